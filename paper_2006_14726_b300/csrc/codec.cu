// codec.cu -- encode splats into the 64-bit position + radius word and 32-bit colour the server
// sends (§4.1, §6; layout: spec S11), and decode such a stream into the float records the LBVH and
// the trace read.  One thread per record, grid-stride loops over the capacity, count on the device.
#include "codec.cuh"

namespace {

__global__ void __launch_bounds__(256) k_encode(const float4* __restrict__ pos_r,
                                                const float4* __restrict__ rgba,
                                                const uint32_t* __restrict__ n_ptr, uint32_t cap,
                                                wrs::CodecConsts k, uint64_t* __restrict__ word,
                                                uint32_t* __restrict__ color,
                                                uint32_t* __restrict__ n_out) {
    const uint32_t n = min(*n_ptr, cap);
    const uint32_t first = blockIdx.x * blockDim.x + threadIdx.x;
    if (first == 0 && n_out) *n_out = n;
    for (uint32_t i = first; i < n; i += gridDim.x * blockDim.x) {
        const float4 p = pos_r[i];
        word[i] = wrs::encode_word(k, p.x, p.y, p.z, p.w);
        color[i] = wrs::encode_color(rgba[i]);
    }
}

__global__ void __launch_bounds__(256) k_decode(const uint64_t* __restrict__ word,
                                                const uint32_t* __restrict__ color,
                                                const uint32_t* __restrict__ n_ptr, uint32_t cap,
                                                wrs::CodecConsts k, float4* __restrict__ pos_r,
                                                float4* __restrict__ rgba, uint32_t* __restrict__ id,
                                                uint32_t* __restrict__ n_out) {
    const uint32_t n = min(*n_ptr, cap);
    const uint32_t first = blockIdx.x * blockDim.x + threadIdx.x;
    if (first == 0) *n_out = n;
    for (uint32_t i = first; i < n; i += gridDim.x * blockDim.x) {
        pos_r[i] = wrs::decode_pos_r(k, word[i]);
        rgba[i] = wrs::decode_color(color[i]);
        id[i] = i;  // the stream keeps the compacted (pixel) order: ties resolve as with pixel ids
    }
}

uint32_t grid_for(uint32_t work) {
    int dev = 0, sms = 148;
    if (cudaGetDevice(&dev) == cudaSuccess)
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const uint32_t blocks = (work + 255) / 256;
    const uint32_t cap = (uint32_t)sms * 8;
    return blocks < 1 ? 1 : (blocks < cap ? blocks : cap);
}

}  // namespace

namespace wrs {

int check_codec(const wrs_codec* c, const char* fn) {
    if (!c) return fail(WRS_ERR_ARG, "%s: codec is NULL", fn);
    for (int a = 0; a < 3; a++) {
        const float ext = c->hi[a] - c->lo[a];
        if (!(fabsf(c->lo[a]) < 1e30f && fabsf(c->hi[a]) < 1e30f && ext > 0.0f && ext < 1e30f))
            return fail(WRS_ERR_ARG, "%s: codec box axis %d is empty or not finite", fn, a);
    }
    if (!(c->r_max > 0.0f && c->r_max < 1e30f))
        return fail(WRS_ERR_ARG, "%s: codec r_max must be positive and finite", fn);
    return WRS_OK;
}

}  // namespace wrs

extern "C" {

int wrs_encode_splats(const wrs_splats* in, const wrs_codec* codec, uint64_t* word,
                      uint32_t* color, uint32_t* n_out, wrs_stream_t stream) {
    const char* fn = "wrs_encode_splats";
    if (int rc = wrs::check_codec(codec, fn)) return rc;
    if (!in || !in->pos_r || !in->rgba || !in->n || !word || !color)
        return wrs::fail(WRS_ERR_ARG, "%s: NULL input or output pointer", fn);
    if ((reinterpret_cast<uintptr_t>(in->pos_r) & 15) | (reinterpret_cast<uintptr_t>(in->rgba) & 15) |
        (reinterpret_cast<uintptr_t>(word) & 7) | (reinterpret_cast<uintptr_t>(color) & 3))
        return wrs::fail(WRS_ERR_ARG, "%s: misaligned array", fn);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    k_encode<<<grid_for(in->capacity ? in->capacity : 1), 256, 0, s>>>(
        reinterpret_cast<const float4*>(in->pos_r), reinterpret_cast<const float4*>(in->rgba), in->n,
        in->capacity, wrs::make_codec(*codec), word, color, n_out);
    WRS_LAUNCH_CHECK("wrs_encode_splats");
    return WRS_OK;
}

int wrs_decode_splats(const uint64_t* word, const uint32_t* color, const uint32_t* n,
                      uint32_t capacity, const wrs_codec* codec, wrs_splats* out,
                      wrs_stream_t stream) {
    const char* fn = "wrs_decode_splats";
    if (int rc = wrs::check_codec(codec, fn)) return rc;
    if (!word || !color || !n || !out || !out->pos_r || !out->rgba || !out->id || !out->n)
        return wrs::fail(WRS_ERR_ARG, "%s: NULL input or output pointer", fn);
    if ((reinterpret_cast<uintptr_t>(out->pos_r) & 15) | (reinterpret_cast<uintptr_t>(out->rgba) & 15) |
        (reinterpret_cast<uintptr_t>(word) & 7) | (reinterpret_cast<uintptr_t>(color) & 3))
        return wrs::fail(WRS_ERR_ARG, "%s: misaligned array", fn);
    if (out->capacity < capacity)
        return wrs::fail(WRS_ERR_CAPACITY, "%s: output capacity %u < stream capacity %u", fn,
                         out->capacity, capacity);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    k_decode<<<grid_for(capacity ? capacity : 1), 256, 0, s>>>(
        word, color, n, capacity, wrs::make_codec(*codec), reinterpret_cast<float4*>(out->pos_r),
        reinterpret_cast<float4*>(out->rgba), out->id, out->n);
    WRS_LAUNCH_CHECK("wrs_decode_splats");
    return WRS_OK;
}

}  // extern "C"
