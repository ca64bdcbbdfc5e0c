// point_splat.cu -- the earlier 2.5D warping the paper compares its sphere tracing against (§2, §5,
// Fig. 3; reading: spec S10): every splat is drawn as an s x s pixel square around its projection
// into the client camera, with one depth per point, and each pixel keeps the nearest point.
//
// Two launches after a 0xFF fill of the key image: a depth pass in which each point min-reduces
// the 64-bit key (bits of its view depth z << 32 | its index) into every pixel it covers (z > 0,
// so the bit pattern orders like the value and ties go to the lower index), and a resolve pass
// that copies the winning point's colour.  The projection is binary32 with the operation order of
// the spec, so the covered pixels and the winner are exact.
#include "common.cuh"

namespace wrs {
int check_camera(const wrs_camera* c, const char* fn);
}

namespace {

constexpr unsigned long long kEmpty = ~0ull;

__global__ void __launch_bounds__(256) k_ps_depth(const float4* __restrict__ pos_r,
                                                  const uint32_t* __restrict__ n_ptr, uint32_t cap,
                                                  wrs_camera cam, int32_t size,
                                                  unsigned long long* __restrict__ key) {
    const uint32_t n = min(*n_ptr, cap);
    const int W = cam.width, H = cam.height;
    const float sx = __fmul_rn(cam.tan_half_fovy, __fdiv_rn((float)W, (float)H));
    const float half = __fmul_rn(0.5f, (float)size);
    const float hw = __fmul_rn(0.5f, (float)W), hh = __fmul_rn(0.5f, (float)H);
    for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const float4 p = pos_r[k];
        const float qx = __fsub_rn(p.x, cam.eye[0]), qy = __fsub_rn(p.y, cam.eye[1]),
                    qz = __fsub_rn(p.z, cam.eye[2]);
        const float z = __fmaf_rn(qz, cam.fwd[2], __fmaf_rn(qy, cam.fwd[1], __fmul_rn(qx, cam.fwd[0])));
        if (!(z > 0.0f)) continue;  // at or behind the eye plane
        const float xr = __fmaf_rn(qz, cam.right[2], __fmaf_rn(qy, cam.right[1], __fmul_rn(qx, cam.right[0])));
        const float yu = __fmaf_rn(qz, cam.up[2], __fmaf_rn(qy, cam.up[1], __fmul_rn(qx, cam.up[0])));
        const float nx = __fdiv_rn(__fdiv_rn(xr, z), sx);
        const float ny = __fdiv_rn(__fdiv_rn(yu, z), cam.tan_half_fovy);
        const float px = __fsub_rn(__fmul_rn(__fadd_rn(nx, 1.0f), hw), 0.5f);
        const float py = __fsub_rn(__fmul_rn(__fsub_rn(1.0f, ny), hh), 0.5f);
        const float x0f = ceilf(__fsub_rn(px, half)), y0f = ceilf(__fsub_rn(py, half));
        if (!(x0f > -(float)size && x0f < (float)W && y0f > -(float)size && y0f < (float)H)) continue;
        const int x0 = (int)x0f, y0 = (int)y0f;
        const unsigned long long kk = ((unsigned long long)__float_as_uint(z) << 32) | k;
        const int ya = max(y0, 0), yb = min(y0 + size, H), xa = max(x0, 0), xb = min(x0 + size, W);
        for (int y = ya; y < yb; y++)
            for (int x = xa; x < xb; x++) atomicMin(key + (size_t)y * W + x, kk);
    }
}

__global__ void __launch_bounds__(256) k_ps_resolve(const unsigned long long* __restrict__ key,
                                                    const float4* __restrict__ rgba, uint32_t npix,
                                                    float4* __restrict__ out,
                                                    int32_t* __restrict__ index_out) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < npix; i += gridDim.x * blockDim.x) {
        const unsigned long long kk = key[i];
        const bool hit = kk != kEmpty;
        const uint32_t k = (uint32_t)kk;
        out[i] = hit ? rgba[k] : make_float4(0.f, 0.f, 0.f, 0.f);
        if (index_out) index_out[i] = hit ? (int32_t)k : -1;
    }
}

uint32_t grid_for(size_t work) {
    int dev = 0, sms = 148;
    if (cudaGetDevice(&dev) == cudaSuccess)
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const size_t blocks = (work + 255) / 256;
    const size_t cap = (size_t)sms * 8;  // a few waves of 256-thread blocks; the loops stride
    return (uint32_t)(blocks < 1 ? 1 : (blocks < cap ? blocks : cap));
}

}  // namespace

extern "C" {

size_t wrs_point_splat_scratch_bytes(int32_t width, int32_t height) {
    if (width <= 0 || height <= 0) return 0;
    return (size_t)width * (size_t)height * sizeof(unsigned long long);
}

int wrs_point_splat(const wrs_splats* splats, const wrs_camera* cam, int32_t point_size,
                    float* rgba_out, int32_t* index_out, void* scratch, size_t scratch_bytes,
                    wrs_stream_t stream) {
    const char* fn = "wrs_point_splat";
    if (int rc = wrs::check_camera(cam, fn)) return rc;
    if (!splats || !splats->pos_r || !splats->rgba || !splats->n || !rgba_out)
        return wrs::fail(WRS_ERR_ARG, "%s: NULL input or output pointer", fn);
    if ((reinterpret_cast<uintptr_t>(splats->pos_r) | reinterpret_cast<uintptr_t>(splats->rgba) |
         reinterpret_cast<uintptr_t>(rgba_out)) & 15)
        return wrs::fail(WRS_ERR_ARG, "%s: float4 arrays must be 16-byte aligned", fn);
    if (point_size < 1 || point_size > 64)
        return wrs::fail(WRS_ERR_ARG, "%s: point_size %d not in 1..64", fn, point_size);
    const size_t npix = (size_t)cam->width * (size_t)cam->height;
    if (npix >= 0x80000000ull)
        return wrs::fail(WRS_ERR_ARG, "%s: image of %zu pixels exceeds 2^31", fn, npix);
    const size_t need = wrs_point_splat_scratch_bytes(cam->width, cam->height);
    if (!scratch || scratch_bytes < need)
        return wrs::fail(WRS_ERR_SCRATCH, "%s: scratch needs %zu bytes, got %zu", fn, need,
                         scratch_bytes);
    if (reinterpret_cast<uintptr_t>(scratch) & 7)
        return wrs::fail(WRS_ERR_ARG, "%s: scratch must be 8-byte aligned", fn);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    unsigned long long* key = static_cast<unsigned long long*>(scratch);
    cudaError_t e = cudaMemsetAsync(key, 0xFF, need, s);
    if (e != cudaSuccess) return wrs::cuda_fail(e, fn);
    if (splats->capacity > 0) {
        k_ps_depth<<<grid_for(splats->capacity), 256, 0, s>>>(
            reinterpret_cast<const float4*>(splats->pos_r), splats->n, splats->capacity, *cam,
            point_size, key);
        WRS_LAUNCH_CHECK("wrs_point_splat depth");
    }
    k_ps_resolve<<<grid_for(npix), 256, 0, s>>>(key, reinterpret_cast<const float4*>(splats->rgba),
                                                (uint32_t)npix, reinterpret_cast<float4*>(rgba_out),
                                                index_out);
    WRS_LAUNCH_CHECK("wrs_point_splat resolve");
    return WRS_OK;
}

}  // extern "C"
