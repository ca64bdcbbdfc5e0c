// unproject.cu -- object-space samples from a colour + depth image (Eq. 1, §4.1) with the
// footprint or voxel radius and a stable compaction of the pixels that carry a sample (§4.1).
//
// Three launches: per-block counts of kept pixels, one-block exclusive scan of the counts (which
// also writes the splat count), and the write pass that re-derives each pixel's rank inside its
// block with warp ballots.  Every pass reads the image with coalesced 16-byte loads.
#include <mutex>

#include "codec.cuh"

namespace wrs {
int check_camera(const wrs_camera* c, const char* fn);
}

namespace {

constexpr int kThreads = 256;
constexpr int kRounds = 4;
constexpr int kTile = kThreads * kRounds;  // pixels per block

__device__ __forceinline__ bool keep_pixel(const float4* __restrict__ rgba,
                                           const float* __restrict__ depth, uint32_t i) {
    const float t = __ldg(depth + i);
    const float a = __ldg(&rgba[i].w);
    return t >= 0.0f && t < __int_as_float(0x7f800000) && a > 0.0f;
}

__device__ __forceinline__ uint32_t block_sum(uint32_t v, uint32_t* s_warp) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) s_warp[warp] = v;
    __syncthreads();
    uint32_t t = 0;
    if (threadIdx.x == 0)
        for (int w = 0; w < kThreads / 32; w++) t += s_warp[w];
    return t;  // valid in thread 0
}

__global__ void __launch_bounds__(kThreads) k_unproject_count(const float4* __restrict__ rgba,
                                                              const float* __restrict__ depth,
                                                              uint32_t npix,
                                                              uint32_t* __restrict__ counts) {
    __shared__ uint32_t s_warp[kThreads / 32];
    const uint32_t base = blockIdx.x * kTile;
    uint32_t c = 0;
#pragma unroll
    for (int k = 0; k < kRounds; k++) {
        const uint32_t i = base + k * kThreads + threadIdx.x;
        if (i < npix && keep_pixel(rgba, depth, i)) c++;
    }
    const uint32_t t = block_sum(c, s_warp);
    if (threadIdx.x == 0) counts[blockIdx.x] = t;
}

// Exclusive scan of nb block counts with one block of 1024 threads.  Plain mode: offsets start at
// 0 and *n_out = total.  APPEND (accumulation over frames): offsets start at the current count
// base = *n_out, and *n_out = min(base + total, capacity); a total above capacity (or a count that
// was already above it) sets WRS_STATUS_SPLAT_OVERFLOW, and the write pass drops the records whose
// slot is >= capacity.  Offsets saturate at 2^32 - 1 (>= capacity, so those records are dropped).
template <bool APPEND>
__global__ void __launch_bounds__(1024) k_scan_counts(const uint32_t* __restrict__ counts,
                                                      uint32_t* __restrict__ offsets, uint32_t nb,
                                                      uint32_t* __restrict__ n_out, uint32_t capacity,
                                                      int32_t* __restrict__ status) {
    __shared__ uint32_t s[1024];
    __shared__ uint32_t s_base;
    const uint32_t per = (nb + 1023) / 1024;
    const uint32_t lo = threadIdx.x * per, hi = min(lo + per, nb);
    uint32_t sum = 0;
    for (uint32_t i = lo; i < hi; i++) sum += counts[i];
    if (APPEND && threadIdx.x == 0) {
        const uint32_t b = *n_out;
        if (b > capacity && status) atomicOr(status, (int32_t)WRS_STATUS_SPLAT_OVERFLOW);
        s_base = min(b, capacity);
    }
    s[threadIdx.x] = sum;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {  // Hillis-Steele inclusive scan
        uint32_t v = threadIdx.x >= (unsigned)o ? s[threadIdx.x - o] : 0;
        __syncthreads();
        s[threadIdx.x] += v;
        __syncthreads();
    }
    const uint64_t base = APPEND ? s_base : 0;
    uint64_t run = base + s[threadIdx.x] - sum;
    for (uint32_t i = lo; i < hi; i++) {
        const uint32_t c = counts[i];
        offsets[i] = (uint32_t)min(run, (uint64_t)0xFFFFFFFFu);
        run += c;
    }
    if (threadIdx.x == 1023) {
        const uint64_t total = base + s[1023];
        if (APPEND && total > capacity && status) atomicOr(status, (int32_t)WRS_STATUS_SPLAT_OVERFLOW);
        *n_out = APPEND ? (uint32_t)min(total, (uint64_t)capacity) : (uint32_t)total;
    }
}

// Output of the write pass.  kPlain: float records at their compacted slot.  kAppend: records go
// after the current count (offsets from the APPEND scan), slots >= capacity are dropped, colours
// are scaled by weight (binary32 product per channel) and ids offset by id_base.  kEncode: the
// 64-bit position + radius word and the 32-bit colour (spec S11) instead of the float records.
enum { kPlain = 0, kAppend = 1, kEncode = 2 };

struct WriteOut {
    float4* pos_r;
    float4* rgba;
    uint32_t* id;
    uint64_t* word;
    uint32_t* color;
    float weight;
    uint32_t id_base;
    uint32_t capacity;
    wrs::CodecConsts codec;
};

template <int MODE>
__global__ void __launch_bounds__(kThreads) k_unproject_write(
    const float4* __restrict__ rgba, const float* __restrict__ depth, wrs_camera cam,
    int32_t mode, float voxel_diag, const uint32_t* __restrict__ offsets, WriteOut out) {
    __shared__ uint32_t s_warp[kThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t npix = (uint32_t)cam.width * (uint32_t)cam.height;
    const uint32_t base = blockIdx.x * kTile;
    uint64_t run = offsets[blockIdx.x];
    // pitch of one pixel at unit depth along the view axis (spec S3)
    const float pitch = __fdiv_rn(__fmul_rn(2.0f, cam.tan_half_fovy), (float)cam.height);
    const float r_vox = __fmul_rn(voxel_diag, 0.5f);
    for (int k = 0; k < kRounds; k++) {
        const uint32_t i = base + k * kThreads + threadIdx.x;
        const bool keep = i < npix && keep_pixel(rgba, depth, i);
        const uint32_t ball = __ballot_sync(0xffffffffu, keep);
        if (lane == 0) s_warp[warp] = __popc(ball);
        __syncthreads();
        uint32_t before = 0, total = 0;
        for (int w = 0; w < kThreads / 32; w++) {
            const uint32_t c = s_warp[w];
            before += (w < warp) ? c : 0;
            total += c;
        }
        const uint64_t slot = run + before + __popc(ball & ((1u << lane) - 1u));
        if (keep && (MODE != kAppend || slot < out.capacity)) {
            const int x = (int)(i % (uint32_t)cam.width), y = (int)(i / (uint32_t)cam.width);
            const wrs::Ray r = wrs::primary_ray(cam, x, y);
            const float t = depth[i];
            float r0;
            if (mode == WRS_RADIUS_FOOTPRINT) {
                const float dz = __fmaf_rn(r.d.z, cam.fwd[2],
                                           __fmaf_rn(r.d.y, cam.fwd[1], __fmul_rn(r.d.x, cam.fwd[0])));
                r0 = __fmul_rn(__fmul_rn(__fmul_rn(t, dz), pitch), 0.70710677f);
            } else {
                r0 = r_vox;
            }
            const float px = __fmaf_rn(r.d.x, t, r.o.x), py = __fmaf_rn(r.d.y, t, r.o.y),
                        pz = __fmaf_rn(r.d.z, t, r.o.z);
            float4 c = rgba[i];
            if (MODE == kEncode) {
                out.word[slot] = wrs::encode_word(out.codec, px, py, pz, r0);
                out.color[slot] = wrs::encode_color(c);
            } else {
                out.pos_r[slot] = make_float4(px, py, pz, r0);
                if (MODE == kAppend) {
                    const float w = out.weight;
                    c = make_float4(__fmul_rn(w, c.x), __fmul_rn(w, c.y), __fmul_rn(w, c.z),
                                    __fmul_rn(w, c.w));
                }
                out.rgba[slot] = c;
                out.id[slot] = MODE == kAppend ? out.id_base + i : i;
            }
        }
        run += total;
        __syncthreads();  // s_warp is reused by the next round
    }
}

// ---- samples smeared along the viewing ray (spec S3b) ------------------------------------------
// Pixel i's chain: its depth interval, radius, chain length n (0 = not a sample) and the colour
// scale of one chain sphere.  Both passes evaluate it the same way.
struct Chain {
    float t_lo, dt, r0, scale;
    int n;
};

__device__ __forceinline__ Chain chain_of(const float4* __restrict__ rgba,
                                          const float* __restrict__ depth_lo,
                                          const float* __restrict__ depth_hi, const wrs_camera& cam,
                                          int32_t mode, float voxel_diag, int max_chain, uint32_t i,
                                          wrs::Ray& ray) {
    Chain c{0.f, 0.f, 0.f, 1.f, 0};
    const float t_lo = __ldg(depth_lo + i);
    const float a = __ldg(&rgba[i].w);
    if (!(t_lo >= 0.0f && t_lo < __int_as_float(0x7f800000) && a > 0.0f)) return c;
    float t_hi = __ldg(depth_hi + i);
    if (!(t_hi < __int_as_float(0x7f800000)) || !(t_hi >= t_lo)) t_hi = t_lo;
    const float dt = __fsub_rn(t_hi, t_lo);
    const float tm = __fmaf_rn(dt, 0.5f, t_lo);
    const int x = (int)(i % (uint32_t)cam.width), y = (int)(i / (uint32_t)cam.width);
    ray = wrs::primary_ray(cam, x, y);
    float r0;
    if (mode == WRS_RADIUS_FOOTPRINT) {
        const float pitch = __fdiv_rn(__fmul_rn(2.0f, cam.tan_half_fovy), (float)cam.height);
        const float dz = __fmaf_rn(ray.d.z, cam.fwd[2],
                                   __fmaf_rn(ray.d.y, cam.fwd[1], __fmul_rn(ray.d.x, cam.fwd[0])));
        r0 = __fmul_rn(__fmul_rn(__fmul_rn(tm, dz), pitch), 0.70710677f);
    } else {
        r0 = __fmul_rn(voxel_diag, 0.5f);
    }
    int n = 1;
    if (r0 > 0.0f) {
        const float q = ceilf(__fdiv_rn(dt, __fmul_rn(2.0f, r0)));
        n = q < 1.0f ? 1 : (q > (float)max_chain ? max_chain : (int)q);
    }
    c.t_lo = t_lo;
    c.dt = dt;
    c.r0 = r0;
    c.n = n;
    if (n > 1) c.scale = __fdiv_rn(-expm1f(__fdiv_rn(log1pf(-a), (float)n)), a);
    return c;
}

__global__ void __launch_bounds__(kThreads) k_interval_count(
    const float4* __restrict__ rgba, const float* __restrict__ depth_lo,
    const float* __restrict__ depth_hi, wrs_camera cam, int32_t mode, float voxel_diag,
    int max_chain, uint32_t* __restrict__ counts) {
    __shared__ uint32_t s_warp[kThreads / 32];
    const uint32_t npix = (uint32_t)cam.width * (uint32_t)cam.height;
    const uint32_t base = blockIdx.x * kTile;
    uint32_t c = 0;
    for (int k = 0; k < kRounds; k++) {
        const uint32_t i = base + k * kThreads + threadIdx.x;
        wrs::Ray ray;
        if (i < npix) c += chain_of(rgba, depth_lo, depth_hi, cam, mode, voxel_diag, max_chain, i, ray).n;
    }
    const uint32_t t = block_sum(c, s_warp);
    if (threadIdx.x == 0) counts[blockIdx.x] = t;
}

// Write pass: a block-wide exclusive scan of the chain lengths gives each pixel's first slot.
__global__ void __launch_bounds__(kThreads) k_interval_write(
    const float4* __restrict__ rgba, const float* __restrict__ depth_lo,
    const float* __restrict__ depth_hi, wrs_camera cam, int32_t mode, float voxel_diag,
    int max_chain, const uint32_t* __restrict__ offsets, float4* __restrict__ pos_r,
    float4* __restrict__ out_rgba, uint32_t* __restrict__ out_id, uint32_t capacity) {
    __shared__ uint32_t s_warp[kThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t npix = (uint32_t)cam.width * (uint32_t)cam.height;
    const uint32_t base = blockIdx.x * kTile;
    uint64_t run = offsets[blockIdx.x];
    for (int k = 0; k < kRounds; k++) {
        const uint32_t i = base + k * kThreads + threadIdx.x;
        wrs::Ray ray;
        Chain ch{0.f, 0.f, 0.f, 1.f, 0};
        if (i < npix) ch = chain_of(rgba, depth_lo, depth_hi, cam, mode, voxel_diag, max_chain, i, ray);
        // inclusive warp scan of the lengths, then the warps' totals
        uint32_t incl = (uint32_t)ch.n;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) s_warp[warp] = incl;
        __syncthreads();
        uint32_t before = 0, total = 0;
        for (int w = 0; w < kThreads / 32; w++) {
            const uint32_t c = s_warp[w];
            before += (w < warp) ? c : 0;
            total += c;
        }
        const uint64_t first = run + before + incl - (uint32_t)ch.n;
        if (ch.n > 0) {
            const float4 c = __ldg(rgba + i);
            const float4 cs = ch.n == 1 ? c
                                        : make_float4(__fmul_rn(c.x, ch.scale), __fmul_rn(c.y, ch.scale),
                                                      __fmul_rn(c.z, ch.scale), __fmul_rn(c.w, ch.scale));
            for (int q = 0; q < ch.n; q++) {
                const uint64_t slot = first + (uint64_t)q;
                if (slot >= capacity) break;
                const float u = __fdiv_rn((float)(2 * q + 1), (float)(2 * ch.n));
                const float tk = __fmaf_rn(u, ch.dt, ch.t_lo);
                pos_r[slot] = make_float4(__fmaf_rn(ray.d.x, tk, ray.o.x), __fmaf_rn(ray.d.y, tk, ray.o.y),
                                          __fmaf_rn(ray.d.z, tk, ray.o.z), ch.r0);
                out_rgba[slot] = cs;
                out_id[slot] = i * (uint32_t)max_chain + (uint32_t)q;
            }
        }
        run += total;
        __syncthreads();  // s_warp is reused by the next round
    }
}

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

WriteOut float_out(const wrs_splats* out, float weight, uint32_t id_base) {
    WriteOut o{};
    o.pos_r = reinterpret_cast<float4*>(out->pos_r);
    o.rgba = reinterpret_cast<float4*>(out->rgba);
    o.id = out->id;
    o.weight = weight;
    o.id_base = id_base;
    o.capacity = out->capacity;
    return o;
}

}  // namespace

extern "C" {

size_t wrs_unproject_scratch_bytes(int32_t width, int32_t height) {
    if (width <= 0 || height <= 0) return 0;
    const size_t npix = (size_t)width * (size_t)height;
    const size_t nb = (npix + kTile - 1) / kTile;
    return 2 * align256(nb * sizeof(uint32_t));
}

int wrs_unproject(const float* rgba, const float* depth, const wrs_camera* cam,
                  int32_t radius_mode, float voxel_diag, wrs_splats* out, void* scratch,
                  size_t scratch_bytes, wrs_stream_t stream) {
    const char* fn = "wrs_unproject";
    if (int rc = wrs::check_camera(cam, fn)) return rc;
    if (!rgba || !depth || !out || !out->pos_r || !out->rgba || !out->id || !out->n)
        return wrs::fail(WRS_ERR_ARG, "%s: NULL input or output pointer", fn);
    if ((reinterpret_cast<uintptr_t>(rgba) | reinterpret_cast<uintptr_t>(out->pos_r) |
         reinterpret_cast<uintptr_t>(out->rgba)) & 15)
        return wrs::fail(WRS_ERR_ARG, "%s: rgba / pos_r arrays must be 16-byte aligned", fn);
    if (radius_mode != WRS_RADIUS_FOOTPRINT && radius_mode != WRS_RADIUS_VOXEL)
        return wrs::fail(WRS_ERR_ARG, "%s: unknown radius_mode %d", fn, radius_mode);
    if (radius_mode == WRS_RADIUS_VOXEL && !(voxel_diag > 0.0f && voxel_diag < 1e30f))
        return wrs::fail(WRS_ERR_ARG, "%s: voxel_diag must be positive and finite", fn);
    const size_t npix = (size_t)cam->width * (size_t)cam->height;
    if (npix >= 0x80000000ull)
        return wrs::fail(WRS_ERR_ARG, "%s: image of %zu pixels exceeds 2^31", fn, npix);
    if (out->capacity < npix)
        return wrs::fail(WRS_ERR_CAPACITY, "%s: splat capacity %u < %zu pixels", fn, out->capacity,
                         npix);
    const size_t need = wrs_unproject_scratch_bytes(cam->width, cam->height);
    if (!scratch || scratch_bytes < need)
        return wrs::fail(WRS_ERR_SCRATCH, "%s: scratch needs %zu bytes, got %zu", fn, need,
                         scratch_bytes);
    const uint32_t nb = (uint32_t)((npix + kTile - 1) / kTile);
    uint32_t* counts = static_cast<uint32_t*>(scratch);
    uint32_t* offsets = reinterpret_cast<uint32_t*>(static_cast<char*>(scratch) +
                                                    align256(nb * sizeof(uint32_t)));
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const float4* in4 = reinterpret_cast<const float4*>(rgba);
    k_unproject_count<<<nb, kThreads, 0, s>>>(in4, depth, (uint32_t)npix, counts);
    WRS_LAUNCH_CHECK("wrs_unproject count");
    k_scan_counts<false><<<1, 1024, 0, s>>>(counts, offsets, nb, out->n, out->capacity, nullptr);
    WRS_LAUNCH_CHECK("wrs_unproject scan");
    k_unproject_write<kPlain><<<nb, kThreads, 0, s>>>(in4, depth, *cam, radius_mode, voxel_diag,
                                                      offsets, float_out(out, 1.0f, 0u));
    WRS_LAUNCH_CHECK("wrs_unproject write");
    return WRS_OK;
}

int wrs_unproject_encode(const float* rgba, const float* depth, const wrs_camera* cam,
                         int32_t radius_mode, float voxel_diag, const wrs_codec* codec,
                         uint64_t* word, uint32_t* color, uint32_t* n, uint32_t capacity,
                         void* scratch, size_t scratch_bytes, wrs_stream_t stream) {
    const char* fn = "wrs_unproject_encode";
    if (int rc = wrs::check_camera(cam, fn)) return rc;
    if (int rc = wrs::check_codec(codec, fn)) return rc;
    if (!rgba || !depth || !word || !color || !n)
        return wrs::fail(WRS_ERR_ARG, "%s: NULL input or output pointer", fn);
    if ((reinterpret_cast<uintptr_t>(rgba) & 15) | (reinterpret_cast<uintptr_t>(word) & 7) |
        (reinterpret_cast<uintptr_t>(color) & 3))
        return wrs::fail(WRS_ERR_ARG, "%s: misaligned array", fn);
    if (radius_mode != WRS_RADIUS_FOOTPRINT && radius_mode != WRS_RADIUS_VOXEL)
        return wrs::fail(WRS_ERR_ARG, "%s: unknown radius_mode %d", fn, radius_mode);
    if (radius_mode == WRS_RADIUS_VOXEL && !(voxel_diag > 0.0f && voxel_diag < 1e30f))
        return wrs::fail(WRS_ERR_ARG, "%s: voxel_diag must be positive and finite", fn);
    const size_t npix = (size_t)cam->width * (size_t)cam->height;
    if (npix >= 0x80000000ull)
        return wrs::fail(WRS_ERR_ARG, "%s: image of %zu pixels exceeds 2^31", fn, npix);
    if (capacity < npix)
        return wrs::fail(WRS_ERR_CAPACITY, "%s: capacity %u < %zu pixels", fn, capacity, npix);
    const size_t need = wrs_unproject_scratch_bytes(cam->width, cam->height);
    if (!scratch || scratch_bytes < need)
        return wrs::fail(WRS_ERR_SCRATCH, "%s: scratch needs %zu bytes, got %zu", fn, need,
                         scratch_bytes);
    const uint32_t nb = (uint32_t)((npix + kTile - 1) / kTile);
    uint32_t* counts = static_cast<uint32_t*>(scratch);
    uint32_t* offsets = reinterpret_cast<uint32_t*>(static_cast<char*>(scratch) +
                                                    align256(nb * sizeof(uint32_t)));
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const float4* in4 = reinterpret_cast<const float4*>(rgba);
    k_unproject_count<<<nb, kThreads, 0, s>>>(in4, depth, (uint32_t)npix, counts);
    WRS_LAUNCH_CHECK("wrs_unproject_encode count");
    k_scan_counts<false><<<1, 1024, 0, s>>>(counts, offsets, nb, n, capacity, nullptr);
    WRS_LAUNCH_CHECK("wrs_unproject_encode scan");
    WriteOut o{};
    o.word = word;
    o.color = color;
    o.capacity = capacity;
    o.codec = wrs::make_codec(*codec);
    k_unproject_write<kEncode><<<nb, kThreads, 0, s>>>(in4, depth, *cam, radius_mode, voxel_diag,
                                                       offsets, o);
    WRS_LAUNCH_CHECK("wrs_unproject_encode write");
    return WRS_OK;
}

int wrs_unproject_interval(const float* rgba, const float* depth_lo, const float* depth_hi,
                           const wrs_camera* cam, int32_t radius_mode, float voxel_diag,
                           int32_t max_chain, wrs_splats* out, void* scratch,
                           size_t scratch_bytes, int32_t* status, wrs_stream_t stream) {
    const char* fn = "wrs_unproject_interval";
    if (int rc = wrs::check_camera(cam, fn)) return rc;
    if (!rgba || !depth_lo || !depth_hi || !out || !out->pos_r || !out->rgba || !out->id || !out->n)
        return wrs::fail(WRS_ERR_ARG, "%s: NULL input or output pointer", fn);
    if ((reinterpret_cast<uintptr_t>(rgba) | reinterpret_cast<uintptr_t>(out->pos_r) |
         reinterpret_cast<uintptr_t>(out->rgba)) & 15)
        return wrs::fail(WRS_ERR_ARG, "%s: rgba / pos_r arrays must be 16-byte aligned", fn);
    if (radius_mode != WRS_RADIUS_FOOTPRINT && radius_mode != WRS_RADIUS_VOXEL)
        return wrs::fail(WRS_ERR_ARG, "%s: unknown radius_mode %d", fn, radius_mode);
    if (radius_mode == WRS_RADIUS_VOXEL && !(voxel_diag > 0.0f && voxel_diag < 1e30f))
        return wrs::fail(WRS_ERR_ARG, "%s: voxel_diag must be positive and finite", fn);
    if (max_chain < 1 || max_chain > 64)
        return wrs::fail(WRS_ERR_ARG, "%s: max_chain %d not in 1..64", fn, max_chain);
    const size_t npix = (size_t)cam->width * (size_t)cam->height;
    if (npix >= 0x80000000ull || npix * (size_t)max_chain > 0x100000000ull)
        return wrs::fail(WRS_ERR_ARG, "%s: %zu pixels x %d exceeds the 32-bit ids", fn, npix,
                         max_chain);
    if (out->capacity == 0) return wrs::fail(WRS_ERR_CAPACITY, "%s: splat capacity is 0", fn);
    const size_t need = wrs_unproject_scratch_bytes(cam->width, cam->height);
    if (!scratch || scratch_bytes < need)
        return wrs::fail(WRS_ERR_SCRATCH, "%s: scratch needs %zu bytes, got %zu", fn, need,
                         scratch_bytes);
    const uint32_t nb = (uint32_t)((npix + kTile - 1) / kTile);
    uint32_t* counts = static_cast<uint32_t*>(scratch);
    uint32_t* offsets = reinterpret_cast<uint32_t*>(static_cast<char*>(scratch) +
                                                    align256(nb * sizeof(uint32_t)));
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const float4* in4 = reinterpret_cast<const float4*>(rgba);
    k_interval_count<<<nb, kThreads, 0, s>>>(in4, depth_lo, depth_hi, *cam, radius_mode, voxel_diag,
                                             max_chain, counts);
    WRS_LAUNCH_CHECK("wrs_unproject_interval count");
    // the count starts at 0; the append form of the scan clamps it to the capacity and flags
    // SPLAT_OVERFLOW when the chains need more records than that
    cudaError_t e = cudaMemsetAsync(out->n, 0, sizeof(uint32_t), s);
    if (e != cudaSuccess) return wrs::cuda_fail(e, fn);
    k_scan_counts<true><<<1, 1024, 0, s>>>(counts, offsets, nb, out->n, out->capacity, status);
    WRS_LAUNCH_CHECK("wrs_unproject_interval scan");
    k_interval_write<<<nb, kThreads, 0, s>>>(in4, depth_lo, depth_hi, *cam, radius_mode, voxel_diag,
                                             max_chain, offsets, reinterpret_cast<float4*>(out->pos_r),
                                             reinterpret_cast<float4*>(out->rgba), out->id,
                                             out->capacity);
    WRS_LAUNCH_CHECK("wrs_unproject_interval write");
    return WRS_OK;
}

int wrs_unproject_append(const float* rgba, const float* depth, const wrs_camera* cam,
                         int32_t radius_mode, float voxel_diag, float weight, uint32_t id_base,
                         wrs_splats* out, void* scratch, size_t scratch_bytes, int32_t* status,
                         wrs_stream_t stream) {
    const char* fn = "wrs_unproject_append";
    if (int rc = wrs::check_camera(cam, fn)) return rc;
    if (!rgba || !depth || !out || !out->pos_r || !out->rgba || !out->id || !out->n)
        return wrs::fail(WRS_ERR_ARG, "%s: NULL input or output pointer", fn);
    if ((reinterpret_cast<uintptr_t>(rgba) | reinterpret_cast<uintptr_t>(out->pos_r) |
         reinterpret_cast<uintptr_t>(out->rgba)) & 15)
        return wrs::fail(WRS_ERR_ARG, "%s: rgba / pos_r arrays must be 16-byte aligned", fn);
    if (radius_mode != WRS_RADIUS_FOOTPRINT && radius_mode != WRS_RADIUS_VOXEL)
        return wrs::fail(WRS_ERR_ARG, "%s: unknown radius_mode %d", fn, radius_mode);
    if (radius_mode == WRS_RADIUS_VOXEL && !(voxel_diag > 0.0f && voxel_diag < 1e30f))
        return wrs::fail(WRS_ERR_ARG, "%s: voxel_diag must be positive and finite", fn);
    if (!(weight > 0.0f && weight <= 1.0f))
        return wrs::fail(WRS_ERR_ARG, "%s: weight must lie in (0, 1]", fn);
    const size_t npix = (size_t)cam->width * (size_t)cam->height;
    if (npix >= 0x80000000ull)
        return wrs::fail(WRS_ERR_ARG, "%s: image of %zu pixels exceeds 2^31", fn, npix);
    if ((uint64_t)id_base + npix > 0x100000000ull)
        return wrs::fail(WRS_ERR_ARG, "%s: id_base %u + %zu pixels exceeds 2^32", fn, id_base, npix);
    if (out->capacity == 0) return wrs::fail(WRS_ERR_CAPACITY, "%s: splat capacity is 0", fn);
    const size_t need = wrs_unproject_scratch_bytes(cam->width, cam->height);
    if (!scratch || scratch_bytes < need)
        return wrs::fail(WRS_ERR_SCRATCH, "%s: scratch needs %zu bytes, got %zu", fn, need,
                         scratch_bytes);
    const uint32_t nb = (uint32_t)((npix + kTile - 1) / kTile);
    uint32_t* counts = static_cast<uint32_t*>(scratch);
    uint32_t* offsets = reinterpret_cast<uint32_t*>(static_cast<char*>(scratch) +
                                                    align256(nb * sizeof(uint32_t)));
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const float4* in4 = reinterpret_cast<const float4*>(rgba);
    k_unproject_count<<<nb, kThreads, 0, s>>>(in4, depth, (uint32_t)npix, counts);
    WRS_LAUNCH_CHECK("wrs_unproject_append count");
    k_scan_counts<true><<<1, 1024, 0, s>>>(counts, offsets, nb, out->n, out->capacity, status);
    WRS_LAUNCH_CHECK("wrs_unproject_append scan");
    k_unproject_write<kAppend><<<nb, kThreads, 0, s>>>(in4, depth, *cam, radius_mode, voxel_diag,
                                                       offsets, float_out(out, weight, id_base));
    WRS_LAUNCH_CHECK("wrs_unproject_append write");
    return WRS_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------------------------
// wrs_unproject_static: the same three kernels with their work buffer (per-block counts, then
// per-block offsets) in a fixed array that lives in this library's device image, for callers that
// cannot hand us device memory.
// ---------------------------------------------------------------------------------------------
namespace {

constexpr uint32_t kStaticMaxPixels = 1u << 26;                  // 67,108,864 = 8192 x 8192
constexpr uint32_t kStaticMaxBlocks = kStaticMaxPixels / kTile;  // 65,536 blocks
constexpr int kStaticMaxDevices = 64;

}  // namespace

// Counts in [0, kStaticMaxBlocks), offsets in [kStaticMaxBlocks, 2 kStaticMaxBlocks): 512 KiB that
// every GPU which loads the library keeps until the process exits.
static __device__ __align__(256) uint32_t g_unproject_static_scratch[2 * kStaticMaxBlocks];

namespace {

std::mutex g_static_mu;
uint32_t* g_static_ptr[kStaticMaxDevices] = {};

// Device address of the static array on the current device.  The host-side symbol is only a
// stand-in, so the address is looked up once per device (with that device current) and cached.
int static_scratch(uint32_t** out, const char* fn) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return wrs::cuda_fail(e, fn);
    if (dev < 0 || dev >= kStaticMaxDevices)
        return wrs::fail(WRS_ERR_ARG, "%s: device ordinal %d beyond %d", fn, dev, kStaticMaxDevices);
    std::lock_guard<std::mutex> lock(g_static_mu);
    if (!g_static_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_unproject_static_scratch);
        if (e != cudaSuccess) return wrs::cuda_fail(e, "wrs_unproject_static: cudaGetSymbolAddress");
        g_static_ptr[dev] = static_cast<uint32_t*>(p);
    }
    *out = g_static_ptr[dev];
    return WRS_OK;
}

}  // namespace

extern "C" int wrs_unproject_static(const float* rgba, const float* depth, const wrs_camera* cam,
                                    int32_t radius_mode, float voxel_diag, wrs_splats* out,
                                    wrs_stream_t stream) {
    const char* fn = "wrs_unproject_static";
    if (int rc = wrs::check_camera(cam, fn)) return rc;
    if (!rgba || !depth || !out || !out->pos_r || !out->rgba || !out->id || !out->n)
        return wrs::fail(WRS_ERR_ARG, "%s: NULL input or output pointer", fn);
    if ((reinterpret_cast<uintptr_t>(rgba) | reinterpret_cast<uintptr_t>(out->pos_r) |
         reinterpret_cast<uintptr_t>(out->rgba)) & 15)
        return wrs::fail(WRS_ERR_ARG, "%s: rgba / pos_r arrays must be 16-byte aligned", fn);
    if (radius_mode != WRS_RADIUS_FOOTPRINT && radius_mode != WRS_RADIUS_VOXEL)
        return wrs::fail(WRS_ERR_ARG, "%s: unknown radius_mode %d", fn, radius_mode);
    if (radius_mode == WRS_RADIUS_VOXEL && !(voxel_diag > 0.0f && voxel_diag < 1e30f))
        return wrs::fail(WRS_ERR_ARG, "%s: voxel_diag must be positive and finite", fn);
    const size_t npix = (size_t)cam->width * (size_t)cam->height;
    if (npix > kStaticMaxPixels)
        return wrs::fail(WRS_ERR_CAPACITY,
                         "%s: image of %zu pixels exceeds the fixed work buffer's limit of %u "
                         "pixels (width x height, e.g. 8192 x 8192 or 16384 x 4096); use "
                         "wrs_unproject with caller scratch",
                         fn, npix, kStaticMaxPixels);
    if (out->capacity < npix)
        return wrs::fail(WRS_ERR_CAPACITY, "%s: splat capacity %u < %zu pixels", fn, out->capacity,
                         npix);
    uint32_t* buf = nullptr;
    if (int rc = static_scratch(&buf, fn)) return rc;
    // Every count and offset the kernels read is written earlier in the same call, so nothing in
    // the shared array has to be cleared between calls.
    const uint32_t nb = (uint32_t)((npix + kTile - 1) / kTile);
    uint32_t* counts = buf;
    uint32_t* offsets = buf + kStaticMaxBlocks;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const float4* in4 = reinterpret_cast<const float4*>(rgba);
    k_unproject_count<<<nb, kThreads, 0, s>>>(in4, depth, (uint32_t)npix, counts);
    WRS_LAUNCH_CHECK("wrs_unproject_static count");
    k_scan_counts<false><<<1, 1024, 0, s>>>(counts, offsets, nb, out->n, out->capacity, nullptr);
    WRS_LAUNCH_CHECK("wrs_unproject_static scan");
    k_unproject_write<kPlain><<<nb, kThreads, 0, s>>>(in4, depth, *cam, radius_mode, voxel_diag,
                                                      offsets, float_out(out, 1.0f, 0u));
    WRS_LAUNCH_CHECK("wrs_unproject_static write");
    return WRS_OK;
}
