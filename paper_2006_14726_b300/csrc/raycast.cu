// raycast.cu -- the server's volume ray marcher with the first-hit depth heuristic (§4.1, §4.2,
// Fig. 2; spec S2) and the readings of the other heuristics of §2 and §5 (spec S2a: max
// contribution, accumulated opacity, max gradient).  One thread per pixel.  Sample positions, trilinear reconstruction and the
// transfer-function alpha that drives the depth decision follow the spec's binary32 operation
// order; the colour composite is ordinary binary32 arithmetic.  The transfer function is staged
// in shared memory; volume reads go through the read-only cache.
#include "common.cuh"

namespace wrs {
int check_camera(const wrs_camera* c, const char* fn);
}

namespace {

template <int DT>
__device__ __forceinline__ float voxel(const void* __restrict__ vol, size_t idx) {
    if (DT == WRS_U8) return (float)__ldg(static_cast<const unsigned char*>(vol) + idx);
    return __ldg(static_cast<const float*>(vol) + idx);
}

__device__ __forceinline__ float lerp_rn(float a, float b, float f) {
    return __fmaf_rn(f, __fsub_rn(b, a), a);
}

template <int DT>
__device__ __forceinline__ float sample(const void* __restrict__ vol, int nx, int ny, int nz,
                                        float px, float py, float pz) {
    const int n[3] = {nx, ny, nz};
    const float p[3] = {px, py, pz};
    int i0[3], i1[3];
    float f[3];
#pragma unroll
    for (int a = 0; a < 3; a++) {
        float g = __fmaf_rn(p[a], (float)n[a], -0.5f);
        g = fminf(fmaxf(g, 0.0f), (float)(n[a] - 1));
        int i = (int)floorf(g);
        if (n[a] >= 2) i = min(i, n[a] - 2);
        else i = 0;
        i0[a] = i;
        i1[a] = n[a] >= 2 ? i + 1 : i;
        f[a] = __fsub_rn(g, (float)i);
    }
    const size_t sx = 1, sy = (size_t)nx, sz = (size_t)nx * ny;
    const size_t b00 = i0[1] * sy + i0[2] * sz, b10 = i1[1] * sy + i0[2] * sz;
    const size_t b01 = i0[1] * sy + i1[2] * sz, b11 = i1[1] * sy + i1[2] * sz;
    const float c00 = lerp_rn(voxel<DT>(vol, b00 + i0[0] * sx), voxel<DT>(vol, b00 + i1[0] * sx), f[0]);
    const float c10 = lerp_rn(voxel<DT>(vol, b10 + i0[0] * sx), voxel<DT>(vol, b10 + i1[0] * sx), f[0]);
    const float c01 = lerp_rn(voxel<DT>(vol, b01 + i0[0] * sx), voxel<DT>(vol, b01 + i1[0] * sx), f[0]);
    const float c11 = lerp_rn(voxel<DT>(vol, b11 + i0[0] * sx), voxel<DT>(vol, b11 + i1[0] * sx), f[0]);
    const float c0 = lerp_rn(c00, c10, f[1]);
    const float c1 = lerp_rn(c01, c11, f[1]);
    float s = lerp_rn(c0, c1, f[2]);
    if (DT == WRS_U8) s = __fdiv_rn(s, 255.0f);
    return fminf(fmaxf(s, 0.0f), 1.0f);
}

// HEUR: WRS_DEPTH_* (spec S2a); param = tau (first hit) or theta (accumulated opacity).
template <int DT, int HEUR>
__global__ void __launch_bounds__(128) k_raycast(const void* __restrict__ vol, int nx, int ny,
                                                 int nz, const float4* __restrict__ tf,
                                                 wrs_camera cam, float step_vox, float param,
                                                 float4* __restrict__ rgba_out,
                                                 float* __restrict__ depth_out) {
    __shared__ float4 s_tf[256];
    for (int i = threadIdx.x; i < 256; i += blockDim.x) s_tf[i] = tf[i];
    __syncthreads();
    // 16x8 pixel tile per block, 8x4 per warp
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int x = blockIdx.x * 16 + (warp & 1) * 8 + (lane & 7);
    const int y = blockIdx.y * 8 + (warp >> 1) * 4 + (lane >> 3);
    if (x >= cam.width || y >= cam.height) return;
    const size_t pix = (size_t)y * cam.width + x;
    const wrs::Ray r = wrs::primary_ray(cam, x, y);

    const float od[3] = {r.o.x, r.o.y, r.o.z}, dd[3] = {r.d.x, r.d.y, r.d.z};
    float lo = 0.0f, hi = __int_as_float(0x7f800000);
    bool miss = false;
#pragma unroll
    for (int a = 0; a < 3; a++) {
        if (dd[a] != 0.0f) {
            const float t0 = __fdiv_rn(__fsub_rn(0.0f, od[a]), dd[a]);
            const float t1 = __fdiv_rn(__fsub_rn(1.0f, od[a]), dd[a]);
            lo = fmaxf(lo, fminf(t0, t1));
            hi = fminf(hi, fmaxf(t0, t1));
        } else if (!(od[a] >= 0.0f && od[a] <= 1.0f)) {
            miss = true;
        }
    }
    float3 C = make_float3(0.f, 0.f, 0.f);
    float A = 0.0f;
    const float kInfF = __int_as_float(0x7f800000);
    float t_first = kInfF, t_any = kInfF;
    float Ad = 0.0f, best = -1.0f, t_best = kInfF, t_acc = kInfF;  // heuristic state (S2a)
    if (!miss && lo < hi) {
        const int n = max(nx, max(ny, nz));
        const float dt = __fdiv_rn(step_vox, (float)n);
        const bool half_step = step_vox == 0.5f;
        for (int j = 0; j < (1 << 24); j++) {  // at most 2^24 samples per ray (spec S2)
            const float tj = __fmaf_rn(__fadd_rn((float)j, 0.5f), dt, lo);
            if (!(tj < hi)) break;
            const float px = __fmaf_rn(r.d.x, tj, r.o.x);
            const float py = __fmaf_rn(r.d.y, tj, r.o.y);
            const float pz = __fmaf_rn(r.d.z, tj, r.o.z);
            const float sv = sample<DT>(vol, nx, ny, nz, px, py, pz);
            const float X = __fmul_rn(sv, 255.0f);
            const int ti = min((int)floorf(X), 254);
            const float ph = __fsub_rn(X, (float)ti);
            const float4 e0 = s_tf[ti], e1 = s_tf[ti + 1];
            const float a = lerp_rn(e0.w, e1.w, ph);  // decision alpha (spec S2)
            if (HEUR == WRS_DEPTH_FIRST_HIT && a >= param && t_first == kInfF) t_first = tj;
            if (a > 0.0f && t_any == kInfF) t_any = tj;
            if (HEUR == WRS_DEPTH_MAX_CONTRIBUTION || HEUR == WRS_DEPTH_ACCUMULATED) {
                const float w = __fmul_rn(__fsub_rn(1.0f, Ad), a);  // this sample's contribution
                Ad = __fadd_rn(Ad, w);
                if (HEUR == WRS_DEPTH_MAX_CONTRIBUTION && w > 0.0f && w > best) { best = w; t_best = tj; }
                if (HEUR == WRS_DEPTH_ACCUMULATED && Ad >= param && t_acc == kInfF) t_acc = tj;
            }
            if (HEUR == WRS_DEPTH_MAX_GRADIENT && a > 0.0f) {
                // squared gradient by central differences one voxel apart
                const float hx = __fdiv_rn(1.0f, (float)nx), hy = __fdiv_rn(1.0f, (float)ny),
                            hz = __fdiv_rn(1.0f, (float)nz);
                const float gx = __fsub_rn(sample<DT>(vol, nx, ny, nz, __fadd_rn(px, hx), py, pz),
                                           sample<DT>(vol, nx, ny, nz, __fsub_rn(px, hx), py, pz));
                const float gy = __fsub_rn(sample<DT>(vol, nx, ny, nz, px, __fadd_rn(py, hy), pz),
                                           sample<DT>(vol, nx, ny, nz, px, __fsub_rn(py, hy), pz));
                const float gz = __fsub_rn(sample<DT>(vol, nx, ny, nz, px, py, __fadd_rn(pz, hz)),
                                           sample<DT>(vol, nx, ny, nz, px, py, __fsub_rn(pz, hz)));
                const float m = __fmaf_rn(gz, gz, __fmaf_rn(gy, gy, __fmul_rn(gx, gx)));
                if (m > best) { best = m; t_best = tj; }
            }
            if (a > 0.0f) {
                const float ac = half_step ? 1.0f - sqrtf(fmaxf(1.0f - a, 0.0f))
                                           : 1.0f - powf(fmaxf(1.0f - a, 0.0f), step_vox);
                const float wgt = (1.0f - A) * ac;
                C.x = fmaf(wgt, fmaf(ph, e1.x - e0.x, e0.x), C.x);
                C.y = fmaf(wgt, fmaf(ph, e1.y - e0.y, e0.y), C.y);
                C.z = fmaf(wgt, fmaf(ph, e1.z - e0.z, e0.z), C.z);
                A = A + wgt;
            }
        }
    }
    rgba_out[pix] = make_float4(C.x, C.y, C.z, A);
    float depth;
    if (HEUR == WRS_DEPTH_MAX_CONTRIBUTION || HEUR == WRS_DEPTH_MAX_GRADIENT) depth = t_best;
    else if (HEUR == WRS_DEPTH_ACCUMULATED) depth = t_acc < kInfF ? t_acc : t_any;
    else depth = t_first < kInfF ? t_first : t_any;
    depth_out[pix] = depth;
}

template <int DT>
void launch_raycast(int heuristic, dim3 grid, cudaStream_t s, const void* vol, int nx, int ny,
                    int nz, const float4* tf, const wrs_camera& cam, float step_vox, float param,
                    float4* o4, float* depth_out) {
    switch (heuristic) {
        case WRS_DEPTH_MAX_CONTRIBUTION:
            k_raycast<DT, WRS_DEPTH_MAX_CONTRIBUTION><<<grid, 128, 0, s>>>(vol, nx, ny, nz, tf, cam,
                                                                            step_vox, param, o4, depth_out);
            break;
        case WRS_DEPTH_ACCUMULATED:
            k_raycast<DT, WRS_DEPTH_ACCUMULATED><<<grid, 128, 0, s>>>(vol, nx, ny, nz, tf, cam,
                                                                       step_vox, param, o4, depth_out);
            break;
        case WRS_DEPTH_MAX_GRADIENT:
            k_raycast<DT, WRS_DEPTH_MAX_GRADIENT><<<grid, 128, 0, s>>>(vol, nx, ny, nz, tf, cam,
                                                                        step_vox, param, o4, depth_out);
            break;
        default:
            k_raycast<DT, WRS_DEPTH_FIRST_HIT><<<grid, 128, 0, s>>>(vol, nx, ny, nz, tf, cam,
                                                                     step_vox, param, o4, depth_out);
    }
}

}  // namespace

extern "C" int wrs_raycast_volume_heuristic(const void* vol, int32_t dtype, int32_t nx,
                                            int32_t ny, int32_t nz, const float* tf,
                                            const wrs_camera* cam, float step_vox,
                                            int32_t heuristic, float param, float* rgba_out,
                                            float* depth_out, wrs_stream_t stream) {
    const char* fn = "wrs_raycast_volume";
    if (int rc = wrs::check_camera(cam, fn)) return rc;
    if (!vol || !tf || !rgba_out || !depth_out)
        return wrs::fail(WRS_ERR_ARG, "%s: NULL pointer", fn);
    if (dtype != WRS_F32 && dtype != WRS_U8)
        return wrs::fail(WRS_ERR_ARG, "%s: unknown dtype %d", fn, dtype);
    if (nx < 1 || ny < 1 || nz < 1 || nx > 16384 || ny > 16384 || nz > 16384)
        return wrs::fail(WRS_ERR_ARG, "%s: volume size %dx%dx%d out of range", fn, nx, ny, nz);
    if (!(step_vox >= 1e-3f && step_vox <= 1e3f))
        return wrs::fail(WRS_ERR_ARG, "%s: step_vox must be in [1e-3, 1e3] voxels", fn);
    if (heuristic < WRS_DEPTH_FIRST_HIT || heuristic > WRS_DEPTH_MAX_GRADIENT)
        return wrs::fail(WRS_ERR_ARG, "%s: unknown depth heuristic %d", fn, heuristic);
    if (!(param == param)) return wrs::fail(WRS_ERR_ARG, "%s: heuristic parameter is NaN", fn);
    if ((reinterpret_cast<uintptr_t>(tf) | reinterpret_cast<uintptr_t>(rgba_out)) & 15)
        return wrs::fail(WRS_ERR_ARG, "%s: tf and rgba_out must be 16-byte aligned", fn);
    dim3 grid((cam->width + 15) / 16, (cam->height + 7) / 8);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const float4* tf4 = reinterpret_cast<const float4*>(tf);
    float4* o4 = reinterpret_cast<float4*>(rgba_out);
    if (dtype == WRS_U8)
        launch_raycast<WRS_U8>(heuristic, grid, s, vol, nx, ny, nz, tf4, *cam, step_vox, param, o4, depth_out);
    else
        launch_raycast<WRS_F32>(heuristic, grid, s, vol, nx, ny, nz, tf4, *cam, step_vox, param, o4, depth_out);
    WRS_LAUNCH_CHECK(fn);
    return WRS_OK;
}

extern "C" int wrs_raycast_volume(const void* vol, int32_t dtype, int32_t nx, int32_t ny,
                                  int32_t nz, const float* tf, const wrs_camera* cam,
                                  float step_vox, float tau, float* rgba_out, float* depth_out,
                                  wrs_stream_t stream) {
    return wrs_raycast_volume_heuristic(vol, dtype, nx, ny, nz, tf, cam, step_vox,
                                        WRS_DEPTH_FIRST_HIT, tau, rgba_out, depth_out, stream);
}
