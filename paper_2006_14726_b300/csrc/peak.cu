// peak.cu -- measurement kernels for the roofline's denominators: binary32 FMA throughput, which
// on this GPU is also the warp-instruction issue rate of ALU-bound code (one FFMA per lane per
// cycle on every scheduler), and a streaming copy (HBM or L2 copy rate, by buffer size).  Not
// part of the method; bench.py times them with CUDA events.
#include "common.cuh"

namespace {

constexpr int kChains = 8;    // independent FMA chains per thread (hide the FMA latency)
constexpr int kUnroll = 16;   // chain steps per loop iteration: 128 FMAs per iteration

__global__ void __launch_bounds__(256) k_fma_peak(float* __restrict__ out, int iters, float a,
                                                  float b) {
    float x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; c++) x[c] = 1.0f + 1e-3f * (float)(threadIdx.x + c);
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int u = 0; u < kUnroll; u++) {
#pragma unroll
            for (int c = 0; c < kChains; c++) x[c] = fmaf(x[c], a, b);
        }
    }
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < kChains; c++) s += x[c];
    // with 0 < a < 1 and b > 0 every chain stays positive: the store never happens, but the
    // compiler cannot know that, so the chains are computed
    if (s < 0.0f) out[blockIdx.x] = s;
}

// Streaming copy, grid-stride, four 16-byte loads in flight per thread before their stores:
// dst[i] = src[i] for n float4, `reps` times over the buffer.  Over a buffer far larger than L2 it
// measures the HBM copy rate; over one that fits in L2 (with reps > 1), the L2 rate.
__global__ void __launch_bounds__(256) k_stream_copy(float4* __restrict__ dst,
                                                     const float4* __restrict__ src, size_t n,
                                                     int reps) {
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (int r = 0; r < reps; r++) {
        size_t i = t;
        for (; i + 3 * stride < n; i += 4 * stride) {
            const float4 a = __ldcg(src + i), b = __ldcg(src + i + stride);
            const float4 c = __ldcg(src + i + 2 * stride), d = __ldcg(src + i + 3 * stride);
            __stcg(dst + i, a);
            __stcg(dst + i + stride, b);
            __stcg(dst + i + 2 * stride, c);
            __stcg(dst + i + 3 * stride, d);
        }
        for (; i < n; i += stride) __stcg(dst + i, __ldcg(src + i));
    }
}

}  // namespace

extern "C" {

int wrs_stream_copy(void* dst, const void* src, size_t bytes, int32_t blocks, int32_t reps,
                    wrs_stream_t stream) {
    if (!dst || !src || blocks < 1 || reps < 1 || (bytes & 15) ||
        ((reinterpret_cast<uintptr_t>(dst) | reinterpret_cast<uintptr_t>(src)) & 15))
        return wrs::fail(WRS_ERR_ARG, "wrs_stream_copy: NULL or misaligned buffer, bytes not a "
                                      "multiple of 16, blocks < 1 or reps < 1");
    k_stream_copy<<<blocks, 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
        static_cast<float4*>(dst), static_cast<const float4*>(src), bytes / 16, reps);
    WRS_LAUNCH_CHECK("wrs_stream_copy");
    return WRS_OK;
}

int wrs_fma_peak(float* out, int32_t blocks, int32_t iters, wrs_stream_t stream) {
    if (!out || blocks < 1 || iters < 1)
        return wrs::fail(WRS_ERR_ARG, "wrs_fma_peak: out NULL, blocks < 1 or iters < 1");
    k_fma_peak<<<blocks, 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(out, iters, 0.999f,
                                                                            0.001f);
    WRS_LAUNCH_CHECK("wrs_fma_peak");
    return WRS_OK;
}

}  // extern "C"
