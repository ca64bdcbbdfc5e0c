// peak.cu -- measurement kernel for the compute side of the roofline: binary32 FMA throughput,
// which on this GPU is also the warp-instruction issue rate of ALU-bound code (one FFMA per lane
// per cycle on every scheduler).  Not part of the method; bench.py times it with CUDA events.
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

}  // namespace

extern "C" {

int wrs_fma_peak(float* out, int32_t blocks, int32_t iters, wrs_stream_t stream) {
    if (!out || blocks < 1 || iters < 1)
        return wrs::fail(WRS_ERR_ARG, "wrs_fma_peak: out NULL, blocks < 1 or iters < 1");
    k_fma_peak<<<blocks, 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(out, iters, 0.999f,
                                                                            0.001f);
    WRS_LAUNCH_CHECK("wrs_fma_peak");
    return WRS_OK;
}

}  // extern "C"
