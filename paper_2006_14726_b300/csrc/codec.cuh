// codec.cuh -- the 64-bit quantised position + radius word and the 32-bit colour the server sends
// (§4.1, §6); the paper gives no bit layout, this library's reading (spec S11):
//   word  = qx | qy << 17 | qz << 34 | qr << 51   (17-bit cells over a caller box, 13-bit radius)
//   color = r | g << 8 | b << 16 | a << 24        (8-bit premultiplied channels)
// All quantisation steps are binary32 with a fixed operation order (the __f*_rn intrinsics).
#pragma once

#include "common.cuh"

namespace wrs {

struct CodecConsts {
    float lo[3];
    float inv[3];   // 131072 / (hi - lo)
    float step[3];  // (hi - lo) * 2^-17
    float rinv;     // 8191 / r_max
    float rstep;    // r_max / 8191
};

__host__ __device__ inline CodecConsts make_codec(const wrs_codec& c) {
    CodecConsts k;
    for (int a = 0; a < 3; a++) {
        const float ext = c.hi[a] - c.lo[a];
        k.lo[a] = c.lo[a];
        k.inv[a] = 131072.0f / ext;
        k.step[a] = ext * 0x1p-17f;
    }
    k.rinv = 8191.0f / c.r_max;
    k.rstep = c.r_max / 8191.0f;
    return k;
}

__device__ __forceinline__ uint32_t quant_floor(float u, uint32_t top) {
    if (!(fabsf(u) <= 3.4028235e38f)) return 0u;  // not finite
    const float f = floorf(u);
    if (f < 0.0f) return 0u;
    if (f > (float)top) return top;
    return (uint32_t)f;
}

__device__ __forceinline__ uint64_t encode_word(const CodecConsts& k, float x, float y, float z,
                                                float r) {
    const uint64_t qx = quant_floor(__fmul_rn(__fsub_rn(x, k.lo[0]), k.inv[0]), 131071u);
    const uint64_t qy = quant_floor(__fmul_rn(__fsub_rn(y, k.lo[1]), k.inv[1]), 131071u);
    const uint64_t qz = quant_floor(__fmul_rn(__fsub_rn(z, k.lo[2]), k.inv[2]), 131071u);
    // the radius is rounded up, so that a decoded sphere still covers its footprint
    const float v = __fmul_rn(r, k.rinv);
    uint64_t qr = 0;
    if (fabsf(v) <= 3.4028235e38f) {
        const float c = ceilf(v);
        qr = c < 0.0f ? 0u : (c > 8191.0f ? 8191u : (uint64_t)c);
    }
    return qx | (qy << 17) | (qz << 34) | (qr << 51);
}

__device__ __forceinline__ uint32_t encode_color(float4 c) {
    const uint32_t r = quant_floor(__fadd_rn(__fmul_rn(c.x, 255.0f), 0.5f), 255u);
    const uint32_t g = quant_floor(__fadd_rn(__fmul_rn(c.y, 255.0f), 0.5f), 255u);
    const uint32_t b = quant_floor(__fadd_rn(__fmul_rn(c.z, 255.0f), 0.5f), 255u);
    const uint32_t a = quant_floor(__fadd_rn(__fmul_rn(c.w, 255.0f), 0.5f), 255u);
    return r | (g << 8) | (b << 16) | (a << 24);
}

__device__ __forceinline__ float4 decode_pos_r(const CodecConsts& k, uint64_t w) {
    const float x = __fmaf_rn(__fadd_rn((float)(uint32_t)(w & 0x1FFFFu), 0.5f), k.step[0], k.lo[0]);
    const float y = __fmaf_rn(__fadd_rn((float)(uint32_t)((w >> 17) & 0x1FFFFu), 0.5f), k.step[1], k.lo[1]);
    const float z = __fmaf_rn(__fadd_rn((float)(uint32_t)((w >> 34) & 0x1FFFFu), 0.5f), k.step[2], k.lo[2]);
    const float r = __fmul_rn((float)(uint32_t)(w >> 51), k.rstep);
    return make_float4(x, y, z, r);
}

__device__ __forceinline__ float4 decode_color(uint32_t c) {
    return make_float4(__fdiv_rn((float)(c & 255u), 255.0f), __fdiv_rn((float)((c >> 8) & 255u), 255.0f),
                       __fdiv_rn((float)((c >> 16) & 255u), 255.0f), __fdiv_rn((float)(c >> 24), 255.0f));
}

// host-side validation shared by the codec entry points
int check_codec(const wrs_codec* c, const char* fn);

}  // namespace wrs
