// common.cuh -- device-side definitions shared by the libwrs kernels.
//
// Decision arithmetic (primary rays, the ray-sphere test, Morton quantisation, volume samples)
// follows the written spec's binary32 operation order exactly.  It is spelled with the __f*_rn
// intrinsics so that nvcc can neither contract a multiply-add nor re-associate: a hit, a hit
// order or a threshold crossing is then decided the same way by every correct implementation of
// the spec.  Continuous quantities (colours, transmittance, gradients) use ordinary arithmetic.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "wrs.h"

namespace wrs {

constexpr uint32_t kLeafBit = 0x80000000u;
constexpr uint32_t kNoChild = 0xFFFFFFFFu;  // unused entry of a 4-wide node
constexpr int kStack = 96;         // traversal stack entries (binary: <= depth; 4-wide: <= 1.5 depth)
constexpr int kMaxLeaf = 16;
constexpr int kBwdChunks = 64;     // backward: traversal passes per ray it can replay

// 64-byte header at the start of an LBVH buffer; internal nodes follow it.
struct LbvhHeader {
    uint32_t n;        // splats
    uint32_t m;        // leaves = ceil(n / leaf)
    uint32_t leaf;     // splats per leaf
    int32_t root;      // internal node 0, or kLeafBit | 0 when there is a single leaf
    float cmin[3];     // centre bounds used by the Morton quantisation
    float cmax[3];
    float maxabs;      // largest |coordinate| of any sphere bound (traversal epsilon scale)
    float rmax;        // largest effective radius
    uint32_t wide_start;  // 64-byte slots of binary nodes before the 4-wide nodes
    uint32_t layout;      // WRS_LBVH_FULL or WRS_LBVH_WIDE (the binary records are not all written)
    uint32_t pad[2];
};
static_assert(sizeof(LbvhHeader) == 64, "header must be 64 bytes");

// Binary internal node = 4 x float4 = 64 B:
//   floats 0..5  : child 0 box (lo.xyz, hi.xyz)
//   floats 6..11 : child 1 box
//   floats 12,13 : child references (int bits; kLeafBit set = leaf index)
//   floats 14,15 : unused
// 4-wide node i (one per binary internal node i) = 8 x float4 = 128 B, structure of arrays over
// the grandchildren of binary node i (a leaf child counts as its own grandchild):
//   float4 0..2: lo.x, lo.y, lo.z of the 4 entries; 3..5: hi.x, hi.y, hi.z; 6: references
//   (int bits; internal references name binary nodes, whose 4-wide node is visited next); 7: zero
//   (written all the same: a 32-byte sector written in part costs DRAM a read-modify-write).
//   Unused entries carry the reference kNoChild, low x = +inf and high x = -inf (their other
//   planes are not written): the direction-ordered slab test (box_test_nf) gets tn = +inf from
//   the x slab and tf = -inf (three-input min/max ignore a NaN in the other planes), so no ray
//   enters them.
__host__ __device__ inline float4* lbvh_nodes(void* buf) {
    return reinterpret_cast<float4*>(reinterpret_cast<char*>(buf) + sizeof(LbvhHeader));
}
__host__ __device__ inline const float4* lbvh_nodes(const void* buf) {
    return reinterpret_cast<const float4*>(reinterpret_cast<const char*>(buf) + sizeof(LbvhHeader));
}
// binary node slots reserved for a capacity (the 4-wide nodes start after them)
__host__ __device__ inline uint32_t lbvh_binary_slots(uint32_t capacity, uint32_t leaf) {
    const uint32_t m = capacity == 0 ? 1 : (capacity + leaf - 1) / leaf;
    return m > 1 ? m - 1 : 1;
}

// ---------------------------------------------------------------------------------------------
// Spec S1: primary ray of pixel (x, y).
// ---------------------------------------------------------------------------------------------
struct Ray {
    float3 o, d;
};

__device__ __forceinline__ Ray primary_ray(const wrs_camera& c, int x, int y) {
    const float W = (float)c.width, H = (float)c.height;
    const float aspect = __fdiv_rn(W, H);
    const float sx = __fmul_rn(c.tan_half_fovy, aspect);
    const float u = __fmul_rn(__fsub_rn(__fdiv_rn((float)(2 * x + 1), W), 1.0f), sx);
    const float v = __fmul_rn(__fsub_rn(1.0f, __fdiv_rn((float)(2 * y + 1), H)), c.tan_half_fovy);
    const float ex = __fmaf_rn(v, c.up[0], __fmaf_rn(u, c.right[0], c.fwd[0]));
    const float ey = __fmaf_rn(v, c.up[1], __fmaf_rn(u, c.right[1], c.fwd[1]));
    const float ez = __fmaf_rn(v, c.up[2], __fmaf_rn(u, c.right[2], c.fwd[2]));
    const float len2 = __fmaf_rn(ez, ez, __fmaf_rn(ey, ey, __fmul_rn(ex, ex)));
    const float inv = __fdiv_rn(1.0f, __fsqrt_rn(len2));
    Ray r;
    r.o = make_float3(c.eye[0], c.eye[1], c.eye[2]);
    r.d = make_float3(__fmul_rn(ex, inv), __fmul_rn(ey, inv), __fmul_rn(ez, inv));
    return r;
}

// ---------------------------------------------------------------------------------------------
// Spec S5: ray-sphere test.  s = (centre, effective radius).  On a hit returns the entry key
// max(b - sqrt(q), 0) and |f|^2 (the squared distance of the centre from the ray).
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ bool sphere_hit(const Ray& r, const float4 s, float& key, float& ff) {
    const float ocx = __fsub_rn(s.x, r.o.x);
    const float ocy = __fsub_rn(s.y, r.o.y);
    const float ocz = __fsub_rn(s.z, r.o.z);
    const float b = __fmaf_rn(ocz, r.d.z, __fmaf_rn(ocy, r.d.y, __fmul_rn(ocx, r.d.x)));
    const float nb = -b;
    const float fx = __fmaf_rn(nb, r.d.x, ocx);
    const float fy = __fmaf_rn(nb, r.d.y, ocy);
    const float fz = __fmaf_rn(nb, r.d.z, ocz);
    ff = __fmaf_rn(fz, fz, __fmaf_rn(fy, fy, __fmul_rn(fx, fx)));
    const float q = __fmaf_rn(s.w, s.w, -ff);
    if (!(q > 0.0f)) return false;
    const float sq = __fsqrt_rn(q);
    if (!(__fadd_rn(b, sq) > 0.0f)) return false;
    const float k0 = __fsub_rn(b, sq);
    key = k0 > 0.0f ? k0 : 0.0f;
    return true;
}

// (key, id) strict lexicographic order of hits (spec S5).
__device__ __forceinline__ bool hit_less(float ka, uint32_t ia, float kb, uint32_t ib) {
    return ka < kb || (ka == kb && ia < ib);
}

// ---------------------------------------------------------------------------------------------
// Conservative ray-box slab test.  Boxes are widened by eps so that no sphere the binary32 test
// would hit is ever culled (the box test only prunes; it never decides a result).
// ---------------------------------------------------------------------------------------------
struct BoxRay {
    float ix, iy, iz;      // 1 / d (guarded against zero components)
    float lx, ly, lz;      // -(o + eps) / d  : offset for the low planes
    float hx, hy, hz;      // -(o - eps) / d  : offset for the high planes
    // the same planes ordered by the ray's direction: the near one of each axis is the low plane
    // when 1/d >= 0, else the high one (used by the 4-wide nodes, whose low and high planes sit in
    // separate float4s, so that the ordering costs an address offset instead of min/max pairs)
    float nx, ny, nz;      // offset of the near plane per axis
    float fx, fy, fz;      // offset of the far plane per axis
    int sx, sy, sz;        // 0 if the near plane is the low one, 3 if it is the high one
};

__device__ __forceinline__ BoxRay make_box_ray(const Ray& r, float eps) {
    auto guard = [](float v) { return fabsf(v) < 1e-12f ? copysignf(1e-12f, v) : v; };
    BoxRay b;
    // correctly rounded reciprocals (the value of 1.0f / x, without the division's slow path)
    b.ix = __frcp_rn(guard(r.d.x));
    b.iy = __frcp_rn(guard(r.d.y));
    b.iz = __frcp_rn(guard(r.d.z));
    b.lx = -(r.o.x + eps) * b.ix;
    b.ly = -(r.o.y + eps) * b.iy;
    b.lz = -(r.o.z + eps) * b.iz;
    b.hx = -(r.o.x - eps) * b.ix;
    b.hy = -(r.o.y - eps) * b.iy;
    b.hz = -(r.o.z - eps) * b.iz;
    const bool px = b.ix >= 0.0f, py = b.iy >= 0.0f, pz = b.iz >= 0.0f;
    b.nx = px ? b.lx : b.hx;  b.fx = px ? b.hx : b.lx;  b.sx = px ? 0 : 3;
    b.ny = py ? b.ly : b.hy;  b.fy = py ? b.hy : b.ly;  b.sy = py ? 0 : 3;
    b.nz = pz ? b.lz : b.hz;  b.fz = pz ? b.hz : b.lz;  b.sz = pz ? 0 : 3;
    return b;
}

// Three-input minimum / maximum (one instruction on sm_100 and later).
__device__ __forceinline__ float max3f(float a, float b, float c) {
    float d;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}
__device__ __forceinline__ float min3f(float a, float b, float c) {
    float d;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}

// Slab test of one box given by its low and high corners (either ray direction).
__device__ __forceinline__ void box_test(const BoxRay& r, float lox, float loy, float loz,
                                         float hix, float hiy, float hiz, float& tn, float& tf) {
    const float ax = fmaf(lox, r.ix, r.lx), bx = fmaf(hix, r.ix, r.hx);
    const float ay = fmaf(loy, r.iy, r.ly), by = fmaf(hiy, r.iy, r.hy);
    const float az = fmaf(loz, r.iz, r.lz), bz = fmaf(hiz, r.iz, r.hz);
    tn = max3f(fminf(ax, bx), fminf(ay, by), fmaxf(fminf(az, bz), 0.0f));
    tf = min3f(fmaxf(ax, bx), fmaxf(ay, by), fmaxf(az, bz));
}

// The same test given the box's near and far plane coordinates for this ray (selected by the
// sign of its direction), with a lower bound `low` >= 0 folded into the near distance: the ray
// meets the box beyond `low` iff tn <= tf.  An empty box (low corner +inf, high corner -inf)
// gives tn = +inf and tf = -inf, so it never passes.
__device__ __forceinline__ void box_test_nf(const BoxRay& r, float nx, float ny, float nz,
                                            float fx, float fy, float fz, float low, float& tn,
                                            float& tf) {
    const float ax = fmaf(nx, r.ix, r.nx), bx = fmaf(fx, r.ix, r.fx);
    const float ay = fmaf(ny, r.iy, r.ny), by = fmaf(fy, r.iy, r.fy);
    const float az = fmaf(nz, r.iz, r.nz), bz = fmaf(fz, r.iz, r.fz);
    tn = max3f(ax, ay, fmaxf(az, low));
    tf = min3f(bx, by, bz);
}

// Two single-precision FMAs in one packed instruction (each lane rounds to nearest, as fmaf).
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) {
    unsigned long long ra, rb, rc, rd;
    asm("mov.b64 %0, {%1, %2};" : "=l"(ra) : "f"(a.x), "f"(a.y));
    asm("mov.b64 %0, {%1, %2};" : "=l"(rb) : "f"(b.x), "f"(b.y));
    asm("mov.b64 %0, {%1, %2};" : "=l"(rc) : "f"(c.x), "f"(c.y));
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(rd) : "l"(ra), "l"(rb), "l"(rc));
    float2 d;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(d.x), "=f"(d.y) : "l"(rd));
    return d;
}

// box_test_nf for two boxes at once (two slots of a 4-wide node, whose planes sit side by side
// in the node's float4s): the six slab products as packed pairs, bitwise the scalar results.
__device__ __forceinline__ void box_test_nf2(const BoxRay& r, float2 nx, float2 ny, float2 nz,
                                             float2 fx, float2 fy, float2 fz, float low,
                                             float& tn0, float& tf0, float& tn1, float& tf1) {
    const float2 ix = make_float2(r.ix, r.ix), iy = make_float2(r.iy, r.iy);
    const float2 iz = make_float2(r.iz, r.iz);
    const float2 ax = fma2(nx, ix, make_float2(r.nx, r.nx)), bx = fma2(fx, ix, make_float2(r.fx, r.fx));
    const float2 ay = fma2(ny, iy, make_float2(r.ny, r.ny)), by = fma2(fy, iy, make_float2(r.fy, r.fy));
    const float2 az = fma2(nz, iz, make_float2(r.nz, r.nz)), bz = fma2(fz, iz, make_float2(r.fz, r.fz));
    tn0 = max3f(ax.x, ay.x, fmaxf(az.x, low));
    tf0 = min3f(bx.x, by.x, bz.x);
    tn1 = max3f(ax.y, ay.y, fmaxf(az.y, low));
    tf1 = min3f(bx.y, by.y, bz.y);
}

// Traversal epsilon: far above the binary32 error of the sphere test (a few units in the last
// place of |o| + |c|), far below a sphere radius.
__device__ __forceinline__ float traversal_eps(const Ray& r, float scene_maxabs) {
    const float om = fmaxf(fmaxf(fabsf(r.o.x), fabsf(r.o.y)), fabsf(r.o.z));
    return 1e-6f * (1.0f + om + scene_maxabs);
}

// Soft edge weight W(rho) of spec S6 and its derivative.
__device__ __forceinline__ float soft_w(float rho, float beta) {
    if (beta <= 0.0f || rho <= 1.0f - beta) return 1.0f;
    float u = fmaxf((1.0f - rho) / beta, 0.0f);
    return u * u * (3.0f - 2.0f * u);
}
__device__ __forceinline__ float soft_dw(float rho, float beta) {
    if (beta <= 0.0f || rho <= 1.0f - beta) return 0.0f;
    float u = (1.0f - rho) / beta;
    if (u < 0.0f) return 0.0f;
    return -6.0f * u * (1.0f - u) / beta;
}

__device__ __forceinline__ void set_status(int32_t* status, uint32_t bits) {
    if (status) atomicOr(reinterpret_cast<unsigned int*>(status), bits);
}

}  // namespace wrs

// host-side error plumbing shared by the entry points
namespace wrs {
int fail(int code, const char* fmt, ...);
int cuda_fail(cudaError_t e, const char* what);
}  // namespace wrs

#define WRS_LAUNCH_CHECK(what)                                         \
    do {                                                               \
        cudaError_t e_ = cudaGetLastError();                           \
        if (e_ != cudaSuccess) return ::wrs::cuda_fail(e_, what);      \
    } while (0)
