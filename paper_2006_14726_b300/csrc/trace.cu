// trace.cu -- ray tracing of the splat spheres (Fig. 2 caption, §4; spec S5, S6), its counting
// variant, several views of one scene in one launch, the multi-session launches, and the adjoint
// (spec S7).
//
// Per ray: ordered BVH traversal with a short stack whose entries carry their boxes' entry
// distances; the K nearest hits beyond the previous pass are kept sorted by (key, id) in
// registers; nodes whose entry lies beyond the K-th key (or whose exit lies before the previous
// pass's last key) are culled, when tested and again when popped; after each pass the K hits are
// composited front to back.  A ray stops once its transmittance reaches t_stop, H hits are used,
// or a pass finds fewer than K hits.  With 4-wide nodes the per-pixel kernels run each lane's
// traversal in warp-wide steps: leaf entries are sorted and stacked with the internal ones, and
// each iteration of the warp takes either a node step or a leaf step for the lanes that want it.  The 4-wide traversal (the default) reads seven float4 of a
// 128-B node per visit (the near and far planes of the ray's direction, and the references); the
// binary traversal reads a 64-B node (four float4); both through the read-only path.  A splat is
// one float4 for the test and one float4 for its colour.
//
// Results do not depend on K, the block shape or the LBVH leaf size: the hit set and order are
// fixed by the binary32 sphere test, and the compositing visits them in the same order.
#include "common.cuh"

namespace wrs {
int check_camera(const wrs_camera* c, const char* fn);
}

namespace {

using wrs::kLeafBit;
using wrs::LbvhHeader;
using wrs::Ray;

struct Scene {
    const LbvhHeader* hdr;
    const float4* __restrict__ nodes;
    const float4* __restrict__ wide;  // 4-wide nodes, or nullptr to traverse the binary nodes
    const float4* __restrict__ pos_r;
    const float4* __restrict__ rgba;
    const uint32_t* __restrict__ id;
    const uint32_t* __restrict__ src;
    const float* __restrict__ opacity;
};

struct Comp {
    int max_hits;
    float t_stop;
    float beta;
    int width;  // 2: binary traversal; 4: 4-wide traversal
};

struct Counts {
    uint32_t nodes, boxes, spheres, gathered, composited, passes;
};

// The composited hits of the rays of a multi-view launch, recorded by the forward pass for a
// traversal-free adjoint: the sorted-splat indices in compositing order, hits[ray * cap + i], and
// their number count[ray] (cap + 1: the ray composited more than cap hits; none are kept and the
// adjoint re-traverses it).  ray = view * pixels + pixel.
struct HitRecord {
    uint32_t* hits;
    uint32_t* count;
    uint32_t cap;
};
// The rays a re-traversing adjoint launch handles: all (count == nullptr), or only those whose
// recorded list went over capacity.
struct HitFilter {
    const uint32_t* count;
    uint32_t cap;
};

constexpr float kInf = __builtin_huge_valf();

// A traversal stack entry: the node reference in the low word and the entry distance of its box
// (>= 0, so its bits order like the value) in the high word.  A popped node whose box starts
// beyond the current K-th nearest hit is dropped without a visit: its children would all fail
// the same cut-off, so the result is unchanged.
using StackEntry = unsigned long long;
__device__ __forceinline__ StackEntry stack_entry(uint32_t ref, float tn) {
    return ((StackEntry)__float_as_uint(tn) << 32) | ref;
}
__device__ __forceinline__ float entry_tn(StackEntry e) { return __uint_as_float((uint32_t)(e >> 32)); }

// Pop the nearest pending node that still starts within the cut-off; false when none is left.
__device__ __forceinline__ bool pop_within(const StackEntry* stack, int& sp, float cutoff,
                                           uint32_t& ref) {
    while (sp > 0) {
        const StackEntry e = stack[--sp];
        if (entry_tn(e) <= cutoff) {
            ref = (uint32_t)e;
            return true;
        }
    }
    return false;
}
// Plain entries (the reference only; the lane-refill state machines keep these: they hold more
// state, and the wider entries cost them registers).
__device__ __forceinline__ int stack_entry_plain(uint32_t ref, float) { return (int)ref; }
__device__ __forceinline__ bool pop_within(const int* stack, int& sp, float, uint32_t& ref) {
    if (sp == 0) return false;
    ref = (uint32_t)stack[--sp];
    return true;
}
template <typename E>
__device__ __forceinline__ E make_entry(uint32_t ref, float tn) {
    return stack_entry(ref, tn);
}
template <>
__device__ __forceinline__ int make_entry<int>(uint32_t ref, float tn) {
    return stack_entry_plain(ref, tn);
}

// Test the splats of leaf `leafref` and insert qualifying hits into the sorted K-buffer: hits
// strictly after (last_key, last_id) when has_last, keeping the K smallest (key, id).  The final
// buffer does not depend on the order in which leaves are visited.
template <int K, bool COUNT>
__device__ __forceinline__ void leaf_hits(const Scene& sc, const Ray& ray, uint32_t leafref,
                                          uint32_t n, uint32_t leaf, bool has_last, float last_key,
                                          uint32_t last_id, float (&kk)[K], uint32_t (&ki)[K],
                                          uint32_t (&kid)[K], int& count, Counts& cnt) {
    const float lower = has_last ? last_key : -kInf;
    const uint32_t j = leafref & ~kLeafBit;
    if (j >= (n + leaf - 1) / leaf) return;  // not a leaf of this tree
    const uint32_t first = j * leaf;
    const uint32_t last = min(first + leaf, n);
    for (uint32_t k = first; k < last; k++) {
        const float4 s = __ldg(sc.pos_r + k);
        float key, ff;
        if (COUNT) cnt.spheres++;
        if (!wrs::sphere_hit(ray, s, key, ff)) continue;
        if (key > kk[K - 1] || key < lower) continue;
        const uint32_t hid = __ldg(sc.id + k);
        if (has_last && !wrs::hit_less(last_key, last_id, key, hid)) continue;
        if (!wrs::hit_less(key, hid, kk[K - 1], kid[K - 1])) continue;
        // bubble the new hit into the sorted buffer; the old K-th entry drops out
        float nk = key;
        uint32_t ni = k, nid = hid;
#pragma unroll
        for (int s2 = 0; s2 < K; s2++) {
            const bool lt = wrs::hit_less(nk, nid, kk[s2], kid[s2]);
            const float tk = kk[s2];
            const uint32_t ti = ki[s2], tid = kid[s2];
            kk[s2] = lt ? nk : tk; ki[s2] = lt ? ni : ti; kid[s2] = lt ? nid : tid;
            nk = lt ? tk : nk; ni = lt ? ti : ni; nid = lt ? tid : nid;
        }
        count = min(count + 1, K);
        if (COUNT) cnt.gathered++;
    }
}

// One visit of internal node `ref`: test both child boxes; the splats of a hit leaf child are
// tested right away (so every traversal step is a node step and lanes do not diverge between
// node and leaf code); hit internal children are descended into, nearer first, the other pushed.
// Returns the next internal node, or kLeafBit when the pass must pop; -1 stack overflow,
// -2 malformed reference.
template <int K, bool COUNT, typename E>
__device__ __forceinline__ int64_t visit_node(const Scene& sc, const Ray& ray,
                                              const wrs::BoxRay& br, uint32_t ref, uint32_t n,
                                              uint32_t leaf, uint32_t m, bool has_last,
                                              float last_key, uint32_t last_id, float (&kk)[K],
                                              uint32_t (&ki)[K], uint32_t (&kid)[K], int& count,
                                              E* stack, int& sp, Counts& cnt) {
    if (ref + 1 >= m) return -2;  // not an internal node of this tree
    const float lower = has_last ? last_key : -kInf;
    const float4* nd = sc.nodes + 4 * (size_t)ref;
    const float4 a = __ldg(nd + 0), b = __ldg(nd + 1), c = __ldg(nd + 2), r = __ldg(nd + 3);
    float tn0, tf0, tn1, tf1;
    wrs::box_test(br, a.x, a.y, a.z, a.w, b.x, b.y, tn0, tf0);
    wrs::box_test(br, b.z, b.w, c.x, c.y, c.z, c.w, tn1, tf1);
    if (COUNT) { cnt.nodes++; cnt.boxes += 2; }
    const uint32_t c0 = __float_as_uint(r.x), c1 = __float_as_uint(r.y);
    bool h0 = tn0 <= tf0 && tn0 <= kk[K - 1] && tf0 >= lower;
    bool h1 = tn1 <= tf1 && tn1 <= kk[K - 1] && tf1 >= lower;
    if (h0 && (c0 & kLeafBit)) {
        leaf_hits<K, COUNT>(sc, ray, c0, n, leaf, has_last, last_key, last_id, kk, ki, kid, count, cnt);
        h0 = false;
    }
    if (h1 && (c1 & kLeafBit)) {
        leaf_hits<K, COUNT>(sc, ray, c1, n, leaf, has_last, last_key, last_id, kk, ki, kid, count, cnt);
        h1 = false;
    }
    if (h0 && h1) {
        const bool first0 = tn0 <= tn1;
        if (sp >= wrs::kStack) return -1;
        stack[sp++] = first0 ? make_entry<E>(c1, tn1) : make_entry<E>(c0, tn0);
        return first0 ? c0 : c1;
    }
    if (h0) return c0;
    if (h1) return c1;
    return kLeafBit;
}

__device__ __forceinline__ void cswap(float& ka, uint32_t& ra, float& kb, uint32_t& rb) {
    const bool s = kb < ka;
    const float tk = s ? kb : ka;
    const uint32_t tr = s ? rb : ra;
    kb = s ? ka : kb;
    rb = s ? ra : rb;
    ka = tk;
    ra = tr;
}

// One visit of the 4-wide node of binary node `ref` (its grandchildren): four box tests from
// structure-of-arrays loads; hit leaf entries are tested right away; hit internal entries are
// sorted by entry distance (5-comparator network), the nearest is returned and the others pushed
// far to near.  Same return convention as visit_node.  (The lane-refill schedule's visit; the
// per-pixel kernels use visit_node4_sorted, which stacks leaf entries too.)
#ifndef WRS_PACKED_MAX_K
#define WRS_PACKED_MAX_K 4  // K 8 and 16 measured faster with one box at a time (register pressure)
#endif
// The four box tests of a 4-wide node visit: slot pairs with packed FMAs (K <= WRS_PACKED_MAX_K)
// or one box at a time; bitwise the same distances.
template <int K>
__device__ __forceinline__ void box_tests4(const wrs::BoxRay& br, const float4& nx,
                                           const float4& ny, const float4& nz, const float4& fx,
                                           const float4& fy, const float4& fz, float low,
                                           float (&tn)[4], float (&tf)[4]) {
    if constexpr (K <= WRS_PACKED_MAX_K) {
        wrs::box_test_nf2(br, make_float2(nx.x, nx.y), make_float2(ny.x, ny.y),
                          make_float2(nz.x, nz.y), make_float2(fx.x, fx.y),
                          make_float2(fy.x, fy.y), make_float2(fz.x, fz.y), low, tn[0], tf[0],
                          tn[1], tf[1]);
        wrs::box_test_nf2(br, make_float2(nx.z, nx.w), make_float2(ny.z, ny.w),
                          make_float2(nz.z, nz.w), make_float2(fx.z, fx.w),
                          make_float2(fy.z, fy.w), make_float2(fz.z, fz.w), low, tn[2], tf[2],
                          tn[3], tf[3]);
    } else {
        wrs::box_test_nf(br, nx.x, ny.x, nz.x, fx.x, fy.x, fz.x, low, tn[0], tf[0]);
        wrs::box_test_nf(br, nx.y, ny.y, nz.y, fx.y, fy.y, fz.y, low, tn[1], tf[1]);
        wrs::box_test_nf(br, nx.z, ny.z, nz.z, fx.z, fy.z, fz.z, low, tn[2], tf[2]);
        wrs::box_test_nf(br, nx.w, ny.w, nz.w, fx.w, fy.w, fz.w, low, tn[3], tf[3]);
    }
}

template <int K, bool COUNT, typename E>
__device__ __forceinline__ int64_t visit_node4(const Scene& sc, const Ray& ray,
                                               const wrs::BoxRay& br, uint32_t ref, uint32_t n,
                                               uint32_t leaf, uint32_t m, bool has_last,
                                               float last_key, uint32_t last_id, float (&kk)[K],
                                               uint32_t (&ki)[K], uint32_t (&kid)[K], int& count,
                                               E* stack, int& sp, Counts& cnt) {
    if (ref + 1 >= m) return -2;  // not an internal node of this tree
    // hits of this pass lie at or beyond max(last key, 0): boxes ending before it are skipped
    const float low = has_last ? fmaxf(last_key, 0.0f) : 0.0f;
    const float4* w = sc.wide + 8 * (size_t)ref;
    // low planes at w[0..2], high planes at w[3..5]: the ray's near plane of each axis is picked
    // by address (br.s* = 0 or 3), so no per-box min/max orders the slab distances
    const float4 nx = __ldg(w + br.sx), ny = __ldg(w + 1 + br.sy), nz = __ldg(w + 2 + br.sz);
    const float4 fx = __ldg(w + 3 - br.sx), fy = __ldg(w + 4 - br.sy), fz = __ldg(w + 5 - br.sz);
    const float4 rf = __ldg(w + 6);
    if (COUNT) { cnt.nodes++; cnt.boxes += 4; }
    float tn[4], tf[4];
    box_tests4<K>(br, nx, ny, nz, fx, fy, fz, low, tn, tf);
    uint32_t r[4] = {__float_as_uint(rf.x), __float_as_uint(rf.y), __float_as_uint(rf.z),
                     __float_as_uint(rf.w)};
    float key[4];
#pragma unroll
    for (int e = 0; e < 4; e++) {
        // an unused slot holds an empty box and never passes; the cut-off is the current K-th
        // nearest hit of this pass (keys of this pass are >= low, so the cut-off is too)
        bool h = tn[e] <= fminf(tf[e], kk[K - 1]);
        if (h && (r[e] & kLeafBit)) {
            leaf_hits<K, COUNT>(sc, ray, r[e], n, leaf, has_last, last_key, last_id, kk, ki, kid,
                                count, cnt);
            h = false;
        }
        key[e] = h ? tn[e] : kInf;
    }
    cswap(key[0], r[0], key[1], r[1]);
    cswap(key[2], r[2], key[3], r[3]);
    cswap(key[0], r[0], key[2], r[2]);
    cswap(key[1], r[1], key[3], r[3]);
    cswap(key[1], r[1], key[2], r[2]);
    if (!(key[0] < kInf)) return kLeafBit;
    if (sp > wrs::kStack - 3) return -1;  // room for the (at most three) pushes: one compare
    if (key[3] < kInf) stack[sp++] = make_entry<E>(r[3], key[3]);
    if (key[2] < kInf) stack[sp++] = make_entry<E>(r[2], key[2]);
    if (key[1] < kInf) stack[sp++] = make_entry<E>(r[1], key[1]);
    return r[0];
}

// One traversal pass of one lane over the binary nodes: the K smallest hits (key, id) strictly
// after (last_key, last_id).  Returns the number gathered (<= K); -1 if the stack overflowed; -2
// if the pass met a reference outside the tree or visited more nodes than the tree has
// (impossible for a well-formed tree; it bounds the loop regardless).  (The 4-wide nodes are
// traversed by the whole warp: gather_warp, gather_packet.)
template <int K, bool COUNT>
__device__ __forceinline__ int gather(const Scene& sc, const Ray& ray, const wrs::BoxRay& br,
                                      uint32_t n, uint32_t leaf, int32_t root, bool has_last,
                                      float last_key, uint32_t last_id, float (&kk)[K],
                                      uint32_t (&ki)[K], uint32_t (&kid)[K], Counts& cnt) {
#pragma unroll
    for (int s = 0; s < K; s++) { kk[s] = kInf; ki[s] = 0xFFFFFFFFu; kid[s] = 0xFFFFFFFFu; }
    int count = 0;
    const uint32_t m = (n + leaf - 1) / leaf;  // leaves; internal nodes = m - 1
    if ((uint32_t)root & kLeafBit) {           // a single leaf: no internal node
        leaf_hits<K, COUNT>(sc, ray, (uint32_t)root, n, leaf, has_last, last_key, last_id, kk, ki,
                            kid, count, cnt);
        return count;
    }
    StackEntry stack[wrs::kStack];
    int sp = 0;
    uint32_t ref = (uint32_t)root;
    uint32_t budget = m + 1;  // internal node visits allowed in one pass
    while (true) {
        if (budget-- == 0) return -2;
        const int64_t next = visit_node<K, COUNT, StackEntry>(sc, ray, br, ref, n, leaf, m,
                                                              has_last, last_key, last_id, kk, ki,
                                                              kid, count, stack, sp, cnt);
        if (next < 0) return (int)next;
        if (next != kLeafBit) { ref = (uint32_t)next; continue; }
        if (!pop_within(stack, sp, kk[K - 1], ref)) break;
    }
    return count;
}

// Per-hit compositing quantities (spec S6).
struct HitTerms {
    float4 c;   // premultiplied rgba
    float op;   // opacity
    float w;    // soft-edge weight
    float rho;  // |f| / r
    float x;    // op * a * w (before the clamp)
    float a;    // clamped alpha
};

__device__ __forceinline__ HitTerms hit_terms(const Scene& sc, const Comp& cp, const Ray& ray,
                                              uint32_t k) {
    HitTerms h;
    h.c = __ldg(sc.rgba + k);
    h.op = sc.opacity ? __ldg(sc.opacity + __ldg(sc.src + k)) : 1.0f;
    h.w = 1.0f;
    h.rho = 0.0f;
    if (cp.beta > 0.0f) {
        const float4 s = __ldg(sc.pos_r + k);
        float key, ff;
        wrs::sphere_hit(ray, s, key, ff);
        h.rho = s.w > 0.0f ? sqrtf(ff) / s.w : 1.0f;
        h.w = wrs::soft_w(h.rho, cp.beta);
    }
    h.x = h.op * h.c.w * h.w;
    h.a = fminf(fmaxf(h.x, 0.0f), 1.0f);
    return h;
}

struct RayCtx {
    Ray ray;
    wrs::BoxRay br;
    uint32_t n, leaf;
    int32_t root;
};

__device__ __forceinline__ RayCtx make_ray_ctx(const Scene& sc, const wrs_camera& cam, int x, int y) {
    RayCtx r;
    r.ray = wrs::primary_ray(cam, x, y);
    const LbvhHeader h = *sc.hdr;
    r.n = h.n;
    r.leaf = h.leaf;
    r.root = h.root;
    r.br = wrs::make_box_ray(r.ray, wrs::traversal_eps(r.ray, h.maxabs));
    return r;
}

// Composite the first `count` gathered hits front to back (spec S6).  Returns true when the ray
// is finished (H hits used, transmittance at or below t_stop, or fewer than K hits were left).
template <int K, bool COUNT>
__device__ __forceinline__ bool composite_chunk(const Scene& sc, const Comp& cp, const Ray& ray,
                                                const uint32_t (&ki)[K], int count, float& T,
                                                float3& C, int& used, Counts& cnt) {
#pragma unroll
    for (int s = 0; s < K; s++) {
        if (s >= count) break;
        if ((cp.max_hits > 0 && used == cp.max_hits) || T <= cp.t_stop) return true;
        const HitTerms h = hit_terms(sc, cp, ray, ki[s]);
        const float tw = T * (h.op * h.w);
        C.x = fmaf(tw, h.c.x, C.x);
        C.y = fmaf(tw, h.c.y, C.y);
        C.z = fmaf(tw, h.c.z, C.z);
        T = T * (1.0f - h.a);
        used++;
        if (COUNT) cnt.composited++;
    }
    if (count < K) return true;
    return (cp.max_hits > 0 && used == cp.max_hits) || T <= cp.t_stop;
}

// Record the hits composited from one gathered chunk (used0 .. used) at their places in the ray's
// list; the ones beyond the list's capacity are dropped (the count marks the list as over).
template <int K>
__device__ __forceinline__ void record_chunk(const uint32_t (&ki)[K], int used0, int used,
                                             uint32_t* rec_hits, uint32_t cap) {
#pragma unroll
    for (int s = 0; s < K; s++) {
        const int i = used0 + s;
        if (i < used && (uint32_t)i < cap) rec_hits[i] = ki[s];
    }
}

// Forward trace of one ray over the binary nodes (spec S6).  overflow_bits: status bits of a
// traversal failure.  With REC, the composited hits go to rec_hits[0 .. cap) and their number
// (cap + 1 beyond cap) to *rec_count.
template <int K, bool COUNT, bool REC = false>
__device__ __forceinline__ float4 trace_ray(const Scene& sc, const Comp& cp, const RayCtx& rc,
                                            uint32_t& overflow_bits, Counts& cnt,
                                            uint32_t* rec_hits = nullptr,
                                            uint32_t* rec_count = nullptr, uint32_t cap = 0) {
    float T = 1.0f;
    float3 C = make_float3(0.f, 0.f, 0.f);
    overflow_bits = 0;
    if (rc.n == 0) {
        if constexpr (REC) *rec_count = 0;
        return make_float4(0.f, 0.f, 0.f, 0.f);
    }
    int used = 0;
    bool has_last = false;
    float last_key = 0.0f;
    uint32_t last_id = 0;
    float kk[K];
    uint32_t ki[K], kid[K];
    while (true) {
        const int count = gather<K, COUNT>(sc, rc.ray, rc.br, rc.n, rc.leaf, rc.root, has_last,
                                           last_key, last_id, kk, ki, kid, cnt);
        if (COUNT) cnt.passes++;
        if (count < 0) { overflow_bits = count == -1 ? WRS_STATUS_STACK_OVERFLOW : WRS_STATUS_MALFORMED_TREE; break; }
        if constexpr (REC) {
            const int u0 = used;
            const bool fin = composite_chunk<K, COUNT>(sc, cp, rc.ray, ki, count, T, C, used, cnt);
            record_chunk<K>(ki, u0, used, rec_hits, cap);
            if (fin) break;
        } else {
            if (composite_chunk<K, COUNT>(sc, cp, rc.ray, ki, count, T, C, used, cnt)) break;
        }
        has_last = true;
        last_key = kk[K - 1];
        last_id = kid[K - 1];
    }
    if constexpr (REC) *rec_count = (uint32_t)used > cap ? cap + 1 : (uint32_t)used;
    return make_float4(C.x, C.y, C.z, 1.0f - T);
}

// ---- per-ray 4-wide traversal with warp-wide leaf steps -------------------------------------
// The per-pixel kernels' 4-wide traversal.  Each lane traverses its own ray, but leaf entries are
// not tested inside the node visit that finds them: they are sorted with the internal entries by
// entry distance, the nearest is the lane's next step and the others are pushed (so a leaf that
// starts beyond the current K-th key is dropped when popped, like a node).  Every iteration of
// the warp runs either a node step, for the lanes whose next entry is an internal node, or a leaf
// step, for the lanes whose next entry is a leaf: the leaf step when at least as many lanes want
// one as want a node step (a ballot), or when no lane wants a node step.  Lanes meet their leaves
// at different visits; tested in the visit that found them, a warp ran about 16 leaf tests of ~3
// active lanes per 32 rays, a divergent block per node slot.  The hit set of each pass, and so
// the image, is that of any other traversal order (the K-buffer keeps the K smallest (key, id)).
// All 32 lanes of the warp call these functions together; a lane without a ray passes
// active = false.
constexpr int64_t kPopNext = (int64_t)1 << 32;  // visit result: no entry hit, pop the next one

template <int K, bool COUNT>
__device__ __forceinline__ int64_t visit_node4_sorted(const Scene& sc, const wrs::BoxRay& br,
                                                      uint32_t ref, uint32_t m, bool has_last,
                                                      float last_key, const float (&kk)[K],
                                                      StackEntry* stack, int& sp, Counts& cnt) {
    if (ref + 1 >= m) return -2;  // not an internal node of this tree
    const float low = has_last ? fmaxf(last_key, 0.0f) : 0.0f;
    const float4* w = sc.wide + 8 * (size_t)ref;
    const float4 nx = __ldg(w + br.sx), ny = __ldg(w + 1 + br.sy), nz = __ldg(w + 2 + br.sz);
    const float4 fx = __ldg(w + 3 - br.sx), fy = __ldg(w + 4 - br.sy), fz = __ldg(w + 5 - br.sz);
    const float4 rf = __ldg(w + 6);
    if (COUNT) { cnt.nodes++; cnt.boxes += 4; }
    float tn[4], tf[4];
    box_tests4<K>(br, nx, ny, nz, fx, fy, fz, low, tn, tf);
    uint32_t r[4] = {__float_as_uint(rf.x), __float_as_uint(rf.y), __float_as_uint(rf.z),
                     __float_as_uint(rf.w)};
    float key[4];
#pragma unroll
    for (int e = 0; e < 4; e++) key[e] = tn[e] <= fminf(tf[e], kk[K - 1]) ? tn[e] : kInf;
    cswap(key[0], r[0], key[1], r[1]);
    cswap(key[2], r[2], key[3], r[3]);
    cswap(key[0], r[0], key[2], r[2]);
    cswap(key[1], r[1], key[3], r[3]);
    cswap(key[1], r[1], key[2], r[2]);
    if (!(key[0] < kInf)) return kPopNext;
    if (sp > wrs::kStack - 3) return -1;  // room for the (at most three) pushes
    if (key[3] < kInf) stack[sp++] = stack_entry(r[3], key[3]);
    if (key[2] < kInf) stack[sp++] = stack_entry(r[2], key[2]);
    if (key[1] < kInf) stack[sp++] = stack_entry(r[1], key[1]);
    return r[0];
}

// One pass of every lane with part = true (gather's contract); the others take part in the
// warp's steps without a ray.
template <int K, bool COUNT>
__device__ __forceinline__ int gather_warp(const Scene& sc, const Ray& ray, const wrs::BoxRay& br,
                                           uint32_t n, uint32_t leaf, int32_t root, bool part,
                                           bool has_last, float last_key, uint32_t last_id,
                                           float (&kk)[K], uint32_t (&ki)[K], uint32_t (&kid)[K],
                                           Counts& cnt) {
#pragma unroll
    for (int s = 0; s < K; s++) { kk[s] = kInf; ki[s] = 0xFFFFFFFFu; kid[s] = 0xFFFFFFFFu; }
    int count = 0;
    const uint32_t m = (n + leaf - 1) / leaf;
    StackEntry stack[wrs::kStack];
    int sp = 0;
    uint32_t cur = (uint32_t)root;  // the lane's next entry (a single-leaf tree starts at a leaf)
    bool live = part;
    int err = 0;
    uint32_t budget = m + 1;  // internal node visits allowed in one pass
    // Every iteration advances at least one lane by a node visit (bounded by the budget) or a
    // pop (bounded by the pushes), so the loop ends; its exit and branches are warp-uniform.
    while (true) {
        const bool at_leaf = live && (cur & kLeafBit);
        const bool at_node = live && !(cur & kLeafBit);
        const unsigned lm = __ballot_sync(0xffffffffu, at_leaf);
        const unsigned nm = __ballot_sync(0xffffffffu, at_node);
        if ((lm | nm) == 0) break;
        if (lm != 0 && (nm == 0 || __popc(lm) >= __popc(nm))) {
            if (at_leaf) {
                leaf_hits<K, COUNT>(sc, ray, cur, n, leaf, has_last, last_key, last_id, kk, ki,
                                    kid, count, cnt);
                live = pop_within(stack, sp, kk[K - 1], cur);
            }
        } else if (at_node) {
            if (budget-- == 0) {
                err = -2;
                live = false;
            } else {
                const int64_t next = visit_node4_sorted<K, COUNT>(sc, br, cur, m, has_last,
                                                                  last_key, kk, stack, sp, cnt);
                if (next < 0) {
                    err = (int)next;
                    live = false;
                } else if (next == kPopNext) {
                    live = pop_within(stack, sp, kk[K - 1], cur);
                } else {
                    cur = (uint32_t)next;
                }
            }
        }
    }
    return err ? err : count;
}

// trace_ray for the whole warp with 4-wide nodes; lanes with active = false take part without a
// ray (and return zero).  Passes continue while any lane of the warp still needs hits.
template <int K, bool COUNT, bool REC = false>
__device__ __forceinline__ float4 trace_ray_warp4(const Scene& sc, const Comp& cp,
                                                  const RayCtx& rc, bool active,
                                                  uint32_t& overflow_bits, Counts& cnt,
                                                  uint32_t* rec_hits = nullptr,
                                                  uint32_t* rec_count = nullptr,
                                                  uint32_t cap = 0) {
    float T = 1.0f;
    float3 C = make_float3(0.f, 0.f, 0.f);
    overflow_bits = 0;
    bool done = !active || rc.n == 0;
    int used = 0;
    bool has_last = false;
    float last_key = 0.0f;
    uint32_t last_id = 0;
    float kk[K];
    uint32_t ki[K], kid[K];
    while (__any_sync(0xffffffffu, !done)) {
        const int count = gather_warp<K, COUNT>(sc, rc.ray, rc.br, rc.n, rc.leaf, rc.root, !done,
                                                has_last, last_key, last_id, kk, ki, kid, cnt);
        if (done) continue;
        if (COUNT) cnt.passes++;
        if (count < 0) {
            overflow_bits = count == -1 ? WRS_STATUS_STACK_OVERFLOW : WRS_STATUS_MALFORMED_TREE;
            done = true;
            continue;
        }
        const int u0 = used;
        done = composite_chunk<K, COUNT>(sc, cp, rc.ray, ki, count, T, C, used, cnt);
        if constexpr (REC) record_chunk<K>(ki, u0, used, rec_hits, cap);
        has_last = true;
        last_key = kk[K - 1];
        last_id = kid[K - 1];
    }
    if constexpr (REC) {
        if (active) *rec_count = (uint32_t)used > cap ? cap + 1 : (uint32_t)used;
    }
    return make_float4(C.x, C.y, C.z, 1.0f - T);
}

// The per-pixel trace of a warp's rays: the warp-wide 4-wide traversal, or per lane with binary
// nodes.  All 32 lanes call it.
template <int K, bool COUNT, bool W4, bool REC = false>
__device__ __forceinline__ float4 trace_ray_warp(const Scene& sc, const Comp& cp, const RayCtx& rc,
                                                 bool active, uint32_t& overflow_bits, Counts& cnt,
                                                 uint32_t* rec_hits = nullptr,
                                                 uint32_t* rec_count = nullptr, uint32_t cap = 0) {
    if constexpr (W4) {
        return trace_ray_warp4<K, COUNT, REC>(sc, cp, rc, active, overflow_bits, cnt, rec_hits,
                                              rec_count, cap);
    } else {
        overflow_bits = 0;
        if (!active) return make_float4(0.f, 0.f, 0.f, 0.f);
        return trace_ray<K, COUNT, REC>(sc, cp, rc, overflow_bits, cnt, rec_hits,
                                               rec_count, cap);
    }
}

// ---- packet schedule: one traversal per warp ------------------------------------------------
// The 32 rays of an 8x4 pixel tile share one traversal of the 4-wide nodes: every lane tests the
// node's four boxes against its own ray (its own pass bound and k-buffer cut-off), a child is
// entered if any lane enters it, and the children are ordered by the smallest entry distance over
// the lanes.  Control flow and the stack are warp-uniform (every lane holds the same stack), so
// the box tests run with all lanes active; a leaf is tested only by the lanes whose ray enters
// it.  Each lane keeps its own k-buffer, so the hits a lane gathers -- and the image -- are those
// of the per-ray traversal; only the set of visited nodes differs (the union over the warp).
// All 32 lanes of a warp must call these functions together (lanes without a ray pass
// part = false).
template <int K>
__device__ __forceinline__ int64_t visit_node4_packet(const Scene& sc, const Ray& ray,
                                                      const wrs::BoxRay& br, uint32_t ref,
                                                      uint32_t n, uint32_t leaf, uint32_t m,
                                                      bool part, bool has_last, float last_key,
                                                      uint32_t last_id, float (&kk)[K],
                                                      uint32_t (&ki)[K], uint32_t (&kid)[K],
                                                      int& count, StackEntry* stack, int& sp) {
    if (ref + 1 >= m) return -2;  // not an internal node of this tree (ref is warp-uniform)
    const float low = has_last ? fmaxf(last_key, 0.0f) : 0.0f;
    const float4* w = sc.wide + 8 * (size_t)ref;
    const float4 nx = __ldg(w + br.sx), ny = __ldg(w + 1 + br.sy), nz = __ldg(w + 2 + br.sz);
    const float4 fx = __ldg(w + 3 - br.sx), fy = __ldg(w + 4 - br.sy), fz = __ldg(w + 5 - br.sz);
    const float4 rf = __ldg(w + 6);
    float tn[4], tf[4];
    box_tests4<K>(br, nx, ny, nz, fx, fy, fz, low, tn, tf);
    uint32_t r[4] = {__float_as_uint(rf.x), __float_as_uint(rf.y), __float_as_uint(rf.z),
                     __float_as_uint(rf.w)};
    float key[4];
    Counts none;
#pragma unroll
    for (int e = 0; e < 4; e++) {
        bool h = part && tn[e] <= fminf(tf[e], kk[K - 1]);
        if (h && (r[e] & kLeafBit)) {
            leaf_hits<K, false>(sc, ray, r[e], n, leaf, has_last, last_key, last_id, kk, ki, kid,
                                count, none);
            h = false;
        }
        // the warp's key of the entry: its smallest entry distance over the lanes that enter it
        // (distances are >= 0, so their bit patterns order like the values; +inf = nobody)
        key[e] = __uint_as_float(__reduce_min_sync(0xffffffffu, __float_as_uint(h ? tn[e] : kInf)));
    }
    cswap(key[0], r[0], key[1], r[1]);
    cswap(key[2], r[2], key[3], r[3]);
    cswap(key[0], r[0], key[2], r[2]);
    cswap(key[1], r[1], key[3], r[3]);
    cswap(key[1], r[1], key[2], r[2]);
    if (!(key[0] < kInf)) return kLeafBit;
    if (sp > wrs::kStack - 3) return -1;  // room for the (at most three) pushes: one compare
    if (key[3] < kInf) stack[sp++] = stack_entry(r[3], key[3]);
    if (key[2] < kInf) stack[sp++] = stack_entry(r[2], key[2]);
    if (key[1] < kInf) stack[sp++] = stack_entry(r[1], key[1]);
    return r[0];
}

template <int K>
__device__ __forceinline__ int gather_packet(const Scene& sc, const Ray& ray,
                                             const wrs::BoxRay& br, uint32_t n, uint32_t leaf,
                                             int32_t root, bool part, bool has_last,
                                             float last_key, uint32_t last_id, float (&kk)[K],
                                             uint32_t (&ki)[K], uint32_t (&kid)[K]) {
#pragma unroll
    for (int s = 0; s < K; s++) { kk[s] = kInf; ki[s] = 0xFFFFFFFFu; kid[s] = 0xFFFFFFFFu; }
    int count = 0;
    Counts none;
    const uint32_t m = (n + leaf - 1) / leaf;
    if ((uint32_t)root & kLeafBit) {
        if (part)
            leaf_hits<K, false>(sc, ray, (uint32_t)root, n, leaf, has_last, last_key, last_id, kk,
                                ki, kid, count, none);
        return count;
    }
    StackEntry stack[wrs::kStack];
    int sp = 0;
    uint32_t ref = (uint32_t)root;
    uint32_t budget = m + 1;
    while (true) {
        if (budget-- == 0) return -2;
        const int64_t next = visit_node4_packet<K>(sc, ray, br, ref, n, leaf, m, part, has_last,
                                                   last_key, last_id, kk, ki, kid, count, stack, sp);
        if (next < 0) return (int)next;
        if (next != kLeafBit) { ref = (uint32_t)next; continue; }
        // the warp's cut-off: the largest K-th key over its rays (a stacked entry's key is the
        // smallest entry distance over the lanes that enter it, so an entry beyond every lane's
        // cut-off holds nothing any lane still needs); warp-uniform like the stack
        const float cut = __uint_as_float(
            __reduce_max_sync(0xffffffffu, __float_as_uint(part ? kk[K - 1] : 0.0f)));
        if (!pop_within(stack, sp, cut, ref)) break;
    }
    return count;
}

// Forward trace of the warp's rays; lanes with active = false take part without a ray.
template <int K, bool REC = false>
__device__ __forceinline__ float4 trace_ray_packet(const Scene& sc, const Comp& cp,
                                                   const RayCtx& rc, bool active,
                                                   uint32_t& overflow_bits,
                                                   uint32_t* rec_hits = nullptr,
                                                   uint32_t* rec_count = nullptr,
                                                   uint32_t cap = 0) {
    float T = 1.0f;
    float3 C = make_float3(0.f, 0.f, 0.f);
    overflow_bits = 0;
    bool done = !active || rc.n == 0;
    int used = 0;
    bool has_last = false;
    float last_key = 0.0f;
    uint32_t last_id = 0;
    float kk[K];
    uint32_t ki[K], kid[K];
    Counts none;
    // passes continue while any lane of the warp still needs hits; each pass is one traversal
    for (uint32_t pass = 0; __any_sync(0xffffffffu, !done); pass++) {
        const int count = gather_packet<K>(sc, rc.ray, rc.br, rc.n, rc.leaf, rc.root, !done,
                                           has_last, last_key, last_id, kk, ki, kid);
        if (count < 0) {  // warp-uniform: the traversal failed for every lane
            if (!done)
                overflow_bits = count == -1 ? WRS_STATUS_STACK_OVERFLOW : WRS_STATUS_MALFORMED_TREE;
            break;
        }
        if (!done) {
            if constexpr (REC) {
                const int u0 = used;
                done = composite_chunk<K, false>(sc, cp, rc.ray, ki, count, T, C, used, none);
                record_chunk<K>(ki, u0, used, rec_hits, cap);
            } else {
                done = composite_chunk<K, false>(sc, cp, rc.ray, ki, count, T, C, used, none);
            }
            has_last = true;
            last_key = kk[K - 1];
            last_id = kid[K - 1];
        }
    }
    if constexpr (REC) {
        if (active) *rec_count = (uint32_t)used > cap ? cap + 1 : (uint32_t)used;
    }
    return make_float4(C.x, C.y, C.z, 1.0f - T);
}

// ---- persistent schedule with lane refill ----------------------------------------------------
// The same per-ray work as trace_ray, run as a per-lane state machine: every loop iteration a
// lane advances its traversal by one node or one leaf; when a ray finishes its lane goes idle,
// and as soon as kRefill lanes of a warp are idle the warp takes that many new rays (ballot +
// one shared-memory atomic).  Each block owns the 8x4 ray tiles blockIdx.x, blockIdx.x + grid, ...
// so that every block gets a mix of cheap and expensive parts of the image.
constexpr int kRefill = 8;

// Minimum resident 128-thread blocks per SM asked of the compiler for the single-view persistent
// kernel with K <= 2 (it caps registers at 65536 / (128 * this)): 10 (48 registers) for the binary
// traversal, 8 (64 registers) for the 4-wide one (1 % faster than 9, 7 % faster than 10), both
// measured on the 1080p, 2 M splat workload; larger K keep more state and get no cap.  Build-time
// tuning knobs (0 = no cap).
#ifndef WRS_PERSISTENT_MIN_BLOCKS
#define WRS_PERSISTENT_MIN_BLOCKS 10
#endif
#ifndef WRS_PERSISTENT_W4_MIN_BLOCKS
#define WRS_PERSISTENT_W4_MIN_BLOCKS 8
#endif
template <int K, bool W4>
struct PersistentMinBlocks {
    static constexpr int value = K > 2 ? 0 : (W4 ? WRS_PERSISTENT_W4_MIN_BLOCKS : WRS_PERSISTENT_MIN_BLOCKS);
};

// Launch bounds of the per-pixel kernel.  With the 4-wide traversal and K <= 2 it runs in blocks
// of at most 128 threads; with K = 1, 9 resident blocks per SM (56 registers, no spills): on the
// 1080p, 2 M splat workload 14 % faster than 10 blocks (48 registers, 112 B spilled), 2 % faster
// than 8 (64 registers) and 8-16 % faster than 7, 6 or no cap (70 registers).  Other instances
// keep blocks of up to 256 threads and no register cap.  A build-time knob:
// WRS_PIXEL_W4_MIN_BLOCKS (resident 128-thread blocks, 0 = no cap).
#ifndef WRS_PIXEL_W4_MIN_BLOCKS
#define WRS_PIXEL_W4_MIN_BLOCKS 9
#endif
#ifndef WRS_PIXEL_W4_K2_MIN_BLOCKS
#define WRS_PIXEL_W4_K2_MIN_BLOCKS 9  // K = 2: 9 blocks (56 registers), 4 % faster than 10
#endif
#ifndef WRS_PIXEL_W4_K4_MIN_BLOCKS
#define WRS_PIXEL_W4_K4_MIN_BLOCKS 8  // K = 4: 8 blocks (64 registers), 5 % faster than no cap (75)
#endif
#ifndef WRS_PIXEL_W4_K8_MIN_BLOCKS
#define WRS_PIXEL_W4_K8_MIN_BLOCKS 7  // K = 8: 7 blocks (72 registers), 9 % faster than no cap (80)
#endif
// Resident 128-thread blocks of the per-pixel kernel for (K, node width) (0 = no cap), and
// whether it is built for blocks of at most 128 threads (the host clamps the block to it).
constexpr int pixel_min_blocks(int K, bool w4) {
    return !w4 ? 0 : K == 1 ? WRS_PIXEL_W4_MIN_BLOCKS : K == 2 ? WRS_PIXEL_W4_K2_MIN_BLOCKS
                   : K == 4 ? WRS_PIXEL_W4_K4_MIN_BLOCKS : K == 8 ? WRS_PIXEL_W4_K8_MIN_BLOCKS : 0;
}
constexpr bool pixel_block_128(int K, bool w4) { return (w4 && K <= 2) || pixel_min_blocks(K, w4) > 0; }
template <int K, bool W4>
struct PixelBounds {
    static constexpr int max_threads = pixel_block_128(K, W4) ? 128 : 256;
    static constexpr int min_blocks = pixel_min_blocks(K, W4);
};

// Resident 128-thread blocks per SM of the multi-session per-tile kernel and of the per-pixel
// backward kernels.  The multi-session kernel with K <= 2 runs 8 (64 registers): on the 64
// sessions 21 % faster than no cap (94 registers) and 10 % faster than 10 blocks.  The backward
// with K = 4 runs 8 (64 registers; with warp-wide leaf steps 12 % faster than no cap at 84
// registers and equal to 6 blocks); with K = 2 the same cap spills and is slower, so the other
// instances keep no cap.  Build-time knobs (0 = no cap).
#ifndef WRS_BATCHED_MIN_BLOCKS
#define WRS_BATCHED_MIN_BLOCKS 8
#endif
#ifndef WRS_BWD_K4_MIN_BLOCKS
#define WRS_BWD_K4_MIN_BLOCKS 8
#endif
// The packet kernels keep no cap: 5 or 6 resident 256-thread blocks (48 or 40 registers) spill
// 180-230 bytes at K 4 and run 4-29 % slower.
#ifndef WRS_PACKET_MIN_BLOCKS
#define WRS_PACKET_MIN_BLOCKS 0
#endif
template <int K, bool W4>
struct BatchedBounds {
    static constexpr int min_blocks = K <= 2 ? WRS_BATCHED_MIN_BLOCKS : 0;
};
template <int K, bool W4>
struct BwdBounds {
    static constexpr int min_blocks = K == 4 ? WRS_BWD_K4_MIN_BLOCKS : 0;
};

template <int K>
struct Lane {
    Ray ray;
    wrs::BoxRay br;
    uint32_t pix;
    float T;
    float3 C;
    int used;
    bool has_last;
    float last_key;
    uint32_t last_id;
    float kk[K];
    uint32_t ki[K], kid[K];
    int count;
    uint32_t ref;
    int sp;
    uint32_t budget;
};

template <int K>
__device__ __forceinline__ void begin_pass(Lane<K>& L, int32_t root, uint32_t m) {
#pragma unroll
    for (int s = 0; s < K; s++) { L.kk[s] = kInf; L.ki[s] = 0xFFFFFFFFu; L.kid[s] = 0xFFFFFFFFu; }
    L.count = 0;
    L.ref = (uint32_t)root;
    L.sp = 0;
    L.budget = m + 1;
}

// One traversal step: one internal-node visit (its leaf children tested inline), as in gather's
// loop.  0: continue; 1: pass finished; -1: stack overflow; -2: malformed tree.
template <int K, bool W4>
__device__ __forceinline__ int lane_step(const Scene& sc, Lane<K>& L, int* stack, uint32_t n,
                                         uint32_t leaf, uint32_t m) {
    Counts cnt;
    if (L.ref & kLeafBit) {  // a single leaf: no internal node
        leaf_hits<K, false>(sc, L.ray, L.ref, n, leaf, L.has_last, L.last_key, L.last_id, L.kk,
                            L.ki, L.kid, L.count, cnt);
        return 1;
    }
    if (L.budget-- == 0) return -2;
    const int64_t next =
        W4 ? visit_node4<K, false, int>(sc, L.ray, L.br, L.ref, n, leaf, m, L.has_last,
                                        L.last_key, L.last_id, L.kk, L.ki, L.kid, L.count, stack,
                                        L.sp, cnt)
           : visit_node<K, false, int>(sc, L.ray, L.br, L.ref, n, leaf, m, L.has_last, L.last_key,
                                       L.last_id, L.kk, L.ki, L.kid, L.count, stack, L.sp, cnt);
    if (next < 0) return (int)next;
    if (next != kLeafBit) { L.ref = (uint32_t)next; return 0; }
    return pop_within(stack, L.sp, L.kk[K - 1], L.ref) ? 0 : 1;
}

template <int K, bool W4>
__global__ void __launch_bounds__(128, PersistentMinBlocks<K, W4>::value) k_trace_pr(Scene sc, Comp cp, wrs_camera cam,
                                                  float4* __restrict__ out, int32_t* status) {
    __shared__ uint32_t s_next;
    if (threadIdx.x == 0) s_next = 0;
    __syncthreads();
    const uint32_t W = (uint32_t)cam.width, H = (uint32_t)cam.height;
    const uint32_t tiles_x = (W + 7) / 8, n_tiles = tiles_x * ((H + 3) / 4);
    const uint32_t G = gridDim.x;
    const uint32_t my_rays = blockIdx.x < n_tiles ? ((n_tiles - 1 - blockIdx.x) / G + 1) * 32 : 0;
    const LbvhHeader hd = *sc.hdr;
    const uint32_t n = hd.n, leaf = hd.leaf;
    const uint32_t m = n == 0 ? 0 : (n + leaf - 1) / leaf;
    const int lane = threadIdx.x & 31;
    Lane<K> L;
    int stack[wrs::kStack];
    Counts cnt;
    bool active = false;
    bool more = my_rays > 0;
    while (true) {
        const uint32_t idle = __ballot_sync(0xffffffffu, !active);
        if (more && __popc(idle) >= kRefill) {
            const uint32_t c = __popc(idle);
            uint32_t base = 0;
            if (lane == 0) base = atomicAdd(&s_next, c);
            base = __shfl_sync(0xffffffffu, base, 0);
            if (base + c >= my_rays) more = false;
            if (!active) {
                const uint32_t r = base + __popc(idle & ((1u << lane) - 1u));
                if (r < my_rays) {
                    const uint32_t tile = blockIdx.x + (r >> 5) * G, pos = r & 31;
                    const uint32_t x = (tile % tiles_x) * 8 + (pos & 7);
                    const uint32_t y = (tile / tiles_x) * 4 + (pos >> 3);
                    if (x < W && y < H) {
                        L.pix = y * W + x;
                        if (n == 0) {
                            out[L.pix] = make_float4(0.f, 0.f, 0.f, 0.f);
                        } else {
                            L.ray = wrs::primary_ray(cam, (int)x, (int)y);
                            L.br = wrs::make_box_ray(L.ray, wrs::traversal_eps(L.ray, hd.maxabs));
                            L.T = 1.0f;
                            L.C = make_float3(0.f, 0.f, 0.f);
                            L.used = 0;
                            L.has_last = false;
                            L.last_key = 0.0f;
                            L.last_id = 0;
                            begin_pass(L, hd.root, m);
                            active = true;
                        }
                    }
                }
            }
        }
        if (!__any_sync(0xffffffffu, active)) {
            if (!more) break;
            continue;
        }
        if (active) {
            const int rc = lane_step<K, W4>(sc, L, stack, n, leaf, m);
            if (rc != 0) {
                bool done = true;
                if (rc < 0) {
                    wrs::set_status(status, rc == -1 ? WRS_STATUS_STACK_OVERFLOW : WRS_STATUS_MALFORMED_TREE);
                } else if (!composite_chunk<K, false>(sc, cp, L.ray, L.ki, L.count, L.T, L.C, L.used, cnt)) {
                    done = false;
                    L.has_last = true;
                    L.last_key = L.kk[K - 1];
                    L.last_id = L.kid[K - 1];
                    begin_pass(L, hd.root, m);
                }
                if (done) {
                    out[L.pix] = make_float4(L.C.x, L.C.y, L.C.z, 1.0f - L.T);
                    active = false;
                }
            }
        }
    }
}

// Pixel of thread t in a (16 x 4*warps/2) tile: warps are 8x4 pixel blocks, two across.
__device__ __forceinline__ void tile_pixel(int t, int& px, int& py) {
    const int warp = t >> 5, lane = t & 31;
    px = (warp & 1) * 8 + (lane & 7);
    py = (warp >> 1) * 4 + (lane >> 3);
}

// The pixel of this thread in the per-pixel grid (blockIdx.x, blockIdx.y) traced and written;
// with REC its composited hits are recorded at ray index ray_base + pixel.  Every lane of the
// block stays to the end (the 4-wide traversal takes warp-wide steps); lanes outside the image
// take part without a ray.
template <int K, bool W4, bool REC = false>
__device__ __forceinline__ void trace_pixel(const Scene& sc, const Comp& cp, const wrs_camera& cam,
                                            float4* __restrict__ out, int32_t* status,
                                            const HitRecord* hr = nullptr, size_t ray_base = 0) {
    int px, py;
    tile_pixel(threadIdx.x, px, py);
    const int tile_h = (blockDim.x >> 6) * 4;
    const int x = blockIdx.x * 16 + px, y = blockIdx.y * tile_h + py;
    const bool active = x < cam.width && y < cam.height;
    const RayCtx rc = make_ray_ctx(sc, cam, active ? x : 0, active ? y : 0);
    uint32_t overflow;
    Counts cnt;
    float4 o;
    if constexpr (REC) {
        const size_t ray = ray_base + (active ? (size_t)y * cam.width + x : 0);
        o = trace_ray_warp<K, false, W4, true>(sc, cp, rc, active, overflow, cnt,
                                               hr->hits + ray * hr->cap, hr->count + ray, hr->cap);
    } else {
        o = trace_ray_warp<K, false, W4>(sc, cp, rc, active, overflow, cnt);
    }
    if (overflow) wrs::set_status(status, overflow);
    // (the output index is formed after the traversal: kept live across it, it costs registers)
    if (active) out[(size_t)y * cam.width + x] = o;
}

template <int K, bool W4>
__global__ void __launch_bounds__(PixelBounds<K, W4>::max_threads, PixelBounds<K, W4>::min_blocks)
k_trace(Scene sc, Comp cp, wrs_camera cam, float4* __restrict__ out, int32_t* status) {
    trace_pixel<K, W4>(sc, cp, cam, out, status);
}

// Several views of one scene in one launch: blockIdx.z is the view; view v's camera is
// vc.cam[v] (read in place from the kernel parameters) and its image starts at out + v * pixels.
constexpr int kMaxViews = 32;
struct ViewCams {
    wrs_camera cam[kMaxViews];
};

template <int K, bool W4>
__global__ void __launch_bounds__(PixelBounds<K, W4>::max_threads, PixelBounds<K, W4>::min_blocks)
k_trace_views(Scene sc, Comp cp, const __grid_constant__ ViewCams vc, float4* __restrict__ out,
              size_t pixels, int32_t* status) {
    trace_pixel<K, W4>(sc, cp, vc.cam[blockIdx.z], out + blockIdx.z * pixels, status);
}

// k_trace_views that records every ray's composited hits (ray = (view0 + view) * pixels + pixel).
template <int K, bool W4>
__global__ void __launch_bounds__(PixelBounds<K, W4>::max_threads, PixelBounds<K, W4>::min_blocks)
k_trace_views_rec(Scene sc, Comp cp, const __grid_constant__ ViewCams vc, float4* __restrict__ out,
                  size_t pixels, HitRecord hr, size_t ray0, int32_t* status) {
    trace_pixel<K, W4, true>(sc, cp, vc.cam[blockIdx.z], out + blockIdx.z * pixels, status, &hr,
                             ray0 + blockIdx.z * pixels);
}

// Packet schedule (4-wide nodes only): every lane of the block stays to the end, lanes outside
// the image take part in their warp's traversal without a ray.
template <int K, bool REC = false>
__device__ __forceinline__ void trace_pixel_packet(const Scene& sc, const Comp& cp,
                                                   const wrs_camera& cam, float4* __restrict__ out,
                                                   int32_t* status, const HitRecord* hr = nullptr,
                                                   size_t ray_base = 0) {
    int px, py;
    tile_pixel(threadIdx.x, px, py);
    const int tile_h = (blockDim.x >> 6) * 4;
    const int x = blockIdx.x * 16 + px, y = blockIdx.y * tile_h + py;
    const bool active = x < cam.width && y < cam.height;
    const RayCtx rc = make_ray_ctx(sc, cam, active ? x : 0, active ? y : 0);
    uint32_t overflow;
    if constexpr (REC) {
        const size_t pix = active ? (size_t)y * cam.width + x : 0, ray = ray_base + pix;
        const float4 o = trace_ray_packet<K, true>(sc, cp, rc, active, overflow,
                                                   hr->hits + ray * hr->cap, hr->count + ray,
                                                   hr->cap);
        if (overflow) wrs::set_status(status, overflow);
        if (active) out[pix] = o;
    } else {
        const float4 o = trace_ray_packet<K>(sc, cp, rc, active, overflow);
        if (overflow) wrs::set_status(status, overflow);
        if (active) out[(size_t)y * cam.width + x] = o;
    }
}

template <int K>
__global__ void __launch_bounds__(256, WRS_PACKET_MIN_BLOCKS) k_trace_packet(Scene sc, Comp cp, wrs_camera cam,
                                                      float4* __restrict__ out, int32_t* status) {
    trace_pixel_packet<K>(sc, cp, cam, out, status);
}

template <int K>
__global__ void __launch_bounds__(256, WRS_PACKET_MIN_BLOCKS) k_trace_packet_views(Scene sc, Comp cp,
                                                            const __grid_constant__ ViewCams vc,
                                                            float4* __restrict__ out,
                                                            size_t pixels, int32_t* status) {
    trace_pixel_packet<K>(sc, cp, vc.cam[blockIdx.z], out + blockIdx.z * pixels, status);
}

template <int K>
__global__ void __launch_bounds__(256, WRS_PACKET_MIN_BLOCKS) k_trace_packet_views_rec(
        Scene sc, Comp cp, const __grid_constant__ ViewCams vc, float4* __restrict__ out,
        size_t pixels, HitRecord hr, size_t ray0, int32_t* status) {
    trace_pixel_packet<K, true>(sc, cp, vc.cam[blockIdx.z], out + blockIdx.z * pixels, status, &hr,
                                ray0 + blockIdx.z * pixels);
}

template <int K, bool W4>
__global__ void __launch_bounds__(256) k_trace_count(Scene sc, Comp cp, wrs_camera cam,
                                                     unsigned long long* counters, int32_t* status) {
    int px, py;
    tile_pixel(threadIdx.x, px, py);
    const int tile_h = (blockDim.x >> 6) * 4;
    const int x = blockIdx.x * 16 + px, y = blockIdx.y * tile_h + py;
    Counts cnt = {0, 0, 0, 0, 0, 0};
    const bool active = x < cam.width && y < cam.height;
    const RayCtx rc = make_ray_ctx(sc, cam, active ? x : 0, active ? y : 0);
    uint32_t overflow;
    trace_ray_warp<K, true, W4>(sc, cp, rc, active, overflow, cnt);
    if (overflow) wrs::set_status(status, overflow);
    unsigned long long v[6] = {cnt.nodes, cnt.boxes, cnt.spheres, cnt.gathered, cnt.composited,
                               cnt.passes};
#pragma unroll
    for (int k = 0; k < 6; k++) {
        unsigned long long s = v[k];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if ((threadIdx.x & 31) == 0) atomicAdd(counters + k, s);
    }
}

// The session owning 8x4 tile `tile` of the concatenated tile space (session s owns tiles
// [tile_begin_s, tile_begin_s + tiles_s)): binary search over the sessions' first tiles.
__device__ __forceinline__ const wrs_session& session_of(const wrs_session* __restrict__ sess,
                                                         int n_sessions, uint32_t tile) {
    int lo = 0, hi = n_sessions - 1;  // last session with tile_begin <= tile
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (sess[mid].tile_begin <= tile) lo = mid; else hi = mid - 1;
    }
    return sess[lo];
}

template <bool W4>
__device__ __forceinline__ Scene session_scene(const wrs_session& S) {
    Scene sc;
    sc.hdr = static_cast<const LbvhHeader*>(S.nodes);
    sc.nodes = wrs::lbvh_nodes(S.nodes);
    sc.wide = W4 ? sc.nodes + 4 * (size_t)sc.hdr->wide_start : nullptr;
    sc.pos_r = reinterpret_cast<const float4*>(S.pos_r);
    sc.rgba = reinterpret_cast<const float4*>(S.rgba);
    sc.id = S.id;
    sc.src = S.src;
    sc.opacity = S.opacity;
    return sc;
}

// Pixel (x, y) of lane `pos` in 8x4 tile `tile`, and the session it belongs to.
__device__ __forceinline__ const wrs_session& tile_pixel_of(const wrs_session* __restrict__ sess,
                                                            int n_sessions, uint32_t tile,
                                                            uint32_t pos, uint32_t& x, uint32_t& y) {
    const wrs_session& S = session_of(sess, n_sessions, tile);
    const uint32_t local = tile - S.tile_begin, tiles_x = ((uint32_t)S.cam.width + 7) / 8;
    x = (local % tiles_x) * 8 + (pos & 7);
    y = (local / tiles_x) * 4 + (pos >> 3);
    return S;
}

// Store the result of lane `pos` of tile `tile`, its output pixel found again: an opaque copy of
// the tile index keeps the compiler from holding the session's output address and the pixel in
// registers through the traversal (in the packet kernel 1 % faster than holding them).
__device__ __forceinline__ void store_tile_pixel(const wrs_session* __restrict__ sess,
                                                 int n_sessions, uint32_t tile, uint32_t pos,
                                                 float4 o) {
    asm volatile("" : "+r"(tile));
    uint32_t x, y;
    const wrs_session& S = tile_pixel_of(sess, n_sessions, tile, pos, x, y);
    const uint32_t W = (uint32_t)S.cam.width;
    if (x < W && y < (uint32_t)S.cam.height)
        reinterpret_cast<float4*>(S.rgba_out)[(size_t)y * W + x] = o;
}

// Multi-session trace, one thread per pixel: warp w of the grid traces 8x4 tile w of the
// concatenated tile space.
template <int K, bool W4>
__global__ void __launch_bounds__(128, BatchedBounds<K, W4>::min_blocks) k_trace_batched_pp(const wrs_session* __restrict__ sess,
                                                          int n_sessions, uint32_t total_tiles,
                                                          Comp cp, int32_t* status) {
    const uint32_t tile = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (tile >= total_tiles) return;
    const uint32_t pos = threadIdx.x & 31u;
    uint32_t x, y;
    const wrs_session& S = tile_pixel_of(sess, n_sessions, tile, pos, x, y);
    const uint32_t W = (uint32_t)S.cam.width;
    const bool active = x < W && y < (uint32_t)S.cam.height;  // the tile is warp-uniform
    const Scene sc = session_scene<W4>(S);
    const RayCtx rc = make_ray_ctx(sc, S.cam, active ? (int)x : 0, active ? (int)y : 0);
    uint32_t overflow;
    Counts cnt;
    const float4 o = trace_ray_warp<K, false, W4>(sc, cp, rc, active, overflow, cnt);
    if (overflow) wrs::set_status(status, overflow);
    // (finding the output pixel again after the traversal, as the packet kernel does, spills
    // less but measured 1 % slower here)
    if (active) reinterpret_cast<float4*>(S.rgba_out)[(size_t)y * W + x] = o;
}

// Multi-session trace, packet schedule (4-wide nodes): warp w traces 8x4 tile w of the
// concatenated tile space with one warp-shared traversal; lanes outside their session's image
// take part without a ray (the tile, and so the session, is warp-uniform).
// Resident 128-thread blocks per SM of the multi-session packet kernel: 8 (64 registers, some
// spilled) takes 15.7 ms on the 64 sessions against 18.1 with 7 and 20.5 with no cap (94
// registers); reading the session's scene pointers from shared memory at each use instead (no
// spills) took 17.1 ms.
#ifndef WRS_BATCHED_PACKET_MIN_BLOCKS
#define WRS_BATCHED_PACKET_MIN_BLOCKS 8
#endif
template <int K>
__global__ void __launch_bounds__(128, WRS_BATCHED_PACKET_MIN_BLOCKS) k_trace_batched_packet(const wrs_session* __restrict__ sess,
                                                              int n_sessions, uint32_t total_tiles,
                                                              Comp cp, int32_t* status) {
    const uint32_t tile = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (tile >= total_tiles) return;
    const uint32_t pos = threadIdx.x & 31u;
    uint32_t x, y;
    const wrs_session& S = tile_pixel_of(sess, n_sessions, tile, pos, x, y);
    const bool active = x < (uint32_t)S.cam.width && y < (uint32_t)S.cam.height;
    const Scene sc = session_scene<true>(S);
    const RayCtx rc = make_ray_ctx(sc, S.cam, active ? (int)x : 0, active ? (int)y : 0);
    uint32_t overflow;
    const float4 o = trace_ray_packet<K>(sc, cp, rc, active, overflow);
    if (overflow) wrs::set_status(status, overflow);
    store_tile_pixel(sess, n_sessions, tile, pos, o);
}

// Multi-session trace with a schedule per session: the warp's tile belongs to one session, whose
// schedule field picks one thread per pixel or one warp-shared traversal (a warp-uniform branch).
#ifndef WRS_BATCHED_MIXED_MIN_BLOCKS
#define WRS_BATCHED_MIXED_MIN_BLOCKS WRS_BATCHED_PACKET_MIN_BLOCKS
#endif
template <int K, bool W4>
__global__ void __launch_bounds__(128, WRS_BATCHED_MIXED_MIN_BLOCKS) k_trace_batched_mixed(
        const wrs_session* __restrict__ sess, int n_sessions, uint32_t total_tiles, Comp cp,
        int32_t* status) {
    const uint32_t tile = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (tile >= total_tiles) return;
    const uint32_t pos = threadIdx.x & 31u;
    uint32_t x, y;
    const wrs_session& S = tile_pixel_of(sess, n_sessions, tile, pos, x, y);
    const uint32_t W = (uint32_t)S.cam.width;
    const bool active = x < W && y < (uint32_t)S.cam.height;
    const Scene sc = session_scene<true>(S);  // the per-pixel traversal reads wide only if W4
    uint32_t overflow;
    float4 o;
    if (S.schedule == WRS_SCHEDULE_PACKET) {
        const RayCtx rc = make_ray_ctx(sc, S.cam, active ? (int)x : 0, active ? (int)y : 0);
        o = trace_ray_packet<K>(sc, cp, rc, active, overflow);
    } else {
        const RayCtx rc = make_ray_ctx(sc, S.cam, active ? (int)x : 0, active ? (int)y : 0);
        Counts cnt;
        o = trace_ray_warp<K, false, W4>(sc, cp, rc, active, overflow, cnt);
    }
    if (overflow) wrs::set_status(status, overflow);
    if (active) reinterpret_cast<float4*>(S.rgba_out)[(size_t)y * W + x] = o;
}

// Persistent multi-session trace with lane refill.  Work is numbered in 8x4 ray tiles over all
// sessions (session s owns tiles [tile_begin_s, tile_begin_s + tiles_s)); a warp grabs chunks of
// kChunkTiles tiles from the global counter and refills its idle lanes from its chunk.  Each lane
// carries the scene of the session its ray belongs to, so one warp may trace several sessions.
constexpr uint32_t kChunkTiles = 4;

template <int K, bool W4>
__global__ void __launch_bounds__(128) k_trace_batched(const wrs_session* __restrict__ sess,
                                                       int n_sessions, uint32_t total_tiles,
                                                       Comp cp, uint32_t* work, int32_t* status) {
    const int lane = threadIdx.x & 31;
    Lane<K> L;
    int stack[wrs::kStack];
    Counts cnt;
    Scene sc;
    float4* out = nullptr;
    uint32_t n = 0, leaf = 1, m = 0;
    int32_t root = 0;
    int si = -1;
    bool active = false;
    bool more = true;                          // warp-uniform
    uint32_t next_ray = 0, end_ray = 0;        // warp-uniform: rays left in the warp's chunk
    while (true) {
        uint32_t idle = __ballot_sync(0xffffffffu, !active);
        if (more && __popc(idle) >= kRefill) {
            while (idle != 0u) {  // warp-uniform loop: hand rays of the chunk to idle lanes
                if (next_ray == end_ray) {
                    uint32_t c = 0;
                    if (lane == 0) c = atomicAdd(work, 1u);
                    c = __shfl_sync(0xffffffffu, c, 0);
                    if ((uint64_t)c * kChunkTiles >= total_tiles) { more = false; break; }
                    next_ray = c * kChunkTiles * 32u;
                    end_ray = min(c * kChunkTiles + kChunkTiles, total_tiles) * 32u;
                }
                const uint32_t take = min(end_ray - next_ray, (uint32_t)__popc(idle));
                const uint32_t rank = __popc(idle & ((1u << lane) - 1u));
                if (((idle >> lane) & 1u) && rank < take) {
                    const uint32_t r = next_ray + rank, tile = r >> 5, pos = r & 31u;
                    int lo = 0, hi = n_sessions - 1;  // last session with tile_begin <= tile
                    while (lo < hi) {
                        const int mid = (lo + hi + 1) >> 1;
                        if (sess[mid].tile_begin <= tile) lo = mid; else hi = mid - 1;
                    }
                    const wrs_session& S = sess[lo];
                    const uint32_t W = (uint32_t)S.cam.width, H = (uint32_t)S.cam.height;
                    const uint32_t local = tile - S.tile_begin, tiles_x = (W + 7) / 8;
                    const uint32_t x = (local % tiles_x) * 8 + (pos & 7);
                    const uint32_t y = (local / tiles_x) * 4 + (pos >> 3);
                    if (x < W && y < H) {
                        if (lo != si) {
                            si = lo;
                            sc.hdr = static_cast<const LbvhHeader*>(S.nodes);
                            sc.nodes = wrs::lbvh_nodes(S.nodes);
                            sc.wide = cp.width == 4 ? sc.nodes + 4 * (size_t)sc.hdr->wide_start
                                                    : nullptr;
                            sc.pos_r = reinterpret_cast<const float4*>(S.pos_r);
                            sc.rgba = reinterpret_cast<const float4*>(S.rgba);
                            sc.id = S.id;
                            sc.src = S.src;
                            sc.opacity = S.opacity;
                            out = reinterpret_cast<float4*>(S.rgba_out);
                            const LbvhHeader hd = *sc.hdr;
                            n = hd.n;
                            leaf = hd.leaf;
                            root = hd.root;
                            m = n == 0 ? 0 : (n + leaf - 1) / leaf;
                        }
                        L.pix = y * W + x;
                        if (n == 0) {
                            out[L.pix] = make_float4(0.f, 0.f, 0.f, 0.f);
                        } else {
                            L.ray = wrs::primary_ray(S.cam, (int)x, (int)y);
                            L.br = wrs::make_box_ray(L.ray, wrs::traversal_eps(L.ray, sc.hdr->maxabs));
                            L.T = 1.0f;
                            L.C = make_float3(0.f, 0.f, 0.f);
                            L.used = 0;
                            L.has_last = false;
                            L.last_key = 0.0f;
                            L.last_id = 0;
                            begin_pass(L, root, m);
                            active = true;
                        }
                    }
                }
                next_ray += take;
                for (uint32_t t = 0; t < take; t++) idle &= idle - 1u;  // drop the served lanes
            }
        }
        if (!__any_sync(0xffffffffu, active)) {
            if (!more) break;
            continue;
        }
        if (active) {
            const int rc = lane_step<K, W4>(sc, L, stack, n, leaf, m);
            if (rc != 0) {
                bool done = true;
                if (rc < 0) {
                    wrs::set_status(status, rc == -1 ? WRS_STATUS_STACK_OVERFLOW : WRS_STATUS_MALFORMED_TREE);
                } else if (!composite_chunk<K, false>(sc, cp, L.ray, L.ki, L.count, L.T, L.C, L.used, cnt)) {
                    done = false;
                    L.has_last = true;
                    L.last_key = L.kk[K - 1];
                    L.last_id = L.kid[K - 1];
                    begin_pass(L, root, m);
                }
                if (done) {
                    out[L.pix] = make_float4(L.C.x, L.C.y, L.C.z, 1.0f - L.T);
                    active = false;
                }
            }
        }
    }
}

// ---- adjoint (spec S7) ---------------------------------------------------------------------
// Pass A replays the forward pass chunk by chunk and records, per chunk, its lower bound and the
// transmittance at its start.  Pass B walks the chunks back to front; each chunk is gathered
// again (same bound, same K hits; the last chunk's hits are still in the k-buffer, so it is not),
// its transmittances recomputed forward from the recorded start, and the hits are then visited
// back to front with the suffix composite S and the suffix transmittance P, so no division by
// (1 - alpha) is needed.
// Pass A for one gathered chunk: advance the transmittance over its used hits exactly as the
// forward compositing does; *u = hits used in this chunk.  Returns true when the ray is finished.
template <int K>
__device__ __forceinline__ bool chunk_forward_T(const Scene& sc, const Comp& cp, const Ray& ray,
                                                const uint32_t (&ki)[K], int count, float& T,
                                                int& used, int& u) {
    u = 0;
#pragma unroll
    for (int s = 0; s < K; s++) {
        if (s >= count) break;
        if ((cp.max_hits > 0 && used == cp.max_hits) || T <= cp.t_stop) return true;
        const HitTerms h = hit_terms(sc, cp, ray, ki[s]);
        T = T * (1.0f - h.a);
        used++;
        u++;
    }
    if (count < K) return true;
    return (cp.max_hits > 0 && used == cp.max_hits) || T <= cp.t_stop;
}

struct GradOut {
    const float* scale;
    float gscale;
    float* g_rgba;
    float* g_op;
    float* g_sc;
};

// The adjoint of one composited hit k (sorted-splat index) with transmittance Ti in front of it,
// given the suffix composite S and suffix transmittance P of the hits behind it (spec S7); S and
// P are then extended over this hit.  Gradients go to the compacted splat order.
__device__ __forceinline__ void hit_adjoint(const Scene& sc, const Comp& cp, const Ray& ray,
                                            uint32_t k, float Ti, const float4 g, float3& S,
                                            float& P, const GradOut& go) {
    const HitTerms h = hit_terms(sc, cp, ray, k);
    const float gC = g.x * h.c.x + g.y * h.c.y + g.z * h.c.z;
    const float gS = g.x * S.x + g.y * S.y + g.z * S.z;
    const float dLda = Ti * (g.w * P - gS);
    const float pass = (h.x >= 0.0f && h.x <= 1.0f) ? 1.0f : 0.0f;
    const uint32_t src = __ldg(sc.src + k);
    const float tow = Ti * h.op * h.w;
    // one 16-byte vector atomic for the four colour components (g_rgba is 16-byte aligned)
    atomicAdd(reinterpret_cast<float4*>(go.g_rgba) + src,
              make_float4(tow * g.x, tow * g.y, tow * g.z, dLda * pass * h.op * h.w));
    if (go.g_op) atomicAdd(go.g_op + src, Ti * h.w * gC + dLda * pass * h.c.w * h.w);
    if (go.g_sc && cp.beta > 0.0f) {
        const float s_val = go.scale ? __ldg(go.scale + src) : go.gscale;
        const float dw = wrs::soft_dw(h.rho, cp.beta);
        if (s_val > 0.0f && dw != 0.0f) {
            const float dLdw = Ti * h.op * gC + dLda * pass * h.op * h.c.w;
            atomicAdd(go.g_sc + src, dLdw * dw * (-h.rho / s_val));
        }
    }
    const float ow = h.op * h.w;
    S.x = fmaf(1.0f - h.a, S.x, ow * h.c.x);
    S.y = fmaf(1.0f - h.a, S.y, ow * h.c.y);
    S.z = fmaf(1.0f - h.a, S.z, ow * h.c.z);
    P = P * (1.0f - h.a);
}

// Pass B for one re-gathered chunk: transmittances forward from the chunk's recorded start T0,
// then the adjoint of its u used hits back to front with the suffix composite S and suffix
// transmittance P of the later chunks.
template <int K>
__device__ __forceinline__ void chunk_adjoint(const Scene& sc, const Comp& cp, const Ray& ray,
                                              const uint32_t (&ki)[K], int u, float T0,
                                              const float4 g, float3& S, float& P,
                                              const GradOut& go) {
    float Tk[K];
    float t = T0;
#pragma unroll
    for (int s = 0; s < K; s++) {
        Tk[s] = t;
        if (s < u) t = t * (1.0f - hit_terms(sc, cp, ray, ki[s]).a);
    }
#pragma unroll
    for (int s = K - 1; s >= 0; s--) {
        if (s >= u) continue;
        hit_adjoint(sc, cp, ray, ki[s], Tk[s], g, S, P, go);
    }
}

// The per-lane backward over the binary nodes (the 4-wide nodes take backward_pixel_packet's
// warp-wide structure).
template <int K>
__device__ __forceinline__ void backward_pixel(const Scene& sc, const Comp& cp,
                                               const wrs_camera& cam,
                                               const float4* __restrict__ dimg, const GradOut& go,
                                               int32_t* status, HitFilter flt = HitFilter{nullptr, 0},
                                               size_t ray_base = 0) {
    int px, py;
    tile_pixel(threadIdx.x, px, py);
    const int tile_h = (blockDim.x >> 6) * 4;
    const int x = blockIdx.x * 16 + px, y = blockIdx.y * tile_h + py;
    if (x >= cam.width || y >= cam.height) return;
    const size_t pix = (size_t)y * cam.width + x;
    if (flt.count && flt.count[ray_base + pix] <= flt.cap) return;  // its recorded list serves
    const float4 g = dimg[pix];
    if (g.x == 0.f && g.y == 0.f && g.z == 0.f && g.w == 0.f) return;
    const RayCtx rc = make_ray_ctx(sc, cam, x, y);
    if (rc.n == 0) return;
    float b_key[wrs::kBwdChunks];
    uint32_t b_id[wrs::kBwdChunks];
    float b_T[wrs::kBwdChunks];
    uint8_t b_used[wrs::kBwdChunks];
    float kk[K];
    uint32_t ki[K], kid[K];
    Counts cnt;
    // pass A
    float T = 1.0f;
    int used = 0, chunks = 0;
    bool has_last = false;
    float last_key = 0.f;
    uint32_t last_id = 0;
    while (true) {
        if (chunks == wrs::kBwdChunks) { wrs::set_status(status, WRS_STATUS_CHUNK_OVERFLOW); return; }
        const int count = gather<K, false>(sc, rc.ray, rc.br, rc.n, rc.leaf, rc.root, has_last,
                                           last_key, last_id, kk, ki, kid, cnt);
        if (count < 0) { wrs::set_status(status, count == -1 ? WRS_STATUS_STACK_OVERFLOW : WRS_STATUS_MALFORMED_TREE); return; }
        b_key[chunks] = has_last ? last_key : -kInf;
        b_id[chunks] = last_id;
        b_T[chunks] = T;
        int u;
        const bool done = chunk_forward_T<K>(sc, cp, rc.ray, ki, count, T, used, u);
        b_used[chunks] = (uint8_t)u;
        chunks++;
        if (done) break;
        has_last = true;
        last_key = kk[K - 1];
        last_id = kid[K - 1];
    }
    // pass B
    float3 S = make_float3(0.f, 0.f, 0.f);
    float P = 1.0f;
    for (int c = chunks - 1; c >= 0; c--) {
        const int u = b_used[c];
        if (u == 0) continue;
        if (c != chunks - 1) {  // the last chunk's hits are still in the k-buffer from pass A
            const bool hl = b_key[c] != -kInf;
            gather<K, false>(sc, rc.ray, rc.br, rc.n, rc.leaf, rc.root, hl, b_key[c], b_id[c],
                                 kk, ki, kid, cnt);
        }
        chunk_adjoint<K>(sc, cp, rc.ray, ki, u, b_T[c], g, S, P, go);
    }
}


// The warp's backward (4-wide nodes): backward_pixel's two passes with every traversal taken by
// the whole warp, either one traversal shared by the warp (PACKET, gather_packet: the replay and
// the re-gathers run with all lanes active) or each lane's own traversal in warp-wide node and
// leaf steps (gather_warp).  Each lane keeps its own chunk table and k-buffer, so its hits are
// those of backward_pixel and its gradients equal backward_pixel's up to the order of the float
// atomics.  All 32 lanes of a warp take part in every gather (lanes without work pass
// part = false); the loops are warp-uniform.  A shared traversal fails for the whole warp; a
// lane's own traversal fails for that lane only (its status bit is set, it adds no more
// gradients).
template <int K, bool PACKET>
__device__ __forceinline__ int gather_bwd(const Scene& sc, const RayCtx& rc, bool part,
                                          bool has_last, float last_key, uint32_t last_id,
                                          float (&kk)[K], uint32_t (&ki)[K], uint32_t (&kid)[K]) {
    if constexpr (PACKET) {
        return gather_packet<K>(sc, rc.ray, rc.br, rc.n, rc.leaf, rc.root, part, has_last,
                                last_key, last_id, kk, ki, kid);
    } else {
        Counts none;
        return gather_warp<K, false>(sc, rc.ray, rc.br, rc.n, rc.leaf, rc.root, part, has_last,
                                     last_key, last_id, kk, ki, kid, none);
    }
}

template <int K, bool PACKET = true>
__device__ __forceinline__ void backward_pixel_packet(const Scene& sc, const Comp& cp,
                                                      const wrs_camera& cam,
                                                      const float4* __restrict__ dimg,
                                                      const GradOut& go, int32_t* status,
                                                      HitFilter flt = HitFilter{nullptr, 0},
                                                      size_t ray_base = 0) {
    int px, py;
    tile_pixel(threadIdx.x, px, py);
    const int tile_h = (blockDim.x >> 6) * 4;
    const int x = blockIdx.x * 16 + px, y = blockIdx.y * tile_h + py;
    const bool inside = x < cam.width && y < cam.height;
    const float4 g = inside ? dimg[(size_t)y * cam.width + x] : make_float4(0.f, 0.f, 0.f, 0.f);
    bool run = inside && !(g.x == 0.f && g.y == 0.f && g.z == 0.f && g.w == 0.f);
    if (run && flt.count && flt.count[ray_base + (size_t)y * cam.width + x] <= flt.cap)
        run = false;  // its recorded list serves
    // a warp none of whose rays runs (no gradient, or every list recorded) has nothing to do: it
    // leaves before the ray set-up (only warp-wide syncs follow, no block barrier)
    if (!__any_sync(0xffffffffu, run)) return;
    const RayCtx rc = make_ray_ctx(sc, cam, inside ? x : 0, inside ? y : 0);
    if (rc.n == 0) return;  // the same for every thread of the launch
    float b_key[wrs::kBwdChunks];
    uint32_t b_id[wrs::kBwdChunks];
    float b_T[wrs::kBwdChunks];
    uint8_t b_used[wrs::kBwdChunks];
    float kk[K];
    uint32_t ki[K], kid[K], last_ki[K];
#pragma unroll
    for (int s = 0; s < K; s++) last_ki[s] = 0xFFFFFFFFu;
    // pass A: replay the forward chunks (the last one's hits are kept for pass B)
    float T = 1.0f;
    int used = 0, chunks = 0;
    bool has_last = false, ok = run;
    float last_key = 0.f;
    uint32_t last_id = 0;
    while (__any_sync(0xffffffffu, run)) {
        if (run && chunks == wrs::kBwdChunks) {
            wrs::set_status(status, WRS_STATUS_CHUNK_OVERFLOW);
            run = false;
            ok = false;
        }
        const int count = gather_bwd<K, PACKET>(sc, rc, run, has_last, last_key, last_id, kk, ki,
                                                kid);
        if (PACKET && count < 0) {  // warp-uniform: the shared traversal failed for every lane
            if (inside)
                wrs::set_status(status, count == -1 ? WRS_STATUS_STACK_OVERFLOW : WRS_STATUS_MALFORMED_TREE);
            return;
        }
        if (!run) continue;
        if (count < 0) {  // this lane's own traversal failed
            wrs::set_status(status, count == -1 ? WRS_STATUS_STACK_OVERFLOW : WRS_STATUS_MALFORMED_TREE);
            run = false;
            ok = false;
            continue;
        }
        b_key[chunks] = has_last ? last_key : -kInf;
        b_id[chunks] = last_id;
        b_T[chunks] = T;
        int u;
        const bool done = chunk_forward_T<K>(sc, cp, rc.ray, ki, count, T, used, u);
        b_used[chunks] = (uint8_t)u;
        chunks++;
        if (done) {
            run = false;
#pragma unroll
            for (int s = 0; s < K; s++) last_ki[s] = ki[s];
        } else {
            has_last = true;
            last_key = kk[K - 1];
            last_id = kid[K - 1];
        }
    }
    if (!ok) chunks = 0;
    // pass B: chunks back to front, in step over the warp's largest chunk count
    float3 S = make_float3(0.f, 0.f, 0.f);
    float P = 1.0f;
    const int cmax = (int)__reduce_max_sync(0xffffffffu, (unsigned)chunks);
    for (int c = cmax - 1; c >= 0; c--) {
        const bool mine = c < chunks && b_used[c] != 0;
        const bool regather = mine && c != chunks - 1;  // the last chunk's hits are in last_ki
        if (__any_sync(0xffffffffu, regather)) {
            const bool hl = regather && b_key[c] != -kInf;
            const int count = gather_bwd<K, PACKET>(sc, rc, regather, hl,
                                                    regather ? b_key[c] : 0.f,
                                                    regather ? b_id[c] : 0u, kk, ki, kid);
            if (PACKET && count < 0) {
                if (inside)
                    wrs::set_status(status, count == -1 ? WRS_STATUS_STACK_OVERFLOW : WRS_STATUS_MALFORMED_TREE);
                return;
            }
            if (!PACKET && regather && count < 0) {  // (pass A traversed the same passes)
                wrs::set_status(status, count == -1 ? WRS_STATUS_STACK_OVERFLOW : WRS_STATUS_MALFORMED_TREE);
                chunks = 0;
                continue;
            }
        }
        if (mine) {
            const uint32_t(&hits)[K] = regather ? ki : last_ki;
            chunk_adjoint<K>(sc, cp, rc.ray, hits, b_used[c], b_T[c], g, S, P, go);
        }
    }
}

// The per-pixel backward: each lane's own traversal, in warp-wide node and leaf steps with 4-wide
// nodes, per lane with binary nodes.
template <int K, bool W4>
__device__ __forceinline__ void backward_pixel_any(const Scene& sc, const Comp& cp,
                                                   const wrs_camera& cam,
                                                   const float4* __restrict__ dimg,
                                                   const GradOut& go, int32_t* status,
                                                   HitFilter flt = HitFilter{nullptr, 0},
                                                   size_t ray_base = 0) {
    if constexpr (W4) backward_pixel_packet<K, false>(sc, cp, cam, dimg, go, status, flt, ray_base);
    else backward_pixel<K>(sc, cp, cam, dimg, go, status, flt, ray_base);
}

template <int K, bool W4>
__global__ void __launch_bounds__(128, BwdBounds<K, W4>::min_blocks) k_trace_bwd(Scene sc, Comp cp, wrs_camera cam,
                                                   const float4* __restrict__ dimg, GradOut go,
                                                   int32_t* status) {
    backward_pixel_any<K, W4>(sc, cp, cam, dimg, go, status);
}

// Several views in one launch (blockIdx.z = view, as k_trace_views); every view's gradients
// accumulate into the same per-splat buffers.
template <int K, bool W4>
__global__ void __launch_bounds__(128, BwdBounds<K, W4>::min_blocks) k_trace_bwd_views(Scene sc, Comp cp,
                                                         const __grid_constant__ ViewCams vc,
                                                         const float4* __restrict__ dimg,
                                                         size_t pixels, GradOut go,
                                                         HitFilter flt, size_t ray0,
                                                         int32_t* status) {
    backward_pixel_any<K, W4>(sc, cp, vc.cam[blockIdx.z], dimg + blockIdx.z * pixels, go, status,
                              flt, ray0 + blockIdx.z * pixels);
}

// 4 resident 256-thread blocks (64 registers): 6 % faster at K 4 and 13 % at K 2 than no cap
// (79-80 registers), 3 % faster than 5 blocks.
#ifndef WRS_BWD_PACKET_MIN_BLOCKS
#define WRS_BWD_PACKET_MIN_BLOCKS 4
#endif
template <int K>
__global__ void __launch_bounds__(256, WRS_BWD_PACKET_MIN_BLOCKS) k_trace_bwd_packet(Scene sc, Comp cp, wrs_camera cam,
                                                          const float4* __restrict__ dimg,
                                                          GradOut go, int32_t* status) {
    backward_pixel_packet<K>(sc, cp, cam, dimg, go, status);
}

template <int K>
__global__ void __launch_bounds__(256, WRS_BWD_PACKET_MIN_BLOCKS) k_trace_bwd_packet_views(Scene sc, Comp cp,
                                                                const __grid_constant__ ViewCams vc,
                                                                const float4* __restrict__ dimg,
                                                                size_t pixels, GradOut go,
                                                                HitFilter flt, size_t ray0,
                                                                int32_t* status) {
    backward_pixel_packet<K>(sc, cp, vc.cam[blockIdx.z], dimg + blockIdx.z * pixels, go, status,
                             flt, ray0 + blockIdx.z * pixels);
}

// The adjoint from recorded hit lists (no traversal): for each ray of each view whose list was
// kept, the transmittances in front of its hits are rebuilt forward from the list (the forward
// pass's own sequence), then the hits are visited back to front with hit_adjoint.  Rays whose list
// went over capacity are left to a re-traversing launch (HitFilter).
constexpr uint32_t kMaxRecord = 32;  // largest hit-list capacity (transmittances kept per thread)
__global__ void __launch_bounds__(128) k_trace_bwd_recorded(Scene sc, Comp cp,
                                                            const __grid_constant__ ViewCams vc,
                                                            const float4* __restrict__ dimg,
                                                            size_t pixels, GradOut go,
                                                            const uint32_t* __restrict__ hits,
                                                            const uint32_t* __restrict__ count,
                                                            uint32_t cap, size_t ray0) {
    const wrs_camera& cam = vc.cam[blockIdx.z];
    int px, py;
    tile_pixel(threadIdx.x, px, py);
    const int tile_h = (blockDim.x >> 6) * 4;
    const int x = blockIdx.x * 16 + px, y = blockIdx.y * tile_h + py;
    if (x >= cam.width || y >= cam.height) return;
    const size_t pix = (size_t)y * cam.width + x;
    const size_t ray = ray0 + blockIdx.z * pixels + pix;
    const uint32_t n = count[ray];
    if (n == 0 || n > cap) return;
    const float4 g = dimg[blockIdx.z * pixels + pix];
    if (g.x == 0.f && g.y == 0.f && g.z == 0.f && g.w == 0.f) return;
    const Ray r = wrs::primary_ray(cam, x, y);
    const uint32_t* h = hits + ray * cap;
    float Tb[kMaxRecord];
    float t = 1.0f;
    for (uint32_t i = 0; i < n; i++) {
        Tb[i] = t;
        t = t * (1.0f - hit_terms(sc, cp, r, __ldg(h + i)).a);
    }
    float3 S = make_float3(0.f, 0.f, 0.f);
    float P = 1.0f;
    for (int i = (int)n - 1; i >= 0; i--) hit_adjoint(sc, cp, r, __ldg(h + i), Tb[i], g, S, P, go);
}

// Persistent backward with lane refill: the per-pixel backward's two phases run as a per-lane
// state machine over the same traversal steps as k_trace_pr.  Phase A replays the forward passes
// and records each chunk's bound and starting transmittance; phase B re-gathers the chunks back
// to front and applies chunk_adjoint.
template <int K, bool W4>
__global__ void __launch_bounds__(128) k_trace_bwd_pr(Scene sc, Comp cp, wrs_camera cam,
                                                      const float4* __restrict__ dimg, GradOut go,
                                                      int32_t* status) {
    __shared__ uint32_t s_next;
    if (threadIdx.x == 0) s_next = 0;
    __syncthreads();
    const uint32_t W = (uint32_t)cam.width, H = (uint32_t)cam.height;
    const uint32_t tiles_x = (W + 7) / 8, n_tiles = tiles_x * ((H + 3) / 4);
    const uint32_t G = gridDim.x;
    const uint32_t my_rays = blockIdx.x < n_tiles ? ((n_tiles - 1 - blockIdx.x) / G + 1) * 32 : 0;
    const LbvhHeader hd = *sc.hdr;
    const uint32_t n = hd.n, leaf = hd.leaf;
    const uint32_t m = n == 0 ? 0 : (n + leaf - 1) / leaf;
    const int lane = threadIdx.x & 31;
    Lane<K> L;
    int stack[wrs::kStack];
    float b_key[wrs::kBwdChunks];
    uint32_t b_id[wrs::kBwdChunks];
    float b_T[wrs::kBwdChunks];
    uint8_t b_used[wrs::kBwdChunks];
    float4 g = make_float4(0.f, 0.f, 0.f, 0.f);
    float3 S = make_float3(0.f, 0.f, 0.f);
    float P = 1.0f;
    int phase = 0, chunks = 0, cur = 0;
    bool active = false;
    bool more = my_rays > 0 && n > 0;
    while (true) {
        const uint32_t idle = __ballot_sync(0xffffffffu, !active);
        if (more && __popc(idle) >= kRefill) {
            const uint32_t c = __popc(idle);
            uint32_t base = 0;
            if (lane == 0) base = atomicAdd(&s_next, c);
            base = __shfl_sync(0xffffffffu, base, 0);
            if (base + c >= my_rays) more = false;
            if (!active) {
                const uint32_t r = base + __popc(idle & ((1u << lane) - 1u));
                if (r < my_rays) {
                    const uint32_t tile = blockIdx.x + (r >> 5) * G, pos = r & 31;
                    const uint32_t x = (tile % tiles_x) * 8 + (pos & 7);
                    const uint32_t y = (tile / tiles_x) * 4 + (pos >> 3);
                    if (x < W && y < H) {
                        g = dimg[(size_t)y * W + x];
                        if (g.x != 0.f || g.y != 0.f || g.z != 0.f || g.w != 0.f) {
                            L.ray = wrs::primary_ray(cam, (int)x, (int)y);
                            L.br = wrs::make_box_ray(L.ray, wrs::traversal_eps(L.ray, hd.maxabs));
                            L.T = 1.0f;
                            L.used = 0;
                            L.has_last = false;
                            L.last_key = 0.0f;
                            L.last_id = 0;
                            phase = 0;
                            chunks = 0;
                            b_key[0] = -kInf;
                            b_id[0] = 0;
                            b_T[0] = 1.0f;
                            begin_pass(L, hd.root, m);
                            active = true;
                        }
                    }
                }
            }
        }
        if (!__any_sync(0xffffffffu, active)) {
            if (!more) break;
            continue;
        }
        if (!active) continue;
        const int rc = lane_step<K, W4>(sc, L, stack, n, leaf, m);
        if (rc == 0) continue;
        if (rc < 0) {
            wrs::set_status(status, rc == -1 ? WRS_STATUS_STACK_OVERFLOW : WRS_STATUS_MALFORMED_TREE);
            active = false;
            continue;
        }
        if (phase == 0) {  // a forward replay pass finished
            int u;
            const bool done = chunk_forward_T<K>(sc, cp, L.ray, L.ki, L.count, L.T, L.used, u);
            b_used[chunks] = (uint8_t)u;
            chunks++;
            if (!done) {
                if (chunks == wrs::kBwdChunks) {
                    wrs::set_status(status, WRS_STATUS_CHUNK_OVERFLOW);
                    active = false;
                    continue;
                }
                L.has_last = true;
                L.last_key = L.kk[K - 1];
                L.last_id = L.kid[K - 1];
                b_key[chunks] = L.last_key;
                b_id[chunks] = L.last_id;
                b_T[chunks] = L.T;
                begin_pass(L, hd.root, m);
                continue;
            }
            phase = 1;
            S = make_float3(0.f, 0.f, 0.f);
            P = 1.0f;
            cur = chunks - 1;  // the last chunk's hits are still in the k-buffer: no re-gather
            if (b_used[cur] != 0)
                chunk_adjoint<K>(sc, cp, L.ray, L.ki, b_used[cur], b_T[cur], g, S, P, go);
        } else {  // chunk `cur` re-gathered: its adjoint
            chunk_adjoint<K>(sc, cp, L.ray, L.ki, b_used[cur], b_T[cur], g, S, P, go);
        }
        do { cur--; } while (cur >= 0 && b_used[cur] == 0);  // next chunk with used hits
        if (cur < 0) {
            active = false;
            continue;
        }
        L.has_last = b_key[cur] != -kInf;
        L.last_key = b_key[cur];
        L.last_id = b_id[cur];
        begin_pass(L, hd.root, m);
    }
}

// Batched trace over binary nodes: flags every session whose tree was built without all its
// binary records (layout WRS_LBVH_WIDE), unless the session's own schedule walks the 4-wide
// nodes (per_session and a packet session).
__global__ void k_check_binary_layout(const wrs_session* __restrict__ sess, int n_sessions,
                                      bool per_session, int32_t* status) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_sessions) return;
    if (per_session && sess[i].schedule == WRS_SCHEDULE_PACKET) return;
    const LbvhHeader* h = static_cast<const LbvhHeader*>(sess[i].nodes);
    if (h->layout != WRS_LBVH_FULL) wrs::set_status(status, WRS_STATUS_MALFORMED_TREE);
}

// ---- host dispatch -------------------------------------------------------------------------
int check_trace_args(const wrs_lbvh* bvh, const wrs_splats* sorted, const wrs_camera* cam,
                     const wrs_trace_params* p, const char* fn) {
    if (int rc = wrs::check_camera(cam, fn)) return rc;
    if (!bvh || !bvh->nodes || !sorted || !p) return wrs::fail(WRS_ERR_ARG, "%s: NULL struct", fn);
    if (!sorted->pos_r || !sorted->rgba || !sorted->id || !sorted->src)
        return wrs::fail(WRS_ERR_ARG, "%s: sorted splats need pos_r, rgba, id and src", fn);
    if ((reinterpret_cast<uintptr_t>(sorted->pos_r) | reinterpret_cast<uintptr_t>(sorted->rgba) |
         reinterpret_cast<uintptr_t>(bvh->nodes)) & 15)
        return wrs::fail(WRS_ERR_ARG, "%s: float4 arrays must be 16-byte aligned", fn);
    const int K = p->k_chunk;
    if (K != 1 && K != 2 && K != 4 && K != 8 && K != 16)
        return wrs::fail(WRS_ERR_ARG, "%s: k_chunk %d not in {1,2,4,8,16}", fn, K);
    if (p->block != 64 && p->block != 128 && p->block != 256)
        return wrs::fail(WRS_ERR_ARG, "%s: block %d not in {64,128,256}", fn, p->block);
    if (p->max_hits < 0) return wrs::fail(WRS_ERR_ARG, "%s: max_hits < 0", fn);
    if (p->schedule != WRS_SCHEDULE_PER_PIXEL && p->schedule != WRS_SCHEDULE_PERSISTENT &&
        p->schedule != WRS_SCHEDULE_PACKET)
        return wrs::fail(WRS_ERR_ARG, "%s: unknown schedule %d", fn, p->schedule);
    if (p->width != 0 && p->width != 2 && p->width != 4)
        return wrs::fail(WRS_ERR_ARG, "%s: width %d not 2 or 4 (0 = 2)", fn, p->width);
    if (bvh->layout != WRS_LBVH_FULL && bvh->layout != WRS_LBVH_WIDE)
        return wrs::fail(WRS_ERR_ARG, "%s: unknown tree layout %u", fn, bvh->layout);
    if (bvh->layout == WRS_LBVH_WIDE && p->width != 4 && p->schedule != WRS_SCHEDULE_PACKET)
        return wrs::fail(WRS_ERR_ARG,
                         "%s: the binary traversal (width %d) needs a tree built with layout "
                         "WRS_LBVH_FULL; this one has only its 4-wide nodes", fn, p->width);
    if (!(p->t_stop >= 0.0f && p->t_stop < 1.0f))
        return wrs::fail(WRS_ERR_ARG, "%s: t_stop must be in [0, 1)", fn);
    if (!(p->edge_softness >= 0.0f && p->edge_softness < 1.0f))
        return wrs::fail(WRS_ERR_ARG, "%s: edge_softness must be in [0, 1)", fn);
    return WRS_OK;
}

Scene make_scene(const wrs_lbvh* bvh, const wrs_splats* sorted, const float* opacity,
                 int width = 2) {
    Scene sc;
    sc.hdr = static_cast<const LbvhHeader*>(bvh->nodes);
    sc.nodes = wrs::lbvh_nodes(bvh->nodes);
    sc.wide = width == 4 ? sc.nodes + 4 * (size_t)wrs::lbvh_binary_slots(bvh->capacity, bvh->leaf_size)
                         : nullptr;
    sc.pos_r = reinterpret_cast<const float4*>(sorted->pos_r);
    sc.rgba = reinterpret_cast<const float4*>(sorted->rgba);
    sc.id = sorted->id;
    sc.src = sorted->src;
    sc.opacity = opacity;
    return sc;
}

// A first-hit query (H small) needs no more than H hits per pass.
int effective_k(const wrs_trace_params* p) {
    int K = p->k_chunk;
    if (p->max_hits > 0) {
        int need = 1;
        while (need < p->max_hits) need <<= 1;
        if (need < K) K = need;
    }
    return K;
}

template <template <int, bool> class Launch, bool W4, typename... A>
void dispatch_k1(int K, A&&... a) {
    switch (K) {
        case 1: Launch<1, W4>::run(a...); break;
        case 2: Launch<2, W4>::run(a...); break;
        case 4: Launch<4, W4>::run(a...); break;
        case 8: Launch<8, W4>::run(a...); break;
        default: Launch<16, W4>::run(a...); break;
    }
}

// launch Launch<K, W4>::run(a...) for the runtime K and traversal width
template <template <int, bool> class Launch, typename... A>
void dispatch_k(int K, int width, A&&... a) {
    if (width == 4) dispatch_k1<Launch, true>(K, a...);
    else dispatch_k1<Launch, false>(K, a...);
}

template <template <int, bool> class Launch>
int blocks_per_sm_kw(int K, int width, int block) {
    const bool w4 = width == 4;
    switch (K) {
        case 1: return w4 ? Launch<1, true>::blocks_per_sm(block) : Launch<1, false>::blocks_per_sm(block);
        case 2: return w4 ? Launch<2, true>::blocks_per_sm(block) : Launch<2, false>::blocks_per_sm(block);
        case 4: return w4 ? Launch<4, true>::blocks_per_sm(block) : Launch<4, false>::blocks_per_sm(block);
        case 8: return w4 ? Launch<8, true>::blocks_per_sm(block) : Launch<8, false>::blocks_per_sm(block);
        default: return w4 ? Launch<16, true>::blocks_per_sm(block) : Launch<16, false>::blocks_per_sm(block);
    }
}

template <int K, bool W4> struct LaunchTrace {
    static void run(dim3 g, int b, cudaStream_t s, Scene sc, Comp cp, wrs_camera cam, float4* o,
                    int32_t* st) {
        k_trace<K, W4><<<g, b, 0, s>>>(sc, cp, cam, o, st);
    }
};
template <int K, bool W4> struct LaunchTraceViews {
    static void run(dim3 g, int b, cudaStream_t s, Scene sc, Comp cp, const ViewCams& vc,
                    float4* o, size_t pixels, int32_t* st) {
        k_trace_views<K, W4><<<g, b, 0, s>>>(sc, cp, vc, o, pixels, st);
    }
};
template <int K, bool W4> struct LaunchPacketViews {  // 4-wide implied, as LaunchTracePacket
    static void run(dim3 g, int b, cudaStream_t s, Scene sc, Comp cp, const ViewCams& vc,
                    float4* o, size_t pixels, int32_t* st) {
        k_trace_packet_views<K><<<g, b, 0, s>>>(sc, cp, vc, o, pixels, st);
    }
};
template <int K, bool W4> struct LaunchBwdViews {
    static void run(dim3 g, int b, cudaStream_t s, Scene sc, Comp cp, const ViewCams& vc,
                    const float4* d, size_t pixels, GradOut go, HitFilter flt, size_t ray0,
                    int32_t* st) {
        k_trace_bwd_views<K, W4><<<g, b, 0, s>>>(sc, cp, vc, d, pixels, go, flt, ray0, st);
    }
};
template <int K, bool W4> struct LaunchTraceViewsRec {
    static void run(dim3 g, int b, cudaStream_t s, Scene sc, Comp cp, const ViewCams& vc,
                    float4* o, size_t pixels, HitRecord hr, size_t ray0, int32_t* st) {
        k_trace_views_rec<K, W4><<<g, b, 0, s>>>(sc, cp, vc, o, pixels, hr, ray0, st);
    }
};
template <int K, bool W4> struct LaunchPacketViewsRec {  // 4-wide implied
    static void run(dim3 g, int b, cudaStream_t s, Scene sc, Comp cp, const ViewCams& vc,
                    float4* o, size_t pixels, HitRecord hr, size_t ray0, int32_t* st) {
        k_trace_packet_views_rec<K><<<g, b, 0, s>>>(sc, cp, vc, o, pixels, hr, ray0, st);
    }
};
template <int K, bool W4> struct LaunchBwdPacket {  // 4-wide implied, as LaunchTracePacket
    static void run(dim3 g, int b, cudaStream_t s, Scene sc, Comp cp, wrs_camera cam,
                    const float4* d, GradOut go, int32_t* st) {
        k_trace_bwd_packet<K><<<g, b, 0, s>>>(sc, cp, cam, d, go, st);
    }
};
template <int K, bool W4> struct LaunchBwdPacketViews {
    static void run(dim3 g, int b, cudaStream_t s, Scene sc, Comp cp, const ViewCams& vc,
                    const float4* d, size_t pixels, GradOut go, HitFilter flt, size_t ray0,
                    int32_t* st) {
        k_trace_bwd_packet_views<K><<<g, b, 0, s>>>(sc, cp, vc, d, pixels, go, flt, ray0, st);
    }
};
template <int K, bool W4> struct LaunchBatchedPP {
    static void run(uint32_t blocks, const wrs_session* ss, int ns, uint32_t tt, Comp cp,
                    int32_t* st, cudaStream_t s) {
        k_trace_batched_pp<K, W4><<<blocks, 128, 0, s>>>(ss, ns, tt, cp, st);
    }
};
template <int K, bool W4> struct LaunchBatchedPacket {  // 4-wide implied, as LaunchTracePacket
    static void run(uint32_t blocks, const wrs_session* ss, int ns, uint32_t tt, Comp cp,
                    int32_t* st, cudaStream_t s) {
        k_trace_batched_packet<K><<<blocks, 128, 0, s>>>(ss, ns, tt, cp, st);
    }
};
template <int K, bool W4> struct LaunchBatchedMixed {
    static void run(uint32_t blocks, const wrs_session* ss, int ns, uint32_t tt, Comp cp,
                    int32_t* st, cudaStream_t s) {
        k_trace_batched_mixed<K, W4><<<blocks, 128, 0, s>>>(ss, ns, tt, cp, st);
    }
};
template <int K, bool W4> struct LaunchTracePacket {  // W4 is implied: the packet traversal is 4-wide
    static void run(dim3 g, int b, cudaStream_t s, Scene sc, Comp cp, wrs_camera cam, float4* o,
                    int32_t* st) {
        k_trace_packet<K><<<g, b, 0, s>>>(sc, cp, cam, o, st);
    }
};
template <int K, bool W4> struct LaunchTracePr {
    static void run(int g, int b, cudaStream_t s, Scene sc, Comp cp, wrs_camera cam, float4* o,
                    int32_t* st) {
        k_trace_pr<K, W4><<<g, b, 0, s>>>(sc, cp, cam, o, st);
    }
    static int blocks_per_sm(int b) {
        int nb = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_trace_pr<K, W4>, b, 0);
        return nb;
    }
};
template <int K, bool W4> struct LaunchCount {
    static void run(dim3 g, int b, cudaStream_t s, Scene sc, Comp cp, wrs_camera cam,
                    unsigned long long* c, int32_t* st) {
        k_trace_count<K, W4><<<g, b, 0, s>>>(sc, cp, cam, c, st);
    }
};
template <int K, bool W4> struct LaunchBatched {
    static void run(int g, int b, cudaStream_t s, const wrs_session* ss, int ns, uint32_t tt,
                    Comp cp, uint32_t* w, int32_t* st) {
        k_trace_batched<K, W4><<<g, b, 0, s>>>(ss, ns, tt, cp, w, st);
    }
    static int blocks_per_sm(int b) {
        int nb = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_trace_batched<K, W4>, b, 0);
        return nb;
    }
};
template <int K, bool W4> struct LaunchBwd {
    static void run(dim3 g, int b, cudaStream_t s, Scene sc, Comp cp, wrs_camera cam,
                    const float4* d, GradOut go, int32_t* st) {
        k_trace_bwd<K, W4><<<g, b, 0, s>>>(sc, cp, cam, d, go, st);
    }
};
template <int K, bool W4> struct LaunchBwdPr {
    static void run(int g, int b, cudaStream_t s, Scene sc, Comp cp, wrs_camera cam,
                    const float4* d, GradOut go, int32_t* st) {
        k_trace_bwd_pr<K, W4><<<g, b, 0, s>>>(sc, cp, cam, d, go, st);
    }
    static int blocks_per_sm(int b) {
        int nb = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_trace_bwd_pr<K, W4>, b, 0);
        return nb;
    }
};

dim3 grid_for(const wrs_camera* cam, int block) {
    const int tile_h = (block / 64) * 4;
    return dim3((cam->width + 15) / 16, (cam->height + tile_h - 1) / tile_h);
}

Comp comp_of(const wrs_trace_params* p) {
    return Comp{p->max_hits, p->t_stop, p->edge_softness, p->width};
}

// One resident wave of 128-thread blocks of a persistent kernel (occupancy x SMs).  Queried once
// per (kernel, K, width) and cached, so that a call made during stream capture issues nothing but
// its memsets and the launch.
template <template <int, bool> class Launch>
int resident_grid(int K, int width) {
    static int cached[5][2] = {{0}};
    const int ki = K == 1 ? 0 : K == 2 ? 1 : K == 4 ? 2 : K == 8 ? 3 : 4;
    const int wi = width == 4 ? 1 : 0;
    if (cached[ki][wi] == 0) {
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const int per_sm = blocks_per_sm_kw<Launch>(K, width, 128);
        cached[ki][wi] = sms * (per_sm < 1 ? 1 : per_sm);
    }
    return cached[ki][wi];
}

}  // namespace

extern "C" {

int wrs_trace(const wrs_lbvh* bvh, const wrs_splats* sorted, const wrs_camera* cam,
              const wrs_trace_params* params, float* rgba_out, int32_t* status,
              wrs_stream_t stream) {
    const char* fn = "wrs_trace";
    if (int rc = check_trace_args(bvh, sorted, cam, params, fn)) return rc;
    if (!rgba_out || (reinterpret_cast<uintptr_t>(rgba_out) & 15))
        return wrs::fail(WRS_ERR_ARG, "%s: rgba_out NULL or not 16-byte aligned", fn);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int K = effective_k(params), W = params->width;
    const Scene sc = make_scene(bvh, sorted, params->opacity, W);
    float4* out = reinterpret_cast<float4*>(rgba_out);
    if (params->schedule == WRS_SCHEDULE_PERSISTENT)
        dispatch_k<LaunchTracePr>(K, W, resident_grid<LaunchTracePr>(K, W), 128, s, sc,
                                  comp_of(params), *cam, out, status);
    else if (params->schedule == WRS_SCHEDULE_PACKET)
        dispatch_k1<LaunchTracePacket, true>(K, grid_for(cam, params->block), params->block, s,
                                             make_scene(bvh, sorted, params->opacity, 4),
                                             comp_of(params), *cam, out, status);
    else {
        // a capped kernel is built for blocks of at most 128 threads
        const int block = (pixel_block_128(K, W == 4) && params->block > 128) ? 128 : params->block;
        dispatch_k<LaunchTrace>(K, W, grid_for(cam, block), block, s, sc, comp_of(params), *cam,
                                out, status);
    }
    WRS_LAUNCH_CHECK(fn);
    return WRS_OK;
}

// Views of one scene: every camera valid and of the first camera's size.
static int check_views(const wrs_lbvh* bvh, const wrs_splats* sorted, const wrs_camera* cams,
                       int n_views, const wrs_trace_params* params, const char* fn) {
    if (!cams || n_views < 1) return wrs::fail(WRS_ERR_ARG, "%s: cams NULL or n_views < 1", fn);
    if (int rc = check_trace_args(bvh, sorted, &cams[0], params, fn)) return rc;
    for (int v = 1; v < n_views; v++) {
        if (int rc = wrs::check_camera(&cams[v], fn)) return rc;
        if (cams[v].width != cams[0].width || cams[v].height != cams[0].height)
            return wrs::fail(WRS_ERR_ARG, "%s: view %d is %dx%d, view 0 is %dx%d", fn, v,
                             cams[v].width, cams[v].height, cams[0].width, cams[0].height);
    }
    return WRS_OK;
}

}  // extern "C"

namespace {
// wrs_trace_views, recording the composited hits when rec is given.
int trace_views_impl(const wrs_lbvh* bvh, const wrs_splats* sorted, const wrs_camera* cams,
                     int32_t n_views, const wrs_trace_params* params, float* rgba_out,
                     const HitRecord* rec, int32_t* status, wrs_stream_t stream, const char* fn) {
    if (int rc = check_views(bvh, sorted, cams, n_views, params, fn)) return rc;
    if (!rgba_out || (reinterpret_cast<uintptr_t>(rgba_out) & 15))
        return wrs::fail(WRS_ERR_ARG, "%s: rgba_out NULL or not 16-byte aligned", fn);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int K = effective_k(params), W = params->width;
    const size_t pixels = (size_t)cams[0].width * cams[0].height;
    const bool packet = params->schedule == WRS_SCHEDULE_PACKET;
    // per-pixel blocks as wrs_trace; the persistent schedule runs per pixel here (the views
    // together fill the GPU, which is what lane refill is for)
    const int block = packet ? params->block
                             : ((pixel_block_128(K, W == 4) && params->block > 128) ? 128 : params->block);
    const Scene sc = make_scene(bvh, sorted, params->opacity, packet ? 4 : W);
    for (int v0 = 0; v0 < n_views; v0 += kMaxViews) {
        const int nv = n_views - v0 < kMaxViews ? n_views - v0 : kMaxViews;
        ViewCams vc;
        for (int v = 0; v < nv; v++) vc.cam[v] = cams[v0 + v];
        dim3 g = grid_for(&cams[0], block);
        g.z = (unsigned)nv;
        float4* out = reinterpret_cast<float4*>(rgba_out) + (size_t)v0 * pixels;
        const size_t ray0 = (size_t)v0 * pixels;
        if (rec && packet)
            dispatch_k1<LaunchPacketViewsRec, true>(K, g, block, s, sc, comp_of(params), vc, out,
                                                    pixels, *rec, ray0, status);
        else if (rec)
            dispatch_k<LaunchTraceViewsRec>(K, W, g, block, s, sc, comp_of(params), vc, out,
                                            pixels, *rec, ray0, status);
        else if (packet)
            dispatch_k1<LaunchPacketViews, true>(K, g, block, s, sc, comp_of(params), vc, out,
                                                 pixels, status);
        else
            dispatch_k<LaunchTraceViews>(K, W, g, block, s, sc, comp_of(params), vc, out, pixels,
                                         status);
        WRS_LAUNCH_CHECK(fn);
    }
    return WRS_OK;
}

int check_record(const uint32_t* hits, const uint32_t* hit_count, uint32_t hit_capacity,
                 const char* fn) {
    if (!hits || !hit_count) return wrs::fail(WRS_ERR_ARG, "%s: hits / hit_count NULL", fn);
    if (hit_capacity < 1 || hit_capacity > kMaxRecord)
        return wrs::fail(WRS_ERR_ARG, "%s: hit_capacity %u not in 1..%u", fn, hit_capacity,
                         kMaxRecord);
    return WRS_OK;
}
}  // namespace

extern "C" {

int wrs_trace_views(const wrs_lbvh* bvh, const wrs_splats* sorted, const wrs_camera* cams,
                    int32_t n_views, const wrs_trace_params* params, float* rgba_out,
                    int32_t* status, wrs_stream_t stream) {
    return trace_views_impl(bvh, sorted, cams, n_views, params, rgba_out, nullptr, status, stream,
                            "wrs_trace_views");
}

int wrs_trace_views_record(const wrs_lbvh* bvh, const wrs_splats* sorted, const wrs_camera* cams,
                           int32_t n_views, const wrs_trace_params* params, float* rgba_out,
                           uint32_t* hits, uint32_t* hit_count, uint32_t hit_capacity,
                           int32_t* status, wrs_stream_t stream) {
    const char* fn = "wrs_trace_views_record";
    if (int rc = check_record(hits, hit_count, hit_capacity, fn)) return rc;
    const HitRecord rec = {hits, hit_count, hit_capacity};
    return trace_views_impl(bvh, sorted, cams, n_views, params, rgba_out, &rec, status, stream, fn);
}

int wrs_trace_count(const wrs_lbvh* bvh, const wrs_splats* sorted, const wrs_camera* cam,
                    const wrs_trace_params* params, unsigned long long* counters,
                    int32_t* status, wrs_stream_t stream) {
    const char* fn = "wrs_trace_count";
    if (int rc = check_trace_args(bvh, sorted, cam, params, fn)) return rc;
    if (!counters) return wrs::fail(WRS_ERR_ARG, "%s: counters is NULL", fn);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemsetAsync(counters, 0, 6 * sizeof(unsigned long long), s);
    if (e != cudaSuccess) return wrs::cuda_fail(e, fn);
    dispatch_k<LaunchCount>(effective_k(params), params->width, grid_for(cam, params->block),
                            params->block, s, make_scene(bvh, sorted, params->opacity, params->width),
                            comp_of(params), *cam, counters, status);
    WRS_LAUNCH_CHECK(fn);
    return WRS_OK;
}

uint32_t wrs_session_tiles(int32_t width, int32_t height) {
    if (width <= 0 || height <= 0) return 0;
    return (uint32_t)((width + 7) / 8) * (uint32_t)((height + 3) / 4);
}

int wrs_trace_batched(const wrs_session* sessions, int32_t n_sessions, uint32_t total_tiles,
                      const wrs_trace_params* params, uint32_t* work_counter, int32_t* status,
                      wrs_stream_t stream) {
    const char* fn = "wrs_trace_batched";
    if (!sessions || !params || !work_counter)
        return wrs::fail(WRS_ERR_ARG, "%s: NULL pointer", fn);
    if (n_sessions <= 0) return wrs::fail(WRS_ERR_ARG, "%s: n_sessions must be > 0", fn);
    const int K0 = params->k_chunk;
    if (K0 != 1 && K0 != 2 && K0 != 4 && K0 != 8 && K0 != 16)
        return wrs::fail(WRS_ERR_ARG, "%s: k_chunk %d not in {1,2,4,8,16}", fn, K0);
    if (params->max_hits < 0 || !(params->t_stop >= 0.0f && params->t_stop < 1.0f) ||
        !(params->edge_softness >= 0.0f && params->edge_softness < 1.0f))
        return wrs::fail(WRS_ERR_ARG, "%s: bad compositing parameters", fn);
    if (params->width != 0 && params->width != 2 && params->width != 4)
        return wrs::fail(WRS_ERR_ARG, "%s: width %d not 2 or 4 (0 = 2)", fn, params->width);
    if (params->schedule < WRS_SCHEDULE_PER_PIXEL || params->schedule > WRS_SCHEDULE_PER_SESSION)
        return wrs::fail(WRS_ERR_ARG, "%s: unknown schedule %d", fn, params->schedule);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemsetAsync(work_counter, 0, sizeof(uint32_t), s);
    if (e != cudaSuccess) return wrs::cuda_fail(e, fn);
    if (total_tiles == 0) return WRS_OK;
    const int K = effective_k(params), W = params->width;
    if (W != 4 && params->schedule != WRS_SCHEDULE_PACKET && status) {
        k_check_binary_layout<<<(n_sessions + 127) / 128, 128, 0, s>>>(
            sessions, n_sessions, params->schedule == WRS_SCHEDULE_PER_SESSION, status);
        WRS_LAUNCH_CHECK(fn);
    }
    if (params->schedule == WRS_SCHEDULE_PER_PIXEL)
        dispatch_k<LaunchBatchedPP>(K, W, (total_tiles + 3) / 4, sessions, n_sessions, total_tiles,
                                    comp_of(params), status, s);
    else if (params->schedule == WRS_SCHEDULE_PACKET)
        dispatch_k<LaunchBatchedPacket>(K, W, (total_tiles + 3) / 4, sessions, n_sessions,
                                        total_tiles, comp_of(params), status, s);
    else if (params->schedule == WRS_SCHEDULE_PER_SESSION)
        dispatch_k<LaunchBatchedMixed>(K, W, (total_tiles + 3) / 4, sessions, n_sessions,
                                       total_tiles, comp_of(params), status, s);
    else
        dispatch_k<LaunchBatched>(K, W, resident_grid<LaunchBatched>(K, W), 128, s, sessions,
                                  n_sessions, total_tiles, comp_of(params), work_counter, status);
    WRS_LAUNCH_CHECK(fn);
    return WRS_OK;
}

static int trace_backward_impl(const wrs_lbvh* bvh, const wrs_splats* sorted,
                               const wrs_camera* cam, const wrs_trace_params* params,
                               const float* radius_scale, float global_scale,
                               const float* dL_drgba, float* g_rgba, float* g_opacity,
                               float* g_scale, int32_t* status, wrs_stream_t stream, bool zero,
                               const char* fn) {
    if (int rc = check_trace_args(bvh, sorted, cam, params, fn)) return rc;
    if (!dL_drgba || !g_rgba ||
        ((reinterpret_cast<uintptr_t>(dL_drgba) | reinterpret_cast<uintptr_t>(g_rgba)) & 15))
        return wrs::fail(WRS_ERR_ARG, "%s: dL_drgba / g_rgba NULL or not 16-byte aligned", fn);
    const size_t cap = sorted->capacity;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (zero) {
        cudaError_t e = cudaMemsetAsync(g_rgba, 0, 4 * sizeof(float) * cap, s);
        if (e == cudaSuccess && g_opacity) e = cudaMemsetAsync(g_opacity, 0, sizeof(float) * cap, s);
        if (e == cudaSuccess && g_scale) e = cudaMemsetAsync(g_scale, 0, sizeof(float) * cap, s);
        if (e != cudaSuccess) return wrs::cuda_fail(e, fn);
    }
    const GradOut go = {radius_scale, global_scale, g_rgba, g_opacity, g_scale};
    const int K = effective_k(params), W = params->width;
    const Scene sc = make_scene(bvh, sorted, params->opacity, W);
    const float4* d4 = reinterpret_cast<const float4*>(dL_drgba);
    if (params->schedule == WRS_SCHEDULE_PERSISTENT) {
        dispatch_k<LaunchBwdPr>(K, W, resident_grid<LaunchBwdPr>(K, W), 128, s, sc,
                                comp_of(params), *cam, d4, go, status);
    } else if (params->schedule == WRS_SCHEDULE_PACKET) {
        dispatch_k1<LaunchBwdPacket, true>(K, grid_for(cam, params->block), params->block, s,
                                           make_scene(bvh, sorted, params->opacity, 4),
                                           comp_of(params), *cam, d4, go, status);
    } else {
        const int block = params->block > 128 ? 128 : params->block;  // keep occupancy
        dispatch_k<LaunchBwd>(K, W, grid_for(cam, block), block, s, sc, comp_of(params), *cam, d4,
                              go, status);
    }
    WRS_LAUNCH_CHECK(fn);
    return WRS_OK;
}

int wrs_trace_backward(const wrs_lbvh* bvh, const wrs_splats* sorted, const wrs_camera* cam,
                       const wrs_trace_params* params, const float* radius_scale,
                       float global_scale, const float* dL_drgba, float* g_rgba,
                       float* g_opacity, float* g_scale, int32_t* status, wrs_stream_t stream) {
    return trace_backward_impl(bvh, sorted, cam, params, radius_scale, global_scale, dL_drgba,
                               g_rgba, g_opacity, g_scale, status, stream, true,
                               "wrs_trace_backward");
}

int wrs_trace_backward_accumulate(const wrs_lbvh* bvh, const wrs_splats* sorted,
                                  const wrs_camera* cam, const wrs_trace_params* params,
                                  const float* radius_scale, float global_scale,
                                  const float* dL_drgba, float* g_rgba, float* g_opacity,
                                  float* g_scale, int32_t* status, wrs_stream_t stream) {
    return trace_backward_impl(bvh, sorted, cam, params, radius_scale, global_scale, dL_drgba,
                               g_rgba, g_opacity, g_scale, status, stream, false,
                               "wrs_trace_backward_accumulate");
}

}  // extern "C"

namespace {
// wrs_trace_backward_views; with filter.count, only the rays whose recorded list is over capacity.
int backward_views_impl(const wrs_lbvh* bvh, const wrs_splats* sorted, const wrs_camera* cams,
                        int32_t n_views, const wrs_trace_params* params, const float* radius_scale,
                        float global_scale, const float* dL_drgba, float* g_rgba,
                        float* g_opacity, float* g_scale, int32_t accumulate, HitFilter filter,
                        int32_t* status, wrs_stream_t stream, const char* fn) {
    if (int rc = check_views(bvh, sorted, cams, n_views, params, fn)) return rc;
    if (!dL_drgba || !g_rgba ||
        ((reinterpret_cast<uintptr_t>(dL_drgba) | reinterpret_cast<uintptr_t>(g_rgba)) & 15))
        return wrs::fail(WRS_ERR_ARG, "%s: dL_drgba / g_rgba NULL or not 16-byte aligned", fn);
    const size_t cap = sorted->capacity;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (!accumulate) {
        cudaError_t e = cudaMemsetAsync(g_rgba, 0, 4 * sizeof(float) * cap, s);
        if (e == cudaSuccess && g_opacity) e = cudaMemsetAsync(g_opacity, 0, sizeof(float) * cap, s);
        if (e == cudaSuccess && g_scale) e = cudaMemsetAsync(g_scale, 0, sizeof(float) * cap, s);
        if (e != cudaSuccess) return wrs::cuda_fail(e, fn);
    }
    const GradOut go = {radius_scale, global_scale, g_rgba, g_opacity, g_scale};
    const int K = effective_k(params), W = params->width;
    const Scene sc = make_scene(bvh, sorted, params->opacity, W);
    const size_t pixels = (size_t)cams[0].width * cams[0].height;
    const bool packet = params->schedule == WRS_SCHEDULE_PACKET;
    // per pixel as wrs_trace_backward (128-thread blocks at most); the packet backward as given
    const int block = packet ? params->block : (params->block > 128 ? 128 : params->block);
    const Scene scp = make_scene(bvh, sorted, params->opacity, 4);
    for (int v0 = 0; v0 < n_views; v0 += kMaxViews) {
        const int nv = n_views - v0 < kMaxViews ? n_views - v0 : kMaxViews;
        ViewCams vc;
        for (int v = 0; v < nv; v++) vc.cam[v] = cams[v0 + v];
        dim3 g = grid_for(&cams[0], block);
        g.z = (unsigned)nv;
        const float4* d = reinterpret_cast<const float4*>(dL_drgba) + (size_t)v0 * pixels;
        if (packet)
            dispatch_k1<LaunchBwdPacketViews, true>(K, g, block, s, scp, comp_of(params), vc, d,
                                                    pixels, go, filter, (size_t)v0 * pixels,
                                                    status);
        else
            dispatch_k<LaunchBwdViews>(K, W, g, block, s, sc, comp_of(params), vc, d, pixels, go,
                                       filter, (size_t)v0 * pixels, status);
        WRS_LAUNCH_CHECK(fn);
    }
    return WRS_OK;
}
}  // namespace

extern "C" {

int wrs_trace_backward_views(const wrs_lbvh* bvh, const wrs_splats* sorted,
                             const wrs_camera* cams, int32_t n_views,
                             const wrs_trace_params* params, const float* radius_scale,
                             float global_scale, const float* dL_drgba, float* g_rgba,
                             float* g_opacity, float* g_scale, int32_t accumulate,
                             int32_t* status, wrs_stream_t stream) {
    return backward_views_impl(bvh, sorted, cams, n_views, params, radius_scale, global_scale,
                               dL_drgba, g_rgba, g_opacity, g_scale, accumulate,
                               HitFilter{nullptr, 0}, status, stream, "wrs_trace_backward_views");
}

int wrs_trace_backward_views_recorded(const wrs_lbvh* bvh, const wrs_splats* sorted,
                                      const wrs_camera* cams, int32_t n_views,
                                      const wrs_trace_params* params, const float* radius_scale,
                                      float global_scale, const uint32_t* hits,
                                      const uint32_t* hit_count, uint32_t hit_capacity,
                                      const float* dL_drgba, float* g_rgba, float* g_opacity,
                                      float* g_scale, int32_t accumulate, int32_t* status,
                                      wrs_stream_t stream) {
    const char* fn = "wrs_trace_backward_views_recorded";
    if (int rc = check_record(hits, hit_count, hit_capacity, fn)) return rc;
    // the rays whose list went over capacity: re-traversed (this also zeroes the gradients and
    // checks every argument)
    const HitFilter over = {hit_count, hit_capacity};
    if (int rc = backward_views_impl(bvh, sorted, cams, n_views, params, radius_scale,
                                     global_scale, dL_drgba, g_rgba, g_opacity, g_scale,
                                     accumulate, over, status, stream, fn))
        return rc;
    // the others from their lists
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const GradOut go = {radius_scale, global_scale, g_rgba, g_opacity, g_scale};
    const Scene sc = make_scene(bvh, sorted, params->opacity, 2);
    const size_t pixels = (size_t)cams[0].width * cams[0].height;
    for (int v0 = 0; v0 < n_views; v0 += kMaxViews) {
        const int nv = n_views - v0 < kMaxViews ? n_views - v0 : kMaxViews;
        ViewCams vc;
        for (int v = 0; v < nv; v++) vc.cam[v] = cams[v0 + v];
        dim3 g = grid_for(&cams[0], 128);
        g.z = (unsigned)nv;
        const float4* d = reinterpret_cast<const float4*>(dL_drgba) + (size_t)v0 * pixels;
        k_trace_bwd_recorded<<<g, 128, 0, s>>>(sc, comp_of(params), vc, d, pixels, go, hits,
                                               hit_count, hit_capacity, (size_t)v0 * pixels);
        WRS_LAUNCH_CHECK(fn);
    }
    return WRS_OK;
}

}  // extern "C"
