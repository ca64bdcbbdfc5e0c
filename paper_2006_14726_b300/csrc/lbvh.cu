// lbvh.cu -- LBVH over the sphere splats (§4.1, §4.2: the LBVH of Lauterbach et al. 2009 as used
// by Zellmann et al. 2019; spec S8).
//
//   k_bounds_partial / k_bounds_final : centre bounds and the largest radius (two-level reduction)
//   k_morton                          : 30-bit Morton code of each centre (binary32 quantisation)
//                                       and the per-tile counts of the first radix digit
//   k_rs_hist (x3) / k_rs_scan / k_rs_scatter (x4) : stable LSD radix sort of (code, index), 8-bit
//                                       digits (the first digit's counts come from k_morton)
//   k_karras                          : binary radix tree over leaf keys (Karras 2012); also
//                                       zeroes the refit's arrival counters
//   k_leaves_refit                    : gathers the splats into leaf order with their effective
//                                       radius, computes leaf boxes and refits the internal nodes
//                                       bottom-up (second thread to reach a node continues); the
//                                       same climb fills the 4-wide nodes
//
// Layout WRS_LBVH_WIDE (a tree for the 4-wide traversal only): k_karras writes no child
// references and the refit no binary record of a node inside one refit block; the records of
// the nodes that span blocks still carry the boxes between blocks.  The 4-wide nodes are the
// same, bitwise.
//
// The splat count is read on the device from the header, so the whole build runs without a host
// synchronisation and can be captured into a CUDA graph.  No kernel waits on another block.
#include "common.cuh"

namespace {

using wrs::LbvhHeader;
using wrs::kLeafBit;

constexpr int kBoundsBlocks = 512;
constexpr int kSortThreads = 256;
#ifndef WRS_SORT_ITEMS
#define WRS_SORT_ITEMS 8
#endif
// keys per thread in a sort tile: 8 and 12 measured fastest on the 2 M-splat build (4: 2 %, 16:
// 3 % slower); a build-time knob
constexpr int kSortItems = WRS_SORT_ITEMS;
constexpr int kSortTile = kSortThreads * kSortItems;  // keys per sort tile
constexpr int kSortWarps = kSortThreads / 32;

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

struct Scratch {
    uint32_t *keys0, *keys1, *vals0, *vals1, *hist, *totals, *leaf_parent, *node_parent, *visit;
    uint4* node_range;  // leaf range [lo, hi] and split of each internal node
    float* partials;
    uint32_t tiles;
};

uint32_t leaves_for(uint32_t cap, uint32_t leaf) { return cap == 0 ? 1 : (cap + leaf - 1) / leaf; }

size_t scratch_layout(uint32_t cap, uint32_t leaf, char* base, Scratch* s) {
    const uint32_t tiles = (cap + kSortTile - 1) / kSortTile;
    const uint32_t m = leaves_for(cap, leaf);
    size_t off = 0;
    auto take = [&](size_t bytes) {
        char* p = base ? base + off : nullptr;
        off += align256(bytes);
        return p;
    };
    char* k0 = take(sizeof(uint32_t) * cap);
    char* k1 = take(sizeof(uint32_t) * cap);
    char* v0 = take(sizeof(uint32_t) * cap);
    char* v1 = take(sizeof(uint32_t) * cap);
    char* h = take(sizeof(uint32_t) * 256 * (size_t)(tiles ? tiles : 1));
    char* tt = take(sizeof(uint32_t) * 256);
    char* lp = take(sizeof(uint32_t) * m);
    char* np = take(sizeof(uint32_t) * m);
    char* vi = take(sizeof(uint32_t) * m);
    char* nr = take(sizeof(uint4) * m);
    char* pa = take(sizeof(float) * 8 * kBoundsBlocks);
    if (s) {
        s->keys0 = (uint32_t*)k0; s->keys1 = (uint32_t*)k1;
        s->vals0 = (uint32_t*)v0; s->vals1 = (uint32_t*)v1;
        s->hist = (uint32_t*)h; s->totals = (uint32_t*)tt; s->leaf_parent = (uint32_t*)lp; s->node_parent = (uint32_t*)np;
        s->visit = (uint32_t*)vi; s->node_range = (uint4*)nr; s->partials = (float*)pa; s->tiles = tiles;
    }
    return off;
}

__device__ __forceinline__ float eff_radius(const float* __restrict__ scale, float gscale,
                                            uint32_t i, float r0) {
    float s = scale ? __ldg(scale + i) : gscale;
    s = s > 0.0f ? s : 0.0f;  // also maps NaN to 0
    return __fmul_rn(s, r0);
}

// ---- bounds --------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_bounds_partial(const float4* __restrict__ pos_r,
                                                        const float* __restrict__ scale,
                                                        float gscale, const uint32_t* __restrict__ n_in,
                                                        uint32_t cap, float* __restrict__ partials) {
    const uint32_t n = min(*n_in, cap);
    float v[7] = {INFINITY, INFINITY, INFINITY, -INFINITY, -INFINITY, -INFINITY, 0.0f};
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float4 p = pos_r[i];
        v[0] = fminf(v[0], p.x); v[1] = fminf(v[1], p.y); v[2] = fminf(v[2], p.z);
        v[3] = fmaxf(v[3], p.x); v[4] = fmaxf(v[4], p.y); v[5] = fmaxf(v[5], p.z);
        v[6] = fmaxf(v[6], eff_radius(scale, gscale, i, p.w));
    }
    __shared__ float s[7][8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 7; k++) {
        float x = v[k];
        for (int o = 16; o > 0; o >>= 1) {
            const float y = __shfl_xor_sync(0xffffffffu, x, o);
            x = (k < 3) ? fminf(x, y) : fmaxf(x, y);
        }
        if (lane == 0) s[k][warp] = x;
    }
    __syncthreads();
    if (threadIdx.x < 7) {
        const int k = threadIdx.x;
        float x = s[k][0];
        for (int w = 1; w < 8; w++) x = (k < 3) ? fminf(x, s[k][w]) : fmaxf(x, s[k][w]);
        partials[blockIdx.x * 8 + k] = x;
    }
}

__global__ void __launch_bounds__(kBoundsBlocks) k_bounds_final(
    const float* __restrict__ partials, const uint32_t* __restrict__ n_in, uint32_t cap,
    uint32_t leaf, uint32_t layout, LbvhHeader* __restrict__ hdr, uint32_t* __restrict__ n_sorted) {
    __shared__ float s[7][kBoundsBlocks / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int b = threadIdx.x;  // one partial per thread
#pragma unroll
    for (int k = 0; k < 7; k++) {
        float x = partials[b * 8 + k];
        for (int o = 16; o > 0; o >>= 1) {
            const float y = __shfl_xor_sync(0xffffffffu, x, o);
            x = (k < 3) ? fminf(x, y) : fmaxf(x, y);
        }
        if (lane == 0) s[k][warp] = x;
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    float v[7];
    for (int k = 0; k < 7; k++) {
        float x = s[k][0];
        for (int w = 1; w < kBoundsBlocks / 32; w++) x = (k < 3) ? fminf(x, s[k][w]) : fmaxf(x, s[k][w]);
        v[k] = x;
    }
    const uint32_t n = min(*n_in, cap);  // a count beyond the capacity is clamped
    LbvhHeader h = {};
    h.n = n;
    h.leaf = leaf;
    h.layout = layout;
    h.wide_start = wrs::lbvh_binary_slots(cap, leaf);
    h.m = n == 0 ? 0 : (n + leaf - 1) / leaf;
    h.root = h.m <= 1 ? (int32_t)kLeafBit : 0;
    float mx = 0.0f;
    for (int k = 0; k < 3; k++) {
        h.cmin[k] = n ? v[k] : 0.0f;
        h.cmax[k] = n ? v[3 + k] : 0.0f;
        mx = fmaxf(mx, fmaxf(fabsf(h.cmin[k]), fabsf(h.cmax[k])));
    }
    h.rmax = v[6];
    h.maxabs = mx + v[6];
    *hdr = h;
    *n_sorted = n;
}

// ---- Morton codes (spec S8) ----------------------------------------------------------------
__device__ __forceinline__ uint32_t spread10(uint32_t v) {
    v = (v * 0x00010001u) & 0xFF0000FFu;
    v = (v * 0x00000101u) & 0x0F00F00Fu;
    v = (v * 0x00000011u) & 0xC30C30C3u;
    v = (v * 0x00000005u) & 0x49249249u;
    return v;
}

__device__ __forceinline__ uint32_t morton_code(const float4 p, const LbvhHeader* __restrict__ hdr) {
    const float c[3] = {p.x, p.y, p.z};
    uint32_t q[3];
#pragma unroll
    for (int k = 0; k < 3; k++) {
        const float ext = __fsub_rn(hdr->cmax[k], hdr->cmin[k]);
        const float sc = ext > 0.0f ? __fdiv_rn(1024.0f, ext) : 0.0f;
        const float v = floorf(__fmul_rn(__fsub_rn(c[k], hdr->cmin[k]), sc));
        q[k] = v >= 1023.0f ? 1023u : (uint32_t)v;
    }
    return (spread10(q[0]) << 2) | (spread10(q[1]) << 1) | spread10(q[2]);
}

// One sort tile per block (kSortTile splats, the sort's item layout): the codes and indices, and
// the tile's counts of the first radix digit (bits 0..7), so the first sort pass needs no
// histogram kernel.  hist is digit-major: hist[d * tiles + tile].
__global__ void __launch_bounds__(kSortThreads) k_morton(const float4* __restrict__ pos_r,
                                                         const LbvhHeader* __restrict__ hdr,
                                                         uint32_t* __restrict__ keys,
                                                         uint32_t* __restrict__ vals,
                                                         uint32_t tiles, uint32_t* __restrict__ hist) {
    __shared__ uint32_t s_cnt[kSortThreads / 32][256];  // one digit histogram per warp
    for (int w = 0; w < kSortThreads / 32; w++) s_cnt[w][threadIdx.x] = 0;
    const uint32_t n = hdr->n;
    const uint32_t base = blockIdx.x * kSortTile;
    const int warp = threadIdx.x >> 5;
    uint32_t code[kSortItems];
#pragma unroll
    for (int k = 0; k < kSortItems; k++) {
        const uint32_t i = base + k * kSortThreads + threadIdx.x;
        code[k] = 0xFFFFFFFFu;
        if (i < n) {
            code[k] = morton_code(pos_r[i], hdr);
            keys[i] = code[k];
            vals[i] = i;
        }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kSortItems; k++)
        if (code[k] != 0xFFFFFFFFu) atomicAdd(&s_cnt[warp][code[k] & 255u], 1u);
    __syncthreads();
    uint32_t c = 0;
    for (int w = 0; w < kSortThreads / 32; w++) c += s_cnt[w][threadIdx.x];
    hist[threadIdx.x * tiles + blockIdx.x] = c;
}

// ---- stable LSD radix sort, 8-bit digits ---------------------------------------------------
// Histogram layout is digit-major: hist[d * tiles + tile], so one exclusive scan over the whole
// array yields each (digit, tile) pair's first output position.
__global__ void __launch_bounds__(kSortThreads) k_rs_hist(const uint32_t* __restrict__ keys,
                                                          const LbvhHeader* __restrict__ hdr,
                                                          int shift, uint32_t tiles,
                                                          uint32_t* __restrict__ hist) {
    __shared__ uint32_t s_cnt[kSortWarps][256];  // one histogram per warp: fewer collisions
    for (int w = 0; w < kSortWarps; w++) s_cnt[w][threadIdx.x] = 0;
    const uint32_t n = hdr->n;
    const uint32_t base = blockIdx.x * kSortTile;
    const int warp = threadIdx.x >> 5;
    uint32_t d[kSortItems];
#pragma unroll
    for (int k = 0; k < kSortItems; k++) {  // all loads in flight before the counting
        const uint32_t i = base + k * kSortThreads + threadIdx.x;
        d[k] = i < n ? (keys[i] >> shift) & 255u : 256u;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kSortItems; k++)
        if (d[k] < 256u) atomicAdd(&s_cnt[warp][d[k]], 1u);
    __syncthreads();
    uint32_t c = 0;
    for (int w = 0; w < kSortWarps; w++) c += s_cnt[w][threadIdx.x];
    hist[threadIdx.x * tiles + blockIdx.x] = c;
}

// One block per digit: exclusive scan of that digit's per-tile counts (contiguous in the
// digit-major layout) in place, and the digit's total.  The scatter adds the digit bases.
__global__ void __launch_bounds__(256) k_rs_scan(uint32_t* __restrict__ hist, uint32_t tiles,
                                                 uint32_t* __restrict__ totals) {
    __shared__ uint32_t s_warp[8];
    __shared__ uint32_t s_carry;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t* h = hist + (size_t)blockIdx.x * tiles;
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    for (uint32_t base = 0; base < tiles; base += 4 * 256) {
        uint32_t v[4], sum = 0;
#pragma unroll
        for (int k = 0; k < 4; k++) {  // 4 consecutive tiles per thread
            const uint32_t i = base + threadIdx.x * 4 + k;
            v[k] = i < tiles ? h[i] : 0u;
            sum += v[k];
        }
        uint32_t inc = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
        }
        if (lane == 31) s_warp[warp] = inc;
        __syncthreads();
        uint32_t wpre = 0, btot = 0;
        for (int w = 0; w < 8; w++) {
            wpre += (w < warp) ? s_warp[w] : 0u;
            btot += s_warp[w];
        }
        uint32_t run = s_carry + wpre + inc - sum;
#pragma unroll
        for (int k = 0; k < 4; k++) {
            const uint32_t i = base + threadIdx.x * 4 + k;
            if (i < tiles) h[i] = run;
            run += v[k];
        }
        __syncthreads();
        if (threadIdx.x == 0) s_carry += btot;
        __syncthreads();
    }
    if (threadIdx.x == 0) totals[blockIdx.x] = s_carry;
}

// Rank every key of the tile stably by digit (warp match + per-warp digit counters), stage the
// tile in shared memory in digit order, then write each digit run to its global position.
__global__ void __launch_bounds__(kSortThreads) k_rs_scatter(
    const uint32_t* __restrict__ keys_in, const uint32_t* __restrict__ vals_in,
    uint32_t* __restrict__ keys_out, uint32_t* __restrict__ vals_out,
    const uint32_t* __restrict__ offsets, const uint32_t* __restrict__ totals,
    const LbvhHeader* __restrict__ hdr, int shift, uint32_t tiles) {
    __shared__ uint32_t s_wcnt[kSortWarps][256];
    __shared__ uint32_t s_start[256];
    __shared__ uint32_t s_glob[256];
    __shared__ uint32_t s_base[256];
    __shared__ uint32_t s_keys[kSortTile];
    __shared__ uint32_t s_vals[kSortTile];
    const uint32_t n = hdr->n;
    const uint32_t base = blockIdx.x * kSortTile;
    if (base >= n) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int d = lane; d < 256; d += 32) s_wcnt[warp][d] = 0;
    __syncwarp();

    uint32_t key[kSortItems], val[kSortItems], rank[kSortItems];
    const uint32_t wbase = base + warp * 32 * kSortItems;
#pragma unroll
    for (int k = 0; k < kSortItems; k++) {
        const uint32_t i = wbase + k * 32 + lane;
        const bool valid = i < n;
        key[k] = valid ? keys_in[i] : 0u;
        val[k] = valid ? vals_in[i] : 0u;
        const uint32_t d = (key[k] >> shift) & 255u;
        const uint32_t label = valid ? d : (256u + lane);  // invalid lanes match nobody
        const uint32_t peers = __match_any_sync(0xffffffffu, label);
        const uint32_t before = __popc(peers & ((1u << lane) - 1u));
        const uint32_t prev = valid ? s_wcnt[warp][d] : 0u;
        __syncwarp();
        if (valid && before == 0) s_wcnt[warp][d] = prev + __popc(peers);
        __syncwarp();
        rank[k] = valid ? prev + before : 0xFFFFFFFFu;
    }
    __syncthreads();
    // per digit: exclusive prefix over warps, then exclusive scan over digits (local starts)
    {
        const int d = threadIdx.x;  // kSortThreads == 256 digits
        uint32_t run = 0;
        for (int w = 0; w < kSortWarps; w++) {
            const uint32_t c = s_wcnt[w][d];
            s_wcnt[w][d] = run;
            run += c;
        }
        s_start[d] = run;  // digit total within the tile, scanned below
        s_glob[d] = offsets[(size_t)d * tiles + blockIdx.x];
        s_base[d] = totals[d];  // digit total over all tiles, scanned below
    }
    __syncthreads();
    if (warp < 2) {  // exclusive scans of the 256 tile totals (warp 0) and global totals (warp 1)
        uint32_t* arr = warp == 0 ? s_start : s_base;
        uint32_t t[8], sum = 0;
#pragma unroll
        for (int j = 0; j < 8; j++) { t[j] = arr[lane * 8 + j]; sum += t[j]; }
        uint32_t inc = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
        }
        uint32_t run = inc - sum;
#pragma unroll
        for (int j = 0; j < 8; j++) { const uint32_t c = t[j]; arr[lane * 8 + j] = run; run += c; }
    }
    __syncthreads();
    s_glob[threadIdx.x] += s_base[threadIdx.x];
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kSortItems; k++) {
        if (rank[k] == 0xFFFFFFFFu) continue;
        const uint32_t d = (key[k] >> shift) & 255u;
        const uint32_t pos = s_start[d] + s_wcnt[warp][d] + rank[k];
        s_keys[pos] = key[k];
        s_vals[pos] = val[k];
    }
    __syncthreads();
    const uint32_t cnt = min((uint32_t)kSortTile, n - base);
    for (uint32_t j = threadIdx.x; j < cnt; j += kSortThreads) {
        const uint32_t kk = s_keys[j];
        const uint32_t d = (kk >> shift) & 255u;
        const uint32_t dst = s_glob[d] + (j - s_start[d]);
        keys_out[dst] = kk;
        vals_out[dst] = s_vals[j];
    }
}

// ---- Karras 2012 binary radix tree over the leaf keys --------------------------------------
// Common prefix length of leaf keys i and j (a = key i, read once by the caller), index
// tie-break for equal keys; -1 outside the leaves.
__device__ __forceinline__ int delta(const uint32_t* __restrict__ codes, uint32_t leaf, int m,
                                     int i, uint32_t a, int j) {
    if (j < 0 || j >= m) return -1;
    const uint32_t b = __ldg(codes + (size_t)j * leaf);
    if (a != b) return __clz(a ^ b);
    return 32 + __clz((uint32_t)i ^ (uint32_t)j);
}

__global__ void __launch_bounds__(256) k_karras(const uint32_t* __restrict__ codes,
                                                const LbvhHeader* __restrict__ hdr,
                                                float4* __restrict__ nodes, bool binary,
                                                uint32_t* __restrict__ leaf_parent,
                                                uint32_t* __restrict__ node_parent,
                                                uint4* __restrict__ node_range,
                                                uint32_t* __restrict__ visit) {
    const int m = (int)hdr->m;
    const uint32_t leaf = hdr->leaf;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m - 1) return;
    visit[i] = 0u;  // the refit's arrival counter of internal node i
    const uint32_t a = __ldg(codes + (size_t)i * leaf);
    const int d = (delta(codes, leaf, m, i, a, i + 1) - delta(codes, leaf, m, i, a, i - 1)) >= 0 ? 1 : -1;
    const int dmin = delta(codes, leaf, m, i, a, i - d);
    int lmax = 2;
    while (delta(codes, leaf, m, i, a, i + lmax * d) > dmin) lmax <<= 1;
    int l = 0;
    for (int t = lmax >> 1; t >= 1; t >>= 1)
        if (delta(codes, leaf, m, i, a, i + (l + t) * d) > dmin) l += t;
    const int j = i + l * d;
    const int dnode = delta(codes, leaf, m, i, a, j);
    int s = 0, t = l;
    do {
        t = (t + 1) >> 1;
        if (s + t < l && delta(codes, leaf, m, i, a, i + (s + t) * d) > dnode) s += t;
    } while (t > 1);
    const int g = i + s * d + min(d, 0);
    const int lo = min(i, j), hi = max(i, j);
    if (binary) {  // the record's child references (its boxes come from the refit)
        const uint32_t left = (lo == g) ? (kLeafBit | (uint32_t)g) : (uint32_t)g;
        const uint32_t right = (hi == g + 1) ? (kLeafBit | (uint32_t)(g + 1)) : (uint32_t)(g + 1);
        nodes[4 * i + 3] = make_float4(__uint_as_float(left), __uint_as_float(right), 0.0f, 0.0f);
    }
    node_range[i] = make_uint4((uint32_t)lo, (uint32_t)hi, (uint32_t)g, 0u);
    if (lo == g) leaf_parent[g] = (uint32_t)i << 1;
    else node_parent[g] = (uint32_t)i << 1;
    if (hi == g + 1) leaf_parent[g + 1] = ((uint32_t)i << 1) | 1u;
    else node_parent[g + 1] = ((uint32_t)i << 1) | 1u;
}

// ---- leaf gather + bottom-up refit ---------------------------------------------------------
// Message passing between the two children of a node: the first child to finish stores its box,
// then increments the node's counter with release semantics; the second child's increment (with
// acquire semantics) observes it and reads both boxes.  Each block owns kRefitBlock consecutive
// leaves.  A node whose leaf range lies inside the block is finished inside the block: its counter
// and child boxes live in shared memory and the ordering is block-scope (cheap).  Only nodes whose
// range spans blocks use global counters with device-scope ordering -- a few per block boundary
// instead of one per node.  128 leaves per block measured fastest on the 2 M-splat build (64 and
// 512: 3-5 % slower, 256: 1.6 % slower); a build-time knob.
#ifndef WRS_REFIT_BLOCK
#define WRS_REFIT_BLOCK 128
#endif
constexpr uint32_t kRefitBlock = WRS_REFIT_BLOCK;

// Counter increments with acquire-release semantics on the atomic itself (one ordered operation
// instead of a fence on each side of a relaxed atomic): the release publishes this child's box,
// the acquire makes the sibling's box visible to the second arrival.
__device__ __forceinline__ uint32_t add_acq_rel_gpu(uint32_t* p) {
    uint32_t old;
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], 1;" : "=r"(old) : "l"(p) : "memory");
    return old;
}
__device__ __forceinline__ uint32_t add_acq_rel_cta_shared(uint32_t* p) {
    uint32_t old;
    const uint32_t a = static_cast<uint32_t>(__cvta_generic_to_shared(p));
    asm volatile("atom.acq_rel.cta.shared::cta.add.u32 %0, [%1], 1;" : "=r"(old) : "r"(a) : "memory");
    return old;
}

// Child box `slot` of binary node `node` (floats 6 slot .. 6 slot + 5 of its 64-byte record) in
// two vector stores: slot 0 = 16 + 8 bytes, slot 1 = 8 + 16 bytes (all naturally aligned).
__device__ __forceinline__ void store_box(float4* nodes, uint32_t node, uint32_t slot,
                                          const float lo[3], const float hi[3]) {
    float* f = reinterpret_cast<float*>(nodes + 4 * (size_t)node);
    if (slot == 0) {
        __stcg(reinterpret_cast<float4*>(f), make_float4(lo[0], lo[1], lo[2], hi[0]));
        __stcg(reinterpret_cast<float2*>(f + 4), make_float2(hi[1], hi[2]));
    } else {
        __stcg(reinterpret_cast<float2*>(f + 6), make_float2(lo[0], lo[1]));
        __stcg(reinterpret_cast<float4*>(f + 8), make_float4(lo[2], hi[0], hi[1], hi[2]));
    }
}

// ---- 4-wide nodes ---------------------------------------------------------------------------
// 4-wide node i lists the grandchildren of binary node i in structure-of-arrays order (float4 q of
// the node holds plane q -- low x, y, z, high x, y, z -- of all four entries; float4 6 holds the
// four references), so that a traversal step loads one coordinate of all four boxes per float4.
// Fixed slots: child c's children go to slots 2c and 2c + 1; a leaf child stands for itself in
// slot 2c and slot 2c + 1 is unused: low x = +inf and high x = -inf (whatever its other planes
// hold, no ray enters it: its x slab is empty) and the reference kNoChild.  The refit fills them
// when a node is finished (by the thread that arrives second): the node's two children as a pair
// of slots of its parent's 4-wide node, a leaf child also as itself in the node's own 4-wide node
// (both slots of a node over two leaves at once).  These are vector stores off the loads of the
// climb.

// Slots 2c and 2c + 1 of 4-wide node i: the boxes b[0..5], b[6..11] with references r0, r1, one
// 8-byte store per plane (the two slots are adjacent in every plane's float4).
__device__ __forceinline__ void write_pair(float4* __restrict__ wide, uint32_t i, uint32_t c,
                                           const float* b, uint32_t r0, uint32_t r1) {
    float* w = reinterpret_cast<float*>(wide + 8 * (size_t)i) + 2 * c;
#pragma unroll
    for (int q = 0; q < 6; q++) *reinterpret_cast<float2*>(w + 4 * q) = make_float2(b[q], b[6 + q]);
    *reinterpret_cast<float2*>(w + 24) = make_float2(__uint_as_float(r0), __uint_as_float(r1));
    *reinterpret_cast<float2*>(w + 28) = make_float2(0.0f, 0.0f);
}

// Slots 2c and 2c + 1 of 4-wide node i for a leaf child c: the leaf (box b[0..5], reference r)
// stands for itself, the slot after it is unused (empty x slab, no reference).
__device__ __forceinline__ void write_leaf_pair(float4* __restrict__ wide, uint32_t i, uint32_t c,
                                                const float* b, uint32_t r) {
    float* w = reinterpret_cast<float*>(wide + 8 * (size_t)i) + 2 * c;
#pragma unroll
    for (int q = 0; q < 6; q++)
        *reinterpret_cast<float2*>(w + 4 * q) =
            make_float2(b[q], q == 0 ? INFINITY : (q == 3 ? -INFINITY : 0.0f));
    *reinterpret_cast<float2*>(w + 24) = make_float2(__uint_as_float(r), __uint_as_float(wrs::kNoChild));
    *reinterpret_cast<float2*>(w + 28) = make_float2(0.0f, 0.0f);
}

// The whole 4-wide node of a binary node whose two children are the leaves l0 (slot 0) and l1
// (slot 1), from their boxes a[0..5] and a[6..11], in seven 16-byte stores: the leaves stand for
// themselves in slots 0 and 2, slots 1 and 3 are unused (empty x slab, no reference).
__device__ __forceinline__ void write_cherry(float4* __restrict__ wide, uint32_t i,
                                             const float (&a)[12], uint32_t l0, uint32_t l1) {
    float4* w = wide + 8 * (size_t)i;
    w[0] = make_float4(a[0], INFINITY, a[6], INFINITY);
    w[1] = make_float4(a[1], 0.0f, a[7], 0.0f);
    w[2] = make_float4(a[2], 0.0f, a[8], 0.0f);
    w[3] = make_float4(a[3], -INFINITY, a[9], -INFINITY);
    w[4] = make_float4(a[4], 0.0f, a[10], 0.0f);
    w[5] = make_float4(a[5], 0.0f, a[11], 0.0f);
    w[6] = make_float4(__uint_as_float(kLeafBit | l0), __uint_as_float(wrs::kNoChild),
                       __uint_as_float(kLeafBit | l1), __uint_as_float(wrs::kNoChild));
    w[7] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
}

__global__ void __launch_bounds__(kRefitBlock) k_leaves_refit(
    const uint32_t* __restrict__ order, const float4* __restrict__ pos_r,
    const float4* __restrict__ rgba, const uint32_t* __restrict__ id,
    const float* __restrict__ scale, float gscale, const LbvhHeader* __restrict__ hdr,
    float4* __restrict__ nodes, bool binary, const uint32_t* __restrict__ leaf_parent,
    const uint32_t* __restrict__ node_parent, const uint4* __restrict__ node_range,
    uint32_t* __restrict__ visit, float4* __restrict__ s_pos, float4* __restrict__ s_rgba,
    uint32_t* __restrict__ s_id, uint32_t* __restrict__ s_src, float4* __restrict__ wide) {
    __shared__ uint32_t sh_cnt[kRefitBlock];
    __shared__ float sh_box[kRefitBlock][12];  // child boxes of local internal node j0 + t
    const uint32_t n = hdr->n, m = hdr->m, leaf = hdr->leaf;
    const uint32_t j0 = blockIdx.x * kRefitBlock;
    sh_cnt[threadIdx.x] = 0;
    __syncthreads();
    const uint32_t j = j0 + threadIdx.x;
    if (j >= m) return;
    const uint32_t j1 = min(j0 + kRefitBlock, m) - 1;  // last leaf of this block
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    const uint32_t first = j * leaf, last = min(first + leaf, n);
    for (uint32_t k = first; k < last; k++) {
        const uint32_t src = order[k];
        const float4 p = pos_r[src];
        const float r = eff_radius(scale, gscale, src, p.w);
        lo[0] = fminf(lo[0], __fsub_rd(p.x, r)); hi[0] = fmaxf(hi[0], __fadd_ru(p.x, r));
        lo[1] = fminf(lo[1], __fsub_rd(p.y, r)); hi[1] = fmaxf(hi[1], __fadd_ru(p.y, r));
        lo[2] = fminf(lo[2], __fsub_rd(p.z, r)); hi[2] = fmaxf(hi[2], __fadd_ru(p.z, r));
        s_pos[k] = make_float4(p.x, p.y, p.z, r);
        s_rgba[k] = rgba[src];
        s_id[k] = id[src];
        s_src[k] = src;
    }
    if (m < 2) return;
    uint32_t pp = leaf_parent[j];
    bool local = true;  // ancestors of a node that spans blocks span blocks too
    // a climb has fewer levels than the tree has leaves; the bound only matters if the links are
    // not those of this splat set (wrs_refit_lbvh with another build's scratch): it then ends
    for (uint32_t level = 0; level < m; level++) {
        const uint32_t node = pp >> 1, slot = pp & 1u;
        if (node + 1 >= m) return;  // never taken for a well-formed tree
        const uint32_t gp = node != 0 ? node_parent[node] : 0u;  // node's own link to its parent
        const uint4 rg = node_range[node];
        float a[12];
        if (local && rg.x >= j0 && rg.y <= j1 && node >= j0 && node <= j1) {
            float* sb = sh_box[node - j0] + 6 * slot;
            sb[0] = lo[0]; sb[1] = lo[1]; sb[2] = lo[2]; sb[3] = hi[0]; sb[4] = hi[1]; sb[5] = hi[2];
            if (add_acq_rel_cta_shared(&sh_cnt[node - j0]) == 0u) return;  // first child: done
#pragma unroll
            for (int k = 0; k < 12; k++) a[k] = sh_box[node - j0][k];
            // the node's binary record (both child boxes) in three 16-byte stores; the binary
            // traversal reads it after the kernel (not written for the 4-wide-only layout)
            if (binary) {
                float4* rec = nodes + 4 * (size_t)node;
                __stcg(rec + 0, make_float4(a[0], a[1], a[2], a[3]));
                __stcg(rec + 1, make_float4(a[4], a[5], a[6], a[7]));
                __stcg(rec + 2, make_float4(a[8], a[9], a[10], a[11]));
            }
        } else {
            // a node spanning blocks: each child's box goes to the record before the release, the
            // second child reads the other one from there
            store_box(nodes, node, slot, lo, hi);
            local = false;
            if (add_acq_rel_gpu(visit + node) == 0u) return;  // first child: done
            const float4* rec = nodes + 4 * (size_t)node;
#pragma unroll
            for (int q = 0; q < 3; q++) {
                const float4 v = __ldcg(rec + q);
                a[4 * q] = v.x; a[4 * q + 1] = v.y; a[4 * q + 2] = v.z; a[4 * q + 3] = v.w;
            }
        }
        // second child: both boxes are final.  The node's children enter the 4-wide nodes here:
        // as grandchildren of its parent (a pair of slots), and a leaf child also as itself in the
        // node's own 4-wide node; then the node's box goes to its parent
        const uint32_t g = rg.z;
        const bool leaf0 = rg.x == g, leaf1 = rg.y == g + 1;
        const uint32_t ref0 = leaf0 ? (kLeafBit | g) : g, ref1 = leaf1 ? (kLeafBit | (g + 1)) : g + 1;
        if (leaf0 && leaf1) write_cherry(wide, node, a, g, g + 1);
        else if (leaf0) write_leaf_pair(wide, node, 0, a, ref0);
        else if (leaf1) write_leaf_pair(wide, node, 1, a + 6, ref1);
        if (node != 0 && (gp >> 1) + 1 < m) write_pair(wide, gp >> 1, gp & 1u, a, ref0, ref1);
        lo[0] = fminf(a[0], a[6]); lo[1] = fminf(a[1], a[7]); lo[2] = fminf(a[2], a[8]);
        hi[0] = fmaxf(a[3], a[9]); hi[1] = fmaxf(a[4], a[10]); hi[2] = fmaxf(a[5], a[11]);
        if (node == 0) return;
        pp = gp;
    }
}

}  // namespace

extern "C" {

size_t wrs_lbvh_bytes(uint32_t capacity, uint32_t leaf_size) {
    if (leaf_size < 1 || leaf_size > (uint32_t)wrs::kMaxLeaf) return 0;
    const size_t slots = wrs::lbvh_binary_slots(capacity, leaf_size);
    return sizeof(LbvhHeader) + 64 * slots + 128 * slots;  // binary nodes, then 4-wide nodes
}

size_t wrs_lbvh_scratch_bytes(uint32_t capacity, uint32_t leaf_size) {
    if (leaf_size < 1 || leaf_size > (uint32_t)wrs::kMaxLeaf) return 0;
    return scratch_layout(capacity, leaf_size, nullptr, nullptr);
}

// Arguments of wrs_build_lbvh and wrs_refit_lbvh.
static int check_lbvh_args(const wrs_splats* in, const float* radius_scale, float global_scale,
                           const wrs_lbvh* bvh, const wrs_splats* sorted, const void* scratch,
                           size_t scratch_bytes, const char* fn) {
    if (!in || !bvh || !sorted) return wrs::fail(WRS_ERR_ARG, "%s: NULL struct", fn);
    if (!in->pos_r || !in->rgba || !in->id || !in->n)
        return wrs::fail(WRS_ERR_ARG, "%s: NULL input splat array", fn);
    if (!sorted->pos_r || !sorted->rgba || !sorted->id || !sorted->src || !sorted->n)
        return wrs::fail(WRS_ERR_ARG, "%s: NULL sorted splat array (src is required)", fn);
    if (!bvh->nodes) return wrs::fail(WRS_ERR_ARG, "%s: bvh->nodes is NULL", fn);
    if (bvh->layout != WRS_LBVH_FULL && bvh->layout != WRS_LBVH_WIDE)
        return wrs::fail(WRS_ERR_ARG, "%s: unknown tree layout %u", fn, bvh->layout);
    const uint32_t leaf = bvh->leaf_size;
    if (leaf < 1 || leaf > (uint32_t)wrs::kMaxLeaf)
        return wrs::fail(WRS_ERR_ARG, "%s: leaf_size %u not in 1..16", fn, leaf);
    if (bvh->capacity < in->capacity || sorted->capacity < in->capacity)
        return wrs::fail(WRS_ERR_CAPACITY, "%s: bvh/sorted capacity below input capacity %u", fn,
                         in->capacity);
    if (in->capacity >= 0x80000000u) return wrs::fail(WRS_ERR_ARG, "%s: capacity >= 2^31", fn);
    if ((reinterpret_cast<uintptr_t>(in->pos_r) | reinterpret_cast<uintptr_t>(in->rgba) |
         reinterpret_cast<uintptr_t>(sorted->pos_r) | reinterpret_cast<uintptr_t>(sorted->rgba) |
         reinterpret_cast<uintptr_t>(bvh->nodes)) & 15)
        return wrs::fail(WRS_ERR_ARG, "%s: float4 arrays and nodes must be 16-byte aligned", fn);
    if (!radius_scale && !(global_scale == global_scale))
        return wrs::fail(WRS_ERR_ARG, "%s: global_scale is NaN", fn);
    const size_t need = scratch_layout(in->capacity, leaf, nullptr, nullptr);
    if (!scratch || scratch_bytes < need)
        return wrs::fail(WRS_ERR_SCRATCH, "%s: scratch needs %zu bytes, got %zu", fn, need,
                         scratch_bytes);
    if (reinterpret_cast<uintptr_t>(scratch) & 255)
        return wrs::fail(WRS_ERR_ARG, "%s: scratch must be 256-byte aligned", fn);
    return WRS_OK;
}

int wrs_build_lbvh(const wrs_splats* in, const float* radius_scale, float global_scale,
                   const wrs_lbvh* bvh, wrs_splats* sorted, void* scratch, size_t scratch_bytes,
                   wrs_stream_t stream) {
    if (int rc = check_lbvh_args(in, radius_scale, global_scale, bvh, sorted, scratch,
                                 scratch_bytes, "wrs_build_lbvh"))
        return rc;
    const uint32_t leaf = bvh->leaf_size;
    const uint32_t cap = in->capacity;
    Scratch S;
    scratch_layout(cap, leaf, static_cast<char*>(scratch), &S);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    LbvhHeader* hdr = static_cast<LbvhHeader*>(bvh->nodes);
    float4* nodes = wrs::lbvh_nodes(bvh->nodes);
    const float4* pos4 = reinterpret_cast<const float4*>(in->pos_r);
    const uint32_t m_cap = leaves_for(cap, leaf);
    const uint32_t gm = (m_cap + 255) / 256;

    k_bounds_partial<<<kBoundsBlocks, 256, 0, s>>>(pos4, radius_scale, global_scale, in->n, cap,
                                                   S.partials);
    WRS_LAUNCH_CHECK("wrs_build_lbvh bounds");
    k_bounds_final<<<1, kBoundsBlocks, 0, s>>>(S.partials, in->n, cap, leaf, bvh->layout, hdr,
                                              sorted->n);
    WRS_LAUNCH_CHECK("wrs_build_lbvh bounds final");
    if (cap == 0) return WRS_OK;
    k_morton<<<S.tiles, kSortThreads, 0, s>>>(pos4, hdr, S.keys0, S.vals0, S.tiles, S.hist);
    WRS_LAUNCH_CHECK("wrs_build_lbvh morton");
    uint32_t *ki = S.keys0, *vi = S.vals0, *ko = S.keys1, *vo = S.vals1;
    for (int shift = 0; shift < 32; shift += 8) {
        if (shift > 0)  // the first digit was counted with the codes
            k_rs_hist<<<S.tiles, kSortThreads, 0, s>>>(ki, hdr, shift, S.tiles, S.hist);
        k_rs_scan<<<256, 256, 0, s>>>(S.hist, S.tiles, S.totals);
        k_rs_scatter<<<S.tiles, kSortThreads, 0, s>>>(ki, vi, ko, vo, S.hist, S.totals, hdr, shift,
                                                      S.tiles);
        WRS_LAUNCH_CHECK("wrs_build_lbvh radix sort");
        uint32_t* t = ki; ki = ko; ko = t;
        t = vi; vi = vo; vo = t;
    }
    // four passes: the sorted keys / values are back in keys0 / vals0
    k_karras<<<gm, 256, 0, s>>>(ki, hdr, nodes, bvh->layout == WRS_LBVH_FULL, S.leaf_parent,
                                S.node_parent, S.node_range, S.visit);
    WRS_LAUNCH_CHECK("wrs_build_lbvh karras");
    const uint32_t grefit = (m_cap + kRefitBlock - 1) / kRefitBlock;
    k_leaves_refit<<<grefit, kRefitBlock, 0, s>>>(vi, pos4, reinterpret_cast<const float4*>(in->rgba),
                                      in->id, radius_scale, global_scale, hdr, nodes,
                                      bvh->layout == WRS_LBVH_FULL, S.leaf_parent,
                                      S.node_parent, S.node_range, S.visit,
                                      reinterpret_cast<float4*>(sorted->pos_r),
                                      reinterpret_cast<float4*>(sorted->rgba), sorted->id,
                                      sorted->src,
                                      nodes + 4 * (size_t)wrs::lbvh_binary_slots(cap, leaf));
    WRS_LAUNCH_CHECK("wrs_build_lbvh refit");
    return WRS_OK;
}

int wrs_refit_lbvh(const wrs_splats* in, const float* radius_scale, float global_scale,
                   const wrs_lbvh* bvh, wrs_splats* sorted, void* scratch, size_t scratch_bytes,
                   wrs_stream_t stream) {
    if (int rc = check_lbvh_args(in, radius_scale, global_scale, bvh, sorted, scratch,
                                 scratch_bytes, "wrs_refit_lbvh"))
        return rc;
    const uint32_t leaf = bvh->leaf_size;
    const uint32_t cap = in->capacity;
    Scratch S;
    scratch_layout(cap, leaf, static_cast<char*>(scratch), &S);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    LbvhHeader* hdr = static_cast<LbvhHeader*>(bvh->nodes);
    float4* nodes = wrs::lbvh_nodes(bvh->nodes);
    const float4* pos4 = reinterpret_cast<const float4*>(in->pos_r);
    const uint32_t m_cap = leaves_for(cap, leaf);
    // the header again (the centre bounds come out as before; the largest radius and the
    // traversal's coordinate bound follow the new radii), then the leaves and the climb over the
    // order and the links the build left in scratch (vals0 and the parent links)
    k_bounds_partial<<<kBoundsBlocks, 256, 0, s>>>(pos4, radius_scale, global_scale, in->n, cap,
                                                   S.partials);
    WRS_LAUNCH_CHECK("wrs_refit_lbvh bounds");
    k_bounds_final<<<1, kBoundsBlocks, 0, s>>>(S.partials, in->n, cap, leaf, bvh->layout, hdr,
                                              sorted->n);
    WRS_LAUNCH_CHECK("wrs_refit_lbvh bounds final");
    if (cap == 0) return WRS_OK;
    cudaError_t e = cudaMemsetAsync(S.visit, 0, sizeof(uint32_t) * m_cap, s);
    if (e != cudaSuccess) return wrs::cuda_fail(e, "wrs_refit_lbvh memset");
    const uint32_t grefit = (m_cap + kRefitBlock - 1) / kRefitBlock;
    k_leaves_refit<<<grefit, kRefitBlock, 0, s>>>(S.vals0, pos4, reinterpret_cast<const float4*>(in->rgba),
                                      in->id, radius_scale, global_scale, hdr, nodes,
                                      bvh->layout == WRS_LBVH_FULL, S.leaf_parent,
                                      S.node_parent, S.node_range, S.visit,
                                      reinterpret_cast<float4*>(sorted->pos_r),
                                      reinterpret_cast<float4*>(sorted->rgba), sorted->id,
                                      sorted->src,
                                      nodes + 4 * (size_t)wrs::lbvh_binary_slots(cap, leaf));
    WRS_LAUNCH_CHECK("wrs_refit_lbvh refit");
    return WRS_OK;
}

}  // extern "C"
