/*
 * oracle.c -- plain, slow, obviously-correct CPU oracle for the ray-traced sphere-splat warping
 * of Zellmann, "Augmenting Image Warping-Based Remote Volume Rendering with Ray Tracing" (2020).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the benchmark's CPU
 * baseline may load this library.  The CUDA library never calls it and it never calls the CUDA
 * library; the two share no source.
 *
 * Precision (the written spec, S0): every discrete decision -- volume sample above the depth
 * threshold, ray-sphere hit or miss, hit key, Morton code, the stop at T_stop -- is taken in
 * binary32 with the exact operation sequence of the spec; every continuous quantity (colour,
 * opacity, transmittance, soft-edge weight, gradient) is computed in binary64.  A second trace
 * path (orc_trace64) takes every decision in binary64 instead.  Compile with -ffp-contract=off so that
 * the compiler never fuses a multiply and an add on its own.
 *
 * Pinning (tests/test_oracle_*.py): camera orientation against an independent projection; single
 * sphere coverage against the closed-form cone angle; two-sphere composite closed form; brute
 * force against this file's own BVH (bitwise); permutation invariance (bitwise); server view
 * reproduced by the warped splats; constant-volume compositing closed form; a step volume whose
 * threshold crossing is known; central finite differences for the adjoint; the radix tree against
 * a brute-force split search.
 */
#include <fenv.h>
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

#pragma STDC FENV_ACCESS ON

typedef struct {
    float eye[3], right[3], up[3], fwd[3];
    float tan_half_fovy;
    int32_t width, height;
} orc_camera;

/* ------------------------------------------------------------------------------------------ */
/* Threads: a parallel-for over [0, n) with interleaved indices.                                */
/* ------------------------------------------------------------------------------------------ */
typedef void (*orc_body)(void* ctx, int64_t i, int tid);
typedef struct { orc_body fn; void* ctx; int64_t n; int tid, nt; } orc_job;

static void* orc_worker(void* p) {
    orc_job* j = (orc_job*)p;
    for (int64_t i = j->tid; i < j->n; i += j->nt) j->fn(j->ctx, i, j->tid);
    return NULL;
}

int orc_default_threads(void) {
    long n = sysconf(_SC_NPROCESSORS_ONLN);
    return n > 0 ? (int)n : 1;
}

static void orc_parallel(orc_body fn, void* ctx, int64_t n, int nt) {
    if (nt <= 0) nt = orc_default_threads();
    if (nt > 256) nt = 256;
    if (nt == 1 || n < 2) {
        for (int64_t i = 0; i < n; i++) fn(ctx, i, 0);
        return;
    }
    pthread_t th[256];
    orc_job jobs[256];
    for (int t = 0; t < nt; t++) {
        jobs[t] = (orc_job){fn, ctx, n, t, nt};
        pthread_create(&th[t], NULL, orc_worker, &jobs[t]);
    }
    for (int t = 0; t < nt; t++) pthread_join(th[t], NULL);
}

/* ------------------------------------------------------------------------------------------ */
/* S1: primary ray of pixel (x, y), binary32 (Eq. 1: r = o + d t).                              */
/* ------------------------------------------------------------------------------------------ */
void orc_primary_ray(const orc_camera* c, int x, int y, float o[3], float d[3]) {
    float W = (float)c->width, H = (float)c->height;
    float aspect = W / H;
    float sx = c->tan_half_fovy * aspect;
    float u = ((float)(2 * x + 1) / W - 1.0f) * sx;
    float v = (1.0f - (float)(2 * y + 1) / H) * c->tan_half_fovy;
    float e[3];
    for (int k = 0; k < 3; k++) e[k] = fmaf(v, c->up[k], fmaf(u, c->right[k], c->fwd[k]));
    float len2 = fmaf(e[2], e[2], fmaf(e[1], e[1], e[0] * e[0]));
    float inv = 1.0f / sqrtf(len2);
    for (int k = 0; k < 3; k++) {
        d[k] = e[k] * inv;
        o[k] = c->eye[k];
    }
}

/* ------------------------------------------------------------------------------------------ */
/* S2: server volume ray caster with the first-hit depth heuristic (§4.1, §4.2, Fig. 2).        */
/* ------------------------------------------------------------------------------------------ */
typedef struct {
    const void* vol; int dtype; int nx, ny, nz;
    const float* tf; const orc_camera* cam; float step_vox; float tau;
    double* rgba_out; float* depth_out; const int32_t* pix;
    int heur; /* S2a: 0 first hit (param tau), 1 max contribution, 2 accumulated (param theta), 3 max gradient */
} rc_ctx;

static float vox32(const rc_ctx* c, int i, int j, int k) {
    size_t idx = ((size_t)k * c->ny + j) * c->nx + i;
    if (c->dtype == 1) return (float)((const uint8_t*)c->vol)[idx];
    return ((const float*)c->vol)[idx];
}

static float lerp32(float a, float b, float f) { return fmaf(f, b - a, a); }

/* Trilinear sample in binary32 following the spec's operation order; used only for decisions. */
static float sample32(const rc_ctx* c, const float p[3]) {
    int n[3] = {c->nx, c->ny, c->nz}, i0[3], i1[3];
    float f[3];
    for (int a = 0; a < 3; a++) {
        float g = fmaf(p[a], (float)n[a], -0.5f);
        g = fminf(fmaxf(g, 0.0f), (float)(n[a] - 1));
        int i = (int)floorf(g);
        if (n[a] >= 2) { if (i > n[a] - 2) i = n[a] - 2; } else i = 0;
        i0[a] = i;
        i1[a] = n[a] >= 2 ? i + 1 : i;
        f[a] = g - (float)i;
    }
    float c00 = lerp32(vox32(c, i0[0], i0[1], i0[2]), vox32(c, i1[0], i0[1], i0[2]), f[0]);
    float c10 = lerp32(vox32(c, i0[0], i1[1], i0[2]), vox32(c, i1[0], i1[1], i0[2]), f[0]);
    float c01 = lerp32(vox32(c, i0[0], i0[1], i1[2]), vox32(c, i1[0], i0[1], i1[2]), f[0]);
    float c11 = lerp32(vox32(c, i0[0], i1[1], i1[2]), vox32(c, i1[0], i1[1], i1[2]), f[0]);
    float c0 = lerp32(c00, c10, f[1]);
    float c1 = lerp32(c01, c11, f[1]);
    float s = lerp32(c0, c1, f[2]);
    if (c->dtype == 1) s = s / 255.0f;
    return fminf(fmaxf(s, 0.0f), 1.0f);
}

static float tf_alpha32(const float* tf, float s) {
    float X = s * 255.0f;
    int i = (int)floorf(X);
    if (i > 254) i = 254;
    float ph = X - (float)i;
    return lerp32(tf[4 * i + 3], tf[4 * (i + 1) + 3], ph);
}

/* Trilinear sample of the same stored values in binary64 at a binary64 position; compositing. */
static double sample64(const rc_ctx* c, const double p[3]) {
    int n[3] = {c->nx, c->ny, c->nz}, i0[3], i1[3];
    double f[3];
    for (int a = 0; a < 3; a++) {
        double g = p[a] * n[a] - 0.5;
        if (g < 0) g = 0;
        if (g > n[a] - 1) g = n[a] - 1;
        int i = (int)floor(g);
        if (n[a] >= 2) { if (i > n[a] - 2) i = n[a] - 2; } else i = 0;
        i0[a] = i;
        i1[a] = n[a] >= 2 ? i + 1 : i;
        f[a] = g - i;
    }
    double s = 0;
    for (int dz = 0; dz < 2; dz++)
        for (int dy = 0; dy < 2; dy++)
            for (int dx = 0; dx < 2; dx++) {
                double w = (dx ? f[0] : 1 - f[0]) * (dy ? f[1] : 1 - f[1]) * (dz ? f[2] : 1 - f[2]);
                s += w * vox32(c, dx ? i1[0] : i0[0], dy ? i1[1] : i0[1], dz ? i1[2] : i0[2]);
            }
    if (c->dtype == 1) s /= 255.0;
    return s < 0 ? 0 : (s > 1 ? 1 : s);
}

static void tf64(const float* tf, double s, double out[4]) {
    double X = s * 255.0;
    int i = (int)floor(X);
    if (i > 254) i = 254;
    double ph = X - i;
    for (int k = 0; k < 4; k++) out[k] = tf[4 * i + k] * (1 - ph) + tf[4 * (i + 1) + k] * ph;
}

static void rc_pixel(void* vctx, int64_t slot, int tid) {
    (void)tid;
    const rc_ctx* c = (const rc_ctx*)vctx;
    int W = c->cam->width;
    int64_t pix = c->pix ? c->pix[slot] : slot;
    int x = (int)(pix % W), y = (int)(pix / W);
    pix = slot; /* outputs are indexed by slot */
    float o[3], d[3];
    orc_primary_ray(c->cam, x, y, o, d);
    double* out = c->rgba_out + 4 * pix;
    out[0] = out[1] = out[2] = out[3] = 0;
    c->depth_out[pix] = INFINITY;

    /* slab clip against the unit cube, binary32 */
    float lo = 0.0f, hi = INFINITY;
    for (int a = 0; a < 3; a++) {
        if (d[a] != 0.0f) {
            float t0 = (0.0f - o[a]) / d[a], t1 = (1.0f - o[a]) / d[a];
            lo = fmaxf(lo, fminf(t0, t1));
            hi = fminf(hi, fmaxf(t0, t1));
        } else if (!(o[a] >= 0.0f && o[a] <= 1.0f)) {
            return;
        }
    }
    if (!(lo < hi)) return;
    int n = c->nx > c->ny ? c->nx : c->ny;
    if (c->nz > n) n = c->nz;
    float dt = c->step_vox / (float)n;

    float t_first = INFINITY, t_any = INFINITY;
    float A32 = 0.0f, best = -1.0f, t_best = INFINITY, t_acc = INFINITY;
    double C[3] = {0, 0, 0}, A = 0;
    for (int j = 0; j < (1 << 24); j++) { /* at most 2^24 samples per ray */
        float tj = fmaf((float)j + 0.5f, dt, lo);
        if (!(tj < hi)) break;
        /* decision path, binary32 */
        float p32[3];
        for (int a = 0; a < 3; a++) p32[a] = fmaf(d[a], tj, o[a]);
        float a32 = tf_alpha32(c->tf, sample32(c, p32));
        if (a32 >= c->tau && t_first == INFINITY) t_first = tj;
        if (a32 > 0.0f && t_any == INFINITY) t_any = tj;
        if (c->heur == 1 || c->heur == 2) {
            /* S2a: contribution of this sample and opacity accumulated through it */
            float w = (1.0f - A32) * a32;
            A32 = A32 + w;
            if (c->heur == 1 && w > 0.0f && w > best) { best = w; t_best = tj; }
            if (c->heur == 2 && A32 >= c->tau && t_acc == INFINITY) t_acc = tj;
        } else if (c->heur == 3 && a32 > 0.0f) {
            /* S2a: squared gradient by central differences one voxel apart */
            int n3[3] = {c->nx, c->ny, c->nz};
            float g[3];
            for (int a = 0; a < 3; a++) {
                float h = 1.0f / (float)n3[a];
                float pp[3] = {p32[0], p32[1], p32[2]}, pm[3] = {p32[0], p32[1], p32[2]};
                pp[a] = p32[a] + h;
                pm[a] = p32[a] - h;
                g[a] = sample32(c, pp) - sample32(c, pm);
            }
            float m = fmaf(g[2], g[2], fmaf(g[1], g[1], g[0] * g[0]));
            if (m > best) { best = m; t_best = tj; }
        }
        /* compositing path, binary64 */
        double p64[3], rgba[4];
        for (int a = 0; a < 3; a++) p64[a] = (double)o[a] + (double)d[a] * (double)tj;
        tf64(c->tf, sample64(c, p64), rgba);
        double ac = 1.0 - pow(1.0 - rgba[3], (double)c->step_vox);
        for (int k = 0; k < 3; k++) C[k] += (1.0 - A) * ac * rgba[k];
        A += (1.0 - A) * ac;
    }
    for (int k = 0; k < 3; k++) out[k] = C[k];
    out[3] = A;
    float depth;
    if (c->heur == 1 || c->heur == 3) depth = t_best;
    else if (c->heur == 2) depth = t_acc < INFINITY ? t_acc : t_any;
    else depth = t_first < INFINITY ? t_first : t_any;
    c->depth_out[pix] = depth;
}

int orc_raycast_heuristic(const void* vol, int dtype, int nx, int ny, int nz, const float* tf,
                          const orc_camera* cam, float step_vox, int heuristic, float param,
                          const int32_t* pix, int64_t npix, double* rgba_out, float* depth_out,
                          int nthreads) {
    if (!vol || !tf || !cam || !rgba_out || !depth_out || nx < 1 || ny < 1 || nz < 1) return -1;
    if (dtype != 0 && dtype != 1) return -1;
    if (heuristic < 0 || heuristic > 3) return -1;
    if (!pix) npix = (int64_t)cam->width * cam->height;
    rc_ctx c = {vol, dtype, nx, ny, nz, tf, cam, step_vox, param, rgba_out, depth_out, pix, heuristic};
    orc_parallel(rc_pixel, &c, npix, nthreads);
    return 0;
}

int orc_raycast(const void* vol, int dtype, int nx, int ny, int nz, const float* tf,
                const orc_camera* cam, float step_vox, float tau, const int32_t* pix,
                int64_t npix, double* rgba_out, float* depth_out, int nthreads) {
    return orc_raycast_heuristic(vol, dtype, nx, ny, nz, tf, cam, step_vox, 0, tau, pix, npix,
                                 rgba_out, depth_out, nthreads);
}

/* ------------------------------------------------------------------------------------------ */
/* S3: unprojection (Eq. 1), footprint or voxel radius (§4.1), stable compaction (§4.1).        */
/* ------------------------------------------------------------------------------------------ */
int64_t orc_unproject(const float* rgba, const float* depth, const orc_camera* cam, int mode,
                      float voxel_diag, float* pos_r, float* rgba_out, uint32_t* id,
                      int64_t capacity) {
    if (!rgba || !depth || !cam || !pos_r || !rgba_out || !id) return -1;
    int W = cam->width, H = cam->height;
    int64_t n = 0;
    float pitch = (2.0f * cam->tan_half_fovy) / (float)H;
    for (int64_t i = 0; i < (int64_t)W * H; i++) {
        float t = depth[i];
        if (!(t >= 0.0f && t < INFINITY && rgba[4 * i + 3] > 0.0f)) continue;
        if (n >= capacity) return -3;
        float o[3], d[3];
        orc_primary_ray(cam, (int)(i % W), (int)(i / W), o, d);
        float r0;
        if (mode == 0) {
            float dz = fmaf(d[2], cam->fwd[2], fmaf(d[1], cam->fwd[1], d[0] * cam->fwd[0]));
            r0 = ((t * dz) * pitch) * 0.70710677f;
        } else {
            r0 = voxel_diag * 0.5f;
        }
        for (int k = 0; k < 3; k++) pos_r[4 * n + k] = fmaf(d[k], t, o[k]);
        pos_r[4 * n + 3] = r0;
        memcpy(rgba_out + 4 * n, rgba + 4 * i, 4 * sizeof(float));
        id[n] = (uint32_t)i;
        n++;
    }
    return n;
}

/* ------------------------------------------------------------------------------------------ */
/* S3b: samples smeared along the viewing ray over their depth interval (future work, §6): each */
/* kept pixel becomes a chain of touching spheres whose opacities compose to the pixel's alpha.  */
/* ------------------------------------------------------------------------------------------ */
int64_t orc_unproject_interval(const float* rgba, const float* depth_lo, const float* depth_hi,
                               const orc_camera* cam, int mode, float voxel_diag, int max_chain,
                               float* pos_r, float* rgba_out, uint32_t* id, int64_t capacity) {
    if (!rgba || !depth_lo || !depth_hi || !cam || !pos_r || !rgba_out || !id) return -1;
    if (max_chain < 1 || max_chain > 64) return -1;
    int W = cam->width, H = cam->height;
    int64_t n_out = 0;
    float pitch = (2.0f * cam->tan_half_fovy) / (float)H;
    for (int64_t i = 0; i < (int64_t)W * H; i++) {
        float tlo = depth_lo[i], thi = depth_hi[i];
        float a = rgba[4 * i + 3];
        if (!(tlo >= 0.0f && tlo < INFINITY && a > 0.0f)) continue;
        if (!(thi < INFINITY) || !(thi >= tlo)) thi = tlo;
        float dt = thi - tlo;
        float tm = fmaf(dt, 0.5f, tlo);
        float o[3], d[3];
        orc_primary_ray(cam, (int)(i % W), (int)(i / W), o, d);
        float r0;
        if (mode == 0) {
            float dz = fmaf(d[2], cam->fwd[2], fmaf(d[1], cam->fwd[1], d[0] * cam->fwd[0]));
            r0 = ((tm * dz) * pitch) * 0.70710677f;
        } else {
            r0 = voxel_diag * 0.5f;
        }
        int n = 1;
        if (r0 > 0.0f) {
            float c = ceilf(dt / (2.0f * r0));
            n = c < 1.0f ? 1 : (c > (float)max_chain ? max_chain : (int)c);
        }
        /* per-sphere opacity so that n of them compose to a along the ray */
        double scale = 1.0;
        if (n > 1) {
            double ap = -expm1(log1p(-(double)a) / (double)n);
            scale = ap / (double)a;
        }
        for (int k = 0; k < n; k++) {
            if (n_out >= capacity) return -3;
            float u = (float)(2 * k + 1) / (float)(2 * n);
            float tk = fmaf(u, dt, tlo);
            for (int q = 0; q < 3; q++) pos_r[4 * n_out + q] = fmaf(d[q], tk, o[q]);
            pos_r[4 * n_out + 3] = r0;
            for (int ch = 0; ch < 4; ch++)
                rgba_out[4 * n_out + ch] = n == 1 ? rgba[4 * i + ch] : (float)((double)rgba[4 * i + ch] * scale);
            id[n_out] = (uint32_t)(i * max_chain + k);
            n_out++;
        }
    }
    return n_out;
}

/* ------------------------------------------------------------------------------------------ */
/* S10: the earlier point-splat warping (§2; compared in §5, Fig. 3): every sample drawn as an    */
/* s x s pixel square around its projection, one depth per point, nearest (z, k) kept, no blend.  */
/* ------------------------------------------------------------------------------------------ */
int orc_point_splat(const float* pos_r, const float* rgba, int64_t n, const orc_camera* cam,
                    int size, float* rgba_out, int64_t* index_out) {
    if (!cam || !rgba_out || !index_out || size < 1 || size > 64) return -1;
    if (n > 0 && (!pos_r || !rgba)) return -1;
    const int W = cam->width, H = cam->height;
    if (W <= 0 || H <= 0) return -1;
    float* zbest = (float*)malloc(sizeof(float) * (size_t)W * (size_t)H);
    if (!zbest) return -2;
    for (int64_t i = 0; i < (int64_t)W * H; i++) {
        zbest[i] = INFINITY;
        index_out[i] = -1;
    }
    const float aspect = (float)W / (float)H;
    const float sx = cam->tan_half_fovy * aspect;
    const float half = 0.5f * (float)size;
    for (int64_t k = 0; k < n; k++) {
        float q[3];
        for (int a = 0; a < 3; a++) q[a] = pos_r[4 * k + a] - cam->eye[a];
        /* depth along the view axis; points at or behind the eye plane are not drawn */
        float z = fmaf(q[2], cam->fwd[2], fmaf(q[1], cam->fwd[1], q[0] * cam->fwd[0]));
        if (!(z > 0.0f)) continue;
        float xr = fmaf(q[2], cam->right[2], fmaf(q[1], cam->right[1], q[0] * cam->right[0]));
        float yu = fmaf(q[2], cam->up[2], fmaf(q[1], cam->up[1], q[0] * cam->up[0]));
        float nx = (xr / z) / sx;
        float ny = (yu / z) / cam->tan_half_fovy;
        /* pixel-centre coordinates: pixel x has its centre at x (camera convention of S1) */
        float px = (nx + 1.0f) * (0.5f * (float)W) - 0.5f;
        float py = (1.0f - ny) * (0.5f * (float)H) - 0.5f;
        float x0f = ceilf(px - half), y0f = ceilf(py - half);
        if (!(x0f > -(float)size && x0f < (float)W && y0f > -(float)size && y0f < (float)H)) continue;
        int x0 = (int)x0f, y0 = (int)y0f;
        for (int y = y0 < 0 ? 0 : y0; y < y0 + size && y < H; y++) {
            for (int x = x0 < 0 ? 0 : x0; x < x0 + size && x < W; x++) {
                int64_t i = (int64_t)y * W + x;
                /* depth test on (z, k): the nearer point wins, equal depths go to the lower index */
                if (z < zbest[i] || (z == zbest[i] && k < index_out[i])) {
                    zbest[i] = z;
                    index_out[i] = k;
                }
            }
        }
    }
    for (int64_t i = 0; i < (int64_t)W * H; i++) {
        int64_t k = index_out[i];
        for (int c = 0; c < 4; c++) rgba_out[4 * i + c] = k >= 0 ? rgba[4 * k + c] : 0.0f;
    }
    free(zbest);
    return 0;
}

/* ------------------------------------------------------------------------------------------ */
/* S11: the 64-bit position + radius word and the 32-bit colour the server sends (§4.1, §6).      */
/* ------------------------------------------------------------------------------------------ */
static uint32_t quant_floor(float u, uint32_t top) {
    if (!(u == u) || u == INFINITY || u == -INFINITY) return 0;
    float f = floorf(u);
    if (f < 0.0f) return 0;
    if (f > (float)top) return top;
    return (uint32_t)f;
}

int orc_encode(const float* pos_r, const float* rgba, int64_t n, const float lo[3],
               const float hi[3], float r_max, uint64_t* word, uint32_t* color) {
    if (n < 0 || (n > 0 && (!pos_r || !rgba || !word || !color))) return -1;
    float inv[3];
    for (int a = 0; a < 3; a++) {
        float ext = hi[a] - lo[a];
        if (!(ext > 0.0f) || ext == INFINITY) return -1;
        inv[a] = 131072.0f / ext;
    }
    if (!(r_max > 0.0f) || r_max == INFINITY) return -1;
    const float rinv = 8191.0f / r_max;
    for (int64_t k = 0; k < n; k++) {
        uint64_t q[3];
        for (int a = 0; a < 3; a++) q[a] = quant_floor((pos_r[4 * k + a] - lo[a]) * inv[a], 131071u);
        /* the radius is rounded up, so that a decoded sphere still covers its footprint */
        float v = pos_r[4 * k + 3] * rinv;
        uint64_t qr = 0;
        if (v == v && v != INFINITY && v != -INFINITY) {
            float c = ceilf(v);
            qr = c < 0.0f ? 0 : (c > 8191.0f ? 8191 : (uint64_t)c);
        }
        word[k] = q[0] | (q[1] << 17) | (q[2] << 34) | (qr << 51);
        uint32_t w = 0;
        for (int ch = 0; ch < 4; ch++) {
            float x = rgba[4 * k + ch] * 255.0f;
            x = x + 0.5f;
            w |= quant_floor(x, 255u) << (8 * ch);
        }
        color[k] = w;
    }
    return 0;
}

int orc_decode(const uint64_t* word, const uint32_t* color, int64_t n, const float lo[3],
               const float hi[3], float r_max, float* pos_r, float* rgba) {
    if (n < 0 || (n > 0 && (!word || !color || !pos_r || !rgba))) return -1;
    float step[3];
    for (int a = 0; a < 3; a++) step[a] = (hi[a] - lo[a]) * 0x1p-17f;
    const float rstep = r_max / 8191.0f;
    for (int64_t k = 0; k < n; k++) {
        uint64_t w = word[k];
        for (int a = 0; a < 3; a++) {
            uint32_t q = (uint32_t)((w >> (17 * a)) & 0x1FFFFu);
            pos_r[4 * k + a] = fmaf((float)q + 0.5f, step[a], lo[a]);  /* the cell's centre */
        }
        pos_r[4 * k + 3] = (float)(uint32_t)(w >> 51) * rstep;
        for (int ch = 0; ch < 4; ch++) rgba[4 * k + ch] = (float)((color[k] >> (8 * ch)) & 255u) / 255.0f;
    }
    return 0;
}

/* ------------------------------------------------------------------------------------------ */
/* S4/S5: sphere test.  Decision in binary32; the binary64 twin feeds only the diagnostic.      */
/* ------------------------------------------------------------------------------------------ */
static inline float eff_radius(const float* pos_r, const float* scale, float gscale, int64_t i) {
    float s = scale ? scale[i] : gscale;
    if (!(s > 0.0f)) s = 0.0f;
    return s * pos_r[4 * i + 3];
}

/* returns 1 on a hit; *key = entry distance (binary32); *ff_out = squared distance of the ray
 * from the centre (binary32, the same value the hit decision used) */
static int sphere32(const float o[3], const float d[3], const float c[3], float r, float* key,
                    float* ff_out) {
    float oc[3];
    for (int k = 0; k < 3; k++) oc[k] = c[k] - o[k];
    float b = fmaf(oc[2], d[2], fmaf(oc[1], d[1], oc[0] * d[0]));
    float f[3];
    for (int k = 0; k < 3; k++) f[k] = fmaf(-b, d[k], oc[k]);
    float ff = fmaf(f[2], f[2], fmaf(f[1], f[1], f[0] * f[0]));
    *ff_out = ff;
    float q = fmaf(r, r, -ff);
    if (!(q > 0.0f)) return 0;
    float sq = sqrtf(q);
    if (!(b + sq > 0.0f)) return 0;
    float k0 = b - sq;
    *key = k0 > 0.0f ? k0 : 0.0f;
    return 1;
}

/* the same test evaluated in binary64; returns hit, key, and rho = |f| / r */
static int sphere64(const float o[3], const float d[3], const float c[3], float r, double* key,
                    double* rho) {
    double oc[3], f[3], b = 0, ff = 0;
    for (int k = 0; k < 3; k++) oc[k] = (double)c[k] - (double)o[k];
    for (int k = 0; k < 3; k++) b += oc[k] * (double)d[k];
    for (int k = 0; k < 3; k++) { f[k] = oc[k] - b * (double)d[k]; ff += f[k] * f[k]; }
    double q = (double)r * (double)r - ff;
    *rho = r > 0 ? sqrt(ff) / (double)r : 1.0;
    if (!(q > 0)) return 0;
    double sq = sqrt(q);
    if (!(b + sq > 0)) return 0;
    *key = b - sq > 0 ? b - sq : 0;
    return 1;
}

/* S6 soft edge */
static double soft_w(double rho, double beta) {
    if (beta <= 0) return 1.0;
    if (rho <= 1.0 - beta) return 1.0;
    double u = (1.0 - rho) / beta;
    if (u < 0) u = 0;
    return u * u * (3.0 - 2.0 * u);
}
static double soft_dw(double rho, double beta) {
    if (beta <= 0 || rho <= 1.0 - beta) return 0.0;
    double u = (1.0 - rho) / beta;
    if (u < 0) return 0.0;
    return 6.0 * u * (1.0 - u) * (-1.0 / beta);
}

/* ------------------------------------------------------------------------------------------ */
/* The oracle's own BVH: top-down median split over sphere boxes in binary64.  It only speeds   */
/* up the search; brute force over all spheres gives bitwise the same images.                  */
/* ------------------------------------------------------------------------------------------ */
typedef struct { double lo[3], hi[3]; int32_t left, right, first, count; } obvh_node;
typedef struct {
    obvh_node* nodes; int32_t n_nodes;
    int32_t* prim;    /* primitive indices, leaf ranges point here */
    int64_t n;
} orc_bvh;

typedef struct { const float* pos_r; const float* scale; float gscale; } prim_src;

static void prim_box(const prim_src* s, int32_t i, double lo[3], double hi[3]) {
    float r = eff_radius(s->pos_r, s->scale, s->gscale, i);
    for (int k = 0; k < 3; k++) {
        lo[k] = (double)s->pos_r[4 * i + k] - (double)r;
        hi[k] = (double)s->pos_r[4 * i + k] + (double)r;
    }
}

/* Partition prim[first, first+count) so that the element of rank k (by centre coordinate on
 * `axis`, ties by index) is in place, smaller before it, larger after it (quickselect). */
static int prim_less(const float* pos, int axis, int32_t i, int32_t j) {
    float x = pos[4 * (int64_t)i + axis], y = pos[4 * (int64_t)j + axis];
    return x < y || (x == y && i < j);
}
static void select_kth(int32_t* a, int32_t n, int32_t k, const float* pos, int axis) {
    int32_t lo = 0, hi = n - 1;
    while (lo < hi) {
        int32_t pivot = a[lo + (hi - lo) / 2];
        int32_t i = lo, j = hi;
        while (i <= j) {
            while (prim_less(pos, axis, a[i], pivot)) i++;
            while (prim_less(pos, axis, pivot, a[j])) j--;
            if (i <= j) { int32_t t = a[i]; a[i] = a[j]; a[j] = t; i++; j--; }
        }
        if (k <= j) hi = j;
        else if (k >= i) lo = i;
        else return;
    }
}

static int32_t obvh_build_rec(orc_bvh* B, const prim_src* s, int32_t first, int32_t count,
                              int leaf) {
    int32_t me = B->n_nodes++;
    obvh_node* nd = &B->nodes[me];
    for (int k = 0; k < 3; k++) { nd->lo[k] = INFINITY; nd->hi[k] = -INFINITY; }
    double clo[3] = {INFINITY, INFINITY, INFINITY}, chi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int32_t a = first; a < first + count; a++) {
        double lo[3], hi[3];
        prim_box(s, B->prim[a], lo, hi);
        for (int k = 0; k < 3; k++) {
            if (lo[k] < nd->lo[k]) nd->lo[k] = lo[k];
            if (hi[k] > nd->hi[k]) nd->hi[k] = hi[k];
            double c = s->pos_r[4 * B->prim[a] + k];
            if (c < clo[k]) clo[k] = c;
            if (c > chi[k]) chi[k] = c;
        }
    }
    nd->first = first;
    nd->count = count;
    nd->left = nd->right = -1;
    if (count <= leaf) return me;
    int axis = 0;
    for (int k = 1; k < 3; k++)
        if (chi[k] - clo[k] > chi[axis] - clo[axis]) axis = k;
    int32_t half = count / 2;
    select_kth(B->prim + first, count, half, s->pos_r, axis);
    int32_t l = obvh_build_rec(B, s, first, half, leaf);
    int32_t r = obvh_build_rec(B, s, first + half, count - half, leaf);
    B->nodes[me].left = l;
    B->nodes[me].right = r;
    B->nodes[me].count = 0;
    return me;
}

void* orc_bvh_build(const float* pos_r, const float* scale, float gscale, int64_t n, int leaf) {
    if (n <= 0 || !pos_r) return NULL;
    if (leaf < 1) leaf = 1;
    orc_bvh* B = (orc_bvh*)calloc(1, sizeof(orc_bvh));
    B->n = n;
    B->prim = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
    for (int64_t i = 0; i < n; i++) B->prim[i] = (int32_t)i;
    B->nodes = (obvh_node*)malloc(sizeof(obvh_node) * (size_t)(2 * n + 1));
    prim_src s = {pos_r, scale, gscale};
    obvh_build_rec(B, &s, 0, (int32_t)n, leaf);
    return B;
}

void orc_bvh_free(void* p) {
    orc_bvh* B = (orc_bvh*)p;
    if (!B) return;
    free(B->nodes);
    free(B->prim);
    free(B);
}

/* conservative ray-box test in binary64; eps widens the box to cover binary32 graze decisions */
static int box_hit(const double lo[3], const double hi[3], const double o[3], const double d[3],
                   double eps) {
    double tmin = 0.0, tmax = INFINITY;
    for (int k = 0; k < 3; k++) {
        double l = lo[k] - eps, h = hi[k] + eps;
        if (d[k] != 0.0) {
            double t0 = (l - o[k]) / d[k], t1 = (h - o[k]) / d[k];
            if (t0 > t1) { double t = t0; t0 = t1; t1 = t; }
            if (t0 > tmin) tmin = t0;
            if (t1 < tmax) tmax = t1;
        } else if (o[k] < l || o[k] > h) {
            return 0;
        }
    }
    return tmin <= tmax;
}

/* ------------------------------------------------------------------------------------------ */
/* Hit collection and compositing (S5, S6).                                                      */
/* ------------------------------------------------------------------------------------------ */
typedef struct {
    const float* pos_r; const float* rgba; const uint32_t* id; int64_t n;
    const float* scale; float global_scale; const float* opacity;
    int32_t max_hits; double t_stop; double beta;
} orc_scene;

typedef struct {
    float key; uint32_t id; int32_t idx; double key64; int hit64; double rho;
    float rho32; /* |f| / r in binary32 from the decision's own |f|^2 (S0: feeds the stop decision) */
} hit_t;

static int cmp_hit(const void* a, const void* b) {
    const hit_t* x = (const hit_t*)a;
    const hit_t* y = (const hit_t*)b;
    if (x->key < y->key) return -1;
    if (x->key > y->key) return 1;
    return (x->id > y->id) - (x->id < y->id);
}

typedef struct { hit_t* h; int64_t n, cap; int amb; } hitlist;

static void hl_push(hitlist* L, hit_t h) {
    if (L->n == L->cap) {
        L->cap = L->cap ? 2 * L->cap : 64;
        L->h = (hit_t*)realloc(L->h, sizeof(hit_t) * (size_t)L->cap);
    }
    L->h[L->n++] = h;
}

static void test_prim(const orc_scene* s, int32_t i, const float o[3], const float d[3],
                      hitlist* L) {
    float r = eff_radius(s->pos_r, s->scale, s->global_scale, i);
    const float* c = s->pos_r + 4 * (int64_t)i;
    float key = 0.0f, ff = 0.0f;
    double key64 = 0.0, rho;
    int h32 = sphere32(o, d, c, r, &key, &ff);
    int h64 = sphere64(o, d, c, r, &key64, &rho);
    if (h32 != h64) L->amb |= 1;
    if (!h32) return;
    float rho32 = r > 0.0f ? sqrtf(ff) / r : 1.0f;
    hit_t h = {key, s->id[i], i, key64, h64, rho, rho32};
    hl_push(L, h);
}

/* Collect every hit of the ray (any order), then sort by (key, id). */
static void collect_hits(const orc_scene* s, const orc_bvh* B, const float o[3], const float d[3],
                         hitlist* L) {
    L->n = 0;
    L->amb = 0;
    if (!B) {
        for (int64_t i = 0; i < s->n; i++) test_prim(s, (int32_t)i, o, d, L);
    } else {
        double o64[3] = {o[0], o[1], o[2]}, d64[3] = {d[0], d[1], d[2]};
        double eps = 1e-6 * (1.0 + fabs(o64[0]) + fabs(o64[1]) + fabs(o64[2]));
        int32_t stack[256];
        int sp = 0;
        stack[sp++] = 0;
        while (sp) {
            const obvh_node* nd = &B->nodes[stack[--sp]];
            if (!box_hit(nd->lo, nd->hi, o64, d64, eps)) continue;
            if (nd->left < 0) {
                for (int32_t a = nd->first; a < nd->first + nd->count; a++)
                    test_prim(s, B->prim[a], o, d, L);
            } else {
                stack[sp++] = nd->left;
                stack[sp++] = nd->right;
            }
        }
    }
    qsort(L->h, (size_t)L->n, sizeof(hit_t), cmp_hit);
    /* diagnostic: would a binary64 evaluation order these hits differently? */
    for (int64_t k = 1; k < L->n; k++) {
        const hit_t* a = &L->h[k - 1];
        const hit_t* b = &L->h[k];
        if (a->key64 > b->key64 || (a->key64 == b->key64 && a->id > b->id)) L->amb |= 2;
    }
}

/* S6 soft edge in binary32 (feeds only the stop decision) */
static float soft_w32(float rho, float beta) {
    if (beta <= 0.0f || rho <= 1.0f - beta) return 1.0f;
    float u = fmaxf((1.0f - rho) / beta, 0.0f);
    return u * u * (3.0f - 2.0f * u);
}

/* Front-to-back compositing of the sorted hits (S6); returns the number of hits used.
 * Colours, alphas and the transmittance are binary64.  The decision to stop at T <= T_stop is
 * a discrete decision, taken (S0) on the binary32 transmittance: alpha = clamp((o a) w) with w
 * from the binary32 distance ratio, T <- T (1 - alpha), compared with T_stop in binary32.
 * *stop64 (optional) is set when the binary64 transmittance would have stopped at another hit
 * (a diagnostic: such a pixel's image moves by about T_stop at most, but the derivatives of its
 * alpha with respect to the earlier hits depend on the later hit). */
static int64_t composite(const orc_scene* s, const hitlist* L, double out[4], double* T_out,
                         double* T_before /* optional, per used hit */, int* stop64) {
    const float t_stop32 = (float)s->t_stop, beta32 = (float)s->beta;
    double T = 1.0, C[3] = {0, 0, 0};
    float T32 = 1.0f;
    int differ = 0;
    int64_t k = 0;
    for (; k < L->n; k++) {
        if (s->max_hits > 0 && k == s->max_hits) break;
        if ((T <= s->t_stop) != (T32 <= t_stop32)) differ = 1;
        if (T32 <= t_stop32) break;
        const hit_t* h = &L->h[k];
        double w = soft_w(h->rho, s->beta);
        double op = s->opacity ? (double)s->opacity[h->idx] : 1.0;
        const float* c = s->rgba + 4 * (int64_t)h->idx;
        double x = op * (double)c[3] * w;
        double a = x < 0 ? 0 : (x > 1 ? 1 : x);
        if (T_before) T_before[k] = T;
        for (int ch = 0; ch < 3; ch++) C[ch] += T * (op * w) * (double)c[ch];
        T *= 1.0 - a;
        float op32 = s->opacity ? s->opacity[h->idx] : 1.0f;
        float w32 = beta32 > 0.0f ? soft_w32(h->rho32, beta32) : 1.0f;
        float x32 = op32 * c[3] * w32;
        float a32 = fminf(fmaxf(x32, 0.0f), 1.0f);
        T32 = T32 * (1.0f - a32);
    }
    out[0] = C[0]; out[1] = C[1]; out[2] = C[2]; out[3] = 1.0 - T;
    if (T_out) *T_out = T;
    if (stop64) *stop64 = differ;
    return k;
}

typedef struct {
    const orc_scene* s; const orc_camera* cam; const orc_bvh* B;
    const int32_t* pix; double* rgba_out; double* T_out; int32_t* nused; int32_t* nhits;
    uint8_t* amb; uint64_t* hash; hitlist* lists;
} tr_ctx;

static void tr_pixel(void* vctx, int64_t i, int tid) {
    tr_ctx* c = (tr_ctx*)vctx;
    int64_t p = c->pix ? c->pix[i] : i;
    int W = c->cam->width;
    float o[3], d[3];
    orc_primary_ray(c->cam, (int)(p % W), (int)(p / W), o, d);
    hitlist* L = &c->lists[tid];
    collect_hits(c->s, c->B, o, d, L);
    double T;
    int stop64 = 0;
    int64_t used = composite(c->s, L, c->rgba_out + 4 * i, &T, NULL, &stop64);
    if (c->T_out) c->T_out[i] = T;
    if (c->nused) c->nused[i] = (int32_t)used;
    if (c->nhits) c->nhits[i] = (int32_t)L->n;
    if (c->amb) c->amb[i] = (uint8_t)(L->amb | (stop64 ? 4 : 0));
    if (c->hash) { /* FNV-1a over the ids of the used hits, in order */
        uint64_t h = 1469598103934665603ull;
        for (int64_t k = 0; k < used; k++) { h ^= L->h[k].id; h *= 1099511628211ull; }
        c->hash[i] = h;
    }
}

int orc_trace(const orc_scene* s, const void* bvh, const orc_camera* cam, const int32_t* pix,
              int64_t npix, double* rgba_out, double* T_out, int32_t* nused, int32_t* nhits,
              uint8_t* amb, uint64_t* hash, int nthreads) {
    if (!s || !cam || !rgba_out) return -1;
    if (!pix) npix = (int64_t)cam->width * cam->height;
    int nt = nthreads > 0 ? nthreads : orc_default_threads();
    if (nt > 256) nt = 256;
    hitlist* lists = (hitlist*)calloc((size_t)nt, sizeof(hitlist));
    tr_ctx c = {s, cam, (const orc_bvh*)bvh, pix, rgba_out, T_out, nused, nhits, amb, hash, lists};
    if (s->n <= 0) {
        for (int64_t i = 0; i < npix; i++) {
            for (int k = 0; k < 4; k++) rgba_out[4 * i + k] = 0;
            if (T_out) T_out[i] = 1;
            if (nused) nused[i] = 0;
            if (nhits) nhits[i] = 0;
            if (amb) amb[i] = 0;
            if (hash) hash[i] = 1469598103934665603ull;
        }
    } else {
        orc_parallel(tr_pixel, &c, npix, nt);
    }
    for (int t = 0; t < nt; t++) free(lists[t].h);
    free(lists);
    return 0;
}

/* ------------------------------------------------------------------------------------------ */
/* The same trace with every decision in binary64 (the plain reading of Fig. 2's transparent   */
/* spheres hit by the client's rays, §4): primary ray, hit or miss, entry distance and hit     */
/* order all in double.  Kept apart from the binary32 path above; nothing is shared but the    */
/* soft-edge weight, the BVH (an accelerator only) and the thread pool.                         */
/*                                                                                              */
/* Ties.  A pixel is a tie at distance t when moving the ray or a sphere by at most t (scene   */
/* units) can change which spheres the pixel composites or their order: a composited sphere    */
/* that the ray grazes within t, a near miss within t that could enter in front of the point   */
/* where compositing stopped, two hits whose entry distances can swap (their ranges under such */
/* a move overlap; a grazing hit's entry distance is ill-conditioned and its range is wide),   */
/* or a sphere whose exit is within reach of the eye.  Arithmetic of another precision decides */
/* such pixels either way; nothing else can differ.                                            */
/* ------------------------------------------------------------------------------------------ */
void orc_primary_ray64(const orc_camera* c, int x, int y, double o[3], double d[3]) {
    double W = c->width, H = c->height, th = c->tan_half_fovy;
    double u = ((2.0 * x + 1.0) / W - 1.0) * th * (W / H);
    double v = (1.0 - (2.0 * y + 1.0) / H) * th;
    double e[3], len = 0;
    for (int k = 0; k < 3; k++) {
        e[k] = (double)c->fwd[k] + u * (double)c->right[k] + v * (double)c->up[k];
        len += e[k] * e[k];
    }
    len = sqrt(len);
    for (int k = 0; k < 3; k++) {
        d[k] = e[k] / len;
        o[k] = c->eye[k];
    }
}

typedef struct {
    double key, rho;
    double key_lo, key_hi;      /* range of the entry distance under a move of at most t */
    int could_miss, could_hit;  /* the hit decision can flip under such a move */
    uint32_t id; int32_t idx; int hit;
} hit64_t;

typedef struct { hit64_t* h; int64_t n, cap; } hitlist64;

static void hl64_push(hitlist64* L, hit64_t h) {
    if (L->n == L->cap) {
        L->cap = L->cap ? 2 * L->cap : 64;
        L->h = (hit64_t*)realloc(L->h, sizeof(hit64_t) * (size_t)L->cap);
    }
    L->h[L->n++] = h;
}

static int cmp_hit64(const void* a, const void* b) {
    const hit64_t* x = (const hit64_t*)a;
    const hit64_t* y = (const hit64_t*)b;
    if (x->key < y->key) return -1;
    if (x->key > y->key) return 1;
    return (x->id > y->id) - (x->id < y->id);
}

static double pos0(double x) { return x > 0 ? x : 0.0; }

/* The ray-sphere test of S5 in binary64 on a binary64 ray: with oc = c - o, b = oc.d,
 * f = oc - b d and q = r^2 - |f|^2, a hit iff q > 0 and the exit distance b + sqrt(q) > 0;
 * key = max(b - sqrt(q), 0).  A move of at most t shifts b by up to t and the ray's distance
 * from the centre |f| by up to t, which bounds the entry and exit distances. */
static void sphere_f64(const double o[3], const double d[3], const float* c, double r, double t,
                       hit64_t* h) {
    double oc[3], f[3], b = 0, ff = 0;
    for (int k = 0; k < 3; k++) oc[k] = (double)c[k] - o[k];
    for (int k = 0; k < 3; k++) b += oc[k] * d[k];
    for (int k = 0; k < 3; k++) { f[k] = oc[k] - b * d[k]; ff += f[k] * f[k]; }
    double dist = sqrt(ff);
    double q = r * r - ff;
    double sq = q > 0 ? sqrt(q) : 0.0;
    h->rho = r > 0 ? dist / r : 1.0;
    h->hit = q > 0 && b + sq > 0;
    h->key = pos0(b - sq);
    double dn = pos0(dist - t), df = dist + t;
    double sq_max = dn < r ? sqrt(r * r - dn * dn) : -1.0; /* -1: no hit under any move */
    double sq_min = df < r ? sqrt(r * r - df * df) : 0.0;
    h->key_lo = sq_max >= 0 ? pos0(b - t - sq_max) : INFINITY;
    h->key_hi = pos0(b + t - sq_min);
    int far_pos = sq_max >= 0 && b + t + sq_max > 0;   /* some move gives an exit beyond the eye */
    int far_neg = !(df < r) || b - t + sq_min <= 0;    /* some move gives a miss */
    h->could_hit = !h->hit && far_pos;
    h->could_miss = h->hit && far_neg;
}

typedef struct {
    const orc_scene* s; const orc_camera* cam; const orc_bvh* B; const int32_t* pix;
    double tie;
    double* rgba_out; double* T_out; int32_t* nused; int32_t* nhits; uint8_t* tie_out;
    hitlist64* hits; hitlist64* near; /* per thread: hits, and misses a move of t can turn into hits */
} tr64_ctx;

static void test_prim64(const tr64_ctx* c, int32_t i, const double o[3], const double d[3],
                        hitlist64* hits, hitlist64* near) {
    const orc_scene* s = c->s;
    double sc = s->scale ? (double)s->scale[i] : (double)s->global_scale;
    if (!(sc > 0)) sc = 0;
    double r = sc * (double)s->pos_r[4 * (int64_t)i + 3];
    hit64_t h;
    sphere_f64(o, d, s->pos_r + 4 * (int64_t)i, r, c->tie, &h);
    h.id = s->id[i];
    h.idx = i;
    if (h.hit) hl64_push(hits, h);
    else if (h.could_hit) hl64_push(near, h);
}

static void tr64_pixel(void* vctx, int64_t i, int tid) {
    tr64_ctx* c = (tr64_ctx*)vctx;
    const orc_scene* s = c->s;
    int64_t p = c->pix ? c->pix[i] : i;
    int W = c->cam->width;
    double o[3], d[3];
    orc_primary_ray64(c->cam, (int)(p % W), (int)(p / W), o, d);
    hitlist64* L = &c->hits[tid];
    hitlist64* N = &c->near[tid];
    L->n = 0;
    N->n = 0;
    if (s->n > 0 && !c->B) {
        for (int64_t k = 0; k < s->n; k++) test_prim64(c, (int32_t)k, o, d, L, N);
    } else if (s->n > 0) {
        double eps = 1e-6 * (1.0 + fabs(o[0]) + fabs(o[1]) + fabs(o[2])) + 2.0 * c->tie;
        int32_t stack[256];
        int sp = 0;
        stack[sp++] = 0;
        while (sp) {
            const obvh_node* nd = &c->B->nodes[stack[--sp]];
            if (!box_hit(nd->lo, nd->hi, o, d, eps)) continue;
            if (nd->left < 0) {
                for (int32_t a = nd->first; a < nd->first + nd->count; a++)
                    test_prim64(c, c->B->prim[a], o, d, L, N);
            } else {
                stack[sp++] = nd->left;
                stack[sp++] = nd->right;
            }
        }
    }
    qsort(L->h, (size_t)L->n, sizeof(hit64_t), cmp_hit64);
    /* front-to-back compositing (S6), as in the binary32 path */
    double T = 1.0, C[3] = {0, 0, 0};
    int64_t used = 0;
    for (; used < L->n; used++) {
        if (s->max_hits > 0 && used == s->max_hits) break;
        if (T <= s->t_stop) break;
        const hit64_t* h = &L->h[used];
        double w = soft_w(h->rho, s->beta);
        double op = s->opacity ? (double)s->opacity[h->idx] : 1.0;
        const float* col = s->rgba + 4 * (int64_t)h->idx;
        double x = op * (double)col[3] * w;
        double a = x < 0 ? 0 : (x > 1 ? 1 : x);
        for (int ch = 0; ch < 3; ch++) C[ch] += T * (op * w) * (double)col[ch];
        T *= 1.0 - a;
    }
    double* out = c->rgba_out + 4 * i;
    out[0] = C[0]; out[1] = C[1]; out[2] = C[2]; out[3] = 1.0 - T;
    if (c->T_out) c->T_out[i] = T;
    if (c->nused) c->nused[i] = (int32_t)used;
    if (c->nhits) c->nhits[i] = (int32_t)L->n;
    if (!c->tie_out) return;
    /* Which decisions can change the pixel.  When compositing stopped early (hit limit or
     * T_stop), a sphere that cannot enter in front of the last composited hit changes nothing. */
    uint8_t flag = 0;
    /* compositing takes no further hit: hits left over, T at or below T_stop, or the limit */
    int stopped = used < L->n || T <= s->t_stop || (s->max_hits > 0 && used >= s->max_hits);
    double reach = INFINITY; /* largest entry distance at which a sphere still changes the pixel */
    if (stopped) reach = used > 0 ? L->h[used - 1].key_hi : -INFINITY;
    for (int64_t k = 0; k < used; k++) {
        const hit64_t* a = &L->h[k];
        if (a->could_miss) flag |= 1;
        for (int64_t j = k + 1; j < L->n; j++) {
            const hit64_t* b = &L->h[j];
            if (a->key_hi == 0 && b->key_hi == 0) continue; /* both around the eye: id order */
            if (b->key_lo <= a->key_hi) flag |= 2;
        }
    }
    for (int64_t k = 0; k < N->n; k++)
        if (N->h[k].key_lo <= reach) flag |= 4;
    c->tie_out[i] = flag;
}

int orc_trace64(const orc_scene* s, const void* bvh, const orc_camera* cam, const int32_t* pix,
                int64_t npix, double tie, double* rgba_out, double* T_out, int32_t* nused,
                int32_t* nhits, uint8_t* tie_out, int nthreads) {
    if (!s || !cam || !rgba_out || !(tie >= 0)) return -1;
    if (!pix) npix = (int64_t)cam->width * cam->height;
    int nt = nthreads > 0 ? nthreads : orc_default_threads();
    if (nt > 256) nt = 256;
    hitlist64* hits = (hitlist64*)calloc((size_t)nt, sizeof(hitlist64));
    hitlist64* near = (hitlist64*)calloc((size_t)nt, sizeof(hitlist64));
    tr64_ctx c = {s, cam, (const orc_bvh*)bvh, pix, tie, rgba_out, T_out, nused, nhits, tie_out,
                  hits, near};
    orc_parallel(tr64_pixel, &c, npix, nt);
    for (int t = 0; t < nt; t++) { free(hits[t].h); free(near[t].h); }
    free(hits);
    free(near);
    return 0;
}

/* ------------------------------------------------------------------------------------------ */
/* S7: adjoint of the ordered compositing, binary64.  Gradients in compacted splat order.       */
/* ------------------------------------------------------------------------------------------ */
typedef struct {
    const orc_scene* s; const orc_camera* cam; const orc_bvh* B; const double* dimg;
    double** g_rgba; double** g_op; double** g_sc; hitlist* lists;
} bw_ctx;

static void bw_pixel(void* vctx, int64_t p, int tid) {
    bw_ctx* c = (bw_ctx*)vctx;
    const orc_scene* s = c->s;
    const double* g = c->dimg + 4 * p;
    if (g[0] == 0 && g[1] == 0 && g[2] == 0 && g[3] == 0) return;
    int W = c->cam->width;
    float o[3], d[3];
    orc_primary_ray(c->cam, (int)(p % W), (int)(p / W), o, d);
    hitlist* L = &c->lists[tid];
    collect_hits(s, c->B, o, d, L);
    if (L->n == 0) return;
    double* Tb = (double*)malloc(sizeof(double) * (size_t)L->n);
    double out[4], Tend;
    int64_t used = composite(s, L, out, &Tend, Tb, NULL);
    double S[3] = {0, 0, 0}, P = 1.0; /* suffix composite and suffix transmittance */
    double* gr = c->g_rgba[tid];
    double* go = c->g_op[tid];
    double* gs = c->g_sc[tid];
    for (int64_t k = used - 1; k >= 0; k--) {
        const hit_t* h = &L->h[k];
        int32_t i = h->idx;
        double w = soft_w(h->rho, s->beta);
        double op = s->opacity ? (double)s->opacity[i] : 1.0;
        const float* col = s->rgba + 4 * (int64_t)i;
        double x = op * (double)col[3] * w;
        double a = x < 0 ? 0 : (x > 1 ? 1 : x);
        double pass = (x >= 0 && x <= 1) ? 1.0 : 0.0;
        double T = Tb[k];
        double gC = g[0] * col[0] + g[1] * col[1] + g[2] * col[2];
        double gS = g[0] * S[0] + g[1] * S[1] + g[2] * S[2];
        double dLda = T * (g[3] * P - gS);                /* dL/d(alpha_h) */
        for (int ch = 0; ch < 3; ch++) gr[4 * i + ch] += T * op * w * g[ch];
        gr[4 * i + 3] += dLda * pass * op * w;
        go[i] += T * w * gC + dLda * pass * col[3] * w;
        double dLdw = T * op * gC + dLda * pass * op * col[3];
        float r = eff_radius(s->pos_r, s->scale, s->global_scale, i);
        if (r > 0 && s->beta > 0) {
            double dw = soft_dw(h->rho, s->beta);
            double r0 = s->pos_r[4 * (int64_t)i + 3];
            gs[i] += dLdw * dw * (-h->rho / (double)r) * r0;
        }
        for (int ch = 0; ch < 3; ch++) S[ch] = op * w * (double)col[ch] + (1.0 - a) * S[ch];
        P *= 1.0 - a;
    }
    free(Tb);
}

int orc_trace_backward(const orc_scene* s, const void* bvh, const orc_camera* cam,
                       const double* dL_dimg, double* g_rgba, double* g_opacity, double* g_scale,
                       int nthreads) {
    if (!s || !cam || !dL_dimg || !g_rgba || !g_opacity || !g_scale) return -1;
    int64_t n = s->n;
    memset(g_rgba, 0, sizeof(double) * 4 * (size_t)(n > 0 ? n : 0));
    memset(g_opacity, 0, sizeof(double) * (size_t)(n > 0 ? n : 0));
    memset(g_scale, 0, sizeof(double) * (size_t)(n > 0 ? n : 0));
    if (n <= 0) return 0;
    int nt = nthreads > 0 ? nthreads : orc_default_threads();
    if (nt < 1) nt = 1;
    if (nt > 64) nt = 64;
    double* gr[64]; double* go[64]; double* gs[64];
    for (int t = 0; t < nt; t++) {
        gr[t] = (double*)calloc(4 * (size_t)n, sizeof(double));
        go[t] = (double*)calloc((size_t)n, sizeof(double));
        gs[t] = (double*)calloc((size_t)n, sizeof(double));
    }
    hitlist* lists = (hitlist*)calloc((size_t)nt, sizeof(hitlist));
    bw_ctx c = {s, cam, (const orc_bvh*)bvh, dL_dimg, gr, go, gs, lists};
    orc_parallel(bw_pixel, &c, (int64_t)cam->width * cam->height, nt);
    for (int t = 0; t < nt; t++) {
        for (int64_t i = 0; i < 4 * n; i++) g_rgba[i] += gr[t][i];
        for (int64_t i = 0; i < n; i++) { g_opacity[i] += go[t][i]; g_scale[i] += gs[t][i]; }
        free(gr[t]); free(go[t]); free(gs[t]); free(lists[t].h);
    }
    free(lists);
    return 0;
}

/* ------------------------------------------------------------------------------------------ */
/* S8: LBVH reference -- Morton codes (binary32 quantisation), stable sort, the binary radix    */
/* tree by its top-down definition, bounds with outward rounding.  Index work: compared bitwise. */
/* ------------------------------------------------------------------------------------------ */
static uint32_t spread10(uint32_t v) {
    uint32_t r = 0;
    for (int b = 0; b < 10; b++) r |= ((v >> b) & 1u) << (3 * b);
    return r;
}

typedef struct { uint32_t code; uint32_t idx; } keyidx;
static int cmp_keyidx(const void* a, const void* b) {
    const keyidx* x = (const keyidx*)a;
    const keyidx* y = (const keyidx*)b;
    if (x->code != y->code) return x->code < y->code ? -1 : 1;
    return (x->idx > y->idx) - (x->idx < y->idx);
}

static int clz32(uint32_t v) { return v ? __builtin_clz(v) : 32; }

static int delta_leaf(const uint32_t* lcode, int64_t M, int64_t i, int64_t j) {
    if (j < 0 || j >= M) return -1;
    uint32_t a = lcode[i], b = lcode[j];
    if (a != b) return clz32(a ^ b);
    return 32 + clz32((uint32_t)i ^ (uint32_t)j);
}

static float round_down_sub(float a, float b) {
    fesetround(FE_DOWNWARD);
    volatile float x = a - b;
    fesetround(FE_TONEAREST);
    return x;
}
static float round_up_add(float a, float b) {
    fesetround(FE_UPWARD);
    volatile float x = a + b;
    fesetround(FE_TONEAREST);
    return x;
}

int orc_lbvh(const float* pos_r, const float* scale, float gscale, int64_t n, int32_t leaf,
             uint32_t* codes_sorted, uint32_t* order, int32_t* child, float* boxes,
             int32_t* root, float* cbounds) {
    if (n <= 0 || leaf < 1 || !pos_r) return -1;
    float cmin[3] = {INFINITY, INFINITY, INFINITY}, cmax[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t i = 0; i < n; i++)
        for (int k = 0; k < 3; k++) {
            cmin[k] = fminf(cmin[k], pos_r[4 * i + k]);
            cmax[k] = fmaxf(cmax[k], pos_r[4 * i + k]);
        }
    if (cbounds) for (int k = 0; k < 3; k++) { cbounds[k] = cmin[k]; cbounds[3 + k] = cmax[k]; }
    float sc[3];
    for (int k = 0; k < 3; k++) {
        float ext = cmax[k] - cmin[k];
        sc[k] = ext > 0.0f ? 1024.0f / ext : 0.0f;
    }
    keyidx* ki = (keyidx*)malloc(sizeof(keyidx) * (size_t)n);
    for (int64_t i = 0; i < n; i++) {
        uint32_t q[3];
        for (int k = 0; k < 3; k++) {
            float v = floorf((pos_r[4 * i + k] - cmin[k]) * sc[k]);
            q[k] = v >= 1023.0f ? 1023u : (uint32_t)v;
        }
        ki[i].code = (spread10(q[0]) << 2) | (spread10(q[1]) << 1) | spread10(q[2]);
        ki[i].idx = (uint32_t)i;
    }
    qsort(ki, (size_t)n, sizeof(keyidx), cmp_keyidx);
    for (int64_t i = 0; i < n; i++) {
        if (codes_sorted) codes_sorted[i] = ki[i].code;
        if (order) order[i] = ki[i].idx;
    }
    int64_t M = (n + leaf - 1) / leaf;
    uint32_t* lcode = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)M);
    for (int64_t j = 0; j < M; j++) lcode[j] = ki[j * leaf].code;

    /* leaf boxes */
    float* lbox = (float*)malloc(sizeof(float) * 6 * (size_t)M);
    for (int64_t j = 0; j < M; j++) {
        float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
        for (int64_t a = j * leaf; a < (j + 1) * leaf && a < n; a++) {
            uint32_t i = ki[a].idx;
            float r = eff_radius(pos_r, scale, gscale, i);
            for (int k = 0; k < 3; k++) {
                lo[k] = fminf(lo[k], round_down_sub(pos_r[4 * i + k], r));
                hi[k] = fmaxf(hi[k], round_up_add(pos_r[4 * i + k], r));
            }
        }
        for (int k = 0; k < 3; k++) { lbox[6 * j + k] = lo[k]; lbox[6 * j + 3 + k] = hi[k]; }
    }
    if (M == 1) {
        if (root) *root = (int32_t)0x80000000u; /* leaf 0 */
        free(lbox); free(lcode); free(ki);
        return 0;
    }
    if (root) *root = 0;
    /* top-down: internal node covering leaves [a, b] */
    int64_t* st = (int64_t*)malloc(sizeof(int64_t) * 3 * (size_t)(M + 1));
    int64_t sp = 0;
    st[sp++] = 0; st[sp++] = M - 1; st[sp++] = 0; /* a, b, node index */
    while (sp) {
        int64_t node = st[--sp], b = st[--sp], a = st[--sp];
        int dn = delta_leaf(lcode, M, a, b);
        int64_t g = a;
        for (int64_t k = a; k < b; k++)
            if (delta_leaf(lcode, M, a, k) > dn) g = k;
        int32_t lref, rref;
        if (g == a) lref = (int32_t)(0x80000000u | (uint32_t)g);
        else { lref = (int32_t)g; st[sp++] = a; st[sp++] = g; st[sp++] = g; }
        if (g + 1 == b) rref = (int32_t)(0x80000000u | (uint32_t)(g + 1));
        else { rref = (int32_t)(g + 1); st[sp++] = g + 1; st[sp++] = b; st[sp++] = g + 1; }
        child[2 * node] = lref;
        child[2 * node + 1] = rref;
    }
    free(st);
    /* bounds of internal nodes: a post-order pass over the child table */
    if (boxes) {
        char* done = (char*)calloc((size_t)M, 1);
        int64_t* stk = (int64_t*)malloc(sizeof(int64_t) * (size_t)(2 * M + 2));
        int64_t top = 0;
        stk[top++] = 0;
        while (top) {
            int64_t node = stk[top - 1];
            int ready = 1;
            for (int c = 0; c < 2; c++) {
                int32_t ref = child[2 * node + c];
                if (ref >= 0 && !done[ref]) { stk[top++] = ref; ready = 0; }
            }
            if (!ready) continue;
            top--;
            float* nb = boxes + 12 * node; /* child0 lo, child0 hi, child1 lo, child1 hi */
            for (int c = 0; c < 2; c++) {
                int32_t ref = child[2 * node + c];
                const float* src;
                float tmp[6];
                if (ref < 0) src = lbox + 6 * (int64_t)((uint32_t)ref & 0x7FFFFFFFu);
                else {
                    const float* cb = boxes + 12 * (int64_t)ref;
                    for (int k = 0; k < 3; k++) {
                        tmp[k] = fminf(cb[k], cb[6 + k]);
                        tmp[3 + k] = fmaxf(cb[3 + k], cb[9 + k]);
                    }
                    src = tmp;
                }
                memcpy(nb + 6 * c, src, 6 * sizeof(float));
            }
            done[node] = 1;
        }
        free(done);
        free(stk);
    }
    free(lbox); free(lcode); free(ki);
    return 0;
}
