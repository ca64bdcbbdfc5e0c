/*
 * wrs.h -- C ABI of libwrs: ray-traced sphere-splat image warping for remote volume rendering
 * (Zellmann, "Augmenting Image Warping-Based Remote Volume Rendering with Ray Tracing", 2020).
 *
 * The client side of the method (§4): each pixel of a server-rendered colour + depth image becomes
 * an object-space sphere (Eq. 1, §4.1); an LBVH is built over the spheres (§4.1, §4.2); every
 * frame the spheres are ray traced from the newer camera and composited front to back (Fig. 2
 * caption, §4).  The server-side volume ray caster with its depth heuristic (§4.1, §4.2) is also
 * exported because it produces the inputs.
 *
 * Conventions for every entry point:
 *  - All array pointers are DEVICE pointers owned by the caller, unless a comment says "host".
 *    The library never allocates, frees or keeps device memory; work buffers ("scratch") are
 *    passed in by the caller, sized by the matching *_bytes() query, 256-byte aligned.
 *  - Every call is asynchronous on the given stream (a cudaStream_t; NULL = the legacy default
 *    stream), performs no host synchronisation and no allocation, and can be captured in a CUDA
 *    graph -- except wrs_check_status(), which synchronises the stream.
 *  - The splat count lives on the device (uint32_t* n) so that unproject -> build -> trace needs
 *    no host round trip; kernels are sized by capacity and skip work beyond *n.
 *  - Return value: WRS_OK (0) or a negative WRS_ERR_* code; wrs_last_error() then describes the
 *    failure (per host thread).  Argument errors are detected on the host before any launch.
 *    Errors found by a kernel (a traversal stack overflow, a backward hit list longer than its
 *    chunk table) are OR-ed into the caller's device status word (int32_t* status, may be NULL
 *    where noted) and surface through wrs_check_status().
 *  - Numerics follow a written spec: discrete decisions (hit/miss, hit order, depth threshold,
 *    Morton code) in binary32 with a fixed operation order; see each function.
 *  - Layouts: images are row-major, y = 0 the top row, RGBA interleaved float32 (16 B / pixel),
 *    premultiplied.  Volumes are x-fastest [nz][ny][nx] over the unit cube [0,1]^3.
 */
#ifndef WRS_H
#define WRS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef void* wrs_stream_t; /* cudaStream_t */

/* return codes */
#define WRS_OK 0
#define WRS_ERR_ARG -1       /* bad argument (NULL pointer, size, camera, parameter) */
#define WRS_ERR_CUDA -2      /* a CUDA runtime call or launch failed */
#define WRS_ERR_CAPACITY -3  /* an output or buffer is smaller than the input requires */
#define WRS_ERR_SCRATCH -4   /* scratch buffer too small */
#define WRS_ERR_DEVICE -5    /* a kernel reported an error in the status word */

/* bits of the device status word */
#define WRS_STATUS_STACK_OVERFLOW 1u  /* BVH traversal stack exceeded; the ray was cut short */
#define WRS_STATUS_CHUNK_OVERFLOW 2u  /* backward: more hit chunks than its table holds */
#define WRS_STATUS_MALFORMED_TREE 4u  /* traversal met an impossible node reference or revisit */
#define WRS_STATUS_SPLAT_OVERFLOW 8u  /* wrs_unproject_append: splats beyond capacity were dropped */

/* volume scalar types */
#define WRS_F32 0
#define WRS_U8 1

/* depth heuristics of wrs_raycast_volume_heuristic (spec S2a; §2 cites them, §5 uses a gradient
 * heuristic, the paper defines none) */
#define WRS_DEPTH_FIRST_HIT 0          /* first sample with alpha >= param (tau), else first alpha > 0 */
#define WRS_DEPTH_MAX_CONTRIBUTION 1   /* sample with the largest (1 - A) alpha, A accumulated */
#define WRS_DEPTH_ACCUMULATED 2        /* first sample where A reaches param (theta), else first alpha > 0 */
#define WRS_DEPTH_MAX_GRADIENT 3       /* sample with alpha > 0 and the largest |grad s|^2 (central
                                          differences one voxel apart) */

/* radius rules for wrs_unproject */
#define WRS_RADIUS_FOOTPRINT 0 /* half diagonal of the pixel footprint at the sample's depth */
#define WRS_RADIUS_VOXEL 1     /* half a voxel's diagonal, the paper's rule (§4.1) */

/* Quantisation box and radius bound of the 64-bit splat word (wrs_encode_splats and friends):
 * positions are quantised to 2^17 cells per axis of [lo, hi] (hi > lo, finite), radii to 8192
 * steps of [0, r_max] (r_max > 0, finite).  Passed by host pointer. */
typedef struct {
    float lo[3], hi[3];
    float r_max;
} wrs_codec;

/* Pinhole camera.  right/up/fwd: orthonormal basis, view along +fwd.  Pixel (x, y), y = 0 top,
 * one ray through each pixel centre: u = ((2x+1)/W - 1) tan_half_fovy W/H,
 * v = (1 - (2y+1)/H) tan_half_fovy, d = normalize(fwd + u right + v up), origin eye (Eq. 1). */
typedef struct {
    float eye[3], right[3], up[3], fwd[3];
    float tan_half_fovy;
    int32_t width, height;
} wrs_camera;

/* A splat set.  pos_r[i] = (x, y, z, r), rgba[i] = premultiplied colour, id[i] = server pixel
 * index y*Ws + x (the tie-break of equal hit distances).  src[i] is filled only for sorted sets
 * (output of wrs_build_lbvh): the compacted index the sorted splat came from; NULL otherwise.
 * n: device uint32 holding the number of valid splats.  capacity: entries allocated. */
typedef struct {
    float* pos_r;     /* [capacity][4] */
    float* rgba;      /* [capacity][4] */
    uint32_t* id;     /* [capacity] */
    uint32_t* src;    /* [capacity] or NULL */
    uint32_t* n;      /* [1] */
    uint32_t capacity;
} wrs_splats;

/* Tree layouts (wrs_lbvh.layout).  Both hold the same 4-wide nodes, bitwise.  FULL also holds
 * every binary record, which the binary traversal (width 2) reads.  WIDE is for the 4-wide
 * traversal only: the build writes the binary records of the nodes whose leaves span several
 * of its refit blocks (it passes boxes between blocks through them) and leaves the others as
 * they were, which saves about a tenth of the build. */
#define WRS_LBVH_FULL 0
#define WRS_LBVH_WIDE 1

/* An LBVH: one device buffer of wrs_lbvh_bytes(capacity, leaf_size) bytes holding a 64-byte
 * header, the binary internal nodes (64 B each: both children's boxes and references) and, for
 * every binary internal node, a 4-wide node over its grandchildren (128 B). */
typedef struct {
    void* nodes;
    uint32_t capacity;  /* maximum splats */
    uint32_t leaf_size; /* splats per leaf, 1..16 */
    uint32_t layout;    /* WRS_LBVH_FULL (0) or WRS_LBVH_WIDE: what the build writes; a trace
                           passes the layout the tree was built with, and width 2 needs FULL */
} wrs_lbvh;

/* Trace schedules (performance only; results are bitwise identical). */
#define WRS_SCHEDULE_PER_PIXEL 0   /* one thread per pixel, grid over the image */
#define WRS_SCHEDULE_PERSISTENT 1  /* one resident wave of 128-thread blocks; warps refill idle
                                      lanes with new rays (block size fixed at 128) */
#define WRS_SCHEDULE_PACKET 2      /* the 32 rays of an 8x4 tile share one traversal of the
                                      4-wide nodes (width is ignored) */
#define WRS_SCHEDULE_PER_SESSION 3 /* wrs_trace_batched only: each session's own schedule field
                                      (PER_PIXEL or PACKET) picks how its tiles are traced */

/* Compositing (spec S6) and performance parameters of a trace.  Results do not depend on
 * k_chunk, block or schedule (bitwise). */
typedef struct {
    int32_t max_hits;     /* H: hits composited at most; 1 = first hit (the paper), 0 = all */
    float t_stop;         /* stop once transmittance <= t_stop (default 1e-5) */
    float edge_softness;  /* beta in [0,1): soft sphere edge for differentiation; 0 = hard */
    const float* opacity; /* device [n] per-splat opacity in COMPACTED order, or NULL (= 1) */
    int32_t k_chunk;      /* hits gathered per traversal pass: 1, 2, 4, 8 or 16 */
    int32_t block;        /* threads per block: 64, 128 or 256 (per-pixel schedule; the 4-wide
                             traversal with k_chunk 1, 2, 4 or 8 uses at most 128) */
    int32_t schedule;     /* WRS_SCHEDULE_PER_PIXEL, WRS_SCHEDULE_PERSISTENT or
                             WRS_SCHEDULE_PACKET; wrs_trace_batched: PER_PIXEL and PACKET = one
                             warp per 8x4 tile of all sessions, PERSISTENT = lane refill */
    int32_t width;        /* traversal: 2 (or 0) = binary nodes, 4 = the LBVH's 4-wide nodes;
                             the binary traversal (width 2 under any schedule but PACKET) of a
                             tree built with layout WRS_LBVH_WIDE is refused: WRS_ERR_ARG */
} wrs_trace_params;

/* One client session of wrs_trace_batched (device array of these). */
typedef struct {
    const void* nodes;     /* the session's LBVH buffer */
    const float* pos_r;    /* its sorted splats */
    const float* rgba;
    const uint32_t* id;
    const uint32_t* src;
    const float* opacity;  /* or NULL */
    float* rgba_out;       /* [height][width][4] */
    wrs_camera cam;
    uint32_t tile_begin;   /* first work item of this session (prefix sum of wrs_session_tiles) */
    uint32_t schedule;     /* under WRS_SCHEDULE_PER_SESSION: WRS_SCHEDULE_PACKET traces this
                              session's tiles with warp-shared traversals, any other value one
                              thread per pixel; ignored by the other schedules */
} wrs_session;

const char* wrs_version(void);
/* Description of the last error on this host thread ("" if none). */
const char* wrs_last_error(void);
/* sizeof(wrs_session) and sizeof(wrs_camera), for bindings that lay the structs out by hand. */
size_t wrs_session_size(void);
size_t wrs_camera_size(void);

/* Colour weight of the server frame of age `age` (0 = newest) in a window accumulated with
 * wrs_unproject_append: decay^age by repeated binary32 multiplication (spec S3a; the paper names
 * accumulation over frames as future work, §6, without a rule).  Host function, no GPU work;
 * decay outside (0, 1] returns NaN. */
float wrs_window_weight(float decay, uint32_t age);

/* Read the device status word (synchronises the stream), clear it, and return WRS_OK or
 * WRS_ERR_DEVICE (with the set bits described by wrs_last_error). */
int wrs_check_status(int32_t* status, wrs_stream_t stream);

/* Server-side volume ray caster with the first-hit depth heuristic (§4.1, §4.2, Fig. 2; the
 * heuristic is cited from earlier work, §2).  Spec S2: samples every step_vox voxels from the ray's
 * entry into the unit cube, trilinear reconstruction, 256-entry RGBA transfer function (tf, device
 * [256][4]), opacity correction to a one-voxel step, front-to-back compositing without early
 * termination, at most 2^24 samples per ray; step_vox in [1e-3, 1e3].  depth_out = first sample distance whose transfer-function alpha >= tau, else the
 * first with alpha > 0, else +inf.  rgba_out: [H][W][4] premultiplied; depth_out: [H][W]. */
int wrs_raycast_volume(const void* vol, int32_t dtype, int32_t nx, int32_t ny, int32_t nz,
                       const float* tf, const wrs_camera* cam, float step_vox, float tau,
                       float* rgba_out, float* depth_out, wrs_stream_t stream);

/* wrs_raycast_volume with another depth heuristic (WRS_DEPTH_*; readings of §2 and §5, spec
 * S2a).  Decisions in binary32 on the same samples and uncorrected alphas; the colour composite
 * is the same for every heuristic.  param: tau for WRS_DEPTH_FIRST_HIT, theta for
 * WRS_DEPTH_ACCUMULATED, ignored otherwise.  wrs_raycast_volume(..., tau, ...) equals
 * heuristic WRS_DEPTH_FIRST_HIT with param tau. */
int wrs_raycast_volume_heuristic(const void* vol, int32_t dtype, int32_t nx, int32_t ny,
                                 int32_t nz, const float* tf, const wrs_camera* cam,
                                 float step_vox, int32_t heuristic, float param, float* rgba_out,
                                 float* depth_out, wrs_stream_t stream);

/* Unprojection with footprint radius and stable compaction (Eq. 1, §4.1).  For every server
 * pixel with finite depth t >= 0 and alpha > 0: p = eye + d t (d the pixel's ray of cam), radius
 * by radius_mode (voxel_diag = length of a voxel's diagonal, used by WRS_RADIUS_VOXEL), colour
 * copied.  Kept pixels are written to out in pixel order, id = pixel index; *out->n = count.
 * Requires out->capacity >= width * height.  Scratch: wrs_unproject_scratch_bytes(w, h). */
size_t wrs_unproject_scratch_bytes(int32_t width, int32_t height);
int wrs_unproject(const float* rgba, const float* depth, const wrs_camera* cam,
                  int32_t radius_mode, float voxel_diag, wrs_splats* out, void* scratch,
                  size_t scratch_bytes, wrs_stream_t stream);

/* The server's record format (§4.1: the position is quantised and packed with the radius into
 * 64 bits; §6: 32 bits of colour; the paper gives no layout -- spec S11 is this library's):
 *   word[i]  = qx | qy << 17 | qz << 34 | qr << 51  (uint64; qa = floor((p_a - lo_a) * 2^17 / ext_a)
 *              clamped to 0..2^17-1, qr = ceil(r * 8191 / r_max) clamped to 0..8191)
 *   color[i] = r | g << 8 | b << 16 | a << 24       (uint32; floor(c * 255 + 0.5) per channel)
 * 12 bytes per splat instead of 36.  Non-finite inputs quantise to 0.
 *
 * wrs_unproject_encode: wrs_unproject (same kept pixels, order, radius) writing the encoded stream
 * directly: word/color [capacity], *n = count (device), capacity >= width * height.  Scratch:
 * wrs_unproject_scratch_bytes(w, h).
 * wrs_encode_splats: encode the first *in->n records of a float splat set (word/color hold
 * in->capacity entries); *n_out (device, may be NULL) = that count.
 * wrs_decode_splats: decode the first min(*n, capacity) records into float splats (position =
 * the cell's centre, radius = qr * r_max / 8191, colour = c8 / 255, id = stream index, which keeps
 * the tie order of pixel ids because the stream is in pixel order); *out->n = that count;
 * out->capacity >= capacity.  The result feeds wrs_build_lbvh unchanged. */
int wrs_unproject_encode(const float* rgba, const float* depth, const wrs_camera* cam,
                         int32_t radius_mode, float voxel_diag, const wrs_codec* codec,
                         uint64_t* word, uint32_t* color, uint32_t* n, uint32_t capacity,
                         void* scratch, size_t scratch_bytes, wrs_stream_t stream);
int wrs_encode_splats(const wrs_splats* in, const wrs_codec* codec, uint64_t* word,
                      uint32_t* color, uint32_t* n_out, wrs_stream_t stream);
int wrs_decode_splats(const uint64_t* word, const uint32_t* color, const uint32_t* n,
                      uint32_t capacity, const wrs_codec* codec, wrs_splats* out,
                      wrs_stream_t stream);

/* Samples smeared along the viewing ray by depth uncertainty (§6 proposes it as future work and
 * gives no rule; spec S3b is this library's reading).  depth_lo / depth_hi: [H][W] the depths at
 * which the accumulated opacity reaches 0.25 and 0.75 (wrs_raycast_volume_heuristic with
 * WRS_DEPTH_ACCUMULATED and those thresholds).  Every pixel kept by the wrs_unproject rule (on
 * depth_lo) becomes a chain of n = clamp(ceil((t_hi - t_lo) / 2 r0), 1, max_chain) spheres of
 * radius r0 (the radius rule at the interval's middle) centred at t_lo + (2k+1)(t_hi - t_lo)/2n on
 * its ray, each with opacity a' = 1 - (1 - a)^(1/n) (colour scaled by a'/a) so that the chain
 * composites back to the pixel along its own ray; id = pixel * max_chain + k; records in pixel
 * order.  max_chain in 1..64, width * height * max_chain <= 2^32.  *out->n = the number of
 * records, clamped to out->capacity (then WRS_STATUS_SPLAT_OVERFLOW is OR-ed into *status, which
 * may be NULL).  With t_hi = t_lo the output equals wrs_unproject's, ids times max_chain.
 * Scratch: wrs_unproject_scratch_bytes(w, h). */
int wrs_unproject_interval(const float* rgba, const float* depth_lo, const float* depth_hi,
                           const wrs_camera* cam, int32_t radius_mode, float voxel_diag,
                           int32_t max_chain, wrs_splats* out, void* scratch,
                           size_t scratch_bytes, int32_t* status, wrs_stream_t stream);

/* Accumulation over server frames (§6 names it as future work and gives no rule; spec S3a is
 * this library's reading): wrs_unproject of one more frame, APPENDED to the splats already in out.
 * With N0 = *out->n on entry (read on the device), the frame's kept pixels (same rule, radius and
 * pixel order as wrs_unproject) are written at N0, N0+1, ... with id = id_base + pixel index and
 * rgba = weight * rgba per channel (binary32; weight in (0, 1], 1 copies bit for bit); then
 * *out->n = N0 + count.  Records whose slot is >= out->capacity are dropped, *out->n is clamped
 * to the capacity and WRS_STATUS_SPLAT_OVERFLOW is OR-ed into *status (status may be NULL: then
 * the overflow is silent).  Requires id_base + width * height <= 2^32 and capacity >= 1; any
 * capacity is accepted (a window of F frames of one size needs F * width * height).  A window
 * of frames is built by one wrs_unproject (newest frame) and one append per older frame; the
 * trace and the LBVH need no change.  Scratch: wrs_unproject_scratch_bytes(w, h). */
int wrs_unproject_append(const float* rgba, const float* depth, const wrs_camera* cam,
                         int32_t radius_mode, float voxel_diag, float weight, uint32_t id_base,
                         wrs_splats* out, void* scratch, size_t scratch_bytes, int32_t* status,
                         wrs_stream_t stream);

/* wrs_unproject for callers that cannot give the library device memory: the paper has no
 * counterpart; this is an interface convenience.  Some hosts fix their device memory when they
 * start (a viewer or plug-in whose embedding application owns the GPU heap, or a process that
 * forbids allocation once its frame loop runs) and so cannot allocate or lend a work buffer per
 * call.  This entry point allocates nothing: its work buffer is a fixed 512 KiB array inside the
 * library's device image, which every GPU that loads the library keeps until the process exits.
 * Inputs and outputs are the caller's, exactly as for wrs_unproject, with the same results.
 *  - Limit: width * height <= 67,108,864 pixels (for example 8192 x 8192 or 16384 x 4096);
 *    larger images return WRS_ERR_CAPACITY.
 *  - The first call on a device looks up that device's address of the array (with the device
 *    current) and caches it for the rest of the process; make that first call before any stream
 *    capture.  The cached address dies with the device's primary context: after cudaDeviceReset
 *    (or anything else that destroys that context) do not call this entry point again in the
 *    same process.
 *  - All calls share the one array per device, which keeps the last call's contents.  Each call
 *    writes every entry it reads before reading it, so nothing needs clearing, but calls that
 *    overlap on the GPU (other streams, other host threads) race on it: serialise them. */
int wrs_unproject_static(const float* rgba, const float* depth, const wrs_camera* cam,
                         int32_t radius_mode, float voxel_diag, wrs_splats* out,
                         wrs_stream_t stream);

/* LBVH over the spheres (§4.1, §4.2; spec S8): 30-bit Morton codes of the centres over their
 * bounds, stable LSD radix sort of (code, index), binary radix tree (Karras 2012) over leaves of
 * leaf_size consecutive sorted splats, bottom-up refit of the sphere boxes.  The effective radius
 * r = max(s, 0) * r0 (s = radius_scale[i] in compacted order, or global_scale if radius_scale is
 * NULL) is baked into sorted->pos_r[.].w; sorted also receives rgba, id, src (= compacted index)
 * and *sorted->n (*in->n is clamped to in->capacity).  bvh->capacity and sorted->capacity must be
 * >= in->capacity.  The build writes the tree header (with bvh->layout), every node a traversal
 * of that layout can reach and rows [0, n) of sorted, so neither buffer needs clearing before
 * the call.  bvh->layout not WRS_LBVH_FULL or WRS_LBVH_WIDE: WRS_ERR_ARG.
 * Buffer sizes: wrs_lbvh_bytes() for bvh->nodes, wrs_lbvh_scratch_bytes() for scratch. */
size_t wrs_lbvh_bytes(uint32_t capacity, uint32_t leaf_size);
size_t wrs_lbvh_scratch_bytes(uint32_t capacity, uint32_t leaf_size);
int wrs_build_lbvh(const wrs_splats* in, const float* radius_scale, float global_scale,
                   const wrs_lbvh* bvh, wrs_splats* sorted, void* scratch, size_t scratch_bytes,
                   wrs_stream_t stream);

/* The same tree with new radii: a tree's leaf order and shape depend on the splat centres only
 * (the Morton codes), so when only the radius scales change (the radius fit) the boxes can be
 * refitted over the existing tree.  Recomputes the header, the effective radii of sorted (and its
 * other arrays), every binary and 4-wide node box, bottom-up over the leaf order and parent links
 * that the last wrs_build_lbvh call left in `scratch`: the result is bitwise the tree
 * wrs_build_lbvh would build with these radius scales, at the cost of the bounds and the refit
 * (no Morton codes, sort or radix tree).  Contract: the same in, bvh (layout included), sorted
 * and scratch as that build, and since then no change to the splat centres or count and no other use of the scratch;
 * otherwise the result is undefined (no access leaves the buffers and the kernels still end).
 * Arguments and errors as wrs_build_lbvh. */
int wrs_refit_lbvh(const wrs_splats* in, const float* radius_scale, float global_scale,
                   const wrs_lbvh* bvh, wrs_splats* sorted, void* scratch, size_t scratch_bytes,
                   wrs_stream_t stream);

/* Trace the client camera's primary rays through the spheres and composite (spec S5, S6; the
 * paper's first-hit query is max_hits = 1).  Hits ordered by (entry distance, id); each
 * composited hit adds T (o w) rgb and multiplies T by 1 - clamp(o a w, 0, 1).  rgba_out:
 * [H][W][4] premultiplied.  status: device word for traversal errors (may be NULL). */
int wrs_trace(const wrs_lbvh* bvh, const wrs_splats* sorted, const wrs_camera* cam,
              const wrs_trace_params* params, float* rgba_out, int32_t* status,
              wrs_stream_t stream);

/* Several client views of one scene in one launch: the novel views a client renders from one
 * server frame (§4), traced together so that small views still fill the GPU.  cams: HOST array of
 * n_views >= 1 cameras, all of the same width W and height H (WRS_ERR_ARG otherwise), read during
 * the call.  rgba_out: device [n_views][H][W][4]; view v is bitwise the image wrs_trace writes for
 * cams[v].  Schedules: PER_PIXEL and PACKET as in wrs_trace; PERSISTENT runs per pixel (the views
 * together fill the GPU, which is what its lane refill is for).  Up to 32 views per launch
 * (more are split into launches of 32). */
int wrs_trace_views(const wrs_lbvh* bvh, const wrs_splats* sorted, const wrs_camera* cams,
                    int32_t n_views, const wrs_trace_params* params, float* rgba_out,
                    int32_t* status, wrs_stream_t stream);

/* Same traversal, counting instead of writing an image: counters (device uint64[6]) receive the
 * totals over all rays of nodes visited, boxes tested, spheres tested, hits gathered, hits
 * composited and traversal passes.  Used for the roofline's algorithmic byte and flop counts. */
int wrs_trace_count(const wrs_lbvh* bvh, const wrs_splats* sorted, const wrs_camera* cam,
                    const wrs_trace_params* params, unsigned long long* counters,
                    int32_t* status, wrs_stream_t stream);

/* Work items (8x4 pixel ray tiles) of one session with the given client size. */
uint32_t wrs_session_tiles(int32_t width, int32_t height);

/* Many client sessions, each with its own LBVH, splats, camera and output, traced in ONE launch
 * of 128-thread blocks (params->block is ignored).  params->schedule WRS_SCHEDULE_PER_PIXEL: one
 * warp per 8x4 ray tile of the concatenated tile space (the warp finds its session by binary
 * search); WRS_SCHEDULE_PACKET: the same tiles, each traced by one warp-shared traversal of the
 * session's 4-wide nodes; WRS_SCHEDULE_PER_SESSION: the same tiles, each session traced as its
 * own schedule field says (a sparse session, with several client pixels per splat, gains from
 * the shared traversal; a dense one does not).  WRS_SCHEDULE_PERSISTENT: one resident wave whose warps take chunks of
 * four ray tiles of any session from *work_counter (device uint32, reset by this call) and refill
 * their idle lanes from them.  sessions: device array of n_sessions descriptors whose tile_begin are the prefix
 * sums of wrs_session_tiles; total_tiles = their sum.  Each session's image equals wrs_trace's
 * bitwise.  A session whose tree was built with layout WRS_LBVH_WIDE and that would be traced
 * over binary nodes (width 2, schedule not PACKET) sets WRS_STATUS_MALFORMED_TREE in *status
 * (checked on the device from the trees' headers; its image is then undefined). */
int wrs_trace_batched(const wrs_session* sessions, int32_t n_sessions, uint32_t total_tiles,
                      const wrs_trace_params* params, uint32_t* work_counter, int32_t* status,
                      wrs_stream_t stream);

/* Adjoint of wrs_trace (spec S7): given dL/d(rgba_out) (device [H][W][4]), re-traverse every ray
 * to rebuild its hit list (nothing is stored by the forward pass) and accumulate, in COMPACTED
 * splat order, g_rgba[n][4] (dL/d rgba; dL_drgba and g_rgba 16-byte aligned), g_opacity[n]
 * (dL/d opacity, may be NULL) and
 * g_scale[n] (dL/d radius scale, may be NULL; zero when edge_softness = 0).  radius_scale /
 * global_scale must be the values the LBVH was built with.  The outputs are zeroed by this call
 * over the first in-capacity entries; accumulation uses float atomics (summation order is not
 * fixed).  status: device word (CHUNK_OVERFLOW if a ray has more than 64 * k_chunk hits).
 * Schedules: PER_PIXEL one thread per pixel (with 4-wide nodes each warp's lanes take their node
 * and leaf steps together, as in wrs_trace); PERSISTENT lane refill; PACKET the same per-ray work
 * with every traversal shared by the warp (4-wide nodes, as wrs_trace's packet schedule). */
int wrs_trace_backward(const wrs_lbvh* bvh, const wrs_splats* sorted, const wrs_camera* cam,
                       const wrs_trace_params* params, const float* radius_scale,
                       float global_scale, const float* dL_drgba, float* g_rgba,
                       float* g_opacity, float* g_scale, int32_t* status, wrs_stream_t stream);

/* wrs_trace_backward without zeroing the outputs: the gradients of this view are added to what
 * g_rgba / g_opacity / g_scale hold, so several views of one splat set (one LBVH) accumulate into
 * one gradient.  Not in the paper; used for multi-view fitting. */
int wrs_trace_backward_accumulate(const wrs_lbvh* bvh, const wrs_splats* sorted,
                                  const wrs_camera* cam, const wrs_trace_params* params,
                                  const float* radius_scale, float global_scale,
                                  const float* dL_drgba, float* g_rgba, float* g_opacity,
                                  float* g_scale, int32_t* status, wrs_stream_t stream);

/* The adjoint of wrs_trace_views (spec S7): dL_drgba is device [n_views][H][W][4] (cams as for
 * wrs_trace_views), and every view's gradients are added into the one set of per-splat outputs
 * (float atomics; summation order not fixed), i.e. the sum of the views' wrs_trace_backward
 * gradients.  accumulate = 0 zeroes the outputs first (as wrs_trace_backward), 1 adds to what
 * they hold (as wrs_trace_backward_accumulate).  Schedule PACKET runs the packet backward, any
 * other one thread per pixel.  Not in the paper; used for multi-view fitting. */
int wrs_trace_backward_views(const wrs_lbvh* bvh, const wrs_splats* sorted,
                             const wrs_camera* cams, int32_t n_views,
                             const wrs_trace_params* params, const float* radius_scale,
                             float global_scale, const float* dL_drgba, float* g_rgba,
                             float* g_opacity, float* g_scale, int32_t accumulate,
                             int32_t* status, wrs_stream_t stream);

/* wrs_trace_views that also records, for the adjoint, the hits each ray composited (spec S6, in
 * compositing order), so that wrs_trace_backward_views_recorded needs no traversal (spec S7: the
 * adjoint holds the hit set and order of the forward pass fixed; recording it is the choice when
 * memory allows, re-traversing it the choice when it does not).  Ray r = v * H * W + y * W + x:
 *  - hits: device [n_views * H * W][hit_capacity] uint32, the sorted-splat indices (positions in
 *    `sorted`) of the composited hits of ray r in hits[r * hit_capacity + i], i < count;
 *  - hit_count: device [n_views * H * W] uint32, the number of composited hits of ray r, or
 *    hit_capacity + 1 when the ray composited more (then its list is incomplete and the adjoint
 *    traces that ray again);
 *  - hit_capacity in 1..32.  Images are bitwise those of wrs_trace_views.  Caller-owned buffers;
 *    entries past a ray's count are left unwritten. */
int wrs_trace_views_record(const wrs_lbvh* bvh, const wrs_splats* sorted, const wrs_camera* cams,
                           int32_t n_views, const wrs_trace_params* params, float* rgba_out,
                           uint32_t* hits, uint32_t* hit_count, uint32_t hit_capacity,
                           int32_t* status, wrs_stream_t stream);

/* wrs_trace_backward_views from the lists of wrs_trace_views_record (same bvh, sorted splats,
 * cameras, parameters, opacity and radius scales as that call; lists unchanged since): the rays
 * whose list is complete are differentiated from it without traversal, the others are traced
 * again as wrs_trace_backward_views does.  The gradients equal wrs_trace_backward_views' up to the
 * order of the float atomics.  accumulate as for wrs_trace_backward_views. */
int wrs_trace_backward_views_recorded(const wrs_lbvh* bvh, const wrs_splats* sorted,
                                      const wrs_camera* cams, int32_t n_views,
                                      const wrs_trace_params* params, const float* radius_scale,
                                      float global_scale, const uint32_t* hits,
                                      const uint32_t* hit_count, uint32_t hit_capacity,
                                      const float* dL_drgba, float* g_rgba, float* g_opacity,
                                      float* g_scale, int32_t accumulate, int32_t* status,
                                      wrs_stream_t stream);

/* The earlier 2.5D warping the paper compares against (§2, §5, Fig. 3): every splat of a set
 * (compacted or sorted; index = its position in that set) drawn as a point_size x point_size pixel
 * square around its projection into cam, one depth per point (the view-axis distance z, points
 * with z <= 0 dropped), the nearest point kept per pixel (ties: lower index), no blending; spec S10
 * gives the binary32 projection and the covering rule.  rgba_out: [H][W][4] premultiplied, the
 * winner's colour or 0; index_out: [H][W] the winner's index or -1 (may be NULL).  point_size in
 * 1..64.  Scratch: wrs_point_splat_scratch_bytes(W, H) (one 64-bit depth key per pixel), 8-byte
 * aligned.  No OpenGL: the rasterisation is restated as a CUDA kernel. */
size_t wrs_point_splat_scratch_bytes(int32_t width, int32_t height);
int wrs_point_splat(const wrs_splats* splats, const wrs_camera* cam, int32_t point_size,
                    float* rgba_out, int32_t* index_out, void* scratch, size_t scratch_bytes,
                    wrs_stream_t stream);

/* Measurement helper, not part of the method: blocks x 256 threads, each running iters x 128
 * binary32 FMAs in 8 independent chains (2 flops each), so that a caller timing the launch gets
 * the FP32 FMA throughput and the warp-instruction issue rate of ALU-bound code under the current
 * clocks.  out: device float[blocks], never written in practice (it keeps the chains alive). */
int wrs_fma_peak(float* out, int32_t blocks, int32_t iters, wrs_stream_t stream);

/* Measurement helper, not part of the method: copy `bytes` (a multiple of 16; both buffers
 * 16-byte aligned device memory) from src to dst, `reps` times over, with `blocks` x 256 threads
 * (four 16-byte loads in flight per thread).  Timed by the caller: over buffers far larger than
 * L2 the HBM copy rate (2 x bytes x reps moved), over buffers that fit in L2 the L2 rate. */
int wrs_stream_copy(void* dst, const void* src, size_t bytes, int32_t blocks, int32_t reps,
                    wrs_stream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* WRS_H */
