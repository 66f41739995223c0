/*
 * sgs.h -- C ABI of the SG-Splatting tile rasterizer for NVIDIA B300 (sm_103a).
 *
 * The method (arXiv 2501.00342, SG-Splatting) renders a set of 3D Gaussians
 * {X, Sigma(q, s), opacity, colour parameters} seen from a pinhole camera into an image
 * (Sec. "Overview" and "Preliminaries": Eq. 2-3, the EWA projection the paper cites, and
 * alpha blending).  Colour is a low-degree SH term plus K spherical-Gaussian lobes
 * (Eq. 4-9).  The hot path has five stages, each a hand-written CUDA kernel:
 *   (a) per-Gaussian preprocess: EWA projection to a 2D conic, 3-sigma radius, tile
 *       rectangle, SH+SG colour                                       -> sgs_preprocess
 *   (b) tile|depth key duplication, (c) LSD radix sort of the 64-bit keys (its depth
 *       half as a sort of the records, its tile half over the instances),
 *   (d) per-tile range identification                                 -> sgs_bin_sort
 *   (e) front-to-back alpha blending per pixel                        -> sgs_render
 * and a hand-written backward pass                                    -> sgs_render_backward
 *
 * Conventions shared by every entry point:
 *  - Memory: the caller owns all device memory and streams.  No entry point allocates
 *    device or host memory.  The caller sizes the workspace with sgs_workspace_size()
 *    and keeps the filled sgs_plan (plain host struct) for the later calls.
 *  - Streams: every call enqueues work on the given stream and returns without
 *    synchronising, except sgs_bin_sort() with a non-NULL count pointer and
 *    sgs_read_device_status(), which synchronise that stream.
 *  - Errors: argument errors are returned at once (SGS_ERR_INVALID).  Errors found on
 *    the device (instance overflow, a bounded wait that ran out) are OR-ed into a
 *    status word in the workspace; read it with sgs_read_device_status().  CUDA launch
 *    errors return SGS_ERR_CUDA.  Nothing traps on the device.
 *  - Numerics: FP32 throughout.  The stages that decide integers (cull, depth bits,
 *    radius, tile rectangle, support membership) use correctly rounded FP32
 *    operations in a fixed order, so keys, sort order and ranges are reproducible
 *    bit for bit.
 *  - Views: B cameras of any resolutions are processed together ("batched"); B = 1 is
 *    the plain single-view path.  Images are planar RGB [3][H_v][W_v] per view, the
 *    views packed one after the other (view v starts at 3 * pixel_offset(v) floats).
 */
#ifndef SGS_H
#define SGS_H

#include <stddef.h>
#include <stdint.h>

#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SGS_MAX_VIEWS 64
#define SGS_MAX_SH_DEGREE 3
#define SGS_MAX_LOBES 4

typedef enum {
    SGS_OK = 0,
    SGS_ERR_INVALID = 1,  /* bad argument, size, alignment or layout */
    SGS_ERR_CAPACITY = 2, /* more (record, tile) instances than the workspace holds */
    SGS_ERR_TIMEOUT = 4,  /* a bounded device-side wait ran out (the result is invalid) */
    SGS_ERR_CUDA = 8      /* a CUDA runtime call or launch failed */
} sgs_status;

typedef enum {
    SGS_AXIS_FREE = 0,        /* each lobe has its own axis mu_k, normalised in the kernel */
    SGS_AXIS_ORTHO_FIXED = 1, /* lobes k = 0,1,2 use the world axes (Eq. 7-8 and
                                 Sec. "Implementation"); no axis is stored, K <= 3 */
    SGS_AXIS_ORTHO_FRAME = 2  /* lobes k = 0,1,2 use the columns of a per-Gaussian rotation
                                 of 3 parameters f (Sec. "Multi-Axis Orthogonal Gaussians":
                                 15 parameters for 3 orthogonal lobes): the unit quaternion
                                 (1, f0, f1, f2) / |(1, f0, f1, f2)|; sg_axis holds f as
                                 [3][stride]; K <= 3 */
} sgs_axis_mode;

/* Pinhole camera, OpenCV axes (+x right, +y down, +z forward).
 * viewmat: world->camera [R | t], 3x4 row-major.  campos: camera centre in world space
 * (the view direction of Eq. 5 is d = (X - campos)/|X - campos|).  Pixel (x, y) has its
 * centre at (x + 0.5, y + 0.5).  88 bytes. */
typedef struct {
    float viewmat[12];
    float campos[3];
    float fx, fy, cx, cy;
    int32_t width, height;
    float near_plane; /* Gaussians with view depth <= near_plane are culled */
} sgs_camera;

/* Gaussian parameters, structure of arrays, device pointers.  Each plane has n valid
 * entries and a row stride of `stride` floats (stride >= n, a multiple of 4, every
 * pointer 16-byte aligned).  Parameters are already activated: scale > 0,
 * opacity in (0, 1), sharpness lambda as given.
 *   mean     [3][stride]              X (Eq. 2)
 *   scale    [3][stride]              s (Eq. 3)
 *   rot      [4][stride]              q = (w, x, y, z), any non-zero norm (Eq. 3)
 *   opacity  [stride]
 *   sh       [(L+1)^2][3][stride]     SH coefficients c_lm per RGB channel (Eq. 4),
 *                                     basis index l*l + l + m, Condon-Shortley phase
 *   sg_amp   [K][3][stride]           lobe amplitudes alpha_k per channel (Eq. 5, 7)
 *   sg_axis  [K][3][stride]           lobe axes mu_k (free-axis mode), or [3][stride] frame
 *                                     parameters (SGS_AXIS_ORTHO_FRAME); NULL otherwise
 *   sg_sharp [K][stride]              lobe sharpness lambda_k
 * colour = max(0, sum_lm c_lm Y_lm(d) + 0.5 + sum_k alpha_k exp(lambda_k (mu_k.d - 1))).
 *
 * Adaptive SH degree (Sec. "Mixing Spherical Harmonics and Spherical Gaussians": the SH
 * degree follows the Gaussian's projected size): with sh_adaptive != 0 the record of
 * Gaussian i in view v sums the SH bands l <= D only, D = 0 if its 3-sigma radius r (the
 * integer pixel radius of the projection) < sh_radius[0], D = 1 if r < sh_radius[1],
 * else D = 2, and never above sh_degree.  Bands above D contribute nothing to that
 * record's colour and receive no gradient from it.  sh_adaptive = 0: D = sh_degree. */
typedef struct {
    int64_t n, stride;
    int32_t sh_degree; /* L in 0..3 */
    int32_t num_lobes; /* K in 0..4 (0..3 in SGS_AXIS_ORTHO_FIXED / _FRAME) */
    int32_t axis_mode; /* sgs_axis_mode */
    const float *mean, *scale, *rot, *opacity, *sh, *sg_amp, *sg_axis, *sg_sharp;
    int32_t sh_adaptive;  /* 0 or 1 */
    float sh_radius[2];   /* pixel thresholds, 0 <= sh_radius[0] <= sh_radius[1] */
} sgs_gaussians;

/* Parameter gradients, same layouts as sgs_gaussians (device pointers, overwritten). */
typedef struct {
    float *mean, *scale, *rot, *opacity, *sh, *sg_amp, *sg_axis, *sg_sharp;
} sgs_grads;

typedef struct {
    int32_t tile_w, tile_h; /* screen tile, pixels; powers of two 8..64, 64..1024 pixels;
                               over 512 pixels needs fwd_pixels and bwd_pixels >= 2 (or 0) */
    int32_t batch_depth;    /* Gaussians staged in shared memory per blend batch: 32..1024 */
    int32_t digit_bits;     /* widest radix-sort digit, 4..10: a sort of b bits takes
                               ceil(b / digit_bits) passes of equal, narrowest width */
    int32_t memory_mode;    /* 0: backward recomputes per tile from the sorted list
                               (no per-pixel contributor lists are ever stored) */
    float bg[3];            /* background colour added as T_final * bg */
    int32_t fwd_pixels;     /* pixels per thread of the forward blend: 0 (auto: 2), 1 or 2 */
    int32_t bwd_pixels;     /* pixels per thread of the backward blend: 0 (auto: 2), 1, 2 or 4
                               (4 needs tile_h a multiple of 16).  Results do not depend on
                               either (the backward's float atomics may add in another order). */
    int32_t count_pairs;    /* 1: sgs_render also writes, per pixel, the number of Gaussians
                               whose support holds it before it finished and the number it
                               blended (region SGS_REGION_PIX_COUNT); 0: not (faster).  May be
                               changed in the plan between calls. */
    int32_t persistent;     /* 1: the two-pixel blend passes (forward and backward) run as
                               persistent kernels -- as many CTAs as fit on the device at once,
                               each claiming the next tile (most expensive first) from a
                               counter in the workspace until none is left; 0: one CTA per
                               tile, in the same order.  Results do not depend on it. */
} sgs_settings;

/* Host-side plan: sizes and workspace offsets.  Filled by sgs_workspace_size(); the
 * caller owns it (stack or heap) and passes it to the stage calls.  Opaque fields. */
typedef struct {
    int64_t n, stride;
    int32_t sh_degree, num_lobes, axis_mode, B;
    sgs_settings settings;
    sgs_camera cams[SGS_MAX_VIEWS];
    int32_t tiles_x[SGS_MAX_VIEWS], tiles_y[SGS_MAX_VIEWS];
    int64_t tile_base[SGS_MAX_VIEWS + 1];  /* first global tile id of each view */
    int64_t pixel_base[SGS_MAX_VIEWS + 1]; /* first pixel of each view */
    int64_t num_records;                   /* B * n */
    int64_t num_tiles, num_pixels;
    int64_t instance_capacity;
    int32_t key_bits, sort_passes;
    int32_t stage; /* last stage run on the bound workspace: 1 preprocess, 2 bin/sort,
                      3 render; a stage call before its predecessor returns SGS_ERR_INVALID */
    cudaEvent_t* events; /* optional caller-owned array[SGS_EV_COUNT] (see sgs_set_events) */
    size_t offsets[40]; /* byte offsets of the workspace regions */
    size_t workspace_bytes;
    void* workspace; /* bound by sgs_preprocess() */
} sgs_plan;

/* Probe points between the kernels of the stage calls.  When a plan carries an event
 * array, each stage call records events[k] (if non-NULL) on its stream at point k. */
typedef enum {
    SGS_EV_PRE_BEGIN = 0, SGS_EV_PRE_END = 1,          /* preprocess kernel */
    SGS_EV_BIN_BEGIN = 2, SGS_EV_SCAN_END = 3,         /* scan of tiles touched */
    SGS_EV_DUP_END = 4,                                /* key duplication */
    SGS_EV_HIST_END = 5,                               /* sort: clears + digit histograms */
    SGS_EV_SORT_END = 6,                               /* sort: all onesweep passes */
    SGS_EV_RANGES_END = 7,                             /* clears + tile ranges */
    SGS_EV_BLEND_BEGIN = 8, SGS_EV_BLEND_END = 9,      /* blend kernel */
    SGS_EV_BWD_BEGIN = 10, SGS_EV_BWD_ZERO_END = 11,   /* the backward's tile order */
    SGS_EV_BWD_BLEND_END = 12,                         /* reverse blend */
    SGS_EV_BWD_PRE_END = 13,                           /* preprocess backward */
    SGS_EV_COUNT = 14
} sgs_event_point;

/* Attaches (events != NULL) or detaches (NULL) a caller-owned array of SGS_EV_COUNT
 * CUDA events (created by the caller, any entry may be NULL) to the plan.  Used to time
 * single kernels inside a running pipeline; the array must outlive its use. */
sgs_status sgs_set_events(sgs_plan* plan, cudaEvent_t* events);

/* Fills *plan and *bytes (device workspace size, 256-byte aligned) for n Gaussians seen
 * by B <= SGS_MAX_VIEWS cameras (host array), at most instance_capacity (record, tile)
 * instances (< 2^32).  Pure host computation.  Returns SGS_ERR_INVALID for bad sizes or
 * settings. */
sgs_status sgs_workspace_size(const sgs_gaussians* g, const sgs_camera* cams, int32_t B,
                              const sgs_settings* settings, int64_t instance_capacity,
                              sgs_plan* plan, size_t* bytes);

/* Stage (a): per (view, Gaussian) record -- cull, depth, screen mean, conic, radius,
 * tile rectangle, colour -- for all B views in one launch (parameters are read once).
 * Binds `workspace` (device, >= plan->workspace_bytes, 256-byte aligned) to the plan
 * and clears the device status word.  g must match the sizes the plan was made for.
 * The workspace keeps state from one call sequence of the plan to the next: the 2D
 * gradient accumulators, which every backward leaves zero, and the previous forward's
 * per-tile costs (a schedule hint).  Both are reset when a workspace is bound whose
 * address differs from the plan's previous one; a workspace that another plan has used
 * in between needs a new plan (sgs_workspace_size) before this one uses it again. */
sgs_status sgs_preprocess(sgs_plan* plan, const sgs_gaussians* g, void* workspace,
                          size_t ws_bytes, cudaStream_t stream);

/* Stages (b)-(d): the (global tile id << 32 | float bits of view depth, record id) pairs in
 * the order of a stable LSD radix sort of the keys, and per-tile [start, end) ranges.  The
 * sort is split: the records are sorted by depth (all instances of a record share its
 * depth), their instances are written in that order (exclusive scan of tiles touched, then
 * duplication), and a second stable sort orders the instances by tile id.  With
 * num_instances != NULL the call synchronises `stream`, stores the instance count M
 * and returns SGS_ERR_CAPACITY if M > capacity (then nothing past the scan ran
 * correctly).  With NULL it does not synchronise (graph capture); overflow is then
 * reported through the status word and the stages write nothing out of bounds. */
sgs_status sgs_bin_sort(sgs_plan* plan, int64_t* num_instances, cudaStream_t stream);

/* Stage (e): front-to-back blending of every pixel of every view.  out_rgb: device
 * float[3 * num_pixels] (planar per view); out_T: device float[num_pixels] final
 * transmittance, or NULL.  The per-pixel state the backward pass needs stays in the
 * workspace. */
sgs_status sgs_render(sgs_plan* plan, float* out_rgb, float* out_T, cudaStream_t stream);

/* Backward of (a)-(e): given dL/d(out_rgb) (device, same layout as out_rgb), writes the
 * gradient of every parameter plane of g into `out` (overwritten; sg_axis ignored in
 * ORTHO_FIXED mode).  Requires sgs_render() on the same plan and workspace before. */
sgs_status sgs_render_backward(sgs_plan* plan, const sgs_gaussians* g, const float* dL_drgb,
                               sgs_grads* out, cudaStream_t stream);

/* Synchronises `stream` and reads the device status word (an OR of sgs_status bits). */
sgs_status sgs_read_device_status(const sgs_plan* plan, int32_t* status, cudaStream_t stream);

/* Device byte offset of workspace region `which` (sgs_region) and its size; lets tests
 * and tools read intermediate results (records, keys, ranges). */
typedef enum {
    SGS_REGION_STATUS = 0,  /* int32 status, uint32 M (clamped), uint64 M (exact) ... */
    SGS_REGION_REC0 = 1,    /* float4[R]: px, py, -A/2, -B           (R = B * n) */
    SGS_REGION_REC1 = 2,    /* float4[R]: -C/2, opacity, view depth, radius */
    SGS_REGION_REC2 = 3,    /* float4[R]: r, g, b, clamp mask bits */
    SGS_REGION_RECT = 4,    /* uint2[R]:  x0 | y0 << 16, x1 | y1 << 16 (0,0 if culled) */
    SGS_REGION_TILES = 5,   /* uint32[R]: tiles touched (0 if culled) */
    SGS_REGION_OFFSETS = 6, /* uint32[R]: exclusive scan of TILES */
    SGS_REGION_KEYS = 7,    /* uint32[capacity]: global tile id of each sorted instance; the
                               full key is (tile id << 32) | float bits of the record's depth
                               (REC1.z of the record in VALS) */
    SGS_REGION_VALS = 8,    /* uint32[capacity]: sorted record ids */
    SGS_REGION_KEYS_IN = 9, /* uint32[capacity]: tile ids before the tile sort, in the order
                               of the depth-sorted records (a ping-pong buffer of the sort) */
    SGS_REGION_VALS_IN = 10,
    SGS_REGION_RANGES = 11, /* uint2[num_tiles]: [start, end) per global tile */
    SGS_REGION_PIX_T = 12,  /* float[num_pixels]: final transmittance */
    SGS_REGION_PIX_LAST = 13, /* uint32[num_pixels]: 1 + position of the last contributor
                                 in the tile's list (0: none) */
    SGS_REGION_GRAD2D = 14, /* float4[2][R] then float[R]: the reverse blend's per-record
                               pixel sums (S_x, S_y, S_xx, S_xy), (S_yy, S_1, dL/dr, dL/dg),
                               then dL/db, where S_m sums gG m over the pixels blending the
                               record below the 0.99 alpha clamp, gG = dL/dalpha exp(power),
                               m in {1, dx, dy, dx^2, dx dy, dy^2}, d = centre - pixel centre
                               (the preprocess backward turns them into dL/d(centre, conic,
                               opacity)); zero outside sgs_render_backward (its last kernel
                               clears what its reverse blend accumulated) */
    SGS_REGION_PIX_COUNT = 15, /* uint2[num_pixels]: list entries the pixel evaluated, and
                                  how many of them it blended */
    SGS_REGION_COUNT = 16
} sgs_region;
sgs_status sgs_region_info(const sgs_plan* plan, int32_t which, size_t* offset, size_t* bytes);

/* Stable LSD radix sort of m (uint64 key, uint32 value) pairs in place on their low
 * key_bits bits (1..64), the same onesweep kernels sgs_bin_sort uses; digit_bits (4..10)
 * is the widest digit.  `temp` is device
 * scratch of at least sgs_sort_temp_bytes(m, key_bits, digit_bits) bytes.  Exposed for
 * tests of the sort alone. */
sgs_status sgs_sort_temp_bytes(int64_t m, int32_t key_bits, int32_t digit_bits, size_t* bytes);
sgs_status sgs_sort_pairs(uint64_t* keys, uint32_t* vals, int64_t m, int32_t key_bits,
                          int32_t digit_bits, void* temp, size_t temp_bytes,
                          cudaStream_t stream);

/* sgs_sort_pairs for 32-bit keys (key_bits <= 32), with the same scratch size
 * (sgs_sort_temp_bytes).  This is the kernel instantiation the rasterizer runs on its
 * 32-bit depth and tile-id keys.  Exposed for tests of the sort alone. */
sgs_status sgs_sort_pairs32(uint32_t* keys, uint32_t* vals, int64_t m, int32_t key_bits,
                            int32_t digit_bits, void* temp, size_t temp_bytes, cudaStream_t stream);

/* Radix sort that allocates nothing and takes no scratch argument.  The paper has no
 * counterpart to this entry point; it exists for callers that may not obtain device
 * memory themselves -- e.g. a host that owns every device allocation through its own pool
 * or budget, or code that runs where a cudaMalloc would be refused or would stall other
 * work.  It sorts like sgs_sort_pairs (same kernels, same stable result on the low
 * key_bits bits, in place), but its scratch is one file-scope device array of
 * SGS_SORT_NOALLOC_SCRATCH_BYTES that every GPU which loads the library holds until the
 * process exits.
 *  - m must not exceed SGS_SORT_NOALLOC_MAX_PAIRS; a larger m (or other bad argument)
 *    returns SGS_ERR_INVALID and enqueues nothing.
 *  - digit_bits must be 4..8 (sgs_sort_pairs takes up to 10): the histogram, offset and
 *    look-back tables of the fixed array are sized for digits of at most 8 bits (radix
 *    256, up to 16 passes); 9 or 10 returns SGS_ERR_INVALID.
 *  - A bounded look-back wait that ran out (SGS_ERR_TIMEOUT in sgs_sort_pairs's status
 *    word) is not reported by this entry point: the status word lives in the fixed array,
 *    which no entry point reads back.  Such a wait only runs out after about a second of
 *    polling an unpublished slot, which a healthy GPU does not do.
 *  - The first call on a device looks up the array's device address
 *    (cudaGetSymbolAddress) with that device current; make that first call before any
 *    stream capture on the device.  A failed lookup returns SGS_ERR_CUDA.
 *  - All calls share the one array, so calls whose work overlaps on the GPU (different
 *    streams, no ordering between them) race and give wrong results; serialise them.
 *  - The array keeps the previous call's contents; each call clears what it reads first.
 *  - No cudaMalloc, cudaFree or allocating library routine is called. */
#define SGS_SORT_NOALLOC_MAX_PAIRS (1 << 18)
#define SGS_SORT_NOALLOC_SCRATCH_BYTES 3320320
sgs_status sgs_sort_pairs_noalloc(uint64_t* keys, uint32_t* vals, int64_t m, int32_t key_bits,
                                  int32_t digit_bits, cudaStream_t stream);

/* Mean absolute error loss of a rendered image against a target, and its gradient:
 * loss[0] = sum |img - target| / count (device float, written), dL_dimg = sign(img -
 * target) / count (sign(0) = 0).  Used for the differentiable training step. */
sgs_status sgs_l1_loss(const float* img, const float* target, int64_t count, float* loss,
                       float* dL_dimg, cudaStream_t stream);

/* sgs_l1_loss with the normaliser given: loss[0] = scale * sum |img - target|, dL_dimg =
 * scale * sign(img - target), scale >= 0 (else SGS_ERR_INVALID).  In view-sharded
 * training each rank renders its own views and passes scale = 1 / (the pixel values of
 * all ranks' views), so that the sum over ranks of the losses and of the parameter
 * gradients is the mean absolute error over every view and its gradient. */
sgs_status sgs_l1_loss_scaled(const float* img, const float* target, int64_t count, float scale, float* loss,
                              float* dL_dimg, cudaStream_t stream);

/* ---- Training: fused Adam step over the parameter planes ----
 * The optimiser works on raw planes (same layouts as sgs_gaussians): scale holds log s and
 * opacity holds logit o (the 3D-GS activations), every other plane is the parameter
 * itself.  One call updates every entry of every plane with Adam (Kingma & Ba 2015):
 *   g  = dL/d(raw) = dL/d(act) * act'(raw)   (exp for scale, sigmoid for opacity)
 *   m  = b1 m + (1 - b1) g,   v = b2 v + (1 - b2) g^2
 *   raw -= lr * (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps)
 *   act = exp(raw) | sigmoid(raw) | raw
 * with the learning rate lr and step t of the entry's group.  A group whose lr is 0 is
 * left untouched (raw, act, m and v): the paper trains the SG lobes only after the first
 * 2,000 iterations, with lr 0.0025 (Sec. "Implementation"), and gives them their own step
 * count from then on.  grad is sgs_render_backward's output (w.r.t. the activated
 * parameters, the ones the renderer reads from `act`).  act planes of identity groups may
 * alias the raw planes.  m and v start at zero (caller-owned).  Asynchronous. */
typedef enum {
    SGS_GROUP_MEAN = 0, SGS_GROUP_SCALE, SGS_GROUP_ROT, SGS_GROUP_OPACITY, SGS_GROUP_SH_DC,
    SGS_GROUP_SH_REST, SGS_GROUP_SG, SGS_GROUP_COUNT
} sgs_param_group;

typedef struct {
    float lr[SGS_GROUP_COUNT];
    int32_t step[SGS_GROUP_COUNT]; /* t >= 1 of each group with lr > 0 */
    float beta1, beta2, eps;
} sgs_adam_config;

sgs_status sgs_adam_step(const sgs_gaussians* layout, const sgs_grads* raw, const sgs_grads* act,
                         const sgs_grads* grad, const sgs_grads* m, const sgs_grads* v,
                         const sgs_adam_config* cfg, cudaStream_t stream);

/* Failure-detection self-test of the bounded device-side waits; the paper has no
 * counterpart.  The scan and the radix sort find each tile's prefix by decoupled look-back,
 * polling a predecessor's 8-byte slot until it is published; every such wait gives up
 * after a fixed number of polls (about a second of GPU time) and sets SGS_ERR_TIMEOUT
 * instead of hanging.  This call runs that same wait once, on one GPU thread, over
 * `num_slots` caller-owned device slots, walking back from slots[num_slots - 1] to
 * slots[0]; a slot is (flag << 62) | value with flag 1 = aggregate (add, keep walking),
 * 2 = inclusive prefix (add, stop), anything else = not yet published (poll again).
 *   sum    device uint64: the sum found (partial after a timeout)
 *   status device int32: SGS_OK, or SGS_ERR_TIMEOUT when a slot was never published
 * The kernel always returns, so the context stays usable.  Arguments are checked on the
 * host (SGS_ERR_INVALID for num_slots < 0 or a null pointer); asynchronous on `stream`. */
sgs_status sgs_selftest_lookback(const uint64_t* slots, int64_t num_slots, uint64_t* sum,
                                 int32_t* status, cudaStream_t stream);

/* Measurement helper (the paper has no counterpart): the device's FP32 arithmetic
 * throughput, the peak against which the blend kernels (bound by the FP32 pipes and issue
 * slots) are reported.  One launch of sgs_alu_probe_size() threads (a multiple of the
 * multiprocessor count), each running 8 independent chains of `iters` multiply-adds,
 * scalar fma.rn.f32 (packed = 0) or packed fma.rn.f32x2 (packed = 1, two FP32 operations
 * per instruction).  out: device float[threads] (written, prevents dead-code removal);
 * *fp32_ops: the FP32 operations enqueued (a multiply-add counted as one), for the caller
 * to divide by the launch time it measures with CUDA events.  Asynchronous on `stream`. */
sgs_status sgs_alu_probe_size(int64_t* threads);
sgs_status sgs_alu_probe(int32_t packed, int32_t iters, float* out, double* fp32_ops, cudaStream_t stream);

const char* sgs_status_string(sgs_status s);

/* sizeof(sgs_plan), sizeof(sgs_camera), sizeof(sgs_gaussians), sizeof(sgs_settings),
 * sizeof(sgs_adam_config), sizeof(sgs_grads) in that order into sizes[6]: lets a
 * foreign-language binding check its struct layouts. */
void sgs_abi_sizes(size_t* sizes);

#ifdef __cplusplus
}
#endif
#endif /* SGS_H */
