/*
 * fvv.h — C ABI of the B300 VINet view-interpolation library (libfvv.so).
 *
 * The operation: given two adjacent camera frames I_left, I_right (H x W RGB)
 * and a viewpoint position t in [0, 1], synthesise the virtual view between
 * them with VINet (arXiv 2112.10603, Sec. 3.1): three VIBlocks estimate the
 * bidirectional flow F_m->l, F_m->r and an occlusion mask M coarse to fine
 * (Eq. 2, Table 3), the frames are backward-warped and blended
 * (Eq. 1:  I_mid(u) = M(u) I_l(u + F_m->l(u)) + (1 - M(u)) I_r(u + F_m->r(u))),
 * and a context-aware U-Net adds a residual (Sec. 3.1 "Refinement Network").
 * The paper interpolates the midpoint and reaches other positions by stacking
 * (Sec. 4.2); here t is also fed to every VIBlock as a constant input plane, so
 * one call can serve any set of positions (t = 0.5 is the paper's midpoint).
 *
 * Conventions shared by every call:
 *  - images are H x W x 3 float32, channels fastest (HWC), values in [0, 1];
 *    several views are stored back to back (n x H x W x 3);
 *  - sizes are padded internally to multiples of 16 with zeros on the bottom and
 *    right, and the output is cropped back to H x W;
 *  - all calls return 0 on success or a negative FVV_E* code; nothing throws
 *    across the ABI; fvv_last_error() returns the calling thread's last message;
 *  - `stream` is a cudaStream_t passed as void*; NULL means the legacy default
 *    stream.  run calls are asynchronous on that stream and never synchronise
 *    unless stated;
 *  - an fvv_interp handle owns its device workspace, is used by one stream at a
 *    time and is not thread-safe; the server (fvv_serve_*) is thread-safe.
 */
#ifndef FVV_H
#define FVV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    FVV_OK = 0,
    FVV_EINVAL = -1,      /* bad argument (NULL pointer, t outside [0,1], bad enum) */
    FVV_ESHAPE = -2,      /* H, W, n_views or weight count out of range */
    FVV_ENOMEM = -3,      /* device or host allocation failed */
    FVV_ECUDA = -4,       /* a CUDA call failed; the message names it */
    FVV_EBUSY = -5,       /* admission refused: the HBM budget or queue is full */
    FVV_ETIMEOUT = -6,    /* a bounded device wait gave up (kernel error flag) */
    FVV_ESUPERSEDED = -7, /* request replaced by a newer one from the same user */
    FVV_ENOTFOUND = -8    /* unknown ticket */
};

enum { FVV_FP32 = 0, FVV_BF16 = 1, FVV_FP8 = 2 };   /* convolution precision */
enum { FVV_PAD_ZERO = 0, FVV_PAD_CIRCULAR = 1 };   /* border handling */
enum { FVV_T_DIRECT = 0, FVV_T_RECURSIVE = 1 };    /* viewpoint handling */

typedef struct {
    int precision; /* FVV_FP32 (SIMT FP32 FMA), FVV_BF16 (tcgen05, FP32 accumulate), FVV_FP8 */
    int pad_mode;  /* FVV_PAD_ZERO: zero conv padding, border-clamped sampling;
                      FVV_PAD_CIRCULAR: everything wraps (needs H, W multiples of 16) */
    int t_mode;    /* FVV_T_DIRECT: the t plane of every VIBlock = t;
                      FVV_T_RECURSIVE: the paper's dense views (Sec. 4.2): only the
                      midpoint network (t plane 0.5) is run, recursively — the view at
                      t = k / 2^n (k odd, n <= 12) is the midpoint of its neighbours at
                      spacing 1 / 2^n; n stages give 2^n - 1 views.  fvv_interp_run
                      only; every dyadic level is one batched forward */
    int max_views; /* views per run call the workspace is sized for (>= 1) */
    int max_cams;  /* cameras per batched call (>= 2) */
    int graphs;    /* 1: each run replays a CUDA graph captured on first use for its
                      view-count bucket (the next power of two of the call's views, at
                      most max_views; launches sized for max_cams cameras): the kernels
                      read the call's view and camera counts from device memory and
                      skip the rest of their grid, so any mix of counts replays one of
                      at most 1 + log2(max_views) graphs; 0: launch kernels directly */
} fvv_opts;

typedef struct fvv_interp fvv_interp;

/* Default options: FP32, zero padding, direct t, max_views 16, max_cams 2, graphs on. */
void fvv_default_opts(fvv_opts *opts);

/* Create an interpolator for H x W frames.
 * weights: host float32 blob, n_floats values, layers in Table 3 order (VIBlock 0,
 *   1, 2, ContextNet, RefineNet), per layer W then b; conv W [Co][Ci][3][3],
 *   convT W [Ci][Co][4][4].  Copied (and packed) at create; the caller keeps it.
 * Returns FVV_ESHAPE if n_floats does not match the architecture or H, W are
 * outside [16, 8192] (circular mode: not multiples of 16). */
int fvv_interp_create(const float *weights, size_t n_floats, int H, int W,
                      const fvv_opts *opts, fvv_interp **out);

/* Synthesise n_views views between one camera pair.
 * left, right: DEVICE pointers, H x W x 3 float32 each (caller-owned).
 * t: HOST array of n_views positions in [0, 1] (0 = left camera, 1 = right).
 * out: DEVICE pointer, n_views x H x W x 3 float32 (caller-owned).
 * Asynchronous on `stream`.  n_views in [1, max_views]. */
int fvv_interp_run(fvv_interp *h, const float *left, const float *right, const float *t,
                   int n_views, float *out, void *stream);

/* Same as fvv_interp_run with HOST buffers: copies left/right to the device,
 * runs, copies the views back into out (host), and synchronises `stream`.
 * Page-locked host memory gives asynchronous copies; pageable memory works too. */
int fvv_interp_run_host(fvv_interp *h, const float *left, const float *right, const float *t,
                        int n_views, float *out, void *stream);

/* Pipelined form of fvv_interp_run_host: enqueues the copy of left/right (HOST, H x W x 3
 * float32) to the device, the forward on `stream` and the copy of the views back into out
 * (HOST, n_views x H x W x 3 float32), and returns without waiting; *ticket receives the
 * call's number (0, 1, 2, ... per handle).  The copies run on the handle's own copy streams,
 * so the copy-out of one call overlaps the forward of the next.  Two calls are in flight at
 * most: a call first waits (host) until the call two before it has delivered its views.
 * left, right and out stay owned by the caller and must not be touched until
 * fvv_interp_wait_host(h, ticket) has returned; page-locked memory is needed for the
 * copies to overlap (pageable memory works, serialised).
 * Errors: FVV_EINVAL (NULL argument, t outside [0, 1]), FVV_ESHAPE (n_views), FVV_ECUDA. */
int fvv_interp_submit_host(fvv_interp *h, const float *left, const float *right, const float *t,
                           int n_views, float *out, void *stream, long long *ticket);

/* Block until the host-buffer call `ticket` has written its views into its out buffer.
 * A ticket that was never issued by this handle gives FVV_EINVAL. */
int fvv_interp_wait_host(fvv_interp *h, long long ticket);

/* Batched rig instant: n_cams frames, n_pairs camera pairs, uneven views per pair.
 * cams: HOST array of n_cams DEVICE pointers (H x W x 3 float32 each).
 * pair_left: HOST, n_pairs camera indices; pair p uses cams pair_left[p] and
 *   pair_left[p] + 1.
 * view_offsets: HOST, n_pairs + 1 prefix offsets; pair p owns views
 *   [view_offsets[p], view_offsets[p+1]).
 * t: HOST, view_offsets[n_pairs] positions.  out: DEVICE, total views x H x W x 3.
 * All views of the call run as one batch (every layer one launch over all views);
 * the total must not exceed max_views and n_cams must not exceed max_cams. */
int fvv_interp_run_batch(fvv_interp *h, const float *const *cams, int n_cams,
                         const int *pair_left, const int *view_offsets, const float *t,
                         int n_pairs, float *out, void *stream);

/* Bytes of device memory the handle holds (weights + workspace). */
size_t fvv_interp_device_bytes(const fvv_interp *h);

/* Number of kernel launches the last run call issued. */
int fvv_interp_last_launches(const fvv_interp *h);

/* Number of CUDA graphs the handle has captured so far (opts.graphs = 1). */
long long fvv_interp_graph_captures(const fvv_interp *h);

/* Copy an intermediate of view `view` from the last run into `dst` (HOST,
 * float32), synchronising the device first.  which: 0, 1, 2 = stage s flows and
 * mask logit F^s, M^s (Eq. 2; Hp/2^(2-s) x Wp/2^(2-s) x 5, padded grid);
 * 3 = I_blend (Eq. 1; Hp x Wp x 3); 4 = RefineNet output z before the sigmoid
 * (Hp x Wp x 3).  n_floats must equal the size of that tensor (FVV_ESHAPE
 * otherwise).  For tests and debugging; not needed on the product path. */
int fvv_interp_peek(fvv_interp *h, int which, int view, float *dst, size_t n_floats);

/* Run one layer of Table 3 (index 0..50, blob order) alone on caller buffers,
 * with the handle's weights and precision: a 3x3 pad-1 conv (stride 1 or 2) or
 * a 4x4 stride-2 pad-1 transposed conv, + bias, + ReLU where Table 3 has one.
 * in: DEVICE, n x H x W pixels, pixel stride in_cs elements, the layer's C_in
 *   channels starting at in_coff; float32 on the FP32 path, bfloat16 otherwise
 *   (then in_cs, in_coff multiples of 8 and, for C_in < 16 or 17..31, the
 *   channels up to 16 / 32 readable, their weights being zero).  ContextNet's
 *   first layer (index 30, 3 input channels) always takes float32 input.
 * out: DEVICE, n x Ho x Wo pixels, pixel stride out_cs, written at out_coff;
 *   float32 if out_f32 or on the FP32 path, else bfloat16.
 * Asynchronous on `stream`.  Used by the kernel-level tests. */
int fvv_interp_layer(fvv_interp *h, int layer, const void *in, int in_cs, int in_coff, int n, int H, int W,
                     void *out, int out_cs, int out_coff, int out_f32, void *stream);

/* One layer of Table 3 with no device allocation at all (the paper has no
 * counterpart: this exists for callers that may not allocate device memory —
 * an application that owns a fixed device-memory budget, a real-time loop that
 * cannot risk the synchronisation an allocation may cause, or a plug-in living in
 * another framework's memory pool; such callers cannot create an fvv_interp).
 * Same operation and FP32 arithmetic as fvv_interp_layer on an FP32 handle, but
 * the weights come from the caller:
 *   w: DEVICE, the layer's weights in the blob layout (conv [Co][Ci][3][3],
 *      convT [Ci][Co][4][4]), float32;  b: DEVICE, Co float32 biases;
 *   in / out: DEVICE float32, as for fvv_interp_layer (zero padding).
 * The repacked weights live in a fixed device array of 2^20 floats (4 MiB, the
 * largest layer of Table 3) that every GPU loading the library keeps until exit;
 * a layer with more weights is rejected with FVV_ESHAPE.  All calls share that
 * array and it keeps the last call's contents, so calls that overlap on the GPU
 * (different streams, or another thread) race: serialise them.  The first call on
 * a device loads this entry point's module, which is when the driver creates the
 * array on that device (that step may synchronise the device), and looks up the
 * array's device address (with that device current).  So make one warm-up call per
 * device at initialisation, before any stream capture and outside any real-time
 * loop; calls after it allocate nothing.  `stream` must belong to the current
 * device (FVV_EINVAL otherwise).  Asynchronous on `stream`. */
int fvv_layer_noalloc(int layer, const float *w, const float *b, const float *in, int in_cs, int in_coff, int n,
                      int H, int W, float *out, int out_cs, int out_coff, void *stream);

/* Multi-view cluster frame (the paper's multiview organizer, Sec. 3.2): the real
 * view of one camera and the views of its neighbourhood along the arc, tiled into
 * one frame for a tile-based encoder.
 *   center: DEVICE, H x W x 3 float32 (the camera's real view).
 *   side_views: HOST array of 2 * n_side DEVICE pointers (H x W x 3 float32 each), in
 *     arc order: the left neighbour camera, the views between it and the centre,
 *     then the views between the centre and the right neighbour, the right camera
 *     (the paper uses n_side = 16: 15 interpolated views + the neighbour per side).
 *   out: DEVICE, W x (H + R * H / scale) x 3 float32 with R = ceil(2 n_side / scale):
 *     rows [0, H) = center; tile k (0 <= k < 2 n_side) = side view k downscaled by the
 *     scale x scale box average, at rows H + (k / scale) * H / scale, columns
 *     (k % scale) * W / scale; unused tiles are zero.
 * Errors: FVV_ESHAPE unless 1 <= n_side <= 64 and scale divides H and W; FVV_EINVAL
 * for NULL pointers.  Asynchronous on `stream`; allocates nothing.  This operation
 * is the system's stitching step, not part of the view interpolation network. */
int fvv_stitch_cluster(const float *center, const float *const *side_views, int n_side, int H, int W, int scale,
                       float *out, void *stream);

/* Laplacian-pyramid loss of Eq. 3 (Sec. 3.1 "Loss functions"), forward only, for n
 * image pairs: loss[v] = sum_{i=1..5} 2^(i-1) || L^i(pred_v) - L^i(gt_v) ||_1, where
 * L^i is level i of the Laplace pyramid (the paper names the pyramid, not its filter:
 * here the Burt-Adelson pyramid of the binomial kernel [1 4 6 4 1]/16 with replicated
 * edges, each level ceil(H/2) x ceil(W/2) of the one before, L^5 = the fifth low-pass
 * image) and ||.||_1 sums |.| over every pixel and channel of the level.
 *   pred, gt: DEVICE, n x H x W x 3 float32 (HWC), e.g. fvv_interp_run's views and the
 *     ground truth;
 *   workspace: DEVICE, at least fvv_lap_loss_workspace(n, H, W) bytes, 256-byte
 *     aligned, owned by the caller (the lower pyramid levels and the partial sums);
 *   loss: DEVICE, n float32 (or NULL); level_norms: DEVICE, n x 5 float32, the five
 *     L1 norms per pair in level order (or NULL; not both NULL).
 * The result does not depend on the launch or the order of blocks (fixed-order sums).
 * Errors: FVV_EINVAL for NULL pointers or a short / misaligned workspace, FVV_ESHAPE
 * unless 1 <= n <= 65535, H, W >= 2 and H x W <= 2^28.  Asynchronous on `stream`;
 * allocates nothing. */
size_t fvv_lap_loss_workspace(int n, int H, int W);
int fvv_lap_loss(const float *pred, const float *gt, int n, int H, int W, void *workspace, size_t workspace_bytes,
                 float *loss, float *level_norms, void *stream);

/* Synchronise the device and report whether any bounded device-side wait of
 * this handle's kernels gave up since the last call (FVV_ETIMEOUT, flag then
 * cleared) or a CUDA error is pending (FVV_ECUDA); FVV_OK otherwise. */
int fvv_interp_status(fvv_interp *h);

/* Fault injection for tests of the failure detection (the paper has no counterpart;
 * its system claims elasticity without a mechanism, Sec. 3.2).  Arms the NEXT
 * fvv_interp_layer call on this handle: in its tensor-core kernel the MMA warp first
 * waits on a shared-memory barrier that nothing signals, for at most `cycles` SM
 * clock cycles.  The wait runs out, the kernel records code 6 in the handle's error
 * word, the other warp roles stop, the copies already issued land, TMEM is freed and
 * the kernel returns without writing its output; fvv_interp_status then returns
 * FVV_ETIMEOUT and clears the word.  No GPU fault is involved and the context stays
 * usable.  The knob is never live inside fvv_interp_run (so no captured graph holds
 * it) and has no effect on the FP32 path, whose kernels have no waits.
 * cycles in [1000, 2^31], else FVV_EINVAL. */
int fvv_interp_inject_stall(fvv_interp *h, long long cycles);

/* FP8 calibration (FVV_FP8 handles only; required before their first run).
 * On FP8 handles every VIBlock conv with 128 or 256 input channels -- c1, the six
 * 256 -> 256 convs and the transposed t0 and t1 (90% of the FLOPs, Table 3) -- runs with
 * E4M3 operands and FP32 accumulation: weights carry one scale
 * per output channel, s_w = max |w| / 448, fixed at create; each such conv's input
 * carries one scale per tensor, s_a = (max |input| over the calibration views) /
 * 448, measured here by running the network in BF16 on n_pairs frame pairs at
 * t = 0.25, 0.5, 0.75.  The producing layer writes E4M3 codes of value / s_a
 * (round to nearest even, saturating); the epilogue dequantises by s_a * s_w[co].
 * frames: DEVICE, n_pairs x 2 x H x W x 3 float32 (left, right of each pair).
 * Synchronises `stream`.  Every other layer and all sampling stay as on FVV_BF16. */
int fvv_calibrate_fp8(fvv_interp *h, const float *frames, int n_pairs, void *stream);

/* Scales of an FP8 layer after calibration: *s_a (input, per tensor) and the first
 * n per-output-channel weight scales s_w.  For tests and inspection. */
int fvv_interp_fp8_scales(fvv_interp *h, int layer, float *s_a, float *s_w, int n);

/* Tile autotuner: times every candidate tile rectangle (128 or 256 output pixels,
 * width 8 ... 256) of every tensor-core layer on a forward of n_views views (with
 * the per-layer events of fvv_interp_profile) and keeps the fastest per layer.
 * cache_path (may be NULL): a JSON file of earlier results keyed by frame size,
 * view count and precision; a matching entry is loaded instead of measuring, and
 * new results are added to the file.  Synchronises the device.  No effect on the
 * FP32 path (its kernel has no tile choice). */
int fvv_interp_autotune(fvv_interp *h, int n_views, const char *cache_path);

/* Per-layer timing (the analogue of the paper's per-module latency, Table 2).
 * fvv_interp_profile(h, 1) brackets every convolution launch of later runs with
 * CUDA events on the run's stream (small overhead); 0 turns it off.  Both reset
 * the counters.  fvv_interp_layer_stats synchronises those events and writes,
 * per layer of Table 3 (n = 51 entries, blob order), the summed kernel time in ms,
 * the summed algorithmic FLOPs (2 x MACs of the unpadded layer) and the number
 * of launches since the last reset; any pointer may be NULL. */
int fvv_interp_profile(fvv_interp *h, int enable);
int fvv_interp_layer_stats(fvv_interp *h, double *ms, double *flops, int *launches, int n);

void fvv_interp_destroy(fvv_interp *h);

/* ------------------------------------------------------------------------
 * Multi-user server: continuous batching of viewpoint requests.
 *
 * The paper's edge media server serves many users from one GPU and organises its
 * modules around FIFO data channels (Sec. 2, Sec. 3.2, supplement S.1).  Here a
 * request = (user, camera pair, t, resolution) -> one synthesised view in device
 * memory.  Per resolution the server holds `slots_per_res` interpolators, each on
 * its own stream: whenever a slot is free the scheduler thread takes up to
 * `max_batch` queued requests of that resolution and runs them as one batched
 * forward, so requests arriving while others run are admitted as slots free up.
 * A new request from a user replaces that user's request still waiting in the
 * queue (latest wins; the old ticket polls FVV_ESUPERSEDED).  Admission: every
 * admitted request holds a view-sized output buffer from a per-resolution pool of
 * `pool_views` buffers, cut to fit `hbm_budget` (bytes, 0 = no limit) after the
 * slots' workspaces; an empty pool makes submit return FVV_EBUSY.  The server is
 * thread-safe.  With fake_ms_per_view > 0 no GPU is used (batches just take
 * fake_ms_per_view per view on the host): for testing the scheduling logic.
 *
 * Dense mode (dense_levels = n > 0; the paper's serving scheme, Sec. 3.2 and the
 * n-stage dense views of Sec. 4.2): for every capture instant the server renders
 * the fixed set t = k / 2^n, k = 1 .. 2^n - 1, of every camera pair once (batches
 * of whole pairs, 2^n - 1 <= max_batch), into one of two per-resolution stores
 * (the newest complete instant is served from one while the next renders into the
 * other).  A request's t snaps to the nearest k / 2^n; k = 0 or 2^n answer with the
 * camera frame itself.  A request is answered at once from the newest complete set
 * when that set belongs to the newest frames (set_frames), else by the first set
 * completed after it arrives; the GPU load does not depend on the number of users.
 * With dense_immediate = 1 a request is answered at once from the newest complete set
 * whatever instant it shows (a set exists once the first instant has rendered); the
 * stats then give, beside the request latency, the age of the answered content (ms
 * from the set_frames call of its instant to the answer) and its staleness (instants
 * between it and the newest frames).  Its view pointer stays valid until the server starts rendering the
 * second instant after it; release() only forgets the ticket.  Frames passed to
 * set_frames must stay valid until their instant has been rendered. */

#define FVV_SERVE_MAX_RES 4

typedef struct {
    int precision;                  /* FVV_BF16, FVV_FP32 or FVV_FP8 (then fvv_serve_calibrate_fp8) */
    int n_res;                      /* resolutions served, 1 .. FVV_SERVE_MAX_RES */
    int res_h[FVV_SERVE_MAX_RES], res_w[FVV_SERVE_MAX_RES];
    int n_cams;                     /* cameras of the rig; pair p = cameras p, p + 1 */
    int slots_per_res;              /* concurrent batches per resolution */
    int max_batch;                  /* views per batch */
    int pool_views;                 /* output buffers per resolution (before the budget cut) */
    size_t hbm_budget;              /* device bytes the server may hold; 0 = unlimited */
    double fake_ms_per_view;        /* > 0: no GPU, simulated batches (tests) */
    int dense_levels;               /* 0: render each request; n > 0: dense mode, 2^n - 1 views per pair */
    int dense_immediate;            /* dense mode: 1 = answer from the newest complete set at once */
} fvv_serve_cfg;

typedef struct {
    long long submitted, completed, superseded, rejected, failed, batches, batched_views, queued;
    double p50_ms, p99_ms, max_ms;  /* latency submit -> view ready, completed requests */
    size_t device_bytes;
    long long dense_instants;       /* dense mode: instants whose view set was rendered */
    double age_p50_ms, age_p99_ms;  /* dense mode: age of the answered content (set_frames -> answer) */
    double stale_mean;              /* dense mode: mean instants between the answered set and the newest frames */
    long long stale_max;
} fvv_serve_stats;

typedef struct fvv_server fvv_server;

/* Defaults: BF16, one resolution 1080 x 1920, 9 cameras, 2 slots, batches of 8,
 * 64 pooled output views, no budget limit, real GPU. */
void fvv_serve_default_cfg(fvv_serve_cfg *cfg);

/* weights: as for fvv_interp_create (may be NULL with fake_ms_per_view > 0). */
int fvv_serve_create(const float *weights, size_t n_floats, const fvv_serve_cfg *cfg, fvv_server **out);

/* FP8 servers (precision FVV_FP8): the activation scales of every slot of resolution
 * res_id, measured as fvv_calibrate_fp8 does (frames: DEVICE, n_pairs x 2 x H x W x 3
 * float32 at that resolution).  Required before the first set_frames of that
 * resolution; FVV_EBUSY if one of its slots is running. */
int fvv_serve_calibrate_fp8(fvv_server *s, int res_id, const float *frames, int n_pairs);

/* Frames of capture instant `instant` at resolution res_id: n_cams DEVICE pointers
 * (H x W x 3 float32, caller-owned, kept valid until replaced).  Batches use the
 * frames set last; a slot reuses its pyramid and ContextNet features while the
 * instant is unchanged. */
int fvv_serve_set_frames(fvv_server *s, int64_t instant, int res_id, const float *const *cams_dev);

/* Queue a request; *ticket identifies it.  FVV_EBUSY when the output pool is full. */
int fvv_serve_submit(fvv_server *s, int user, int pair, float t, int res_id, uint64_t *ticket);

/* 0 = done (*out_dev: the view, H x W x 3 float32 DEVICE, valid until release;
 * *latency_ms: submit -> ready), 1 = pending, FVV_ESUPERSEDED, FVV_ENOTFOUND, or
 * FVV_ECUDA if its batch failed. */
int fvv_serve_poll(fvv_server *s, uint64_t ticket, const float **out_dev, double *latency_ms);

/* Forget a finished ticket and return its output buffer to the pool (1 if still pending). */
int fvv_serve_release(fvv_server *s, uint64_t ticket);

int fvv_serve_stats_get(fvv_server *s, fvv_serve_stats *out);

/* Stops the scheduler, waits for batches on the device, frees everything. */
void fvv_serve_destroy(fvv_server *s);

/* Thread-local message of the last failing call on this thread ("" if none). */
const char *fvv_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* FVV_H */
