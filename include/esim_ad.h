/*
 * esim_ad.h - C ABI of the GB300 (sm_103a) event-camera simulator with adaptive
 * weighted-local-regression denoising (Tsuji, Yatagawa, Kubo, Morishima,
 * "Event-based Camera Simulation using Monte Carlo Path Tracing with Adaptive
 * Denoising", arXiv 2303.02608).
 *
 * The library turns noisy path-traced frames (radiance plus first-bounce
 * normal, depth and albedo buffers, Section 3) into DVS events (Eq. 1).  Per
 * pixel and frame it
 *   1. converts radiance to log brightness y = ln(Y + eps) (Section 1.1, 2.1),
 *   2. tests, with the model kept from the pixel's last event, whether the
 *      brightness change can reach C: Delta R = (beta^T (x^c - xhat^c))^2 >= C^2
 *      (Proposition 1, Eqs. 6-9),
 *   3. for flagged pixels only, solves the first-order weighted local
 *      regression of Eqs. 3-5 over a (2r+1)^2 x T spatio-temporal window,
 *   4. emits floor(|alpha - L_last| / C) events of polarity sign(alpha - L_last)
 *      at the frame time (Eq. 1, Section 3 footnote) and, after an event,
 *      replaces the pixel's model (Fig. 1, Section 3).
 * In exhaustive mode step 2 is skipped and every pixel is regressed every
 * frame (the WLR+ESIM baseline of Section 3).
 *
 * Conventions for every entry point:
 *   - All functions return esim_ad_status; output pointers are left untouched
 *     on error.  No function throws, aborts or prints.
 *   - Work is enqueued on the CUDA stream given to esim_ad_init and runs
 *     asynchronously; only the functions documented as synchronising wait for
 *     it.  Errors raised by asynchronous device work surface at the next
 *     synchronising call.
 *   - ESIM_AD_EOVERFLOW (device event buffer overflowed) and ESIM_AD_ETIMEOUT
 *     (a bounded device wait expired) are sticky: every later call except
 *     esim_ad_stats, esim_ad_reset and esim_ad_destroy returns ESIM_AD_ESTATE.
 *   - Planar image buffers are [channel][height][pitch], row-major; the pitch
 *     is esim_ad_frame.pitch_elems (0 = width, densely packed).
 *   - A context is not thread-safe; use one context per host thread.
 */
#ifndef ESIM_AD_H
#define ESIM_AD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct esim_ad_ctx esim_ad_ctx;   /* opaque, owned by the library */

typedef enum esim_ad_status {
    ESIM_AD_OK = 0,
    ESIM_AD_EINVAL = -1,      /* bad argument or configuration                 */
    ESIM_AD_ENOMEM = -2,      /* device or host allocation failed              */
    ESIM_AD_ECUDA = -3,       /* a CUDA runtime/driver call failed             */
    ESIM_AD_EOVERFLOW = -4,   /* device event buffer overflowed (sticky)       */
    ESIM_AD_ETIMEOUT = -5,    /* a bounded device wait expired (sticky)        */
    ESIM_AD_ESTATE = -6,      /* context unusable after a sticky error         */
    ESIM_AD_ENOSPACE = -7     /* caller's buffer too small; *n_out = required  */
} esim_ad_status;

enum { ESIM_AD_ADAPTIVE = 0, ESIM_AD_EXHAUSTIVE = 1 };
/* radiance input: linear luminance, linear RGB (Rec.709 luminance is taken), or
 * log brightness y = ln(Y + eps) already computed by the renderer, as FP16 */
enum { ESIM_AD_LUMA_F32 = 0, ESIM_AD_RGB_F32 = 1, ESIM_AD_LOGLUMA_F16 = 2 };
/* feature input: separate float32 planes, or one [7][H][W] BF16 stack
 * (normal xyz, depth, albedo rgb) whose values are multiplied by feature_scale */
enum { ESIM_AD_FEAT_F32 = 0, ESIM_AD_FEAT_BF16 = 1 };
/* arithmetic form: FP32 storage and solve, or the mixed form (FP16 log
 * brightness and BF16 features in the frame ring, FP32 accumulation, FP32
 * Cholesky with one refinement step, FP64 re-solve when the estimated
 * condition number exceeds 1e6) */
enum { ESIM_AD_FP32 = 0, ESIM_AD_MIXED = 1 };

/*
 * Simulation parameters.  Paper symbols: C (Eq. 1), h and b_j (Eq. 5), the
 * window Omega_c (Eq. 4, Fig. 1).  Choices the paper leaves open are fixed as:
 *   - image-coordinate regressors are the pixel offset divided by radius, with
 *     coordinate bandwidth 1 (h still applies);
 *   - the window spans frames t-T+1..t (truncated at the sequence start) and is
 *     clipped at the image border;
 *   - the regression adds ridge * W * |beta|^2 to the unnormalised objective
 *     (ridge on the slopes only, so Proposition 1 stays an identity);
 *   - kernel w(u) = exp(-u^2/2).
 * The paper's experiments use h = 1 and b_j = 1 (Section 3, bandwidth
 * optimisation).
 */
typedef struct esim_ad_config {
    uint32_t struct_size;    /* = sizeof(esim_ad_config); ABI versioning        */
    int32_t  width;          /* W >= 1                                          */
    int32_t  height;         /* H >= 1                                          */
    int32_t  radius;         /* r in [1, 15]: (2r+1)^2 spatial window           */
    int32_t  frames;         /* T in [1, 16]: temporal window                   */
    int32_t  mode;           /* ESIM_AD_ADAPTIVE | ESIM_AD_EXHAUSTIVE           */
    int32_t  radiance_fmt;   /* ESIM_AD_LUMA_F32 (1 plane) | RGB_F32 (3) | LOGLUMA_F16 */
    int32_t  feature_fmt;    /* ESIM_AD_FEAT_F32 | ESIM_AD_FEAT_BF16             */
    int32_t  precision;      /* ESIM_AD_FP32 | ESIM_AD_MIXED                     */
    int32_t  reserved0;
    float    contrast;       /* C > 0                                           */
    float    h;              /* global bandwidth h > 0                          */
    float    bandwidth[7];   /* b_j > 0: normal x,y,z, depth, albedo r,g,b      */
    float    log_eps;        /* eps >= 0 in y = ln(Y + eps)                     */
    float    ridge;          /* lambda > 0                                      */
    float    feature_scale[7]; /* > 0; BF16 feature j stores x_j / scale_j (inputs
                                  in FEAT_BF16 and the MIXED ring); powers of two
                                  keep the round trip exact. Ignored otherwise. */
    float    guard_kappa;    /* optional variance guard of the test (a project
                                extension, off for parity with the paper): with
                                guard_kappa > 0 an adaptive frame also flags a
                                pixel when |y_t(c) - L_last| >= C + guard_kappa *
                                sigma_y, sigma_y = sqrt(Var[Y]) / (Y + eps) (delta
                                method, Var[Y] from the frame's variance plane;
                                0 when that plane is NULL).  <= 0: off.        */
    uint64_t event_capacity; /* device event buffer size in events, >= 1        */
} esim_ad_config;

/*
 * One input frame: the renderer's noisy radiance and first-bounce features.
 * Pointers are device memory, or host memory when on_host != 0 (the library
 * then copies them in on its stream; host memory should be pinned for the copy
 * to be asynchronous).  The caller keeps ownership; buffers are read in stream
 * order and may be reused once later work on the same stream has been
 * enqueued and completed.
 */
typedef struct esim_ad_frame {
    const void*  radiance;   /* [1 or 3][H][W] float32, or [H][W] FP16 log (radiance_fmt) */
    const float* variance;   /* [H][W] sample variance of the luminance Y, may be
                                NULL; read only by the optional guard
                                (guard_kappa > 0), unused by the paper's method */
    const float* normal;     /* [3][H][W] float32 (FEAT_F32)                    */
    const float* albedo;     /* [3][H][W] float32 (FEAT_F32)                    */
    const float* depth;      /* [H][W] float32 (FEAT_F32)                       */
    const void*  features;   /* [7][H][W] BF16 (FEAT_BF16): normal xyz, depth,
                                albedo rgb, each stored as x_j / feature_scale_j */
    int32_t      on_host;    /* 0: device pointers, 1: host pointers            */
    int32_t      reserved0;
    int64_t      pitch_elems; /* row pitch of every input plane in elements (0 =
                                width); a plane is then [H][pitch], and plane c
                                of a multi-plane input starts c*H*pitch elements
                                in.  EINVAL if nonzero and below width.        */
} esim_ad_frame;

/* One DVS event e = (q_k, t_l, p_k) of Eq. 1; 12 bytes. */
typedef struct esim_ad_event {
    uint32_t frame;          /* frame index t (fixed-interval timestamps)       */
    uint16_t x, y;           /* pixel q_k                                       */
    int8_t   polarity;       /* p_k in {-1, +1}                                 */
    uint8_t  pad[3];
} esim_ad_event;

typedef struct esim_ad_stats {
    uint64_t frames;         /* frames pushed since init/reset                  */
    uint64_t regressions;    /* pixels regressed (all frames); exhaustive: W*H*frames */
    uint64_t events;         /* events emitted since init/reset                 */
    uint64_t pixels;         /* W*H                                             */
    uint64_t fp64_solves;    /* MIXED: regressions re-solved in FP64 (cond > 1e6) */
    uint64_t staged_ingests; /* frames ingested by the staged (TMA, persistent) kernel:
                                MIXED with FP16/BF16 frames whose planes are 16-byte
                                aligned with a row pitch of a multiple of 8 elements;
                                the others take the one-tile kernel (same results) */
} esim_ad_stats;

/*
 * Create a simulator context bound to `cuda_stream` (a cudaStream_t; NULL =
 * legacy default stream) on the current CUDA device.  Allocates the frame
 * ring, per-pixel model state, work queues and the event buffer in device
 * memory (owned by the context).  Returns EINVAL for a NULL or malformed
 * config (struct_size mismatch, out-of-range sizes or parameters), ENOMEM on
 * allocation failure, ECUDA if no usable device.  *out is set only on success.
 */
esim_ad_status esim_ad_init(const esim_ad_config* cfg, void* cuda_stream, esim_ad_ctx** out);

/*
 * Push the next frame (index t = frames pushed so far) and enqueue the hot
 * path for it on the context's stream: ingest to log brightness, the
 * Proposition-1 test with stream compaction of flagged pixels (adaptive mode,
 * t >= 1), the weighted local regression of flagged pixels (every pixel at
 * t = 0 and in exhaustive mode), and event emission with the last-event update
 * (Eq. 1).  Frame 0 only initialises L_last and the models and emits no events.
 * In the MIXED precision with LOGLUMA_F16 + FEAT_BF16 frames of at least
 * 32 x 8 pixels whose planes start on 16-byte boundaries with a row pitch
 * that is a multiple of 8 elements, the ingest reads the frame by TMA
 * (persistent CTAs, each tile's loads issued a tile ahead); other frames take the one-tile
 * ingest kernel, with identical results (esim_ad_stats.staged_ingests counts
 * the former).  Pinned host frames land in such a layout when W*H is a
 * multiple of 4 and W a multiple of 8.
 * Does not synchronise unless frame->on_host (then it waits for its own
 * host-to-device copies only).  EINVAL on NULL/missing planes (normal, albedo
 * and depth for FEAT_F32, features for FEAT_BF16), ESTATE after a sticky
 * error, ECUDA if a launch fails.  The frame's ordered event writer runs on
 * an internal stream that the context's stream joins before the next frame's
 * solve and in every synchronising call (esim_ad_events, esim_ad_denoised,
 * esim_ad_stats_get, ...), so events are only ever read complete; work the
 * caller enqueues on the context's stream after this call is ordered after
 * the frame's regression, not after its event writer.
 */
esim_ad_status esim_ad_push_frame(esim_ad_ctx* ctx, const esim_ad_frame* frame);

/*
 * Drain the events emitted since the last drain into `dst` (device memory if
 * dst_is_device, else host), in canonical order: frame, then row y, then
 * column x, repeated events of a pixel adjacent.  Synchronises the stream.
 * *n_out receives the number of events.  If cap is smaller than that number,
 * nothing is drained, *n_out holds the required count and ENOSPACE is
 * returned.  The device buffer (event_capacity records) is a ring: a frame's
 * records are lost when, with those not yet drained, they would exceed it;
 * then this returns EOVERFLOW (sticky) with *n_out = the number of events
 * produced since the last drain.  dst may be NULL when cap == 0 (query).
 */
esim_ad_status esim_ad_events(esim_ad_ctx* ctx, esim_ad_event* dst, uint64_t cap,
                              uint64_t* n_out, int dst_is_device);

/*
 * Drain the events of the frames up to and including `frame` (an index of a
 * pushed frame, t = 0, 1, ...; at most 7 frames older than the latest), with
 * the semantics of esim_ad_events otherwise.  It waits for that frame's event
 * writer only, copying on an internal stream: frames pushed after it keep
 * computing (and their host-to-device copies keep landing) meanwhile, so a
 * caller can push frame t + 1 before draining frame t.  Events of that frame
 * already drained by a wider drain give 0.  No paper counterpart: a
 * streaming interface.  EINVAL for a frame not pushed or too old.
 */
esim_ad_status esim_ad_events_frame(esim_ad_ctx* ctx, uint64_t frame, esim_ad_event* dst, uint64_t cap,
                                    uint64_t* n_out, int dst_is_device);

/*
 * Copy the last frame's per-pixel results: alpha = f(x^c) of Eq. 4 (denoised
 * log brightness, [H][W] float32; pixels not regressed in that frame keep the
 * value of their last regression) and flags ([H][W] uint8, 1 where the
 * regression ran in that frame).  Either pointer may be NULL.  Device or host
 * destination per dst_is_device.  Synchronises the stream.
 */
esim_ad_status esim_ad_denoised(esim_ad_ctx* ctx, float* alpha, uint8_t* flags, int dst_is_device);

/*
 * Read (get) or overwrite (set) the per-pixel model kept since each pixel's
 * last event (Fig. 1): l_last [H*W] = brightness reference L(t - Delta t) of
 * Eq. 1, beta [H*W][7] = feature slopes of Eq. 3 (normal xyz, depth, albedo
 * rgb), xc [H*W][7] = the centre feature x^c at the last event.  Host
 * pointers; any may be NULL to skip.  Both synchronise the stream.  Used for
 * checkpoint/resume and for lock-step comparison against a reference.
 */
esim_ad_status esim_ad_get_state(esim_ad_ctx* ctx, float* l_last, float* beta, float* xc);
esim_ad_status esim_ad_set_state(esim_ad_ctx* ctx, const float* l_last, const float* beta,
                                 const float* xc);

/*
 * Kernel timing for tracing and roofline accounting (no paper counterpart:
 * instrumentation).  While enabled, every kernel launch of esim_ad_push_frame
 * is bracketed by CUDA events on the context's stream, and each frame's event
 * writer runs there after the frame's solve, so that every kernel is timed
 * alone.  (Otherwise the writer runs on an internal stream beside the next
 * frame's ingest and regression pass 1; every synchronising call of this API
 * waits for it.)  Classes: 0 = ingest +
 * Proposition-1 test, 1 = weighted local regression + emission, 2 = ordered
 * event writer (class 1 covers both regression launches of an adaptive
 * frame).  `kernels` counts every kernel launch the library issued while
 * enabled.  `neighbours` counts (pixel, window neighbour) pairs
 * accumulated by the regression since init/reset, the unit of its arithmetic.
 * esim_ad_profile_enable(ctx, 1) clears the timings; esim_ad_profile_get
 * synchronises and returns totals since then.
 */
typedef struct esim_ad_profile {
    uint64_t launches[3];    /* timed launch groups per kernel class              */
    uint64_t kernels;        /* kernel launches issued since enabled             */
    double   ms[3];          /* summed device time per class, milliseconds       */
    uint64_t neighbours;     /* (pixel, neighbour) pairs regressed since init     */
    uint64_t regressions;    /* pixels regressed since init/reset                */
} esim_ad_profile;

esim_ad_status esim_ad_profile_enable(esim_ad_ctx* ctx, int on);
esim_ad_status esim_ad_profile_get(esim_ad_ctx* ctx, esim_ad_profile* out);

/*
 * Batching form: many independent sequences of uneven resolution advanced one
 * frame each per step.  The paper has no batched mode; this is the serving
 * shape of the same per-sequence method (every sequence behaves exactly as a
 * context of esim_ad_init would, up to floating-point summation order).
 *
 * Per step: one ingest/test launch over the tiles of all sequences, one
 * persistent accumulation launch over a single compacted queue of flagged
 * (sequence, pixel) entries of all sequences, one solve launch, one
 * event-writer launch; the whole step is a CUDA graph instantiated at init
 * and replayed per step (the per-step frame pointers travel in a small table
 * copied by the graph).  The tile shape that groups flagged pixels into the
 * queue (16x16, 32x8 or 64x4 pixels) and the regression's lanes per pixel
 * (8, 16, 32) are chosen jointly by an autotuner that times the nine pairs on
 * the first adaptive steps and caches the choice per (radius, frames,
 * precision, SM count) in $ESIM_AD_CACHE (default
 * ~/.cache/esim_ad_autotune.txt); ESIM_AD_BATCH_TILE=16|32|64 together with
 * ESIM_AD_BATCH_LANES=8|16|32 forces a pair.
 */
typedef struct esim_ad_batch esim_ad_batch;

/* One batched event: as esim_ad_event plus the sequence index. 12 bytes. */
typedef struct esim_ad_batch_event {
    uint32_t frame;          /* the sequence's own frame index                   */
    uint16_t x, y;
    int8_t   polarity;
    uint8_t  pad;
    uint16_t seq;            /* index into the configs given at init            */
} esim_ad_batch_event;

/*
 * cfgs[n_seq] (1 <= n_seq <= 255): width, height and contrast may differ per
 * sequence; every other field must equal cfgs[0]'s, and event_capacity is
 * taken from cfgs[0] for the whole batch; each sequence has at most 16,777,216
 * pixels.  EINVAL otherwise; ENOMEM / ECUDA as esim_ad_init.  Synchronises.
 */
esim_ad_status esim_ad_batch_init(const esim_ad_config* cfgs, int32_t n_seq, void* cuda_stream,
                                  esim_ad_batch** out);

/*
 * Advance every sequence whose frames[i].radiance is non-NULL by one frame
 * (device pointers; the others are idle this step and keep their state).
 * frames[n_seq].  Asynchronous: the frames must stay valid until the step has
 * run on the stream.  ESTATE after a sticky error, ECUDA on a launch failure.
 */
esim_ad_status esim_ad_batch_step(esim_ad_batch* b, const esim_ad_frame* frames);

/* Drain all sequences' events (order: step, sequence, row, column, repeat);
 * semantics as esim_ad_events.  Synchronises. */
esim_ad_status esim_ad_batch_events(esim_ad_batch* b, esim_ad_batch_event* dst, uint64_t cap,
                                    uint64_t* n_out, int dst_is_device);

/* Restart sequence `seq` at frame 0 (its next step initialises it again). */
esim_ad_status esim_ad_batch_reset_sequence(esim_ad_batch* b, int32_t seq);

/* Per-sequence read-back, as esim_ad_denoised / esim_ad_get_state for sequence
 * `seq` (its last step; host pointers for the state).  Synchronise. */
esim_ad_status esim_ad_batch_denoised(esim_ad_batch* b, int32_t seq, float* alpha, uint8_t* flags,
                                      int dst_is_device);
esim_ad_status esim_ad_batch_get_state(esim_ad_batch* b, int32_t seq, float* l_last, float* beta,
                                       float* xc);

/* Counters and kernel timing as for a context: stats over all sequences, and
 * the profile of the steps run while enabled (class 1 = the one persistent
 * regression launch per step).  lanes_out receives the autotuned lanes per pixel. */
esim_ad_status esim_ad_batch_stats(esim_ad_batch* b, esim_ad_stats* out, int32_t* lanes_out);
/* The tile shape (width x height in pixels) and lanes per pixel in use: the
 * autotuned pair once tuning has finished, else the default 32x8 / 8 (or the
 * pair being timed on the current tuning step's successor).  Null outputs are
 * skipped.  EINVAL for a NULL batch. */
esim_ad_status esim_ad_batch_tiling(esim_ad_batch* b, int32_t* tile_w, int32_t* tile_h, int32_t* lanes);
esim_ad_status esim_ad_batch_profile_enable(esim_ad_batch* b, int on);
esim_ad_status esim_ad_batch_profile_get(esim_ad_batch* b, esim_ad_profile* out);

void esim_ad_batch_destroy(esim_ad_batch* b);

/*
 * Differentiation form: the dense weighted local regression of Eqs. 3-5 over a
 * whole sequence, as a differentiable function of the noisy radiance E and of
 * the seven feature bandwidths b_j of Eq. 5 (the paper fixes h = 1, b_j = 1
 * and names bandwidth selection, Section 3, as the costly alternative; fitting
 * b by gradient descent is this library's extension).  Stateless: the caller
 * owns every buffer, including a workspace of esim_ad_wlr_workspace_size bytes.
 *
 * Per frame t and pixel c, alpha_t(c) solves Eq. 4 over frames t-T+1..t with
 * the ridge of esim_ad_config.  The adjoint uses v = A^-1 e_0 and the residuals
 * r_i = y_i - z_i^T theta:  d alpha/d y_i = w_i v^T z_i,
 * d alpha/d w_i = v^T z_i r_i - lambda v^T P theta (P = diag(0,1,..,1), from the
 * ridge lambda W |beta|^2 with dW/dw_i = 1),  d w_i/d b_j = w_i d_ij^2 / (h^2 b_j^3),
 * d y/d E = (luminance weight) / (Y + eps).  Weights are recomputed, not stored.
 */
typedef struct esim_ad_wlr_desc {
    uint32_t struct_size;    /* = sizeof(esim_ad_wlr_desc)                      */
    int32_t  width, height;  /* W, H >= 1                                       */
    int32_t  sequence;       /* F >= 1 frames in the sequence                   */
    int32_t  radius;         /* r in [1, 15]                                    */
    int32_t  frames;         /* T in [1, 16]                                    */
    int32_t  radiance_fmt;   /* ESIM_AD_LUMA_F32 | ESIM_AD_RGB_F32              */
    float    h;              /* > 0                                             */
    float    log_eps;        /* >= 0                                            */
    float    ridge;          /* > 0                                             */
} esim_ad_wlr_desc;

/* Bytes of device workspace the forward and backward calls need (0 on a bad desc). */
size_t esim_ad_wlr_workspace_size(const esim_ad_wlr_desc* d);

/*
 * radiance  [F][C][H][W] float32, C = 1 or 3 (device, input)
 * features  [F][7][H][W] float32: normal xyz, depth, albedo rgb (device, input)
 * bandwidth [7] float32 b_j > 0 (device, input; read by the kernels, no host copy)
 * alpha     [F][H][W] float32 (device, output)
 * saved     [F][20][H][W] float32 (device, output; theta and v for the backward)
 * workspace esim_ad_wlr_workspace_size bytes (device, caller-owned scratch)
 * Asynchronous on cuda_stream.  EINVAL on a bad desc or NULL pointer.
 */
esim_ad_status esim_ad_wlr_forward(const esim_ad_wlr_desc* d, const float* radiance,
                                   const float* features, const float* bandwidth, float* alpha,
                                   float* saved, void* workspace, void* cuda_stream);

/*
 * g_alpha     [F][H][W] dL/d alpha (device, input)
 * g_radiance  [F][C][H][W] dL/dE (device, output, overwritten)
 * g_bandwidth [7] dL/db (device, output, overwritten)
 * Other arguments as for the forward, with `saved` and `workspace` from it
 * (the workspace must not have been reused in between).  The sums are taken in
 * a fixed order: results are deterministic.  Asynchronous on cuda_stream.
 */
esim_ad_status esim_ad_wlr_backward(const esim_ad_wlr_desc* d, const float* radiance,
                                    const float* features, const float* bandwidth,
                                    const float* saved, const float* g_alpha, float* g_radiance,
                                    float* g_bandwidth, void* workspace, void* cuda_stream);

/*
 * Second-order form: the dense regression of Eqs. 4-5 with the Taylor
 * expansion of Eq. 3 carried to second order, the non-linear regression that
 * the paper's conclusion (Section 4) names as its extension.  Per frame t and
 * pixel c, over the same window and weights as esim_ad_wlr_forward, it fits
 *     y ~ alpha + beta^T d + sum_{a<=b} gamma_ab d_a d_b,   d = x^i - x^c
 * (55 unknowns over the 9-D feature: coordinate offset (q - c)/r, normal,
 * depth, albedo), minimising sum_i w^i (y^i - theta^T z^i)^2 +
 * lambda W sum_{k>=1} theta_k^2 (ridge on every coefficient but alpha, in
 * these natural units), and returns alpha.  Stateless and dense: every pixel of
 * every frame.  FP32 accumulation and Cholesky; the window's neighbours are
 * summed in up to eight interleaved partial sums, so results are deterministic.
 *
 * radiance  [F][C][H][W] float32, C = 1 or 3 (device, input)
 * features  [F][7][H][W] float32: normal xyz, depth, albedo rgb (device, input)
 * bandwidth [7] float32 b_j > 0 (device, input)
 * alpha     [F][H][W] float32 (device, output)
 * workspace esim_ad_wlr2_workspace_size bytes (device, caller-owned scratch:
 *           the packed log brightness and features, 32 bytes per pixel-frame)
 * Asynchronous on cuda_stream.  EINVAL on a bad desc, a NULL pointer or more
 * than 65535 frames; ECUDA if a launch fails.
 */
size_t esim_ad_wlr2_workspace_size(const esim_ad_wlr_desc* d);
esim_ad_status esim_ad_wlr2_forward(const esim_ad_wlr_desc* d, const float* radiance,
                                    const float* features, const float* bandwidth, float* alpha,
                                    void* workspace, void* cuda_stream);

/*
 * Write the events of one frame from a map of signed per-pixel event counts
 * (polarity times number of events at each pixel), in canonical order (row,
 * column, repeat), without allocating anything.  The paper has no
 * counterpart: this is a deployment entry point.
 *
 * Who it is for: callers that cannot call cudaMalloc where they need events
 * written - latency-critical loops where cudaMalloc's implicit device-wide
 * synchronisation would stall other work, and plugins of a host framework that
 * owns all device memory.  It runs the same kernels as the context's event
 * writer, with their scratch (about 32 KB) in a fixed array inside the library
 * that every GPU loading the library keeps until the process exits.
 *
 * counts       [height][width] int32, device memory (input, caller-owned);
 *              each |count| at most 524,288 (2^19).
 * frame        frame index written into each record.
 * events       device memory for `capacity` records (output, caller-owned);
 *              may be NULL when capacity == 0.
 * total_device one uint64 in device memory (output): the number of events the
 *              counts call for; records past `capacity` are dropped, so
 *              *total_device > capacity means the buffer was too small.  If a
 *              count lies outside +-2^19, nothing is written and
 *              *total_device is UINT64_MAX.
 * cuda_stream  cudaStream_t the work is enqueued on; nothing is synchronised.
 * Limit: width * height <= 16,777,216 pixels (and each side <= 65535);
 * larger frames return EINVAL.  EINVAL also for NULL counts/total_device or
 * NULL events with capacity > 0; ECUDA if a CUDA call fails.
 * The first call on a device looks up the array's device address (once per
 * device, with that device current); make that first call before any stream
 * capture.  All calls on a device share the one array, so calls whose work
 * overlaps on the GPU (different streams without ordering) race; the array's
 * control block is cleared at the start of each call.
 */
esim_ad_status esim_ad_write_events_noalloc(const int32_t* counts, int32_t width, int32_t height,
                                            uint32_t frame, esim_ad_event* events, uint64_t capacity,
                                            uint64_t* total_device, void* cuda_stream);

/* ------------------------------------------------------------------------
 * Evaluation (Section 3, quantitative comparison).
 *
 * esim_ad_esim_frame: one frame of the plain ESIM simulator the paper compares
 * against (and, run on noise-free frames, the stand-in for its reference
 * events): Eq. 1 applied to the log brightness y = ln(Y + log_eps) of the frame
 * itself (Y = Rec.709 luminance of RGB radiance, or the radiance itself with
 * one channel), with the simulator's crossing rule: dL = y - L_last,
 * n = floor(|dL| / C), counts = sign(dL) n, L_last += counts C.  init != 0:
 * L_last = y and counts = 0 (frame 0).
 *
 * radiance  [channels][n_pix] float32, device (input, caller-owned); channels 1 or 3.
 * l_last    [n_pix] float32, device (in/out, caller-owned).
 * counts    [n_pix] int32, device (output, caller-owned).
 * Asynchronous on cuda_stream.  EINVAL for NULL pointers, channels not 1 or
 * 3, n_pix < 0 or contrast <= 0; ECUDA if the launch fails.
 */
esim_ad_status esim_ad_esim_frame(const float* radiance, int32_t channels, float log_eps, float contrast,
                                  int32_t init, float* l_last, int32_t* counts, int64_t n_pix,
                                  void* cuda_stream);

/* Result of esim_ad_quality; tau values as passed, up to 16. */
typedef struct {
    int32_t n_tau;
    float tau[16];
    double precision[16];   /* P(tau), Eq. 10a */
    double recall[16];      /* R(tau), Eq. 10b */
    double fscore[16];      /* harmonic mean of the two (0 where both are 0) */
    double chamfer;         /* polarity-aware chamfer distance; +inf if an event has no same-polarity partner */
    uint64_t n_gen, n_ref;  /* events in each set */
} esim_ad_quality_result;

/*
 * Precision, recall, F-score and chamfer distance of generated events against
 * reference events, both given as signed per-pixel count maps (p*n per pixel
 * and frame, as the simulators produce).  Events are signed points
 * (x / width, y / height, t / frames); for every event the distance to the
 * nearest event of the same polarity in the other set is found exactly on the
 * GPU: a per-column pass records, for each pixel, the squared distance to the
 * nearest event in its column (per frame and polarity), then each event
 * searches outward in x and t with the bound of its best distance so far.
 * P(tau) = fraction of generated events within tau of a reference event,
 * R(tau) = fraction of reference events within tau of a generated event; the
 * chamfer distance is the mean squared distance generated -> reference plus
 * the mean squared distance reference -> generated.  Distances are evaluated
 * in FP32 (squared, then compared with tau^2); sums in FP64, reduced in a
 * fixed order (the result is deterministic).
 *
 * gen, ref   [frames][height][width] int32, device (input, caller-owned).
 * tau        n_tau (1..16) thresholds, host.
 * workspace  device memory of esim_ad_quality_workspace_size() bytes,
 *            caller-owned, any content.
 * out        host (output); written after the stream has been synchronised.
 * Synchronises cuda_stream.  EINVAL for NULL pointers, sizes <= 0, n_tau out
 * of range or a workspace that is too small; ECUDA if a CUDA call fails.
 */
size_t esim_ad_quality_workspace_size(int32_t width, int32_t height, int32_t frames);
esim_ad_status esim_ad_quality(const int32_t* gen, const int32_t* ref, int32_t width, int32_t height,
                               int32_t frames, const float* tau, int32_t n_tau, void* workspace,
                               size_t workspace_bytes, esim_ad_quality_result* out, void* cuda_stream);

/* ------------------------------------------------------------------------
 * Monte Carlo renderer for analytic test scenes (a stand-in for the paper's
 * PBRT-v4 renders, Section 3): it produces exactly the simulator's inputs -
 * noisy RGB radiance at spp samples per pixel, the variance of the luminance
 * estimate, and first-hit normal, depth and albedo.
 *
 * Scene: an open-fronted room x in [-box0, box0], y in [-box1, box1],
 * z in [-box2, box2] (no wall at z = +box2) with diffuse walls (the back wall
 * checkered when checker > 0), a rectangular area light of radiance
 * light_radiance on the ceiling over [light0, light1] x [light2, light3] in
 * x and z, and up to 8 diffuse spheres whose centres move by `velocity` per
 * frame.  Pinhole camera at cam_pos looking along -z (up +y).
 *
 * Estimator per sample: a jittered camera ray; at each of up to max_bounces
 * surface interactions, next-event estimation towards one uniform point of
 * the light (shadowed by spheres), then a cosine-weighted bounce; emission
 * counted for camera rays only.  Random numbers: Philox4x32-10 (Salmon et al.
 * 2011) with key (seed, frame) and counter (pixel, sample, call, 0).  All
 * arithmetic is IEEE FP32 with one rounding per operation (no contraction),
 * so the result is a fixed function of the scene, frame and seed.
 * Features are means over the samples of the camera rays' first hits; depth
 * is the distance along the ray.
 * ------------------------------------------------------------------------ */
typedef struct esim_ad_sphere {
    float center[3];    /* at frame 0 */
    float velocity[3];  /* per frame  */
    float radius;       /* > 0        */
    float albedo[3];
} esim_ad_sphere;

typedef struct esim_ad_render_scene {
    uint32_t struct_size;       /* = sizeof(esim_ad_render_scene)               */
    int32_t  width, height;     /* >= 1, width * height < 2^31                  */
    int32_t  spp;               /* samples per pixel, 1..65536                  */
    int32_t  max_bounces;       /* surface interactions per path, 1..8          */
    int32_t  n_spheres;         /* 0..8                                         */
    uint32_t seed;
    float    cam_pos[3];        /* inside the room                              */
    float    tan_half_fov_y;    /* > 0                                          */
    float    box[3];            /* half extents > 0                             */
    float    wall_albedo[5][3]; /* left, right, floor, ceiling, back            */
    float    back_albedo2[3];   /* second colour of the back wall's checker     */
    float    checker;           /* checker cell size; <= 0: plain back wall     */
    float    light[4];          /* x0 < x1, z0 < z1 of the ceiling light        */
    float    light_radiance[3];
    float    eps;               /* minimum hit distance > 0                     */
    esim_ad_sphere spheres[8];
} esim_ad_render_scene;

/*
 * Render frame `frame` of the scene into caller-owned device buffers:
 * radiance [3][H][W], variance [H][W] (variance of the mean luminance,
 * unbiased over the samples; 0 when spp == 1), normal [3][H][W],
 * albedo [3][H][W], depth [H][W], all float32.  Asynchronous on cuda_stream.
 * EINVAL for NULL pointers or out-of-range fields; ECUDA if the launch fails.
 */
esim_ad_status esim_ad_render(const esim_ad_render_scene* scene, int32_t frame, float* radiance,
                              float* variance, float* normal, float* albedo, float* depth,
                              void* cuda_stream);

/* Restart the sequence at frame 0 and clear events, counters and sticky errors. */
esim_ad_status esim_ad_reset(esim_ad_ctx* ctx);

/* Counters since init/reset; synchronises the stream. */
esim_ad_status esim_ad_stats_get(esim_ad_ctx* ctx, esim_ad_stats* out);

/* Release every resource of the context (synchronises its stream). NULL is a no-op. */
void esim_ad_destroy(esim_ad_ctx* ctx);

/* Static, human-readable name of a status code. */
const char* esim_ad_status_string(esim_ad_status status);

#ifdef __cplusplus
}
#endif
#endif /* ESIM_AD_H */
