/*
 * glt: GB300-native pose-only direct photometric tracking.
 *
 * C ABI of the library libglt.so.  The method is GLidE-SLAM's direct tracker
 * (arXiv 2607.16897, Sec. IV "Direct Photometric Tracking"): a new frame is
 * aligned to a reference frame whose sparse map points have known depth, by
 * a coarse-to-fine Gauss-Newton / Levenberg-Marquardt solve over an SE(3) pose
 * plus an affine brightness pair (a, b).  Per pyramid level and iteration
 * every map point's 8-pixel pattern is projected through the current pose,
 * the current image and its gradient are sampled bilinearly, the residual
 * r = I(u(T) + du_k) - e^a I0_k - b is Huber-weighted, the image gradient is
 * chained through the projection Jacobian and everything is reduced into the
 * 8x8 normal equations (Eqs. 1-5).  The whole level x iteration loop, the
 * FP64 Cholesky solve and the SE(3) update run on the GPU.
 *
 * Conventions shared by every entry point
 *  - Poses are row-major 3x4 [R|t] doubles, T maps reference-camera
 *    coordinates to current-camera coordinates: x_c = R x_r + t.  The paper's
 *    u_i(T) = pi(T P_i), u_i^0 = pi(T0 P_i) (Eq. 1) is this with x_r = T0 P_i.
 *  - Increments are applied on the right: T <- T exp(delta) (Sec. IV-A), twist
 *    order (translation, rotation).
 *  - Images are 8-bit gray, row-major with a row pitch in bytes (>= width).
 *    Pixel centres sit at integer coordinates.
 *  - Map points are float triples (u0, v0, depth): the level-0 reference pixel
 *    position (sub-pixel) and the camera-z depth in metres.
 *  - Streams: every call is ordered on the caller's CUDA stream (a
 *    cudaStream_t passed as void*; NULL = legacy default stream).  Only the
 *    calls that return host results synchronise that stream.
 *  - Ownership: the caller owns all buffers it passes.  Host inputs are copied
 *    before the call returns; device inputs are read by work enqueued on the
 *    stream, so they must stay valid until that work has run.  The library
 *    owns the device memory it allocates in glt_create / glt_batch_create and
 *    frees it in the matching destroy call; nothing else allocates.
 *  - Errors: every int-returning call returns GLT_OK (0) or a negative
 *    GLT_ERR_* code; no exception crosses the ABI.  glt_last_error() gives a
 *    thread-local message for the last failure.  Per-frame solver outcomes are
 *    bits in glt_result.status, not errors.
 *  - Threads: one tracker must not be used from two host threads at once.
 */
#ifndef GLT_H
#define GLT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GLT_MAX_LEVELS 8

/* return codes */
#define GLT_OK 0
#define GLT_ERR_INVALID_ARG (-1)
#define GLT_ERR_CUDA (-2)
#define GLT_ERR_NO_REFERENCE (-3)
#define GLT_ERR_CAPACITY (-4)
#define GLT_ERR_UNSUPPORTED (-5)
#define GLT_ERR_IO (-6)              /* a file could not be opened, read or written */

/* glt_result.status bits (per-frame solver outcomes) */
#define GLT_TRACK_TOO_FEW_POINTS 1 /* a level had fewer than min_valid samples */
#define GLT_TRACK_NOT_PD 2         /* the damped normal matrix was not positive definite */
#define GLT_TRACK_DIVERGED 4       /* a non-finite start, pass sum (FP32 overflow) or
                                      candidate state; the state before it is returned */
#define GLT_TRACK_TIMEOUT 8        /* a CTA of the stream's cluster waited longer than its
                                      limit (about a second) for a peer's partial sums; the
                                      accepted state before that pass is returned */

/* pyramid slots */
#define GLT_REF 0
#define GLT_CUR 1

/* precision modes */
#define GLT_FP32 0  /* uint8 levels, FP32 residuals/Jacobians/sums; the solve and the state
                       update in the precision glt_config.solve selects (FP64 by default) */
#define GLT_MIXED 1 /* FP16 (I, gx, gy) levels, FP32 math, Kahan FP32 block sums; solve and
                       state as GLT_FP32 */

/* solve modes (glt_config.solve) */
#define GLT_SOLVE_FP64 0
#define GLT_SOLVE_FP32 1

/* Jacobian forms (Sec. IV-B) */
#define GLT_FORWARD 0 /* current image's gradient at the warped location, every pass */
#define GLT_IC 1      /* inverse compositional: reference-side rows cached per reference */

/* Normal matrix of the solve (Sec. IV-B / IV-C) */
#define GLT_HESSIAN_PASS 0   /* J^T W J summed again in every pass */
#define GLT_HESSIAN_CACHED 1 /* the paper's cache: H = J^T J of the reference-side rows over
                                the reference's usable points, once per reference and
                                level; each pass reduces only g, E and n */

typedef struct glt_tracker glt_tracker;
typedef struct glt_batch glt_batch;
typedef struct glt_nn glt_nn;

typedef struct glt_config {
    int width, height;          /* level-0 frame size in pixels (>= 16 each) */
    int levels;                 /* pyramid levels, 1..GLT_MAX_LEVELS; level l is
                                   floor(size / 2^l) and must be >= 8 pixels */
    double fx, fy, cx, cy;      /* level-0 pinhole intrinsics; level l uses f/2^l, c/2^l */
    int max_points;             /* capacity of glt_set_map_points */
    int max_iters[GLT_MAX_LEVELS]; /* LM candidate evaluations per level (0 skips a level) */
    double huber_k;             /* Huber threshold in gray levels (weight k/|r| beyond it) */
    double lambda0;             /* initial LM damping of diag(H) at each level start
                                   (>= 0; 0 with accept_step huge is plain Gauss-Newton) */
    double lambda_up;           /* damping factor after a rejected candidate */
    double lambda_down;         /* damping factor after an accepted candidate */
    double eps_step;            /* stop the finest level once max |delta_xi| < eps_step */
    double eps_step_coarse;     /* ... and every coarser level once max |delta_xi| <
                                   eps_step_coarse; such a final step (if also below
                                   accept_step) is taken without a pass of its own */
    double eps_cost;            /* ... or once a rejected candidate raised the cost by
                                   no more than eps_cost * cost */
    double accept_step;         /* candidates with max |delta_xi| < accept_step are taken
                                   even if the cost rose (Gauss-Newton steps near
                                   convergence); larger ones only if it fell */
    int min_valid;              /* minimum valid residual samples per pass */
    double zmin;                /* minimum current-camera depth of a usable point (m) */
    int precision;              /* GLT_FP32 or GLT_MIXED */
    int cluster;                /* CTAs cooperating on one stream (1..16, 0 = auto) */
    int threads;                /* threads per CTA (128, 256 or 512; 0 = auto; p x p
                                   patches 256, the cached Hessian 512) */
    int jacobian;               /* GLT_FORWARD or GLT_IC.  GLT_IC (Sec. IV-B, IV-C
                                   "Precompute IC"): glt_set_map_points also caches
                                   the reference gradient at every pattern sample of
                                   every level, and each pass uses the rows
                                   e^a grad I0(u0_l + du_k) dpi/dx(x_r) [I | -[x_r]x]
                                   instead of the current image's gradient (the
                                   inverse-compositional template approximation;
                                   T <- T exp(delta) as in the paper) */
    int pattern;                /* 0: the 8-pixel sparse pattern; odd p in 3..11: the
                                   paper's p x p patch (Sec. IV-A; 7 x 7 and 11 x 11 in
                                   Sec. V), samples row by row from (-(p-1)/2, -(p-1)/2);
                                   p x p needs precision GLT_FP32 and 256 (or 0) threads */
    int affine;                 /* 1: estimate (a, b); 0: keep the initial (a, b) (the
                                   paper estimates no brightness change) */
    int hessian;                /* GLT_HESSIAN_PASS or GLT_HESSIAN_CACHED.  CACHED (Sec.
                                   IV-B: with the rows on the reference side H = J^T J is
                                   constant while the reference is, so it is precomputed
                                   once per reference update; Sec. IV-C "Precompute IC":
                                   per-point H_i reduced into one H per level):
                                   glt_set_map_points also reduces H over the points usable
                                   on each level of the reference and inverts it in FP64;
                                   every pass then reduces only g = J^T W r, E and n (over
                                   the points usable at the pass state) and steps by
                                   delta = -(e^{2a} H)^-1 g (the rows are e^a times the
                                   reference rows).  Points out of view stay in H, as in
                                   the paper.  Needs jacobian GLT_IC, affine 0, lambda0 0
                                   (plain Gauss-Newton), precision GLT_FP32 and 512 (or 0)
                                   threads (7 x 7 and 11 x 11 patches are split over four
                                   threads each); an H that is not positive definite ends
                                   the level with GLT_TRACK_NOT_PD */
    int solve;                  /* the 8x8 solve and the SE(3) step (the state, the
                                   accept/reject decision and the composition are FP64 in
                                   both modes): GLT_SOLVE_FP64 (default) the L D L^T
                                   factorisation and the exponential in FP64;
                                   GLT_SOLVE_FP32 the factorisation and exp(delta) - I in
                                   FP32 (H and g are FP32 sums; the increment's entries
                                   are O(|delta|)), the composition in FP64 and one FP64
                                   orthonormalisation of the frame's final pose; a
                                   system with an FP32 pivot below 1e-4 of its damped
                                   diagonal is factorised in FP64, so "not positive
                                   definite" is always the FP64 decision */
} glt_config;

typedef struct glt_result {
    double T[12];               /* final pose, row-major 3x4 */
    double a, b;                /* final affine brightness, cur ~ e^a ref + b */
    double cost;                /* mean Huber energy sum(rho)/n of the last evaluated state
                                   on the last level that ran (NaN if none ran); a level's
                                   final step below its stop threshold is taken without a
                                   pass of its own, so T may differ from that state by a
                                   step below eps_step */
    int n_valid;                /* valid residual samples behind `cost` */
    int iters_total;            /* candidate evaluations over all levels */
    int iters[GLT_MAX_LEVELS];  /* candidate evaluations per level */
    int passes;                 /* linearisation passes (level starts + candidates) */
    int status;                 /* GLT_TRACK_* bits */
} glt_result;

/* Fills `cfg` with the defaults: 4 levels, 10 iterations per level, Huber 9,
 * lambda0 1e-4 (x4 up, x0.5 down), eps_step 1e-6 (finest level),
 * eps_step_coarse 3e-4 (coarser levels), eps_cost 0 (off),
 * accept_step 1e-3, min_valid 16, zmin 1e-3, FP32, automatic cluster/threads,
 * max_points 4096, GLT_FORWARD, the 8-pixel pattern, affine estimated,
 * GLT_HESSIAN_PASS.
 * The paper's configuration is levels 6, pattern 7 (or 11), affine 0,
 * jacobian GLT_IC, hessian GLT_HESSIAN_CACHED, huber_k very large (no robust
 * weights), lambda0 0, accept_step very large and eps_step =
 * eps_step_coarse = 0 (plain Gauss-Newton with a fixed number of iterations
 * per level). */
void glt_default_config(glt_config* cfg, int width, int height, double fx, double fy,
                        double cx, double cy);

/* Creates a tracker on the current CUDA device and allocates all its device
 * memory (both pyramids, map-point arrays for max_points, solver state).
 * Errors: INVALID_ARG for a bad config, CUDA on allocation failure. */
int glt_create(const glt_config* cfg, glt_tracker** out);

/* Frees everything glt_create allocated.  NULL is a no-op.  The caller must
 * ensure no work using the tracker is still pending on any stream. */
void glt_destroy(glt_tracker* trk);

/* Sec. IV-C "Image pyramids": copies `img` (width x height, `pitch_bytes` per
 * row, host or device memory per `is_device`) into level 0 of pyramid `slot`
 * (GLT_REF or GLT_CUR) and builds levels 1..L-1 by a 5-tap binomial blur
 * [1 4 6 4 1]/16 in x and y with clamp-to-edge borders and even-sample
 * decimation, summed exactly in integers and rounded half up.  In GLT_MIXED
 * mode it also writes the FP16 (I, gx, gy) copy of every CUR level.
 * A host frame is first copied into a device staging buffer of the tracker (so
 * two host-frame builds on different streams must not overlap).
 * Asynchronous on `stream`.  Errors: INVALID_ARG (slot, pitch < width, NULL). */
int glt_build_pyramid(glt_tracker* trk, int slot, const uint8_t* img, int pitch_bytes,
                      int is_device, void* stream);

/* Sec. IV-C "Precompute" (the part the forward form needs): uploads n map
 * points uvd[n][3] = (u0, v0, depth) (host or device memory), back-projects
 * them and samples each point's reference patch I0 (8 pattern pixels) on every
 * level of the REF pyramid, marking points whose pattern leaves the image.
 * Must follow glt_build_pyramid(GLT_REF).  Asynchronous on `stream`.
 * Errors: CAPACITY if n > max_points, NO_REFERENCE if no REF pyramid. */
int glt_set_map_points(glt_tracker* trk, const float* uvd, int n, int is_device, void* stream);

/* Sec. IV-A/IV-C "Track": coarse-to-fine LM from (T_init, ab_init) against the
 * current REF data and CUR pyramid, one persistent launch; writes the result
 * to the host struct `out` after synchronising `stream`.  The rotation of
 * T_init is first projected onto SO(3) (Gram-Schmidt on its rows).
 * T_init = NULL (or ab_init = NULL) starts from the tracker's state instead:
 * the constant-velocity prediction of glt_state_predict.  Every call then
 * advances the tracker's state with the result (glt_state_update).
 * Errors: NO_REFERENCE without map points, INVALID_ARG for non-finite input. */
int glt_track_frame(glt_tracker* trk, const double T_init[12], const double ab_init[2],
                    glt_result* out, void* stream);

/* As glt_track_frame, fully asynchronous: the initial state is read on the
 * device from init_dev[14] = (T[12], a, b) and the result written to the
 * device struct out_dev.  No host synchronisation. */
int glt_track_frame_async(glt_tracker* trk, const double* init_dev, glt_result* out_dev,
                          void* stream);

/* Sec. IV-C "Image pyramids" + "Track" for one frame:
 * glt_build_pyramid(GLT_CUR) from the DEVICE frame `frame_dev` (width x
 * height, `pitch_bytes` per row) followed by glt_track_frame_async, issued as
 * one chain: each pyramid kernel after the first, and the track kernel, is a
 * programmatic dependent launch of the kernel before it, so it starts while
 * that kernel runs (the track kernel loads its descriptor and initial state
 * then) and waits on the device for the data it needs.  Same results as the
 * two calls.  The frame must stay unchanged until the work completes.
 * Asynchronous.  Errors: NO_REFERENCE, INVALID_ARG (NULL, pitch < width). */
int glt_track_image_async(glt_tracker* trk, const uint8_t* frame_dev, int pitch_bytes,
                          const double* init_dev, glt_result* out_dev, void* stream);

/* Sec. IV-C "Image pyramids" + "Track" for one frame, from the host:
 * glt_build_pyramid(GLT_CUR) + glt_track_frame in one call, the form a
 * per-frame caller uses: the frame `img` (host memory, uploaded first through
 * the tracker's staging buffer, or device memory per `is_device`; `pitch_bytes`
 * per row) is chained with the solve as in glt_track_image_async, the result
 * is written to the host struct `out` after synchronising `stream`, and the
 * tracker's state advances.  T_init / ab_init NULL: start from the state's
 * constant-velocity prediction (glt_state_predict).
 * Errors: NO_REFERENCE, INVALID_ARG (NULL img / out, pitch < width,
 * non-finite initial state). */
int glt_track_image(glt_tracker* trk, const uint8_t* img, int pitch_bytes, int is_device,
                    const double T_init[12], const double ab_init[2], glt_result* out,
                    void* stream);

/* One linearisation (Eqs. 3-5 at a given state) on `level` of the CUR pyramid:
 * the full symmetric H (64 doubles, row-major), g = J^T W r (8; the paper's
 * right-hand side b of Eq. 5 is -g), the Huber energy E and the number of
 * valid samples n, all written to host memory; if `res` is not NULL it gets
 * the N*K FP32 residuals, K samples of the pattern per point (8, or p*p),
 * NaN for samples of unused points.  With GLT_HESSIAN_CACHED these are the
 * normal equations the solve uses: H is e^{2a} times the level's cached
 * reference Hessian in its pose block (the affine rows and columns zero) and
 * g keeps its pose part (g[6] = g[7] = 0).  Synchronous.
 * Uses a multi-block kernel with a single-pass last-block finish. */
int glt_debug_linearize(glt_tracker* trk, int level, const double T[12], double a, double b,
                        double H[64], double g[8], double* E, int* n, float* res,
                        void* stream);

/* ---------------------------------------------------------------------------
 * Tracking state of one stream (checkpoint / resume; the paper keeps none of
 * its own: its tracker starts every frame from a constant-velocity motion
 * model, Sec. IV-A).  Host memory, 216 bytes, no device work:
 *   T_cr    the last tracked pose, row-major 3x4 [R|t], reference -> current
 *           camera (x_c = R x_r + t), identity after glt_set_map_points;
 *   a, b    the last affine pair (0, 0 after glt_set_map_points);
 *   motion  M = T_k T_{k-1}^{-1}, the camera motion between the last two
 *           tracked frames in the newer frame's camera coordinates (identity
 *           at creation; a new reference keeps it);
 *   reference  version of the map points T_cr is relative to (0 before the
 *           first glt_set_map_points, +1 for every call);
 *   frames  frames tracked against that reference.
 * A new reference resets T_cr and (a, b), i.e. the library reads the new
 * reference as the last tracked frame (what an indirect pipeline's keyframe
 * refresh gives); a caller whose reference is another frame sets the pose
 * with glt_set_state.  glt_track_frame reads and advances the state;
 * glt_track_frame_async and the batch leave it alone (their callers can run
 * glt_state_predict / glt_state_update on their own copies).
 * ------------------------------------------------------------------------- */
typedef struct glt_state {
    double T_cr[12];
    double a, b;
    double motion[12];
    unsigned reference;
    int frames;
} glt_state;

/* Constant-velocity prediction from `state`: T_init = motion T_cr (FP64,
 * rotation re-orthonormalised by Gram-Schmidt on its rows) and ab_init =
 * (a, b).  Host only.  Errors: INVALID_ARG (NULL, non-finite state). */
int glt_state_predict(const glt_state* state, double T_init[12], double ab_init[2]);

/* Advances `state` by one tracked frame: motion = T T_cr^{-1}, T_cr = T,
 * (a, b) from `result`, frames + 1.  Host only.  A result with a non-finite
 * pose or affine pair leaves the state unchanged and returns INVALID_ARG. */
int glt_state_update(glt_state* state, const glt_result* result);

/* Copies the tracker's state to host memory `out`.  Host only, no sync. */
int glt_get_state(const glt_tracker* trk, glt_state* out);

/* Replaces the tracker's state (a checkpoint taken by glt_get_state, or the
 * pose of the last frame relative to a new reference); `reference` is
 * ignored and set to the tracker's current map-point version.  Host only.
 * Errors: INVALID_ARG (NULL, non-finite values, frames < 0). */
int glt_set_state(glt_tracker* trk, const glt_state* in);

/* Test access to the solver's FP64 reciprocal (the pivot reciprocals of the
 * L D L^T factorisation inside the track kernel): r_dev[i] = 1 / d_dev[i] for
 * n DEVICE doubles, computed as the kernel computes it (one Newton-Raphson
 * step on an FP32 seed for 2^-100 <= |d| < 2^100, relative error below 1e-13;
 * an IEEE division elsewhere).  Not part of the method; no paper counterpart.
 * Asynchronous.  Errors: INVALID_ARG (n < 0, NULL with n > 0), CUDA. */
int glt_debug_rcp(const double* d_dev, double* r_dev, int n, void* stream);

/* Latency floor of one tracker pass: times (CUDA events, after one warm-up
 * launch) a launch of one stream's cluster (`cluster` CTAs of `threads`
 * threads) that runs `passes` passes of the track kernel's fixed part --
 * the block reduction, the cluster exchange of the CTA partials and the
 * solver tail (the LM decision, the solve -- the L D L^T factorisation, or
 * with `cached` the product with a cached H^-1 -- and the SE(3) exponential
 * and composition, in solve mode `solve`: GLT_SOLVE_FP64 or GLT_SOLVE_FP32)
 * on a fixed normal system -- with no map point, and writes the
 * microseconds per pass to *us_per_pass.  What a real pass costs beyond it
 * is the linearisation of its points.  Not part of the method; no paper
 * counterpart.  Synchronous; allocates 8 bytes.
 * Errors: INVALID_ARG (passes outside [1, 100000], an unknown solve mode, a
 * shape that cannot launch: cached needs 512 threads), CUDA. */
int glt_debug_pass_floor(int cluster, int threads, int cached, int solve, int passes,
                         float* us_per_pass, void* stream);

/* Failure test of the cluster exchange (no counterpart in the paper): one
 * pass of the latency-floor kernel on a `cluster`-CTA cluster whose CTA 0
 * withholds its partial sums, so every CTA's bounded wait runs out (about a
 * second, twice: the wait and the drain before the CTAs leave together).
 * *status = GLT_TRACK_TIMEOUT when the kernel reported the timeout, else 0;
 * the context stays usable.  Synchronous.
 * Errors: INVALID_ARG (cluster outside [2, 16], a shape that cannot launch),
 * CUDA. */
int glt_debug_exchange_timeout(int cluster, int threads, int* status, void* stream);

/* Bounds-checked build (libglt_checked.so, the same sources compiled with
 * GLT_CHECKED; the paper has no counterpart): every gather and table access
 * of the pyramid, map-point and track kernels checks its range against its
 * buffer, and an access outside sets a flag bit (1: uint8 level window, 2:
 * FP16-packed texels, 4: per-point reference tables, 8: point arrays, 16:
 * pyramid source, 32: pyramid destination, 64: map-point table writes) and
 * goes to the buffer's first element instead.  Waits for the device, writes
 * the flags of every kernel run since the last call to *flags and clears
 * them.  Errors: INVALID_ARG (flags NULL), UNSUPPORTED (the normal build:
 * *flags = 0), CUDA. */
int glt_debug_checked_flags(unsigned* flags);

/* Positive control of the bounds-checked build: a one-thread kernel reads
 * one element inside a 64-float device buffer and one 5 elements past its
 * end through the range check, which sends the second to the buffer's first
 * element and sets flag 4; *flags = the flags that kernel set.  Synchronous.
 * Errors: INVALID_ARG (flags NULL), UNSUPPORTED (the normal build: nothing is
 * launched, *flags = 0), CUDA. */
int glt_debug_checked_probe(unsigned* flags);

/* The (cluster, threads) shape the tracker's solve launches with (chosen at
 * glt_create and again when the point count changes, or set in the config). */
int glt_get_shape(const glt_tracker* trk, int* cluster, int* threads);

/* Copies level `level` of pyramid `slot` (unpadded, W_l * H_l bytes) to host
 * memory `out`.  Synchronous. */
int glt_get_pyramid(glt_tracker* trk, int slot, int level, uint8_t* out, void* stream);

/* Copies the per-pass trace of the last track into host arrays of length
 * `max`: cost[k] = E/n of pass k (INFINITY when too few samples) and
 * info[k] = level * 4 + 2 * accepted + is_candidate; *count = passes recorded.
 * Synchronous. */
int glt_get_trace(glt_tracker* trk, double* cost, int* info, int max, int* count, void* stream);

/* ---------------------------------------------------------------------------
 * Batched form: S independent trackers (own sizes, points and configs) tracked
 * in ONE persistent launch, one thread-block cluster per stream.
 * ------------------------------------------------------------------------- */

/* Builds a batch over `trackers[0..S-1]` (all created on the current device,
 * all with the same precision, and all or none with GLT_HESSIAN_CACHED).  The
 * batch references, but does not own, the trackers; they must outlive it.
 * Errors: INVALID_ARG. */
int glt_batch_create(glt_tracker* const* trackers, int S, glt_batch** out);
void glt_batch_destroy(glt_batch* batch);

/* Builds the CUR pyramids of all S trackers in one launch per level from
 * frames_dev, a DEVICE array of S device pointers to contiguous frames
 * (pitch = each tracker's width).  The pointer array is read at run time, so
 * a captured graph stays valid when its contents change. */
int glt_batch_build_pyramid(glt_batch* batch, const uint8_t* const* frames_dev, void* stream);

/* Tracks all S streams: init_dev[S][14] (T[12], a, b) and out_dev[S] are
 * device arrays.  One launch; no host synchronisation. */
int glt_batch_track(glt_batch* batch, const double* init_dev, glt_result* out_dev,
                    void* stream);

/* Captures glt_batch_build_pyramid + glt_batch_track with these arguments into
 * a CUDA graph owned by the batch (replacing any previous one).  The kernels
 * are chained as programmatic dependent launches, as in
 * glt_track_image_async (the track kernel only without a proposal stage). */
int glt_batch_capture(glt_batch* batch, const uint8_t* const* frames_dev, const double* init_dev,
                      glt_result* out_dev, void* stream);

/* Replays the captured graph on `stream`.  Errors: INVALID_ARG if none. */
int glt_batch_replay(glt_batch* batch, void* stream);

/* Autotuner: times the batched track on the current inputs (`reps` timed
 * launches each) over the candidate launch configurations and keeps the
 * fastest: one (cluster, threads) shape for every stream; two launch classes
 * (see glt_batch_set_classes) with the first quarter or half of the launch
 * order as the heavy class on a wide shape and the rest on a narrow one; or
 * clusters in proportion to each stream's points (glt_batch_set_proportional)
 * at several points per CTA.  Results are cached for the process, keyed by
 * the batch's signature (kernel variant and, in launch order, every stream's
 * width, height, point capacity and levels): a batch with a known signature
 * takes the cached configuration without timing.  Reports the first class's
 * shape (the only one for a single class; glt_batch_get_class_table gives all
 * of them) and the measured ms per track.  Synchronous; invalidates a
 * captured graph.  The proposal stage is not timed. */
int glt_batch_autotune(glt_batch* batch, const double* init_dev, glt_result* out_dev, int reps,
                       int* best_cluster, int* best_threads, float* best_ms, void* stream);

/* Sets one (cluster, threads) shape for every stream of the batch.
 * Invalidates a captured graph. */
int glt_batch_set_shape(glt_batch* batch, int cluster, int threads);

/* Launch classes: the streams in the batch's launch order (heaviest first,
 * by point capacity times samples per point, then frame width) split into a
 * heavy class, the first
 * `heavy` streams, tracked with (heavy_cluster, heavy_threads), and a light
 * class, the rest, with (light_cluster, light_threads).  The two classes run
 * as concurrent launches: glt_batch_track forks the light class onto an
 * internal stream and joins it back into the caller's stream; a captured
 * graph holds them as parallel nodes.  heavy = S (or 0) is one launch with
 * the heavy (light) shape.  Invalidates a captured graph.
 * Errors: INVALID_ARG (heavy outside [0, S], a shape that cannot launch). */
int glt_batch_set_classes(glt_batch* batch, int heavy, int heavy_cluster, int heavy_threads,
                          int light_cluster, int light_threads);

/* The batch's first two launch classes (any pointer may be NULL): heavy = the
 * first stream of class 1 (S with one class), the shapes of classes 0 and 1
 * (class 0's twice with one class). */
int glt_batch_get_classes(const glt_batch* batch, int* heavy, int* heavy_cluster,
                          int* heavy_threads, int* light_cluster, int* light_threads);

/* Launch classes in proportion to work (the paper has no counterpart: a
 * batching policy).  Stream i of the launch order gets the smallest
 * power-of-two cluster c <= 16 with c * points_per_cta >= its point capacity
 * in 8-sample units (max_points * samples per point / 8), reduced to the
 * largest size that can launch with `threads`; the streams of one cluster
 * size form a class (at most 5, contiguous in the launch order) and the
 * classes run as concurrent launches, as in glt_batch_set_classes.  Keeps the
 * points per thread about equal across streams, so that the streams with the
 * most points do not set the batch's critical path.  Invalidates a captured
 * graph.  Errors: INVALID_ARG (points_per_cta < 1, a thread count with which
 * no cluster size can launch). */
int glt_batch_set_proportional(glt_batch* batch, int points_per_cta, int threads);

/* All launch classes: *nclass = their number; for k < min(*nclass, max),
 * first[k] = the class's first stream in the launch order (it runs to the
 * next class's first, the last to S), cluster[k] and threads[k] its shape
 * (any array may be NULL).  Errors: INVALID_ARG (batch or nclass NULL,
 * max < 0). */
int glt_batch_get_class_table(const glt_batch* batch, int max, int* first, int* cluster,
                              int* threads, int* nclass);

/* Allocation-free linearisation.  The paper has no counterpart.  It serves
 * callers that may not allocate device memory at the point where they need a
 * linearisation and therefore cannot use glt_create: real-time loops whose
 * memory budget is fixed at start-up, and plugins whose host framework owns
 * every device allocation.  It computes what glt_debug_linearize computes
 * (same arithmetic) on caller-owned DEVICE buffers: the REF and CUR images of
 * pyramid level `level` (uint8, (width >> level) x (height >> level), row
 * pitches in bytes >= the level width), n map points uvd_dev[n][3] =
 * (u0, v0, depth) at level-0 pixels, level-0 intrinsics, the state (T
 * host-side 3x4, a, b), Huber k and zmin; the reference patch is sampled on
 * the fly.  It writes out_dev[46] (device doubles): the 36 upper-triangle
 * entries of H row by row, g (8), the Huber energy E and the valid-sample
 * count n.  Asynchronous on `stream`; calls no cudaMalloc or cudaFree.
 * Scratch: a file-scope device array of 512 block partial sums plus a ticket
 * (n <= 65536 points; larger n returns GLT_ERR_CAPACITY before any GPU work),
 * which every GPU that loads the library keeps until the process exits.
 * The first call on a device looks up that array's device address
 * (cudaGetSymbolAddress) and keeps it for the device; make that first call
 * before any stream capture.  The kept address does not survive
 * cudaDeviceReset (or any other reset of the device's primary context):
 * after one, this entry point must not be called again in the process.
 * Every call shares the array and clears its ticket counter first, so calls
 * that overlap on the GPU (on different streams, or concurrently from several
 * host threads) race and must be serialised by the caller. */
int glt_linearize_noalloc(const uint8_t* ref_dev, int ref_pitch, const uint8_t* cur_dev,
                          int cur_pitch, int width, int height, int level, double fx, double fy,
                          double cx, double cy, const float* uvd_dev, int n, const double T[12],
                          double a, double b, double huber_k, double zmin, double* out_dev,
                          void* stream);

/* ---------------------------------------------------------------------------
 * Learned initial-pose proposal.  The paper has no counterpart: it seeds each
 * frame with a constant-velocity guess only.  This optional stage maps the
 * coarsest-level residual image of a stream (current minus reference at the
 * identity warp, 40 x 30, divided by 64) and the stream's previous inter-frame
 * motion (a 6-vector: log of that motion divided by 0.02, computed by the
 * proposal stage from the motion itself) to an increment of the initial
 * state, which then starts the same LM solve.
 * Network: 3 x (conv 3x3, stride 2, zero padding 1, ReLU) with 16, 32, 64
 * channels -> flatten (1280) ++ motion (6) -> fc 128 + ReLU -> fc 8.
 * The 8 outputs y give delta = (0.01 y[0..6], y[7]) and the proposal
 * T' = T_init exp(delta[0..5]), a' = a + delta[6], b' = b + delta[7].
 * Parameters are one flat FP32 array of GLT_NN_PARAMS values: conv1.w
 * [16,1,3,3], conv1.b [16], conv2.w [32,16,3,3], conv2.b [32], conv3.w
 * [64,32,3,3], conv3.b [64], fc1.w [128,1286], fc1.b [128], fc2.w [8,128],
 * fc2.b [8], each row-major.  The kernels use BF16 copies of the weights
 * (rounded to nearest even from the FP32 master copy), FP32 activations and
 * FP32 accumulation in a fixed order (results are deterministic).
 * Inputs x are [B][1200] (row-major 30 x 40 images), motions m [B][6],
 * outputs and targets [B][8], all FP32 DEVICE arrays.
 * A network object is not thread-safe; work on it is ordered on the stream
 * passed to each call, and it must not be used on two streams at once.
 * ------------------------------------------------------------------------- */
#define GLT_NN_PARAMS 189064
#define GLT_NN_INPUT 1200
#define GLT_NN_MOTION 6
#define GLT_NN_OUTPUT 8

/* Allocates a network for batches of up to max_batch (1..65536) samples:
 * FP32 master weights, BF16 copy, Adam moments, activations.  Weights are
 * uninitialised until glt_nn_set_params.  Errors: INVALID_ARG, CUDA. */
int glt_nn_create(int max_batch, glt_nn** out);
void glt_nn_destroy(glt_nn* nn);

/* Copies `count` (= GLT_NN_PARAMS) FP32 host values into the master weights,
 * refreshes the BF16 copy and resets the Adam state.  Synchronous. */
int glt_nn_set_params(glt_nn* nn, const float* params_host, int count);

/* Copies the FP32 master weights to host memory.  Synchronous. */
int glt_nn_get_params(glt_nn* nn, float* params_host, int count);

/* Inference: y_dev[B][8] = network(x_dev, m_dev).  Asynchronous. */
int glt_nn_forward(glt_nn* nn, const float* x_dev, const float* m_dev, float* y_dev, int B,
                   void* stream);

/* Loss L = 0.5/B sum_b ||y_b - t_b||^2 and its gradient with respect to every
 * parameter (with the BF16 weights used in the forward and backward passes),
 * written to host grad_host[GLT_NN_PARAMS] and *loss_host (may be NULL).
 * Synchronous.  Changes no weights. */
int glt_nn_gradient(glt_nn* nn, const float* x_dev, const float* m_dev, const float* t_dev, int B,
                    float* grad_host, float* loss_host, void* stream);

/* One training step: forward, backward, Adam (beta1 0.9, beta2 0.999,
 * eps 1e-8, bias-corrected, learning rate lr > 0) on the FP32 master weights,
 * BF16 refresh.  The pre-update loss goes to the device float *loss_dev (may
 * be NULL).  Asynchronous. */
int glt_nn_train_step(glt_nn* nn, const float* x_dev, const float* m_dev, const float* t_dev,
                      int B, float lr, float* loss_dev, void* stream);

/* Writes a training checkpoint of `nn` to the file `path` (binary,
 * little-endian): the 8 bytes "GLTNNCK1", int32 GLT_NN_PARAMS, int32 Adam step
 * count, then GLT_NN_PARAMS FP32 values each of the master weights and of the
 * Adam first and second moments.  Synchronous (waits for the device).
 * Errors: INVALID_ARG (NULL), IO, CUDA. */
int glt_nn_save(glt_nn* nn, const char* path);

/* Reads `path` into `nn`: a checkpoint written by glt_nn_save (weights, Adam
 * moments and step restored, so training resumes bit for bit), or a NumPy
 * .npy file holding GLT_NN_PARAMS little-endian FP32 values in one dimension
 * (weights only, as glt_nn_set_params: Adam state reset).  Refreshes the BF16
 * copy.  Synchronous.  Errors: INVALID_ARG (NULL, unknown format, wrong
 * size), IO (cannot open, short file), CUDA. */
int glt_nn_load(glt_nn* nn, const char* path);

/* Attaches `nn` (or detaches it, nn = NULL) as the proposal stage of the
 * batch: from then on glt_batch_track and glt_batch_capture first build each
 * stream's residual image from its REF and CUR coarsest levels, compute each
 * stream's motion input log(M) / 0.02 in FP64 from motion_dev[S][12] (a DEVICE
 * array of doubles read at run time: the last inter-frame motion M of every
 * stream, row-major 3x4, as glt_state.motion holds it; the identity for a
 * stream without two tracked frames), run the network on all S streams and
 * start every stream's LM from the proposed state instead of init_dev.  Every tracker of the batch needs a 40 x 30 coarsest
 * level (640 x 480 with 5 levels, 320 x 240 with 4).  The batch references
 * the network, which must outlive it and must not be trained while the batch
 * uses it.  Invalidates a captured graph.  The autotuner ignores the stage.
 * Errors: INVALID_ARG (size, max_batch < S), CUDA. */
int glt_batch_set_proposal(glt_batch* batch, glt_nn* nn, const double* motion_dev);

/* Name of a return code (GLT_OK, GLT_ERR_*) or, for a positive value, of the
 * glt_result.status bits it holds ("ok", "too few points", "not positive
 * definite", "diverged", joined by "|"); never NULL, static storage. */
const char* glt_status_string(int code);

/* Thread-local message of the last error (never NULL). */
const char* glt_last_error(void);

/* Library version string. */
const char* glt_version(void);

#ifdef __cplusplus
}
#endif
#endif /* GLT_H */
