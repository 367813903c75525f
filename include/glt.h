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

/* glt_result.status bits (per-frame solver outcomes) */
#define GLT_TRACK_TOO_FEW_POINTS 1 /* a level had fewer than min_valid samples */
#define GLT_TRACK_NOT_PD 2         /* the damped normal matrix was not positive definite */

/* pyramid slots */
#define GLT_REF 0
#define GLT_CUR 1

/* precision modes */
#define GLT_FP32 0  /* uint8 levels, FP32 residuals/Jacobians/sums, FP64 solve */
#define GLT_MIXED 1 /* FP16 (I, gx, gy) levels, FP32 math, Kahan FP32 block sums, FP64 solve */

typedef struct glt_tracker glt_tracker;
typedef struct glt_batch glt_batch;

typedef struct glt_config {
    int width, height;          /* level-0 frame size in pixels (>= 16 each) */
    int levels;                 /* pyramid levels, 1..GLT_MAX_LEVELS; level l is
                                   floor(size / 2^l) and must be >= 8 pixels */
    double fx, fy, cx, cy;      /* level-0 pinhole intrinsics; level l uses f/2^l, c/2^l */
    int max_points;             /* capacity of glt_set_map_points */
    int max_iters[GLT_MAX_LEVELS]; /* LM candidate evaluations per level (0 skips a level) */
    double huber_k;             /* Huber threshold in gray levels (weight k/|r| beyond it) */
    double lambda0;             /* initial LM damping of diag(H) at each level start */
    double lambda_up;           /* damping factor after a rejected candidate */
    double lambda_down;         /* damping factor after an accepted candidate */
    double eps_step;            /* stop a level once max |delta_xi| < eps_step */
    double eps_cost;            /* ... or once a rejected candidate raised the cost by
                                   no more than eps_cost * cost */
    double accept_step;         /* candidates with max |delta_xi| < accept_step are taken
                                   even if the cost rose (Gauss-Newton steps near
                                   convergence); larger ones only if it fell */
    int min_valid;              /* minimum valid residual samples per pass */
    double zmin;                /* minimum current-camera depth of a usable point (m) */
    int precision;              /* GLT_FP32 or GLT_MIXED */
    int cluster;                /* CTAs cooperating on one stream (1..16, 0 = auto) */
    int threads;                /* threads per CTA (128, 256 or 512; 0 = auto) */
} glt_config;

typedef struct glt_result {
    double T[12];               /* final pose, row-major 3x4 */
    double a, b;                /* final affine brightness, cur ~ e^a ref + b */
    double cost;                /* mean Huber energy sum(rho)/n at the final state on the
                                   last level that ran (NaN if none ran) */
    int n_valid;                /* valid residual samples behind `cost` */
    int iters_total;            /* candidate evaluations over all levels */
    int iters[GLT_MAX_LEVELS];  /* candidate evaluations per level */
    int passes;                 /* linearisation passes (level starts + candidates) */
    int status;                 /* GLT_TRACK_* bits */
} glt_result;

/* Fills `cfg` with the defaults: 4 levels, 10 iterations per level, Huber 9,
 * lambda0 1e-4 (x4 up, x0.5 down), eps_step 1e-6, eps_cost 0 (off),
 * accept_step 1e-3, min_valid 16, zmin 1e-3, FP32, automatic cluster/threads,
 * max_points 4096. */
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
 * Errors: NO_REFERENCE without map points, INVALID_ARG for non-finite input. */
int glt_track_frame(glt_tracker* trk, const double T_init[12], const double ab_init[2],
                    glt_result* out, void* stream);

/* As glt_track_frame, fully asynchronous: the initial state is read on the
 * device from init_dev[14] = (T[12], a, b) and the result written to the
 * device struct out_dev.  No host synchronisation. */
int glt_track_frame_async(glt_tracker* trk, const double* init_dev, glt_result* out_dev,
                          void* stream);

/* One linearisation (Eqs. 3-5 at a given state) on `level` of the CUR pyramid:
 * the full symmetric H (64 doubles, row-major), g = J^T W r (8; the paper's
 * right-hand side b of Eq. 5 is -g), the Huber energy E and the number of
 * valid samples n, all written to host memory; if `res` is not NULL it gets
 * the N*8 FP32 residuals (NaN for samples of unused points).  Synchronous.
 * Uses a multi-block kernel with a single-pass last-block finish. */
int glt_debug_linearize(glt_tracker* trk, int level, const double T[12], double a, double b,
                        double H[64], double g[8], double* E, int* n, float* res,
                        void* stream);

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
 * all with the same precision).  The batch references, but does not own, the
 * trackers; they must outlive it.  Errors: INVALID_ARG. */
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
 * a CUDA graph owned by the batch (replacing any previous one). */
int glt_batch_capture(glt_batch* batch, const uint8_t* const* frames_dev, const double* init_dev,
                      glt_result* out_dev, void* stream);

/* Replays the captured graph on `stream`.  Errors: INVALID_ARG if none. */
int glt_batch_replay(glt_batch* batch, void* stream);

/* Autotuner: times the batched track over the candidate (cluster, threads)
 * shapes on the current inputs (replaying `reps` times each), keeps the
 * fastest, and reports it.  Synchronous; invalidates a captured graph. */
int glt_batch_autotune(glt_batch* batch, const double* init_dev, glt_result* out_dev, int reps,
                       int* best_cluster, int* best_threads, float* best_ms, void* stream);

/* Sets the (cluster, threads) shape used by glt_batch_track / capture. */
int glt_batch_set_shape(glt_batch* batch, int cluster, int threads);

/* Allocation-free linearisation.  The paper has no counterpart: this entry
 * point exists for callers that must not allocate device memory where they
 * call it -- code recorded into a CUDA graph by stream capture, real-time
 * loops with a memory budget fixed at start-up, plugins whose host framework
 * owns all device memory -- and who therefore cannot use glt_create.
 * It runs one linearisation of Eqs. 3-5 (same arithmetic as
 * glt_debug_linearize) on caller-owned DEVICE buffers: the REF and CUR images
 * of pyramid level `level` (uint8, (width >> level) x (height >> level), row
 * pitches in bytes >= the level width), n map points uvd_dev[n][3] =
 * (u0, v0, depth) at level-0 pixels, level-0 intrinsics, the state (T
 * host-side 3x4, a, b), Huber k and zmin; the reference patch is sampled on
 * the fly.  It writes out_dev[46] (device doubles): the 36 upper-triangle
 * entries of H row by row, g (8), the Huber energy E and the valid-sample
 * count n.  Asynchronous on `stream`; allocates nothing.
 * Scratch: a file-scope device array holding up to 512 block partial sums
 * (n <= 65536 points; larger n returns GLT_ERR_CAPACITY), which every GPU
 * that loads the library keeps until the process exits.  The first call on a
 * device looks up that array's device address (cudaGetSymbolAddress); make
 * that first call before any stream capture.  Every call shares the array
 * and clears its ticket counter first, so calls that overlap on the GPU (on
 * different streams, or concurrently from several host threads) race and
 * must be serialised by the caller. */
int glt_linearize_noalloc(const uint8_t* ref_dev, int ref_pitch, const uint8_t* cur_dev,
                          int cur_pitch, int width, int height, int level, double fx, double fy,
                          double cx, double cy, const float* uvd_dev, int n, const double T[12],
                          double a, double b, double huber_k, double zmin, double* out_dev,
                          void* stream);

/* Thread-local message of the last error (never NULL). */
const char* glt_last_error(void);

/* Library version string. */
const char* glt_version(void);

#ifdef __cplusplus
}
#endif
#endif /* GLT_H */
