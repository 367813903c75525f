/*
 * FP64 CPU oracle of pose-only direct photometric tracking (GLidE-SLAM,
 * Sec. IV "Direct Photometric Tracking").
 *
 * TEST INFRASTRUCTURE ONLY.  This library is the slow, plain reference that
 * the CUDA path is checked against.  Only the test suite, the smoke check and
 * the benchmark's CPU-baseline leg may load it; the product path never does.
 * It shares no code, header, table or helper with the CUDA path.
 *
 * Conventions
 *  - Poses are row-major 3x4 [R|t] doubles.  T maps reference-camera
 *    coordinates to current-camera coordinates: x_c = R x_r + t.  The paper's
 *    world-frame form u_i(T) = pi(T P_i), u_i^0 = pi(T0 P_i) (Eq. 1) is this
 *    with x_r = T0 P_i and T = T_cur * T0^-1.
 *  - Increment delta = (upsilon (3, translation), omega (3, rotation), da, db),
 *    applied as T <- T exp(delta_xi) (Sec. IV-A), a += da, b += db.
 *  - Residual r = I(u(T) + du_k) - e^a I0_k - b (the paper's Eq. 2 has the
 *    opposite sign and no affine term; the sign cancels in the normal
 *    equations).  g = J^T W r, so the paper's right-hand side b of Eq. 5 is -g.
 *  - Level-l intrinsics: f_l = f / 2^l, c_l = c / 2^l.
 *  - Images passed to the linearisation are doubles (uint8 pyramid levels
 *    converted exactly), so that analytic test images can be used too.
 */
#ifndef GLT_ORACLE_H
#define GLT_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    double fx, fy, cx, cy;
} orc_cam;

typedef struct {
    int levels;
    int max_iters[8];
    double huber_k;
    double lambda0, lambda_up, lambda_down;
    double eps_step;
    double eps_step_coarse;
    double eps_cost;
    double accept_step;
    int min_valid;
    double zmin;
    int ic; /* 0: forward Jacobian (current image), 1: inverse-compositional (reference side) */
    int pattern; /* 0: the 8-pixel sparse pattern; odd p (3..11): the paper's p x p patch */
    int affine;  /* 1: estimate (a, b); 0: keep them at their initial values (the paper's form) */
    int hcache;  /* 1 (with ic, affine 0): the pose block of the normal matrix is the
                    per-reference Hessian of orc_ic_hessian times e^{2a}, not the per-pass
                    sum (Sec. IV-B: H precomputed once per reference update) */
} orc_config;

typedef struct {
    double T[12];
    double a, b, cost;
    int n_valid;
    int iters_total;
    int iters[8];
    int passes;
    int status; /* bit 0 too few points, bit 1 not positive definite, bit 2 diverged */
} orc_result;

enum { ORC_TOO_FEW_POINTS = 1, ORC_NOT_PD = 2, ORC_DIVERGED = 4 };

/* the 8-pixel sparse pattern, offsets in level pixels */
extern const int orc_pattern_dx[8];
extern const int orc_pattern_dy[8];

/* Sample offsets of a pattern (0: the 8-pixel pattern; odd p: the p x p patch
 * of Sec. IV-A, row by row from (-(p-1)/2, -(p-1)/2)).  Returns the number of
 * samples K (at most 121), or 0 for an unknown pattern. */
int orc_pattern(int pattern, int* dx, int* dy);

/* As orc_ref_patch for any pattern: I0[N*K]. */
void orc_ref_patch2(const double* img, int W, int H, int level, const float* uvd, int N,
                    int pattern, double* I0, uint8_t* valid);

/* Pyramid (Sec. IV-C "Image pyramids"): one level down. dst is
 * (W/2) x (H/2), row-major contiguous. */
void orc_pyr_down(const uint8_t* src, int W, int H, int pitch, uint8_t* dst);
/* All levels, concatenated row-major (level 0 first, unpadded). */
void orc_build_pyramid(const uint8_t* img, int W, int H, int pitch, int L, uint8_t* out);

/* SE(3) (Sec. IV-A, T <- T exp(delta)) */
void orc_se3_exp(const double xi[6], double T[12]);
void orc_se3_log(const double T[12], double xi[6]);
void orc_se3_mul(const double A[12], const double B[12], double C[12]);

/* map points: x_r = d K^-1 [u0 v0 1] */
void orc_backproject(orc_cam K0, const float* uvd, int N, double* x_r);

/* reference patch I0 at level l (Sec. IV-C "Precompute"): I0[N*8], valid[N] */
void orc_ref_patch(const double* img, int W, int H, int level, const float* uvd, int N,
                   double* I0, uint8_t* valid);

/* One linearisation at state (T, a, b) on level l (Eqs. 1-5 with affine and
 * Huber weights).  I0[N*8] and valid_ref[N] are this level's reference data.
 * Outputs the full symmetric H[64], g[8], energy E = sum rho and n = number
 * of valid residual samples.  Optional per-sample outputs (NULL to skip):
 * res[N*8] (NaN where invalid), jac[N*8*8], wts[N*8], pvalid[N]. */
void orc_linearize(const double* img, int W, int H, orc_cam K0, int level, const double* x_r,
                   const double* I0, const uint8_t* valid_ref, int N, const double T[12],
                   double a, double b, double huber_k, double zmin, double* Hout, double* g,
                   double* E, int* n, double* res, double* jac, double* wts, uint8_t* pvalid);

/* Inverse-compositional cache (Sec. IV-B, the IC Jacobian equation; Sec. IV-C
 * "Precompute IC") on level l of the REFERENCE image: for every point and
 * pattern sample k, J_ic[(8 i + k) * 6 + c] = grad I0(u0_l + du_k) dpi/dx(x_r)
 * [I | -[x_r]x], the pose Jacobian evaluated on the reference side (at the
 * identity pose).  Rows of points with valid_ref[i] = 0 are zero.  Layout
 * [N][K][6] for the pattern's K samples. */
void orc_ic_jacobian(const double* ref, int W, int H, orc_cam K0, int level, const double* x_r,
                     const float* uvd, const uint8_t* valid_ref, int N, int pattern, double* Jic);

/* Per-reference Hessian of one level (Sec. IV-B: with the IC rows fixed, H =
 * J^T J is constant while the reference is; Sec. IV-C "Precompute IC": the
 * per-point contributions H_i reduced over the points into one per-level H):
 * H6[36] (row-major 6x6) = sum over the points with valid_ref[i] of
 * sum_k J_ic(i,k)^T J_ic(i,k), from the [N][K][6] cache of orc_ic_jacobian. */
void orc_ic_hessian(const double* Jic, const uint8_t* valid_ref, int N, int K, double H6[36]);

/* As orc_linearize for any pattern (I0[N*K], per-sample outputs with K
 * samples per point); with Jic non-NULL the pose columns of each Jacobian row
 * are e^a J_ic (the template approximation of the current-side Jacobian: the
 * current image's gradient is not used), the affine columns unchanged. */
void orc_linearize2(const double* img, int W, int H, orc_cam K0, int level, const double* x_r,
                    const double* I0, const uint8_t* valid_ref, const double* Jic, int N,
                    int pattern, const double T[12], double a, double b, double huber_k,
                    double zmin, double* Hout, double* g, double* E, int* n, double* res,
                    double* jac, double* wts, uint8_t* pvalid);

/* Coarse-to-fine LM (Sec. IV-A and the accept/reject schedule of this
 * library).  cur: concatenated double pyramid of the current frame
 * (level-0 first, unpadded, dims from W0, H0).  I0: [L][N][8], valid: [L][N].
 * Optional trace (NULL to skip), one entry per linearisation pass, at most
 * max_trace entries: trace_cost = E/n of that pass (INFINITY if too few
 * samples), trace_info = level * 4 + 2 * accepted + is_candidate,
 * trace_step = max |delta_xi| of the candidate (0 for a level start). */
void orc_track(const double* cur, int W0, int H0, orc_cam K0, const double* x_r,
               const double* I0, const uint8_t* valid, int N, const orc_config* cfg,
               const double T_init[12], double a0, double b0, orc_result* out,
               double* trace_cost, int* trace_info, double* trace_step, int max_trace);
/* As orc_track with cfg->pattern (I0 [L][N][K]) and cfg->affine; with cfg->ic
 * set, Jic is the [L][N*K*6] inverse-compositional cache of orc_ic_jacobian,
 * used by every linearisation of the solve; with cfg->hcache also set (and
 * cfg->affine 0) every pass solves with the per-reference Hessian of
 * orc_ic_hessian scaled by e^{2a} (the rows are e^a J_ic) instead of the pass's
 * own sum, while g, the energy and the sample count stay per pass. */
void orc_track2(const double* cur, int W0, int H0, orc_cam K0, const double* x_r,
                const double* I0, const uint8_t* valid, const double* Jic, int N,
                const orc_config* cfg, const double T_init[12], double a0, double b0,
                orc_result* out, double* trace_cost, int* trace_info, double* trace_step,
                int max_trace);

#ifdef __cplusplus
}
#endif
#endif
