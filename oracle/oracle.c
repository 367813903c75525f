/*
 * FP64 CPU oracle of pose-only direct photometric tracking (GLidE-SLAM,
 * Sec. IV).  TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check
 * and the benchmark's CPU-baseline leg, never by the product path.
 *
 * Every function below is the plain definition written out, in the order the
 * paper states the method, with the readings this library takes where the
 * paper is silent (each one marked "reading:").  No blocking, fusion or
 * reordering beyond the definitions.
 */
#include "oracle.h"

#include <float.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define ORC_PI 3.14159265358979323846

/* Reading: 8-pixel sparse pattern (a DSO-style diamond) instead of the
 * paper's p x p patch (Sec. IV-A, Eq. 2 uses offsets du_k of a patch). */
const int orc_pattern_dx[8] = {0, -2, 2, 0, 0, -1, 1, -1};
const int orc_pattern_dy[8] = {0, 0, 0, -2, 2, -1, -1, 1};

/* ------------------------------------------------------------------------
 * Image pyramid (Sec. IV-C "Image pyramids": blur, then downsample; level 0
 * is full resolution).  Reading: 5-tap binomial kernel [1 4 6 4 1]/16 in
 * each direction, clamp-to-edge borders, even-sample decimation, exact
 * integer sum with round-half-up: p_l(x,y) = (sum w_i w_j p(2x+i, 2y+j) + 128) >> 8.
 * ------------------------------------------------------------------------ */
int orc_pattern(int pattern, int* dx, int* dy)
{
    if (pattern == 0) {
        for (int k = 0; k < 8; ++k) {
            dx[k] = orc_pattern_dx[k];
            dy[k] = orc_pattern_dy[k];
        }
        return 8;
    }
    if (pattern < 3 || pattern > 11 || (pattern & 1) == 0) return 0;
    int h = (pattern - 1) / 2, K = 0;
    for (int j = -h; j <= h; ++j)
        for (int i = -h; i <= h; ++i) {
            dx[K] = i;
            dy[K] = j;
            ++K;
        }
    return K;
}

static int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

void orc_pyr_down(const uint8_t* src, int W, int H, int pitch, uint8_t* dst)
{
    static const int w[5] = {1, 4, 6, 4, 1};
    int Wd = W / 2, Hd = H / 2;
    for (int y = 0; y < Hd; ++y) {
        for (int x = 0; x < Wd; ++x) {
            int s = 0;
            for (int j = -2; j <= 2; ++j) {
                for (int i = -2; i <= 2; ++i) {
                    int sx = clampi(2 * x + i, 0, W - 1);
                    int sy = clampi(2 * y + j, 0, H - 1);
                    s += w[i + 2] * w[j + 2] * (int)src[(size_t)sy * pitch + sx];
                }
            }
            dst[(size_t)y * Wd + x] = (uint8_t)((s + 128) >> 8);
        }
    }
}

void orc_build_pyramid(const uint8_t* img, int W, int H, int pitch, int L, uint8_t* out)
{
    for (int y = 0; y < H; ++y) memcpy(out + (size_t)y * W, img + (size_t)y * pitch, (size_t)W);
    const uint8_t* prev = out;
    size_t off = (size_t)W * H;
    int w = W, h = H;
    for (int l = 1; l < L; ++l) {
        orc_pyr_down(prev, w, h, w, out + off);
        prev = out + off;
        w /= 2;
        h /= 2;
        off += (size_t)w * h;
    }
}

/* ------------------------------------------------------------------------
 * SE(3) (Sec. IV-A: 6-D twist, T <- T exp(delta)).  Closed-form exponential
 * (Rodrigues for R, left Jacobian V for t); series coefficients below a small
 * angle.  Twist order (upsilon, omega): reading, the paper only says three
 * rotational and three translational components.
 * ------------------------------------------------------------------------ */
static void hat(const double w[3], double W[9])
{
    W[0] = 0;     W[1] = -w[2]; W[2] = w[1];
    W[3] = w[2];  W[4] = 0;     W[5] = -w[0];
    W[6] = -w[1]; W[7] = w[0];  W[8] = 0;
}

static void mat3_mul(const double A[9], const double B[9], double C[9])
{
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double s = 0;
            for (int k = 0; k < 3; ++k) s += A[3 * i + k] * B[3 * k + j];
            C[3 * i + j] = s;
        }
}

void orc_se3_exp(const double xi[6], double T[12])
{
    const double* v = xi;
    const double* w = xi + 3;
    double th2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
    double th = sqrt(th2);
    /* R = I + A W + B W^2,  V = I + B W + C W^2 with
     * A = sin(th)/th, B = (1-cos th)/th^2 = 2 sin^2(th/2)/th^2, C = (th - sin th)/th^3;
     * Taylor series of the same functions where the closed forms cancel. */
    double A, B, C;
    if (th < 1e-4) {
        A = 1.0 - th2 / 6.0 + th2 * th2 / 120.0;
        B = 0.5 - th2 / 24.0 + th2 * th2 / 720.0;
    } else {
        double sh = sin(0.5 * th);
        A = sin(th) / th;
        B = 2.0 * sh * sh / th2;
    }
    if (th < 0.1) {
        double t4 = th2 * th2;
        C = 1.0 / 6.0 - th2 / 120.0 + t4 / 5040.0 - t4 * th2 / 362880.0 + t4 * t4 / 39916800.0;
    } else {
        C = (th - sin(th)) / (th2 * th);
    }
    double Wm[9], W2[9];
    hat(w, Wm);
    mat3_mul(Wm, Wm, W2);
    double R[9], V[9];
    for (int i = 0; i < 9; ++i) {
        double I = (i % 4 == 0) ? 1.0 : 0.0;
        R[i] = I + A * Wm[i] + B * W2[i];
        V[i] = I + B * Wm[i] + C * W2[i];
    }
    for (int r = 0; r < 3; ++r) {
        T[4 * r + 0] = R[3 * r + 0];
        T[4 * r + 1] = R[3 * r + 1];
        T[4 * r + 2] = R[3 * r + 2];
        T[4 * r + 3] = V[3 * r + 0] * v[0] + V[3 * r + 1] * v[1] + V[3 * r + 2] * v[2];
    }
}

void orc_se3_log(const double T[12], double xi[6])
{
    double R[9] = {T[0], T[1], T[2], T[4], T[5], T[6], T[8], T[9], T[10]};
    double t[3] = {T[3], T[7], T[11]};
    double vee[3] = {R[7] - R[5], R[2] - R[6], R[3] - R[1]}; /* (R - R^T)^v */
    double s = 0.5 * sqrt(vee[0] * vee[0] + vee[1] * vee[1] + vee[2] * vee[2]);
    double c = 0.5 * (R[0] + R[4] + R[8] - 1.0);
    double th = atan2(s, c);
    double w[3];
    if (th < 1e-4) {
        double k = 0.5 * (1.0 + th * th / 6.0);
        for (int i = 0; i < 3; ++i) w[i] = k * vee[i];
    } else if (th < ORC_PI - 1e-4) {
        double k = th / (2.0 * sin(th));
        for (int i = 0; i < 3; ++i) w[i] = k * vee[i];
    } else {
        /* near pi: axis from the symmetric part R + I = 2 a a^T (approx) */
        int m = 0;
        for (int i = 1; i < 3; ++i)
            if (R[4 * i] > R[4 * m]) m = i;
        double a[3];
        double d = sqrt(0.5 * (R[4 * m] + 1.0));
        for (int i = 0; i < 3; ++i) a[i] = (i == m) ? d : 0.5 * (R[3 * i + m] + R[3 * m + i]) / (2.0 * d);
        double na = sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
        double sgn = (a[0] * vee[0] + a[1] * vee[1] + a[2] * vee[2]) < 0 ? -1.0 : 1.0;
        for (int i = 0; i < 3; ++i) w[i] = sgn * th * a[i] / na;
    }
    /* upsilon = V^-1 t,  V^-1 = I - W/2 + k W^2,  k = (1 - A/(2B)) / th^2 */
    double th2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
    double k;
    if (th < 0.1) {
        double t4 = th2 * th2;
        k = 1.0 / 12.0 + th2 / 720.0 + t4 / 30240.0 + t4 * th2 / 1209600.0;
    } else {
        double sh = sin(0.5 * th);
        double A = sin(th) / th, B = 2.0 * sh * sh / th2;
        k = (1.0 - A / (2.0 * B)) / th2;
    }
    double Wm[9], W2[9];
    hat(w, Wm);
    mat3_mul(Wm, Wm, W2);
    for (int r = 0; r < 3; ++r) {
        double acc = 0;
        for (int j = 0; j < 3; ++j) {
            double I = (r == j) ? 1.0 : 0.0;
            acc += (I - 0.5 * Wm[3 * r + j] + k * W2[3 * r + j]) * t[j];
        }
        xi[r] = acc;
        xi[3 + r] = w[r];
    }
}

void orc_se3_mul(const double A[12], const double B[12], double C[12])
{
    double out[12];
    for (int r = 0; r < 3; ++r) {
        for (int c = 0; c < 4; ++c) {
            double s = (c == 3) ? A[4 * r + 3] : 0.0;
            for (int k = 0; k < 3; ++k) s += A[4 * r + k] * B[4 * k + c];
            out[4 * r + c] = s;
        }
    }
    memcpy(C, out, sizeof(out));
}

/* ------------------------------------------------------------------------
 * Map points and reference patches (Sec. IV-A Eq. 1 and Sec. IV-C
 * "Precompute": sample the reference patch I0 around u_i^0 on every level).
 * Reading: the map point arrives as its reference pixel (u0, v0) and its
 * camera-z depth d, so x_r = d ((u0-cx)/fx, (v0-cy)/fy, 1) and u_i^0 = (u0, v0).
 * ------------------------------------------------------------------------ */
void orc_backproject(orc_cam K0, const float* uvd, int N, double* x_r)
{
    for (int i = 0; i < N; ++i) {
        double u = uvd[3 * i], v = uvd[3 * i + 1], d = uvd[3 * i + 2];
        x_r[3 * i + 0] = d * (u - K0.cx) / K0.fx;
        x_r[3 * i + 1] = d * (v - K0.cy) / K0.fy;
        x_r[3 * i + 2] = d;
    }
}

/* Reading: a sample q is usable iff 1 <= q_x < W-2 and 1 <= q_y < H-2, so
 * both bilinear taps and both central-difference neighbours of each tap lie
 * inside the image; a point is used only if all 8 of its samples are. */
static int sample_inside(double qx, double qy, int W, int H)
{
    return qx >= 1.0 && qx < (double)(W - 2) && qy >= 1.0 && qy < (double)(H - 2);
}

static double px(const double* img, int W, int x, int y) { return img[(size_t)y * W + x]; }

/* Bilinear interpolation (Sec. IV-A, "intensities are sampled bilinearly"). */
static double bilinear(const double* img, int W, double qx, double qy)
{
    int x0 = (int)floor(qx), y0 = (int)floor(qy);
    double al = qx - x0, be = qy - y0;
    return (1 - al) * (1 - be) * px(img, W, x0, y0) + al * (1 - be) * px(img, W, x0 + 1, y0) +
           (1 - al) * be * px(img, W, x0, y0 + 1) + al * be * px(img, W, x0 + 1, y0 + 1);
}

/* Image differentiation (Sec. IV-C): central differences per pixel, then the
 * gradient images are interpolated with the same bilinear weights. */
static double grad_x(const double* img, int W, int x, int y)
{
    return 0.5 * (px(img, W, x + 1, y) - px(img, W, x - 1, y));
}
static double grad_y(const double* img, int W, int x, int y)
{
    return 0.5 * (px(img, W, x, y + 1) - px(img, W, x, y - 1));
}
static void bilinear_grad(const double* img, int W, double qx, double qy, double* gx, double* gy)
{
    int x0 = (int)floor(qx), y0 = (int)floor(qy);
    double al = qx - x0, be = qy - y0;
    double w00 = (1 - al) * (1 - be), w10 = al * (1 - be), w01 = (1 - al) * be, w11 = al * be;
    *gx = w00 * grad_x(img, W, x0, y0) + w10 * grad_x(img, W, x0 + 1, y0) +
          w01 * grad_x(img, W, x0, y0 + 1) + w11 * grad_x(img, W, x0 + 1, y0 + 1);
    *gy = w00 * grad_y(img, W, x0, y0) + w10 * grad_y(img, W, x0 + 1, y0) +
          w01 * grad_y(img, W, x0, y0 + 1) + w11 * grad_y(img, W, x0 + 1, y0 + 1);
}

void orc_ref_patch(const double* img, int W, int H, int level, const float* uvd, int N,
                   double* I0, uint8_t* valid)
{
    orc_ref_patch2(img, W, H, level, uvd, N, 0, I0, valid);
}

void orc_ref_patch2(const double* img, int W, int H, int level, const float* uvd, int N,
                    int pattern, double* I0, uint8_t* valid)
{
    int dx[121], dy[121];
    int K = orc_pattern(pattern, dx, dy);
    double s = ldexp(1.0, -level);
    for (int i = 0; i < N; ++i) {
        double u = uvd[3 * i] * s, v = uvd[3 * i + 1] * s;
        int ok = uvd[3 * i + 2] > 0; /* a map point needs a positive depth */
        for (int k = 0; k < K && ok; ++k) ok = sample_inside(u + dx[k], v + dy[k], W, H);
        valid[i] = (uint8_t)ok;
        for (int k = 0; k < K; ++k)
            I0[(size_t)K * i + k] = ok ? bilinear(img, W, u + dx[k], v + dy[k]) : 0.0;
    }
}

/* ------------------------------------------------------------------------
 * Inverse-compositional cache (Sec. IV-B: J_ik = grad I0(u_i^0 + du_k)
 * dpi/dx dx/ddelta with x = T0 P_i, i.e. evaluated on the reference side;
 * Sec. IV-C "Precompute IC": computed once per reference and level).
 * ------------------------------------------------------------------------ */
void orc_ic_jacobian(const double* ref, int W, int H, orc_cam K0, int level, const double* x_r,
                     const float* uvd, const uint8_t* valid_ref, int N, int pattern, double* Jic)
{
    int dx[121], dy[121];
    int K = orc_pattern(pattern, dx, dy);
    double s = ldexp(1.0, -level);
    double fx = K0.fx * s, fy = K0.fy * s;
    (void)H;
    for (int i = 0; i < N; ++i) {
        double* Ji = Jic + (size_t)i * K * 6;
        memset(Ji, 0, (size_t)K * 6 * sizeof(double));
        if (!valid_ref[i]) continue;
        const double* X = x_r + 3 * i;
        /* dpi/dx at x_r and [I | -[x_r]x] */
        double dpi[6] = {fx / X[2], 0, -fx * X[0] / (X[2] * X[2]),
                         0, fy / X[2], -fy * X[1] / (X[2] * X[2])};
        double Xh[9];
        hat(X, Xh);
        double Jg[12];
        for (int r = 0; r < 2; ++r)
            for (int c = 0; c < 6; ++c) {
                double acc = 0;
                for (int k = 0; k < 3; ++k) {
                    double m = c < 3 ? (k == c ? 1.0 : 0.0) : -Xh[3 * k + (c - 3)];
                    acc += dpi[3 * r + k] * m;
                }
                Jg[6 * r + c] = acc;
            }
        double u = uvd[3 * i] * s, v = uvd[3 * i + 1] * s;
        for (int k = 0; k < K; ++k) {
            double gx, gy;
            bilinear_grad(ref, W, u + dx[k], v + dy[k], &gx, &gy);
            for (int c = 0; c < 6; ++c) Ji[6 * k + c] = gx * Jg[c] + gy * Jg[6 + c];
        }
    }
}

void orc_ic_hessian(const double* Jic, const uint8_t* valid_ref, int N, int K, double H6[36])
{
    memset(H6, 0, 36 * sizeof(double));
    for (int i = 0; i < N; ++i) {
        if (!valid_ref[i]) continue;
        for (int k = 0; k < K; ++k) {
            const double* J = Jic + ((size_t)K * i + k) * 6;
            for (int p = 0; p < 6; ++p)
                for (int q = 0; q < 6; ++q) H6[6 * p + q] += J[p] * J[q];
        }
    }
}

/* ------------------------------------------------------------------------
 * Linearisation (Sec. IV-A Eqs. 1-5; forward form of Sec. IV-B: J uses the
 * current image's gradient at the warped location; with Jic, the
 * inverse-compositional form: J uses the cached reference-side rows).
 * ------------------------------------------------------------------------ */
void orc_linearize(const double* img, int W, int H, orc_cam K0, int level, const double* x_r,
                   const double* I0, const uint8_t* valid_ref, int N, const double T[12],
                   double a, double b, double huber_k, double zmin, double* Hout, double* g,
                   double* E, int* n, double* res, double* jac, double* wts, uint8_t* pvalid)
{
    orc_linearize2(img, W, H, K0, level, x_r, I0, valid_ref, NULL, N, 0, T, a, b, huber_k, zmin,
                   Hout, g, E, n, res, jac, wts, pvalid);
}

void orc_linearize2(const double* img, int W, int H, orc_cam K0, int level, const double* x_r,
                    const double* I0, const uint8_t* valid_ref, const double* Jic, int N,
                    int pattern, const double T[12], double a, double b, double huber_k,
                    double zmin, double* Hout, double* g, double* E, int* n, double* res,
                    double* jac, double* wts, uint8_t* pvalid)
{
    int pdx[121], pdy[121];
    int K = orc_pattern(pattern, pdx, pdy);
    double s = ldexp(1.0, -level);
    double fx = K0.fx * s, fy = K0.fy * s, cx = K0.cx * s, cy = K0.cy * s;
    double R[9] = {T[0], T[1], T[2], T[4], T[5], T[6], T[8], T[9], T[10]};
    double t[3] = {T[3], T[7], T[11]};
    double ea = exp(a);
    memset(Hout, 0, 64 * sizeof(double));
    memset(g, 0, 8 * sizeof(double));
    *E = 0;
    *n = 0;
    for (int i = 0; i < N; ++i) {
        const double* X = x_r + 3 * i;
        if (res)
            for (int k = 0; k < K; ++k) res[(size_t)K * i + k] = NAN;
        if (jac) memset(jac + (size_t)K * 8 * i, 0, (size_t)K * 8 * sizeof(double));
        if (wts) memset(wts + (size_t)K * i, 0, (size_t)K * sizeof(double));
        if (pvalid) pvalid[i] = 0;
        if (!valid_ref[i]) continue;
        /* x_c = R x_r + t; pi(x_c) with level intrinsics (Eq. 1) */
        double xc[3];
        for (int r = 0; r < 3; ++r) xc[r] = R[3 * r] * X[0] + R[3 * r + 1] * X[1] + R[3 * r + 2] * X[2] + t[r];
        if (!(xc[2] > zmin)) continue;
        double u = fx * xc[0] / xc[2] + cx;
        double v = fy * xc[1] / xc[2] + cy;
        int ok = 1;
        for (int k = 0; k < K && ok; ++k) ok = sample_inside(u + pdx[k], v + pdy[k], W, H);
        if (!ok) continue;
        if (pvalid) pvalid[i] = 1;
        /* geometric Jacobian d u / d delta_xi = dpi/dx_c * R [I | -[x_r]x]
         * (right perturbation T exp(delta): x_c(delta) = R exp(delta) x_r + t) */
        double dpi[6] = {fx / xc[2], 0, -fx * xc[0] / (xc[2] * xc[2]),
                         0, fy / xc[2], -fy * xc[1] / (xc[2] * xc[2])};
        double M[18]; /* 3x6 = R [I | -[x_r]x] */
        double Xh[9];
        hat(X, Xh);
        for (int r = 0; r < 3; ++r) {
            for (int c = 0; c < 3; ++c) {
                M[6 * r + c] = R[3 * r + c];
                double acc = 0;
                for (int k = 0; k < 3; ++k) acc += R[3 * r + k] * Xh[3 * k + c];
                M[6 * r + 3 + c] = -acc;
            }
        }
        double Jg[12]; /* 2x6 */
        for (int r = 0; r < 2; ++r)
            for (int c = 0; c < 6; ++c) {
                double acc = 0;
                for (int k = 0; k < 3; ++k) acc += dpi[3 * r + k] * M[6 * k + c];
                Jg[6 * r + c] = acc;
            }
        for (int k = 0; k < K; ++k) {
            double qx = u + pdx[k], qy = v + pdy[k];
            double I = bilinear(img, W, qx, qy);
            double gx, gy;
            bilinear_grad(img, W, qx, qy, &gx, &gy);
            double i0 = I0[(size_t)K * i + k];
            double r = I - ea * i0 - b;
            /* Huber weight and energy (k = huber_k) */
            double ar = fabs(r);
            double w = ar <= huber_k ? 1.0 : huber_k / ar;
            double rho = ar <= huber_k ? 0.5 * r * r : huber_k * ar - 0.5 * huber_k * huber_k;
            double J[8];
            if (Jic)
                for (int c = 0; c < 6; ++c) J[c] = ea * Jic[((size_t)K * i + k) * 6 + c];
            else
                for (int c = 0; c < 6; ++c) J[c] = gx * Jg[c] + gy * Jg[6 + c];
            J[6] = -ea * i0;
            J[7] = -1.0;
            for (int p = 0; p < 8; ++p) {
                for (int q = 0; q < 8; ++q) Hout[8 * p + q] += w * J[p] * J[q];
                g[p] += w * J[p] * r;
            }
            *E += rho;
            *n += 1;
            if (res) res[(size_t)K * i + k] = r;
            if (jac) memcpy(jac + ((size_t)K * i + k) * 8, J, sizeof(J));
            if (wts) wts[(size_t)K * i + k] = w;
        }
    }
}

/* ------------------------------------------------------------------------
 * Coarse-to-fine solve (Sec. IV-A: coarser level initialises the finer one,
 * bounded iterations per level; Sec. IV-C "Track": Cholesky solve of the
 * normal equations, then T <- T exp(delta)).
 * Reading: Gauss-Newton steps safeguarded by Levenberg-Marquardt damping of
 * diag(H).  A candidate is taken if it lowers the mean Huber energy E/n, or
 * if its rotational/translational part is below accept_step (small steps are
 * Gauss-Newton steps, as in the paper; the safeguard only screens large
 * ones).  A level stops after max_iters candidates, once a step is
 * below eps_step (eps_step_coarse on the levels above the finest), or when a
 * rejected candidate raised the cost by no more than eps_cost * cost.
 * Reading (a level's final step): a step below the level's stop threshold
 * (eps_step_coarse above the finest level, eps_step on it) that is also below
 * accept_step would be taken whatever its cost and would end the level; it is
 * therefore taken without a pass of its own.  Above the finest level the next
 * level's start pass is the first evaluation of the new state; on the finest
 * level the reported cost and sample count are those of the last evaluated
 * state, which the returned pose differs from by that final step.
 * ------------------------------------------------------------------------ */
static int cholesky_solve8(const double A[64], const double g[8], double delta[8])
{
    double L[64];
    memset(L, 0, sizeof(L));
    for (int j = 0; j < 8; ++j) {
        double d = A[8 * j + j];
        for (int k = 0; k < j; ++k) d -= L[8 * j + k] * L[8 * j + k];
        if (!(d > 0.0) || !(d > 1e-13 * A[8 * j + j])) return 0;
        L[8 * j + j] = sqrt(d);
        for (int i = j + 1; i < 8; ++i) {
            double s = A[8 * i + j];
            for (int k = 0; k < j; ++k) s -= L[8 * i + k] * L[8 * j + k];
            L[8 * i + j] = s / L[8 * j + j];
        }
    }
    double y[8];
    for (int i = 0; i < 8; ++i) { /* L y = -g */
        double s = -g[i];
        for (int k = 0; k < i; ++k) s -= L[8 * i + k] * y[k];
        y[i] = s / L[8 * i + i];
    }
    for (int i = 7; i >= 0; --i) { /* L^T delta = y */
        double s = y[i];
        for (int k = i + 1; k < 8; ++k) s -= L[8 * k + i] * delta[k];
        delta[i] = s / L[8 * i + i];
    }
    return 1;
}

/* Sec. IV-B / IV-C: the pose block of the pass's normal matrix replaced by
 * the per-reference Hessian H6 of the level, scaled by e^{2a} because the
 * rows the pass uses are e^a J_ic; the affine rows and columns are cleared
 * (the affine pair is held fixed in this form, so the solve never uses them). */
static void use_cached_hessian(double Hm[64], double g[8], const double H6[36], double a)
{
    double s = exp(2.0 * a);
    memset(Hm, 0, 64 * sizeof(double));
    for (int p = 0; p < 6; ++p)
        for (int q = 0; q < 6; ++q) Hm[8 * p + q] = s * H6[6 * p + q];
    g[6] = 0.0;
    g[7] = 0.0;
}

static int sums_are_finite(const double Hm[64], const double g[8], double E)
{
    int ok = isfinite(E);
    for (int i = 0; i < 64; ++i) ok = ok && isfinite(Hm[i]);
    for (int i = 0; i < 8; ++i) ok = ok && isfinite(g[i]);
    return ok;
}

static void trace_pass(orc_result* out, double* tc, int* ti, double* ts, int max_trace,
                       double cost, int level, int accepted, int candidate, double step)
{
    int k = out->passes;
    if (tc && k < max_trace) tc[k] = cost;
    if (ti && k < max_trace) ti[k] = level * 4 + 2 * accepted + candidate;
    if (ts && k < max_trace) ts[k] = step;
    out->passes = k + 1;
}

void orc_track(const double* cur, int W0, int H0, orc_cam K0, const double* x_r,
               const double* I0, const uint8_t* valid, int N, const orc_config* cfg,
               const double T_init[12], double a0, double b0, orc_result* out,
               double* trace_cost, int* trace_info, double* trace_step, int max_trace)
{
    orc_config c = *cfg;
    c.pattern = 0;
    c.ic = 0;
    orc_track2(cur, W0, H0, K0, x_r, I0, valid, NULL, N, &c, T_init, a0, b0, out, trace_cost,
               trace_info, trace_step, max_trace);
}

void orc_track2(const double* cur, int W0, int H0, orc_cam K0, const double* x_r,
                const double* I0, const uint8_t* valid, const double* Jic, int N,
                const orc_config* cfg, const double T_init[12], double a0, double b0,
                orc_result* out, double* trace_cost, int* trace_info, double* trace_step,
                int max_trace)
{
    int L = cfg->levels;
    size_t off[8];
    int Ws[8], Hs[8];
    size_t o = 0;
    int w = W0, h = H0;
    for (int l = 0; l < L; ++l) {
        off[l] = o;
        Ws[l] = w;
        Hs[l] = h;
        o += (size_t)w * h;
        w /= 2;
        h /= 2;
    }
    double T[12], a = a0, b = b0;
    memcpy(T, T_init, sizeof(T));
    /* Reading: the initial rotation is projected back onto SO(3) by
     * Gram-Schmidt on its rows (r0 normalised, r1 made orthogonal to r0 and
     * normalised, r2 = r0 x r1) once per frame, so a caller's accumulated
     * rounding does not carry into the solve; inside a frame poses are only
     * composed with exact exponentials. */
    {
        double n0 = sqrt(T[0] * T[0] + T[1] * T[1] + T[2] * T[2]);
        for (int c = 0; c < 3; ++c) T[c] /= n0;
        double d = T[4] * T[0] + T[5] * T[1] + T[6] * T[2];
        for (int c = 0; c < 3; ++c) T[4 + c] -= d * T[c];
        double n1 = sqrt(T[4] * T[4] + T[5] * T[5] + T[6] * T[6]);
        for (int c = 0; c < 3; ++c) T[4 + c] /= n1;
        T[8] = T[1] * T[6] - T[2] * T[5];
        T[9] = T[2] * T[4] - T[0] * T[6];
        T[10] = T[0] * T[5] - T[1] * T[4];
    }
    memset(out, 0, sizeof(*out));
    out->cost = NAN;
    /* Reading (failure detection): a start that is not finite (or whose
     * rotation Gram-Schmidt cannot orthonormalise) is not solved;
     * a pass whose sums are not finite is unusable (like one with too few
     * samples) and a candidate state that is not finite ends the level; each
     * sets the DIVERGED bit. */
    {
        int finite_start = isfinite(a) && isfinite(b);
        for (int i = 0; i < 12; ++i) finite_start = finite_start && isfinite(T[i]);
        if (!finite_start) {
            out->status |= ORC_DIVERGED;
            memcpy(out->T, T, sizeof(T));
            out->a = a;
            out->b = b;
            return;
        }
    }
    double Hm[64], g[8], E;
    int n;
    int pdx[121], pdy[121];
    const int K = orc_pattern(cfg->pattern, pdx, pdy);
    const int hcache = cfg->hcache && cfg->ic && Jic && !cfg->affine;
    for (int l = L - 1; l >= 0; --l) {
        if (cfg->max_iters[l] <= 0) continue;
        const double* img = cur + off[l];
        const double* I0l = I0 + (size_t)l * N * K;
        const uint8_t* vl = valid + (size_t)l * N;
        const double* Jl = (cfg->ic && Jic) ? Jic + (size_t)l * N * K * 6 : NULL;
        double H6[36];
        if (hcache) orc_ic_hessian(Jl, vl, N, K, H6);
        orc_linearize2(img, Ws[l], Hs[l], K0, l, x_r, I0l, vl, Jl, N, cfg->pattern, T, a, b,
                       cfg->huber_k, cfg->zmin, Hm, g, &E, &n, NULL, NULL, NULL, NULL);
        if (hcache) use_cached_hessian(Hm, g, H6, a);
        int sums_finite = sums_are_finite(Hm, g, E);
        int enough = n >= cfg->min_valid && n > 0 && sums_finite;
        trace_pass(out, trace_cost, trace_info, trace_step, max_trace, enough ? E / n : INFINITY,
                   l, 0, 0, 0.0);
        if (!enough) {
            out->status |= sums_finite ? ORC_TOO_FEW_POINTS : ORC_DIVERGED;
            continue;
        }
        double cost = E / n;
        double lambda = cfg->lambda0;
        int it = 0;
        while (it < cfg->max_iters[l]) {
            double A[64], delta[8], gs[8];
            memcpy(A, Hm, sizeof(A));
            memcpy(gs, g, sizeof(gs));
            if (!cfg->affine) {
                /* (a, b) held fixed: the affine rows and columns become the
                 * identity and their right-hand side zero, so da = db = 0 and
                 * the pose block is solved alone */
                for (int r = 6; r < 8; ++r) {
                    for (int c = 0; c < 8; ++c) A[8 * r + c] = A[8 * c + r] = 0.0;
                    A[8 * r + r] = 1.0;
                    gs[r] = 0.0;
                }
            }
            for (int d = 0; d < 8; ++d) A[8 * d + d] += lambda * A[8 * d + d];
            if (!cholesky_solve8(A, gs, delta)) {
                out->status |= ORC_NOT_PD;
                break;
            }
            double dT[12], Tn[12];
            orc_se3_exp(delta, dT);
            orc_se3_mul(T, dT, Tn);
            double an = a + delta[6], bn = b + delta[7];
            int cand_finite = isfinite(an) && isfinite(bn);
            for (int d = 0; d < 12; ++d) cand_finite = cand_finite && isfinite(Tn[d]);
            if (!cand_finite) {
                out->status |= ORC_DIVERGED;
                break;
            }
            double m = 0;
            for (int d = 0; d < 6; ++d) m = fmax(m, fabs(delta[d]));
            if (m < (l > 0 ? cfg->eps_step_coarse : cfg->eps_step) && m < cfg->accept_step) {
                /* the level's last step, taken without a pass of its own */
                memcpy(T, Tn, sizeof(T));
                a = an;
                b = bn;
                ++it;
                break;
            }
            double Hn[64], gn[8], En;
            int nn;
            orc_linearize2(img, Ws[l], Hs[l], K0, l, x_r, I0l, vl, Jl, N, cfg->pattern, Tn, an,
                           bn, cfg->huber_k, cfg->zmin, Hn, gn, &En, &nn, NULL, NULL, NULL, NULL);
            if (hcache) use_cached_hessian(Hn, gn, H6, an);
            ++it;
            int nfin = sums_are_finite(Hn, gn, En);
            if (!nfin) out->status |= ORC_DIVERGED;
            double cn = (nn >= cfg->min_valid && nn > 0 && nfin) ? En / nn : INFINITY;
            int accepted = cn < cost || (cn < INFINITY && m < cfg->accept_step);
            trace_pass(out, trace_cost, trace_info, trace_step, max_trace, cn, l, accepted, 1, m);
            int flat = !accepted && cn - cost <= cfg->eps_cost * cost;
            if (accepted) {
                memcpy(T, Tn, sizeof(T));
                a = an;
                b = bn;
                memcpy(Hm, Hn, sizeof(Hm));
                memcpy(g, gn, sizeof(g));
                cost = cn;
                n = nn;
                lambda *= cfg->lambda_down;
            } else {
                lambda *= cfg->lambda_up;
            }
            if (m < (l > 0 ? cfg->eps_step_coarse : cfg->eps_step) || flat) break;
        }
        out->iters[l] = it;
        out->iters_total += it;
        out->cost = cost;
        out->n_valid = n;
    }
    memcpy(out->T, T, sizeof(T));
    out->a = a;
    out->b = b;
}
