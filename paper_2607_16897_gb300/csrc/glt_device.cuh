// Device-side building blocks of the tracker: per-stream descriptors, the
// per-point linearisation (projection, bilinear gather of I and grad I,
// residual, Huber weight, forward Jacobian, 44-term normal-equation
// accumulation), the warp reduce-scatter, and the FP64 LM solver tail
// (Cholesky 8x8, SE(3) exponential, pose composition).
//
// Method: GLidE-SLAM Sec. IV (Eqs. 1-5) in the forward form of Sec. IV-B
// (Jacobian from the current image's gradient at the warped location), with
// affine brightness, Huber weights and LM damping added by this library.
#pragma once

#include <cooperative_groups.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "glt.h"

namespace glt {

constexpr int kMaxLevels = GLT_MAX_LEVELS;
constexpr int kNumH = 36;        // upper triangle of the 8x8 H
constexpr int kIdxG = 36;        // g = J^T W r, 8 entries
constexpr int kIdxE = 44;        // Huber energy
constexpr int kIdxN = 45;        // valid sample count
constexpr int kNumAcc = 46;
constexpr int kAccPad = 48;      // padded for the 5-stage reduce-scatter
// cached-Hessian form: g0 = sum w r J_ic (6), Huber energy, sample count
constexpr int kHcAcc = 8;
constexpr int kHcE = 6;
constexpr int kHcN = 7;

// 8-pixel sparse pattern (offsets du_k of Eq. 2), level pixels.
__host__ __device__ constexpr int pat_dx(int k) { return k == 1 ? -2 : k == 2 ? 2 : k == 5 ? -1 : k == 6 ? 1 : k == 7 ? -1 : 0; }
__host__ __device__ constexpr int pat_dy(int k) { return k == 3 ? -2 : k == 4 ? 2 : (k == 5 || k == 6) ? -1 : k == 7 ? 1 : 0; }

// Programmatic dependent launch (sm_90 and later): a kernel launched with
// cudaLaunchAttributeProgrammaticStreamSerialization may begin while the
// previous kernel of its stream still runs.  griddep_wait() returns once that
// kernel has completed and its writes are visible; griddep_launch_dependents()
// lets the next such kernel begin.  Both are no-ops for an ordinary launch.
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void griddep_launch_dependents()
{
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// The uint8 CUR levels may be written by a pyramid kernel that was still
// running when the track kernel started (a programmatic dependent launch), so
// the gathers read them with ld.global.ca (weak, L1-cached loads ordered by
// the dependency wait), never through the read-only path, which assumes data
// that is final for the whole lifetime of the kernel.
struct LevelDev {
    const uint8_t* img;   // uint8 level, `pitch` bytes per row (pitch >= W + 8, multiple of 16)
    const uint2* packed;  // GLT_MIXED: FP16 (I, gx, gy, 0) per pixel, W pixels per row
    int W, H, pitch;
};

// One tracked stream as the kernels see it (device memory).
struct StreamDesc {
    LevelDev lv[kMaxLevels];
    int L, N, Npad;
    float fx, fy;          // level-0 focal lengths
    float huber_k, zmin;
    const float4* pt;      // (u0, v0, (u0-cx)/fx, (v0-cy)/fy)
    const float2* dz;      // (depth, 1/depth)
    const float* I0;       // [L][Npad][K]; I0[l][p][0] is NaN where the point is unusable
    const float2* G0;      // GLT_IC: reference gradient (gx, gy) [L][Npad][K], else null
    int pattern, K;        // 0 and 8: the 8-pixel pattern; p and p*p: the p x p patch
    int affine;            // 0: (a, b) held at their initial values
    const double* Hc;      // GLT_HESSIAN_CACHED: per level H (36) then H^-1 (36), row-major
                           // 6x6 pose blocks of the reference rows; H^-1[0] NaN if H is not PD
    int max_iters[kMaxLevels];
    int min_valid;
    int max_trace;
    double lambda0, lambda_up, lambda_down, eps_step, eps_step_coarse, eps_cost, accept_step;
    double* trace_E;       // [max_trace] Huber energy of each pass, or null
    int* trace_n;          // [max_trace] valid samples of each pass
    int* trace_info;       // [max_trace] level * 4 + 2 * accepted + is_candidate
    int* trace_count;      // passes of the last track, or null
    int solve;             // GLT_SOLVE_FP64 or GLT_SOLVE_FP32
};

// Bounds-checked build (compiled with -DGLT_CHECKED into libglt_checked.so):
// every gather and table access of the hot path checks its element range
// [p, p + n) against its buffer [base, base + size); an access outside sets
// bit `site` of this translation unit's check flags and goes to the buffer's
// first element instead (no trap, no access outside the buffer).  In the
// normal build checked() is the pointer itself.
enum CheckSite {
    CK_IMAGE = 0,      // uint8 level window rows
    CK_PACKED = 1,     // FP16-packed level texels
    CK_TABLE = 2,      // per-point reference tables (I0, G0)
    CK_POINTS = 3,     // point arrays (pt, dz)
    CK_PYR_SRC = 4,    // pyramid source rows
    CK_PYR_DST = 5,    // pyramid destination and level-0 copy
    CK_SET_POINTS = 6  // reference-table writes of set_points
};
#ifdef GLT_CHECKED
static __device__ unsigned g_check_flags;
template <class T>
__device__ __forceinline__ T* checked(T* p, size_t n, T* base, size_t size, int site)
{
    if (p < base || p + n > base + size) {
        atomicOr(&g_check_flags, 1u << site);
        return base;
    }
    return p;
}
#else
template <class T>
__device__ __forceinline__ T* checked(T* p, size_t, T*, size_t, int)
{
    return p;
}
#endif

// The state one linearisation pass is evaluated at, in the form the FP32
// gather uses: R - I and t rounded from the FP64 pose, e^a, b.
struct PassParams {
    float Rm[9];
    float t[3];
    float ea, b;
    float scale;           // 2^-level
    int level;
    int done;
};

// ---------------------------------------------------------------------------
// Per-point linearisation
// ---------------------------------------------------------------------------
__device__ __forceinline__ float u8f(uint32_t w, int byte) { return (float)((w >> (8 * byte)) & 0xffu); }

struct PointGeom {
    float al, be;          // bilinear weights' fractions (shared by all 8 samples)
    int xb, yb;            // integer base of sample 0
    float a0[3], a1[3];    // rows of d(pi)/d(x_c) * R (level intrinsics)
    float xr[3];           // x_r
};

// Projects point p through the pass state. Returns false if the point is not
// usable (invalid reference, behind zmin, or a pattern sample outside
// 1 <= q < W-2, 1 <= q < H-2).
//
// Projection is evaluated relative to the reference pixel to keep FP32
// accurate at any image width:  with m = ((u0-cx)/fx, (v0-cy)/fy, 1) and
// D = (R - I) m + t / d,  x_c = d (m + D)  and
// u - u0 = fx (D_x - m_x D_z) / (1 + D_z)   (exactly Eq. 1's pi(R x_r + t)).
// A point's data for one level: position, depth, reference patch (I0[0..7];
// for a p x p patch only I0[0], the validity marker).  Loaded once per level
// and kept across that level's passes when a thread owns a single point.
struct PointCache {
    float4 q;
    float2 dz;
    float4 ia, ib;
    int p, level;
};

__device__ __forceinline__ void load_point(const StreamDesc& D, int level, int p, PointCache& c)
{
    c.q = *checked(D.pt + p, 1, D.pt, (size_t)D.Npad, CK_POINTS);
    c.dz = *checked(D.dz + p, 1, D.dz, (size_t)D.Npad, CK_POINTS);
    const size_t tab = (size_t)D.L * D.Npad * D.K;
    const float* I0b = checked(D.I0 + ((size_t)level * D.Npad + p) * D.K, (size_t)D.K, D.I0, tab, CK_TABLE);
    if (D.pattern) {
        c.ia = make_float4(I0b[0], 0.f, 0.f, 0.f);   // the p x p path reads its samples itself
        c.ib = make_float4(0.f, 0.f, 0.f, 0.f);
    } else {
        const float4* I0p = reinterpret_cast<const float4*>(I0b);   // K = 8: 32-byte rows
        c.ia = I0p[0];
        c.ib = I0p[1];
    }
    c.p = p;
    c.level = level;
}

template <bool SQUARE = false>
__device__ __forceinline__ bool project_point(const StreamDesc& D, const PassParams& P,
                                              const LevelDev& lv, const PointCache& c, PointGeom& G)
{
    const float4 q = c.q;
    const float2 dz = c.dz;
    const float ub = q.z, vb = q.w, d = dz.x, rho = dz.y;
    const float Dx = fmaf(P.Rm[0], ub, fmaf(P.Rm[1], vb, fmaf(P.t[0], rho, P.Rm[2])));
    const float Dy = fmaf(P.Rm[3], ub, fmaf(P.Rm[4], vb, fmaf(P.t[1], rho, P.Rm[5])));
    const float Dz = fmaf(P.Rm[6], ub, fmaf(P.Rm[7], vb, fmaf(P.t[2], rho, P.Rm[8])));
    const float onez = 1.0f + Dz;
    if (!(d * onez > D.zmin)) return false;
    const float iz = 1.0f / onez;
    const float du = D.fx * fmaf(-ub, Dz, Dx) * iz;
    const float dv = D.fy * fmaf(-vb, Dz, Dy) * iz;
    if (!(fabsf(du) < 1e6f && fabsf(dv) < 1e6f)) return false;
    const float s = P.scale;
    const float U = q.x * s, V = q.y * s;
    const float Ui = floorf(U), Vi = floorf(V);
    const float su = (U - Ui) + du * s;
    const float sv = (V - Vi) + dv * s;
    const float fu = floorf(su), fv = floorf(sv);
    G.al = su - fu;
    G.be = sv - fv;
    G.xb = (int)Ui + (int)fu;
    G.yb = (int)Vi + (int)fv;
    const int h = (SQUARE && D.pattern) ? (D.pattern - 1) / 2 : 2;   // half extent of the pattern
    if (G.xb < 1 + h || G.xb > lv.W - 3 - h || G.yb < 1 + h || G.yb > lv.H - 3 - h) return false;
    // d(pi)/d(x_c) R, with x_c / z_c = (m + D) / (1 + D_z) and 1/z_c = rho / (1 + D_z)
    const float xn = (ub + Dx) * iz, yn = (vb + Dy) * iz;
    const float fxl = D.fx * s * rho * iz, fyl = D.fy * s * rho * iz;
    const float R0[3] = {1.0f + P.Rm[0], P.Rm[1], P.Rm[2]};
    const float R1[3] = {P.Rm[3], 1.0f + P.Rm[4], P.Rm[5]};
    const float R2[3] = {P.Rm[6], P.Rm[7], 1.0f + P.Rm[8]};
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        G.a0[c] = fxl * fmaf(-xn, R2[c], R0[c]);
        G.a1[c] = fyl * fmaf(-yn, R2[c], R1[c]);
    }
    G.xr[0] = d * ub;
    G.xr[1] = d * vb;
    G.xr[2] = d;
    return true;
}

// Accumulates one residual sample into acc (upper triangle of w J J^T, w J r,
// Huber energy, count).
__device__ __forceinline__ void accumulate_sample(const PointGeom& G, float I, float gx, float gy,
                                                  float i0, float ea, float b, float k,
                                                  float* acc, float* res_out)
{
    float J[8];
    const float Jt0 = fmaf(gx, G.a0[0], gy * G.a1[0]);
    const float Jt1 = fmaf(gx, G.a0[1], gy * G.a1[1]);
    const float Jt2 = fmaf(gx, G.a0[2], gy * G.a1[2]);
    J[0] = Jt0;
    J[1] = Jt1;
    J[2] = Jt2;
    // rotational columns: row vector (Jt) * (-[x_r]x) = x_r x Jt
    J[3] = fmaf(G.xr[1], Jt2, -G.xr[2] * Jt1);
    J[4] = fmaf(G.xr[2], Jt0, -G.xr[0] * Jt2);
    J[5] = fmaf(G.xr[0], Jt1, -G.xr[1] * Jt0);
    J[6] = -ea * i0;
    J[7] = -1.0f;
    const float r = fmaf(-ea, i0, I) - b;
    const float ar = fabsf(r);
    const float w = ar <= k ? 1.0f : k / ar;
    const float rho = ar <= k ? 0.5f * r * r : k * (ar - 0.5f * k);
    if (res_out) *res_out = r;
    float wJ[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) wJ[i] = w * J[i];
    int idx = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
#pragma unroll
        for (int j = i; j < 8; ++j) {
            acc[idx] = fmaf(wJ[i], J[j], acc[idx]);
            ++idx;
        }
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) acc[kIdxG + i] = fmaf(wJ[i], r, acc[kIdxG + i]);
    acc[kIdxE] += rho;
    acc[kIdxN] += 1.0f;
}

// Cached-Hessian form (Sec. IV-B: with the rows on the reference side H is
// fixed per reference and level; Sec. IV-C "Track": each point contributes
// only its right-hand side b_i = -sum_k J_ik^T r_ik).  A sample adds its
// Huber-weighted residual times the cached reference gradient to the point's
// (sx, sy); the point then folds them into g0 = sum w r J_ic:
// J_k = [Jt_k, x_r x Jt_k] with Jt_k = gx_k a0 + gy_k a1, so
// sum_k w_k r_k J_k = [v, x_r x v] with v = sx a0 + sy a1.
__device__ __forceinline__ void hc_sample(float I, float i0, float2 g0, float ea, float b, float k,
                                          float& sx, float& sy, float* acc, float* res_out)
{
    const float r = fmaf(-ea, i0, I) - b;
    const float ar = fabsf(r);
    const float w = ar <= k ? 1.0f : k / ar;
    const float rho = ar <= k ? 0.5f * r * r : k * (ar - 0.5f * k);
    if (res_out) *res_out = r;
    const float wr = w * r;
    sx = fmaf(wr, g0.x, sx);
    sy = fmaf(wr, g0.y, sy);
    acc[kHcE] += rho;
    acc[kHcN] += 1.0f;
}

__device__ __forceinline__ void hc_fold(const PointGeom& G, float sx, float sy, float* acc)
{
    const float v0 = fmaf(sx, G.a0[0], sy * G.a1[0]);
    const float v1 = fmaf(sx, G.a0[1], sy * G.a1[1]);
    const float v2 = fmaf(sx, G.a0[2], sy * G.a1[2]);
    acc[0] += v0;
    acc[1] += v1;
    acc[2] += v2;
    acc[3] += fmaf(G.xr[1], v2, -G.xr[2] * v1);
    acc[4] += fmaf(G.xr[2], v0, -G.xr[0] * v2);
    acc[5] += fmaf(G.xr[0], v1, -G.xr[1] * v0);
}

// Geometric rows at the reference point (identity pose), for the
// inverse-compositional form.
__device__ __forceinline__ void ic_geometry(const StreamDesc& D, const PassParams& P, int p, PointGeom& G)
{
    const float4 q = *checked(D.pt + p, 1, D.pt, (size_t)D.Npad, CK_POINTS);
    const float rho = checked(D.dz + p, 1, D.dz, (size_t)D.Npad, CK_POINTS)->y;
    const float fxl = D.fx * P.scale * rho, fyl = D.fy * P.scale * rho;
    G.a0[0] = fxl;
    G.a0[1] = 0.0f;
    G.a0[2] = -fxl * q.z;
    G.a1[0] = 0.0f;
    G.a1[1] = fyl;
    G.a1[2] = -fyl * q.w;
}

// The p x p patch (the paper's Sec. IV-A patch) for p = 7 and 11: the point's
// window of (p + 1) x (p + 1) bytes (inverse compositional) or (p + 3) x (p + 3)
// (forward: the gradient taps) is loaded once with three aligned 8-byte loads
// per row and funnel shifts, and all p*p samples are interpolated from
// registers.  FP32 levels only.
template <int PS, bool ICF, bool HC = false>
__device__ __forceinline__ void linearize_square_t(const StreamDesc& D, const PassParams& P, int p,
                                                   PointGeom& G, float* acc, float* res)
{
    static_assert(!HC || ICF, "the cached Hessian needs the inverse-compositional rows");
    float sx = 0.0f, sy = 0.0f;
    constexpr int h = (PS - 1) / 2, B = ICF ? 0 : 1, R = PS + 1 + 2 * B, NWD = (R + 3) / 4;
    const LevelDev& lv = D.lv[P.level];
    if (ICF) ic_geometry(D, P, p, G);
    const int xs = G.xb - h - B, ys = G.yb - h - B;
    const int a8 = xs & ~7, sh = xs - a8;
    const int wb = sh >> 2, s8 = (sh & 3) * 8;
    const uint8_t* base = lv.img + (size_t)ys * lv.pitch + a8;
    uint32_t win[R][NWD];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const uint2* rp = checked(reinterpret_cast<const uint2*>(base + (size_t)r * lv.pitch), 3,
                                  reinterpret_cast<const uint2*>(lv.img), (size_t)lv.pitch * lv.H / 8, CK_IMAGE);
        const uint2 u0 = __ldca(rp), u1 = __ldca(rp + 1), u2 = __ldca(rp + 2);
        const uint32_t v[6] = {u0.x, u0.y, u1.x, u1.y, u2.x, u2.y};
#pragma unroll
        for (int i = 0; i < NWD; ++i) {
            const uint32_t lo = wb ? v[i + 1] : v[i];
            const uint32_t hi = wb ? v[i + 2] : v[i + 1];
            win[r][i] = __funnelshift_r(lo, hi, s8);
        }
    }
#define GLT_WX(r, c) ((float)((win[(r)][(c) >> 2] >> (8 * ((c) & 3))) & 0xffu))
    const float w00 = (1.0f - G.al) * (1.0f - G.be), w10 = G.al * (1.0f - G.be);
    const float w01 = (1.0f - G.al) * G.be, w11 = G.al * G.be;
    const size_t tab = (size_t)D.L * D.Npad * (PS * PS);
    const float* I0p = checked(D.I0 + ((size_t)P.level * D.Npad + p) * (PS * PS), (size_t)(PS * PS), D.I0,
                               tab, CK_TABLE);
    const float2* G0p = ICF ? checked(D.G0 + ((size_t)P.level * D.Npad + p) * (PS * PS), (size_t)(PS * PS),
                                      D.G0, tab, CK_TABLE)
                            : nullptr;
#pragma unroll
    for (int j = 0; j < PS; ++j) {
#pragma unroll
        for (int i = 0; i < PS; ++i) {
            const int r0 = j + B, c0 = i + B, k = j * PS + i;
            const float I00 = GLT_WX(r0, c0), I10 = GLT_WX(r0, c0 + 1);
            const float I01 = GLT_WX(r0 + 1, c0), I11 = GLT_WX(r0 + 1, c0 + 1);
            const float I = fmaf(w00, I00, fmaf(w10, I10, fmaf(w01, I01, w11 * I11)));
            if (HC) {
                hc_sample(I, I0p[k], G0p[k], P.ea, P.b, D.huber_k, sx, sy, acc,
                          res ? res + (size_t)(PS * PS) * p + k : nullptr);
                continue;
            }
            float gx, gy;
            if (ICF) {
                const float2 g0 = G0p[k];
                gx = P.ea * g0.x;
                gy = P.ea * g0.y;
            } else {
                gx = 0.5f * fmaf(w00, I10 - GLT_WX(r0, c0 - 1),
                            fmaf(w10, GLT_WX(r0, c0 + 2) - I00,
                            fmaf(w01, I11 - GLT_WX(r0 + 1, c0 - 1),
                                 w11 * (GLT_WX(r0 + 1, c0 + 2) - I01))));
                gy = 0.5f * fmaf(w00, I01 - GLT_WX(r0 - 1, c0),
                            fmaf(w10, I11 - GLT_WX(r0 - 1, c0 + 1),
                            fmaf(w01, GLT_WX(r0 + 2, c0) - I00,
                                 w11 * (GLT_WX(r0 + 2, c0 + 1) - I10))));
            }
            accumulate_sample(G, I, gx, gy, I0p[k], P.ea, P.b, D.huber_k, acc,
                              res ? res + (size_t)(PS * PS) * p + k : nullptr);
        }
    }
#undef GLT_WX
    if (HC) hc_fold(G, sx, sy, acc);
}

// Any other odd p (3..11): samples read one by one (four taps, plus the
// gradient taps in the forward form) through the read-only cache.
template <bool HC = false>
__device__ __forceinline__ void linearize_square_any(const StreamDesc& D, const PassParams& P, int p,
                                                     PointGeom& G, float* acc, float* res)
{
    float sx = 0.0f, sy = 0.0f;
    const LevelDev& lv = D.lv[P.level];
    const int K = D.K, h = (D.pattern - 1) / 2, S = lv.pitch;
    const bool ic = D.G0 != nullptr;
    if (ic) ic_geometry(D, P, p, G);
    const float w00 = (1.0f - G.al) * (1.0f - G.be), w10 = G.al * (1.0f - G.be);
    const float w01 = (1.0f - G.al) * G.be, w11 = G.al * G.be;
    const size_t tab = (size_t)D.L * D.Npad * K;
    const float* I0p = checked(D.I0 + ((size_t)P.level * D.Npad + p) * K, (size_t)K, D.I0, tab, CK_TABLE);
    const float2* G0p = ic ? checked(D.G0 + ((size_t)P.level * D.Npad + p) * K, (size_t)K, D.G0, tab, CK_TABLE)
                           : nullptr;
    for (int k = 0; k < K; ++k) {
        const int dx = k % D.pattern - h, dy = k / D.pattern - h;
        // taps t - S - 1 .. t + 2 S + 2 (intensity and central differences)
        const uint8_t* t = checked(lv.img + (size_t)(G.yb + dy - 1) * S + (G.xb + dx - 1), (size_t)3 * S + 4,
                                   lv.img, (size_t)S * lv.H, CK_IMAGE) + S + 1;
        const float I00 = __ldca(t), I10 = __ldca(t + 1), I01 = __ldca(t + S), I11 = __ldca(t + S + 1);
        const float I = fmaf(w00, I00, fmaf(w10, I10, fmaf(w01, I01, w11 * I11)));
        if (HC) {
            hc_sample(I, I0p[k], G0p[k], P.ea, P.b, D.huber_k, sx, sy, acc,
                      res ? res + (size_t)K * p + k : nullptr);
            continue;
        }
        float gx, gy;
        if (ic) {
            const float2 g0 = G0p[k];
            gx = P.ea * g0.x;
            gy = P.ea * g0.y;
        } else {
            gx = 0.5f * fmaf(w00, I10 - (float)__ldca(t - 1),
                        fmaf(w10, (float)__ldca(t + 2) - I00,
                        fmaf(w01, I11 - (float)__ldca(t + S - 1),
                             w11 * ((float)__ldca(t + S + 2) - I01))));
            gy = 0.5f * fmaf(w00, I01 - (float)__ldca(t - S),
                        fmaf(w10, I11 - (float)__ldca(t - S + 1),
                        fmaf(w01, (float)__ldca(t + 2 * S) - I00,
                             w11 * ((float)__ldca(t + 2 * S + 1) - I10))));
        }
        accumulate_sample(G, I, gx, gy, I0p[k], P.ea, P.b, D.huber_k, acc, res ? res + (size_t)K * p + k : nullptr);
    }
    if (HC) hc_fold(G, sx, sy, acc);
}

// Inlined so the accumulators stay in registers.
template <bool HC = false>
__device__ __forceinline__ void linearize_square(const StreamDesc& D, const PassParams& P, int p,
                                                 PointGeom& G, float* acc, float* res)
{
    if (HC) {
        if (D.pattern == 7) linearize_square_t<7, true, true>(D, P, p, G, acc, res);
        else if (D.pattern == 11) linearize_square_t<11, true, true>(D, P, p, G, acc, res);
        else linearize_square_any<true>(D, P, p, G, acc, res);
        return;
    }
    const bool ic = D.G0 != nullptr;
    if (D.pattern == 7) {
        if (ic) linearize_square_t<7, true>(D, P, p, G, acc, res);
        else linearize_square_t<7, false>(D, P, p, G, acc, res);
    } else if (D.pattern == 11) {
        if (ic) linearize_square_t<11, true>(D, P, p, G, acc, res);
        else linearize_square_t<11, false>(D, P, p, G, acc, res);
    } else {
        linearize_square_any(D, P, p, G, acc, res);
    }
}

// The cached-Hessian form splits a p x p patch (p = 7 or 11) into
// kHcGroups groups of consecutive rows, one thread per group: each of the
// point's threads projects the point (the same FP32 arithmetic, so the same
// validity decision), samples its rows from its own (rows + 1) x (p + 1)
// byte window and folds its rows' sums into g0; the fold is linear, so the
// threads of a point exchange nothing.
constexpr int kHcGroups = 4;

template <int PS>
__device__ __forceinline__ void linearize_rows_hc(const StreamDesc& D, const PassParams& P, int p,
                                                  int group, PointGeom& G, float* acc)
{
    constexpr int h = (PS - 1) / 2, RG = (PS + kHcGroups - 1) / kHcGroups, R = RG + 1;
    constexpr int NWD = (PS + 1 + 3) / 4;
    const LevelDev& lv = D.lv[P.level];
    ic_geometry(D, P, p, G);
    const int j0 = group * RG;
    const int xs = G.xb - h, ys = G.yb - h + j0;
    const int a8 = xs & ~7, sh = xs - a8;
    const int wb = sh >> 2, s8 = (sh & 3) * 8;
    const uint8_t* base = lv.img + (size_t)ys * lv.pitch + a8;
    uint32_t win[R][NWD];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        // rows of the patch (and the lower bilinear tap of its last row) only
        if (j0 + r <= PS) {
            const uint2* rp = checked(reinterpret_cast<const uint2*>(base + (size_t)r * lv.pitch), 3,
                                      reinterpret_cast<const uint2*>(lv.img), (size_t)lv.pitch * lv.H / 8,
                                      CK_IMAGE);
            const uint2 u0 = __ldca(rp), u1 = __ldca(rp + 1), u2 = __ldca(rp + 2);
            const uint32_t v[6] = {u0.x, u0.y, u1.x, u1.y, u2.x, u2.y};
#pragma unroll
            for (int i = 0; i < NWD; ++i) {
                const uint32_t lo = wb ? v[i + 1] : v[i];
                const uint32_t hi = wb ? v[i + 2] : v[i + 1];
                win[r][i] = __funnelshift_r(lo, hi, s8);
            }
        } else {
#pragma unroll
            for (int i = 0; i < NWD; ++i) win[r][i] = 0u;
        }
    }
#define GLT_WR(r, c) ((float)((win[(r)][(c) >> 2] >> (8 * ((c) & 3))) & 0xffu))
    const float w00 = (1.0f - G.al) * (1.0f - G.be), w10 = G.al * (1.0f - G.be);
    const float w01 = (1.0f - G.al) * G.be, w11 = G.al * G.be;
    const size_t tab = (size_t)D.L * D.Npad * (PS * PS);
    const float* I0p = checked(D.I0 + ((size_t)P.level * D.Npad + p) * (PS * PS), (size_t)(PS * PS), D.I0,
                               tab, CK_TABLE);
    const float2* G0p = checked(D.G0 + ((size_t)P.level * D.Npad + p) * (PS * PS), (size_t)(PS * PS), D.G0,
                                tab, CK_TABLE);
    float sx = 0.0f, sy = 0.0f;
#pragma unroll
    for (int j = 0; j < RG; ++j) {
        if (j0 + j < PS) {
#pragma unroll
            for (int i = 0; i < PS; ++i) {
                const int k = (j0 + j) * PS + i;
                const float I00 = GLT_WR(j, i), I10 = GLT_WR(j, i + 1);
                const float I01 = GLT_WR(j + 1, i), I11 = GLT_WR(j + 1, i + 1);
                const float I = fmaf(w00, I00, fmaf(w10, I10, fmaf(w01, I01, w11 * I11)));
                hc_sample(I, I0p[k], G0p[k], P.ea, P.b, D.huber_k, sx, sy, acc, nullptr);
            }
        }
    }
#undef GLT_WR
    hc_fold(G, sx, sy, acc);
}

// Linearises map point p at the pass state into acc.  RES: also write the K
// residuals (NaN for an unusable point) to res[Kp..Kp+K-1].
// SQUARE: the p x p path is compiled in; IC: the inverse-compositional rows
// are compiled in (both decided per stream at run time when compiled in).
// HC: the cached-Hessian accumulation (acc holds kHcAcc values; FP32 levels
// and inverse-compositional rows only).
template <bool MIXED, bool RES, bool SQUARE = false, bool IC = true, bool HC = false>
__device__ __forceinline__ void linearize_point(const StreamDesc& D, const PassParams& P,
                                                const PointCache& c, float* acc, float* res)
{
    static_assert(!HC || (IC && !MIXED), "the cached Hessian needs FP32 levels and IC rows");
    const LevelDev& lv = D.lv[P.level];
    const int p = c.p;
    const float4 ia = c.ia, ib = c.ib;
    PointGeom G;
    bool ok = !isnan(ia.x) && project_point<SQUARE>(D, P, lv, c, G);
    if (!ok) {
        if (RES) {
            for (int k = 0; k < D.K; ++k) res[(size_t)D.K * p + k] = __int_as_float(0x7fc00000);
        }
        return;
    }
    if (SQUARE && D.pattern) {
        linearize_square<HC>(D, P, p, G, acc, RES ? res : nullptr);
        return;
    }
    const float i0[8] = {ia.x, ia.y, ia.z, ia.w, ib.x, ib.y, ib.z, ib.w};
    // inverse-compositional form: geometric rows at the reference point
    // (identity pose) and the cached reference gradients times e^a
    const bool ic = IC && D.G0 != nullptr;
    const float2* G0p = nullptr;
    if (ic) {
        ic_geometry(D, P, p, G);
        G0p = checked(D.G0 + ((size_t)P.level * D.Npad + p) * 8, (size_t)8, D.G0, (size_t)D.L * D.Npad * 8,
                      CK_TABLE);
    }
    const float w00 = (1.0f - G.al) * (1.0f - G.be), w10 = G.al * (1.0f - G.be);
    const float w01 = (1.0f - G.al) * G.be, w11 = G.al * G.be;
    if (!MIXED) {
        // 8x8 byte window, rows yb-3..yb+4, columns xb-3..xb+4: two aligned
        // 8-byte loads per row, then a funnel shift to the window start.
        float hsx = 0.0f, hsy = 0.0f;   // cached-Hessian form: the point's (sx, sy)
        const int xs = G.xb - 3;
        const int a8 = xs & ~7;
        const int sh = (xs - a8) * 8;
        const uint8_t* base = lv.img + (size_t)(G.yb - 3) * lv.pitch + a8;
        uint32_t rw[8][2];
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            const uint2* rp = checked(reinterpret_cast<const uint2*>(base + (size_t)r * lv.pitch), 2,
                                      reinterpret_cast<const uint2*>(lv.img), (size_t)lv.pitch * lv.H / 8,
                                      CK_IMAGE);
            const uint2 w0 = __ldca(rp), w1 = __ldca(rp + 1);
            if (sh < 32) {
                rw[r][0] = __funnelshift_r(w0.x, w0.y, sh);
                rw[r][1] = __funnelshift_r(w0.y, w1.x, sh);
            } else {
                rw[r][0] = __funnelshift_r(w0.y, w1.x, sh - 32);
                rw[r][1] = __funnelshift_r(w1.x, w1.y, sh - 32);
            }
        }
#define GLT_PX(r, c) u8f(rw[(r)][(c) >> 2], (c) & 3)
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int r0 = pat_dy(k) + 3, c0 = pat_dx(k) + 3;
            const float I00 = GLT_PX(r0, c0), I10 = GLT_PX(r0, c0 + 1);
            const float I01 = GLT_PX(r0 + 1, c0), I11 = GLT_PX(r0 + 1, c0 + 1);
            const float I = fmaf(w00, I00, fmaf(w10, I10, fmaf(w01, I01, w11 * I11)));
            if (HC) {
                hc_sample(I, i0[k], G0p[k], P.ea, P.b, D.huber_k, hsx, hsy, acc,
                          RES ? res + 8 * p + k : nullptr);
                continue;
            }
            float gx, gy;
            if (ic) {
                const float2 g0 = G0p[k];
                gx = P.ea * g0.x;
                gy = P.ea * g0.y;
            } else {
                // central differences at the four taps (the 1/2 is applied after interpolation)
                gx = 0.5f * fmaf(w00, I10 - GLT_PX(r0, c0 - 1),
                            fmaf(w10, GLT_PX(r0, c0 + 2) - I00,
                            fmaf(w01, I11 - GLT_PX(r0 + 1, c0 - 1),
                                 w11 * (GLT_PX(r0 + 1, c0 + 2) - I01))));
                gy = 0.5f * fmaf(w00, I01 - GLT_PX(r0 - 1, c0),
                            fmaf(w10, I11 - GLT_PX(r0 - 1, c0 + 1),
                            fmaf(w01, GLT_PX(r0 + 2, c0) - I00,
                                 w11 * (GLT_PX(r0 + 2, c0 + 1) - I10))));
            }
            accumulate_sample(G, I, gx, gy, i0[k], P.ea, P.b, D.huber_k, acc,
                              RES ? res + 8 * p + k : nullptr);
        }
#undef GLT_PX
        if (HC) hc_fold(G, hsx, hsy, acc);
    } else {
        const uint2* pk = lv.packed;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int x0 = G.xb + pat_dx(k), y0 = G.yb + pat_dy(k);
            const uint2* t0 = checked(pk + (size_t)y0 * lv.W + x0, (size_t)lv.W + 2, pk, (size_t)lv.W * lv.H,
                                      CK_PACKED);
            const uint2* t1 = t0 + lv.W;
            const uint2 p00 = __ldca(t0), p10 = __ldca(t0 + 1), p01 = __ldca(t1), p11 = __ldca(t1 + 1);
            const float2 a00 = __half22float2(*reinterpret_cast<const __half2*>(&p00.x));
            const float2 a10 = __half22float2(*reinterpret_cast<const __half2*>(&p10.x));
            const float2 a01 = __half22float2(*reinterpret_cast<const __half2*>(&p01.x));
            const float2 a11 = __half22float2(*reinterpret_cast<const __half2*>(&p11.x));
            const float y00 = __low2float(*reinterpret_cast<const __half2*>(&p00.y));
            const float y10 = __low2float(*reinterpret_cast<const __half2*>(&p10.y));
            const float y01 = __low2float(*reinterpret_cast<const __half2*>(&p01.y));
            const float y11 = __low2float(*reinterpret_cast<const __half2*>(&p11.y));
            const float I = fmaf(w00, a00.x, fmaf(w10, a10.x, fmaf(w01, a01.x, w11 * a11.x)));
            const float2 g0 = ic ? G0p[k] : make_float2(0.0f, 0.0f);
            const float gx = ic ? P.ea * g0.x : fmaf(w00, a00.y, fmaf(w10, a10.y, fmaf(w01, a01.y, w11 * a11.y)));
            const float gy = ic ? P.ea * g0.y : fmaf(w00, y00, fmaf(w10, y10, fmaf(w01, y01, w11 * y11)));
            accumulate_sample(G, I, gx, gy, i0[k], P.ea, P.b, D.huber_k, acc,
                              RES ? res + 8 * p + k : nullptr);
        }
    }
}

// One task of a cached-Hessian pass: row group `group` of point c.p for the
// 7 x 7 and 11 x 11 patches (groups = kHcGroups), the whole point otherwise
// (groups = 1).
__device__ __forceinline__ void linearize_task_hc(const StreamDesc& D, const PassParams& P,
                                                  const PointCache& c, int group, int groups,
                                                  float* acc)
{
    if (groups == 1) {
        linearize_point<false, false, true, true, true>(D, P, c, acc, nullptr);
        return;
    }
    const LevelDev& lv = D.lv[P.level];
    PointGeom G;
    if (isnan(c.ia.x) || !project_point<true>(D, P, lv, c, G)) return;
    if (D.pattern == 7)
        linearize_rows_hc<7>(D, P, c.p, group, G, acc);
    else
        linearize_rows_hc<11>(D, P, c.p, group, G, acc);
}

__host__ __device__ inline int hc_groups(int pattern)
{
    return (pattern == 7 || pattern == 11) ? kHcGroups : 1;
}

// ---------------------------------------------------------------------------
// Reductions
// ---------------------------------------------------------------------------
// Butterfly reduce-scatter of 48 values over a warp: 48 shuffles instead of
// 5 x 48.  Afterwards lane L holds the warp sums of indices
// base(L) + {0,1,2}, base = 24*b4 + 12*b3 + 6*b2 + 3*b1 (b_i = bit i of L).
__device__ __forceinline__ int rs_base(int lane)
{
    return ((lane >> 4) & 1) * 24 + ((lane >> 3) & 1) * 12 + ((lane >> 2) & 1) * 6 + ((lane >> 1) & 1) * 3;
}

__device__ __forceinline__ void warp_reduce_scatter48(float (&v)[kAccPad], int lane)
{
    const unsigned full = 0xffffffffu;
#define GLT_RS_STAGE(HALF, OFF)                                            \
    {                                                                      \
        const bool hi = (lane & (OFF)) != 0;                               \
        _Pragma("unroll") for (int i = 0; i < (HALF); ++i) {               \
            const float send = hi ? v[i] : v[i + (HALF)];                  \
            const float keep = hi ? v[i + (HALF)] : v[i];                  \
            v[i] = keep + __shfl_xor_sync(full, send, (OFF));              \
        }                                                                  \
    }
    GLT_RS_STAGE(24, 16)
    GLT_RS_STAGE(12, 8)
    GLT_RS_STAGE(6, 4)
    GLT_RS_STAGE(3, 2)
#undef GLT_RS_STAGE
#pragma unroll
    for (int i = 0; i < 3; ++i) v[i] += __shfl_xor_sync(full, v[i], 1);
}

// Butterfly reduce-scatter of the 8 cached-Hessian accumulators (7 shuffles),
// then two pair stages: afterwards lanes with (lane & 3) == 0 hold the warp
// sum of value ((lane >> 4) & 1) * 4 + ((lane >> 3) & 1) * 2 + ((lane >> 2) & 1).
__device__ __forceinline__ int rs8_index(int lane)
{
    return ((lane >> 4) & 1) * 4 + ((lane >> 3) & 1) * 2 + ((lane >> 2) & 1);
}

__device__ __forceinline__ void warp_reduce_scatter8(float (&v)[kHcAcc], int lane)
{
    const unsigned full = 0xffffffffu;
#pragma unroll
    for (int half = 4, off = 16; half >= 1; half >>= 1, off >>= 1) {
        const bool hi = (lane & off) != 0;
#pragma unroll
        for (int i = 0; i < half; ++i) {
            const float send = hi ? v[i] : v[i + half];
            const float keep = hi ? v[i + half] : v[i];
            v[i] = keep + __shfl_xor_sync(full, send, off);
        }
    }
    v[0] += __shfl_xor_sync(full, v[0], 2);
    v[0] += __shfl_xor_sync(full, v[0], 1);
}

// Block reduction of the 8 cached-Hessian accumulators into out[0..8).
// Ends with __syncthreads().
template <int THREADS>
__device__ __forceinline__ void block_reduce8(float (&acc)[kHcAcc], float (*red)[kAccPad], float* out)
{
    constexpr int NW = THREADS / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    warp_reduce_scatter8(acc, lane);
    if ((lane & 3) == 0) red[warp][rs8_index(lane)] = acc[0];
    __syncthreads();
    if (threadIdx.x < kHcAcc) {
        float s = 0.0f;
#pragma unroll
        for (int w = 0; w < NW; ++w) s += red[w][threadIdx.x];
        out[threadIdx.x] = s;
    }
    __syncthreads();
}

// Block reduction of the per-thread accumulators into out[0..kNumAcc).
// KAHAN: compensated FP32 sum across warps, compensation in out_c.
// Ends with __syncthreads().
template <int THREADS, bool KAHAN>
__device__ __forceinline__ void block_reduce(float (&acc)[kAccPad], float (*red)[kAccPad], float* out,
                                             float* out_c)
{
    constexpr int NW = THREADS / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    warp_reduce_scatter48(acc, lane);
    if ((lane & 1) == 0) {
        const int b = rs_base(lane);
        red[warp][b + 0] = acc[0];
        red[warp][b + 1] = acc[1];
        red[warp][b + 2] = acc[2];
    }
    __syncthreads();
    if (threadIdx.x < kNumAcc) {
        const int j = threadIdx.x;
        float s = 0.0f, c = 0.0f;
#pragma unroll
        for (int w = 0; w < NW; ++w) {
            if (KAHAN) {
                const float y = red[w][j] - c;
                const float t = s + y;
                c = (t - s) - y;
                s = t;
            } else {
                s += red[w][j];
            }
        }
        out[j] = s;
        if (KAHAN) out_c[j] = -c;
    }
    __syncthreads();
}

// ---------------------------------------------------------------------------
// Solver tail, run by one warp of every CTA
//
// GB300 runs FP64 at a small fraction of its FP32 rate with long dependent
// latencies (measured on the part: ~64 cycles per DFMA, ~420 per divide or
// reciprocal, ~670 per square root, ~1700 per sincos), and this tail sits on
// the critical path of every pass.  The state, the normal equations, the
// accept/reject decision and the composition are FP64 in both solve modes;
// GLT_SOLVE_FP64 (the default) also factorises and exponentiates in FP64,
// GLT_SOLVE_FP32 does those two in FP32 (their inputs carry FP32 rounding
// anyway, or their result is a small increment):
//  * the damped normal matrix is factored as L D L^T (no square roots), one
//    row per lane, columns eliminated right-looking with warp shuffles; in
//    GLT_SOLVE_FP32 first in FP32, and a pivot below 1e-4 of its damped
//    diagonal sends the system to the FP64 elimination, which alone decides
//    "not positive definite";
//  * FP64 pivot reciprocals are an FP32 seed refined by one Newton step
//    (relative error ~4e-15);
//  * the SE(3) exponential uses the power series of its coefficients in
//    theta^2 below theta = 0.1 (sincos only beyond), each lane one element
//    of exp(delta) (GLT_SOLVE_FP32: of exp(delta) - I in FP32, composed with
//    the FP64 pose as T + T (exp(delta) - I), and the frame's final pose
//    orthonormalised once in FP64);
//  * FP64 <-> FP32 conversions go through the bit pattern (integer
//    instructions), and accept/reject compares E' n <= E n' instead of
//    dividing.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double rcp_d(double d)
{
    // Reciprocal by one Newton-Raphson iteration for f(r) = 1/r - d,
    // r' = r + r (1 - d r), from an FP32 seed: the seed is rcp.approx.ftz.f32
    // of d rounded to FP32 through its bit pattern (no F2F conversions on the
    // FP64 pipe), relative error e0 <= 2^-22, and the iteration squares it
    // (e1 = e0^2 plus FP64 rounding): relative error < 1e-13.  Only for
    // 2^-100 <= |d| < 2^100 (exponent tested as an integer), where the
    // exponent fits FP32; zero, infinities, NaN and the rest divide.
    const int hi = __double2hiint(d);
    const unsigned lo = (unsigned)__double2loint(d);
    const int ebits = (hi >> 20) & 0x7ff;
    if (ebits < 1023 - 100 || ebits >= 1023 + 100) return 1.0 / d;
    const int e32 = ebits - 896;
    const unsigned fb = ((unsigned)hi & 0x80000000u) | ((unsigned)e32 << 23) |
                        (((unsigned)hi & 0xfffffu) << 3) | (lo >> 29);
    float rf;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rf) : "f"(__uint_as_float(fb)));
    const unsigned rb = __float_as_uint(rf);
    const int rhi = (int)((rb & 0x80000000u) | ((((rb >> 23) & 0xffu) + 896u) << 20) | ((rb >> 3) & 0xfffffu));
    double r = __hiloint2double(rhi, (int)(rb << 29));
    const double e = fma(-d, r, 1.0);
    return fma(r, e, r);
}

// FP64 -> FP32 through the bit pattern (integer instructions only, nothing on
// the FP64 pipe): the significand truncated to 23 bits (relative error
// < 2^-23); magnitudes below 2^-126 give a signed zero and above FP32's range
// infinity; infinities and NaN are kept.
__device__ __forceinline__ float f32_of(double x)
{
    const int hi = __double2hiint(x);
    const unsigned lo = (unsigned)__double2loint(x);
    const int eb = (hi >> 20) & 0x7ff;
    const unsigned sign = (unsigned)hi & 0x80000000u;
    const unsigned man = (((unsigned)hi & 0xfffffu) << 3) | (lo >> 29);
    unsigned b;
    if (eb == 0x7ff)
        b = sign | 0x7f800000u | ((((unsigned)hi & 0xfffffu) | lo) ? 0x400000u : 0u);
    else if (eb > 1023 + 127)
        b = sign | 0x7f800000u;
    else if (eb < 1023 - 126)
        b = sign;
    else
        b = sign | ((unsigned)(eb - 896) << 23) | man;
    return __uint_as_float(b);
}

// FP32 -> FP64 through the bit pattern: exact for zero and normal numbers
// (subnormals give a signed zero); infinities and NaN are kept.
__device__ __forceinline__ double f64_of(float f)
{
    const unsigned b = __float_as_uint(f);
    const unsigned e = (b >> 23) & 0xffu;
    const unsigned sign = b & 0x80000000u;
    unsigned hi = sign, lo = 0u;
    if (e != 0u) {
        hi = sign | ((e == 0xffu ? 0x7ffu : e + 896u) << 20) | ((b & 0x7fffffu) >> 3);
        if (e == 0xffu && (b & 0x7fffffu)) hi |= 0x80000u;
        lo = b << 29;
    }
    return __hiloint2double((int)hi, (int)lo);
}

// |x| compared through the bit pattern: for non-negative doubles the IEEE
// ordering is the integer ordering of the bits (no FP64 instructions).
__device__ __forceinline__ long long abs_bits(double x)
{
    return __double_as_longlong(x) & 0x7fffffffffffffffll;
}

// Bits of +infinity: x is finite iff abs_bits(x) < kInfBits.
constexpr long long kInfBits = 0x7ff0000000000000ll;

// Pass parameters for state (T, a, b) on `level` (single thread).
__device__ __host__ inline void make_pass_params(const double* T, double a, double b, int level,
                                                 PassParams& P)
{
    P.Rm[0] = (float)(T[0] - 1.0);
    P.Rm[1] = (float)T[1];
    P.Rm[2] = (float)T[2];
    P.Rm[3] = (float)T[4];
    P.Rm[4] = (float)(T[5] - 1.0);
    P.Rm[5] = (float)T[6];
    P.Rm[6] = (float)T[8];
    P.Rm[7] = (float)T[9];
    P.Rm[8] = (float)(T[10] - 1.0);
    P.t[0] = (float)T[3];
    P.t[1] = (float)T[7];
    P.t[2] = (float)T[11];
    P.ea = expf((float)a);
    P.b = (float)b;
    P.level = level;
    P.scale = ldexpf(1.0f, -level);
    P.done = 0;
}

// Same, one element per lane (lanes 0-13), for the pose in T (12 doubles).
__device__ __forceinline__ void make_pass_params_warp(const double* T, double a, double b,
                                                      int level, PassParams& P, int lane)
{
    if (lane < 12) {
        const int r = lane >> 2, c = lane & 3;
        const double v = T[lane] - ((c == r) ? 1.0 : 0.0);
        if (c < 3)
            P.Rm[3 * r + c] = (float)v;
        else
            P.t[r] = (float)v;
    } else if (lane == 12) {
        P.ea = expf((float)a);
    } else if (lane == 13) {
        P.b = (float)b;
        P.level = level;
        P.scale = ldexpf(1.0f, -level);
        P.done = 0;
    }
}

// Same, with lane l < 12 holding pose entry l in `v` (no shared-memory read).
__device__ __forceinline__ void make_pass_params_lane(double v, double a, double b, int level,
                                                      PassParams& P, int lane)
{
    if (lane < 12) {
        const int r = lane >> 2, c = lane & 3;
        const double m = v - ((c == r) ? 1.0 : 0.0);
        if (c < 3)
            P.Rm[3 * r + c] = (float)m;
        else
            P.t[r] = (float)m;
    } else if (lane == 12) {
        P.ea = expf((float)a);
    } else if (lane == 13) {
        P.b = (float)b;
        P.level = level;
        P.scale = ldexpf(1.0f, -level);
        P.done = 0;
    }
}

// LM state machine, replicated in every CTA of a stream's cluster (each CTA
// runs it on bit-identical inputs, so all take the same decisions).
enum { PH_START = 0, PH_CAND = 1 };

struct Solver {
    double T[12], a, b;       // accepted state
    double ema;               // cached-Hessian form: e^-a (a is held fixed there)
    double Tc[12], ac, bc;    // candidate under evaluation
    double H[64], g[8];       // normal equations at the accepted state
    double E, nd, lambda, res_E;   // energy / samples (as double) at the accepted state
    long long maxstep_bits;   // max |delta_xi| of the candidate, as abs_bits
    int n, res_n, level, it, phase, status, passes, done;
    int moved;                // the pose changed since the initial state
    int iters[kMaxLevels];
};

// Upper-triangle index of (i, j), i <= j, in the accumulator layout.
__device__ __forceinline__ int upper_index(int i, int j) { return i * 8 - (i * (i - 1)) / 2 + (j - i); }

// Initial state (one thread): Gram-Schmidt the initial rotation, first level.
__device__ inline void solver_init(const StreamDesc& D, const double* init, Solver& S, PassParams& P)
{
    for (int i = 0; i < 12; ++i) S.T[i] = init[i];
    {
        double* T = S.T;
        const double n0 = sqrt(T[0] * T[0] + T[1] * T[1] + T[2] * T[2]);
        for (int c = 0; c < 3; ++c) T[c] /= n0;
        const double d = T[4] * T[0] + T[5] * T[1] + T[6] * T[2];
        for (int c = 0; c < 3; ++c) T[4 + c] -= d * T[c];
        const double n1 = sqrt(T[4] * T[4] + T[5] * T[5] + T[6] * T[6]);
        for (int c = 0; c < 3; ++c) T[4 + c] /= n1;
        T[8] = T[1] * T[6] - T[2] * T[5];
        T[9] = T[2] * T[4] - T[0] * T[6];
        T[10] = T[0] * T[5] - T[1] * T[4];
    }
    S.a = init[12];
    S.b = init[13];
    S.status = 0;
    bool finite_start = true;
    for (int i = 0; i < 12; ++i) finite_start &= abs_bits(S.T[i]) < kInfBits;
    finite_start &= abs_bits(S.a) < kInfBits && abs_bits(S.b) < kInfBits;
    S.passes = 0;
    S.it = 0;
    S.n = 0;
    S.nd = 0.0;
    S.E = 0.0;
    S.maxstep_bits = 0;
    S.res_n = 0;
    S.res_E = __longlong_as_double(0x7ff8000000000000ll);
    S.done = 0;
    S.moved = 0;
    for (int l = 0; l < kMaxLevels; ++l) S.iters[l] = 0;
    S.ema = (D.Hc && finite_start) ? exp(-S.a) : 1.0;
    int l = D.L - 1;
    while (l >= 0 && D.max_iters[l] <= 0) --l;
    if (!finite_start) {
        // a start that is not finite (or whose rotation is degenerate) is
        // not solved: the result is the start, flagged
        S.status |= GLT_TRACK_DIVERGED;
        l = -1;
    }
    S.level = l;
    S.phase = PH_START;
    if (l < 0) {
        S.done = 1;
        P.done = 1;
    } else {
        make_pass_params(S.T, S.a, S.b, l, P);
    }
}

// One LM decision after a pass whose cluster-wide sums are `tot`; executed
// by all 32 lanes of one warp with uniform control flow.  FP64 instructions
// are kept to the minimum the method needs (each costs ~64 issue cycles).
// HC: the cached-Hessian form (tot holds g0 = sum w r J_ic, E and n; the
// step is -e^-a H^-1 g0 with the level's per-reference H^-1, since the rows
// are e^a J_ic and the normal matrix e^2a H).
template <bool HC = false>
__device__ inline void solver_step_warp(const StreamDesc& D, const double* tot, Solver& S,
                                        PassParams& P, int lane, bool write_trace)
{
    const unsigned full = 0xffffffffu;
    const int row = lane & 7;
    const double E = tot[HC ? kHcE : kIdxE];
    const double nd = tot[HC ? kHcN : kIdxN];   // exact integer count
    const int n = (int)nd;
    // sums that are not finite (an FP32 overflow) make the pass unusable
    bool fin = true;
#pragma unroll
    for (int i = lane; i < (HC ? kHcE : kIdxE); i += 32) fin &= abs_bits(tot[i]) < kInfBits;
    const bool sums_finite = __all_sync(full, fin) && abs_bits(E) < kInfBits;
    const bool enough = n >= D.min_valid && n > 0 && sums_finite;
    int status = S.status;
    if (!sums_finite) status |= GLT_TRACK_DIVERGED;
    const int level = S.level;
    const int phase = S.phase;
    int it = S.it;
    double lambda = S.lambda;
    const long long step_bits = S.maxstep_bits;
    bool load_normal = false, accept = false, finish = false, candidate = false;
    if (phase == PH_START) {
        if (!enough) {
            if (sums_finite) status |= GLT_TRACK_TOO_FEW_POINTS;
        } else {
            load_normal = true;
            lambda = D.lambda0;
            it = 0;
            candidate = true;
        }
    } else {
        ++it;
        // c' < c  <=>  E' n < E n'  (both counts positive); flat: c' - c <= eps c
        const double En = E * S.nd;
        const double Ecn = S.E * nd;
        const bool small = step_bits < abs_bits(D.accept_step);
        accept = enough && (En < Ecn || small);
        const bool flat = !accept && enough && __double_as_longlong(D.eps_cost) != 0 &&
                          (En - Ecn <= D.eps_cost * Ecn);   // off (no FP64 work) when eps_cost = 0
        lambda *= accept ? D.lambda_down : D.lambda_up;
        load_normal = accept;
        if (it >= D.max_iters[level] ||
            step_bits < abs_bits(level > 0 ? D.eps_step_coarse : D.eps_step) || flat)
            finish = true;
        else
            candidate = true;
    }
    if (write_trace && lane == 0 && D.trace_E && S.passes < D.max_trace) {
        D.trace_E[S.passes] = E;
        D.trace_n[S.passes] = n;
        D.trace_info[S.passes] = level * 4 + (phase == PH_CAND ? 1 + (accept ? 2 : 0) : 0);
    }
    __syncwarp();
    // commit the pass outcome to the shared state
    if (accept && lane < 12) S.T[lane] = S.Tc[lane];
    if (HC) {
        if (load_normal) {
            // g0 of the accepted state, and the level's H^-1 (read again at every
            // acceptance: two loads per lane)
            if (lane < 6) S.g[lane] = tot[lane];
            const double* Hi = D.Hc + 72 * level + 36;
            S.H[lane] = Hi[lane];
            if (lane < 4) S.H[32 + lane] = Hi[32 + lane];
        }
    } else if (load_normal && lane < 8) {
        // with (a, b) held fixed their rows and columns become the identity and
        // their right-hand side zero, so the solve gives da = db = 0
        const bool fixed_ab = !D.affine;
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            double v = tot[c >= lane ? upper_index(lane, c) : upper_index(c, lane)];
            if (fixed_ab && (lane >= 6 || c >= 6)) v = lane == c ? 1.0 : 0.0;
            S.H[8 * lane + c] = v;
        }
        S.g[lane] = (fixed_ab && lane >= 6) ? 0.0 : tot[kIdxG + lane];
    }
    if (lane == 0) {
        S.passes += 1;
        S.it = it;
        S.lambda = lambda;
        S.status = status;
        if (accept) {
            S.a = S.ac;
            S.b = S.bc;
            S.moved = 1;
        }
        if (load_normal) {
            S.E = E;
            S.nd = nd;
            S.n = n;
        }
    }
    __syncwarp();

    bool next_level = (phase == PH_START && !enough) || finish;
    bool solved = false;
    double dl[8];
    if (candidate && HC) {
        // ---- delta = -e^-a H^-1 g0, one row per lane (lanes 0-5); the affine
        // pair is held fixed in this form
        if (!(abs_bits(S.H[0]) < kInfBits)) {
            if (lane == 0) S.status |= GLT_TRACK_NOT_PD;
            finish = true;
            next_level = true;
        } else {
            const int r6 = lane < 6 ? lane : 0;
            double x = 0.0;
#pragma unroll
            for (int j = 0; j < 6; ++j) x = fma(S.H[6 * r6 + j], S.g[j], x);
            x *= -S.ema;
#pragma unroll
            for (int c = 0; c < 6; ++c) dl[c] = __shfl_sync(full, x, c);
            dl[6] = 0.0;
            dl[7] = 0.0;
            solved = true;
        }
    } else if (candidate) {
        // ---- (H + lambda diag H) delta = -g by L D L^T, right-looking, one
        // matrix entry per lane: lanes 0-27 hold the strictly lower entries
        // (i, k), i > k, column by column; lanes 0-7 also hold the diagonal
        // entry of row `lane`.  Each column costs one reciprocal, one scale
        // and two FMAs per warp (trailing entries and diagonal) instead of
        // one FMA per trailing column.
        const int ek = lane < 7 ? 0 : lane < 13 ? 1 : lane < 18 ? 2 : lane < 22 ? 3 : lane < 25 ? 4
                     : lane < 27 ? 5 : lane < 28 ? 6 : 7;
        const int ei = lane < 28 ? lane - (ek * 7 - (ek * (ek - 1)) / 2) + ek + 1 : 8;
        // GLT_SOLVE_FP32 first factorises in FP32 (H and g are FP32 sums,
        // relative error ~1e-7, so the step they define is known to ~cond x
        // 1e-7 however it is solved; the FP32 elimination adds an error of the
        // same order, ~cond x 2^-23).  Used when every FP32 pivot is above 1e-4
        // of its damped diagonal, where its rounding (~1e-6 of the diagonal)
        // cannot change its sign; otherwise, and always for GLT_SOLVE_FP64
        // (the default), the FP64 elimination below decides, as for every
        // system it accepts or rejects as not positive definite.
        bool ok32 = false;
        if (D.solve != GLT_SOLVE_FP64) {
            float e = lane < 28 ? f32_of(S.H[8 * ei + ek]) : 0.0f;
            const double diag = S.H[8 * row + row];
            const double a0 = fma(lambda, diag, diag);
            const float a0f = f32_of(a0);
            float dg = a0f, dinv = 0.0f;
            float y = -f32_of(S.g[row]);
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const float d = __shfl_sync(full, dg, j);
                const float r = __frcp_rn(d);
                if (lane == j) dinv = r;
                if (j < 7) {
                    const float l = e * r;
                    const int cj = j * 7 - (j * (j - 1)) / 2 - j - 1;
                    const bool trail = lane < 28 && ek > j;
                    const bool drow = lane > j && lane < 8;
                    const float li = __shfl_sync(full, l, cj + (trail ? ei : j + 1));
                    const float ak = __shfl_sync(full, e, cj + (trail ? ek : j + 1));
                    const float ld = __shfl_sync(full, l, cj + (drow ? lane : j + 1));
                    const float ad = __shfl_sync(full, e, cj + (drow ? lane : j + 1));
                    const float yj = __shfl_sync(full, y, j);
                    if (trail) e = fmaf(-li, ak, e);
                    if (drow) {
                        dg = fmaf(-ld, ad, dg);
                        y = fmaf(-ld, yj, y);
                    }
                    if (lane < 28 && ek == j) e = l;
                }
            }
            ok32 = __all_sync(full, dg > 1e-4f * a0f || lane >= 8);
            if (ok32) {
                // column `row` of L (entries below the diagonal) gathered into the row's lane
                float Lcol[8];
#pragma unroll
                for (int i = 1; i < 8; ++i) {
                    const int cr = row * 7 - (row * (row - 1)) / 2 - row - 1;
                    const float v = __shfl_sync(full, e, row < i ? cr + i : 0);
                    Lcol[i] = row < i ? v : 0.0f;
                }
                // diagonal, backward (L^T x = D^-1 y)
                float x = y * dinv;
#pragma unroll
                for (int j = 7; j >= 1; --j) {
                    const float xj = __shfl_sync(full, x, j);
                    if (row < j) x = fmaf(-Lcol[j], xj, x);
                }
                const double x64 = f64_of(x);
#pragma unroll
                for (int c = 0; c < 8; ++c) dl[c] = __shfl_sync(full, x64, c);
                solved = true;
            }
        }
        if (!ok32) {
            // ---- the FP64 elimination (the layout above, FP64 reciprocals)
            double e = lane < 28 ? S.H[8 * ei + ek] : 0.0;
            const double diag = S.H[8 * row + row];
            const double a0 = fma(lambda, diag, diag);   // damped diagonal (lanes 0-7)
            double dg = a0;
            double dinv = 0.0;
            // the forward substitution L y = -g rides along: y_i -= l_ij y_j with the
            // l_ij the diagonal update already fetched (lanes 0-7 hold y_i)
            double y = -S.g[row];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const double d = __shfl_sync(full, dg, j);
                const double r = rcp_d(d);
                if (lane == j) dinv = r;
                if (j < 7) {
                    const double l = e * r;                         // l_ij on the lanes of column j
                    const int cj = j * 7 - (j * (j - 1)) / 2 - j - 1;   // lane of (i, j) is cj + i
                    const bool trail = lane < 28 && ek > j;        // entry (i, k), k > j: -= l_ij a_kj
                    const bool drow = lane > j && lane < 8;          // diagonal d_i, i > j: -= l_ij a_ij
                    const double li = __shfl_sync(full, l, cj + (trail ? ei : j + 1));
                    const double ak = __shfl_sync(full, e, cj + (trail ? ek : j + 1));
                    const double ld = __shfl_sync(full, l, cj + (drow ? lane : j + 1));
                    const double ad = __shfl_sync(full, e, cj + (drow ? lane : j + 1));
                    const double yj = __shfl_sync(full, y, j);
                    if (trail) e = fma(-li, ak, e);
                    if (drow) {
                        dg = fma(-ld, ad, dg);
                        y = fma(-ld, yj, y);
                    }
                    if (lane < 28 && ek == j) e = l;
                }
            }
            // pivots checked once, each lane its own: d > 0 and d > 1e-13 * damped diagonal
            const bool piv_ok = dg > 1e-13 * a0 && dg > 0.0;
            const bool ok = __all_sync(full, piv_ok || lane >= 8);
            if (!ok) {
                if (lane == 0) S.status |= GLT_TRACK_NOT_PD;
                finish = true;
                next_level = true;
            } else {
                // column `row` of L (entries below the diagonal) gathered into the row's lane
                double Lcol[8];
#pragma unroll
                for (int i = 1; i < 8; ++i) {
                    const int cr = row * 7 - (row * (row - 1)) / 2 - row - 1;
                    const double v = __shfl_sync(full, e, row < i ? cr + i : 0);
                    Lcol[i] = row < i ? v : 0.0;
                }
                // diagonal, backward (L^T x = D^-1 y)
                double x = y * dinv;
#pragma unroll
                for (int j = 7; j >= 1; --j) {
                    const double xj = __shfl_sync(full, x, j);
                    if (row < j) x = fma(-Lcol[j], xj, x);
                }
#pragma unroll
                for (int c = 0; c < 8; ++c) dl[c] = __shfl_sync(full, x, c);
                solved = true;
            }
        }
    }
    if (solved) {
        {
            long long mbits = 0;
#pragma unroll
            for (int c = 0; c < 6; ++c) mbits = max(mbits, abs_bits(dl[c]));
            double tc;
            if (D.solve == GLT_SOLVE_FP32) {
                // ---- exp(delta_xi) - I in FP32: its entries are O(|delta|), so FP32
                // rounding leaves ~1e-7 |delta| (absolute); the product with T is FP64.
                //   R_e - I = A [w]x + B [w]x^2,  t_e = v + B (w x v) + C w x (w x v),
                // A = sin th / th, B = (1 - cos th) / th^2, C = (th - sin th) / th^3
                // (power series below th^2 = 0.25, truncation < 3e-11 relative)
                const float v0 = f32_of(dl[0]), v1 = f32_of(dl[1]), v2 = f32_of(dl[2]);
                const float w0 = f32_of(dl[3]), w1 = f32_of(dl[4]), w2 = f32_of(dl[5]);
                const float th2 = fmaf(w0, w0, fmaf(w1, w1, w2 * w2));
                float A, B, Cc;
                if (th2 < 0.25f) {
                    A = fmaf(fmaf(fmaf(fmaf(th2, 1.0f / 362880.0f, -1.0f / 5040.0f), th2, 1.0f / 120.0f), th2, -1.0f / 6.0f), th2, 1.0f);
                    B = fmaf(fmaf(fmaf(fmaf(th2, 1.0f / 3628800.0f, -1.0f / 40320.0f), th2, 1.0f / 720.0f), th2, -1.0f / 24.0f), th2, 0.5f);
                    Cc = fmaf(fmaf(fmaf(fmaf(th2, 1.0f / 39916800.0f, -1.0f / 362880.0f), th2, 1.0f / 5040.0f), th2, -1.0f / 120.0f), th2, 1.0f / 6.0f);
                } else {
                    const float th = sqrtf(th2);
                    const float sn = sinf(th), sh = sinf(0.5f * th);
                    A = sn / th;
                    B = 2.0f * sh * sh / th2;
                    Cc = (th - sn) / (th2 * th);
                }
                // one element (r, c) of the 3x4 increment per lane 0-11, every lane
                // running the same instructions on its own operands:
                //   (R_e - I)(r, c) = A W_rc + B (w_r w_c - d_rc th2)        (W = [w]x)
                //   t_e(r)          = v_r + B (w x v)_r + C (w_r (w . v) - v_r th2)
                // as  base + cA (a1 b1 - a2 b2) + cB (p q - d th2).
                const float wv = fmaf(w0, v0, fmaf(w1, v1, w2 * v2));
                const int er = (lane >> 2) % 3, ec = lane & 3;
                const float wr = er == 0 ? w0 : (er == 1 ? w1 : w2);
                const float wr1 = er == 0 ? w1 : (er == 1 ? w2 : w0);   // w_{r+1}
                const float wr2 = er == 0 ? w2 : (er == 1 ? w0 : w1);   // w_{r+2}
                const float vr = er == 0 ? v0 : (er == 1 ? v1 : v2);
                const float vr1 = er == 0 ? v1 : (er == 1 ? v2 : v0);
                const float vr2 = er == 0 ? v2 : (er == 1 ? v0 : v1);
                const float wc = ec == 0 ? w0 : (ec == 1 ? w1 : w2);
                const bool rot = ec < 3;
                const float drc = (rot && er == ec) ? 1.0f : 0.0f;
                // W_rc = +w_{r+2} if c = r+1, -w_{r+1} if c = r+2, 0 on the diagonal
                const float Wrc = ec == (er + 1) % 3 ? -wr2 : (ec == (er + 2) % 3 ? wr1 : 0.0f);
                const float base = rot ? 0.0f : vr;
                const float a1 = rot ? Wrc : wr1, b1 = rot ? 1.0f : vr2;
                const float a2 = rot ? 0.0f : wr2, b2 = rot ? 0.0f : vr1;
                const float pq = rot ? wc : wv, dd = rot ? drc : vr;
                const float ex = fmaf(a1, b1, -(a2 * b2));
                const float ey = fmaf(wr, pq, -(dd * th2));
                const float dE = fmaf(rot ? B : Cc, ey, fmaf(rot ? A : B, ex, base));
                // ---- Tc = T exp(delta) = T + T (exp(delta) - I) in FP64:
                // Tc(r, c) = T(r, c) + sum_k T(r, k) dE(k, c)   (c = 3: dE(k, 3) = t_e(k))
                const double e0 = f64_of(__shfl_sync(full, dE, ec));
                const double e1 = f64_of(__shfl_sync(full, dE, 4 + ec));
                const double e2 = f64_of(__shfl_sync(full, dE, 8 + ec));
                tc = lane < 12 ? fma(S.T[4 * er], e0, fma(S.T[4 * er + 1], e1, fma(S.T[4 * er + 2], e2, S.T[4 * er + ec])))
                               : 0.0;
            } else {
                // ---- exp(delta_xi): R_e = I + A [w]x + B [w]x^2, t_e = v + B (w x v) + C w x (w x v)
                const double w0 = dl[3], w1 = dl[4], w2 = dl[5];
                const double th2 = fma(w0, w0, fma(w1, w1, w2 * w2));
                double A, B, Cc;
                if (th2 < 1e-4) {
                    A = fma(fma(th2, 1.0 / 120.0, -1.0 / 6.0), th2, 1.0);
                    B = fma(fma(th2, 1.0 / 720.0, -1.0 / 24.0), th2, 0.5);
                    Cc = fma(fma(th2, 1.0 / 5040.0, -1.0 / 120.0), th2, 1.0 / 6.0);
                } else if (th2 < 0.01) {
                    A = fma(fma(fma(fma(th2, 1.0 / 362880.0, -1.0 / 5040.0), th2, 1.0 / 120.0), th2, -1.0 / 6.0), th2, 1.0);
                    B = fma(fma(fma(fma(th2, 1.0 / 3628800.0, -1.0 / 40320.0), th2, 1.0 / 720.0), th2, -1.0 / 24.0), th2, 0.5);
                    Cc = fma(fma(fma(fma(th2, 1.0 / 39916800.0, -1.0 / 362880.0), th2, 1.0 / 5040.0), th2, -1.0 / 120.0), th2, 1.0 / 6.0);
                } else {
                    const double th = sqrt(th2);
                    double sn, cs, sh, ch;
                    sincos(th, &sn, &cs);
                    sincos(0.5 * th, &sh, &ch);
                    A = sn / th;
                    B = 2.0 * sh * sh / th2;
                    Cc = (th - sn) / (th2 * th);
                }
                // ---- E = exp(delta_xi) as a 3x4 [R_e | t_e], one element (r, c) per lane
                // 0-11, every lane running the same FP64 instructions on its own operands:
                //   R_e(r, c) = d_rc + A W_rc + B (w_r w_c - d_rc th2)            (W = [w]x)
                //   t_e(r)    = v_r + B (w x v)_r + C (w_r (w . v) - v_r th2)
                // as  base + cA (a1 b1 - a2 b2) + cB (p q - d th2).
                const double v0 = dl[0], v1 = dl[1], v2 = dl[2];
                const double wv = fma(w0, v0, fma(w1, v1, w2 * v2));
                const int er = (lane >> 2) % 3, ec = lane & 3;
                const double wr = er == 0 ? w0 : (er == 1 ? w1 : w2);
                const double wr1 = er == 0 ? w1 : (er == 1 ? w2 : w0);   // w_{r+1}
                const double wr2 = er == 0 ? w2 : (er == 1 ? w0 : w1);   // w_{r+2}
                const double vr = er == 0 ? v0 : (er == 1 ? v1 : v2);
                const double vr1 = er == 0 ? v1 : (er == 1 ? v2 : v0);
                const double vr2 = er == 0 ? v2 : (er == 1 ? v0 : v1);
                const double wc = ec == 0 ? w0 : (ec == 1 ? w1 : w2);
                const bool rot = ec < 3;
                const double drc = (rot && er == ec) ? 1.0 : 0.0;
                // W_rc = +w_{r+2} if c = r+1, -w_{r+1} if c = r+2, 0 on the diagonal
                const double Wrc = ec == (er + 1) % 3 ? -wr2 : (ec == (er + 2) % 3 ? wr1 : 0.0);
                const double base = rot ? drc : vr;
                const double a1 = rot ? Wrc : wr1, b1 = rot ? 1.0 : vr2;
                const double a2 = rot ? 0.0 : wr2, b2 = rot ? 0.0 : vr1;
                const double pq = rot ? wc : wv, dd = rot ? drc : vr;
                const double ex = fma(a1, b1, -(a2 * b2));
                const double ey = fma(wr, pq, -(dd * th2));
                const double E = fma(rot ? B : Cc, ey, fma(rot ? A : B, ex, base));
                // ---- Tc = T E: Tc(r, c) = sum_k T(r, k) E(k, c) (+ T(r, 3) for c = 3)
                const double e0 = __shfl_sync(full, E, ec);
                const double e1 = __shfl_sync(full, E, 4 + ec);
                const double e2 = __shfl_sync(full, E, 8 + ec);
                tc = lane < 12 ? fma(S.T[4 * er], e0, fma(S.T[4 * er + 1], e1,
                                      fma(S.T[4 * er + 2], e2, rot ? 0.0 : S.T[4 * er + 3])))
                               : 0.0;
            }
            const double ac = S.a + dl[6], bc = S.b + dl[7];
            const bool cand_finite = __all_sync(full, abs_bits(tc) < kInfBits) &&
                                     abs_bits(ac) < kInfBits && abs_bits(bc) < kInfBits;
            // a step below the level's stop threshold (and below accept_step)
            // would be taken whatever its cost and would end the level, so it
            // is taken here without a pass of its own: the next level's start
            // pass is the first evaluation of the new state; on the finest
            // level the result keeps the cost and count of the last evaluated
            // state
            const bool take_now = mbits < abs_bits(level > 0 ? D.eps_step_coarse : D.eps_step) &&
                                  mbits < abs_bits(D.accept_step);
            if (!cand_finite) {
                // the solve produced a state that is not finite: keep the
                // accepted one and end the level
                if (lane == 0) S.status |= GLT_TRACK_DIVERGED;
                finish = true;
                next_level = true;
            } else if (take_now) {
                if (lane < 12) S.T[lane] = tc;
                if (lane == 0) {
                    S.a = ac;
                    S.b = bc;
                    S.moved = 1;
                }
                ++it;
                finish = true;
                next_level = true;
            } else {
                if (lane < 12) S.Tc[lane] = tc;
                if (lane == 0) {
                    S.ac = ac;
                    S.bc = bc;
                    S.maxstep_bits = mbits;
                    S.phase = PH_CAND;
                }
                make_pass_params_lane(tc, ac, bc, level, P, lane);
            }
        }
    }
    if (finish && lane == 0) {
        S.iters[level] = it;
        S.res_E = S.E;
        S.res_n = S.n;
    }
    __syncwarp();
    if (next_level) {
        int l = level - 1;
        while (l >= 0 && D.max_iters[l] <= 0) --l;
        if (l < 0) {
            // GLT_SOLVE_FP32: the poses composed from FP32 increments drift
            // from orthonormal by ~1e-9 per step: one Newton step R' = R (3 I - R^T R) / 2 =
            // R + R (I - R^T R) / 2 on the final pose (FP64; the deviation
            // becomes its square)
            if (S.moved && D.solve == GLT_SOLVE_FP32) {
                const int i = lane / 3, j = lane % 3;
                double dlt = lane < 9 ? (i == j ? 1.0 : 0.0) : 0.0;
                if (lane < 9) {
#pragma unroll
                    for (int k = 0; k < 3; ++k) dlt = fma(-S.T[4 * k + i], S.T[4 * k + j], dlt);
                }
                const int r = lane >> 2, c = lane & 3;
                const int cc = c < 3 ? c : 0;
                const double d0 = __shfl_sync(full, dlt, cc), d1 = __shfl_sync(full, dlt, 3 + cc),
                             d2 = __shfl_sync(full, dlt, 6 + cc);
                double v = 0.0;
                if (lane < 12 && c < 3)
                    v = fma(0.5, fma(S.T[4 * r], d0, fma(S.T[4 * r + 1], d1, S.T[4 * r + 2] * d2)),
                            S.T[lane]);
                __syncwarp();
                if (lane < 12 && c < 3) S.T[lane] = v;
            }
            if (lane == 0) {
                S.done = 1;
                P.done = 1;
            }
        } else {
            if (lane == 0) {
                S.level = l;
                S.phase = PH_START;
            }
            make_pass_params_warp(S.T, S.a, S.b, l, P, lane);
        }
    }
    __syncwarp();
}

__device__ inline void solver_write_result(const StreamDesc& D, const Solver& S, glt_result* out)
{
    if (D.trace_count) *D.trace_count = S.passes;
    for (int i = 0; i < 12; ++i) out->T[i] = S.T[i];
    out->a = S.a;
    out->b = S.b;
    out->cost = S.res_n > 0 ? S.res_E / (double)S.res_n : S.res_E;
    out->n_valid = S.res_n;
    int tot = 0;
    for (int l = 0; l < kMaxLevels; ++l) {
        out->iters[l] = S.iters[l];
        tot += S.iters[l];
    }
    out->iters_total = tot;
    out->passes = S.passes;
    out->status = S.status;
}

}  // namespace glt
