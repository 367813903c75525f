// Map-point upload (GLidE-SLAM Sec. IV-C "Precompute"): back-project each
// point and sample its reference patch I0 at the 8 pattern offsets on every
// REF level (Eq. 2's I0(u_i^0 + du_k)); in the inverse-compositional form
// also the reference gradient there (the image part of the cached Jacobian
// rows of Sec. IV-B; the geometric part at x_r follows from the point).
#include "glt_internal.h"

namespace glt {

// One thread per point.  Level-l reference position u0 / 2^l is exact in
// FP32; the 8 samples share its fractional part, so their bilinear weights
// are computed once.  A point is unusable on a level (I0[..][0] = NaN) if its
// depth is not positive or a sample leaves 1 <= q < W-2, 1 <= q < H-2.
struct RefLevels {
    const uint8_t* img[kMaxLevels];
};

__global__ void set_points_kernel(StreamDesc* __restrict__ desc, int n, RefLevels ref,
                                  const float* __restrict__ uvd, float cx, float cy,
                                  float4* __restrict__ pt, float2* __restrict__ dz,
                                  float* __restrict__ I0, float2* __restrict__ G0)
{
    const StreamDesc& D = *desc;
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p == 0) desc->N = n;      // the point count the kernels of later passes read
    if (p >= n) return;
    const float u0 = uvd[3 * p], v0 = uvd[3 * p + 1], d = uvd[3 * p + 2];
    const bool finite = isfinite(u0) && isfinite(v0) && isfinite(d) && d > 0.0f &&
                        fabsf(u0) < 1e7f && fabsf(v0) < 1e7f;
    *checked(pt + p, 1, pt, (size_t)D.Npad, CK_SET_POINTS) = make_float4(u0, v0, (u0 - cx) / D.fx, (v0 - cy) / D.fy);
    *checked(dz + p, 1, dz, (size_t)D.Npad, CK_SET_POINTS) = make_float2(d, 1.0f / d);
    const int K = D.K, h = D.pattern ? (D.pattern - 1) / 2 : 2;
    for (int l = 0; l < D.L; ++l) {
        const size_t tab = (size_t)D.L * D.Npad * K;
        float* out = checked(I0 + ((size_t)l * D.Npad + p) * K, (size_t)K, I0, tab, CK_SET_POINTS);
        float2* gout = G0 ? checked(G0 + ((size_t)l * D.Npad + p) * K, (size_t)K, G0, tab, CK_SET_POINTS) : nullptr;
        const LevelDev& lv = D.lv[l];
        const float s = ldexpf(1.0f, -l);
        const float U = u0 * s, V = v0 * s;
        const float fu = floorf(U), fv = floorf(V);
        const int xb = finite ? (int)fu : -1000, yb = finite ? (int)fv : -1000;
        // every sample q = (U + dx, V + dy) must satisfy 1 <= q < W-2, 1 <= q < H-2
        if (!finite || xb < 1 + h || xb > lv.W - 3 - h || yb < 1 + h || yb > lv.H - 3 - h) {
            for (int k = 0; k < K; ++k) {
                out[k] = k == 0 ? __int_as_float(0x7fc00000) : 0.0f;
                if (gout) gout[k] = make_float2(0.0f, 0.0f);
            }
            continue;
        }
        const float al = U - fu, be = V - fv;
        const float w00 = (1.0f - al) * (1.0f - be), w10 = al * (1.0f - be);
        const float w01 = (1.0f - al) * be, w11 = al * be;
        const uint8_t* img = ref.img[l];
        const int P = lv.pitch;
        for (int k = 0; k < K; ++k) {
            const int dx = D.pattern ? k % D.pattern - h : pat_dx(k);
            const int dy = D.pattern ? k / D.pattern - h : pat_dy(k);
            const uint8_t* t = img + (size_t)(yb + dy) * P + (xb + dx);
            const float I00 = t[0], I10 = t[1], I01 = t[P], I11 = t[P + 1];
            out[k] = fmaf(w00, I00, fmaf(w10, I10, fmaf(w01, I01, w11 * I11)));
            if (gout) {
                // central differences at the four taps, bilinear weights, then the 1/2
                const float gx = 0.5f * fmaf(w00, I10 - (float)t[-1],
                                        fmaf(w10, (float)t[2] - I00,
                                        fmaf(w01, I11 - (float)t[P - 1],
                                             w11 * ((float)t[P + 2] - I01))));
                const float gy = 0.5f * fmaf(w00, I01 - (float)t[-P],
                                        fmaf(w10, I11 - (float)t[1 - P],
                                        fmaf(w01, (float)t[2 * P] - I00,
                                             w11 * ((float)t[2 * P + 1] - I10))));
                gout[k] = make_float2(gx, gy);
            }
        }
    }
}

// Sec. IV-B: with the inverse-compositional rows J_ik evaluated on the
// reference, H = sum_i sum_k J_ik^T J_ik is fixed while the reference is;
// Sec. IV-C "Precompute IC": each point's H_i is reduced into one H per level.
// One block per level: every thread sums the 21 upper-triangle products of
// its points' rows in FP32 per point (J_k = [Jt_k, x_r x Jt_k], Jt_k =
// gx_k a0 + gy_k a1 with the cached reference gradient and the projection
// rows at x_r, e^a = 1) and in FP64 across its points; the block adds the
// thread sums in a fixed tree order; thread 0 factorises H = L D L^T in FP64
// (pivots d > 0 and d > 1e-13 H_jj, else H^-1[0] = NaN: not positive
// definite) and writes H and H^-1 to Hc[72 l ..].
constexpr int kHessThreads = 256;

__global__ void __launch_bounds__(kHessThreads) ic_hessian_kernel(const StreamDesc* __restrict__ desc,
                                                                  double* __restrict__ Hc)
{
    __shared__ double red[kHessThreads][21];
    const StreamDesc& D = *desc;
    const int l = blockIdx.x;
    const int tid = threadIdx.x;
    const float s = ldexpf(1.0f, -l);
    double acc[21];
#pragma unroll
    for (int i = 0; i < 21; ++i) acc[i] = 0.0;
    for (int p = tid; p < D.N; p += kHessThreads) {
        const size_t base = ((size_t)l * D.Npad + p) * D.K;
        if (isnan(D.I0[base])) continue;          // not usable on this level of the reference
        const float4 q = D.pt[p];
        const float2 dz = D.dz[p];
        const float fxl = D.fx * s * dz.y, fyl = D.fy * s * dz.y;
        const float a0[3] = {fxl, 0.0f, -fxl * q.z};
        const float a1[3] = {0.0f, fyl, -fyl * q.w};
        const float xr[3] = {dz.x * q.z, dz.x * q.w, dz.x};
        float h[21];
#pragma unroll
        for (int i = 0; i < 21; ++i) h[i] = 0.0f;
        for (int k = 0; k < D.K; ++k) {
            const float2 g0 = D.G0[base + k];
            float J[6];
            J[0] = fmaf(g0.x, a0[0], g0.y * a1[0]);
            J[1] = fmaf(g0.x, a0[1], g0.y * a1[1]);
            J[2] = fmaf(g0.x, a0[2], g0.y * a1[2]);
            J[3] = fmaf(xr[1], J[2], -xr[2] * J[1]);
            J[4] = fmaf(xr[2], J[0], -xr[0] * J[2]);
            J[5] = fmaf(xr[0], J[1], -xr[1] * J[0]);
            int idx = 0;
#pragma unroll
            for (int i = 0; i < 6; ++i)
#pragma unroll
                for (int j = i; j < 6; ++j) {
                    h[idx] = fmaf(J[i], J[j], h[idx]);
                    ++idx;
                }
        }
#pragma unroll
        for (int i = 0; i < 21; ++i) acc[i] += (double)h[i];
    }
#pragma unroll
    for (int i = 0; i < 21; ++i) red[tid][i] = acc[i];
    __syncthreads();
    for (int half = kHessThreads / 2; half > 0; half >>= 1) {
        if (tid < half)
            for (int i = 0; i < 21; ++i) red[tid][i] += red[tid + half][i];
        __syncthreads();
    }
    if (tid != 0) return;
    double H[36], L[36] = {}, d[6], Hi[36];
    int idx = 0;
    for (int i = 0; i < 6; ++i)
        for (int j = i; j < 6; ++j) {
            H[6 * i + j] = H[6 * j + i] = red[0][idx];
            ++idx;
        }
    bool pd = true;
    for (int j = 0; j < 6 && pd; ++j) {
        double dj = H[6 * j + j];
        for (int k = 0; k < j; ++k) dj -= L[6 * j + k] * L[6 * j + k] * d[k];
        pd = dj > 0.0 && dj > 1e-13 * H[6 * j + j];
        d[j] = dj;
        L[6 * j + j] = 1.0;
        for (int i = j + 1; i < 6 && pd; ++i) {
            double v = H[6 * i + j];
            for (int k = 0; k < j; ++k) v -= L[6 * i + k] * L[6 * j + k] * d[k];
            L[6 * i + j] = v / dj;
        }
    }
    for (int c = 0; c < 6 && pd; ++c) {
        // column c of H^-1: L y = e_c, z = D^-1 y, L^T x = z
        double y[6], x[6];
        for (int i = 0; i < 6; ++i) {
            double v = i == c ? 1.0 : 0.0;
            for (int k = 0; k < i; ++k) v -= L[6 * i + k] * y[k];
            y[i] = v;
        }
        for (int i = 5; i >= 0; --i) {
            double v = y[i] / d[i];
            for (int k = i + 1; k < 6; ++k) v -= L[6 * k + i] * x[k];
            x[i] = v;
        }
        for (int i = 0; i < 6; ++i) Hi[6 * i + c] = x[i];
    }
    double* out = Hc + 72 * l;
    for (int i = 0; i < 36; ++i) {
        out[i] = H[i];
        out[36 + i] = pd ? Hi[i] : __longlong_as_double(0x7ff8000000000000ll);
    }
}

cudaError_t launch_ic_hessian(const glt_tracker* t, cudaStream_t s)
{
    ic_hessian_kernel<<<t->L, kHessThreads, 0, s>>>(t->desc_dev, t->Hc);
    return cudaGetLastError();
}

cudaError_t launch_set_points(const glt_tracker* t, const float* uvd_dev, int n, cudaStream_t s)
{
    const int threads = 128;
    const int blocks = n > 0 ? (n + threads - 1) / threads : 1;
    RefLevels ref{};
    for (int l = 0; l < t->L; ++l) ref.img[l] = t->pyr[GLT_REF].base + t->pyr[GLT_REF].off[l];
    set_points_kernel<<<blocks, threads, 0, s>>>(t->desc_dev, n, ref, uvd_dev, (float)t->cfg.cx,
                                                 (float)t->cfg.cy, t->pt, t->dz, t->I0, t->G0);
    return cudaGetLastError();
}

#ifdef GLT_CHECKED
unsigned check_flags_points()
{
    unsigned v = 0, z = 0;
    cudaMemcpyFromSymbol(&v, g_check_flags, sizeof(v));
    cudaMemcpyToSymbol(g_check_flags, &z, sizeof(z));
    return v;
}
#endif

}  // namespace glt

