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
    pt[p] = make_float4(u0, v0, (u0 - cx) / D.fx, (v0 - cy) / D.fy);
    dz[p] = make_float2(d, 1.0f / d);
    const int K = D.K, h = D.pattern ? (D.pattern - 1) / 2 : 2;
    for (int l = 0; l < D.L; ++l) {
        float* out = I0 + ((size_t)l * D.Npad + p) * K;
        float2* gout = G0 ? G0 + ((size_t)l * D.Npad + p) * K : nullptr;
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

}  // namespace glt
