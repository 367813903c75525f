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

__global__ void set_points_kernel(const StreamDesc* __restrict__ desc, RefLevels ref,
                                  const float* __restrict__ uvd, float cx, float cy,
                                  float4* __restrict__ pt, float2* __restrict__ dz,
                                  float* __restrict__ I0, float2* __restrict__ G0)
{
    const StreamDesc& D = *desc;
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= D.N) return;
    const float u0 = uvd[3 * p], v0 = uvd[3 * p + 1], d = uvd[3 * p + 2];
    const bool finite = isfinite(u0) && isfinite(v0) && isfinite(d) && d > 0.0f &&
                        fabsf(u0) < 1e7f && fabsf(v0) < 1e7f;
    pt[p] = make_float4(u0, v0, (u0 - cx) / D.fx, (v0 - cy) / D.fy);
    dz[p] = make_float2(d, 1.0f / d);
    for (int l = 0; l < D.L; ++l) {
        float4* out = reinterpret_cast<float4*>(I0 + ((size_t)l * D.Npad + p) * 8);
        const LevelDev& lv = D.lv[l];
        const float s = ldexpf(1.0f, -l);
        const float U = u0 * s, V = v0 * s;
        const float fu = floorf(U), fv = floorf(V);
        const int xb = finite ? (int)fu : -1000, yb = finite ? (int)fv : -1000;
        if (!finite || xb < 3 || xb > lv.W - 5 || yb < 3 || yb > lv.H - 5) {
            const float nan = __int_as_float(0x7fc00000);
            out[0] = make_float4(nan, 0.f, 0.f, 0.f);
            out[1] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (G0) {
                float4* g = reinterpret_cast<float4*>(G0 + ((size_t)l * D.Npad + p) * 8);
#pragma unroll
                for (int k = 0; k < 4; ++k) g[k] = make_float4(0.f, 0.f, 0.f, 0.f);
            }
            continue;
        }
        const float al = U - fu, be = V - fv;
        const float w00 = (1.0f - al) * (1.0f - be), w10 = al * (1.0f - be);
        const float w01 = (1.0f - al) * be, w11 = al * be;
        const uint8_t* img = ref.img[l];
        float v[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const uint8_t* t = img + (size_t)(yb + pat_dy(k)) * lv.pitch + (xb + pat_dx(k));
            v[k] = fmaf(w00, (float)t[0], fmaf(w10, (float)t[1], fmaf(w01, (float)t[lv.pitch], w11 * (float)t[lv.pitch + 1])));
        }
        out[0] = make_float4(v[0], v[1], v[2], v[3]);
        out[1] = make_float4(v[4], v[5], v[6], v[7]);
        if (G0) {
            // central differences at the four taps, bilinear weights, then the 1/2
            float gg[16];
            const int P = lv.pitch;
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const uint8_t* t = img + (size_t)(yb + pat_dy(k)) * P + (xb + pat_dx(k));
                const float I00 = t[0], I10 = t[1], I01 = t[P], I11 = t[P + 1];
                gg[2 * k] = 0.5f * fmaf(w00, I10 - (float)t[-1],
                                   fmaf(w10, (float)t[2] - I00,
                                   fmaf(w01, I11 - (float)t[P - 1],
                                        w11 * ((float)t[P + 2] - I01))));
                gg[2 * k + 1] = 0.5f * fmaf(w00, I01 - (float)t[-P],
                                       fmaf(w10, I11 - (float)t[1 - P],
                                       fmaf(w01, (float)t[2 * P] - I00,
                                            w11 * ((float)t[2 * P + 1] - I10))));
            }
            float4* g = reinterpret_cast<float4*>(G0 + ((size_t)l * D.Npad + p) * 8);
#pragma unroll
            for (int k = 0; k < 4; ++k) g[k] = make_float4(gg[4 * k], gg[4 * k + 1], gg[4 * k + 2], gg[4 * k + 3]);
        }
    }
}

cudaError_t launch_set_points(const glt_tracker* t, const float* uvd_dev, int n, cudaStream_t s)
{
    const int threads = 128;
    const int blocks = (n + threads - 1) / threads;
    if (blocks == 0) return cudaSuccess;
    RefLevels ref{};
    for (int l = 0; l < t->L; ++l) ref.img[l] = t->pyr[GLT_REF].base + t->pyr[GLT_REF].off[l];
    set_points_kernel<<<blocks, threads, 0, s>>>(t->desc_dev, ref, uvd_dev, (float)t->cfg.cx,
                                                 (float)t->cfg.cy, t->pt, t->dz, t->I0, t->G0);
    return cudaGetLastError();
}

}  // namespace glt
