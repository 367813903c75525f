// glt_linearize_noalloc: one linearisation pass on caller-owned device
// buffers that allocates nothing.
//
// Who needs it: callers that are not allowed to allocate device memory at
// the point where they want a linearisation -- real-time loops that fix their
// memory budget at start-up, and plugins whose host framework owns every
// device allocation.  glt_create allocates, so such a caller cannot build a
// tracker there; this entry point needs none.
//
// The only memory it uses besides the caller's inputs and outputs is a
// file-scope scratch array (block partial sums and the last-block ticket),
// which every GPU that loads the library holds until the process exits.
#include <cmath>
#include <cstring>
#include <mutex>

#include "glt_internal.h"

namespace glt {
namespace {

constexpr int kNaThreads = 128;
constexpr int kNaMaxBlocks = 512;
constexpr int kNaMaxPoints = kNaThreads * kNaMaxBlocks;   // 65536 map points
constexpr int kNaTicket = kNaMaxBlocks * kAccPad;         // index of the ticket word
constexpr int kNaWords = kNaTicket + 64;

// block partial sums (floats) followed by the ticket counter (as unsigned)
static __device__ __align__(256) float g_noalloc_scratch[kNaWords];

struct NaArgs {
    const uint8_t* ref;
    const uint8_t* cur;
    int W, H, ref_pitch, cur_pitch;
    float fx, fy, cx, cy;   // level-0 intrinsics
    const float* uvd;       // N x (u0, v0, depth), level-0 reference pixels
    int N;
    float huber_k, zmin;
};

// Reference sample (same bilinear weights for all 8 pattern pixels).
__device__ __forceinline__ float na_tap(const uint8_t* img, int pitch, int x, int y, float w00,
                                        float w10, float w01, float w11)
{
    const uint8_t* t = img + (size_t)y * pitch + x;
    return fmaf(w00, (float)t[0], fmaf(w10, (float)t[1], fmaf(w01, (float)t[pitch], w11 * (float)t[pitch + 1])));
}

__global__ void __launch_bounds__(kNaThreads)
    linearize_noalloc_kernel(NaArgs A, PassParams P, float* __restrict__ scratch,
                             double* __restrict__ out)
{
    constexpr int NW = kNaThreads / 32;
    __shared__ float red[NW][kAccPad];
    __shared__ float part[kAccPad];
    __shared__ int is_last;
    float acc[kAccPad];
#pragma unroll
    for (int i = 0; i < kAccPad; ++i) acc[i] = 0.0f;
    const int p = blockIdx.x * kNaThreads + threadIdx.x;
    const float s = P.scale;
    bool ok = p < A.N;
    float u0 = 0.f, v0 = 0.f, d = 0.f;
    if (ok) {
        u0 = A.uvd[3 * p];
        v0 = A.uvd[3 * p + 1];
        d = A.uvd[3 * p + 2];
        ok = isfinite(u0) && isfinite(v0) && isfinite(d) && d > 0.0f && fabsf(u0) < 1e7f && fabsf(v0) < 1e7f;
    }
    // reference patch I0 on this level
    float i0[8];
    if (ok) {
        const float U = u0 * s, V = v0 * s;
        const float fu = floorf(U), fv = floorf(V);
        const int xr = (int)fu, yr = (int)fv;
        ok = xr >= 3 && xr <= A.W - 5 && yr >= 3 && yr <= A.H - 5;
        if (ok) {
            const float al = U - fu, be = V - fv;
            const float w00 = (1.0f - al) * (1.0f - be), w10 = al * (1.0f - be);
            const float w01 = (1.0f - al) * be, w11 = al * be;
#pragma unroll
            for (int k = 0; k < 8; ++k)
                i0[k] = na_tap(A.ref, A.ref_pitch, xr + pat_dx(k), yr + pat_dy(k), w00, w10, w01, w11);
        }
    }
    // projection relative to the reference pixel (as in the tracker)
    PointGeom G;
    if (ok) {
        const float ub = (u0 - A.cx) / A.fx, vb = (v0 - A.cy) / A.fy, rho = 1.0f / d;
        const float Dx = fmaf(P.Rm[0], ub, fmaf(P.Rm[1], vb, fmaf(P.t[0], rho, P.Rm[2])));
        const float Dy = fmaf(P.Rm[3], ub, fmaf(P.Rm[4], vb, fmaf(P.t[1], rho, P.Rm[5])));
        const float Dz = fmaf(P.Rm[6], ub, fmaf(P.Rm[7], vb, fmaf(P.t[2], rho, P.Rm[8])));
        const float onez = 1.0f + Dz;
        ok = d * onez > A.zmin;
        if (ok) {
            const float iz = 1.0f / onez;
            const float du = A.fx * fmaf(-ub, Dz, Dx) * iz;
            const float dv = A.fy * fmaf(-vb, Dz, Dy) * iz;
            ok = fabsf(du) < 1e6f && fabsf(dv) < 1e6f;
            if (ok) {
                const float U = u0 * s, V = v0 * s;
                const float Ui = floorf(U), Vi = floorf(V);
                const float su = (U - Ui) + du * s, sv = (V - Vi) + dv * s;
                const float fu = floorf(su), fv = floorf(sv);
                G.al = su - fu;
                G.be = sv - fv;
                G.xb = (int)Ui + (int)fu;
                G.yb = (int)Vi + (int)fv;
                ok = G.xb >= 3 && G.xb <= A.W - 5 && G.yb >= 3 && G.yb <= A.H - 5;
                const float xn = (ub + Dx) * iz, yn = (vb + Dy) * iz;
                const float fxl = A.fx * s * rho * iz, fyl = A.fy * s * rho * iz;
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
            }
        }
    }
    if (ok) {
        const float w00 = (1.0f - G.al) * (1.0f - G.be), w10 = G.al * (1.0f - G.be);
        const float w01 = (1.0f - G.al) * G.be, w11 = G.al * G.be;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const uint8_t* t = A.cur + (size_t)(G.yb + pat_dy(k)) * A.cur_pitch + (G.xb + pat_dx(k));
            const int pc = A.cur_pitch;
            const float I00 = t[0], I10 = t[1], I01 = t[pc], I11 = t[pc + 1];
            const float I = fmaf(w00, I00, fmaf(w10, I10, fmaf(w01, I01, w11 * I11)));
            const float gx = 0.5f * fmaf(w00, I10 - (float)t[-1],
                                   fmaf(w10, (float)t[2] - I00,
                                   fmaf(w01, I11 - (float)t[pc - 1], w11 * ((float)t[pc + 2] - I01))));
            const float gy = 0.5f * fmaf(w00, I01 - (float)t[-pc],
                                   fmaf(w10, I11 - (float)t[1 - pc],
                                   fmaf(w01, (float)t[2 * pc] - I00, w11 * ((float)t[2 * pc + 1] - I10))));
            accumulate_sample(G, I, gx, gy, i0[k], P.ea, P.b, A.huber_k, acc, nullptr);
        }
    }
    block_reduce<kNaThreads, false>(acc, red, part, nullptr);
    if (threadIdx.x < kNumAcc) scratch[(size_t)blockIdx.x * kAccPad + threadIdx.x] = part[threadIdx.x];
    __threadfence();
    __syncthreads();
    unsigned* ticket = reinterpret_cast<unsigned*>(scratch + kNaTicket);
    if (threadIdx.x == 0) is_last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    __syncthreads();
    if (is_last) {
        __threadfence();
        if (threadIdx.x < kNumAcc) {
            double acc_d = 0.0;
            for (unsigned b = 0; b < gridDim.x; ++b)
                acc_d += (double)__ldcg(scratch + (size_t)b * kAccPad + threadIdx.x);
            out[threadIdx.x] = acc_d;
        }
        if (threadIdx.x == 0) *ticket = 0u;
    }
}

// Device address of the scratch array, looked up once per device and kept
// (an address that a reset of the device's primary context would invalidate).
constexpr int kNaMaxDevices = 64;
std::mutex g_na_mutex;
float* g_na_ptr[kNaMaxDevices] = {};

int na_scratch(float** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= kNaMaxDevices) {
        set_error("device ordinal beyond the scratch table");
        return GLT_ERR_UNSUPPORTED;
    }
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (!g_na_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(noalloc scratch)");
        g_na_ptr[dev] = static_cast<float*>(p);
    }
    *out = g_na_ptr[dev];
    return GLT_OK;
}

}  // namespace
}  // namespace glt

using namespace glt;

extern "C" int glt_linearize_noalloc(const uint8_t* ref_dev, int ref_pitch, const uint8_t* cur_dev,
                                     int cur_pitch, int width, int height, int level, double fx,
                                     double fy, double cx, double cy, const float* uvd_dev, int n,
                                     const double T[12], double a, double b, double huber_k,
                                     double zmin, double* out_dev, void* stream)
{
    if (!ref_dev || !cur_dev || !out_dev || !T || (n > 0 && !uvd_dev)) {
        set_error("glt_linearize_noalloc: NULL argument");
        return GLT_ERR_INVALID_ARG;
    }
    if (n < 0 || n > kNaMaxPoints) {
        set_error("glt_linearize_noalloc: n must be in [0, 65536] (size of the static scratch)");
        return n < 0 ? GLT_ERR_INVALID_ARG : GLT_ERR_CAPACITY;
    }
    if (level < 0 || level >= GLT_MAX_LEVELS || width < 16 || height < 16 || (width >> level) < 8 ||
        (height >> level) < 8 || ref_pitch < (width >> level) || cur_pitch < (width >> level)) {
        set_error("glt_linearize_noalloc: bad level size or pitch (pitch must be >= level width)");
        return GLT_ERR_INVALID_ARG;
    }
    if (!(fx > 0) || !(fy > 0) || !(huber_k > 0) || !(zmin > 0) || !std::isfinite(a) ||
        !std::isfinite(b)) {
        set_error("glt_linearize_noalloc: bad intrinsics or state");
        return GLT_ERR_INVALID_ARG;
    }
    for (int i = 0; i < 12; ++i)
        if (!std::isfinite(T[i])) {
            set_error("glt_linearize_noalloc: non-finite pose");
            return GLT_ERR_INVALID_ARG;
        }
    float* scratch = nullptr;
    int rc = na_scratch(&scratch);
    if (rc != GLT_OK) return rc;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    // the ticket must start at zero (a previous call that was cut short
    // could have left it non-zero)
    cudaError_t e = cudaMemsetAsync(scratch + kNaTicket, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return cuda_fail(e, "glt_linearize_noalloc ticket reset");
    if (n == 0) {
        e = cudaMemsetAsync(out_dev, 0, kNumAcc * sizeof(double), s);
        return e == cudaSuccess ? GLT_OK : cuda_fail(e, "glt_linearize_noalloc");
    }
    NaArgs A;
    A.ref = ref_dev;
    A.cur = cur_dev;
    A.W = width >> level;
    A.H = height >> level;
    A.ref_pitch = ref_pitch;
    A.cur_pitch = cur_pitch;
    A.fx = (float)fx;
    A.fy = (float)fy;
    A.cx = (float)cx;
    A.cy = (float)cy;
    A.uvd = uvd_dev;
    A.N = n;
    A.huber_k = (float)huber_k;
    A.zmin = (float)zmin;
    PassParams P;
    make_pass_params(T, a, b, level, P);
    const int blocks = (n + kNaThreads - 1) / kNaThreads;
    linearize_noalloc_kernel<<<blocks, kNaThreads, 0, s>>>(A, P, scratch, out_dev);
    e = cudaGetLastError();
    return e == cudaSuccess ? GLT_OK : cuda_fail(e, "glt_linearize_noalloc kernel");
}
