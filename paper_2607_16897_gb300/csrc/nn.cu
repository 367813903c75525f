// Learned initial-pose proposal: a 3 x (conv 3x3 stride 2 pad 1 + ReLU) +
// 2-layer MLP network (189064 parameters) mapping the coarsest-level residual
// image (1 x 30 x 40) and the previous inter-frame motion (6) to an 8-vector
// increment of the initial state.  Hand-written training and inference
// kernels: BF16 weights (rounded from FP32 master weights after every Adam
// step), FP32 activations and accumulation, deterministic reductions (fixed
// summation order, no atomics).
//
// Flat parameter layout: conv1.w [16,1,3,3], conv1.b [16], conv2.w [32,16,3,3],
// conv2.b [32], conv3.w [64,32,3,3], conv3.b [64], fc1.w [128,1286],
// fc1.b [128], fc2.w [8,128], fc2.b [8], row-major, in that order.
#include <cuda_bf16.h>

#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <vector>

#include <cooperative_groups.h>

#include "glt_internal.h"

namespace glt {
namespace nn {

constexpr int kIn = 1200, kMotion = 6, kOut = 8, kFlat = 1280, kF = 1286, kHid = 128;
struct Layer {
    int w, b;  // offsets of weight and bias in the flat layout
};
constexpr Layer kC1 = {0, 144}, kC2 = {160, 4768}, kC3 = {4800, 23232}, kF1 = {23296, 187904},
                kF2 = {188032, 189056};
constexpr int kParams = 189064;

__device__ __forceinline__ float wv(const __nv_bfloat16* w, int i) { return __bfloat162float(w[i]); }

// out[b,o,i,j] = bias_o + sum_{c,di,dj} w[o,c,di,dj] in[b,c,2i+di-1,2j+dj-1]; stores the
// pre-activation z and a = max(z, 0).
__global__ void conv_fwd(const float* __restrict__ in, const __nv_bfloat16* __restrict__ w, int woff,
                         int boff, int B, int C, int H, int W, int O, float* __restrict__ z,
                         float* __restrict__ a)
{
    const int Ho = (H + 1) / 2, Wo = (W + 1) / 2;
    const int n = B * O * Ho * Wo;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
        const int j = t % Wo, i = (t / Wo) % Ho, o = (t / (Wo * Ho)) % O, b = t / (Wo * Ho * O);
        float s = wv(w, boff + o);
        for (int c = 0; c < C; ++c) {
            const float* x = in + ((size_t)(b * C + c) * H) * W;
            const int wb = woff + (o * C + c) * 9;
#pragma unroll
            for (int di = 0; di < 3; ++di) {
                const int r = 2 * i + di - 1;
                if (r < 0 || r >= H) continue;
#pragma unroll
                for (int dj = 0; dj < 3; ++dj) {
                    const int q = 2 * j + dj - 1;
                    if (q < 0 || q >= W) continue;
                    s = fmaf(wv(w, wb + di * 3 + dj), x[r * W + q], s);
                }
            }
        }
        z[t] = s;
        a[t] = fmaxf(s, 0.0f);
    }
}

// out[b,o] = bias_o + sum_i w[o,i] in[b,i], in = (in0[b, 0:n0], in1[b, 0:n1]);
// one warp per output, lanes stride over i, fixed-order shuffle reduction.
__global__ void fc_fwd(const float* __restrict__ in0, int n0, const float* __restrict__ in1, int n1,
                       const __nv_bfloat16* __restrict__ w, int woff, int boff, int B, int O,
                       float* __restrict__ z, float* __restrict__ a, int relu)
{
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= B * O) return;
    const int b = warp / O, o = warp % O;
    const int n = n0 + n1;
    const __nv_bfloat16* wr = w + woff + (size_t)o * n;
    float s = 0.0f;
    for (int i = lane; i < n; i += 32) {
        const float x = i < n0 ? in0[(size_t)b * n0 + i] : in1[(size_t)b * n1 + (i - n0)];
        s = fmaf(wv(wr, i), x, s);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if (lane == 0) {
        s += wv(w, boff + o);
        z[warp] = s;
        a[warp] = relu ? fmaxf(s, 0.0f) : s;
    }
}

// dy = (y - t) / B and loss = 0.5 * sum (y - t)^2 / B (one block).
__global__ void loss_grad(const float* __restrict__ y, const float* __restrict__ t, int B,
                          float* __restrict__ dy, float* __restrict__ loss)
{
    __shared__ float red[256];
    float s = 0.0f;
    const int n = B * kOut;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const float d = y[i] - t[i];
        dy[i] = d / (float)B;
        s = fmaf(d, d, s);
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
        if (threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
        __syncthreads();
    }
    if (threadIdx.x == 0 && loss) *loss = 0.5f * red[0] / (float)B;
}

// fully connected backward: dW[o,i] = sum_b dz[b,o] in[b,i] (one thread per
// weight), db[o] = sum_b dz[b,o].
__global__ void fc_bwd_w(const float* __restrict__ dz, const float* __restrict__ in0, int n0,
                         const float* __restrict__ in1, int n1, int B, int O,
                         float* __restrict__ grad, int woff, int boff)
{
    const int n = n0 + n1;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < O * n) {
        const int o = t / n, i = t % n;
        float s = 0.0f;
        for (int b = 0; b < B; ++b) {
            const float x = i < n0 ? in0[(size_t)b * n0 + i] : in1[(size_t)b * n1 + (i - n0)];
            s = fmaf(dz[b * O + o], x, s);
        }
        grad[woff + t] = s;
    } else if (t < O * n + O) {
        const int o = t - O * n;
        float s = 0.0f;
        for (int b = 0; b < B; ++b) s += dz[b * O + o];
        grad[boff + o] = s;
    }
}

// input gradient of a fully connected layer, times the ReLU mask of the
// input's pre-activation: din[b,i] = (sum_o w[o,i] dz[b,o]) * (zin[b,i] > 0), i < nout.
__global__ void fc_bwd_in(const float* __restrict__ dz, const __nv_bfloat16* __restrict__ w, int woff,
                          int n, int B, int O, int nout, const float* __restrict__ zin,
                          float* __restrict__ din)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= B * nout) return;
    const int b = t / nout, i = t % nout;
    float s = 0.0f;
    for (int o = 0; o < O; ++o) s = fmaf(wv(w, woff + (size_t)o * n + i), dz[b * O + o], s);
    din[t] = zin[t] > 0.0f ? s : 0.0f;
}

// conv weight and bias gradients: one block per weight (or bias), strided
// loop over (b, i, j) and a fixed-order block reduction.
__global__ void conv_bwd_w(const float* __restrict__ dz, const float* __restrict__ in, int B, int C,
                           int H, int W, int O, float* __restrict__ grad, int woff, int boff)
{
    __shared__ float red[128];
    const int Ho = (H + 1) / 2, Wo = (W + 1) / 2;
    const int nw = O * C * 9;
    const int k = blockIdx.x;
    float s = 0.0f;
    const int n = B * Ho * Wo;
    if (k < nw) {
        const int o = k / (C * 9), c = (k / 9) % C, di = (k % 9) / 3, dj = k % 3;
        for (int t = threadIdx.x; t < n; t += blockDim.x) {
            const int j = t % Wo, i = (t / Wo) % Ho, b = t / (Wo * Ho);
            const int r = 2 * i + di - 1, q = 2 * j + dj - 1;
            if (r >= 0 && r < H && q >= 0 && q < W)
                s = fmaf(dz[((size_t)(b * O + o) * Ho + i) * Wo + j], in[((size_t)(b * C + c) * H + r) * W + q], s);
        }
    } else {
        const int o = k - nw;
        for (int t = threadIdx.x; t < n; t += blockDim.x) {
            const int j = t % Wo, i = (t / Wo) % Ho, b = t / (Wo * Ho);
            s += dz[((size_t)(b * O + o) * Ho + i) * Wo + j];
        }
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int st = 64; st > 0; st >>= 1) {
        if (threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
        __syncthreads();
    }
    if (threadIdx.x == 0) grad[k < nw ? woff + k : boff + (k - nw)] = red[0];
}

// conv input gradient times the input pre-activation's ReLU mask.
__global__ void conv_bwd_in(const float* __restrict__ dz, const __nv_bfloat16* __restrict__ w, int woff,
                            int B, int C, int H, int W, int O, const float* __restrict__ zin,
                            float* __restrict__ din)
{
    const int Ho = (H + 1) / 2, Wo = (W + 1) / 2;
    const int n = B * C * H * W;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
        const int x = t % W, y = (t / W) % H, c = (t / (W * H)) % C, b = t / (W * H * C);
        float s = 0.0f;
        for (int o = 0; o < O; ++o) {
#pragma unroll
            for (int di = 0; di < 3; ++di) {
                const int r2 = y + 1 - di;
                if (r2 < 0 || (r2 & 1) || (r2 >> 1) >= Ho) continue;
#pragma unroll
                for (int dj = 0; dj < 3; ++dj) {
                    const int q2 = x + 1 - dj;
                    if (q2 < 0 || (q2 & 1) || (q2 >> 1) >= Wo) continue;
                    s = fmaf(wv(w, woff + (o * C + c) * 9 + di * 3 + dj),
                             dz[((size_t)(b * O + o) * Ho + (r2 >> 1)) * Wo + (q2 >> 1)], s);
                }
            }
        }
        din[t] = zin[t] > 0.0f ? s : 0.0f;
    }
}

// Adam (Kingma and Ba) on the FP32 master weights, then the BF16 copy.
__global__ void adam(float* __restrict__ w, __nv_bfloat16* __restrict__ wbf, const float* __restrict__ g,
                     float* __restrict__ m, float* __restrict__ v, int n, float lr, float b1, float b2,
                     float eps, float c1, float c2)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = fmaf(b1, m[i], (1.0f - b1) * gi);
    const float vi = fmaf(b2, v[i], (1.0f - b2) * gi * gi);
    m[i] = mi;
    v[i] = vi;
    const float wi = w[i] - lr * (mi * c1) / (sqrtf(vi * c2) + eps);
    w[i] = wi;
    wbf[i] = __float2bfloat16_rn(wi);
}

__global__ void to_bf16(const float* __restrict__ w, __nv_bfloat16* __restrict__ wbf, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) wbf[i] = __float2bfloat16_rn(w[i]);
}

// conv2 / conv3 BF16 weights transposed to [K][O] (K = input channel x tap),
// the layout the proposal stage stages into shared memory as one contiguous
// copy; rewritten after every change of the BF16 weights.
constexpr int kW2 = 144 * 32, kW3 = 288 * 64;

__global__ void conv_relayout(const __nv_bfloat16* __restrict__ wbf, __nv_bfloat16* __restrict__ wt)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q < kW2)
        wt[(q % 144) * 32 + q / 144] = wbf[kC2.w + q];
    else if (q < kW2 + kW3)
        wt[kW2 + ((q - kW2) % 288) * 64 + (q - kW2) / 288] = wbf[kC3.w + (q - kW2)];
}

}  // namespace nn
}  // namespace glt

struct glt_nn {
    int max_batch = 0;
    int step = 0;
    float* w = nullptr;               // FP32 master
    __nv_bfloat16* wbf = nullptr;     // BF16 copy used by the kernels
    __nv_bfloat16* wt = nullptr;      // conv2 / conv3 BF16 weights as [K][O] (proposal stage)
    float* g = nullptr;
    float* m = nullptr;
    float* v = nullptr;
    float *z1, *a1, *z2, *a2, *z3, *a3, *z4, *h, *y, *dy, *dh, *d3, *d2, *d1;
    float* loss = nullptr;
};

using namespace glt;
using namespace glt::nn;

namespace {

int nn_alloc(glt_nn* n)
{
    const int B = n->max_batch;
    auto al = [](float** p, size_t count) {
        return cudaMalloc(reinterpret_cast<void**>(p), count * sizeof(float));
    };
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = al(&n->w, kParams);
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&n->wbf), kParams * sizeof(__nv_bfloat16));
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&n->wt), (kW2 + kW3) * sizeof(__nv_bfloat16));
    if (e == cudaSuccess) e = al(&n->g, kParams);
    if (e == cudaSuccess) e = al(&n->m, kParams);
    if (e == cudaSuccess) e = al(&n->v, kParams);
    if (e == cudaSuccess) e = al(&n->z1, (size_t)B * 16 * 15 * 20);
    if (e == cudaSuccess) e = al(&n->a1, (size_t)B * 16 * 15 * 20);
    if (e == cudaSuccess) e = al(&n->z2, (size_t)B * 32 * 8 * 10);
    if (e == cudaSuccess) e = al(&n->a2, (size_t)B * 32 * 8 * 10);
    if (e == cudaSuccess) e = al(&n->z3, (size_t)B * kFlat);
    if (e == cudaSuccess) e = al(&n->a3, (size_t)B * kFlat);
    if (e == cudaSuccess) e = al(&n->z4, (size_t)B * kHid);
    if (e == cudaSuccess) e = al(&n->h, (size_t)B * kHid);
    if (e == cudaSuccess) e = al(&n->y, (size_t)B * kOut);
    if (e == cudaSuccess) e = al(&n->dy, (size_t)B * kOut);
    if (e == cudaSuccess) e = al(&n->dh, (size_t)B * kHid);
    if (e == cudaSuccess) e = al(&n->d3, (size_t)B * kFlat);
    if (e == cudaSuccess) e = al(&n->d2, (size_t)B * 32 * 8 * 10);
    if (e == cudaSuccess) e = al(&n->d1, (size_t)B * 16 * 15 * 20);
    if (e == cudaSuccess) e = al(&n->loss, 1);
    if (e == cudaSuccess) e = cudaMemset(n->m, 0, kParams * sizeof(float));
    if (e == cudaSuccess) e = cudaMemset(n->v, 0, kParams * sizeof(float));
    return e == cudaSuccess ? GLT_OK : cuda_fail(e, "proposal network allocation");
}

void nn_free(glt_nn* n)
{
    if (!n) return;
    for (float* p : {n->w, n->g, n->m, n->v, n->z1, n->a1, n->z2, n->a2, n->z3, n->a3, n->z4, n->h,
                     n->y, n->dy, n->dh, n->d3, n->d2, n->d1, n->loss})
        cudaFree(p);
    cudaFree(n->wbf);
    cudaFree(n->wt);
    delete n;
}

int grid_for(int n, int t) { return (n + t - 1) / t; }

}  // namespace

cudaError_t glt::nn_forward(glt_nn* n, const float* x, const float* mo, int B, cudaStream_t s)
{
    conv_fwd<<<grid_for(B * 16 * 15 * 20, 128), 128, 0, s>>>(x, n->wbf, kC1.w, kC1.b, B, 1, 30, 40, 16, n->z1, n->a1);
    conv_fwd<<<grid_for(B * 32 * 8 * 10, 128), 128, 0, s>>>(n->a1, n->wbf, kC2.w, kC2.b, B, 16, 15, 20, 32, n->z2, n->a2);
    conv_fwd<<<grid_for(B * kFlat, 128), 128, 0, s>>>(n->a2, n->wbf, kC3.w, kC3.b, B, 32, 8, 10, 64, n->z3, n->a3);
    fc_fwd<<<grid_for(B * kHid * 32, 256), 256, 0, s>>>(n->a3, kFlat, mo, kMotion, n->wbf, kF1.w, kF1.b, B, kHid, n->z4, n->h, 1);
    fc_fwd<<<grid_for(B * kOut * 32, 256), 256, 0, s>>>(n->h, kHid, nullptr, 0, n->wbf, kF2.w, kF2.b, B, kOut, n->y, n->y, 0);
    return cudaGetLastError();
}

namespace {

cudaError_t nn_backward(glt_nn* n, const float* x, const float* mo, const float* t, int B, cudaStream_t s)
{
    loss_grad<<<1, 256, 0, s>>>(n->y, t, B, n->dy, n->loss);
    fc_bwd_w<<<grid_for(kOut * kHid + kOut, 256), 256, 0, s>>>(n->dy, n->h, kHid, nullptr, 0, B, kOut, n->g, kF2.w, kF2.b);
    fc_bwd_in<<<grid_for(B * kHid, 256), 256, 0, s>>>(n->dy, n->wbf, kF2.w, kHid, B, kOut, kHid, n->z4, n->dh);
    fc_bwd_w<<<grid_for(kHid * kF + kHid, 256), 256, 0, s>>>(n->dh, n->a3, kFlat, mo, kMotion, B, kHid, n->g, kF1.w, kF1.b);
    fc_bwd_in<<<grid_for(B * kFlat, 256), 256, 0, s>>>(n->dh, n->wbf, kF1.w, kF, B, kHid, kFlat, n->z3, n->d3);
    conv_bwd_w<<<64 * 32 * 9 + 64, 128, 0, s>>>(n->d3, n->a2, B, 32, 8, 10, 64, n->g, kC3.w, kC3.b);
    conv_bwd_in<<<grid_for(B * 32 * 8 * 10, 128), 128, 0, s>>>(n->d3, n->wbf, kC3.w, B, 32, 8, 10, 64, n->z2, n->d2);
    conv_bwd_w<<<32 * 16 * 9 + 32, 128, 0, s>>>(n->d2, n->a1, B, 16, 15, 20, 32, n->g, kC2.w, kC2.b);
    conv_bwd_in<<<grid_for(B * 16 * 15 * 20, 128), 128, 0, s>>>(n->d2, n->wbf, kC2.w, B, 16, 15, 20, 32, n->z1, n->d1);
    conv_bwd_w<<<16 * 1 * 9 + 16, 128, 0, s>>>(n->d1, x, B, 1, 30, 40, 16, n->g, kC1.w, kC1.b);
    return cudaGetLastError();
}

int check_batch(const glt_nn* n, int B)
{
    if (!n) return invalid_arg_msg("network is NULL");
    if (B < 1 || B > n->max_batch) return invalid_arg_msg("batch size outside [1, max_batch]");
    return GLT_OK;
}

}  // namespace

int glt::invalid_arg_msg(const char* msg)
{
    set_error(msg);
    return GLT_ERR_INVALID_ARG;
}

// ---------------------------------------------------------------------------
// Proposal stage of the batched tracker
// ---------------------------------------------------------------------------
namespace glt {
namespace nn {

// Proposal stage: one thread block per stream runs the whole inference with
// the activations in shared memory and the BF16 weights read through the
// read-only cache (they stay L2-resident across blocks):
//   x = (I_cur - I_ref) / 64 on the 40 x 30 coarsest level,
//   conv1 -> conv2 -> conv3 (ReLU) -> fc1 (ReLU) on [flatten, motion] -> fc2,
//   then T' = T exp(0.01 y[0:6]), a' = a + 0.01 y[6], b' = b + y[7].
// Conv inputs are stored with a one-pixel zero border, so every 3x3 window is
// read without bounds tests.  conv1 gives each thread 4 output channels of one
// pixel; conv2 and conv3 run as small GEMMs (output pixels x channels, K =
// input channel x tap) with register tiles of PT pixels x 4 channels, on the
// layer's weights in the [K][O] layout (a tile's 4 weights are one 8-byte
// load), copied into shared memory with asynchronous 16-byte copies issued at
// the start and awaited just before conv2.  The sum order per output (bias,
// then channel, row, column) is that of conv_fwd.
constexpr int kPropThreads = 512;
constexpr int kXp = 32 * 42, kA1p = 16 * 17 * 22, kA2p = 32 * 10 * 12;
constexpr int kPropSmemFloats = kXp + kA1p + kA2p + (kF + 2) + kHid + kOut;
constexpr size_t kPropSmemBytes = kPropSmemFloats * sizeof(float) + (kW2 + kW3) * sizeof(__nv_bfloat16);
static_assert(kPropSmemFloats % 4 == 0, "the BF16 weights must start on a 16-byte boundary");
static_assert((kXp + kA1p + kA2p) % 4 == 0, "the bordered planes are cleared as float4");
static_assert((kW2 + kW3) * sizeof(__nv_bfloat16) % 16 == 0, "the weight copy is made of 16-byte pieces");

// Bordered activation planes keep each row as its even columns followed by
// its odd columns (column c of a row of Wp at (c & 1) * Wp / 2 + c / 2): the
// stride-2 3x3 windows of consecutive output pixels then read consecutive
// words, where the plain layout read every other one (two-way bank
// conflicts).
__device__ __forceinline__ int split_col(int c, int Wp) { return (c & 1) * (Wp >> 1) + (c >> 1); }

// GEMM form of a stride-2 3x3 conv on a zero-bordered, column-split input:
// thread t < tasks computes PT output pixels p = pg + u PG (consecutive
// lanes, consecutive pixels) x 4 channels.  Output planes bordered and
// column-split if PADOUT, else flat.
template <int C, int H, int W, int O, int PT, bool PADOUT>
__device__ __forceinline__ void conv_gemm(const float* __restrict__ in, const __nv_bfloat16* __restrict__ wt,
                                          const __nv_bfloat16* __restrict__ w, int boff,
                                          float* __restrict__ out)
{
    constexpr int Ho = (H + 1) / 2, Wo = (W + 1) / 2, Wp = W + 2, plane = (H + 2) * (W + 2), half = Wp / 2;
    constexpr int PG = Ho * Wo / PT, tasks = PG * (O / 4);
    static_assert(Ho * Wo % PT == 0, "pixel tiles must cover the output");
    static_assert(tasks <= kPropThreads, "one tile per thread");
    static_assert(Wp % 2 == 0, "column-split rows need an even padded width");
    const int t = threadIdx.x;
    if (t >= tasks) return;
    const int pg = t % PG, cg = t / PG;
    int base[PT];
#pragma unroll
    for (int u = 0; u < PT; ++u) {
        const int p = pg + u * PG;
        base[u] = 2 * (p / Wo) * Wp + (p % Wo);     // window row 2i, split column of 2j
    }
    float acc[PT][4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float b = __bfloat162float(__ldg(w + boff + cg * 4 + k));
#pragma unroll
        for (int u = 0; u < PT; ++u) acc[u][k] = b;
    }
    for (int c = 0; c < C; ++c) {
        const float* xc = in + c * plane;
        const __nv_bfloat16* wc = wt + (c * 9) * O + cg * 4;
#pragma unroll
        for (int q = 0; q < 9; ++q) {
            const uint2 raw = *reinterpret_cast<const uint2*>(wc + q * O);
            const float2 w01 = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&raw.x));
            const float2 w23 = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&raw.y));
            const int di = q / 3, dj = q % 3;
            const int off = di * Wp + (dj & 1) * half + (dj >> 1);   // column 2j + dj
#pragma unroll
            for (int u = 0; u < PT; ++u) {
                const float a = xc[base[u] + off];
                acc[u][0] = fmaf(w01.x, a, acc[u][0]);
                acc[u][1] = fmaf(w01.y, a, acc[u][1]);
                acc[u][2] = fmaf(w23.x, a, acc[u][2]);
                acc[u][3] = fmaf(w23.y, a, acc[u][3]);
            }
        }
    }
#pragma unroll
    for (int u = 0; u < PT; ++u) {
        const int p = pg + u * PG, i = p / Wo, j = p % Wo;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int o = cg * 4 + k;
            const float r = fmaxf(acc[u][k], 0.0f);
            if (PADOUT)
                out[o * (Ho + 2) * (Wo + 2) + (i + 1) * (Wo + 2) + split_col(j + 1, Wo + 2)] = r;
            else
                out[(o * Ho + i) * Wo + j] = r;
        }
    }
}

__device__ __forceinline__ float2 wv2(const __nv_bfloat16* w, int i)
{
    return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(w + i));
}

// in: C planes of (H+2) x (W+2) with a zero border, rows column-split; out: O
// planes of the (H+1)/2 x (W+1)/2 result, bordered and column-split if
// PADOUT, else flat.
template <int C, int H, int W, int O, int KO, bool PADOUT>
__device__ __forceinline__ void conv_block(const float* __restrict__ in, const __nv_bfloat16* __restrict__ w,
                                           int woff, int boff, float* __restrict__ out)
{
    constexpr int Ho = (H + 1) / 2, Wo = (W + 1) / 2, Wp = W + 2, plane = (H + 2) * (W + 2);
    constexpr int tasks = (O / KO) * Ho * Wo;
    for (int t = threadIdx.x; t < tasks; t += kPropThreads) {
        const int p = t % (Ho * Wo), og = t / (Ho * Wo);
        const int i = p / Wo, j = p % Wo;
        float acc[KO];
#pragma unroll
        for (int k = 0; k < KO; ++k) acc[k] = __bfloat162float(__ldg(w + boff + og * KO + k));
        const float* xb = in + (2 * i) * Wp + j;      // column-split rows: column 2j + dj
        for (int c = 0; c < C; ++c) {
            float v[9];
#pragma unroll
            for (int di = 0; di < 3; ++di)
#pragma unroll
                for (int dj = 0; dj < 3; ++dj)
                    v[di * 3 + dj] = xb[c * plane + di * Wp + (dj & 1) * (Wp >> 1) + (dj >> 1)];
#pragma unroll
            for (int k = 0; k < KO; ++k) {
                const __nv_bfloat16* wk = w + woff + ((og * KO + k) * C + c) * 9;
#pragma unroll
                for (int q = 0; q < 9; ++q) acc[k] = fmaf(__bfloat162float(__ldg(wk + q)), v[q], acc[k]);
            }
        }
#pragma unroll
        for (int k = 0; k < KO; ++k) {
            const int o = og * KO + k;
            const float r = fmaxf(acc[k], 0.0f);
            if (PADOUT)
                out[o * (Ho + 2) * (Wo + 2) + (i + 1) * (Wo + 2) + split_col(j + 1, Wo + 2)] = r;
            else
                out[(o * Ho + i) * Wo + j] = r;
        }
    }
}

// Network motion input from the stream's last inter-frame motion M = [R | t]
// (row-major 3x4): log(M) / 0.02 as (upsilon, omega).  The input is FP32, and
// so is this evaluation after the differences of M's entries it starts from
// (vee(R - R^T), trace R - 1 and, near pi, the symmetric part), which are
// formed in FP64.  sin th = |vee| / 2 and cos th = (trace - 1) / 2, th their
// atan2; omega = th / (2 sin th) vee (its series below th = 1e-4; near pi the
// axis comes from the symmetric part instead); upsilon = V^-1 t with
// V^-1 = I - W/2 + k W^2, k = (1 - A / (2 B)) / th^2, A = sin th / th,
// B = (1 - cos th) / th^2, taken below th = 0.5 as its series
// k = sum_n |B_2n| th^(2n-2) / (2n)! (Bernoulli numbers), to th^8.
constexpr float kMotionScale = 0.02f;

__device__ void motion_feature(const double* __restrict__ M, float* __restrict__ f6)
{
    const float vee[3] = {(float)(M[9] - M[6]), (float)(M[2] - M[8]), (float)(M[4] - M[1])};
    const float t[3] = {(float)M[3], (float)M[7], (float)M[11]};
    const float sn = 0.5f * sqrtf(vee[0] * vee[0] + vee[1] * vee[1] + vee[2] * vee[2]);
    const float cs = (float)(0.5 * (M[0] + M[5] + M[10] - 1.0));
    const float th = atan2f(sn, cs);
    const float pi = 3.14159265358979f;
    float w[3];
    if (th < 1e-4f) {
        const float k = 0.5f * (1.0f + th * th / 6.0f);
        for (int i = 0; i < 3; ++i) w[i] = k * vee[i];
    } else if (th < pi - 1e-4f) {
        const float k = th / (2.0f * sn);
        for (int i = 0; i < 3; ++i) w[i] = k * vee[i];
    } else {
        const double Rd[3] = {M[0], M[5], M[10]};
        int m = 0;
        for (int i = 1; i < 3; ++i)
            if (Rd[i] > Rd[m]) m = i;
        const float d = sqrtf((float)(0.5 * (Rd[m] + 1.0)));
        float a[3];
        for (int i = 0; i < 3; ++i)
            a[i] = i == m ? d : (float)(0.5 * (M[4 * i + m] + M[4 * m + i])) / (2.0f * d);
        const float na = sqrtf(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
        const float sg = (a[0] * vee[0] + a[1] * vee[1] + a[2] * vee[2]) < 0.0f ? -1.0f : 1.0f;
        for (int i = 0; i < 3; ++i) w[i] = sg * th * a[i] / na;
    }
    const float th2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
    float k;
    if (th < 0.5f) {
        k = 1.0f / 12.0f + th2 * (1.0f / 720.0f + th2 * (1.0f / 30240.0f +
                                 th2 * (1.0f / 1209600.0f + th2 * (1.0f / 47900160.0f))));
    } else {
        const float sh = sinf(0.5f * th);
        const float A = sinf(th) / th, B = 2.0f * sh * sh / th2;
        k = (1.0f - A / (2.0f * B)) / th2;
    }
    // W = [w]x;  V^-1 t = t - (w x t) / 2 + k w x (w x t)
    const float wt[3] = {w[1] * t[2] - w[2] * t[1], w[2] * t[0] - w[0] * t[2], w[0] * t[1] - w[1] * t[0]};
    const float wwt[3] = {w[1] * wt[2] - w[2] * wt[1], w[2] * wt[0] - w[0] * wt[2],
                          w[0] * wt[1] - w[1] * wt[0]};
    for (int i = 0; i < 3; ++i) {
        f6[i] = (t[i] - 0.5f * wt[i] + k * wwt[i]) / kMotionScale;
        f6[3 + i] = w[i] / kMotionScale;
    }
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem)
{
    const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}

// fc1 is shared by the kPropCluster blocks of a thread-block cluster (one
// stream each; blocks past the last stream only help): block r computes
// hidden units [r kHid / kPropCluster, (r + 1) kHid / kPropCluster) for every
// stream of its cluster, from the streams' feature vectors copied out of the
// peers' shared memory, and writes each result into its stream's block, so
// the 329 KB of fc1 weights are read from L2 once per cluster instead of once
// per stream.  Each output keeps conv_fwd's lane split and reduction order.
constexpr int kPropCluster = 4;
static_assert(kHid % (kPropCluster * (kPropThreads / 32)) == 0, "whole rows per warp");
static_assert(kPropCluster * (kF + 2) <= kA1p, "the peers' feature vectors fit where conv1's output was");

__global__ void __launch_bounds__(kPropThreads)
proposal_kernel(const PropJob* __restrict__ jobs, const double* __restrict__ motion,
                const double* __restrict__ init, const __nv_bfloat16* __restrict__ w,
                const __nv_bfloat16* __restrict__ wt, double* __restrict__ out, int S)
{
    namespace cg = cooperative_groups;
    cg::cluster_group cluster = cg::this_cluster();
    extern __shared__ __align__(16) float sm[];
    float* xp = sm;
    float* a1 = xp + kXp;
    float* a2 = a1 + kA1p;
    float* f = a2 + kA2p;
    float* h = f + (kF + 2);
    float* y = h + kHid;
    __nv_bfloat16* w2t = reinterpret_cast<__nv_bfloat16*>(y + kOut);
    __nv_bfloat16* w3t = w2t + kW2;
    const int s = blockIdx.x;
    const bool valid = s < S;      // block-uniform: blocks past the last stream only share fc1
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // conv2 / conv3 weights: one contiguous [K][O] copy, in flight until conv2
    for (int v = tid; v < (kW2 + kW3) / 8; v += kPropThreads) cp_async16(w2t + 8 * v, wt + 8 * v);
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    // the rows of T each lane of warp 0 composes at the end (lanes 12, 13: a, b)
    double Tr[4] = {0.0, 0.0, 0.0, 0.0};
    if (valid && warp == 0 && lane < 14) {
        const double* T = init + 14 * s;
        if (lane < 12) {
            for (int k = 0; k < 4; ++k) Tr[k] = T[4 * (lane >> 2) + k];
        } else {
            Tr[0] = T[lane];
        }
    }
    float4* z4 = reinterpret_cast<float4*>(sm);
    for (int q = tid; q < (kXp + kA1p + kA2p) / 4; q += kPropThreads) z4[q] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    __syncthreads();
    if (valid) {
        const PropJob J = jobs[s];
        for (int p = tid; p < kIn; p += kPropThreads) {
            const int r = p / 40, c = p % 40;
            xp[(r + 1) * 42 + split_col(c + 1, 42)] =
                ((float)J.cur[r * J.pitch + c] - (float)J.ref[r * J.pitch + c]) * (1.0f / 64.0f);
        }
        __syncthreads();
        conv_block<1, 30, 40, 16, 4, true>(xp, w, kC1.w, kC1.b, a1);
    }
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    __syncthreads();
    if (valid) {
        // the motion input, on a thread that conv2's 320 tiles leave idle
        if (tid == kPropThreads - 1) motion_feature(motion + 12 * s, f + kFlat);
        conv_gemm<16, 15, 20, 32, 2, true>(a1, w2t, w, kC2.b, a2);
        __syncthreads();
        conv_gemm<32, 8, 10, 64, 1, false>(a2, w3t, w, kC3.b, f);
    } else {
        for (int i = tid; i < kF + 2; i += kPropThreads) f[i] = 0.0f;
    }
    // every block's feature vector is complete; copy the cluster's into the
    // (dead) conv1 output area
    cluster.sync();
    float* fl = a1;
    for (int q = 0; q < kPropCluster; ++q) {
        const float* src = cluster.map_shared_rank(f, q);
        for (int i = tid; i < kF + 2; i += kPropThreads) fl[q * (kF + 2) + i] = src[i];
    }
    __syncthreads();
    // fc1: this block's kHid / kPropCluster rows for every stream of the
    // cluster, two rows per warp, BF16 pairs along the rows; each result goes
    // to its stream's block
    {
        constexpr int RPB = kHid / kPropCluster, RPW = RPB / (kPropThreads / 32);
        const int rank = (int)cluster.block_rank();
        const int o0 = rank * RPB + warp * RPW;
        float acc[RPW][kPropCluster];
#pragma unroll
        for (int k = 0; k < RPW; ++k)
#pragma unroll
            for (int q = 0; q < kPropCluster; ++q) acc[k][q] = 0.0f;
#pragma unroll 4
        for (int i = 2 * lane; i < kF; i += 64) {
            float2 fq[kPropCluster];
#pragma unroll
            for (int q = 0; q < kPropCluster; ++q) fq[q] = make_float2(fl[q * (kF + 2) + i], fl[q * (kF + 2) + i + 1]);
#pragma unroll
            for (int k = 0; k < RPW; ++k) {
                const float2 wp = wv2(w, kF1.w + (o0 + k) * kF + i);
#pragma unroll
                for (int q = 0; q < kPropCluster; ++q) {
                    acc[k][q] = fmaf(wp.x, fq[q].x, acc[k][q]);
                    acc[k][q] = fmaf(wp.y, fq[q].y, acc[k][q]);
                }
            }
        }
#pragma unroll
        for (int k = 0; k < RPW; ++k)
#pragma unroll
            for (int q = 0; q < kPropCluster; ++q)
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) acc[k][q] += __shfl_xor_sync(0xffffffffu, acc[k][q], off);
        if (lane < RPW * kPropCluster) {
            const int k = lane / kPropCluster, q = lane % kPropCluster;
            float v = 0.0f;
#pragma unroll
            for (int kk = 0; kk < RPW; ++kk)
#pragma unroll
                for (int qq = 0; qq < kPropCluster; ++qq)
                    if (kk == k && qq == q) v = acc[kk][qq];
            cluster.map_shared_rank(h, q)[o0 + k] = fmaxf(v + wv(w, kF1.b + o0 + k), 0.0f);
        }
    }
    // every stream's hidden vector is complete (and no block reads a peer after this)
    cluster.sync();
    if (!valid) return;
    if (warp < kOut) {
        const int row = kF2.w + warp * kHid;
        float acc = 0.0f;
        for (int i = 2 * lane; i < kHid; i += 64) {
            const float2 wp = wv2(w, row + i);
            acc = fmaf(wp.x, h[i], acc);
            acc = fmaf(wp.y, h[i + 1], acc);
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
        if (lane == 0) y[warp] = acc + wv(w, kF2.b + warp);
    }
    __syncthreads();
    if (warp != 0 || lane >= 14) return;
    // T' = T exp(d) = T + T (exp(d) - I): the increment exp(d) - I, whose
    // entries are O(|d|), in FP32 (every lane the whole 3 x 4 matrix;
    // A = sin th / th, B = (1 - cos th) / th^2, C = (th - sin th) / th^3 as
    // series below th^2 = 0.25, truncation below 1e-10 relative), the
    // composition in FP64: lane 4 r + c writes entry (r, c), lanes 12 and 13
    // the affine pair
    double* O = out + 14 * s;
    if (lane >= 12) {
        O[lane] = Tr[0] + (double)y[lane - 6] * (lane == 12 ? 0.01 : 1.0);
        return;
    }
    float d[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) d[k] = y[k] * 0.01f;
    const float w0 = d[3], w1 = d[4], w2 = d[5];
    const float th2 = w0 * w0 + w1 * w1 + w2 * w2;
    float A, B, C;
    if (th2 < 0.25f) {
        A = 1.0f - th2 * (1.0f / 6.0f - th2 * (1.0f / 120.0f - th2 * (1.0f / 5040.0f - th2 * (1.0f / 362880.0f))));
        B = 0.5f - th2 * (1.0f / 24.0f - th2 * (1.0f / 720.0f - th2 * (1.0f / 40320.0f - th2 * (1.0f / 3628800.0f))));
        C = 1.0f / 6.0f - th2 * (1.0f / 120.0f - th2 * (1.0f / 5040.0f - th2 * (1.0f / 362880.0f - th2 * (1.0f / 39916800.0f))));
    } else {
        const float th = sqrtf(th2), sn = sinf(th), sh = sinf(0.5f * th);
        A = sn / th;
        B = 2.0f * sh * sh / th2;
        C = (th - sn) / (th2 * th);
    }
    // W = [w]x, W^2 = w w^T - th^2 I; rotation increment A W + B W^2,
    // translation V t - t = B W t + C W^2 t with t = d[0:3]
    const float Wm[3][3] = {{0.0f, -w2, w1}, {w2, 0.0f, -w0}, {-w1, w0, 0.0f}};
    const float ww[3] = {w0, w1, w2};
    float dE[3][4];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        float wt = 0.0f, w2t = 0.0f;
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const float W2 = ww[k] * ww[j] - (k == j ? th2 : 0.0f);
            dE[k][j] = fmaf(A, Wm[k][j], B * W2);
            wt = fmaf(Wm[k][j], d[j], wt);
            w2t = fmaf(W2, d[j], w2t);
        }
        dE[k][3] = d[k] + fmaf(B, wt, C * w2t);
    }
    const int c = lane & 3;
    double v = c == 0 ? Tr[0] : c == 1 ? Tr[1] : c == 2 ? Tr[2] : Tr[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float e = c == 0 ? dE[k][0] : c == 1 ? dE[k][1] : c == 2 ? dE[k][2] : dE[k][3];
        v = fma(Tr[k], (double)e, v);
    }
    O[lane] = v;
}

}  // namespace nn

cudaError_t launch_proposal(glt_batch* b, const double* init_dev, cudaStream_t s)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)((b->S + nn::kPropCluster - 1) / nn::kPropCluster * nn::kPropCluster), 1, 1);
    cfg.blockDim = dim3(nn::kPropThreads, 1, 1);
    cfg.dynamicSmemBytes = nn::kPropSmemBytes;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = nn::kPropCluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, nn::proposal_kernel, b->prop_jobs, b->motion_dev, init_dev,
                              (const __nv_bfloat16*)b->nn->wbf, (const __nv_bfloat16*)b->nn->wt,
                              b->prop_init, b->S);
}

}  // namespace glt

extern "C" {

int glt_batch_set_proposal(glt_batch* b, glt_nn* n, const double* motion_dev)
{
    if (!b) return invalid_arg_msg("batch is NULL");
    if (b->exec) {
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
    }
    if (b->graph) {
        cudaGraphDestroy(b->graph);
        b->graph = nullptr;
    }
    if (!n) {
        b->nn = nullptr;
        b->motion_dev = nullptr;
        return GLT_OK;
    }
    if (!motion_dev) return invalid_arg_msg("motion_dev is NULL");
    if (n->max_batch < b->S) return invalid_arg_msg("network max_batch is smaller than the batch");
    std::vector<PropJob> jobs(b->S);
    for (int i = 0; i < b->S; ++i) {
        glt_tracker* t = b->trk[i];
        const int l = t->L - 1;
        if (t->W[l] != 40 || t->H[l] != 30)
            return invalid_arg_msg("the proposal needs every stream's coarsest level to be 40 x 30");
        jobs[i].ref = t->pyr[GLT_REF].base + t->pyr[GLT_REF].off[l];
        jobs[i].cur = t->pyr[GLT_CUR].base + t->pyr[GLT_CUR].off[l];
        jobs[i].pitch = t->pitch[l];
    }
    cudaError_t e = cudaSuccess;
    if (!b->prop_jobs) {
        e = cudaMalloc(reinterpret_cast<void**>(&b->prop_jobs), b->S * sizeof(PropJob));
        if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&b->prop_init), (size_t)b->S * 14 * sizeof(double));
        if (e != cudaSuccess) return cuda_fail(e, "proposal buffers");
    }
    e = cudaMemcpy(b->prop_jobs, jobs.data(), b->S * sizeof(PropJob), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(nn::proposal_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)nn::kPropSmemBytes);
    if (e != cudaSuccess) return cuda_fail(e, "proposal jobs");
    b->nn = n;
    b->motion_dev = motion_dev;
    return GLT_OK;
}

int glt_nn_create(int max_batch, glt_nn** out)
{
    if (!out) return invalid_arg_msg("out is NULL");
    *out = nullptr;
    if (max_batch < 1 || max_batch > 65536) return invalid_arg_msg("max_batch must be in [1, 65536]");
    glt_nn* n = new glt_nn();
    n->max_batch = max_batch;
    int rc = nn_alloc(n);
    if (rc != GLT_OK) {
        nn_free(n);
        return rc;
    }
    *out = n;
    return GLT_OK;
}

void glt_nn_destroy(glt_nn* n) { nn_free(n); }

int glt_nn_set_params(glt_nn* n, const float* host, int count)
{
    if (!n || !host) return invalid_arg_msg("NULL argument");
    if (count != kParams) return invalid_arg_msg("count must equal GLT_NN_PARAMS");
    cudaError_t e = cudaMemcpy(n->w, host, kParams * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(n->m, 0, kParams * sizeof(float));
    if (e == cudaSuccess) e = cudaMemset(n->v, 0, kParams * sizeof(float));
    if (e != cudaSuccess) return cuda_fail(e, "glt_nn_set_params");
    to_bf16<<<grid_for(kParams, 256), 256>>>(n->w, n->wbf, kParams);
    conv_relayout<<<grid_for(kW2 + kW3, 256), 256>>>(n->wbf, n->wt);
    e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(e, "glt_nn_set_params");
    n->step = 0;
    return GLT_OK;
}

int glt_nn_get_params(glt_nn* n, float* host, int count)
{
    if (!n || !host) return invalid_arg_msg("NULL argument");
    if (count != kParams) return invalid_arg_msg("count must equal GLT_NN_PARAMS");
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(host, n->w, kParams * sizeof(float), cudaMemcpyDeviceToHost);
    return e == cudaSuccess ? GLT_OK : cuda_fail(e, "glt_nn_get_params");
}

int glt_nn_forward(glt_nn* n, const float* x_dev, const float* m_dev, float* y_dev, int B, void* stream)
{
    int rc = check_batch(n, B);
    if (rc != GLT_OK) return rc;
    if (!x_dev || !m_dev || !y_dev) return invalid_arg_msg("NULL argument");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = nn_forward(n, x_dev, m_dev, B, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(y_dev, n->y, (size_t)B * kOut * sizeof(float), cudaMemcpyDeviceToDevice, s);
    return e == cudaSuccess ? GLT_OK : cuda_fail(e, "glt_nn_forward");
}

int glt_nn_gradient(glt_nn* n, const float* x_dev, const float* m_dev, const float* t_dev, int B,
                    float* grad_host, float* loss_host, void* stream)
{
    int rc = check_batch(n, B);
    if (rc != GLT_OK) return rc;
    if (!x_dev || !m_dev || !t_dev || !grad_host) return invalid_arg_msg("NULL argument");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = nn_forward(n, x_dev, m_dev, B, s);
    if (e == cudaSuccess) e = nn_backward(n, x_dev, m_dev, t_dev, B, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(grad_host, n->g, kParams * sizeof(float), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && loss_host) e = cudaMemcpyAsync(loss_host, n->loss, sizeof(float), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return e == cudaSuccess ? GLT_OK : cuda_fail(e, "glt_nn_gradient");
}

int glt_nn_train_step(glt_nn* n, const float* x_dev, const float* m_dev, const float* t_dev, int B,
                      float lr, float* loss_dev, void* stream)
{
    int rc = check_batch(n, B);
    if (rc != GLT_OK) return rc;
    if (!x_dev || !m_dev || !t_dev) return invalid_arg_msg("NULL argument");
    if (!(lr > 0.0f)) return invalid_arg_msg("lr must be > 0");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = nn_forward(n, x_dev, m_dev, B, s);
    if (e == cudaSuccess) e = nn_backward(n, x_dev, m_dev, t_dev, B, s);
    if (e != cudaSuccess) return cuda_fail(e, "glt_nn_train_step");
    n->step += 1;
    const double b1 = 0.9, b2 = 0.999;
    const float c1 = (float)(1.0 / (1.0 - std::pow(b1, n->step)));
    const float c2 = (float)(1.0 / (1.0 - std::pow(b2, n->step)));
    adam<<<grid_for(kParams, 256), 256, 0, s>>>(n->w, n->wbf, n->g, n->m, n->v, kParams, lr, (float)b1,
                                                (float)b2, 1e-8f, c1, c2);
    conv_relayout<<<grid_for(kW2 + kW3, 256), 256, 0, s>>>(n->wbf, n->wt);
    if (loss_dev) e = cudaMemcpyAsync(loss_dev, n->loss, sizeof(float), cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaGetLastError();
    return e == cudaSuccess ? GLT_OK : cuda_fail(e, "glt_nn_train_step");
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Checkpoints and weight files

namespace {

const char kCkptTag[8] = {'G', 'L', 'T', 'N', 'N', 'C', 'K', '1'};

int io_fail(const char* what, const char* path)
{
    set_error(std::string(what) + ": " + (path ? path : "(null)"));
    return GLT_ERR_IO;
}

// Little-endian int32 from 4 bytes, independent of the host's byte order.
int32_t le32(const unsigned char* p)
{
    return (int32_t)((uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16) |
                     ((uint32_t)p[3] << 24));
}

void put_le32(unsigned char* p, int32_t v)
{
    const uint32_t u = (uint32_t)v;
    for (int i = 0; i < 4; ++i) p[i] = (unsigned char)(u >> (8 * i));
}

bool read_floats(FILE* f, std::vector<float>& out, size_t n)
{
    std::vector<unsigned char> raw(n * 4);
    if (std::fread(raw.data(), 1, raw.size(), f) != raw.size()) return false;
    out.resize(n);
    for (size_t i = 0; i < n; ++i) {
        const uint32_t u = (uint32_t)le32(&raw[4 * i]);
        std::memcpy(&out[i], &u, 4);
    }
    return true;
}

bool write_floats(FILE* f, const std::vector<float>& v)
{
    std::vector<unsigned char> raw(v.size() * 4);
    for (size_t i = 0; i < v.size(); ++i) {
        uint32_t u;
        std::memcpy(&u, &v[i], 4);
        put_le32(&raw[4 * i], (int32_t)u);
    }
    return std::fwrite(raw.data(), 1, raw.size(), f) == raw.size();
}

// The header of a NumPy .npy file (format versions 1-3): checks that it
// describes GLT_NN_PARAMS little-endian float32 values in one C-order
// dimension and leaves `f` at the data.
int npy_header(FILE* f, const unsigned char* head8, const char* path)
{
    const int major = head8[6];
    size_t hlen = 0;
    if (major == 1) {
        unsigned char b[2];
        if (std::fread(b, 1, 2, f) != 2) return io_fail("short .npy header", path);
        hlen = (size_t)b[0] | ((size_t)b[1] << 8);
    } else if (major == 2 || major == 3) {
        unsigned char b[4];
        if (std::fread(b, 1, 4, f) != 4) return io_fail("short .npy header", path);
        hlen = (size_t)(uint32_t)le32(b);
    } else {
        return invalid_arg_msg("unsupported .npy version");
    }
    if (hlen == 0 || hlen > 65536) return invalid_arg_msg("bad .npy header length");
    std::string h(hlen, ' ');
    if (std::fread(&h[0], 1, hlen, f) != hlen) return io_fail("short .npy header", path);
    char shape[32];
    std::snprintf(shape, sizeof(shape), "(%d,)", kParams);
    if (h.find("'<f4'") == std::string::npos || h.find("'fortran_order': False") == std::string::npos ||
        h.find(shape) == std::string::npos)
        return invalid_arg_msg(".npy file is not GLT_NN_PARAMS little-endian float32 values");
    return GLT_OK;
}

}  // namespace

extern "C" {

int glt_nn_save(glt_nn* n, const char* path)
{
    if (!n || !path) return invalid_arg_msg("NULL argument");
    std::vector<float> w(kParams), m(kParams), v(kParams);
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(w.data(), n->w, kParams * sizeof(float), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(m.data(), n->m, kParams * sizeof(float), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(v.data(), n->v, kParams * sizeof(float), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "glt_nn_save");
    FILE* f = std::fopen(path, "wb");
    if (!f) return io_fail("cannot open for writing", path);
    unsigned char head[16];
    std::memcpy(head, kCkptTag, 8);
    put_le32(head + 8, kParams);
    put_le32(head + 12, n->step);
    bool ok = std::fwrite(head, 1, 16, f) == 16 && write_floats(f, w) && write_floats(f, m) &&
              write_floats(f, v);
    ok = (std::fclose(f) == 0) && ok;
    return ok ? GLT_OK : io_fail("write failed", path);
}

int glt_nn_load(glt_nn* n, const char* path)
{
    if (!n || !path) return invalid_arg_msg("NULL argument");
    FILE* f = std::fopen(path, "rb");
    if (!f) return io_fail("cannot open", path);
    unsigned char head[8];
    std::vector<float> w, m, v;
    int step = 0;
    int rc = GLT_OK;
    if (std::fread(head, 1, 8, f) != 8) {
        rc = io_fail("short file", path);
    } else if (std::memcmp(head, kCkptTag, 8) == 0) {
        unsigned char b[8];
        if (std::fread(b, 1, 8, f) != 8) {
            rc = io_fail("short checkpoint header", path);
        } else if (le32(b) != kParams || le32(b + 4) < 0) {
            rc = invalid_arg_msg("checkpoint of another network size");
        } else {
            step = le32(b + 4);
            if (!read_floats(f, w, kParams) || !read_floats(f, m, kParams) || !read_floats(f, v, kParams))
                rc = io_fail("short checkpoint", path);
        }
    } else if (std::memcmp(head, "\x93NUMPY", 6) == 0) {
        rc = npy_header(f, head, path);
        if (rc == GLT_OK && !read_floats(f, w, kParams)) rc = io_fail("short .npy data", path);
    } else {
        rc = invalid_arg_msg("neither a network checkpoint nor a .npy file");
    }
    std::fclose(f);
    if (rc != GLT_OK) return rc;
    if (m.empty()) {
        m.assign(kParams, 0.0f);
        v.assign(kParams, 0.0f);
    }
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(n->w, w.data(), kParams * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(n->m, m.data(), kParams * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(n->v, v.data(), kParams * sizeof(float), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "glt_nn_load");
    to_bf16<<<grid_for(kParams, 256), 256>>>(n->w, n->wbf, kParams);
    conv_relayout<<<grid_for(kW2 + kW3, 256), 256>>>(n->wbf, n->wt);
    e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(e, "glt_nn_load");
    n->step = step;
    return GLT_OK;
}

}  // extern "C"
