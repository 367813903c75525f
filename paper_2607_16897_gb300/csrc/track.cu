// The persistent tracker kernel (whole coarse-to-fine LM in one launch, one
// thread-block cluster per stream) and the single-pass multi-block
// linearisation kernel.
//
// GLidE-SLAM Sec. IV-C "Track": per level and iteration, per-point residuals
// and Jacobians, a tree reduction, a Cholesky solve and T <- T exp(delta),
// all on the GPU.  Here the level x iteration loop stays inside one kernel:
// each CTA of the cluster linearises a slice of the map points, the CTA sums
// are exchanged through distributed shared memory, and every CTA runs the
// (bit-identical) FP64 LM decision, so only one cluster barrier per pass is
// needed.
#include <cooperative_groups.h>

#include "glt_internal.h"

namespace cg = cooperative_groups;

namespace glt {

constexpr int kMaxCluster = 16;   // largest cluster a stream may use (config.cluster)

// ---------------------------------------------------------------------------
// Cluster exchange of the CTA partial sums.  Every CTA pushes its partial
// (48 floats; with the Kahan compensations 96) into a slot of every CTA of
// the cluster, itself included, with st.async stores that complete bytes on
// the receiver's mbarrier; a CTA sums its slots in rank order once its
// barrier's phase has completed.  One mbarrier and one slot array per pass
// parity: pass k + 2 writes a CTA's parity-k slots only after every CTA has
// finished pass k + 1, which needs this CTA's pass k + 1 partial, pushed after
// it read its pass k slots.  Waits are bounded (kExchangeLimit cycles); a
// wait that runs out ends the solve with GLT_TRACK_TIMEOUT.
constexpr long long kExchangeLimit = 1ll << 31;    // ~1 s at 2 GHz

template <int W>
struct Exchange {
    float slot[2][kMaxCluster][W];
    unsigned long long mbar[2];
};

__device__ __forceinline__ unsigned smem_addr(const void* p)
{
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(unsigned long long* m, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(m)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect(unsigned long long* m, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(m)), "r"(bytes)
                 : "memory");
}

// true once the phase of parity `parity` has completed; false after `limit` cycles
__device__ __forceinline__ bool mbar_wait(unsigned long long* m, unsigned parity, long long limit)
{
    const long long t0 = clock64();
    while (true) {
        unsigned done;
        asm volatile("{\n\t.reg .pred p;\n\t"
                     "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}"
                     : "=r"(done)
                     : "r"(smem_addr(m)), "r"(parity)
                     : "memory");
        if (done) return true;
        if (clock64() - t0 > limit) return false;
    }
}

// 16 bytes to CTA `cta`'s copy of the local address `dst`, completing on its copy of `m`
__device__ __forceinline__ void push16(float* dst, float4 v, unsigned long long* m, unsigned cta)
{
    unsigned rd, rm;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(rd) : "r"(smem_addr(dst)), "r"(cta));
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(rm) : "r"(smem_addr(m)), "r"(cta));
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v4.b32 [%0], {%1, %2, %3, %4}, [%5];"
                 ::"r"(rd), "r"(__float_as_uint(v.x)), "r"(__float_as_uint(v.y)), "r"(__float_as_uint(v.z)),
                   "r"(__float_as_uint(v.w)), "r"(rm)
                 : "memory");
}

// Arm this pass's receive, push the CTA partial src[0:W] (16-byte chunks) to
// every CTA of the cluster.  Called by all threads after the block reduction.
template <int THREADS, int W>
__device__ __forceinline__ void exchange_push(Exchange<W>& X, int par, const float* src, int C, int rank)
{
    constexpr int CH = W / 4;
    if (threadIdx.x == 0) mbar_arrive_expect(&X.mbar[par], (unsigned)(C * W * 4));
    for (int t = threadIdx.x; t < C * CH; t += THREADS) {
        const int r = t / CH, q = t % CH;
        push16(&X.slot[par][rank][4 * q], reinterpret_cast<const float4*>(src)[q], &X.mbar[par], (unsigned)r);
    }
}

// The 128-thread shape is capped at 128 registers so four CTAs fit on an SM
// (batches of many small clusters); the wider shapes keep the registers the
// compiler wants (a single stream's latency).

// VAR: 0 FP32 levels, forward Jacobian; 1 FP16-packed levels (GLT_MIXED);
// 2 FP32 with the p x p patch path compiled in; 3 FP32 with the
// inverse-compositional rows compiled in; 4 the cached-Hessian form (FP32,
// inverse-compositional rows, any pattern: per pass only g, E and n are
// reduced and the step uses the per-reference H^-1).  Variants 1-3 decide the
// Jacobian form (and 2 the pattern) per stream, so one batch may mix them;
// variant 4 runs only streams of that form.
template <int THREADS, int VAR>
__global__ void __launch_bounds__(THREADS, THREADS == 128 ? 4 : 1) track_kernel(const StreamDesc* const* __restrict__ descs,
                                                        const int* __restrict__ users,
                                                        const double* __restrict__ init,
                                                        glt_result* __restrict__ results)
{
    constexpr int NW = THREADS / 32;
    constexpr bool MIXED = VAR == 1, SQUARE = VAR == 2 || VAR == 4, IC = VAR != 0, HC = VAR == 4;
    constexpr int NACC = HC ? kHcAcc : kAccPad;    // accumulators per thread
    constexpr int NSUM = HC ? kHcAcc : kNumAcc;    // sums exchanged per pass
    // CTA partial per pass parity: the sums (MIXED: their compensations at +kAccPad)
    constexpr int XW = HC ? kHcAcc : MIXED ? 2 * kAccPad : kAccPad;
    __shared__ StreamDesc sD;
    __shared__ PassParams P;
    __shared__ Solver S;
    __shared__ float red[NW][kAccPad];
    __shared__ __align__(16) float part[2][XW];
    __shared__ __align__(16) Exchange<XW> X;
    __shared__ double tot[kAccPad];
    __shared__ int xfail;

    cg::cluster_group cluster = cg::this_cluster();
    const int C = (int)cluster.num_blocks();
    const int rank = (int)cluster.block_rank();
    const int stream = blockIdx.x / C;
    const int tid = threadIdx.x;

    const int user = users[stream];
    {
        const int* src = reinterpret_cast<const int*>(descs[stream]);
        int* dst = reinterpret_cast<int*>(&sD);
        for (int i = tid; i < (int)(sizeof(StreamDesc) / sizeof(int)); i += THREADS) dst[i] = src[i];
    }
    __syncthreads();
    if (tid == 0) {
        solver_init(sD, init + 14 * user, S, P);
        xfail = 0;
        if (C > 1) {
            mbar_init(&X.mbar[0], 1);
            mbar_init(&X.mbar[1], 1);
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
    }
    // every CTA's barriers exist before the first push
    if (C > 1)
        cluster.sync();
    else
        __syncthreads();
    // Everything above reads data that was final before the previous kernel
    // of the stream started; the CUR levels it may still be writing are read
    // only after this wait (a no-op unless launched as a programmatic
    // dependent, which is how glt_track_image_async and the batch graph chain
    // the track launch behind the pyramid kernels).
    griddep_wait();

    const int tail_warp = (int)(blockIdx.x % NW);
    int par = 0;
    unsigned xph = 0;    // bit p: parity of the phase of X.mbar[p] the next wait completes
    PointCache pc;
    pc.p = -1;
    pc.level = -1;
    while (!P.done) {
        float acc[NACC];
#pragma unroll
        for (int i = 0; i < NACC; ++i) acc[i] = 0.0f;
        if constexpr (HC) {
            // tasks: row groups of the p x p patches (kHcGroups per point) or whole points
            const int groups = hc_groups(sD.pattern);
            const int tasks = sD.N * groups;
            for (int t = rank * THREADS + tid; t < tasks; t += C * THREADS) {
                const int p = groups == 1 ? t : t / kHcGroups;
                if (pc.p != p || pc.level != P.level) load_point(sD, P.level, p, pc);
                linearize_task_hc(sD, P, pc, t - p * groups, groups, acc);
            }
        } else {
            for (int p = rank * THREADS + tid; p < sD.N; p += C * THREADS) {
                // a thread that owns one point keeps its data for the whole level
                // (the 128-thread shape, capped at 128 registers for batches of
                // many streams, reloads it instead)
                if (THREADS == 128 || pc.p != p || pc.level != P.level) load_point(sD, P.level, p, pc);
                linearize_point<MIXED, false, SQUARE, IC, HC>(sD, P, pc, acc, nullptr);
            }
        }
        if constexpr (HC)
            block_reduce8<THREADS>(acc, red, part[par]);
        else
            block_reduce<THREADS, MIXED>(acc, red, part[par], MIXED ? part[par] + kAccPad : nullptr);
        if (C > 1) exchange_push<THREADS, XW>(X, par, part[par], C, rank);
        if (tid < NSUM) {
            // finish over the CTAs of the cluster: a compensated FP32 sum
            // (TwoSum, error-free per step) of the pushed partials in rank
            // order, converted to FP64 once; the FP64 pipe of this GPU is too
            // slow to carry a chain of C adds
            if (C > 1 && !mbar_wait(&X.mbar[par], (xph >> par) & 1u, kExchangeLimit)) xfail = 1;
            const float* src = C > 1 ? &X.slot[par][0][0] : &part[par][0];
            float v[kMaxCluster], vc[kMaxCluster];
#pragma unroll
            for (int r = 0; r < kMaxCluster; ++r) {
                if (r < C) {
                    v[r] = src[r * XW + tid];
                    if (MIXED) vc[r] = src[r * XW + kAccPad + tid];
                }
            }
            float hi = 0.0f, lo = 0.0f;
#pragma unroll
            for (int r = 0; r < kMaxCluster; ++r) {
                if (r < C) {
                    if (MIXED) lo += vc[r];
                    const float s = hi + v[r];
                    const float bb = s - hi;
                    lo += (hi - (s - bb)) + (v[r] - bb);
                    hi = s;
                }
            }
            tot[tid] = (double)hi + (double)lo;
        }
        xph ^= 1u << par;
        __syncthreads();
        if (xfail) {
            // a peer's partial did not arrive within the limit: end the solve
            // with the accepted state
            if (tid == 0) {
                S.status |= GLT_TRACK_TIMEOUT;
                S.done = 1;
            }
            break;
        }
        // the FP64 tail runs on one warp; CTAs of different streams that share an
        // SM use different warps so their tails spread over the SM's sub-partitions
        if ((tid >> 5) == tail_warp) solver_step_warp<HC>(sD, tot, S, P, tid & 31, rank == 0);
        __syncthreads();
        par ^= 1;
    }
    if (xfail && tid == 0) {
        // let pushes still in flight into this CTA land (bounded) before it leaves
        mbar_wait(&X.mbar[par], ((xph >> par) & 1u) ^ 1u, kExchangeLimit);
    }
    // leave together: no CTA exits while a peer may still push into it
    if (C > 1) cluster.sync();
    if (rank == 0 && tid == 0) solver_write_result(sD, S, results + user);
}

// The fixed part of a tracker pass, for its latency floor: the block
// reduction, the cluster barrier, the distributed-shared-memory finish and the
// FP64 tail, exactly as in track_kernel, with no point linearised.  The sums
// the tail sees are replaced by a fixed, well-conditioned normal system whose
// steps are small, so that every pass is an accepted candidate (a full
// decision, factorisation or H^-1 product, exponential and composition).
// CTA 0 of the cluster records the cycles of the pass loop.
__device__ double g_floor_Hc[72];   // H and H^-1 of the cached-Hessian floor (device data)

template <int THREADS, bool HC>
__global__ void __launch_bounds__(THREADS, 1) pass_floor_kernel(int passes, int drop_rank, int solve,
                                                                 long long* __restrict__ cycles)
{
    constexpr int NW = THREADS / 32;
    constexpr int NSUM = HC ? kHcAcc : kNumAcc;
    constexpr int XW = HC ? kHcAcc : kAccPad;
    __shared__ StreamDesc sD;
    __shared__ PassParams P;
    __shared__ Solver S;
    __shared__ float red[NW][kAccPad];
    __shared__ __align__(16) float part[2][XW];
    __shared__ __align__(16) Exchange<XW> X;
    __shared__ double tot[kAccPad];
    __shared__ int xfail;
    cg::cluster_group cluster = cg::this_cluster();
    const int C = (int)cluster.num_blocks();
    const int rank = (int)cluster.block_rank();
    const int tid = threadIdx.x;
    if (tid == 0) {
        int* z = reinterpret_cast<int*>(&sD);
        for (int i = 0; i < (int)(sizeof(StreamDesc) / sizeof(int)); ++i) z[i] = 0;
        sD.L = 1;
        sD.max_iters[0] = passes + 1;
        sD.min_valid = 1;
        sD.affine = 1;
        sD.lambda0 = 1e-4;
        sD.lambda_up = 4.0;
        sD.lambda_down = 0.5;
        sD.accept_step = 1e-3;
        sD.solve = solve;
        sD.Hc = HC ? g_floor_Hc : nullptr;
        if (HC && blockIdx.x == 0)
            for (int i = 0; i < 72; ++i) {
                const int r = (i % 36) / 6, c = i % 6;
                g_floor_Hc[i] = r == c ? (i < 36 ? 100.0 + 10.0 * r : 1.0 / (100.0 + 10.0 * r)) : 0.0;
            }
        double init[14];
        for (int i = 0; i < 14; ++i) init[i] = (i < 12 && i % 5 == 0) ? 1.0 : 0.0;
        solver_init(sD, init, S, P);
        xfail = 0;
        if (C > 1) {
            mbar_init(&X.mbar[0], 1);
            mbar_init(&X.mbar[1], 1);
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
    }
    if (C > 1) cluster.sync();
    __syncthreads();
    const long long t0 = clock64();
    int par = 0;
    unsigned xph = 0;
    for (int it = 0; it < passes; ++it) {
        float acc[kAccPad];
#pragma unroll
        for (int i = 0; i < kAccPad; ++i) acc[i] = 0.0f;
        if constexpr (HC) {
            float a8[kHcAcc];
#pragma unroll
            for (int i = 0; i < kHcAcc; ++i) a8[i] = acc[i];
            block_reduce8<THREADS>(a8, red, part[par]);
        } else {
            block_reduce<THREADS, false>(acc, red, part[par], nullptr);
        }
        // drop_rank >= 0 (the timeout test): that CTA withholds its first push
        if (C > 1 && !(it == 0 && rank == drop_rank)) exchange_push<THREADS, XW>(X, par, part[par], C, rank);
        if (tid < NSUM) {
            if (C > 1 && !mbar_wait(&X.mbar[par], (xph >> par) & 1u, kExchangeLimit)) xfail = 1;
            const float* src = C > 1 ? &X.slot[par][0][0] : &part[par][0];
            float v[kMaxCluster];
#pragma unroll
            for (int r = 0; r < kMaxCluster; ++r)
                if (r < C) v[r] = src[r * XW + tid];
            float hi = 0.0f, lo = 0.0f;
#pragma unroll
            for (int r = 0; r < kMaxCluster; ++r) {
                if (r < C) {
                    const float sum = hi + v[r];
                    const float bb = sum - hi;
                    lo += (hi - (sum - bb)) + (v[r] - bb);
                    hi = sum;
                }
            }
            // the fixed system (the reduced zeros are added so the finish is not dead code)
            double x;
            if (HC) {
                x = tid < 6 ? 1e-3 * (tid + 1) : (tid == kHcE ? 1000.0 : 1000.0);
            } else {
                x = tid == kIdxE ? 1000.0 : tid == kIdxN ? 1000.0 : tid >= kIdxG ? 1e-3 * (tid - kIdxG + 1) : 1.0;
                for (int i = 0; i < 8; ++i)
                    if (tid == upper_index(i, i)) x = 100.0 + 10.0 * i;
            }
            tot[tid] = x + (double)hi + (double)lo;
        }
        xph ^= 1u << par;
        __syncthreads();
        if (xfail) break;
        if ((tid >> 5) == (int)(blockIdx.x % NW)) solver_step_warp<HC>(sD, tot, S, P, tid & 31, false);
        __syncthreads();
        par ^= 1;
    }
    const long long t1 = clock64();
    if (xfail && tid == 0) mbar_wait(&X.mbar[par], ((xph >> par) & 1u) ^ 1u, kExchangeLimit);
    if (C > 1) cluster.sync();
    if (blockIdx.x == 0 && tid == 0) cycles[0] = xfail ? -1 : t1 - t0;
}

// One linearisation pass over all points of one tracker, many blocks, with a
// single-pass finish: each block writes its 46 sums, the last block to arrive
// (ticket counter) adds the block sums in block order in FP64.
template <int THREADS, int VAR>
__global__ void __launch_bounds__(THREADS) linearize_kernel(const StreamDesc* __restrict__ desc,
                                                            PassParams P,
                                                            float* __restrict__ partials,
                                                            unsigned* __restrict__ counter,
                                                            double* __restrict__ out,
                                                            float* __restrict__ res)
{
    constexpr int NW = THREADS / 32;
    constexpr bool MIXED = VAR == 1, SQUARE = VAR == 2 || VAR == 4, IC = VAR != 0, HC = VAR == 4;
    constexpr int NACC = HC ? kHcAcc : kAccPad;
    constexpr int NSUM = HC ? kHcAcc : kNumAcc;
    __shared__ float red[NW][kAccPad];
    __shared__ float part[kAccPad];
    __shared__ float part_c[kAccPad];
    __shared__ int is_last;
    const StreamDesc& D = *desc;
    float acc[NACC];
#pragma unroll
    for (int i = 0; i < NACC; ++i) acc[i] = 0.0f;
    const int p = blockIdx.x * THREADS + threadIdx.x;
    if (p < D.N) {
        PointCache pc;
        load_point(D, P.level, p, pc);
        if (res)
            linearize_point<MIXED, true, SQUARE, IC, HC>(D, P, pc, acc, res);
        else
            linearize_point<MIXED, false, SQUARE, IC, HC>(D, P, pc, acc, nullptr);
    }
    if constexpr (HC)
        block_reduce8<THREADS>(acc, red, part);
    else
        block_reduce<THREADS, MIXED>(acc, red, part, part_c);
    if (threadIdx.x < NSUM)
        partials[(size_t)blockIdx.x * kAccPad + threadIdx.x] = part[threadIdx.x] + (MIXED ? part_c[threadIdx.x] : 0.0f);
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) is_last = atomicAdd(counter, 1u) == gridDim.x - 1;
    __syncthreads();
    if (is_last) {
        __threadfence();
        if (threadIdx.x < NSUM) {
            double s = 0.0;
            for (unsigned b = 0; b < gridDim.x; ++b)
                s += (double)__ldcg(partials + (size_t)b * kAccPad + threadIdx.x);
            out[threadIdx.x] = s;
        }
        if (threadIdx.x == 0) *counter = 0u;  // ready for the next launch
    }
}

namespace {

template <int THREADS, int VAR>
cudaError_t launch_track_t(const StreamDesc* const* descs, const int* users, int S, int cluster,
                           const double* init, glt_result* results, cudaStream_t s, bool pdl)
{
    auto kern = track_kernel<THREADS, VAR>;
    if (cluster > 8) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(S * cluster), 1, 1);
    cfg.blockDim = dim3(THREADS, 1, 1);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)cluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 2 : 1;
    return cudaLaunchKernelEx(&cfg, kern, descs, users, init, results);
}

template <int THREADS, int VAR>
bool shape_ok_t(int cluster)
{
    auto kern = track_kernel<THREADS, VAR>;
    if (cluster > 8 &&
        cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)cluster, 1, 1);
    cfg.blockDim = dim3(THREADS, 1, 1);
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)cluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    cudaError_t e = cudaOccupancyMaxActiveClusters(&n, kern, &cfg);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return n > 0;
}

template <int VAR>
bool shape_ok_v(int cluster, int threads)
{
    switch (threads) {
    case 128: return shape_ok_t<128, VAR>(cluster);
    case 256: return shape_ok_t<256, VAR>(cluster);
    case 512: return shape_ok_t<512, VAR>(cluster);
    default: return false;
    }
}

// the p x p variant is built for 256 threads only (its unrolled patches are long)
template <>
bool shape_ok_v<2>(int cluster, int threads)
{
    return threads == 256 && shape_ok_t<256, 2>(cluster);
}

template <int VAR>
cudaError_t launch_track_v(const StreamDesc* const* descs, const int* users, int S, int cluster,
                           int threads, const double* init, glt_result* results, cudaStream_t s,
                           bool pdl)
{
    switch (threads) {
    case 128: return launch_track_t<128, VAR>(descs, users, S, cluster, init, results, s, pdl);
    case 256: return launch_track_t<256, VAR>(descs, users, S, cluster, init, results, s, pdl);
    case 512: return launch_track_t<512, VAR>(descs, users, S, cluster, init, results, s, pdl);
    default: return cudaErrorInvalidValue;
    }
}

template <>
cudaError_t launch_track_v<2>(const StreamDesc* const* descs, const int* users, int S, int cluster,
                              int threads, const double* init, glt_result* results, cudaStream_t s,
                              bool pdl)
{
    if (threads != 256) return cudaErrorInvalidValue;
    return launch_track_t<256, 2>(descs, users, S, cluster, init, results, s, pdl);
}

// the cached-Hessian variant is built for 512 threads only (a p x p point is
// split over kHcGroups threads, so it wants many threads per stream)
template <>
bool shape_ok_v<4>(int cluster, int threads)
{
    return threads == 512 && shape_ok_t<512, 4>(cluster);
}

template <>
cudaError_t launch_track_v<4>(const StreamDesc* const* descs, const int* users, int S, int cluster,
                              int threads, const double* init, glt_result* results, cudaStream_t s,
                              bool pdl)
{
    if (threads != 512) return cudaErrorInvalidValue;
    return launch_track_t<512, 4>(descs, users, S, cluster, init, results, s, pdl);
}

}  // namespace

bool track_shape_ok(int cluster, int threads, int variant)
{
    if (cluster < 1 || cluster > 16) return false;
    switch (variant) {
    case 0: return shape_ok_v<0>(cluster, threads);
    case 1: return shape_ok_v<1>(cluster, threads);
    case 2: return shape_ok_v<2>(cluster, threads);
    case 3: return shape_ok_v<3>(cluster, threads);
    case 4: return shape_ok_v<4>(cluster, threads);
    default: return false;
    }
}

cudaError_t launch_track(const StreamDesc* const* descs, const int* users, int S, int cluster,
                         int threads, int variant, const double* init, glt_result* results,
                         cudaStream_t s, bool pdl)
{
    switch (variant) {
    case 0: return launch_track_v<0>(descs, users, S, cluster, threads, init, results, s, pdl);
    case 1: return launch_track_v<1>(descs, users, S, cluster, threads, init, results, s, pdl);
    case 2: return launch_track_v<2>(descs, users, S, cluster, threads, init, results, s, pdl);
    case 3: return launch_track_v<3>(descs, users, S, cluster, threads, init, results, s, pdl);
    case 4: return launch_track_v<4>(descs, users, S, cluster, threads, init, results, s, pdl);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_linearize(const glt_tracker* t, const PassParams& P, bool want_res,
                             cudaStream_t s)
{
    constexpr int T = 128;
    const int blocks = (t->N + T - 1) / T;
    if (blocks <= 0 || blocks > t->lin_blocks) return cudaErrorInvalidValue;
    float* res = want_res ? t->lin_res : nullptr;
    const int v = track_variant(t->cfg);
    if (v == 1)
        linearize_kernel<T, 1><<<blocks, T, 0, s>>>(t->desc_dev, P, t->lin_partials,
                                                    t->lin_counter, t->lin_out, res);
    else if (v == 2)
        linearize_kernel<T, 2><<<blocks, T, 0, s>>>(t->desc_dev, P, t->lin_partials,
                                                    t->lin_counter, t->lin_out, res);
    else if (v == 3)
        linearize_kernel<T, 3><<<blocks, T, 0, s>>>(t->desc_dev, P, t->lin_partials,
                                                    t->lin_counter, t->lin_out, res);
    else if (v == 4)
        linearize_kernel<T, 4><<<blocks, T, 0, s>>>(t->desc_dev, P, t->lin_partials,
                                                    t->lin_counter, t->lin_out, res);
    else
        linearize_kernel<T, 0><<<blocks, T, 0, s>>>(t->desc_dev, P, t->lin_partials,
                                                    t->lin_counter, t->lin_out, res);
    return cudaGetLastError();
}

}  // namespace glt

namespace glt {

cudaError_t launch_pass_floor(int cluster, int threads, bool cached, int passes, long long* cycles,
                              cudaStream_t s, int drop_rank, int solve)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)cluster, 1, 1);
    cfg.blockDim = dim3((unsigned)threads, 1, 1);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)cluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
#define GLT_FLOOR(T, HC)                                                                        \
    {                                                                                           \
        auto k = pass_floor_kernel<T, HC>;                                                      \
        if (cluster > 8) {                                                                      \
            cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1); \
            if (e != cudaSuccess) return e;                                                     \
        }                                                                                       \
        return cudaLaunchKernelEx(&cfg, k, passes, drop_rank, solve, cycles);                   \
    }
    if (cached) {
        if (threads == 512) GLT_FLOOR(512, true)
    } else {
        if (threads == 128) GLT_FLOOR(128, false)
        if (threads == 256) GLT_FLOOR(256, false)
        if (threads == 512) GLT_FLOOR(512, false)
    }
#undef GLT_FLOOR
    return cudaErrorInvalidValue;
}

#ifdef GLT_CHECKED
unsigned check_flags_track()
{
    unsigned v = 0, z = 0;
    cudaMemcpyFromSymbol(&v, g_check_flags, sizeof(v));
    cudaMemcpyToSymbol(g_check_flags, &z, sizeof(z));
    return v;
}
#endif

}  // namespace glt

