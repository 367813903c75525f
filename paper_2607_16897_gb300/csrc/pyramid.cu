// Image pyramid kernels (GLidE-SLAM Sec. IV-C "Image pyramids": blur, then
// downsample; level 0 is the full-resolution frame).
//
// Level l from level l-1: out(x, y) = (sum_{i,j=-2..2} w_i w_j in(2x+i, 2y+j) + 128) >> 8
// with w = [1 4 6 4 1], clamp-to-edge, computed exactly in integers.  One CTA
// produces a 64 x 16 output tile: it stages the input window (2*64+8 columns
// from the 4-byte aligned column 2*x0-4, 2*16+3 rows) in shared memory with
// 4-byte loads, runs the vertical pass into a 16-bit buffer and the horizontal
// pass, and stores 4 output bytes per thread.
// Jobs (one per stream) index blockIdx.z, so a whole batch of streams builds a
// level in one launch.  Level 1 reads the caller's frame and writes the
// level-0 copy from its staged windows, so a frame is read from HBM once.
#include "glt_internal.h"

namespace glt {

namespace {
constexpr int TW = 64;               // output tile width
constexpr int TH = 16;               // output tile height
constexpr int IW = 2 * TW + 8;       // staged input columns 2*ox0-4 .. 2*ox0+2*TW+3
constexpr int IH = 2 * TH + 3;
constexpr int PYR_THREADS = 256;
}  // namespace

int pyr_tiles_x(int dW) { return (dW + TW - 1) / TW; }
int pyr_tiles_y(int dH) { return (dH + TH - 1) / TH; }

// One 64 x 16 output tile of J's level.  COHERENT selects L2 loads
// (ld.global.cg) for a source level written earlier in the same launch; a
// source that is read-only for the launch goes through the read-only cache.
template <bool COHERENT>
__device__ __forceinline__ uint32_t ld_word(const uint8_t* p)
{
    return COHERENT ? __ldcg(reinterpret_cast<const unsigned int*>(p))
                    : __ldg(reinterpret_cast<const unsigned int*>(p));
}
template <bool COHERENT>
__device__ __forceinline__ uint8_t ld_byte(const uint8_t* p)
{
    return COHERENT ? __ldcg(p) : __ldg(p);
}

// If copy0 is set (level 1 built straight from the source frame), the tile
// also writes its share of the level-0 copy (pitch cp) from the staged window:
// source rows [2 oy0, 2 oy0 + 2 TH) and columns [2 ox0, 2 ox0 + 2 TW), extended
// to the frame's last row / column on the last tile row / column, so the
// tiles partition level 0.
template <bool COHERENT>
__device__ __forceinline__ void pyr_tile(const PyrJob& J, int ox0, int oy0, uint8_t (*in)[IW],
                                         uint16_t (*vs)[IW], uint8_t* copy0 = nullptr, int cp = 0)
{
    const int ix0 = 2 * ox0 - 4, iy0 = 2 * oy0 - 2;
    // stage the input window (clamp-to-edge); 4-byte loads when the whole
    // window row lies inside the image and is aligned, bytes otherwise
    const bool interior_x = ix0 >= 0 && ix0 + IW <= J.sW && ((J.sp & 3) == 0) &&
                            ((reinterpret_cast<uintptr_t>(J.src) & 3) == 0);
    // all of a thread's loads are issued before any store, so the window
    // costs about one memory round trip instead of one per loop iteration
    if (interior_x) {
        constexpr int WPR = IW / 4, NW = IH * WPR, PER = (NW + PYR_THREADS - 1) / PYR_THREADS;
        uint32_t v[PER];
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            const int i = threadIdx.x + k * PYR_THREADS;
            if (i < NW) {
                const int r = i / WPR, c = i % WPR;
                const int gy = min(max(iy0 + r, 0), J.sH - 1);
                v[k] = ld_word<COHERENT>(J.src + (size_t)gy * J.sp + ix0 + 4 * c);
            }
        }
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            const int i = threadIdx.x + k * PYR_THREADS;
            if (i < NW) *reinterpret_cast<uint32_t*>(&in[i / WPR][4 * (i % WPR)]) = v[k];
        }
    } else {
        constexpr int NB = IH * IW, PER = (NB + PYR_THREADS - 1) / PYR_THREADS;
        uint8_t v[PER];
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            const int i = threadIdx.x + k * PYR_THREADS;
            if (i < NB) {
                const int r = i / IW, c = i % IW;
                const int gy = min(max(iy0 + r, 0), J.sH - 1);
                const int gx = min(max(ix0 + c, 0), J.sW - 1);
                v[k] = ld_byte<COHERENT>(J.src + (size_t)gy * J.sp + gx);
            }
        }
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            const int i = threadIdx.x + k * PYR_THREADS;
            if (i < NB) in[i / IW][i % IW] = v[k];
        }
    }
    __syncthreads();
    if (copy0) {
        const int y0 = 2 * oy0, y1 = oy0 + TH >= J.dH ? J.sH : 2 * oy0 + 2 * TH;
        const int x0 = 2 * ox0, x1 = ox0 + TW >= J.dW ? J.sW : 2 * ox0 + 2 * TW;
        const int nw = (x1 - x0) >> 2;          // whole 4-byte words (x0 is a multiple of 128)
        const int tail = (x1 - x0) & 3;
        const int per_row = nw + tail;
        for (int i = threadIdx.x; i < (y1 - y0) * per_row; i += PYR_THREADS) {
            const int r = i / per_row, k = i % per_row;
            uint8_t* drow = copy0 + (size_t)(y0 + r) * cp + x0;
            const uint8_t* srow = &in[r + 2][4];  // staged column 4 is source column x0
            if (k < nw)
                reinterpret_cast<uint32_t*>(drow)[k] = *reinterpret_cast<const uint32_t*>(srow + 4 * k);
            else
                drow[4 * nw + (k - nw)] = srow[4 * nw + (k - nw)];
        }
    }
    // vertical 5-tap pass on every staged column
    for (int i = threadIdx.x; i < TH * IW; i += PYR_THREADS) {
        const int y = i / IW, c = i % IW;
        const int r = 2 * y;
        vs[y][c] = (uint16_t)(in[r][c] + 4 * in[r + 1][c] + 6 * in[r + 2][c] + 4 * in[r + 3][c] + in[r + 4][c]);
    }
    __syncthreads();
    // horizontal pass: each thread produces 4 consecutive output pixels
    for (int i = threadIdx.x; i < TH * (TW / 4); i += PYR_THREADS) {
        const int y = i / (TW / 4), x4 = (i % (TW / 4)) * 4;
        const int gy = oy0 + y;
        if (gy >= J.dH) continue;
        uint32_t packed = 0;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int c = 2 * (x4 + k) + 2;   // staged column of input x = 2*(ox0+x4+k) - 2
            const uint32_t s = vs[y][c] + 4u * vs[y][c + 1] + 6u * vs[y][c + 2] + 4u * vs[y][c + 3] + vs[y][c + 4];
            packed |= ((s + 128u) >> 8) << (8 * k);
        }
        const int gx = ox0 + x4;
        uint8_t* dst = J.dst + (size_t)gy * J.dp + gx;
        if (gx + 4 <= J.dW && ((reinterpret_cast<uintptr_t>(dst) & 3) == 0)) {
            *reinterpret_cast<uint32_t*>(dst) = packed;
        } else {
            for (int k = 0; k < 4 && gx + k < J.dW; ++k) dst[k] = (uint8_t)(packed >> (8 * k));
        }
    }
    __syncthreads();   // the staging buffers are reused by the next tile
}

// One level of S streams (blockIdx.z = stream).  For level 1 the source can
// be the caller's frame instead of the level-0 buffer: `frames` (a device table
// of S contiguous frames, pitch = width) or `src` / `sp` (one stream); the
// tiles then also write the level-0 copy into the job's source buffer.
__global__ void __launch_bounds__(PYR_THREADS) pyr_down_kernel(const PyrJob* __restrict__ jobs,
                                                               const uint8_t* const* __restrict__ frames,
                                                               const uint8_t* __restrict__ src, int sp)
{
    __shared__ __align__(16) uint8_t in[IH][IW];
    __shared__ __align__(16) uint16_t vs[TH][IW];
    // the next level's kernel (or the track kernel) may start its setup now;
    // this level's source is read only once the previous kernel is done
    griddep_launch_dependents();
    PyrJob J = jobs[blockIdx.z];
    griddep_wait();
    const int ox0 = blockIdx.x * TW, oy0 = blockIdx.y * TH;
    if (ox0 >= J.dW || oy0 >= J.dH) return;
    if (frames || src) {
        uint8_t* level0 = const_cast<uint8_t*>(J.src);
        const int p0 = J.sp;
        J.src = frames ? frames[blockIdx.z] : src;
        J.sp = frames ? J.sW : sp;
        pyr_tile<false>(J, ox0, oy0, in, vs, level0, p0);
    } else {
        // a level written by the previous kernel: L2 loads, not the read-only path
        pyr_tile<true>(J, ox0, oy0, in, vs);
    }
}

namespace {
// ordinary or programmatic-dependent launch of a pyramid-family kernel
template <typename... KArgs, typename... Args>
cudaError_t launch_ex(void (*kern)(KArgs...), dim3 grid, int threads, cudaStream_t s, bool pdl,
                      Args... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = dim3((unsigned)threads, 1, 1);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kern, args...);
}
}  // namespace

cudaError_t launch_pyr_down(const PyrJob* jobs_dev, int njobs, int tiles_x, int tiles_y,
                            cudaStream_t s, const uint8_t* const* frames, const uint8_t* src, int sp,
                            bool pdl)
{
    dim3 grid((unsigned)tiles_x, (unsigned)tiles_y, (unsigned)njobs);
    return launch_ex(pyr_down_kernel, grid, PYR_THREADS, s, pdl, jobs_dev, frames, src, sp);
}

// Batched level-0 copy: frame s (contiguous, pitch W) -> pitched level 0.
__global__ void copy_frames_kernel(const uint8_t* const* __restrict__ frames,
                                   const CopyJob* __restrict__ jobs)
{
    griddep_launch_dependents();
    griddep_wait();
    const CopyJob J = jobs[blockIdx.y];
    const uint8_t* src = frames[blockIdx.y];
    const int n = J.W * J.H;
    const bool vec = ((J.W & 3) == 0) && ((reinterpret_cast<uintptr_t>(src) & 3) == 0);
    if (vec) {
        const int wpr = J.W / 4;
        for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < wpr * J.H; i += gridDim.x * blockDim.x) {
            const int y = i / wpr, c = i % wpr;
            const uint32_t w = __ldg(reinterpret_cast<const uint32_t*>(src + (size_t)y * J.W) + c);
            *reinterpret_cast<uint32_t*>(J.dst + (size_t)y * J.dp + 4 * c) = w;
        }
    } else {
        for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
            const int y = i / J.W, x = i % J.W;
            J.dst[(size_t)y * J.dp + x] = __ldg(src + i);
        }
    }
}

cudaError_t launch_copy_frames(const uint8_t* const* frames, const CopyJob* jobs, int njobs,
                               int max_bytes, cudaStream_t s, bool pdl)
{
    const int threads = 256;
    int bx = (max_bytes / 4 + threads - 1) / threads;
    if (bx > 256) bx = 256;
    if (bx < 1) bx = 1;
    return launch_ex(copy_frames_kernel, dim3((unsigned)bx, (unsigned)njobs), threads, s, pdl, frames, jobs);
}

// Mixed precision storage: FP16 (I, gx, gy, 0) per pixel, central differences
// halved (exact in FP16: multiples of 1/2 with |g| <= 127.5), 0 on the border.
__global__ void pack_kernel(const PackJob* __restrict__ jobs)
{
    griddep_launch_dependents();
    griddep_wait();
    const PackJob J = jobs[blockIdx.y];
    const int n = J.W * J.H;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int y = i / J.W, x = i % J.W;
        const uint8_t* row = J.src + (size_t)y * J.sp;
        const float I = row[x];
        float gx = 0.0f, gy = 0.0f;
        if (x > 0 && x < J.W - 1) gx = 0.5f * ((float)row[x + 1] - (float)row[x - 1]);
        if (y > 0 && y < J.H - 1) gy = 0.5f * ((float)row[x + J.sp] - (float)row[x - J.sp]);
        const __half2 ig = __floats2half2_rn(I, gx);
        const __half2 yz = __floats2half2_rn(gy, 0.0f);
        uint2 v;
        v.x = *reinterpret_cast<const uint32_t*>(&ig);
        v.y = *reinterpret_cast<const uint32_t*>(&yz);
        J.dst[i] = v;
    }
}

cudaError_t launch_pack(const PackJob* jobs, int njobs, int max_pixels, cudaStream_t s, bool pdl)
{
    const int threads = 256;
    int bx = (max_pixels + threads - 1) / threads;
    if (bx > 512) bx = 512;
    if (bx < 1) bx = 1;
    return launch_ex(pack_kernel, dim3((unsigned)bx, (unsigned)njobs), threads, s, pdl, jobs);
}

}  // namespace glt
