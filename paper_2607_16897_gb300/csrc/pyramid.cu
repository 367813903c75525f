// Image pyramid kernels (GLidE-SLAM Sec. IV-C "Image pyramids": blur, then
// downsample; level 0 is the full-resolution frame).
//
// Level l from level l-1: out(x, y) = (sum_{i,j=-2..2} w_i w_j in(2x+i, 2y+j) + 128) >> 8
// with w = [1 4 6 4 1], clamp-to-edge, computed exactly in integers.  Work is
// cut into 64 x 16 output tiles: a CTA stages a tile's input window (2*64+8
// columns from the 4-byte aligned column 2*x0-4, 2*16+3 rows) in shared memory
// with 4-byte loads, runs the vertical pass (two columns per 32-bit lane pair)
// and the horizontal pass, and stores 4 output bytes per thread.  The
// grid has one CTA per tile over all jobs (one job per stream, so a whole
// batch of streams builds a level in one launch).  Level 1 reads the caller's frame and
// writes the level-0 copy from its staged windows, so a frame is read from HBM
// once.
#include <algorithm>

#include "glt_internal.h"

namespace glt {

namespace {
constexpr int TW = 64;               // output tile width
constexpr int TH = 16;               // output tile height
constexpr int IW = 2 * TW + 8;       // staged input columns 2*ox0-4 .. 2*ox0+2*TW+3
constexpr int IH = 2 * TH + 3;
constexpr int PYR_THREADS = 256;
}  // namespace

__host__ __device__ int pyr_tiles_x(int dW) { return (dW + TW - 1) / TW; }
__host__ __device__ int pyr_tiles_y(int dH) { return (dH + TH - 1) / TH; }

// One output tile of a launch: the level job (for level 1 with the caller's
// frame as its source and the level-0 buffer as copy0), its corner, and
// whether the source rows are 4-byte aligned (word loads; `interior`) or need
// byte loads throughout.
struct Tile {
    PyrJob J;
    uint8_t* copy0;
    int cp, ox0, oy0;
    bool interior;
};

// Tile f of the launch: tile_map[f] = (job << 16) | tile within the job
// (row-major), or, for one job without a map, f itself.
__device__ __forceinline__ Tile tile_at(const PyrJob* __restrict__ jobs, const unsigned* __restrict__ tile_map,
                                        const uint8_t* const* frames, const uint8_t* src, int sp, int f)
{
    int z = 0, local = f;
    if (tile_map) {
        const unsigned m = tile_map[f];
        z = (int)(m >> 16);
        local = (int)(m & 0xffffu);
    }
    Tile t;
    t.J = jobs[z];
    const int tx = pyr_tiles_x(t.J.dW);
    const int ty = local / tx;
    t.ox0 = (local - ty * tx) * TW;
    t.oy0 = ty * TH;
    t.copy0 = nullptr;
    t.cp = 0;
    if (frames || src) {
        // level 1 from the caller's frame; the tiles also write the level-0 copy
        t.copy0 = const_cast<uint8_t*>(t.J.src);
        t.cp = t.J.sp;
        t.J.src = frames ? frames[z] : src;
        t.J.sp = frames ? t.J.sW : sp;
    }
    t.interior = ((t.J.sp & 3) == 0) && ((reinterpret_cast<uintptr_t>(t.J.src) & 3) == 0);
    return t;
}

constexpr int kWordsPerRow = IW / 4, kWords = IH * kWordsPerRow;
constexpr int kPer = (kWords + PYR_THREADS - 1) / PYR_THREADS;

// Source loads: a level written by the previous kernel of a programmatic
// chain is read from L2 (ld.global.cg); the caller's frame, which no kernel
// of the chain writes (level 1 is launched as an ordinary kernel), through
// the read-only path.
__device__ __forceinline__ uint32_t src_word(const Tile& t, const uint8_t* p)
{
    p = checked(p, 4, t.J.src, (size_t)t.J.sp * t.J.sH, CK_PYR_SRC);
    const unsigned int* w = reinterpret_cast<const unsigned int*>(p);
    return t.copy0 ? __ldg(w) : __ldcg(w);
}
__device__ __forceinline__ uint8_t src_byte(const Tile& t, const uint8_t* p)
{
    p = checked(p, 1, t.J.src, (size_t)t.J.sp * t.J.sH, CK_PYR_SRC);
    return t.copy0 ? __ldg(p) : __ldcg(p);
}

// The staged window's 4-byte words for a tile with aligned source rows,
// issued into registers (all of a thread's loads before any use: one memory
// round trip).  A word whose 4 source columns lie inside the row is one load;
// a word at the left or right border is assembled from its clamped columns.
__device__ __forceinline__ void issue_window(const Tile& t, uint32_t (&v)[kPer])
{
    const int ix0 = 2 * t.ox0 - 4, iy0 = 2 * t.oy0 - 2;
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
        const int i = threadIdx.x + k * PYR_THREADS;
        if (i < kWords) {
            const int r = i / kWordsPerRow, c = i % kWordsPerRow;
            const uint8_t* row = t.J.src + (size_t)min(max(iy0 + r, 0), t.J.sH - 1) * t.J.sp;
            const int x = ix0 + 4 * c;
            if (x >= 0 && x + 3 < t.J.sW) {
                v[k] = src_word(t, row + x);
            } else {
                uint32_t w = 0;
#pragma unroll
                for (int b = 0; b < 4; ++b)
                    w |= (uint32_t)src_byte(t, row + min(max(x + b, 0), t.J.sW - 1)) << (8 * b);
                v[k] = w;
            }
        }
    }
}

// Lands the window in shared memory: the issued words of an aligned tile,
// or (unaligned source rows) byte loads with clamped columns, in groups of 8
// per thread.
__device__ __forceinline__ void land_window(const Tile& t, const uint32_t (&v)[kPer], uint8_t (*in)[IW])
{
    if (t.interior) {
#pragma unroll
        for (int k = 0; k < kPer; ++k) {
            const int i = threadIdx.x + k * PYR_THREADS;
            if (i < kWords) *reinterpret_cast<uint32_t*>(&in[i / kWordsPerRow][4 * (i % kWordsPerRow)]) = v[k];
        }
        return;
    }
    const int ix0 = 2 * t.ox0 - 4, iy0 = 2 * t.oy0 - 2;
    constexpr int NB = IH * IW, PER = (NB + PYR_THREADS - 1) / PYR_THREADS, G = 8;
#pragma unroll
    for (int k0 = 0; k0 < PER; k0 += G) {
        uint8_t b[G];
#pragma unroll
        for (int k = 0; k < G; ++k) {
            const int i = threadIdx.x + (k0 + k) * PYR_THREADS;
            if (k0 + k < PER && i < NB) {
                const int r = i / IW, c = i % IW;
                const int gy = min(max(iy0 + r, 0), t.J.sH - 1);
                const int gx = min(max(ix0 + c, 0), t.J.sW - 1);
                b[k] = src_byte(t, t.J.src + (size_t)gy * t.J.sp + gx);
            }
        }
#pragma unroll
        for (int k = 0; k < G; ++k) {
            const int i = threadIdx.x + (k0 + k) * PYR_THREADS;
            if (k0 + k < PER && i < NB) in[i / IW][i % IW] = b[k];
        }
    }
}

// The tile's outputs from its staged window.  If copy0 is set (level 1 built
// straight from the source frame), the tile also writes its share of the
// level-0 copy (pitch cp): source rows [2 oy0, 2 oy0 + 2 TH) and columns
// [2 ox0, 2 ox0 + 2 TW), extended to the frame's last row / column on the last
// tile row / column, so the tiles partition level 0.
__device__ __forceinline__ void tile_outputs(const Tile& t, uint8_t (*in)[IW], uint32_t* vs)
{
    const PyrJob& J = t.J;
    const int ox0 = t.ox0, oy0 = t.oy0;
    if (t.copy0) {
        const int y0 = 2 * oy0, y1 = oy0 + TH >= J.dH ? J.sH : 2 * oy0 + 2 * TH;
        const int x0 = 2 * ox0, x1 = ox0 + TW >= J.dW ? J.sW : 2 * ox0 + 2 * TW;
        const int nw = (x1 - x0) >> 2;          // whole 4-byte words (x0 is a multiple of 128): <= 32
        const int tail = (x1 - x0) & 3;
        // staged row r + 2 is source row y0 + r, staged column 4 source column x0;
        // 32 word slots per row, then the 0-3 tail bytes of every row
        for (int i = threadIdx.x; i < (y1 - y0) * 32; i += PYR_THREADS) {
            const int r = i >> 5, k = i & 31;
            if (k < nw)
                *reinterpret_cast<uint32_t*>(checked(t.copy0 + (size_t)(y0 + r) * t.cp + x0 + 4 * k, 4, t.copy0,
                                                     (size_t)t.cp * J.sH, CK_PYR_DST)) =
                    *reinterpret_cast<const uint32_t*>(&in[r + 2][4 + 4 * k]);
        }
        if (tail) {
            for (int i = threadIdx.x; i < (y1 - y0) * 4; i += PYR_THREADS) {
                const int r = i >> 2, k = i & 3;
                if (k < tail)
                    *checked(t.copy0 + (size_t)(y0 + r) * t.cp + x0 + 4 * nw + k, 1, t.copy0, (size_t)t.cp * J.sH,
                             CK_PYR_DST) = in[r + 2][4 + 4 * nw + k];
            }
        }
    }
    // vertical 5-tap pass, one 4-byte word (4 staged columns) per item: both
    // 16-bit lanes of a u32 carry one column's sum (at most 16 * 255), so one
    // 32-bit multiply-add serves two columns; the sums go to two planes by
    // column parity, ve[y][w] = (V[4w], V[4w+2]) and vo[y][w] = (V[4w+1], V[4w+3])
    uint32_t* ve = vs;
    uint32_t* vo = vs + TH * (IW / 4);
    for (int i = threadIdx.x; i < TH * (IW / 4); i += PYR_THREADS) {
        const int y = i / (IW / 4), w = i - y * (IW / 4);
        const uint32_t* col = reinterpret_cast<const uint32_t*>(&in[2 * y][0]) + w;
        uint32_t lo = 0, hi = 0;
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            const uint32_t a = col[k * (IW / 4)];
            const uint32_t wk = k == 2 ? 6u : (k == 1 || k == 3) ? 4u : 1u;
            lo += wk * (a & 0x00ff00ffu);
            hi += wk * ((a >> 8) & 0x00ff00ffu);
        }
        ve[i] = lo;
        vo[i] = hi;
    }
    __syncthreads();
    // horizontal pass, 4 output pixels per item, two per 32-bit lane pair:
    // output x (tile-local) takes staged columns 2x+2 .. 2x+6, i.e.
    // Ve[x+1] + 4 Vo[x+1] + 6 Ve[x+2] + 4 Vo[x+2] + Ve[x+3], where Ve[e] = V[2e]
    // and Vo[e] = V[2e+1]; a lane sum is at most 16 * 16 * 255 + 128 < 2^16
    for (int i = threadIdx.x; i < TH * (TW / 4); i += PYR_THREADS) {
        const int y = i / (TW / 4), x4 = (i % (TW / 4)) * 4;
        const int gy = oy0 + y;
        if (gy >= J.dH) continue;
        const uint32_t* e = ve + y * (IW / 4) + (x4 >> 1);
        const uint32_t* o = vo + y * (IW / 4) + (x4 >> 1);
        const uint32_t e0 = e[0], e1 = e[1], e2 = e[2], e3 = e[3];
        const uint32_t o0 = o[0], o1 = o[1], o2 = o[2];
        // pair (x4, x4+1): A = Ve(x+1, x+2), B = Ve(x+2, x+3), C = Ve(x+3, x+4),
        // D = Vo(x+1, x+2), E = Vo(x+2, x+3) with x = x4; pair (x4+2, x4+3) one word on
        const uint32_t s01 = __byte_perm(e0, e1, 0x5432) + 6u * e1 + __byte_perm(e1, e2, 0x5432) +
                             4u * (__byte_perm(o0, o1, 0x5432) + o1) + 0x00800080u;
        const uint32_t s23 = __byte_perm(e1, e2, 0x5432) + 6u * e2 + __byte_perm(e2, e3, 0x5432) +
                             4u * (__byte_perm(o1, o2, 0x5432) + o2) + 0x00800080u;
        const uint32_t packed = __byte_perm(s01 >> 8, s23 >> 8, 0x6420);
        const int gx = ox0 + x4;
        uint8_t* dst = J.dst + (size_t)gy * J.dp + gx;
        if (gx < J.dW) dst = checked(dst, (size_t)min(4, J.dW - gx), J.dst, (size_t)J.dp * J.dH, CK_PYR_DST);
        if (gx + 4 <= J.dW && ((reinterpret_cast<uintptr_t>(dst) & 3) == 0)) {
            *reinterpret_cast<uint32_t*>(dst) = packed;
        } else {
            for (int k = 0; k < 4 && gx + k < J.dW; ++k) dst[k] = (uint8_t)(packed >> (8 * k));
        }
    }
}

// One level of S streams, one CTA per output tile over all jobs (no idle
// CTAs for the smaller streams of a batch).  For level 1 the source can be
// the caller's frame instead of the level-0 buffer: `frames` (a device table
// of S contiguous frames, pitch = width) or `src` / `sp` (one stream); the
// tiles then also write the level-0 copy into the job's source buffer.
__global__ void __launch_bounds__(PYR_THREADS, 8) pyr_down_kernel(const PyrJob* __restrict__ jobs,
                                                                  const unsigned* __restrict__ tile_map,
                                                                  const uint8_t* const* frames,
                                                                  const uint8_t* src, int sp)
{
    __shared__ __align__(16) uint8_t in[IH][IW];
    __shared__ __align__(16) uint32_t vs[2 * TH * (IW / 4)];   // the two parity planes
    // the next level's kernel (or the track kernel) may start its setup now;
    // the tile's description (tables written before the chain started) is
    // read at once, this level's source only once the previous kernel is done
    griddep_launch_dependents();
    const Tile t = tile_at(jobs, tile_map, frames, src, sp, (int)blockIdx.x);
    griddep_wait();
    uint32_t v[kPer];
    if (t.interior) issue_window(t, v);
    land_window(t, v, in);
    __syncthreads();
    tile_outputs(t, in, vs);
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

cudaError_t launch_pyr_down(const PyrJob* jobs_dev, const unsigned* tile_map_dev, int total, cudaStream_t s,
                            const uint8_t* const* frames, const uint8_t* src, int sp, bool pdl)
{
    if (total <= 0) return cudaSuccess;
    return launch_ex(pyr_down_kernel, dim3((unsigned)total), PYR_THREADS, s, pdl, jobs_dev, tile_map_dev,
                     frames, src, sp);
}

// Batched level-0 copy: frame s (contiguous, pitch W) -> pitched level 0.
__global__ void copy_frames_kernel(const uint8_t* const* __restrict__ frames,
                                   const CopyJob* __restrict__ jobs)
{
    griddep_launch_dependents();
    const CopyJob J = jobs[blockIdx.y];   // tables written before the chain started
    const uint8_t* src = frames[blockIdx.y];
    griddep_wait();
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
    const PackJob J = jobs[blockIdx.y];   // written before the chain started
    griddep_wait();
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

#ifdef GLT_CHECKED
unsigned check_flags_pyramid()
{
    unsigned v = 0, z = 0;
    cudaMemcpyFromSymbol(&v, g_check_flags, sizeof(v));
    cudaMemcpyToSymbol(g_check_flags, &z, sizeof(z));
    return v;
}
#endif

}  // namespace glt

