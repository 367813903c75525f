// Test entry points for device building blocks that have no host-visible
// effect of their own.
#include "glt_internal.h"

namespace glt {
namespace {

__global__ void rcp_kernel(const double* __restrict__ d, double* __restrict__ r, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) r[i] = rcp_d(d[i]);
}

}  // namespace
}  // namespace glt

using namespace glt;

extern "C" int glt_debug_rcp(const double* d_dev, double* r_dev, int n, void* stream)
{
    if (n < 0 || (n > 0 && (!d_dev || !r_dev))) return invalid_arg_msg("glt_debug_rcp: bad argument");
    if (n == 0) return GLT_OK;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    rcp_kernel<<<(n + 255) / 256, 256, 0, s>>>(d_dev, r_dev, n);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? GLT_OK : cuda_fail(e, "glt_debug_rcp kernel");
}

extern "C" int glt_debug_pass_floor(int cluster, int threads, int cached, int solve, int passes,
                                    float* us_per_pass, void* stream)
{
    if (!us_per_pass || passes < 1 || passes > 100000 || cluster < 1 || cluster > 16 ||
        (solve != GLT_SOLVE_FP64 && solve != GLT_SOLVE_FP32))
        return invalid_arg_msg("glt_debug_pass_floor: bad argument");
    if (!track_shape_ok(cluster, threads, cached ? 4 : 0))
        return invalid_arg_msg("glt_debug_pass_floor: shape cannot launch");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    long long* cyc = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&cyc), sizeof(long long));
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    // one launch to warm up, then the timed one
    if (e == cudaSuccess) e = launch_pass_floor(cluster, threads, cached != 0, passes, cyc, s, -1, solve);
    if (e == cudaSuccess) e = cudaEventRecord(e0, s);
    if (e == cudaSuccess) e = launch_pass_floor(cluster, threads, cached != 0, passes, cyc, s, -1, solve);
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(cyc);
    if (e != cudaSuccess) return cuda_fail(e, "glt_debug_pass_floor");
    *us_per_pass = 1000.0f * ms / (float)passes;
    return GLT_OK;
}

extern "C" int glt_debug_exchange_timeout(int cluster, int threads, int* status, void* stream)
{
    if (!status || cluster < 2 || cluster > 16)
        return invalid_arg_msg("glt_debug_exchange_timeout: bad argument");
    if (!track_shape_ok(cluster, threads, 0))
        return invalid_arg_msg("glt_debug_exchange_timeout: shape cannot launch");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    long long* cyc = nullptr;
    long long host = 0;
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&cyc), sizeof(long long));
    if (e == cudaSuccess) e = launch_pass_floor(cluster, threads, false, 1, cyc, s, 0);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&host, cyc, sizeof(long long), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(cyc);
    if (e != cudaSuccess) return cuda_fail(e, "glt_debug_exchange_timeout");
    *status = host < 0 ? GLT_TRACK_TIMEOUT : 0;
    return GLT_OK;
}

#ifdef GLT_CHECKED
namespace glt {
namespace {
// Positive control of the bounds-checked build: one index inside a buffer of
// n floats and one 5 elements past its end go through checked(); the second
// is redirected to the buffer's first element (no access outside it) and
// sets the CK_TABLE flag.  Compiled only into the checked build.
__global__ void checked_probe_kernel(const float* __restrict__ buf, int n, float* __restrict__ out)
{
    out[0] = *checked(buf + n / 2, 1, buf, (size_t)n, CK_TABLE);
    out[1] = *checked(buf + n + 5, 1, buf, (size_t)n, CK_TABLE);
}
}  // namespace
unsigned check_flags_debug()
{
    unsigned v = 0, z = 0;
    cudaMemcpyFromSymbol(&v, g_check_flags, sizeof(v));
    cudaMemcpyToSymbol(g_check_flags, &z, sizeof(z));
    return v;
}
}  // namespace glt
#endif

extern "C" int glt_debug_checked_probe(unsigned* flags)
{
    if (!flags) return invalid_arg_msg("glt_debug_checked_probe: flags is NULL");
    *flags = 0;
#ifdef GLT_CHECKED
    float* buf = nullptr;
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&buf), 66 * sizeof(float));
    if (e == cudaSuccess) e = cudaMemset(buf, 0, 66 * sizeof(float));
    if (e == cudaSuccess) {
        checked_probe_kernel<<<1, 1>>>(buf, 64, buf + 64);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e == cudaSuccess) *flags = check_flags_debug();
    cudaFree(buf);
    return e == cudaSuccess ? GLT_OK : cuda_fail(e, "glt_debug_checked_probe");
#else
    set_error("glt_debug_checked_probe: not a bounds-checked build (libglt_checked.so)");
    return GLT_ERR_UNSUPPORTED;
#endif
}

extern "C" int glt_debug_checked_flags(unsigned* flags)
{
    if (!flags) return invalid_arg_msg("glt_debug_checked_flags: flags is NULL");
#ifdef GLT_CHECKED
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(e, "glt_debug_checked_flags");
    *flags = check_flags_track() | check_flags_pyramid() | check_flags_points();
    return GLT_OK;
#else
    *flags = 0;
    set_error("glt_debug_checked_flags: not a bounds-checked build (libglt_checked.so)");
    return GLT_ERR_UNSUPPORTED;
#endif
}
