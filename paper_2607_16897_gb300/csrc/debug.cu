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
