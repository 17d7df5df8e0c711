// Diagnostics entry points (not part of the method): expose device helpers
// so the tests can compare them with CUDA's own routines.
#include "axi_internal.h"
#include "trig.cuh"

namespace axi {
namespace {

__global__ void diag_sincos_kernel(const double *__restrict__ x, int n, double *__restrict__ s,
                                   double *__restrict__ c) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    trig::sincos_ring(x[i], &s[i], &c[i]);
}

}  // namespace
}  // namespace axi

extern "C" axi_status axi_diag_sincos(const double *d_x, int32_t n, double *d_sin, double *d_cos,
                                      void *stream) {
  if (n < 0 || (n > 0 && (!d_x || !d_sin || !d_cos))) return AXI_ERR_ARG;
  if (n == 0) return AXI_OK;
  int blocks = (n + 255) / 256;
  if (blocks > 152 * 8) blocks = 152 * 8;
  axi::diag_sincos_kernel<<<blocks, 256, 0, static_cast<cudaStream_t>(stream)>>>(d_x, n, d_sin,
                                                                                 d_cos);
  return cudaGetLastError() == cudaSuccess ? AXI_OK : AXI_ERR_CUDA;
}
