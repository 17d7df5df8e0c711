// Diagnostics entry points (not part of the method): expose device helpers
// so the tests can compare them with CUDA's own routines.
#include "axi_internal.h"
#include "trig.cuh"

#include <mutex>
#include <vector>

namespace axi {
namespace {

__global__ void diag_sincos_kernel(const double *__restrict__ x, int n, double *__restrict__ s,
                                   double *__restrict__ c) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    trig::sincos_ring(x[i], &s[i], &c[i]);
}

__global__ void diag_sincos_tab_kernel(const double *__restrict__ x, int n, const double2 *__restrict__ gtab,
                                       double *__restrict__ s, double *__restrict__ c) {
  __shared__ double2 tab[trig::kRingTab];
  for (int i = threadIdx.x; i < trig::kRingTab; i += blockDim.x) tab[i] = gtab[i];
  __syncthreads();
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    trig::sincos_ring_tab(x[i], tab, &s[i], &c[i]);
}

// the table variant's table, uploaded once per device on first use
__device__ double2 g_diag_ring_tab[trig::kRingTab];

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

extern "C" axi_status axi_diag_sincos_table(const double *d_x, int32_t n, double *d_sin, double *d_cos,
                                            void *stream) {
  if (n < 0 || (n > 0 && (!d_x || !d_sin || !d_cos))) return AXI_ERR_ARG;
  if (n == 0) return AXI_OK;
  static std::mutex mu;
  static bool loaded[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return AXI_ERR_CUDA;
  {
    std::lock_guard<std::mutex> lock(mu);
    if (!loaded[dev]) {
      std::vector<double2> tab(axi::trig::kRingTab);
      axi::trig::ring_table_host(tab.data());
      if (cudaMemcpyToSymbol(axi::g_diag_ring_tab, tab.data(), sizeof(double2) * tab.size()) != cudaSuccess)
        return AXI_ERR_CUDA;
      loaded[dev] = true;
    }
  }
  double2 *gtab = nullptr;
  if (cudaGetSymbolAddress(reinterpret_cast<void **>(&gtab), axi::g_diag_ring_tab) != cudaSuccess)
    return AXI_ERR_CUDA;
  int blocks = (n + 255) / 256;
  if (blocks > 152 * 8) blocks = 152 * 8;
  axi::diag_sincos_tab_kernel<<<blocks, 256, 0, static_cast<cudaStream_t>(stream)>>>(d_x, n, gtab, d_sin,
                                                                                     d_cos);
  return cudaGetLastError() == cudaSuccess ? AXI_OK : AXI_ERR_CUDA;
}
