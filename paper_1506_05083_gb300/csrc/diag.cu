// Diagnostics entry points (not part of the method): expose device helpers
// so the tests can compare them with CUDA's own routines.
#include "axi_internal.h"
#include "tcgen05.cuh"
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

// the fixed-point variant's table (ring_table_q62.inc)
__device__ const long long g_diag_ring_q62[trig::kRingTab][2] = {
#include "ring_table_q62.inc"
};

__global__ void diag_sincos_q_kernel(const double *__restrict__ x, int n, double *__restrict__ s,
                                     double *__restrict__ c) {
  __shared__ longlong2 tab[trig::kRingTab];
  for (int i = threadIdx.x; i < trig::kRingTab; i += blockDim.x)
    tab[i] = make_longlong2(g_diag_ring_q62[i][0], g_diag_ring_q62[i][1]);
  __syncthreads();
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    trig::sincos_ring_q(x[i], tab, &s[i], &c[i]);
}

// The failure path of the tcgen05 kernels, without their work: one CTA takes
// tensor memory, waits with the kernels' bounded wait (tc::mbar_wait) on an
// mbarrier that nothing completes, and when the limit runs out latches the
// timeout bit of the status word, releases its tensor memory and returns.
__global__ void __launch_bounds__(128)
diag_wait_timeout_kernel(long long max_cycles, int *__restrict__ status) {
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t tmem_base;
  const int warp = threadIdx.x >> 5;
  if (warp == 0) tc::tmem_alloc(&tmem_base, 32);
  if (threadIdx.x == 0) tc::mbar_init(&bar, 1);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (threadIdx.x == 0 && !tc::mbar_wait(&bar, 0, max_cycles)) atomicOr(status, kStatTimeout);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (warp == 0) {
    __syncwarp();
    tc::tmem_dealloc(tmem_base, 32);
  }
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

extern "C" axi_status axi_diag_sincos_fixed(const double *d_x, int32_t n, double *d_sin, double *d_cos,
                                            void *stream) {
  if (n < 0 || (n > 0 && (!d_x || !d_sin || !d_cos))) return AXI_ERR_ARG;
  if (n == 0) return AXI_OK;
  int blocks = (n + 255) / 256;
  if (blocks > 152 * 8) blocks = 152 * 8;
  axi::diag_sincos_q_kernel<<<blocks, 256, 0, static_cast<cudaStream_t>(stream)>>>(d_x, n, d_sin, d_cos);
  return cudaGetLastError() == cudaSuccess ? AXI_OK : AXI_ERR_CUDA;
}

extern "C" axi_status axi_diag_wait_timeout(const axi_operator *op, int64_t max_cycles, void *stream) {
  if (!op || max_cycles < 1 || max_cycles > ((int64_t)1 << 34)) return AXI_ERR_ARG;
  axi::diag_wait_timeout_kernel<<<1, 128, 0, static_cast<cudaStream_t>(stream)>>>(
      (long long)max_cycles, axi::operator_status_word(op));
  return cudaGetLastError() == cudaSuccess ? AXI_OK : AXI_ERR_CUDA;
}
