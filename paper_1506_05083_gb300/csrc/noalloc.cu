// axi_apply_operator_noalloc: the apply with its scratch in a static device
// array instead of a caller-provided buffer.
//
// Some callers cannot allocate device memory when they need to apply the
// operator: a host application that owns the GPU's whole memory budget and
// hands plug-ins only their input and output buffers, or a latency-critical
// loop in which a cudaMalloc (which may synchronise the device) is not
// allowed. This entry point lets them apply a built operator with no
// allocation at all: the RHS blocks live in g_apply_scratch below, a
// file-scope device array that every GPU loading this library holds until
// the process exits.
#include <mutex>

#include "axi_internal.h"

namespace {

constexpr size_t kNoAllocScratchBytes = size_t(32) << 20;  // 32 MiB
static __device__ __align__(256) unsigned char g_apply_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_scratch_addr[kMaxDevices] = {};

// Device address of g_apply_scratch on device `dev` (the current device). In
// host code the symbol is only a host-side stand-in, so the address is
// looked up once per device with that device current and cached; a device
// reset (cudaDeviceReset) would make the cached address stale, so calls
// after a reset in the same process are not supported.
axi_status scratch_address(int dev, void **out) {
  if (dev < 0 || dev >= kMaxDevices) return AXI_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_addr[dev]) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_apply_scratch) != cudaSuccess || !p) return AXI_ERR_CUDA;
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return AXI_OK;
}

}  // namespace

extern "C" size_t axi_noalloc_scratch_bytes(void) { return kNoAllocScratchBytes; }

extern "C" axi_status axi_apply_operator_noalloc(const axi_operator *op, int32_t obs, int32_t W,
                                                 const axi_c128 *d_f, axi_c128 *d_coef,
                                                 axi_c128 *d_sigma, void *stream) {
  if (!op || !d_f || !d_coef || W < 1) return AXI_ERR_ARG;
  // The library, not the caller, picks the scratch: it must be the array of
  // the device that holds the operator, and the stream must belong to it.
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return AXI_ERR_CUDA;
  if (dev != axi::operator_device(op)) return AXI_ERR_ARG;
  if (stream) {
    int sdev = -1;
    if (cudaStreamGetDevice(static_cast<cudaStream_t>(stream), &sdev) != cudaSuccess)
      return AXI_ERR_ARG;
    if (sdev != dev) return AXI_ERR_ARG;
  }
  size_t need = 0;
  axi_status s = axi_apply_workspace_bytes(op, obs, W, &need);
  if (s != AXI_OK) return s;
  if (need > kNoAllocScratchBytes) return AXI_ERR_WORKSPACE;  // too large for the static scratch
  void *scratch = nullptr;
  s = scratch_address(dev, &scratch);
  if (s != AXI_OK) return s;
  // Every element of the scratch that the apply reads is written by it first
  // (the transform to modes fills all D x 2W RHS columns), so no clearing is
  // needed between calls.
  return axi_apply_operator(op, obs, W, d_f, d_coef, d_sigma, scratch, kNoAllocScratchBytes, stream);
}
