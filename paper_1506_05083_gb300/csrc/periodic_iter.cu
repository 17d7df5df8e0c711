// The two steps of one application of the preconditioned periodic operator
// (Sec. 4.2, eq. iter) that no other kernel covers:
//
//   matvec_kernel      C eta: the dense C block of the full system (Sec. 4.1,
//                      eq. full; column-major, 8 M1^2 rows x P N columns)
//                      times W coefficient vectors, split over column slices
//                      with a second, fixed-order pass over the slices
//                      (deterministic: no atomics);
//   iter_combine_kernel  y = g + A_else A_0^+ g - B xi: the spherical-wave
//                      part d of xi through B~ (block diagonal in the mode,
//                      mode -n = (-1)^n mode n) to the modal data of the P
//                      modes -P/2 < n <= P/2, carried back to the P ring
//                      nodes by f_l = sum_n fhat_n e^{2 pi i n l / P}.
//
// The other steps are the operator's apply (A_0^+), the near-image sum
// (A_else) and the SVD solve (Q^+), each with its own entry point.
#include <algorithm>

#include "axi_internal.h"

namespace {

constexpr int kMvRows = 256;    // rows per CTA (one per thread)
constexpr int kMvChunk = 64;    // columns of X staged in shared memory per pass
constexpr int kMvMaxRhs = 16;

__device__ __forceinline__ double2 cmul_acc(double2 acc, double2 a, double2 x) {
  acc.x = fma(a.x, x.x, fma(-a.y, x.y, acc.x));
  acc.y = fma(a.x, x.y, fma(a.y, x.x, acc.y));
  return acc;
}

// Y[w][r] (or the slice partial work[s][w][r]) = sum over the slice's columns
// c of A[c * lda + r] X[w * ldx + c]. NR >= nrhs; columns of X beyond nrhs
// are staged as zeros and never written.
template <int NR>
__global__ void __launch_bounds__(kMvRows) matvec_kernel(const double2 *__restrict__ A, int64_t lda,
                                                         int64_t rows, int64_t cols,
                                                         const double2 *__restrict__ X, int64_t ldx,
                                                         int nrhs, int64_t cols_per_slice,
                                                         double2 *__restrict__ out, int64_t ldo,
                                                         int64_t slice_stride) {
  __shared__ double2 xs[kMvChunk][NR];
  const int64_t r = (int64_t)blockIdx.x * kMvRows + threadIdx.x;
  const int64_t c_begin = (int64_t)blockIdx.y * cols_per_slice;
  const int64_t c_end = min(cols, c_begin + cols_per_slice);
  double2 acc[NR];
#pragma unroll
  for (int w = 0; w < NR; ++w) acc[w] = make_double2(0.0, 0.0);
  for (int64_t c0 = c_begin; c0 < c_end; c0 += kMvChunk) {
    const int nc = c_end - c0 < kMvChunk ? (int)(c_end - c0) : kMvChunk;
    __syncthreads();
    for (int i = threadIdx.x; i < kMvChunk * NR; i += kMvRows) {
      const int cc = i / NR, w = i % NR;
      xs[cc][w] = (cc < nc && w < nrhs) ? X[(int64_t)w * ldx + c0 + cc] : make_double2(0.0, 0.0);
    }
    __syncthreads();
    if (r < rows) {
      const double2 *a = A + c0 * lda + r;
      int cc = 0;
      for (; cc + 2 <= nc; cc += 2) {
        const double2 a0 = a[(int64_t)cc * lda], a1 = a[(int64_t)(cc + 1) * lda];
#pragma unroll
        for (int w = 0; w < NR; ++w) acc[w] = cmul_acc(cmul_acc(acc[w], a0, xs[cc][w]), a1, xs[cc + 1][w]);
      }
      if (cc < nc) {
        const double2 a0 = a[(int64_t)cc * lda];
#pragma unroll
        for (int w = 0; w < NR; ++w) acc[w] = cmul_acc(acc[w], a0, xs[cc][w]);
      }
    }
  }
  if (r < rows) {
    double2 *o = out + (int64_t)blockIdx.y * slice_stride + r;
#pragma unroll
    for (int w = 0; w < NR; ++w)
      if (w < nrhs) o[(int64_t)w * ldo] = acc[w];
  }
}

// Y[w * ldy + r] = sum over slices s in order of work[(s nrhs + w) rows + r].
__global__ void matvec_slice_sum_kernel(const double2 *__restrict__ work, int64_t rows, int nrhs,
                                        int slices, double2 *__restrict__ Y, int64_t ldy) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= rows * nrhs) return;
  const int64_t w = i / rows, r = i % rows;
  double2 s = make_double2(0.0, 0.0);
  for (int k = 0; k < slices; ++k) {
    const double2 v = work[((int64_t)k * nrhs + w) * rows + r];
    s.x += v.x;
    s.y += v.y;
  }
  Y[w * ldy + r] = s;
}

// Column slices for a matrix of `rows` x `cols`: enough CTAs for four per SM
// of a 152-SM part, each slice at least one staged chunk wide.
int matvec_slices(int64_t rows, int64_t cols) {
  const int64_t tiles = (rows + kMvRows - 1) / kMvRows;
  const int64_t want = (4 * 152 + tiles - 1) / tiles;
  const int64_t most = (cols + kMvChunk - 1) / kMvChunk;
  return (int)std::max<int64_t>(1, std::min<int64_t>({want, most, 4096}));
}

constexpr int kCombineThreads = 128;
constexpr int kCombineMaxP = 1536;  // twiddles + modal values: 32 P bytes <= 48 KB

// One CTA per (row r, wave w); y may alias g or a (each thread reads its own
// elements before writing them). Shared: the twiddles e^{2 pi i t / P}, t < P,
// and the modal values fhat_n of the row for the P modes (zero for |n| > p).
__global__ void __launch_bounds__(kCombineThreads) iter_combine_kernel(
    int rows, int P, int p, const double2 *g, const double2 *a, const double *__restrict__ bt,
    const double2 *__restrict__ d, int64_t ldd, double2 *y) {
  extern __shared__ double2 sh[];
  double2 *tw = sh;        // [P]
  double2 *fh = sh + P;    // [P], mode n at n mod P
  const int r = blockIdx.x, w = blockIdx.y;
  const int nmax = min(p, P / 2);
  for (int t = threadIdx.x; t < P; t += blockDim.x) {
    double s, c;
    sincospi(2.0 * t / P, &s, &c);
    tw[t] = make_double2(c, s);
    // Mode of slot t: n = t for t <= P/2, else t - P (mode -P/2 is not held).
    const int n = t <= P / 2 ? t : t - P;
    const int an = n < 0 ? -n : n;
    double2 acc = make_double2(0.0, 0.0);
    if (an <= nmax) {
      // Block of |n|: rows x (p + 1 - |n|) column-major, after the blocks of
      // modes 0 .. |n| - 1 (sum of their widths p + 1 - m).
      const double *blk = bt + (int64_t)rows * ((int64_t)an * (p + 1) - (int64_t)an * (an - 1) / 2);
      const double2 *dw = d + (int64_t)w * ldd;
      for (int l = an; l <= p; ++l) {
        const double b = blk[(int64_t)(l - an) * rows + r];
        const double2 dv = dw[l * l + l + n];
        acc.x = fma(b, dv.x, acc.x);
        acc.y = fma(b, dv.y, acc.y);
      }
      if (n < 0 && (an & 1)) acc = make_double2(-acc.x, -acc.y);
    }
    fh[t] = acc;
  }
  __syncthreads();
  const int64_t base = ((int64_t)w * rows + r) * P;
  for (int l = threadIdx.x; l < P; l += blockDim.x) {
    // sum over the held modes; e^{2 pi i n l / P} = tw[(n l) mod P] with the
    // index reduced exactly in integers.
    double2 s = make_double2(0.0, 0.0);
    for (int n = -min(p, (P - 1) / 2); n <= nmax; ++n) {
      const int t = n < 0 ? n + P : n;
      const int k = (int)(((int64_t)t * l) % P);
      s = cmul_acc(s, fh[t], tw[k]);
    }
    double2 v = make_double2(-s.x, -s.y);
    if (g) { const double2 gv = g[base + l]; v.x += gv.x; v.y += gv.y; }
    if (a) { const double2 av = a[base + l]; v.x += av.x; v.y += av.y; }
    y[base + l] = v;
  }
}

bool aligned(const void *p, uintptr_t a) { return (reinterpret_cast<uintptr_t>(p) & (a - 1)) == 0; }

axi_status launch_status() {
  return cudaGetLastError() == cudaSuccess ? AXI_OK : AXI_ERR_CUDA;
}

}  // namespace

extern "C" axi_status axi_matvec_workspace_bytes(int64_t rows, int64_t cols, int32_t nrhs,
                                                 size_t *bytes) {
  if (!bytes || rows < 1 || cols < 1 || nrhs < 1 || nrhs > kMvMaxRhs) return AXI_ERR_ARG;
  const int s = matvec_slices(rows, cols);
  *bytes = s > 1 ? (size_t)s * nrhs * rows * sizeof(double2) : 0;
  return AXI_OK;
}

extern "C" axi_status axi_matvec_c128(const axi_c128 *d_A, int64_t lda, int64_t rows, int64_t cols,
                                      const axi_c128 *d_X, int64_t ldx, int32_t nrhs, axi_c128 *d_Y,
                                      int64_t ldy, void *d_work, size_t work_bytes, void *stream) {
  if (!d_A || !d_X || !d_Y || rows < 1 || cols < 1 || lda < rows || ldx < cols || ldy < rows ||
      nrhs < 1 || nrhs > kMvMaxRhs || (rows + kMvRows - 1) / kMvRows > INT32_MAX ||
      !aligned(d_A, 16) || !aligned(d_X, 16) || !aligned(d_Y, 16) || !aligned(d_work, 16))
    return AXI_ERR_ARG;
  size_t need = 0;
  axi_matvec_workspace_bytes(rows, cols, nrhs, &need);
  if (need > 0 && (!d_work || work_bytes < need)) return AXI_ERR_WORKSPACE;
  const int slices = matvec_slices(rows, cols);
  const int64_t per = (cols + slices - 1) / slices;
  const dim3 grid((unsigned)((rows + kMvRows - 1) / kMvRows), (unsigned)slices);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const double2 *A = reinterpret_cast<const double2 *>(d_A);
  const double2 *X = reinterpret_cast<const double2 *>(d_X);
  double2 *out = slices > 1 ? static_cast<double2 *>(d_work) : reinterpret_cast<double2 *>(d_Y);
  const int64_t ldo = slices > 1 ? rows : ldy;
  const int64_t sstride = slices > 1 ? (int64_t)nrhs * rows : 0;
#define AXI_MV(NR) \
  matvec_kernel<NR><<<grid, kMvRows, 0, st>>>(A, lda, rows, cols, X, ldx, nrhs, per, out, ldo, sstride)
  if (nrhs <= 1) AXI_MV(1);
  else if (nrhs <= 2) AXI_MV(2);
  else if (nrhs <= 4) AXI_MV(4);
  else if (nrhs <= 8) AXI_MV(8);
  else AXI_MV(16);
#undef AXI_MV
  if (slices > 1) {
    const int64_t n = rows * nrhs;
    matvec_slice_sum_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(
        static_cast<const double2 *>(d_work), rows, nrhs, slices, reinterpret_cast<double2 *>(d_Y), ldy);
  }
  return launch_status();
}

extern "C" axi_status axi_iter_combine(int32_t W, int32_t rows, int32_t P, int32_t p,
                                       const axi_c128 *d_g, const axi_c128 *d_a,
                                       const double *d_btilde, size_t btilde_count,
                                       const axi_c128 *d_d, int64_t ldd, axi_c128 *d_y,
                                       void *stream) {
  if (!d_btilde || !d_d || !d_y || W < 1 || W > 65535 || rows < 1 || rows > (1 << 30) || P < 1 ||
      P > kCombineMaxP || p < 0 || p > AXI_BTILDE_MAX_DEGREE || ldd < (int64_t)(p + 1) * (p + 1) ||
      !aligned(d_g, 16) || !aligned(d_a, 16) || !aligned(d_d, 16) || !aligned(d_y, 16) ||
      !aligned(d_btilde, 8))
    return AXI_ERR_ARG;
  const int64_t nmax = std::min(p, P / 2);
  const int64_t need = (int64_t)rows * ((nmax + 1) * (p + 1) - nmax * (nmax + 1) / 2);
  if ((int64_t)btilde_count < need) return AXI_ERR_ARG;
  const size_t smem = 2 * (size_t)P * sizeof(double2);
  iter_combine_kernel<<<dim3((unsigned)rows, (unsigned)W), kCombineThreads, smem,
                        static_cast<cudaStream_t>(stream)>>>(
      rows, P, p, reinterpret_cast<const double2 *>(d_g), reinterpret_cast<const double2 *>(d_a), d_btilde,
      reinterpret_cast<const double2 *>(d_d), ldd, reinterpret_cast<double2 *>(d_y));
  return launch_status();
}
