// FFT-based transforms of the apply (FP64), replacing the direct O(P^2) sums
// when P = 2^a 3^b 5^c:
//   boundary data to modes   fhat_n = (1/P) sum_l f_l e^{-2 pi i n l / P}  (eq. fhatquad, q = P)
//   modes to point strengths sigma_l = (1/P) sum_n c_n e^{+2 pi i n l / P}  (Sec. 4.1)
// One warp per sequence (fft.cuh); 8 sequences per CTA.
#include "axi_internal.h"
#include "fft.cuh"

namespace axi {
namespace {

constexpr int kSeq = 8;   // sequences (warps) per CTA

// X[d][2w + s][row]: s = 0 holds mode +d, s = 1 mode -d (duplicated for d = 0, P/2).
__global__ void __launch_bounds__(256)
rhs_fft_kernel(const ObsDev *__restrict__ od, int W, const double2 *__restrict__ f,
               double2 *__restrict__ X) {
  const ObsDev &o = *od;
  const int P = o.P, rows = o.rows;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int w = blockIdx.y, row = blockIdx.x * kSeq + warp;
  extern __shared__ double2 sh[];
  double2 *tw = sh;                      // [P]
  int *perm = reinterpret_cast<int *>(sh + P);                      // [P]
  double2 *seq = sh + P + (P + 1) / 2 + warp * P;                   // [kSeq][P]
  for (int i = threadIdx.x; i < P; i += blockDim.x) { tw[i] = o.tw_P[i]; perm[i] = o.fft_perm[i]; }
  if (row < rows)
    for (int l = lane; l < P; l += 32) seq[l] = f[((size_t)w * rows + row) * P + l];
  __syncthreads();
  if (row >= rows) return;
  fft::warp_fft(seq, P, tw, o.fft_rad, o.fft_nst, lane);
  const double invP = 1.0 / P;
  const int ncol = 2 * W;
  for (int ni = lane; ni < P; ni += 32) {
    const double2 v = seq[perm[ni]];
    const double2 acc = make_double2(v.x * invP, v.y * invP);
    const int dmode = ni <= P / 2 ? ni : P - ni;
    const int s = ni <= P / 2 ? 0 : 1;
    X[((size_t)dmode * ncol + 2 * w + s) * rows + row] = acc;
    if (dmode == 0 || 2 * dmode == P) X[((size_t)dmode * ncol + 2 * w + 1) * rows + row] = acc;
  }
}

// sigma[w][j][l] from coef[w][n][j]: sigma = conj(DFT(conj(c))) / P.
__global__ void __launch_bounds__(256)
point_fft_kernel(const ObsDev *__restrict__ od, int W, const double2 *__restrict__ coef,
                 double2 *__restrict__ sigma) {
  const ObsDev &o = *od;
  const int P = o.P, cols = o.cols;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int w = blockIdx.y, j = blockIdx.x * kSeq + warp;
  extern __shared__ double2 sh[];
  double2 *tw = sh;
  int *perm = reinterpret_cast<int *>(sh + P);
  double2 *seq = sh + P + (P + 1) / 2 + warp * P;
  for (int i = threadIdx.x; i < P; i += blockDim.x) { tw[i] = o.tw_P[i]; perm[i] = o.fft_perm[i]; }
  if (j < cols)
    for (int n = lane; n < P; n += 32) {
      const double2 c = coef[((size_t)w * P + n) * cols + j];
      seq[n] = make_double2(c.x, -c.y);
    }
  __syncthreads();
  if (j >= cols) return;
  fft::warp_fft(seq, P, tw, o.fft_rad, o.fft_nst, lane);
  const double invP = 1.0 / P;
  for (int l = lane; l < P; l += 32) {
    const double2 v = seq[perm[l]];
    sigma[((size_t)w * cols + j) * P + l] = make_double2(v.x * invP, -v.y * invP);
  }
}

size_t fft_smem(int P) { return sizeof(double2) * (P + (P + 1) / 2 + (size_t)kSeq * P); }

}  // namespace

cudaError_t launch_rhs_fft(const ObsDev *d_o, const ObsDev &h, int W, const double2 *f, double2 *X,
                           cudaStream_t st) {
  dim3 grid((h.rows + kSeq - 1) / kSeq, W);
  rhs_fft_kernel<<<grid, 256, fft_smem(h.P), st>>>(d_o, W, f, X);
  return cudaGetLastError();
}

cudaError_t launch_point_fft(const ObsDev *d_o, const ObsDev &h, int W, const double2 *coef,
                             double2 *sigma, cudaStream_t st) {
  dim3 grid((h.cols + kSeq - 1) / kSeq, W);
  point_fft_kernel<<<grid, 256, fft_smem(h.P), st>>>(d_o, W, coef, sigma);
  return cudaGetLastError();
}

}  // namespace axi
