// Q^+ of the periodizing system (Sec. 4.2: Q is inverted through its SVD):
// a one-sided (Hestenes) Jacobi SVD of a dense complex m x n matrix, m >= n,
// and the truncated pseudo-inverse solve x = V Sigma^+ U^H b.
//
// A sweep visits every column pair once, in n' - 1 rounds of n'/2 disjoint
// pairs (n' = n rounded up to even; the circle method: position 0 holds
// index n' - 1, the others rotate by the round). One CTA per pair and round:
// alpha = ||x||^2, beta = ||y||^2, gamma = x^H y = |gamma| e^{i phi} over the
// m rows; unless |gamma| <= tol sqrt(alpha beta), the unitary rotation
//   x' = c x - s e^{-i phi} y,   y' = s e^{i phi} x + c y,
//   zeta = (beta - alpha) / (2 |gamma|), t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)),
//   c = 1 / sqrt(1 + t^2), s = c t,
// makes the pair orthogonal, and the same rotation updates V's columns. Each
// sweep first orders the columns by decreasing norm and pairs them in that
// order (25 sweeps became 20 for the cup cell's Q). The
// largest |gamma| / sqrt(alpha beta) of a sweep is kept as an ordered 64-bit
// key; the host reads it after each sweep and stops below tol. On return A
// holds U Sigma (orthogonal columns), V the right singular vectors, sigma
// the column norms of U Sigma, so A_in = (U Sigma) V^H.
#include <algorithm>
#include <cstring>
#include <vector>

#include "axi_internal.h"

namespace axi {
namespace {

constexpr int kJT = 256;

// The sweep's largest off-diagonal ratio, as the bits of a non-negative
// double (they order like the values). One per device: calls that overlap
// on a device would share it.
__device__ unsigned long long g_jac_off;

__device__ __forceinline__ int circle_index(int x, int r, int np) {
  return x == 0 ? np - 1 : (x - 1 + r) % (np - 1);
}

// sums of 4 values over the CTA, every thread gets them
__device__ __forceinline__ void block_sum4(double (&v)[4], double (*red)[4]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < 4; ++q)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);
  if (lane == 0)
#pragma unroll
    for (int q = 0; q < 4; ++q) red[warp][q] = v[q];
  __syncthreads();
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    double s = 0.0;
    for (int w = 0; w < kJT / 32; ++w) s += red[w][q];
    v[q] = s;
  }
}

__global__ void __launch_bounds__(kJT)
jacobi_round_kernel(double2 *__restrict__ A, long long lda, int m, double2 *__restrict__ V,
                    long long ldv, int n, int np, int r, double tol, const int *__restrict__ perm) {
  int i = circle_index(blockIdx.x, r, np), j = circle_index(np - 1 - blockIdx.x, r, np);
  if (i >= n || j >= n) return;                        // the padding index: uniform over the CTA
  i = perm[i];
  j = perm[j];
  if (i > j) { const int t = i; i = j; j = t; }
  __shared__ double red[kJT / 32][4];
  double2 *x = A + (long long)i * lda, *y = A + (long long)j * lda;
  double v[4] = {0.0, 0.0, 0.0, 0.0};                  // alpha, beta, Re gamma, Im gamma
  for (int k = threadIdx.x; k < m; k += kJT) {
    const double2 a = x[k], b = y[k];
    v[0] = fma(a.x, a.x, fma(a.y, a.y, v[0]));
    v[1] = fma(b.x, b.x, fma(b.y, b.y, v[1]));
    v[2] = fma(a.x, b.x, fma(a.y, b.y, v[2]));
    v[3] = fma(a.x, b.y, fma(-a.y, b.x, v[3]));
  }
  block_sum4(v, red);
  const double al = v[0], be = v[1], g = hypot(v[2], v[3]);
  const double off = (al > 0.0 && be > 0.0) ? g / sqrt(al * be) : 0.0;
  if (threadIdx.x == 0)
    atomicMax(&g_jac_off, (unsigned long long)__double_as_longlong(isfinite(off) ? off : 1e300));
  if (!(off > tol)) return;                            // uniform: every thread has the same sums
  const double zeta = (be - al) / (2.0 * g);
  const double t = copysign(1.0, zeta) / (fabs(zeta) + sqrt(fma(zeta, zeta, 1.0)));
  const double c = 1.0 / sqrt(fma(t, t, 1.0)), s = c * t;
  const double ph_r = v[2] / g, ph_i = v[3] / g;       // e^{i phi}
  // s e^{-i phi} and s e^{i phi}
  const double sm_r = s * ph_r, sm_i = -s * ph_i, sp_r = s * ph_r, sp_i = s * ph_i;
  for (int k = threadIdx.x; k < m; k += kJT) {
    const double2 a = x[k], b = y[k];
    x[k] = make_double2(c * a.x - (sm_r * b.x - sm_i * b.y), c * a.y - (sm_r * b.y + sm_i * b.x));
    y[k] = make_double2(sp_r * a.x - sp_i * a.y + c * b.x, sp_r * a.y + sp_i * a.x + c * b.y);
  }
  double2 *vx = V + (long long)i * ldv, *vy = V + (long long)j * ldv;
  for (int k = threadIdx.x; k < n; k += kJT) {
    const double2 a = vx[k], b = vy[k];
    vx[k] = make_double2(c * a.x - (sm_r * b.x - sm_i * b.y), c * a.y - (sm_r * b.y + sm_i * b.x));
    vy[k] = make_double2(sp_r * a.x - sp_i * a.y + c * b.x, sp_r * a.y + sp_i * a.x + c * b.y);
  }
}

__global__ void identity_kernel(double2 *V, long long ldv, int n) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)n * n) return;
  const int col = (int)(e / n), row = (int)(e - (long long)col * n);
  V[(long long)col * ldv + row] = make_double2(row == col ? 1.0 : 0.0, 0.0);
}

// sigma_i = ||A(:, i)||, one CTA per column
__global__ void __launch_bounds__(kJT)
column_norm_kernel(const double2 *__restrict__ A, long long lda, int m, double *__restrict__ sigma) {
  __shared__ double red[kJT / 32][4];
  const double2 *x = A + (long long)blockIdx.x * lda;
  double v[4] = {0.0, 0.0, 0.0, 0.0};
  for (int k = threadIdx.x; k < m; k += kJT) v[0] = fma(x[k].x, x[k].x, fma(x[k].y, x[k].y, v[0]));
  block_sum4(v, red);
  if (threadIdx.x == 0) sigma[blockIdx.x] = sqrt(v[0]);
}

// W(i, r) = [sigma_i > cut sigma_max] (U Sigma)(:, i)^H B(:, r) / sigma_i^2:
// one CTA per column i and group of NR right-hand sides, so each column of
// U Sigma is read once per group; sigma_max is reduced by the CTA (the
// values are not sorted). Columns r past nrhs read the last one and are not
// written.
template <int NR>
__global__ void __launch_bounds__(kJT)
svd_project_kernel(const double2 *__restrict__ US, long long lda, int m, const double *__restrict__ sigma,
                   int n, double cutoff, const double2 *__restrict__ B, long long ldb, int nrhs,
                   double2 *__restrict__ W) {
  __shared__ double red[kJT / 32][2 * NR];
  __shared__ double smax_w[kJT / 32];
  const int i = blockIdx.x, r0 = blockIdx.y * NR;
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  double smax = 0.0;
  for (int q = threadIdx.x; q < n; q += kJT) smax = fmax(smax, sigma[q]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) smax = fmax(smax, __shfl_xor_sync(0xffffffffu, smax, o));
  if (lane == 0) smax_w[wp] = smax;
  const double2 *u = US + (long long)i * lda;
  const double2 *b[NR];
#pragma unroll
  for (int j = 0; j < NR; ++j) b[j] = B + (long long)min(r0 + j, nrhs - 1) * ldb;
  double2 acc[NR];
#pragma unroll
  for (int j = 0; j < NR; ++j) acc[j] = make_double2(0.0, 0.0);
  for (int k = threadIdx.x; k < m; k += kJT) {
    const double2 a = u[k];
#pragma unroll
    for (int j = 0; j < NR; ++j) {
      const double2 y = b[j][k];
      acc[j].x = fma(a.x, y.x, fma(a.y, y.y, acc[j].x));
      acc[j].y = fma(a.x, y.y, fma(-a.y, y.x, acc[j].y));
    }
  }
#pragma unroll
  for (int j = 0; j < NR; ++j) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      acc[j].x += __shfl_xor_sync(0xffffffffu, acc[j].x, o);
      acc[j].y += __shfl_xor_sync(0xffffffffu, acc[j].y, o);
    }
    if (lane == 0) {
      red[wp][2 * j] = acc[j].x;
      red[wp][2 * j + 1] = acc[j].y;
    }
  }
  __syncthreads();
  if (threadIdx.x < NR && r0 + (int)threadIdx.x < nrhs) {
    double sm = 0.0, re = 0.0, im = 0.0;
    for (int q = 0; q < kJT / 32; ++q) {               // fixed order: reproducible
      sm = fmax(sm, smax_w[q]);
      re += red[q][2 * threadIdx.x];
      im += red[q][2 * threadIdx.x + 1];
    }
    const double si = sigma[i];
    const double w = si > cutoff * sm ? 1.0 / (si * si) : 0.0;
    W[(long long)(r0 + threadIdx.x) * n + i] = make_double2(re * w, im * w);
  }
}

// X(:, r) = V W(:, r): one CTA per 32 rows and group of NR right-hand sides;
// its 8 warps take the terms i = warp (mod 8), the lanes the rows, and the
// warps' partial sums are added in a fixed order through shared memory.
template <int NR>
__global__ void __launch_bounds__(kJT)
svd_expand_kernel(const double2 *__restrict__ V, long long ldv, int n, const double2 *__restrict__ W,
                  int nrhs, double2 *__restrict__ X, long long ldx) {
  __shared__ double2 red[kJT / 32][32];
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  const int row = blockIdx.x * 32 + lane, r0 = blockIdx.y * NR;
  const int rr = min(row, n - 1);
  const double2 *w[NR];
#pragma unroll
  for (int j = 0; j < NR; ++j) w[j] = W + (long long)min(r0 + j, nrhs - 1) * n;
  double2 acc[NR];
#pragma unroll
  for (int j = 0; j < NR; ++j) acc[j] = make_double2(0.0, 0.0);
  for (int i = wp; i < n; i += kJT / 32) {
    const double2 a = V[(long long)i * ldv + rr];
#pragma unroll
    for (int j = 0; j < NR; ++j) {
      const double2 y = w[j][i];
      acc[j].x = fma(a.x, y.x, fma(-a.y, y.y, acc[j].x));
      acc[j].y = fma(a.x, y.y, fma(a.y, y.x, acc[j].y));
    }
  }
#pragma unroll
  for (int j = 0; j < NR; ++j) {
    red[wp][lane] = acc[j];
    __syncthreads();
    if (wp == 0 && row < n && r0 + j < nrhs) {
      double2 s = red[0][lane];
      for (int q = 1; q < kJT / 32; ++q) {
        s.x += red[q][lane].x;
        s.y += red[q][lane].y;
      }
      X[(long long)(r0 + j) * ldx + row] = s;
    }
    __syncthreads();
  }
}

}  // namespace

cudaError_t svd_jacobi(double2 *A, long long m, long long n, long long lda, double2 *V, long long ldv,
                       double *sigma, double tol, int max_sweeps, int *sweeps, bool *converged,
                       cudaStream_t st) {
  *sweeps = 0;
  *converged = false;
  const long long nn = n * n;
  identity_kernel<<<(unsigned)((nn + 255) / 256), 256, 0, st>>>(V, ldv, (int)n);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int np = (int)(n + (n & 1));
  // each sweep pairs the columns in the order of decreasing norm (the
  // permutation lives in sigma's buffer until the final norms)
  int *perm_d = reinterpret_cast<int *>(sigma);
  std::vector<double> nrm((size_t)n);
  std::vector<int> perm((size_t)n);
  for (int sw = 0; sw < max_sweeps && np > 1; ++sw) {
    column_norm_kernel<<<(unsigned)n, kJT, 0, st>>>(A, lda, (int)m, sigma);
    e = cudaGetLastError();
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(nrm.data(), sigma, sizeof(double) * n, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return e;
    for (int q = 0; q < (int)n; ++q) perm[q] = q;
    std::stable_sort(perm.begin(), perm.end(), [&](int a, int b) { return nrm[a] > nrm[b]; });
    e = cudaMemcpyAsync(perm_d, perm.data(), sizeof(int) * n, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return e;
    const unsigned long long zero = 0ull;
    e = cudaMemcpyToSymbolAsync(g_jac_off, &zero, sizeof(zero), 0, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return e;
    for (int r = 0; r < np - 1; ++r) {
      jacobi_round_kernel<<<np / 2, kJT, 0, st>>>(A, lda, (int)m, V, ldv, (int)n, np, r, tol, perm_d);
      e = cudaGetLastError();
      if (e != cudaSuccess) return e;
    }
    unsigned long long off_bits = 0ull;
    e = cudaMemcpyFromSymbolAsync(&off_bits, g_jac_off, sizeof(off_bits), 0, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return e;
    double off;
    std::memcpy(&off, &off_bits, sizeof(off));
    *sweeps = sw + 1;
    if (off <= tol) {
      *converged = true;
      break;
    }
  }
  if (np <= 1) *converged = true;
  column_norm_kernel<<<(unsigned)n, kJT, 0, st>>>(A, lda, (int)m, sigma);
  return cudaGetLastError();
}

template <int NR>
cudaError_t svd_solve_nr(const double2 *US, const double2 *V, const double *sigma, long long m, long long n,
                         long long lda, long long ldv, double cutoff, const double2 *B, long long ldb,
                         long long nrhs, double2 *X, long long ldx, double2 *W, cudaStream_t st) {
  const unsigned groups = (unsigned)((nrhs + NR - 1) / NR);
  svd_project_kernel<NR><<<dim3((unsigned)n, groups), kJT, 0, st>>>(US, lda, (int)m, sigma, (int)n, cutoff,
                                                                     B, ldb, (int)nrhs, W);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  svd_expand_kernel<NR><<<dim3((unsigned)((n + 31) / 32), groups), kJT, 0, st>>>(V, ldv, (int)n, W,
                                                                                  (int)nrhs, X, ldx);
  return cudaGetLastError();
}

cudaError_t svd_solve(const double2 *US, const double2 *V, const double *sigma, long long m, long long n,
                      long long lda, long long ldv, double cutoff, const double2 *B, long long ldb,
                      long long nrhs, double2 *X, long long ldx, double2 *W, cudaStream_t st) {
  if (nrhs <= 1) return svd_solve_nr<1>(US, V, sigma, m, n, lda, ldv, cutoff, B, ldb, nrhs, X, ldx, W, st);
  if (nrhs <= 2) return svd_solve_nr<2>(US, V, sigma, m, n, lda, ldv, cutoff, B, ldb, nrhs, X, ldx, W, st);
  if (nrhs <= 4) return svd_solve_nr<4>(US, V, sigma, m, n, lda, ldv, cutoff, B, ldb, nrhs, X, ldx, W, st);
  if (nrhs <= 8) return svd_solve_nr<8>(US, V, sigma, m, n, lda, ldv, cutoff, B, ldb, nrhs, X, ldx, W, st);
  return svd_solve_nr<16>(US, V, sigma, m, n, lda, ldv, cutoff, B, ldb, nrhs, X, ldx, W, st);
}

}  // namespace axi
