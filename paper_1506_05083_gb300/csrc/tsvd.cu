// Truncated-SVD form of the one-obstacle operator (Sec. 4.2: each block's
// pseudo-inverse applied as V_n Sigma_n^+ (U_n^* x), truncation 1e-10,
// never formed explicitly), built on the Householder QR: A_n = Q R and
//   R = U_R Sigma V^H   (one-sided Jacobi, FP64),
// so A_n = (Q U_R) Sigma V^H and
//   c = V Sigma^+ U_R^H (Q^H fhat_n)_{1:N},
// Sigma^+ keeping the singular values >= 1e-10 sigma_max.
//
// One-sided (Hestenes) Jacobi: the columns g_i of G (initially R) are made
// mutually orthogonal by plane rotations from the right, G <- G J, V <- V J.
// For a pair (i, j) with alpha = |g_i|^2, beta = |g_j|^2, gamma = g_i^H g_j,
// the phase e = conj(gamma)/|gamma| makes the off-diagonal real, and the
// rotation with zeta = (beta - alpha) / (2 |gamma|),
// t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)), c = 1/sqrt(1 + t^2), s = c t
//   g_i <- c g_i - s e g_j,   g_j <- s g_i + c e g_j
// zeroes it. A sweep visits every pair once in round-robin order (n - 1
// rounds of n/2 disjoint pairs, one warp per pair); sweeps repeat until no
// pair has |gamma| > n eps sqrt(alpha beta) (the rounding of a length-n dot
// product is about sqrt(n) eps of it, so a tighter test never settles), at
// most kMaxSweeps. Then sigma_j = |g_j| and U_R = G Sigma^{-1}.
#include "axi_internal.h"

namespace axi {
namespace {

constexpr int kJThreads = 512;
constexpr int kMaxSweeps = 40;
constexpr double kEps = 2.220446049250313e-16;

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Column k of round r of the circle method over m (even) positions.
__device__ __forceinline__ int circle_pos(int k, int r, int m) {
  return k == 0 ? 0 : 1 + (k - 1 + r) % (m - 1);
}

__global__ void __launch_bounds__(kJThreads)
tsvd_jacobi_kernel(const ObsDev *__restrict__ od) {
  const ObsDev &o = *od;
  const int d = blockIdx.x;
  if (!owns_mode(o, d)) return;
  const int n = o.cols, ld = o.rows;
  const int m = (n + 1) & ~1;                      // positions (a dummy when n is odd)
  const double tol = n * kEps;
  double2 *G = o.svdU + (size_t)d * n * n;         // column-major, column j at G + j n
  double2 *V = o.svdV + (size_t)d * n * n;
  const double2 *R = o.A + (size_t)d * o.cols * ld;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int nw = kJThreads / 32;
  __shared__ int rotations;
  // columns ordered by decreasing norm (Jacobi converges in fewer sweeps when
  // the large columns come first): rank of column j among the column norms
  // of R (ties by index), then G = R P, V = P
  extern __shared__ double jsm[];
  double *cn = jsm;                                // [n] column norms^2
  int *pos = reinterpret_cast<int *>(jsm + n);     // [n] new position of column j
  for (int j = warp; j < n; j += nw) {
    double s2 = 0.0;
    for (int q = lane; q <= j; q += 32) {
      const double2 r = R[(size_t)j * ld + q];
      s2 = fma(r.x, r.x, fma(r.y, r.y, s2));
    }
    s2 = warp_sum_d(s2);
    if (lane == 0) cn[j] = s2;
  }
  __syncthreads();
  for (int j = tid; j < n; j += kJThreads) {
    int rk = 0;
    for (int q = 0; q < n; ++q) rk += (cn[q] > cn[j] || (cn[q] == cn[j] && q < j)) ? 1 : 0;
    pos[j] = rk;
  }
  __syncthreads();
  for (size_t e = tid; e < (size_t)n * n; e += kJThreads) {
    const int j = (int)(e / n), i = (int)(e % n);
    const size_t to = (size_t)pos[j] * n + i;
    G[to] = i <= j ? R[(size_t)j * ld + i] : make_double2(0.0, 0.0);
    V[to] = make_double2(i == j ? 1.0 : 0.0, 0.0);
  }
  __syncthreads();
  int sweep = 0;
  for (; sweep < kMaxSweeps; ++sweep) {
    if (tid == 0) rotations = 0;
    __syncthreads();
    for (int r = 0; r < m - 1; ++r) {
      for (int k = warp; k < m / 2; k += nw) {
        int i = circle_pos(k, r, m), j = circle_pos(m - 1 - k, r, m);
        if (i > j) { const int t = i; i = j; j = t; }
        if (j >= n) continue;                      // the dummy position
        double2 *gi = G + (size_t)i * n, *gj = G + (size_t)j * n;
        double al = 0.0, be = 0.0, gr = 0.0, gm = 0.0;
        for (int q = lane; q < n; q += 32) {
          const double2 a = gi[q], b = gj[q];
          al = fma(a.x, a.x, fma(a.y, a.y, al));
          be = fma(b.x, b.x, fma(b.y, b.y, be));
          gr = fma(a.x, b.x, fma(a.y, b.y, gr));      // conj(a) b
          gm = fma(a.x, b.y, fma(-a.y, b.x, gm));
        }
        al = warp_sum_d(al);
        be = warp_sum_d(be);
        gr = warp_sum_d(gr);
        gm = warp_sum_d(gm);
        const double ag = sqrt(gr * gr + gm * gm);
        if (!(ag > tol * sqrt(al * be))) continue;     // already orthogonal (uniform in the warp)
        const double zeta = (be - al) / (2.0 * ag);
        const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
        const double c = 1.0 / sqrt(1.0 + t * t), s = c * t;
        const double er = gr / ag, ei = -gm / ag;      // e = conj(gamma) / |gamma|
        auto rotate = [&](double2 *xi, double2 *xj) {
          for (int q = lane; q < n; q += 32) {
            const double2 a = xi[q], b = xj[q];
            const double2 eb = make_double2(er * b.x - ei * b.y, er * b.y + ei * b.x);
            xi[q] = make_double2(c * a.x - s * eb.x, c * a.y - s * eb.y);
            xj[q] = make_double2(s * a.x + c * eb.x, s * a.y + c * eb.y);
          }
        };
        rotate(gi, gj);
        rotate(V + (size_t)i * n, V + (size_t)j * n);
        if (lane == 0) atomicAdd(&rotations, 1);
      }
      __syncthreads();
    }
    if (rotations == 0) break;
    __syncthreads();
  }
  // sigma_j = |g_j|, u_j = g_j / sigma_j
  for (int j = warp; j < n; j += nw) {
    double2 *gj = G + (size_t)j * n;
    double s2 = 0.0;
    for (int q = lane; q < n; q += 32) s2 = fma(gj[q].x, gj[q].x, fma(gj[q].y, gj[q].y, s2));
    const double sg = sqrt(warp_sum_d(s2));
    const double inv = sg > 0.0 ? 1.0 / sg : 0.0;
    for (int q = lane; q < n; q += 32) gj[q] = make_double2(gj[q].x * inv, gj[q].y * inv);
    if (lane == 0) {
      o.svdS[(size_t)d * n + j] = sg;
      if (!isfinite(sg)) atomicOr(o.status, kStatNonFinite);
    }
  }
  if (tid == 0) {
    o.svdSweeps[d] = sweep + 1;
    if (sweep == kMaxSweeps) atomicOr(o.status, kStatTimeout);   // no convergence
  }
}

// X[d][c][0..n) <- V Sigma^+ U^H X[d][c][0..n) for kTC right-hand-side
// columns per CTA: z = U^H y (one warp per output k), scaled by 1/sigma_k
// where sigma_k >= 1e-10 sigma_max (else 0), then x = V z (threads over rows).
constexpr int kTC = 8;
__global__ void __launch_bounds__(256)
tsvd_apply_kernel(const ObsDev *__restrict__ od, double2 *__restrict__ X, int ncols_total) {
  const ObsDev &o = *od;
  const int d = blockIdx.x;
  const int c0 = blockIdx.y * kTC;
  if (c0 >= ncols_total || !owns_mode(o, d)) return;
  const int nc = min(kTC, ncols_total - c0);
  const int n = o.cols;
  const double2 *U = o.svdU + (size_t)d * n * n;
  const double2 *V = o.svdV + (size_t)d * n * n;
  const double *sg = o.svdS + (size_t)d * n;
  double2 *Xd = X + ((size_t)d * ncols_total + c0) * o.rows;
  extern __shared__ double2 tsm[];
  double2 *y = tsm;                 // [kTC][n]
  double2 *z = tsm + kTC * n;       // [kTC][n]
  __shared__ double smax;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int e = tid; e < kTC * n; e += 256) {
    const int c = e / n, i = e % n;
    y[e] = c < nc ? Xd[(size_t)c * o.rows + i] : make_double2(0.0, 0.0);
  }
  if (warp == 0) {
    double mx = 0.0;
    for (int k = lane; k < n; k += 32) mx = fmax(mx, sg[k]);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, off));
    if (lane == 0) smax = mx;
  }
  __syncthreads();
  const double cut = 1e-10 * smax;
  for (int k = warp; k < n; k += 8) {
    const double2 *uk = U + (size_t)k * n;
    double2 acc[kTC];
#pragma unroll
    for (int c = 0; c < kTC; ++c) acc[c] = make_double2(0.0, 0.0);
    for (int i = lane; i < n; i += 32) {
      const double2 u = uk[i];
#pragma unroll
      for (int c = 0; c < kTC; ++c) {
        const double2 v = y[c * n + i];
        acc[c].x = fma(u.x, v.x, fma(u.y, v.y, acc[c].x));      // conj(u) v
        acc[c].y = fma(u.x, v.y, fma(-u.y, v.x, acc[c].y));
      }
    }
    const double s = sg[k];
    const double w = s >= cut && s > 0.0 ? 1.0 / s : 0.0;
#pragma unroll
    for (int c = 0; c < kTC; ++c) {
      const double re = warp_sum_d(acc[c].x), im = warp_sum_d(acc[c].y);
      if (lane == 0) z[c * n + k] = make_double2(re * w, im * w);
    }
  }
  __syncthreads();
  for (int i = tid; i < n; i += 256) {
    double2 acc[kTC];
#pragma unroll
    for (int c = 0; c < kTC; ++c) acc[c] = make_double2(0.0, 0.0);
    for (int k = 0; k < n; ++k) {
      const double2 v = V[(size_t)k * n + i];
#pragma unroll
      for (int c = 0; c < kTC; ++c) {
        const double2 zz = z[c * n + k];
        acc[c].x = fma(v.x, zz.x, fma(-v.y, zz.y, acc[c].x));
        acc[c].y = fma(v.x, zz.y, fma(v.y, zz.x, acc[c].y));
      }
    }
    for (int c = 0; c < nc; ++c) Xd[(size_t)c * o.rows + i] = acc[c];
  }
}

}  // namespace

cudaError_t launch_tsvd(const ObsDev *d_o, const ObsDev &h, cudaStream_t st) {
  const size_t smem = (sizeof(double) + sizeof(int)) * (size_t)h.cols + 16;
  static size_t granted = 0;
  cudaError_t e = ensure_dynamic_smem(tsvd_jacobi_kernel, smem, granted);
  if (e != cudaSuccess) return e;
  tsvd_jacobi_kernel<<<h.D, kJThreads, smem, st>>>(d_o);
  return cudaGetLastError();
}

cudaError_t launch_tsvd_apply(const ObsDev *d_o, const ObsDev &h, double2 *X, int ncol,
                              cudaStream_t st) {
  const size_t smem = sizeof(double2) * 2 * kTC * (size_t)h.cols;
  static size_t granted = 0;
  cudaError_t e = ensure_dynamic_smem(tsvd_apply_kernel, smem, granted);
  if (e != cudaSuccess) return e;
  tsvd_apply_kernel<<<dim3(h.D, (ncol + kTC - 1) / kTC), 256, smem, st>>>(d_o, X, ncol);
  return cudaGetLastError();
}

}  // namespace axi
