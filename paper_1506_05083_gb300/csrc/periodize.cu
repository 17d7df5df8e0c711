// The periodizing scheme's spherical-wave block B~ (Sec. 4, eq. urep; Sec.
// 4.1, the B~ display): the effect of the auxiliary regular waves
// u_lm = j_l(k r) Y_lm(theta, phi), l <= p, on the obstacle's modal boundary
// data.
//
// With the obstacle's axis on the expansion's z axis, the mean over phi of
// F[u_lm] e^{-i n phi} (F the boundary functional of a collocation ring:
// the normal derivative for Neumann rows, the value and the normal
// derivative for transmission rows) is delta_{mn} times F applied to the
// meridian-plane function j_l(k r) Pbar_l^n(cos theta), Pbar the
// orthonormal associated Legendre function with the Condon-Shortley phase
// (Y_lm = Pbar_l^m(cos theta) e^{i m phi}). So B~ is block diagonal in the
// mode and real: mode n keeps the p + 1 - n columns l = n .. p, and mode -n
// is (-1)^n mode n. The trapezoid rule the paper prints gives the same
// blocks for q > |m| + |n| nodes; forming them directly costs O(M p^2)
// instead of O(M P p^2 q).
//
// One warp per collocation point (rho_i, z_i), r = |(rho_i, z_i)|, theta the
// polar angle:
//   * lane 0: j_0 .. j_max(p, 1) of x = k r by the backward three-term
//     recurrence f_{l-1} = (2l + 1)/x f_l - f_{l+1} from l = p + x + 32
//     (Miller's algorithm: the recurrence's minimal solution is j_l),
//     rescaled by 2^-664 whenever a value passes 2^664, and normalised by
//     j_0 = sin x / x or j_1 = sin x / x^2 - cos x / x, whichever is larger;
//   * lanes over the order m = n: Pbar_m^m = -sqrt((2m+1)/(2m)) sin(theta)
//     Pbar_{m-1}^{m-1} from Pbar_0^0 = 1/sqrt(4 pi), then in l
//       Pbar_{m+1}^m = sqrt(2m+3) cos(theta) Pbar_m^m,
//       Pbar_l^m = a_lm (cos(theta) Pbar_{l-1}^m - b_lm Pbar_{l-2}^m),
//       a_lm = sqrt((4l^2-1)/(l^2-m^2)), b_lm = sqrt(((l-1)^2-m^2)/(4(l-1)^2-1)),
//     dPbar_l^m/dtheta = (l cos(theta) Pbar_l^m - c_lm Pbar_{l-1}^m)/sin(theta),
//       c_lm = sqrt((2l+1)(l-m)(l+m)/(2l-1));
//   * f = j_l(x) Pbar, d_r f = k j_l'(x) Pbar (j_l' = j_{l-1} - (l+1)/x j_l,
//     j_0' = -j_1), d_theta f = j_l(x) dPbar, and
//       d_rho f = sin(theta) d_r f + cos(theta)/r d_theta f,
//       d_z f   = cos(theta) d_r f - sin(theta)/r d_theta f,
//     the normal derivative n_rho d_rho f + n_z d_z f.
#include "axi_internal.h"

namespace axi {
namespace {

constexpr int kBtWarps = 4;

__device__ __forceinline__ size_t bt_block_offset(int n, int p, int rows) {
  return (size_t)rows * ((size_t)n * (p + 1) - (size_t)n * (n - 1) / 2);
}

__global__ void __launch_bounds__(32 * kBtWarps)
btilde_kernel(const ObsDev *__restrict__ obs_arr, int oi, int p, int nmax, double *__restrict__ out) {
  const ObsDev &o = obs_arr[oi];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int i = blockIdx.x * kBtWarps + warp;
  extern __shared__ double bt_j[];                  // [kBtWarps][jn]: j_0 .. j_{jn-1}
  const int jn = (p > 1 ? p : 1) + 1;
  double *jl = bt_j + (size_t)warp * jn;
  if (i >= o.M) return;                             // whole warp; no block barriers below
  const double rho = o.coll[4 * i], z = o.coll[4 * i + 1];
  const double nr = o.coll[4 * i + 2], nz = o.coll[4 * i + 3];
  const double r = hypot(rho, z), x = o.k * r;
  const double st = rho / r, ct = z / r;            // sin, cos of the polar angle
  if (lane == 0) {
    const int L0 = p + (int)x + 32;
    double f1 = 0.0, f0 = 1.0;                      // f_{l+1}, f_l at l = L0
    for (int l = L0; l >= 1; --l) {
      const double fm = (2.0 * l + 1.0) / x * f0 - f1;
      f1 = f0;
      f0 = fm;                                      // f_{l-1}
      if (l - 1 < jn) jl[l - 1] = fm;
      if (fabs(fm) > 0x1p664) {                     // keep the sequence in range
        const double s = 0x1p-664;
        f0 *= s;
        f1 *= s;
        for (int u = l - 1; u < jn && u <= L0; ++u) jl[u] *= s;
      }
    }
    double sn, cs;
    sincos(x, &sn, &cs);
    const double j0 = sn / x, j1 = sn / (x * x) - cs / x;
    const double sc = fabs(j0) >= fabs(j1) ? j0 / jl[0] : j1 / jl[1];
    for (int u = 0; u < jn; ++u) jl[u] *= sc;
  }
  __syncwarp();
  const int rows = o.rows, M = o.M;
  const bool trans = o.bc == AXI_BC_TRANSMISSION;
  bool finite = true;
  for (int m = lane; m <= nmax; m += 32) {
    double pmm = 0.28209479177387814347;            // 1 / sqrt(4 pi)
    for (int u = 1; u <= m; ++u) pmm *= -sqrt((2.0 * u + 1.0) / (2.0 * u)) * st;
    double *blk = out + bt_block_offset(m, p, rows);
    double prev = 0.0, cur = pmm;                   // Pbar_{l-1}^m, Pbar_l^m
    for (int l = m; l <= p; ++l) {
      if (l == m + 1) {
        prev = cur;
        cur = sqrt(2.0 * m + 3.0) * ct * prev;
      } else if (l > m + 1) {
        const double ll = (double)l * l, mm = (double)m * m, l1 = (double)(l - 1) * (l - 1);
        const double a = sqrt((4.0 * ll - 1.0) / (ll - mm)), b = sqrt((l1 - mm) / (4.0 * l1 - 1.0));
        const double nxt = a * (ct * cur - b * prev);
        prev = cur;
        cur = nxt;
      }
      const double c = l > m ? sqrt((2.0 * l + 1.0) * (l - m) * (l + m) / (2.0 * l - 1.0)) : 0.0;
      const double dP = (l * ct * cur - c * (l > m ? prev : 0.0)) / st;
      const double j = jl[l];
      const double dj = l == 0 ? -jl[1] : jl[l - 1] - (l + 1.0) / x * j;
      const double fr = o.k * dj * cur, ft = j * dP;
      const double drho = st * fr + ct / r * ft, dz = ct * fr - st / r * ft;
      const double dn = nr * drho + nz * dz;
      double *col = blk + (size_t)(l - m) * rows;
      if (trans) {
        const double v = j * cur;
        col[i] = v;
        col[M + i] = dn;
        finite = finite && isfinite(v);
      } else {
        col[i] = dn;
      }
      finite = finite && isfinite(dn);
    }
  }
  if (!finite) atomicOr(o.status, kStatNonFinite);
}

}  // namespace

size_t btilde_count(const ObsDev &h, int p) {
  const int nmax = min(h.D - 1, p);
  return (size_t)h.rows * ((size_t)(nmax + 1) * (p + 1) - (size_t)(nmax + 1) * nmax / 2);
}

cudaError_t launch_btilde(const ObsDev *d_obs, const ObsDev &h, int oi, int p, double *out,
                          cudaStream_t st) {
  if (h.M <= 0) return cudaSuccess;
  const int nmax = min(h.D - 1, p);
  const int jn = (p > 1 ? p : 1) + 1;
  const size_t smem = sizeof(double) * (size_t)kBtWarps * jn;
  btilde_kernel<<<(h.M + kBtWarps - 1) / kBtWarps, 32 * kBtWarps, smem, st>>>(d_obs, oi, p, nmax, out);
  return cudaGetLastError();
}

}  // namespace axi
