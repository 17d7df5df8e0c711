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
// Layout on the GPU: a CTA takes 32 collocation points (one per lane); each
// warp takes the orders m and nmax - m (nmax = min(P/2, p)), whose degree
// ranges l = m .. p and l = nmax - m .. p add up to the same length for
// every warp; the grid covers all points and all orders, so the FP64 work
// spreads evenly over the SMs. For a point (rho_i, z_i), r = |(rho_i, z_i)|
// and theta its polar angle:
//   * warp 0: j_0 .. j_max(p, 1) of x = k r for its 32 points into shared
//     memory, by the backward three-term recurrence
//     f_{l-1} = (2l + 1)/x f_l - f_{l+1} from l = p + max x + 32 (Miller's
//     algorithm: the recurrence's minimal solution is j_l), rescaled by
//     2^-664 whenever a value passes 2^664, and normalised by
//     j_0 = sin x / x or j_1 = sin x / x^2 - cos x / x, whichever is larger;
//   * meanwhile each warp writes its orders' recurrence coefficients for
//     l = m .. p into shared memory, one l per lane (they depend on (l, m)
//     only):
//       Pbar_{m+1}^m = sqrt(2m+3) cos(theta) Pbar_m^m,
//       Pbar_l^m = a_lm (cos(theta) Pbar_{l-1}^m - b_lm Pbar_{l-2}^m),
//       a_lm = sqrt((4l^2-1)/(l^2-m^2)), b_lm = sqrt(((l-1)^2-m^2)/(4(l-1)^2-1)),
//       dPbar_l^m/dtheta = (l cos(theta) Pbar_l^m - c_lm Pbar_{l-1}^m)/sin(theta),
//       c_lm = sqrt((2l+1)(l-m)(l+m)/(2l-1));
//     Pbar_m^m = (-1)^m sqrt((1/(4 pi)) prod_{u<=m} (2u+1)/(2u)) sin(theta)^m;
//   * then per l, for all 32 points at once: f = j_l(x) Pbar,
//     d_r f = k j_l'(x) Pbar (j_l' = j_{l-1} - (l+1)/x j_l, j_0' = -j_1),
//     d_theta f = j_l(x) dPbar; with
//       d_rho f = sin(theta) d_r f + cos(theta)/r d_theta f,
//       d_z f   = cos(theta) d_r f - sin(theta)/r d_theta f,
//     the normal derivative is A d_r f + B d_theta f, A = n_rho sin(theta) +
//     n_z cos(theta), B = (n_rho cos(theta) - n_z sin(theta))/r, formed once
//     per point; the 32 points' entries of a column are written as one
//     coalesced segment.
#include "axi_internal.h"

namespace axi {
namespace {

constexpr int kBtWarps = 2;                         // order pairs per CTA

__device__ __forceinline__ size_t bt_block_offset(int n, int p, int rows) {
  return (size_t)rows * ((size_t)n * (p + 1) - (size_t)n * (n - 1) / 2);
}

// the recurrence coefficients (a, b, c) of order m for l = m .. p, one l per lane
__device__ __forceinline__ void bt_coefficients(double *cf, int m, int p, int lane) {
  for (int l = m + lane; l <= p; l += 32) {
    double a = 0.0, b = 0.0, c = 0.0;
    if (l == m + 1) {
      a = sqrt(2.0 * m + 3.0);
    } else if (l > m + 1) {
      const double ll = (double)l * l, mm = (double)m * m, l1 = (double)(l - 1) * (l - 1);
      a = sqrt((4.0 * ll - 1.0) / (ll - mm));
      b = sqrt((l1 - mm) / (4.0 * l1 - 1.0));
    }
    if (l > m) c = sqrt((2.0 * l + 1.0) * (l - m) * (l + m) / (2.0 * l - 1.0));
    cf[l] = a;
    cf[(p + 1) + l] = b;
    cf[2 * (p + 1) + l] = c;
  }
}

__global__ void __launch_bounds__(32 * kBtWarps)
btilde_kernel(const ObsDev *__restrict__ obs_arr, int oi, int p, int nmax, double *__restrict__ out) {
  const ObsDev &o = obs_arr[oi];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int jn = (p > 1 ? p : 1) + 1;
  extern __shared__ double bt_sh[];
  double *jl = bt_sh;                               // [jn][32]: j_l of lane's point
  double *cf = bt_sh + (size_t)jn * 32 + (size_t)warp * 6 * (p + 1);   // [2 orders][3][p + 1]
  const int i = blockIdx.x * 32 + lane;
  const int m0 = blockIdx.y * kBtWarps + warp, m1 = nmax - m0;   // this warp's orders
  const bool has0 = m0 <= m1, has1 = m0 < m1;
  const bool live = i < o.M;
  const int ic = live ? i : o.M - 1;                // a valid point for idle lanes
  const double rho = o.coll[4 * ic], z = o.coll[4 * ic + 1];
  const double nr = o.coll[4 * ic + 2], nz = o.coll[4 * ic + 3];
  const double r = hypot(rho, z), x = o.k * r;
  const double st = rho / r, ct = z / r;            // sin, cos of the polar angle
  const double ix = 1.0 / x;
  if (warp == 0) {
    double xmax = x;
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) xmax = fmax(xmax, __shfl_xor_sync(0xffffffffu, xmax, s));
    const int L0 = p + (int)xmax + 32;
    double f1 = 0.0, f0 = 1.0;                      // f_{l+1}, f_l at l = L0
    double t = (2.0 * L0 + 1.0) * ix;               // (2l + 1)/x, one subtraction per step
    const double dt = 2.0 * ix;
    for (int l = L0; l >= 1; --l) {
      const double fm = fma(t, f0, -f1);
      t -= dt;
      f1 = f0;
      f0 = fm;                                      // f_{l-1}
      if (l - 1 < jn) jl[(l - 1) * 32 + lane] = fm;
      // |f_{l-1}| above 2^664, tested on the exponent bits (integer instructions)
      if (((unsigned long long)__double_as_longlong(fm) & 0x7ff0000000000000ull) > 0x6970000000000000ull) {
        const double s = 0x1p-664;
        f0 *= s;
        f1 *= s;
        for (int u = l - 1; u < jn; ++u) jl[u * 32 + lane] *= s;
      }
    }
    double sn, cs;
    sincos(x, &sn, &cs);
    const double j0 = sn * ix, j1 = (sn * ix - cs) * ix;
    const double sc = fabs(j0) >= fabs(j1) ? j0 / jl[lane] : j1 / jl[32 + lane];
    for (int u = 0; u < jn; ++u) jl[u * 32 + lane] *= sc;
  }
  if (has0) bt_coefficients(cf, m0, p, lane);
  if (has1) bt_coefficients(cf + 3 * (p + 1), m1, p, lane);
  __syncthreads();                                  // j_l of the CTA's points, the coefficients
  const int rows = o.rows, M = o.M;
  const bool trans = o.bc == AXI_BC_TRANSMISSION;
  const double ist = 1.0 / st;
  const double Ak = o.k * (nr * st + nz * ct), B = (nr * ct - nz * st) / r;
  bool finite = true;
  for (int t = 0; t < 2; ++t) {
    if (!(t == 0 ? has0 : has1)) continue;
    const int m = t == 0 ? m0 : m1;
    const double *ca = cf + t * 3 * (p + 1), *cb = ca + (p + 1), *cc = ca + 2 * (p + 1);
    double prod = 1.0 / (4.0 * 3.14159265358979323846), spow = 1.0;
    for (int u = 1; u <= m; ++u) {
      prod *= (2.0 * u + 1.0) / (2.0 * u);
      spow *= st;
    }
    double cur = ((m & 1) ? -sqrt(prod) : sqrt(prod)) * spow;   // Pbar_m^m
    double prev = 0.0;
    double *blk = out + bt_block_offset(m, p, rows);
    double lct = m * ct;                            // l cos(theta)
    for (int l = m; l <= p; ++l) {
      if (l > m) {
        const double nxt = ca[l] * fma(ct, cur, -cb[l] * prev);
        prev = cur;
        cur = nxt;
        lct += ct;
      }
      const double dP = fma(lct, cur, -cc[l] * prev) * ist;
      const double j = jl[l * 32 + lane];
      const double dj = l == 0 ? -jl[32 + lane] : fma(-(l + 1.0) * ix, j, jl[(l - 1) * 32 + lane]);
      const double dn = fma(Ak * dj, cur, B * j * dP);
      double *col = blk + (size_t)(l - m) * rows;
      if (live) {
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
  const size_t smem = sizeof(double) * ((size_t)jn * 32 + (size_t)kBtWarps * 6 * (p + 1));
  static size_t granted = 0;
  cudaError_t e = ensure_dynamic_smem(btilde_kernel, smem, granted);
  if (e != cudaSuccess) return e;
  const int pairs = nmax / 2 + 1;                   // warps per 32 points: orders m and nmax - m
  const dim3 grid((h.M + 31) / 32, (pairs + kBtWarps - 1) / kBtWarps);
  btilde_kernel<<<grid, 32 * kBtWarps, smem, st>>>(d_obs, oi, p, nmax, out);
  return cudaGetLastError();
}

}  // namespace axi
