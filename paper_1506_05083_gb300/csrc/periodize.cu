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
#include <cmath>

#include "axi_internal.h"
#include "fft.cuh"

namespace axi {
namespace {

constexpr int kQMaxM1 = 64;
constexpr int kQMaxRows = 128;

// The unit cell and Rayleigh-Bloch set of a Q fill, by value (kernel
// parameter): Gauss nodes on [-1, 1] and, per m = rb_m0 + u, the first n
// and the count of the modes with |kappa| <= pi N0 (host enumeration).
struct QCell {
  double kx, ky, ex, ey, z0;
  int p, m1, n0, nrb, nrows, rb_m0;
  double g[kQMaxM1];
  int rb_n0[kQMaxRows], rb_count[kQMaxRows];
};

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

// ---------------------------------------------------------------------------
// Q, the periodizing rows of eq. full for the unknowns [d; a; b]: the S
// blocks put the spherical waves and one Cartesian derivative at the
// M1 x M1 product Gauss nodes of the unit cell's faces, as the
// discrepancies of eqs. qp1-qp4 (u_R - alpha u_L, d_x u_R - alpha d_x u_L,
// u_F - beta u_B, d_y u_F - beta d_y u_B) and the Cauchy data on T and D
// (u, d_z u); the W blocks put the Rayleigh-Bloch waves on T and D (eqs.
// rb1-rb2, T-nD): -e^{i(kap_x x + kap_y y)} and -i k_z e^{...} on T for the
// a's, -e^{...} and +i k_z e^{...} on D for the b's. Column-major output,
// columns l^2 + l + m, then the a's, then the b's.
//
// S kernel: the lanes of a warp take 32 row pairs (a node of L and its
// partner on R, of B and F, or one node of T or D), each warp the orders m
// and p - m, both signs: for real k, u_{l,-m} = (-1)^m conj(u_lm). At a
// point with r, cos(theta) = z/r, sin(theta) = rho/r and e^{i phi} =
// (x + i y)/rho (rho > 0: with M1 even no node lies on the axis), and
// E = e^{i m phi}, u = j_l(k r) Pbar_l^m E and, with A = k j_l' Pbar,
// B = j_l dPbar / r, C = m j_l Pbar / (r sin(theta)),
//   d_x u = E ((A sin + B cos) cos(phi) - i C sin(phi)),
//   d_y u = E ((A sin + B cos) sin(phi) + i C cos(phi)),
//   d_z u = E (A cos(theta) - B sin(theta)),
// from grad u = d_r u e_r + d_theta u e_theta / r + d_phi u e_phi / (r sin).
// ---------------------------------------------------------------------------

constexpr int kQWarps = 2;

struct QPoint {
  double r, st, ct, cp, sp, ix, ist, ir;
};

__device__ __forceinline__ QPoint q_point(double x, double y, double z, double k) {
  QPoint q;
  const double rho = hypot(x, y);
  q.r = hypot(rho, z);
  q.st = rho / q.r;
  q.ct = z / q.r;
  q.cp = x / rho;
  q.sp = y / rho;
  q.ix = 1.0 / (k * q.r);
  q.ist = 1.0 / q.st;
  q.ir = 1.0 / q.r;
  return q;
}

// j_0 .. j_{jn-1}(k r) of each lane's point into jl[u * 32 + lane] (Miller's
// backward recurrence as in btilde_kernel); L0 is uniform over the warp
__device__ void q_bessel(double *jl, int jn, int L0, double ix, int lane) {
  double f1 = 0.0, f0 = 1.0;
  double t = (2.0 * L0 + 1.0) * ix;
  const double dt = 2.0 * ix;
  for (int l = L0; l >= 1; --l) {
    const double fm = fma(t, f0, -f1);
    t -= dt;
    f1 = f0;
    f0 = fm;
    if (l - 1 < jn) jl[(l - 1) * 32 + lane] = fm;
    if (((unsigned long long)__double_as_longlong(fm) & 0x7ff0000000000000ull) > 0x6970000000000000ull) {
      const double s = 0x1p-664;
      f0 *= s;
      f1 *= s;
      for (int u = l - 1; u < jn; ++u) jl[u * 32 + lane] *= s;
    }
  }
  const double x = 1.0 / ix;
  double sn, cs;
  sincos(x, &sn, &cs);
  const double j0 = sn * ix, j1 = (sn * ix - cs) * ix;
  const double sc = fabs(j0) >= fabs(j1) ? j0 / jl[lane] : j1 / jl[32 + lane];
  for (int u = 0; u < jn; ++u) jl[u * 32 + lane] *= sc;
}

__device__ __forceinline__ double2 cmul2(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

__global__ void __launch_bounds__(32 * kQWarps)
q_s_kernel(const ObsDev *__restrict__ obs_arr, int oi, QCell cell, double2 *__restrict__ out, long long ld) {
  const ObsDev &o = obs_arr[oi];
  const double k = o.k;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int p = cell.p, m1 = cell.m1, nr = m1 * m1;
  const int jn = (p > 1 ? p : 1) + 1;
  extern __shared__ double q_sh[];
  double *cf = q_sh + (size_t)warp * (2 * jn * 32 + 6 * (p + 1));   // [2 orders][3][p + 1]
  double *jl0 = cf + 6 * (p + 1), *jl1 = jl0 + (size_t)jn * 32;     // [jn][32] per point
  const int row = blockIdx.x * 32 + lane;                            // row pair
  const int g0 = blockIdx.y * (blockDim.x >> 5) + warp;
  const int m0 = g0, m1o = p - g0;
  const bool has0 = m0 <= m1o, has1 = m0 < m1o;
  const bool live = row < 4 * nr;
  const int rr = live ? row : 4 * nr - 1;
  const int grp = rr / nr, idx = rr - grp * nr, ia = idx / m1, ib = idx - ia * m1;
  const double ga = cell.g[ia], gb = cell.g[ib];
  const double hx = 0.5 * cell.ex, hy = 0.5 * cell.ey, z0 = cell.z0;
  // the row pair's points: P1 - phase * P2 .. written as u(P2) - ph u(P1)
  double x1, y1, z1, x2, y2, z2;
  if (grp == 0) { x1 = -hx; y1 = hy * ga; z1 = z0 * gb; x2 = hx; y2 = y1; z2 = z1; }
  else if (grp == 1) { x1 = hx * ga; y1 = -hy; z1 = z0 * gb; x2 = x1; y2 = hy; z2 = z1; }
  else { x1 = hx * ga; y1 = hy * gb; z1 = grp == 2 ? z0 : -z0; x2 = x1; y2 = y1; z2 = z1; }
  const bool two = grp < 2;
  double2 ph = make_double2(0.0, 0.0);              // alpha or beta
  if (grp == 0) sincos(cell.kx * cell.ex, &ph.y, &ph.x);
  if (grp == 1) sincos(cell.ky * cell.ey, &ph.y, &ph.x);
  const QPoint P1 = q_point(x1, y1, z1, k), P2 = q_point(x2, y2, z2, k);
  double xm = fmax(k * P1.r, k * P2.r);
#pragma unroll
  for (int s = 16; s > 0; s >>= 1) xm = fmax(xm, __shfl_xor_sync(0xffffffffu, xm, s));
  const int L0 = p + (int)xm + 32;
  q_bessel(jl1, jn, L0, P2.ix, lane);               // the point every row uses
  if (__any_sync(0xffffffffu, two)) q_bessel(jl0, jn, L0, P1.ix, lane);
  if (has0) bt_coefficients(cf, m0, p, lane);
  if (has1) bt_coefficients(cf + 3 * (p + 1), m1o, p, lane);
  __syncwarp();
  const long long r0 = (long long)(2 * grp) * nr + idx, r1 = r0 + nr;   // value, derivative rows
  bool finite = true;
  for (int t = 0; t < 2; ++t) {
    if (!(t == 0 ? has0 : has1)) continue;
    const int m = t == 0 ? m0 : m1o;
    const double *ca = cf + t * 3 * (p + 1), *cb = ca + (p + 1), *cc = ca + 2 * (p + 1);
    double prod = 1.0 / (4.0 * 3.14159265358979323846);
    for (int u = 1; u <= m; ++u) prod *= (2.0 * u + 1.0) / (2.0 * u);
    const double pmm = (m & 1) ? -sqrt(prod) : sqrt(prod);
    // per point: Pbar recurrence state and E = e^{i m phi}
    double cur[2], prv[2], lct[2];
    double2 E[2];
    const QPoint *PP[2] = {&P1, &P2};
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const QPoint &P = *PP[q];
      double sp = 1.0;
      double2 e = make_double2(1.0, 0.0), base = make_double2(P.cp, P.sp);
      for (int u = m; u > 0; u >>= 1) {             // e^{i m phi}, sin(theta)^m by squaring
        if (u & 1) e = cmul2(e, base);
        base = cmul2(base, base);
      }
      for (int u = 0; u < m; ++u) sp *= P.st;
      cur[q] = pmm * sp;
      prv[q] = 0.0;
      lct[q] = m * P.ct;
      E[q] = e;
    }
    const double sgn = (m & 1) ? -1.0 : 1.0;
    for (int l = m; l <= p; ++l) {
      double2 val[2], der[2];
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        if (q == 0 && !two) continue;               // T and D rows have one point
        const QPoint &P = *PP[q];
        const double *jl = q == 0 ? jl0 : jl1;
        if (l > m) {
          const double nxt = ca[l] * fma(P.ct, cur[q], -cb[l] * prv[q]);
          prv[q] = cur[q];
          cur[q] = nxt;
          lct[q] += P.ct;
        }
        const double dP = fma(lct[q], cur[q], -cc[l] * prv[q]) * P.ist;
        const double j = jl[l * 32 + lane];
        const double dj = l == 0 ? -jl[32 + lane] : fma(-(l + 1.0) * P.ix, j, jl[(l - 1) * 32 + lane]);
        const double A = k * dj * cur[q], B = j * dP * P.ir, Cc = m * j * cur[q] * P.ir * P.ist;
        const double jp = j * cur[q];
        val[q] = make_double2(jp * E[q].x, jp * E[q].y);
        double2 w;                                  // the derivative's factor of E
        if (grp == 0) w = make_double2(fma(A, P.st, B * P.ct) * P.cp, -Cc * P.sp);
        else if (grp == 1) w = make_double2(fma(A, P.st, B * P.ct) * P.sp, Cc * P.cp);
        else w = make_double2(fma(A, P.ct, -B * P.st), 0.0);
        der[q] = cmul2(E[q], w);
      }
      // +m: u(P2) - ph u(P1); -m: (-1)^m (conj u(P2) - ph conj u(P1))
      double2 vp = val[1], dp2 = der[1], vm = make_double2(val[1].x, -val[1].y),
              dm = make_double2(der[1].x, -der[1].y);
      if (two) {
        const double2 a = cmul2(ph, val[0]), b = cmul2(ph, der[0]);
        const double2 ac = cmul2(ph, make_double2(val[0].x, -val[0].y));
        const double2 bc = cmul2(ph, make_double2(der[0].x, -der[0].y));
        vp = make_double2(vp.x - a.x, vp.y - a.y);
        dp2 = make_double2(dp2.x - b.x, dp2.y - b.y);
        vm = make_double2(vm.x - ac.x, vm.y - ac.y);
        dm = make_double2(dm.x - bc.x, dm.y - bc.y);
      }
      if (live) {
        const long long cpos = (long long)l * l + l + m, cneg = (long long)l * l + l - m;
        out[cpos * ld + r0] = vp;
        out[cpos * ld + r1] = dp2;
        if (m > 0) {
          out[cneg * ld + r0] = make_double2(sgn * vm.x, sgn * vm.y);
          out[cneg * ld + r1] = make_double2(sgn * dm.x, sgn * dm.y);
        }
        finite = finite && isfinite(vp.x + vp.y + dp2.x + dp2.y);
      }
    }
  }
  if (!finite) atomicOr(o.status, kStatNonFinite);
}

// W kernel: one warp per Rayleigh-Bloch column (the a's, then the b's), the
// lanes over rows; e^{i kap_x x_a} and e^{i kap_y y_b} formed once per
// column in shared memory, their products on the wall's nodes.
constexpr int kWWarps = 4;

__global__ void __launch_bounds__(32 * kWWarps)
q_w_kernel(const ObsDev *__restrict__ obs_arr, int oi, QCell cell, double2 *__restrict__ out, long long ld,
           long long col0) {
  const ObsDev &o = obs_arr[oi];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int m1 = cell.m1, nr = m1 * m1;
  const int c = blockIdx.x * kWWarps + warp;        // 0 .. 2 nrb - 1
  __shared__ double2 phx[kWWarps][kQMaxM1], phy[kWWarps][kQMaxM1];
  if (c >= 2 * cell.nrb) return;                    // whole warp; no block barriers below
  const bool top = c < cell.nrb;
  const int j = top ? c : c - cell.nrb;
  int mm = 0, nn = 0, acc = 0;                      // decode the mode: rows of m, each an n range
  for (int u = 0; u < cell.nrows; ++u) {
    if (j < acc + cell.rb_count[u]) { mm = cell.rb_m0 + u; nn = cell.rb_n0[u] + (j - acc); break; }
    acc += cell.rb_count[u];
  }
  const double kapx = cell.kx + 2.0 * 3.14159265358979323846 * mm / cell.ex;
  const double kapy = cell.ky + 2.0 * 3.14159265358979323846 * nn / cell.ey;
  const double kz2 = o.k * o.k - kapx * kapx - kapy * kapy;
  // i k_z with the principal root: real k_z when kz2 >= 0, else i sqrt(-kz2)
  const double2 ikz = kz2 >= 0.0 ? make_double2(0.0, sqrt(kz2)) : make_double2(-sqrt(-kz2), 0.0);
  const double hx = 0.5 * cell.ex, hy = 0.5 * cell.ey;
  for (int a = lane; a < m1; a += 32) {
    double s, cs;
    sincos(kapx * hx * cell.g[a], &s, &cs);
    phx[warp][a] = make_double2(cs, s);
    sincos(kapy * hy * cell.g[a], &s, &cs);
    phy[warp][a] = make_double2(cs, s);
  }
  __syncwarp();
  double2 *col = out + (col0 + c) * ld;
  const int b0 = top ? 4 : 6;                       // the wall's value and derivative blocks
  const double dsg = top ? -1.0 : 1.0;              // -i k_z on T, +i k_z on D
  for (int r = lane; r < 8 * nr; r += 32) {
    const int blk = r / nr, idx = r - blk * nr;
    double2 v = make_double2(0.0, 0.0);
    if (blk == b0 || blk == b0 + 1) {
      const int ia = idx / m1, ib = idx - ia * m1;
      const double2 e = cmul2(phx[warp][ia], phy[warp][ib]);
      v = blk == b0 ? make_double2(-e.x, -e.y) : cmul2(make_double2(dsg * ikz.x, dsg * ikz.y), e);
    }
    col[r] = v;
  }
}

// ---------------------------------------------------------------------------
// C, the periodizing rows applied to the ring part of eq. urep (Neumann
// obstacles): u = sum_{n,j} c_nj Phi^near_nj, Phi^near the 3 x 3 phased
// images of eq. Phinear, Phi_nj(x) = (1/P) sum_s G(x, y_j(2 pi s/P))
// e^{+i n 2 pi s/P} (the P point sources per ring of Sec. 4.1). With
// u(x) = sum_{a,b} alpha^a beta^b Psi(x - a e_x - b e_y) the near terms cancel
// between the walls of a pair (Sec. 4.1), leaving six distant ones:
//   u_R - alpha u_L = sum_b beta^b (alpha^-1 Psi(x_L + 2 e_x - b e_y)
//                                   - alpha^2 Psi(x_L - e_x - b e_y)),
//   u_F - beta u_B  = sum_a alpha^a (beta^-1 Psi(x_B - a e_x + 2 e_y)
//                                    - beta^2 Psi(x_B - a e_x - e_y)),
// and the same for the derivative rows; T and D keep all nine images. One
// warp per (row pair, ring j): per image point the lanes form the P samples
// of G and of one Cartesian derivative of G, two warp FFTs give every mode,
// and the image's coefficient times both is added in shared memory; the
// row pair's two rows are written for all P modes (column (n mod P) N + j).
// ---------------------------------------------------------------------------

constexpr int kCWarps = 4;

__global__ void __launch_bounds__(32 * kCWarps)
c_kernel(const ObsDev *__restrict__ obs_arr, int oi, QCell cell, double2 *__restrict__ out, long long ld) {
  const ObsDev &o = obs_arr[oi];
  const int P = o.P, N = o.N;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  extern __shared__ double2 c_sh[];
  double2 *tw = c_sh;                                           // [P] e^{-2 pi i r / P}
  int *perm = reinterpret_cast<int *>(c_sh + P);                // [P]
  double2 *ws = c_sh + P + (P + 1) / 2 + (size_t)warp * 4 * P;  // value, derivative, their sums
  double2 *sv = ws, *sd = ws + P, *av = ws + 2 * P, *ad = ws + 3 * P;
  const bool fft = o.fft_nst > 0;
  for (int i = threadIdx.x; i < P; i += blockDim.x) {
    tw[i] = o.tw_P[i];
    perm[i] = fft ? o.fft_perm[i] : i;
  }
  __syncthreads();
  const int m1 = cell.m1, nr = m1 * m1;
  const long long w = (long long)blockIdx.x * kCWarps + warp;   // row pair fastest, then ring
  if (w >= 4LL * nr * N) return;                                // whole warp; no block barriers below
  const int rp = (int)(w % (4LL * nr)), j = (int)(w / (4LL * nr));
  const int grp = rp / nr, idx = rp - grp * nr, ia = idx / m1, ib = idx - ia * m1;
  const double ga = cell.g[ia], gb = cell.g[ib];
  const double ex = cell.ex, ey = cell.ey, hx = 0.5 * ex, hy = 0.5 * ey, z0 = cell.z0;
  const double k = o.k, rs = o.src[2 * j], zs = o.src[2 * j + 1];
  const double wgt = 1.0 / (4.0 * 3.14159265358979323846 * P);
  double2 al, be;
  sincos(cell.kx * ex, &al.y, &al.x);
  sincos(cell.ky * ey, &be.y, &be.x);
  const double2 al_inv = make_double2(al.x, -al.y), be_inv = make_double2(be.x, -be.y);
  const double2 al2 = cmul2(al, al), be2 = cmul2(be, be);
  for (int n = lane; n < P; n += 32) {
    av[n] = make_double2(0.0, 0.0);
    ad[n] = make_double2(0.0, 0.0);
  }
  const int axis = grp == 0 ? 0 : grp == 1 ? 1 : 2;
  const int npts = grp < 2 ? 6 : 9;
  bool finite = true;
  for (int t = 0; t < npts; ++t) {
    double x, y, z;
    double2 cf;
    if (grp == 0) {                                  // b = t % 3 - 1; far right / far left images
      const int b = t % 3 - 1;
      const double2 bb = b < 0 ? be_inv : b > 0 ? be : make_double2(1.0, 0.0);
      const bool right = t < 3;
      x = right ? -hx + 2.0 * ex : -hx - ex;
      y = hy * ga - b * ey;
      z = z0 * gb;
      cf = right ? cmul2(al_inv, bb) : cmul2(make_double2(-al2.x, -al2.y), bb);
    } else if (grp == 1) {
      const int a = t % 3 - 1;
      const double2 aa = a < 0 ? al_inv : a > 0 ? al : make_double2(1.0, 0.0);
      const bool front = t < 3;
      x = hx * ga - a * ex;
      y = front ? -hy + 2.0 * ey : -hy - ey;
      z = z0 * gb;
      cf = front ? cmul2(aa, be_inv) : cmul2(aa, make_double2(-be2.x, -be2.y));
    } else {
      const int a = t / 3 - 1, b = t % 3 - 1;
      const double2 aa = a < 0 ? al_inv : a > 0 ? al : make_double2(1.0, 0.0);
      const double2 bb = b < 0 ? be_inv : b > 0 ? be : make_double2(1.0, 0.0);
      x = hx * ga - a * ex;
      y = hy * gb - b * ey;
      z = grp == 2 ? z0 : -z0;
      cf = cmul2(aa, bb);
    }
    for (int sidx = lane; sidx < P; sidx += 32) {
      // y_j(psi_s) = (rs cos psi_s, rs sin psi_s, zs); cos, sin from the twiddle table
      const double dx = x - rs * tw[sidx].x, dy = y + rs * tw[sidx].y, dz = z - zs;
      const double R2 = dx * dx + dy * dy + dz * dz;
      const double iR = rsqrt(R2), R = R2 * iR, kR = k * R;
      double sn, cs;
      sincos(kR, &sn, &cs);
      const double g = wgt * iR;
      sv[sidx] = make_double2(cs * g, sn * g);
      const double dc = axis == 0 ? dx : axis == 1 ? dy : dz;
      const double f = dc * g * iR * iR;               // (x - y)_c (ikR - 1) e^{ikR} / (4 pi P R^3)
      sd[sidx] = make_double2(f * fma(-kR, sn, -cs), f * fma(kR, cs, -sn));
    }
    __syncwarp();
    if (fft) {
      fft::warp_fft(sv, P, tw, o.fft_rad, o.fft_nst, lane);
      fft::warp_fft(sd, P, tw, o.fft_rad, o.fft_nst, lane);
      // sum_s a_s e^{+2 pi i n s / P} is the forward transform at -n mod P
      for (int n = lane; n < P; n += 32) {
        const int pos = perm[(P - n) % P];
        const double2 v = cmul2(cf, sv[pos]), d = cmul2(cf, sd[pos]);
        av[n] = make_double2(av[n].x + v.x, av[n].y + v.y);
        ad[n] = make_double2(ad[n].x + d.x, ad[n].y + d.y);
      }
    } else {                                          // direct sums for P with other prime factors
      for (int n = lane; n < P; n += 32) {
        double2 v = make_double2(0.0, 0.0), d = make_double2(0.0, 0.0);
        for (int sidx = 0; sidx < P; ++sidx) {
          const double2 e = make_double2(tw[((long long)n * sidx) % P].x, -tw[((long long)n * sidx) % P].y);
          v = make_double2(v.x + sv[sidx].x * e.x - sv[sidx].y * e.y, v.y + sv[sidx].x * e.y + sv[sidx].y * e.x);
          d = make_double2(d.x + sd[sidx].x * e.x - sd[sidx].y * e.y, d.y + sd[sidx].x * e.y + sd[sidx].y * e.x);
        }
        v = cmul2(cf, v);
        d = cmul2(cf, d);
        av[n] = make_double2(av[n].x + v.x, av[n].y + v.y);
        ad[n] = make_double2(ad[n].x + d.x, ad[n].y + d.y);
      }
    }
    __syncwarp();
  }
  const long long r0 = (long long)(2 * grp) * nr + idx, r1 = r0 + nr;
  for (int n = lane; n < P; n += 32) {
    const long long col = (long long)n * N + j;
    out[col * ld + r0] = av[n];
    out[col * ld + r1] = ad[n];
    finite = finite && isfinite(av[n].x + av[n].y + ad[n].x + ad[n].y);
  }
  if (!__all_sync(0xffffffffu, finite) && lane == 0) atomicOr(o.status, kStatNonFinite);
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

// Gauss-Legendre nodes on [-1, 1], ascending: Newton's method on P_n from
// cos(pi (i + 3/4) / (n + 1/2)), P_n and P_n' by the three-term recurrence.
static void gauss_legendre_nodes(int n, double *g) {
  for (int i = 0; i < n; ++i) {
    double x = std::cos(3.14159265358979323846 * (i + 0.75) / (n + 0.5));
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = x;
      for (int j = 2; j <= n; ++j) {
        const double p2 = ((2.0 * j - 1.0) * x * p1 - (j - 1.0) * p0) / j;
        p0 = p1;
        p1 = p2;
      }
      const double dp = n * (x * p1 - p0) / (x * x - 1.0);
      const double dx = p1 / dp;
      x -= dx;
      if (std::fabs(dx) < 1e-16) break;
    }
    g[n - 1 - i] = x;
  }
}

// The cell by value, with the Rayleigh-Bloch set |kappa| <= pi N0 enumerated
// by m, then n (kappa = (kx + 2 pi m / ex, ky + 2 pi n / ey)).
static bool make_qcell(const axi_cell &c, QCell &q) {
  if (c.m1 < 2 || c.m1 > kQMaxM1 || (c.m1 & 1) || c.p < 0 || c.p > AXI_BTILDE_MAX_DEGREE ||
      c.n0 < 0 || !(c.ex > 0.0) || !(c.ey > 0.0) || !(c.z0 > 0.0))
    return false;
  q.kx = c.kx; q.ky = c.ky; q.ex = c.ex; q.ey = c.ey; q.z0 = c.z0;
  q.p = c.p; q.m1 = c.m1; q.n0 = c.n0;
  gauss_legendre_nodes(c.m1, q.g);
  const double tp = 2.0 * 3.14159265358979323846, R = 3.14159265358979323846 * c.n0;
  const int mlo = (int)std::floor((-R - c.kx) * c.ex / tp) - 1, mhi = (int)std::ceil((R - c.kx) * c.ex / tp) + 1;
  const int nlo = (int)std::floor((-R - c.ky) * c.ey / tp) - 1, nhi = (int)std::ceil((R - c.ky) * c.ey / tp) + 1;
  if (mhi - mlo + 1 > kQMaxRows) return false;
  q.rb_m0 = mlo;
  q.nrows = mhi - mlo + 1;
  q.nrb = 0;
  for (int u = 0; u < q.nrows; ++u) {
    const double kx = c.kx + tp * (mlo + u) / c.ex;
    int first = 0, cnt = 0;
    for (int n = nlo; n <= nhi; ++n) {
      const double ky = c.ky + tp * n / c.ey;
      if (kx * kx + ky * ky <= R * R) {
        if (cnt == 0) first = n;
        ++cnt;
      }
    }
    q.rb_n0[u] = first;
    q.rb_count[u] = cnt;
    q.nrb += cnt;
  }
  return true;
}

bool q_shape(const axi_cell &c, long long &rows, long long &cols, long long &nrb) {
  static thread_local QCell q;
  if (!make_qcell(c, q)) return false;
  rows = 8LL * c.m1 * c.m1;
  nrb = q.nrb;
  cols = (long long)(c.p + 1) * (c.p + 1) + 2LL * q.nrb;
  return true;
}

bool q_modes(const axi_cell &c, int *mn, long long cap) {
  static thread_local QCell q;
  if (!make_qcell(c, q) || cap < q.nrb) return false;
  long long j = 0;
  for (int u = 0; u < q.nrows; ++u)
    for (int v = 0; v < q.rb_count[u]; ++v, ++j) {
      mn[2 * j] = q.rb_m0 + u;
      mn[2 * j + 1] = q.rb_n0[u] + v;
    }
  return true;
}

cudaError_t launch_q(const ObsDev *d_obs, const ObsDev &h, int oi, const axi_cell &c, double2 *out,
                     long long ld, cudaStream_t st) {
  static thread_local QCell q;
  if (!make_qcell(c, q)) return cudaErrorInvalidValue;
  const int p = q.p, jn = (p > 1 ? p : 1) + 1, nr = q.m1 * q.m1;
  // two warps per CTA while their Bessel tables fit, else one (large p)
  const size_t per_warp = sizeof(double) * (2 * (size_t)jn * 32 + 6 * (size_t)(p + 1));
  const int nw = 2 * per_warp <= (size_t)160 * 1024 ? kQWarps : 1;
  const size_t smem = per_warp * nw;
  static size_t granted = 0;
  cudaError_t e = ensure_dynamic_smem(q_s_kernel, smem, granted);
  if (e != cudaSuccess) return e;
  const dim3 grid((4 * nr + 31) / 32, (p / 2 + 1 + nw - 1) / nw);
  q_s_kernel<<<grid, 32 * nw, smem, st>>>(d_obs, oi, q, out, ld);
  e = cudaGetLastError();
  if (e != cudaSuccess || q.nrb == 0) return e;
  q_w_kernel<<<(2 * q.nrb + kWWarps - 1) / kWWarps, 32 * kWWarps, 0, st>>>(
      d_obs, oi, q, out, ld, (long long)(p + 1) * (p + 1));
  return cudaGetLastError();
}

bool c_shape(const ObsDev &h, const axi_cell &c, long long &rows, long long &cols) {
  static thread_local QCell q;
  if (!make_qcell(c, q)) return false;
  rows = 8LL * c.m1 * c.m1;
  cols = (long long)h.P * h.N;
  return true;
}

cudaError_t launch_c(const ObsDev *d_obs, const ObsDev &h, int oi, const axi_cell &c, double2 *out,
                     long long ld, cudaStream_t st) {
  static thread_local QCell q;
  if (!make_qcell(c, q)) return cudaErrorInvalidValue;
  const int P = h.P;
  const size_t smem = sizeof(double2) * ((size_t)P + (P + 1) / 2 + (size_t)kCWarps * 4 * P);
  static size_t granted = 0;
  cudaError_t e = ensure_dynamic_smem(c_kernel, smem, granted);
  if (e != cudaSuccess) return e;
  const long long warps = 4LL * q.m1 * q.m1 * h.N;
  c_kernel<<<(unsigned)((warps + kCWarps - 1) / kCWarps), 32 * kCWarps, smem, st>>>(d_obs, oi, q, out, ld);
  return cudaGetLastError();
}

}  // namespace axi
