// Host-side discretisation of the generating curve (step A1 of the path).
//
// Sec. 3: the body is the rotation of gamma = (rho(t), z(t)), t in [0, pi],
// about the z axis. Collocation points sit at t_m = pi (m - 1/2) / M.
// Sec. 3.2, scheme (c): proxies are obtained by complexifying the
// parametrisation, y_j = gamma(t_j + i tau), t_j = pi (j - 1/2) / N; we
// identify (z, rho) with zeta = z + i rho so that the complexified point is
// zeta(t_j + i s tau) read back as (rho', z') = (Im, Re). The sign s makes
// the proxies fall inside the body (for the sphere s = +1 gives radius
// e^{-tau}); exterior proxies of the transmission problem (Sec. 3.4) use -tau.
// Shapes: Fig. 2 caption (polar bodies and the erf-rounded cup).
#include <cmath>
#include <complex>
#include <vector>

#include "../../include/axi_mfs.h"

namespace {

using cd = std::complex<double>;
constexpr double kPi = 3.14159265358979323846;

// Complex error function for the cup's complexified parameter.
// |z| <= 3.5: erf(z) = (2/sqrt(pi)) e^{-z^2} sum_n 2^n z^{2n+1} / (2n+1)!!
//   (Abramowitz & Stegun 7.1.6; terms stay in phase for small Im z).
// otherwise:  erfc(z) = e^{-z^2}/sqrt(pi) * 1/(z + (1/2)/(z + 1/(z + (3/2)/(z + ...))))
//   (Laplace continued fraction, A&S 7.1.14), evaluated bottom-up, for Re z > 0;
//   erf(-z) = -erf(z) covers Re z < 0.
cd erf_c(cd z) {
  if (z.real() < 0.0) return -erf_c(-z);
  const double two_over_sqrtpi = 1.12837916709551257390;
  if (std::abs(z) <= 3.5) {
    cd term = z, sum = z, z2 = z * z;
    for (int n = 0; n < 200; ++n) {
      term *= 2.0 * z2 / double(2 * n + 3);
      sum += term;
      if (std::abs(term) < 1e-18 * std::abs(sum)) break;
    }
    return two_over_sqrtpi * std::exp(-z2) * sum;
  }
  cd f = z;
  for (int n = 80; n >= 1; --n) f = z + (0.5 * n) / f;
  cd erfc = std::exp(-z * z) / (std::sqrt(kPi) * f);
  return 1.0 - erfc;
}

struct Curve {
  int shape;
  const double *p;
  int np;
  // zeta(t) = z(t) + i rho(t) and dzeta/dt for complex t.
  void eval(cd t, cd &zeta, cd &dzeta) const {
    if (shape == AXI_SHAPE_POLAR) {
      cd r = p[0], dr = 0.0;
      for (int j = 1; j < np; ++j) {
        r += p[j] * std::cos(double(j) * t);
        dr -= p[j] * double(j) * std::sin(double(j) * t);
      }
      cd e = std::exp(cd(0, 1) * t);
      zeta = r * e;
      dzeta = (dr + cd(0, 1) * r) * e;
    } else {
      const double a = p[0], b = p[1];
      cd x = t - kPi / 2;
      cd er = erf_c(x / a);
      cd g = std::exp(-(x / a) * (x / a));
      cd r = 1.0 - a * er;
      cd dr = -(2.0 / std::sqrt(kPi)) * g;
      double c = 2.0 * (1.0 - (b - a) / kPi);
      cd sa = (a / std::sqrt(kPi)) * g + x * er;
      cd th = b - a + c * sa;
      cd dth = c * er;
      cd e = std::exp(cd(0, 1) * th);
      zeta = r * e;
      dzeta = (dr + cd(0, 1) * r * dth) * e;
    }
  }
};

// +1 when gamma runs counter-clockwise in the (z, rho) plane (closed along
// the axis), i.e. the body lies to the left of the direction of travel.
double orientation(const Curve &c) {
  const int n = 4096;
  double area = 0.0, z0 = 0, r0 = 0, zp = 0, rp = 0;
  for (int i = 0; i < n; ++i) {
    cd zeta, dz;
    c.eval(cd(kPi * i / (n - 1), 0.0), zeta, dz);
    double z = zeta.real(), r = zeta.imag();
    if (i == 0) { z0 = z; r0 = r; }
    else area += zp * r - z * rp;
    zp = z; rp = r;
  }
  area += zp * r0 - z0 * rp;
  return area > 0 ? 1.0 : -1.0;
}

bool is_fin(double x) { return std::isfinite(x); }

}  // namespace

extern "C" axi_status axi_geometry(int32_t shape, const double *h_params, int32_t n_params,
                                   int32_t M, int32_t N, double tau, double *h_coll,
                                   double *h_src, double *h_src_ext) {
  if (!h_params || !h_coll || !h_src) return AXI_ERR_ARG;
  if (shape == AXI_SHAPE_POLAR) {
    if (n_params < 1) return AXI_ERR_ARG;
  } else if (shape == AXI_SHAPE_CUP) {
    if (n_params < 2 || !(h_params[0] > 0)) return AXI_ERR_ARG;
  } else {
    return AXI_ERR_ARG;
  }
  if (M < 1 || N < 1) return AXI_ERR_SHAPE;
  Curve c{shape, h_params, n_params};
  const double s = orientation(c);
  for (int m = 0; m < M; ++m) {
    double t = kPi * (m + 0.5) / M;
    cd zeta, dz;
    c.eval(cd(t, 0.0), zeta, dz);
    cd nrm = s * (cd(0, -1) * dz) / std::abs(dz);
    double *o = h_coll + 4 * m;
    o[0] = zeta.imag(); o[1] = zeta.real(); o[2] = nrm.imag(); o[3] = nrm.real();
    for (int i = 0; i < 4; ++i) if (!is_fin(o[i])) return AXI_ERR_GEOMETRY;
  }
  for (int j = 0; j < N; ++j) {
    double t = kPi * (j + 0.5) / N;
    cd zeta, dz;
    c.eval(cd(t, s * tau), zeta, dz);
    h_src[2 * j] = zeta.imag();
    h_src[2 * j + 1] = zeta.real();
    if (!(h_src[2 * j] > 0) || !is_fin(h_src[2 * j + 1])) return AXI_ERR_GEOMETRY;
    if (h_src_ext) {
      c.eval(cd(t, -s * tau), zeta, dz);
      h_src_ext[2 * j] = zeta.imag();
      h_src_ext[2 * j + 1] = zeta.real();
      if (!(h_src_ext[2 * j] > 0) || !is_fin(h_src_ext[2 * j + 1])) return AXI_ERR_GEOMETRY;
    }
  }
  return AXI_OK;
}

namespace {
bool smooth235(int n) {
  for (int p : {2, 3, 5}) while (n % p == 0) n /= p;
  return n == 1;
}
double min_rate(int M, int N, const double *coll, const double *src) {
  double best = INFINITY;
  for (int m = 0; m < M; ++m) {
    const double rho = coll[4 * m], z = coll[4 * m + 1];
    for (int j = 0; j < N; ++j) {
      const double rs = src[2 * j], zs = src[2 * j + 1];
      const double d2 = (rho - rs) * (rho - rs) + (z - zs) * (z - zs);
      // Theorem 1: alpha = Im acos(1 + d^2/(2 rho rho')) = acosh(...)
      const double a = std::acosh(1.0 + d2 / (2.0 * rho * rs));
      if (a < best) best = a;
    }
  }
  return best;
}
}  // namespace

extern "C" axi_status axi_choose_q(int32_t M, int32_t N, int32_t P, const double *h_coll,
                                   const double *h_src, const double *h_src_ext, int32_t *q) {
  if (!h_coll || !h_src || !q) return AXI_ERR_ARG;
  if (M < 1 || N < 1 || P < 2 || (P & 1)) return AXI_ERR_SHAPE;
  double al = min_rate(M, N, h_coll, h_src);
  if (h_src_ext) al = std::fmin(al, min_rate(M, N, h_coll, h_src_ext));
  if (!(al > 0) || !std::isfinite(al)) return AXI_ERR_GEOMETRY;
  double lo = std::fmax(2.0 * P, 37.0 / al + P / 2.0);
  int n = (int)std::ceil(lo);
  if (n < 2) n = 2;
  while (!(n % 2 == 0 && smooth235(n))) ++n;
  *q = n;
  return AXI_OK;
}

// Sub-grid stride of each ring pair's fill samples (Sec. 3.1, Theorem 1):
// the largest s in {4, 2, 1} with (q/2) mod s = 0 and
//   q/s >= max(P, 37/alpha + P/2),  alpha = acosh(1 + d^2/(2 rho rho')),
// the pair's own convergence rate, so that the q/s-node trapezoid rule of the
// pair meets the accuracy the q-node rule was chosen for.
extern "C" axi_status axi_fill_subgrid(int32_t M, int32_t N, int32_t P, int32_t q,
                                       const double *h_coll, const double *h_src,
                                       uint8_t *h_stride) {
  if (!h_coll || !h_src || !h_stride) return AXI_ERR_ARG;
  if (M < 1 || N < 1 || P < 2 || (P & 1) || q < P || (q & 1)) return AXI_ERR_SHAPE;
  for (int m = 0; m < M; ++m) {
    const double rho = h_coll[4 * m], z = h_coll[4 * m + 1];
    for (int j = 0; j < N; ++j) {
      const double rs = h_src[2 * j], zs = h_src[2 * j + 1];
      const double d2 = (rho - rs) * (rho - rs) + (z - zs) * (z - zs);
      const double alpha = std::acosh(1.0 + d2 / (2.0 * rho * rs));
      if (!(alpha > 0)) return AXI_ERR_GEOMETRY;
      const double need = std::fmax((double)P, 37.0 / alpha + P / 2.0);
      int sg = 1;
      for (int c : {4, 2})
        if ((q / 2) % c == 0 && (double)(q / c) >= need) { sg = c; break; }
      h_stride[(size_t)m * N + j] = (uint8_t)sg;
    }
  }
  return AXI_OK;
}
