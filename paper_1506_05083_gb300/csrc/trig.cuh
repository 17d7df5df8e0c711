// sin and cos of one FP64 argument for the ring-kernel samples, written from
// the mathematics to spend fewer FP64 issue slots than the general library
// routine (which also covers huge arguments):
//   * Cody-Waite reduction: j = rint(x 2/pi) by the 1.5 * 2^52 rounding
//     trick, r = x - j pi/2 with pi/2 split into three doubles (computed to
//     300 bits with mpmath) and one FMA per part, so r is accurate to a few
//     units of 2^-53 for |x| < 2^20;
//   * Taylor series on |r| <= pi/4: sin through r^15 and cos through r^16
//     (truncation below 7e-17 relative), evaluated by Horner in r^2;
//   * the quadrant j mod 4 swaps and negates the pair with integer
//     instructions on the bit patterns.
// 23 FP64 operations. Valid for |x| < 2^20 (the samples use x = k R, far
// below that); tests/test_gpu_trig.py checks it against CUDA's sincos.
#pragma once
#include <cmath>
#include <cuda_runtime.h>

namespace axi {
namespace trig {

__device__ __forceinline__ void sincos_ring(double x, double *sp, double *cp) {
  constexpr double kRound = 6755399441055744.0;            // 1.5 * 2^52
  constexpr double kTwoOverPi = 0.6366197723675814;
  constexpr double kPio2_1 = 1.5707963267948966;
  constexpr double kPio2_2 = 6.123233995736766e-17;
  constexpr double kPio2_3 = -1.4973849048591698e-33;
  const double t = fma(x, kTwoOverPi, kRound);
  const double j = t - kRound;
  const unsigned q = (unsigned)__double2loint(t) & 3u;     // j mod 4
  double r = fma(-j, kPio2_1, x);
  r = fma(-j, kPio2_2, r);
  r = fma(-j, kPio2_3, r);
  const double z = r * r;
  // sin r = r + r z P(z),  P = -1/3! + z/5! - ... - z^6/15!
  double ps = fma(z, -1.0 / 1307674368000.0, 1.0 / 6227020800.0);
  ps = fma(z, ps, -1.0 / 39916800.0);
  ps = fma(z, ps, 1.0 / 362880.0);
  ps = fma(z, ps, -1.0 / 5040.0);
  ps = fma(z, ps, 1.0 / 120.0);
  ps = fma(z, ps, -1.0 / 6.0);
  const double s = fma(r * z, ps, r);
  // cos r = 1 - z/2 + z^2 Q(z),  Q = 1/4! - z/6! + ... + z^6/16!
  double pc = fma(z, 1.0 / 20922789888000.0, -1.0 / 87178291200.0);
  pc = fma(z, pc, 1.0 / 479001600.0);
  pc = fma(z, pc, -1.0 / 3628800.0);
  pc = fma(z, pc, 1.0 / 40320.0);
  pc = fma(z, pc, -1.0 / 720.0);
  pc = fma(z, pc, 1.0 / 24.0);
  const double c = fma(z * z, pc, fma(-0.5, z, 1.0));
  // quadrant: (sin, cos)(r + q pi/2) = (s, c), (c, -s), (-s, -c), (-c, s)
  long long sb = __double_as_longlong(s), cb = __double_as_longlong(c);
  const long long sw = (q & 1u) ? cb : sb;
  const long long cw = (q & 1u) ? sb : cb;
  const long long sgn = 1ll << 63;
  *sp = __longlong_as_double((q & 2u) ? sw ^ sgn : sw);
  *cp = __longlong_as_double(((q + 1u) & 2u) ? cw ^ sgn : cw);
}

// Table form for kernels that can hold a 16 KB table in shared memory:
//   x = j delta + r,  delta = 2 pi / 1024,  j = rint(x / delta),  |r| <= delta / 2,
// (cos, sin)(j delta) from the table (entry j mod 1024), sin r and cos r from
// three- and two-term Taylor series (|r| <= 0.00307: truncation below 2e-19
// relative), then the angle-addition formulas. delta's two Cody-Waite parts
// are the pi/2 parts above divided by 256 (exact); the third part would
// change r by less than 1e-26 for |x| < 2^20 and is dropped. 14 FP64
// operations; entries of the table are accurate to half a unit in the last
// place, so the result is within a few units of 2^-53 of the true value.
constexpr int kRingTab = 1024;

// (cos, sin)(2 pi i / 1024), i = 0 .. 1023, on the host.
inline void ring_table_host(double2 *tab) {
  const double twopi = 6.283185307179586476925286766559;
  for (int i = 0; i < kRingTab; ++i) {
    const double a = twopi * i / kRingTab;
    tab[i] = make_double2(std::cos(a), std::sin(a));
  }
}

__device__ __forceinline__ void sincos_ring_tab(double x, const double2 *__restrict__ tab, double *sp,
                                                double *cp) {
  constexpr double kRound = 6755399441055744.0;            // 1.5 * 2^52
  constexpr double kInvDelta = 162.97466172610083;         // 512 / pi
  constexpr double kDelta1 = 1.5707963267948966 / 256.0;   // exact scalings of the pi/2 parts
  constexpr double kDelta2 = 6.123233995736766e-17 / 256.0;
  const double t = fma(x, kInvDelta, kRound);
  const double j = t - kRound;
  const unsigned idx = (unsigned)__double2loint(t) & (kRingTab - 1);   // j mod 1024
  double r = fma(-j, kDelta1, x);
  r = fma(-j, kDelta2, r);
  const double z = r * r;
  const double s = fma(r * z, fma(z, 1.0 / 120.0, -1.0 / 6.0), r);  // sin r
  const double c = fma(z, fma(z, 1.0 / 24.0, -0.5), 1.0);            // cos r
  const double2 e = tab[idx];                                        // (cos, sin)(j delta)
  *sp = fma(s, e.x, c * e.y);
  *cp = fma(c, e.x, -(s * e.y));
}

}  // namespace trig
}  // namespace axi
