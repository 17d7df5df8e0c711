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

}  // namespace trig
}  // namespace axi
