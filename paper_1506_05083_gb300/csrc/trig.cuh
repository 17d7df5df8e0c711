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
#include "ozaki.cuh"

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

// Fixed-point form of sincos_ring_tab for kernels bound by the FP64 pipe (on
// this part one FP64 warp instruction holds a sub-partition's FP64 unit for
// about 64 cycles, an integer one issues in one or two): the same reduction
// x = j delta + r in FP64 (four operations), then everything in 64-bit
// integers:
//   v = round(r 2^71) from r's bits (|r| <= delta / 2 < 2^-8.3);
//   sin r = r - r^3/6 + r^5/120 at 2^-71, cos r = 1 - r^2/2 + r^4/24 at 2^-62
//   (the next terms are below 2^-70 and 2^-59.5 of 1), products as the high
//   halves of signed 64 x 64-bit products (__mul64hi), 1/6, 1/20, 1/24 as
//   2^64-scaled constants;
//   the angle addition against a table of (cos, sin)(2 pi i / 1024) with 62
//   fractional bits (ring_table_q62.inc, rounded to nearest), giving sin x
//   and cos x with 60 fractional bits, about 2^-58 from the exact values of
//   the reduced argument; one rounding to double at the end (integer
//   instructions, no conversion unit).
// 4 FP64 operations instead of 14. The caller holds the table (1024 pairs of
// long long, 16 KB) in shared memory.
__device__ __forceinline__ long long fixed_from_double(double r, int frac_bits) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(r);
  const int E = (int)((b >> 52) & 0x7ff);
  unsigned long long M = b & 0xfffffffffffffull;
  int Ee = E;
  if (E == 0) Ee = 1; else M |= 1ull << 52;
  const int sh = Ee - 1075 + frac_bits;                // |r| 2^frac_bits = M 2^sh
  long long m;
  if (sh >= 0) m = (long long)(M << sh);                // callers keep this below 2^63
  else if (sh > -60) m = (long long)((M + (1ull << (-sh - 1))) >> (-sh));
  else m = 0;
  return (b >> 63) ? -m : m;
}

__device__ __forceinline__ void sincos_ring_q(double x, const longlong2 *__restrict__ tab, double *sp,
                                              double *cp) {
  constexpr double kRound = 6755399441055744.0;            // 1.5 * 2^52
  constexpr double kInvDelta = 162.97466172610083;         // 512 / pi
  constexpr double kDelta1 = 1.5707963267948966 / 256.0;
  constexpr double kDelta2 = 6.123233995736766e-17 / 256.0;
  constexpr long long kC6 = 3074457345618258603ll;         // round(2^64 / 6)
  constexpr long long kC20 = 922337203685477581ll;         // round(2^64 / 20)
  constexpr long long kC24 = 768614336404564651ll;         // round(2^64 / 24)
  const double t = fma(x, kInvDelta, kRound);
  const double j = t - kRound;
  const unsigned idx = (unsigned)__double2loint(t) & (kRingTab - 1);
  double r = fma(-j, kDelta1, x);
  r = fma(-j, kDelta2, r);
  const long long v = fixed_from_double(r, 71);           // r 2^71
  const long long v2 = __mul64hi(v, v);                   // r^2 2^78
  const long long s3 = __mul64hi(__mul64hi(v2, v), kC6);  // r^3/6 2^85
  const long long s5 = __mul64hi(__mul64hi(s3, v2), kC20);   // r^5/120 2^99
  const long long sr = v - (s3 >> 14) + (s5 >> 28);      // sin r 2^71
  const long long c4 = __mul64hi(__mul64hi(v2, v2), kC24) >> 30;   // r^4/24 2^62
  const long long cr = (1ll << 62) - (v2 >> 17) + c4;    // cos r 2^62
  const longlong2 e = tab[idx];                           // (cos, sin)(j delta) 2^62
  const long long sn = __mul64hi(e.y, cr) + (__mul64hi(e.x, sr) >> 9);   // 2^60
  const long long cs = __mul64hi(e.x, cr) - (__mul64hi(e.y, sr) >> 9);
  *sp = oz::scaled_to_double(sn, -60);
  *cp = oz::scaled_to_double(cs, -60);
}

}  // namespace trig
}  // namespace axi
