// Step A3's Householder panel (Sec. 3: unpivoted, backward-stable QR of each
// mode's least-squares matrix) for split plans, in 58-bit fixed point.
//
// The FP64 panel of qr.cu is bound by the FP64 pipe, which on this part
// retires about two FP64 operations per clock per SM against 64 lanes of
// 32-bit integer multiply-add. This kernel factors the same panel (same
// reflector convention, same T) with integer arithmetic in the row sweep and
// FP64 only for the per-column scalars:
//
//   * Column c of the panel (rows k0.. of the mode's matrix, K rows) is held
//     as X = round(a 2^{58 - E_c}), with 2^{E_c} above the column's 2-norm
//     (largest entry times sqrt(K), rounded up to a power of two). The
//     reflectors H_j are unitary on the rows they touch, so every entry stays
//     below the column norm: |X| <= 2^58 all through the panel. Reflector
//     columns are held as V = round(v 2^58) (|v| <= 1: v = x / (alpha - beta)
//     and |alpha - beta| >= |beta| >= ||x||).
//   * A 58-bit value is split as X = h 2^29 + l (|h| <= 2^29, |l| <= 2^28),
//     and a product as h h' 2^58 + (h l' + l h') 2^29 + l l', four 32 x 32
//     -> 64-bit multiply-adds (mad.wide.s32).
//   * The sums of a column step (||x||^2, x^H a_c, v_a^H x) are EXACT: each
//     thread keeps a sum as a1 2^58 + a2 in two 64-bit integers, the warp
//     and CTA reductions add integers, and the scalars convert the exact
//     sums to FP64 once. A sum whose terms cancel keeps its full relative
//     precision, as the FP64 sums would to rounding.
//   * The updates a_c - v w_c (w_c = conj(tau) v^H a_c, held as
//     round(w_c 2^{58 - E_c}), |w_c| <= 2 ||a_c||) drop the l l' term and
//     round once: an error below one unit of 2^{E_c - 58}, i.e. 2^-58 of the
//     column norm, where an FP64 update errs by about 2^-53 of it.
//   * v = x scale is formed from the scalar's 58-bit mantissa in 128-bit
//     products and rounded once to 2^-58.
// The scalars (alpha, ||x||, beta, tau, 1/(alpha - beta), the w_c and the
// Gram entries for T) and T itself are FP64 as in qr.cu; beta is kept in
// FP64 and written back as R's diagonal. Integer sums are independent of
// their order, so the factors do not depend on the thread count.
// It is a tuning choice (panel_fixed 2), not the default: the sums of a
// column step take 255 registers, so only one or two warps per SM
// sub-partition run the sweep, and they issue on under a fifth of the
// cycles (dependency latency); the panel then takes about as long as the
// FP64 one, which keeps the FP64 pipe busy from the same single warp.
#include "axi_internal.h"
#include "ozaki.cuh"

namespace axi {
namespace {

constexpr int kQ = 58;                               // fraction bits of a column's values
constexpr long long kMask29 = (1ll << 29) - 1;
constexpr long long kMask58 = (1ll << 58) - 1;
constexpr int kX = kNB - 1;                          // complex partial sums per column step

// d = a b + c with a 32 x 32 -> 64-bit signed product
__device__ __forceinline__ long long mw(int a, int b, long long c) {
  long long d;
  asm("mad.wide.s32 %0, %1, %2, %3;" : "=l"(d) : "r"(a), "r"(b), "l"(c));
  return d;
}

// x = h 2^29 + l, l the low 29 bits sign-extended (|l| <= 2^28)
__device__ __forceinline__ void split29(long long x, int &h, int &l) {
  l = ((int)((unsigned)x << 3)) >> 3;
  h = (int)((x - (long long)l) >> 29);
}

// A complex value split per component; the negated parts serve the
// imaginary halves of conjugated products.
struct Sp {
  int rh, rl, ih, il;
};
struct SpN {
  int rh, rl, ih, il, nrh, nrl, nih, nil;
};
__device__ __forceinline__ Sp split(longlong2 x) {
  Sp s;
  split29(x.x, s.rh, s.rl);
  split29(x.y, s.ih, s.il);
  return s;
}
__device__ __forceinline__ SpN splitn(longlong2 x) {
  SpN s;
  split29(x.x, s.rh, s.rl);
  split29(x.y, s.ih, s.il);
  s.nrh = -s.rh; s.nrl = -s.rl; s.nih = -s.ih; s.nil = -s.il;
  return s;
}
__device__ __forceinline__ longlong2 join(int4 s) {
  return make_longlong2(((long long)s.x << 29) + s.y, ((long long)s.z << 29) + s.w);
}

// An exact sum a1 2^58 + a2 (a2 kept below 2^62 between normalisations).
struct Acc {
  long long a1, a2;
};
__device__ __forceinline__ void fold_mid(Acc &s, long long m) {
  s.a1 += m >> 29;                       // floor; the low 29 bits go to a2
  s.a2 += (m & kMask29) << 29;
}
// s += Re(conj(a) b), t += Im(conj(a) b) exactly, with b's real part negated
// in bn (Im(conj(a) b) = ar bi + ai (-br)).
__device__ __forceinline__ void mac_conj_b(Acc &s, Acc &t, int arh, int arl, int aih, int ail,
                                           const SpN &b) {
  s.a1 = mw(arh, b.rh, s.a1);
  s.a1 = mw(aih, b.ih, s.a1);
  long long m = mw(arh, b.rl, 0);
  m = mw(arl, b.rh, m);
  m = mw(aih, b.il, m);
  m = mw(ail, b.ih, m);
  s.a2 = mw(arl, b.rl, s.a2);
  s.a2 = mw(ail, b.il, s.a2);
  fold_mid(s, m);
  t.a1 = mw(arh, b.ih, t.a1);
  t.a1 = mw(aih, b.nrh, t.a1);
  m = mw(arh, b.il, 0);
  m = mw(arl, b.ih, m);
  m = mw(aih, b.nrl, m);
  m = mw(ail, b.nrh, m);
  t.a2 = mw(arl, b.il, t.a2);
  t.a2 = mw(ail, b.nrl, t.a2);
  fold_mid(t, m);
}
// the same with a's imaginary part negated in a (Im = ar bi + (-ai) br)
__device__ __forceinline__ void mac_conj_a(Acc &s, Acc &t, const SpN &a, const Sp &b) {
  s.a1 = mw(a.rh, b.rh, s.a1);
  s.a1 = mw(a.ih, b.ih, s.a1);
  long long m = mw(a.rh, b.rl, 0);
  m = mw(a.rl, b.rh, m);
  m = mw(a.ih, b.il, m);
  m = mw(a.il, b.ih, m);
  s.a2 = mw(a.rl, b.rl, s.a2);
  s.a2 = mw(a.il, b.il, s.a2);
  fold_mid(s, m);
  t.a1 = mw(a.rh, b.ih, t.a1);
  t.a1 = mw(a.nih, b.rh, t.a1);
  m = mw(a.rh, b.il, 0);
  m = mw(a.rl, b.ih, m);
  m = mw(a.nih, b.rl, m);
  m = mw(a.nil, b.rh, m);
  t.a2 = mw(a.rl, b.il, t.a2);
  t.a2 = mw(a.nil, b.rl, t.a2);
  fold_mid(t, m);
}
// s += |a|^2 exactly
__device__ __forceinline__ void mac_abs2(Acc &s, const SpN &a) {
  s.a1 = mw(a.rh, a.rh, s.a1);
  s.a1 = mw(a.ih, a.ih, s.a1);
  long long m = mw(2 * a.rh, a.rl, 0);
  m = mw(2 * a.ih, a.il, m);
  s.a2 = mw(a.rl, a.rl, s.a2);
  s.a2 = mw(a.il, a.il, s.a2);
  fold_mid(s, m);
}

// y <- y - v w, with w given as the split of -w (nw) and of Im w (wi):
//   Re: v_r (-w_r) + v_i w_i,   Im: v_r (-w_i) + v_i (-w_r);
// the l l' terms are dropped and the middle terms rounded once (the 2^28
// start), so the result errs by less than one unit.
__device__ __forceinline__ void upd(longlong2 &y, const Sp &v, int4 nw, int2 wi) {
  y.x = mw(v.rh, nw.x, y.x);
  y.x = mw(v.ih, wi.x, y.x);
  long long m = mw(v.rh, nw.y, 1ll << 28);
  m = mw(v.rl, nw.x, m);
  m = mw(v.ih, wi.y, m);
  m = mw(v.il, wi.x, m);
  y.x += m >> 29;
  y.y = mw(v.rh, nw.z, y.y);
  y.y = mw(v.ih, nw.x, y.y);
  m = mw(v.rh, nw.w, 1ll << 28);
  m = mw(v.rl, nw.z, m);
  m = mw(v.ih, nw.y, m);
  m = mw(v.il, nw.x, m);
  y.y += m >> 29;
}

// round(p 2^-sh) for a 128-bit p; sh <= 0 shifts left, exactly, by at most
// 60 places (the caller's result is below 2^59, so p is small there)
__device__ __forceinline__ long long shr_round(__int128 p, int sh) {
  if (sh <= 0) return (long long)(p << (sh < -60 ? 60 : -sh));
  if (sh >= 126) return 0;
  return (long long)((p + ((__int128)1 << (sh - 1))) >> sh);
}

// the full 128-bit product of two signed 64-bit integers
__device__ __forceinline__ __int128 mul128(long long a, long long b) {
  const unsigned long long lo = (unsigned long long)a * (unsigned long long)b;
  const long long hi = __mul64hi(a, b);
  return (__int128)(((unsigned __int128)(unsigned long long)hi << 64) | lo);
}

// v (2^58 units) = x s 2^-sh for a complex 58-bit mantissa s
__device__ __forceinline__ longlong2 mul_scalar(longlong2 x, longlong2 s, int sh) {
  const __int128 pr = mul128(x.x, s.x) - mul128(x.y, s.y);
  const __int128 pi = mul128(x.x, s.y) + mul128(x.y, s.x);
  return make_longlong2(shr_round(pr, sh), shr_round(pi, sh));
}

// (a1 2^58 + a2) 2^e as the nearest double (to within one rounding of a
// 62-bit intermediate), integer instructions only
__device__ __forceinline__ double acc_to_double(long long a1, long long a2, int e) {
  const __int128 v = ((__int128)a1 << 58) + a2;
  const long long lo = (long long)v;
  if ((long long)(v >> 64) == (lo >> 63)) return oz::scaled_to_double(lo, e);
  const unsigned __int128 u = v < 0 ? (unsigned __int128)(-v) : (unsigned __int128)v;
  const unsigned long long hi = (unsigned long long)(u >> 64);
  const int L = hi ? 128 - __clzll((long long)hi) : 64 - __clzll((long long)(unsigned long long)u);
  const int s = L - 62;
  long long t = (long long)((u + ((unsigned __int128)1 << (s - 1))) >> s);
  if (v < 0) t = -t;
  return oz::scaled_to_double(t, e + s);
}

// round(x 2^{58 - e}) for |x| < 2^{e + 2}
__device__ __forceinline__ long long to_fx(double x, int e) {
  unsigned sgn;
  const long long m = (long long)oz::mag_fixed(x, e, kQ, sgn);
  return sgn ? -m : m;
}

__device__ __forceinline__ double fx_to_double(long long x, int e) {
  return oz::scaled_to_double(x, e - kQ);
}

// Reduce-scatter of 16 exact sums (a1, a2 with 0 <= a2 < 2^58) over the
// warp: afterwards lanes 2k and 2k + 1 hold the warp-wide sum of value k
// (a2 below 2^63). Four halving levels and one exchange between lane pairs:
// the sums of a column step go through in two batches, which keeps half as
// many of them live at once.
__device__ __forceinline__ void reduce_scatter16(long long (&a1)[16], long long (&a2)[16],
                                                 long long &o1, long long &o2) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 16, n = 8; o >= 2; o >>= 1, n >>= 1) {
    const bool upper = (lane & o) != 0;
#pragma unroll
    for (int i = 0; i < n; ++i) {
      const long long s1 = upper ? a1[i] : a1[i + n], k1 = upper ? a1[i + n] : a1[i];
      const long long s2 = upper ? a2[i] : a2[i + n], k2 = upper ? a2[i + n] : a2[i];
      a1[i] = k1 + __shfl_xor_sync(0xffffffffu, s1, o);
      a2[i] = k2 + __shfl_xor_sync(0xffffffffu, s2, o);
    }
  }
  o1 = a1[0] + __shfl_xor_sync(0xffffffffu, a1[0], 1);
  o2 = a2[0] + __shfl_xor_sync(0xffffffffu, a2[0], 1);
}

__device__ __forceinline__ double2 cmulf(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cfmaf(double2 acc, double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, fma(-a.y, b.y, acc.x)), fma(a.x, b.y, fma(a.y, b.x, acc.y)));
}
__device__ __forceinline__ double2 cfma_conjf(double2 acc, double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, fma(a.y, b.y, acc.x)), fma(a.x, b.y, fma(-a.y, b.x, acc.y)));
}

}  // namespace
}  // namespace axi

namespace axi {
namespace {

// One CTA of NT threads per (obstacle, mode) task; thread t owns the rows
// t, t + NT, ... of the panel (K = rows - k0 rows, all in shared memory).
// Per column jj: the exact partial sums of the previous sweep are reduced
// (warp reduce-scatter, then warp 0 over the warps); warp 0 forms the FP64
// scalars and, for every later column c, w_c as a 58-bit fixed-point
// number; one sweep then forms v = x scale, applies H_jj to the later
// columns and accumulates the sums for column jj + 1:
//   ||x||^2, P_c = x^H a_c (c > jj + 1), Q_a = v_a^H x (a <= jj)
// (the Gram entries G(a, jj + 1) = conj(v_a[jj + 1]) + scale Q_a of T).
template <int NT>
__global__ void __launch_bounds__(NT)
qr_panel_fx_kernel(const ObsDev *__restrict__ obs, const int *__restrict__ task_obs,
                   const int *__restrict__ task_mode, int p) {
  constexpr int kW = NT / 32;
  const int task = blockIdx.x;
  const ObsDev &o = obs[task_obs[task]];
  const int d = task_mode[task];
  const int lda = o.rows;
  const int k0 = p * kNB;
  const int nbp = min(kNB, o.cols - k0);
  const int K = o.rows - k0;
  double2 *A = o.A + (size_t)d * o.cols * lda;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // [nbp][K]: column c holds X (rows <= c) and, once H_c is formed, the
  // split V (rows > c, read as int4); FP64 values before and after
  extern __shared__ longlong2 Pf[];
  int4 *Pv = reinterpret_cast<int4 *>(Pf);
  double2 *Pd = reinterpret_cast<double2 *>(Pf);
  __shared__ long long red1[kW][32], red2[kW][32];
  __shared__ long long tot1[32], tot2[32];
  __shared__ unsigned long long wkey[kW][kNB];
  __shared__ int colE[kNB];
  __shared__ int4 wn4[kX];                      // split of -w_c, c = x + 1
  __shared__ int2 wi2[kX];                      // split of Im w_c
  __shared__ longlong2 svS;                     // 2^{E_jj} scale = svS 2^{-svSh}
  __shared__ int svSh;
  __shared__ double2 Gsh[kNB][kNB];             // Gsh[a][j] = v_a^H v_j, a < j
  __shared__ double2 Tsh[kNB][kNB + 1];
  __shared__ double2 taush[kNB];
  __shared__ double betash[kNB];

  auto t_column = [&](int j) {                  // column j of T, as in qr.cu
    const double2 tj = taush[j];
    if (lane < j) {
      double2 z = make_double2(0.0, 0.0);
      for (int l = lane; l < j; ++l) z = cfmaf(z, Tsh[lane][l], Gsh[l][j]);
      const double2 t = cmulf(tj, z);
      Tsh[lane][j] = make_double2(-t.x, -t.y);
    } else if (lane == j) {
      Tsh[j][j] = tj;
    }
  };

  // load, with the largest component of each column
  {
    unsigned long long m[kNB];
#pragma unroll
    for (int a = 0; a < kNB; ++a) m[a] = 0ull;
    for (int i = tid; i < K; i += NT) {
#pragma unroll
      for (int a = 0; a < kNB; ++a) {
        if (a >= nbp) break;
        const double2 v = A[(size_t)(k0 + a) * lda + k0 + i];
        Pd[a * K + i] = v;
        const unsigned long long k = oz::abs_key2(v);
        m[a] = k > m[a] ? k : m[a];
      }
    }
#pragma unroll
    for (int a = 0; a < kNB; ++a) {
#pragma unroll
      for (int s = 16; s > 0; s >>= 1) {
        const unsigned long long w = __shfl_xor_sync(0xffffffffu, m[a], s);
        m[a] = w > m[a] ? w : m[a];
      }
      if (lane == 0) wkey[warp][a] = m[a];
    }
  }
  for (int e = tid; e < kNB * (kNB + 1); e += NT) (&Tsh[0][0])[e] = make_double2(0.0, 0.0);
  __syncthreads();
  if (tid < kNB) {
    unsigned long long m = 0ull;
    for (int w = 0; w < kW; ++w) m = wkey[w][tid] > m ? wkey[w][tid] : m;
    // ||a_c|| <= sqrt(2 K) max |component| < 2^{e + h}, 4^h >= 2 K
    const int bits = 32 - __clz(2 * K - 1);
    colE[tid] = oz::key_exponent(m) + ((bits + 1) >> 1);
  }
  __syncthreads();
  for (int e = tid; e < nbp * K; e += NT) {
    const int Ec = colE[e / K];
    const double2 v = Pd[e];
    Pf[e] = make_longlong2(to_fx(v.x, Ec), to_fx(v.y, Ec));
  }
  __syncthreads();

  // exact sums for column 0: slot x holds P_{x+1}
  Acc pr[kX], pi[kX], qr, qi, xn2;
#pragma unroll
  for (int x = 0; x < kX; ++x) pr[x] = pi[x] = Acc{0, 0};
  qr = qi = xn2 = Acc{0, 0};
  int qslot = -1;                               // slot whose sums are in (qr, qi)
  for (int i = tid; i < K; i += NT) {
    if (i == 0) continue;
    const SpN xs = splitn(Pf[i]);
    mac_abs2(xn2, xs);
#pragma unroll
    for (int x = 0; x < kX; ++x) {
      if (x + 1 >= nbp) break;
      mac_conj_a(pr[x], pi[x], xs, split(Pf[(x + 1) * K + i]));
    }
  }

  for (int jj = 0; jj < nbp; ++jj) {
    {
      // slots: (Re, Im) of partial x at 2x, 2x + 1, ||x||^2 at 30; each
      // normalised to 0 <= a2 < 2^58, reduced in two batches of 16
#pragma unroll
      for (int b = 0; b < 2; ++b) {
        long long v1[16], v2[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) {
          const int slot = 16 * b + k, x = slot >> 1;
          Acc r;
          if (slot == 30) r = xn2;
          else if (slot == 31) r = Acc{0, 0};
          else if (slot & 1) r = x == qslot ? qi : pi[x];    // slot qslot holds no other sum:
          else r = x == qslot ? qr : pr[x];                   // select, not add
          v1[k] = r.a1 + (r.a2 >> 58);
          v2[k] = r.a2 & kMask58;
        }
        long long o1, o2;
        reduce_scatter16(v1, v2, o1, o2);
        if ((lane & 1) == 0) {
          red1[warp][16 * b + (lane >> 1)] = o1 + (o2 >> 58);
          red2[warp][16 * b + (lane >> 1)] = o2 & kMask58;
        }
      }
    }
    __syncthreads();                                           // sums of column jj
    if (warp == 1 && jj > 0) t_column(jj - 1);                 // beside warp 0's scalars
    if (warp == 0) {
      long long s1 = 0, s2 = 0;
#pragma unroll
      for (int w = 0; w < kW; ++w) {
        s1 += red1[w][lane];
        s2 += red2[w][lane];
      }
      tot1[lane] = s1;
      tot2[lane] = s2;
      __syncwarp();
      const int Ej = colE[jj];
      const double xn2d = acc_to_double(tot1[30], tot2[30], 2 * Ej - 2 * kQ);
      const longlong2 ax = Pf[jj * K + jj];
      const double2 alpha = make_double2(fx_to_double(ax.x, Ej), fx_to_double(ax.y, Ej));
      double beta;
      double2 tau, scale;
      if (xn2d == 0.0 && alpha.y == 0.0) {
        beta = alpha.x; tau = make_double2(0.0, 0.0); scale = make_double2(0.0, 0.0);
      } else {
        const double s2d = fma(alpha.x, alpha.x, fma(alpha.y, alpha.y, xn2d));
        const double rs = rsqrt(s2d);
        beta = -copysign(s2d * rs, alpha.x);
        const double ib = -copysign(rs, alpha.x);
        tau = make_double2((beta - alpha.x) * ib, -alpha.y * ib);
        const double2 den = make_double2(alpha.x - beta, alpha.y);
        const double idd = 1.0 / (den.x * den.x + den.y * den.y);
        scale = make_double2(den.x * idd, -den.y * idd);        // 1 / (alpha - beta)
      }
      if (lane < kX) {
        if (lane < jj) {                                       // Q_a, v_a in units of 2^-58
          const double2 val = make_double2(acc_to_double(tot1[2 * lane], tot2[2 * lane], Ej - 2 * kQ),
                                           acc_to_double(tot1[2 * lane + 1], tot2[2 * lane + 1], Ej - 2 * kQ));
          const longlong2 va = join(Pv[lane * K + jj]);
          const double2 vac = make_double2(fx_to_double(va.x, 0), -fx_to_double(va.y, 0));
          Gsh[lane][jj] = cfmaf(vac, scale, val);              // conj(v_a[jj]) + scale Q_a
        } else if (lane + 1 < nbp) {                           // P_c, c = lane + 1
          const int Ec = colE[lane + 1];
          const int e = Ej + Ec - 2 * kQ;
          const double2 val = make_double2(acc_to_double(tot1[2 * lane], tot2[2 * lane], e),
                                           acc_to_double(tot1[2 * lane + 1], tot2[2 * lane + 1], e));
          const longlong2 ac = Pf[(lane + 1) * K + jj];
          const double2 acd = make_double2(fx_to_double(ac.x, Ec), fx_to_double(ac.y, Ec));
          const double2 vh = cfma_conjf(acd, scale, val);       // a_c[jj] + conj(scale) P_c
          const double2 w = make_double2(tau.x * vh.x + tau.y * vh.y, tau.x * vh.y - tau.y * vh.x);
          int4 nw;
          split29(-to_fx(w.x, Ec), nw.x, nw.y);
          split29(-to_fx(w.y, Ec), nw.z, nw.w);
          wn4[lane] = nw;
          wi2[lane] = make_int2(-nw.z, -nw.w);
        }
      }
      if (lane == 0) {
        betash[jj] = beta;
        taush[jj] = tau;
        if (!isfinite(beta)) atomicOr(o.status, kStatNonFinite);
        // v = x scale = X 2^{E_jj - 58} scale: V = X (2^{E_jj} scale) in units of 2^-58
        const unsigned long long ka = oz::abs_key(scale.x), kb = oz::abs_key(scale.y);
        const int se = oz::key_exponent(ka > kb ? ka : kb);
        svS = make_longlong2(to_fx(scale.x, se), to_fx(scale.y, se));
        svSh = kQ - se - Ej;
      }
    }
    __syncthreads();                                           // scalars of column jj
    // H_jj on the owner's rows: v, the later columns, and the exact sums of
    // column jn = jj + 1 (slot x < jn: Q_x; x >= jn: P_{x+1})
    const longlong2 S = svS;
    const int vsh = svSh;
    const int jn = jj + 1;
    int4 nwj = make_int4(0, 0, 0, 0);
    int2 wij = make_int2(0, 0);
    if (jn < nbp) {
      nwj = wn4[jj];
      wij = wi2[jj];
    }
#pragma unroll
    for (int x = 0; x < kX; ++x) pr[x] = pi[x] = Acc{0, 0};
    qr = qi = xn2 = Acc{0, 0};
    qslot = jj;
    for (int i = tid; i < K; i += NT) {
      if (i < jj) continue;
      Sp v;
      if (i == jj) {
        v.rh = 1 << 29; v.rl = 0; v.ih = 0; v.il = 0;           // v = 1 on the diagonal
      } else {
        v = split(mul_scalar(Pf[jj * K + i], S, vsh));
        Pv[jj * K + i] = make_int4(v.rh, v.rl, v.ih, v.il);
      }
      if (jn >= nbp) continue;
      const bool acc = i > jn;
      longlong2 xn = Pf[jn * K + i];
      upd(xn, v, nwj, wij);
      Pf[jn * K + i] = xn;
      const SpN xs = splitn(xn);
      if (acc) {
        mac_abs2(xn2, xs);
        mac_conj_b(qr, qi, v.rh, v.rl, v.ih, v.il, xs);
      }
#pragma unroll
      for (int x = kX - 1; x >= 0; --x) {                      // columns c = x + 1 > jn
        if (x < jn) break;
        if (x + 1 >= nbp) continue;
        longlong2 y = Pf[(x + 1) * K + i];
        upd(y, v, wn4[x], wi2[x]);
        Pf[(x + 1) * K + i] = y;
        if (acc) mac_conj_a(pr[x], pi[x], xs, split(y));
      }
      if (acc) {
#pragma unroll
        for (int x = 0; x < kX; ++x) {                         // Gram with earlier reflectors a < jj
          if (x >= jj) break;
          const int4 va = Pv[x * K + i];
          mac_conj_b(pr[x], pi[x], va.x, va.y, va.z, va.w, xs);
        }
      }
    }
  }
  __syncthreads();
  if (warp == 1) t_column(nbp - 1);
  // back to FP64 in place: R above the diagonal, beta on it, v below
  for (int e = tid; e < nbp * K; e += NT) {
    const int a = e / K, i = e - a * K;
    double2 r;
    if (i < a) {
      const longlong2 X = Pf[e];
      const int Ea = colE[a];
      r = make_double2(fx_to_double(X.x, Ea), fx_to_double(X.y, Ea));
    } else if (i == a) {
      r = make_double2(betash[a], 0.0);
    } else {
      const longlong2 V = join(Pv[e]);
      r = make_double2(fx_to_double(V.x, 0), fx_to_double(V.y, 0));
    }
    Pd[e] = r;
  }
  __syncthreads();
  for (int e = tid; e < nbp * K; e += NT) {
    const int a = e / K, i = e - a * K;
    A[(size_t)(k0 + a) * lda + k0 + i] = Pd[e];
  }
  if (tid < nbp) o.tau[(size_t)d * o.cols + k0 + tid] = taush[tid];
  double2 *Tg = o.T + ((size_t)d * o.npanels + p) * kNB * kNB;
  for (int e = tid; e < kNB * kNB; e += NT) Tg[e] = Tsh[e % kNB][e / kNB];
  if (o.slices == 0) return;

  // the exponent of each reflector column (largest |V(i, a)|, unit diagonal
  // included) for vdigits_kernel (qr_split.cu), as the FP64 panel writes it
  const int kp = o.kp;
  const int dslot = o.dig_kept ? p : (p & 1);
  int *vex = o.vexp + ((size_t)d * o.dig_nslot + dslot) * (kNB + kp);
  {
    unsigned long long m[kNB];
#pragma unroll
    for (int a = 0; a < kNB; ++a) m[a] = 0ull;
    for (int i = tid; i < K; i += NT) {
#pragma unroll
      for (int a = 0; a < kNB; ++a) {
        const double2 v = (a >= nbp || i < a) ? make_double2(0.0, 0.0)
                          : (i == a ? make_double2(1.0, 0.0) : Pd[a * K + i]);
        const unsigned long long k = oz::abs_key2(v);
        m[a] = k > m[a] ? k : m[a];
      }
    }
#pragma unroll
    for (int a = 0; a < kNB; ++a) {
#pragma unroll
      for (int s = 16; s > 0; s >>= 1) {
        const unsigned long long w = __shfl_xor_sync(0xffffffffu, m[a], s);
        m[a] = w > m[a] ? w : m[a];
      }
      if (lane == 0) wkey[warp][a] = m[a];
    }
  }
  __syncthreads();
  if (tid < kNB) {
    unsigned long long m = 0ull;
    for (int w = 0; w < kW; ++w) m = wkey[w][tid] > m ? wkey[w][tid] : m;
    // the column maxima of Y = V T (y_rows_kernel) start from zero
    o.ykey[((size_t)d * 2 + (p & 1)) * kNB + tid] = 0ull;
    vex[tid] = oz::key_exponent(m);
  }
}

template <int NT>
size_t panel_fx_static_smem() {
  static size_t bytes = 0;
  if (bytes == 0) {
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, qr_panel_fx_kernel<NT>) == cudaSuccess) bytes = fa.sharedSizeBytes;
  }
  return bytes;
}

template <int NT>
cudaError_t launch_fx(const ObsDev *d_obs, const int *d_task_obs, const int *d_task_mode,
                      int ntasks, int p, int rows, cudaStream_t st) {
  const size_t smem = sizeof(longlong2) * (size_t)kNB * rows;
  static size_t granted = 0;
  cudaError_t e = ensure_dynamic_smem(qr_panel_fx_kernel<NT>, smem, granted);
  if (e != cudaSuccess) return e;
  static const bool carve = (prefer_max_shared(qr_panel_fx_kernel<NT>), true);
  (void)carve;
  qr_panel_fx_kernel<NT><<<ntasks, NT, smem, st>>>(d_obs, d_task_obs, d_task_mode, p);
  return cudaGetLastError();
}

}  // namespace

bool panel_fx_fits(int rows, int threads) {
  static int optin = -1;
  if (optin < 0) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
      return false;
  }
  const size_t st = threads == 256 ? panel_fx_static_smem<256>() : panel_fx_static_smem<128>();
  return st > 0 && st + sizeof(longlong2) * (size_t)kNB * rows <= (size_t)optin;
}

cudaError_t launch_qr_panel_fx(const ObsDev *d_obs, const int *d_task_obs, const int *d_task_mode,
                               int ntasks, int p, int max_panel_rows, int threads, cudaStream_t st) {
  if (ntasks <= 0) return cudaSuccess;
  if (threads == 256)
    return launch_fx<256>(d_obs, d_task_obs, d_task_mode, ntasks, p, max_panel_rows, st);
  return launch_fx<128>(d_obs, d_task_obs, d_task_mode, ntasks, p, max_panel_rows, st);
}

}  // namespace axi
