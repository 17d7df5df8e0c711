// Split-precision (Ozaki-scheme) building blocks for FP64 complex GEMMs on
// BF16 tensor cores.
//
// A row (or column) of FP64 values is scaled by one power of two 2^-e so that
// every |value| < 1, written as a 56-bit fixed-point integer, and cut into
// S base-128 digits d_1..d_S (|d_1| <= 128, |d_s| <= 64 after it; all exact
// in BF16):  x = 2^e sum_s d_s 2^{-7s} + O(2^{e - 7S - 1}).
// A product of two such numbers is sum_{s,t} d_s d_t 2^{-7(s+t)}. The BF16
// mma.sync (m16n8k16, FP32 accumulate) forms the integer sums
// sum_k d_{s,ik} d_{t,kj} exactly as long as every partial sum stays below
// 2^24 in magnitude (all terms are integers, so the tensor core's alignment
// and rounding lose nothing). Pairs with s + t = g share one FP32
// accumulator ("group" g); groups are flushed after at most 32 products of
// the contraction: with |d_1| <= 128 and |d_s| <= 64 otherwise, a group sum
// of one complex component stays below 32 * 2 * 2^12 (g + 1) <= 2^22, so the
// FP32 sums are exact and convert to integers by a magic-number add. Only pairs with
// s + t <= S + 1 are formed: the dropped terms are below 2^{-7S} S relative to
// the row/column maxima, the same order as the truncation of the digits.
#pragma once
#include <cuda_bf16.h>
#include <stdint.h>

namespace axi {
namespace oz {

__device__ __forceinline__ void mma16816(float (&c)[4], uint32_t a0, uint32_t a1, uint32_t a2,
                                         uint32_t a3, uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// On this part the FP64 pipe is ~1/1600 of the BF16 tensor rate, so the
// split and the recombination below use integer and FP32 instructions only:
// exponents and digits come from the IEEE-754 bit patterns, and FP32 group
// sums are turned into integers and accumulated in 64-bit integers.

// |x| as an ordered 64-bit key (IEEE bit patterns of non-negative doubles
// sort like the values).
__device__ __forceinline__ unsigned long long abs_key(double x) {
  return (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffull;
}

// Largest key of the real and imaginary parts of a complex value.
__device__ __forceinline__ unsigned long long abs_key2(double2 v) {
  const unsigned long long a = abs_key(v.x), b = abs_key(v.y);
  return a > b ? a : b;
}

// Exponent e with |x| < 2^e for the largest key (0 for an all-zero set).
__device__ __forceinline__ int key_exponent(unsigned long long key) {
  if (key == 0) return 0;
  const int E = (int)(key >> 52);
  return E == 0 ? -1022 : E - 1022;
}

// BF16 bit pattern of a small integer (|d| <= 255): d + 256 is placed in the
// mantissa of 2^23 (an OR, the sum staying below 2^23), 2^23 + 256 is taken
// off exactly in FP32, and the FP32 result, having at most 8 significant
// bits, truncates to BF16 without rounding (0 gives +0).
__device__ __forceinline__ unsigned short int_to_bf16_bits(int d) {
  const float f = __uint_as_float(0x4B000000u | (unsigned)(d + 256)) - 8388864.0f;
  return (unsigned short)(__float_as_uint(f) >> 16);
}

// Balanced digits of x * 2^{-e} (|x| < 2^e): m = round(x * 2^{7S - e}) is
// formed exactly from the mantissa and exponent bits, then written in base 128
// with digits d_2..d_S in [-64, 63] and a leading digit |d_1| <= 128:
//   x = 2^e sum_s d_s 2^{-7s} + err,  |err| <= 2^{e - 7S - 1}.
// Rounding (not truncation) keeps the digit errors unbiased, so they do not
// add up coherently along a contraction.
template <int S>
__device__ __forceinline__ void split_store(double x, int e, __nv_bfloat16 *dst, int stride) {
  static_assert(S >= 1 && S <= 8, "1..8 digits");
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int E = (int)((b >> 52) & 0x7ff);
  unsigned long long M = b & 0xfffffffffffffull;
  int Ee = E;
  if (E == 0) Ee = 1; else M |= 1ull << 52;
  const int sh = Ee - 1075 + 7 * S - e;             // x * 2^{7S-e} = M * 2^sh, sh <= 3
  long long m;
  if (sh >= 0) m = (long long)(M << sh);
  else if (sh > -60) m = (long long)((M + (1ull << (-sh - 1))) >> (-sh));
  else m = 0;
  if (b >> 63) m = -m;
  unsigned short *out = reinterpret_cast<unsigned short *>(dst);
#pragma unroll
  for (int s = S; s >= 2; --s) {
    int d = (int)(m & 127);
    if (d >= 64) d -= 128;
    out[(s - 1) * stride] = int_to_bf16_bits(d);
    m = (m - d) >> 7;
  }
  out[0] = int_to_bf16_bits((int)m);
}

// split_store with a run-time digit count S (1..8) into raw BF16 bit patterns.
__device__ __forceinline__ void split_store_n(double x, int e, int S, unsigned short *dst,
                                              size_t stride) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int E = (int)((b >> 52) & 0x7ff);
  unsigned long long M = b & 0xfffffffffffffull;
  int Ee = E;
  if (E == 0) Ee = 1; else M |= 1ull << 52;
  const int sh = Ee - 1075 + 7 * S - e;
  long long m;
  if (sh >= 0) m = (long long)(M << sh);
  else if (sh > -60) m = (long long)((M + (1ull << (-sh - 1))) >> (-sh));
  else m = 0;
  if (b >> 63) m = -m;
  for (int s = S; s >= 2; --s) {
    int d = (int)(m & 127);
    if (d >= 64) d -= 128;
    dst[(s - 1) * stride] = int_to_bf16_bits(d);
    m = (m - d) >> 7;
  }
  dst[0] = int_to_bf16_bits((int)m);
}

// Faster digits for an operand that is split on every use (the trailing
// matrix in the QR update). m = round(|x| 2^{7S - e}) with one bit of
// headroom in e (|x| < 2^{e-1}, so m <= 2^{7S-1}); the signed value is
// offset by K = 64 (1 + 2^7 + ... + 2^{7(S-1)}) so that a = K +- m >= 0 and
// its base-128 fields f_s give balanced digits d_s = f_s - 64 without a
// carry chain: d_s in [-64, 63], the top field left unmasked so d_1 <= 65.
// Rounding happens once, at the last digit, so digit errors stay unbiased.
// BF16 bits of d come from one FP32 add: (2^23 + f) - (2^23 + 64) is exact.
// Two values (consecutive rows) are packed per 32-bit word: low half x0,
// high half x1.
__device__ __forceinline__ unsigned long long mag_fixed(double x, int e, int S7, unsigned &sign) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  sign = (unsigned)(b >> 63);
  const int E = (int)((b >> 52) & 0x7ff);
  unsigned long long M = b & 0xfffffffffffffull;
  int Ee = E;
  if (E == 0) Ee = 1; else M |= 1ull << 52;
  const int sh = Ee - 1075 + S7 - e;
  if (sh >= 0) return M << sh;
  if (sh > -60) return (M + (1ull << (-sh - 1))) >> (-sh);
  return 0;
}
__device__ __forceinline__ unsigned bf16_bits_bal(unsigned f) {
  return __float_as_uint(__uint_as_float(0x4B000000u | f) - 8388672.0f) >> 16;
}
template <int S>
__device__ __forceinline__ void split2_fast(double x0, double x1, int e, uint32_t *dst,
                                            int stride_words) {
  unsigned long long K = 0;
#pragma unroll
  for (int s = 0; s < S; ++s) K = (K << 7) | 64ull;
  unsigned s0, s1;
  const unsigned long long m0 = mag_fixed(x0, e, 7 * S, s0), m1 = mag_fixed(x1, e, 7 * S, s1);
  const unsigned long long a0 = s0 ? K - m0 : K + m0, a1 = s1 ? K - m1 : K + m1;
#pragma unroll
  for (int s = 1; s <= S; ++s) {
    const unsigned mask = s == 1 ? 0xffffu : 127u;
    const unsigned f0 = (unsigned)(a0 >> (7 * (S - s))) & mask;
    const unsigned f1 = (unsigned)(a1 >> (7 * (S - s))) & mask;
    dst[(s - 1) * stride_words] = bf16_bits_bal(f0) | (bf16_bits_bal(f1) << 16);
  }
}

// Exact FP32 integer (|v| < 2^22) -> int32 without a conversion instruction.
__device__ __forceinline__ int f32_int(float v) {
  return __float_as_int(v + 12582912.0f) - 0x4B400000;
}

// Group accumulators folded into two 64-bit integers: groups g = 2..4 into
// hi (weight 2^{7(4-g)}), groups g = 5..S+1 into lo (weight 2^{7(S+1-g)}).
// The represented value is hi 2^-28 + lo 2^{-7(S+1)}.
template <int S>
__device__ __forceinline__ void fold_group(long long &hi, long long &lo, int g, float acc) {
  const long long v = (long long)f32_int(acc);
  if (g <= 4) hi += v << (7 * (4 - g));
  else lo += v << (7 * (S + 1 - g));
}

// t 2^e rounded to the nearest double (ties to even), built from the bits
// with integer instructions only: on this part an integer-to-FP64
// conversion occupies the FP64 pipe like an FMA. Falls back to ldexp when
// the result is not a normal number.
__device__ __forceinline__ double scaled_to_double(long long t, int e) {
  if (t == 0) return 0.0;
  const unsigned long long sgn = t < 0 ? 0x8000000000000000ull : 0ull;
  unsigned long long a = t < 0 ? 0ull - (unsigned long long)t : (unsigned long long)t;
  const int lz = __clzll((long long)a);
  a <<= lz;                                              // leading one at bit 63
  unsigned long long m = a >> 11;                        // 53 significant bits
  const unsigned rem = (unsigned)(a & 0x7ffu);
  m += (rem > 0x400u || (rem == 0x400u && (m & 1ull))) ? 1ull : 0ull;
  const int E = 63 - lz + e;                             // value in [2^E, 2^{E+1}]
  if (E < -1021 || E > 1022) return ldexp((double)t, e);
  // the hidden bit of m (or its carry) adds to the biased exponent field
  return __longlong_as_double((long long)(sgn | (((unsigned long long)(E + 1022) << 52) + m)));
}

// Group sum `acc` (an exact integer, |acc| < 2^22) of digit group g added to
// a fixed-point accumulator of resolution 2^-R: t += acc 2^{R - 7g}, rounded
// to nearest where R < 7g. With g a compile-time constant (unrolled group
// loops) the shift direction folds away.
template <int R>
__device__ __forceinline__ void fold_fixed(long long &t, int g, float acc) {
  const long long v = (long long)f32_int(acc);
  const int sh = R - 7 * g;
  if (sh >= 0) t += v << sh;
  else t += (v + (1ll << (-sh - 1))) >> (-sh);
}

// fold_fixed for the adjacent groups g and g + 1 at once: their exact sums
// (|acc| < 2^22) combine as acc_g 2^7 + acc_g1 in 32 bits (below 2^30), so
// the pair costs one 64-bit shift and add. For R >= 7 g (group g lands at or
// above the resolution) it is bit-identical to two fold_fixed calls: a right
// shift of the pair drops at most 7 bits, all of them from acc_g1.
template <int R>
__device__ __forceinline__ void fold_fixed_pair(long long &t, int g, float acc_g, float acc_g1) {
  const int v = f32_int(acc_g) * 128 + f32_int(acc_g1);
  const int sh = R - 7 * (g + 1);
  if (sh >= 0) t += (long long)v << sh;
  else t += ((long long)v + (1ll << (-sh - 1))) >> (-sh);
}

// x - t 2^e for a double x and an integer t (|t| < 2^59), with integer
// instructions only. The difference is formed in 64-bit integers at the finer
// of the two resolutions that keeps x within 62 bits: 2^e when x's last bit
// is at most 2^9 above it (x exact there, or rounded to nearest when x is
// finer than 2^e), else 2^(e + k) with k chosen so that x is exact and t is
// rounded to nearest (an error below 2^-10 of x's last bit); then one
// rounding by scaled_to_double. Non-finite x falls back to FP64.
__device__ __forceinline__ double sub_scaled(double x, long long t, int e) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int E = (int)((b >> 52) & 0x7ff);
  if (E == 0x7ff) return x - scaled_to_double(t, e);
  unsigned long long M = b & 0xfffffffffffffull;
  int Ee = E;
  if (E == 0) Ee = 1; else M |= 1ull << 52;
  const int sh = Ee - 1075 - e;                      // x = M 2^sh in units of 2^e
  long long m;
  if (sh > 9) {                                      // work at 2^(e + k), x exact
    const int k = sh - 9;
    m = (long long)(M << 9);
    t = k >= 62 ? 0ll : (t + (1ll << (k - 1))) >> k;
    e += k;
  } else if (sh >= 0) {
    m = (long long)(M << sh);
  } else if (sh > -60) {
    m = (long long)((M + (1ull << (-sh - 1))) >> (-sh));
  } else {
    m = 0;
  }
  if (b >> 63) m = -m;
  return scaled_to_double(m - t, e);
}

// The S balanced digits of split_store, as BF16 bit patterns in registers.
template <int S>
__device__ __forceinline__ void split_regs(double x, int e, unsigned short (&out)[S]) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int E = (int)((b >> 52) & 0x7ff);
  unsigned long long M = b & 0xfffffffffffffull;
  int Ee = E;
  if (E == 0) Ee = 1; else M |= 1ull << 52;
  const int sh = Ee - 1075 + 7 * S - e;
  long long m;
  if (sh >= 0) m = (long long)(M << sh);
  else if (sh > -60) m = (long long)((M + (1ull << (-sh - 1))) >> (-sh));
  else m = 0;
  if (b >> 63) m = -m;
#pragma unroll
  for (int s = S; s >= 2; --s) {
    int d = (int)(m & 127);
    if (d >= 64) d -= 128;
    out[s - 1] = int_to_bf16_bits(d);
    m = (m - d) >> 7;
  }
  out[0] = int_to_bf16_bits((int)m);
}

// fold_group for group sums up to 2^24 (exact FP32 integers beyond the
// magic-number range): a rounding conversion instead of the add trick.
template <int S>
__device__ __forceinline__ void fold_group_rn(long long &hi, long long &lo, int g, float acc) {
  const long long v = (long long)__float2int_rn(acc);
  if (g <= 4) hi += v << (7 * (4 - g));
  else lo += v << (7 * (S + 1 - g));
}

// hi 2^{-28} + lo 2^{-7(S+1)}, times 2^E.
template <int S>
__device__ __forceinline__ double unfold(long long hi, long long lo, int E) {
  return scaled_to_double(hi, E - 28) + scaled_to_double(lo, E - 7 * (S + 1));
}

// hi 2^{-28} + lo 2^{-7(S+1)} as one 64-bit integer t, the value being
// t 2^{unfold1_shift<S>()} (times 2^E). Valid when |hi| < 2^34, which holds
// for a single k16 step of a complex contraction (group g = 2 sums at most
// 32 products of two digits <= 128, weight 2^14): one integer-to-FP64
// conversion instead of two.
template <int S>
__device__ __forceinline__ long long unfold1_int(long long hi, long long lo) {
  constexpr int sh = 7 * (S + 1) - 28;
  constexpr int shh = sh < 28 ? sh : 28;
  constexpr int drop = sh - shh;
  if constexpr (drop > 0) return (hi << shh) + ((lo + (1ll << (drop - 1))) >> drop);
  else return (hi << shh) + lo;
}
template <int S>
__host__ __device__ constexpr int unfold1_shift() {
  return -7 * (S + 1) + ((7 * (S + 1) - 28) - ((7 * (S + 1) - 28) < 28 ? (7 * (S + 1) - 28) : 28));
}

__device__ __forceinline__ uint32_t neg2(uint32_t v) { return v ^ 0x80008000u; }

// ldmatrix: four 8x8 b16 matrices from shared memory; lane l gives the row
// address of row (l mod 8) of matrix (l / 8), and receives in r[m] the pair
// (row l / 4, columns 2 (l mod 4), +1) of matrix m, i.e. mma fragment order.
__device__ __forceinline__ void ldsm_x4(uint32_t (&r)[4], const void *p) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(a));
}

// Asynchronous 16-byte global -> shared copy (L2 only); with valid == false
// nothing is read and the 16 bytes are zero-filled.
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem, bool valid) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  const int n = valid ? 16 : 0;
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(s), "l"(gmem), "r"(n));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N)); }

// Complex slice product for one k16 step: acc_re += Ar Br - Ai Bi, acc_im += Ar Bi + Ai Br.
__device__ __forceinline__ void cmma(float (&re)[4], float (&im)[4], const uint32_t (&ar)[4],
                                     const uint32_t (&ai)[4], const uint32_t (&br)[2],
                                     const uint32_t (&bi)[2]) {
  mma16816(re, ar[0], ar[1], ar[2], ar[3], br[0], br[1]);
  mma16816(re, neg2(ai[0]), neg2(ai[1]), neg2(ai[2]), neg2(ai[3]), bi[0], bi[1]);
  mma16816(im, ar[0], ar[1], ar[2], ar[3], bi[0], bi[1]);
  mma16816(im, ai[0], ai[1], ai[2], ai[3], br[0], br[1]);
}

}  // namespace oz
}  // namespace axi
