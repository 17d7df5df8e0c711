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
// accumulator ("group" g); groups are flushed into FP64 after at most 32
// products of the contraction, far inside the 2^24 bound
// (32 * 7 pairs * 2^14 * 2 real products < 2^24). Only pairs with
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

// Exponent e with max|x| < 2^e (0 for an all-zero set).
__device__ __forceinline__ int scale_exponent(double maxabs) {
  if (!(maxabs > 0.0)) return 0;
  int e;
  frexp(maxabs, &e);
  return e;
}

// Balanced digits of x * 2^{-e} (|x| < 2^e): x * 2^{56-e} is rounded to the
// nearest integer, rounded again to its top 7S bits, and written in base 128
// with digits d_2..d_S in [-64, 63] and a leading digit |d_1| <= 128, so that
//   x = 2^e sum_s d_s 2^{-7s} + err,  |err| <= 2^{e - 7S - 1} (1 + 2^-7).
// Rounding (not truncation) keeps the digit errors unbiased, so they do not
// add up coherently along a contraction. All steps after the rounding are
// exact integer operations.
template <int S>
__device__ __forceinline__ void split_store(double x, int e, __nv_bfloat16 *dst, int stride) {
  static_assert(S >= 1 && S <= 8, "1..8 digits");
  const long long n = __double2ll_rn(ldexp(x, 56 - e));   // |n| <= 2^56
  constexpr int drop = 56 - 7 * S;
  long long m = drop > 0 ? ((n + (1ll << (drop > 0 ? drop - 1 : 0))) >> drop) : n;
#pragma unroll
  for (int s = S; s >= 2; --s) {
    int d = (int)(m & 127);
    if (d >= 64) d -= 128;
    dst[(s - 1) * stride] = __float2bfloat16_rn((float)d);
    m = (m - d) >> 7;
  }
  dst[0] = __float2bfloat16_rn((float)m);
}

__device__ __forceinline__ uint32_t ld32(const __nv_bfloat16 *p) {
  return *reinterpret_cast<const uint32_t *>(p);
}
__device__ __forceinline__ uint32_t neg2(uint32_t v) { return v ^ 0x80008000u; }

// A fragment (16 x 16, row-major, k contiguous) at tile origin `base` with row stride ld.
__device__ __forceinline__ void load_a(const __nv_bfloat16 *base, int ld, int lane, uint32_t (&a)[4]) {
  const int g = lane >> 2, t = lane & 3;
  a[0] = ld32(base + g * ld + 2 * t);
  a[1] = ld32(base + (g + 8) * ld + 2 * t);
  a[2] = ld32(base + g * ld + 8 + 2 * t);
  a[3] = ld32(base + (g + 8) * ld + 8 + 2 * t);
}
// B fragment (16 x 8, stored [n][k] with k contiguous) at origin `base` with n stride ld.
__device__ __forceinline__ void load_b(const __nv_bfloat16 *base, int ld, int lane, uint32_t (&b)[2]) {
  const int g = lane >> 2, t = lane & 3;
  b[0] = ld32(base + g * ld + 2 * t);
  b[1] = ld32(base + g * ld + 8 + 2 * t);
}

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
