// Split-precision back substitution R X = Y of the apply (Sec. 4.2): the
// blocked substitution of trsm_kernel with its off-diagonal updates on BF16
// tensor cores.
//
// R (cols x cols, upper triangular, real diagonal) is taken in 32-column
// blocks from the bottom. For block b (rows/columns r0 = 32 b .. r0 + nb):
//   1. the 32 x 32 diagonal block is solved in FP64, one warp per RHS column,
//      after scaling the block's rows and the RHS by the reciprocal diagonal
//      (a unit-diagonal elimination: four FMAs per step);
//   2. the rows above are updated, Y(0:r0, :) -= R(0:r0, block) X_b, as a
//      digit GEMM: R's rows are split once, at the end of the build
//      (r_digits_kernel, one exponent per row and block, balanced digits,
//      kept in the operator), X_b per block (one
//      exponent per column, carry-free balanced digits), every digit pair
//      s + t <= S + 1 on BF16 mma.sync (group sums over the 32-term complex
//      contraction stay below 2^23: exact in FP32), recombined with integer instructions
//      into the FP64 read-modify-write of Y.
// One CTA per (mode, 16 RHS columns): warp w solves columns w and w + 8 of
// each diagonal block as two interleaved (independent) chains, and the
// update's two n8 tiles go to warps 0-3 and 4-7. With two CTAs per SM the
// 32 columns of 16 waves on the cup's 91 modes fit in one wave of CTAs.
#include "axi_internal.h"
#include "ozaki.cuh"

namespace axi {
namespace {

constexpr int kTB = 32;          // block size of the substitution
constexpr int kTC = 16;          // RHS columns per CTA (warp w solves columns w and w + 8)
constexpr int kTT = 256;         // threads
constexpr int kRM = 64;          // rows of R per staged chunk of the update
constexpr int kLDR = kTB + 8;    // padded k stride (bf16) of the staged digits

__device__ __forceinline__ unsigned long long key2(double2 v) {
  const unsigned long long a = oz::abs_key(v.x), b = oz::abs_key(v.y);
  return a > b ? a : b;
}

// Digits of R(0:r0, r0:r0+nb) for every mode d and block b (layout in
// ObsDev::rdig): block b holds rb = r0 rounded up to 64 rows, rows r0..rb-1
// zero, so the update reads whole 64-row chunks. One CTA per (mode, block,
// 64-row chunk): the 64 x 32 tile is read column by column (coalesced) into
// shared memory, then each warp splits whole rows, lane k taking column k,
// so every digit store is one contiguous 64-byte row segment.
__global__ void __launch_bounds__(kTT)
r_digits_kernel(const ObsDev *__restrict__ od) {
  const ObsDev &o = *od;
  const int S = o.slices;
  const int d = blockIdx.x, b = blockIdx.y, m0 = 64 * blockIdx.z;
  const int rb = r_digit_block_rows(b);
  if (m0 >= rb || !owns_mode(o, d)) return;
  const int n = o.cols, ld = o.rows;
  const int r0 = b * kTB, nb = min(kTB, n - r0);
  const double2 *R = o.A + (size_t)d * o.cols * o.rows;
  const size_t before = r_digit_rows_before(b);
  const size_t mrows = r_digit_rows_before((n + kTB - 1) / kTB);
  unsigned short *dg = o.rdig + ((size_t)d * mrows * S + before * S) * 2 * kTB;
  int *ex = o.rex + (size_t)d * mrows + before;
  const size_t dstride = (size_t)2 * rb * kTB;            // between digits
  __shared__ double2 tile[kTB][64 + 1];
  for (int e = threadIdx.x; e < kTB * 64; e += kTT) {
    const int c = e / 64, r = e % 64, i = m0 + r;
    tile[c][r] = (i < r0 && c < nb) ? R[(size_t)(r0 + c) * ld + i] : make_double2(0.0, 0.0);
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int r = warp; r < 64; r += kTT / 32) {
    const int i = m0 + r;
    const double2 x = tile[lane][r];
    unsigned long long m = key2(x);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const unsigned long long w = __shfl_xor_sync(0xffffffffu, m, off);
      m = w > m ? w : m;
    }
    const int e = oz::key_exponent(m);               // 0 for the zero rows i >= r0
    if (lane == 0) ex[i] = e;
    oz::split_store_n(x.x, e, S, dg + (size_t)i * kTB + lane, dstride);
    oz::split_store_n(x.y, e, S, dg + (size_t)(rb + i) * kTB + lane, dstride);
  }
}

template <int S>
struct TrsmSmem {
  union {                                // the diagonal block, then the R chunks of the update
    double2 Rb[kTB][kTB + 1];
    __nv_bfloat16 A[S][2][kRM][kLDR];    // digits of an R chunk ([row][column of the block])
  };
  double2 Yb[kTB][kTC + 1];
  double rinv[kTB];
  int eX[kTC];
  int eR[kRM];
  __nv_bfloat16 B[S][2][kTC][kLDR];      // digits of X_b ([column][row of the block])
};

template <int S>
__global__ void __launch_bounds__(kTT)
trsm_split_kernel(const ObsDev *__restrict__ od, double2 *__restrict__ X, int ncols_total) {
  const ObsDev &o = *od;
  const int d = blockIdx.x;
  const int c0 = blockIdx.y * kTC;
  if (c0 >= ncols_total || !owns_mode(o, d)) return;
  const int ncols = min(kTC, ncols_total - c0);
  const int n = o.cols, ld = o.rows, nblk = (n + kTB - 1) / kTB;
  const size_t mrows = r_digit_rows_before(nblk);
  const double2 *R = o.A + (size_t)d * o.cols * o.rows;
  double2 *Xd = X + ((size_t)d * ncols_total + c0) * o.rows;
  extern __shared__ __align__(16) unsigned char tsraw[];
  TrsmSmem<S> &sm = *reinterpret_cast<TrsmSmem<S> *>(tsraw);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int grp = lane >> 2, tig = lane & 3;
  const int lrow = lane & 7, lmat = lane >> 3;
  const int a_row = lrow + 8 * (lmat & 1), a_k = 8 * (lmat >> 1);
  for (int ib = nblk - 1; ib >= 0; --ib) {
    const int r0 = ib * kTB, nb = min(kTB, n - r0);
    __syncthreads();
    for (int e = tid; e < kTB * kTB; e += kTT) {
      const int r = e % kTB, c = e / kTB;
      sm.Rb[r][c] = (r < nb && c < nb) ? R[(size_t)(r0 + c) * ld + r0 + r] : make_double2(0.0, 0.0);
    }
    for (int e = tid; e < kTB * kTC; e += kTT) {
      const int r = e % kTB, c = e / kTB;
      sm.Yb[r][c] = (r < nb && c < ncols) ? Xd[(size_t)c * ld + r0 + r] : make_double2(0.0, 0.0);
    }
    if (tid < kTB) sm.rinv[tid] = tid < nb ? 1.0 / R[(size_t)(r0 + tid) * ld + r0 + tid].x : 0.0;
    __syncthreads();
    // rows of the block scaled by the reciprocal (real) diagonal: the solve
    // then runs on a unit-diagonal triangle and each step is four FMAs
    for (int e = tid; e < kTB * kTB; e += kTT) {
      const int r = e % kTB, c = e / kTB;
      if (r < c) {
        const double inv = sm.rinv[r];
        sm.Rb[r][c] = make_double2(sm.Rb[r][c].x * inv, sm.Rb[r][c].y * inv);
      }
    }
    __syncthreads();
    // 1. diagonal block in FP64, warp w solves columns w and w + 8
    if (warp < ncols) {
      const int c0w = warp, c1w = warp + kTC / 2;
      const double inv = sm.rinv[lane];
      double2 y = sm.Yb[lane][c0w], z = sm.Yb[lane][c1w];   // column c1w is zero when unused
      y = make_double2(y.x * inv, y.y * inv);
      z = make_double2(z.x * inv, z.y * inv);
      for (int rr = nb - 1; rr >= 0; --rr) {
        double2 x, w;
        x.x = __shfl_sync(0xffffffffu, y.x, rr);              // final once the rows below are done
        x.y = __shfl_sync(0xffffffffu, y.y, rr);
        w.x = __shfl_sync(0xffffffffu, z.x, rr);
        w.y = __shfl_sync(0xffffffffu, z.y, rr);
        if (lane < rr) {
          const double2 rv = sm.Rb[lane][rr];
          y = make_double2(fma(-rv.x, x.x, fma(rv.y, x.y, y.x)), fma(-rv.x, x.y, fma(-rv.y, x.x, y.y)));
          z = make_double2(fma(-rv.x, w.x, fma(rv.y, w.y, z.x)), fma(-rv.x, w.y, fma(-rv.y, w.x, z.y)));
        }
      }
      sm.Yb[lane][c0w] = y;
      if (c1w < ncols) sm.Yb[lane][c1w] = z;
    }
    __syncthreads();
    for (int e = tid; e < kTB * kTC; e += kTT) {
      const int r = e % kTB, c = e / kTB;
      if (r < nb && c < ncols) Xd[(size_t)c * ld + r0 + r] = sm.Yb[r][c];
    }
    if (r0 == 0) break;
    // 2. digits of X_b: one exponent (with headroom) per column
#pragma unroll
    for (int h = 0; h < kTC / 8; ++h) {
      const int c = warp + 8 * h;
      const unsigned long long m = (lane < nb && c < ncols) ? key2(sm.Yb[lane][c]) : 0ull;
      unsigned long long mm = m;
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        const unsigned long long w = __shfl_xor_sync(0xffffffffu, mm, off);
        mm = w > mm ? w : mm;
      }
      if (lane == 0) sm.eX[c] = oz::key_exponent(mm) + 1;
    }
    __syncthreads();
    if (tid < kTC * (kTB / 2)) {
      const int c = tid / (kTB / 2), rp = tid % (kTB / 2);
      const double2 y0 = sm.Yb[2 * rp][c], y1 = sm.Yb[2 * rp + 1][c];
      uint32_t *wr = reinterpret_cast<uint32_t *>(&sm.B[0][0][c][0]) + rp;
      uint32_t *wi = reinterpret_cast<uint32_t *>(&sm.B[0][1][c][0]) + rp;
      oz::split2_fast<S>(y0.x, y1.x, sm.eX[c], wr, 2 * kTC * kLDR / 2);
      oz::split2_fast<S>(y0.y, y1.y, sm.eX[c], wi, 2 * kTC * kLDR / 2);
    }
    // 3. rows above: Y(0:r0) -= R(0:r0, block) X_b, 64 rows per chunk; warps
    // 0..3 take columns 0..7, warps 4..7 columns 8..15, 16 rows each
    const size_t before = r_digit_rows_before(ib);
    const int rb = r_digit_block_rows(ib);
    const unsigned short *dg = o.rdig + ((size_t)d * mrows * S + before * S) * 2 * kTB;
    const int *ex = o.rex + (size_t)d * mrows + before;
    for (int m0 = 0; m0 < r0; m0 += kRM) {
      __syncthreads();
      // R digits of rows m0..m0+63: [S][2][64][32] -> A, 4 x 16-byte pieces per row
      for (int e = tid; e < S * 2 * kRM * 4; e += kTT) {
        const int u = e & 3, row = e >> 2;                   // row = (s * 2 + part) * kRM + r
        const int sp = row / kRM, r = row % kRM;
        const uint4 v = *reinterpret_cast<const uint4 *>(dg + ((size_t)sp * rb + m0 + r) * kTB + 8 * u);
        *reinterpret_cast<uint4 *>(&sm.A[0][0][0][0] + (size_t)row * kLDR + 8 * u) = v;
      }
      if (tid < kRM) sm.eR[tid] = ex[m0 + tid];
      __syncthreads();
      const int wr = warp & 3, nt = warp >> 2;                  // row group, n8 tile
      if (m0 + 16 * wr < r0 && 8 * nt < ncols) {
        float acc[S][2][4];
#pragma unroll
        for (int g = 0; g < S; ++g)
#pragma unroll
          for (int e = 0; e < 4; ++e) acc[g][0][e] = acc[g][1][e] = 0.0f;
#pragma unroll
        for (int kk = 0; kk < kTB; kk += 16) {
#pragma unroll
          for (int s = 1; s <= S; ++s) {
            uint32_t ar[4], ai[4];
            oz::ldsm_x4(ar, &sm.A[s - 1][0][16 * wr + a_row][kk + a_k]);
            oz::ldsm_x4(ai, &sm.A[s - 1][1][16 * wr + a_row][kk + a_k]);
#pragma unroll
            for (int t = 1; t <= S + 1 - s; ++t) {
              uint32_t b4[4];                               // re k0-7, re k8-15, im k0-7, im k8-15
              oz::ldsm_x4(b4, &sm.B[t - 1][lmat >> 1][8 * nt + lrow][kk + 8 * (lmat & 1)]);
              const uint32_t br[2] = {b4[0], b4[1]}, bi[2] = {b4[2], b4[3]};
              oz::cmma(acc[s + t - 2][0], acc[s + t - 2][1], ar, ai, br, bi);
            }
          }
        }
        long long hi[2][4] = {}, lo[2][4] = {};
#pragma unroll
        for (int g = 2; g <= S + 1; ++g)
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            oz::fold_group_rn<S>(hi[0][e], lo[0][e], g, acc[g - 2][0][e]);
            oz::fold_group_rn<S>(hi[1][e], lo[1][e], g, acc[g - 2][1][e]);
          }
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int r = 16 * wr + grp + (e >= 2 ? 8 : 0);
          const int i = m0 + r, c = 8 * nt + 2 * tig + (e & 1);
          if (i < r0 && c < ncols) {
            const int E = sm.eR[r] + sm.eX[c] + oz::unfold1_shift<S>();
            double2 *y = &Xd[(size_t)c * ld + i];
            double2 v = *y;
            v.x -= oz::scaled_to_double(oz::unfold1_int<S>(hi[0][e], lo[0][e]), E);
            v.y -= oz::scaled_to_double(oz::unfold1_int<S>(hi[1][e], lo[1][e]), E);
            *y = v;
          }
        }
      }
    }
  }
}

template <int S>
cudaError_t launch_trsm_s(const ObsDev *d_o, const ObsDev &h, double2 *X, int ncol, cudaStream_t st) {
  const size_t smem = sizeof(TrsmSmem<S>);
  static size_t granted = 0;
  cudaError_t e = ensure_dynamic_smem(trsm_split_kernel<S>, smem, granted);
  if (e != cudaSuccess) return e;
  trsm_split_kernel<S><<<dim3(h.D, (ncol + kTC - 1) / kTC), kTT, smem, st>>>(d_o, X, ncol);
  return cudaGetLastError();
}

}  // namespace

size_t r_digit_bytes(const ObsDev &h) {
  if (h.slices <= 0) return 0;
  const size_t rows = r_digit_rows_before((h.cols + kTB - 1) / kTB);
  return (size_t)h.D * rows * h.slices * 2 * kTB * sizeof(unsigned short);
}
size_t r_exponent_bytes(const ObsDev &h) {
  if (h.slices <= 0) return 0;
  return (size_t)h.D * r_digit_rows_before((h.cols + kTB - 1) / kTB) * sizeof(int);
}

cudaError_t launch_r_digits(const ObsDev *d_o, const ObsDev &h, cudaStream_t st) {
  const int nblk = (h.cols + kTB - 1) / kTB;
  if (h.slices <= 0 || nblk < 2) return cudaSuccess;
  r_digits_kernel<<<dim3(h.D, nblk, r_digit_block_rows(nblk - 1) / 64), kTT, 0, st>>>(d_o);
  return cudaGetLastError();
}

cudaError_t launch_trsm_split(const ObsDev *d_o, const ObsDev &h, double2 *X, int ncol,
                              cudaStream_t st) {
  switch (h.slices) {
    case 4: return launch_trsm_s<4>(d_o, h, X, ncol, st);
    case 5: return launch_trsm_s<5>(d_o, h, X, ncol, st);
    case 6: return launch_trsm_s<6>(d_o, h, X, ncol, st);
    case 7: return launch_trsm_s<7>(d_o, h, X, ncol, st);
    case 8: return launch_trsm_s<8>(d_o, h, X, ncol, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace axi
