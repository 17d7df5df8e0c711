// Split-precision (AXI_PREC_SPLIT_BF16) block-reflector update on tensor cores.
//
// The trailing update of the blocked Householder QR and the Q^H of the apply
// both compute, for one panel's reflectors V (K x nb, unit lower trapezoidal)
// and compact-WY factor T,
//     X <- X - V (T^H (V^H X))         (Sec. 3 eq. linsys; Sec. 4.2),
// on a tile of kTN target columns. Here the two GEMMs run as Ozaki slice
// products on BF16 mma.sync (ozaki.cuh) and T^H in FP64:
//   digits  the panel's reflectors are split once per factorisation
//           (panel_digits_kernel) into V^H digits (exponent per reflector)
//           and V row digits (exponent per row);
//   pass 0  exponents of X's columns (carried from the previous step);
//   pass 1  W = V^H X, contraction over the K rows in chunks of 32;
//   pass 2  W' = T^H W (FP64), per-column exponents and digits of W';
//   pass 3  X -= V W', contraction nb = 16 (one k16 step), FP64
//           read-modify-write of X.
// Native FP64 work per X element and panel step: the final recombination
// and subtraction, a handful of operations against 256 for the FP64 kernel.
#include "axi_internal.h"
#include "ozaki.cuh"
#include <cooperative_groups.h>

namespace cg = cooperative_groups;

namespace axi {
namespace {

constexpr int kThreads = 128;          // 4 warps
constexpr int kTN = 32;                // target columns per CTA
constexpr int kKC = 32;                // contraction rows per chunk (pass 1)
constexpr int kRC = 64;                // output rows per chunk (pass 3): 4 warps x 16
constexpr int kLD1 = kKC + 8;          // padded k stride (conflict-free fragment loads)
constexpr int kLD2 = kNB + 8;

template <int S>
struct Pass1 {
  __nv_bfloat16 A[S][2][kNB][kLD1];    // digits of V^H chunk (rows = panel columns)
  __nv_bfloat16 B[S][2][kTN][kLD1];    // digits of X chunk ([column][row])
};
template <int S>
struct Pass3 {
  __nv_bfloat16 A[S][2][kRC][kLD2];    // digits of V rows chunk ([row][panel column])
  __nv_bfloat16 B[S][2][kTN][kLD2];    // digits of W' ([column][panel column])
};
template <int S>
struct OzSmem {
  union {
    Pass1<S> p1;
    Pass3<S> p3;
  } u;
  double2 W[kNB][kTN + 1];
  double2 T[kNB][kNB + 1];
  int eVH[kNB], eX[kTN], eW[kTN], eV[kRC];
  unsigned long long kNext[kTN];
};
// Cluster form (rows split over C CTAs): W' slices and the cluster-summed W
// of this CTA's column slice.
struct ClExtra {
  double2 Wq[kNB][kTN + 1];
  double2 Wsum[kNB][kTN / 2 + 1];
};

__device__ __forceinline__ double2 vget(const double2 *A, int lda, int rows, int k0, int nbp, int i,
                                        int a) {
  if (a >= nbp || i >= rows) return make_double2(0.0, 0.0);
  const int c = k0 + a;
  if (i < c) return make_double2(0.0, 0.0);
  if (i == c) return make_double2(1.0, 0.0);
  return A[(size_t)c * lda + i];
}

__device__ __forceinline__ unsigned long long key2(double2 v) {
  const unsigned long long a = oz::abs_key(v.x), b = oz::abs_key(v.y);
  return a > b ? a : b;
}

__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
    v = w > v ? w : v;
  }
  return v;
}

// Digits and exponents of one panel's reflectors. Blocks are stored per mode
// in `nslot` slots: the QR keeps one slot (the current panel), the apply's
// scratch one slot per panel. Block of 4*S*kNB*kp entries: V^H digits
// [S][2][kNB][kp], then V row digits [S][2][kp][kNB]; exponents [kNB + kp].
struct PanelDigits {
  const unsigned short *vh;   // digits of the left factor of the first product (V^H, or Y^H)
  const unsigned short *v;    // V row digits
  const int *ex;              // [kNB + kp]: exponents of vh's rows, then of V's rows
  const int *exh;             // exponents of vh's rows (ex unless given apart)
  int kp;
  bool pre_t;                 // vh holds Y^H = (V T)^H: the first product is already W'
};

template <int S>
__device__ __forceinline__ size_t digit_block(int kp) { return (size_t)4 * S * kNB * kp; }

template <int S>
__device__ __forceinline__ PanelDigits panel_digits(const unsigned short *dig, const int *ex, int kp,
                                                    int d, int nslot, int slot) {
  const size_t blk = digit_block<S>(kp);
  PanelDigits pd;
  pd.vh = dig + ((size_t)d * nslot + slot) * blk;
  pd.v = pd.vh + blk / 2;
  pd.ex = ex + ((size_t)d * nslot + slot) * (kNB + kp);
  pd.exh = pd.ex;
  pd.kp = kp;
  pd.pre_t = false;
  return pd;
}

// W' = T^H W for T upper triangular: output (a, j) is a sum of a + 1 terms,
// so outputs a and 15 - a are taken together (17 terms) to give every thread
// the same FP64 chain. th_pair returns (a, 15 - a) of column j, lo = a.
__device__ __forceinline__ void th_pair(const double2 (*T)[kNB + 1], const double2 *W, int ldw,
                                        int j, int lo, double2 &out_lo, double2 &out_hi) {
  const int hi = kNB - 1 - lo;
  double2 al = make_double2(0.0, 0.0), ah = make_double2(0.0, 0.0);
#pragma unroll 4
  for (int it = 0; it <= kNB; ++it) {               // kNB + 1 = 17 terms per pair
    const bool low = it <= lo;
    const int b = low ? it : it - lo - 1, a = low ? lo : hi;
    const double2 tv = T[b][a], w = W[b * ldw + j];
    const double re = tv.x * w.x + tv.y * w.y;      // conj(t) * w
    const double im = tv.x * w.y - tv.y * w.x;
    if (low) { al.x += re; al.y += im; } else { ah.x += re; ah.y += im; }
  }
  out_lo = al;
  out_hi = ah;
}

// A pair (a, 15 - a) split over two threads (half 0: 9 terms, half 1: 8):
// half 0 sums all of output lo and terms b = 0 .. 7 - lo of output hi, half 1
// terms b = 8 - lo .. hi of output hi.
__device__ __forceinline__ void th_pair_half(const double2 (*T)[kNB + 1], const double2 *W,
                                             int ldw, int j, int lo, int half, double2 &al,
                                             double2 &ah) {
  const int hi = kNB - 1 - lo;
  al = make_double2(0.0, 0.0);
  ah = make_double2(0.0, 0.0);
#pragma unroll 3
  for (int it = 0; it <= kNB / 2; ++it) {
    const bool low = half == 0 && it <= lo;
    const int b = half == 0 ? (low ? it : it - lo - 1) : kNB / 2 - lo + it;
    const int a = low ? lo : hi;
    if (half == 1 && it == kNB / 2) break;
    const double2 tv = T[b][a], w = W[b * ldw + j];
    const double re = tv.x * w.x + tv.y * w.y;      // conj(t) * w
    const double im = tv.x * w.y - tv.y * w.x;
    if (low) { al.x += re; al.y += im; } else { ah.x += re; ah.y += im; }
  }
}

// Column-max keys of X: `kin` (global, per column) when the previous update
// left them, else `carry` (the previous panel's pass 3 of this CTA left them
// in sm.kNext), else a scan of rows k0..rows-1. Pass 3 always leaves the keys
// of the updated X over rows k0+kNB.. (the next panel step's rows) in
// sm.kNext, and in `kout` when that is given.
// This CTA handles rows [rlo, rhi) of X (rlo a multiple of 32); with C > 1 the
// CTA is one of a cluster of C that splits the rows: their partial V^H X are
// summed through distributed shared memory, CTA r forms W' = T^H W for
// columns [r kTN/C, (r+1) kTN/C), and every CTA gathers the whole W'.
// FE: the pass-3 epilogue folds into one fixed-point int64 and subtracts in
// integers (sub_scaled); otherwise two int64 folds, one integer-built double
// and an FP64 subtraction (measured faster in the apply's Q^H, where the
// cluster's warps interleave with the FP64 T^H W of other CTAs).
template <int S, int C = 1, bool FE = true>
__device__ void oz_block_reflector_update(const PanelDigits pd, int rows, int k0,
                                          const double2 *__restrict__ Tg,
                                          double2 *__restrict__ X, int ldx, int ncols,
                                          const unsigned long long *__restrict__ kin, bool carry,
                                          unsigned long long *__restrict__ kout, OzSmem<S> &sm,
                                          ClExtra *cx = nullptr, int rlo = 0, int rhi = -1,
                                          int xoff = 0) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int grp = lane >> 2, tig = lane & 3;
  if (rhi < 0) rhi = rows;
  const int r1st = max(k0, rlo);

  // ---- pass 0: exponents of X's columns over rows k0..rows-1 (V's are stored)
  if (tid < kNB) sm.eVH[tid] = pd.exh[tid];
  if (kin != nullptr || carry) {
    if (tid < kTN) {
      const unsigned long long m = tid < ncols ? (carry ? sm.kNext[tid] : kin[tid]) : 0ull;
      sm.eX[tid] = oz::key_exponent(m) + 1;                   // headroom for split2_fast
    }
  } else {
    for (int j = warp; j < kTN; j += kThreads / 32) {
      unsigned long long m = 0;
      if (j < ncols)
        for (int i = r1st + lane; i < rhi; i += 32) {
          const unsigned long long k = key2(X[(size_t)j * ldx + i - xoff]);
          m = k > m ? k : m;
        }
      m = warp_max_u64(m);
      if (lane == 0) sm.eX[j] = oz::key_exponent(m) + 1;
    }
  }
  for (int e = tid; e < kNB * kNB; e += kThreads) sm.T[e % kNB][e / kNB] = Tg[e];
  __syncthreads();
  if (tid < kTN) sm.kNext[tid] = 0ull;

  // ---- pass 1: W = V^H X (16 x kTN); warp w owns columns 8w..8w+7. The next
  // chunk's V^H digits and X values are loaded into registers while the
  // current chunk's slice products run.
  constexpr int kVU = S * 2 * kNB * (kKC / 8) / kThreads;      // uint4 of V^H digits per thread
  constexpr int kXU = kTN * (kKC / 2) / kThreads;              // row pairs of X per thread
  static_assert(S * 2 * kNB * (kKC / 8) % kThreads == 0 && kTN * (kKC / 2) % kThreads == 0, "");
  uint4 vst[kVU];
  double2 xst[kXU][2];
  auto stage = [&](int r0) {
    const int rr0 = r0 - k0;
#pragma unroll
    for (int u = 0; u < kVU; ++u) {
      const int e = tid + u * kThreads, row = e >> 2, w4 = e & 3;  // row = (s*2 + part)*kNB + a
      vst[u] = *reinterpret_cast<const uint4 *>(pd.vh + (size_t)row * pd.kp + rr0 + 8 * w4);
    }
#pragma unroll
    for (int u = 0; u < kXU; ++u) {
      const int e = tid + u * kThreads, j = e / (kKC / 2), rp = e % (kKC / 2), i = r0 + 2 * rp;
      xst[u][0] = xst[u][1] = make_double2(0.0, 0.0);
      if (j < ncols) {
        if (i < rhi) xst[u][0] = X[(size_t)j * ldx + i - xoff];
        if (i + 1 < rhi) xst[u][1] = X[(size_t)j * ldx + i + 1 - xoff];
      }
    }
  };
  // ldmatrix lane roles: row (l mod 8) of matrix l / 8
  const int lrow = lane & 7, lmat = lane >> 3;
  const int a_row = lrow + 8 * (lmat & 1), a_k = 8 * (lmat >> 1);
  long long whi[2][4] = {}, wlo[2][4] = {};
  if (r1st < rhi) stage(r1st);
  for (int r0 = r1st; r0 < rhi; r0 += kKC) {
    __syncthreads();
#pragma unroll
    for (int u = 0; u < kVU; ++u) {
      const int e = tid + u * kThreads, row = e >> 2, w4 = e & 3;
      *reinterpret_cast<uint4 *>(&sm.u.p1.A[0][0][0][0] + row * kLD1 + 8 * w4) = vst[u];
    }
    // X digits, two consecutive rows per thread and 32-bit word
#pragma unroll
    for (int u = 0; u < kXU; ++u) {
      const int e = tid + u * kThreads, j = e / (kKC / 2), rp = e % (kKC / 2);
      if (8 * (j >> 3) >= ncols) continue;           // no warp reads this column group
      const int ex = sm.eX[j];
      uint32_t *wr = reinterpret_cast<uint32_t *>(&sm.u.p1.B[0][0][j][0]) + rp;
      uint32_t *wi = reinterpret_cast<uint32_t *>(&sm.u.p1.B[0][1][j][0]) + rp;
      oz::split2_fast<S>(xst[u][0].x, xst[u][1].x, ex, wr, kTN * kLD1);
      oz::split2_fast<S>(xst[u][0].y, xst[u][1].y, ex, wi, kTN * kLD1);
    }
    __syncthreads();
    if (r0 + kKC < rhi) stage(r0 + kKC);
    // All S groups accumulate at once (independent accumulators): digit s of
    // V^H is loaded once, then every digit t of X with s + t <= S + 1. A warp
    // whose 8 columns all lie beyond ncols has nothing to add.
    if (8 * warp >= ncols) continue;
    float acc[S][2][4];
#pragma unroll
    for (int g = 0; g < S; ++g)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[g][0][q] = acc[g][1][q] = 0.0f;
#pragma unroll
    for (int s = 1; s <= S; ++s) {
      uint32_t ar0[4], ar1[4], ai0[4], ai1[4];
      oz::ldsm_x4(ar0, &sm.u.p1.A[s - 1][0][a_row][a_k]);
      oz::ldsm_x4(ar1, &sm.u.p1.A[s - 1][0][a_row][16 + a_k]);
      oz::ldsm_x4(ai0, &sm.u.p1.A[s - 1][1][a_row][a_k]);
      oz::ldsm_x4(ai1, &sm.u.p1.A[s - 1][1][a_row][16 + a_k]);
#pragma unroll
      for (int t = 1; t <= S + 1 - s; ++t) {
        uint32_t br[4], bi[4];
        oz::ldsm_x4(br, &sm.u.p1.B[t - 1][0][8 * warp + lrow][8 * lmat]);
        oz::ldsm_x4(bi, &sm.u.p1.B[t - 1][1][8 * warp + lrow][8 * lmat]);
        const uint32_t br0[2] = {br[0], br[1]}, bi0[2] = {bi[0], bi[1]};
        const uint32_t br1[2] = {br[2], br[3]}, bi1[2] = {bi[2], bi[3]};
        oz::cmma(acc[s + t - 2][0], acc[s + t - 2][1], ar0, ai0, br0, bi0);
        oz::cmma(acc[s + t - 2][0], acc[s + t - 2][1], ar1, ai1, br1, bi1);
      }
    }
    // group sums: at most 7 pairs x 2 products x 32 rows x 128 x 65 < 2^22,
    // exact integers in FP32
#pragma unroll
    for (int g = 2; g <= S + 1; ++g)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const long long vr = (long long)__float2int_rn(acc[g - 2][0][q]);
        const long long vi = (long long)__float2int_rn(acc[g - 2][1][q]);
        if (g <= 4) {
          whi[0][q] += vr << (7 * (4 - g));
          whi[1][q] += vi << (7 * (4 - g));
        } else {
          wlo[0][q] += vr << (7 * (S + 1 - g));
          wlo[1][q] += vi << (7 * (S + 1 - g));
        }
      }
  }
  // c-fragment element q: row grp (+8 for q >= 2), column 8w + 2 tig + (q & 1)
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int a = grp + (q >= 2 ? 8 : 0), j = 8 * warp + 2 * tig + (q & 1);
    const int e = sm.eVH[a] + sm.eX[j];
    sm.W[a][j] = make_double2(oz::unfold<S>(whi[0][q], wlo[0][q], e),
                              oz::unfold<S>(whi[1][q], wlo[1][q], e));
  }
  __syncthreads();

  // ---- pass 2: W' = T^H W (T upper triangular) in FP64, then digits of W'
  if constexpr (C > 1) {
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    // columns of W' formed here: the live columns split evenly over the cluster
    const int cw = (ncols + C - 1) / C;                     // <= kTN / C
    cl.sync();                                              // every CTA's partial W ready
    for (int e = tid; e < kNB * cw; e += kThreads) {
      const int a = e / cw, jl = e % cw, j = rank * cw + jl;
      double2 acc = make_double2(0.0, 0.0);
#pragma unroll
      for (int r = 0; r < C; ++r) {
        const double2 *wr = cl.map_shared_rank(&sm.W[0][0], r);
        const double2 w = wr[a * (kTN + 1) + j];
        acc.x += w.x;
        acc.y += w.y;
      }
      cx->Wsum[a][jl] = acc;
    }
    __syncthreads();
    // kNB / 2 pairs (a, 15 - a) per column of the slice: one per two threads
    // when there are enough threads, else one per thread
    static_assert((kNB / 2) * (kTN / C) <= kThreads, "one pair per thread");
    const int npair = (kNB / 2) * cw;
    if (2 * npair <= kThreads) {
      const int half = tid & 1, pi = tid >> 1;
      const bool act = pi < npair;
      const int jl = act ? pi % cw : 0, lo = act ? pi / cw : 0;
      double2 al, ah;
      th_pair_half(sm.T, &cx->Wsum[0][0], kTN / 2 + 1, jl, lo, half, al, ah);
      ah.x += __shfl_xor_sync(0xffffffffu, ah.x, 1);
      ah.y += __shfl_xor_sync(0xffffffffu, ah.y, 1);
      if (act && half == 0) {
        cx->Wq[lo][rank * cw + jl] = al;
        cx->Wq[kNB - 1 - lo][rank * cw + jl] = ah;
      }
    } else if (tid < npair) {
      const int jl = tid % cw, lo = tid / cw;
      double2 olo, ohi;
      th_pair(sm.T, &cx->Wsum[0][0], kTN / 2 + 1, jl, lo, olo, ohi);
      cx->Wq[lo][rank * cw + jl] = olo;
      cx->Wq[kNB - 1 - lo][rank * cw + jl] = ohi;
    }
    cl.sync();                                              // W' slices ready
    for (int e = tid; e < kNB * kTN; e += kThreads) {
      const int a = e / kTN, j = e % kTN;
      if (j < C * cw) {
        const double2 *q = cl.map_shared_rank(&cx->Wq[0][0], j / cw);
        sm.W[a][j] = q[a * (kTN + 1) + j];
      } else {
        sm.W[a][j] = make_double2(0.0, 0.0);                // beyond every slice: unused
      }
    }
    __syncthreads();
  } else if (!pd.pre_t) {
  constexpr int kPairs = (kNB / 2) * kTN / kThreads;          // pairs (a, 15 - a) per thread
  double2 wp[kPairs][2];
#pragma unroll
  for (int u = 0; u < kPairs; ++u) {
    const int e = tid + u * kThreads, j = e % kTN, lo = e / kTN;
    wp[u][0] = wp[u][1] = make_double2(0.0, 0.0);
    if (j < ncols) th_pair(sm.T, &sm.W[0][0], kTN + 1, j, lo, wp[u][0], wp[u][1]);
  }
  __syncthreads();
#pragma unroll
  for (int u = 0; u < kPairs; ++u) {
    const int e = tid + u * kThreads, j = e % kTN, lo = e / kTN;
    sm.W[lo][j] = wp[u][0];
    sm.W[kNB - 1 - lo][j] = wp[u][1];
  }
  __syncthreads();
  }
  if (tid < kTN) {
    unsigned long long m = 0;
    for (int a = 0; a < kNB; ++a) {
      const unsigned long long k = key2(sm.W[a][tid]);
      m = k > m ? k : m;
    }
    sm.eW[tid] = oz::key_exponent(m);
  }
  __syncthreads();
  for (int e = tid; e < kNB * kTN; e += kThreads) {
    const int j = e / kNB, a = e % kNB;
    if (8 * (j >> 3) >= ncols) continue;             // column group beyond ncols: not read
    const double2 w = sm.W[a][j];
    oz::split_store<S>(w.x, sm.eW[j], &sm.u.p3.B[0][0][j][a], 2 * kTN * kLD2);
    oz::split_store<S>(w.y, sm.eW[j], &sm.u.p3.B[0][1][j][a], 2 * kTN * kLD2);
  }

  // ---- pass 3: X -= V W'; warp w owns rows 16w..16w+15 of each 64-row chunk
  // and the target columns as n8 tiles (those below ncols). For each tile all
  // S groups accumulate at once; the tile's X values are loaded before its
  // products. The groups are folded into one int64 per entry (resolution
  // 2^-50 of the row and column scales) and subtracted from X in that fixed
  // point (sub_scaled): integer instructions only.
  const int knext = k0 + kNB;
  for (int r0 = r1st; r0 < rhi; r0 += kRC) {
    __syncthreads();
    const int rr0 = r0 - k0;
    if (tid < kRC) sm.eV[tid] = pd.ex[kNB + rr0 + tid];
    // V row digits of local rows rr0 .. rr0+63: 8 words per (digit, part, row)
    for (int e = tid; e < S * 2 * kRC * (kNB / 8); e += kThreads) {
      const int w4 = e % (kNB / 8), rowi = e / (kNB / 8);     // rowi = (s*2 + part)*kRC + r
      const int sp = rowi / kRC, r = rowi % kRC;
      const uint4 val =
          reinterpret_cast<const uint4 *>(pd.v + ((size_t)sp * pd.kp + rr0 + r) * kNB)[w4];
      reinterpret_cast<uint4 *>(&sm.u.p3.A[0][0][0][0] + rowi * kLD2)[w4] = val;
    }
    __syncthreads();
    if (r0 + 16 * warp >= rhi) continue;
    // X values of tile nt + 1 are loaded while tile nt's products run
    auto load_x = [&](int nt, double2 (&xv)[4]) {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int i = r0 + 16 * warp + grp + (q >= 2 ? 8 : 0);
        const int j = 8 * nt + 2 * tig + (q & 1);
        xv[q] = (i < rhi && j < ncols) ? X[(size_t)j * ldx + i - xoff] : make_double2(0.0, 0.0);
      }
    };
    double2 xnext[4];
    load_x(0, xnext);
#pragma unroll 1
    for (int nt = 0; nt < kTN / 8; ++nt) {
      if (8 * nt >= ncols) break;
      double2 xv[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) xv[q] = xnext[q];
      if (nt + 1 < kTN / 8 && 8 * (nt + 1) < ncols) load_x(nt + 1, xnext);
      float acc[S][2][4];
#pragma unroll
      for (int g = 0; g < S; ++g)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[g][0][q] = acc[g][1][q] = 0.0f;
#pragma unroll
      for (int s = 1; s <= S; ++s) {
        uint32_t ar[4], ai[4];
        oz::ldsm_x4(ar, &sm.u.p3.A[s - 1][0][16 * warp + a_row][a_k]);
        oz::ldsm_x4(ai, &sm.u.p3.A[s - 1][1][16 * warp + a_row][a_k]);
#pragma unroll
        for (int t = 1; t <= S + 1 - s; ++t) {
          uint32_t b[4];                    // re k0-7, re k8-15, im k0-7, im k8-15
          oz::ldsm_x4(b, &sm.u.p3.B[t - 1][lmat >> 1][8 * nt + lrow][8 * (lmat & 1)]);
          const uint32_t br[2] = {b[0], b[1]}, bi[2] = {b[2], b[3]};
          oz::cmma(acc[s + t - 2][0], acc[s + t - 2][1], ar, ai, br, bi);
        }
      }
      long long ta[2][4] = {}, tb[2][4] = {};
      if constexpr (FE) {
#pragma unroll
        for (int g = 2; g <= S + 1; g += 2)
#pragma unroll
          for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int c = 0; c < 2; ++c) {
              if (g + 1 <= S + 1 && 50 >= 7 * g) {
                oz::fold_fixed_pair<50>(ta[c][q], g, acc[g - 2][c][q], acc[g - 1][c][q]);
              } else {
                oz::fold_fixed<50>(ta[c][q], g, acc[g - 2][c][q]);
                if (g + 1 <= S + 1) oz::fold_fixed<50>(ta[c][q], g + 1, acc[g - 1][c][q]);
              }
            }
      } else {
#pragma unroll
        for (int g = 2; g <= S + 1; ++g)
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            oz::fold_group<S>(ta[0][q], tb[0][q], g, acc[g - 2][0][q]);
            oz::fold_group<S>(ta[1][q], tb[1][q], g, acc[g - 2][1][q]);
          }
      }
      unsigned long long cm[2] = {0ull, 0ull};
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int r = 16 * warp + grp + (q >= 2 ? 8 : 0);
        const int i = r0 + r, j = 8 * nt + 2 * tig + (q & 1);
        if (i < rhi && j < ncols) {
          double2 v;
          if constexpr (FE) {
            const int e = sm.eV[r] + sm.eW[j] - 50;
            v.x = oz::sub_scaled(xv[q].x, ta[0][q], e);
            v.y = oz::sub_scaled(xv[q].y, ta[1][q], e);
          } else {
            const int e = sm.eV[r] + sm.eW[j] + oz::unfold1_shift<S>();
            v.x = xv[q].x - oz::scaled_to_double(oz::unfold1_int<S>(ta[0][q], tb[0][q]), e);
            v.y = xv[q].y - oz::scaled_to_double(oz::unfold1_int<S>(ta[1][q], tb[1][q]), e);
          }
          X[(size_t)j * ldx + i - xoff] = v;
          if (i >= knext) {
            const unsigned long long k = key2(v);
            cm[q & 1] = k > cm[q & 1] ? k : cm[q & 1];
          }
        }
      }
      // column keys over rows >= k0 + kNB: lanes with the same tig share columns
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        unsigned long long m = cm[c];
#pragma unroll
        for (int o = 4; o < 32; o <<= 1) {
          const unsigned long long w = __shfl_xor_sync(0xffffffffu, m, o);
          m = w > m ? w : m;
        }
        if (grp == 0 && m != 0ull) atomicMax(&sm.kNext[8 * nt + 2 * tig + c], m);
      }
    }
  }
  __syncthreads();
  if (kout != nullptr && tid < ncols) kout[tid] = sm.kNext[tid];
}

// Work items (task, column tile) taken blockIdx.x, blockIdx.x + gridDim.x,
// ...: a grid of one CTA per item, or a persistent grid of one CTA per SM
// (the tuning's choice). Three CTAs' worth of registers per SM (at most 170
// each), so two update CTAs leave room for a panel CTA on the same SM.
template <int S>
__global__ void __launch_bounds__(kThreads, 3)
qr_update_split_kernel(const ObsDev *__restrict__ obs, const int *__restrict__ task_obs,
                       const int *__restrict__ task_mode, int p, int col_off, int max_cols,
                       int ntasks, int ntiles, bool use_y) {
  extern __shared__ __align__(16) unsigned char smraw[];
  OzSmem<S> &sm = *reinterpret_cast<OzSmem<S> *>(smraw);
  for (int item = blockIdx.x; item < ntasks * ntiles; item += gridDim.x) {
    const int task = item % ntasks, tile = item / ntasks;
    const ObsDev &o = obs[task_obs[task]];
    const int d = task_mode[task];
    const int k0 = p * kNB;
    const int nbp = min(kNB, o.cols - k0);
    const int c0 = k0 + nbp + col_off + tile * kTN;
    if (c0 >= o.cols) continue;                           // uniform over the CTA
    const int ncols = min(min(kTN, max_cols), o.cols - c0);
    double2 *A = o.A + (size_t)d * o.cols * o.rows;
    const double2 *Tg = o.T + ((size_t)d * o.npanels + p) * kNB * kNB;
    // carried column keys: slot p mod 2 written by step p-1, slot (p+1) mod 2 for step p+1
    const unsigned long long *kin =
        p > 0 ? o.ckey + ((size_t)d * 2 + (p & 1)) * o.cols + c0 : nullptr;
    unsigned long long *kout = o.ckey + ((size_t)d * 2 + ((p + 1) & 1)) * o.cols + c0;
    const int dslot = o.dig_kept ? p : (p & 1);
    PanelDigits pd = panel_digits<S>(o.vdig, o.vexp, o.kp, d, o.dig_nslot, dslot);
    if (use_y) {                                          // W' = Y^H X in one product
      pd.vh = o.ydig + ((size_t)d * 2 + (p & 1)) * (size_t)2 * S * kNB * o.kp;
      pd.exh = o.yexp + ((size_t)d * 2 + (p & 1)) * kNB;
      pd.pre_t = true;
    }
    __syncthreads();                                      // shared memory of the previous item
    oz_block_reflector_update<S>(pd, o.rows, k0, Tg, A + (size_t)c0 * o.rows, o.rows, ncols, kin,
                                 false, kout, sm);
  }
}

// The next panel's columns (the kNB after panel p) in split precision, with
// each mode's rows [k0, rows) split over a cluster of C CTAs (grid.x =
// ntasks * C): on the critical path of the factorisation, so the rows of
// one mode are spread over C SMs. Column exponents come from the keys the
// previous step's trailing update carried (scanned at the first step).
template <int S, int C>
__global__ void __launch_bounds__(kThreads)
qr_update_next_split_kernel(const ObsDev *__restrict__ obs, const int *__restrict__ task_obs,
                            const int *__restrict__ task_mode, int p) {
  const int rank = (int)cg::this_cluster().block_rank();
  const int task = blockIdx.x / C;
  const ObsDev &o = obs[task_obs[task]];
  const int d = task_mode[task];
  const int k0 = p * kNB;
  const int nbp = min(kNB, o.cols - k0);
  const int c0 = k0 + nbp;
  if (c0 >= o.cols) return;                             // uniform over the cluster
  const int ncols = min(kNB, o.cols - c0);
  const int RB = ((o.rows - k0 + C - 1) / C + 31) / 32 * 32;
  const int rlo = k0 + rank * RB, rhi = min(o.rows, rlo + RB);
  extern __shared__ __align__(16) unsigned char smraw[];
  OzSmem<S> &sm = *reinterpret_cast<OzSmem<S> *>(smraw);
  ClExtra *cx = reinterpret_cast<ClExtra *>(smraw + (sizeof(OzSmem<S>) + 15) / 16 * 16);
  double2 *A = o.A + (size_t)d * o.cols * o.rows;
  const double2 *Tg = o.T + ((size_t)d * o.npanels + p) * kNB * kNB;
  const unsigned long long *kin =
      p > 0 ? o.ckey + ((size_t)d * 2 + (p & 1)) * o.cols + c0 : nullptr;
  const int dslot = o.dig_kept ? p : (p & 1);
  oz_block_reflector_update<S, C>(panel_digits<S>(o.vdig, o.vexp, o.kp, d, o.dig_nslot, dslot),
                                  o.rows, k0, Tg, A + (size_t)c0 * o.rows, o.rows, ncols, kin,
                                  false, nullptr, sm, cx, rlo, rhi);
  cg::this_cluster().sync();                            // no CTA leaves while W' is being read
}

// L2 prefetch of what panel step p reads in the apply: this CTA's rows of the
// V^H and V digit blocks and T. The kept digit blocks of a whole operator
// exceed L2, so without it every panel step starts with DRAM-latency loads.
template <int S>
__device__ __forceinline__ void prefetch_panel_l2(const PanelDigits &pd, int k0, int rlo, int rhi,
                                                  const double2 *Tg) {
  auto pf = [](const void *p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); };
  const int tid = threadIdx.x;
  const int r1 = max(k0, rlo) - k0, r2 = rhi - k0;        // local rows of the panel's block
  if (r2 <= r1) return;
  // V^H digits: S * 2 * kNB rows of kp, this CTA's columns r1 .. r2 (128-byte lines)
  const int l1 = (r1 * 2) >> 7, l2 = ((r2 * 2 - 1) >> 7) + 1;        // lines per row
  const int nl = l2 - l1;
  for (int e = tid; e < S * 2 * kNB * nl; e += kThreads) {
    const int row = e / nl, l = l1 + e % nl;
    pf(reinterpret_cast<const char *>(pd.vh + (size_t)row * pd.kp) + 128 * l);
  }
  // V row digits: per (digit, part) the rows r1 .. r2 of kNB entries, contiguous
  const int bytes = (r2 - r1) * kNB * 2, nb = (bytes + 127) / 128;
  for (int e = tid; e < S * 2 * nb; e += kThreads) {
    const int sp = e / nb, l = e % nb;
    pf(reinterpret_cast<const char *>(pd.v + ((size_t)sp * pd.kp + r1) * kNB) + 128 * l);
  }
  if (tid < kNB * kNB * 16 / 128) pf(reinterpret_cast<const char *>(Tg) + 128 * tid);
}

// Q^H on RHS blocks with the rows of each (mode, 32-column tile) split over a
// cluster of C CTAs (grid.x = D * C): the panels stay sequential, but each
// CTA multiplies only its share of the rows, so a handful of waves' columns
// still keep C x the SMs busy.
template <int S, int C>
__global__ void __launch_bounds__(kThreads)
apply_qh_cluster_kernel(const ObsDev *__restrict__ od, double2 *__restrict__ X, int ncols_total,
                        const unsigned short *__restrict__ dig, const int *__restrict__ dex) {
  const ObsDev &o = *od;
  const int rank = (int)cg::this_cluster().block_rank();
  const int d = blockIdx.x / C;
  const int c0 = blockIdx.y * kTN;
  if (c0 >= ncols_total || !owns_mode(o, d)) return;  // uniform over the cluster
  const int ncols = min(kTN, ncols_total - c0);
  const int RB = ((o.rows + C - 1) / C + 31) / 32 * 32;
  const int rlo = rank * RB, rhi = min(o.rows, rlo + RB);
  extern __shared__ __align__(16) unsigned char smraw[];
  OzSmem<S> &sm = *reinterpret_cast<OzSmem<S> *>(smraw);
  ClExtra *cx = reinterpret_cast<ClExtra *>(smraw + (sizeof(OzSmem<S>) + 15) / 16 * 16);
  double2 *Xd = X + ((size_t)d * ncols_total + c0) * o.rows;
  prefetch_panel_l2<S>(panel_digits<S>(dig, dex, o.kp, d, o.npanels, 0), 0, rlo, rhi,
                       o.T + (size_t)d * o.npanels * kNB * kNB);
  for (int p = 0; p < o.npanels; ++p) {
    const double2 *Tg = o.T + ((size_t)d * o.npanels + p) * kNB * kNB;
    if (p + 1 < o.npanels)                              // the next step's digits into L2
      prefetch_panel_l2<S>(panel_digits<S>(dig, dex, o.kp, d, o.npanels, p + 1), (p + 1) * kNB, rlo,
                           rhi, Tg + kNB * kNB);
    oz_block_reflector_update<S, C, false>(panel_digits<S>(dig, dex, o.kp, d, o.npanels, p),
                                           o.rows, p * kNB, Tg, Xd, o.rows, ncols, nullptr, p > 0,
                                           nullptr, sm, cx, rlo, rhi);
  }
  cg::this_cluster().sync();                            // no CTA leaves while W' is being read
}

// Digits of one panel's reflectors for every active task (one CTA each).
// One CTA per (task, panel): tasks from the QR task list at panel step p
// (QR: slot p mod 2 of the mode), or every (mode, panel) of one obstacle (apply:
// task_obs == nullptr, blockIdx.x = mode, blockIdx.y = panel).
template <int S>
__global__ void __launch_bounds__(256)
panel_digits_kernel(const ObsDev *__restrict__ obs, const int *__restrict__ task_obs,
                    const int *__restrict__ task_mode, int p_qr, unsigned short *__restrict__ dig,
                    int *__restrict__ dex) {
  const bool qr = task_obs != nullptr;
  const ObsDev &o = qr ? obs[task_obs[blockIdx.x]] : obs[0];
  const int d = qr ? task_mode[blockIdx.x] : blockIdx.x;
  if (!owns_mode(o, d)) return;
  const int p = qr ? p_qr : blockIdx.y;
  // QR: two slots per mode alternating with the step, because the look-ahead
  // lets step p's trailing update still read its digits while step p+1's are
  // written; apply: one slot per panel.
  const int nslot = qr ? o.dig_nslot : o.npanels;
  const int slot = (qr && !o.dig_kept) ? (p & 1) : p;
  const int k0 = p * kNB, nbp = min(kNB, o.cols - k0), rows = o.rows, kp = o.kp;
  const double2 *A = o.A + (size_t)d * o.cols * o.rows;
  const size_t blk = digit_block<S>(kp);
  unsigned short *base = qr ? o.vdig : dig;
  int *ebase = qr ? o.vexp : dex;
  unsigned short *vh = base + ((size_t)d * nslot + slot) * blk;
  unsigned short *v = vh + blk / 2;
  int *ex = ebase + ((size_t)d * nslot + slot) * (kNB + kp);
  extern __shared__ int sexp[];                 // [kNB + kp]
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int a = warp; a < kNB; a += 8) {
    unsigned long long m = 0;
    for (int i = k0 + lane; i < rows; i += 32) {
      const unsigned long long k = key2(vget(A, rows, rows, k0, nbp, i, a));
      m = k > m ? k : m;
    }
    m = warp_max_u64(m);
    if (lane == 0) sexp[a] = oz::key_exponent(m);
  }
  for (int r = tid; r < kp; r += 256) {
    unsigned long long m = 0;
    for (int a = 0; a < kNB; ++a) {
      const unsigned long long k = key2(vget(A, rows, rows, k0, nbp, k0 + r, a));
      m = k > m ? k : m;
    }
    sexp[kNB + r] = oz::key_exponent(m);
  }
  __syncthreads();
  for (int e = tid; e < kNB + kp; e += 256) ex[e] = sexp[e];
  // V^H digits: [s][part][a][r]
  for (int e = tid; e < kNB * kp; e += 256) {
    const int a = e / kp, r = e % kp;
    const double2 x = vget(A, rows, rows, k0, nbp, k0 + r, a);
    const int ev = sexp[a];
    oz::split_store_n(x.x, ev, S, vh + (size_t)a * kp + r, (size_t)2 * kNB * kp);
    oz::split_store_n(-x.y, ev, S, vh + (size_t)(kNB + a) * kp + r, (size_t)2 * kNB * kp);
  }
  // V row digits: [s][part][r][a]
  for (int e = tid; e < kp * kNB; e += 256) {
    const int r = e / kNB, a = e % kNB;
    const double2 x = vget(A, rows, rows, k0, nbp, k0 + r, a);
    const int ev = sexp[kNB + r];
    oz::split_store_n(x.x, ev, S, v + (size_t)r * kNB + a, (size_t)2 * kp * kNB);
    oz::split_store_n(x.y, ev, S, v + (size_t)(kp + r) * kNB + a, (size_t)2 * kp * kNB);
  }
}

// Digits of panel p's reflectors over the whole GPU (split plans whose panel
// kernel wrote the reflector columns' exponents): one CTA per (task, 64 rows
// of the digit block), the same layout as panel_digits_kernel. The block's
// V rows are staged in shared memory by coalesced column reads; row
// exponents are formed here; the V^H digits are stored with consecutive
// threads on consecutive rows, the V row digits with consecutive threads on
// consecutive reflectors, so every store instruction writes contiguous bytes.
constexpr int kVdRows = 64;
template <int S>
__global__ void __launch_bounds__(256)
vdigits_kernel(const ObsDev *__restrict__ obs, const int *__restrict__ task_obs,
               const int *__restrict__ task_mode, int p) {
  const ObsDev &o = obs[task_obs[blockIdx.x]];
  const int d = task_mode[blockIdx.x];
  const int r0 = blockIdx.y * kVdRows;
  const int kp = o.kp;
  if (r0 >= kp) return;
  const int slot = o.dig_kept ? p : (p & 1);
  const int k0 = p * kNB, nbp = min(kNB, o.cols - k0), rows = o.rows;
  const double2 *A = o.A + (size_t)d * o.cols * o.rows;
  const size_t blk = (size_t)4 * S * kNB * kp;
  unsigned short *vh = o.vdig + ((size_t)d * o.dig_nslot + slot) * blk;
  unsigned short *vr = vh + blk / 2;
  int *ex = o.vexp + ((size_t)d * o.dig_nslot + slot) * (kNB + kp);
  __shared__ double2 Vs[kNB][kVdRows + 1];
  __shared__ int ecol[kNB], erow[kVdRows];
  const int tid = threadIdx.x;
  for (int e = tid; e < kNB * kVdRows; e += 256) {
    const int a = e / kVdRows, rr = e % kVdRows;
    Vs[a][rr] = vget(A, rows, rows, k0, nbp, k0 + r0 + rr, a);
  }
  if (tid < kNB) ecol[tid] = ex[tid];                    // written by the panel kernel
  __syncthreads();
  if (tid < kVdRows) {
    unsigned long long m = 0ull;
#pragma unroll
    for (int a = 0; a < kNB; ++a) {
      const unsigned long long k = key2(Vs[a][tid]);
      m = k > m ? k : m;
    }
    erow[tid] = oz::key_exponent(m);
    ex[kNB + r0 + tid] = erow[tid];
  }
  __syncthreads();
  const size_t sh = (size_t)2 * kNB * kp, sv = (size_t)2 * kp * kNB;
  for (int e = tid; e < kNB * kVdRows; e += 256) {        // V^H: [s][part][a][r]
    const int a = e / kVdRows, rr = e % kVdRows;
    const double2 x = Vs[a][rr];
    oz::split_store<S>(x.x, ecol[a], reinterpret_cast<__nv_bfloat16 *>(vh + (size_t)a * kp + r0 + rr), (int)sh);
    oz::split_store<S>(-x.y, ecol[a], reinterpret_cast<__nv_bfloat16 *>(vh + (size_t)(kNB + a) * kp + r0 + rr),
                       (int)sh);
  }
  for (int e = tid; e < kNB * kVdRows; e += 256) {        // V rows: [s][part][r][a]
    const int rr = e / kNB, a = e % kNB;
    const double2 x = Vs[a][rr];
    oz::split_store<S>(x.x, erow[rr], reinterpret_cast<__nv_bfloat16 *>(vr + (size_t)(r0 + rr) * kNB + a), (int)sv);
    oz::split_store<S>(x.y, erow[rr], reinterpret_cast<__nv_bfloat16 *>(vr + (size_t)(kp + r0 + rr) * kNB + a),
                       (int)sv);
  }
}

// Y = V T for panel p (the trailing update then forms W' = Y^H X in one
// product, with no FP64 T^H W per column tile): one CTA per (task, 64 rows),
// rows of V staged with their unit diagonal, Y written column by column
// ([16][kp] per mode and slot p mod 2), the largest |Y| of each column into
// ykey by atomic maximum (cleared by the panel kernel of step p).
__global__ void __launch_bounds__(256)
y_rows_kernel(const ObsDev *__restrict__ obs, const int *__restrict__ task_obs,
              const int *__restrict__ task_mode, int p) {
  const ObsDev &o = obs[task_obs[blockIdx.x]];
  const int d = task_mode[blockIdx.x];
  const int r0 = blockIdx.y * kVdRows, kp = o.kp;
  if (r0 >= kp) return;
  const int k0 = p * kNB, nbp = min(kNB, o.cols - k0), rows = o.rows;
  const double2 *A = o.A + (size_t)d * o.cols * o.rows;
  const double2 *Tg = o.T + ((size_t)d * o.npanels + p) * kNB * kNB;
  double2 *Y = o.ybuf + ((size_t)d * 2 + (p & 1)) * kNB * kp;
  unsigned long long *yk = o.ykey + ((size_t)d * 2 + (p & 1)) * kNB;
  __shared__ double2 Vs[kVdRows][kNB + 1], Ts[kNB][kNB + 1];
  __shared__ unsigned long long wk[8][kNB];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int e = tid; e < kNB * kVdRows; e += 256) {
    const int a = e / kVdRows, rr = e % kVdRows;
    Vs[rr][a] = vget(A, rows, rows, k0, nbp, k0 + r0 + rr, a);
  }
  for (int e = tid; e < kNB * kNB; e += 256) Ts[e % kNB][e / kNB] = Tg[e];
  __syncthreads();
  // thread = (column b = tid / 16, 4 rows)
  const int b = tid >> 4, rq = (tid & 15) * 4;
  unsigned long long mk = 0ull;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int rr = rq + u;
    double2 y = make_double2(0.0, 0.0);
    for (int a = 0; a <= b; ++a) {
      const double2 v = Vs[rr][a], t = Ts[a][b];
      y.x = fma(v.x, t.x, fma(-v.y, t.y, y.x));
      y.y = fma(v.x, t.y, fma(v.y, t.x, y.y));
    }
    Y[(size_t)b * kp + r0 + rr] = y;
    const unsigned long long k = key2(y);
    mk = k > mk ? k : mk;
  }
  // column maxima: the 16 threads of a column are consecutive lanes
#pragma unroll
  for (int off = 8; off > 0; off >>= 1) {
    const unsigned long long w = __shfl_xor_sync(0xffffffffu, mk, off);
    mk = w > mk ? w : mk;
  }
  if ((lane & 15) == 0) wk[warp][lane >> 4] = mk;       // warp w holds columns 2w, 2w + 1
  __syncthreads();
  if (tid < kNB) {
    const unsigned long long m = wk[tid >> 1][tid & 1];
    if (m) atomicMax(yk + tid, m);
  }
}

// Digits of Y^H (conjugated, one exponent per column of Y, the layout of the
// V^H digits) from y_rows_kernel's Y and column maxima.
template <int S>
__global__ void __launch_bounds__(256)
ydigits_kernel(const ObsDev *__restrict__ obs, const int *__restrict__ task_obs,
               const int *__restrict__ task_mode, int p) {
  const ObsDev &o = obs[task_obs[blockIdx.x]];
  const int d = task_mode[blockIdx.x];
  const int r0 = blockIdx.y * kVdRows, kp = o.kp;
  if (r0 >= kp) return;
  const int slot = p & 1;
  const double2 *Y = o.ybuf + ((size_t)d * 2 + slot) * kNB * kp;
  const unsigned long long *yk = o.ykey + ((size_t)d * 2 + slot) * kNB;
  unsigned short *yh = o.ydig + ((size_t)d * 2 + slot) * (size_t)2 * S * kNB * kp;
  int *ye = o.yexp + ((size_t)d * 2 + slot) * kNB;
  __shared__ int ecol[kNB];
  const int tid = threadIdx.x;
  if (tid < kNB) {
    ecol[tid] = oz::key_exponent(yk[tid]);
    if (blockIdx.y == 0) ye[tid] = ecol[tid];
  }
  __syncthreads();
  const size_t sh = (size_t)2 * kNB * kp;
  for (int e = tid; e < kNB * kVdRows; e += 256) {        // [s][part][b][r]
    const int b = e / kVdRows, rr = e % kVdRows;
    const double2 y = Y[(size_t)b * kp + r0 + rr];
    oz::split_store<S>(y.x, ecol[b], reinterpret_cast<__nv_bfloat16 *>(yh + (size_t)b * kp + r0 + rr), (int)sh);
    oz::split_store<S>(-y.y, ecol[b], reinterpret_cast<__nv_bfloat16 *>(yh + (size_t)(kNB + b) * kp + r0 + rr),
                       (int)sh);
  }
}

template <int S>
cudaError_t launch_digits_s(const ObsDev *d_obs, const int *d_task_obs, const int *d_task_mode,
                            int ntasks, int p, int kp_max, cudaStream_t st) {
  const size_t smem = sizeof(int) * (kNB + kp_max);     // exponents of the tallest task
  static size_t granted = 0;
  const cudaError_t e = ensure_dynamic_smem(panel_digits_kernel<S>, smem, granted);
  if (e != cudaSuccess) return e;
  static const bool carve = (prefer_max_shared(panel_digits_kernel<S>), true);
  (void)carve;
  panel_digits_kernel<S><<<ntasks, 256, smem, st>>>(d_obs, d_task_obs, d_task_mode, p, nullptr,
                                                    nullptr);
  return cudaGetLastError();
}

template <int S>
cudaError_t launch_update_s(const ObsDev *d_obs, const int *d_task_obs, const int *d_task_mode,
                            int ntasks, int p, int col_off, int ntiles, int max_cols,
                            bool persistent, bool use_y, cudaStream_t st) {
  const size_t smem = sizeof(OzSmem<S>);
  static size_t granted = 0;
  cudaError_t e = ensure_dynamic_smem(qr_update_split_kernel<S>, smem, granted);
  if (e != cudaSuccess) return e;
  static const bool carve = (prefer_max_shared(qr_update_split_kernel<S>), true);
  (void)carve;
  const int items = ntasks * ntiles;
  const int grid = persistent ? min(items, sm_count()) : items;
  qr_update_split_kernel<S><<<grid, kThreads, smem, st>>>(d_obs, d_task_obs, d_task_mode, p,
                                                          col_off, max_cols, ntasks, ntiles, use_y);
  return cudaGetLastError();
}

template <int S, int C>
cudaError_t launch_next_split_s(const ObsDev *d_obs, const int *d_task_obs, const int *d_task_mode,
                                int ntasks, int p, cudaStream_t st) {
  const size_t smem = (sizeof(OzSmem<S>) + 15) / 16 * 16 + sizeof(ClExtra);
  static size_t granted = 0;
  cudaError_t e = ensure_dynamic_smem(qr_update_next_split_kernel<S, C>, smem, granted);
  if (e != cudaSuccess) return e;
  static const bool carve = (prefer_max_shared(qr_update_next_split_kernel<S, C>), true);
  (void)carve;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(ntasks * C);
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = C;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, qr_update_next_split_kernel<S, C>, d_obs, d_task_obs, d_task_mode, p);
}

template <int S>
cudaError_t launch_next_split_c(const ObsDev *d_obs, const int *d_task_obs, const int *d_task_mode,
                                int ntasks, int p, int max_rows, int cluster, cudaStream_t st) {
  // cluster 0 (auto): rows per CTA a 64-row chunk or more in each member of
  // the cluster, at most about one CTA per SM (the trailing update holds one
  // CTA on each); else the tuning's 1, 2 or 4
  int C = cluster;
  if (C == 0) C = (max_rows >= 256 && 4 * ntasks <= sm_count()) ? 4 : 2;
  if (C == 4) return launch_next_split_s<S, 4>(d_obs, d_task_obs, d_task_mode, ntasks, p, st);
  if (C == 1) return launch_next_split_s<S, 1>(d_obs, d_task_obs, d_task_mode, ntasks, p, st);
  return launch_next_split_s<S, 2>(d_obs, d_task_obs, d_task_mode, ntasks, p, st);
}

template <int S, int C>
cudaError_t launch_apply_cluster_s(const ObsDev *d_o, const ObsDev &h, double2 *X, int ncol,
                                   unsigned short *dig, int *dex, cudaStream_t st) {
  const size_t smem = (sizeof(OzSmem<S>) + 15) / 16 * 16 + sizeof(ClExtra);
  static size_t granted = 0;
  cudaError_t e = ensure_dynamic_smem(apply_qh_cluster_kernel<S, C>, smem, granted);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(h.D * C, (ncol + kTN - 1) / kTN);
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = C;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, apply_qh_cluster_kernel<S, C>, d_o, X, ncol,
                            (const unsigned short *)dig, (const int *)dex);
}

template <int S>
cudaError_t launch_apply_qh_s(const ObsDev *d_o, const ObsDev &h, double2 *X, int ncol,
                              unsigned short *dig, int *dex, bool kept, cudaStream_t st) {
  if (!kept) {
    static size_t granted_d = 0;
    cudaError_t e = ensure_dynamic_smem(panel_digits_kernel<S>, sizeof(int) * (kNB + h.kp), granted_d);
    if (e != cudaSuccess) return e;
    panel_digits_kernel<S><<<dim3(h.D, h.npanels), 256, sizeof(int) * (kNB + h.kp), st>>>(
        d_o, nullptr, nullptr, 0, dig, dex);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  // rows split over a cluster of 4 CTAs (2 for short panels); every cluster
  // loops over all panels, so clusters that do not find room beside the
  // first wave of CTAs (two per SM) would run a whole second pass: auto takes
  // 4 only when D x 4 CTAs fit in one wave
  int C = h.apply_cluster;
  if (C == 0) {
    const int tiles = (ncol + kTN - 1) / kTN;
    C = (h.rows >= 192 && (long long)h.D * tiles * 4 <= 2ll * sm_count()) ? 4 : 2;
  }
  if (C == 4) return launch_apply_cluster_s<S, 4>(d_o, h, X, ncol, dig, dex, st);
  return launch_apply_cluster_s<S, 2>(d_o, h, X, ncol, dig, dex, st);
}

}  // namespace

bool split_slices_supported(int s) { return s >= 4 && s <= 8; }


int split_update_tile_cols() { return kTN; }

cudaError_t launch_qr_update_split(const ObsDev *d_obs, const int *d_task_obs,
                                   const int *d_task_mode, int ntasks, int p, int slices,
                                   int col_off, int ntiles, int max_cols, bool persistent,
                                   bool use_y, cudaStream_t st) {
  switch (slices) {
    case 4: return launch_update_s<4>(d_obs, d_task_obs, d_task_mode, ntasks, p, col_off, ntiles,
                                          max_cols, persistent, use_y, st);
    case 5: return launch_update_s<5>(d_obs, d_task_obs, d_task_mode, ntasks, p, col_off, ntiles,
                                          max_cols, persistent, use_y, st);
    case 6: return launch_update_s<6>(d_obs, d_task_obs, d_task_mode, ntasks, p, col_off, ntiles,
                                          max_cols, persistent, use_y, st);
    case 7: return launch_update_s<7>(d_obs, d_task_obs, d_task_mode, ntasks, p, col_off, ntiles,
                                          max_cols, persistent, use_y, st);
    case 8: return launch_update_s<8>(d_obs, d_task_obs, d_task_mode, ntasks, p, col_off, ntiles,
                                          max_cols, persistent, use_y, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_vdigits(const ObsDev *d_obs, const int *d_task_obs, const int *d_task_mode,
                           int ntasks, int p, int kp_max, int slices, cudaStream_t st) {
  if (ntasks <= 0) return cudaSuccess;
  const dim3 grid(ntasks, kp_max / kVdRows);
  switch (slices) {
    case 4: vdigits_kernel<4><<<grid, 256, 0, st>>>(d_obs, d_task_obs, d_task_mode, p); break;
    case 5: vdigits_kernel<5><<<grid, 256, 0, st>>>(d_obs, d_task_obs, d_task_mode, p); break;
    case 6: vdigits_kernel<6><<<grid, 256, 0, st>>>(d_obs, d_task_obs, d_task_mode, p); break;
    case 7: vdigits_kernel<7><<<grid, 256, 0, st>>>(d_obs, d_task_obs, d_task_mode, p); break;
    case 8: vdigits_kernel<8><<<grid, 256, 0, st>>>(d_obs, d_task_obs, d_task_mode, p); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_y_digits(const ObsDev *d_obs, const int *d_task_obs, const int *d_task_mode,
                            int ntasks, int p, int kp_max, int slices, cudaStream_t st) {
  if (ntasks <= 0) return cudaSuccess;
  const dim3 grid(ntasks, kp_max / kVdRows);
  y_rows_kernel<<<grid, 256, 0, st>>>(d_obs, d_task_obs, d_task_mode, p);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  switch (slices) {
    case 4: ydigits_kernel<4><<<grid, 256, 0, st>>>(d_obs, d_task_obs, d_task_mode, p); break;
    case 5: ydigits_kernel<5><<<grid, 256, 0, st>>>(d_obs, d_task_obs, d_task_mode, p); break;
    case 6: ydigits_kernel<6><<<grid, 256, 0, st>>>(d_obs, d_task_obs, d_task_mode, p); break;
    case 7: ydigits_kernel<7><<<grid, 256, 0, st>>>(d_obs, d_task_obs, d_task_mode, p); break;
    case 8: ydigits_kernel<8><<<grid, 256, 0, st>>>(d_obs, d_task_obs, d_task_mode, p); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_qr_update_next_split(const ObsDev *d_obs, const int *d_task_obs,
                                        const int *d_task_mode, int ntasks, int p, int slices,
                                        int max_rows, int cluster, cudaStream_t st) {
  if (ntasks <= 0) return cudaSuccess;
  switch (slices) {
    case 4: return launch_next_split_c<4>(d_obs, d_task_obs, d_task_mode, ntasks, p, max_rows, cluster, st);
    case 5: return launch_next_split_c<5>(d_obs, d_task_obs, d_task_mode, ntasks, p, max_rows, cluster, st);
    case 6: return launch_next_split_c<6>(d_obs, d_task_obs, d_task_mode, ntasks, p, max_rows, cluster, st);
    case 7: return launch_next_split_c<7>(d_obs, d_task_obs, d_task_mode, ntasks, p, max_rows, cluster, st);
    case 8: return launch_next_split_c<8>(d_obs, d_task_obs, d_task_mode, ntasks, p, max_rows, cluster, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_panel_digits(const ObsDev *d_obs, const int *d_task_obs, const int *d_task_mode,
                                int ntasks, int p, int slices, int kp_max, cudaStream_t st) {
  if (ntasks <= 0) return cudaSuccess;
  switch (slices) {
    case 4: return launch_digits_s<4>(d_obs, d_task_obs, d_task_mode, ntasks, p, kp_max, st);
    case 5: return launch_digits_s<5>(d_obs, d_task_obs, d_task_mode, ntasks, p, kp_max, st);
    case 6: return launch_digits_s<6>(d_obs, d_task_obs, d_task_mode, ntasks, p, kp_max, st);
    case 7: return launch_digits_s<7>(d_obs, d_task_obs, d_task_mode, ntasks, p, kp_max, st);
    case 8: return launch_digits_s<8>(d_obs, d_task_obs, d_task_mode, ntasks, p, kp_max, st);
    default: return cudaErrorInvalidValue;
  }
}

size_t apply_digit_bytes(const ObsDev &h) {
  if (h.slices <= 0 || h.dig_kept) return 0;                 // kept from the build
  const size_t blocks = (size_t)h.D * h.npanels;
  const size_t dig = blocks * 4 * (size_t)h.slices * kNB * h.kp * sizeof(unsigned short);
  return ((dig + 255) & ~(size_t)255) + blocks * (kNB + h.kp) * sizeof(int);
}

cudaError_t launch_apply_qh_split(const ObsDev *d_o, const ObsDev &h, double2 *X, int ncol,
                                  void *digit_scratch, cudaStream_t st) {
  const size_t blocks = (size_t)h.D * h.npanels;
  const size_t dig = blocks * 4 * (size_t)h.slices * kNB * h.kp * sizeof(unsigned short);
  const bool kept = h.dig_kept != 0;                    // the build left every panel's digits
  unsigned short *dg = kept ? h.vdig : static_cast<unsigned short *>(digit_scratch);
  int *dx = kept ? h.vexp
                 : reinterpret_cast<int *>(static_cast<char *>(digit_scratch) +
                                           ((dig + 255) & ~(size_t)255));
  switch (h.slices) {
    case 4: return launch_apply_qh_s<4>(d_o, h, X, ncol, dg, dx, kept, st);
    case 5: return launch_apply_qh_s<5>(d_o, h, X, ncol, dg, dx, kept, st);
    case 6: return launch_apply_qh_s<6>(d_o, h, X, ncol, dg, dx, kept, st);
    case 7: return launch_apply_qh_s<7>(d_o, h, X, ncol, dg, dx, kept, st);
    case 8: return launch_apply_qh_s<8>(d_o, h, X, ncol, dg, dx, kept, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace axi
