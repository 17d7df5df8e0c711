// Trailing update of the split-precision QR on fifth-generation tensor cores.
//
// For panel p, a tile of 64 trailing columns X (rows k0 .. rows-1) of one mode
// is updated as
//     X <- X - V W',   W' = Y^H X,   Y = V T          (compact WY, Sec. 3)
// with both products as BF16 digit products on tcgen05.mma (kind::f16, FP32
// accumulators in tensor memory), the digits as in ozaki.cuh: X split on the
// fly with one bit of headroom (digits in [-64, 65]), Y^H (ydigits_kernel), V's
// rows (vdigits_kernel) and W' balanced (|d| <= 128).
//
// First product, W'^T = X^T conj(Y) contracted over the rows in 16-row chunks:
// the 128 MMA rows are [Re X ; Im X] of the 64 columns, the N columns the
// 16 columns of Re Y^H then Im Y^H, per digit; one MMA per digit s of X against
// the stacked digits t = 1 .. S+1-s of Y^H lands digit group g = s + t at
// tensor-memory columns 32 (g - 2). A group sums at most 16 rows x 7 pairs x
// 65 x 128 < 2^20 per chunk, so the accumulators are read every 4 chunks (sums
// below 2^22, exact in FP32) into one int64 per entry, a fixed point of
// resolution 2^-47 relative to the column scales (exact but for the rounding
// of groups g > 6; no FP64 instruction until W' is formed). Then
//   W'_re = P(Re X, Re Y^H) - P(Im X, Im Y^H),  W'_im = P(Im X, Re Y^H) + P(Re X, Im Y^H),
// exchanged through shared memory.
//
// Second product, for 128 rows and 16 columns at a time:
//   D_re = [Vr | Vi] [W'r ; -W'i],   D_im = [Vr | Vi] [W'i ; W'r]     (K = 32),
// one pair of K = 16 MMAs per digit s of V against the stacked digits of W'
// (group g at columns 16 (g - 2), imaginary parts 16 S further); a group sums at
// most 32 x 7 x 128 x 128 < 2^22, exact in one pass. The epilogue folds the
// groups into one int64 per entry (resolution 2^-50 relative to the row and
// column scales), subtracts it from X in that fixed point (ozaki.cuh
// sub_scaled: integer instructions, one rounding) and
// keeps, per column, the high word of the largest |entry|'s IEEE key over the
// next step's rows (the exponent is all the next step's split needs).
//
// Loads are asynchronous and one step ahead: the raw X values and Y^H digits of
// chunk c + 1 are copied (cp.async, 16 bytes per copy) while chunk c is split,
// the V-row digits of a 128-row block likewise, and the X values the epilogue
// subtracts from are loaded before it waits for its MMAs. Digit tiles sit in
// shared memory in the no-swizzle K-major layout (tcgen05.cuh), made visible
// to the tensor core with a proxy fence; thread 0 issues the MMAs; completion
// comes back through mbarriers with bounded waits (on expiry the timeout bit of the status word
// is set, in-flight MMAs are waited for with a bound, tensor memory is freed
// and the CTA returns; the decision to stop is block-uniform, taken by
// __syncthreads_or).
#include "axi_internal.h"
#include "ozaki.cuh"
#include "tcgen05.cuh"

namespace axi {
namespace {

constexpr int kUC = 64;                 // X columns per CTA
constexpr int kUT = 256;                // threads
constexpr int kFold = 4;                // 16-row chunks per fold of the first product
constexpr int kR1 = 47;                 // fixed-point resolution bits, first product
constexpr int kR2 = 50;                 // and second product
constexpr uint32_t kTmemCols = 256;
constexpr long long kWaitCycles = 2000000000ll;
constexpr int kRawLd = 17;             // raw X column stride (complex): conflict-free 16-byte reads
constexpr uint32_t kRawBytes = kRawLd * kUC * 16;   // one chunk of raw X: [64 columns][16 rows] complex

__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// K-major no-swizzle core-matrix offset (bytes) of element (r, k) of a tile
// whose rows are `kw` elements wide (kw = 16: SBO 256; kw = 32: SBO 512).
__device__ __forceinline__ uint32_t core_off(int r, int k, int kw) {
  return (uint32_t)((r >> 3) * (kw * 16) + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

template <int S>
struct TcLayout {
  // first product: A1 [S][128 x 16] (4 KB per digit), two stages of raw X
  // chunks and two of B1 [S][32 x 16] (1 KB per digit)
  static constexpr uint32_t kA1 = S * 4096;
  static constexpr uint32_t kRaw = kA1;
  static constexpr uint32_t kB1 = kRaw + 2 * kRawBytes;
  static constexpr uint32_t kOps = kB1 + 2 * S * 1024;
  // second product (aliases the first's area): A2 [S][128 x 32] (8 KB per
  // digit), B2 [2 variants][S][16 x 32] (1 KB per digit)
  static constexpr uint32_t kA2 = S * 8192, kB2 = 2 * S * 1024;
  static_assert(kA2 + kB2 <= kOps, "second product fits the operand area");
  // FP64 exchange of the first product (aliases the operand area after it)
  static_assert(128 * 33 * 8 <= kOps, "exchange fits the operand area");
  static constexpr uint32_t kW = 16 * kUC * 16;      // W' [16][64] complex
  static constexpr uint32_t kTotal = kOps + kW;
};

template <int S>
__global__ void __launch_bounds__(kUT, 2)
qr_update_tc_kernel(const ObsDev *__restrict__ obs, const int *__restrict__ task_obs,
                    const int *__restrict__ task_mode, int p, int ntasks) {
  using L = TcLayout<S>;
  const int task = blockIdx.x % ntasks, tile = blockIdx.x / ntasks;
  const ObsDev &o = obs[task_obs[task]];
  const int d = task_mode[task];
  const int k0 = p * kNB, nbp = min(kNB, o.cols - k0);
  const int c0 = k0 + nbp + kNB + tile * kUC;          // beyond the next panel's columns
  if (c0 >= o.cols) return;                             // uniform over the CTA
  const int ncols = min(kUC, o.cols - c0);
  const int rows = o.rows, K = rows - k0, nch = (K + 15) / 16, kp = o.kp;
  double2 *X = o.A + (size_t)d * o.cols * rows + (size_t)c0 * rows;
  const unsigned short *yh = o.ydig + ((size_t)d * 2 + (p & 1)) * (size_t)2 * S * kNB * kp;
  const int *yex = o.yexp + ((size_t)d * 2 + (p & 1)) * kNB;
  const int dslot = o.dig_kept ? p : (p & 1);
  const size_t vblk = (size_t)4 * S * kNB * kp;
  const unsigned short *vr = o.vdig + ((size_t)d * o.dig_nslot + dslot) * vblk + vblk / 2;
  const int *vex = o.vexp + ((size_t)d * o.dig_nslot + dslot) * (kNB + kp) + kNB;
  const unsigned long long *kin = p > 0 ? o.ckey + ((size_t)d * 2 + (p & 1)) * o.cols + c0 : nullptr;
  unsigned long long *kout = o.ckey + ((size_t)d * 2 + ((p + 1) & 1)) * o.cols + c0;

  extern __shared__ __align__(1024) unsigned char usm[];
  unsigned char *A1 = usm;
  double2 *Wp = reinterpret_cast<double2 *>(usm + L::kOps);           // W' [b][j]
  __shared__ __align__(8) uint64_t mma_done, acc_full, d_full, drain;
  __shared__ uint32_t tmem_base;
  __shared__ int eX[kUC], eW[kUC], eY[kNB];
  __shared__ unsigned knext[kUC];        // high words of the column keys (exponent bits)
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int quad = warp & 3, half = warp >> 2;

  if (warp == 0) tc::tmem_alloc(&tmem_base, kTmemCols);
  if (tid == 0) {
    tc::mbar_init(&mma_done, 1);
    tc::mbar_init(&acc_full, 1);
    tc::mbar_init(&d_full, 1);
    tc::mbar_init(&drain, 1);
  }
  // Chunk c's raw X (thread: column tid / 4, rows 4 (tid % 4) .. +3, the
  // values it splits itself) and Y^H digits (row n = 16 part + b' of digit t:
  // Y^H digit (part, b') at rows i0 .. i0 + 15, two 16-byte pieces from the
  // [t][part][b'][kp] layout) into stage c mod 2, one commit group per chunk.
  const int xj = tid >> 2, xk = (tid & 3) * 4;
  auto issue = [&](int c) {
    const int stg = c & 1, i0 = k0 + 16 * c;
    double2 *raw = reinterpret_cast<double2 *>(usm + L::kRaw + stg * kRawBytes);
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int i = i0 + xk + u;
      const bool valid = xj < ncols && i < rows;
      oz::cp_async16(raw + xj * kRawLd + xk + u, valid ? X + (size_t)xj * rows + i : X, valid);
    }
    unsigned char *B1 = usm + L::kB1 + stg * S * 1024;
    for (int e = tid; e < S * 32 * 2; e += kUT) {
      const int t = e / 64, n = (e / 2) & 31, kg = e & 1;
      oz::cp_async16(B1 + t * 1024 + core_off(n, 8 * kg, 16),
                     yh + ((size_t)(t * 2 + (n >> 4)) * kNB + (n & 15)) * kp + (i0 - k0) + 8 * kg, true);
    }
    oz::cp_async_commit();
  };
  issue(0);                                             // overlaps the set-up below
  if (tid < kNB) eY[tid] = yex[tid];
  if (tid < kUC) knext[tid] = 0u;
  // column exponents of X over rows k0.. (carried keys, else a scan), one bit of headroom
  if (kin != nullptr) {
    if (tid < kUC) eX[tid] = tid < ncols ? oz::key_exponent(kin[tid]) + 1 : 0;
  } else {
    for (int j = warp; j < kUC; j += kUT / 32) {
      unsigned long long m = 0;
      if (j < ncols) {
#pragma unroll 4
        for (int i = k0 + lane; i < rows; i += 32) {
          const unsigned long long k = oz::abs_key2(X[(size_t)j * rows + i]);
          m = k > m ? k : m;
        }
      }
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        const unsigned long long w = __shfl_xor_sync(0xffffffffu, m, off);
        m = w > m ? w : m;
      }
      if (lane == 0) eX[j] = oz::key_exponent(m) + 1;
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tmem_base;
  const uint32_t lane_addr = (uint32_t)(32 * quad) << 16;

  // ---- first product: W'^T = X^T conj(Y) over the rows
  // fixed-point sums (resolution 2^-kR1 of the scale 2^(eX + eY)): below
  // 2^(22 + kR1 - 14) per fold, so 256 folds (16384 rows) fit 63 bits
  long long tacc[16];
#pragma unroll
  for (int q = 0; q < 16; ++q) tacc[q] = 0;
  const int prow = 32 * quad + lane, pj = prow & 63;
  int nfold = 0;
  bool ok = true;
  for (int c = 0; c < nch; ++c) {
    // MMA(c - 1) done: A1 and stage (c + 1) mod 2 are free
    bool w = true;
    if (c >= 1) w = tc::mbar_wait(&mma_done, (c - 1) & 1, kWaitCycles);
    if (__syncthreads_or(!w)) { ok = false; break; }
    if (c + 1 < nch) issue(c + 1);
    else oz::cp_async_commit();                         // empty group: chunk c's is the older one
    oz::cp_async_wait<1>();
    // A1: rows r < 64 Re X(:, r), r >= 64 Im X(:, r - 64); k = row i0 + k
    {
      const double2 *raw = reinterpret_cast<const double2 *>(usm + L::kRaw + (c & 1) * kRawBytes);
      const int e = eX[xj];
#pragma unroll
      for (int pr = 0; pr < 2; ++pr) {
        const double2 x0 = raw[xj * kRawLd + xk + 2 * pr], x1 = raw[xj * kRawLd + xk + 2 * pr + 1];
        uint32_t *dre = reinterpret_cast<uint32_t *>(A1 + core_off(xj, xk + 2 * pr, 16));
        uint32_t *dim = reinterpret_cast<uint32_t *>(A1 + core_off(64 + xj, xk + 2 * pr, 16));
        oz::split2_fast<S>(x0.x, x1.x, e, dre, 1024);
        oz::split2_fast<S>(x0.y, x1.y, e, dim, 1024);
      }
    }
    fence_proxy_async();                                // A1 writes and B1 copies -> tensor core
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const bool first = (c % kFold) == 0, fold = c % kFold == kFold - 1 || c == nch - 1;
    if (tid == 0) {
      const uint32_t a0 = tc::smem_u32(A1), b0 = tc::smem_u32(usm + L::kB1 + (c & 1) * S * 1024);
#pragma unroll
      for (int s = 1; s <= S; ++s) {
        const uint64_t da = tc::smem_desc(a0 + (s - 1) * 4096, 128, 256);
        const uint64_t db = tc::smem_desc(b0, 128, 256);
        tc::mma_bf16(tmem + (uint32_t)(32 * (s - 1)), da, db, tc::idesc_bf16_f32(128, 32 * (S + 1 - s)),
                     !(first && s == 1));
      }
      tc::commit(&mma_done);
      if (fold) tc::commit(&acc_full);
    }
    if (fold) {                                         // fold the groups
      const bool wf = tc::mbar_wait(&acc_full, nfold & 1, kWaitCycles);
      ++nfold;
      if (__syncthreads_or(!wf)) { ok = false; break; }
      tc::fence_after_sync();
#pragma unroll
      for (int qh = 0; qh < 2; ++qh) {
#pragma unroll
        for (int g = 2; g <= S + 1; g += 2) {
          uint32_t r[8], r2[8];
          tc::ld8(tmem + lane_addr + (uint32_t)(32 * (g - 2) + 16 * half + 8 * qh), r);
          if (g + 1 <= S + 1) tc::ld8(tmem + lane_addr + (uint32_t)(32 * (g - 1) + 16 * half + 8 * qh), r2);
          tc::ld_wait();
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            if (g + 1 <= S + 1 && kR1 >= 7 * g)
              oz::fold_fixed_pair<kR1>(tacc[8 * qh + q], g, __uint_as_float(r[q]), __uint_as_float(r2[q]));
            else {
              oz::fold_fixed<kR1>(tacc[8 * qh + q], g, __uint_as_float(r[q]));
              if (g + 1 <= S + 1) oz::fold_fixed<kR1>(tacc[8 * qh + q], g + 1, __uint_as_float(r2[q]));
            }
          }
        }
      }
      tc::fence_before_sync();
      __syncthreads();                                  // TMEM read before the next MMAs
    }
  }
  oz::cp_async_wait<0>();                               // no copy outlives the loop
  if (ok) {
    // P(r, n) in FP64: r = part_x * 64 + j, n = part_y * 16 + b'
    __syncthreads();
    double *P = reinterpret_cast<double *>(usm);
#pragma unroll
    for (int q = 0; q < 16; ++q)
      P[prow * 33 + 16 * half + q] = oz::scaled_to_double(tacc[q], eX[pj] + eY[q] - kR1);
    __syncthreads();
    // W'(b', j) = Y^H X: re = P(Re, Re) - P(Im, Im), im = P(Im, Re) + P(Re, Im)
    for (int e = tid; e < kNB * kUC; e += kUT) {
      const int bb = e / kUC, jj = e % kUC;
      Wp[bb * kUC + jj] = make_double2(P[jj * 33 + bb] - P[(64 + jj) * 33 + 16 + bb],
                                       P[(64 + jj) * 33 + bb] + P[jj * 33 + 16 + bb]);
    }
    __syncthreads();
    if (tid < kUC) {
      unsigned long long m = 0;
      for (int bb = 0; bb < kNB; ++bb) {
        const unsigned long long k = oz::abs_key2(Wp[bb * kUC + tid]);
        m = k > m ? k : m;
      }
      eW[tid] = oz::key_exponent(m);
    }
    __syncthreads();
  }

  // ---- second product: X -= V W', 128 rows x 16 columns per unit
  unsigned char *A2 = usm, *B2 = usm + L::kA2;
  constexpr uint32_t kDim = 16 * S;                     // TMEM column of the imaginary parts
  const int knext_row = k0 + kNB;
  double *Xd = reinterpret_cast<double *>(X);
  int nunit = 0;
  for (int rb = 0; ok && 128 * rb < K; ++rb) {
    const int r0 = 128 * rb;                            // rows k0 + r0 .. of the block
    // A2: row rr, k < 16 Vr(rr, k), k >= 16 Vi(rr, k - 16) from the [s][part][r][16] layout
    for (int e = tid; e < S * 128 * 4; e += kUT) {
      const int s = e / 512, rr = (e >> 2) & 127, piece = e & 3;    // piece = part * 2 + kg
      oz::cp_async16(A2 + s * 8192 + core_off(rr, 8 * piece, 32),
                     vr + ((size_t)(s * 2 + (piece >> 1)) * kp + r0 + rr) * kNB + 8 * (piece & 1), true);
    }
    oz::cp_async_commit();
    const int er = vex[r0 + 32 * quad + lane];
    const int i = k0 + r0 + 32 * quad + lane;
    const bool row_ok = i < rows;
    oz::cp_async_wait<0>();
    for (int u = 0; u < kUC / 16 && 16 * u < ncols; ++u) {
      // B2: variant 0 rows jj: k < 16 W'r(k, jj), k >= 16 -W'i; variant 1: W'i, W'r.
      // Thread: W'(bb, jj), bb = tid / 16, jj = tid % 16; each part split once,
      // the negation a sign flip of its digits.
      {
        const int bb = tid >> 4, jj = tid & 15;
        const double2 wv = Wp[bb * kUC + 16 * u + jj];
        const int ew = eW[16 * u + jj];
        unsigned short dr[S], di[S];
        oz::split_regs<S>(wv.x, ew, dr);
        oz::split_regs<S>(wv.y, ew, di);
        unsigned short *b0 = reinterpret_cast<unsigned short *>(B2);
        const uint32_t o_lo = core_off(jj, bb, 32) / 2, o_hi = core_off(jj, 16 + bb, 32) / 2;
#pragma unroll
        for (int s2 = 0; s2 < S; ++s2) {
          b0[s2 * 512 + o_lo] = dr[s2];
          b0[s2 * 512 + o_hi] = di[s2] ^ 0x8000;
          b0[(S + s2) * 512 + o_lo] = di[s2];
          b0[(S + s2) * 512 + o_hi] = dr[s2];
        }
      }
      fence_proxy_async();                              // B2 writes (and the A2 copies) -> tensor core
      tc::fence_before_sync();
      __syncthreads();
      tc::fence_after_sync();
      if (tid == 0) {
        const uint32_t a0 = tc::smem_u32(A2), b0 = tc::smem_u32(B2);
#pragma unroll
        for (int s = 1; s <= S; ++s) {
          const uint32_t idesc = tc::idesc_bf16_f32(128, 16 * (S + 1 - s));
#pragma unroll
          for (int var = 0; var < 2; ++var)
#pragma unroll
            for (int kh = 0; kh < 2; ++kh) {
              const uint64_t da = tc::smem_desc(a0 + (s - 1) * 8192 + kh * 256, 128, 512);
              const uint64_t db = tc::smem_desc(b0 + var * S * 1024 + kh * 256, 128, 512);
              tc::mma_bf16(tmem + (uint32_t)(kDim * var + 16 * (s - 1)), da, db, idesc,
                           !(s == 1 && kh == 0));
            }
        }
        tc::commit(&d_full);
      }
      // the X values this thread updates, loaded while the MMAs run: row i,
      // the unit's 16 columns, real (half 0) or imaginary (half 1) part
      double xv[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int jj = 16 * u + q;
        xv[q] = (row_ok && jj < ncols) ? Xd[2 * ((size_t)jj * rows + i) + half] : 0.0;
      }
      const bool wd = tc::mbar_wait(&d_full, nunit & 1, kWaitCycles);
      ++nunit;
      if (__syncthreads_or(!wd)) { ok = false; break; }
      tc::fence_after_sync();
      // epilogue: warp (quad, half) takes TMEM lanes 32 quad .. (rows) and the
      // real (half 0) or imaginary (half 1) accumulators of the 16 columns
#pragma unroll
      for (int qh = 0; qh < 2; ++qh) {
        double xn[8];         // the next eight columns' X values, loaded during this fold
        if (qh == 0) {
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const int jj = 16 * u + 8 + q;
            xn[q] = (row_ok && jj < ncols) ? Xd[2 * ((size_t)jj * rows + i) + half] : 0.0;
          }
        }
        long long ta[8];      // fixed point, resolution 2^-kR2 of the scale 2^(er + eW)
#pragma unroll
        for (int q = 0; q < 8; ++q) ta[q] = 0;
        // groups two at a time: two loads in flight per wait
#pragma unroll
        for (int g = 2; g <= S + 1; g += 2) {
          uint32_t rv[8], rw[8];
          tc::ld8(tmem + lane_addr + (uint32_t)(kDim * half + 16 * (g - 2) + 8 * qh), rv);
          if (g + 1 <= S + 1)
            tc::ld8(tmem + lane_addr + (uint32_t)(kDim * half + 16 * (g - 1) + 8 * qh), rw);
          tc::ld_wait();
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            if (g + 1 <= S + 1 && kR2 >= 7 * g)
              oz::fold_fixed_pair<kR2>(ta[q], g, __uint_as_float(rv[q]), __uint_as_float(rw[q]));
            else {
              oz::fold_fixed<kR2>(ta[q], g, __uint_as_float(rv[q]));
              if (g + 1 <= S + 1) oz::fold_fixed<kR2>(ta[q], g + 1, __uint_as_float(rw[q]));
            }
          }
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int jj = 16 * u + 8 * qh + q;
          unsigned hk = 0u;       // the key's high word: all that the exponent needs
          if (row_ok && jj < ncols) {
            const double v = oz::sub_scaled(xv[q], ta[q], er + eW[jj] - kR2);
            Xd[2 * ((size_t)jj * rows + i) + half] = v;
            if (i >= knext_row) hk = (unsigned)(oz::abs_key(v) >> 32);
          }
          hk = __reduce_max_sync(0xffffffffu, hk);
          if (lane == 0 && hk != 0u) atomicMax(&knext[jj], hk);
        }
        if (qh == 0) {
#pragma unroll
          for (int q = 0; q < 8; ++q) xv[q] = xn[q];
        }
      }
      tc::fence_before_sync();
      __syncthreads();                                  // TMEM and B2 free for the next unit
    }
    __syncthreads();                                    // A2 free for the next row block
  }
  if (!ok) {
    // a wait ran out: let any MMA still in flight finish (bounded) before the
    // tensor memory is released, and report the timeout
    if (tid == 0) {
      tc::commit(&drain);
      (void)tc::mbar_wait(&drain, 0, kWaitCycles);
      atomicOr(o.status, kStatTimeout);
    }
  } else if (tid < ncols) {
    kout[tid] = (unsigned long long)knext[tid] << 32;
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (warp == 0) tc::tmem_dealloc(tmem, kTmemCols);
}

// one_per_sm: pad the dynamic shared memory so that a second update CTA does
// not fit on an SM, leaving registers and shared memory for a panel or a
// next-panel update CTA of the critical path beside it.
constexpr size_t kOnePerSmSmem = 120 * 1024;

template <int S>
cudaError_t launch_tc_s(const ObsDev *d_obs, const int *d_task_obs, const int *d_task_mode,
                        int ntasks, int p, int ntiles, bool one_per_sm, cudaStream_t st) {
  const size_t smem = one_per_sm && TcLayout<S>::kTotal < kOnePerSmSmem ? kOnePerSmSmem
                                                                        : TcLayout<S>::kTotal;
  static size_t granted = 0;
  cudaError_t e = ensure_dynamic_smem(qr_update_tc_kernel<S>, smem, granted);
  if (e != cudaSuccess) return e;
  static const bool carve = (prefer_max_shared(qr_update_tc_kernel<S>), true);
  (void)carve;
  qr_update_tc_kernel<S><<<ntasks * ntiles, kUT, smem, st>>>(d_obs, d_task_obs, d_task_mode, p,
                                                            ntasks);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_qr_update_tc(const ObsDev *d_obs, const int *d_task_obs, const int *d_task_mode,
                                int ntasks, int p, int slices, int max_rest_cols, bool one_per_sm,
                                cudaStream_t st) {
  if (ntasks <= 0 || max_rest_cols <= 0) return cudaSuccess;
  const int ntiles = (max_rest_cols + kUC - 1) / kUC;
  switch (slices) {
    case 4: return launch_tc_s<4>(d_obs, d_task_obs, d_task_mode, ntasks, p, ntiles, one_per_sm, st);
    case 5: return launch_tc_s<5>(d_obs, d_task_obs, d_task_mode, ntasks, p, ntiles, one_per_sm, st);
    case 6: return launch_tc_s<6>(d_obs, d_task_obs, d_task_mode, ntasks, p, ntiles, one_per_sm, st);
    case 7: return launch_tc_s<7>(d_obs, d_task_obs, d_task_mode, ntasks, p, ntiles, one_per_sm, st);
    case 8: return launch_tc_s<8>(d_obs, d_task_obs, d_task_mode, ntasks, p, ntiles, one_per_sm, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace axi
