// Step A2 in split precision: the modal transform of the fill as a digit GEMM
// on BF16 tensor cores (plans with AXI_PREC_SPLIT_BF16).
//
// The q/2 + 1 ring samples g_l of each (m, j) pair are even in l (Sec. 3.1,
// eq. ptr), so with h = q/2
//   A_n = g_0 + (-1)^n g_h + 2 sum_{0<l<h} g_l cos(pi n l / h)     (1/q, 1/4pi in g).
// Pairing l with h - l (cos(pi n (h - l)/h) = (-1)^n cos(pi n l/h)) folds it to
//   A_n = sum_{l<L} w_l cos(pi n l / h) u_l,   u = e (n even), o (n odd),
//   e_l = g_l + g_{h-l},  o_l = g_l - g_{h-l}  (l < h/2),  e_{h/2} = g_{h/2},
// w_0 = 1, w_l = 2 otherwise; L = h/2 + 1 (h even) or (h + 1)/2 (h odd).
// That is two real GEMMs per plan: [cos table of the even modes] x [e of every
// pair, real and imaginary part as separate columns], likewise odd/o.
//
//   fill_samples_kernel  one warp per (pair, kind): FP64 samples (sin/cos of
//                        k R in 64-bit fixed point, trig::sincos_ring_q), the fold,
//                        per-column exponents and S = 8 balanced digits of
//                        e and o (split2_fast), written to a scratch buffer;
//   fill_gemm_tc_kernel  (Lp <= 448, MR <= 64) the same GEMM on the fifth-
//                        generation tensor cores: CTA = 128 real columns x
//                        the MR modes of one parity, tcgen05.mma (M = 128,
//                        N = MR, K = 16) from shared-memory tiles in the
//                        no-swizzle K-major layout (tcgen05.cuh), one FP32
//                        accumulator per digit group g = s + t in tensor
//                        memory, cp.async pipeline (2 stages and two CTAs
//                        per SM for MR <= 32, else 4 stages) released by
//                        tcgen05.commit; group sums stay exact over the whole
//                        contraction (at most 36,928 per row of K, times
//                        Lp <= 448 < 2^24), so the int64 fold happens once,
//                        in the epilogue (tcgen05.ld);
//   fill_gemm_kernel     (other sizes) CTA tile = all modes x NT real columns; the cos
//                        table's digits (computed once per plan on the host)
//                        and the sample digits are staged per 32-row chunk of
//                        the contraction; every digit pair s + t <= 9 on BF16
//                        mma.sync, FP32 group sums folded into int64 every
//                        128 products (a group sums at most 8 pairs x 128 x
//                        65 x 128 < 2^24: exact), doubles rebuilt with integer
//                        instructions, written into the modal matrices.
// The samples keep the FP64 pipe busy; the transform (the FFT's half of the
// FP64 work) moves to the tensor pipe.
#include "axi_internal.h"
#include "ozaki.cuh"
#include "tcgen05.cuh"
#include "trig.cuh"

namespace axi {
namespace {
// (cos, sin)(2 pi i / 1024) with 62 fractional bits for trig::sincos_ring_q
__device__ const long long g_ring_q62[1024][2] = {
#include "ring_table_q62.inc"
};
}  // namespace
namespace {

constexpr double kInv4Pi = 0.07957747154594766788;
constexpr int kFS = kFillDigits;          // digits of both operands (8)
constexpr int kFKC = 32;                  // contraction rows per staged chunk
constexpr int kFLD = kFKC + 8;            // padded k stride in shared memory (bf16)
constexpr int kFWarpsA = 8;               // pairs per CTA in the sample kernel
constexpr int kFThreadsB = 512;           // 16 warps in the GEMM kernel

__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
    v = w > v ? w : v;
  }
  return v;
}

// Sample kernel. gdig: [2 parts][cols2][kFS][Lp] BF16 bit patterns, read as
// 32-bit words (two k per word); gex: [2 parts][cols2] exponents (one bit of
// headroom, as split2_fast wants). Column c2 = 2 (pair_local * kinds + kind)
// + (0 re, 1 im).
__global__ void __launch_bounds__(256, 5)
fill_samples_kernel(const ObsDev *__restrict__ obs_arr, int oi, int pair0, int npairs, int kinds,
                    uint32_t *__restrict__ gdig, int *__restrict__ gex) {
  const ObsDev &o = obs_arr[oi];
  const int q = o.q, h = q / 2, L = o.fill_L, Lp = o.fill_Lp;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  extern __shared__ double2 fseq[];
  longlong2 *ring = reinterpret_cast<longlong2 *>(fseq);   // [1024] (cos, sin) 2^62
  for (int i = threadIdx.x; i < trig::kRingTab; i += blockDim.x)
    ring[i] = make_longlong2(g_ring_q62[i][0], g_ring_q62[i][1]);
  __syncthreads();
  double2 *seq = fseq + trig::kRingTab + (size_t)warp * (h + 1);
  const int pl = blockIdx.x * kFWarpsA + warp;
  if (pl >= npairs) return;                       // whole warp; no block barriers below
  const int kind = blockIdx.y;
  const int p = pair0 + pl;
  const int m = p / o.N, j = p % o.N;
  const bool deriv = (o.bc == AXI_BC_NEUMANN) ? true : (kind & 1);
  const bool ext = (o.bc == AXI_BC_TRANSMISSION) && kind >= 2;
  const double k = ext ? o.km : o.k;
  const double *Sp = ext ? o.srcx : o.src;
  const double rs = Sp[2 * j], zs = Sp[2 * j + 1];
  const double rho = o.coll[4 * m], z = o.coll[4 * m + 1];
  const double nr = o.coll[4 * m + 2], nz = o.coll[4 * m + 3];
  const double dr = rho - rs, dz = z - zs;
  const double base = dr * dr + dz * dz, fourrr = 4.0 * rho * rs;
  // sub-grid: nodes l = 0, sg, 2 sg, .. (sg divides h), weight sg / (4 pi q);
  // the other nodes stay zero, so the transform below is the (q/sg)-node rule
  const int sg = o.fill_sig[((size_t)(ext ? 1 : 0) * o.M + m) * o.N + j];
  const double wq = kInv4Pi * sg / q;
  // n . (x - y_l) = (n_r rho + n_z dz) - n_r rho' cos(phi_l), with sg/(4 pi q) folded in
  const double an = (nr * rho + nz * dz) * wq, bn = nr * rs * wq;
  if (sg > 1)
    for (int l = lane; l <= h; l += 32)
      if (l % sg) seq[l] = make_double2(0.0, 0.0);
  for (int i = lane; i * sg <= h; i += 32) {
    const int l = i * sg;
    const double R2 = fma(fourrr, o.tab_s2[l], base);
    const double inv = rsqrt(R2);
    const double R = R2 * inv, kR = k * R;
    double sn, cs;
    trig::sincos_ring_q(kR, ring, &sn, &cs);
    double2 s;
    if (!deriv) {
      const double iw = inv * wq;
      s = make_double2(cs * iw, sn * iw);
    } else {
      const double f = fma(-bn, o.tab_cos[l], an) * (inv * inv * inv);
      s = make_double2(f * fma(-kR, sn, -cs), f * fma(kR, cs, -sn));
    }
    seq[l] = s;
  }
  __syncwarp();
  // fold in place: e_l at l, o_l at h - l (l < h/2); the middle e_{h/2} stays
  const bool mid = (h & 1) == 0;
  for (int l = lane; l < L; l += 32) {
    if (mid && l == h / 2) continue;
    const double2 a = seq[l], b = seq[h - l];
    seq[l] = make_double2(a.x + b.x, a.y + b.y);
    seq[h - l] = make_double2(a.x - b.x, a.y - b.y);
  }
  __syncwarp();
  auto eval = [&](int l) { return l < L ? seq[l] : make_double2(0.0, 0.0); };
  auto oval = [&](int l) {
    return (l < L && !(mid && l == h / 2)) ? seq[h - l] : make_double2(0.0, 0.0);
  };
  unsigned long long ke_r = 0, ke_i = 0, ko_r = 0, ko_i = 0;
  for (int l = lane; l < L; l += 32) {
    const double2 e = eval(l), od = oval(l);
    ke_r = max(ke_r, oz::abs_key(e.x));
    ke_i = max(ke_i, oz::abs_key(e.y));
    ko_r = max(ko_r, oz::abs_key(od.x));
    ko_i = max(ko_i, oz::abs_key(od.y));
  }
  ke_r = warp_max_u64(ke_r);
  ke_i = warp_max_u64(ke_i);
  ko_r = warp_max_u64(ko_r);
  ko_i = warp_max_u64(ko_i);
  const int xe_r = oz::key_exponent(ke_r) + 1, xe_i = oz::key_exponent(ke_i) + 1;
  const int xo_r = oz::key_exponent(ko_r) + 1, xo_i = oz::key_exponent(ko_i) + 1;
  const size_t cols2 = (size_t)npairs * kinds * 2;
  const size_t c2 = 2 * ((size_t)pl * kinds + kind);
  if (lane == 0) {
    gex[c2] = xe_r;
    gex[c2 + 1] = xe_i;
    gex[cols2 + c2] = xo_r;
    gex[cols2 + c2 + 1] = xo_i;
  }
  const int wpr = Lp / 2;                                  // words per digit row
  if (!o.fill_tc) {
    // [part][cols2][kFS][Lp]
    uint32_t *de_r = gdig + (c2 * kFS) * wpr;
    uint32_t *de_i = gdig + ((c2 + 1) * kFS) * wpr;
    uint32_t *do_r = gdig + ((cols2 + c2) * kFS) * wpr;
    uint32_t *do_i = gdig + ((cols2 + c2 + 1) * kFS) * wpr;
    for (int w = lane; w < wpr; w += 32) {
      const double2 e0 = eval(2 * w), e1 = eval(2 * w + 1);
      const double2 o0 = oval(2 * w), o1 = oval(2 * w + 1);
      oz::split2_fast<kFS>(e0.x, e1.x, xe_r, de_r + w, wpr);
      oz::split2_fast<kFS>(e0.y, e1.y, xe_i, de_i + w, wpr);
      oz::split2_fast<kFS>(o0.x, o1.x, xo_r, do_r + w, wpr);
      oz::split2_fast<kFS>(o0.y, o1.y, xo_i, do_i + w, wpr);
    }
  } else {
    // tcgen05 tiles: [part][128-column block][16-k chunk][digit] K-major
    // no-swizzle tiles of 128 rows x 16 k (4096 bytes, 1024 words); column c
    // is row c mod 128, word w holds k = 2w, 2w + 1
    const int nch = Lp / 16, nblk = ((int)cols2 + 127) / 128;
    auto tile = [&](int pt, size_t c) {
      const int cb = (int)(c >> 7), r = (int)(c & 127);
      return gdig + ((size_t)(pt * nblk + cb) * nch) * kFS * 1024 + (r >> 3) * 64 + (r & 7) * 4;
    };
    uint32_t *de_r = tile(0, c2), *de_i = tile(0, c2 + 1);
    uint32_t *do_r = tile(1, c2), *do_i = tile(1, c2 + 1);
    for (int w = lane; w < wpr; w += 32) {
      const double2 e0 = eval(2 * w), e1 = eval(2 * w + 1);
      const double2 o0 = oval(2 * w), o1 = oval(2 * w + 1);
      const size_t off = (size_t)(w >> 3) * kFS * 1024 + ((w & 7) >> 2) * 32 + (w & 3);
      oz::split2_fast<kFS>(e0.x, e1.x, xe_r, de_r + off, 1024);
      oz::split2_fast<kFS>(e0.y, e1.y, xe_i, de_i + off, 1024);
      oz::split2_fast<kFS>(o0.x, o1.x, xo_r, do_r + off, 1024);
      oz::split2_fast<kFS>(o0.y, o1.y, xo_i, do_i + off, 1024);
    }
  }
}

// GEMM kernel. Rows: 2 MR (MR even-mode rows, then MR odd-mode rows; mode
// n = 2 r' + part, rows with n >= D are zero). Columns: NT real columns per
// CTA. Warp w < MT * NT / 8 computes the 16 x 8 tile (w / (NT/8), w % (NT/8)).
__global__ void __launch_bounds__(kFThreadsB)
fill_gemm_kernel(const ObsDev *__restrict__ obs_arr, int oi, int pair0, int npairs, int kinds,
                 int NT, const uint32_t *__restrict__ gdig, const int *__restrict__ gex,
                 double2 *__restrict__ out, int ld_rows, int ld_cols) {
  const ObsDev &o = obs_arr[oi];
  const int Lp = o.fill_Lp, MR = o.fill_MR, D = o.D;
  const int rows = 2 * MR, MT = rows / 16, nt8 = NT / 8;
  const int cols2 = npairs * kinds * 2;
  const int c0 = blockIdx.x * NT;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int grp = lane >> 2, tig = lane & 3;
  const int lrow = lane & 7, lmat = lane >> 3;
  const int a_row = lrow + 8 * (lmat & 1), a_k = 8 * (lmat >> 1);
  extern __shared__ __align__(16) unsigned char fgs[];
  // digit-major layouts: consecutive rows (columns) 80 bytes apart, so the
  // eight rows of every ldmatrix 8x8 matrix fall in distinct bank groups
  // two stages, each [kFS][rows][kFLD] cos-table digits then [2][kFS][NT][kFLD]
  __nv_bfloat16 *Cs = reinterpret_cast<__nv_bfloat16 *>(fgs);
  const bool active = warp < MT * nt8;
  const int mt = active ? warp / nt8 : 0, nt = active ? warp % nt8 : 0;
  const int part = (mt * 16) / MR;
  float acc[kFS][4];
  long long hi[4] = {0, 0, 0, 0}, lo[4] = {0, 0, 0, 0};
#pragma unroll
  for (int g = 0; g < kFS; ++g)
#pragma unroll
    for (int e = 0; e < 4; ++e) acc[g][e] = 0.0f;
  const int nchunks = Lp / kFKC;
  const int wpr = Lp / 2;
  const size_t stage_elems = (size_t)kFS * kFLD * (rows + 2 * NT);
  // chunk ch of the cos-table digits ([kFS][rows][32 k]) and the sample digits
  // ([2][kFS][NT][32 k]) into stage buffer b, as asynchronous 16-byte copies
  auto stage = [&](int ch, int b) {
    __nv_bfloat16 *cs = Cs + b * stage_elems;
    __nv_bfloat16 *gs = cs + (size_t)rows * kFS * kFLD;
    for (int e = tid; e < rows * kFS * 4; e += kFThreadsB) {
      const int u = e & 3, sr = e >> 2;                     // sr = s * rows + row
      oz::cp_async16(cs + (size_t)sr * kFLD + 8 * u,
                     o.fill_cdig + (size_t)sr * Lp + ch * kFKC + 8 * u, true);
    }
    for (int e = tid; e < 2 * NT * kFS * 4; e += kFThreadsB) {
      const int u = e & 3, r = e >> 2;                      // r = (pt * kFS + s) * NT + c
      const int c = r % NT, s = (r / NT) % kFS, pt = r / (kFS * NT);
      const int col = c0 + c;
      const bool ok = col < cols2;
      const uint32_t *src =
          gdig + (((size_t)pt * cols2 + (ok ? col : 0)) * kFS + s) * wpr + ch * (kFKC / 2) + 4 * u;
      oz::cp_async16(gs + (size_t)r * kFLD + 8 * u, src, ok);
    }
    oz::cp_async_commit();
  };
  stage(0, 0);
  for (int ch = 0; ch < nchunks; ++ch) {
    if (ch + 1 < nchunks) {
      stage(ch + 1, (ch + 1) & 1);
      oz::cp_async_wait<1>();
    } else {
      oz::cp_async_wait<0>();
    }
    __syncthreads();                                        // chunk ch visible to all warps
    const __nv_bfloat16 *Cc = Cs + (ch & 1) * stage_elems;
    const __nv_bfloat16 *Gc = Cc + (size_t)rows * kFS * kFLD;
    if (active) {
#pragma unroll
      for (int kk = 0; kk < kFKC; kk += 16) {
        // digits t = 1..8 of the warp's 8 columns: two digits per ldmatrix.x4
        uint32_t b[kFS][2];
#pragma unroll
        for (int t = 0; t < kFS; t += 2) {
          uint32_t r4[4];
          const int col = nt * 8 + lrow, dg = t + (lmat >> 1), kq = kk + 8 * (lmat & 1);
          oz::ldsm_x4(r4, Gc + (((size_t)part * kFS + dg) * NT + col) * kFLD + kq);
          b[t][0] = r4[0];
          b[t][1] = r4[1];
          b[t + 1][0] = r4[2];
          b[t + 1][1] = r4[3];
        }
#pragma unroll
        for (int s = 1; s <= kFS; ++s) {
          uint32_t a[4];
          oz::ldsm_x4(a, Cc + ((size_t)(s - 1) * rows + mt * 16 + a_row) * kFLD + kk + a_k);
#pragma unroll
          for (int t = 1; t <= kFS + 1 - s; ++t)
            oz::mma16816(acc[s + t - 2], a[0], a[1], a[2], a[3], b[t - 1][0], b[t - 1][1]);
        }
      }
    }
    __syncthreads();                                        // buffer ch & 1 free for chunk ch + 2
    // fold every 4 chunks (128 products per group pair) and at the end
    if (active && (((ch + 1) & 3) == 0 || ch == nchunks - 1)) {
#pragma unroll
      for (int g = 2; g <= kFS + 1; ++g)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const long long v = (long long)__float2int_rn(acc[g - 2][e]);
          if (g <= 4) hi[e] += v << (7 * (4 - g));
          else lo[e] += v << (7 * (kFS + 1 - g));
          acc[g - 2][e] = 0.0f;
        }
    }
  }
  if (!active) return;
  // c-fragment element e: row grp (+8 for e >= 2), column 2 tig + (e & 1):
  // the (re, im) pair of one complex column
  bool bad = false;
  const size_t mode_stride = (size_t)ld_cols * ld_rows;
#pragma unroll
  for (int hf = 0; hf < 2; ++hf) {
    const int row = mt * 16 + grp + 8 * hf;
    const int n = 2 * (row % MR) + row / MR;
    const int colc = c0 + nt * 8 + 2 * tig;                 // real column of the real part
    if (n >= D || colc >= cols2) continue;
    const int ce = o.fill_cex[row];
    double vv[2];
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const int e = 2 * hf + c;
      const int E = ce + gex[(size_t)part * cols2 + colc + c];
      vv[c] = oz::scaled_to_double(hi[e], E - 28) + oz::scaled_to_double(lo[e], E - 7 * (kFS + 1));
    }
    const int cp = colc / 2, kind = cp % kinds, pl = cp / kinds;
    const int p = pair0 + pl, m = p / o.N, j = p % o.N;
    int orow = m, ocol = j;
    double sign = 1.0;
    if (o.bc == AXI_BC_TRANSMISSION) {
      const bool ext = kind >= 2;
      orow += (kind & 1) ? o.M : 0;
      ocol += ext ? o.N : 0;
      sign = ext ? -1.0 : 1.0;
    }
    const double2 v = make_double2(sign * vv[0], sign * vv[1]);
    bad |= !isfinite(v.x) || !isfinite(v.y);
    out[(size_t)n * mode_stride + (size_t)ocol * ld_rows + orow] = v;
  }
  if (bad) atomicOr(o.status, kStatNonFinite);
}


// ---------------------------------------------------------------------------
// tcgen05 form, persistent. A tile is (parity, 128-column block); the sample
// digits arrive in fill_samples_kernel's tcgen05 layout: per (parity,
// column block, 16-k chunk) the eight digits' K-major no-swizzle tiles of 128
// rows x 16 k, 32 KB contiguous; the cos-table digits likewise per (parity,
// chunk), MR rows each. Each CTA walks the tiles blockIdx.x, + gridDim.x, ...
// with its warps specialised:
//   thread 0     streams chunks through kTcStages shared-memory buffers with
//                two bulk copies (TMA) each, completing on full[b]; issues the
//                MMAs of a chunk once full[b] flips (one per sample digit s,
//                N = (9 - s) MR: every cos digit t <= 9 - s at once, column
//                block t accumulating into group s + t) and frees the buffer with
//                tcgen05.commit on empty[b]; after a tile's last chunk it
//                commits acc_full[a], and before a tile's first MMA it waits
//                for tmem_free[a] (the epilogue has read accumulator set a;
//                kTcAcc = 2 sets when 16 MR columns fit tensor memory, so the
//                next tile's MMAs run while the epilogue reads the last);
//   warps 4..11  the epilogue, two warps per SM sub-partition to hide the
//                TMEM-load and integer latencies: warp w reads TMEM lanes
//                32 (w mod 4) .. + 31 (the tile's columns) for the 16-mode
//                slices (w - 4) / 4, + 2, ..., turns them into int64,
//                doubles, the modal matrices; one arrival each on tmem_free.
// The next tile's copies stream in while the epilogue of the current runs.
constexpr int kTcCols = 128;              // real columns per tile (MMA M)
constexpr int kTcThreads = 384;
constexpr int kTcEpiWarps = 8;
constexpr int kTcTileA = kTcCols * 16 * 2;        // bytes of one digit's A tile per chunk

__host__ __device__ inline int tc_stage_bytes(int MR) { return kFS * kTcTileA + kFS * MR * 32; }
__host__ __device__ inline uint32_t tc_tmem_cols(int MR) {
  uint32_t n = 32;
  while (n < (uint32_t)(kFS * MR)) n <<= 1;
  return n;
}

__device__ __forceinline__ void mbar_arrive(uint64_t *mbar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::smem_u32(mbar)) : "memory");
}

template <int kTcStages, int kTcAcc>
__global__ void __launch_bounds__(kTcThreads, 1)
fill_gemm_tc_kernel(const ObsDev *__restrict__ obs_arr, int oi, int pair0, int npairs, int kinds,
                    const uint32_t *__restrict__ gdig, const int *__restrict__ gex,
                    double2 *__restrict__ out, int ld_rows, int ld_cols) {
  const ObsDev &o = obs_arr[oi];
  const int Lp = o.fill_Lp, MR = o.fill_MR, D = o.D;
  const int cols2 = npairs * kinds * 2;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nch = Lp / 16, nblk = (cols2 + kTcCols - 1) / kTcCols;
  const int ntiles = 2 * nblk;
  const int my_tiles = blockIdx.x < ntiles ? (ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  const uint32_t a_bytes = kFS * kTcTileA, b_bytes = kFS * MR * 32;
  const uint32_t stage_bytes = a_bytes + b_bytes;
  const uint32_t ncols_tmem = tc_tmem_cols(kTcAcc * MR);
  constexpr long long kWaitCycles = 2000000000ll;     // about a second per wait
  extern __shared__ __align__(1024) unsigned char tsm[];
  __shared__ __align__(8) uint64_t full[kTcStages], empty[kTcStages], acc_full[kTcAcc],
      tmem_free[kTcAcc];
  __shared__ uint32_t tmem_base;
  __shared__ int fail;

  if (warp == 0) tc::tmem_alloc(&tmem_base, ncols_tmem);
  if (tid == 0) {
    for (int b = 0; b < kTcStages; ++b) {
      tc::mbar_init(&full[b], 1);
      tc::mbar_init(&empty[b], 1);
    }
    for (int a = 0; a < kTcAcc; ++a) {
      tc::mbar_init(&acc_full[a], 1);
      tc::mbar_init(&tmem_free[a], kTcEpiWarps);        // one arrival per epilogue warp
    }
    fail = 0;
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tmem_base;
  auto tile_of = [&](int i, int &part, int &cb) {
    const int tt = blockIdx.x + i * gridDim.x;
    part = tt / nblk;
    cb = tt % nblk;
  };

  if (tid == 0) {
    const int total = my_tiles * nch;
    auto issue = [&](int gc) {
      int part, cb;
      tile_of(gc / nch, part, cb);
      const int ch = gc % nch, b = gc % kTcStages;
      unsigned char *buf = tsm + (size_t)b * stage_bytes;
      const unsigned char *ga = reinterpret_cast<const unsigned char *>(gdig) +
                                ((size_t)(part * nblk + cb) * nch + ch) * a_bytes;
      const unsigned char *gb = reinterpret_cast<const unsigned char *>(o.fill_cdig) +
                                ((size_t)part * nch + ch) * b_bytes;
      tc::mbar_arrive_expect_tx(&full[b], a_bytes + b_bytes);
      tc::bulk_g2s(buf, ga, a_bytes, &full[b]);
      tc::bulk_g2s(buf + a_bytes, gb, b_bytes, &full[b]);
    };
    int issued = 0, consumed = 0, committed = -1;
    for (; issued < kTcStages && issued < total; ++issued) issue(issued);
    bool ok = true;
    for (int i = 0; i < my_tiles && ok; ++i) {
      const int ab = i % kTcAcc;
      const uint32_t acc = tmem + (uint32_t)(ab * kFS * MR);
      if (i >= kTcAcc && !tc::mbar_wait(&tmem_free[ab], (i / kTcAcc - 1) & 1, kWaitCycles)) {
        ok = false;
        break;
      }
      tc::fence_after_sync();
      for (int ch = 0; ch < nch; ++ch) {
        const int gc = i * nch + ch, b = gc % kTcStages;
        if (!tc::mbar_wait(&full[b], (gc / kTcStages) & 1, kWaitCycles)) { ok = false; break; }
        consumed = gc + 1;
        const uint32_t a0 = tc::smem_u32(tsm + (size_t)b * stage_bytes), b0 = a0 + a_bytes;
        // Digit s of the samples against the cos-table digits t = 1 .. 9 - s at
        // once: the stacked B tiles (row (t - 1) MR + mode) form one K-major
        // tile, and D's column block t lands on group s + t's accumulator at
        // TMEM column (s + t - 2) MR. N is cut into pieces of at most 256.
#pragma unroll
        for (int s = 1; s <= kFS; ++s) {
          const uint64_t da = tc::smem_desc(a0 + (s - 1) * kTcTileA, 128, 256);
          const int ntot = (kFS + 1 - s) * MR;
          for (int off = 0; off < ntot; off += 256) {
            const int n = min(256, ntot - off);
            const uint64_t db = tc::smem_desc(b0 + off * 32, 128, 256);
            tc::mma_bf16(acc + (uint32_t)((s - 1) * MR + off), da, db, tc::idesc_bf16_f32(kTcCols, n),
                         ch > 0 || s > 1);
          }
        }
        tc::commit(&empty[b]);
        committed = gc;
        if (ch == nch - 1) tc::commit(&acc_full[ab]);   // the tile's accumulators are final
        // refill the buffer of chunk gc - 1 once its MMAs are done
        if (gc >= 1 && issued < total) {
          const int pg = gc - 1;
          if (!tc::mbar_wait(&empty[pg % kTcStages], (pg / kTcStages) & 1, kWaitCycles)) { ok = false; break; }
          issue(issued++);
        }
      }
    }
    if (!ok) {
      // let the copies and MMAs in flight finish before shared memory and TMEM go
      for (int c = consumed; c < issued; ++c)
        (void)tc::mbar_wait(&full[c % kTcStages], (c / kTcStages) & 1, kWaitCycles);
      if (committed >= 0)
        (void)tc::mbar_wait(&empty[committed % kTcStages], (committed / kTcStages) & 1, kWaitCycles);
      atomicOr(&fail, 1);
      atomicOr(o.status, kStatTimeout);
    }
  } else if (warp >= 4) {
    // epilogue warps
    const int lb = 32 * (warp & 3);
    const size_t mode_stride = (size_t)ld_cols * ld_rows;
    bool bad = false;
    for (int i = 0; i < my_tiles; ++i) {
      const int ab = i % kTcAcc;
      const uint32_t acc = tmem + (uint32_t)(ab * kFS * MR);
      const bool w = tc::mbar_wait(&acc_full[ab], (i / kTcAcc) & 1, kWaitCycles);
      if (!__all_sync(0xffffffffu, w) || *(volatile int *)&fail) break;
      tc::fence_after_sync();
      int part, cb;
      tile_of(i, part, cb);
      const int col = cb * kTcCols + lb + lane;
      const int ex_col = col < cols2 ? gex[(size_t)part * cols2 + col] : 0;
      const int cp = col / 2, kind = cp % kinds, pl = cp / kinds;
      const int p = pair0 + pl, m = p / o.N, j = p % o.N;
      int orow = m, ocol = j;
      double sign = 1.0;
      if (o.bc == AXI_BC_TRANSMISSION) {
        const bool ext = kind >= 2;
        orow += (kind & 1) ? o.M : 0;
        ocol += ext ? o.N : 0;
        sign = ext ? -1.0 : 1.0;
      }
      const bool writer = (lane & 1) == 0 && col < cols2;
      const int sl0 = (warp - 4) >> 2;
      if (sl0 >= MR / 16) {                             // no slice here (MR = 16)
        tc::fence_before_sync();
        __syncwarp();
        if (lane == 0) mbar_arrive(&tmem_free[ab]);
      }
      for (int sl = sl0; sl < MR / 16; sl += kTcEpiWarps / 4) {
        long long hi[16], lo[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) hi[q] = lo[q] = 0;
#pragma unroll
        for (int g = 2; g <= kFS + 1; ++g) {
          uint32_t r[16];
          tc::ld16(acc + ((uint32_t)lb << 16) + (uint32_t)((g - 2) * MR + 16 * sl), r);
          tc::ld_wait();
#pragma unroll
          for (int q = 0; q < 16; ++q) {
            const long long v = (long long)__float2int_rn(__uint_as_float(r[q]));
            if (g <= 4) hi[q] += v << (7 * (4 - g));
            else lo[q] += v << (7 * (kFS + 1 - g));
          }
        }
        if (sl + kTcEpiWarps / 4 >= MR / 16) {          // this warp's last slice: its TMEM reads are done
          tc::fence_before_sync();
          __syncwarp();
          if (lane == 0) mbar_arrive(&tmem_free[ab]);
        }
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          const int mr = 16 * sl + q, n = 2 * mr + part;
          const int E = o.fill_cex[part * MR + mr] + ex_col;
          const double val =
              oz::scaled_to_double(hi[q], E - 28) + oz::scaled_to_double(lo[q], E - 7 * (kFS + 1));
          const double vim = __shfl_down_sync(0xffffffffu, val, 1);
          if (writer && n < D) {
            const double2 v = make_double2(sign * val, sign * vim);
            bad |= !isfinite(v.x) || !isfinite(v.y);
            out[(size_t)n * mode_stride + (size_t)ocol * ld_rows + orow] = v;
          }
        }
      }
    }
    if (bad) atomicOr(o.status, kStatNonFinite);
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (warp == 0) {
    __syncwarp();
    tc::tmem_dealloc(tmem, ncols_tmem);
  }
}

}  // namespace

int fill_gemm_cols(int MR) {
  const int mt = 2 * MR / 16;
  return 8 * (16 / mt);
}

size_t fill_gemm_smem(int MR) {
  return 2 * sizeof(__nv_bfloat16) * kFS * kFLD * ((size_t)2 * MR + 2 * (size_t)fill_gemm_cols(MR));
}

cudaError_t launch_fill_mma(const ObsDev *d_obs, const ObsDev &h, int oi, double2 *out,
                            int ld_rows, int ld_cols, int chunk_mb, cudaStream_t st) {
  const int kinds = h.bc == AXI_BC_TRANSMISSION ? 4 : 1;
  const int npairs_total = h.M * h.N;
  // ring pairs per chunk: the plan's (its scratch holds that many), or fewer
  // so that one chunk's sample digits stay in L2 between the two kernels
  int chunk = h.fill_chunk_pairs;
  if (chunk_mb > 0) {
    const size_t per_pair = (size_t)2 * 2 * kinds * kFillDigits * h.fill_Lp * sizeof(unsigned short);
    const size_t want = ((size_t)chunk_mb << 20) / per_pair;
    chunk = (int)std::max<size_t>(8, std::min<size_t>((size_t)chunk, want));
  }
  const int NT = fill_gemm_cols(h.fill_MR);
  const size_t smemA = sizeof(double2) * ((size_t)trig::kRingTab + (size_t)kFWarpsA * (h.q / 2 + 1));
  const bool tc = h.fill_tc != 0;
  // one CTA per SM, 4 stages; two accumulator sets when 16 MR TMEM columns fit
  const bool two = h.fill_MR <= 32;
  const size_t smemB = tc ? (size_t)4 * tc_stage_bytes(h.fill_MR) : fill_gemm_smem(h.fill_MR);
  static size_t grantedA = 0, grantedB = 0, grantedT2 = 0, grantedT1 = 0;
  cudaError_t e = ensure_dynamic_smem(fill_samples_kernel, smemA, grantedA);
  if (e != cudaSuccess) return e;
  e = !tc ? ensure_dynamic_smem(fill_gemm_kernel, smemB, grantedB)
          : two ? ensure_dynamic_smem(fill_gemm_tc_kernel<4, 2>, smemB, grantedT2)
                : ensure_dynamic_smem(fill_gemm_tc_kernel<4, 1>, smemB, grantedT1);
  if (e != cudaSuccess) return e;
  for (int pair0 = 0; pair0 < npairs_total; pair0 += chunk) {
    const int np = min(chunk, npairs_total - pair0);
    fill_samples_kernel<<<dim3((np + kFWarpsA - 1) / kFWarpsA, kinds), 32 * kFWarpsA, smemA, st>>>(
        d_obs, oi, pair0, np, kinds, h.fill_gdig, h.fill_gex);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int cols2 = np * kinds * 2;
    // persistent: one CTA per SM
    const int ntiles = 2 * ((cols2 + kTcCols - 1) / kTcCols);
    const dim3 tgrid(min(ntiles, sm_count()));
    if (tc && two)
      fill_gemm_tc_kernel<4, 2><<<tgrid, kTcThreads, smemB, st>>>(
          d_obs, oi, pair0, np, kinds, h.fill_gdig, h.fill_gex, out, ld_rows, ld_cols);
    else if (tc)
      fill_gemm_tc_kernel<4, 1><<<tgrid, kTcThreads, smemB, st>>>(
          d_obs, oi, pair0, np, kinds, h.fill_gdig, h.fill_gex, out, ld_rows, ld_cols);
    else
      fill_gemm_kernel<<<(cols2 + NT - 1) / NT, kFThreadsB, smemB, st>>>(
          d_obs, oi, pair0, np, kinds, NT, h.fill_gdig, h.fill_gex, out, ld_rows, ld_cols);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace axi
