// Step A7: the eight phased nearest-image sums at all ring nodes (Sec. 4.1,
// the action of A_else), as a split-precision GEMM on tensor cores.
//
//   U_w(x_t) = sum_{img != 0} ph_w(img) sum_s dG/dn_t(x_t, y_s + d_img) sigma_w(s),
//   ph_w(a, b) = e^{i k (d_x a e_x + d_y b e_y)},   d_(a,b) = (a e_x, b e_y, 0),
//
// targets x_t = ring nodes (rho_m, phi_l = 2 pi l / P, z_m) with their normals,
// sources y_s = point sources (rho'_j, phi_l', z'_j) with strengths sigma.
//
// Lattice symmetry: when e_x = e_y and 4 | P, rotating targets, sources and
// image by 90 degrees (l -> l + P/4, (a, b) -> (-b, a)) leaves the kernel
// unchanged, so the images (1,0), (0,1), (-1,0), (0,-1) share the kernel of
// (1,0) and the diagonal images that of (1,1):
//   sum_s K_{R^r rep}(t, s) sigma(s) = [K_rep sigma_r](R^{-r} t),  sigma_r(s) = sigma(R^r s).
// Each representative image is then one GEMM  C = K_rep [sigma_0 .. sigma_3]
// (targets x sources times sources x 4W), and U collects C's rows rotated back
// with the image phases. Without the symmetry every image is its own
// representative with one rotation.
//
// Arithmetic: kernel values are generated in FP64 (rsqrt, table sin/cos) and
// both operands are split into S balanced base-128 digits (ozaki.cuh), written
// straight into K-major no-swizzle tiles (core matrices of 8 rows x 8 k) of
// 128 targets x 16 sources (A) and 32 columns x 16 sources (B). The GEMM runs
// on tcgen05 (near_gemm_tc_kernel): per 16-source chunk, for every kernel
// digit s and part, one MMA against the stacked strength digits t <= S + 1 - s,
// whose column blocks land on the FP32 group accumulators s + t in tensor
// memory (real and imaginary parts separately; -Ai Bi through the
// instruction's negate-A bit). Both operands are split with one bit of
// headroom so every digit satisfies |d| <= 64; a group sum then stays below
// 256 * 2 * 7 * 2^12 < 2^24 over 256 sources, after which the epilogue warps
// fold the accumulators into exact int64 sums and the MMAs start over.
#include "axi_internal.h"
#include "trig.cuh"
#include "ozaki.cuh"
#include "tcgen05.cuh"

namespace axi {
namespace {

constexpr double kInv4Pi = 0.07957747154594766788;
constexpr int kGK = 32;        // sources padded to a multiple of this

__device__ __forceinline__ void mbar_arrive_cta(uint64_t *mbar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::smem_u32(mbar)) : "memory");
}

struct NearGeom {
  int M, N, P, nrot, nrep, W, S, Sp;   // S = N*P sources, Sp padded to kGK
  int sld;                             // stride of one wave in the strengths array
  double k, ex, ey;
  int rep_a[8], rep_b[8];
};

__device__ __forceinline__ void target_point(const ObsDev &o, int t, double &x, double &y, double &z,
                                             double &nx, double &ny, double &nz) {
  const int m = t / o.P, l = t % o.P;
  const double2 tw = o.tw_P[l];
  const double c = tw.x, s = -tw.y;
  const double rho = o.coll[4 * m], nr = o.coll[4 * m + 2];
  x = rho * c; y = rho * s; z = o.coll[4 * m + 1];
  nx = nr * c; ny = nr * s; nz = o.coll[4 * m + 3];
}

__device__ __forceinline__ void source_point(const ObsDev &o, int s, double &x, double &y, double &z) {
  const int j = s / o.P, l = s % o.P;
  const double2 tw = o.tw_P[l];
  const double rs = o.src[2 * j];
  x = rs * tw.x; y = -rs * tw.y; z = o.src[2 * j + 1];
}

// Per target row: exponent of an upper bound of |dG/dn| over all sources of
// the representative image: |dG/dn| <= sqrt(1 + k^2 R^2) / (4 pi R^2), decreasing
// in R, at the smallest distance. One extra bit of headroom keeps the leading
// digit within 64. The smallest squared distance is searched in FP32 (any
// lower bound of it keeps the bound valid) and shrunk by 1% to cover FP32
// rounding of the coordinates.
// It also leaves, per target, the target shifted by minus the image offset and
// the normal times 1/(4 pi) (ttab[ti][0..5]) for the kernel-value kernel.
__global__ void __launch_bounds__(256)
near_rowexp_kernel(const ObsDev *__restrict__ od, NearGeom g, int rep, int t0, int nt,
                   int *__restrict__ erow, double *__restrict__ ttab) {
  const ObsDev &o = *od;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ti = blockIdx.x * 8 + warp;
  if (ti >= nt) return;
  double tx, ty, tz, nx, ny, nz;
  target_point(o, t0 + ti, tx, ty, tz, nx, ny, nz);
  if (lane < 6) {
    const double v[6] = {tx - g.rep_a[rep] * g.ex, ty - g.rep_b[rep] * g.ey, tz,
                         nx * kInv4Pi, ny * kInv4Pi, nz * kInv4Pi};
    ttab[(size_t)ti * 8 + lane] = v[lane];
  }
  const float px = (float)(tx - g.rep_a[rep] * g.ex), py = (float)(ty - g.rep_b[rep] * g.ey);
  const float pz = (float)tz;
  float r2f = 3.0e38f;
  for (int s = lane; s < g.S; s += 32) {
    const int j = s / o.P, l = s % o.P;
    const double2 tw = o.tw_P[l];
    const float rs = (float)o.src[2 * j];
    const float dx = px - rs * (float)tw.x, dy = py + rs * (float)tw.y, dz = pz - (float)o.src[2 * j + 1];
    r2f = fminf(r2f, fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) r2f = fminf(r2f, __shfl_xor_sync(0xffffffffu, r2f, off));
  if (lane == 0) {
    const double r2min = 0.99 * (double)r2f;
    const double bound = sqrt(1.0 + g.k * g.k * r2min) / r2min * kInv4Pi;
    erow[ti] = oz::key_exponent(oz::abs_key(bound)) + 1;
  }
}

// Kernel-value digits of the representative image for targets [t0, t0 + nt),
// in tiles: per (128-target block, 16-source chunk) the 2 SD planes (part-major:
// re digits 1..SD, then im) of 128 x 16, 4096 bytes each, element (r, kk) at
// (r / 8) 256 + (kk / 8) 128 + (r % 8) 16 + (kk % 8) 2; zero beyond S.
// Target data come from near_rowexp_kernel's table (shift and 1/(4 pi) folded
// in), source coordinates from near_sources_kernel's, so a kernel value costs
// only the distance, rsqrt, the table sin/cos and the products.
template <int SD>
__global__ void __launch_bounds__(256)
near_adigits_kernel(const ObsDev *__restrict__ od, NearGeom g, int nt, const int *__restrict__ erow,
                    const double *__restrict__ ttab, const double *__restrict__ sxyz,
                    unsigned short *__restrict__ A) {
  const ObsDev &o = *od;
  const int ti = blockIdx.y;
  const int s = blockIdx.x * 256 + threadIdx.x;
  if (ti >= nt || s >= g.Sp) return;
  double2 kv = make_double2(0.0, 0.0);
  if (s < g.S) {
    const double *tt = ttab + (size_t)ti * 8;
    const double dx = tt[0] - sxyz[s], dy = tt[1] - sxyz[g.Sp + s], dz = tt[2] - sxyz[2 * g.Sp + s];
    const double R2 = fma(dx, dx, fma(dy, dy, dz * dz));
    const double inv = rsqrt(R2);
    const double R = R2 * inv, kR = g.k * R;
    double sn, cs;
    trig::sincos_ring_tab(kR, o.tab_ring, &sn, &cs);   // table through L1
    const double f = fma(tt[3], dx, fma(tt[4], dy, tt[5] * dz)) * (inv * inv) * inv;
    kv = make_double2(f * fma(-kR, sn, -cs), f * fma(kR, cs, -sn));   // (ikR - 1) e^{ikR}
  }
  const int e = erow[ti];
  const int r = ti & 127, kk = s & 15;
  unsigned short *dst = A + ((size_t)(ti >> 7) * (g.Sp / 16) + (s >> 4)) * 2 * SD * 2048 +
                        (r >> 3) * 128 + (kk >> 3) * 64 + (r & 7) * 8 + (kk & 7);
  oz::split_store_n(kv.x, e, SD, dst, 2048);                   // planes 4096 bytes apart
  oz::split_store_n(kv.y, e, SD, dst + SD * 2048, 2048);
}

// Source coordinates, sxyz = [x | y | z] with Sp entries each.
__global__ void __launch_bounds__(256)
near_sources_kernel(const ObsDev *__restrict__ od, NearGeom g, double *__restrict__ sxyz) {
  const ObsDev &o = *od;
  for (int s = blockIdx.x * 256 + threadIdx.x; s < g.S; s += gridDim.x * 256) {
    double x, y, z;
    source_point(o, s, x, y, z);
    sxyz[s] = x;
    sxyz[g.Sp + s] = y;
    sxyz[2 * g.Sp + s] = z;
  }
}

// Exponent of each wave's strengths (max over all sources).
__global__ void __launch_bounds__(256)
near_sigexp_kernel(NearGeom g, const double2 *__restrict__ sigma, int *__restrict__ ecol) {
  const int w = blockIdx.x;
  unsigned long long m = 0;
  for (int s = threadIdx.x; s < g.S; s += 256) {
    const double2 v = sigma[(size_t)w * g.sld + s];
    const unsigned long long a = oz::abs_key(v.x), b = oz::abs_key(v.y);
    m = a > m ? a : m;
    m = b > m ? b : m;
  }
  __shared__ unsigned long long red[256];
  red[threadIdx.x] = m;
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if (threadIdx.x < h && red[threadIdx.x + h] > red[threadIdx.x]) red[threadIdx.x] = red[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) ecol[w] = oz::key_exponent(red[0]) + 1;   // headroom: |d| <= 64
}

// Strength digits: column c = r W + w holds sigma_w(R^r s), s = j P + l -> (j, l + r P/4);
// tiles per (32-column block, 16-source chunk): 2 SD planes (re digits, then
// im) of 32 x 16, 1024 bytes each, the A tile layout with 32 rows.
template <int SD>
__global__ void __launch_bounds__(256)
near_bdigits_kernel(NearGeom g, const double2 *__restrict__ sigma, const int *__restrict__ ecol,
                    unsigned short *__restrict__ B) {
  const int c = blockIdx.y;
  const int s = blockIdx.x * 256 + threadIdx.x;
  if (s >= g.Sp) return;
  const int r = c / g.W, w = c % g.W;
  double2 v = make_double2(0.0, 0.0);
  if (s < g.S) {
    const int j = s / g.P, l = s % g.P;
    const int lr = (l + r * (g.P / 4)) % g.P;
    v = sigma[(size_t)w * g.sld + j * g.P + lr];
  }
  const int rr = c & 31, kk = s & 15;
  unsigned short *dst = B + ((size_t)(c >> 5) * (g.Sp / 16) + (s >> 4)) * 2 * SD * 512 +
                        (rr >> 3) * 128 + (kk >> 3) * 64 + (rr & 7) * 8 + (kk & 7);
  oz::split_store_n(v.x, ecol[w], SD, dst, 512);               // planes 1024 bytes apart
  oz::split_store_n(v.y, ecol[w], SD, dst + SD * 512, 512);
}

// C[ti][c] = sum_s K[ti][s] B[s][c] for one block of targets on tcgen05. CTA
// tile: 128 targets (MMA M) x 32 columns; 384 threads. Thread 0 streams the
// 16-source chunks (two bulk copies each: 2 SD A planes, 2 SD B planes) through
// 3 shared-memory stages and issues per chunk 4 SD MMAs:
//   re += Ar_s [Br_1 .. Br_{SD+1-s}] - Ai_s [Bi_1 ..]  (negate-A bit),
//   im += Ar_s [Bi_1 .. ] + Ai_s [Br_1 .. ],
// N = (SD + 1 - s) 32, column block t landing on group s + t (TMEM columns
// (g - 2) 32 for re, SD 32 + (g - 2) 32 for im). Every kNearFold chunks (256
// sources) the epilogue warps 4..11 (TMEM lanes 32 (w mod 4) .., 16 columns
// each) convert the group sums to int64 and add them to exact hi/lo sums, then
// release the accumulators; at the end they write C in FP64.
constexpr int kNearCols = 32;
constexpr int kNearThreads = 384;
constexpr int kNearStages = 3;
constexpr int kNearFold = 16;                 // chunks of 16 sources per fold

template <int SD>
__host__ __device__ constexpr int near_stage_bytes() { return 2 * SD * 4096 + 2 * SD * 1024; }

template <int SD>
__global__ void __launch_bounds__(kNearThreads, 1)
near_gemm_tc_kernel(NearGeom g, int nt, const unsigned short *__restrict__ A,
                    const unsigned short *__restrict__ B, const int *__restrict__ erow,
                    const int *__restrict__ ecol, double2 *__restrict__ C, int *__restrict__ status) {
  const int NC = g.nrot * g.W;
  const int mb = blockIdx.x, nb = blockIdx.y;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nch = g.Sp / 16;
  const int nfold = (nch + kNearFold - 1) / kNearFold;
  constexpr uint32_t a_bytes = 2 * SD * 4096, b_bytes = 2 * SD * 1024;
  constexpr uint32_t stage_bytes = a_bytes + b_bytes;
  constexpr uint32_t ncols_tmem = 512;               // 2 SD x 32 <= 448 columns used
  constexpr long long kWaitCycles = 2000000000ll;
  extern __shared__ __align__(1024) unsigned char nsm[];
  __shared__ __align__(8) uint64_t full[kNearStages], empty[kNearStages], acc_full, tmem_free;
  __shared__ uint32_t tmem_base;
  __shared__ int fail;

  if (warp == 0) tc::tmem_alloc(&tmem_base, ncols_tmem);
  if (tid == 0) {
    for (int b = 0; b < kNearStages; ++b) {
      tc::mbar_init(&full[b], 1);
      tc::mbar_init(&empty[b], 1);
    }
    tc::mbar_init(&acc_full, 1);
    tc::mbar_init(&tmem_free, 8);                     // one arrival per epilogue warp
    fail = 0;
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tmem_base;

  if (tid == 0) {
    const unsigned char *gA = reinterpret_cast<const unsigned char *>(A) + (size_t)mb * nch * a_bytes;
    const unsigned char *gB = reinterpret_cast<const unsigned char *>(B) + (size_t)nb * nch * b_bytes;
    auto issue = [&](int c) {
      const int b = c % kNearStages;
      unsigned char *buf = nsm + (size_t)b * stage_bytes;
      tc::mbar_arrive_expect_tx(&full[b], a_bytes + b_bytes);
      tc::bulk_g2s(buf, gA + (size_t)c * a_bytes, a_bytes, &full[b]);
      tc::bulk_g2s(buf + a_bytes, gB + (size_t)c * b_bytes, b_bytes, &full[b]);
    };
    int issued = 0, consumed = 0, committed = -1;
    for (; issued < kNearStages && issued < nch; ++issued) issue(issued);
    bool ok = true;
    for (int ch = 0; ch < nch && ok; ++ch) {
      const int f = ch / kNearFold, first = ch % kNearFold == 0;
      if (first && f > 0) {
        if (!tc::mbar_wait(&tmem_free, (f - 1) & 1, kWaitCycles)) { ok = false; break; }
        tc::fence_after_sync();
      }
      const int b = ch % kNearStages;
      if (!tc::mbar_wait(&full[b], (ch / kNearStages) & 1, kWaitCycles)) { ok = false; break; }
      consumed = ch + 1;
      const uint32_t a0 = tc::smem_u32(nsm + (size_t)b * stage_bytes), b0 = a0 + a_bytes;
      const uint32_t bre = b0, bim = b0 + SD * 1024;
#pragma unroll
      for (int s = 1; s <= SD; ++s) {
        const int nn = (SD + 1 - s) * kNearCols;
        const uint32_t idesc = tc::idesc_bf16_f32(128, nn);
        const uint32_t idesc_neg = tc::idesc_bf16_f32(128, nn, true);
        const uint64_t dar = tc::smem_desc(a0 + (s - 1) * 4096, 128, 256);
        const uint64_t dai = tc::smem_desc(a0 + (SD + s - 1) * 4096, 128, 256);
        const uint64_t dbr = tc::smem_desc(bre, 128, 256), dbi = tc::smem_desc(bim, 128, 256);
        const uint32_t dre = tmem + (uint32_t)((s - 1) * kNearCols);
        const uint32_t dim = tmem + (uint32_t)((SD + s - 1) * kNearCols);
        const bool acc = !(first && s == 1);
        tc::mma_bf16(dre, dar, dbr, idesc, acc);
        tc::mma_bf16(dre, dai, dbi, idesc_neg, true);
        tc::mma_bf16(dim, dar, dbi, idesc, acc);
        tc::mma_bf16(dim, dai, dbr, idesc, true);
      }
      tc::commit(&empty[b]);
      committed = ch;
      if (ch % kNearFold == kNearFold - 1 || ch == nch - 1) tc::commit(&acc_full);
      if (ch >= 1 && issued < nch) {
        const int pg = ch - 1;
        if (!tc::mbar_wait(&empty[pg % kNearStages], (pg / kNearStages) & 1, kWaitCycles)) { ok = false; break; }
        issue(issued++);
      }
    }
    if (!ok) {
      for (int c = consumed; c < issued; ++c)
        (void)tc::mbar_wait(&full[c % kNearStages], (c / kNearStages) & 1, kWaitCycles);
      if (committed >= 0)
        (void)tc::mbar_wait(&empty[committed % kNearStages], (committed / kNearStages) & 1, kWaitCycles);
      atomicOr(&fail, 1);
      atomicOr(status, kStatTimeout);
    }
  } else if (warp >= 4) {
    const int lb = 32 * (warp & 3), hf = (warp - 4) >> 2;     // TMEM lanes, 16-column half
    long long hi[2][16], lo[2][16];
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
      for (int q = 0; q < 16; ++q) hi[c][q] = lo[c][q] = 0;
    bool ok = true;
    for (int f = 0; f < nfold; ++f) {
      const bool w = tc::mbar_wait(&acc_full, f & 1, kWaitCycles);
      if (!__all_sync(0xffffffffu, w) || *(volatile int *)&fail) { ok = false; break; }
      tc::fence_after_sync();
#pragma unroll
      for (int c = 0; c < 2; ++c)
#pragma unroll
        for (int gg = 2; gg <= SD + 1; ++gg) {
          uint32_t r[16];
          tc::ld16(tmem + ((uint32_t)lb << 16) + (uint32_t)((c * SD + gg - 2) * kNearCols + 16 * hf), r);
          tc::ld_wait();
#pragma unroll
          for (int q = 0; q < 16; ++q) {
            const long long v = (long long)__float2int_rn(__uint_as_float(r[q]));
            if (gg <= 4) hi[c][q] += v << (7 * (4 - gg));
            else lo[c][q] += v << (7 * (SD + 1 - gg));
          }
        }
      tc::fence_before_sync();
      __syncwarp();
      if (lane == 0) mbar_arrive_cta(&tmem_free);
    }
    if (ok) {
      const int r = mb * 128 + lb + lane;
      if (r < nt) {
        const int er = erow[r];
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          const int c = nb * kNearCols + 16 * hf + q;
          if (c < NC) {
            const int ex = er + ecol[c % g.W];
            C[(size_t)r * NC + c] = make_double2(oz::unfold<SD>(hi[0][q], lo[0][q], ex),
                                                 oz::unfold<SD>(hi[1][q], lo[1][q], ex));
          }
        }
      }
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (warp == 0) {
    __syncwarp();
    tc::tmem_dealloc(tmem, ncols_tmem);
  }
}

// U[w][t0 + ti] += sum_r ph_w(R^r rep) C[(m, l - r P/4)][r W + w] for the block's targets.
__global__ void __launch_bounds__(256)
near_combine_kernel(NearGeom g, int rep, int t0, int nt, const double *__restrict__ dirs,
                    const double2 *__restrict__ C, double2 *__restrict__ U, int T) {
  const int NC = g.nrot * g.W;
  const size_t total = (size_t)nt * g.W;
  for (size_t idx = blockIdx.x * (size_t)256 + threadIdx.x; idx < total; idx += (size_t)gridDim.x * 256) {
    const int ti = (int)(idx % nt), w = (int)(idx / nt);
    const int tg = t0 + ti;
    const int m = tg / g.P, l = tg % g.P;
    double2 u = U[(size_t)w * T + tg];
    int a = g.rep_a[rep], b = g.rep_b[rep];
    for (int r = 0; r < g.nrot; ++r) {
      const int lr = ((l - r * (g.P / 4)) % g.P + g.P) % g.P;
      const int src_ti = m * g.P + lr - t0;
      const double2 cv = C[(size_t)src_ti * NC + r * g.W + w];
      double sn, cs;
      sincos(g.k * (dirs[3 * w] * a * g.ex + dirs[3 * w + 1] * b * g.ey), &sn, &cs);
      u.x = fma(cs, cv.x, fma(-sn, cv.y, u.x));
      u.y = fma(cs, cv.y, fma(sn, cv.x, u.y));
      const int na = -b, nb = a;                 // rotate the image by 90 degrees
      a = na;
      b = nb;
    }
    U[(size_t)w * T + tg] = u;
  }
}

__global__ void ring_targets_kernel(const ObsDev *__restrict__ od, double *__restrict__ X,
                                    double *__restrict__ Nrm, int T) {
  const ObsDev &o = *od;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < T; t += gridDim.x * blockDim.x) {
    double x, y, z, nx, ny, nz;
    target_point(o, t, x, y, z, nx, ny, nz);
    X[3 * t] = x; X[3 * t + 1] = y; X[3 * t + 2] = z;
    Nrm[3 * t] = nx; Nrm[3 * t + 1] = ny; Nrm[3 * t + 2] = nz;
  }
}

NearGeom make_geom(const ObsDev &h, int W, double ex, double ey) {
  NearGeom g;
  g.M = h.M; g.N = h.N; g.P = h.P; g.W = W; g.k = h.k; g.ex = ex; g.ey = ey;
  g.sld = h.cols * h.P;
  g.S = h.N * h.P;
  g.Sp = (g.S + kGK - 1) / kGK * kGK;
  const bool sym = (ex == ey) && (h.P % 4 == 0);
  if (sym) {
    g.nrot = 4; g.nrep = 2;
    g.rep_a[0] = 1; g.rep_b[0] = 0;
    g.rep_a[1] = 1; g.rep_b[1] = 1;
  } else {
    g.nrot = 1; g.nrep = 8;
    int n = 0;
    for (int a = -1; a <= 1; ++a)
      for (int b = -1; b <= 1; ++b)
        if (a || b) { g.rep_a[n] = a; g.rep_b[n] = b; ++n; }
  }
  return g;
}

int block_targets(const ObsDev &h, int W, int nrot) {
  // whole rings per block (rotations stay inside the block), sized so the
  // kernel-value digits stay near 3 GB
  const double per_target = 2.0 * 8 * h.N * h.P * 2;  // SD <= 8 digits, re/im, 2 bytes
  int rings = (int)(3.0e9 / (per_target * h.P));
  if (rings < 1) rings = 1;
  if (rings > h.M) rings = h.M;
  (void)W; (void)nrot;
  return rings * h.P;
}

}  // namespace

size_t near_image_scratch_bytes(const ObsDev &h, int W, double ex, double ey, int slices) {
  const NearGeom g = make_geom(h, W, ex, ey);
  const size_t T = (size_t)h.M * h.P;
  size_t b = 0;
  auto add = [&](size_t n) { b += (n + 255) & ~(size_t)255; };
  add(sizeof(double2) * (size_t)W * h.cols * h.P);     // sigma
  if (slices <= 0) {
    add(sizeof(double) * 3 * T);
    add(sizeof(double) * 3 * T);
    return b;
  }
  const int tb = block_targets(h, W, g.nrot);
  const int NC = g.nrot * W;
  add(sizeof(int) * tb);                                 // row exponents
  add(sizeof(double) * 8 * tb);                          // target table
  add(sizeof(double) * 3 * g.Sp);                        // source coordinates
  add(sizeof(int) * W);                                  // column exponents
  add(sizeof(unsigned short) * 2 * (size_t)slices * ((tb + 127) / 128 * 128) * g.Sp);   // A digit tiles
  add(sizeof(unsigned short) * 2 * (size_t)slices * ((NC + 31) / 32 * 32) * g.Sp);     // B digit tiles
  add(sizeof(double2) * (size_t)tb * NC);                          // C block
  return b;
}

template <int SD>
static cudaError_t near_split(const ObsDev *d_o, const ObsDev &h, const NearGeom &g,
                              const double2 *sigma, const double *dirs, double2 *U, char *sc,
                              cudaStream_t st) {
  const int T = h.M * h.P;
  const int tb = block_targets(h, g.W, g.nrot);
  const int NC = g.nrot * g.W;
  auto take = [&](size_t n) { char *p = sc; sc += (n + 255) & ~(size_t)255; return p; };
  int *erow = reinterpret_cast<int *>(take(sizeof(int) * tb));
  double *ttab = reinterpret_cast<double *>(take(sizeof(double) * 8 * tb));
  double *sxyz = reinterpret_cast<double *>(take(sizeof(double) * 3 * g.Sp));
  int *ecol = reinterpret_cast<int *>(take(sizeof(int) * g.W));
  unsigned short *A = reinterpret_cast<unsigned short *>(
      take(sizeof(unsigned short) * 2 * (size_t)SD * ((tb + 127) / 128 * 128) * g.Sp));
  unsigned short *B = reinterpret_cast<unsigned short *>(
      take(sizeof(unsigned short) * 2 * (size_t)SD * ((NC + 31) / 32 * 32) * g.Sp));
  double2 *C = reinterpret_cast<double2 *>(take(sizeof(double2) * (size_t)tb * NC));
  const size_t gemm_smem = (size_t)kNearStages * near_stage_bytes<SD>();
  static size_t granted = 0;
  cudaError_t e = ensure_dynamic_smem(near_gemm_tc_kernel<SD>, gemm_smem, granted);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(U, 0, sizeof(double2) * (size_t)g.W * T, st);
  if (e != cudaSuccess) return e;
  near_sigexp_kernel<<<g.W, 256, 0, st>>>(g, sigma, ecol);
  near_sources_kernel<<<(g.S + 255) / 256, 256, 0, st>>>(d_o, g, sxyz);
  near_bdigits_kernel<SD><<<dim3((g.Sp + 255) / 256, NC), 256, 0, st>>>(g, sigma, ecol, B);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  for (int t0 = 0; t0 < T; t0 += tb) {
    const int nt = T - t0 < tb ? T - t0 : tb;
    for (int rep = 0; rep < g.nrep; ++rep) {
      near_rowexp_kernel<<<(nt + 7) / 8, 256, 0, st>>>(d_o, g, rep, t0, nt, erow, ttab);
      near_adigits_kernel<SD><<<dim3((g.Sp + 255) / 256, nt), 256, 0, st>>>(d_o, g, nt, erow, ttab,
                                                                              sxyz, A);
      near_gemm_tc_kernel<SD><<<dim3((nt + 127) / 128, (NC + kNearCols - 1) / kNearCols), kNearThreads,
                                gemm_smem, st>>>(g, nt, A, B, erow, ecol, C, h.status);
      near_combine_kernel<<<152 * 8, 256, 0, st>>>(g, rep, t0, nt, dirs, C, U, T);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
  }
  return cudaSuccess;
}

cudaError_t launch_near_image(const ObsDev *d_o, const ObsDev &h, int W, const double2 *coef,
                              double ex, double ey, const double *dirs, int slices, double2 *U,
                              void *scratch, cudaStream_t st) {
  const int T = h.M * h.P;
  char *sc = static_cast<char *>(scratch);
  double2 *sigma = reinterpret_cast<double2 *>(sc);
  sc += (sizeof(double2) * (size_t)W * h.cols * h.P + 255) & ~(size_t)255;
  // strengths of the exterior field (the first N columns of each wave)
  cudaError_t e = launch_point_strengths(d_o, h, W, coef, sigma, st);
  if (e != cudaSuccess) return e;
  if (slices <= 0) {
    double *X = reinterpret_cast<double *>(sc);
    double *Nrm = reinterpret_cast<double *>(sc + ((sizeof(double) * 3 * T + 255) & ~(size_t)255));
    ring_targets_kernel<<<152 * 4, 256, 0, st>>>(d_o, X, Nrm, T);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    axi_lattice lat{ex, ey};
    return launch_eval(d_o, h, W, sigma, T, X, Nrm, AXI_EVAL_NORMAL_DERIV, &lat, dirs, U, st);
  }
  // The point strengths are stored [W][cols][P]; the exterior field's N rows
  // come first in each wave (transmission appends the interior field's).
  const NearGeom g = make_geom(h, W, ex, ey);
  switch (slices) {
    case 4: return near_split<4>(d_o, h, g, sigma, dirs, U, sc, st);
    case 5: return near_split<5>(d_o, h, g, sigma, dirs, U, sc, st);
    case 6: return near_split<6>(d_o, h, g, sigma, dirs, U, sc, st);
    case 7: return near_split<7>(d_o, h, g, sigma, dirs, U, sc, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace axi
