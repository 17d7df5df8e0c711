// Step A2: ring-kernel modal fill (Sec. 3.1, eqs. ringkernel, ringkernelderiv, ptr).
//
// For a collocation point x_m = (rho_m, 0, z_m) with outward normal n_m and a
// proxy ring (rho'_j, z'_j), the q-node periodic trapezoid rule gives
//   A_n(m, j) = (1/q) sum_{l=0}^{q-1} g_l e^{-2 pi i n l / q},
// g_l = G_k(x_m, y_j(phi_l)) or dG_k/dn_m, phi_l = 2 pi l / q. The samples are
// even in l (g_l = g_{q-l}: the distance depends on cos phi only), so only
// l = 0..q/2 are evaluated and the transform folds to a real cosine sum
//   A_n = (1/q) [g_0 + (-1)^n g_{q/2} + 2 sum_{l=1}^{q/2-1} g_l cos(2 pi n l / q)],
// which also shows A_n = A_{-n}: only n = 0..P/2 are produced.
//
// This direct-sum form (used only when q has prime factors other than 2, 3
// and 5) evaluates every pair on all q nodes; the FFT and split forms use
// each pair's sub-grid (ObsDev::fill_sig).
//
// Mapping: one CTA = 32 consecutive collocation points (one per lane) x one
// proxy ring x one kernel kind; 8 warps. Samples for a chunk of 32 nodes are
// evaluated by all warps into shared memory, then warp w accumulates modes
// n = w, w+8, ... in registers from the shared samples and a shared cosine
// table indexed by (n l) mod q. Stores are 512-byte coalesced columns.
// Arithmetic is native FP64 throughout (the ill-conditioned MFS matrices need
// the full precision); the kernel is bound by the FP64 pipe.
#include "axi_internal.h"
#include "trig.cuh"
#include "fft.cuh"

namespace axi {
namespace {

constexpr int kThreads = 256;
constexpr int kLanes = 32;
constexpr int kChunk = 32;                 // trapezoid nodes per shared-memory chunk
constexpr int kAcc = kMaxModes / 8;        // modes per thread
constexpr double kInv4Pi = 0.07957747154594766788;

__global__ void __launch_bounds__(kThreads)
fill_kernel(const ObsDev *__restrict__ obs_arr, int oi, double2 *__restrict__ out,
            int ld_rows, int ld_cols) {
  const ObsDev &o = obs_arr[oi];
  extern __shared__ double smem[];
  double *tcos = smem;                                             // [q]
  double2 *samp = reinterpret_cast<double2 *>(smem + ((o.q + 1) & ~1));  // [kChunk][kLanes]

  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int m = blockIdx.x * kLanes + lane;
  const int j = blockIdx.y;
  const int kind = blockIdx.z;
  // Neumann: one kind (dG/dn, k, interior proxies). Transmission (eq. trans):
  // 0: A (value, k, interior), 1: A' (derivative, k, interior),
  // 2: A^- (value, k_-, exterior), 3: A'^- (derivative, k_-, exterior);
  // the minus blocks enter the system with a negative sign.
  const bool deriv = (o.bc == AXI_BC_NEUMANN) ? true : (kind & 1);
  const bool ext = (o.bc == AXI_BC_TRANSMISSION) && kind >= 2;
  const double k = ext ? o.km : o.k;
  const double *S = ext ? o.srcx : o.src;
  const double rs = S[2 * j], zs = S[2 * j + 1];
  const int mm = m < o.M ? m : o.M - 1;
  const double rho = o.coll[4 * mm], z = o.coll[4 * mm + 1];
  const double nr = o.coll[4 * mm + 2], nz = o.coll[4 * mm + 3];
  const int q = o.q, half = q / 2, D = o.D;
  const int na = (D - warp + 7) / 8;          // modes n = warp + 8a < D handled by this warp

  for (int i = threadIdx.x; i < q; i += kThreads) tcos[i] = o.tab_cos[i];

  double2 acc[kAcc];
#pragma unroll
  for (int a = 0; a < kAcc; ++a) acc[a] = make_double2(0.0, 0.0);

  const double dr = rho - rs, dz = z - zs;
  const double base = dr * dr + dz * dz, fourrr = 4.0 * rho * rs;
  const double wq = kInv4Pi / q;

  for (int l0 = 0; l0 <= half; l0 += kChunk) {
    __syncthreads();
#pragma unroll
    for (int i = 0; i < kChunk / 8; ++i) {
      const int ll = warp + 8 * i;
      const int l = l0 + ll;
      double2 s = make_double2(0.0, 0.0);
      if (l <= half) {
        // R^2 = (rho - rho')^2 + 4 rho rho' sin^2(phi/2) + (z - z')^2 (no cancellation)
        // one reciprocal square root gives both 1/R and R (FP64 rsqrt, <= 1 ulp)
        const double R2 = base + fourrr * o.tab_s2[l];
        const double inv = rsqrt(R2);
        const double R = R2 * inv;
        double sn, cs;
        trig::sincos_ring(k * R, &sn, &cs);
        const double w = ((l == 0 || l == half) ? 1.0 : 2.0) * wq;
        if (!deriv) {
          s = make_double2(cs * inv * w, sn * inv * w);
        } else {
          // dG/dn_x = (n . (x - y)) (i k R - 1) e^{ikR} / (4 pi R^3)
          const double ndot = nr * (rho - rs * tcos[l]) + nz * dz;
          const double f = ndot * inv * inv * inv * w, kR = k * R;
          s = make_double2(f * (-cs - kR * sn), f * (-sn + kR * cs));
        }
      }
      samp[ll * kLanes + lane] = s;
    }
    __syncthreads();
    const int lmax = min(kChunk, half + 1 - l0);
    for (int ll = 0; ll < lmax; ++ll) {
      const double2 s = samp[ll * kLanes + lane];
      const int l = l0 + ll;
      const int step = (8 * l) % q;
      int idx = (warp * l) % q;
      // uniform early exit: predicated-off FP64 FMAs would still occupy the pipe
#pragma unroll
      for (int a = 0; a < kAcc; ++a) {
        if (a >= na) break;
        const double c = tcos[idx];
        acc[a].x = fma(c, s.x, acc[a].x);
        acc[a].y = fma(c, s.y, acc[a].y);
        idx += step;
        if (idx >= q) idx -= q;
      }
    }
  }

  if (m >= o.M) return;
  int row = m, col = j;
  double sign = 1.0;
  if (o.bc == AXI_BC_TRANSMISSION) {
    row += (kind & 1) ? o.M : 0;
    col += ext ? o.N : 0;
    sign = ext ? -1.0 : 1.0;
  }
  const size_t mode_stride = (size_t)ld_cols * ld_rows;
  double2 *dst = out + (size_t)col * ld_rows + row;
  bool bad = false;
#pragma unroll
  for (int a = 0; a < kAcc; ++a) {
    const int n = warp + 8 * a;
    if (n < D) {
      const double2 v = make_double2(sign * acc[a].x, sign * acc[a].y);
      bad |= !isfinite(v.x) || !isfinite(v.y);
      dst[n * mode_stride] = v;
    }
  }
  if (bad) atomicOr(o.status, kStatNonFinite);
}

// FFT variant (q = 2^a 3^b 5^c): one warp per (m, j) pair evaluates the
// q/2 + 1 samples, mirrors them into the full even sequence of length q and
// transforms it in shared memory with the mixed-radix warp FFT (fft.cuh):
//   A_n = (1/q) sum_{l=0}^{q-1} g_l e^{-2 pi i n l / q},  n = 0 .. D-1.
// Per sample this costs ~5 log2(q) FP64 operations instead of 2 D FMAs.
__global__ void __launch_bounds__(256)
fill_fft_kernel(const ObsDev *__restrict__ obs_arr, int oi, double2 *__restrict__ out,
                int ld_rows, int ld_cols) {
  const ObsDev &o = obs_arr[oi];
  const int q = o.q, half = q / 2, D = o.D;
  const int nw = blockDim.x >> 5;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  extern __shared__ double2 fsm[];
  double2 *tw = fsm;                                        // [q]
  int *perm = reinterpret_cast<int *>(fsm + q);             // [q]
  double2 *seq = fsm + q + (q + 1) / 2 + warp * q;          // [nw][q]
  for (int i = threadIdx.x; i < q; i += blockDim.x) { tw[i] = o.tw_q[i]; perm[i] = o.fft_perm_q[i]; }
  const int m = blockIdx.x * nw + warp;
  const int j = blockIdx.y;
  const int kind = blockIdx.z;
  const bool deriv = (o.bc == AXI_BC_NEUMANN) ? true : (kind & 1);
  const bool ext = (o.bc == AXI_BC_TRANSMISSION) && kind >= 2;
  const double k = ext ? o.km : o.k;
  const double *S = ext ? o.srcx : o.src;
  const double rs = S[2 * j], zs = S[2 * j + 1];
  const int mm = m < o.M ? m : o.M - 1;
  const double rho = o.coll[4 * mm], z = o.coll[4 * mm + 1];
  const double nr = o.coll[4 * mm + 2], nz = o.coll[4 * mm + 3];
  const double dr = rho - rs, dz = z - zs;
  const double base = dr * dr + dz * dz, fourrr = 4.0 * rho * rs;
  // sub-grid of the pair (nodes l = 0, sg, 2 sg, ..; sg divides q/2): the other
  // nodes are zero and the weight is sg / (4 pi q), i.e. the (q/sg)-node rule
  const int sg = o.fill_sig[((size_t)(ext ? 1 : 0) * o.M + mm) * o.N + j];
  const double wq = kInv4Pi * sg / q;
  // n . (x - y_l) = (n_r rho + n_z dz) - n_r rho' cos(phi_l), with sg/(4 pi q) folded in
  const double an = (nr * rho + nz * dz) * wq, bn = nr * rs * wq;
  if (sg > 1)
    for (int l = lane; l < q; l += 32)
      if (l % sg) seq[l] = make_double2(0.0, 0.0);
  for (int i = lane; i * sg <= half; i += 32) {
    const int l = i * sg;
    const double R2 = fma(fourrr, o.tab_s2[l], base);
    const double inv = rsqrt(R2);
    const double R = R2 * inv, kR = k * R;
    double sn, cs;
    trig::sincos_ring_tab(kR, o.tab_ring, &sn, &cs);   // table in global memory (L1-resident)
    double2 s;
    if (!deriv) {
      const double iw = inv * wq;
      s = make_double2(cs * iw, sn * iw);
    } else {
      const double f = fma(-bn, o.tab_cos[l], an) * (inv * inv * inv);
      s = make_double2(f * fma(-kR, sn, -cs), f * fma(kR, cs, -sn));
    }
    seq[l] = s;
    if (l > 0 && l < half) seq[q - l] = s;
  }
  __syncthreads();                                          // tables and sequences ready
  // With fft_sum_last_q the last stage is not run: each needed mode is the
  // sum of its last-stage block (twiddle 1, output 0).
  const int rl = o.fft_sum_last_q ? o.fft_rad_q[o.fft_nst_q - 1] : 1;
  fft::warp_fft(seq, q, tw, o.fft_rad_q, o.fft_nst_q - (rl > 1 ? 1 : 0), lane);
  if (m >= o.M) return;
  int row = m, col = j;
  double sign = 1.0;
  if (o.bc == AXI_BC_TRANSMISSION) {
    row += (kind & 1) ? o.M : 0;
    col += ext ? o.N : 0;
    sign = ext ? -1.0 : 1.0;
  }
  const size_t mode_stride = (size_t)ld_cols * ld_rows;
  double2 *dst = out + (size_t)col * ld_rows + row;
  bool bad = false;
  for (int n = lane; n < D; n += 32) {
    const double2 *blk = seq + perm[n];
    double2 v0 = blk[0];
    for (int k = 1; k < rl; ++k) v0 = make_double2(v0.x + blk[k].x, v0.y + blk[k].y);
    const double2 v = make_double2(sign * v0.x, sign * v0.y);
    bad |= !isfinite(v.x) || !isfinite(v.y);
    dst[n * mode_stride] = v;
  }
  if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(o.status, kStatNonFinite);
}

}  // namespace

cudaError_t launch_fill(const ObsDev *d_obs, const ObsDev &h, int oi, double2 *out, int ld_rows,
                        int ld_cols, cudaStream_t st, int chunk_mb) {
  // split-precision plans: samples in FP64, the transform on tensor cores
  if (h.slices > 0 && h.fill_cdig != nullptr)
    return launch_fill_mma(d_obs, h, oi, out, ld_rows, ld_cols, chunk_mb, st);
  if (h.fft_nst_q > 0) {
    const int nw = h.q <= 512 ? 8 : 4;                      // pairs (warps) per CTA
    const size_t smem = sizeof(double2) * (h.q + (h.q + 1) / 2 + (size_t)nw * h.q);
    static size_t granted = 0;
    cudaError_t e = ensure_dynamic_smem(fill_fft_kernel, smem, granted);
    if (e != cudaSuccess) return e;
    dim3 grid((h.M + nw - 1) / nw, h.N, h.bc == AXI_BC_TRANSMISSION ? 4 : 1);
    fill_fft_kernel<<<grid, 32 * nw, smem, st>>>(d_obs, oi, out, ld_rows, ld_cols);
    return cudaGetLastError();
  }
  dim3 grid((h.M + kLanes - 1) / kLanes, h.N, h.bc == AXI_BC_TRANSMISSION ? 4 : 1);
  size_t smem = sizeof(double) * ((h.q + 1) & ~1) + sizeof(double2) * kChunk * kLanes;
  static size_t granted = 0;
  cudaError_t e = ensure_dynamic_smem(fill_kernel, smem, granted);
  if (e != cudaSuccess) return e;
  fill_kernel<<<grid, kThreads, smem, st>>>(d_obs, oi, out, ld_rows, ld_cols);
  return cudaGetLastError();
}

}  // namespace axi
