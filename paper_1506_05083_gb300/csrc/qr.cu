// Steps A3 and A5: blocked complex Householder QR of every distinct modal
// matrix, and application of the factors to right-hand sides.
//
// Sec. 3 (eq. linsys) solves each mode's rectangular system by a dense
// backward-stable least-squares method; Sec. 4.2 applies the factors, never
// an explicit inverse. We use unpivoted Householder QR with the LAPACK
// reflector convention: H = I - tau v v^H, v[0] = 1, and H^H maps the column
// (alpha; x) to (beta; 0) with real beta = -sign(Re alpha) ||(alpha; x)||,
// tau = (beta - alpha)/beta, v = x/(alpha - beta).
//
// Blocking (compact WY): a panel of kNB columns is factored by one CTA per
// (obstacle, mode); its reflectors combine into H_1 ... H_nb = I - V T V^H
// with T upper triangular, and the trailing matrix is updated by
//   A22 <- (I - V T^H V^H) A22 = A22 - V (T^H (V^H A22)),
// in a second launch whose CTAs each own a tile of trailing columns. The
// apply runs the same block-reflector product over the stored panels for a
// tile of right-hand-side columns, then a blocked back substitution with R.
#include "axi_internal.h"
#include "ozaki.cuh"
#include <cooperative_groups.h>

namespace cg = cooperative_groups;

namespace axi {
namespace {

constexpr int kThreads = 256;
// The shared-memory panel is bound by the FP64 pipe of one SM: 128 threads
// (about two rows each) keep the per-warp reductions and scalar work small;
// 256 threads give each SM sub-partition a second warp to cover the FP64
// latency (the tuning chooses).
constexpr int kPanelThreads = 128;
constexpr int kTN = 16;   // columns of the target per CTA in block-reflector kernels
constexpr int kRC = 32;   // rows per shared-memory chunk

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cjmul(double2 a, double2 b) {  // conj(a) * b
  return make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ double2 cadd(double2 a, double2 b) {
  return make_double2(a.x + b.x, a.y + b.y);
}
// Complex multiply-accumulate as four explicit FMAs (acc + a b, acc + conj(a) b,
// acc - a b). Written as a product plus an addition, the compiler cannot
// reassociate and issues six FP64 instructions; these kernels are bound by
// the FP64 pipe.
__device__ __forceinline__ double2 cfma(double2 acc, double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, fma(-a.y, b.y, acc.x)), fma(a.x, b.y, fma(a.y, b.x, acc.y)));
}
__device__ __forceinline__ double2 cfma_conj(double2 acc, double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, fma(a.y, b.y, acc.x)), fma(a.x, b.y, fma(-a.y, b.x, acc.y)));
}
__device__ __forceinline__ double2 cfms(double2 acc, double2 a, double2 b) {
  return make_double2(fma(-a.x, b.x, fma(a.y, b.y, acc.x)), fma(-a.x, b.y, fma(-a.y, b.x, acc.y)));
}
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Reduce-scatter of 32 values per lane over the warp: afterwards lane l holds
// the warp-wide sum of value l. Each level sends half of the remaining values
// to the partner lane and adds the other half: 31 shuffles and 31 additions
// per lane, against 160 for 32 separate butterfly sums.
__device__ __forceinline__ double warp_reduce_scatter32(double (&v)[32]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 16, n = 16; o >= 1; o >>= 1, n >>= 1) {
    const bool upper = (lane & o) != 0;
#pragma unroll
    for (int i = 0; i < n; ++i) {
      const double send = upper ? v[i] : v[i + n];
      const double keep = upper ? v[i + n] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
  }
  return v[0];
}

// Sum `n` complex partials over the CTA; result in out[0..n). Contains syncs.
__device__ void block_sum_c(double2 *part, int n, double (*red)[2 * kNB], double2 *out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int r = 0; r < n; ++r) {
    double x = warp_sum(part[r].x), y = warp_sum(part[r].y);
    if (lane == 0) { red[warp][2 * r] = x; red[warp][2 * r + 1] = y; }
  }
  __syncthreads();
  if (threadIdx.x < n) {
    double x = 0, y = 0;
    for (int w = 0; w < kThreads / 32; ++w) { x += red[w][2 * threadIdx.x]; y += red[w][2 * threadIdx.x + 1]; }
    out[threadIdx.x] = make_double2(x, y);
  }
  __syncthreads();
}

// Element (i, a) of the panel's reflector matrix V (rows i >= k0; unit
// diagonal, zeros above it, stored entries below it).
__device__ __forceinline__ double2 vget(const double2 *A, int lda, int rows, int k0, int nbp,
                                        int i, int a) {
  if (a >= nbp || i >= rows) return make_double2(0.0, 0.0);
  const int c = k0 + a;
  if (i < c) return make_double2(0.0, 0.0);
  if (i == c) return make_double2(1.0, 0.0);
  return A[(size_t)c * lda + i];
}

// ---------------------------------------------------------------------------
// Panel: unblocked Householder on columns [k0, k0+nbp) of one modal matrix,
// then the T factor of the compact WY form (forward, column-wise):
//   T(j, j) = tau_j,  T(0:j, j) = -tau_j T(0:j, 0:j) (V(:, 0:j)^H v_j).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads)
qr_panel_kernel(const ObsDev *__restrict__ obs, const int *__restrict__ task_obs,
                const int *__restrict__ task_mode, int p) {
  const ObsDev &o = obs[task_obs[blockIdx.x]];
  const int d = task_mode[blockIdx.x];
  const int lda = o.rows, rows = o.rows;
  const int k0 = p * kNB;
  const int nbp = min(kNB, o.cols - k0);
  double2 *A = o.A + (size_t)d * o.cols * lda;
  const int tid = threadIdx.x;

  __shared__ double red[kThreads / 32][2 * kNB];
  __shared__ double2 wsh[kNB];
  __shared__ double2 G[kNB][kNB];
  __shared__ double2 Tsh[kNB][kNB];
  __shared__ double2 taush[kNB];

  for (int jj = 0; jj < nbp; ++jj) {
    const int c = k0 + jj;
    double2 *col = A + (size_t)c * lda;
    // ||x||^2 of the part below the diagonal
    double s = 0.0;
    for (int i = c + 1 + tid; i < rows; i += kThreads) {
      const double2 v = col[i];
      s = fma(v.x, v.x, fma(v.y, v.y, s));
    }
    double2 part[kNB];
    part[0] = make_double2(s, 0.0);
    block_sum_c(part, 1, red, wsh);
    const double xn2 = wsh[0].x;
    const double2 alpha = col[c];
    double beta;
    double2 tau, scale;
    if (xn2 == 0.0 && alpha.y == 0.0) {
      beta = alpha.x; tau = make_double2(0.0, 0.0); scale = make_double2(0.0, 0.0);
    } else {
      const double nrm = sqrt(alpha.x * alpha.x + alpha.y * alpha.y + xn2);
      beta = -copysign(nrm, alpha.x);
      tau = make_double2((beta - alpha.x) / beta, -alpha.y / beta);
      const double2 den = make_double2(alpha.x - beta, alpha.y);
      const double dd = den.x * den.x + den.y * den.y;
      scale = make_double2(den.x / dd, -den.y / dd);       // 1 / (alpha - beta)
    }
    const int nrem = nbp - jj - 1;
#pragma unroll
    for (int r = 0; r < kNB; ++r) part[r] = make_double2(0.0, 0.0);
    for (int i = c + 1 + tid; i < rows; i += kThreads) {
      const double2 v = cmul(col[i], scale);
      col[i] = v;
#pragma unroll
      for (int r = 0; r < kNB - 1; ++r)
        if (r < nrem) part[r] = cfma_conj(part[r], v, A[(size_t)(c + 1 + r) * lda + i]);
    }
    if (tid == 0) {
#pragma unroll
      for (int r = 0; r < kNB - 1; ++r)
        if (r < nrem) part[r] = cadd(part[r], A[(size_t)(c + 1 + r) * lda + c]);
    }
    if (nrem > 0) block_sum_c(part, nrem, red, wsh);
    // A(c:, c2) -= v conj(tau) w_c2   (H^H applied to the rest of the panel)
    const double2 ctau = make_double2(tau.x, -tau.y);
    for (int i = c + tid; i < rows; i += kThreads) {
      const double2 v = (i == c) ? make_double2(1.0, 0.0) : col[i];
      for (int r = 0; r < nrem; ++r) {
        const double2 w = cmul(ctau, wsh[r]);
        double2 *x = &A[(size_t)(c + 1 + r) * lda + i];
        const double2 vw = cmul(v, w);
        *x = make_double2(x->x - vw.x, x->y - vw.y);
      }
    }
    __syncthreads();
    if (tid == 0) {
      col[c] = make_double2(beta, 0.0);
      o.tau[(size_t)d * o.cols + c] = tau;
      taush[jj] = tau;
      if (!isfinite(beta)) atomicOr(o.status, kStatNonFinite);
    }
    __syncthreads();
  }

  // Gram matrix G(a, b) = v_a^H v_b, a < b (v_b vanishes above row k0 + b).
  const int lane = tid & 31, warp = tid >> 5;
  const int npair = nbp * (nbp - 1) / 2;
  for (int pi = warp; pi < npair; pi += kThreads / 32) {
    int b = 1, acc = 0;
    while (acc + b <= pi) { acc += b; ++b; }
    const int a = pi - acc;
    const double2 *va = A + (size_t)(k0 + a) * lda;
    const double2 *vb = A + (size_t)(k0 + b) * lda;
    double2 g = make_double2(0.0, 0.0);
    for (int i = k0 + b + 1 + lane; i < rows; i += 32) g = cfma_conj(g, va[i], vb[i]);
    g.x = warp_sum(g.x);
    g.y = warp_sum(g.y);
    if (lane == 0) {
      const double2 vab = va[k0 + b];  // v_a at row k0+b, times v_b = 1 there
      G[a][b] = make_double2(g.x + vab.x, g.y - vab.y);
    }
  }
  __syncthreads();
  if (tid == 0) {
    for (int j = 0; j < kNB; ++j)
      for (int i = 0; i < kNB; ++i) Tsh[i][j] = make_double2(0.0, 0.0);
    for (int j = 0; j < nbp; ++j) {
      const double2 tj = taush[j];
      Tsh[j][j] = tj;
      for (int i = 0; i < j; ++i) {
        double2 zz = make_double2(0.0, 0.0);
        for (int l = i; l < j; ++l) zz = cadd(zz, cmul(Tsh[i][l], G[l][j]));
        const double2 t = cmul(tj, zz);
        Tsh[i][j] = make_double2(-t.x, -t.y);
      }
    }
  }
  __syncthreads();
  double2 *Tg = o.T + ((size_t)d * o.npanels + p) * kNB * kNB;
  for (int e = tid; e < kNB * kNB; e += kThreads) Tg[e] = Tsh[e % kNB][e / kNB];
}

// ---------------------------------------------------------------------------
// Panel held in shared memory, factored by a cluster of C CTAs (C = 1: one
// CTA, K = rows - k0 <= kPanelSmemRows). Thread t of CTA r owns the rows
// i = r NT + t + u C NT (NT threads per CTA) for the whole panel, so only
// reductions cross threads. Column jj needs, from the rows i > jj of its
// unscaled column x,
//   xn2 = sum |x_i|^2,  P_c = sum conj(x_i) a_c[i] (c > jj),  Q_a = sum conj(v_a[i]) x_i (a < jj);
// with scale = 1 / (alpha - beta) and v = (1; x scale),
//   v^H a_c = a_c[jj] + conj(scale) P_c,   v_a^H v = conj(v_a[jj]) + scale Q_a,
// so one reduction per column suffices. The partial sums for column jj + 1
// are formed in the same sweep that applies reflector jj to the owner's rows.
// Per column: partials reduced per warp and, with C > 1, exchanged through
// distributed shared memory (one cluster barrier; double-buffered with the
// row jj the owner publishes), then every CTA's warp 0 forms the same
// scalars, and a CTA barrier publishes them. T follows at the end from the
// Gram entries:
//   T(jj, jj) = tau_jj,  T(0:jj, jj) = -tau_jj T(0:jj, 0:jj) (V(:, 0:jj)^H v_jj).
// ---------------------------------------------------------------------------
template <int C, int NT>
__global__ void __launch_bounds__(NT)
qr_panel_smem_kernel(const ObsDev *__restrict__ obs, const int *__restrict__ task_obs,
                     const int *__restrict__ task_mode, int p) {
  constexpr int kStride = C * NT;
  constexpr int kBuf = C > 1 ? 2 : 1;
  const int rank = C > 1 ? (int)cg::this_cluster().block_rank() : 0;
  const int task = blockIdx.x / C;
  const ObsDev &o = obs[task_obs[task]];
  const int d = task_mode[task];
  const int lda = o.rows;
  const int k0 = p * kNB;
  const int nbp = min(kNB, o.cols - k0);
  const int K = o.rows - k0;
  const int Kl = C > 1 ? NT * ((K + kStride - 1) / kStride) : K;   // local rows per column
  double2 *A = o.A + (size_t)d * o.cols * lda;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int kW = NT / 32;
  constexpr int kX = kNB - 1;                  // complex partials per column
  extern __shared__ double2 Ps[];              // [nbp][Kl]; slot u NT + t holds row r NT + t + u C NT
  __shared__ double red[kBuf][kW][32];         // per-warp sums: complex x at 2x, 2x+1; xn2 at 30
  __shared__ double2 rowbuf[kBuf][kNB];        // row jj as published by its owner (C > 1)
  __shared__ double tot[32];
  __shared__ double2 wsh[kX];                  // conj(tau) v^H a_c, index c - 1
  __shared__ double2 Gsh[kNB][kNB];            // Gsh[a][j] = v_a^H v_j, a < j
  __shared__ double2 Tsh[kNB][kNB + 1];
  __shared__ double2 taush[kNB];
  __shared__ double2 sc_scale;
  auto row_of = [&](int slot) { return (slot / NT) * kStride + rank * NT + slot % NT; };
  auto owner_of = [&](int i) { return (i % kStride) / NT; };
  auto slot_of = [&](int i) { return (i / kStride) * NT + i % NT; };
  // Column j of T (one warp; columns < j, tau_j and the Gram column j are
  // complete). Done while warp 0 forms the next column's scalars, on another
  // SM sub-partition's FP64 unit.
  auto t_column = [&](int j) {
    const double2 tj = taush[j];
    if (lane < j) {
      double2 z = make_double2(0.0, 0.0);
      for (int l = lane; l < j; ++l) z = cfma(z, Tsh[lane][l], Gsh[l][j]);
      const double2 t = cmul(tj, z);
      Tsh[lane][j] = make_double2(-t.x, -t.y);
    } else if (lane == j) {
      Tsh[j][j] = tj;
    }
  };
  auto csync = [&]() {
    if constexpr (C > 1) cg::this_cluster().sync();
    else __syncthreads();
  };

  for (int e = tid; e < nbp * Kl; e += NT) {
    const int a = e / Kl, i = row_of(e % Kl);
    Ps[e] = i < K ? A[(size_t)(k0 + a) * lda + k0 + i] : make_double2(0.0, 0.0);
  }
  for (int e = tid; e < kNB * (kNB + 1); e += NT) (&Tsh[0][0])[e] = make_double2(0.0, 0.0);
  __syncthreads();
  if (C > 1 && rank == 0 && tid < nbp) rowbuf[0][tid] = Ps[tid * Kl];   // row 0 (slot 0)

  // partial sums for column 0: slot x holds P_{x+1}
  double2 part[kX];
  double2 qjj = make_double2(0.0, 0.0);        // Q of the latest reflector, for slot qslot
  int qslot = -1;
  double xn2p = 0.0;
#pragma unroll
  for (int x = 0; x < kX; ++x) part[x] = make_double2(0.0, 0.0);
  for (int slot = tid; slot < Kl; slot += NT) {
    const int i = row_of(slot);
    if (i >= K) break;
    if (i == 0) continue;
    const double2 xi = Ps[slot];
    xn2p = fma(xi.x, xi.x, fma(xi.y, xi.y, xn2p));
#pragma unroll
    for (int x = 0; x < kX; ++x) {
      if (x + 1 >= nbp) break;
      part[x] = cfma_conj(part[x], xi, Ps[(x + 1) * Kl + slot]);
    }
  }

  for (int jj = 0; jj < nbp; ++jj) {
    const int buf = kBuf > 1 ? (jj & 1) : 0;
    {
      // lane l ends with the warp sum of component l
      double v[32];
#pragma unroll
      for (int x = 0; x < kX; ++x) {
        // slot qslot holds no other partial: select, not add (an FP64 add each)
        v[2 * x] = x == qslot ? qjj.x : part[x].x;
        v[2 * x + 1] = x == qslot ? qjj.y : part[x].y;
      }
      v[30] = xn2p;
      v[31] = 0.0;
      red[buf][warp][lane] = warp_reduce_scatter32(v);
    }
    csync();                                                   // partials (and row jj) of column jj
    if (warp == 1 && jj > 0) t_column(jj - 1);                 // beside warp 0's scalars
    if (warp == 0) {
      double s = 0.0;
#pragma unroll
      for (int r = 0; r < C; ++r) {
        const double *rr = &red[buf][0][0];
        if constexpr (C > 1) rr = cg::this_cluster().map_shared_rank(rr, r);
#pragma unroll
        for (int w = 0; w < kW; ++w) s += rr[w * 32 + lane];
      }
      tot[lane] = s;
      // row jj: local shared memory (C = 1) or the owner's published copy
      const int own = owner_of(jj);
      const double2 *rowj;
      int rstride;
      if constexpr (C > 1) {
        rowj = cg::this_cluster().map_shared_rank(&rowbuf[buf][0], own);
        rstride = 1;
      } else {
        rowj = Ps + jj;
        rstride = Kl;
      }
      __syncwarp();
      const double xn2 = tot[30];
      const double2 alpha = rowj[jj * rstride];
      double beta;
      double2 tau, scale;
      if (xn2 == 0.0 && alpha.y == 0.0) {
        beta = alpha.x; tau = make_double2(0.0, 0.0); scale = make_double2(0.0, 0.0);
      } else {
        // one reciprocal square root gives both |beta| and 1 / beta
        const double s2 = fma(alpha.x, alpha.x, fma(alpha.y, alpha.y, xn2));
        const double rs = rsqrt(s2);
        beta = -copysign(s2 * rs, alpha.x);
        const double ib = -copysign(rs, alpha.x);
        tau = make_double2((beta - alpha.x) * ib, -alpha.y * ib);
        const double2 den = make_double2(alpha.x - beta, alpha.y);
        const double idd = 1.0 / (den.x * den.x + den.y * den.y);
        scale = make_double2(den.x * idd, -den.y * idd);        // 1 / (alpha - beta)
      }
      if (lane < kX) {
        const double2 val = make_double2(tot[2 * lane], tot[2 * lane + 1]);
        if (lane < jj) {
          const double2 va = rowj[lane * rstride];
          Gsh[lane][jj] = cfma(make_double2(va.x, -va.y), scale, val);      // conj(v_a[jj]) + scale Q_a
        } else if (lane + 1 < nbp) {
          const double2 vh = cfma_conj(rowj[(lane + 1) * rstride], scale, val);  // a_c[jj] + conj(scale) P_c
          wsh[lane] = cjmul(tau, vh);
        }
      }
      if (lane == 0) {
        if (rank == own) Ps[jj * Kl + slot_of(jj)] = make_double2(beta, 0.0);
        taush[jj] = tau;
        sc_scale = scale;
        if (rank == 0 && !isfinite(beta)) atomicOr(o.status, kStatNonFinite);
      }
    }
    __syncthreads();                                           // scalars of column jj
    // Apply reflector jj to the owner's rows, scale v, and form the partial
    // sums of column jn = jj + 1 (slot x < jn: Q_x; x >= jn: P_{x+1}).
    const double2 scale = sc_scale;
    const int jn = jj + 1;
    double2 w[kX];
#pragma unroll
    for (int x = kX - 1; x >= 0; --x) {
      if (x < jj) break;
      w[x] = wsh[x];
    }
#pragma unroll
    for (int x = 0; x < kX; ++x) part[x] = make_double2(0.0, 0.0);
    qjj = make_double2(0.0, 0.0);
    qslot = jj;
    xn2p = 0.0;
    const double2 wj = jn < nbp ? wsh[jj] : make_double2(0.0, 0.0);   // column jn's coefficient
    for (int slot = tid; slot < Kl; slot += NT) {
      const int i = row_of(slot);
      if (i >= K) break;
      if (i < jj) continue;
      // Row jj (v = 1) takes the same instruction path as the rows below it:
      // a separate branch would add its FP64 instructions to the warp's count.
      const bool diag = i == jj;
      double2 v = cmul(Ps[jj * Kl + slot], scale);
      if (diag) v = make_double2(1.0, 0.0);
      else Ps[jj * Kl + slot] = v;
      if (jn >= nbp) continue;
      const bool acc = i > jn;
      const double2 xn = cfms(Ps[jn * Kl + slot], v, wj);
      Ps[jn * Kl + slot] = xn;
      if (acc) {
        xn2p = fma(xn.x, xn.x, fma(xn.y, xn.y, xn2p));
        qjj = cfma_conj(qjj, v, xn);
      }
#pragma unroll
      for (int x = kX - 1; x >= 0; --x) {                      // columns c = x + 1 > jn
        if (x < jn) break;
        if (x + 1 >= nbp) continue;
        double2 *y = Ps + (x + 1) * Kl + slot;
        const double2 yn = cfms(*y, v, w[x]);
        *y = yn;
        if (acc) part[x] = cfma_conj(part[x], xn, yn);
      }
      if (acc) {
#pragma unroll
        for (int x = 0; x < kX; ++x) {                         // Gram with earlier reflectors a < jj
          if (x >= jj) break;
          part[x] = cfma_conj(part[x], Ps[x * Kl + slot], xn);
        }
      }
      if (C > 1 && i == jn) {                                  // publish row jn for its scalars
        for (int c = 0; c < nbp; ++c) rowbuf[jn & 1][c] = Ps[c * Kl + slot];
      }
    }
  }
  csync();        // no CTA leaves while another may still read its shared memory
  if (warp == 1) t_column(nbp - 1);
  __syncthreads();
  for (int e = tid; e < nbp * Kl; e += NT) {
    const int a = e / Kl, i = row_of(e % Kl);
    if (i < K) A[(size_t)(k0 + a) * lda + k0 + i] = Ps[e];
  }
  if (rank == 0) {
    if (tid < nbp) o.tau[(size_t)d * o.cols + k0 + tid] = taush[tid];
    double2 *Tg = o.T + ((size_t)d * o.npanels + p) * kNB * kNB;
    for (int e = tid; e < kNB * kNB; e += NT) Tg[e] = Tsh[e % kNB][e / kNB];
  }
  if (o.slices == 0) return;

  // Split plans: the exponent of each reflector column (the largest |V(i, a)|
  // over all rows, unit diagonal included) for the digits of V^H, which
  // vdigits_kernel (qr_split.cu) writes next over the whole GPU.
  const int kp = o.kp;
  const int dslot = o.dig_kept ? p : (p & 1);
  int *vex = o.vexp + ((size_t)d * o.dig_nslot + dslot) * (kNB + kp);
  __shared__ unsigned long long colkey[kNB], wkey[kW][kNB];
  {
    unsigned long long m[kNB];
#pragma unroll
    for (int a = 0; a < kNB; ++a) m[a] = 0ull;
    for (int sl = tid; sl < Kl; sl += NT) {
      const int i = row_of(sl);
      if (i >= K) break;
#pragma unroll
      for (int a = 0; a < kNB; ++a) {
        const double2 v = (a >= nbp || i < a) ? make_double2(0.0, 0.0)
                          : (i == a ? make_double2(1.0, 0.0) : Ps[a * Kl + sl]);
        const unsigned long long k = oz::abs_key2(v);
        m[a] = k > m[a] ? k : m[a];
      }
    }
#pragma unroll
    for (int a = 0; a < kNB; ++a) {
#pragma unroll
      for (int o2 = 16; o2 > 0; o2 >>= 1) {
        const unsigned long long w = __shfl_xor_sync(0xffffffffu, m[a], o2);
        m[a] = w > m[a] ? w : m[a];
      }
      if (lane == 0) wkey[warp][a] = m[a];
    }
  }
  __syncthreads();
  if (tid < kNB) {
    unsigned long long m = 0ull;
    for (int w = 0; w < kW; ++w) m = wkey[w][tid] > m ? wkey[w][tid] : m;
    colkey[tid] = m;
  }
  csync();                                       // every CTA's column maxima
  if (rank == 0 && tid < kNB) {
    // the column maxima of Y = V T (y_rows_kernel) start from zero
    o.ykey[((size_t)d * 2 + (p & 1)) * kNB + tid] = 0ull;
    unsigned long long m = 0ull;
#pragma unroll
    for (int r = 0; r < C; ++r) {
      const unsigned long long *ck = colkey;
      if constexpr (C > 1) ck = cg::this_cluster().map_shared_rank(colkey, r);
      m = ck[tid] > m ? ck[tid] : m;
    }
    vex[tid] = oz::key_exponent(m);
  }
  csync();                                       // remote reads done before any CTA leaves
}

// ---------------------------------------------------------------------------
// X(k0:rows, 0:ncols) <- (I - V T^H V^H) X(k0:rows, 0:ncols) for one panel.
// One CTA, kTN target columns; FP64. Thread (a, c) = (tid / kTN, tid % kTN).
// ---------------------------------------------------------------------------
template <int TN>
struct BrSmem {
  double2 W[kNB][TN + 1];
  double2 T[kNB][kNB + 1];
};

template <int TN>
__device__ void apply_block_reflector_h(const double2 *__restrict__ A, int lda, int rows, int k0,
                                        int nbp, const double2 *__restrict__ Tg,
                                        double2 *__restrict__ X, int ldx, int ncols,
                                        BrSmem<TN> &sm) {
  constexpr int NT = kNB * TN;             // threads: one per (reflector, column) of W
  const int tid = threadIdx.x;
  const int ta = tid / TN, tc = tid % TN;
  for (int e = tid; e < kNB * kNB; e += NT) sm.T[e % kNB][e / kNB] = Tg[e];
  // W(ta, tc) = v_ta^H x_tc straight from global memory (L1-cached; no
  // block barriers in the loop): v is 1 at row k0 + ta and zero above it.
  double2 w = make_double2(0.0, 0.0);
  if (ta < nbp && tc < ncols) {
    const int c = k0 + ta;
    const double2 *va = A + (size_t)c * lda;
    const double2 *xc = X + (size_t)tc * ldx;
    w = xc[c];
#pragma unroll 4
    for (int r = c + 1; r < rows; ++r) w = cfma_conj(w, va[r], xc[r]);
  }
  sm.W[ta][tc] = w;
  __syncthreads();
  // W' = T^H W  (T upper triangular, so T^H is lower)
  double2 wp = make_double2(0.0, 0.0);
  for (int b = 0; b <= ta; ++b) wp = cfma_conj(wp, sm.T[b][ta], sm.W[b][tc]);
  __syncthreads();
  sm.W[ta][tc] = wp;
  __syncthreads();
  // X -= V W'
  const int r = tid % kRC, cg = tid / kRC;  // 8 column groups
  for (int r0 = k0; r0 < rows; r0 += kRC) {
    const int i = r0 + r;
    double2 vrow[kNB];
#pragma unroll
    for (int a = 0; a < kNB; ++a) vrow[a] = vget(A, lda, rows, k0, nbp, i, a);
    if (i < rows) {
      for (int c = cg; c < ncols; c += NT / kRC) {
        double2 x = X[(size_t)c * ldx + i];
#pragma unroll
        for (int a = 0; a < kNB; ++a) x = cfms(x, vrow[a], sm.W[a][c]);
        X[(size_t)c * ldx + i] = x;
      }
    }
  }
  __syncthreads();
}

template <int TN>
__global__ void __launch_bounds__(kNB * TN)
qr_update_kernel(const ObsDev *__restrict__ obs, const int *__restrict__ task_obs,
                 const int *__restrict__ task_mode, int p, int col_off) {
  const ObsDev &o = obs[task_obs[blockIdx.x]];
  const int d = task_mode[blockIdx.x];
  const int k0 = p * kNB;
  const int nbp = min(kNB, o.cols - k0);
  const int c0 = k0 + nbp + col_off + blockIdx.y * TN;
  if (c0 >= o.cols) return;
  const int ncols = min(TN, o.cols - c0);
  __shared__ BrSmem<TN> sm;
  double2 *A = o.A + (size_t)d * o.cols * o.rows;
  const double2 *Tg = o.T + ((size_t)d * o.npanels + p) * kNB * kNB;
  apply_block_reflector_h<TN>(A, o.rows, o.rows, k0, nbp, Tg, A + (size_t)c0 * o.rows, o.rows,
                              ncols, sm);
}

// Q^H applied to the RHS block of mode d: X_d is [2W][rows] column-major.
// Narrow tiles (kTA columns, 128 threads) give several CTAs per mode: the 12+
// panel applications of one tile are sequential, so parallelism comes from
// modes x tiles.
constexpr int kTA = 8;
__global__ void __launch_bounds__(kNB * kTA)
apply_qh_kernel(const ObsDev *__restrict__ od, double2 *__restrict__ X, int ncols_total) {
  const ObsDev &o = *od;
  const int d = blockIdx.x;
  if (!owns_mode(o, d)) return;
  const int c0 = blockIdx.y * kTA;
  if (c0 >= ncols_total) return;
  const int ncols = min(kTA, ncols_total - c0);
  __shared__ BrSmem<kTA> sm;
  const double2 *A = o.A + (size_t)d * o.cols * o.rows;
  double2 *Xd = X + ((size_t)d * ncols_total + c0) * o.rows;
  for (int p = 0; p < o.npanels; ++p) {
    const int k0 = p * kNB;
    const int nbp = min(kNB, o.cols - k0);
    const double2 *Tg = o.T + ((size_t)d * o.npanels + p) * kNB * kNB;
    apply_block_reflector_h<kTA>(A, o.rows, o.rows, k0, nbp, Tg, Xd, o.rows, ncols, sm);
  }
}

// Blocked back substitution R X = Y on the first `cols` rows of each RHS
// column (R real-diagonal upper triangle of the packed factors). One warp
// per RHS column inside 32x32 diagonal blocks; rows above are updated with
// the solved block before moving up.
constexpr int kTB = 32;
constexpr int kTS = 8;    // RHS columns per CTA in the triangular solve (one warp each)
__global__ void __launch_bounds__(kThreads)
trsm_kernel(const ObsDev *__restrict__ od, double2 *__restrict__ X, int ncols_total) {
  const ObsDev &o = *od;
  const int d = blockIdx.x;
  if (!owns_mode(o, d)) return;
  const int c0 = blockIdx.y * kTS;
  if (c0 >= ncols_total) return;
  const int ncols = min(kTS, ncols_total - c0);
  const double2 *R = o.A + (size_t)d * o.cols * o.rows;
  const int ld = o.rows, n = o.cols;
  double2 *Xd = X + ((size_t)d * ncols_total + c0) * o.rows;
  __shared__ double2 Rb[kTB][kTB + 1];
  __shared__ double2 Yb[kTB][kTS + 1];
  __shared__ double rinv[kTB];              // 1 / R_ii of the block (real diagonal)
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nblk = (n + kTB - 1) / kTB;
  for (int ib = nblk - 1; ib >= 0; --ib) {
    const int r0 = ib * kTB, nb = min(kTB, n - r0);
    __syncthreads();
    for (int e = tid; e < kTB * kTB; e += kThreads) {
      const int r = e % kTB, c = e / kTB;
      Rb[r][c] = (r < nb && c < nb) ? R[(size_t)(r0 + c) * ld + r0 + r] : make_double2(0.0, 0.0);
    }
    for (int e = tid; e < kTB * kTS; e += kThreads) {
      const int r = e % kTB, c = e / kTB;
      Yb[r][c] = (r < nb && c < ncols) ? Xd[(size_t)c * ld + r0 + r] : make_double2(0.0, 0.0);
    }
    // the block's reciprocals in one parallel division (a division per
    // elimination step would sit on every warp's sequential chain)
    if (tid < kTB) rinv[tid] = tid < nb ? 1.0 / R[(size_t)(r0 + tid) * ld + r0 + tid].x : 0.0;
    __syncthreads();
    for (int c = warp; c < ncols; c += kThreads / 32) {
      double2 y = Yb[lane][c];
      for (int rr = nb - 1; rr >= 0; --rr) {
        double2 x = make_double2(0.0, 0.0);
        if (lane == rr) {
          const double inv = rinv[rr];            // real diagonal (beta of the reflector)
          y = make_double2(y.x * inv, y.y * inv);
          x = y;
        }
        x.x = __shfl_sync(0xffffffffu, x.x, rr);
        x.y = __shfl_sync(0xffffffffu, x.y, rr);
        if (lane < rr) y = cfms(y, Rb[lane][rr], x);
      }
      Yb[lane][c] = y;
    }
    __syncthreads();
    for (int e = tid; e < kTB * kTS; e += kThreads) {
      const int r = e % kTB, c = e / kTB;
      if (r < nb && c < ncols) Xd[(size_t)c * ld + r0 + r] = Yb[r][c];
    }
    // rows above: Y(0:r0, c) -= R(0:r0, r0:r0+nb) X_b(:, c)
    for (int e = tid; e < r0 * kTS; e += kThreads) {
      const int r = e % r0, c = e / r0;
      if (c >= ncols) continue;
      double2 acc = Xd[(size_t)c * ld + r];
      for (int b = 0; b < nb; ++b) acc = cfms(acc, R[(size_t)(r0 + b) * ld + r], Yb[b][c]);
      Xd[(size_t)c * ld + r] = acc;
    }
  }
}

// fhat_n = (1/P) sum_l f_l e^{-2 pi i n l / P} (eq. fhatquad with q = P),
// written as RHS blocks X[d][2w + s][row]: s = 0 holds mode +d, s = 1 mode -d.
constexpr int kDR = 16;  // rows per CTA
__global__ void __launch_bounds__(kThreads)
rhs_dft_kernel(const ObsDev *__restrict__ od, int W, const double2 *__restrict__ f,
               double2 *__restrict__ X) {
  const ObsDev &o = *od;
  const int P = o.P, rows = o.rows;
  const int w = blockIdx.y;
  const int r0 = blockIdx.x * kDR;
  extern __shared__ double2 sh[];
  double2 *tw = sh;            // [P]
  double2 *F = sh + P;         // [kDR][P + 1] (padded rows: conflict-free reads)
  const int ldF = P + 1;
  for (int i = threadIdx.x; i < P; i += kThreads) tw[i] = o.tw_P[i];
  for (int e = threadIdx.x; e < kDR * P; e += kThreads) {
    const int r = e / P, l = e % P;
    F[r * ldF + l] = (r0 + r < rows) ? f[((size_t)w * rows + r0 + r) * P + l] : make_double2(0.0, 0.0);
  }
  __syncthreads();
  const int r = threadIdx.x % kDR, tn = threadIdx.x / kDR;  // 16 mode lanes
  const int row = r0 + r;
  const double invP = 1.0 / P;
  const int ncol = 2 * W;
  for (int ni = tn; ni < P; ni += kThreads / kDR) {
    double2 acc = make_double2(0.0, 0.0);
    int idx = 0;
    for (int l = 0; l < P; ++l) {
      acc = cfma(acc, F[r * ldF + l], tw[idx]);
      idx += ni;
      if (idx >= P) idx -= P;
    }
    acc.x *= invP;
    acc.y *= invP;
    if (row < rows) {
      const int dmode = ni <= P / 2 ? ni : P - ni;
      const int s = ni <= P / 2 ? 0 : 1;
      X[((size_t)dmode * ncol + 2 * w + s) * rows + row] = acc;
      if (dmode == 0 || 2 * dmode == P)  // +-n coincide: duplicate to keep X defined
        X[((size_t)dmode * ncol + 2 * w + 1) * rows + row] = acc;
    }
  }
}

// coef[w][n mod P][j] from the solved blocks.
__global__ void scatter_coef_kernel(const ObsDev *__restrict__ od, int W,
                                    const double2 *__restrict__ X, double2 *__restrict__ coef) {
  const ObsDev &o = *od;
  const int P = o.P, cols = o.cols, rows = o.rows;
  const int ni = blockIdx.x, w = blockIdx.y;
  const int dmode = ni <= P / 2 ? ni : P - ni;
  const int s = ni <= P / 2 ? 0 : 1;
  const double2 *src = X + ((size_t)dmode * 2 * W + 2 * w + s) * rows;
  double2 *dst = coef + ((size_t)w * P + ni) * cols;
  const bool own = owns_mode(o, dmode);              // other processes own the rest
  for (int j = threadIdx.x; j < cols; j += blockDim.x) dst[j] = own ? src[j] : make_double2(0.0, 0.0);
}

// sigma[w][j][l] = (1/P) sum_n c[w][n][j] e^{+2 pi i n l / P}  (Sec. 4.1)
__global__ void __launch_bounds__(kThreads)
point_strength_kernel(const ObsDev *__restrict__ od, int W, const double2 *__restrict__ coef,
                      double2 *__restrict__ sigma) {
  const ObsDev &o = *od;
  const int P = o.P, cols = o.cols;
  const int w = blockIdx.y;
  const int j = blockIdx.x * 32 + (threadIdx.x & 31);
  extern __shared__ double2 sh[];
  double2 *tw = sh;  // e^{-2 pi i r / P}
  for (int i = threadIdx.x; i < P; i += kThreads) tw[i] = o.tw_P[i];
  __syncthreads();
  if (j >= cols) return;
  const double invP = 1.0 / P;
  for (int l = threadIdx.x >> 5; l < P; l += kThreads / 32) {
    double2 acc = make_double2(0.0, 0.0);
    for (int ni = 0; ni < P; ++ni) {
      const int nn = ni <= P / 2 ? ni : ni - P;      // signed mode
      int idx = (int)(((long long)nn * l) % P);
      if (idx < 0) idx += P;
      const double2 e = tw[idx];                      // e^{-2 pi i n l / P}
      const double2 ep = make_double2(e.x, -e.y);     // e^{+2 pi i n l / P}
      acc = cfma(acc, coef[((size_t)w * P + ni) * cols + j], ep);
    }
    sigma[((size_t)w * cols + j) * P + l] = make_double2(acc.x * invP, acc.y * invP);
  }
}

}  // namespace

namespace {

template <int C, int NT>
cudaError_t launch_panel_cluster(const ObsDev *d_obs, const int *d_task_obs, const int *d_task_mode,
                                 int ntasks, int p, int max_panel_rows, cudaStream_t st) {
  auto local_rows = [](int K) {
    return C > 1 ? NT * ((K + C * NT - 1) / (C * NT)) : K;
  };
  // the step's own panel height (the first step is the tallest, so the grant
  // made there covers the rest of the build)
  const size_t smem = sizeof(double2) * (size_t)kNB * local_rows(max_panel_rows);
  static size_t granted = 0;
  cudaError_t e = ensure_dynamic_smem(qr_panel_smem_kernel<C, NT>, smem, granted);
  if (e != cudaSuccess) return e;
  static const bool carve = (prefer_max_shared(qr_panel_smem_kernel<C, NT>), true);
  (void)carve;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(ntasks * C);
  cfg.blockDim = dim3(NT);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = C;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = C > 1 ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, qr_panel_smem_kernel<C, NT>, d_obs, d_task_obs, d_task_mode, p);
}

}  // namespace

int sm_count() {
  static int n = 0;
  if (n == 0) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0)
      n = 1;
  }
  return n;
}

// Whether one CTA of NT threads can hold a panel of `rows` rows (dynamic)
// beside the kernel's static shared arrays.
template <int NT>
bool panel_fits_one_cta(int rows) {
  static int limit = -1;
  static size_t static_bytes = 0;
  if (limit < 0) {
    int dev = 0, optin = 0;
    cudaFuncAttributes fa;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
        cudaFuncGetAttributes(&fa, qr_panel_smem_kernel<1, NT>) != cudaSuccess)
      return false;
    limit = optin;
    static_bytes = fa.sharedSizeBytes;
  }
  return static_bytes + sizeof(double2) * (size_t)kNB * rows <= (size_t)limit;
}

// The panel is bound by the FP64 pipe of the SMs that factor it: when the
// step has few tasks, each is spread over a cluster of 2 or 4 CTAs (SMs).
template <int NT>
cudaError_t launch_panel_nt(const ObsDev *d_obs, const int *d_task_obs, const int *d_task_mode,
                            int ntasks, int p, int max_panel_rows, int cluster, cudaStream_t st) {
  const int sms = sm_count();
  if (cluster == 4 || (cluster == 0 && 4 * ntasks <= sms))
    return launch_panel_cluster<4, NT>(d_obs, d_task_obs, d_task_mode, ntasks, p, max_panel_rows, st);
  if (cluster == 2 || (cluster == 0 && 2 * ntasks <= sms))
    return launch_panel_cluster<2, NT>(d_obs, d_task_obs, d_task_mode, ntasks, p, max_panel_rows, st);
  if (!panel_fits_one_cta<NT>(max_panel_rows))   // the panel and the static arrays exceed one CTA
    return launch_panel_cluster<2, NT>(d_obs, d_task_obs, d_task_mode, ntasks, p, max_panel_rows, st);
  return launch_panel_cluster<1, NT>(d_obs, d_task_obs, d_task_mode, ntasks, p, max_panel_rows, st);
}

// The panel is bound by the FP64 pipe of the SMs that factor it: when the
// step has few tasks, each is spread over a cluster of 2 or 4 CTAs (SMs).
cudaError_t launch_qr_panel(const ObsDev *d_obs, const int *d_task_obs, const int *d_task_mode,
                            int ntasks, int p, int max_panel_rows, int slices, int cluster,
                            int threads, int fixed, cudaStream_t st, bool *digits_written) {
  // the shared-memory panel also writes the reflector columns' exponents,
  // after which vdigits_kernel writes split plans' digits (launch_vdigits)
  *digits_written = slices > 0 && max_panel_rows <= kPanelSmemRows;
  if (ntasks <= 0) return cudaSuccess;
  if (slices > 0 && max_panel_rows <= kPanelSmemRows && fixed == 2 && cluster <= 1) {
    // split plans, on request: the panel in fixed point on one CTA per mode
    // (threads 0: 256 above 128 rows, else 128), where the panel fits one CTA
    const int nt = threads != 0 ? threads : (max_panel_rows > 128 ? 256 : 128);
    if (panel_fx_fits(max_panel_rows, nt))
      return launch_qr_panel_fx(d_obs, d_task_obs, d_task_mode, ntasks, p, max_panel_rows, nt, st);
    return cudaErrorInvalidConfiguration;                     // asked for, but it does not fit
  }
  if (max_panel_rows <= kPanelSmemRows) {
    // threads 0 (auto): 256 when the panel runs on one CTA and has more than
    // 128 rows (two warps per SM sub-partition hide the FP64 latency of the
    // per-row sweep; in clusters the wider CTAs' exchanges cost more), else 128
    const int sms = sm_count();
    const int c_auto = (cluster == 0 && 4 * ntasks <= sms) ? 4 : (cluster == 0 && 2 * ntasks <= sms) ? 2 : 1;
    const int c_eff = cluster != 0 ? cluster : c_auto;
    const bool wide = threads == 256 || (threads == 0 && c_eff == 1 && max_panel_rows > 128);
    if (wide)
      return launch_panel_nt<256>(d_obs, d_task_obs, d_task_mode, ntasks, p, max_panel_rows,
                                  cluster, st);
    return launch_panel_nt<kPanelThreads>(d_obs, d_task_obs, d_task_mode, ntasks, p,
                                          max_panel_rows, cluster, st);
  }
  qr_panel_kernel<<<ntasks, kThreads, 0, st>>>(d_obs, d_task_obs, d_task_mode, p);
  return cudaGetLastError();
}

// The next panel's kNB columns, in native FP64 with narrow tiles (two CTAs
// per mode): this update is on the critical path of the factorisation, where
// the split path would first need the panel's digits.
cudaError_t launch_qr_update_next(const ObsDev *d_obs, const int *d_task_obs,
                                  const int *d_task_mode, int ntasks, int p, cudaStream_t st) {
  if (ntasks <= 0) return cudaSuccess;
  static const bool carve = (prefer_max_shared(qr_update_kernel<kTA>), true);
  (void)carve;
  qr_update_kernel<kTA><<<dim3(ntasks, kNB / kTA), kNB * kTA, 0, st>>>(d_obs, d_task_obs,
                                                                      d_task_mode, p, 0);
  return cudaGetLastError();
}

// Columns from kNB past the panel onward, native FP64 or split digits.
cudaError_t launch_qr_update_rest(const ObsDev *d_obs, const int *d_task_obs,
                                  const int *d_task_mode, int ntasks, int p, int slices,
                                  int max_rest_cols, int rest_grid, bool use_y, cudaStream_t st) {
  if (ntasks <= 0 || max_rest_cols <= 0) return cudaSuccess;
  if (slices > 0 && use_y && (rest_grid == 0 || rest_grid == 2 || rest_grid == 3))
    return launch_qr_update_tc(d_obs, d_task_obs, d_task_mode, ntasks, p, slices, max_rest_cols,
                               rest_grid == 3, st);
  if (slices > 0)
    return launch_qr_update_split(d_obs, d_task_obs, d_task_mode, ntasks, p, slices, kNB,
                                  (max_rest_cols + split_update_tile_cols() - 1) /
                                      split_update_tile_cols(),
                                  split_update_tile_cols(), rest_grid == 1, use_y, st);
  static const bool carve = (prefer_max_shared(qr_update_kernel<kTN>), true);
  (void)carve;
  qr_update_kernel<kTN><<<dim3(ntasks, (max_rest_cols + kTN - 1) / kTN), kThreads, 0, st>>>(
      d_obs, d_task_obs, d_task_mode, p, kNB);
  return cudaGetLastError();
}

cudaError_t launch_apply(const ObsDev *d_o, const ObsDev &h, int W, const double2 *f,
                         double2 *coef, double2 *sigma, double2 *X, void *digit_scratch,
                         cudaStream_t st) {
  const int ncol = 2 * W;
  // algorithmic flops over the W x P right-hand sides: Q^H 16 rows cols - 8 cols^2,
  // back substitution 4 cols^2 each
  const double rhs = (double)W * h.P;
  int pid = prof_begin(AXI_KERNEL_APPLY_RHS, st);
  if (h.fft_nst > 0) {
    cudaError_t e = launch_rhs_fft(d_o, h, W, f, X, st);
    if (e != cudaSuccess) return e;
  } else {
    dim3 grid((h.rows + kDR - 1) / kDR, W);
    size_t smem = sizeof(double2) * (h.P + (size_t)kDR * (h.P + 1));
    static size_t granted = 0;
    cudaError_t ea = ensure_dynamic_smem(rhs_dft_kernel, smem, granted);
    if (ea != cudaSuccess) return ea;
    rhs_dft_kernel<<<grid, kThreads, smem, st>>>(d_o, W, f, X);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  prof_end(pid, st);
  cudaError_t e;
  pid = prof_begin(AXI_KERNEL_APPLY_QH, st);
  if (h.slices > 0 && W >= kSplitApplyMinWaves) {
    e = launch_apply_qh_split(d_o, h, X, ncol, digit_scratch, st);
  } else {
    apply_qh_kernel<<<dim3(h.D, (ncol + kTA - 1) / kTA), kNB * kTA, 0, st>>>(d_o, X, ncol);
    e = cudaGetLastError();
  }
  prof_end(pid, st, rhs * (16.0 * h.rows * h.cols - 8.0 * h.cols * h.cols));
  if (e != cudaSuccess) return e;
  pid = prof_begin(AXI_KERNEL_APPLY_TRSM, st);
  if (h.tsvd) {
    e = launch_tsvd_apply(d_o, h, X, ncol, st);     // V Sigma^+ U_R^H instead of R^{-1}
  } else if (h.slices > 0) {
    e = launch_trsm_split(d_o, h, X, ncol, st);
  } else {
    trsm_kernel<<<dim3(h.D, (ncol + kTS - 1) / kTS), kThreads, 0, st>>>(d_o, X, ncol);
    e = cudaGetLastError();
  }
  prof_end(pid, st, rhs * 4.0 * h.cols * h.cols);
  if (e != cudaSuccess) return e;
  pid = prof_begin(AXI_KERNEL_APPLY_OUT, st);
  scatter_coef_kernel<<<dim3(h.P, W), 128, 0, st>>>(d_o, W, X, coef);
  e = cudaGetLastError();
  if (e == cudaSuccess && sigma) e = launch_point_strengths(d_o, h, W, coef, sigma, st);
  prof_end(pid, st);
  return e;
}

cudaError_t launch_point_strengths(const ObsDev *d_o, const ObsDev &h, int W, const double2 *coef,
                                   double2 *sigma, cudaStream_t st) {
  if (h.fft_nst > 0) return launch_point_fft(d_o, h, W, coef, sigma, st);
  dim3 grid((h.cols + 31) / 32, W);
  point_strength_kernel<<<grid, kThreads, sizeof(double2) * h.P, st>>>(d_o, W, coef, sigma);
  return cudaGetLastError();
}

}  // namespace axi
