// Step A7: the eight phased nearest-image sums at all ring nodes (Sec. 4.2,
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
// Arithmetic: kernel values are generated in FP64 (rsqrt, sincos) and both
// operands are split into S balanced base-128 digits (ozaki.cuh); the GEMM
// runs on BF16 mma.sync with all digit groups' FP32 sums live, folded into
// int64 every 256 products of the contraction. Both operands are split with
// one bit of headroom so every digit satisfies |d| <= 64; a group sum of one
// complex component then stays below 256 * 2 * 7 * 2^12 < 2^24, an exact FP32
// integer converted with __float2int_rn.
#include "axi_internal.h"
#include "trig.cuh"
#include "ozaki.cuh"

namespace axi {
namespace {

constexpr double kInv4Pi = 0.07957747154594766788;
constexpr int kGM = 64;        // targets per GEMM CTA
constexpr int kGN = 32;        // (rotation, wave) columns per GEMM CTA
constexpr int kGK = 32;        // contraction chunk
constexpr int kLDK = kGK + 8;  // padded k stride in shared memory
constexpr int kFlushChunks = 8;  // fold FP32 group sums every 8 chunks (256 products)

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
// digit within 64.
__global__ void __launch_bounds__(256)
near_rowexp_kernel(const ObsDev *__restrict__ od, NearGeom g, int rep, int t0, int nt,
                   int *__restrict__ erow) {
  const ObsDev &o = *od;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ti = blockIdx.x * 8 + warp;
  if (ti >= nt) return;
  double tx, ty, tz, nx, ny, nz;
  target_point(o, t0 + ti, tx, ty, tz, nx, ny, nz);
  const double sx = g.rep_a[rep] * g.ex, sy = g.rep_b[rep] * g.ey;
  double r2min = 1e300;
  for (int s = lane; s < g.S; s += 32) {
    double x, y, z;
    source_point(o, s, x, y, z);
    const double dx = tx - x - sx, dy = ty - y - sy, dz = tz - z;
    r2min = fmin(r2min, fma(dx, dx, fma(dy, dy, dz * dz)));
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) r2min = fmin(r2min, __shfl_xor_sync(0xffffffffu, r2min, off));
  if (lane == 0) {
    const double bound = sqrt(1.0 + g.k * g.k * r2min) / r2min * kInv4Pi;
    erow[ti] = oz::key_exponent(oz::abs_key(bound)) + 1;
  }
}

// Kernel-value digits of the representative image for targets [t0, t0 + nt):
// A[s][part][ti][Sp] (k = source index contiguous), zero beyond S.
template <int SD>
__global__ void __launch_bounds__(256)
near_adigits_kernel(const ObsDev *__restrict__ od, NearGeom g, int rep, int t0, int nt,
                    const int *__restrict__ erow, unsigned short *__restrict__ A) {
  const ObsDev &o = *od;
  const int ti = blockIdx.y;
  const int s = blockIdx.x * 256 + threadIdx.x;
  if (ti >= nt || s >= g.Sp) return;
  double2 kv = make_double2(0.0, 0.0);
  if (s < g.S) {
    double tx, ty, tz, nx, ny, nz, x, y, z;
    target_point(o, t0 + ti, tx, ty, tz, nx, ny, nz);
    source_point(o, s, x, y, z);
    const double dx = tx - x - g.rep_a[rep] * g.ex, dy = ty - y - g.rep_b[rep] * g.ey, dz = tz - z;
    const double R2 = fma(dx, dx, fma(dy, dy, dz * dz));
    const double inv = rsqrt(R2);
    const double R = R2 * inv;
    double sn, cs;
    trig::sincos_ring_tab(g.k * R, o.tab_ring, &sn, &cs);   // table through L1
    const double f = (nx * dx + ny * dy + nz * dz) * inv * inv * inv * kInv4Pi, kR = g.k * R;
    kv = make_double2(f * fma(-kR, sn, -cs), f * fma(kR, cs, -sn));   // (ikR - 1) e^{ikR}
  }
  const size_t plane = (size_t)nt * g.Sp;
  const int e = erow[ti];
  unsigned short *dst = A + (size_t)ti * g.Sp + s;
  oz::split_store_n(kv.x, e, SD, dst, 2 * plane);
  oz::split_store_n(kv.y, e, SD, dst + plane, 2 * plane);
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

// Strength digits: column c = r W + w holds sigma_w(R^r s), s = j P + l -> (j, l + r P/4).
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
  const int NC = g.nrot * g.W;
  const size_t plane = (size_t)NC * g.Sp;
  unsigned short *dst = B + (size_t)c * g.Sp + s;
  oz::split_store_n(v.x, ecol[w], SD, dst, 2 * plane);
  oz::split_store_n(v.y, ecol[w], SD, dst + plane, 2 * plane);
}

// C[ti][c] = sum_s K[ti][s] B[s][c] for one block of targets; 8 warps, each a
// 16 x 16 output tile (one m16 fragment x two n8 fragments); int64 folds of
// every digit group, FP64 at the end.
template <int SD>
__global__ void __launch_bounds__(256)
near_gemm_kernel(NearGeom g, int nt, const unsigned short *__restrict__ A,
                 const unsigned short *__restrict__ B, const int *__restrict__ erow,
                 const int *__restrict__ ecol, double2 *__restrict__ C) {
  constexpr int NG = SD;                         // groups g = 2 .. SD + 1
  extern __shared__ __align__(16) unsigned char near_smem[];
  typedef __nv_bfloat16 ATile[2][kGM][kLDK];
  typedef __nv_bfloat16 BTile[2][kGN][kLDK];
  ATile *As = reinterpret_cast<ATile *>(near_smem);                       // [SD]
  BTile *Bs = reinterpret_cast<BTile *>(near_smem + sizeof(ATile) * SD);  // [SD]
  const int NC = g.nrot * g.W;
  const int m0 = blockIdx.x * kGM, n0 = blockIdx.y * kGN;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wm = warp & 3, wn = warp >> 2;       // 4 x 2 warps: rows 16 wm, columns 16 wn
  const int grp = lane >> 2, tig = lane & 3;
  const size_t aplane = (size_t)nt * g.Sp, bplane = (size_t)NC * g.Sp;

  float acc[NG][2][2][4];                        // [group][re/im][n-fragment][element]
  long long hi[2][2][4], lo[2][2][4];
#pragma unroll
  for (int q = 0; q < NG; ++q)
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
      for (int f = 0; f < 2; ++f)
#pragma unroll
        for (int e = 0; e < 4; ++e) acc[q][c][f][e] = 0.f;
#pragma unroll
  for (int c = 0; c < 2; ++c)
#pragma unroll
    for (int f = 0; f < 2; ++f)
#pragma unroll
      for (int e = 0; e < 4; ++e) hi[c][f][e] = lo[c][f][e] = 0;

  const int nchunk = g.Sp / kGK;
  for (int ch = 0; ch < nchunk; ++ch) {
    const int k0 = ch * kGK;
    __syncthreads();
    // A: SD*2*kGM rows of kGK digits (64 bytes = 4 x 16 B); B likewise with kGN rows
    for (int e = tid; e < SD * 2 * kGM * 4; e += 256) {
      const int q = e & 3, row = e >> 2;                  // row = (s*2 + part)*kGM + r
      const int sp = row / kGM, r = row % kGM;
      uint4 v = make_uint4(0, 0, 0, 0);
      if (m0 + r < nt)
        v = reinterpret_cast<const uint4 *>(A + (size_t)sp * aplane + (size_t)(m0 + r) * g.Sp + k0)[q];
      reinterpret_cast<uint4 *>(&As[0][0][0][0] + row * kLDK)[q] = v;
    }
    for (int e = tid; e < SD * 2 * kGN * 4; e += 256) {
      const int q = e & 3, row = e >> 2;
      const int sp = row / kGN, r = row % kGN;
      uint4 v = make_uint4(0, 0, 0, 0);
      if (n0 + r < NC)
        v = reinterpret_cast<const uint4 *>(B + (size_t)sp * bplane + (size_t)(n0 + r) * g.Sp + k0)[q];
      reinterpret_cast<uint4 *>(&Bs[0][0][0][0] + row * kLDK)[q] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kGK; kk += 16) {
#pragma unroll
      for (int s = 1; s <= SD; ++s) {
        uint32_t ar[4], ai[4];
        oz::load_a(&As[s - 1][0][16 * wm][kk], kLDK, lane, ar);
        oz::load_a(&As[s - 1][1][16 * wm][kk], kLDK, lane, ai);
#pragma unroll
        for (int t = 1; t <= SD + 1 - s; ++t) {
#pragma unroll
          for (int f = 0; f < 2; ++f) {
            uint32_t br[2], bi[2];
            oz::load_b(&Bs[t - 1][0][16 * wn + 8 * f][kk], kLDK, lane, br);
            oz::load_b(&Bs[t - 1][1][16 * wn + 8 * f][kk], kLDK, lane, bi);
            oz::cmma(acc[s + t - 2][0][f], acc[s + t - 2][1][f], ar, ai, br, bi);
          }
        }
      }
    }
    if ((ch + 1) % kFlushChunks == 0 || ch + 1 == nchunk) {
#pragma unroll
      for (int q = 0; q < NG; ++q)
#pragma unroll
        for (int c = 0; c < 2; ++c)
#pragma unroll
          for (int f = 0; f < 2; ++f)
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              const long long v = (long long)__float2int_rn(acc[q][c][f][e]);
              const int g2 = q + 2;
              if (g2 <= 4) hi[c][f][e] += v << (7 * (4 - g2));
              else lo[c][f][e] += v << (7 * (SD + 1 - g2));
              acc[q][c][f][e] = 0.f;
            }
    }
  }
#pragma unroll
  for (int f = 0; f < 2; ++f)
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int r = m0 + 16 * wm + grp + (e >= 2 ? 8 : 0);
      const int c = n0 + 16 * wn + 8 * f + 2 * tig + (e & 1);
      if (r < nt && c < NC) {
        const int ex = erow[r] + ecol[c % g.W];
        C[(size_t)r * NC + c] = make_double2(oz::unfold<SD>(hi[0][f][e], lo[0][f][e], ex),
                                             oz::unfold<SD>(hi[1][f][e], lo[1][f][e], ex));
      }
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
  add(sizeof(int) * W);                                  // column exponents
  add(sizeof(unsigned short) * 2 * (size_t)slices * tb * g.Sp);   // A digits
  add(sizeof(unsigned short) * 2 * (size_t)slices * NC * g.Sp);   // B digits
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
  int *ecol = reinterpret_cast<int *>(take(sizeof(int) * g.W));
  unsigned short *A = reinterpret_cast<unsigned short *>(take(sizeof(unsigned short) * 2 * (size_t)SD * tb * g.Sp));
  unsigned short *B = reinterpret_cast<unsigned short *>(take(sizeof(unsigned short) * 2 * (size_t)SD * NC * g.Sp));
  double2 *C = reinterpret_cast<double2 *>(take(sizeof(double2) * (size_t)tb * NC));
  const size_t gemm_smem = sizeof(__nv_bfloat16) * SD * 2 * (kGM + kGN) * kLDK;
  static size_t granted = 0;
  cudaError_t e = ensure_dynamic_smem(near_gemm_kernel<SD>, gemm_smem, granted);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(U, 0, sizeof(double2) * (size_t)g.W * T, st);
  if (e != cudaSuccess) return e;
  near_sigexp_kernel<<<g.W, 256, 0, st>>>(g, sigma, ecol);
  near_bdigits_kernel<SD><<<dim3((g.Sp + 255) / 256, NC), 256, 0, st>>>(g, sigma, ecol, B);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  for (int t0 = 0; t0 < T; t0 += tb) {
    const int nt = T - t0 < tb ? T - t0 : tb;
    for (int rep = 0; rep < g.nrep; ++rep) {
      near_rowexp_kernel<<<(nt + 7) / 8, 256, 0, st>>>(d_o, g, rep, t0, nt, erow);
      near_adigits_kernel<SD><<<dim3((g.Sp + 255) / 256, nt), 256, 0, st>>>(d_o, g, rep, t0, nt, erow, A);
      near_gemm_kernel<SD><<<dim3((nt + kGM - 1) / kGM, (NC + kGN - 1) / kGN), 256, gemm_smem, st>>>(
          g, nt, A, B, erow, ecol, C);
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
