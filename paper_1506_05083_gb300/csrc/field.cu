// Incident-wave boundary data and field evaluation from point strengths.
//
// Incident data (Sec. 2 eqs. ui, neu; Sec. 3.4 eq. trans) is sampled on the
// M x P ring nodes (rho_m, phi_l = 2 pi l / P, z_m) that the RHS transform
// (eq. fhatquad with q = P) consumes.
//
// Field evaluation (Sec. 4.1): each ring source of mode n is replaced by P
// point sources with strengths sigma_jl (the inverse transform of c_nj over
// n), so u(x) = sum_{j,l} G_k(x, y_jl) sigma_jl. With a lattice the sum runs
// over the eight phased nearest images, the action A_else of Sec. 4.1 done by
// direct summation instead of an FMM.
#include "axi_internal.h"
#include "trig.cuh"

namespace axi {
namespace {

constexpr int kThreads = 256;
constexpr double kInv4Pi = 0.07957747154594766788;

__global__ void incident_kernel(const ObsDev *__restrict__ od, int W, const double *__restrict__ dirs,
                                double2 *__restrict__ f) {
  const ObsDev &o = *od;
  const int P = o.P, rows = o.rows;
  const size_t total = (size_t)W * rows * P;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    const int l = (int)(e % P);
    const int row = (int)((e / P) % rows);
    const int w = (int)(e / ((size_t)P * rows));
    const int m = row % o.M;
    const double rho = o.coll[4 * m], z = o.coll[4 * m + 1];
    const double nr = o.coll[4 * m + 2], nz = o.coll[4 * m + 3];
    const double2 t = o.tw_P[l];       // (cos phi_l, -sin phi_l)
    const double c = t.x, s = -t.y;
    const double dx = dirs[3 * w], dy = dirs[3 * w + 1], dz = dirs[3 * w + 2];
    const double dxv = dx * rho * c + dy * rho * s + dz * z;     // d . x
    const double dnv = dx * nr * c + dy * nr * s + dz * nz;      // d . n
    double sn, cs;
    sincos(o.k * dxv, &sn, &cs);
    double2 v;
    const bool value_row = (o.bc == AXI_BC_TRANSMISSION) && row < o.M;
    if (value_row) {
      v = make_double2(-cs, -sn);                              // -u_i
    } else {
      const double a = o.k * dnv;                              // -du/dn = -i k (d.n) u_i
      v = make_double2(a * sn, -a * cs);
    }
    f[e] = v;
  }
}

// One CTA per (target, group of kWG waves); threads stride over the sources
// s = (j, l) of the exterior field (first N columns) and, with a lattice,
// over the eight images. Kernel values are generated once per (target,
// source, image) and reused for every wave of the group.
constexpr int kWG = 8;
__global__ void __launch_bounds__(kThreads)
eval_kernel(const ObsDev *__restrict__ od, int W, const double2 *__restrict__ sigma, int T,
            const double *__restrict__ targets, const double *__restrict__ normals, int kind,
            int use_lattice, double ex, double ey, const double *__restrict__ dirs,
            double2 *__restrict__ out) {
  const ObsDev &o = *od;
  const int t = blockIdx.x;
  const int w0 = blockIdx.y * kWG;
  const int nw = min(kWG, W - w0);
  const int P = o.P, N = o.N, cols = o.cols;
  const double k = o.k;
  const double tx = targets[3 * t], ty = targets[3 * t + 1], tz = targets[3 * t + 2];
  double nx = 0, ny = 0, nz = 0;
  if (kind == AXI_EVAL_NORMAL_DERIV) { nx = normals[3 * t]; ny = normals[3 * t + 1]; nz = normals[3 * t + 2]; }
  __shared__ double2 phase[kWG][9];
  if (threadIdx.x < kWG * 9) {
    const int w = threadIdx.x / 9, im = threadIdx.x % 9;
    const int a = im / 3 - 1, b = im % 3 - 1;
    double2 ph = make_double2(1.0, 0.0);
    if (use_lattice && w < nw) {
      const double arg = k * (dirs[3 * (w0 + w)] * a * ex + dirs[3 * (w0 + w) + 1] * b * ey);
      double sn, cs;
      sincos(arg, &sn, &cs);
      ph = make_double2(cs, sn);
    }
    phase[w][im] = ph;
  }
  __syncthreads();
  double2 acc[kWG];
#pragma unroll
  for (int w = 0; w < kWG; ++w) acc[w] = make_double2(0.0, 0.0);
  const int S = N * P;
  for (int s = threadIdx.x; s < S; s += kThreads) {
    const int j = s / P, l = s % P;
    const double2 tw = o.tw_P[l];
    const double rs = o.src[2 * j], zs = o.src[2 * j + 1];
    const double yx = rs * tw.x, yy = -rs * tw.y, yz = zs;
    double2 ksum[kWG];
#pragma unroll
    for (int w = 0; w < kWG; ++w) ksum[w] = make_double2(0.0, 0.0);
    const int nimg = use_lattice ? 9 : 1;
    for (int im = 0; im < nimg; ++im) {
      double sx = 0, sy = 0;
      if (use_lattice) {
        if (im == 4) continue;  // central copy excluded (A_else)
        sx = (im / 3 - 1) * ex;
        sy = (im % 3 - 1) * ey;
      }
      double2 kv;
      if (kind == AXI_EVAL_FAR_FIELD) {
        double sn, cs;
        sincos(-k * (tx * (yx + sx) + ty * (yy + sy) + tz * yz), &sn, &cs);
        kv = make_double2(cs * kInv4Pi, sn * kInv4Pi);
      } else {
        const double dx = tx - yx - sx, dy = ty - yy - sy, dz = tz - yz;
        const double R = sqrt(dx * dx + dy * dy + dz * dz);
        const double inv = 1.0 / R;
        double sn, cs;
        trig::sincos_ring(k * R, &sn, &cs);
        if (kind == AXI_EVAL_POTENTIAL) {
          kv = make_double2(cs * inv * kInv4Pi, sn * inv * kInv4Pi);
        } else {
          const double nd = nx * dx + ny * dy + nz * dz;
          const double f = nd * inv * inv * inv * kInv4Pi, kR = k * R;
          kv = make_double2(f * (-cs - kR * sn), f * (-sn + kR * cs));
        }
      }
      const int imi = use_lattice ? im : 4;
#pragma unroll
      for (int w = 0; w < kWG; ++w) {
        const double2 ph = phase[w][imi];
        ksum[w].x = fma(ph.x, kv.x, fma(-ph.y, kv.y, ksum[w].x));
        ksum[w].y = fma(ph.x, kv.y, fma(ph.y, kv.x, ksum[w].y));
      }
    }
#pragma unroll
    for (int w = 0; w < kWG; ++w) {
      if (w < nw) {
        const double2 sg = sigma[((size_t)(w0 + w) * cols + j) * P + l];
        acc[w].x = fma(ksum[w].x, sg.x, fma(-ksum[w].y, sg.y, acc[w].x));
        acc[w].y = fma(ksum[w].x, sg.y, fma(ksum[w].y, sg.x, acc[w].y));
      }
    }
  }
  __shared__ double red[kThreads / 32][2 * kWG];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int w = 0; w < kWG; ++w) {
    double x = acc[w].x, y = acc[w].y;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      x += __shfl_xor_sync(0xffffffffu, x, off);
      y += __shfl_xor_sync(0xffffffffu, y, off);
    }
    if (lane == 0) { red[warp][2 * w] = x; red[warp][2 * w + 1] = y; }
  }
  __syncthreads();
  if (threadIdx.x < nw) {
    double x = 0, y = 0;
    for (int i = 0; i < kThreads / 32; ++i) { x += red[i][2 * threadIdx.x]; y += red[i][2 * threadIdx.x + 1]; }
    out[(size_t)(w0 + threadIdx.x) * T + t] = make_double2(x, y);
  }
}

}  // namespace

cudaError_t launch_incident(const ObsDev *d_o, const ObsDev &h, int W, const double *dirs,
                            double2 *f, cudaStream_t st) {
  const size_t total = (size_t)W * h.rows * h.P;
  int blocks = (int)((total + kThreads - 1) / kThreads);
  if (blocks > 152 * 16) blocks = 152 * 16;
  if (blocks < 1) blocks = 1;
  incident_kernel<<<blocks, kThreads, 0, st>>>(d_o, W, dirs, f);
  return cudaGetLastError();
}

cudaError_t launch_eval(const ObsDev *d_o, const ObsDev &h, int W, const double2 *sigma, int T,
                        const double *targets, const double *normals, int kind,
                        const axi_lattice *lat, const double *dirs, double2 *out,
                        cudaStream_t st) {
  dim3 grid(T, (W + kWG - 1) / kWG);
  eval_kernel<<<grid, kThreads, 0, st>>>(d_o, W, sigma, T, targets, normals, kind, lat ? 1 : 0,
                                         lat ? lat->ex : 0.0, lat ? lat->ey : 0.0, dirs, out);
  return cudaGetLastError();
}

}  // namespace axi
