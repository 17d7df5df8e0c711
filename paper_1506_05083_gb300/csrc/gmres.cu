// Restarted GMRES (the Krylov method the paper applies to eq. iter, Sec.
// 4.2) for W independent right-hand sides of length n sharing one operator,
// by reverse communication: axi_gmres_iterate returns whenever it needs the
// operator applied to a block of W vectors, so the caller composes the
// operator from whatever entry points it needs.
//
// Per wave: Arnoldi with classical Gram-Schmidt applied twice (CGS2; the dot
// products and the updates run as device kernels over all waves at once),
// the Hessenberg column reduced by complex Givens rotations on the host
// (k <= restart scalars), the residual estimate |g_{j+1}| checked against
// tol ||b||. A wave that has converged has its next basis vector set to
// zero, so the shared operator applications leave it unchanged; its Krylov
// count for the cycle is frozen. At the end of a cycle every wave solves its
// triangular system and updates x; a restart forms the true residual
// b - A x by one more application.
#include <cmath>
#include <complex>
#include <cstring>
#include <new>
#include <vector>

#include "axi_internal.h"

namespace {

constexpr int kGT = 256;

// out[w * ldo + j] = V_j(w)^H x(w) for j < k: V_j(w) = V + (j W + w) n.
__global__ void __launch_bounds__(kGT) gm_dots_kernel(const double2 *__restrict__ V, int64_t n, int W,
                                                      const double2 *__restrict__ x,
                                                      double2 *__restrict__ out, int ldo) {
  __shared__ double red[kGT / 32][2];
  const int j = blockIdx.x, w = blockIdx.y;
  const double2 *v = V + ((int64_t)j * W + w) * n, *xx = x + (int64_t)w * n;
  double re = 0.0, im = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += kGT) {
    const double2 a = v[i], b = xx[i];
    re = fma(a.x, b.x, fma(a.y, b.y, re));
    im = fma(a.x, b.y, fma(-a.y, b.x, im));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    re += __shfl_xor_sync(0xffffffffu, re, o);
    im += __shfl_xor_sync(0xffffffffu, im, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red[threadIdx.x >> 5][0] = re;
    red[threadIdx.x >> 5][1] = im;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double sr = 0.0, si = 0.0;
    for (int q = 0; q < kGT / 32; ++q) {                 // fixed order: reproducible
      sr += red[q][0];
      si += red[q][1];
    }
    out[(int64_t)w * ldo + j] = make_double2(sr, si);
  }
}

// x(w) += sign sum_{j < k} c[w * ldc + j] V_j(w)
__global__ void gm_update_kernel(const double2 *__restrict__ V, int64_t n, int W, int k,
                                 const double2 *__restrict__ c, int ldc, double sign,
                                 double2 *__restrict__ x) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int w = blockIdx.y;
  if (i >= n) return;
  double2 acc = make_double2(0.0, 0.0);
  for (int j = 0; j < k; ++j) {
    const double2 a = V[((int64_t)j * W + w) * n + i], s = c[(int64_t)w * ldc + j];
    acc.x = fma(a.x, s.x, fma(-a.y, s.y, acc.x));
    acc.y = fma(a.x, s.y, fma(a.y, s.x, acc.y));
  }
  double2 v = x[(int64_t)w * n + i];
  v.x = fma(sign, acc.x, v.x);
  v.y = fma(sign, acc.y, v.y);
  x[(int64_t)w * n + i] = v;
}

// dst(w) = a[w] (x(w) - y(w)) (y may be null: dst = a x); dst may alias x or y.
__global__ void gm_axmy_kernel(int64_t n, const double *__restrict__ a, const double2 *x, const double2 *y,
                               double2 *dst) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int w = blockIdx.y;
  if (i >= n) return;
  const int64_t e = (int64_t)w * n + i;
  double2 v = x[e];
  if (y) {
    const double2 u = y[e];
    v.x -= u.x;
    v.y -= u.y;
  }
  dst[e] = make_double2(a[w] * v.x, a[w] * v.y);
}

__global__ void gm_scale_kernel(int64_t count, double alpha, double2 *x) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) x[i] = make_double2(alpha * x[i].x, alpha * x[i].y);
}

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

}  // namespace

using cplx = std::complex<double>;

struct axi_gmres {
  int64_t n;
  int W, m, max_iter;
  double tol;
  // device: basis V [(m+1)][W][n], w [W][n], coefficients [W][m+1] x 2, scalars [W]
  double2 *V, *w, *c1, *c2;
  double *a;
  int state;                 // 0 start, 1 after an Arnoldi apply, 2 after a restart apply, 3 done
  bool nonfinite;            // a residual estimate was not finite
  int j;                     // Arnoldi step of the cycle
  std::vector<cplx> H;       // [W][(m+1) m], column-major per wave
  std::vector<double> cs;    // [W][m]
  std::vector<cplx> sn;      // [W][m]
  std::vector<cplx> g;       // [W][m+1]
  std::vector<double> bnorm, relres;
  std::vector<int> iters, kcyc;
  std::vector<char> conv, live;   // converged for good; still stepping in this cycle
  cudaStream_t st;
};

namespace {

cplx &Hat(axi_gmres *s, int w, int r, int c) { return s->H[(size_t)w * (s->m + 1) * s->m + (size_t)c * (s->m + 1) + r]; }

axi_status cuda_ok(cudaError_t e) { return e == cudaSuccess ? AXI_OK : AXI_ERR_CUDA; }

// c1[w][0..k) = V_{0..k}(w)^H x(w), read back to host h[w][k]
cudaError_t dots(axi_gmres *s, const double2 *V, int k, const double2 *x, double2 *dev_out, std::vector<double2> &h) {
  gm_dots_kernel<<<dim3((unsigned)k, (unsigned)s->W), kGT, 0, s->st>>>(V, s->n, s->W, x, dev_out, s->m + 1);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  h.resize((size_t)s->W * (s->m + 1));
  e = cudaMemcpyAsync(h.data(), dev_out, sizeof(double2) * h.size(), cudaMemcpyDeviceToHost, s->st);
  if (e != cudaSuccess) return e;
  return cudaStreamSynchronize(s->st);
}

dim3 vec_grid(const axi_gmres *s) { return dim3((unsigned)((s->n + 255) / 256), (unsigned)s->W); }

// dst(w) = a_w (x(w) - y(w)) with host scalars a_w
cudaError_t axmy(axi_gmres *s, const std::vector<double> &aw, const double2 *x, const double2 *y, double2 *dst) {
  cudaError_t e = cudaMemcpyAsync(s->a, aw.data(), sizeof(double) * s->W, cudaMemcpyHostToDevice, s->st);
  if (e != cudaSuccess) return e;
  gm_axmy_kernel<<<vec_grid(s), 256, 0, s->st>>>(s->n, s->a, x, y, dst);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return cudaStreamSynchronize(s->st);   // aw is the caller's: keep it alive until the copy is done
}

// Start a cycle from r (in V_0, already formed unscaled): beta = ||r||.
cudaError_t start_cycle(axi_gmres *s) {
  std::vector<double2> h;
  cudaError_t e = dots(s, s->V, 1, s->V, s->c1, h);
  if (e != cudaSuccess) return e;
  std::vector<double> aw((size_t)s->W, 0.0);
  for (int w = 0; w < s->W; ++w) {
    const double beta = std::sqrt(std::fmax(h[(size_t)w * (s->m + 1)].x, 0.0));
    s->kcyc[w] = 0;
    std::fill(s->g.begin() + (size_t)w * (s->m + 1), s->g.begin() + (size_t)(w + 1) * (s->m + 1), cplx(0.0));
    s->g[(size_t)w * (s->m + 1)] = beta;
    if (!s->conv[w]) {
      s->relres[w] = s->bnorm[w] > 0.0 ? beta / s->bnorm[w] : 0.0;
      if (beta <= s->tol * s->bnorm[w] || beta == 0.0) s->conv[w] = 1;
    }
    s->live[w] = !s->conv[w] && s->iters[w] < s->max_iter;
    aw[w] = s->live[w] ? 1.0 / beta : 0.0;
  }
  s->j = 0;
  return axmy(s, aw, s->V, nullptr, s->V);
}

// End of a cycle: y_w = H_w^{-1} g_w over its kcyc steps, x += V y.
cudaError_t end_cycle(axi_gmres *s, double2 *x) {
  const int m1 = s->m + 1;
  std::vector<double2> y((size_t)s->W * m1, make_double2(0.0, 0.0));
  int kmax = 0;
  for (int w = 0; w < s->W; ++w) {
    const int k = s->kcyc[w];
    kmax = std::max(kmax, k);
    std::vector<cplx> yy((size_t)k);
    for (int r = k - 1; r >= 0; --r) {
      cplx acc = s->g[(size_t)w * m1 + r];
      for (int c = r + 1; c < k; ++c) acc -= Hat(s, w, r, c) * yy[c];
      const cplx d = Hat(s, w, r, r);
      yy[r] = d != cplx(0.0) ? acc / d : cplx(0.0);
    }
    for (int r = 0; r < k; ++r) y[(size_t)w * m1 + r] = make_double2(yy[r].real(), yy[r].imag());
  }
  if (kmax == 0) return cudaSuccess;
  cudaError_t e = cudaMemcpyAsync(s->c2, y.data(), sizeof(double2) * y.size(), cudaMemcpyHostToDevice, s->st);
  if (e != cudaSuccess) return e;
  gm_update_kernel<<<vec_grid(s), 256, 0, s->st>>>(s->V, s->n, s->W, kmax, s->c2, m1, 1.0, x);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return cudaStreamSynchronize(s->st);
}

// After w = A V_j: CGS2 against V_0..V_j, the new column of H, its Givens
// rotation and the residual estimate; V_{j+1} = w / h_{j+1,j} for live waves.
cudaError_t arnoldi_step(axi_gmres *s) {
  const int m1 = s->m + 1, k = s->j + 1;
  std::vector<double2> h1, h2, nr;
  cudaError_t e = dots(s, s->V, k, s->w, s->c1, h1);
  if (e != cudaSuccess) return e;
  gm_update_kernel<<<vec_grid(s), 256, 0, s->st>>>(s->V, s->n, s->W, k, s->c1, m1, -1.0, s->w);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = dots(s, s->V, k, s->w, s->c2, h2)) != cudaSuccess) return e;
  gm_update_kernel<<<vec_grid(s), 256, 0, s->st>>>(s->V, s->n, s->W, k, s->c2, m1, -1.0, s->w);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  // ||w||^2 through the dots kernel with w itself as the one basis vector
  gm_dots_kernel<<<dim3(1, (unsigned)s->W), kGT, 0, s->st>>>(s->w, s->n, s->W, s->w, s->c1, m1);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  nr.resize((size_t)s->W * m1);
  if ((e = cudaMemcpyAsync(nr.data(), s->c1, sizeof(double2) * nr.size(), cudaMemcpyDeviceToHost, s->st)) !=
      cudaSuccess)
    return e;
  if ((e = cudaStreamSynchronize(s->st)) != cudaSuccess) return e;
  std::vector<double> aw((size_t)s->W, 0.0);
  const int j = s->j;
  for (int w = 0; w < s->W; ++w) {
    if (!s->live[w]) continue;
    for (int r = 0; r < k; ++r) {
      const double2 a = h1[(size_t)w * m1 + r], b = h2[(size_t)w * m1 + r];
      Hat(s, w, r, j) = cplx(a.x + b.x, a.y + b.y);
    }
    const double hn = std::sqrt(std::fmax(nr[(size_t)w * m1].x, 0.0));
    Hat(s, w, j + 1, j) = hn;
    for (int r = 0; r < j; ++r) {                        // earlier rotations
      const double c = s->cs[(size_t)w * s->m + r];
      const cplx sn = s->sn[(size_t)w * s->m + r];
      const cplx a = Hat(s, w, r, j), b = Hat(s, w, r + 1, j);
      Hat(s, w, r, j) = c * a + sn * b;
      Hat(s, w, r + 1, j) = -std::conj(sn) * a + c * b;
    }
    const cplx a = Hat(s, w, j, j), b = Hat(s, w, j + 1, j);
    const double aa = std::abs(a), t = std::hypot(aa, std::abs(b));
    double c;
    cplx sn;
    if (t == 0.0) {
      c = 1.0;
      sn = 0.0;
    } else if (aa == 0.0) {
      c = 0.0;
      sn = std::conj(b) / t;
    } else {
      c = aa / t;
      sn = (a / aa) * std::conj(b) / t;
    }
    s->cs[(size_t)w * s->m + j] = c;
    s->sn[(size_t)w * s->m + j] = sn;
    Hat(s, w, j, j) = c * a + sn * b;
    Hat(s, w, j + 1, j) = 0.0;
    cplx &gj = s->g[(size_t)w * m1 + j];
    s->g[(size_t)w * m1 + j + 1] = -std::conj(sn) * gj;
    gj = c * gj;
    s->kcyc[w] = j + 1;
    s->iters[w] += 1;
    const double res = std::abs(s->g[(size_t)w * m1 + j + 1]);
    s->relres[w] = s->bnorm[w] > 0.0 ? res / s->bnorm[w] : 0.0;
    if (!std::isfinite(res)) {
      s->nonfinite = true;
      s->live[w] = 0;
      continue;
    }
    if (res <= s->tol * s->bnorm[w] || hn == 0.0) {
      s->conv[w] = 1;
      s->live[w] = 0;
    } else if (s->iters[w] >= s->max_iter) {
      s->live[w] = 0;
    }
    aw[w] = s->live[w] ? 1.0 / hn : 0.0;
  }
  return axmy(s, aw, s->w, nullptr, s->V + (size_t)(j + 1) * s->W * s->n);
}

}  // namespace

extern "C" axi_status axi_gmres_workspace_bytes(int64_t n, int32_t W, int32_t restart, size_t *bytes) {
  if (!bytes || n < 1 || W < 1 || W > 65535 || restart < 1 || restart > 512) return AXI_ERR_ARG;
  const size_t vec = sizeof(double2) * (size_t)n * W;
  *bytes = align256(vec * (restart + 1)) + align256(vec) +
           2 * align256(sizeof(double2) * (size_t)W * (restart + 1)) + align256(sizeof(double) * W);
  return AXI_OK;
}

extern "C" axi_status axi_gmres_create(int64_t n, int32_t W, int32_t restart, int32_t max_iter, double tol,
                                       void *d_work, size_t work_bytes, axi_gmres **out) {
  size_t need = 0;
  if (!out || max_iter < 1 || !(tol >= 0.0)) return AXI_ERR_ARG;
  axi_status s = axi_gmres_workspace_bytes(n, W, restart, &need);
  if (s != AXI_OK) return s;
  if (!d_work || work_bytes < need || (reinterpret_cast<uintptr_t>(d_work) & 255)) return AXI_ERR_WORKSPACE;
  // host state: no exception may leave this C entry point
  axi_gmres *g = new (std::nothrow) axi_gmres();
  if (!g) return AXI_ERR_WORKSPACE;
  try {
    g->n = n;
    g->W = W;
    g->m = restart;
    g->max_iter = max_iter;
    g->tol = tol;
    const size_t vec = sizeof(double2) * (size_t)n * W;
    char *p = static_cast<char *>(d_work);
    g->V = reinterpret_cast<double2 *>(p);
    p += align256(vec * (restart + 1));
    g->w = reinterpret_cast<double2 *>(p);
    p += align256(vec);
    g->c1 = reinterpret_cast<double2 *>(p);
    p += align256(sizeof(double2) * (size_t)W * (restart + 1));
    g->c2 = reinterpret_cast<double2 *>(p);
    p += align256(sizeof(double2) * (size_t)W * (restart + 1));
    g->a = reinterpret_cast<double *>(p);
    g->state = 0;
    g->nonfinite = false;
    g->j = 0;
    g->H.assign((size_t)W * (restart + 1) * restart, cplx(0.0));
    g->cs.assign((size_t)W * restart, 0.0);
    g->sn.assign((size_t)W * restart, cplx(0.0));
    g->g.assign((size_t)W * (restart + 1), cplx(0.0));
    g->bnorm.assign(W, 0.0);
    g->relres.assign(W, 1.0);
    g->iters.assign(W, 0);
    g->kcyc.assign(W, 0);
    g->conv.assign(W, 0);
    g->live.assign(W, 0);
    g->st = nullptr;
  } catch (const std::bad_alloc &) {
    delete g;
    return AXI_ERR_WORKSPACE;
  }
  *out = g;
  return AXI_OK;
}

extern "C" axi_status axi_gmres_destroy(axi_gmres *g) {
  delete g;
  return AXI_OK;
}

extern "C" axi_status axi_gmres_iterate(axi_gmres *g, const axi_c128 *d_b, axi_c128 *d_x, int32_t *need_apply,
                                        const axi_c128 **d_in, axi_c128 **d_out, void *stream) {
  if (!g || !d_b || !d_x || !need_apply || !d_in || !d_out || !aligned16(d_b) || !aligned16(d_x))
    return AXI_ERR_ARG;
  g->st = static_cast<cudaStream_t>(stream);
  const double2 *b = reinterpret_cast<const double2 *>(d_b);
  double2 *x = reinterpret_cast<double2 *>(d_x);
  cudaError_t e = cudaSuccess;
  *need_apply = 0;
  auto request = [&](const double2 *in) {
    *d_in = reinterpret_cast<const axi_c128 *>(in);
    *d_out = reinterpret_cast<axi_c128 *>(g->w);
    *need_apply = 1;
  };
  auto all_stopped = [&]() {
    for (int w = 0; w < g->W; ++w)
      if (g->live[w]) return false;
    return true;
  };
  auto finished = [&]() {
    for (int w = 0; w < g->W; ++w)
      if (!g->conv[w] && g->iters[w] < g->max_iter) return false;
    return true;
  };
  try {
    switch (g->state) {
      case 0: {  // x = 0, r = b
        const std::vector<double> zero((size_t)g->W, 0.0), one((size_t)g->W, 1.0);
        if ((e = axmy(g, zero, b, nullptr, x)) != cudaSuccess) break;
        if ((e = axmy(g, one, b, nullptr, g->V)) != cudaSuccess) break;
        std::vector<double2> h;
        if ((e = dots(g, g->V, 1, g->V, g->c1, h)) != cudaSuccess) break;
        for (int w = 0; w < g->W; ++w) g->bnorm[w] = std::sqrt(std::fmax(h[(size_t)w * (g->m + 1)].x, 0.0));
        if ((e = start_cycle(g)) != cudaSuccess) break;
        if (all_stopped()) {
          g->state = 3;
          break;
        }
        g->state = 1;
        request(g->V);
        break;
      }
      case 1: {  // w = A V_j
        if ((e = arnoldi_step(g)) != cudaSuccess) break;
        g->j += 1;
        if (!all_stopped() && g->j < g->m) {
          request(g->V + (size_t)g->j * g->W * g->n);
          break;
        }
        if ((e = end_cycle(g, x)) != cudaSuccess) break;
        if (finished()) {
          g->state = 3;
          break;
        }
        g->state = 2;
        request(x);
        break;
      }
      case 2: {  // w = A x: V_0 = b - w, a new cycle
        const std::vector<double> one((size_t)g->W, 1.0);
        if ((e = axmy(g, one, b, g->w, g->V)) != cudaSuccess) break;
        if ((e = start_cycle(g)) != cudaSuccess) break;
        if (all_stopped()) {
          g->state = 3;
          break;
        }
        g->state = 1;
        request(g->V);
        break;
      }
      default:
        break;
    }
  } catch (const std::bad_alloc &) {
    g->state = 3;
    *need_apply = 0;
    return AXI_ERR_WORKSPACE;
  }
  if (e != cudaSuccess) return AXI_ERR_CUDA;
  if (g->nonfinite) {
    g->state = 3;
    *need_apply = 0;
    return AXI_ERR_NUMERIC;
  }
  return AXI_OK;
}

extern "C" axi_status axi_gmres_result(const axi_gmres *g, int32_t *h_iters, double *h_relres,
                                       int32_t *h_converged) {
  if (!g) return AXI_ERR_ARG;
  for (int w = 0; w < g->W; ++w) {
    if (h_iters) h_iters[w] = g->iters[w];
    if (h_relres) h_relres[w] = g->relres[w];
    if (h_converged) h_converged[w] = g->conv[w];
  }
  return AXI_OK;
}

extern "C" axi_status axi_vec_scale(int64_t count, double alpha, axi_c128 *d_x, void *stream) {
  if (!d_x || count < 0 || !aligned16(d_x)) return AXI_ERR_ARG;
  if (count == 0) return AXI_OK;
  gm_scale_kernel<<<(unsigned)((count + 255) / 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(
      count, alpha, reinterpret_cast<double2 *>(d_x));
  return cuda_ok(cudaGetLastError());
}
