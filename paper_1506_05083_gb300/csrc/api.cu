// C-ABI entry points: validation, workspace layout, launch sequencing.
// The device work is in fill.cu (A2), qr.cu (A3, A4-A6) and field.cu.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <cstdio>
#include <cstdlib>
#include <new>
#include <string>
#include <vector>

#include "axi_internal.h"
#include "trig.cuh"

using axi::ObsDev;

namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr size_t kAlign = 256;

size_t align_up(size_t x) { return (x + kAlign - 1) & ~(kAlign - 1); }

struct ObsHost {
  ObsDev dev;  // device pointers are filled at build time from the offsets below
  std::vector<double> coll, src, srcx, tab_cos, tab_s2;
  std::vector<double2> tw_P;
  std::vector<int> fft_perm, fft_perm_q;
  std::vector<double2> tw_q;
  size_t off_coll, off_src, off_srcx, off_cos, off_s2, off_tw, off_A, off_tau, off_T;
  size_t off_ring = 0;
  std::vector<double2> tab_ring;
  size_t off_svdU = 0, off_svdV = 0, off_svdS = 0, off_svdSw = 0;
  size_t off_ybuf = 0, off_ykey = 0, off_ydig = 0, off_yexp = 0;
  size_t off_vdig = 0, off_vexp = 0, off_ckey = 0, off_rdig = 0, off_rex = 0, off_perm = 0, off_perm_q = 0, off_tw_q = 0;
  std::vector<unsigned short> fill_cdig;   // split fill: cos-table digits [S][2 MR][Lp]
  std::vector<int> fill_cex;               // and row exponents [2 MR]
  size_t off_fcdig = 0, off_fcex = 0;
  std::vector<unsigned char> fill_sig;     // [2][M][N] sub-grid stride per ring pair
  size_t off_fsig = 0;
  std::vector<unsigned char> owned;        // [D] modes this process factors (axi_plan_shard)
  size_t off_owned = 0;
};

// Digits of the folded cosine table of the split fill (fill_mma.cu): row
// r < 2 MR holds mode n = 2 (r mod MR) + r / MR, entries w_l cos(2 pi n l / q)
// for l < L (w_0 = 1, else 2), zero elsewhere; balanced base-128 digits of
// round(x 2^{7S - e}) with e the row's exponent (|x| < 2^e).
void fill_cos_digits(ObsHost &h, int S) {
  const ObsDev &d = h.dev;
  const int q = d.q, rows = 2 * d.fill_MR, Lp = d.fill_Lp, L = d.fill_L;
  h.fill_cdig.assign((size_t)S * rows * Lp, 0);
  h.fill_cex.assign(rows, 0);
  std::vector<double> v(L);
  for (int r = 0; r < rows; ++r) {
    const int n = 2 * (r % d.fill_MR) + r / d.fill_MR;
    if (n >= d.D) continue;
    double mx = 0.0;
    for (int l = 0; l < L; ++l) {
      v[l] = (l == 0 ? 1.0 : 2.0) * h.tab_cos[(size_t)n * l % q];
      if ((n & 1) && 2 * l == q / 2) v[l] = 0.0;          // cos(pi n / 2) = 0 for odd n
      mx = std::max(mx, std::fabs(v[l]));
    }
    if (mx == 0.0) continue;
    const int e = std::ilogb(mx) + 1;
    h.fill_cex[r] = e;
    for (int l = 0; l < L; ++l) {
      long long m = std::llround(std::ldexp(v[l], 7 * S - e));
      for (int s = S; s >= 1; --s) {
        int dg;
        if (s > 1) {
          dg = (int)(m & 127);
          if (dg >= 64) dg -= 128;
          m = (m - dg) / 128;
        } else {
          dg = (int)m;
        }
        const float f = (float)dg;
        uint32_t b;
        std::memcpy(&b, &f, sizeof(b));
        h.fill_cdig[((size_t)(s - 1) * rows + r) * Lp + l] = (unsigned short)(b >> 16);
      }
    }
  }
  if (!d.fill_tc) return;
  // tcgen05 layout: per (parity, 16-row chunk of the contraction, digit) one
  // K-major no-swizzle tile of MR rows x 16 k (core matrices of 8 rows x 8 k,
  // 128 bytes apart along k, 256 bytes apart along rows), so that one bulk
  // copy brings a chunk's tiles of all digits
  const int MR = d.fill_MR, nch = Lp / 16;
  std::vector<unsigned short> tcl(h.fill_cdig.size(), 0);
  for (int part = 0; part < 2; ++part)
    for (int ch = 0; ch < nch; ++ch)
      for (int s = 0; s < S; ++s)
        for (int r = 0; r < MR; ++r)
          for (int kk = 0; kk < 16; ++kk) {
            const size_t tile = ((size_t)(part * nch + ch) * S + s) * MR * 16;
            const size_t in = (size_t)(r / 8) * 128 + (kk / 8) * 64 + (r % 8) * 8 + (kk % 8);
            tcl[tile + in] = h.fill_cdig[((size_t)s * rows + part * MR + r) * Lp + ch * 16 + kk];
          }
  h.fill_cdig.swap(tcl);
}

// Sub-grid strides of the fill (axi_fill_subgrid per proxy set); `full`
// gives stride 1 everywhere.
axi_status fill_strides(ObsHost &h, int M, int N, int P, int q, bool transmission, bool full) {
  h.fill_sig.assign((size_t)2 * M * N, 1);
  if (full) return AXI_OK;
  axi_status s = axi_fill_subgrid(M, N, P, q, h.coll.data(), h.src.data(), h.fill_sig.data());
  if (s == AXI_OK && transmission)
    s = axi_fill_subgrid(M, N, P, q, h.coll.data(), h.srcx.data(), h.fill_sig.data() + (size_t)M * N);
  return s;
}

}  // namespace

struct axi_plan_s {
  std::vector<ObsHost> obs;
  int prec = 0;
  axi::Tuning tune;                       // schedule choices (axi_plan_set_tuning / autotune)
  size_t off_fgdig = 0, off_fgex = 0;     // split fill: sample-digit scratch (shared)
  std::vector<int> task_obs, task_mode;   // sorted by obstacle panel count, descending
  std::vector<int> all_task_obs, all_task_mode;   // every task, before axi_plan_shard
  std::vector<int> step_tasks;            // tasks active at panel step p (a prefix)
  std::vector<int> step_cols;             // widest trailing matrix at step p
  std::vector<int> step_rows;             // tallest panel at step p
  // algorithmic FP64-equivalent flops of step p's panel, next-panel update and
  // trailing update over all active tasks (for the kernel profile)
  std::vector<double> step_fl_panel, step_fl_next, step_fl_rest;
  size_t off_obsdev = 0, off_task_obs = 0, off_task_mode = 0, off_status = 0;
  size_t bytes = 0;
};

// Event pairs around launch classes (axi_operator_profile).
struct OpProfiler final : axi::KernelProfiler {
  struct Rec { int kind; cudaEvent_t a, b; double flops; };
  std::vector<Rec> recs;
  std::vector<cudaEvent_t> pool;
  size_t used = 0;
  cudaEvent_t take() {
    if (used == pool.size()) {
      cudaEvent_t e = nullptr;
      if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
      pool.push_back(e);
    }
    return pool[used++];
  }
  int begin(int kind, cudaStream_t st) override {
    Rec r{kind, take(), take(), 0.0};
    if (!r.a || !r.b || cudaEventRecord(r.a, st) != cudaSuccess) return -1;
    recs.push_back(r);
    return (int)recs.size() - 1;
  }
  void end(int id, cudaStream_t st, double flops) override {
    recs[id].flops = flops;
    if (cudaEventRecord(recs[id].b, st) != cudaSuccess) recs[id].kind = -1;
  }
  void clear() { recs.clear(); used = 0; }
  ~OpProfiler() override {
    for (cudaEvent_t e : pool) cudaEventDestroy(e);
  }
};

namespace axi {
thread_local KernelProfiler *t_prof = nullptr;
}

// Points axi::t_prof at a profiled operator's recorder for one entry point.
struct ProfScope {
  explicit ProfScope(OpProfiler *p) { axi::t_prof = p; }
  ~ProfScope() { axi::t_prof = nullptr; }
};

struct axi_operator_s {
  axi_plan_s *plan;
  OpProfiler *rec = nullptr;   // launch record of the last profile (owned)
  bool profiling = false;       // recording into `rec` (axi_operator_profile)
  OpProfiler *prof() const { return profiling ? rec : nullptr; }
  int device = -1;          // CUDA device the operator was built on (its workspace lives there)
  char *ws;
  ObsDev *d_obs;
  int *d_task_obs, *d_task_mode, *d_status;
  // look-ahead: the bulk of each trailing update runs on `side` while the
  // next panel runs on `crit` (highest stream priority, so its CTAs are
  // dispatched ahead of queued trailing-update CTAs) or on the caller's
  // stream; fork/join through the events
  cudaStream_t side = nullptr, crit = nullptr;
  cudaEvent_t ev_panel = nullptr, ev_rest = nullptr, ev_fork = nullptr, ev_join = nullptr;
};

namespace {

axi_status cuda_status(cudaError_t e) { return e == cudaSuccess ? AXI_OK : AXI_ERR_CUDA; }

}  // namespace

int axi::operator_device(const axi_operator *op) { return op ? op->device : -1; }
int *axi::operator_status_word(const axi_operator *op) { return op ? op->d_status : nullptr; }

namespace {

// Mixed-radix plan of length n: radices (4s first, then 2, 3, 5) and the
// position of output k after the in-place decimation-in-frequency FFT,
//   pos(k) = (k mod r1) (n / r1) + pos'(k div r1).
// Returns the number of stages, 0 if n has other prime factors.
// Radices of n (4s, then 2, 3, 5) and the output positions of the in-place
// DIF FFT. With `needed` > 0 (only outputs n < needed are read), the largest
// radix r with n / r >= needed is moved to the last stage and *sum_last is
// set: every needed output is then output 0 of a last-stage block, i.e. the
// plain sum of the block's r entries, and that stage need not run.
int fft_plan(int n, int *rad_out, std::vector<int> &perm, int needed = 0,
             int *sum_last = nullptr) {
  std::vector<int> rad;
  int m = n;
  while (m % 4 == 0) { rad.push_back(4); m /= 4; }
  while (m % 2 == 0) { rad.push_back(2); m /= 2; }
  while (m % 3 == 0) { rad.push_back(3); m /= 3; }
  while (m % 5 == 0) { rad.push_back(5); m /= 5; }
  perm.assign(n, 0);
  if (sum_last) *sum_last = 0;
  if (m != 1 || rad.size() > 8) return 0;
  if (sum_last && needed > 0 && rad.size() > 1) {
    int best = -1;
    for (size_t s = 0; s < rad.size(); ++s)
      if (n / rad[s] >= needed && (best < 0 || rad[s] > rad[best])) best = (int)s;
    if (best >= 0) {
      const int r = rad[best];
      rad.erase(rad.begin() + best);
      rad.push_back(r);
      *sum_last = 1;
    }
  }
  for (size_t s = 0; s < rad.size(); ++s) rad_out[s] = rad[s];
  std::vector<int> cur(1, 0);
  int len = 1;
  for (int s = (int)rad.size() - 1; s >= 0; --s) {
    const int r = rad[s];
    std::vector<int> nxt(len * r);
    for (int k = 0; k < len * r; ++k) nxt[k] = (k % r) * len + cur[k / r];
    cur.swap(nxt);
    len *= r;
  }
  perm = cur;
  return (int)rad.size();
}

axi_status validate(const axi_obstacle &o) {
  if (!o.h_coll || !o.h_src) return AXI_ERR_ARG;
  if (o.bc != AXI_BC_NEUMANN && o.bc != AXI_BC_TRANSMISSION) return AXI_ERR_ARG;
  if (o.bc == AXI_BC_TRANSMISSION && !o.h_src_ext) return AXI_ERR_ARG;
  if (o.M < 1 || o.N < 1 || o.M < o.N) return AXI_ERR_SHAPE;
  if (o.P < 2 || (o.P & 1) || o.P > axi::kMaxP) return AXI_ERR_SHAPE;
  if (o.q < o.P || (o.q & 1)) return AXI_ERR_SHAPE;
  if (!(o.k > 0) || !std::isfinite(o.k)) return AXI_ERR_ARG;
  if (o.bc == AXI_BC_TRANSMISSION && (!(o.k_minus > 0) || !std::isfinite(o.k_minus)))
    return AXI_ERR_ARG;
  for (int m = 0; m < o.M; ++m)
    for (int i = 0; i < 4; ++i)
      if (!std::isfinite(o.h_coll[4 * m + i])) return AXI_ERR_GEOMETRY;
  for (int s = 0; s < (o.bc == AXI_BC_TRANSMISSION ? 2 : 1); ++s) {
    const double *S = s ? o.h_src_ext : o.h_src;
    for (int j = 0; j < o.N; ++j) {
      if (!(S[2 * j] > 0) || !std::isfinite(S[2 * j + 1])) return AXI_ERR_GEOMETRY;
      for (int m = 0; m < o.M; ++m) {
        const double dr = o.h_coll[4 * m] - S[2 * j], dz = o.h_coll[4 * m + 1] - S[2 * j + 1];
        if (dr * dr + dz * dz == 0.0) return AXI_ERR_GEOMETRY;  // target on a source ring
      }
    }
  }
  return AXI_OK;
}

// Tuning as a flat JSON object of integers, e.g.
// {"next_update": 2, "panel_cluster": 1, "rest_grid": 0}; unknown keys are
// ignored, missing keys keep their value.
bool parse_tuning(const char *js, axi::Tuning &t) {
  if (!js) return false;
  const char *c = js;
  while (*c && *c != '{') ++c;
  if (*c != '{') return false;
  ++c;
  while (true) {
    while (*c == ' ' || *c == '\n' || *c == '\t' || *c == '\r' || *c == ',') ++c;
    if (*c == '}') return true;
    if (*c != '"') return false;
    const char *k0 = ++c;
    while (*c && *c != '"') ++c;
    if (*c != '"') return false;
    const std::string key(k0, c - k0);
    ++c;
    while (*c == ' ') ++c;
    if (*c != ':') return false;
    ++c;
    char *end = nullptr;
    const double v = std::strtod(c, &end);
    if (end == c) return false;
    c = end;
    const int iv = (int)v;
    if (key == "next_update") {
      if (iv < 0 || iv > 2) return false;
      t.next_update = iv;
    } else if (key == "panel_cluster") {
      if (iv != 0 && iv != 1 && iv != 2 && iv != 4) return false;
      t.panel_cluster = iv;
    } else if (key == "rest_grid") {
      if (iv < 0 || iv > 4) return false;
      t.rest_grid = iv;
    } else if (key == "fill_chunk_mb") {
      if (iv < 0 || iv > 4096) return false;
      t.fill_chunk_mb = iv;
    } else if (key == "next_cluster") {
      if (iv != 0 && iv != 1 && iv != 2 && iv != 4) return false;
      t.next_cluster = iv;
    } else if (key == "apply_cluster") {
      if (iv != 0 && iv != 2 && iv != 4) return false;
      t.apply_cluster = iv;
    } else if (key == "crit_stream") {
      if (iv < 0 || iv > 1) return false;
      t.crit_stream = iv;
    } else if (key == "panel_fixed") {
      if (iv < 0 || iv > 2) return false;
      t.panel_fixed = iv;
    } else if (key == "rest_start") {
      if (iv < 0 || iv > 1) return false;
      t.rest_start = iv;
    } else if (key == "panel_threads") {
      if (iv != 0 && iv != 128 && iv != 256) return false;
      t.panel_threads = iv;
    }
  }
}

std::string tuning_json(const axi::Tuning &t) {
  char buf[320];
  std::snprintf(buf, sizeof(buf),
                "{\"next_update\": %d, \"panel_cluster\": %d, \"rest_grid\": %d, \"panel_threads\": %d, "
                "\"crit_stream\": %d, \"fill_chunk_mb\": %d, \"next_cluster\": %d, "
                "\"panel_fixed\": %d, \"rest_start\": %d, \"apply_cluster\": %d}",
                t.next_update, t.panel_cluster, t.rest_grid, t.panel_threads, t.crit_stream,
                t.fill_chunk_mb, t.next_cluster, t.panel_fixed, t.rest_start, t.apply_cluster);
  return buf;
}

axi_status copy_out(const std::string &js, char *buf, size_t n) {
  if (!buf || n < js.size() + 1) return AXI_ERR_ARG;
  std::memcpy(buf, js.c_str(), js.size() + 1);
  return AXI_OK;
}

// Per panel step of the current task list (sorted by panel count, so the
// tasks active at step s form a prefix): active tasks, widest trailing
// matrix, tallest panel, and the algorithmic flops of the step's panels and
// updates (for the kernel profile).
void step_tables(axi_plan_s *p) {
  int maxpan = 0;
  for (size_t t = 0; t < p->task_obs.size(); ++t)
    maxpan = std::max(maxpan, p->obs[p->task_obs[t]].dev.npanels);
  p->step_tasks.assign(maxpan, 0);
  p->step_cols.assign(maxpan, 0);
  p->step_rows.assign(maxpan, 0);
  p->step_fl_panel.assign(maxpan, 0.0);
  p->step_fl_next.assign(maxpan, 0.0);
  p->step_fl_rest.assign(maxpan, 0.0);
  for (int s = 0; s < maxpan; ++s) {
    for (int t = 0; t < (int)p->task_obs.size(); ++t) {
      const ObsDev &d = p->obs[p->task_obs[t]].dev;
      if (d.npanels > s) {
        p->step_tasks[s] = t + 1;
        const int k0 = s * axi::kNB, nbp = std::min(axi::kNB, d.cols - k0);
        p->step_cols[s] = std::max(p->step_cols[s], d.cols - k0 - nbp);
        p->step_rows[s] = std::max(p->step_rows[s], d.rows - k0);
        // reflector j (height K - j) costs 16 (K - j) flops per column it updates
        const double K = d.rows - k0;
        double pan = 0.0, hsum = 0.0;
        for (int j = 0; j < nbp; ++j) {
          pan += 16.0 * (K - j) * (nbp - 1 - j);
          hsum += 16.0 * (K - j);
        }
        const int rest = d.cols - k0 - nbp;
        const int nnext = std::min(axi::kNB, std::max(rest, 0));
        p->step_fl_panel[s] += pan;
        p->step_fl_next[s] += hsum * nnext;
        p->step_fl_rest[s] += hsum * std::max(rest - nnext, 0);
      }
    }
  }
}

}  // namespace

extern "C" {

const char *axi_status_string(int32_t s) {
  switch (s) {
    case AXI_OK: return "ok";
    case AXI_ERR_ARG: return "invalid argument";
    case AXI_ERR_SHAPE: return "invalid sizes";
    case AXI_ERR_GEOMETRY: return "invalid geometry";
    case AXI_ERR_WORKSPACE: return "workspace too small or misaligned";
    case AXI_ERR_CUDA: return "CUDA runtime error";
    case AXI_ERR_TIMEOUT: return "device wait timed out";
    case AXI_ERR_NUMERIC: return "non-finite value on the device";
    case AXI_ERR_UNSUPPORTED: return "unsupported option";
    default: return "unknown status";
  }
}

axi_status axi_plan_create(const axi_obstacle *obs, int32_t n_obs, int32_t prec, axi_plan **out) {
  if (!obs || !out || n_obs < 1) return AXI_ERR_ARG;
  const bool full_grid = (prec & axi::kPlanFullFillGrid) != 0;
  const bool tsvd = (prec & axi::kPlanTsvd) != 0;
  prec &= ~(axi::kPlanFullFillGrid | axi::kPlanTsvd);
  const int mode = prec & 0xff;
  int slices = 0;
  if (mode == AXI_PREC_SPLIT_BF16) {
    slices = (prec >> 8) & 0xff;
    if (slices == 0) slices = 7;
    if (!axi::split_slices_supported(slices)) return AXI_ERR_UNSUPPORTED;
  } else if (prec != AXI_PREC_FP64) {
    return AXI_ERR_ARG;
  }
  for (int i = 0; i < n_obs; ++i) {
    axi_status s = validate(obs[i]);
    if (s != AXI_OK) return s;
  }
  axi_plan_s *p = new (std::nothrow) axi_plan_s;
  if (!p) return AXI_ERR_ARG;
  p->prec = prec;
  p->obs.resize(n_obs);
  size_t off = 0;
  p->off_obsdev = off; off = align_up(off + sizeof(ObsDev) * n_obs);
  int ntask = 0;
  for (int i = 0; i < n_obs; ++i) ntask += obs[i].P / 2 + 1;
  p->off_task_obs = off; off = align_up(off + sizeof(int) * ntask);
  p->off_task_mode = off; off = align_up(off + sizeof(int) * ntask);
  p->off_status = off; off = align_up(off + sizeof(int));
  size_t fill_gdig_bytes = 0, fill_gex_bytes = 0;
  // Split plans keep every panel's reflector digits (written by the QR, read
  // by every apply) when they fit in 4 GB over the plan; otherwise the QR
  // alternates two blocks per mode and each apply recomputes the digits.
  bool keep_digits = false;
  if (slices > 0) {
    size_t total = 0;
    for (int i = 0; i < n_obs; ++i) {
      const int rows = obs[i].bc == AXI_BC_TRANSMISSION ? 2 * obs[i].M : obs[i].M;
      const int cols = obs[i].bc == AXI_BC_TRANSMISSION ? 2 * obs[i].N : obs[i].N;
      const size_t kp = (size_t)(rows + 63) / 64 * 64 + 64;
      const size_t np = (size_t)(cols + axi::kNB - 1) / axi::kNB;
      total += (size_t)(obs[i].P / 2 + 1) * np * (4 * slices * axi::kNB * kp * 2 + (axi::kNB + kp) * 4);
    }
    keep_digits = total <= ((size_t)4 << 30);
  }
  for (int i = 0; i < n_obs; ++i) {
    const axi_obstacle &o = obs[i];
    ObsHost &h = p->obs[i];
    ObsDev &d = h.dev;
    std::memset(&d, 0, sizeof(d));
    d.M = o.M; d.N = o.N; d.P = o.P; d.q = o.q; d.bc = o.bc;
    d.rows = o.bc == AXI_BC_TRANSMISSION ? 2 * o.M : o.M;
    d.cols = o.bc == AXI_BC_TRANSMISSION ? 2 * o.N : o.N;
    d.D = o.P / 2 + 1;
    d.npanels = (d.cols + axi::kNB - 1) / axi::kNB;
    d.slices = slices;
    d.k = o.k; d.km = o.bc == AXI_BC_TRANSMISSION ? o.k_minus : 0.0;
    h.coll.assign(o.h_coll, o.h_coll + 4 * o.M);
    h.src.assign(o.h_src, o.h_src + 2 * o.N);
    if (o.bc == AXI_BC_TRANSMISSION) h.srcx.assign(o.h_src_ext, o.h_src_ext + 2 * o.N);
    h.tab_cos.resize(o.q);
    for (int r = 0; r < o.q; ++r) h.tab_cos[r] = std::cos(2.0 * kPi * r / o.q);
    h.tab_s2.resize(o.q / 2 + 1);
    for (int l = 0; l <= o.q / 2; ++l) {
      const double s = std::sin(kPi * l / o.q);
      h.tab_s2[l] = s * s;
    }
    h.tw_P.resize(o.P);
    for (int r = 0; r < o.P; ++r)
      h.tw_P[r] = make_double2(std::cos(2.0 * kPi * r / o.P), -std::sin(2.0 * kPi * r / o.P));
    // radices 4, 2, 3, 5 and output permutations for the FFTs of length P
    // (apply) and q (fill)
    d.fft_nst = fft_plan(o.P, d.fft_rad, h.fft_perm);
    d.fft_nst_q = fft_plan(o.q, d.fft_rad_q, h.fft_perm_q, d.D, &d.fft_sum_last_q);
    h.tw_q.resize(o.q);
    for (int r = 0; r < o.q; ++r)
      h.tw_q[r] = make_double2(std::cos(2.0 * kPi * r / o.q), -std::sin(2.0 * kPi * r / o.q));
    h.off_perm_q = off; off = align_up(off + sizeof(int) * h.fft_perm_q.size());
    h.off_tw_q = off; off = align_up(off + sizeof(double2) * h.tw_q.size());
    h.off_coll = off; off = align_up(off + sizeof(double) * h.coll.size());
    h.off_perm = off; off = align_up(off + sizeof(int) * h.fft_perm.size());
    h.off_src = off; off = align_up(off + sizeof(double) * h.src.size());
    h.off_srcx = off; off = align_up(off + sizeof(double) * h.srcx.size());
    h.off_cos = off; off = align_up(off + sizeof(double) * h.tab_cos.size());
    h.off_s2 = off; off = align_up(off + sizeof(double) * h.tab_s2.size());
    h.off_tw = off; off = align_up(off + sizeof(double2) * h.tw_P.size());
    h.tab_ring.resize(axi::trig::kRingTab);
    axi::trig::ring_table_host(h.tab_ring.data());
    h.off_ring = off; off = align_up(off + sizeof(double2) * h.tab_ring.size());
    if (fill_strides(h, o.M, o.N, o.P, o.q, o.bc == AXI_BC_TRANSMISSION, full_grid) != AXI_OK) {
      delete p;
      return AXI_ERR_GEOMETRY;
    }
    h.off_fsig = off; off = align_up(off + h.fill_sig.size());
    h.owned.assign(d.D, 1);
    h.off_owned = off; off = align_up(off + h.owned.size());
    h.off_A = off; off = align_up(off + sizeof(double2) * (size_t)d.D * d.cols * d.rows);
    h.off_tau = off; off = align_up(off + sizeof(double2) * (size_t)d.D * d.cols);
    h.off_T = off; off = align_up(off + sizeof(double2) * (size_t)d.D * d.npanels * axi::kNB * axi::kNB);
    d.tsvd = tsvd ? 1 : 0;
    if (tsvd) {
      h.off_svdU = off; off = align_up(off + sizeof(double2) * (size_t)d.D * d.cols * d.cols);
      h.off_svdV = off; off = align_up(off + sizeof(double2) * (size_t)d.D * d.cols * d.cols);
      h.off_svdS = off; off = align_up(off + sizeof(double) * (size_t)d.D * d.cols);
      h.off_svdSw = off; off = align_up(off + sizeof(int) * (size_t)d.D);
    }
    if (slices > 0) {
      // digit rows: rounded up to 64, plus 64 zero rows so that a 64-row chunk
      // starting at any row of X stays inside the block
      d.kp = (d.rows + 63) / 64 * 64 + 64;
      const size_t blocks = (size_t)d.D * d.npanels;
      (void)blocks;
      d.dig_kept = keep_digits ? 1 : 0;
      d.dig_nslot = keep_digits ? d.npanels : 2;
      h.off_vdig = off; off = align_up(off + sizeof(unsigned short) * (size_t)d.D * d.dig_nslot * 4 * slices * axi::kNB * d.kp);
      h.off_vexp = off; off = align_up(off + sizeof(int) * (size_t)d.D * d.dig_nslot * (axi::kNB + d.kp));
      h.off_ckey = off; off = align_up(off + sizeof(unsigned long long) * (size_t)d.D * 2 * d.cols);
      h.off_ybuf = off; off = align_up(off + sizeof(double2) * (size_t)d.D * 2 * axi::kNB * d.kp);
      h.off_ykey = off; off = align_up(off + sizeof(unsigned long long) * (size_t)d.D * 2 * axi::kNB);
      h.off_ydig = off; off = align_up(off + sizeof(unsigned short) * (size_t)d.D * 2 * 2 * slices * axi::kNB * d.kp);
      h.off_yexp = off; off = align_up(off + sizeof(int) * (size_t)d.D * 2 * axi::kNB);
      h.off_rdig = off; off = align_up(off + axi::r_digit_bytes(d));
      h.off_rex = off; off = align_up(off + axi::r_exponent_bytes(d));
      // split fill: folded length, padding, cos-table digits, pair chunk
      const int hh = d.q / 2;
      d.fill_L = (hh % 2 == 0) ? hh / 2 + 1 : (hh + 1) / 2;
      d.fill_Lp = (d.fill_L + 31) / 32 * 32;
      d.fill_MR = ((d.D + 1) / 2 + 15) / 16 * 16;
      d.fill_tc = axi::fill_uses_tc(d.fill_Lp, d.fill_MR) ? 1 : 0;
      const int kinds = o.bc == AXI_BC_TRANSMISSION ? 4 : 1;
      const size_t per_pair = (size_t)2 * 2 * kinds * axi::kFillDigits * d.fill_Lp * sizeof(unsigned short);
      const size_t cap = (size_t)512 << 20;
      d.fill_chunk_pairs = (int)std::max<size_t>(8, std::min<size_t>((size_t)o.M * o.N, cap / per_pair));
      // the tcgen05 layout pads the columns to whole 128-column tiles
      const size_t pad = d.fill_tc ? (size_t)2 * 128 * axi::kFillDigits * d.fill_Lp * sizeof(unsigned short) : 0;
      fill_gdig_bytes = std::max(fill_gdig_bytes, per_pair * d.fill_chunk_pairs + pad);
      fill_gex_bytes = std::max(fill_gex_bytes, sizeof(int) * 2 * 2 * kinds * (size_t)d.fill_chunk_pairs);
      fill_cos_digits(h, axi::kFillDigits);
      h.off_fcdig = off; off = align_up(off + sizeof(unsigned short) * h.fill_cdig.size());
      h.off_fcex = off; off = align_up(off + sizeof(int) * h.fill_cex.size());
    }
  }
  if (fill_gdig_bytes > 0) {
    p->off_fgdig = off; off = align_up(off + fill_gdig_bytes);
    p->off_fgex = off; off = align_up(off + fill_gex_bytes);
  }
  p->bytes = off;
  // QR task list: (obstacle, mode), obstacles with more panels first so the
  // tasks still active at panel step s form a prefix of the list.
  std::vector<int> order(n_obs);
  for (int i = 0; i < n_obs; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    return p->obs[a].dev.npanels > p->obs[b].dev.npanels;
  });
  for (int i : order)
    for (int m = 0; m < p->obs[i].dev.D; ++m) { p->task_obs.push_back(i); p->task_mode.push_back(m); }
  p->all_task_obs = p->task_obs;
  p->all_task_mode = p->task_mode;
  step_tables(p);
  *out = p;
  return AXI_OK;
}

axi_status axi_plan_workspace_bytes(const axi_plan *plan, size_t *bytes) {
  if (!plan || !bytes) return AXI_ERR_ARG;
  *bytes = plan->bytes;
  return AXI_OK;
}

axi_status axi_plan_shard(axi_plan *plan, int32_t rank, int32_t world) {
  if (!plan || world < 1 || rank < 0 || rank >= world) return AXI_ERR_ARG;
  // longest processing time first: tasks by decreasing QR flops (ties in
  // task-list order) each to the least loaded rank (ties to the lowest), the
  // same assignment on every process
  const size_t nt = plan->all_task_obs.size();
  std::vector<double> fl(nt);
  for (size_t t = 0; t < nt; ++t) {
    const ObsDev &d = plan->obs[plan->all_task_obs[t]].dev;
    fl[t] = 8.0 * d.rows * (double)d.cols * d.cols - 8.0 / 3.0 * (double)d.cols * d.cols * d.cols;
  }
  std::vector<size_t> order(nt);
  for (size_t t = 0; t < nt; ++t) order[t] = t;
  std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) { return fl[a] > fl[b]; });
  std::vector<double> load(world, 0.0);
  std::vector<int> owner(nt, 0);
  for (size_t t : order) {
    int best = 0;
    for (int r = 1; r < world; ++r)
      if (load[r] < load[best]) best = r;
    owner[t] = best;
    load[best] += fl[t];
  }
  plan->task_obs.clear();
  plan->task_mode.clear();
  for (auto &h : plan->obs) std::fill(h.owned.begin(), h.owned.end(), 0);
  for (size_t t = 0; t < nt; ++t) {
    if (owner[t] != rank) continue;
    plan->task_obs.push_back(plan->all_task_obs[t]);
    plan->task_mode.push_back(plan->all_task_mode[t]);
    plan->obs[plan->all_task_obs[t]].owned[plan->all_task_mode[t]] = 1;
  }
  step_tables(plan);
  return AXI_OK;
}

axi_status axi_plan_owned_modes(const axi_plan *plan, int32_t obs, uint8_t *h_mask) {
  if (!plan || !h_mask || obs < 0 || obs >= (int)plan->obs.size()) return AXI_ERR_ARG;
  const auto &o = plan->obs[obs].owned;
  std::memcpy(h_mask, o.data(), o.size());
  return AXI_OK;
}

axi_status axi_plan_set_tuning(axi_plan *plan, const char *json) {
  if (!plan) return AXI_ERR_ARG;
  axi::Tuning t = plan->tune;
  if (!parse_tuning(json, t)) return AXI_ERR_ARG;
  plan->tune = t;
  return AXI_OK;
}

axi_status axi_plan_get_tuning(const axi_plan *plan, char *buf, size_t n) {
  if (!plan) return AXI_ERR_ARG;
  return copy_out(tuning_json(plan->tune), buf, n);
}

axi_status axi_plan_destroy(axi_plan *plan) {
  delete plan;
  return AXI_OK;
}

// Fill, then the panel steps with look-ahead. For step p:
//   caller's stream: panel(p) -> record ev_panel -> wait ev_rest(p-1)
//                    -> FP64 update of the next panel's columns
//   side stream:     wait ev_panel -> [reflector digits (split)] -> update of
//                    the columns beyond (split or FP64) -> record ev_rest
// so panel(p+1) and the small next-panel update form the critical path while
// the bulk of each trailing update runs beside them. The columns beyond of
// step p-1 include the next panel's columns of step p, hence the wait.
static axi_status run_build(axi_operator_s *op, cudaStream_t st,
                            const axi_c128 *const *modes = nullptr) {
  axi_plan_s *p = op->plan;
  ProfScope scope(op->prof());
  cudaError_t e = cudaMemsetAsync(op->d_status, 0, sizeof(int), st);
  if (e != cudaSuccess) return AXI_ERR_CUDA;
  for (size_t i = 0; i < p->obs.size(); ++i) {
    const ObsDev &d = p->obs[i].dev;
    if (modes && modes[i]) {              // the caller's modal matrices instead of the fill
      e = cudaMemcpyAsync(d.A, modes[i], sizeof(double2) * (size_t)d.D * d.cols * d.rows,
                          cudaMemcpyDeviceToDevice, st);
      if (e != cudaSuccess) return AXI_ERR_CUDA;
      continue;
    }
    const int pid = axi::prof_begin(AXI_KERNEL_FILL, st);
    e = axi::launch_fill(op->d_obs, d, (int)i, d.A, d.rows, d.cols, st, p->tune.fill_chunk_mb);
    axi::prof_end(pid, st);
    if (e != cudaSuccess) return AXI_ERR_CUDA;
  }
  const int slices = p->obs[0].dev.slices;
  int kp_max = 0;
  for (const auto &ob : p->obs) kp_max = ob.dev.kp > kp_max ? ob.dev.kp : kp_max;
  // the panel chain on the high-priority stream, joined back below
  const cudaStream_t caller = st;
  if (p->tune.crit_stream == 1 && !p->step_tasks.empty()) {
    if (cudaEventRecord(op->ev_fork, caller) != cudaSuccess ||
        cudaStreamWaitEvent(op->crit, op->ev_fork, 0) != cudaSuccess)
      return AXI_ERR_CUDA;
    st = op->crit;
  }
  bool rest_pending = false, side_used = false;
  for (size_t s = 0; s < p->step_tasks.size(); ++s) {
    const int nt = p->step_tasks[s];
    int pid = axi::prof_begin(AXI_KERNEL_PANEL, st);
    bool panel_digits = false;
    e = axi::launch_qr_panel(op->d_obs, op->d_task_obs, op->d_task_mode, nt, (int)s,
                             p->step_rows[s], slices, p->tune.panel_cluster,
                             p->tune.panel_threads, p->tune.panel_fixed, st, &panel_digits);
    axi::prof_end(pid, st, p->step_fl_panel[s]);
    if (e != cudaSuccess) return AXI_ERR_CUDA;
    if (panel_digits) {                 // the digits right behind the panel, over the whole GPU
      pid = axi::prof_begin(AXI_KERNEL_PANEL_DIGITS, st);
      e = axi::launch_vdigits(op->d_obs, op->d_task_obs, op->d_task_mode, nt, (int)s, kp_max, slices,
                                st);
      axi::prof_end(pid, st);
      if (e != cudaSuccess) return AXI_ERR_CUDA;
    }
    const int rest_cols = p->step_cols[s] - axi::kNB;
    // kept digits: every panel's digits are written (the apply reads them),
    // also at the last steps that have no trailing update
    const bool digits_here = slices > 0 && (rest_cols > 0 || p->obs[0].dev.dig_kept);
    // the side stream's work of this step starts behind the panel (and its
    // digits), or, with rest_start 1, behind the next-panel update as well
    const bool fork_late = p->tune.rest_start == 1 && p->step_cols[s] > 0;
    if ((rest_cols > 0 || digits_here) && !fork_late) {
      if (cudaEventRecord(op->ev_panel, st) != cudaSuccess ||
          cudaStreamWaitEvent(op->side, op->ev_panel, 0) != cudaSuccess)
        return AXI_ERR_CUDA;
    }
    if (rest_pending && cudaStreamWaitEvent(st, op->ev_rest, 0) != cudaSuccess) return AXI_ERR_CUDA;
    rest_pending = false;
    if (p->step_cols[s] > 0) {
      pid = axi::prof_begin(AXI_KERNEL_UPDATE_NEXT, st);
      // split plans whose panel wrote its digits update the next panel's
      // columns in split precision too; otherwise in native FP64
      e = panel_digits && p->tune.next_update != 1
              ? axi::launch_qr_update_next_split(op->d_obs, op->d_task_obs, op->d_task_mode, nt,
                                                 (int)s, slices, p->step_rows[s],
                                                 p->tune.next_cluster, st)
              : axi::launch_qr_update_next(op->d_obs, op->d_task_obs, op->d_task_mode, nt, (int)s, st);
      axi::prof_end(pid, st, p->step_fl_next[s]);
      if (e != cudaSuccess) return AXI_ERR_CUDA;
    }
    if ((rest_cols > 0 || digits_here) && fork_late) {
      if (cudaEventRecord(op->ev_panel, st) != cudaSuccess ||
          cudaStreamWaitEvent(op->side, op->ev_panel, 0) != cudaSuccess)
        return AXI_ERR_CUDA;
    }
    if (digits_here && !panel_digits) {
      pid = axi::prof_begin(AXI_KERNEL_PANEL_DIGITS, op->side);
      e = axi::launch_panel_digits(op->d_obs, op->d_task_obs, op->d_task_mode, nt, (int)s, slices,
                                   kp_max, op->side);
      axi::prof_end(pid, op->side);
      if (e != cudaSuccess) return AXI_ERR_CUDA;
    }
    if (rest_cols > 0 || digits_here) side_used = true;
    if (rest_cols > 0) {
      // split plans whose panel wrote its column exponents: Y = V T beside
      // the critical path, so the trailing update forms W' in one product
      const bool use_y = slices > 0 && panel_digits;
      if (use_y) {
        pid = axi::prof_begin(AXI_KERNEL_PANEL_DIGITS, op->side);
        e = axi::launch_y_digits(op->d_obs, op->d_task_obs, op->d_task_mode, nt, (int)s, kp_max, slices,
                                 op->side);
        axi::prof_end(pid, op->side);
        if (e != cudaSuccess) return AXI_ERR_CUDA;
      }
      pid = axi::prof_begin(AXI_KERNEL_UPDATE_REST, op->side);
      e = axi::launch_qr_update_rest(op->d_obs, op->d_task_obs, op->d_task_mode, nt, (int)s, slices,
                                     rest_cols, p->tune.rest_grid, use_y, op->side);
      axi::prof_end(pid, op->side, p->step_fl_rest[s]);
      if (e != cudaSuccess || cudaEventRecord(op->ev_rest, op->side) != cudaSuccess)
        return AXI_ERR_CUDA;
      rest_pending = true;
    }
  }
  // join the side stream (its last kernels may be digit blocks only the apply reads)
  if (side_used && (cudaEventRecord(op->ev_rest, op->side) != cudaSuccess ||
                    cudaStreamWaitEvent(st, op->ev_rest, 0) != cudaSuccess))
    return AXI_ERR_CUDA;
  if (st != caller) {
    if (cudaEventRecord(op->ev_join, st) != cudaSuccess ||
        cudaStreamWaitEvent(caller, op->ev_join, 0) != cudaSuccess)
      return AXI_ERR_CUDA;
    st = caller;
  }
  for (size_t i = 0; i < p->obs.size(); ++i) {
    const ObsDev &d = p->obs[i].dev;
    if (d.tsvd) {                         // SVD of R: the apply uses V Sigma^+ U_R^H
      const int pid = axi::prof_begin(AXI_KERNEL_R_DIGITS, st);
      e = axi::launch_tsvd(op->d_obs + i, d, st);
      axi::prof_end(pid, st);
    } else {                              // digits of R's off-diagonal blocks for the back substitution
      const int pid = axi::prof_begin(AXI_KERNEL_R_DIGITS, st);
      e = axi::launch_r_digits(op->d_obs + i, d, st);
      axi::prof_end(pid, st);
    }
    if (e != cudaSuccess) return AXI_ERR_CUDA;
  }
  return AXI_OK;
}

axi_status axi_build_operator(axi_plan *plan, void *d_workspace, size_t bytes, void *stream,
                              axi_operator **out) {
  if (!plan || !d_workspace || !out) return AXI_ERR_ARG;
  if (bytes < plan->bytes || (reinterpret_cast<uintptr_t>(d_workspace) & (kAlign - 1)))
    return AXI_ERR_WORKSPACE;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  char *ws = static_cast<char *>(d_workspace);
  std::vector<ObsDev> devs(plan->obs.size());
  for (size_t i = 0; i < plan->obs.size(); ++i) {
    ObsHost &h = plan->obs[i];
    ObsDev &d = h.dev;
    d.coll = reinterpret_cast<const double *>(ws + h.off_coll);
    d.src = reinterpret_cast<const double *>(ws + h.off_src);
    d.srcx = h.srcx.empty() ? nullptr : reinterpret_cast<const double *>(ws + h.off_srcx);
    d.tab_cos = reinterpret_cast<const double *>(ws + h.off_cos);
    d.tab_s2 = reinterpret_cast<const double *>(ws + h.off_s2);
    d.tw_P = reinterpret_cast<const double2 *>(ws + h.off_tw);
    d.tab_ring = reinterpret_cast<const double2 *>(ws + h.off_ring);
    d.fill_sig = reinterpret_cast<const unsigned char *>(ws + h.off_fsig);
    d.mode_owned = reinterpret_cast<const unsigned char *>(ws + h.off_owned);
    d.fft_perm = reinterpret_cast<const int *>(ws + h.off_perm);
    d.fft_perm_q = reinterpret_cast<const int *>(ws + h.off_perm_q);
    d.tw_q = reinterpret_cast<const double2 *>(ws + h.off_tw_q);
    d.A = reinterpret_cast<double2 *>(ws + h.off_A);
    d.tau = reinterpret_cast<double2 *>(ws + h.off_tau);
    d.T = reinterpret_cast<double2 *>(ws + h.off_T);
    d.svdU = d.tsvd ? reinterpret_cast<double2 *>(ws + h.off_svdU) : nullptr;
    d.svdV = d.tsvd ? reinterpret_cast<double2 *>(ws + h.off_svdV) : nullptr;
    d.svdS = d.tsvd ? reinterpret_cast<double *>(ws + h.off_svdS) : nullptr;
    d.svdSweeps = d.tsvd ? reinterpret_cast<int *>(ws + h.off_svdSw) : nullptr;
    d.vdig = d.slices > 0 ? reinterpret_cast<unsigned short *>(ws + h.off_vdig) : nullptr;
    d.vexp = d.slices > 0 ? reinterpret_cast<int *>(ws + h.off_vexp) : nullptr;
    d.ckey = d.slices > 0 ? reinterpret_cast<unsigned long long *>(ws + h.off_ckey) : nullptr;
    d.rdig = d.slices > 0 ? reinterpret_cast<unsigned short *>(ws + h.off_rdig) : nullptr;
    d.ybuf = d.slices > 0 ? reinterpret_cast<double2 *>(ws + h.off_ybuf) : nullptr;
    d.ykey = d.slices > 0 ? reinterpret_cast<unsigned long long *>(ws + h.off_ykey) : nullptr;
    d.ydig = d.slices > 0 ? reinterpret_cast<unsigned short *>(ws + h.off_ydig) : nullptr;
    d.yexp = d.slices > 0 ? reinterpret_cast<int *>(ws + h.off_yexp) : nullptr;
    d.rex = d.slices > 0 ? reinterpret_cast<int *>(ws + h.off_rex) : nullptr;
    if (d.slices > 0) {
      d.fill_cdig = reinterpret_cast<const unsigned short *>(ws + h.off_fcdig);
      d.fill_cex = reinterpret_cast<const int *>(ws + h.off_fcex);
      d.fill_gdig = reinterpret_cast<uint32_t *>(ws + plan->off_fgdig);
      d.fill_gex = reinterpret_cast<int *>(ws + plan->off_fgex);
    }
    d.status = reinterpret_cast<int *>(ws + plan->off_status);
    devs[i] = d;
    struct { size_t off; const void *src; size_t n; } cp[] = {
        {h.off_coll, h.coll.data(), sizeof(double) * h.coll.size()},
        {h.off_src, h.src.data(), sizeof(double) * h.src.size()},
        {h.off_srcx, h.srcx.data(), sizeof(double) * h.srcx.size()},
        {h.off_cos, h.tab_cos.data(), sizeof(double) * h.tab_cos.size()},
        {h.off_s2, h.tab_s2.data(), sizeof(double) * h.tab_s2.size()},
        {h.off_tw, h.tw_P.data(), sizeof(double2) * h.tw_P.size()},
        {h.off_ring, h.tab_ring.data(), sizeof(double2) * h.tab_ring.size()},
        {h.off_fsig, h.fill_sig.data(), h.fill_sig.size()},
        {h.off_owned, h.owned.data(), h.owned.size()},
        {h.off_perm, h.fft_perm.data(), sizeof(int) * h.fft_perm.size()},
        {h.off_perm_q, h.fft_perm_q.data(), sizeof(int) * h.fft_perm_q.size()},
        {h.off_tw_q, h.tw_q.data(), sizeof(double2) * h.tw_q.size()},
        {h.off_fcdig, h.fill_cdig.data(), sizeof(unsigned short) * h.fill_cdig.size()},
        {h.off_fcex, h.fill_cex.data(), sizeof(int) * h.fill_cex.size()},
    };
    for (auto &c : cp) {
      if (!c.n) continue;
      if (cudaMemcpyAsync(ws + c.off, c.src, c.n, cudaMemcpyHostToDevice, st) != cudaSuccess)
        return AXI_ERR_CUDA;
    }
  }
  if (cudaMemcpyAsync(ws + plan->off_obsdev, devs.data(), sizeof(ObsDev) * devs.size(),
                      cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(ws + plan->off_task_obs, plan->task_obs.data(),
                      sizeof(int) * plan->task_obs.size(), cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(ws + plan->off_task_mode, plan->task_mode.data(),
                      sizeof(int) * plan->task_mode.size(), cudaMemcpyHostToDevice, st) != cudaSuccess)
    return AXI_ERR_CUDA;
  // the host staging vectors above must not be released before the copies finish
  if (cudaStreamSynchronize(st) != cudaSuccess) return AXI_ERR_CUDA;
  axi_operator_s *op = new (std::nothrow) axi_operator_s;
  if (!op) return AXI_ERR_ARG;
  op->plan = plan;
  op->ws = ws;
  if (cudaGetDevice(&op->device) != cudaSuccess) {
    delete op;
    return AXI_ERR_CUDA;
  }
  op->d_obs = reinterpret_cast<ObsDev *>(ws + plan->off_obsdev);
  op->d_task_obs = reinterpret_cast<int *>(ws + plan->off_task_obs);
  op->d_task_mode = reinterpret_cast<int *>(ws + plan->off_task_mode);
  op->d_status = reinterpret_cast<int *>(ws + plan->off_status);
  int prio_least = 0, prio_greatest = 0;
  if (cudaDeviceGetStreamPriorityRange(&prio_least, &prio_greatest) != cudaSuccess ||
      cudaStreamCreateWithFlags(&op->side, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithPriority(&op->crit, cudaStreamNonBlocking, prio_greatest) != cudaSuccess ||
      cudaEventCreateWithFlags(&op->ev_panel, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&op->ev_rest, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&op->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&op->ev_join, cudaEventDisableTiming) != cudaSuccess) {
    axi_operator_destroy(op);
    return AXI_ERR_CUDA;
  }
  axi_status s = run_build(op, st);
  if (s != AXI_OK) { axi_operator_destroy(op); return s; }
  *out = op;
  return AXI_OK;
}

axi_status axi_refactor_operator(axi_operator *op, void *stream) {
  if (!op) return AXI_ERR_ARG;
  return run_build(op, static_cast<cudaStream_t>(stream));
}

axi_status axi_refactor_operator_modes(axi_operator *op, const axi_c128 *const *h_modes, void *stream) {
  if (!op || !h_modes) return AXI_ERR_ARG;
  return run_build(op, static_cast<cudaStream_t>(stream), h_modes);
}

axi_status axi_fill_modes(const axi_operator *op, int32_t obs, axi_c128 *d_out, void *stream) {
  if (!op || !d_out || obs < 0 || obs >= (int)op->plan->obs.size()) return AXI_ERR_ARG;
  const ObsDev &d = op->plan->obs[obs].dev;
  return cuda_status(axi::launch_fill(op->d_obs, d, obs, reinterpret_cast<double2 *>(d_out), d.rows,
                                      d.cols, static_cast<cudaStream_t>(stream),
                                      op->plan->tune.fill_chunk_mb));
}

axi_status axi_btilde_count(const axi_operator *op, int32_t obs, int32_t p, size_t *count) {
  if (!op || !count || obs < 0 || obs >= (int)op->plan->obs.size() || p < 0 ||
      p > AXI_BTILDE_MAX_DEGREE)
    return AXI_ERR_ARG;
  *count = axi::btilde_count(op->plan->obs[obs].dev, p);
  return AXI_OK;
}

axi_status axi_fill_btilde(const axi_operator *op, int32_t obs, int32_t p, double *d_out,
                           size_t count, void *stream) {
  if (!op || !d_out || obs < 0 || obs >= (int)op->plan->obs.size() || p < 0 ||
      p > AXI_BTILDE_MAX_DEGREE || (reinterpret_cast<uintptr_t>(d_out) & 7))
    return AXI_ERR_ARG;
  const ObsDev &d = op->plan->obs[obs].dev;
  if (count < axi::btilde_count(d, p)) return AXI_ERR_ARG;
  return cuda_status(axi::launch_btilde(op->d_obs, d, obs, p, d_out, static_cast<cudaStream_t>(stream)));
}

axi_status axi_q_shape(const axi_cell *cell, int64_t *rows, int64_t *cols, int64_t *n_rb) {
  if (!cell || !rows || !cols || !n_rb) return AXI_ERR_ARG;
  long long r = 0, c = 0, n = 0;
  if (!axi::q_shape(*cell, r, c, n)) return AXI_ERR_ARG;
  *rows = r; *cols = c; *n_rb = n;
  return AXI_OK;
}

axi_status axi_q_modes(const axi_cell *cell, int32_t *h_mn, int64_t cap) {
  if (!cell || !h_mn) return AXI_ERR_ARG;
  return axi::q_modes(*cell, reinterpret_cast<int *>(h_mn), cap) ? AXI_OK : AXI_ERR_ARG;
}

axi_status axi_fill_q(const axi_operator *op, int32_t obs, const axi_cell *cell, axi_c128 *d_out,
                      int64_t ld, void *stream) {
  if (!op || !cell || !d_out || obs < 0 || obs >= (int)op->plan->obs.size() ||
      (reinterpret_cast<uintptr_t>(d_out) & 15))
    return AXI_ERR_ARG;
  long long r = 0, c = 0, n = 0;
  if (!axi::q_shape(*cell, r, c, n) || ld < r) return AXI_ERR_ARG;
  const ObsDev &d = op->plan->obs[obs].dev;
  return cuda_status(axi::launch_q(op->d_obs, d, obs, *cell, reinterpret_cast<double2 *>(d_out), ld,
                                   static_cast<cudaStream_t>(stream)));
}

axi_status axi_c_shape(const axi_operator *op, int32_t obs, const axi_cell *cell, int64_t *rows,
                       int64_t *cols) {
  if (!op || !cell || !rows || !cols || obs < 0 || obs >= (int)op->plan->obs.size()) return AXI_ERR_ARG;
  const ObsDev &d = op->plan->obs[obs].dev;
  if (d.bc != AXI_BC_NEUMANN) return AXI_ERR_UNSUPPORTED;
  long long r = 0, c = 0;
  if (!axi::c_shape(d, *cell, r, c)) return AXI_ERR_ARG;
  *rows = r; *cols = c;
  return AXI_OK;
}

axi_status axi_fill_c(const axi_operator *op, int32_t obs, const axi_cell *cell, axi_c128 *d_out,
                      int64_t ld, void *stream) {
  if (!op || !cell || !d_out || obs < 0 || obs >= (int)op->plan->obs.size() ||
      (reinterpret_cast<uintptr_t>(d_out) & 15))
    return AXI_ERR_ARG;
  const ObsDev &d = op->plan->obs[obs].dev;
  if (d.bc != AXI_BC_NEUMANN) return AXI_ERR_UNSUPPORTED;
  long long r = 0, c = 0;
  if (!axi::c_shape(d, *cell, r, c) || ld < r) return AXI_ERR_ARG;
  return cuda_status(axi::launch_c(op->d_obs, d, obs, *cell, reinterpret_cast<double2 *>(d_out), ld,
                                   static_cast<cudaStream_t>(stream)));
}

axi_status axi_svd_jacobi(axi_c128 *d_A, int64_t m, int64_t n, int64_t lda, axi_c128 *d_V, int64_t ldv,
                          double *d_sigma, double tol, int32_t max_sweeps, int32_t *sweeps,
                          void *stream) {
  if (!d_A || !d_V || !d_sigma || !sweeps || n < 1 || m < n || lda < m || ldv < n || max_sweeps < 1 ||
      n > (int64_t)1 << 20 || m > (int64_t)1 << 30 || !(tol >= 0.0) ||
      (reinterpret_cast<uintptr_t>(d_A) & 15) || (reinterpret_cast<uintptr_t>(d_V) & 15) ||
      (reinterpret_cast<uintptr_t>(d_sigma) & 7))
    return AXI_ERR_ARG;
  int sw = 0;
  bool conv = false;
  const cudaError_t e = axi::svd_jacobi(reinterpret_cast<double2 *>(d_A), m, n, lda,
                                        reinterpret_cast<double2 *>(d_V), ldv, d_sigma, tol, max_sweeps,
                                        &sw, &conv, static_cast<cudaStream_t>(stream));
  *sweeps = sw;
  if (e != cudaSuccess) return AXI_ERR_CUDA;
  return conv ? AXI_OK : AXI_ERR_NUMERIC;
}

axi_status axi_svd_solve(const axi_c128 *d_US, const axi_c128 *d_V, const double *d_sigma, int64_t m,
                         int64_t n, int64_t lda, int64_t ldv, double cutoff, const axi_c128 *d_B,
                         int64_t ldb, int64_t nrhs, axi_c128 *d_X, int64_t ldx, axi_c128 *d_work,
                         void *stream) {
  if (!d_US || !d_V || !d_sigma || !d_B || !d_X || !d_work || n < 1 || m < n || lda < m || ldv < n ||
      ldb < m || ldx < n || nrhs < 1 || nrhs > 65535 || n > (int64_t)1 << 20 || !(cutoff >= 0.0))
    return AXI_ERR_ARG;
  return cuda_status(axi::svd_solve(reinterpret_cast<const double2 *>(d_US),
                                    reinterpret_cast<const double2 *>(d_V), d_sigma, m, n, lda, ldv, cutoff,
                                    reinterpret_cast<const double2 *>(d_B), ldb, nrhs,
                                    reinterpret_cast<double2 *>(d_X), ldx,
                                    reinterpret_cast<double2 *>(d_work), static_cast<cudaStream_t>(stream)));
}

axi_status axi_operator_factors(const axi_operator *op, int32_t obs, axi_factor_view *v) {
  if (!op || !v || obs < 0 || obs >= (int)op->plan->obs.size()) return AXI_ERR_ARG;
  const ObsDev &d = op->plan->obs[obs].dev;
  v->rows = d.rows; v->cols = d.cols; v->D = d.D; v->nb = axi::kNB; v->npanels = d.npanels;
  v->d_A = reinterpret_cast<const axi_c128 *>(d.A);
  v->d_tau = reinterpret_cast<const axi_c128 *>(d.tau);
  v->d_T = reinterpret_cast<const axi_c128 *>(d.T);
  return AXI_OK;
}

axi_status axi_operator_svd(const axi_operator *op, int32_t obs, axi_svd_view *v) {
  if (!op || !v || obs < 0 || obs >= (int)op->plan->obs.size()) return AXI_ERR_ARG;
  const ObsDev &d = op->plan->obs[obs].dev;
  if (!d.tsvd) return AXI_ERR_UNSUPPORTED;
  v->n = d.cols;
  v->D = d.D;
  v->d_U = reinterpret_cast<const axi_c128 *>(d.svdU);
  v->d_V = reinterpret_cast<const axi_c128 *>(d.svdV);
  v->d_sigma = d.svdS;
  v->d_sweeps = d.svdSweeps;
  return AXI_OK;
}

axi_status axi_incident_planewaves(const axi_operator *op, int32_t obs, int32_t W,
                                   const double *d_dirs, axi_c128 *d_f, void *stream) {
  if (!op || !d_dirs || !d_f || obs < 0 || obs >= (int)op->plan->obs.size() || W < 1)
    return AXI_ERR_ARG;
  const ObsDev &d = op->plan->obs[obs].dev;
  return cuda_status(axi::launch_incident(op->d_obs + obs, d, W, d_dirs,
                                          reinterpret_cast<double2 *>(d_f),
                                          static_cast<cudaStream_t>(stream)));
}

axi_status axi_apply_workspace_bytes(const axi_operator *op, int32_t obs, int32_t W, size_t *bytes) {
  if (!op || !bytes || obs < 0 || obs >= (int)op->plan->obs.size() || W < 1) return AXI_ERR_ARG;
  const ObsDev &d = op->plan->obs[obs].dev;
  *bytes = align_up(sizeof(double2) * (size_t)d.D * 2 * W * d.rows);
  if (d.slices > 0 && W >= axi::kSplitApplyMinWaves) *bytes += align_up(axi::apply_digit_bytes(d));
  return AXI_OK;
}

axi_status axi_apply_operator(const axi_operator *op, int32_t obs, int32_t W, const axi_c128 *d_f,
                              axi_c128 *d_coef, axi_c128 *d_sigma, void *d_scratch,
                              size_t scratch_bytes, void *stream) {
  if (!op || !d_f || !d_coef || !d_scratch || obs < 0 || obs >= (int)op->plan->obs.size() || W < 1)
    return AXI_ERR_ARG;
  size_t need = 0;
  axi_apply_workspace_bytes(op, obs, W, &need);
  if (scratch_bytes < need) return AXI_ERR_WORKSPACE;
  ObsDev d = op->plan->obs[obs].dev;                      // host copy with the plan's tuning
  d.apply_cluster = op->plan->tune.apply_cluster;
  char *digit_scratch = static_cast<char *>(d_scratch) + align_up(sizeof(double2) * (size_t)d.D * 2 * W * d.rows);
  ProfScope scope(op->prof());
  return cuda_status(axi::launch_apply(op->d_obs + obs, d, W, reinterpret_cast<const double2 *>(d_f),
                                       reinterpret_cast<double2 *>(d_coef),
                                       reinterpret_cast<double2 *>(d_sigma),
                                       static_cast<double2 *>(d_scratch), digit_scratch,
                                       static_cast<cudaStream_t>(stream)));
}

axi_status axi_eval_field(const axi_operator *op, int32_t obs, int32_t W, const axi_c128 *d_coef,
                          int32_t T, const double *d_targets, const double *d_normals, int32_t kind,
                          const axi_lattice *lattice, const double *d_dirs, axi_c128 *d_out,
                          void *d_scratch, size_t scratch_bytes, void *stream) {
  if (!op || !d_coef || !d_targets || !d_out || !d_scratch || obs < 0 ||
      obs >= (int)op->plan->obs.size() || W < 1 || T < 1)
    return AXI_ERR_ARG;
  if (kind < AXI_EVAL_POTENTIAL || kind > AXI_EVAL_FAR_FIELD) return AXI_ERR_ARG;
  if (kind == AXI_EVAL_NORMAL_DERIV && !d_normals) return AXI_ERR_ARG;
  if (lattice && !d_dirs) return AXI_ERR_ARG;
  const ObsDev &d = op->plan->obs[obs].dev;
  if (scratch_bytes < sizeof(double2) * (size_t)W * d.cols * d.P) return AXI_ERR_WORKSPACE;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  double2 *sigma = static_cast<double2 *>(d_scratch);
  cudaError_t e = axi::launch_point_strengths(op->d_obs + obs, d, W,
                                              reinterpret_cast<const double2 *>(d_coef), sigma, st);
  if (e != cudaSuccess) return AXI_ERR_CUDA;
  return cuda_status(axi::launch_eval(op->d_obs + obs, d, W, sigma, T, d_targets, d_normals, kind,
                                      lattice, d_dirs, reinterpret_cast<double2 *>(d_out), st));
}

axi_status axi_near_image_workspace_bytes(const axi_operator *op, int32_t obs, int32_t W,
                                          const axi_lattice *lattice, int32_t slices,
                                          size_t *bytes) {
  if (!op || !lattice || !bytes || obs < 0 || obs >= (int)op->plan->obs.size() || W < 1)
    return AXI_ERR_ARG;
  if (slices != 0 && (slices < 4 || slices > 7)) return AXI_ERR_UNSUPPORTED;
  *bytes = axi::near_image_scratch_bytes(op->plan->obs[obs].dev, W, lattice->ex, lattice->ey, slices);
  return AXI_OK;
}

axi_status axi_near_image_sum(const axi_operator *op, int32_t obs, int32_t W, const axi_c128 *d_coef,
                              const axi_lattice *lattice, const double *d_dirs, int32_t slices,
                              axi_c128 *d_out, void *d_scratch, size_t scratch_bytes,
                              void *stream) {
  if (!op || !d_coef || !lattice || !d_dirs || !d_out || !d_scratch || obs < 0 ||
      obs >= (int)op->plan->obs.size() || W < 1)
    return AXI_ERR_ARG;
  if (slices != 0 && (slices < 4 || slices > 7)) return AXI_ERR_UNSUPPORTED;
  if (!(lattice->ex > 0) || !(lattice->ey > 0)) return AXI_ERR_ARG;
  const ObsDev &d = op->plan->obs[obs].dev;
  if (scratch_bytes < axi::near_image_scratch_bytes(d, W, lattice->ex, lattice->ey, slices))
    return AXI_ERR_WORKSPACE;
  return cuda_status(axi::launch_near_image(op->d_obs + obs, d, W,
                                            reinterpret_cast<const double2 *>(d_coef),
                                            lattice->ex, lattice->ey, d_dirs, slices,
                                            reinterpret_cast<double2 *>(d_out), d_scratch,
                                            static_cast<cudaStream_t>(stream)));
}

axi_status axi_operator_status(const axi_operator *op) {
  if (!op) return AXI_ERR_ARG;
  int s = 0;
  if (cudaMemcpy(&s, op->d_status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
    return AXI_ERR_CUDA;
  if (s & axi::kStatTimeout) return AXI_ERR_TIMEOUT;
  if (s & axi::kStatNonFinite) return AXI_ERR_NUMERIC;
  return AXI_OK;
}

axi_status axi_operator_autotune(axi_operator *op, int32_t reps, void *stream, char *json_out,
                                 size_t n) {
  if (!op || reps < 1 || reps > 100) return AXI_ERR_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  axi_plan_s *p = op->plan;
  const axi::Tuning keep = p->tune;
  const bool split = p->obs[0].dev.slices > 0;
  cudaEvent_t a = nullptr, b = nullptr;
  if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
    if (a) cudaEventDestroy(a);
    return AXI_ERR_CUDA;
  }
  axi::Tuning best = keep;
  double best_ms = 1e300;
  int tried = 0, skipped = 0;
  // one warm-up build of the plan's current tuning, then `reps` timed builds
  auto time_it = [&](double &ms_out) -> axi_status {
    axi_status s = run_build(op, st);
    if (s != AXI_OK) return s;
    if (cudaEventRecord(a, st) != cudaSuccess) return AXI_ERR_CUDA;
    for (int r = 0; r < reps && s == AXI_OK; ++r) s = run_build(op, st);
    if (s != AXI_OK) return s;
    float ms = 0.0f;
    if (cudaEventRecord(b, st) != cudaSuccess || cudaEventSynchronize(b) != cudaSuccess ||
        cudaEventElapsedTime(&ms, a, b) != cudaSuccess)
      return AXI_ERR_CUDA;
    ms_out = ms / reps;
    ++tried;
    return AXI_OK;
  };
  axi_status s = AXI_OK;
  // the panel chain's schedule first
  for (int nu : {1, 2}) {
    if (nu == 2 && !split) continue;
    for (int pc : {0, 1, 2, 4})
      for (int rg : {4, 1, 2, 3})
        for (int pt : {0, 128, 256})
          for (int cs : {0, 1}) {
            if (rg >= 2 && nu != 2) continue;         // the tcgen05 update reads Y^H digits
            p->tune = keep;
            p->tune.next_update = nu;
            p->tune.panel_cluster = pc;
            p->tune.rest_grid = rg;
            p->tune.panel_threads = pt;
            p->tune.crit_stream = cs;
            double ms = 0.0;
            s = time_it(ms);
            if (s != AXI_OK) {                        // a candidate that cannot run here
              (void)cudaGetLastError();
              ++skipped;
              s = AXI_OK;
              continue;
            }
            if (ms < best_ms) {
              best_ms = ms;
              best = p->tune;
            }
          }
  }
  // then, one choice at a time with the best so far: the next-panel update's
  // cluster (split plans whose panels write digits) and the split fill's
  // chunk size (smaller chunks keep the sample digits in L2)
  if (s == AXI_OK && split) {
    for (int nc : {1, 2, 4}) {
      if (best.next_update == 1 || nc == best.next_cluster) continue;
      p->tune = best;
      p->tune.next_cluster = nc;
      double ms = 0.0;
      s = time_it(ms);
      if (s != AXI_OK) {
        (void)cudaGetLastError();
        ++skipped;
        s = AXI_OK;
        continue;
      }
      if (ms < best_ms) {
        best_ms = ms;
        best = p->tune;
      }
    }
  }
  // split plans: the fixed-point panel (one CTA of 128 or 256 threads per mode)
  if (s == AXI_OK && split) {
    const axi::Tuning base = best;
    for (int pt : {128, 256}) {
      p->tune = base;
      p->tune.panel_fixed = 2;
      p->tune.panel_cluster = 1;
      p->tune.panel_threads = pt;
      double ms = 0.0;
      s = time_it(ms);
      if (s != AXI_OK) {
        (void)cudaGetLastError();
        ++skipped;
        s = AXI_OK;
        continue;
      }
      if (ms < best_ms) {
        best_ms = ms;
        best = p->tune;
      }
    }
  }
  if (s == AXI_OK && split && p->obs[0].dev.fill_cdig != nullptr) {
    const axi::Tuning base = best;
    for (int fc : {0, 256, 128, 96, 64}) {
      if (fc == base.fill_chunk_mb) continue;
      p->tune = base;
      p->tune.fill_chunk_mb = fc;
      double ms = 0.0;
      s = time_it(ms);
      if (s != AXI_OK) {
        (void)cudaGetLastError();
        ++skipped;
        s = AXI_OK;
        continue;
      }
      if (ms < best_ms) {
        best_ms = ms;
        best = p->tune;
      }
    }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (s == AXI_OK && best_ms >= 1e300) s = AXI_ERR_CUDA;  // no candidate ran
  if (s != AXI_OK) {
    p->tune = keep;
    return s;
  }
  p->tune = best;
  s = run_build(op, st);                                 // leave the operator built with it
  if (s != AXI_OK) return s;
  if (json_out) {
    std::string js = tuning_json(best);
    char tail[96];
    std::snprintf(tail, sizeof(tail), ", \"build_ms\": %.4f, \"candidates\": %d, \"skipped\": %d}",
                  best_ms, tried, skipped);
    js.pop_back();
    js += tail;
    return copy_out(js, json_out, n);
  }
  return AXI_OK;
}

axi_status axi_operator_profile(axi_operator *op, int32_t enable) {
  if (!op) return AXI_ERR_ARG;
  if (enable) {
    if (!op->rec) op->rec = new (std::nothrow) OpProfiler;
    if (!op->rec) return AXI_ERR_ARG;
    op->rec->clear();
  }
  op->profiling = enable != 0;      // stopping keeps the record for axi_operator_profile_read
  return AXI_OK;
}

axi_status axi_operator_profile_read(axi_operator *op, axi_kernel_stat *h_stats) {
  if (!op || !h_stats) return AXI_ERR_ARG;
  for (int k = 0; k < AXI_KERNEL_KINDS; ++k) h_stats[k] = axi_kernel_stat{0, 0.0, 0.0};
  if (!op->rec) return AXI_OK;
  for (const auto &r : op->rec->recs) {
    if (r.kind < 0 || r.kind >= AXI_KERNEL_KINDS) continue;
    float ms = 0.0f;
    if (cudaEventSynchronize(r.b) != cudaSuccess || cudaEventElapsedTime(&ms, r.a, r.b) != cudaSuccess)
      return AXI_ERR_CUDA;
    h_stats[r.kind].launches += 1;
    h_stats[r.kind].ms += ms;
    h_stats[r.kind].flops += r.flops;
  }
  return AXI_OK;
}

axi_status axi_operator_destroy(axi_operator *op) {
  if (!op) return AXI_OK;
  delete op->rec;
  if (op->side) {
    cudaStreamSynchronize(op->side);
    cudaStreamDestroy(op->side);
  }
  if (op->crit) {
    cudaStreamSynchronize(op->crit);
    cudaStreamDestroy(op->crit);
  }
  if (op->ev_panel) cudaEventDestroy(op->ev_panel);
  if (op->ev_rest) cudaEventDestroy(op->ev_rest);
  if (op->ev_fork) cudaEventDestroy(op->ev_fork);
  if (op->ev_join) cudaEventDestroy(op->ev_join);
  delete op;
  return AXI_OK;
}

}  // extern "C"
