// Internal types shared by the host API and the kernels. Not part of the ABI.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "../../include/axi_mfs.h"

namespace axi {

constexpr int kNB = 16;        // Householder panel width (columns per block reflector)
constexpr int kMaxModes = 128; // D = P/2 + 1 <= 128, i.e. P <= 254
constexpr int kMaxP = 254;
constexpr int kFillDigits = 8;        // digits of the split fill transform (both operands)
constexpr int kPanelSmemRows = 864;  // panels up to this many rows are factored in shared memory
constexpr int kPlanFullFillGrid = 1 << 16;   // AXI_PLAN_FULL_FILL_GRID
constexpr int kPlanTsvd = 1 << 17;           // AXI_PLAN_TSVD

// Schedule choices of a plan (axi_plan_set_tuning, axi_operator_autotune).
struct Tuning {
  int next_update = 0;    // 0 auto, 1 native FP64, 2 split digits (split plans)
  int panel_cluster = 0;  // 0 auto (by the number of tasks), else 1, 2 or 4 CTAs per mode
  int rest_grid = 0;      // split trailing update: 0 auto (2 where the update reads Y^H digits,
                          // else 4), 1 mma.sync persistent (one CTA per SM), 2 tcgen05 kernel,
                          // 3 the same with one CTA per SM (room for a critical-path CTA beside it),
                          // 4 mma.sync, one CTA per (task, column tile)
  int panel_threads = 0;  // 0 auto (256 on one CTA with more than 128 rows, else 128), 128, 256
  int crit_stream = 0;    // 0 the panel chain on the caller's stream, 1 on a stream of the
                          // operator with the device's highest priority
  int fill_chunk_mb = 0;  // split fill: 0 the plan's chunk (up to 512 MB of sample digits),
                          // else at most this many MB per chunk (small chunks stay in L2)
  int next_cluster = 0;   // split next-panel update: CTAs per mode, 0 auto (4 when every
                          // mode's four fit one per SM and the panel has 256 rows, else 2), 1, 2, 4
  int panel_fixed = 0;    // split plans' panel: 0 auto (FP64), 1 FP64, 2 fixed point (one CTA per
                          // mode)
  int rest_start = 0;     // trailing update of a step: 0 starts after the panel's digits (beside
                          // the next-panel update), 1 after the next-panel update (beside the
                          // next panel only)
  int apply_cluster = 0;  // split Q^H of the apply: CTAs per (mode, column tile) cluster,
                          // 0 auto (4 when every cluster fits in one wave of CTAs, else 2)
};

// Device status bits latched by kernels (OR-ed into ObsDev::status).
enum : int { kStatNonFinite = 1, kStatTimeout = 2 };

// Per-obstacle view of the operator in the caller's workspace (device side).
struct ObsDev {
  int M, N, P, q;         // discretisation
  int rows, cols;         // modal matrix size: M x N (Neumann), 2M x 2N (transmission)
  int D;                  // distinct modes n = 0..P/2
  int bc;                 // axi_bc
  int npanels;            // ceil(cols / kNB)
  int slices;             // 0: native FP64 updates; 4..8: BF16 digits per FP64 value
  double k, km;           // exterior / interior wavenumber
  const double *coll;     // [M][4] rho, z, n_rho, n_z
  const double *src;      // [N][2] interior proxies
  const double *srcx;     // [N][2] exterior proxies (transmission) or null
  const double *tab_cos;  // [q]   cos(2 pi r / q)
  const double *tab_s2;   // [q/2+1] sin^2(pi l / q)
  const double2 *tw_P;    // [P]   e^{-2 pi i r / P}
  const double2 *tab_ring;  // [1024] (cos, sin)(2 pi i / 1024), the fill samples' sin/cos table
  // [2][M][N] azimuthal sub-grid stride (1, 2 or 4) of each ring pair's
  // samples: interior proxies, then exterior proxies (transmission); the
  // fill evaluates nodes l = 0, s, 2s, .. only (Theorem 1 rate of the pair).
  const unsigned char *fill_sig;
  // [D] 1 for the modes this process factors and applies (axi_plan_shard);
  // the apply leaves the other modes' coefficients zero
  const unsigned char *mode_owned;
  double2 *A;             // [D][cols][rows] packed QR factors (column-major)
  double2 *tau;           // [D][cols] reflector scalars
  double2 *T;             // [D][npanels][kNB][kNB] compact-WY T blocks (col-major)
  int *status;            // device status word
  // split precision only: BF16 digits of the current panel's reflectors for
  // the trailing updates: two blocks per mode, used by alternate panel steps.
  // Block of 4*slices*kNB*kp entries: V^H digits [slices][re/im][kNB][kp]
  // (conjugated), then V row digits [slices][re/im][kp][kNB]; exponents
  // [kNB + kp] (per reflector column, then per row).
  unsigned short *vdig;
  int *vexp;
  int kp;                 // digit row stride: rows rounded up to a multiple of 64, + 64
  int dig_kept;           // 1: every panel's digits are kept for the apply (slot = panel)
  int dig_nslot;          // digit blocks per mode: npanels (kept) or 2 (QR steps alternate)
  // split precision only: [D][2][cols] largest |entry| key (IEEE bits) of each
  // trailing column over the next panel step's rows, written by one split
  // update and read by the next (alternating slots), so the trailing matrix
  // is not scanned for its exponents at every step.
  unsigned long long *ckey;
  // split precision only: digits of R's off-diagonal blocks for the back
  // substitution, written at the end of the build. Per mode, 32-column block
  // b (b >= 1) holds rb = r_digit_block_rows(b) rows starting at row offset
  // r_digit_rows_before(b): digits [slices][re/im][rb][32] (row i, column
  // 32 b + k), exponents [rb] (one per row of the block).
  unsigned short *rdig;
  int *rex;
  // split precision only: Y = V T of the current panel for the trailing
  // update (slots p mod 2): Y [D][2][kNB][kp] FP64, column maxima ykey
  // [D][2][kNB], digits of Y^H [D][2][slices][re/im][kNB][kp], exponents
  // yexp [D][2][kNB]
  double2 *ybuf;
  unsigned long long *ykey;
  unsigned short *ydig;
  int *yexp;
  // split precision only: the fill's transform as a digit GEMM (fill_mma.cu).
  // Folded length L, padded Lp (multiple of 32), MR rows per parity part;
  // cos-table digits [kFillDigits][2 MR][Lp] and row exponents [2 MR];
  // sample-digit scratch for fill_chunk_pairs ring pairs at a time.
  int fill_L, fill_Lp, fill_MR, fill_chunk_pairs;
  int fill_tc;            // 1: tcgen05 transform (fill_uses_tc), digit tiles in its layout
  int apply_cluster;      // host side only: Tuning::apply_cluster for the split Q^H launch
  const unsigned short *fill_cdig;
  const int *fill_cex;
  uint32_t *fill_gdig;
  int *fill_gex;
  // truncated-SVD plans (AXI_PLAN_TSVD): R = U_R Sigma V^H per mode
  int tsvd;
  double2 *svdU, *svdV;   // [D][cols][cols] column-major
  double *svdS;           // [D][cols]
  int *svdSweeps;         // [D] Jacobi sweeps taken
  int fft_nst;            // radices of P for the apply's FFTs (0: P has other prime factors)
  int fft_rad[8];
  const int *fft_perm;    // [P] position of output n after the in-place FFT
  int fft_nst_q;          // radices of q for the fill's FFT (0: direct cosine sums)
  int fft_sum_last_q;     // 1: the needed modes are sums over the last stage's blocks
  int fft_rad_q[8];
  const int *fft_perm_q;  // [q]
  const double2 *tw_q;    // [q] e^{-2 pi i r / q}
};

__host__ __device__ inline bool owns_mode(const ObsDev &o, int d) {
  return o.mode_owned == nullptr || o.mode_owned[d] != 0;
}

// Streaming multiprocessors of the current device (cached).
int sm_count();

// Optional per-launch timing (axi_operator_profile): while an entry point of
// a profiled operator runs, t_prof points at its recorder, and the launch
// sites bracket each launch class with prof_begin / prof_end, which record
// CUDA events on the launch's own stream and the launch's algorithmic
// FP64-equivalent flops (axi_kernel_kind numbers the classes).
struct KernelProfiler {
  virtual int begin(int kind, cudaStream_t st) = 0;
  virtual void end(int id, cudaStream_t st, double flops) = 0;
  virtual ~KernelProfiler() {}
};
extern thread_local KernelProfiler *t_prof;
inline int prof_begin(int kind, cudaStream_t st) { return t_prof ? t_prof->begin(kind, st) : -1; }
inline void prof_end(int id, cudaStream_t st, double flops = 0.0) {
  if (id >= 0 && t_prof) t_prof->end(id, st, flops);
}

// CUDA device an operator was built on (api.cu); -1 for a null handle.
int operator_device(const axi_operator *op);
// The operator's device status word (api.cu).
int *operator_status_word(const axi_operator *op);

// The split fill's transform runs on tcgen05 when its group sums stay exact
// in FP32 over the whole contraction (folded length Lp <= 448) and the
// accumulators of one parity fit tensor memory (MR <= 64 modes).
constexpr int kFillTcMaxLp = 448;
inline bool fill_uses_tc(int Lp, int MR) { return Lp <= kFillTcMaxLp && MR <= 64; }

// Rows of R above 32-column block b, rounded up to 64, and their running
// total over blocks 0..b-1 (sum of 64 ceil(j/2) for j < b = 64 floor(b^2/4)).
__host__ __device__ inline int r_digit_block_rows(int b) { return 64 * ((b + 1) / 2); }
__host__ __device__ inline size_t r_digit_rows_before(int b) { return (size_t)64 * ((size_t)b * b / 4); }

// Kernels of one factorisation step run side by side (panel and next-panel
// update on the critical path, digits and trailing update beside them). With
// the default carveout an SM sized for one kernel's shared memory can refuse
// the CTAs of another; asking for the largest shared-memory carveout lets
// them co-reside. Called once per kernel, outside stream capture.
template <typename Kernel>
inline void prefer_max_shared(Kernel *kernel) {
  (void)cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared);
}

// Raise a kernel's dynamic shared-memory limit only when a launch needs more
// than any earlier launch did. The first (largest) request happens when an
// operator is built, so later launches made under stream capture issue no
// attribute calls.
template <typename Kernel>
inline cudaError_t ensure_dynamic_smem(Kernel *kernel, size_t bytes, size_t &granted) {
  if (bytes <= 48 * 1024 || bytes <= granted) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) granted = bytes;
  return e;
}

// Launch wrappers (each returns the cudaError_t of its launch).
// fill_mma.cu: the split-precision transform of the fill
// chunk_mb > 0 caps the ring pairs per chunk at that many MB of sample digits
// (Tuning::fill_chunk_mb; the plan's chunk otherwise).
cudaError_t launch_fill_mma(const ObsDev *d_obs, const ObsDev &h, int oi, double2 *out,
                            int ld_rows, int ld_cols, int chunk_mb, cudaStream_t st);
size_t fill_gemm_smem(int MR);
cudaError_t launch_fill(const ObsDev *d_obs, const ObsDev &h_obs, int obs_index,
                        double2 *out, int ld_rows, int ld_cols, cudaStream_t st, int chunk_mb = 0);
// Sets *digits_written when the panel kernel also wrote the exponents of the
// panel's reflector columns, so that launch_vdigits can write the digits
// (split plans, panels in shared memory).
// cluster: CTAs per mode for shared-memory panels (0 = by the number of tasks).
// fixed: split plans' panel arithmetic, 0 and 1 FP64, 2 fixed point
// (qr_panel_fx.cu; one CTA per mode, so only with cluster 0 or 1).
cudaError_t launch_qr_panel(const ObsDev *d_obs, const int *d_task_obs, const int *d_task_mode,
                            int ntasks, int panel, int max_panel_rows, int slices, int cluster,
                            int threads, int fixed, cudaStream_t st, bool *digits_written);
// The spherical-wave block B~ of the periodizing scheme (periodize.cu):
// doubles of the packed mode blocks for degree p, and their fill.
size_t btilde_count(const ObsDev &h, int p);
cudaError_t launch_btilde(const ObsDev *d_obs, const ObsDev &h, int oi, int p, double *out,
                          cudaStream_t st);
// The periodizing rows Q (periodize.cu): shape and Rayleigh-Bloch modes of a
// cell (false when a field is out of range), and the fill.
bool q_shape(const axi_cell &c, long long &rows, long long &cols, long long &nrb);
bool q_modes(const axi_cell &c, int *mn, long long cap);
cudaError_t launch_q(const ObsDev *d_obs, const ObsDev &h, int oi, const axi_cell &c, double2 *out,
                     long long ld, cudaStream_t st);
// Dense SVD for Q^+ (svd_dense.cu): one-sided Jacobi (A <- U Sigma, V, sigma;
// *converged false when max_sweeps ran out) and the truncated solve.
cudaError_t svd_jacobi(double2 *A, long long m, long long n, long long lda, double2 *V, long long ldv,
                       double *sigma, double tol, int max_sweeps, int *sweeps, bool *converged,
                       cudaStream_t st);
cudaError_t svd_solve(const double2 *US, const double2 *V, const double *sigma, long long m, long long n,
                      long long lda, long long ldv, double cutoff, const double2 *B, long long ldb,
                      long long nrhs, double2 *X, long long ldx, double2 *W, cudaStream_t st);
// The C block (periodize.cu; Neumann obstacles): shape for a cell, and the fill.
bool c_shape(const ObsDev &h, const axi_cell &c, long long &rows, long long &cols);
cudaError_t launch_c(const ObsDev *d_obs, const ObsDev &h, int oi, const axi_cell &c, double2 *out,
                     long long ld, cudaStream_t st);
// The fixed-point panel (qr_panel_fx.cu): whether a panel of `rows` rows fits
// one CTA of `threads` (128 or 256), and its launch.
bool panel_fx_fits(int rows, int threads);
cudaError_t launch_qr_panel_fx(const ObsDev *d_obs, const int *d_task_obs, const int *d_task_mode,
                               int ntasks, int panel, int max_panel_rows, int threads,
                               cudaStream_t st);
// Trailing update of panel step `panel`: the next panel's kNB columns (native
// FP64, critical path), and the columns beyond (split or FP64; col_off = kNB).
cudaError_t launch_qr_update_next(const ObsDev *d_obs, const int *d_task_obs,
                                  const int *d_task_mode, int ntasks, int panel, cudaStream_t st);
// Split plans: digits of panel p's reflectors over the whole GPU, after a
// panel kernel that wrote the reflector columns' exponents.
cudaError_t launch_vdigits(const ObsDev *d_obs, const int *d_task_obs, const int *d_task_mode,
                           int ntasks, int p, int kp_max, int slices, cudaStream_t st);
// Split plans: the next panel's columns in split precision, rows of each mode
// spread over a cluster (needs the panel's digits; max_rows = tallest panel).
cudaError_t launch_qr_update_next_split(const ObsDev *d_obs, const int *d_task_obs,
                                        const int *d_task_mode, int ntasks, int panel, int slices,
                                        int max_rows, int cluster, cudaStream_t st);
// use_y: the trailing update reads Y^H digits (launch_y_digits) and skips T^H W.
// rest_grid: Tuning::rest_grid.
cudaError_t launch_qr_update_rest(const ObsDev *d_obs, const int *d_task_obs,
                                  const int *d_task_mode, int ntasks, int panel, int slices,
                                  int max_rest_cols, int rest_grid, bool use_y, cudaStream_t st);
// The trailing update of split plans on tcgen05 (W' = Y^H X, X -= V W'),
// 64 columns per CTA; needs the Y^H digits.
cudaError_t launch_qr_update_tc(const ObsDev *d_obs, const int *d_task_obs, const int *d_task_mode,
                                int ntasks, int p, int slices, int max_rest_cols, bool one_per_sm,
                                cudaStream_t st);
// Y = V T of panel p and the digits of Y^H (split plans, after launch_vdigits).
cudaError_t launch_y_digits(const ObsDev *d_obs, const int *d_task_obs, const int *d_task_mode,
                            int ntasks, int p, int kp_max, int slices, cudaStream_t st);
int split_update_tile_cols();
cudaError_t launch_qr_update_split(const ObsDev *d_obs, const int *d_task_obs,
                                   const int *d_task_mode, int ntasks, int panel, int slices,
                                   int col_off, int ntiles, int max_cols, bool persistent,
                                   bool use_y, cudaStream_t st);
cudaError_t launch_apply_qh_split(const ObsDev *d_o, const ObsDev &h, double2 *X, int ncol,
                                  void *digit_scratch, cudaStream_t st);
size_t apply_digit_bytes(const ObsDev &h);
// trsm_split.cu: back substitution with its off-diagonal updates on tensor
// cores; R's digits are written once per build (launch_r_digits)
size_t r_digit_bytes(const ObsDev &h);
size_t r_exponent_bytes(const ObsDev &h);
cudaError_t launch_r_digits(const ObsDev *d_o, const ObsDev &h, cudaStream_t st);
cudaError_t launch_trsm_split(const ObsDev *d_o, const ObsDev &h, double2 *X, int ncol,
                              cudaStream_t st);
// Split plans apply Q^H with split digits from this many waves up (the
// cluster kernel is faster than the FP64 one at every batch size measured).
constexpr int kSplitApplyMinWaves = 1;
bool split_slices_supported(int slices);
// kp_max: the largest digit row stride (kp) over the tasks of the launch
cudaError_t launch_panel_digits(const ObsDev *d_obs, const int *d_task_obs, const int *d_task_mode,
                                int ntasks, int panel, int slices, int kp_max, cudaStream_t st);
// tsvd.cu: SVD of every mode's R (after the QR) and its truncated apply
cudaError_t launch_tsvd(const ObsDev *d_o, const ObsDev &h, cudaStream_t st);
cudaError_t launch_tsvd_apply(const ObsDev *d_o, const ObsDev &h, double2 *X, int ncol,
                              cudaStream_t st);
cudaError_t launch_incident(const ObsDev *d_o, const ObsDev &h_o, int W, const double *dirs,
                            double2 *f, cudaStream_t st);
cudaError_t launch_apply(const ObsDev *d_o, const ObsDev &h_o, int W, const double2 *f,
                         double2 *coef, double2 *sigma, double2 *X, void *digit_scratch,
                         cudaStream_t st);
cudaError_t launch_eval(const ObsDev *d_o, const ObsDev &h_o, int W, const double2 *sigma,
                        int T, const double *targets, const double *normals, int kind,
                        const axi_lattice *lat, const double *dirs, double2 *out,
                        cudaStream_t st);
cudaError_t launch_rhs_fft(const ObsDev *d_o, const ObsDev &h_o, int W, const double2 *f,
                           double2 *X, cudaStream_t st);
cudaError_t launch_point_fft(const ObsDev *d_o, const ObsDev &h_o, int W, const double2 *coef,
                             double2 *sigma, cudaStream_t st);
size_t near_image_scratch_bytes(const ObsDev &h, int W, double ex, double ey, int slices);
cudaError_t launch_near_image(const ObsDev *d_o, const ObsDev &h, int W, const double2 *coef,
                              double ex, double ey, const double *dirs, int slices, double2 *U,
                              void *scratch, cudaStream_t st);
cudaError_t launch_point_strengths(const ObsDev *d_o, const ObsDev &h_o, int W,
                                   const double2 *coef, double2 *sigma, cudaStream_t st);

}  // namespace axi
