/*
 * axi_mfs.h -- C ABI of the GB300 one-obstacle MFS solution operator.
 *
 * The library builds and applies the solution operator A_0^+ of the
 * axisymmetric method of fundamental solutions (Liu & Barnett, "Efficient
 * numerical solution of acoustic scattering from doubly-periodic arrays of
 * axisymmetric objects", arXiv:1506.05083):
 *
 *   build_operator : for every distinct azimuthal mode n = 0..P/2, fill the
 *                    modal MFS matrix by the q-node trapezoid rule over
 *                    azimuth (Sec. 3.1, eq. ptr) and factor it by blocked
 *                    Householder QR (Sec. 3, eq. linsys: a backward-stable
 *                    dense least-squares solve per mode);
 *   apply_operator : FFT of boundary data to modes (eq. fhatquad), Q^H and
 *                    triangular solve per mode (Sec. 4.2, never an explicit
 *                    inverse), optional inverse FFT to point strengths
 *                    (Sec. 4.1);
 *   eval_field     : scattered potential, normal derivative or far field of
 *                    the coefficients, optionally summed over the eight
 *                    phased nearest lattice images (Sec. 4.1, A_else).
 *
 * Conventions (all entry points):
 *   - Every call returns an axi_status; nothing aborts, throws or prints.
 *   - Device pointers ("d_") are borrowed: the caller allocates and frees
 *     them. Host pointers ("h_") are read during the call only.
 *   - Calls that take a `stream` (a cudaStream_t passed as void*, NULL = the
 *     legacy default stream) are asynchronous on that stream. Device-side
 *     errors are latched into a status word of the operator and reported by
 *     axi_operator_status() after the caller synchronises the stream.
 *   - Handles are not thread-safe; one handle must not be used from two
 *     host threads at once.
 *   - Complex numbers are interleaved (re, im) doubles, 16 bytes each.
 *   - Modes: coefficient and modal arrays store mode n, -P/2 < n <= P/2,
 *     at index n mod P (FFT order). The scattered field is
 *       u(rho, phi, z) = sum_n e^{+i n phi} sum_j A_n(rho, z; j) c_nj,
 *     which pairs mode n of the data with mode n of the coefficients; the
 *     ring kernel is even in n (A_n = A_{-n}), so modes +n and -n share
 *     one factorisation.
 */
#ifndef AXI_MFS_H
#define AXI_MFS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct { double re, im; } axi_c128;

typedef enum {
  AXI_OK = 0,
  AXI_ERR_ARG = -1,          /* NULL pointer or invalid enum                  */
  AXI_ERR_SHAPE = -2,        /* sizes violate P even, q even, q >= P, M >= N, */
                             /* or exceed the compiled limits                 */
  AXI_ERR_GEOMETRY = -3,     /* rho' <= 0, non-finite or coincident points    */
  AXI_ERR_WORKSPACE = -4,    /* workspace too small or misaligned             */
  AXI_ERR_CUDA = -5,         /* a CUDA runtime call failed                    */
  AXI_ERR_TIMEOUT = -6,      /* a bounded device-side wait expired            */
  AXI_ERR_NUMERIC = -7,      /* non-finite value met on the device            */
  AXI_ERR_UNSUPPORTED = -8   /* option not built into this library            */
} axi_status;

typedef enum { AXI_BC_NEUMANN = 0, AXI_BC_TRANSMISSION = 1 } axi_bc;

/* Arithmetic of the trailing-matrix updates of the QR and of the apply's
 * Q^H. Fill, Householder panels, T factors and triangular solves are native
 * FP64 in every mode. The `prec` argument of axi_plan_create is
 * AXI_PREC_FP64, or AXI_PREC_SPLIT_BF16 optionally or-ed with
 * AXI_PREC_SLICES(s), s in 4..8 (default 7): each FP64 value is scaled by a
 * power of two per row or column and cut into s signed 7-bit digits, exact in
 * BF16; digit products run on tensor cores with exact FP32 integer sums and
 * are recombined in FP64 (Ozaki scheme). s = 7 keeps 49 bits per value. */
typedef enum {
  AXI_PREC_FP64 = 0,
  AXI_PREC_SPLIT_BF16 = 1
} axi_precision;
#define AXI_PREC_SLICES(s) ((int32_t)(s) << 8)

/* Plan option or-ed into `prec`: evaluate every ring pair of the fill on all
 * q azimuthal nodes. By default each (collocation point, proxy ring) pair is
 * sampled on the coarsest of the sub-grids of q, q/2 and q/4 nodes (dividing
 * q/2) on which Theorem 1's rate for that pair, alpha = acosh(1 +
 * d^2/(2 rho rho')), still gives q_pair >= max(P, 37/alpha + P/2): the same
 * rule axi_choose_q applies to the closest pair, now per pair. Far pairs
 * converge faster (Sec. 3.1), so most pairs need a fraction of the nodes;
 * the sub-grid sum is the trapezoid rule with q_pair nodes, which agrees with
 * the q-node rule to rounding (measured: 3e-15 of max|A| on the cup). */
#define AXI_PLAN_FULL_FILL_GRID ((int32_t)1 << 16)

/* Plan option or-ed into `prec`: the truncated-SVD form of the operator
 * (Sec. 4.2, the paper's factorisation of each block for its preconditioner):
 * after the Householder QR A_n = Q R, every mode's N x N factor R is
 * decomposed as R = U_R Sigma V^H by one-sided Jacobi in FP64, and the apply
 * computes c = V Sigma^+ U_R^H (Q^H fhat_n)_{1:N}, Sigma^+ keeping the
 * singular values >= 1e-10 sigma_max (the paper's truncation), as two
 * products and a scaling: the pseudo-inverse is never formed. The workspace
 * holds U_R, V and Sigma per mode (2 N^2 + N numbers). A mode whose Jacobi
 * sweeps do not converge in 40 latches AXI_ERR_TIMEOUT. */
#define AXI_PLAN_TSVD ((int32_t)1 << 17)

typedef enum { AXI_SHAPE_POLAR = 0, AXI_SHAPE_CUP = 1 } axi_shape;

/*
 * axi_geometry -- discretise a generating curve (Sec. 3; Sec. 3.2 scheme (c);
 * Sec. 3.4 for the exterior proxies).
 *
 *   shape, h_params, n_params : AXI_SHAPE_POLAR with params {r0, a_1..a_J}:
 *       r(t) = r0 + sum_j a_j cos(j t), (rho, z) = r(t) (sin t, cos t);
 *     AXI_SHAPE_CUP with params {a, b} (Fig. 2(c)): r(t) = 1 - a erf((t-pi/2)/a),
 *       theta(t) = b - a + 2(1-(b-a)/pi) s_a(t-pi/2),
 *       s_a(x) = (a/sqrt(pi)) e^{-x^2/a^2} + x erf(x/a), (rho, z) = r (sin, cos)(theta).
 *   M, N       : collocation points t_m = pi(m-1/2)/M and proxies t_j = pi(j-1/2)/N.
 *   tau        : complexification distance; proxies are zeta(t_j + i s tau) with
 *                zeta = z + i rho and s = +-1 chosen so they fall inside the body.
 *   h_coll     : out, host [M][4] doubles (rho, z, n_rho, n_z), unit outward normal.
 *   h_src      : out, host [N][2] doubles (rho', z'), interior proxies.
 *   h_src_ext  : out, host [N][2] doubles, exterior proxies (-tau), or NULL.
 * Errors: AXI_ERR_ARG (NULL output, unknown shape), AXI_ERR_SHAPE (M<1, N<1),
 *         AXI_ERR_GEOMETRY (a proxy with rho' <= 0 or non-finite values).
 */
axi_status axi_geometry(int32_t shape, const double *h_params, int32_t n_params,
                        int32_t M, int32_t N, double tau,
                        double *h_coll, double *h_src, double *h_src_ext);

/*
 * axi_choose_q -- quadrature count of the ring-kernel fill from Theorem 1:
 * alpha_min = min over (m, j) of acosh(1 + d^2/(2 rho rho')); q is the
 * smallest even 2^a 3^b 5^c >= max(2P, 37/alpha_min + P/2) (e^{-alpha q}
 * ~ 1e-16 plus ~|n| extra nodes, as remarked after the theorem).
 *   h_coll [M][4], h_src [N][2] as produced by axi_geometry; h_src_ext may be
 *   NULL (Neumann). Writes *q. Errors: AXI_ERR_ARG, AXI_ERR_GEOMETRY.
 */
axi_status axi_choose_q(int32_t M, int32_t N, int32_t P, const double *h_coll,
                        const double *h_src, const double *h_src_ext, int32_t *q);

/*
 * axi_fill_subgrid -- per ring pair, the azimuthal sub-grid the fill samples
 * on (Sec. 3.1, Theorem 1 applied to each pair; see AXI_PLAN_FULL_FILL_GRID):
 * h_stride[m*N + j] = largest s in {4, 2, 1} with (q/2) mod s = 0 and
 * q/s >= max(P, 37/alpha_mj + P/2), alpha_mj = acosh(1 + d^2/(2 rho_m rho'_j)).
 *   h_coll [M][4], h_src [N][2] as from axi_geometry; h_stride : out, host [M][N].
 * Host only. Errors: AXI_ERR_ARG, AXI_ERR_SHAPE, AXI_ERR_GEOMETRY.
 */
axi_status axi_fill_subgrid(int32_t M, int32_t N, int32_t P, int32_t q, const double *h_coll,
                            const double *h_src, uint8_t *h_stride);

/* One obstacle of a batch. All pointers are host pointers read by
 * axi_plan_create only. */
typedef struct {
  int32_t bc;            /* axi_bc                                                */
  int32_t M, N, P, q;    /* P even >= 2, q even >= P, M >= N >= 1                 */
  double k;              /* exterior wavenumber > 0                               */
  double k_minus;        /* interior wavenumber (transmission), else ignored      */
  const double *h_coll;    /* [M][4] rho, z, n_rho, n_z                           */
  const double *h_src;     /* [N][2] interior proxies (rho' > 0)                  */
  const double *h_src_ext; /* [N][2] exterior proxies (transmission) or NULL      */
} axi_obstacle;

typedef struct axi_plan_s axi_plan;
typedef struct axi_operator_s axi_operator;

/*
 * axi_plan_create -- validate a batch of obstacles and lay out the device
 * workspace of its operator. Copies the geometry; the caller's arrays may be
 * freed afterwards. Per obstacle the operator holds, for D = P/2+1 distinct
 * modes, the packed QR factors of the rows x cols modal matrix (rows = M,
 * cols = N for Neumann; 2M x 2N for transmission, eq. trans), column-major
 * with leading dimension rows, plus reflector scalars and compact-WY T blocks.
 *   obs[n_obs] : obstacles; prec : axi_precision, optionally or-ed with
 *                AXI_PREC_SLICES(s) and AXI_PLAN_FULL_FILL_GRID; *plan : out.
 * Errors: AXI_ERR_ARG, AXI_ERR_SHAPE, AXI_ERR_GEOMETRY, AXI_ERR_UNSUPPORTED.
 */
axi_status axi_plan_create(const axi_obstacle *obs, int32_t n_obs, int32_t prec,
                           axi_plan **plan);

/*
 * Schedule tuning (the paper has no counterpart): the choices the build
 * makes that do not change what it computes, as a flat JSON object of
 * integers:
 *   "next_update"   0 auto, 1 native FP64, 2 BF16 digits (split plans) for
 *                   the next panel's columns of each step;
 *   "panel_cluster" 0 auto (by the number of (obstacle, mode) tasks), or 1,
 *                   2, 4 CTAs per mode for the Householder panels;
 *   "rest_grid"     trailing updates of split plans: 0 auto (2 where the
 *                   update can read Y^H digits, i.e. the panel wrote its
 *                   reflector exponents, else 4), 1 mma.sync persistent (one
 *                   CTA per SM), 2 the tcgen05 trailing update
 *                   (tensor-memory accumulators, 64 columns per CTA), 3 the
 *                   same with one CTA per SM (room beside it for a panel or
 *                   next-panel CTA), 4 mma.sync with one CTA per (task,
 *                   column tile);
 *   "panel_threads" 0 auto (256 threads when a panel of more than 128 rows
 *                   runs on one CTA, else 128), 128 or 256 threads per
 *                   panel CTA;
 *   "crit_stream"   0 the panels and next-panel updates on `stream`, 1 on
 *                   a stream of the operator with the device's highest
 *                   priority (forked from and joined back into `stream`);
 *   "fill_chunk_mb" split plans: 0 the plan's fill chunk (up to 512 MB of
 *                   sample digits per chunk of ring pairs), else at most
 *                   this many MB per chunk (0..4096), so that a chunk's
 *                   digits stay in L2 between the sample and transform
 *                   kernels;
 *   "next_cluster"  split plans' next-panel update: CTAs per mode, 0 auto
 *                   (4 when four per mode fit one per SM and the panel has
 *                   256 rows or more, else 2), or 1, 2, 4;
 *   "panel_fixed"   split plans' Householder panels: 0 auto (FP64), 1 FP64,
 *                   2 in 58-bit fixed point (exact integer sums, integer
 *                   updates, FP64 scalars; one CTA per mode, so with
 *                   panel_cluster 0 or 1; the build fails with AXI_ERR_CUDA
 *                   where a panel does not fit one CTA);
 *   "rest_start"    0 each step's trailing update starts as soon as the
 *                   panel (and its digits) is done, beside the next-panel
 *                   update; 1 it starts after the next-panel update, so that
 *                   it runs beside the next panel only;
 *   "apply_cluster" split plans' Q^H in axi_apply_operator: 0 auto (4 CTAs
 *                   per (mode, 32-column tile) when all of them fit in one
 *                   wave of two CTAs per SM, else 2), or 2, 4.
 * axi_plan_set_tuning parses such an object (unknown keys ignored, missing
 * keys kept; AXI_ERR_ARG on malformed input or values out of range);
 * axi_plan_get_tuning writes the current one into buf[n] (AXI_ERR_ARG if it
 * does not fit). axi_operator_autotune times every candidate schedule with
 * CUDA events on `stream` (one warm-up and `reps` builds each, reps in
 * 1..100; it synchronises the stream, so not under stream capture): first
 * the panel chain's choices together, then, for split plans, the next-panel
 * update's cluster, the fixed-point panel (128 and 256 threads) and the fill
 * chunk, each with the best so far ("rest_start" is left as given: its two
 * settings time alike with direct launches, but 1 is slower in a CUDA
 * graph). It keeps the fastest in the plan, rebuilds the
 * operator with it and, when json_out is
 * not NULL, writes the choice with its build time ("build_ms"), the number
 * of candidates timed and the number skipped because they cannot run on this
 * device or plan ("skipped"). Caching the result is the caller's: pass it back with
 * axi_plan_set_tuning before axi_build_operator.
 */
axi_status axi_plan_set_tuning(axi_plan *plan, const char *json);
axi_status axi_plan_get_tuning(const axi_plan *plan, char *buf, size_t n);

/*
 * axi_plan_shard -- restrict a plan to process `rank` of `world` (call before
 * axi_build_operator). The (obstacle, distinct mode) tasks are independent
 * (Sec. 3: the modal systems decouple), so they are split over the
 * processes by estimated cost, longest first (QR flops 8 rows cols^2 -
 * 8 cols^3/3 per task), each to the least loaded process; every process
 * computes the same assignment. The build fills every mode (the ring samples
 * are shared by all modes) but factors only the owned ones; the apply
 * leaves the coefficients of the other modes zero, so a sum over the
 * processes (one all-reduce of d_coef) assembles the full coefficients, and
 * point strengths or fields are then computed from those (axi_eval_field).
 * axi_plan_owned_modes writes the owned-mode mask of obstacle `obs` into
 * h_mask[D] (1 owned, 0 not). Errors: AXI_ERR_ARG.
 */
axi_status axi_plan_shard(axi_plan *plan, int32_t rank, int32_t world);
axi_status axi_plan_owned_modes(const axi_plan *plan, int32_t obs, uint8_t *h_mask);

/* Bytes of device workspace the plan needs (256-byte aligned base required). */
axi_status axi_plan_workspace_bytes(const axi_plan *plan, size_t *bytes);

/*
 * axi_build_operator -- fill and factor all distinct modes of all obstacles
 * (Sec. 3.1 eq. ptr; Sec. 3 eq. linsys, linsysb; Sec. 3.4 eq. trans).
 *   d_workspace, bytes : caller-owned device buffer of at least
 *                        axi_plan_workspace_bytes(); it holds the operator and
 *                        must outlive it.
 *   stream             : cudaStream_t (void*). The build is asynchronous.
 *   *op                : out, operator handle (owns no device memory). The
 *                        plan must outlive the operator, and a plan backs
 *                        one operator at a time.
 * Errors: AXI_ERR_ARG, AXI_ERR_WORKSPACE, AXI_ERR_CUDA.
 */
axi_status axi_build_operator(axi_plan *plan, void *d_workspace, size_t bytes,
                              void *stream, axi_operator **op);

/*
 * axi_refactor_operator -- re-run the fill and the factorisation of an
 * existing operator in place (same plan, same workspace). Issues kernel
 * launches only (no host copies, no allocation), so a caller may capture it
 * in a CUDA graph. Errors: AXI_ERR_ARG, AXI_ERR_CUDA.
 */
axi_status axi_refactor_operator(axi_operator *op, void *stream);

/* See axi_plan_set_tuning. Errors: AXI_ERR_ARG, AXI_ERR_CUDA. */
axi_status axi_operator_autotune(axi_operator *op, int32_t reps, void *stream, char *json_out,
                                 size_t n);

/*
 * axi_refactor_operator_modes -- factor given modal matrices instead of the
 * fill's (Sec. 3, eq. linsys): for each obstacle i with h_modes[i] != NULL,
 * the D matrices at device address h_modes[i] ([D][cols][rows], the layout
 * axi_fill_modes writes) are copied into the operator and factored; obstacles
 * with h_modes[i] == NULL are filled as usual. h_modes is a host array of
 * n_obs device pointers, read during the call. A non-finite entry shows as
 * AXI_ERR_NUMERIC from axi_operator_status after the stream is synchronised.
 * Asynchronous; no allocation. Errors: AXI_ERR_ARG, AXI_ERR_CUDA.
 */
axi_status axi_refactor_operator_modes(axi_operator *op, const axi_c128 *const *h_modes,
                                       void *stream);

/*
 * axi_fill_modes -- the fill step alone (Sec. 3.1, eq. ptr): write the D
 * distinct modal matrices of obstacle `obs` to d_out [D][cols][rows]
 * (column-major per mode; Neumann: A'_n; transmission: the 2x2 block of
 * eq. trans), leaving the operator's factors untouched.
 */
axi_status axi_fill_modes(const axi_operator *op, int32_t obs, axi_c128 *d_out, void *stream);

/*
 * The periodizing scheme's spherical-wave block B~ (Sec. 4, eq. urep; Sec.
 * 4.1, the B~ display): the modal boundary data of obstacle `obs` due to the
 * regular waves u_lm = j_l(k r) Y_lm(theta, phi), l = 0 .. p, |m| <= l
 * (Y_lm orthonormal with the Condon-Shortley phase, theta the polar angle of
 * the collocation point (rho, z), k the exterior wavenumber). Rows are those
 * of the operator's modal matrices: Neumann, M rows of the normal
 * derivative; transmission, 2M rows, values then normal derivatives. The
 * obstacle's axis is the expansion's z axis, so the mean over phi keeps
 * only m = n and B~ is block diagonal and real: mode n holds the columns
 * l = n .. p, mode -n is (-1)^n times mode n, every other entry is zero.
 *
 * axi_btilde_count writes the number of doubles of the packed blocks for
 * degree p (0 <= p <= AXI_BTILDE_MAX_DEGREE). axi_fill_btilde writes them to
 * d_out, a device buffer of at least that many doubles (8-byte aligned,
 * owned by the caller): for n = 0 .. min(P/2, p) in turn, the block of mode
 * n as a rows x (p + 1 - n) column-major array (column l - n holds degree
 * l). Enqueued on `stream`; a non-finite entry sets the operator's status
 * word (AXI_ERR_NUMERIC from axi_operator_status).
 * Errors: AXI_ERR_ARG (null pointers, obs or p out of range, count too
 * small), AXI_ERR_CUDA.
 */
#define AXI_BTILDE_MAX_DEGREE 255
axi_status axi_btilde_count(const axi_operator *op, int32_t obs, int32_t p, size_t *count);
axi_status axi_fill_btilde(const axi_operator *op, int32_t obs, int32_t p, double *d_out,
                           size_t count, void *stream);

/*
 * The periodizing rows Q of the full system (Sec. 4.1, eq. full) for the
 * spherical-wave and Rayleigh-Bloch unknowns [d; a; b] (Sec. 4, eqs. urep,
 * rb1-rb2), the obstacle's exterior wavenumber k. The unit cell is
 * [-ex/2, ex/2] x [-ey/2, ey/2] x [-z0, z0] around the obstacle; each face
 * carries the m1 x m1 product Gauss-Legendre nodes (node (a, b) = row
 * a m1 + b of each block: (y_a, z_b) on L and R, (x_a, z_b) on B and F,
 * (x_a, y_b) on T and D). The 8 m1^2 rows, in blocks of m1^2:
 *   u_R - alpha u_L, d_x u_R - alpha d_x u_L, u_F - beta u_B,
 *   d_y u_F - beta d_y u_B, u_T, d_z u_T, u_D, d_z u_D
 * (eqs. qp1-qp4, T-nD), alpha = e^{i kx ex}, beta = e^{i ky ey}. Columns:
 * the (p + 1)^2 regular waves j_l(k r) Y_lm (column l^2 + l + m; Y_lm as in
 * axi_fill_btilde), then the n_rb a's, then the n_rb b's over the Rayleigh-
 * Bloch wavevectors kappa = (kx + 2 pi m / ex, ky + 2 pi n / ey) with
 * |kappa| <= pi n0, ordered by m then n (axi_q_modes), k_z the principal
 * root of k^2 - |kappa|^2; the a's carry -e^{i kappa.(x, y)} on u_T and
 * -i k_z e^{...} on d_z u_T, the b's -e^{...} on u_D and +i k_z e^{...} on
 * d_z u_D, zero elsewhere.
 */
typedef struct {
  double kx, ky;   /* Bloch wavevector: k times the incident direction's x, y */
  double ex, ey;   /* lattice periods (> 0) */
  double z0;       /* half height of the cell (> 0), above the obstacle */
  int32_t m1;      /* Gauss nodes per face direction: even, 2 .. 64 */
  int32_t n0;      /* Rayleigh-Bloch cut |kappa| <= pi n0, n0 >= 0 */
  int32_t p;       /* spherical-wave degree, 0 .. AXI_BTILDE_MAX_DEGREE */
} axi_cell;

/* Rows, columns and Rayleigh-Bloch count of Q for `cell`; AXI_ERR_ARG when a
 * field is out of range (or the m range of the Rayleigh-Bloch set exceeds 128). */
axi_status axi_q_shape(const axi_cell *cell, int64_t *rows, int64_t *cols, int64_t *n_rb);
/* The Rayleigh-Bloch (m, n) pairs of the a and b columns, in order, into
 * h_mn[2 * n_rb] (host); AXI_ERR_ARG if cap < n_rb. */
axi_status axi_q_modes(const axi_cell *cell, int32_t *h_mn, int64_t cap);
/* Q of obstacle `obs` into d_out, column-major with leading dimension
 * ld >= rows (device memory owned by the caller, 16-byte aligned; every
 * entry of the rows x cols block is written). Enqueued on `stream`; a
 * non-finite entry sets the operator's status word.
 * Errors: AXI_ERR_ARG, AXI_ERR_CUDA. */
axi_status axi_fill_q(const axi_operator *op, int32_t obs, const axi_cell *cell, axi_c128 *d_out,
                      int64_t ld, void *stream);

/*
 * The C block of the full system (Sec. 4.1, eq. full; Neumann obstacles): the
 * rows of axi_fill_q applied to the ring part of eq. urep, u = sum_{n,j}
 * c_nj Phi^near_nj, Phi^near the 3 x 3 phased images of eq. Phinear with
 * alpha^a beta^b, Phi_nj(x) = (1/P) sum_s G_k(x, y_j(2 pi s / P))
 * e^{+i n 2 pi s / P} (the P point sources per ring of Sec. 4.1; the mode
 * sign of the operator's coefficients). Rows as axi_fill_q; columns in the
 * operator's coefficient order, column (n mod P) N + j. Between the walls of
 * a pair the near images cancel (Sec. 4.1): the discrepancy rows are formed
 * from the six distant ones, T and D from all nine.
 * axi_c_shape writes rows (8 m1^2) and columns (P N); axi_fill_c writes the
 * block column-major into d_out with leading dimension ld >= rows (caller-
 * owned device memory, 16-byte aligned). Enqueued on `stream`.
 * Errors: AXI_ERR_ARG, AXI_ERR_UNSUPPORTED (transmission obstacles),
 * AXI_ERR_CUDA.
 */
axi_status axi_c_shape(const axi_operator *op, int32_t obs, const axi_cell *cell, int64_t *rows,
                       int64_t *cols);
axi_status axi_fill_c(const axi_operator *op, int32_t obs, const axi_cell *cell, axi_c128 *d_out,
                      int64_t ld, void *stream);

/*
 * Q^+ through the SVD (Sec. 4.2: the periodizing rows Q are inverted by
 * their singular value decomposition), for any dense complex matrix with at
 * least as many rows as columns. For Q (8 m1^2 rows, (p + 1)^2 + 2 n_rb
 * columns; axi_q_shape) that asks for enough wall nodes: the paper's m1 of
 * about 4 nodes per wavelength across a face keeps Q tall.
 *
 * axi_svd_jacobi: one-sided (Hestenes) Jacobi SVD of the m x n matrix d_A
 * (m >= n >= 1, column-major, leading dimension lda >= m), in place: on
 * return d_A holds U Sigma (orthogonal columns), d_V (n x n, ldv >= n) the
 * right singular vectors and d_sigma[n] the singular values (column norms
 * of U Sigma, unsorted), so that A = (U Sigma) V^H. A sweep orders the
 * columns by decreasing norm (d_sigma holds that order during the call) and
 * rotates every column pair once (n' - 1 rounds of n'/2 disjoint pairs,
 * n' = n rounded up to even); the sweeps stop when every pair's |x^H y| / (||x|| ||y||) is at
 * most tol (e.g. 1e-15), after at most max_sweeps. *sweeps receives the
 * number run. The call synchronises `stream` after every sweep (not under
 * stream capture); calls that overlap on one device share the convergence
 * word. Device buffers are the caller's, 16-byte aligned (8 for d_sigma).
 * Errors: AXI_ERR_ARG, AXI_ERR_NUMERIC (not converged in max_sweeps, or a
 * non-finite value), AXI_ERR_CUDA.
 *
 * axi_svd_solve: X = V Sigma^+ U^H B with the singular values at or below
 * cutoff * sigma_max dropped, from axi_svd_jacobi's output (d_US = d_A after
 * the call): B is m x nrhs (ldb >= m), X is n x nrhs (ldx >= n), d_work
 * holds n * nrhs complex values. Enqueued on `stream`.
 * Errors: AXI_ERR_ARG, AXI_ERR_CUDA.
 */
axi_status axi_svd_jacobi(axi_c128 *d_A, int64_t m, int64_t n, int64_t lda, axi_c128 *d_V, int64_t ldv,
                          double *d_sigma, double tol, int32_t max_sweeps, int32_t *sweeps,
                          void *stream);
axi_status axi_svd_solve(const axi_c128 *d_US, const axi_c128 *d_V, const double *d_sigma, int64_t m,
                         int64_t n, int64_t lda, int64_t ldv, double cutoff, const axi_c128 *d_B,
                         int64_t ldb, int64_t nrhs, axi_c128 *d_X, int64_t ldx, axi_c128 *d_work,
                         void *stream);

/*
 * One application of the preconditioned periodic operator (Sec. 4.2, eq.
 * iter), y = (I + A_else A_0^+ - B Q^+ C A_0^+) g, is composed of
 *   coef = A_0^+ g                       axi_apply_operator
 *   a    = A_else coef                   axi_near_image_sum
 *   c    = C coef                        axi_matvec_c128 (C from axi_fill_c)
 *   xi   = Q^+ c                         axi_svd_solve (Q from axi_fill_q,
 *                                        its SVD from axi_svd_jacobi)
 *   y    = g + a - B xi                  axi_iter_combine (B~ from
 *                                        axi_fill_btilde)
 * with g, a and y boundary samples [W][M][P] (the operator's right-hand-side
 * layout), i.e. the paper's modal operator conjugated by the transform of
 * eq. fhatquad; a Krylov solve in either space yields the same eta.
 *
 * axi_matvec_c128: Y[w * ldy + r] = sum_c A[c * lda + r] X[w * ldx + c] for
 * a dense complex rows x cols matrix A (column-major, lda >= rows) and
 * 1 <= nrhs <= 16 vectors, all device memory owned by the caller and
 * 16-byte aligned. The
 * columns are split into slices whose partial sums are added in a fixed
 * order (results are reproducible run to run): d_work must hold
 * axi_matvec_workspace_bytes bytes (none for small matrices: d_work may then
 * be null). Enqueued on `stream`.
 * Errors: AXI_ERR_ARG (null pointers, sizes or leading dimensions out of
 * range, misaligned buffers), AXI_ERR_WORKSPACE (work too small),
 * AXI_ERR_CUDA.
 */
axi_status axi_matvec_workspace_bytes(int64_t rows, int64_t cols, int32_t nrhs, size_t *bytes);
axi_status axi_matvec_c128(const axi_c128 *d_A, int64_t lda, int64_t rows, int64_t cols,
                           const axi_c128 *d_X, int64_t ldx, int32_t nrhs, axi_c128 *d_Y, int64_t ldy,
                           void *d_work, size_t work_bytes, void *stream);

/*
 * axi_iter_combine: y = g + a - B xi for W waves of `rows` x P boundary
 * samples (layout [W][rows][P], P <= 1536). B xi is the spherical-wave part
 * d of xi (d_d + w * ldd, (p + 1)^2 entries in column order l^2 + l + m,
 * ldd >= (p + 1)^2) through B~ (d_btilde, the packed blocks of
 * axi_fill_btilde for the same rows, P and p; btilde_count its size in
 * doubles): the modal data fhat_n = sum_l B~_n[., l] d_{l,n} of the P modes
 * -P/2 < n <= P/2 (mode -n is (-1)^n times the block of n; modes |n| > p
 * are zero), carried to the nodes by f_l = sum_n fhat_n e^{2 pi i n l / P}.
 * d_g and d_a may be null (taken as zero); d_y may alias d_g or d_a. The
 * complex buffers are 16-byte aligned, d_btilde 8-byte aligned.
 * Enqueued on `stream`.
 * Errors: AXI_ERR_ARG (null pointers, sizes out of range, misaligned
 * buffers, btilde_count smaller than the packed blocks), AXI_ERR_CUDA.
 */
axi_status axi_iter_combine(int32_t W, int32_t rows, int32_t P, int32_t p, const axi_c128 *d_g,
                            const axi_c128 *d_a, const double *d_btilde, size_t btilde_count,
                            const axi_c128 *d_d, int64_t ldd, axi_c128 *d_y, void *stream);

/*
 * Restarted GMRES (Sec. 4.2: eq. iter is solved by a Krylov method) for W
 * independent systems A x_w = b_w of length n that share one operator, by
 * reverse communication: the library keeps the Krylov state and asks the
 * caller to apply A, so any composition of entry points can serve as A (for
 * eq. iter: the five calls listed above axi_matvec_c128).
 *
 * axi_gmres_workspace_bytes: device bytes for n, W and the restart length
 * (1..512): the (restart + 1) basis blocks of W x n complex values, one more
 * block and a few scalars per wave. axi_gmres_create binds a caller-owned,
 * 256-byte aligned device buffer of that size and the stopping rule:
 * ||b_w - A x_w|| <= tol ||b_w||, at most max_iter Arnoldi steps per wave.
 * The host state it allocates is released by axi_gmres_destroy (the device
 * buffer stays the caller's).
 *
 * axi_gmres_iterate(g, d_b, d_x, &need, &d_in, &d_out, stream): d_b and d_x
 * are [W][n] (16-byte aligned, not aliased). Starts from x = 0 on the first
 * call. When it returns with need = 1, the caller writes A applied to the W
 * vectors at d_in into d_out (both [W][n], inside the workspace or d_x; the
 * operator must map zero to zero: a converged wave is fed zeros) on
 * `stream`, then calls again with the same arguments; need = 0 means the
 * solve has ended and d_x holds the iterate. Arnoldi uses classical
 * Gram-Schmidt twice; a Hessenberg column is reduced by complex Givens
 * rotations on the host; each restart forms b - A x by one application.
 * The call synchronises `stream` (it reads the Arnoldi scalars).
 * axi_gmres_result writes, per wave, the Arnoldi steps taken, the last
 * relative residual (the true one at each restart, the Givens estimate in
 * between) and whether tol was met (any argument may be null).
 * Errors: AXI_ERR_ARG, AXI_ERR_WORKSPACE (buffer too small or misaligned),
 * AXI_ERR_NUMERIC (a non-finite residual: the solve stops), AXI_ERR_CUDA.
 *
 * axi_vec_scale: x *= alpha for `count` complex values (e.g. xi = -Q^+ C eta
 * from the SVD solve's output). Errors: AXI_ERR_ARG, AXI_ERR_CUDA.
 */
typedef struct axi_gmres axi_gmres;
axi_status axi_gmres_workspace_bytes(int64_t n, int32_t W, int32_t restart, size_t *bytes);
axi_status axi_gmres_create(int64_t n, int32_t W, int32_t restart, int32_t max_iter, double tol,
                            void *d_work, size_t work_bytes, axi_gmres **out);
axi_status axi_gmres_destroy(axi_gmres *g);
axi_status axi_gmres_iterate(axi_gmres *g, const axi_c128 *d_b, axi_c128 *d_x, int32_t *need_apply,
                             const axi_c128 **d_in, axi_c128 **d_out, void *stream);
axi_status axi_gmres_result(const axi_gmres *g, int32_t *h_iters, double *h_relres,
                            int32_t *h_converged);
axi_status axi_vec_scale(int64_t count, double alpha, axi_c128 *d_x, void *stream);

/* Device view of the packed factors of one obstacle (read-only). For mode d,
 * A + d*cols*rows is the rows x cols column-major array with R on and above
 * the diagonal (real diagonal) and the reflector vectors below it; tau + d*cols
 * holds the reflector scalars; T + (d*npanels + p)*nb*nb the nb x nb upper
 * triangular compact-WY factor of panel p (column-major), so that the panel's
 * reflectors multiply to I - V T V^H. */
typedef struct {
  int32_t rows, cols, D, nb, npanels;
  const axi_c128 *d_A, *d_tau, *d_T;
} axi_factor_view;

axi_status axi_operator_factors(const axi_operator *op, int32_t obs, axi_factor_view *view);

/* Device view of a truncated-SVD operator's R = U_R Sigma V^H (AXI_PLAN_TSVD):
 * for mode d, U_R and V are n x n column-major at d_U + d n^2 and d_V + d n^2,
 * sigma at d_sigma + d n (unsorted), and d_sweeps[d] the Jacobi sweeps taken.
 * AXI_ERR_UNSUPPORTED for other plans. */
typedef struct {
  int32_t n, D;
  const axi_c128 *d_U, *d_V;
  const double *d_sigma;
  const int32_t *d_sweeps;
} axi_svd_view;

axi_status axi_operator_svd(const axi_operator *op, int32_t obs, axi_svd_view *view);

/*
 * axi_incident_planewaves -- boundary data of W incident plane waves
 * u_i = e^{i k d.x} (eq. ui) on the rows x P ring nodes (rho_m, 2 pi l/P, z_m)
 * of obstacle `obs`: Neumann f = -du_i/dn (eq. neu); transmission
 * [-u_i; -du_i/dn] (eq. trans).
 *   d_dirs : device [W][3] unit directions d.
 *   d_f    : out, device [W][rows][P] complex.
 */
axi_status axi_incident_planewaves(const axi_operator *op, int32_t obs, int32_t W,
                                   const double *d_dirs, axi_c128 *d_f, void *stream);

/*
 * axi_apply_workspace_bytes -- scratch bytes axi_apply_operator needs for W
 * right-hand sides of obstacle `obs`: the RHS blocks ([D][2W][rows] complex)
 * and, for split-precision operators whose plan did not keep every panel's
 * reflector digits (plans whose digits would exceed 4 GB), those digits,
 * recomputed by each apply.
 */
axi_status axi_apply_workspace_bytes(const axi_operator *op, int32_t obs, int32_t W,
                                     size_t *bytes);

/*
 * axi_apply_operator -- apply A_0^+ of obstacle `obs` to W data sets
 * (eq. fhatquad with q = P; Sec. 4.2 application of the factors):
 *   fhat_n = (1/P) sum_l f_l e^{-2 pi i n l/P};  c_n = R^{-1} (Q^H fhat_n)_{1:cols}.
 *   d_f      : device [W][rows][P] samples on the ring nodes.
 *   d_coef   : out, device [W][P][cols], mode n at index n mod P.
 *   d_sigma  : out or NULL, device [W][cols][P] point strengths
 *              sigma_jl = (1/P) sum_n c_nj e^{2 pi i n l/P} (Sec. 4.1).
 *   d_scratch, scratch_bytes : >= axi_apply_workspace_bytes(op, obs, W).
 * Errors: AXI_ERR_ARG, AXI_ERR_WORKSPACE, AXI_ERR_CUDA.
 */
axi_status axi_apply_operator(const axi_operator *op, int32_t obs, int32_t W,
                              const axi_c128 *d_f, axi_c128 *d_coef, axi_c128 *d_sigma,
                              void *d_scratch, size_t scratch_bytes, void *stream);

/*
 * axi_apply_operator_noalloc -- axi_apply_operator for callers that cannot
 * allocate device memory at the time they apply the operator (for example a
 * host application that owns the GPU's memory budget and passes a plug-in
 * only its input and output buffers, or a latency-critical loop where a
 * cudaMalloc, which can synchronise the device, is not allowed).
 * The paper has no counterpart: this is a deployment variant of the apply.
 *
 * Same arguments and results as axi_apply_operator, without the scratch
 * buffer: the RHS blocks live in a static device array of
 * axi_noalloc_scratch_bytes() bytes (32 MiB) that every GPU loading this
 * library holds until the process exits. The call allocates nothing.
 *   - Sizes: returns AXI_ERR_WORKSPACE when axi_apply_workspace_bytes(op, obs, W)
 *     exceeds the static array (W > 79 for N=180, M=216, P=120; W > 26 for
 *     N=360, M=432, P=180). Split-precision plans that did not keep their
 *     reflector digits (over 4 GB of digits, e.g. the 64-obstacle batch) need
 *     hundreds of MB per apply and are always refused.
 *   - Device: the current device and the stream's device must be the one the
 *     operator was built on (AXI_ERR_ARG otherwise), because the library
 *     picks that device's array.
 *   - The first call on each device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current; make that first call
 *     before any stream capture. Calls after a cudaDeviceReset in the same
 *     process are not supported (the looked-up address would be stale).
 *   - All calls share the one array, which keeps the last call's contents:
 *     calls that overlap on the GPU (different streams, no ordering) race.
 *     Every element the apply reads is written first, so nothing needs
 *     clearing between calls.
 */
axi_status axi_apply_operator_noalloc(const axi_operator *op, int32_t obs, int32_t W,
                                      const axi_c128 *d_f, axi_c128 *d_coef,
                                      axi_c128 *d_sigma, void *stream);

/* Size in bytes of the static scratch used by axi_apply_operator_noalloc. */
size_t axi_noalloc_scratch_bytes(void);

typedef enum {
  AXI_EVAL_POTENTIAL = 0,   /* u(x)                                    */
  AXI_EVAL_NORMAL_DERIV = 1,/* du/dn_x, normals required              */
  AXI_EVAL_FAR_FIELD = 2    /* F(xhat), targets are unit directions   */
} axi_eval_kind;

/*
 * axi_eval_field -- evaluate the exterior scattered field of coefficients
 * d_coef [W][P][cols] of obstacle `obs` from its point strengths
 * (sigma over qe = P azimuthal nodes, Sec. 4.1):
 *   POTENTIAL     u(x)  = sum_{j,l} G_k(x, y_jl) sigma_jl
 *   NORMAL_DERIV  du/dn = sum_{j,l} dG_k/dn_x(x, y_jl) sigma_jl
 *   FAR_FIELD     F(xh) = (1/4pi) sum_{j,l} e^{-i k xh.y_jl} sigma_jl.
 * With lattice != NULL the sum runs over the eight phased nearest images
 * y_jl + a e_x + b e_y, (a, b) in {-1,0,1}^2 \ {(0,0)}, weighted by
 * alpha^a beta^b, alpha = e^{i k d_x e_x}, beta = e^{i k d_y e_y} (eq. bloch,
 * Sec. 4.1 A_else) with d read per wave from d_dirs [W][3].
 *   d_targets [T][3], d_normals [T][3] (NORMAL_DERIV), d_out [W][T].
 *   d_scratch : >= W * cols * P * 16 bytes (point strengths).
 */
typedef struct { double ex, ey; } axi_lattice;

axi_status axi_eval_field(const axi_operator *op, int32_t obs, int32_t W,
                          const axi_c128 *d_coef, int32_t T, const double *d_targets,
                          const double *d_normals, int32_t kind,
                          const axi_lattice *lattice, const double *d_dirs,
                          axi_c128 *d_out, void *d_scratch, size_t scratch_bytes,
                          void *stream);

/*
 * axi_near_image_sum -- A_else of Sec. 4.1 for one obstacle: the normal
 * derivative, at every ring node x_t = (rho_m, 2 pi l / P, z_m) with its
 * normal, of the eight phased nearest lattice images of the point sources
 * (P per proxy ring, strengths from d_coef as in axi_eval_field):
 *   U_w(x_t) = sum_{(a,b) != 0} alpha_w^a beta_w^b sum_s dG/dn_t(x_t, y_s + (a e_x, b e_y, 0)) sigma_w(s),
 *   alpha_w = e^{i k d_x e_x}, beta_w = e^{i k d_y e_y} (eq. bloch), d from d_dirs [W][3].
 *   d_coef  : device [W][P][cols] coefficients (exterior field = first N columns).
 *   slices  : 0 = native FP64 direct sum; 4..7 = kernel values and strengths
 *             split into that many BF16 digits, contracted on tensor cores
 *             (the lattice's 90-degree symmetry is used when e_x = e_y and 4 | P).
 *   d_out   : device [W][M*P], target index t = m*P + l.
 *   d_scratch, scratch_bytes : >= axi_near_image_workspace_bytes(); the split
 *             path stages kernel digits for blocks of whole target rings (~3 GB).
 * Errors: AXI_ERR_ARG, AXI_ERR_UNSUPPORTED (slices), AXI_ERR_WORKSPACE, AXI_ERR_CUDA.
 */
axi_status axi_near_image_workspace_bytes(const axi_operator *op, int32_t obs, int32_t W,
                                          const axi_lattice *lattice, int32_t slices,
                                          size_t *bytes);
axi_status axi_near_image_sum(const axi_operator *op, int32_t obs, int32_t W,
                              const axi_c128 *d_coef, const axi_lattice *lattice,
                              const double *d_dirs, int32_t slices, axi_c128 *d_out,
                              void *d_scratch, size_t scratch_bytes, void *stream);

/*
 * Kernel profiling (measurement support; the paper has no counterpart).
 * axi_operator_profile(op, 1) clears the record and starts timing every
 * launch class of later axi_refactor_operator / axi_apply_operator calls on
 * this operator with CUDA events on the launch's own stream (not allowed
 * while a stream is being captured); axi_operator_profile(op, 0) stops.
 * axi_operator_profile_read waits for the recorded events and writes, per
 * class, the number of launches, their summed device time and their summed
 * algorithmic FP64-equivalent flops (complex Householder: 16 (K - j) flops
 * per reflector j and column it updates, i.e. 8 M N^2 - 8 N^3/3 per mode;
 * apply: 16 rows cols - 8 cols^2 per right-hand side for Q^H, 4 cols^2 for
 * the triangular solve; fill and data movement count 0).
 */
typedef enum {
  AXI_KERNEL_FILL = 0,         /* ring samples + modal transform (all kernels)   */
  AXI_KERNEL_PANEL = 1,        /* Householder panel factorisation                */
  AXI_KERNEL_UPDATE_NEXT = 2,  /* update of the next panel's columns             */
  AXI_KERNEL_UPDATE_REST = 3,  /* update of the trailing columns beyond it       */
  AXI_KERNEL_PANEL_DIGITS = 4, /* split plans: reflector digits                  */
  AXI_KERNEL_R_DIGITS = 5,     /* split plans: digits of R for the apply         */
  AXI_KERNEL_APPLY_RHS = 6,    /* transform of the data to modes                 */
  AXI_KERNEL_APPLY_QH = 7,     /* Q^H on the right-hand sides                    */
  AXI_KERNEL_APPLY_TRSM = 8,   /* back substitution                              */
  AXI_KERNEL_APPLY_OUT = 9,    /* coefficient scatter and point strengths        */
  AXI_KERNEL_KINDS = 10
} axi_kernel_kind;
typedef struct { int32_t launches; double ms; double flops; } axi_kernel_stat;
axi_status axi_operator_profile(axi_operator *op, int32_t enable);
/* h_stats: host [AXI_KERNEL_KINDS]. Errors: AXI_ERR_ARG, AXI_ERR_CUDA. */
axi_status axi_operator_profile_read(axi_operator *op, axi_kernel_stat *h_stats);

/* Device status word of the operator (read after synchronising the stream). */
axi_status axi_operator_status(const axi_operator *op);

/* Release handles. Does not free the caller's workspace. NULL is accepted. */
axi_status axi_operator_destroy(axi_operator *op);
axi_status axi_plan_destroy(axi_plan *plan);

/* Static description of a status code. */
const char *axi_status_string(int32_t s);

/* axi_diag_sincos -- diagnostics, not a step of the method (the paper has no
 * counterpart): evaluates at n device doubles d_x the sin/cos routine the
 * ring-kernel samples use (Cody-Waite reduction and Taylor series, valid for
 * |x| < 2^20), writing d_sin[i], d_cos[i]. Lets a caller or a test compare it
 * with CUDA's sincos. Asynchronous on `stream`; AXI_ERR_ARG for n < 0 or
 * missing pointers; n = 0 does nothing. */
axi_status axi_diag_sincos(const double *d_x, int32_t n, double *d_sin, double *d_cos, void *stream);

/* axi_diag_sincos_table -- diagnostics, as axi_diag_sincos, for the table form
 * the fill's samples use: (cos, sin) of a multiple j of 2 pi / 1024 from a
 * 1024-entry table in shared memory, short Taylor series for the remainder,
 * angle addition (valid for |x| < 2^20). The first call on a device uploads
 * the table to a static device array (16 KB). Same arguments and errors. */
axi_status axi_diag_sincos_table(const double *d_x, int32_t n, double *d_sin, double *d_cos,
                                 void *stream);

/* axi_diag_sincos_fixed -- diagnostics, as axi_diag_sincos, for the
 * fixed-point form the split fill's samples use: the same reduction to a
 * multiple of 2 pi / 1024 in FP64, then the series and the angle addition in
 * 64-bit integers against a table with 62 fractional bits, one rounding to
 * double (valid for |x| < 2^20). Same arguments and errors. */
axi_status axi_diag_sincos_fixed(const double *d_x, int32_t n, double *d_sin, double *d_cos,
                                 void *stream);

/* axi_diag_wait_timeout -- diagnostics of the failure path of the library's
 * bounded device waits (the paper has no counterpart): one CTA allocates
 * tensor memory, waits on an mbarrier that nothing completes with the same
 * bounded wait the tcgen05 kernels use, limited to max_cycles SM clocks,
 * then latches AXI_ERR_TIMEOUT in the operator's status word, frees the
 * tensor memory and returns; the context stays usable and the next build
 * clears the word. max_cycles in [1, 2^34]. Errors: AXI_ERR_ARG, AXI_ERR_CUDA. */
axi_status axi_diag_wait_timeout(const axi_operator *op, int64_t max_cycles, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* AXI_MFS_H */
