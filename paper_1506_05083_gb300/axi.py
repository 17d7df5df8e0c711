"""Thin ctypes binding of libaxi_mfs.so (include/axi_mfs.h).

Argument marshalling only: every step of the path runs in the library's CUDA
kernels. PyTorch supplies device memory and the current stream. If the
library has not been built this module raises at first use; there is no
fallback implementation.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import List, Optional, Sequence

import math

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libaxi_mfs.so")

BC_NEUMANN, BC_TRANSMISSION = 0, 1
PREC_FP64, PREC_SPLIT_BF16 = 0, 1
PLAN_FULL_FILL_GRID = 1 << 16                   # or-ed into prec: every ring pair on all q nodes
PLAN_TSVD = 1 << 17                             # or-ed into prec: truncated-SVD form of A_n^+
SHAPE_POLAR, SHAPE_CUP = 0, 1
EVAL_POTENTIAL, EVAL_NORMAL_DERIV, EVAL_FAR_FIELD = 0, 1, 2
OK, ERR_ARG, ERR_SHAPE = 0, -1, -2              # axi_status values (include/axi_mfs.h)

_dp = C.POINTER(C.c_double)
_vp = C.c_void_p


def svd_jacobi(A: torch.Tensor, tol=None, max_sweeps=30, stream=None):
    """axi_svd_jacobi on a [n][m] complex128 CUDA tensor holding the m x n
    matrix column-major (transposed view of the rows; m >= n, so a Q from
    `Operator.q_matrix` needs at least as many wall rows as columns); A is
    overwritten with U Sigma. tol defaults to sqrt(m) times the double
    rounding unit. Returns (V as [n][n] column-major, sigma [n], sweeps)."""
    if A.dtype != torch.complex128 or not A.is_cuda or not A.is_contiguous() or A.dim() != 2:
        raise ValueError("svd_jacobi: A must be a contiguous complex128 CUDA tensor [n][m]")
    n, m = A.shape
    if tol is None:
        tol = math.sqrt(m) * 2.0 ** -52
    V = torch.empty((n, n), dtype=torch.complex128, device=A.device)
    sigma = torch.empty(n, dtype=torch.float64, device=A.device)
    sw = C.c_int32()
    _check(lib().axi_svd_jacobi(_dev(A), m, n, m, _dev(V), n, _dev(sigma), tol, max_sweeps, C.byref(sw),
                                _stream(stream)), "axi_svd_jacobi")
    return V, sigma, sw.value


def svd_solve(US: torch.Tensor, V: torch.Tensor, sigma: torch.Tensor, B: torch.Tensor, cutoff=1e-10,
              stream=None) -> torch.Tensor:
    """axi_svd_solve: X = V Sigma^+ U^H B (singular values at or below cutoff
    sigma_max dropped); US [n][m], V [n][n], B [nrhs][m] column-major views.
    Returns X as [nrhs][n]."""
    n, m = US.shape
    for t in (US, V, B):
        if t.dtype != torch.complex128 or not t.is_cuda or not t.is_contiguous():
            raise ValueError("svd_solve: complex128 contiguous CUDA tensors expected")
    if V.shape != (n, n) or B.dim() != 2 or B.shape[1] != m or sigma.numel() != n:
        raise ValueError("svd_solve: shapes do not match")
    nrhs = B.shape[0]
    X = torch.empty((nrhs, n), dtype=torch.complex128, device=US.device)
    W = torch.empty((nrhs, n), dtype=torch.complex128, device=US.device)
    _check(lib().axi_svd_solve(_dev(US), _dev(V), _dev(sigma), m, n, m, n, cutoff, _dev(B), m, nrhs, _dev(X),
                               n, _dev(W), _stream(stream)), "axi_svd_solve")
    return X


def matvec_c128(A: torch.Tensor, X: torch.Tensor, out=None, work=None, stream=None) -> torch.Tensor:
    """axi_matvec_c128: Y = A X for a column-major A held as [cols][ld >= rows]
    (the layout of `Operator.c_block`) and X [nrhs][cols]; rows = A's ld.
    Returns Y [nrhs][rows]."""
    cols, rows = A.shape
    nrhs = X.shape[0]
    for t in (A, X):
        if t.dtype != torch.complex128 or not t.is_cuda or not t.is_contiguous() or t.dim() != 2:
            raise ValueError("matvec_c128: contiguous complex128 CUDA matrices expected")
    if X.shape[1] != cols:
        raise ValueError("matvec_c128: X must be [nrhs][cols of A]")
    if out is None:
        out = torch.empty((nrhs, rows), dtype=torch.complex128, device=A.device)
    nb = C.c_size_t()
    _check(lib().axi_matvec_workspace_bytes(rows, cols, nrhs, C.byref(nb)), "axi_matvec_workspace_bytes")
    if work is None and nb.value:
        work = torch.empty(nb.value, dtype=torch.uint8, device=A.device)
    _check(lib().axi_matvec_c128(_dev(A), rows, rows, cols, _dev(X), cols, nrhs, _dev(out), out.shape[1],
                                 _dev(work), 0 if work is None else work.numel() * work.element_size(),
                                 _stream(stream)), "axi_matvec_c128")
    return out


def iter_combine(g, a, bt: torch.Tensor, d: torch.Tensor, p: int, out=None, stream=None) -> torch.Tensor:
    """axi_iter_combine: y = g + a - (B~ d carried to the ring nodes) for
    samples [W][rows][P] (g or a may be None: zero); bt the packed buffer of
    `Operator.btilde`, d [W][ldd >= (p+1)^2] the leading part of xi."""
    ref = g if g is not None else a
    if ref is None:
        raise ValueError("iter_combine: the sample shape comes from g or a")
    W, rows, P = ref.shape
    for t in [x for x in (g, a, d) if x is not None]:
        if t.dtype != torch.complex128 or not t.is_cuda or not t.is_contiguous():
            raise ValueError("iter_combine: contiguous complex128 CUDA tensors expected")
    for t in [x for x in (g, a) if x is not None]:
        if tuple(t.shape) != (W, rows, P):
            raise ValueError("iter_combine: g and a must have the same [W][rows][P] shape")
    if d.dim() != 2 or d.shape[0] != W:
        raise ValueError("iter_combine: d must be [W][ldd]")
    if out is None:
        out = torch.empty((W, rows, P), dtype=torch.complex128, device=ref.device)
    _check(lib().axi_iter_combine(W, rows, P, p, _dev(g), _dev(a), _dev(bt), bt.numel(), _dev(d),
                                  d.shape[1], _dev(out), _stream(stream)), "axi_iter_combine")
    return out


class Cell(C.Structure):
    """axi_cell: the unit cell of the periodizing rows Q (include/axi_mfs.h)."""
    _fields_ = [("kx", C.c_double), ("ky", C.c_double), ("ex", C.c_double), ("ey", C.c_double),
                ("z0", C.c_double), ("m1", C.c_int32), ("n0", C.c_int32), ("p", C.c_int32)]


def q_shape(cell: Cell):
    """axi_q_shape: (rows, cols, n_rb) of Q for the cell."""
    r, c, n = C.c_int64(), C.c_int64(), C.c_int64()
    _check(lib().axi_q_shape(C.byref(cell), C.byref(r), C.byref(c), C.byref(n)), "axi_q_shape")
    return r.value, c.value, n.value


def q_modes(cell: Cell) -> np.ndarray:
    """axi_q_modes: the Rayleigh-Bloch (m, n) of the a and b columns, [n_rb][2]."""
    _, _, n = q_shape(cell)
    out = np.zeros((max(n, 1), 2), dtype=np.int32)
    _check(lib().axi_q_modes(C.byref(cell), C.c_void_p(out.ctypes.data), n), "axi_q_modes")
    return out[:n]


class _Obstacle(C.Structure):
    _fields_ = [("bc", C.c_int32), ("M", C.c_int32), ("N", C.c_int32), ("P", C.c_int32),
                ("q", C.c_int32), ("k", C.c_double), ("k_minus", C.c_double),
                ("h_coll", _dp), ("h_src", _dp), ("h_src_ext", _dp)]


class _FactorView(C.Structure):
    _fields_ = [("rows", C.c_int32), ("cols", C.c_int32), ("D", C.c_int32), ("nb", C.c_int32),
                ("npanels", C.c_int32), ("d_A", _vp), ("d_tau", _vp), ("d_T", _vp)]


class _KernelStat(C.Structure):
    _fields_ = [("launches", C.c_int32), ("ms", C.c_double), ("flops", C.c_double)]


KERNEL_KINDS = ["fill", "panel", "update_next", "update_rest", "panel_digits", "r_digits",
                "apply_rhs", "apply_qh", "apply_trsm", "apply_out"]   # axi_kernel_kind order


class _SvdView(C.Structure):
    _fields_ = [("n", C.c_int32), ("D", C.c_int32), ("d_U", _vp), ("d_V", _vp),
                ("d_sigma", _vp), ("d_sweeps", _vp)]


class _Lattice(C.Structure):
    _fields_ = [("ex", C.c_double), ("ey", C.c_double)]


# (name, restype, argtypes); every entry point declared in include/axi_mfs.h
SIGNATURES = [
    ("axi_geometry", C.c_int, [C.c_int32, _dp, C.c_int32, C.c_int32, C.c_int32, C.c_double, _dp, _dp, _dp]),
    ("axi_choose_q", C.c_int, [C.c_int32, C.c_int32, C.c_int32, _dp, _dp, _dp, C.POINTER(C.c_int32)]),
    ("axi_fill_subgrid", C.c_int, [C.c_int32, C.c_int32, C.c_int32, C.c_int32, _dp, _dp,
                                   C.POINTER(C.c_uint8)]),
    ("axi_plan_create", C.c_int, [C.POINTER(_Obstacle), C.c_int32, C.c_int32, C.POINTER(_vp)]),
    ("axi_plan_workspace_bytes", C.c_int, [_vp, C.POINTER(C.c_size_t)]),
    ("axi_plan_shard", C.c_int, [_vp, C.c_int32, C.c_int32]),
    ("axi_plan_owned_modes", C.c_int, [_vp, C.c_int32, C.POINTER(C.c_uint8)]),
    ("axi_plan_set_tuning", C.c_int, [_vp, C.c_char_p]),
    ("axi_plan_get_tuning", C.c_int, [_vp, C.c_char_p, C.c_size_t]),
    ("axi_operator_autotune", C.c_int, [_vp, C.c_int32, _vp, C.c_char_p, C.c_size_t]),
    ("axi_build_operator", C.c_int, [_vp, _vp, C.c_size_t, _vp, C.POINTER(_vp)]),
    ("axi_refactor_operator", C.c_int, [_vp, _vp]),
    ("axi_refactor_operator_modes", C.c_int, [_vp, C.POINTER(_vp), _vp]),
    ("axi_diag_wait_timeout", C.c_int, [_vp, C.c_int64, _vp]),
    ("axi_fill_modes", C.c_int, [_vp, C.c_int32, _vp, _vp]),
    ("axi_btilde_count", C.c_int, [_vp, C.c_int32, C.c_int32, C.POINTER(C.c_size_t)]),
    ("axi_q_shape", C.c_int, [_vp, C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
    ("axi_q_modes", C.c_int, [_vp, _vp, C.c_int64]),
    ("axi_fill_q", C.c_int, [_vp, C.c_int32, _vp, _vp, C.c_int64, _vp]),
    ("axi_c_shape", C.c_int, [_vp, C.c_int32, _vp, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
    ("axi_fill_c", C.c_int, [_vp, C.c_int32, _vp, _vp, C.c_int64, _vp]),
    ("axi_svd_jacobi", C.c_int, [_vp, C.c_int64, C.c_int64, C.c_int64, _vp, C.c_int64, _vp, C.c_double,
                                 C.c_int32, C.POINTER(C.c_int32), _vp]),
    ("axi_svd_solve", C.c_int, [_vp, _vp, _vp, C.c_int64, C.c_int64, C.c_int64, C.c_int64, C.c_double, _vp,
                                C.c_int64, C.c_int64, _vp, C.c_int64, _vp, _vp]),
    ("axi_fill_btilde", C.c_int, [_vp, C.c_int32, C.c_int32, _vp, C.c_size_t, _vp]),
    ("axi_matvec_workspace_bytes", C.c_int, [C.c_int64, C.c_int64, C.c_int32, C.POINTER(C.c_size_t)]),
    ("axi_matvec_c128", C.c_int, [_vp, C.c_int64, C.c_int64, C.c_int64, _vp, C.c_int64, C.c_int32, _vp,
                                  C.c_int64, _vp, C.c_size_t, _vp]),
    ("axi_iter_combine", C.c_int, [C.c_int32, C.c_int32, C.c_int32, C.c_int32, _vp, _vp, _vp, C.c_size_t,
                                   _vp, C.c_int64, _vp, _vp]),
    ("axi_gmres_workspace_bytes", C.c_int, [C.c_int64, C.c_int32, C.c_int32, C.POINTER(C.c_size_t)]),
    ("axi_gmres_create", C.c_int, [C.c_int64, C.c_int32, C.c_int32, C.c_int32, C.c_double, _vp, C.c_size_t,
                                   C.POINTER(_vp)]),
    ("axi_gmres_destroy", C.c_int, [_vp]),
    ("axi_gmres_iterate", C.c_int, [_vp, _vp, _vp, C.POINTER(C.c_int32), C.POINTER(_vp), C.POINTER(_vp),
                                    _vp]),
    ("axi_gmres_result", C.c_int, [_vp, C.POINTER(C.c_int32), C.POINTER(C.c_double), C.POINTER(C.c_int32)]),
    ("axi_vec_scale", C.c_int, [C.c_int64, C.c_double, _vp, _vp]),
    ("axi_operator_factors", C.c_int, [_vp, C.c_int32, C.POINTER(_FactorView)]),
    ("axi_operator_svd", C.c_int, [_vp, C.c_int32, C.POINTER(_SvdView)]),
    ("axi_incident_planewaves", C.c_int, [_vp, C.c_int32, C.c_int32, _vp, _vp, _vp]),
    ("axi_apply_workspace_bytes", C.c_int, [_vp, C.c_int32, C.c_int32, C.POINTER(C.c_size_t)]),
    ("axi_apply_operator", C.c_int, [_vp, C.c_int32, C.c_int32, _vp, _vp, _vp, _vp, C.c_size_t, _vp]),
    ("axi_apply_operator_noalloc", C.c_int, [_vp, C.c_int32, C.c_int32, _vp, _vp, _vp, _vp]),
    ("axi_noalloc_scratch_bytes", C.c_size_t, []),
    ("axi_diag_sincos", C.c_int, [_vp, C.c_int32, _vp, _vp, _vp]),
    ("axi_diag_sincos_table", C.c_int, [_vp, C.c_int32, _vp, _vp, _vp]),
    ("axi_diag_sincos_fixed", C.c_int, [_vp, C.c_int32, _vp, _vp, _vp]),
    ("axi_eval_field", C.c_int, [_vp, C.c_int32, C.c_int32, _vp, C.c_int32, _vp, _vp, C.c_int32,
                                 C.POINTER(_Lattice), _vp, _vp, _vp, C.c_size_t, _vp]),
    ("axi_near_image_workspace_bytes", C.c_int, [_vp, C.c_int32, C.c_int32, C.POINTER(_Lattice),
                                                 C.c_int32, C.POINTER(C.c_size_t)]),
    ("axi_near_image_sum", C.c_int, [_vp, C.c_int32, C.c_int32, _vp, C.POINTER(_Lattice), _vp,
                                     C.c_int32, _vp, _vp, C.c_size_t, _vp]),
    ("axi_operator_profile", C.c_int, [_vp, C.c_int32]),
    ("axi_operator_profile_read", C.c_int, [_vp, _vp]),
    ("axi_operator_status", C.c_int, [_vp]),
    ("axi_operator_destroy", C.c_int, [_vp]),
    ("axi_plan_destroy", C.c_int, [_vp]),
    ("axi_status_string", C.c_char_p, [C.c_int32]),
]

_lib = None


def lib():
    """Load libaxi_mfs.so; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with __graft_entry__.build()")
        L = C.CDLL(LIB_PATH)
        for name, res, args in SIGNATURES:
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


class AxiError(RuntimeError):
    def __init__(self, code, where):
        super().__init__(f"{where}: {lib().axi_status_string(code).decode()} ({code})")
        self.code = code


def _check(code, where):
    if code != 0:
        raise AxiError(code, where)


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(_dp)


def _dev(t: Optional[torch.Tensor]):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def geometry(shape: int, params: Sequence[float], M: int, N: int, tau: float):
    """axi_geometry: (coll [M][4], src [N][2], src_ext [N][2]) as numpy arrays."""
    p = np.ascontiguousarray(params, dtype=np.float64)
    coll = np.zeros((M, 4))
    src = np.zeros((N, 2))
    srcx = np.zeros((N, 2))
    _check(lib().axi_geometry(shape, _ptr(p), len(p), M, N, tau, _ptr(coll), _ptr(src), _ptr(srcx)),
           "axi_geometry")
    return coll, src, srcx


def choose_q(M, N, P, coll, src, src_ext=None) -> int:
    q = C.c_int32(0)
    coll = np.ascontiguousarray(coll, dtype=np.float64)
    src = np.ascontiguousarray(src, dtype=np.float64)
    sx = None if src_ext is None else np.ascontiguousarray(src_ext, dtype=np.float64)
    _check(lib().axi_choose_q(M, N, P, _ptr(coll), _ptr(src), None if sx is None else _ptr(sx),
                              C.byref(q)), "axi_choose_q")
    return q.value


class Plan:
    """A host-only plan (axi_plan_create) without device memory: for the
    mode partition of axi_plan_shard and other host queries."""

    def __init__(self, specs: List[ObstacleSpec], prec: int = PREC_FP64):
        self.specs = specs
        arr = (_Obstacle * len(specs))()
        for i, s in enumerate(specs):
            arr[i] = _Obstacle(s.bc, s.M, s.N, s.P, s.q, s.k, s.k_minus, _ptr(s.coll), _ptr(s.src),
                               _ptr(s.src_ext) if s.src_ext is not None else None)
        plan = C.c_void_p()
        _check(lib().axi_plan_create(arr, len(specs), prec, C.byref(plan)), "axi_plan_create")
        self._plan = plan

    def __del__(self):
        try:
            if getattr(self, "_plan", None):
                lib().axi_plan_destroy(self._plan)
        except Exception:
            pass

    def shard(self, rank: int, world: int):
        _check(lib().axi_plan_shard(self._plan, rank, world), "axi_plan_shard")

    def owned_modes(self, obs=0) -> np.ndarray:
        mask = np.zeros(self.specs[obs].P // 2 + 1, dtype=np.uint8)
        _check(lib().axi_plan_owned_modes(self._plan, obs,
                                          mask.ctypes.data_as(C.POINTER(C.c_uint8))),
               "axi_plan_owned_modes")
        return mask.astype(bool)


def gather_coefficients(coef: torch.Tensor, group=None) -> torch.Tensor:
    """Sum of the processes' coefficient arrays (each holds its owned modes,
    zeros elsewhere) in place: one all-reduce of the real view."""
    import torch.distributed as dist
    dist.all_reduce(torch.view_as_real(coef), op=dist.ReduceOp.SUM, group=group)
    return coef


def fill_subgrid(M, N, P, q, coll, src) -> np.ndarray:
    """axi_fill_subgrid: [M][N] azimuthal sub-grid stride of each ring pair's fill samples."""
    coll = np.ascontiguousarray(coll, dtype=np.float64)
    src = np.ascontiguousarray(src, dtype=np.float64)
    out = np.zeros((M, N), dtype=np.uint8)
    _check(lib().axi_fill_subgrid(M, N, P, q, _ptr(coll), _ptr(src),
                                  out.ctypes.data_as(C.POINTER(C.c_uint8))), "axi_fill_subgrid")
    return out


class ObstacleSpec:
    """Host description of one obstacle (arguments of axi_obstacle)."""

    def __init__(self, bc, M, N, P, q, k, k_minus, coll, src, src_ext=None):
        self.bc, self.M, self.N, self.P, self.q = int(bc), int(M), int(N), int(P), int(q)
        self.k, self.k_minus = float(k), float(k_minus)
        self.coll = np.ascontiguousarray(coll, dtype=np.float64)
        self.src = np.ascontiguousarray(src, dtype=np.float64)
        self.src_ext = None if src_ext is None else np.ascontiguousarray(src_ext, dtype=np.float64)

    @property
    def rows(self):
        return self.M * (2 if self.bc == BC_TRANSMISSION else 1)

    @property
    def cols(self):
        return self.N * (2 if self.bc == BC_TRANSMISSION else 1)


class Operator:
    """Plan + workspace + built operator (axi_plan_create / axi_build_operator)."""

    def __init__(self, specs: List[ObstacleSpec], prec: int = PREC_FP64, device="cuda",
                 stream=None, tuning: Optional[str] = None, shard=None):
        self.specs = specs
        arr = (_Obstacle * len(specs))()
        for i, s in enumerate(specs):
            arr[i] = _Obstacle(s.bc, s.M, s.N, s.P, s.q, s.k, s.k_minus, _ptr(s.coll), _ptr(s.src),
                               _ptr(s.src_ext) if s.src_ext is not None else None)
        plan = C.c_void_p()
        _check(lib().axi_plan_create(arr, len(specs), prec, C.byref(plan)), "axi_plan_create")
        self._plan = plan
        if tuning is not None:
            _check(lib().axi_plan_set_tuning(plan, tuning.encode()), "axi_plan_set_tuning")
        if shard is not None:                       # (rank, world)
            _check(lib().axi_plan_shard(plan, int(shard[0]), int(shard[1])), "axi_plan_shard")
        nb = C.c_size_t(0)
        _check(lib().axi_plan_workspace_bytes(plan, C.byref(nb)), "axi_plan_workspace_bytes")
        self.workspace = torch.empty(nb.value, dtype=torch.uint8, device=device)
        op = C.c_void_p()
        _check(lib().axi_build_operator(plan, _dev(self.workspace), nb.value, _stream(stream),
                                        C.byref(op)), "axi_build_operator")
        self._op = op

    def __del__(self):
        try:
            if getattr(self, "_op", None):
                lib().axi_operator_destroy(self._op)
            if getattr(self, "_plan", None):
                lib().axi_plan_destroy(self._plan)
        except Exception:
            pass

    def tuning(self) -> str:
        """axi_plan_get_tuning: the plan's schedule choices as JSON."""
        buf = C.create_string_buffer(512)
        _check(lib().axi_plan_get_tuning(self._plan, buf, 512), "axi_plan_get_tuning")
        return buf.value.decode()

    def set_tuning(self, json_text: str):
        """axi_plan_set_tuning (takes effect at the next build)."""
        _check(lib().axi_plan_set_tuning(self._plan, json_text.encode()), "axi_plan_set_tuning")

    def autotune(self, reps=3, stream=None) -> str:
        """axi_operator_autotune: time every candidate schedule, keep the fastest."""
        buf = C.create_string_buffer(512)
        _check(lib().axi_operator_autotune(self._op, reps, _stream(stream), buf, 512),
               "axi_operator_autotune")
        return buf.value.decode()

    def refactor(self, stream=None):
        _check(lib().axi_refactor_operator(self._op, _stream(stream)), "axi_refactor_operator")

    def profile(self, enable: bool):
        """axi_operator_profile: start (clearing the record) or stop per-launch timing."""
        _check(lib().axi_operator_profile(self._op, 1 if enable else 0), "axi_operator_profile")

    def profile_read(self) -> dict:
        """axi_operator_profile_read: {kind: (launches, ms, algorithmic flops)}."""
        arr = (_KernelStat * len(KERNEL_KINDS))()
        _check(lib().axi_operator_profile_read(self._op, C.cast(arr, C.c_void_p)),
               "axi_operator_profile_read")
        return {k: (arr[i].launches, arr[i].ms, arr[i].flops) for i, k in enumerate(KERNEL_KINDS)}

    def refactor_from_modes(self, modes, stream=None):
        """axi_refactor_operator_modes: factor the given [D][cols][rows] complex128
        device tensors (None = fill that obstacle as usual)."""
        arr = (_vp * len(self.specs))()
        for i, m in enumerate(modes):
            if m is not None:
                s = self.specs[i]
                if (tuple(m.shape) != (s.P // 2 + 1, s.cols, s.rows) or m.dtype != torch.complex128
                        or not m.is_contiguous() or m.device != self.workspace.device):
                    raise ValueError(f"modes[{i}] must be a contiguous complex128 tensor of shape "
                                     f"{(s.P // 2 + 1, s.cols, s.rows)} on {self.workspace.device}")
                arr[i] = m.data_ptr()
        _check(lib().axi_refactor_operator_modes(self._op, arr, _stream(stream)),
               "axi_refactor_operator_modes")

    def diag_wait_timeout(self, max_cycles: int, stream=None):
        """axi_diag_wait_timeout: a bounded device wait that runs out (status AXI_ERR_TIMEOUT)."""
        _check(lib().axi_diag_wait_timeout(self._op, int(max_cycles), _stream(stream)),
               "axi_diag_wait_timeout")

    def status(self) -> int:
        return lib().axi_operator_status(self._op)

    def fill_modes(self, obs=0, out=None, stream=None) -> torch.Tensor:
        s = self.specs[obs]
        if out is None:
            out = torch.empty((s.P // 2 + 1, s.cols, s.rows), dtype=torch.complex128,
                              device=self.workspace.device)
        _check(lib().axi_fill_modes(self._op, obs, _dev(out), _stream(stream)), "axi_fill_modes")
        return out

    def btilde(self, p, obs=0, out=None, stream=None):
        """axi_fill_btilde: the spherical-wave block B~ of degree p as a list of
        per-mode [p + 1 - n][rows] views (mode n = 0 .. min(P/2, p)) into one
        packed float64 buffer (returned second)."""
        n = C.c_size_t()
        _check(lib().axi_btilde_count(self._op, obs, p, C.byref(n)), "axi_btilde_count")
        if out is None:
            out = torch.empty(n.value, dtype=torch.float64, device=self.workspace.device)
        if out.dtype != torch.float64 or not out.is_contiguous() or out.numel() < n.value:
            raise ValueError("btilde: out must be a contiguous float64 tensor of the count's size")
        _check(lib().axi_fill_btilde(self._op, obs, p, _dev(out), out.numel(), _stream(stream)),
               "axi_fill_btilde")
        s = self.specs[obs]
        blocks, off = [], 0
        for m in range(min(s.P // 2, p) + 1):
            sz = (p + 1 - m) * s.rows
            blocks.append(out[off:off + sz].view(p + 1 - m, s.rows))
            off += sz
        return blocks, out

    def q_matrix(self, cell: Cell, obs=0, out=None, stream=None):
        """axi_fill_q: the periodizing rows Q for the cell as a [cols][rows]
        complex128 tensor (column-major Q)."""
        rows, cols, _ = q_shape(cell)
        if out is None:
            out = torch.empty((cols, rows), dtype=torch.complex128, device=self.workspace.device)
        if out.dtype != torch.complex128 or not out.is_contiguous() or out.shape[0] < cols \
                or out.shape[1] < rows:
            raise ValueError("q_matrix: out must be a contiguous complex128 [cols][ld >= rows] tensor")
        _check(lib().axi_fill_q(self._op, obs, C.byref(cell), _dev(out), out.shape[1], _stream(stream)),
               "axi_fill_q")
        return out

    def c_block(self, cell: Cell, obs=0, out=None, stream=None):
        """axi_fill_c: the C block for the cell as a [cols][rows] complex128
        tensor (column-major C; column (n mod P) N + j)."""
        r, c = C.c_int64(), C.c_int64()
        _check(lib().axi_c_shape(self._op, obs, C.byref(cell), C.byref(r), C.byref(c)), "axi_c_shape")
        if out is None:
            out = torch.empty((c.value, r.value), dtype=torch.complex128, device=self.workspace.device)
        if out.dtype != torch.complex128 or not out.is_contiguous() or out.shape[0] < c.value \
                or out.shape[1] < r.value:
            raise ValueError("c_block: out must be a contiguous complex128 [cols][ld >= rows] tensor")
        _check(lib().axi_fill_c(self._op, obs, C.byref(cell), _dev(out), out.shape[1], _stream(stream)),
               "axi_fill_c")
        return out

    def factors(self, obs=0):
        """(A [D][cols][rows], tau [D][cols], T [D][npanels][nb][nb] col-major) views."""
        v = _FactorView()
        _check(lib().axi_operator_factors(self._op, obs, C.byref(v)), "axi_operator_factors")
        base = self.workspace.data_ptr()

        def view(ptr, shape):
            off = ptr - base
            n = int(np.prod(shape))
            return self.workspace[off:off + 16 * n].view(torch.complex128).view(*shape)

        A = view(v.d_A, (v.D, v.cols, v.rows))
        tau = view(v.d_tau, (v.D, v.cols))
        T = view(v.d_T, (v.D, v.npanels, v.nb, v.nb))
        return A, tau, T, v.nb

    def svd(self, obs=0):
        """(U [D][n][n] col-major, V, sigma [D][n], sweeps [D]) views of a truncated-SVD operator."""
        v = _SvdView()
        _check(lib().axi_operator_svd(self._op, obs, C.byref(v)), "axi_operator_svd")
        base = self.workspace.data_ptr()

        def view(ptr, nbytes, dtype, shape):
            off = ptr - base
            return self.workspace[off:off + nbytes].view(dtype).view(*shape)

        n, D = v.n, v.D
        return (view(v.d_U, 16 * D * n * n, torch.complex128, (D, n, n)),
                view(v.d_V, 16 * D * n * n, torch.complex128, (D, n, n)),
                view(v.d_sigma, 8 * D * n, torch.float64, (D, n)),
                view(v.d_sweeps, 4 * D, torch.int32, (D,)))

    def incident(self, dirs: torch.Tensor, obs=0, stream=None) -> torch.Tensor:
        s = self.specs[obs]
        W = dirs.shape[0]
        f = torch.empty((W, s.rows, s.P), dtype=torch.complex128, device=dirs.device)
        _check(lib().axi_incident_planewaves(self._op, obs, W, _dev(dirs), _dev(f), _stream(stream)),
               "axi_incident_planewaves")
        return f

    def apply_scratch_bytes(self, W, obs=0) -> int:
        nb = C.c_size_t(0)
        _check(lib().axi_apply_workspace_bytes(self._op, obs, W, C.byref(nb)),
               "axi_apply_workspace_bytes")
        return nb.value

    def apply(self, f: torch.Tensor, obs=0, want_sigma=False, scratch=None, coef=None,
              sigma=None, stream=None):
        s = self.specs[obs]
        W = f.shape[0]
        dev = f.device
        if coef is None:
            coef = torch.empty((W, s.P, s.cols), dtype=torch.complex128, device=dev)
        if want_sigma and sigma is None:
            sigma = torch.empty((W, s.cols, s.P), dtype=torch.complex128, device=dev)
        need = self.apply_scratch_bytes(W, obs)
        if scratch is None:
            scratch = torch.empty(need, dtype=torch.uint8, device=dev)
        _check(lib().axi_apply_operator(self._op, obs, W, _dev(f), _dev(coef),
                                        _dev(sigma) if want_sigma else None, _dev(scratch),
                                        scratch.numel() * scratch.element_size(), _stream(stream)),
               "axi_apply_operator")
        return (coef, sigma) if want_sigma else coef

    def apply_noalloc(self, f: torch.Tensor, coef: torch.Tensor, sigma=None, obs=0, stream=None):
        """axi_apply_operator_noalloc into caller-provided coef (and sigma)."""
        s = self.specs[obs]
        W = f.shape[0]
        dev = self.workspace.device
        want = [(f, (W, s.rows, s.P), "f"), (coef, (W, s.P, s.cols), "coef")]
        if sigma is not None:
            want.append((sigma, (W, s.cols, s.P), "sigma"))
        for t, shape, name in want:
            if (tuple(t.shape) != shape or t.dtype != torch.complex128 or not t.is_contiguous()
                    or t.device != dev):
                raise ValueError(f"apply_noalloc: {name} must be a contiguous complex128 tensor "
                                 f"of shape {shape} on {dev}")
        code = lib().axi_apply_operator_noalloc(self._op, obs, W, _dev(f), _dev(coef),
                                                _dev(sigma), _stream(stream))
        _check(code, "axi_apply_operator_noalloc")

    def eval_field(self, coef: torch.Tensor, targets: torch.Tensor, kind=EVAL_FAR_FIELD, obs=0,
                   normals=None, lattice=None, dirs=None, scratch=None, stream=None):
        s = self.specs[obs]
        W = coef.shape[0]
        T = targets.shape[0]
        out = torch.empty((W, T), dtype=torch.complex128, device=coef.device)
        need = 16 * W * s.cols * s.P
        if scratch is None:
            scratch = torch.empty(need, dtype=torch.uint8, device=coef.device)
        lat = C.byref(_Lattice(*lattice)) if lattice is not None else None
        _check(lib().axi_eval_field(self._op, obs, W, _dev(coef), T, _dev(targets), _dev(normals),
                                    kind, lat, _dev(dirs), _dev(out), _dev(scratch),
                                    scratch.numel() * scratch.element_size(), _stream(stream)),
               "axi_eval_field")
        return out


def _near_bytes(op, obs, W, lattice, slices):
    nb = C.c_size_t(0)
    _check(lib().axi_near_image_workspace_bytes(op._op, obs, W, C.byref(_Lattice(*lattice)), slices,
                                                C.byref(nb)), "axi_near_image_workspace_bytes")
    return nb.value


def near_image_sum(op, coef: torch.Tensor, lattice, dirs: torch.Tensor, slices=6, obs=0,
                   out=None, scratch=None, stream=None):
    """axi_near_image_sum: [W][M*P] normal derivative of the eight phased images at the ring nodes."""
    s = op.specs[obs]
    W = coef.shape[0]
    if out is None:
        out = torch.empty((W, s.M * s.P), dtype=torch.complex128, device=coef.device)
    need = _near_bytes(op, obs, W, lattice, slices)
    if scratch is None:
        scratch = torch.empty(need, dtype=torch.uint8, device=coef.device)
    _check(lib().axi_near_image_sum(op._op, obs, W, _dev(coef), C.byref(_Lattice(*lattice)),
                                    _dev(dirs), slices, _dev(out), _dev(scratch),
                                    scratch.numel() * scratch.element_size(), _stream(stream)),
           "axi_near_image_sum")
    return out


def spec_from_obstacle(ob, q: Optional[int] = None) -> ObstacleSpec:
    """ObstacleSpec from a synth.Obstacle, discretised by axi_geometry."""
    coll, src, srcx = geometry(ob.shape, ob.params, ob.M, ob.N, ob.tau)
    if q is None:
        q = ob.q if ob.q else choose_q(ob.M, ob.N, ob.P, coll, src,
                                       srcx if ob.bc == BC_TRANSMISSION else None)
    return ObstacleSpec(ob.bc, ob.M, ob.N, ob.P, q, ob.k, ob.k_minus, coll, src,
                        srcx if ob.bc == BC_TRANSMISSION else None)


def periodic_iter_apply(op, g: torch.Tensor, lattice, dirs: torch.Tensor, C_blk: torch.Tensor,
                        US: torch.Tensor, V: torch.Tensor, sigma: torch.Tensor, bt: torch.Tensor, p: int,
                        cutoff=1e-10, near_slices=0, obs=0, want_coef=False, out=None, stream=None):
    """One application of eq. iter's operator, y = (I + A_else A_0^+ -
    B Q^+ C A_0^+) g, on Neumann boundary samples g [W][M][P]: the operator's
    apply, the near-image sum (FP64 direct for near_slices 0, else split into
    that many digits on tensor cores), C eta, the SVD solve with Q's factors
    (US, V, sigma of `svd_jacobi`) and the combine, each through its own C
    entry point on `stream`. C_blk from `Operator.c_block`, bt from
    `Operator.btilde` (degree p). Returns y [W][M][P] (and A_0^+ g, [W][P][N],
    when want_coef)."""
    W = g.shape[0]
    coef = op.apply(g, obs=obs, stream=stream)                                 # [W][P][N]
    a = near_image_sum(op, coef, lattice, dirs, slices=near_slices, obs=obs, stream=stream)
    c = matvec_c128(C_blk, coef.view(W, -1), stream=stream)                   # [W][8 M1^2]
    xi = svd_solve(US, V, sigma, c, cutoff=cutoff, stream=stream)              # [W][nQ]
    y = iter_combine(g, a.view(g.shape), bt, xi, p, out=out, stream=stream)
    return (y, coef) if want_coef else y


def gmres(apply_fn, b: torch.Tensor, tol=1e-12, restart=40, max_iter=400, stream=None):
    """axi_gmres_*: solve A x_w = b_w for every wave w of b [W][...] (complex128,
    CUDA) by restarted GMRES from x = 0; apply_fn(v, out) writes A v into out
    (both shaped like b). Returns (x, iterations, relative residuals,
    converged flags)."""
    if b.dtype != torch.complex128 or not b.is_cuda or not b.is_contiguous():
        raise ValueError("gmres: b must be a contiguous complex128 CUDA tensor")
    W = b.shape[0]
    n = b[0].numel()
    x = torch.empty_like(b)
    nb = C.c_size_t()
    _check(lib().axi_gmres_workspace_bytes(n, W, restart, C.byref(nb)), "axi_gmres_workspace_bytes")
    work = torch.empty(nb.value, dtype=torch.uint8, device=b.device)
    g = C.c_void_p()
    _check(lib().axi_gmres_create(n, W, restart, max_iter, tol, _dev(work), nb.value, C.byref(g)),
           "axi_gmres_create")
    blk = 16 * W * n

    def view(ptr):
        if ptr == x.data_ptr():
            return x
        off = ptr - work.data_ptr()
        if off < 0 or off + blk > nb.value:
            raise RuntimeError("gmres: the driver asked for a block outside its buffers")
        return work[off:off + blk].view(torch.complex128).view(b.shape)

    try:
        need, din, dout = C.c_int32(), C.c_void_p(), C.c_void_p()
        while True:
            _check(lib().axi_gmres_iterate(g, _dev(b), _dev(x), C.byref(need), C.byref(din), C.byref(dout),
                                           _stream(stream)), "axi_gmres_iterate")
            if not need.value:
                break
            apply_fn(view(din.value), view(dout.value))
        its = (C.c_int32 * W)()
        rel = (C.c_double * W)()
        conv = (C.c_int32 * W)()
        _check(lib().axi_gmres_result(g, its, rel, conv), "axi_gmres_result")
    finally:
        lib().axi_gmres_destroy(g)
    return x, list(its), list(rel), [bool(c) for c in conv]


def periodic_solve(op, f: torch.Tensor, lattice, dirs: torch.Tensor, C_blk: torch.Tensor, US: torch.Tensor,
                   V: torch.Tensor, sigma: torch.Tensor, bt: torch.Tensor, p: int, cutoff=1e-10, near_slices=0,
                   tol=1e-12, restart=40, max_iter=400, obs=0, stream=None):
    """Eq. iter solved by GMRES for Neumann boundary samples f [W][M][P], then
    eta = A_0^+ eta~ and xi = -Q^+ C eta (Sec. 4.2). Returns (eta~ [W][M][P],
    eta [W][P][N], xi [W][nQ], iterations, relative residuals, converged)."""
    def apply_fn(v, out):
        periodic_iter_apply(op, v, lattice, dirs, C_blk, US, V, sigma, bt, p, cutoff=cutoff,
                            near_slices=near_slices, obs=obs, out=out, stream=stream)

    et, its, rel, conv = gmres(apply_fn, f, tol=tol, restart=restart, max_iter=max_iter, stream=stream)
    eta = op.apply(et, obs=obs, stream=stream)
    W = f.shape[0]
    c = matvec_c128(C_blk, eta.view(W, -1), stream=stream)
    xi = svd_solve(US, V, sigma, c, cutoff=cutoff, stream=stream)
    _check(lib().axi_vec_scale(xi.numel(), -1.0, _dev(xi), _stream(stream)), "axi_vec_scale")
    return et, eta, xi, its, rel, conv
