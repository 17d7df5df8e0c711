"""Edge cases of the CUDA path, against the FP64 oracle.

* sizes without an FFT plan: P and q with the prime factor 7 take the direct
  transforms (fill by the folded cosine sum, RHS by a direct DFT, point
  strengths by a direct inverse DFT);
* panels taller than the shared-memory panel (rows > 864) take the
  global-memory panel kernel, in both precisions;
* an empty batch (W = 0) is refused with AXI_ERR_ARG and launches nothing.
Tolerances as in test_gpu_parity: e_A <= 1e-13, e_bd and e_ff <= 1e-10.
"""
import ctypes as C
import dataclasses
import math

import numpy as np
import pytest

import oracle as O
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _prepare(wl):
    ob = wl.obstacles[0]
    coll, src, srcx = O.geometry(ob)
    if not ob.q:
        ob = dataclasses.replace(ob, q=O.choose_q(ob, coll, src, srcx))
    A, fac = O.factor_operator(ob, coll, src, srcx)
    return ob, (coll, src, srcx), A, fac


def _e_bd(A, ob, c_gpu, c_ora, fh):
    num = 0.0
    for idx in range(ob.P):
        n = idx if idx <= ob.P // 2 else ob.P - idx
        num += np.linalg.norm(A[n] @ (c_gpu[:, idx, :] - c_ora[:, idx, :]).T) ** 2
    return math.sqrt(num) / np.linalg.norm(fh)


def _check_apply(axi, op, wl, ob, coll, src, A, fac, want_sigma=True):
    dirs_np = synth.plane_wave_directions(wl.n_waves, wl.wave_seed)
    f = op.incident(torch.tensor(dirs_np, device="cuda"))
    coef, sigma = op.apply(f, want_sigma=True)
    xh = synth.plane_wave_directions(64, 99)
    F = op.eval_field(coef, torch.tensor(xh, device="cuda"), axi.EVAL_FAR_FIELD).cpu().numpy()
    torch.cuda.synchronize()
    assert op.status() == 0
    fh = O.rhs_modes(O.incident_samples(ob, coll, dirs_np))
    c_ora = O.solve_modes(ob, fac, fh)
    c_gpu = coef.cpu().numpy()
    e_bd = _e_bd(A, ob, c_gpu, c_ora, fh)
    assert e_bd < 1e-10, e_bd
    F_ora = O.far_field(ob, src, c_ora, xh)
    e_ff = np.abs(F - F_ora).max() / np.abs(F_ora).max()
    assert e_ff < 1e-10, e_ff
    if want_sigma:
        sig_ora = O.point_strengths(c_gpu, ob.P)
        assert np.abs(sigma.cpu().numpy() - sig_ora).max() < 1e-12 * np.abs(sig_ora).max()


def test_direct_transforms_without_fft_plan():
    """P = 14 and q = 112 (factor 7): no mixed-radix plan, direct transforms."""
    from paper_1506_05083_gb300 import axi
    wl = synth.small_case(seed=21, k=2.5, M=40, N=30, P=14, q=112)
    ob, (coll, src, srcx), A, fac = _prepare(wl)
    op = axi.Operator([axi.spec_from_obstacle(wl.obstacles[0])])
    Ag = op.fill_modes().cpu().numpy().transpose(0, 2, 1)
    assert np.abs(Ag - A).max() / np.abs(A).max() < 1e-13
    _check_apply(axi, op, wl, ob, coll, src, A, fac)


@pytest.mark.parametrize("prec", ["fp64", "split7"])
def test_panel_taller_than_shared_memory(prec):
    """M = 900 collocation rings: 900-row panels use the global-memory panel."""
    from paper_1506_05083_gb300 import axi
    wl = synth.small_case(seed=23, k=2.0, M=900, N=40, P=4)
    ob, (coll, src, srcx), A, fac = _prepare(wl)
    p = axi.PREC_FP64 if prec == "fp64" else axi.PREC_SPLIT_BF16 | (7 << 8)
    op = axi.Operator([axi.spec_from_obstacle(wl.obstacles[0])], prec=p)
    Af = op.fill_modes().cpu().numpy().transpose(0, 2, 1)
    Ap, tau, T, nb = op.factors()
    Ap = Ap.cpu().numpy().transpose(0, 2, 1)
    tau = tau.cpu().numpy()
    rows, cols = Ap.shape[1], Ap.shape[2]
    assert rows == 900
    for d in range(ob.P // 2 + 1):
        # Q R = A through the reflectors, applied to R's columns
        R = np.triu(Ap[d][:cols])
        X = np.zeros((rows, cols), dtype=np.complex128)
        X[:cols] = R
        for j in range(cols - 1, -1, -1):
            v = np.zeros(rows, dtype=np.complex128)
            v[j] = 1.0
            v[j + 1:] = Ap[d][j + 1:, j]
            X -= tau[d][j] * np.outer(v, v.conj() @ X)
        tol = 1e-13 if prec == "fp64" else 1e-11
        assert np.linalg.norm(X - Af[d]) < tol * np.linalg.norm(Af[d])
    _check_apply(axi, op, wl, ob, coll, src, A, fac)


def test_empty_batch_is_refused():
    from paper_1506_05083_gb300 import axi
    wl = synth.small_case()
    op = axi.Operator([axi.spec_from_obstacle(wl.obstacles[0])])
    L = axi.lib()
    null = C.c_void_p(0)
    code = L.axi_apply_operator(op._op, 0, 0, null, null, null, null, 0, null)
    assert code == axi.ERR_ARG
    code = L.axi_incident_planewaves(op._op, 0, 0, null, null, null)
    assert code == axi.ERR_ARG
    torch.cuda.synchronize()
    assert op.status() == 0
