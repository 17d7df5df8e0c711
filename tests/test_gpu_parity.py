"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances follow the parity metric of the one-obstacle operator:
  e_A  = max|A_gpu - A_ora| / max|A_ora|                <= 1e-13 (fill)
  QR   ||A - Q R|| / ||A||, ||I - V T V^H - H_1..H_nb|| <= 1e-13
  e_bd = ||A_ora (c_gpu - c_ora)|| / ||fhat||          <= 1e-10 (all modes and waves jointly)
  e_ff = max|F_gpu - F_ora| / max|F_ora|                <= 1e-10
Coefficients and R are not compared entry by entry: on the ill-conditioned
MFS blocks they are not reproducible across rounding orders; what the method
fixes (boundary data, far field) is.
"""
import dataclasses
import math

import numpy as np
import pytest

import oracle as O
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

_cache = {}


def _case(name):
    """(workload, obstacle, oracle geometry, oracle matrices, oracle factors)."""
    if name in _cache:
        return _cache[name]
    if name == "sphere":
        wl = synth.config_sphere()
    elif name == "small":
        wl = synth.small_case()
    elif name == "small_trans":
        wl = synth.small_case(seed=11, k=2.0, M=44, N=36, P=20, bc=synth.BC_TRANSMISSION)
    elif name == "medium":
        # enough columns (80) that trailing updates reach beyond the next panel
        wl = synth.small_case(seed=13, k=4.0, M=96, N=80, P=16)
    elif name == "smooth":
        wl = synth.config_smooth()
    else:
        raise KeyError(name)
    ob = wl.obstacles[0]
    coll, src, srcx = O.geometry(ob)
    if not ob.q:
        # each side applies the Theorem 1 rule to its own geometry
        ob = dataclasses.replace(ob, q=O.choose_q(ob, coll, src, srcx))
    A, fac = O.factor_operator(ob, coll, src, srcx)
    _cache[name] = (wl, ob, (coll, src, srcx), A, fac)
    return _cache[name]


def _operator(obs_list):
    from paper_1506_05083_gb300 import axi
    specs = []
    for ob_ora, ob_in in obs_list:
        spec = axi.spec_from_obstacle(ob_in)
        assert spec.q == ob_ora.q
        specs.append(spec)
    return axi, axi.Operator(specs)


def _e_bd(A, ob, c_gpu, c_ora, fh):
    P = ob.P
    num = 0.0
    for idx in range(P):
        n = idx if idx <= P // 2 else P - idx
        num += np.linalg.norm(A[n] @ (c_gpu[:, idx, :] - c_ora[:, idx, :]).T) ** 2
    return math.sqrt(num) / np.linalg.norm(fh)


@pytest.mark.parametrize("name", ["small", "small_trans", "sphere"])
def test_fill_parity(name):
    wl, ob, geo, A, fac = _case(name)
    axi, op = _operator([(ob, wl.obstacles[0])])
    Ag = op.fill_modes().cpu().numpy().transpose(0, 2, 1)
    torch.cuda.synchronize()
    assert op.status() == 0
    err = np.abs(Ag - A).max() / np.abs(A).max()
    assert err < 1e-13, err


def _householder_q(Vp, tau, rows, cols):
    Q = np.eye(rows, dtype=np.complex128)
    for j in range(cols - 1, -1, -1):
        v = np.zeros(rows, dtype=np.complex128)
        v[j] = 1.0
        v[j + 1:] = Vp[j + 1:, j]
        Q -= tau[j] * np.outer(v, v.conj() @ Q)
    return Q


@pytest.mark.parametrize("name", ["small", "small_trans"])
def test_qr_invariants(name):
    wl, ob, geo, A, fac = _case(name)
    axi, op = _operator([(ob, wl.obstacles[0])])
    Af = op.fill_modes().cpu().numpy().transpose(0, 2, 1)
    Ap, tau, T, nb = op.factors()
    Ap = Ap.cpu().numpy().transpose(0, 2, 1)
    tau = tau.cpu().numpy()
    T = T.cpu().numpy()
    rows, cols = Ap.shape[1], Ap.shape[2]
    for d in (0, 1, ob.P // 4, ob.P // 2):
        Q = _householder_q(Ap[d], tau[d], rows, cols)
        R = np.triu(Ap[d][:cols])
        assert np.all(np.diag(R).imag == 0)
        assert np.linalg.norm(Q[:, :cols] @ R - Af[d]) < 1e-13 * np.linalg.norm(Af[d])
        assert np.abs(Q.conj().T @ Q - np.eye(rows)).max() < 1e-13
        # leading |R_jj| are well determined: compare with the oracle's factor
        Ro = np.abs(np.diag(fac[d][0][:cols]))
        assert np.allclose(np.abs(np.diag(R))[:4], Ro[:4], rtol=1e-11)
        # compact WY: I - V T V^H equals the product of the panel's reflectors
        for p in range(T.shape[1]):
            k0 = p * nb
            nbp = min(nb, cols - k0)
            V = np.zeros((rows, nbp), dtype=np.complex128)
            Hprod = np.eye(rows, dtype=np.complex128)
            for a in range(nbp):
                c = k0 + a
                V[c, a] = 1.0
                V[c + 1:, a] = Ap[d][c + 1:, c]
                Hprod = Hprod @ (np.eye(rows) - tau[d][c] * np.outer(V[:, a], V[:, a].conj()))
            Tp = T[d, p].T[:nbp, :nbp]          # stored column-major
            assert np.abs(np.eye(rows) - V @ Tp @ V.conj().T - Hprod).max() < 1e-13


@pytest.mark.parametrize("name", ["small", "small_trans", "sphere"])
def test_apply_parity(name):
    wl, ob, (coll, src, srcx), A, fac = _case(name)
    axi, op = _operator([(ob, wl.obstacles[0])])
    dirs_np = synth.plane_wave_directions(wl.n_waves, wl.wave_seed)
    dirs = torch.tensor(dirs_np, device="cuda")
    f_gpu = op.incident(dirs)
    coef, sigma = op.apply(f_gpu, want_sigma=True)
    xh_np = synth.plane_wave_directions(64, 99)
    F_gpu = op.eval_field(coef, torch.tensor(xh_np, device="cuda"), axi.EVAL_FAR_FIELD)
    torch.cuda.synchronize()
    assert op.status() == 0
    f_ora = O.incident_samples(ob, coll, dirs_np)
    assert np.abs(f_gpu.cpu().numpy() - f_ora).max() < 1e-13 * np.abs(f_ora).max()
    fh = O.rhs_modes(f_ora)
    c_ora = O.solve_modes(ob, fac, fh)
    c_gpu = coef.cpu().numpy()
    assert _e_bd(A, ob, c_gpu, c_ora, fh) < 1e-10
    F_ora = O.far_field(ob, src, c_ora, xh_np)
    e_ff = np.abs(F_gpu.cpu().numpy() - F_ora).max() / np.abs(F_ora).max()
    assert e_ff < 1e-10, e_ff
    sig_ora = O.point_strengths(c_gpu, ob.P)
    assert np.abs(sigma.cpu().numpy() - sig_ora).max() < 1e-12 * np.abs(sig_ora).max()


def test_sphere_series_on_gpu():
    wl, ob, geo, A, fac = _case("sphere")
    axi, op = _operator([(ob, wl.obstacles[0])])
    d = synth.plane_wave_directions(1, wl.wave_seed)
    coef = op.apply(op.incident(torch.tensor(d, device="cuda")))
    xh = synth.plane_wave_directions(64, 99)
    F = op.eval_field(coef, torch.tensor(xh, device="cuda"), axi.EVAL_FAR_FIELD).cpu().numpy()[0]
    Fs = O.sphere_series_far_field(ob.k, 1.0, d[0], xh)
    assert np.abs(F - Fs).max() < 1e-10 * np.abs(Fs).max()


@pytest.mark.parametrize("kind", [0, 1, 2])
def test_eval_kinds(kind):
    wl, ob, (coll, src, srcx), A, fac = _case("small")
    axi, op = _operator([(ob, wl.obstacles[0])])
    rng = np.random.default_rng(17)
    W = 3
    c = rng.standard_normal((W, ob.P, ob.N)) + 1j * rng.standard_normal((W, ob.P, ob.N))
    if kind == 2:
        T = synth.plane_wave_directions(40, 3)
    else:
        T = rng.uniform(-4, 4, (40, 3))
        T[:, 2] += 6.0
    nv = rng.standard_normal((40, 3))
    nv /= np.linalg.norm(nv, axis=1, keepdims=True)
    ct = torch.tensor(c, device="cuda")
    out = op.eval_field(ct, torch.tensor(T, device="cuda"), kind,
                        normals=torch.tensor(nv, device="cuda") if kind == 1 else None)
    out = out.cpu().numpy()
    if kind == 2:
        ref = O.far_field(ob, src, c, T)
    else:
        ref = O.potential(ob, src, c, T, normals=nv if kind == 1 else None)
    assert np.abs(out - ref).max() < 1e-12 * np.abs(ref).max()


def test_near_image_sum_parity():
    wl, ob, (coll, src, srcx), A, fac = _case("small")
    axi, op = _operator([(ob, wl.obstacles[0])])
    rng = np.random.default_rng(5)
    W = 4
    c = rng.standard_normal((W, ob.P, ob.N)) + 1j * rng.standard_normal((W, ob.P, ob.N))
    d = synth.plane_wave_directions(W, 77)
    lat = (3.3, 2.9)
    idx = np.arange(0, ob.M * ob.P, 7)
    phi = 2 * math.pi * np.arange(ob.P) / ob.P
    X = np.array([[cm[0] * math.cos(p), cm[0] * math.sin(p), cm[1]] for cm in coll for p in phi])[idx]
    Nn = np.array([[cm[2] * math.cos(p), cm[2] * math.sin(p), cm[3]] for cm in coll for p in phi])[idx]
    out = op.eval_field(torch.tensor(c, device="cuda"), torch.tensor(X, device="cuda"),
                        axi.EVAL_NORMAL_DERIV, normals=torch.tensor(Nn, device="cuda"),
                        lattice=lat, dirs=torch.tensor(d, device="cuda")).cpu().numpy()
    ref = O.near_image_sum(ob, coll, src, c, d, lat, target_idx=idx)
    assert np.abs(out - ref).max() < 1e-12 * np.abs(ref).max()


def test_batched_uneven_obstacles():
    cases = [_case(n) for n in ("small", "small_trans", "sphere")]
    axi, op = _operator([(c[1], c[0].obstacles[0]) for c in cases])
    for i, (wl, ob, (coll, src, srcx), A, fac) in enumerate(cases):
        dirs_np = synth.plane_wave_directions(3, 40 + i)
        coef = op.apply(op.incident(torch.tensor(dirs_np, device="cuda"), obs=i), obs=i)
        fh = O.rhs_modes(O.incident_samples(ob, coll, dirs_np))
        c_ora = O.solve_modes(ob, fac, fh)
        assert _e_bd(A, ob, coef.cpu().numpy(), c_ora, fh) < 1e-10
    torch.cuda.synchronize()
    assert op.status() == 0


def test_smooth_full_size():
    """The smooth-body workload at full size (N=180, M=216, P=120, q=400, 16 waves)."""
    wl, ob, (coll, src, srcx), A, fac = _case("smooth")
    axi, op = _operator([(ob, wl.obstacles[0])])
    Ag = op.fill_modes().cpu().numpy().transpose(0, 2, 1)
    assert np.abs(Ag - A).max() / np.abs(A).max() < 1e-13
    dirs_np = synth.plane_wave_directions(wl.n_waves, wl.wave_seed)
    coef = op.apply(op.incident(torch.tensor(dirs_np, device="cuda")))
    xh_np = synth.plane_wave_directions(64, 99)
    F_gpu = op.eval_field(coef, torch.tensor(xh_np, device="cuda"), axi.EVAL_FAR_FIELD).cpu().numpy()
    torch.cuda.synchronize()
    assert op.status() == 0
    fh = O.rhs_modes(O.incident_samples(ob, coll, dirs_np))
    c_ora = O.solve_modes(ob, fac, fh)
    assert _e_bd(A, ob, coef.cpu().numpy(), c_ora, fh) < 1e-10
    F_ora = O.far_field(ob, src, c_ora, xh_np)
    assert np.abs(F_gpu - F_ora).max() / np.abs(F_ora).max() < 1e-10


@pytest.mark.parametrize("prec", ["fp64", "split"])
def test_fill_subgrid_and_full_grid(prec):
    """The smooth body at full size: the fill on each ring pair's sub-grid
    (default; 92% of pairs on q/2 nodes) and on the full q-node grid
    (AXI_PLAN_FULL_FILL_GRID) both match the oracle's full-grid fill to
    e_A <= 1e-13, and each other to rounding."""
    from paper_1506_05083_gb300 import axi
    wl, ob, (coll, src, srcx), A, fac = _case("smooth")
    spec = axi.spec_from_obstacle(wl.obstacles[0])
    base = axi.PREC_FP64 if prec == "fp64" else axi.PREC_SPLIT_BF16
    out = []
    for flag in (0, axi.PLAN_FULL_FILL_GRID):
        op = axi.Operator([spec], prec=base | flag)
        out.append(op.fill_modes().cpu().numpy().transpose(0, 2, 1))
        torch.cuda.synchronize()
        assert op.status() == 0
        del op
    scale = np.abs(A).max()
    for Ag in out:
        assert np.abs(Ag - A).max() / scale < 1e-13
    assert np.abs(out[0] - out[1]).max() / scale < 1e-13
