"""Split-precision (Ozaki, BF16 digits on tensor cores) QR updates and apply,
against the FP64 oracle. Parity bar as for the native path: e_bd, e_ff <= 1e-10
at the default 7 digits; fewer digits must degrade gracefully and monotonically.
"""
import dataclasses
import math

import numpy as np
import pytest

import oracle as O
import synth
from test_gpu_parity import _case, _e_bd, _householder_q

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _op(name, slices):
    from paper_1506_05083_gb300 import axi
    wl, ob, geo, A, fac = _case(name)
    spec = axi.spec_from_obstacle(wl.obstacles[0])
    assert spec.q == ob.q
    prec = axi.PREC_SPLIT_BF16 | (slices << 8)
    return axi, axi.Operator([spec], prec=prec), (wl, ob, geo, A, fac)


@pytest.mark.parametrize("name", ["small", "small_trans", "sphere", "medium", "smooth"])
def test_split_fill_parity(name):
    """Split plans fill with the tensor-core transform (8 digits, fill_mma.cu):
    same bar as the FP64 fill, e_A <= 1e-13 against the oracle's direct sums."""
    axi, op, (wl, ob, geo, A, fac) = _op(name, 7)
    Ag = op.fill_modes().cpu().numpy().transpose(0, 2, 1)
    torch.cuda.synchronize()
    assert op.status() == 0
    err = np.abs(Ag - A).max() / np.abs(A).max()
    assert err < 1e-13, err


@pytest.mark.parametrize("P,q", [(180, 0), (240, 0), (8, 1728), (8, 1800)])
def test_split_fill_parity_shapes(P, q):
    """Mode counts that fill the tensor-core accumulators (P = 180: 48 modes per
    parity, N = 48; P = 240: 64, every TMEM column), the longest contraction the
    tcgen05 transform takes in one pass (q = 1728: 433 folded nodes, padded to
    448), and one too long for exact FP32 group sums over one pass (q = 1800:
    451 folded nodes), which takes the mma.sync transform with periodic int64
    folds."""
    from paper_1506_05083_gb300 import axi
    wl = synth.small_case(seed=29, k=3.0, M=24, N=20, P=P, q=q)
    ob = wl.obstacles[0]
    coll, src, srcx = O.geometry(ob)
    if not ob.q:
        ob = dataclasses.replace(ob, q=O.choose_q(ob, coll, src, srcx))
    A = O.system_matrix(ob, coll, src, srcx)
    op = axi.Operator([axi.spec_from_obstacle(wl.obstacles[0])],
                      prec=axi.PREC_SPLIT_BF16 | (7 << 8))
    Ag = op.fill_modes().cpu().numpy().transpose(0, 2, 1)
    torch.cuda.synchronize()
    assert op.status() == 0
    err = np.abs(Ag - A).max() / np.abs(A).max()
    assert err < 1e-13, err


@pytest.mark.parametrize("name", ["medium", "small_trans"])
def test_split_qr_invariants(name):
    axi, op, (wl, ob, geo, A, fac) = _op(name, 7)
    Af = op.fill_modes().cpu().numpy().transpose(0, 2, 1)
    Ap, tau, T, nb = op.factors()
    Ap = Ap.cpu().numpy().transpose(0, 2, 1)
    tau = tau.cpu().numpy()
    torch.cuda.synchronize()
    assert op.status() == 0
    rows, cols = Ap.shape[1], Ap.shape[2]
    for d in (0, 1, ob.P // 2):
        Q = _householder_q(Ap[d], tau[d], rows, cols)
        R = np.triu(Ap[d][:cols])
        assert np.linalg.norm(Q[:, :cols] @ R - Af[d]) < 1e-12 * np.linalg.norm(Af[d])


@pytest.mark.parametrize("name", ["medium", "small_trans", "sphere", "smooth"])
def test_split_apply_parity(name):
    axi, op, (wl, ob, (coll, src, srcx), A, fac) = _op(name, 7)
    dirs_np = synth.plane_wave_directions(wl.n_waves, wl.wave_seed)
    coef = op.apply(op.incident(torch.tensor(dirs_np, device="cuda")))
    xh = synth.plane_wave_directions(64, 99)
    F = op.eval_field(coef, torch.tensor(xh, device="cuda"), axi.EVAL_FAR_FIELD).cpu().numpy()
    torch.cuda.synchronize()
    assert op.status() == 0
    fh = O.rhs_modes(O.incident_samples(ob, coll, dirs_np))
    c_ora = O.solve_modes(ob, fac, fh)
    assert _e_bd(A, ob, coef.cpu().numpy(), c_ora, fh) < 1e-10
    F_ora = O.far_field(ob, src, c_ora, xh)
    assert np.abs(F - F_ora).max() / np.abs(F_ora).max() < 1e-10


def test_split_digits_sweep():
    """Error against the oracle shrinks as digits are added (4 -> 8)."""
    errs = []
    for s in (4, 5, 6, 7, 8):
        axi, op, (wl, ob, (coll, src, srcx), A, fac) = _op("medium", s)
        dirs_np = synth.plane_wave_directions(wl.n_waves, wl.wave_seed)
        coef = op.apply(op.incident(torch.tensor(dirs_np, device="cuda")))
        fh = O.rhs_modes(O.incident_samples(ob, coll, dirs_np))
        c_ora = O.solve_modes(ob, fac, fh)
        errs.append(_e_bd(A, ob, coef.cpu().numpy(), c_ora, fh))
    assert errs[-1] < 1e-11
    assert errs[0] > errs[-1]
    assert all(e < 1e-3 for e in errs)


@pytest.mark.parametrize("name", ["medium", "smooth", "small_trans"])
def test_split_tc_update_parity(name):
    """The trailing update on tcgen05 (tuning rest_grid 2, 3 with one CTA
    per SM, and 0 = auto; 4 is the mma.sync form: W' = Y^H X and X -= V W' as BF16 digit products with
    tensor-memory accumulators): Q R reproduces the filled modes, the apply
    meets the oracle bar, the coefficients agree with the mma.sync update's
    to the digits' precision, and the occupancy choice changes no bit."""
    from paper_1506_05083_gb300 import axi
    wl, ob, (coll, src, srcx), A, fac = _case(name)
    spec = axi.spec_from_obstacle(wl.obstacles[0])
    prec = axi.PREC_SPLIT_BF16 | (7 << 8)
    dirs_np = synth.plane_wave_directions(wl.n_waves, wl.wave_seed)
    coefs = {}
    for rg in (4, 0, 2, 3):
        op = axi.Operator([spec], prec=prec, tuning='{"next_update": 2, "rest_grid": %d}' % rg)
        assert '"rest_grid": %d' % rg in op.tuning()
        coefs[rg] = op.apply(op.incident(torch.tensor(dirs_np, device="cuda"))).cpu().numpy()
        if rg == 2:
            Af = op.fill_modes().cpu().numpy().transpose(0, 2, 1)
            Ap, tau, T, nb = op.factors()
            Ap = Ap.cpu().numpy().transpose(0, 2, 1)
            tau = tau.cpu().numpy()
        torch.cuda.synchronize()
        assert op.status() == 0
    rows, cols = Ap.shape[1], Ap.shape[2]
    for d in (0, 1, ob.P // 2):
        Q = _householder_q(Ap[d], tau[d], rows, cols)
        R = np.triu(Ap[d][:cols])
        assert np.linalg.norm(Q[:, :cols] @ R - Af[d]) < 1e-12 * np.linalg.norm(Af[d])
    fh = O.rhs_modes(O.incident_samples(ob, coll, dirs_np))
    c_ora = O.solve_modes(ob, fac, fh)
    for rg in (2, 3):       # tcgen05 update, two or one CTA per SM
        assert _e_bd(A, ob, coefs[rg], c_ora, fh) < 1e-10
        assert _e_bd(A, ob, coefs[rg], coefs[4], fh) < 1e-10
    assert np.array_equal(coefs[2], coefs[3])
    assert np.array_equal(coefs[0], coefs[2])      # auto picks the tcgen05 update here


def test_split_fill_chunking_is_exact():
    """The fill's chunk of ring pairs (tuning fill_chunk_mb) only changes how
    many pairs each pair of fill launches covers: the modal matrices, and so
    the factors and coefficients, are bit-identical for every chunk size,
    including chunks far smaller than one launch's natural size."""
    from paper_1506_05083_gb300 import axi
    wl, ob, (coll, src, srcx), A, fac = _case("smooth")
    spec = axi.spec_from_obstacle(wl.obstacles[0])
    prec = axi.PREC_SPLIT_BF16 | (7 << 8)
    dirs = torch.tensor(synth.plane_wave_directions(wl.n_waves, wl.wave_seed), device="cuda")
    out = {}
    for mb in (0, 8, 1):
        op = axi.Operator([spec], prec=prec, tuning='{"fill_chunk_mb": %d}' % mb)
        out[mb] = (op.fill_modes().cpu().numpy(), op.apply(op.incident(dirs)).cpu().numpy())
        torch.cuda.synchronize()
        assert op.status() == 0
    for mb in (8, 1):
        assert np.array_equal(out[mb][0], out[0][0])
        assert np.array_equal(out[mb][1], out[0][1])
    err = np.abs(out[1][0].transpose(0, 2, 1) - A).max() / np.abs(A).max()
    assert err < 1e-13, err


@pytest.mark.parametrize("name", ["medium", "smooth"])
def test_split_next_cluster_parity(name):
    """The next panel's columns updated by clusters of 1, 2 or 4 CTAs per mode
    (tuning next_cluster): each meets the oracle bar, and they agree with each
    other to the digits' precision (the row split changes only the order in
    which the cluster's partial V^H X are added)."""
    from paper_1506_05083_gb300 import axi
    wl, ob, (coll, src, srcx), A, fac = _case(name)
    spec = axi.spec_from_obstacle(wl.obstacles[0])
    dirs_np = synth.plane_wave_directions(wl.n_waves, wl.wave_seed)
    fh = O.rhs_modes(O.incident_samples(ob, coll, dirs_np))
    c_ora = O.solve_modes(ob, fac, fh)
    coefs = {}
    for nc in (1, 2, 4):
        op = axi.Operator([spec], prec=axi.PREC_SPLIT_BF16 | (7 << 8),
                          tuning='{"next_update": 2, "next_cluster": %d}' % nc)
        coefs[nc] = op.apply(op.incident(torch.tensor(dirs_np, device="cuda"))).cpu().numpy()
        torch.cuda.synchronize()
        assert op.status() == 0
        assert _e_bd(A, ob, coefs[nc], c_ora, fh) < 1e-10
    assert _e_bd(A, ob, coefs[1], coefs[2], fh) < 1e-10
    assert _e_bd(A, ob, coefs[4], coefs[2], fh) < 1e-10


@pytest.mark.parametrize("name", ["medium", "smooth"])
def test_split_rest_start_is_exact(name):
    """Starting each trailing update after the next-panel update (tuning
    rest_start 1), on either stream priority, changes only when kernels run,
    not what they compute: the coefficients equal those of rest_start 0 bit
    for bit, and meet the oracle bar."""
    from paper_1506_05083_gb300 import axi
    wl, ob, (coll, src, srcx), A, fac = _case(name)
    spec = axi.spec_from_obstacle(wl.obstacles[0])
    dirs_np = synth.plane_wave_directions(wl.n_waves, wl.wave_seed)
    fh = O.rhs_modes(O.incident_samples(ob, coll, dirs_np))
    c_ora = O.solve_modes(ob, fac, fh)
    coefs = []
    for rs, cs in ((0, 0), (1, 0), (1, 1)):
        op = axi.Operator([spec], prec=axi.PREC_SPLIT_BF16 | (7 << 8),
                          tuning='{"next_update": 2, "rest_start": %d, "crit_stream": %d}' % (rs, cs))
        coefs.append(op.apply(op.incident(torch.tensor(dirs_np, device="cuda"))).cpu().numpy())
        torch.cuda.synchronize()
        assert op.status() == 0
    assert _e_bd(A, ob, coefs[0], c_ora, fh) < 1e-10
    assert np.array_equal(coefs[1], coefs[0])
    assert np.array_equal(coefs[2], coefs[0])


@pytest.mark.parametrize("name", ["small", "medium", "smooth"])
def test_split_panel_fixed_parity(name):
    """The Householder panel in 58-bit fixed point (tuning panel_fixed 2:
    exact integer sums, integer updates, FP64 scalars): Q R reproduces the
    filled modes, Q is unitary, every panel's I - V T V^H equals the product
    of its reflectors, the apply meets the oracle bar and agrees with the
    FP64 panel's, and 128 and 256 threads give the same bits (integer sums
    do not depend on their order)."""
    from paper_1506_05083_gb300 import axi
    wl, ob, (coll, src, srcx), A, fac = _case(name)
    spec = axi.spec_from_obstacle(wl.obstacles[0])
    prec = axi.PREC_SPLIT_BF16 | (7 << 8)
    dirs_np = synth.plane_wave_directions(wl.n_waves, wl.wave_seed)
    coefs, facs = {}, {}
    for key, t in (("fp64", '{"next_update": 2, "panel_fixed": 1}'),
                   ("fx128", '{"next_update": 2, "panel_fixed": 2, "panel_threads": 128}'),
                   ("fx256", '{"next_update": 2, "panel_fixed": 2, "panel_threads": 256}')):
        op = axi.Operator([spec], prec=prec, tuning=t)
        coefs[key] = op.apply(op.incident(torch.tensor(dirs_np, device="cuda"))).cpu().numpy()
        Ap, tau, T, nb = op.factors()
        facs[key] = (Ap.cpu().numpy().transpose(0, 2, 1), tau.cpu().numpy(), T.cpu().numpy())
        if key == "fx128":
            Af = op.fill_modes().cpu().numpy().transpose(0, 2, 1)
        torch.cuda.synchronize()
        assert op.status() == 0
    Ap, tau, T = facs["fx128"]
    rows, cols = Ap.shape[1], Ap.shape[2]
    for d in (0, 1, ob.P // 2):
        Q = _householder_q(Ap[d], tau[d], rows, cols)
        R = np.triu(Ap[d][:cols])
        assert np.all(np.diag(R).imag == 0)
        assert np.linalg.norm(Q[:, :cols] @ R - Af[d]) < 1e-12 * np.linalg.norm(Af[d])
        assert np.abs(Q.conj().T @ Q - np.eye(rows)).max() < 1e-13
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
            Tp = T[d, p].T[:nbp, :nbp]
            assert np.abs(np.eye(rows) - V @ Tp @ V.conj().T - Hprod).max() < 1e-13
    for k in range(3):
        assert np.array_equal(facs["fx256"][k], facs["fx128"][k])
    assert np.array_equal(coefs["fx256"], coefs["fx128"])
    fh = O.rhs_modes(O.incident_samples(ob, coll, dirs_np))
    c_ora = O.solve_modes(ob, fac, fh)
    assert _e_bd(A, ob, coefs["fx128"], c_ora, fh) < 1e-10
    assert _e_bd(A, ob, coefs["fx128"], coefs["fp64"], fh) < 1e-10
