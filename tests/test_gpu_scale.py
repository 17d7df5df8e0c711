"""Full-scale workloads against the oracle: the 64-obstacle batch (sampled
obstacles), the cup precision table (native FP64 vs 5..8 BF16 digits), and
the split-precision apply for a large batch of waves."""
import dataclasses
import json
import math
import os

import numpy as np
import pytest

import oracle as O
import synth
from test_gpu_parity import _e_bd

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _oracle(ob):
    coll, src, srcx = O.geometry(ob)
    if not ob.q:
        ob = dataclasses.replace(ob, q=O.choose_q(ob, coll, src, srcx))
    A, fac = O.factor_operator(ob, coll, src, srcx)
    return ob, coll, src, A, fac


def _sensitivity(ob, A, fh, c_ora, rng):
    """e_bd between the oracle solution and the oracle re-solved with every
    modal matrix perturbed by u * max|A_n| complex Gaussian noise: how far
    boundary data moves per unit-roundoff normwise change of the matrix."""
    u = np.finfo(float).eps / 2
    num = 0.0
    for idx in range(ob.P):
        n = idx if idx <= ob.P // 2 else ob.P - idx
        noise = rng.standard_normal(A[n].shape) + 1j * rng.standard_normal(A[n].shape)
        Ap = A[n] + u * np.abs(A[n]).max() * noise / math.sqrt(2)
        QR, tau = O.householder_qr(Ap)
        y = O.apply_qh(QR, tau, fh[:, idx, :].T)[:A.shape[2]]
        cp = O.back_substitute(np.triu(QR[:A.shape[2], :A.shape[2]]), y)
        num += np.linalg.norm(A[n] @ (c_ora[:, idx].T - cp)) ** 2
    return math.sqrt(num) / np.linalg.norm(fh)


@pytest.mark.parametrize("prec", ["fp64", "split"])
def test_batched_64_obstacles_sampled(prec):
    """All 64 obstacles in one plan; five of them checked against the oracle.

    The batched workload draws N, P and k independently, so some obstacles are
    unresolved (oracle residual 1e-5..1e-4, coefficient norms up to ~1e11) and
    their least-squares solutions are sensitive to rounding-level changes of the
    matrix. Bar: e_bd <= max(1e-10, 1e3 * s), s = the oracle's own sensitivity
    to a u*max|A| normwise perturbation (the fill parity bar, 1e-13*max|A|, is
    ~1e3 u). Resolved obstacles (9, 35; residual < 1e-6) have s ~ 1e-15, so
    the bar there is the plain 1e-10.
    """
    from paper_1506_05083_gb300 import axi
    wl = synth.config_batched()
    specs = [axi.spec_from_obstacle(ob) for ob in wl.obstacles]
    p = axi.PREC_FP64 if prec == "fp64" else axi.PREC_SPLIT_BF16
    op = axi.Operator(specs, prec=p)
    torch.cuda.synchronize()
    assert op.status() == 0
    rng = np.random.default_rng(123)
    for i in (9, 35, 24, 7, 15):
        ob_in = wl.obstacles[i]
        ob, coll, src, A, fac = _oracle(ob_in)
        assert specs[i].q == ob.q
        dirs = synth.plane_wave_directions(4, 500 + i)
        coef = op.apply(op.incident(torch.tensor(dirs, device="cuda"), obs=i), obs=i).cpu().numpy()
        fh = O.rhs_modes(O.incident_samples(ob, coll, dirs))
        c_ora = O.solve_modes(ob, fac, fh)
        res = math.sqrt(sum(
            np.linalg.norm(A[idx if idx <= ob.P // 2 else ob.P - idx] @ c_ora[:, idx].T
                           - fh[:, idx].T) ** 2 for idx in range(ob.P))) / np.linalg.norm(fh)
        s = _sensitivity(ob, A, fh, c_ora, rng)
        e = _e_bd(A, ob, coef, c_ora, fh)
        assert e <= max(1e-10, 1e3 * s), (i, e, s)
        if res < 1e-6:
            assert e < 1e-10, (i, e)


def test_split_apply_many_waves():
    """W >= 33 switches the apply's Q^H to tensor cores; check it against the oracle."""
    from paper_1506_05083_gb300 import axi
    wl = synth.small_case()
    ob, coll, src, A, fac = _oracle(wl.obstacles[0])
    op = axi.Operator([axi.spec_from_obstacle(wl.obstacles[0])], prec=axi.PREC_SPLIT_BF16)
    dirs = synth.plane_wave_directions(40, 4040)
    coef = op.apply(op.incident(torch.tensor(dirs, device="cuda"))).cpu().numpy()
    torch.cuda.synchronize()
    assert op.status() == 0
    fh = O.rhs_modes(O.incident_samples(ob, coll, dirs))
    c_ora = O.solve_modes(ob, fac, fh)
    assert _e_bd(A, ob, coef, c_ora, fh) < 1e-10


def test_cup_precision_table():
    """Cup, k=25, N=360, M=432, P=180: boundary-data and far-field error per arithmetic."""
    from paper_1506_05083_gb300 import axi
    wl = synth.config_cup()
    ob, coll, src, A, fac = _oracle(wl.obstacles[0])
    dirs = synth.plane_wave_directions(wl.n_waves, wl.wave_seed)
    fh = O.rhs_modes(O.incident_samples(ob, coll, dirs))
    c_ora = O.solve_modes(ob, fac, fh)
    xh = synth.plane_wave_directions(64, 99)
    F_ora = O.far_field(ob, src, c_ora, xh)
    spec = axi.spec_from_obstacle(wl.obstacles[0])
    table = {}
    for name, prec in [("fp64", axi.PREC_FP64)] + [
            (f"split{s}", axi.PREC_SPLIT_BF16 | (s << 8)) for s in (5, 6, 7, 8)]:
        op = axi.Operator([spec], prec=prec)
        coef = op.apply(op.incident(torch.tensor(dirs, device="cuda")))
        F = op.eval_field(coef, torch.tensor(xh, device="cuda"), axi.EVAL_FAR_FIELD).cpu().numpy()
        torch.cuda.synchronize()
        assert op.status() == 0
        e_bd = _e_bd(A, ob, coef.cpu().numpy(), c_ora, fh)
        e_ff = float(np.abs(F - F_ora).max() / np.abs(F_ora).max())
        table[name] = {"e_bd": e_bd, "e_ff": e_ff}
        del op
    print("cup precision table:", json.dumps(table))
    out = os.environ.get("AXI_PRECISION_TABLE")
    if out:
        with open(out, "w") as fh_:
            json.dump(table, fh_, indent=1)
    assert table["fp64"]["e_bd"] < 1e-10 and table["fp64"]["e_ff"] < 1e-10
    assert table["split7"]["e_bd"] < 1e-10 and table["split7"]["e_ff"] < 1e-10
    assert table["split8"]["e_bd"] < 1e-10
    assert table["split5"]["e_bd"] >= table["split8"]["e_bd"]
