"""Full-scale workloads against the oracle: the 64-obstacle batch (17 sampled
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


GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "batched_residuals.json")
# 17 of the 64 obstacles: P = 240 (17, 51, 61, 14, 35, 5), the two largest N
# the oracle factors in seconds (5: N = 359, 59: N = 350), transmission
# (7, 58, 50, 14, 44, 34, 35), k from 3 to 27, resolved and unresolved bodies
BATCH_CHECKED = (15, 24, 9, 45, 17, 28, 51, 7, 58, 61, 50, 14, 44, 34, 35, 59, 5)


@pytest.mark.parametrize("prec", ["fp64", "split"])
def test_batched_64_obstacles_sampled(prec):
    """All 64 obstacles in one plan; 17 of them checked against the oracle.

    The batched workload draws N, P and k independently, so some obstacles are
    unresolved (oracle residual above 1e-6) and their least-squares solutions
    are sensitive to rounding-level changes of the matrix. The oracle's
    residual r and its sensitivity s (e_bd after a u*max|A| normwise
    perturbation of every modal matrix) come from tests/golden/
    batched_residuals.json, written by the committed oracle-only script
    beside it. Bar: e_bd <= max(1e-10, 1e3 s) for every obstacle: 1e-10
    where the discrete problem is conditioned to that level, else what a
    backward-stable FP64 solver can reach (the fill's parity bar, 1e-13
    max|A|, is ~1e3 u). The residual r only labels obstacles as resolved
    (r < 1e-6) in the report; a resolved body can still be ill conditioned.
    """
    from paper_1506_05083_gb300 import axi
    golden = json.load(open(GOLDEN))
    wl = synth.config_batched()
    specs = [axi.spec_from_obstacle(ob) for ob in wl.obstacles]
    p = axi.PREC_FP64 if prec == "fp64" else axi.PREC_SPLIT_BF16
    op = axi.Operator(specs, prec=p)
    torch.cuda.synchronize()
    assert op.status() == 0
    unresolved = sum(1 for g in golden.values() if g["residual"] >= 1e-6)
    print(f"batched workload: {unresolved} of {len(golden)} obstacles unresolved (residual >= 1e-6)")
    report = []
    for i in BATCH_CHECKED:
        g = golden[str(i)]
        ob, coll, src, A, fac = _oracle(wl.obstacles[i])
        assert specs[i].q == ob.q == g["q"]
        dirs = synth.plane_wave_directions(4, 500 + i)
        coef = op.apply(op.incident(torch.tensor(dirs, device="cuda"), obs=i), obs=i).cpu().numpy()
        fh = O.rhs_modes(O.incident_samples(ob, coll, dirs))
        c_ora = O.solve_modes(ob, fac, fh)
        e = _e_bd(A, ob, coef, c_ora, fh)
        bar = max(1e-10, 1e3 * g["sensitivity"])
        report.append((i, g["N"], g["P"], g["bc"], g["residual"], g["sensitivity"], e, bar))
    torch.cuda.synchronize()
    assert op.status() == 0
    for row in report:
        print("obstacle %d N=%d P=%d bc=%d residual %.1e sensitivity %.1e e_bd %.2e bar %.1e" % row)
    for i, N, P, bc, r, s_, e, bar in report:
        assert e <= bar, (i, e, bar)


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
