"""Truncated-SVD form of the operator (AXI_PLAN_TSVD; Sec. 4.2: A_n^+ applied as
V Sigma^+ U^* x with a 1e-10 relative truncation) against the oracle: singular
values against LAPACK's on the oracle's modal matrices, orthonormal factors
that reconstruct R, Jacobi convergence, and the solution against the oracle's
truncated-SVD solve on boundary data."""
import dataclasses
import json
import os

import numpy as np
import pytest

import oracle as O
import synth
from test_gpu_parity import _e_bd

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _case(name):
    wl = synth.small_case() if name == "small" else synth.config_smooth()
    ob = wl.obstacles[0]
    coll, src, srcx = O.geometry(ob)
    if not ob.q:
        ob = dataclasses.replace(ob, q=O.choose_q(ob, coll, src, srcx))
    return wl, ob, coll, src, srcx


@pytest.mark.parametrize("name,prec", [("small", "fp64"), ("small", "split"), ("smooth", "fp64"),
                                       ("smooth", "split")])
def test_tsvd_operator(name, prec):
    from paper_1506_05083_gb300 import axi
    wl, ob, coll, src, srcx = _case(name)
    base = axi.PREC_FP64 if prec == "fp64" else axi.PREC_SPLIT_BF16
    op = axi.Operator([axi.spec_from_obstacle(wl.obstacles[0])], prec=base | axi.PLAN_TSVD)
    U, V, sg, sweeps = (t.cpu().numpy() for t in op.svd())
    Ap, tau, T, nb = op.factors()
    Ap = Ap.cpu().numpy().transpose(0, 2, 1)
    torch.cuda.synchronize()
    assert op.status() == 0
    A = O.system_matrix(ob, coll, src, srcx)
    n = A.shape[2]
    s_all = max(np.linalg.norm(A[d], 2) for d in range(A.shape[0]))   # the operator's sigma_max
    worst = {}
    for d in range(A.shape[0]):
        Ud, Vd = U[d].T, V[d].T                            # column-major storage -> [row][col]
        R = np.triu(Ap[d][:n])
        s_ora = np.linalg.svd(A[d], compute_uv=False)           # the oracle's matrix
        s_R = np.linalg.svd(R, compute_uv=False)                # the GPU's factor R
        smax = s_ora[0]
        # the Jacobi SVD of R against LAPACK on the same R (relative to the
        # mode's sigma_max); R against the oracle's matrix, relative to the
        # operator's sigma_max like the fill's e_A (high modes are orders of
        # magnitude smaller than mode 0)
        worst["sigma"] = max(worst.get("sigma", 0), np.abs(np.sort(sg[d])[::-1] - s_R).max() / smax)
        worst["sigma_R"] = max(worst.get("sigma_R", 0), np.abs(s_R - s_ora).max() / s_all)
        worst["orthU"] = max(worst.get("orthU", 0), np.abs(Ud.conj().T @ Ud - np.eye(n)).max())
        worst["orthV"] = max(worst.get("orthV", 0), np.abs(Vd.conj().T @ Vd - np.eye(n)).max())
        worst["recon"] = max(worst.get("recon", 0),
                             np.abs((Ud * sg[d]) @ Vd.conj().T - R).max() / np.abs(R).max())
    dirs = synth.plane_wave_directions(wl.n_waves, wl.wave_seed)
    coef = op.apply(op.incident(torch.tensor(dirs, device="cuda"))).cpu().numpy()
    torch.cuda.synchronize()
    assert op.status() == 0
    fh = O.rhs_modes(O.incident_samples(ob, coll, dirs))
    c_ora = O.solve_modes_tsvd(ob, A, fh)
    e = _e_bd(A, ob, coef, c_ora, fh)
    print(name, prec, json.dumps({k: float(v) for k, v in worst.items()}), "sweeps",
          int(sweeps.max()), "e_bd vs oracle tsvd", e)
    assert sweeps.max() < 40
    assert worst["sigma"] < 1e-12 and worst["sigma_R"] < 1e-13
    assert worst["orthU"] < 1e-12 and worst["orthV"] < 1e-12
    assert worst["recon"] < 1e-12
    assert e < 1e-10
