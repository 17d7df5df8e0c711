"""Failure paths of the device code, exercised without faulting or hanging the
GPU: a bounded device wait that runs out (a host-set short limit on an
mbarrier nothing completes) must return with AXI_ERR_TIMEOUT latched and the
context usable; a non-finite modal matrix must surface as AXI_ERR_NUMERIC;
the next build clears the status word. Also: factoring the oracle's own modal
matrices checks the QR and the apply independently of the GPU fill."""
import dataclasses

import numpy as np
import pytest

import oracle as O
import synth
from test_gpu_parity import _e_bd

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

AXI_ERR_TIMEOUT, AXI_ERR_NUMERIC = -6, -7


def _small(prec_name="fp64"):
    from paper_1506_05083_gb300 import axi
    ob = synth.small_case().obstacles[0]
    prec = axi.PREC_FP64 if prec_name == "fp64" else axi.PREC_SPLIT_BF16
    return axi, ob, axi.Operator([axi.spec_from_obstacle(ob)], prec=prec)


def test_bounded_wait_times_out_and_context_survives():
    axi, ob, op = _small()
    torch.cuda.synchronize()
    assert op.status() == 0
    op.diag_wait_timeout(2_000_000)          # about a millisecond of SM clocks
    torch.cuda.synchronize()
    assert op.status() == AXI_ERR_TIMEOUT
    # the context is intact: rebuild (clears the word) and solve
    op.refactor()
    dirs = synth.plane_wave_directions(3, 41)
    coef = op.apply(op.incident(torch.tensor(dirs, device="cuda"))).cpu().numpy()
    torch.cuda.synchronize()
    assert op.status() == 0
    coll, src, srcx = O.geometry(ob)
    ob = dataclasses.replace(ob, q=O.choose_q(ob, coll, src, srcx))
    A, fac = O.factor_operator(ob, coll, src, srcx)
    fh = O.rhs_modes(O.incident_samples(ob, coll, dirs))
    assert _e_bd(A, ob, coef, O.solve_modes(ob, fac, fh), fh) < 1e-10


@pytest.mark.parametrize("prec", ["fp64", "split"])
def test_non_finite_modal_matrix_is_reported(prec):
    axi, ob, op = _small(prec)
    A = op.fill_modes()
    A[3, 5, 7] = complex("nan")
    op.refactor_from_modes([A])
    torch.cuda.synchronize()
    assert op.status() == AXI_ERR_NUMERIC
    op.refactor()
    torch.cuda.synchronize()
    assert op.status() == 0


@pytest.mark.parametrize("prec", ["fp64", "split"])
def test_factor_oracle_modal_matrices(prec):
    """The oracle's modal matrices factored and applied on the GPU match the
    oracle's own least-squares solution (no GPU fill involved)."""
    axi, ob, op = _small(prec)
    coll, src, srcx = O.geometry(ob)
    ob = dataclasses.replace(ob, q=O.choose_q(ob, coll, src, srcx))
    A, fac = O.factor_operator(ob, coll, src, srcx)            # [D][rows][cols]
    modes = torch.tensor(np.ascontiguousarray(A.transpose(0, 2, 1)), device="cuda")
    op.refactor_from_modes([modes])
    dirs = synth.plane_wave_directions(4, 43)
    coef = op.apply(op.incident(torch.tensor(dirs, device="cuda"))).cpu().numpy()
    torch.cuda.synchronize()
    assert op.status() == 0
    fh = O.rhs_modes(O.incident_samples(ob, coll, dirs))
    assert _e_bd(A, ob, coef, O.solve_modes(ob, fac, fh), fh) < 1e-11
    with pytest.raises(ValueError):
        op.refactor_from_modes([modes[:1]])
