"""The build (fill + look-ahead QR with its side-stream fork/join) and the
apply captured in CUDA graphs and replayed give the same results as direct
calls, for both arithmetic modes."""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", ["fp64", "split"])
def test_graph_replay_matches_direct(prec):
    from paper_1506_05083_gb300 import axi
    wl = synth.small_case(seed=29, k=3.0, M=72, N=60, P=24)
    p = axi.PREC_FP64 if prec == "fp64" else axi.PREC_SPLIT_BF16
    op = axi.Operator([axi.spec_from_obstacle(wl.obstacles[0])], prec=p)
    spec = op.specs[0]
    dirs = torch.tensor(synth.plane_wave_directions(6, 77), device="cuda")
    coef = torch.empty((6, spec.P, spec.cols), dtype=torch.complex128, device="cuda")
    scratch = torch.empty(op.apply_scratch_bytes(6), dtype=torch.uint8, device="cuda")
    op.refactor()
    direct = op.apply(op.incident(dirs), scratch=scratch).clone()
    factors = op.factors()[0].clone()
    torch.cuda.synchronize()
    gb, ga = torch.cuda.CUDAGraph(), torch.cuda.CUDAGraph()
    with torch.cuda.graph(gb):
        op.refactor()
    with torch.cuda.graph(ga):
        op.apply(op.incident(dirs), scratch=scratch, coef=coef)
    for _ in range(3):
        op.factors()[0].zero_()
        coef.zero_()
        gb.replay()
        ga.replay()
    torch.cuda.synchronize()
    assert op.status() == 0
    assert torch.equal(op.factors()[0], factors)
    assert torch.equal(coef, direct)
