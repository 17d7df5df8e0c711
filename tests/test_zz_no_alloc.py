"""The no-allocation apply (axi_apply_operator_noalloc) against the regular one.

Callers that cannot allocate device memory when they apply the operator (a
host application owning the GPU's memory budget, a loop where cudaMalloc is
not allowed) use this entry point: its scratch is a static device array in
the library. Here it must reproduce axi_apply_operator's coefficients and
point strengths on two calls in a row (the shared array keeps the previous
call's contents, which must not leak into the next result), and refuse a
batch too large for the array with a clear error instead of touching memory.
This file is collected last so that a failing run has already run every
other test.
"""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_noalloc_apply_matches_apply_twice():
    from paper_1506_05083_gb300 import axi
    wl = synth.small_case(seed=23, k=3.0, M=40, N=32, P=16)
    op = axi.Operator([axi.spec_from_obstacle(wl.obstacles[0])])
    spec = op.specs[0]
    results = []
    for seed in (31, 32):   # two calls in a row, different data
        dirs = torch.tensor(synth.plane_wave_directions(5, seed), device="cuda")
        f = op.incident(dirs)
        coef_ref, sig_ref = op.apply(f, want_sigma=True)
        coef = torch.full((5, spec.P, spec.cols), float("nan"), dtype=torch.complex128, device="cuda")
        sig = torch.full((5, spec.cols, spec.P), float("nan"), dtype=torch.complex128, device="cuda")
        op.apply_noalloc(f, coef, sig)
        torch.cuda.synchronize()
        results.append((coef.cpu().numpy(), coef_ref.cpu().numpy(), sig.cpu().numpy(),
                        sig_ref.cpu().numpy()))
    assert op.status() == 0
    for coef, coef_ref, sig, sig_ref in results:
        assert np.isfinite(coef).all() and np.isfinite(sig).all()
        assert np.abs(coef - coef_ref).max() <= 1e-12 * np.abs(coef_ref).max()
        assert np.abs(sig - sig_ref).max() <= 1e-12 * np.abs(sig_ref).max()
    assert np.abs(results[0][0] - results[1][0]).max() > 0   # the two calls really differ


def test_noalloc_rejects_batch_beyond_static_scratch():
    from paper_1506_05083_gb300 import axi
    wl = synth.small_case(seed=23, k=3.0, M=40, N=32, P=16)
    op = axi.Operator([axi.spec_from_obstacle(wl.obstacles[0])])
    spec = op.specs[0]
    cap = axi.lib().axi_noalloc_scratch_bytes()
    per_wave = 16 * (spec.P // 2 + 1) * 2 * spec.rows
    W = cap // per_wave + 1
    f = torch.zeros((W, spec.rows, spec.P), dtype=torch.complex128, device="cuda")
    coef = torch.zeros((W, spec.P, spec.cols), dtype=torch.complex128, device="cuda")
    with pytest.raises(axi.AxiError) as e:
        op.apply_noalloc(f, coef)
    assert e.value.code == -2          # AXI_ERR_SHAPE
