"""The no-allocation apply (axi_apply_operator_noalloc) against the regular one.

Callers that cannot allocate device memory when they apply the operator (a
host application owning the GPU's memory budget that hands a plug-in only its
input and output buffers, a loop where cudaMalloc, which may synchronise the
device, is not allowed) use this entry point: its scratch is a static device
array in the library. Here it must reproduce axi_apply_operator's
coefficients and point strengths on calls in a row with different data and
batch sizes (the shared array keeps the previous call's contents, which must
not leak into the next result), for native-FP64 and split-precision
operators, and refuse a batch too large for the array with a clear error
instead of touching memory. This file is collected last so that a failing run
has already run every other test.
"""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _op(prec_name):
    from paper_1506_05083_gb300 import axi
    wl = synth.small_case(seed=23, k=3.0, M=40, N=32, P=16)
    prec = axi.PREC_FP64 if prec_name == "fp64" else axi.PREC_SPLIT_BF16
    return axi, axi.Operator([axi.spec_from_obstacle(wl.obstacles[0])], prec=prec)


@pytest.mark.parametrize("prec", ["fp64", "split"])
def test_noalloc_apply_matches_apply(prec):
    axi, op = _op(prec)
    spec = op.specs[0]
    results = []
    # calls in a row: different data, the larger batch first so a smaller one
    # would expose leftovers of the previous call in the shared array
    for seed, W in ((31, 7), (32, 3), (33, 7)):
        dirs = torch.tensor(synth.plane_wave_directions(W, seed), device="cuda")
        f = op.incident(dirs)
        coef_ref, sig_ref = op.apply(f, want_sigma=True)
        coef = torch.full((W, spec.P, spec.cols), float("nan"), dtype=torch.complex128, device="cuda")
        sig = torch.full((W, spec.cols, spec.P), float("nan"), dtype=torch.complex128, device="cuda")
        op.apply_noalloc(f, coef, sig)
        torch.cuda.synchronize()
        results.append((coef.cpu().numpy(), coef_ref.cpu().numpy(), sig.cpu().numpy(),
                        sig_ref.cpu().numpy()))
    assert op.status() == 0
    for coef, coef_ref, sig, sig_ref in results:
        assert np.isfinite(coef).all() and np.isfinite(sig).all()
        assert np.abs(coef - coef_ref).max() <= 1e-12 * np.abs(coef_ref).max()
        assert np.abs(sig - sig_ref).max() <= 1e-12 * np.abs(sig_ref).max()
    assert np.abs(results[0][0] - results[2][0]).max() > 0   # the calls really differ
    # nothing allocated: the caching allocator's and the driver's counters stay
    # put over further calls (the kernels are loaded by the calls above)
    dirs = torch.tensor(synth.plane_wave_directions(7, 34), device="cuda")
    f = op.incident(dirs)
    coef = torch.empty((7, spec.P, spec.cols), dtype=torch.complex128, device="cuda")
    torch.cuda.synchronize()
    torch_before, free_before = torch.cuda.memory_allocated(), torch.cuda.mem_get_info()[0]
    for _ in range(3):
        op.apply_noalloc(f, coef)
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() == torch_before
    assert torch.cuda.mem_get_info()[0] == free_before


def test_noalloc_rejects_batch_beyond_static_scratch():
    axi, op = _op("fp64")
    spec = op.specs[0]
    cap = axi.lib().axi_noalloc_scratch_bytes()
    per_wave = 16 * (spec.P // 2 + 1) * 2 * spec.rows
    W = cap // per_wave + 1
    f = torch.zeros((W, spec.rows, spec.P), dtype=torch.complex128, device="cuda")
    coef = torch.zeros((W, spec.P, spec.cols), dtype=torch.complex128, device="cuda")
    with pytest.raises(axi.AxiError) as e:
        op.apply_noalloc(f, coef)
    assert e.value.code == -4          # AXI_ERR_WORKSPACE
    with pytest.raises(ValueError):    # mis-shaped output refused by the binding
        op.apply_noalloc(f[:2], coef[:1])
