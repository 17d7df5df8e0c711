"""The ring-kernel sin/cos routines (csrc/trig.cuh) against CUDA's sincos
(torch.sin / torch.cos on the device) and numpy's, through the diagnostics
entry points: axi_diag_sincos (Cody-Waite reduction + Taylor series),
axi_diag_sincos_table (1024-entry table + short series + angle addition) and
axi_diag_sincos_fixed (the same reduction, then series and angle addition in
64-bit fixed point: the form the split fill's samples use).

Bound: absolute error <= 1e-15 (about 4.5 units of 2^-52 at 1.0) for
|x| <= 2000, which covers k R for every workload here (k <= 45, R <= 10).
"""
import ctypes as C
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("entry", ["axi_diag_sincos", "axi_diag_sincos_table", "axi_diag_sincos_fixed"])
def test_sincos_ring_against_cuda_and_numpy(entry):
    from paper_1506_05083_gb300 import axi
    rng = np.random.default_rng(3)
    x = np.concatenate([
        rng.uniform(0.0, 2000.0, 200_000),
        rng.uniform(-50.0, 50.0, 50_000),
        np.arange(-40, 41) * (math.pi / 4),                  # octant boundaries
        np.arange(-40, 41) * (math.pi / 2) + 1e-9,
        np.arange(-3000, 3001) * (2 * math.pi / 1024),        # table points
        np.arange(-3000, 3001) * (2 * math.pi / 1024) + math.pi / 1024,   # half-way
        [0.0, -0.0, 1e-300, 5e-324, 1e-8, math.pi, 1000.0 * math.pi],
    ])
    xd = torch.tensor(x, device="cuda")
    s = torch.empty_like(xd)
    c = torch.empty_like(xd)
    code = getattr(axi.lib(), entry)(C.c_void_p(xd.data_ptr()), len(x), C.c_void_p(s.data_ptr()),
                                     C.c_void_p(c.data_ptr()), None)
    assert code == axi.OK
    torch.cuda.synchronize()
    s_cuda, c_cuda = torch.sin(xd), torch.cos(xd)
    for ours, ref in ((s, s_cuda), (c, c_cuda)):
        assert (ours - ref).abs().max().item() <= 1e-15
    s_np, c_np = np.sin(x), np.cos(x)
    assert np.abs(s.cpu().numpy() - s_np).max() <= 1e-15
    assert np.abs(c.cpu().numpy() - c_np).max() <= 1e-15
    # Pythagorean identity as an independent check
    assert np.abs(s.cpu().numpy() ** 2 + c.cpu().numpy() ** 2 - 1.0).max() <= 1e-15


@pytest.mark.parametrize("entry", ["axi_diag_sincos", "axi_diag_sincos_table", "axi_diag_sincos_fixed"])
def test_diag_sincos_arguments(entry):
    from paper_1506_05083_gb300 import axi
    f = getattr(axi.lib(), entry)
    assert f(None, -1, None, None, None) == axi.ERR_ARG
    assert f(None, 0, None, None, None) == axi.OK
    assert f(None, 5, None, None, None) == axi.ERR_ARG
