"""Near-image sum (the action of A_else, Sec. 4.1) at every ring node: the
split-precision GEMM path against the direct FP64 path (all targets) and both
against the oracle's direct 3D sum (target subsample). Lattices with and
without the 90-degree symmetry, and P not divisible by 4."""
import math

import numpy as np
import pytest

import oracle as O
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _setup(wl_ob, W, seed):
    from paper_1506_05083_gb300 import axi
    spec = axi.spec_from_obstacle(wl_ob)
    op = axi.Operator([spec])
    rng = np.random.default_rng(seed)
    c = rng.standard_normal((W, spec.P, spec.cols)) + 1j * rng.standard_normal((W, spec.P, spec.cols))
    d = synth.plane_wave_directions(W, seed + 1)
    return axi, op, spec, c, d


@pytest.mark.parametrize("P,lat", [(16, (3.1, 3.1)), (16, (3.3, 2.9)), (18, (3.1, 3.1))])
def test_near_split_vs_fp64_vs_oracle(P, lat):
    ob = synth.small_case(seed=31, k=2.5, M=28, N=24, P=P).obstacles[0]
    axi, op, spec, c, d = _setup(ob, 5, 11)
    ct = torch.tensor(c, device="cuda")
    dt = torch.tensor(d, device="cuda")
    U64 = axi.near_image_sum(op, ct, lat, dt, slices=0).cpu().numpy()
    U6 = axi.near_image_sum(op, ct, lat, dt, slices=6).cpu().numpy()
    U7 = axi.near_image_sum(op, ct, lat, dt, slices=7).cpu().numpy()
    torch.cuda.synchronize()
    assert op.status() == 0
    scale = np.abs(U64).max()
    assert np.abs(U7 - U64).max() < 1e-11 * scale
    assert np.abs(U6 - U64).max() < 1e-10 * scale
    coll, src, srcx = O.geometry(ob)
    idx = np.arange(0, ob.M * ob.P, 5)
    ref = O.near_image_sum(ob, coll, src, c, d, lat, target_idx=idx)
    assert np.abs(U64[:, idx] - ref).max() < 1e-12 * np.abs(ref).max()
    assert np.abs(U7[:, idx] - ref).max() < 1e-11 * np.abs(ref).max()


def test_near_cup_scale_sampled():
    """The cup (N=360, M=432, P=180) with 256 waves, lattice period 13
    wavelengths, 6 digits: 2 waves (the first and the last) x 2048 seeded
    random targets of the 77,760 ring nodes against the oracle's direct 3D
    sum over the eight phased images (computed in blocks of 256 targets)."""
    wl = synth.config_cup_apply()
    ob = wl.obstacles[0]
    axi, op, spec, c, d = _setup(ob, wl.n_waves, 5)
    lat = wl.lattice
    U = axi.near_image_sum(op, torch.tensor(c, device="cuda"), lat,
                           torch.tensor(d, device="cuda"), slices=6).cpu().numpy()
    torch.cuda.synchronize()
    assert op.status() == 0
    coll, src, srcx = O.geometry(ob)
    rng = np.random.default_rng(3)
    idx = np.sort(rng.choice(ob.M * ob.P, 2048, replace=False))
    waves = [0, wl.n_waves - 1]
    ref = np.concatenate([O.near_image_sum(ob, coll, src, c[waves], d[waves], lat,
                                           target_idx=idx[b:b + 256])
                          for b in range(0, idx.size, 256)], axis=1)
    err = np.abs(U[waves][:, idx] - ref).max() / np.abs(ref).max()
    assert err < 1e-10, err
