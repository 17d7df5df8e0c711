"""The mode-sharded operator (axi_plan_shard) on one GPU: the operators of
process 0 and 1 of 2 factor and apply disjoint modes; their coefficient
arrays sum to the unsharded operator's, mode by mode the same arithmetic."""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", ["fp64", "split"])
def test_sharded_operators_sum_to_the_whole(prec):
    from paper_1506_05083_gb300 import axi
    obs = [synth.small_case(seed=7).obstacles[0],
           synth.small_case(seed=11, k=2.0, M=44, N=36, P=20, bc=synth.BC_TRANSMISSION).obstacles[0]]
    specs = [axi.spec_from_obstacle(ob) for ob in obs]
    p = axi.PREC_FP64 if prec == "fp64" else axi.PREC_SPLIT_BF16
    whole = axi.Operator(specs, prec=p)
    parts = [axi.Operator(specs, prec=p, shard=(r, 2)) for r in range(2)]
    for i in range(len(obs)):
        dirs = torch.tensor(synth.plane_wave_directions(5, 80 + i), device="cuda")
        ref = whole.apply(whole.incident(dirs, obs=i), obs=i)
        got = sum(op.apply(op.incident(dirs, obs=i), obs=i) for op in parts)
        torch.cuda.synchronize()
        assert np.abs((got - ref).cpu().numpy()).max() <= 1e-14 * np.abs(ref.cpu().numpy()).max()
    for op in [whole] + parts:
        assert op.status() == 0
