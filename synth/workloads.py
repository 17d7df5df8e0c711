"""Workload definitions for the one-obstacle MFS solution operator.

Shapes follow the test bodies of the paper (Sec. 2, Fig. 2 caption; Sec. 3.3):
  * 'polar': r(t) = r0 + sum_j amp_j cos(j t), rho = r sin t, z = r cos t,
    t in [0, pi] measured from the +z axis (a sphere when all amp_j are 0);
  * 'cup':   r(t) = 1 - a erf((t - pi/2)/a), angle theta(t) from the +z axis
    as in the Fig. 2(c) caption, half-thickness a, opening half-angle b.
Only parameters live here; evaluating the curves is the method's business.

Every random quantity is drawn from numpy's PCG64 generator with a stated
seed, so the CUDA path and the oracle see identical inputs.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional, Tuple

import numpy as np

SHAPE_POLAR = 0
SHAPE_CUP = 1

BC_NEUMANN = 0
BC_TRANSMISSION = 1


@dataclass
class Obstacle:
    """One axisymmetric obstacle and its discretisation parameters."""
    shape: int                    # SHAPE_POLAR or SHAPE_CUP
    params: List[float]           # polar: [r0, amp_1, ..., amp_J]; cup: [a, b]
    k: float                      # exterior wavenumber
    M: int                        # collocation points on the generating curve
    N: int                        # proxy (MFS source) rings
    P: int                        # azimuthal modes, even
    q: int                        # azimuthal quadrature nodes of the fill, even, q >= P
    tau: float                    # complexification distance of the proxies
    bc: int = BC_NEUMANN
    k_minus: float = 0.0          # interior wavenumber (transmission only)


@dataclass
class Workload:
    name: str
    obstacles: List[Obstacle]
    n_waves: int
    wave_seed: int
    lattice: Optional[Tuple[float, float]] = None   # (e_x, e_y) for the near-image sum
    meta: dict = field(default_factory=dict)


def plane_wave_directions(n: int, seed: int) -> np.ndarray:
    """[n][3] unit incident directions: theta ~ U[0, pi/2], phi ~ U[0, 2 pi).

    theta is the polar angle from +z, phi the azimuth; uniform in the angles.
    """
    rng = np.random.default_rng(seed)
    th = rng.uniform(0.0, math.pi / 2, n)
    ph = rng.uniform(0.0, 2 * math.pi, n)
    return np.stack([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)], axis=1)


def sphere(k=2.0, M=72, N=60, P=32, q=128) -> Obstacle:
    # proxies on the sphere of radius 0.7: complexification distance ln(1/0.7)
    return Obstacle(SHAPE_POLAR, [1.0], k, M, N, P, q, math.log(1 / 0.7))


def perturbed_polar(seed: int, k: float, M: int, N: int, P: int, q: int, tau=0.1,
                    amp=0.2, J=4) -> Obstacle:
    rng = np.random.default_rng(seed)
    a = rng.uniform(-1.0, 1.0, J)
    return Obstacle(SHAPE_POLAR, [1.0] + [amp * float(x) for x in a], k, M, N, P, q, tau)


def cup(k=25.0, M=432, N=360, P=180, q=1000, tau=0.05, a=0.2, b=math.pi / 2) -> Obstacle:
    return Obstacle(SHAPE_CUP, [a, b], k, M, N, P, q, tau)


def config_sphere() -> Workload:
    """Sound-hard unit sphere, k=2, N=60, M=72, P=32, one seeded plane wave."""
    return Workload("sphere_k2_N60_M72_P32", [sphere()], 1, 1)


def config_smooth() -> Workload:
    """Seeded smooth body r=1+0.2 sum a_j cos(js), k=10, N=180, M=216, P=120, 16 waves."""
    return Workload("smooth_k10_N180_M216_P120_W16",
                    [perturbed_polar(2, 10.0, 216, 180, 120, 400)], 16, 3)


def config_cup() -> Workload:
    """Hemispherical thick-shell cup, k=25, N=360, M=432, P=180 (NP=64800)."""
    return Workload("cup_k25_N360_M432_P180", [cup()], 16, 5)


def config_cup_apply() -> Workload:
    """Cup factors with 256 seeded waves and the 3x3 near-image lattice sum."""
    k = 25.0
    period = 13 * 2 * math.pi / k
    return Workload("cup_k25_apply_W256_lattice13", [cup()], 256, 5, lattice=(period, period))


def q_candidates(lo: int) -> int:
    """Smallest even integer >= lo of the form 2^a 3^b 5^c."""
    n = max(2, int(lo))
    while True:
        m = n
        for p in (2, 3, 5):
            while m % p == 0:
                m //= p
        if m == 1 and n % 2 == 0:
            return n
        n += 1


def config_batched(n_obs=64, seed=4, max_N=360) -> Workload:
    """64 seeded obstacles of uneven size, wavenumber and boundary condition.

    N ~ U[60, max_N], M = ceil(1.2 N), P from {32, 64, 120, 180, 240},
    k ~ U[1, 30], transmission with probability 1/2 (k_minus = 1.5 k).
    q is recorded as 0 here: it is chosen from the geometry by the rule of
    Theorem 1 on each side.
    """
    rng = np.random.default_rng(seed)
    obs = []
    for i in range(n_obs):
        N = int(rng.integers(60, max_N + 1))
        M = int(math.ceil(1.2 * N))
        P = int(rng.choice([32, 64, 120, 180, 240]))
        k = float(rng.uniform(1.0, 30.0))
        bc = BC_TRANSMISSION if rng.uniform() < 0.5 else BC_NEUMANN
        a = rng.uniform(-1.0, 1.0, 4)
        # amplitude 0.1 keeps r >= 0.6 so both proxy curves (+-tau) stay off the axis
        o = Obstacle(SHAPE_POLAR, [1.0] + [0.1 * float(x) for x in a], k, M, N, P, 0, 0.1,
                     bc=bc, k_minus=1.5 * k if bc == BC_TRANSMISSION else 0.0)
        obs.append(o)
    return Workload("batched64_N60-360_P32-240_k1-30", obs, 4, 6)


def small_case(seed=7, k=3.0, M=40, N=32, P=16, q=0, bc=BC_NEUMANN) -> Workload:
    """A small perturbed body for quick parity tests (several tiles, ragged tail).

    q = 0: each side picks q from its geometry by the Theorem 1 rule.
    """
    o = perturbed_polar(seed, k, M, N, P, q)
    if bc == BC_TRANSMISSION:
        o.bc = BC_TRANSMISSION
        o.k_minus = 1.5 * k
    return Workload(f"small_seed{seed}_M{M}_N{N}_P{P}", [o], 4, seed + 100)
