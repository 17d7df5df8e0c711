"""Pins of the oracle's spherical-wave block B~ (Sec. 4, eq. urep; Sec. 4.1)
against facts fixed outside it (no GPU): closed forms of the special
functions, the plane-wave (Rayleigh) expansion, and the oracle's own
independent incident-data path."""
import math

import numpy as np
import pytest

import oracle as O
import synth
from oracle import periodizing as OP


def _small(bc=0, P=32, k=3.0):
    wl = synth.small_case(seed=7, k=k, M=40, N=32, P=P, bc=bc)
    ob = wl.obstacles[0]
    coll, src, srcx = O.geometry(ob)
    return ob, coll


def test_spherical_bessel_closed_forms():
    x = np.array([0.3, 1.0, 2.7, 9.5, 31.0])
    s, c = np.sin(x), np.cos(x)
    assert np.allclose(OP.sph_jn(0, x), s / x, rtol=1e-14, atol=0)
    assert np.allclose(OP.sph_jn(1, x), s / x**2 - c / x, rtol=1e-13, atol=1e-16)
    assert np.allclose(OP.sph_jn(2, x), (3 / x**3 - 1 / x) * s - 3 * c / x**2, rtol=1e-12, atol=1e-16)
    assert np.allclose(OP.sph_jn(0, x, derivative=True), -OP.sph_jn(1, x), rtol=1e-14, atol=1e-17)


def test_spherical_harmonics_closed_forms():
    th, ph = 0.83, 2.1
    st, ct, e = math.sin(th), math.cos(th), np.exp(1j * ph)
    cases = {
        (0, 0): 0.5 / math.sqrt(math.pi),
        (1, 0): 0.5 * math.sqrt(3 / math.pi) * ct,
        (1, 1): -0.5 * math.sqrt(1.5 / math.pi) * st * e,          # Condon-Shortley phase
        (1, -1): 0.5 * math.sqrt(1.5 / math.pi) * st / e,
        (2, 2): 0.25 * math.sqrt(7.5 / math.pi) * st**2 * e**2,
        (2, 1): -0.5 * math.sqrt(7.5 / math.pi) * st * ct * e,
    }
    for (l, m), ref in cases.items():
        assert abs(OP.sph_y(l, m, th, ph)[0] - ref) < 1e-15


@pytest.mark.parametrize("d", [(0.0, 0.0, 1.0), (0.36, -0.48, 0.8), (1.0, 0.0, 0.0)])
def test_plane_wave_expansion_value_and_normal_derivative(d):
    """e^{ik d.x} = sum_lm d_lm j_l(kr) Y_lm(x^) and its gradient i k d e^{ik d.x}:
    pins the value and the chain-rule gradient of the spherical waves."""
    rng = np.random.default_rng(3)
    k, p = 2.5, 34
    x = rng.uniform(-1.2, 1.2, (40, 3))
    nvec = rng.normal(size=(40, 3))
    nvec /= np.linalg.norm(nvec, axis=1, keepdims=True)
    d = np.asarray(d)
    coef = OP.plane_wave_coefficients(p, d)
    u = np.zeros(40, dtype=np.complex128)
    dn = np.zeros(40, dtype=np.complex128)
    for l in range(p + 1):
        for m in range(-l, l + 1):
            v, g = OP.sph_wave_value_grad(l, m, k, x)
            u += coef[l * l + l + m] * v
            dn += coef[l * l + l + m] * np.sum(g * nvec, axis=1)
    ref = np.exp(1j * k * (x @ d))
    assert np.abs(u - ref).max() < 1e-13
    assert np.abs(dn - 1j * k * (nvec @ d) * ref).max() < 1e-12


@pytest.mark.parametrize("bc", [0, 1])
def test_btilde_block_structure(bc):
    """Only m = n survives the mean over phi (axis on the expansion's z axis),
    and the surviving entries are real for real k."""
    ob, coll = _small(bc=bc, P=16)
    p = 6
    B = OP.btilde(ob, coll, p, q=64, rows=range(0, 40, 5))
    scale = np.abs(B).max()
    for n in range(B.shape[0]):
        keep = OP.btilde_columns(p, n)
        mask = np.ones(B.shape[2], bool)
        mask[keep] = False
        assert np.abs(B[n][:, mask]).max() < 1e-14 * scale
        if keep.size:
            assert np.abs(B[n][:, keep].imag).max() < 1e-14 * scale


@pytest.mark.parametrize("bc", [0, 1])
def test_btilde_reproduces_incident_modes(bc):
    """B~ applied to a plane wave's spherical-wave coefficients gives the
    plane wave's modal boundary data, computed independently by
    `incident_samples` (value, normal derivative at the ring nodes) and
    `rhs_modes` (the DFT over phi), which hold minus that data."""
    ob, coll = _small(bc=bc, P=32)
    p = 30
    d = np.array([math.sin(0.3), 0.0, math.cos(0.3)])
    B = OP.btilde(ob, coll, p, q=96, modes=range(0, 6))
    fh = O.rhs_modes(O.incident_samples(ob, coll, d[None, :]))[0]     # [P][rows]
    coef = OP.plane_wave_coefficients(p, d)
    for n in range(6):
        got = B[n] @ coef
        assert np.abs(got + fh[n]).max() < 1e-12 * np.abs(fh[0]).max()


def test_gauss_nodes_two_point_rule():
    nodes = OP.wall_nodes(2.0, 4.0, 3.0, 2)
    g = 1.0 / math.sqrt(3.0)
    assert np.allclose(np.sort(np.unique(nodes["T"][:, 0])), [-g, g], atol=1e-15)
    assert np.allclose(np.sort(np.unique(nodes["L"][:, 2])), [-3 * g, 3 * g], atol=1e-15)
    assert np.allclose(nodes["R"][:, 0], 1.0) and np.allclose(nodes["F"][:, 1], 2.0)


@pytest.mark.parametrize("up", [True, False])
def test_q_quasi_periodic_plane_wave(up):
    """A plane wave e^{ik d.x} is quasi-periodic with alpha = e^{ik d_x e_x},
    beta = e^{ik d_y e_y} (eq. per) and is the (0,0) Rayleigh-Bloch wave on
    the wall it leaves through: with its spherical-wave coefficients and that
    mode's amplitude, every discrepancy row (eqs. qp1-qp4) and the Cauchy rows
    of that wall (eqs. T-nD) vanish, and the other wall's rows carry the wave."""
    k, p, ex, ey, z0, m1, n0 = 3.0, 30, 2.0, 1.7, 1.5, 6, 3
    d = np.array([0.36, -0.28, math.sqrt(1 - 0.36**2 - 0.28**2)])
    if not up:
        d[2] = -d[2]
    kx, ky = k * d[0], k * d[1]
    Q, modes = OP.q_matrix(k, p, kx, ky, ex, ey, z0, m1, n0)
    nh, nrb, nr = OP.n_harmonics(p), modes.shape[0], m1 * m1
    j0 = int(np.where((modes[:, 0] == 0) & (modes[:, 1] == 0))[0][0])
    xi = np.zeros(nh + 2 * nrb, dtype=np.complex128)
    xi[:nh] = OP.plane_wave_coefficients(p, d)
    if up:
        xi[nh + j0] = np.exp(1j * k * d[2] * z0)
    else:
        xi[nh + nrb + j0] = np.exp(-1j * k * d[2] * z0)
    r = Q @ xi
    nodes = OP.wall_nodes(ex, ey, z0, m1)
    zero_blocks = [0, 1, 2, 3, 4, 5] if up else [0, 1, 2, 3, 6, 7]
    for b in zero_blocks:
        assert np.abs(r[b * nr:(b + 1) * nr]).max() < 1e-12, b
    f = "D" if up else "T"
    b0 = 6 if up else 4
    u = np.exp(1j * k * (nodes[f] @ d))
    assert np.abs(r[b0 * nr:(b0 + 1) * nr] - u).max() < 1e-12
    assert np.abs(r[(b0 + 1) * nr:(b0 + 2) * nr] - 1j * k * d[2] * u).max() < 1e-12


def test_c_rows_match_potential_image_sums():
    """C c equals the 3 x 3 phased image sums of the field `potential`
    computes from the same coefficients (point strengths, point sources;
    pinned against the sphere series), combined into the discrepancy and
    Cauchy rows."""
    wl = synth.small_case(seed=7, k=3.0, M=40, N=32, P=16)
    ob = wl.obstacles[0]
    coll, src, srcx = O.geometry(ob)
    kx, ky, ex, ey, z0, m1 = 1.1, -0.7, 2.6, 2.3, 1.6, 4
    C = OP.c_matrix(ob, src, kx, ky, ex, ey, z0, m1)
    rng = np.random.default_rng(5)
    coef = rng.normal(size=(1, ob.P, ob.N)) + 1j * rng.normal(size=(1, ob.P, ob.N))
    got = C @ coef.reshape(-1)
    nodes = OP.wall_nodes(ex, ey, z0, m1)
    alpha, beta = np.exp(1j * kx * ex), np.exp(1j * ky * ey)

    def u(X, axis=None):
        out = 0.0
        for a in (-1, 0, 1):
            for b in (-1, 0, 1):
                nrm = None
                if axis is not None:
                    nrm = np.zeros_like(X)
                    nrm[:, axis] = 1.0
                out = out + alpha ** a * beta ** b * O.potential(
                    ob, src, coef, X - np.array([a * ex, b * ey, 0.0]), qe=ob.P, normals=nrm)[0]
        return out

    want = np.concatenate([u(nodes["R"]) - alpha * u(nodes["L"]), u(nodes["R"], 0) - alpha * u(nodes["L"], 0),
                           u(nodes["F"]) - beta * u(nodes["B"]), u(nodes["F"], 1) - beta * u(nodes["B"], 1),
                           u(nodes["T"]), u(nodes["T"], 2), u(nodes["D"]), u(nodes["D"], 2)])
    assert np.abs(got - want).max() < 1e-12 * np.abs(want).max()


def test_q_pinv_solve_prescribed_singular_values():
    rng = np.random.default_rng(9)
    m, n = 40, 24
    U, _ = np.linalg.qr(rng.normal(size=(m, n)) + 1j * rng.normal(size=(m, n)))
    V, _ = np.linalg.qr(rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n)))
    s = np.concatenate([np.logspace(0, -3, 12), np.logspace(-13, -14, n - 12)])   # a clear gap
    A = (U * s) @ V.conj().T
    x_true = V[:, :12] @ (rng.normal(size=12) + 0j)          # in the span of the kept values
    X, sv = OP.q_pinv_solve(A, (A @ x_true)[:, None], 1e-10)
    assert np.allclose(sv[:12], s[:12], rtol=1e-12)
    assert np.abs(sv[12:] - s[12:]).max() < 1e-15
    assert np.abs(X[:, 0] - x_true).max() < 1e-11


def test_btilde_samples_direct_expansion():
    """B~ d carried back to the P ring nodes equals the normal derivative of
    the truncated expansion sum d_lm u_lm evaluated at those nodes directly
    (p < P/2, so every mode the waves hold is among the P modes): pins the
    mode index of each column, the sign of the negative modes and the sign of
    the transform back to samples."""
    P, p = 16, 6
    ob, coll = _small(P=P)
    rng = np.random.default_rng(11)
    d = rng.normal(size=(2, OP.n_harmonics(p))) + 1j * rng.normal(size=(2, OP.n_harmonics(p)))
    X, Nv = OP._ring_nodes(coll, P)                                     # [M][P][3]
    ref = np.zeros((2, coll.shape[0], P), dtype=np.complex128)
    for l in range(p + 1):
        for m in range(-l, l + 1):
            _, g = OP.sph_wave_value_grad(l, m, ob.k, X)
            dn = np.sum(g * Nv, axis=-1)
            ref += d[:, l * l + l + m][:, None, None] * dn[None]
    got = OP.btilde_samples(ob, coll, p, d)
    assert np.abs(got - ref).max() < 1e-12 * np.abs(ref).max()


def test_periodic_solve_dense_assembly():
    """The dense matrix of eq. iter's operator (columns = images of the unit
    vectors) reproduces the operator on a random vector, and its solution
    leaves a residual at rounding level: pins the assembly's orientation."""
    wl = synth.small_case(seed=7, k=3.0, M=20, N=16, P=8)
    ob = wl.obstacles[0]
    coll, src, srcx = O.geometry(ob)
    ob.q = O.choose_q(ob, coll, src, srcx)
    A, fac = O.factor_operator(ob, coll, src, srcx)
    d = np.array([0.36, -0.28, np.sqrt(1 - 0.36**2 - 0.28**2)])
    ex, ey, z0, m1, n0, p = 2.6, 2.3, 1.6, 6, 2, 3
    C = OP.c_matrix(ob, src, ob.k * d[0], ob.k * d[1], ex, ey, z0, m1)
    Q, _ = OP.q_matrix(ob.k, p, ob.k * d[0], ob.k * d[1], ex, ey, z0, m1, n0)
    rng = np.random.default_rng(2)
    f = rng.normal(size=(2, ob.M, ob.P)) + 1j * rng.normal(size=(2, ob.M, ob.P))
    et, eta, xi, Aop = OP.periodic_solve_dense(ob, coll, src, fac, f, d, (ex, ey), C, Q, p)
    v = rng.normal(size=(1, ob.M, ob.P)) + 1j * rng.normal(size=(1, ob.M, ob.P))
    Av = OP.periodic_operator_apply(ob, coll, src, fac, v, d[None], (ex, ey), C, Q, p)
    assert np.abs(Aop @ v.ravel() - Av.ravel()).max() < 1e-12 * np.abs(Av).max()
    back = OP.periodic_operator_apply(ob, coll, src, fac, et, np.stack([d, d]), (ex, ey), C, Q, p)
    assert np.abs(back - f).max() < 1e-10 * np.abs(f).max()
    assert xi.shape == (2, Q.shape[1]) and eta.shape == (2, ob.P, ob.N)


def test_a0_plus_forms_agree_when_nothing_is_truncated():
    """With every modal singular value above the 1e-10 cutoff, the truncated-
    SVD A_0^+ (("tsvd", A)) and the QR solve give the same eq. iter operator:
    pins the dispatch between the two forms."""
    wl = synth.small_case(seed=7, k=3.0, M=20, N=16, P=8)
    ob = wl.obstacles[0]
    coll, src, srcx = O.geometry(ob)
    ob.q = O.choose_q(ob, coll, src, srcx)
    A, fac = O.factor_operator(ob, coll, src, srcx)
    assert min(np.linalg.svd(A[d], compute_uv=False)[-1] / np.linalg.norm(A[d], 2)
               for d in range(A.shape[0])) > 1e-8
    d = np.array([0.36, -0.28, np.sqrt(1 - 0.36**2 - 0.28**2)])
    ex, ey, z0, m1, n0, p = 2.6, 2.3, 1.6, 6, 2, 3
    C = OP.c_matrix(ob, src, ob.k * d[0], ob.k * d[1], ex, ey, z0, m1)
    Q, _ = OP.q_matrix(ob.k, p, ob.k * d[0], ob.k * d[1], ex, ey, z0, m1, n0)
    g = np.random.default_rng(4).normal(size=(2, ob.M, ob.P)) + 0j
    y_qr = OP.periodic_operator_apply(ob, coll, src, fac, g, np.stack([d, d]), (ex, ey), C, Q, p)
    y_sv = OP.periodic_operator_apply(ob, coll, src, ("tsvd", A), g, np.stack([d, d]), (ex, ey), C, Q, p)
    assert np.abs(y_qr - y_sv).max() < 1e-10 * np.abs(y_qr).max()
