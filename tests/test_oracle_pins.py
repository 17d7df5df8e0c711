"""Pins of the oracle against facts fixed outside it (no GPU).

Each test names the passage of the paper (or the textbook result) that fixes
the expected value; none re-types the oracle's own formula.
"""
import math

import numpy as np
import pytest
import scipy.integrate as si
import scipy.special as sps

import oracle as O
import synth


def _small(k=3.0, M=40, N=32, P=16, seed=7, bc=0):
    wl = synth.small_case(seed=seed, k=k, M=M, N=N, P=P, bc=bc)
    ob = wl.obstacles[0]
    coll, src, srcx = O.geometry(ob)
    ob.q = O.choose_q(ob, coll, src, srcx)
    return ob, coll, src, srcx


# --- geometry (Sec. 3, Sec. 3.2 scheme (c)) ---------------------------------

def test_sphere_geometry_closed_form():
    ob = synth.sphere()
    coll, src, _ = O.geometry(ob)
    t = math.pi * (np.arange(ob.M) + 0.5) / ob.M
    assert np.allclose(coll[:, 0], np.sin(t), atol=1e-15)
    assert np.allclose(coll[:, 1], np.cos(t), atol=1e-15)
    assert np.allclose(coll[:, 2:], coll[:, :2], atol=1e-15)    # outward normal = position
    r = np.hypot(src[:, 0], src[:, 1])
    assert np.allclose(r, 0.7, atol=1e-15)                      # shrunk by 0.3 toward the centre


@pytest.mark.parametrize("which", ["smooth", "cup"])
def test_normals_and_proxies(which):
    ob = synth.config_smooth().obstacles[0] if which == "smooth" else synth.cup()
    coll, src, srcx = O.geometry(ob)
    # normals: unit, orthogonal to a finite-difference tangent
    t = math.pi * (np.arange(ob.M) + 0.5) / ob.M
    h = 1e-6
    zp, _ = O.curve(ob, t + h)
    zm, _ = O.curve(ob, t - h)
    tan = (zp - zm) / (2 * h)
    assert np.allclose(np.hypot(coll[:, 2], coll[:, 3]), 1.0, atol=1e-14)
    dot = coll[:, 3] * tan.real + coll[:, 2] * tan.imag
    assert np.abs(dot).max() < 1e-8 * np.abs(tan).max()
    # complexification to first order: y(t + i s tau) ~ zeta + i s tau zeta'
    s = O.orientation(ob)
    tj = math.pi * (np.arange(ob.N) + 0.5) / ob.N
    zeta, dz = O.curve(ob, tj)
    approx = zeta + 1j * s * ob.tau * dz
    y = src[:, 1] + 1j * src[:, 0]
    assert np.abs(y - approx).max() < 3 * ob.tau ** 2 * np.abs(dz).max() ** 2 + 0.05
    # proxies strictly inside: winding test against the closed curve (gamma + axis)
    tt = np.linspace(0, math.pi, 20001)
    zc, _ = O.curve(ob, tt)
    poly = np.concatenate([zc, [zc[0]]])
    for yy, inside in ((src, True), (srcx, False)):
        pts = yy[:, 1] + 1j * yy[:, 0]
        ang = np.angle((poly[1:, None] - pts) / (poly[:-1, None] - pts)).sum(0)
        wind = np.abs(np.round(ang / (2 * math.pi)))
        assert np.all(wind == (1 if inside else 0))


# --- fill (Sec. 3.1, eq. ptr, Theorem 1) -------------------------------------

def test_fill_against_adaptive_quadrature():
    ob, coll, src, _ = _small()
    for deriv in (False, True):
        A = O.fill(ob.k, coll, src, ob.q, ob.P, deriv)
        for (m, j, n) in [(0, 0, 0), (5, 7, 3), (20, 19, 8), (39, 31, 1), (13, 2, 6)]:
            x = coll[m]
            def integrand(phi, part):
                y = np.array([src[j, 0] * math.cos(phi), src[j, 0] * math.sin(phi), src[j, 1]])
                xv = np.array([x[0], 0.0, x[1]])
                d = xv - y
                R = np.linalg.norm(d)
                g = np.exp(1j * ob.k * R) / (4 * math.pi * R)
                if deriv:
                    nd = x[2] * d[0] + x[3] * d[2]
                    g = g * nd * (1j * ob.k * R - 1) / R ** 2
                v = g * np.exp(-1j * n * phi) / (2 * math.pi)
                return v.real if part == 0 else v.imag
            re = si.quad(integrand, 0, 2 * math.pi, args=(0,), epsabs=1e-14, epsrel=1e-13, limit=400)[0]
            im = si.quad(integrand, 0, 2 * math.pi, args=(1,), epsabs=1e-14, epsrel=1e-13, limit=400)[0]
            assert abs(A[n, m, j] - (re + 1j * im)) < 1e-12, (deriv, m, j, n)


def test_fill_laplace_elliptic_closed_form():
    ob, coll, src, _ = _small()
    A0 = O.fill(0.0, coll, src, ob.q, 2, False)[0]
    rho, z = coll[:, 0][:, None], coll[:, 1][:, None]
    rs, zs = src[:, 0][None], src[:, 1][None]
    s2 = (rho + rs) ** 2 + (z - zs) ** 2
    exact = sps.ellipk(4 * rho * rs / s2) / (2 * math.pi ** 2 * np.sqrt(s2))
    assert np.abs(A0 - exact).max() < 1e-13 * np.abs(exact).max()


def test_normal_derivative_finite_difference():
    ob, coll, src, _ = _small()
    h = 1e-5
    cp, cm = coll.copy(), coll.copy()
    cp[:, 0] += h * coll[:, 2]; cp[:, 1] += h * coll[:, 3]
    cm[:, 0] -= h * coll[:, 2]; cm[:, 1] -= h * coll[:, 3]
    g = O.ring_samples(ob.k, coll, src, 16, True)
    fd = (O.ring_samples(ob.k, cp, src, 16, False) - O.ring_samples(ob.k, cm, src, 16, False)) / (2 * h)
    assert np.abs(g - fd).max() < 1e-7 * np.abs(g).max()


def test_theorem1_rate_fig4_pairs():
    # Fig. 4 caption: k = 10, source (0.45, 0.44); targets (0.5, 0.49), (0.6, 0.2)
    src = np.array([[0.45, 0.44]])
    for tgt in ([0.5, 0.49], [0.6, 0.2]):
        coll = np.array([[tgt[0], tgt[1], 1.0, 0.0]])
        alpha = float(O.theorem1_rate(tgt[0], tgt[1], 0.45, 0.44))
        ref = O.fill(10.0, coll, src, 4000, 2, False)[0, 0, 0]
        qs = [q for q in range(20, 2000, 10)]
        err = [abs(O.fill(10.0, coll, src, q, 2, False)[0, 0, 0] - ref) for q in qs]
        err = np.array(err)
        sel = (err > 1e-13) & (err < 1e-4)
        slope = np.polyfit(np.array(qs)[sel], np.log(err[sel]), 1)[0]
        assert abs(-slope - alpha) < 0.15 * alpha, (tgt, slope, alpha)


def test_fill_even_in_mode():
    ob, coll, src, _ = _small()
    g = O.ring_samples(ob.k, coll, src, ob.q, True)
    l = np.arange(ob.q)
    for n in (1, 5, 8):
        neg = (g * np.exp(2j * math.pi * n * l / ob.q)).mean(-1)      # A_{-n}
        pos = O.fill(ob.k, coll, src, ob.q, ob.P, True)[n]
        assert np.abs(neg - pos).max() < 1e-14 * np.abs(pos).max() + 1e-17


def test_q_rule_converged():
    ob, coll, src, _ = _small()
    A1 = O.fill(ob.k, coll, src, ob.q, ob.P, True)
    A2 = O.fill(ob.k, coll, src, O.mfs._smooth_int(int(1.5 * ob.q)), ob.P, True)
    assert np.abs(A1 - A2).max() < 1e-14 * np.abs(A1).max()


# --- least squares (Sec. 3 eq. linsys; Sec. 4.2) -----------------------------

def test_householder_against_lapack():
    rng = np.random.default_rng(0)
    A = rng.standard_normal((30, 20)) + 1j * rng.standard_normal((30, 20))
    QR, tau = O.householder_qr(A)
    R = np.triu(QR[:20])
    Q = O.apply_qh(QR, tau, np.eye(30)).conj().T            # Q = (Q^H)^H
    assert np.abs(Q.conj().T @ Q - np.eye(30)).max() < 1e-14
    assert np.abs(Q[:, :20] @ R - A).max() < 1e-13
    assert np.allclose(np.abs(np.diag(R)), np.abs(np.diag(np.linalg.qr(A)[1])), rtol=1e-13)
    assert np.all(np.abs(np.diag(R).imag) == 0)
    b = rng.standard_normal((30, 3)) + 1j * rng.standard_normal((30, 3))
    x = O.back_substitute(R, O.apply_qh(QR, tau, b)[:20])
    assert np.abs(x - np.linalg.lstsq(A, b, rcond=None)[0]).max() < 1e-12


def test_qr_invariants_on_mfs_block():
    ob, coll, src, _ = _small()
    A = O.fill(ob.k, coll, src, ob.q, ob.P, True)[3]
    QR, tau = O.householder_qr(A)
    Q = O.apply_qh(QR, tau, np.eye(A.shape[0])).conj().T
    R = np.triu(QR[:A.shape[1]])
    assert np.linalg.norm(Q[:, :A.shape[1]] @ R - A) < 1e-14 * np.linalg.norm(A) * A.shape[1]


# --- RHS transform and mode structure (eq. fhatquad) -------------------------

def test_rhs_against_numpy_fft():
    rng = np.random.default_rng(1)
    f = rng.standard_normal((3, 7, 12)) + 1j * rng.standard_normal((3, 7, 12))
    fh = O.rhs_modes(f)
    assert np.abs(fh - np.moveaxis(np.fft.fft(f, axis=-1) / 12, -1, -2)).max() < 1e-14


def test_axial_incidence_single_mode():
    ob, coll, src, srcx = _small()
    A, fac = O.factor_operator(ob, coll, src, srcx)
    fh = O.rhs_modes(O.incident_samples(ob, coll, np.array([[0.0, 0.0, 1.0]])))
    assert np.abs(fh[0, 1:]).max() < 1e-14 * np.abs(fh[0, 0]).max()
    c = O.solve_modes(ob, fac, fh)
    assert np.abs(c[0, 1:]).max() < 1e-10 * np.abs(c[0, 0]).max()


def test_rotation_covariance():
    ob, coll, src, srcx = _small()
    A, fac = O.factor_operator(ob, coll, src, srcx)
    d = synth.plane_wave_directions(1, 11)[0]
    s = 3
    psi = 2 * math.pi * s / ob.P
    Rz = np.array([[math.cos(psi), -math.sin(psi), 0], [math.sin(psi), math.cos(psi), 0], [0, 0, 1]])
    c1 = O.solve_modes(ob, fac, O.rhs_modes(O.incident_samples(ob, coll, d[None])))
    c2 = O.solve_modes(ob, fac, O.rhs_modes(O.incident_samples(ob, coll, (Rz @ d)[None])))
    n = np.arange(ob.P)
    n = np.where(n > ob.P // 2, n - ob.P, n)
    # the Nyquist mode P/2 aliases with -P/2 under the shift; skip it
    keep = np.abs(n) < ob.P // 2
    lhs = c2[0, keep]
    rhs = (c1[0] * np.exp(-1j * n * psi)[:, None])[keep]
    assert np.abs(lhs - rhs).max() < 1e-11 * np.abs(c1).max()


# --- solve + synthesis against closed forms ----------------------------------

def test_sound_hard_sphere_series():
    wl = synth.config_sphere()
    ob = wl.obstacles[0]
    coll, src, srcx = O.geometry(ob)
    A, fac = O.factor_operator(ob, coll, src, srcx)
    d = synth.plane_wave_directions(1, wl.wave_seed)
    c = O.solve_modes(ob, fac, O.rhs_modes(O.incident_samples(ob, coll, d)))
    xh = synth.plane_wave_directions(64, 99)
    F = O.far_field(ob, src, c, xh)[0]
    Fs = O.sphere_series_far_field(ob.k, 1.0, d[0], xh)
    assert np.abs(F - Fs).max() < 1e-12 * np.abs(Fs).max()
    x = np.array([[10.0, 10.0, 10.0], [3.0, -2.0, 1.0], [0.0, 0.0, -4.0]])
    u = O.potential(ob, src, c, x)[0]
    us = O.sphere_series_potential(ob.k, 1.0, d[0], x)
    assert np.abs(u - us).max() < 1e-12 * np.abs(us).max()
    # normal derivative variant: finite difference of the potential
    nv = np.array([[0.6, 0.0, 0.8]] * 3)
    du = O.potential(ob, src, c, x, normals=nv)[0]
    h = 1e-5
    fd = (O.potential(ob, src, c, x + h * nv)[0] - O.potential(ob, src, c, x - h * nv)[0]) / (2 * h)
    assert np.abs(du - fd).max() < 1e-8 * np.abs(du).max()


def test_brute_force_3d_point_source_mfs():
    # q = P: the modal systems are the block DFT of the dense point-source system
    wl = synth.small_case(seed=3, k=2.0, M=15, N=12, P=8)
    ob = wl.obstacles[0]
    ob.q = ob.P
    coll, src, srcx = O.geometry(ob)
    A, fac = O.factor_operator(ob, coll, src, srcx)
    d = synth.plane_wave_directions(1, 5)
    f = O.incident_samples(ob, coll, d)[0]                     # [M][P]
    c = O.solve_modes(ob, fac, O.rhs_modes(f[None]))
    sig = O.point_strengths(c, ob.P)[0]                        # [N][P]
    P = ob.P
    phi = 2 * math.pi * np.arange(P) / P
    X = np.array([[cm[0] * math.cos(p), cm[0] * math.sin(p), cm[1]] for cm in coll for p in phi])
    Nn = np.array([[cm[2] * math.cos(p), cm[2] * math.sin(p), cm[3]] for cm in coll for p in phi])
    Y = np.array([[s[0] * math.cos(p), s[0] * math.sin(p), s[1]] for s in src for p in phi])
    Dv = X[:, None, :] - Y[None]
    R = np.linalg.norm(Dv, axis=-1)
    nd = np.einsum("tc,tsc->ts", Nn, Dv)
    Kd = nd * (1j * ob.k * R - 1) * np.exp(1j * ob.k * R) / (4 * math.pi * R ** 3)
    s_bf = np.linalg.lstsq(Kd, f.reshape(-1), rcond=None)[0].reshape(ob.N, P)
    assert np.abs(sig - s_bf).max() < 1e-9 * np.abs(s_bf).max()


def test_reciprocity():
    wl = synth.small_case(seed=9, k=3.0, M=144, N=120, P=48)
    ob = wl.obstacles[0]
    coll, src, srcx = O.geometry(ob)
    ob.q = O.choose_q(ob, coll, src)
    A, fac = O.factor_operator(ob, coll, src, srcx)
    d = synth.plane_wave_directions(2, 21)
    d[1] = -d[1]
    xh = np.array([[0.3, -0.4, math.sqrt(1 - 0.25)], [-0.6, 0.0, 0.8]])
    c = O.solve_modes(ob, fac, O.rhs_modes(O.incident_samples(ob, coll, d)))
    F_ab = O.far_field(ob, src, c[:1], xh[:1])[0, 0]             # F(xh0; d0)
    c2 = O.solve_modes(ob, fac, O.rhs_modes(O.incident_samples(ob, coll, -xh[:1])))
    F_ba = O.far_field(ob, src, c2, -d[:1])[0, 0]                 # F(-d0; -xh0)
    assert abs(F_ab - F_ba) < 1e-9 * abs(F_ab)


def test_transmission_null_case():
    # k_minus = k: the transmission problem has u = 0 outside (Sec. 3.4)
    wl = synth.small_case(seed=5, k=2.5, M=120, N=100, P=32, bc=synth.BC_TRANSMISSION)
    ob = wl.obstacles[0]
    ob.k_minus = ob.k
    coll, src, srcx = O.geometry(ob)
    ob.q = O.choose_q(ob, coll, src, srcx)
    A, fac = O.factor_operator(ob, coll, src, srcx)
    d = synth.plane_wave_directions(2, 8)
    c = O.solve_modes(ob, fac, O.rhs_modes(O.incident_samples(ob, coll, d)))
    xh = synth.plane_wave_directions(16, 4)
    F = O.far_field(ob, src, c, xh)
    assert np.abs(F).max() < 1e-8
    # the interior field reproduces u_i inside
    xin = np.array([[0.1, 0.2, -0.1], [0.0, 0.3, 0.2]])
    um = O.potential(ob, srcx, c[:, :, ob.N:], xin, k=ob.k_minus)
    ui = np.exp(1j * ob.k * (xin @ d.T)).T
    assert np.abs(um - ui).max() < 1e-8


def test_near_image_sum_translation():
    ob, coll, src, srcx = _small(k=2.0, M=20, N=16, P=8)
    A, fac = O.factor_operator(ob, coll, src, srcx)
    d = synth.plane_wave_directions(2, 13)
    c = O.solve_modes(ob, fac, O.rhs_modes(O.incident_samples(ob, coll, d)))
    lat = (3.1, 2.7)
    idx = np.array([0, 7, 33, 100, 159])
    U = O.near_image_sum(ob, coll, src, c, d, lat, target_idx=idx)
    phi = 2 * math.pi * np.arange(ob.P) / ob.P
    X = np.array([[cm[0] * math.cos(p), cm[0] * math.sin(p), cm[1]] for cm in coll for p in phi])[idx]
    Nn = np.array([[cm[2] * math.cos(p), cm[2] * math.sin(p), cm[3]] for cm in coll for p in phi])[idx]
    ref = np.zeros_like(U)
    for a in (-1, 0, 1):
        for b in (-1, 0, 1):
            if a == b == 0:
                continue
            shift = np.array([a * lat[0], b * lat[1], 0.0])
            ph = np.exp(1j * ob.k * (d[:, 0] * a * lat[0] + d[:, 1] * b * lat[1]))
            ref += ph[:, None] * O.potential(ob, src, c, X - shift, normals=Nn)
    assert np.abs(U - ref).max() < 1e-13 * np.abs(ref).max()


# --- cup generating curve (Fig. 2(c) caption; Sec. 3 smoothness on the axis) --

def test_cup_curve_facts():
    """Facts the cup's description fixes, independent of how the curve is coded:
    both ends lie on the axis (rho = 0) with z' = 0 there to rounding (Sec. 3
    says the cup meets this to double precision because erf saturates); away
    from the rim the outer arc has radius 1 + a = 1.2 and the inner arc
    1 - a = 0.8 (half-thickness a); the rim, the extreme polar angle of the
    curve, sits within a of the opening half-angle b; outward normals point
    away from the shell material (radially out on the outer arc, towards the
    centre on the inner arc)."""
    for b in (math.pi / 2, math.pi / 6):
        ob = synth.cup(b=b)
        a = ob.params[0]
        zeta, dz = O.curve(ob, np.array([0.0, math.pi]))
        assert np.abs(zeta.imag).max() < 1e-15                      # rho = 0 at both ends
        assert np.abs(dz.real).max() < 1e-15                        # z'(0) = z'(pi) = 0
        assert np.abs(np.abs(zeta) - np.array([1 + a, 1 - a])).max() < 1e-15
        assert np.all(zeta.real < 0)                                # closed end at -z (opening at +z)
        t = np.linspace(0.0, math.pi, 20001)
        zt, _ = O.curve(ob, t)
        far = np.abs(t - math.pi / 2) >= 5 * a
        outer, inner = far & (t < math.pi / 2), far & (t > math.pi / 2)
        assert np.abs(np.abs(zt[outer]) - (1 + a)).max() < 1e-12
        assert np.abs(np.abs(zt[inner]) - (1 - a)).max() < 1e-12
        assert zt.imag[1:-1].min() > 0                              # rho > 0 between the ends
        theta = np.arctan2(np.abs(zt.imag), zt.real)                # polar angle from +z
        assert abs(theta.min() - b) < a
        # collocation normals: radial on the outer arc, anti-radial on the inner
        ob_c = synth.cup(b=b, M=200, N=160)
        coll, _, _ = O.geometry(ob_c)
        tm = math.pi * (np.arange(ob_c.M) + 0.5) / ob_c.M
        rad = coll[:, :2] / np.hypot(coll[:, 0], coll[:, 1])[:, None]
        fo = (tm < math.pi / 2 - 6 * a)
        fi = (tm > math.pi / 2 + 6 * a)
        assert np.abs(coll[fo, 2:] - rad[fo]).max() < 1e-12
        assert np.abs(coll[fi, 2:] + rad[fi]).max() < 1e-12


# --- Bloch phases of the near images (eqs. per, bloch; A_else in Sec. 4.1) ----

@pytest.mark.parametrize("specular", [False, True])
def test_near_image_phases_zeroth_bragg_order(specular):
    """Quasi-periodicity (eq. per) makes the copy of the obstacle at lattice
    offset (a e_x, b e_y) radiate with the Bloch factor alpha^a beta^b of the
    incident wave, and such an array radiates coherently in its zeroth Bragg
    orders: the directions whose components along the lattice plane equal the
    incident direction's (straight through, and the specular reflection). So at
    a very distant target in such a direction, the eight-image sum of the
    target-normal derivative equals 8 times the central copy's own
    contribution, (i k e^{ikR}/R) F_0(xhat) with F_0 the far field. A wrong
    sign of either phase exponent, or alpha and beta exchanged, breaks it."""
    ob, coll, src, srcx = _small(k=2.0, M=20, N=16, P=12)
    A, fac = O.factor_operator(ob, coll, src, srcx)
    # incident direction with azimuth on a ring node (phi_1 = 2 pi / P, 30
    # degrees: d_x != d_y, so exchanging alpha and beta shows) so the far
    # target can sit at node l = 1 of a one-row "collocation" array
    th, phi = 0.7, 2 * math.pi / ob.P
    d = np.array([[math.sin(th) * math.cos(phi), math.sin(th) * math.sin(phi), math.cos(th)]])
    c = O.solve_modes(ob, fac, O.rhs_modes(O.incident_samples(ob, coll, d)))
    xz = -math.cos(th) if specular else math.cos(th)
    xhat = np.array([math.sin(th) * math.cos(phi), math.sin(th) * math.sin(phi), xz])
    R = 1e8
    far = np.array([[R * math.sin(th), R * xz, math.sin(th), xz]])  # rho, z, n_rho, n_z
    lat = (3.1, 2.7)
    U = O.near_image_sum(ob, far, src, c, d, lat, target_idx=np.array([1]))[0, 0]
    F0 = O.far_field(ob, src, c, xhat[None])[0, 0]
    ratio = U / (1j * ob.k * np.exp(1j * ob.k * R) / R * F0)
    assert abs(ratio - 8.0) < 1e-4, ratio


# --- truncated-SVD pseudo-inverse (Sec. 4.2) ---------------------------------

def _unitary(rng, n):
    Z = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    Q, R = np.linalg.qr(Z)
    return Q * (np.diag(R) / np.abs(np.diag(R)))


def test_tsvd_solve_on_known_factors():
    """A = U diag(s) V^H built from known unitary factors, with singular values
    far on either side of the 1e-10 relative cutoff: the solution must be
    V_k diag(1/s_k) U_k^H F over exactly the kept ones (computed from the
    constructed factors, not from an SVD)."""
    rng = np.random.default_rng(5)
    M, N = 40, 24
    U = _unitary(rng, M)[:, :N]
    V = _unitary(rng, N)
    s = np.logspace(0, -16, N)
    s[(s > 1e-12) & (s < 1e-8)] = 1e-7             # nothing near the cutoff
    s = 1e3 * np.sort(s)[::-1]                      # relative cutoff: 1e-7 here, not 1e-10
    A = (U * s) @ V.conj().T
    F = rng.standard_normal((M, 3)) + 1j * rng.standard_normal((M, 3))
    k = s >= 1e-10 * s[0]
    assert 0 < k.sum() < N
    x_ref = V[:, k] @ ((U[:, k].conj().T @ F) / s[k][:, None])
    x = O.tsvd_solve(A, F)
    assert np.abs(x - x_ref).max() < 1e-6 * np.abs(x_ref).max()
    # the kept part of the residual vanishes: U_k^H (A x - F) = 0
    assert np.abs(U[:, k].conj().T @ (A @ x - F)).max() < 1e-13 * np.abs(x).max()


def test_tsvd_equals_qr_when_well_conditioned():
    rng = np.random.default_rng(6)
    A = rng.standard_normal((50, 30)) + 1j * rng.standard_normal((50, 30))
    F = rng.standard_normal((50, 2)) + 1j * rng.standard_normal((50, 2))
    QR, tau = O.householder_qr(A)
    x_qr = O.back_substitute(np.triu(QR[:30]), O.apply_qh(QR, tau, F)[:30])
    assert np.abs(O.tsvd_solve(A, F) - x_qr).max() < 1e-12 * np.abs(x_qr).max()
