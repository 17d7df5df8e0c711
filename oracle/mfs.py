"""Oracle: the one-obstacle axisymmetric MFS solution operator, plain FP64.

TEST INFRASTRUCTURE ONLY (see the package docstring): imported by `tests/`,
`__graft_entry__.smoke()` and `bench.py`'s CPU-baseline leg, never by the
product path.

Notation follows the paper (Liu & Barnett, arXiv:1506.05083):
  gamma         generating curve (rho(t), z(t)), t in [0, pi]        (Sec. 3)
  M, N          collocation points / proxy rings on the curve        (Sec. 3, eq. linsys)
  P             azimuthal modes n in (-P/2, P/2]                     (Sec. 3)
  q             trapezoid nodes of the ring-kernel quadrature        (Sec. 3.1, eq. ptr)
  A_n, A'_n     value / target-normal-derivative ring-kernel matrices
  c_n           coefficients of mode n, eta = [c_{-P/2+1}; ...; c_{P/2}]

Readings where the paper is silent or garbled (shared with the CUDA path,
which implements them independently):
  * u(rho, phi, z) = sum_n e^{+i n phi} sum_j A_n(rho, z; j) c_nj and
    A_n c_n = fhat_n; since the ring kernel depends on cos(phi) only,
    A_n = A_{-n} and modes +-n share one factorisation.
  * (1/2pi) int d(phi) normalisation everywhere, i.e. the 1/q quadrature.
  * collocation t_m = pi (m - 1/2) / M, proxies t_j = pi (j - 1/2) / N.
  * proxies by complexification of zeta(t) = z(t) + i rho(t):
    y_j = zeta(t_j + i s tau), s = +1 if gamma runs counter-clockwise in the
    (z, rho) plane (interior on the left), else -1; exterior proxies use -tau.
  * unpivoted Householder QR (LAPACK reflector convention), no column
    scaling, no rank truncation; R is never inverted explicitly.
  * time convention e^{-i omega t}: G = e^{ikR}/(4 pi R), far field
    u ~ e^{ikr}/r F(xhat).

Pins (tests/test_oracle_pins.py) for each function:
  curve/geometry      closed-form sphere points, finite-difference normals,
                      proxies inside the body, Taylor check of complexification;
                      cup: both ends on the axis with z' = 0, arc radii 1 +- a,
                      rim within a of the opening angle b, normals away from
                      the shell (Fig. 2(c) caption, Sec. 3)
  ring_samples        finite-difference normal derivative of G
  fill                adaptive quadrature (scipy.integrate.quad) of the ring
                      integral; Laplace k=0, n=0 elliptic-K closed form;
                      Theorem 1 convergence rate; evenness A_n = A_{-n}
  householder_qr,     Q^H Q = I, QR = A, |R_jj| against LAPACK, LS solution
  apply_qh, back_substitute   against numpy lstsq
  rhs_modes           numpy FFT; axial incidence gives mode 0 only
  solve + synthesis   sound-hard sphere series (far field and potential);
                      brute-force 3D point-source MFS with q = P;
                      rotation covariance; reciprocity
  transmission        k_minus = k null case (u = 0 outside)
  tsvd_solve          matrices of known singular values (cutoff applied to the
                      constructed factors); equals the QR solution when the
                      matrix is well conditioned
  near_image_sum      direct 3D summation over explicit image points; the
                      Bloch phases by the coherent zeroth Bragg order of the
                      eight images at a distant target (eq. per)
"""
from __future__ import annotations

import math
from typing import Dict, Tuple

import numpy as np
import scipy.special as sps

__all__ = [
    "curve", "orientation", "geometry", "theorem1_rate", "choose_q",
    "ring_samples", "fill", "system_matrix", "householder_qr", "apply_qh",
    "back_substitute", "factor_operator", "incident_samples", "rhs_modes",
    "solve_modes", "point_strengths", "far_field", "potential",
    "near_image_sum", "sphere_series_far_field", "sphere_series_potential",
    "n_rows", "n_cols", "tsvd_solve", "solve_modes_tsvd", "TSVD_CUTOFF",
]

FOUR_PI = 4.0 * math.pi


# ----------------------------------------------------------------------------
# A1: geometry (Sec. 3, Sec. 3.2 scheme (c), Sec. 3.4 exterior proxies)
# ----------------------------------------------------------------------------

def curve(ob, t):
    """zeta(t) = z(t) + i rho(t) and its t-derivative, for real or complex t.

    Polar shapes (Fig. 2 (a),(b) and the seeded bodies): r(t) = r0 + sum_j
    amp_j cos(j t), zeta = r(t) e^{i t}.  Cup (Fig. 2 (c)): r(t) = 1 - a
    erf((t - pi/2)/a), theta(t) = b - a + 2 (1 - (b - a)/pi) s_a(t - pi/2),
    s_a(x) = (a/sqrt(pi)) e^{-x^2/a^2} + x erf(x/a) (the caption's formula is
    garbled; this is the rounded |x| it describes), zeta = r e^{i theta}.
    """
    t = np.asarray(t)
    if ob.shape == 0:
        r0, amps = ob.params[0], ob.params[1:]
        r = r0 + sum(a * np.cos((j + 1) * t) for j, a in enumerate(amps))
        dr = -sum(a * (j + 1) * np.sin((j + 1) * t) for j, a in enumerate(amps))
        e = np.exp(1j * t)
        return r * e, (dr + 1j * r) * e
    a, b = ob.params[0], ob.params[1]
    x = t - math.pi / 2
    er = sps.erf(x / a)
    r = 1.0 - a * er
    dr = -(2.0 / math.sqrt(math.pi)) * np.exp(-(x / a) ** 2)
    c = 2.0 * (1.0 - (b - a) / math.pi)
    sa = (a / math.sqrt(math.pi)) * np.exp(-(x / a) ** 2) + x * er
    th = b - a + c * sa
    dth = c * er
    e = np.exp(1j * th)
    return r * e, (dr + 1j * r * dth) * e


def orientation(ob, n=4096):
    """+1 if gamma runs counter-clockwise in the (z, rho) plane, else -1.

    Signed area of the closed polygon gamma + axis segment (shoelace).
    """
    t = np.linspace(0.0, math.pi, n)
    zeta, _ = curve(ob, t)
    z, rho = zeta.real, zeta.imag
    area = 0.5 * np.sum(z[:-1] * rho[1:] - z[1:] * rho[:-1])
    area += 0.5 * (z[-1] * rho[0] - z[0] * rho[-1])
    return 1.0 if area > 0 else -1.0


def geometry(ob):
    """Collocation points with outward normals, interior and exterior proxies.

    Returns coll [M][4] = (rho, z, n_rho, n_z), src [N][2] = (rho', z'),
    src_ext [N][2] (exterior proxies, -tau, Sec. 3.4).
    """
    s = orientation(ob)
    tm = math.pi * (np.arange(1, ob.M + 1) - 0.5) / ob.M
    tj = math.pi * (np.arange(1, ob.N + 1) - 0.5) / ob.N
    zeta, dzeta = curve(ob, tm)
    nrm = s * (-1j * dzeta) / np.abs(dzeta)
    coll = np.stack([zeta.imag, zeta.real, nrm.imag, nrm.real], axis=1)
    yi, _ = curve(ob, tj + 1j * s * ob.tau)
    ye, _ = curve(ob, tj - 1j * s * ob.tau)
    src = np.stack([yi.imag, yi.real], axis=1)
    src_ext = np.stack([ye.imag, ye.real], axis=1)
    return coll, src, src_ext


def theorem1_rate(rho, z, rho_s, z_s):
    """Theorem 1: PTR rate alpha = Im acos(1 + d^2/(2 rho rho'))."""
    d2 = (rho - rho_s) ** 2 + (z - z_s) ** 2
    return np.arccosh(1.0 + d2 / (2.0 * rho * rho_s))


def _smooth_int(lo):
    n = max(2, int(math.ceil(lo)))
    while True:
        m = n
        for p in (2, 3, 5):
            while m % p == 0:
                m //= p
        if m == 1 and n % 2 == 0:
            return n
        n += 1


def choose_q(ob, coll, src, src_ext=None):
    """Quadrature count from Theorem 1 (Sec. 3.1): e^{-alpha_min q} ~ 1e-16.

    Reading of the paper's convergence test: q = smallest even 2^a 3^b 5^c
    >= max(2P, 37/alpha_min + P/2), the P/2 covering the "+|n| extra nodes"
    remark after Theorem 1.
    """
    al = theorem1_rate(coll[:, 0:1], coll[:, 1:2], src[None, :, 0], src[None, :, 1]).min()
    if src_ext is not None and ob.bc == 1:
        al = min(al, theorem1_rate(coll[:, 0:1], coll[:, 1:2],
                                   src_ext[None, :, 0], src_ext[None, :, 1]).min())
    return _smooth_int(max(2 * ob.P, 37.0 / al + ob.P / 2))


# ----------------------------------------------------------------------------
# A2: ring-kernel fill (Sec. 3.1, eqs. ringkernel, ringkernelderiv, ptr)
# ----------------------------------------------------------------------------

def ring_samples(k, coll, src, q, deriv):
    """Samples of G_k or dG_k/dn_x between target x_m = (rho_m, 0, z_m) and
    the rotated source y_j(phi_l) = (rho'_j cos phi_l, rho'_j sin phi_l, z'_j),
    phi_l = 2 pi l / q, l = 0..q-1.  Returns [M][N][q] complex.

    G = e^{ikR}/(4 pi R) (eq. G); dG/dn_x = (n . (x - y)) (ikR - 1) e^{ikR}/(4 pi R^3).
    """
    phi = 2.0 * math.pi * np.arange(q) / q
    rho = coll[:, 0][:, None, None]
    z = coll[:, 1][:, None, None]
    rs = src[:, 0][None, :, None]
    zs = src[:, 1][None, :, None]
    dx = rho - rs * np.cos(phi)
    dy = -rs * np.sin(phi)
    dz = z - zs
    R = np.sqrt(dx * dx + dy * dy + dz * dz)
    e = np.exp(1j * k * R)
    if not deriv:
        return e / (FOUR_PI * R)
    ndot = coll[:, 2][:, None, None] * dx + coll[:, 3][:, None, None] * dz
    return ndot * (1j * k * R - 1.0) * e / (FOUR_PI * R ** 3)


def fill(k, coll, src, q, P, deriv, chunk=16):
    """Distinct modal matrices A_n (or A'_n), n = 0..P/2, by the q-node PTR
    (eq. ptr): A_n(m, j) = (1/q) sum_l g_l e^{-2 pi i n l / q}.  Direct
    summation over all q nodes.  Returns [P/2+1][M][N] complex.
    """
    D = P // 2 + 1
    M, N = coll.shape[0], src.shape[0]
    l = np.arange(q)
    E = np.exp(-2j * math.pi * np.outer(l, np.arange(D)) / q) / q     # [q][D]
    out = np.empty((D, M, N), dtype=np.complex128)
    for m0 in range(0, M, chunk):
        g = ring_samples(k, coll[m0:m0 + chunk], src, q, deriv)      # [c][N][q]
        out[:, m0:m0 + chunk, :] = np.moveaxis(g @ E, 2, 0)
    return out


def n_rows(ob):
    return ob.M * (2 if ob.bc == 1 else 1)


def n_cols(ob):
    return ob.N * (2 if ob.bc == 1 else 1)


def system_matrix(ob, coll, src, src_ext):
    """A_0's distinct diagonal blocks, [P/2+1][rows][cols] (eqs. linsysb, trans).

    Neumann: A'_n.  Transmission: [[A_n, -A^-_n], [A'_n, -A'^-_n]] with the
    interior wavenumber k_minus and the exterior proxies for the minus blocks.
    """
    if ob.bc == 0:
        return fill(ob.k, coll, src, ob.q, ob.P, True)
    A = fill(ob.k, coll, src, ob.q, ob.P, False)
    Ad = fill(ob.k, coll, src, ob.q, ob.P, True)
    Am = fill(ob.k_minus, coll, src_ext, ob.q, ob.P, False)
    Amd = fill(ob.k_minus, coll, src_ext, ob.q, ob.P, True)
    top = np.concatenate([A, -Am], axis=2)
    bot = np.concatenate([Ad, -Amd], axis=2)
    return np.concatenate([top, bot], axis=1)


# ----------------------------------------------------------------------------
# A3: dense backward-stable least squares per mode (Sec. 3, eq. linsys)
# ----------------------------------------------------------------------------

def householder_qr(A):
    """Unblocked complex Householder QR, A = Q R, Q = H_1 H_2 ... H_N.

    H_j = I - tau_j v_j v_j^H with v_j[0] = 1; H_j^H maps the column
    (alpha; x) to (beta; 0), beta = -sign(Re alpha) ||(alpha; x)|| real,
    tau = (beta - alpha)/beta, v = x/(alpha - beta).  Returns the packed
    array (R on and above the diagonal, v below it) and tau.
    """
    A = np.array(A, dtype=np.complex128, copy=True)
    M, N = A.shape
    tau = np.zeros(N, dtype=np.complex128)
    for j in range(N):
        alpha = A[j, j]
        x = A[j + 1:, j]
        xn = np.linalg.norm(x)
        if xn == 0.0 and alpha.imag == 0.0:
            continue
        nrm = math.hypot(abs(alpha), xn)
        beta = -math.copysign(nrm, alpha.real)
        tau[j] = (beta - alpha) / beta
        v = x / (alpha - beta)
        A[j + 1:, j] = v
        A[j, j] = beta
        if j + 1 < N:
            w = A[j, j + 1:] + v.conj() @ A[j + 1:, j + 1:]
            w *= np.conj(tau[j])
            A[j, j + 1:] -= w
            A[j + 1:, j + 1:] -= np.outer(v, w)
    return A, tau


def apply_qh(QR, tau, B):
    """Q^H B = H_N^H ... H_1^H B for B [M][r]."""
    B = np.array(B, dtype=np.complex128, copy=True)
    M, N = QR.shape
    for j in range(N):
        v = QR[j + 1:, j]
        w = B[j] + v.conj() @ B[j + 1:]
        w *= np.conj(tau[j])
        B[j] -= w
        B[j + 1:] -= np.outer(v, w)
    return B


def back_substitute(R, Y):
    """Solve R X = Y for upper-triangular R [N][N], Y [N][r], row by row."""
    N = R.shape[0]
    X = np.zeros_like(Y, dtype=np.complex128)
    for i in range(N - 1, -1, -1):
        X[i] = (Y[i] - R[i, i + 1:] @ X[i + 1:]) / R[i, i]
    return X


def factor_operator(ob, coll, src, src_ext):
    """Fill and factor every distinct mode: list of (packed QR, tau)."""
    A = system_matrix(ob, coll, src, src_ext)
    return A, [householder_qr(A[d]) for d in range(A.shape[0])]


# ----------------------------------------------------------------------------
# A4-A6: apply (Sec. 3 eq. fhatquad; Sec. 4.2 application of A_n^+; Sec. 4.1)
# ----------------------------------------------------------------------------

def incident_samples(ob, coll, dirs):
    """Boundary data on the M x P ring nodes (rho_m, phi_l = 2 pi l/P, z_m).

    Neumann (eq. neu): f = -du_i/dn, u_i = e^{ik d.x} (eq. ui).
    Transmission (eq. trans): rows [f; f'] = [-u_i; -du_i/dn].
    Returns [W][rows][P] complex.
    """
    P = ob.P
    phi = 2.0 * math.pi * np.arange(P) / P
    rho, z, nr, nz = (coll[:, i][:, None] for i in range(4))
    X = np.stack([rho * np.cos(phi), rho * np.sin(phi), np.broadcast_to(z, (coll.shape[0], P))], -1)
    Nv = np.stack([nr * np.cos(phi), nr * np.sin(phi), np.broadcast_to(nz, (coll.shape[0], P))], -1)
    out = []
    for d in np.atleast_2d(dirs):
        ui = np.exp(1j * ob.k * (X @ d))
        dui = 1j * ob.k * (Nv @ d) * ui
        out.append(-dui if ob.bc == 0 else np.concatenate([-ui, -dui], axis=0))
    return np.array(out)


def rhs_modes(f):
    """fhat_n = (1/P) sum_l f_l e^{-2 pi i n l / P} (eq. fhatquad with q = P),
    by direct summation; mode n stored at index n mod P.  f: [W][rows][P] ->
    [W][P][rows].
    """
    P = f.shape[-1]
    l = np.arange(P)
    n = np.arange(P)
    n = np.where(n > P // 2, n - P, n)
    E = np.exp(-2j * math.pi * np.outer(l, n) / P) / P
    return np.moveaxis(f @ E, -1, -2)


def solve_modes(ob, factors, fhat):
    """c_n = R^{-1} (Q^H fhat_n)_{1:cols} for every mode n (Sec. 4.2: apply the
    factors, never an explicit inverse); modes +-n use the factors of |n|.
    fhat [W][P][rows] -> coef [W][P][cols].
    """
    W, P, rows = fhat.shape
    cols = n_cols(ob)
    coef = np.zeros((W, P, cols), dtype=np.complex128)
    for idx in range(P):
        n = idx if idx <= P // 2 else idx - P
        QR, tau = factors[abs(n)]
        Y = apply_qh(QR, tau, fhat[:, idx, :].T)[:cols]
        coef[:, idx, :] = back_substitute(np.triu(QR[:cols, :cols]), Y).T
    return coef


TSVD_CUTOFF = 1e-10


def tsvd_solve(A, F, cutoff=TSVD_CUTOFF):
    """Truncated-SVD least squares (Sec. 4.2, application of A_n^+): with
    A = U diag(s) V^H, x = V diag(1/s_k) U^H F over the singular values
    s_k >= cutoff * s_max, applied as two products and a scaling, never as an
    explicit pseudo-inverse. F [M][r] -> x [N][r]."""
    U, sv, Vh = np.linalg.svd(A, full_matrices=False)
    keep = sv >= cutoff * sv[0]
    y = (U[:, keep].conj().T @ F) / sv[keep][:, None]
    return Vh[keep].conj().T @ y


def solve_modes_tsvd(ob, A, fhat, cutoff=TSVD_CUTOFF):
    """Truncated-SVD variant of solve_modes: c_n = A_n^+ fhat_n with the
    1e-10 relative cutoff of Sec. 4.2; modes +-n use the matrix of |n|.
    A [P/2+1][rows][cols], fhat [W][P][rows] -> coef [W][P][cols]."""
    W, P, rows = fhat.shape
    coef = np.zeros((W, P, A.shape[2]), dtype=np.complex128)
    for idx in range(P):
        n = idx if idx <= P // 2 else P - idx
        coef[:, idx, :] = tsvd_solve(A[n], fhat[:, idx, :].T, cutoff).T
    return coef


def point_strengths(coef, qe):
    """Ring -> point sources (Sec. 4.1): sigma_{j,l} = (1/qe) sum_n c_nj
    e^{i n phi_l}, phi_l = 2 pi l / qe.  coef [W][P][N] -> [W][N][qe].
    """
    W, P, N = coef.shape
    n = np.arange(P)
    n = np.where(n > P // 2, n - P, n)
    l = np.arange(qe)
    E = np.exp(2j * math.pi * np.outer(n, l) / qe) / qe                # [P][qe]
    return np.einsum("wpn,pl->wnl", coef, E)


def _source_points(src, qe):
    phi = 2.0 * math.pi * np.arange(qe) / qe
    x = src[:, 0][:, None] * np.cos(phi)
    y = src[:, 0][:, None] * np.sin(phi)
    z = np.broadcast_to(src[:, 1][:, None], x.shape)
    return np.stack([x, y, z], -1)                                      # [N][qe][3]


def far_field(ob, src, coef, xhat, qe=None):
    """F(xhat) = (1/4 pi) sum_{j,l} sigma_jl e^{-ik xhat . y_jl} of the
    exterior field (u ~ e^{ikr}/r F).  coef [W][P][cols] -> [W][T].
    """
    qe = qe or ob.P
    sig = point_strengths(coef[:, :, :ob.N], qe)                       # [W][N][qe]
    Y = _source_points(src, qe).reshape(-1, 3)
    K = np.exp(-1j * ob.k * (np.asarray(xhat) @ Y.T)) / FOUR_PI        # [T][N*qe]
    return sig.reshape(sig.shape[0], -1) @ K.T


def potential(ob, src, coef, targets, qe=None, k=None, normals=None):
    """u(x) = sum_{j,l} G_k(x, y_jl) sigma_jl at 3D targets (or dG/dn_x when
    normals are given).  coef [W][P][N] (one block of columns)."""
    qe = qe or ob.P
    k = ob.k if k is None else k
    sig = point_strengths(coef, qe)
    Y = _source_points(src, qe).reshape(-1, 3)
    T = np.asarray(targets)
    D = T[:, None, :] - Y[None, :, :]
    R = np.linalg.norm(D, axis=-1)
    e = np.exp(1j * k * R)
    if normals is None:
        K = e / (FOUR_PI * R)
    else:
        nd = np.einsum("tc,tsc->ts", np.asarray(normals), D)
        K = nd * (1j * k * R - 1.0) * e / (FOUR_PI * R ** 3)
    return sig.reshape(sig.shape[0], -1) @ K.T


def near_image_sum(ob, coll, src, coef, dirs, lattice, target_idx=None):
    """A7 (Sec. 4.1, action of A_else): normal derivative at the ring nodes
    x_{m,l} (rho_m, phi_l = 2 pi l / P, z_m) of the eight phased images of the
    point sources (q = P), omitting the central copy:
      U_w(x_t) = sum_{(a,b) != (0,0)} alpha_w^a beta_w^b
                 sum_s dG/dn_t(x_t, y_s + a e_x + b e_y) sigma_{w,s},
    alpha_w = e^{i k d_x e_x}, beta_w = e^{i k d_y e_y} (eq. bloch with its
    e_y typo read as e_y).  Returns [W][M*P] in target order t = m*P + l, or
    only the targets listed in target_idx.
    """
    P = ob.P
    ex, ey = lattice
    sig = point_strengths(coef[:, :, :ob.N], P).reshape(coef.shape[0], -1)    # [W][N*P]
    Y = _source_points(src, P).reshape(-1, 3)
    phi = 2.0 * math.pi * np.arange(P) / P
    rho, z, nr, nz = (coll[:, i][:, None] for i in range(4))
    X = np.stack([rho * np.cos(phi), rho * np.sin(phi),
                  np.broadcast_to(z, (coll.shape[0], P))], -1).reshape(-1, 3)
    Nv = np.stack([nr * np.cos(phi), nr * np.sin(phi),
                   np.broadcast_to(nz, (coll.shape[0], P))], -1).reshape(-1, 3)
    if target_idx is not None:
        X, Nv = X[target_idx], Nv[target_idx]
    dirs = np.atleast_2d(dirs)
    out = np.zeros((dirs.shape[0], X.shape[0]), dtype=np.complex128)
    for a in (-1, 0, 1):
        for b in (-1, 0, 1):
            if a == 0 and b == 0:
                continue
            shift = np.array([a * ex, b * ey, 0.0])
            Dv = X[:, None, :] - (Y[None, :, :] + shift)
            R = np.linalg.norm(Dv, axis=-1)
            nd = np.einsum("tc,tsc->ts", Nv, Dv)
            K = nd * (1j * ob.k * R - 1.0) * np.exp(1j * ob.k * R) / (FOUR_PI * R ** 3)
            ph = np.exp(1j * ob.k * (dirs[:, 0] * a * ex + dirs[:, 1] * b * ey))
            out += ph[:, None] * (sig @ K.T)
    return out


# ----------------------------------------------------------------------------
# External pins: sound-hard sphere series (Colton-Kress separation of variables)
# ----------------------------------------------------------------------------

def _sphere_ratio(k, a, L):
    l = np.arange(L + 1)
    jp = sps.spherical_jn(l, k * a, derivative=True)
    hp = jp + 1j * sps.spherical_yn(l, k * a, derivative=True)
    return l, jp / hp


def sphere_series_far_field(k, a, d, xhat, L=None):
    """Sound-hard sphere: F(xhat) = (i/k) sum_l (2l+1) [j_l'(ka)/h_l'(ka)] P_l(xhat.d)."""
    L = L or int(k * a + 40)
    l, ratio = _sphere_ratio(k, a, L)
    c = np.asarray(xhat) @ np.asarray(d)
    Pl = np.array([sps.eval_legendre(ll, c) for ll in l])
    return (1j / k) * np.sum(((2 * l + 1) * ratio)[:, None] * Pl, axis=0)


def sphere_series_potential(k, a, d, x, L=None):
    """u^s(x) = -sum_l i^l (2l+1) [j_l'(ka)/h_l'(ka)] h_l(k|x|) P_l(xhat.d)."""
    L = L or int(k * a + 40)
    l, ratio = _sphere_ratio(k, a, L)
    x = np.asarray(x)
    r = np.linalg.norm(x, axis=-1)
    c = (x @ np.asarray(d)) / r
    out = np.zeros(x.shape[0], dtype=np.complex128)
    for ll in l:
        h = sps.spherical_jn(ll, k * r) + 1j * sps.spherical_yn(ll, k * r)
        out -= (1j ** ll) * (2 * ll + 1) * ratio[ll] * h * sps.eval_legendre(ll, c)
    return out
