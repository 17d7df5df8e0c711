"""Oracle: the auxiliary spherical-harmonic block B~ of the periodizing
scheme (Sec. 4, eq. urep; Sec. 4.1, the B~ display), plain FP64.

TEST INFRASTRUCTURE ONLY (see the package docstring): imported by `tests/`
and never by the product path.

The periodic field in the unit cell carries, besides the ring sources, the
regular spherical waves u_lm(x) = j_l(k r) Y_lm(theta, phi), l <= p, |m| <= l
(eq. urep). B~ maps their coefficients d_lm to the modal boundary data the
obstacle's rows hold (Sec. 4.1):

  B~_{n i, lm} = (1/2pi) int_0^{2pi} F_i[u_lm](phi) e^{-i n phi} dphi
              ~= (1/q) sum_{s=0}^{q-1} F_i[u_lm](2 pi s/q) e^{-2 pi i n s/q},

F_i the boundary functional of collocation ring i: the normal derivative for
the Neumann problem (eq. neu), the value and the normal derivative (rows
[value; normal derivative]) for the transmission problem (eq. trans), as in
A's rows (`system_matrix`).

Readings (shared with the CUDA path, which implements them independently):
  * theta is the polar angle of (rho_i, z_i), atan2(rho_i, z_i); the printed
    tan^-1(z_i / rho_i) is the elevation, which is not the argument of the
    standard Y_lm of eq. urep.
  * Y_lm is the orthonormal spherical harmonic with the Condon-Shortley phase,
    Y_lm = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!) P_l^m(cos theta) e^{i m phi}
    (the normalisation the paper leaves to its cited library).
  * the B~ printed with the value j_l Y_lm is the Dirichlet functional; the
    Neumann rows take the normal derivative, as A's rows do.
  * with the obstacle's axis on the expansion's z axis the mean over phi is
    delta_{mn} times the meridian-plane functional of j_l(k r) P_l^m-part:
    B~ is block diagonal in the mode (only m = n), and real for real k; the
    trapezoid rule reproduces this exactly for q > |m| + |n| nodes.

Q (the periodizing rows of eq. full for the unknowns [d; a; b]): the S
blocks put the spherical waves and their x-, y-, z-derivatives at M1 x M1
product Gauss nodes of the unit cell's faces, combined into the
discrepancies of eqs. qp1-qp4 and the Cauchy data on T and D; the W blocks
put the Rayleigh-Bloch waves on T and D (eqs. rb1-rb2, T-nD). Readings:
the cell is [-ex/2, ex/2] x [-ey/2, ey/2] x [-z0, z0] around the obstacle;
(kx, ky) = k (d_x, d_y) of the incident direction, alpha = e^{i kx ex},
beta = e^{i ky ey}; the Rayleigh-Bloch set is |kappa| <= pi N0, ordered by
m then n; k_z takes the principal square root (+i sqrt for evanescent
waves).

C (eq. full's C block, Neumann): the same rows applied to the ring part of
eq. urep with the nine phased images of eq. Phinear, by definition on both
walls of each pair. Readings: the ring integrals use the P-node trapezoid
rule with absolute nodes 2 pi s / P (the point sources of Sec. 4.1, "q = P
is sufficient" for distant interactions) and the repository's mode sign
e^{+i n psi} (`point_strengths`); columns follow the operator's
coefficients, mode n at n mod P.

Pins (tests/test_oracle_periodizing.py):
  sph_jn             closed forms of j_0, j_1, j_2 and j_0' = -j_1
  sph_y              closed forms of Y_00, Y_1m, Y_22 (fixes the phase)
  sph_wave_*         the plane-wave expansion e^{ik d.x} = 4 pi sum i^l
                     j_l(kr) Y_lm(x^) conj(Y_lm(d^)), value and normal
                     derivative against i k (n.d) e^{ik d.x}
  btilde             m != n entries vanish, m = n entries are real; B~ times
                     the plane wave's coefficients equals minus the modal
                     incident data of `incident_samples` + `rhs_modes`
  q_matrix           a quasi-periodic plane wave (its spherical-wave
                     coefficients, and its own Rayleigh-Bloch mode as a or b)
                     leaves every discrepancy row zero, and the Cauchy rows
                     of the wall it radiates through; the Gauss nodes against
                     the closed form of the 2-node rule
  c_matrix           C times a coefficient vector equals the phased image
                     sums of `potential` (value and Cartesian derivatives) at
                     the shifted wall nodes, combined into the same rows
  q_pinv_solve       a matrix built with prescribed singular values (random
                     unitary factors): the values come back, and the solve
                     inverts the kept part exactly
  btilde_samples     for p < P/2, the direct value of the truncated expansion's
                     normal derivative, sum d_lm dn u_lm, at the P ring nodes
                     (no trapezoid sum, no transform)
  periodic_operator_apply   composed of the functions above, each pinned
  periodic_solve_dense      the assembled matrix reproduces the operator on
                     a random vector; the solve is LAPACK's
  _a0_plus           the truncated-SVD and QR forms agree when no singular
                     value falls below the cutoff
"""
from __future__ import annotations

import math

import numpy as np
import scipy.special as sps

from .mfs import near_image_sum, rhs_modes, solve_modes, solve_modes_tsvd

__all__ = ["sph_jn", "sph_y", "sph_wave_value_grad", "plane_wave_coefficients",
           "btilde", "btilde_columns", "n_harmonics", "rb_modes", "wall_nodes", "q_matrix",
           "c_matrix", "q_pinv_solve", "btilde_samples",
           "periodic_operator_apply", "periodic_solve_dense"]


def n_harmonics(p):
    """(p + 1)^2 coefficients d_lm, column index l^2 + l + m."""
    return (p + 1) ** 2


def sph_jn(l, x, derivative=False):
    """Spherical Bessel function j_l(x) (or its derivative), scipy's routine."""
    return sps.spherical_jn(l, x, derivative=derivative)


def sph_y(l, m, theta, phi):
    """Orthonormal Y_lm(theta polar, phi azimuth) with the Condon-Shortley phase,
    and its (d/dtheta, d/dphi)."""
    y, g = sps.sph_harm_y(l, m, theta, phi, diff_n=1)
    return y, g[..., 0], g[..., 1]


def sph_wave_value_grad(l, m, k, x):
    """u_lm(x) = j_l(k r) Y_lm(theta, phi) at Cartesian points x [..., 3] and
    its Cartesian gradient [..., 3], by the chain rule through (r, theta, phi):
      grad u = d_r u e_r + (1/r) d_theta u e_theta + 1/(r sin theta) d_phi u e_phi.
    m may be an array that broadcasts against x[..., 0] (all orders of one
    degree in one call).
    """
    x = np.asarray(x, dtype=np.float64)
    X, Y, Z = x[..., 0], x[..., 1], x[..., 2]
    rho = np.hypot(X, Y)
    r = np.hypot(rho, Z)
    theta = np.arctan2(rho, Z)
    phi = np.mod(np.arctan2(Y, X), 2.0 * math.pi)
    jl = sph_jn(l, k * r)
    djl = sph_jn(l, k * r, derivative=True)
    yv, yt, yp = sph_y(l, m, theta, phi)
    u = jl * yv
    du_r = k * djl * yv
    du_t = jl * yt / r
    du_p = jl * yp / (r * np.sin(theta))
    st, ct = np.sin(theta), np.cos(theta)
    cp, sp = np.cos(phi), np.sin(phi)
    e_r = np.stack([st * cp, st * sp, ct], -1)
    e_t = np.stack([ct * cp, ct * sp, -st], -1)
    e_p = np.stack([-sp, cp, np.zeros_like(sp)], -1)
    grad = du_r[..., None] * e_r + du_t[..., None] * e_t + du_p[..., None] * e_p
    return u, grad


def plane_wave_coefficients(p, d):
    """d_lm of e^{ik d.x} = 4 pi sum_lm i^l j_l(kr) Y_lm(x^) conj(Y_lm(d^)), l <= p
    (the Rayleigh plane-wave expansion), in column order l^2 + l + m."""
    d = np.asarray(d, dtype=np.float64)
    th = math.atan2(math.hypot(d[0], d[1]), d[2])
    ph = math.atan2(d[1], d[0]) % (2.0 * math.pi)
    out = np.zeros(n_harmonics(p), dtype=np.complex128)
    for l in range(p + 1):
        for m in range(-l, l + 1):
            out[l * l + l + m] = 4.0 * math.pi * (1j ** l) * np.conj(sph_y(l, m, th, ph)[0])
    return out


def _ring_nodes(coll, q):
    """Ring nodes x_{i s} = (rho_i cos phi_s, rho_i sin phi_s, z_i) and their
    normals (n_rho cos phi_s, n_rho sin phi_s, n_z), phi_s = 2 pi s / q."""
    phi = 2.0 * math.pi * np.arange(q) / q
    rho, z, nr, nz = (coll[:, i][:, None] for i in range(4))
    X = np.stack([rho * np.cos(phi), rho * np.sin(phi), np.broadcast_to(z, (coll.shape[0], q))], -1)
    Nv = np.stack([nr * np.cos(phi), nr * np.sin(phi), np.broadcast_to(nz, (coll.shape[0], q))], -1)
    return X, Nv


def btilde(ob, coll, p, q, modes=None, rows=None):
    """B~ by the printed trapezoid rule: [len(modes)][n_rows][(p+1)^2] complex.

    modes: the distinct modes n to form (default 0 .. P/2); rows: indices of
    the collocation points (default all). Neumann: rows are the normal
    derivative; transmission: [value; normal derivative] (2 len(rows) rows).
    The sum over the q nodes of each mode is a matrix product with
    e^{-2 pi i n s / q} / q.
    """
    if modes is None:
        modes = range(ob.P // 2 + 1)
    modes = list(modes)
    c = coll if rows is None else coll[np.asarray(rows)]
    X, Nv = _ring_nodes(c, q)
    nr = c.shape[0]
    F_val = np.zeros((nr, n_harmonics(p), q), dtype=np.complex128)
    F_dn = np.zeros_like(F_val)
    for l in range(p + 1):
        ms = np.arange(-l, l + 1)[:, None, None]
        u, g = sph_wave_value_grad(l, ms, ob.k, X[None])               # [2l+1][rows][q]
        F_val[:, l * l:(l + 1) ** 2, :] = np.moveaxis(u, 0, 1)
        F_dn[:, l * l:(l + 1) ** 2, :] = np.moveaxis(np.sum(g * Nv[None], axis=-1), 0, 1)
    s = np.arange(q)
    E = np.exp(-2j * math.pi * np.outer(s, np.asarray(modes)) / q) / q     # [q][modes]
    dn = np.einsum("ics,sn->nic", F_dn, E)
    if ob.bc == 0:
        return dn
    val = np.einsum("ics,sn->nic", F_val, E)
    return np.concatenate([val, dn], axis=1)


def btilde_columns(p, n):
    """Column indices l^2 + l + n (l = |n| .. p) of mode n's non-zero block."""
    return np.array([l * l + l + n for l in range(abs(n), p + 1)], dtype=np.int64)


# ----------------------------------------------------------------------------
# Q: the periodizing rows of the full system (Sec. 4.1, eq. full): the S
# blocks (spherical waves on the walls) and the W blocks (Rayleigh-Bloch
# waves on T and D, eqs. rb1-rb2 and T-nD)
# ----------------------------------------------------------------------------

def rb_modes(kx, ky, ex, ey, n0):
    """The Rayleigh-Bloch wavevectors kappa = (kx + 2 pi m/ex, ky + 2 pi n/ey)
    with |kappa| <= pi N0 (Sec. 4, after eq. Phinear), ordered by m, then n,
    and k_z = +sqrt(k^2 - |kappa|^2) taken later (principal branch).
    Returns an int array [n_rb][2] of (m, n)."""
    R = math.pi * n0
    out = []
    mlo = math.floor((-R - kx) * ex / (2 * math.pi)) - 1
    mhi = math.ceil((R - kx) * ex / (2 * math.pi)) + 1
    nlo = math.floor((-R - ky) * ey / (2 * math.pi)) - 1
    nhi = math.ceil((R - ky) * ey / (2 * math.pi)) + 1
    for m in range(mlo, mhi + 1):
        for n in range(nlo, nhi + 1):
            kap_x = kx + 2 * math.pi * m / ex
            kap_y = ky + 2 * math.pi * n / ey
            if kap_x * kap_x + kap_y * kap_y <= R * R:
                out.append((m, n))
    return np.array(out, dtype=np.int64).reshape(-1, 2)


def wall_nodes(ex, ey, z0, m1):
    """M1 x M1 product Gauss-Legendre nodes on the faces of the unit cell
    U = [-ex/2, ex/2] x [-ey/2, ey/2] x [-z0, z0] (Sec. 4.1), per row block:
    L/R share (y, z) (node a b -> y_a, z_b), B/F share (x, z), T/D share (x, y).
    Returns dict of [M1*M1][3] points for L, R, B, F, T, D (row index a*M1 + b)."""
    g, _ = np.polynomial.legendre.leggauss(m1)
    A, Bn = np.meshgrid(g, g, indexing="ij")
    a, b = A.ravel(), Bn.ravel()
    one = np.ones_like(a)
    return {
        "L": np.stack([-ex / 2 * one, ey / 2 * a, z0 * b], -1),
        "R": np.stack([ex / 2 * one, ey / 2 * a, z0 * b], -1),
        "B": np.stack([ex / 2 * a, -ey / 2 * one, z0 * b], -1),
        "F": np.stack([ex / 2 * a, ey / 2 * one, z0 * b], -1),
        "T": np.stack([ex / 2 * a, ey / 2 * b, z0 * one], -1),
        "D": np.stack([ex / 2 * a, ey / 2 * b, -z0 * one], -1),
    }


def q_matrix(k, p, kx, ky, ex, ey, z0, m1, n0):
    """Q of eq. full for the spherical-wave and Rayleigh-Bloch unknowns
    [d_lm; a; b]: 8 M1^2 rows in the printed order
      u_R - alpha u_L, d_x u_R - alpha d_x u_L, u_F - beta u_B, d_y u_F - beta d_y u_B,
      u_T, d_z u_T, u_D, d_z u_D
    (eqs. qp1-qp4, T-nD with all normals along +x, +y, +z), alpha = e^{i kx ex},
    beta = e^{i ky ey}; columns (p+1)^2 spherical waves (l^2 + l + m), then
    a and b over `rb_modes` (the W blocks enter with a minus sign:
    -e^{i(kap_x x + kap_y y)} and -i k_z e^{...} on T, -e^{...} and
    +i k_z e^{...} on D). Returns (Q [rows][cols] complex, modes)."""
    nodes = wall_nodes(ex, ey, z0, m1)
    modes = rb_modes(kx, ky, ex, ey, n0)
    nr = m1 * m1
    nh = n_harmonics(p)
    nrb = modes.shape[0]
    alpha, beta = np.exp(1j * kx * ex), np.exp(1j * ky * ey)
    Q = np.zeros((8 * nr, nh + 2 * nrb), dtype=np.complex128)
    for l in range(p + 1):
        ms = np.arange(-l, l + 1)[:, None]
        cols = slice(l * l, (l + 1) ** 2)
        U = {}
        for f in "LRBFTD":
            u, g = sph_wave_value_grad(l, ms, k, nodes[f][None])    # [2l+1][nr], [2l+1][nr][3]
            U[f] = (u, g)
        Q[0 * nr:1 * nr, cols] = (U["R"][0] - alpha * U["L"][0]).T
        Q[1 * nr:2 * nr, cols] = (U["R"][1][..., 0] - alpha * U["L"][1][..., 0]).T
        Q[2 * nr:3 * nr, cols] = (U["F"][0] - beta * U["B"][0]).T
        Q[3 * nr:4 * nr, cols] = (U["F"][1][..., 1] - beta * U["B"][1][..., 1]).T
        Q[4 * nr:5 * nr, cols] = U["T"][0].T
        Q[5 * nr:6 * nr, cols] = U["T"][1][..., 2].T
        Q[6 * nr:7 * nr, cols] = U["D"][0].T
        Q[7 * nr:8 * nr, cols] = U["D"][1][..., 2].T
    kap_x = kx + 2 * math.pi * modes[:, 0] / ex
    kap_y = ky + 2 * math.pi * modes[:, 1] / ey
    kz = np.sqrt((k * k - kap_x ** 2 - kap_y ** 2).astype(np.complex128))
    for f, r0, c0, sgn in (("T", 4, nh, 1.0), ("D", 6, nh + nrb, -1.0)):
        x = nodes[f]
        E = np.exp(1j * (np.outer(x[:, 0], kap_x) + np.outer(x[:, 1], kap_y)))   # [nr][nrb]
        Q[r0 * nr:(r0 + 1) * nr, c0:c0 + nrb] = -E
        Q[(r0 + 1) * nr:(r0 + 2) * nr, c0:c0 + nrb] = -sgn * 1j * kz[None, :] * E
    return Q, modes


# ----------------------------------------------------------------------------
# C: the periodizing rows' dependence on the ring coefficients eta (Sec. 4.1,
# eq. full and the C-block paragraph), Neumann obstacles
# ----------------------------------------------------------------------------

def _ring_modes(k, src, P, X, axis=None):
    """Phi_nj(X) (or its Cartesian derivative along `axis`) for every mode and
    proxy ring, by the P-node trapezoid rule with absolute nodes
    psi_s = 2 pi s / P (the point sources of Sec. 4.1):
      Phi_nj(x) = (1/P) sum_s G_k(x, y_j(psi_s)) e^{+i n psi_s}
    (the repository's mode convention, as in `point_strengths`).
    X [T][3] -> [T][P (n mod P)][N]."""
    N = src.shape[0]
    psi = 2.0 * math.pi * np.arange(P) / P
    Y = np.stack([src[:, 0][:, None] * np.cos(psi), src[:, 0][:, None] * np.sin(psi),
                  np.broadcast_to(src[:, 1][:, None], (N, P))], -1)            # [N][P][3]
    D = X[:, None, None, :] - Y[None]                                           # [T][N][P][3]
    R = np.linalg.norm(D, axis=-1)
    e = np.exp(1j * k * R)
    if axis is None:
        K = e / (4.0 * math.pi * R)
    else:
        K = D[..., axis] * (1j * k * R - 1.0) * e / (4.0 * math.pi * R ** 3)
    n = np.arange(P)
    n = np.where(n > P // 2, n - P, n)
    E = np.exp(1j * np.outer(psi, n)) / P                                       # [P s][P n]
    return np.einsum("tjs,sn->tnj", K, E)


def c_matrix(ob, src, kx, ky, ex, ey, z0, m1, row_pairs=None):
    """C of eq. full for a Neumann obstacle: the rows of `q_matrix` applied to
    the ring part of u (eq. urep), u = sum_{n,j} c_nj Phi^near_nj with the
    3 x 3 phased images of eq. Phinear,
      Phi^near_nj(x) = sum_{|a|,|b| <= 1} alpha^a beta^b Phi_nj(x - a e_x - b e_y),
    evaluated by its definition on both walls of each pair (18 terms, then
    u_R - alpha u_L etc.; the cancellation of Sec. 4.1 is left to the
    arithmetic). Columns: mode n at n mod P, then ring j (col = (n mod P) N + j),
    the operator's coefficient order. row_pairs: indices a*M1 + b of the node
    pairs to form (default all); returns [8 len][P N], blocks as q_matrix."""
    P, k = ob.P, ob.k
    nodes = wall_nodes(ex, ey, z0, m1)
    idx = np.arange(m1 * m1) if row_pairs is None else np.asarray(row_pairs)
    alpha, beta = np.exp(1j * kx * ex), np.exp(1j * ky * ey)

    def near(X, axis=None):
        out = 0.0
        for a in (-1, 0, 1):
            for b in (-1, 0, 1):
                sh = np.array([a * ex, b * ey, 0.0])
                out = out + alpha ** a * beta ** b * _ring_modes(k, src, P, X - sh, axis)
        return out.reshape(X.shape[0], -1)                                      # [T][P N]

    L, R, B, F, T, Dn = (nodes[f][idx] for f in "LRBFTD")
    blocks = [near(R) - alpha * near(L), near(R, 0) - alpha * near(L, 0),
              near(F) - beta * near(B), near(F, 1) - beta * near(B, 1),
              near(T), near(T, 2), near(Dn), near(Dn, 2)]
    return np.concatenate(blocks, axis=0)


# ----------------------------------------------------------------------------
# Q^+ by the SVD (Sec. 4.2: "rapid to invert (via SVD)"; the O(k^6) stage)
# ----------------------------------------------------------------------------

def q_pinv_solve(Q, B, cutoff):
    """x = Q^+ b through the SVD with singular values below cutoff * sigma_max
    dropped (LAPACK's SVD through numpy, a library primitive); returns
    (X, singular values in descending order)."""
    U, s, Vh = np.linalg.svd(Q, full_matrices=False)
    keep = s > cutoff * s[0]
    W = (U[:, keep].conj().T @ B) / s[keep][:, None]
    return Vh[keep].conj().T @ W, s


# ----------------------------------------------------------------------------
# One application of the preconditioned periodic operator (Sec. 4.2, eq. iter)
# ----------------------------------------------------------------------------

def btilde_samples(ob, coll, p, d):
    """The B~ term of eq. iter carried back to the ring nodes: with the modal
    data fhat_n = sum_lm B~_{n,lm} d_lm for the P modes the rows hold,
    -P/2 < n <= P/2 (mode -P/2 is not among them, as in `rhs_modes`),
      f_{m,l} = sum_n fhat_{n,m} e^{2 pi i n l / P}
    (the inverse of eq. fhatquad's sum). Neumann rows; d [W][(p+1)^2] ->
    [W][M][P]. B~ by `btilde` with q = 2 (p + P) + 2 nodes, more than
    |m| + |n| for every pair, so its trapezoid sums are exact."""
    P = ob.P
    nm = np.arange(P)
    nm = np.where(nm > P // 2, nm - P, nm)
    Bt = btilde(ob, coll, p, 2 * (p + P) + 2, modes=list(nm))                 # [P][M][(p+1)^2]
    fB = np.einsum("nrc,wc->wnr", Bt, np.atleast_2d(d))                        # [W][P][M]
    E = np.exp(2j * math.pi * np.outer(nm, np.arange(P)) / P)                  # [n][l]
    return np.einsum("wnr,nl->wrl", fB, E)


def _a0_plus(ob, factors, fhat):
    """A_0^+ fhat: `solve_modes` for the list of (packed QR, tau), or the
    truncated SVD of Sec. 4.2 (`solve_modes_tsvd`, 1e-10 cutoff) when factors
    is ("tsvd", A) with A the modal matrices [P/2+1][rows][cols]."""
    if isinstance(factors, tuple) and factors[0] == "tsvd":
        return solve_modes_tsvd(ob, factors[1], fhat)
    return solve_modes(ob, factors, fhat)


def periodic_operator_apply(ob, coll, src, factors, g, dirs, lattice, C, Q, p, cutoff=1e-10):
    """y = (I + A_else A_0^+ - B Q^+ C A_0^+) g, eq. iter, for a Neumann
    obstacle. Reading: the paper states the operator on modal data; it acts
    here on boundary samples g [W][M][P], i.e. conjugated by the transform of
    eq. fhatquad, so that the device apply (samples in) and the near-image
    sum (samples out) compose without extra transforms; a solve in either
    space gives the same eta. Steps:
      coef = A_0^+ g          `rhs_modes`, then `solve_modes` (the QR factors)
      A_else coef             `near_image_sum` with the waves' Bloch phases
      xi = Q^+ (C coef)       the rows of `c_matrix`, `q_pinv_solve` with
                              the paper's 1e-10 relative cutoff
      B xi                    `btilde_samples` of xi's spherical-wave part d
    factors: the list of (packed QR, tau) of `factor_operator`, or ("tsvd",
    A) for the paper's truncated-SVD A_0^+ (see `_a0_plus`). Returns y
    [W][M][P]."""
    W, M, P = g.shape
    coef = _a0_plus(ob, factors, rhs_modes(g))                                 # [W][P][N]
    ae = near_image_sum(ob, coll, src, coef, dirs, lattice).reshape(W, M, P)
    yC = coef.reshape(W, -1) @ C.T                                             # [W][8 M1^2]
    xi, _ = q_pinv_solve(Q, yC.T, cutoff)                                      # [nQ][W]
    return g + ae - btilde_samples(ob, coll, p, xi[:n_harmonics(p)].T)


def periodic_solve_dense(ob, coll, src, factors, f, dirs, lattice, C, Q, p, cutoff=1e-10):
    """Eq. iter solved directly, for small cases (Sec. 4.2): the operator's
    matrix over the n = M P samples, column i the image of unit vector i
    under `periodic_operator_apply`, solved by LAPACK for every wave of f
    [W][M][P]; then eta = A_0^+ eta~ (`solve_modes`) and xi = -Q^+ C eta
    (`q_pinv_solve`). dirs [3] is the Bloch direction; factors as in
    `periodic_operator_apply`. Returns (eta~ [W][M][P],
    eta [W][P][N], xi [W][nQ], the operator matrix [n][n])."""
    W, M, P = f.shape
    n = M * P
    E = np.eye(n, dtype=np.complex128).reshape(n, M, P)
    Aop = periodic_operator_apply(ob, coll, src, factors, E, np.stack([np.asarray(dirs)] * n), lattice,
                                  C, Q, p, cutoff).reshape(n, n).T
    et = np.linalg.solve(Aop, f.reshape(W, n).T).T.reshape(W, M, P)
    eta = _a0_plus(ob, factors, rhs_modes(et))
    xi, _ = q_pinv_solve(Q, (eta.reshape(W, -1) @ C.T).T, cutoff)
    return et, eta, -xi.T, Aop
