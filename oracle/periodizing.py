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

Pins (tests/test_oracle_periodizing.py):
  sph_jn             closed forms of j_0, j_1, j_2 and j_0' = -j_1
  sph_y              closed forms of Y_00, Y_1m, Y_22 (fixes the phase)
  sph_wave_*         the plane-wave expansion e^{ik d.x} = 4 pi sum i^l
                     j_l(kr) Y_lm(x^) conj(Y_lm(d^)), value and normal
                     derivative against i k (n.d) e^{ik d.x}
  btilde             m != n entries vanish, m = n entries are real; B~ times
                     the plane wave's coefficients equals minus the modal
                     incident data of `incident_samples` + `rhs_modes`
"""
from __future__ import annotations

import math

import numpy as np
import scipy.special as sps

__all__ = ["sph_jn", "sph_y", "sph_wave_value_grad", "plane_wave_coefficients",
           "btilde", "btilde_columns", "n_harmonics"]


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
