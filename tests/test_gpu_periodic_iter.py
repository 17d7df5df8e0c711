"""One application of the preconditioned periodic operator (Sec. 4.2, eq.
iter) on the GPU against the oracle: the dense C eta product, the B~ term
carried back to the ring nodes with the combine, and the whole composite
y = (I + A_else A_0^+ - B Q^+ C A_0^+) g."""
import numpy as np
import pytest

import oracle as O
import synth
from oracle import mfs as OM
from oracle import periodizing as OP

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("rows,cols,nrhs", [(300, 1000, 1), (300, 1000, 3), (97, 5000, 16), (64, 50, 5),
                                            (1, 1, 1)])
def test_matvec_parity(rows, cols, nrhs):
    """Y = A X against numpy's product: within 1e-13 of sum |A| |X| per row
    (the summation order differs), and the same bits on a second run."""
    from paper_1506_05083_gb300 import axi
    rng = np.random.default_rng(rows + cols + nrhs)
    A = rng.normal(size=(cols, rows)) + 1j * rng.normal(size=(cols, rows))      # column-major A
    X = rng.normal(size=(nrhs, cols)) + 1j * rng.normal(size=(nrhs, cols))
    At, Xt = torch.tensor(A, device="cuda"), torch.tensor(X, device="cuda")
    Y1 = axi.matvec_c128(At, Xt)
    Y2 = axi.matvec_c128(At, Xt)
    torch.cuda.synchronize()
    ref = X @ A                                                                  # [nrhs][rows]
    bound = np.abs(X) @ np.abs(A)
    assert np.all(np.abs(Y1.cpu().numpy() - ref) <= 1e-13 * bound + 1e-300)
    assert torch.equal(Y1, Y2)


def _small_op(P=16):
    from paper_1506_05083_gb300 import axi
    wl = synth.small_case(seed=7, k=3.0, M=40, N=32, P=P)
    ob = wl.obstacles[0]
    coll, src, srcx = O.geometry(ob)
    op = axi.Operator([axi.spec_from_obstacle(ob)], prec=axi.PREC_FP64)
    return axi, wl, ob, coll, src, srcx, op


@pytest.mark.parametrize("p", [6, 8, 12])
def test_iter_combine_btilde_term(p):
    """y = g + a - B d against g + a - `btilde_samples`: p below, at and above
    P/2 (modes |n| > P/2 of the waves are not held by the rows), and with g
    and a left out (B d alone, negated)."""
    axi, wl, ob, coll, src, srcx, op = _small_op()
    rng = np.random.default_rng(p)
    W, nh = 2, OP.n_harmonics(p)
    d = rng.normal(size=(W, nh + 3)) + 1j * rng.normal(size=(W, nh + 3))         # ldd > (p+1)^2
    g = rng.normal(size=(W, ob.M, ob.P)) + 1j * rng.normal(size=(W, ob.M, ob.P))
    a = rng.normal(size=g.shape) + 1j * rng.normal(size=g.shape)
    _, bt = op.btilde(p)
    dt, gt, at = (torch.tensor(x, device="cuda") for x in (d, g, a))
    y = axi.iter_combine(gt, at, bt, dt, p).cpu().numpy()
    y0 = axi.iter_combine(None, at * 0, bt, dt, p).cpu().numpy()
    torch.cuda.synchronize()
    assert op.status() == 0
    Bd = OP.btilde_samples(ob, coll, p, d[:, :nh])
    scale = np.abs(Bd).max()
    assert np.abs(y0 + Bd).max() < 1e-12 * scale
    assert np.abs(y - (g + a - Bd)).max() < 1e-12 * max(scale, np.abs(g).max())


def _abs_image_bound(ob, coll, src, coef, lattice):
    """max over targets and waves of sum |dG/dn| |sigma| over the eight
    images: the scale a digit split's rounding is relative to (large
    coefficients whose images cancel leave the sum itself far smaller)."""
    P, k = ob.P, ob.k
    sig = np.abs(O.point_strengths(coef, P).reshape(coef.shape[0], -1))
    X, Nv = OP._ring_nodes(coll, P)
    X, Nv = X.reshape(-1, 3), Nv.reshape(-1, 3)
    Y = OM._source_points(src, P).reshape(-1, 3)
    B = 0.0
    for a in (-1, 0, 1):
        for b in (-1, 0, 1):
            if a or b:
                Dv = X[:, None, :] - (Y[None] + np.array([a * lattice[0], b * lattice[1], 0.0]))
                R = np.linalg.norm(Dv, axis=-1)
                K = np.abs(np.einsum("tc,tsc->ts", Nv, Dv)) * np.abs(1j * k * R - 1.0) / (4 * np.pi * R ** 3)
                B = B + sig @ K.T
    return np.max(B)


@pytest.mark.parametrize("near_slices", [0, 6, 7])
def test_periodic_iter_apply_parity(near_slices):
    """The composite on the small obstacle in a cell of the same Bloch phases
    as the near-image sum's waves: (1) every step after A_0^+ against the
    oracle's steps on the device's own coefficients, 1e-11 of the output
    scale; (2) the coefficients against the oracle's QR solve by the boundary
    residual (they are not unique); (3) the whole output against the oracle's
    composite, within the spread the coefficients' non-uniqueness allows.
    With the near-image sum split into digits, (1) and (3) are bounded by the
    split's rounding, relative to sum |dG/dn| |sigma| (2^-37 of it for 6
    digits of 7 bits, 2^-44 for 7, with the FP32 group sums' margin)."""
    axi, wl, ob, coll, src, srcx, op = _small_op()
    ob.q = O.choose_q(ob, coll, src, srcx)
    d = np.array([0.36, -0.28, np.sqrt(1 - 0.36**2 - 0.28**2)])
    ex, ey, z0, m1, n0, p = 2.6, 2.3, 1.6, 6, 3, 8
    cell = axi.Cell(ob.k * d[0], ob.k * d[1], ex, ey, z0, m1, n0, p)
    W = 2
    rng = np.random.default_rng(5)
    g = rng.normal(size=(W, ob.M, ob.P)) + 1j * rng.normal(size=(W, ob.M, ob.P))
    dirs = np.stack([d] * W)
    Cg = op.c_block(cell)
    Qg = op.q_matrix(cell)
    US = Qg.clone()
    V, sig, sweeps = axi.svd_jacobi(US)
    _, bt = op.btilde(p)
    y, coef = axi.periodic_iter_apply(op, torch.tensor(g, device="cuda"), (ex, ey),
                                      torch.tensor(dirs, device="cuda"), Cg, US, V, sig, bt, p,
                                      near_slices=near_slices, want_coef=True)
    torch.cuda.synchronize()
    assert op.status() == 0
    y, c_gpu = y.cpu().numpy(), coef.cpu().numpy()
    Co = OP.c_matrix(ob, src, cell.kx, cell.ky, ex, ey, z0, m1)
    Qo, _ = OP.q_matrix(ob.k, p, cell.kx, cell.ky, ex, ey, z0, m1, n0)
    # (1) the steps after A_0^+ on the device's coefficients
    ae = O.near_image_sum(ob, coll, src, c_gpu, dirs, (ex, ey)).reshape(g.shape)
    xi, _ = OP.q_pinv_solve(Qo, (c_gpu.reshape(W, -1) @ Co.T).T, 1e-10)
    y_steps = g + ae - OP.btilde_samples(ob, coll, p, xi[:OP.n_harmonics(p)].T)
    e1 = np.abs(y - y_steps).max() / np.abs(y_steps).max()
    # (2) A_0^+ against the oracle's factors by the boundary residual
    A, fac = O.factor_operator(ob, coll, src, srcx)
    fh = O.rhs_modes(g)
    c_ora = O.solve_modes(ob, fac, fh)
    An = A[np.minimum(np.arange(ob.P), ob.P - np.arange(ob.P))]                # mode slot -> |n|
    res = np.abs(np.einsum("prc,wpc->wpr", An, c_gpu - c_ora)).max() / np.abs(fh).max()
    # (3) the whole composite
    y_ora = OP.periodic_operator_apply(ob, coll, src, fac, g, dirs, (ex, ey), Co, Qo, p)
    e3 = np.abs(y - y_ora).max() / np.abs(y_ora).max()
    print(f"slices {near_slices}: steps {e1:.3e}  coef residual {res:.3e}  composite {e3:.3e}  "
          f"sweeps {sweeps}")
    if near_slices:
        bound = _abs_image_bound(ob, coll, src, c_gpu, (ex, ey)) / np.abs(y_steps).max()
        print(f"  sum|K||sigma| / max|y| = {bound:.3e}; error / bound: {e1 / bound:.3e}")
        tol = 2.0 ** (-7 * near_slices + 5) * bound + 1e-11
    else:
        tol = 1e-11
    assert e1 < tol
    assert res < 1e-10
    assert e3 < max(tol, 1e-11)


def test_gmres_dense_operator():
    """The GMRES driver alone on A = I + K (K Gaussian, spectral radius about
    1/2; n = 300) applied by the matvec kernel, restart 10 so that the true
    residual is re-formed several times; a zero right-hand side stays zero
    with no steps. Against LAPACK's solve."""
    from paper_1506_05083_gb300 import axi
    rng = np.random.default_rng(8)
    n, W = 300, 3
    K = (rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))) / (2 * np.sqrt(2 * n))
    A = np.eye(n) + K
    b = rng.normal(size=(W, n)) + 1j * rng.normal(size=(W, n))
    b[2] = 0.0
    At = torch.tensor(np.ascontiguousarray(A.T), device="cuda")                 # column-major A
    x, its, rel, conv = axi.gmres(lambda v, out: axi.matvec_c128(At, v, out=out),
                                  torch.tensor(b, device="cuda"), tol=1e-12, restart=10, max_iter=400)
    torch.cuda.synchronize()
    xr = np.linalg.solve(A, b[:2].T).T
    assert conv == [True, True, True]
    assert its[2] == 0 and np.all(x[2].cpu().numpy() == 0)
    assert max(rel[:2]) <= 1e-12
    assert np.abs(x[:2].cpu().numpy() - xr).max() < 1e-10 * np.abs(xr).max()
    assert 10 < its[0] <= 400


def test_periodic_solve_small():
    """Eq. iter solved by GMRES on the GPU (tol 1e-12) for the small obstacle's
    incident data in its cell: eta~ against the oracle's dense solve; the
    residual of eq. iter and xi = -Q^+ C eta recomputed by the oracle's steps
    from the device's eta~, eta and xi."""
    axi, wl, ob, coll, src, srcx, op = _small_op()
    ob.q = O.choose_q(ob, coll, src, srcx)
    d = np.array([0.36, -0.28, np.sqrt(1 - 0.36**2 - 0.28**2)])
    ex, ey, z0, m1, n0, p = 2.6, 2.3, 1.6, 6, 3, 8
    cell = axi.Cell(ob.k * d[0], ob.k * d[1], ex, ey, z0, m1, n0, p)
    dirs = np.stack([d, d])
    f = O.incident_samples(ob, coll, dirs)                                       # [W][M][P]
    Cg, US = op.c_block(cell), op.q_matrix(cell)
    V, sig, _ = axi.svd_jacobi(US)
    _, bt = op.btilde(p)
    et, eta, xi, its, rel, conv = axi.periodic_solve(op, torch.tensor(f, device="cuda"), (ex, ey),
                                                     torch.tensor(dirs, device="cuda"), Cg, US, V, sig,
                                                     bt, p, tol=1e-12, restart=40)
    torch.cuda.synchronize()
    assert op.status() == 0 and all(conv), (its, rel)
    et, eta, xi = et.cpu().numpy(), eta.cpu().numpy(), xi.cpu().numpy()
    A, fac = O.factor_operator(ob, coll, src, srcx)
    Co = OP.c_matrix(ob, src, cell.kx, cell.ky, ex, ey, z0, m1)
    Qo, _ = OP.q_matrix(ob.k, p, cell.kx, cell.ky, ex, ey, z0, m1, n0)
    et_o, _, _, Aop = OP.periodic_solve_dense(ob, coll, src, fac, f, d, (ex, ey), Co, Qo, p)
    e_et = np.abs(et - et_o).max() / np.abs(et_o).max()
    ae = O.near_image_sum(ob, coll, src, eta, dirs, (ex, ey)).reshape(f.shape)
    res = et + ae + OP.btilde_samples(ob, coll, p, xi[:, :OP.n_harmonics(p)]) - f
    e_res = np.abs(res).max() / np.abs(f).max()
    xo, _ = OP.q_pinv_solve(Qo, (eta.reshape(2, -1) @ Co.T).T, 1e-10)
    e_xi = np.abs(xi + xo.T).max() / np.abs(xo).max()
    print(f"iters {its} relres {rel}  eta~ {e_et:.2e}  residual {e_res:.2e}  xi {e_xi:.2e}  "
          f"cond {np.linalg.cond(Aop):.1f}")
    assert e_et < 1e-10
    assert e_res < 1e-10
    assert e_xi < 1e-10


def test_periodic_solve_ill_conditioned_tsvd():
    """An obstacle with 140 proxies, whose worst modal block has sigma_min /
    sigma_max near 3e-13, below the paper's 1e-10 truncation: with A_0^+ as the
    truncated SVD (the operator's AXI_PLAN_TSVD form, Sec. 4.2) the Krylov
    vectors' coefficients stay bounded, so the near-image sum split into 7
    digits stays accurate and GMRES reaches 1e-10 (measured: 16 steps,
    1.0e-11). eta~ against the oracle's dense solve with the same
    truncated-SVD A_0^+, within kappa times the two solutions' residuals;
    the residual of eq. iter
    from the device's eta~, eta and xi by the oracle's steps, against the
    same residual of the oracle's own solution (A_0^+ still amplifies
    rounding by up to 1e10 / sigma_max, so neither is at rounding level)."""
    from paper_1506_05083_gb300 import axi
    wl = synth.small_case(seed=7, k=3.0, M=160, N=140, P=16)
    ob = wl.obstacles[0]
    coll, src, srcx = O.geometry(ob)
    ob.q = O.choose_q(ob, coll, src, srcx)
    op = axi.Operator([axi.spec_from_obstacle(ob)], prec=axi.PREC_FP64 | axi.PLAN_TSVD)
    d = np.array([0.36, -0.28, np.sqrt(1 - 0.36**2 - 0.28**2)])
    ex, ey, z0, m1, n0, p = 2.6, 2.3, 1.6, 6, 3, 8
    cell = axi.Cell(ob.k * d[0], ob.k * d[1], ex, ey, z0, m1, n0, p)
    dirs = np.stack([d])
    f = O.incident_samples(ob, coll, dirs)
    Cg, US = op.c_block(cell), op.q_matrix(cell)
    V, sig, _ = axi.svd_jacobi(US)
    _, bt = op.btilde(p)
    et, eta, xi, its, rel, conv = axi.periodic_solve(op, torch.tensor(f, device="cuda"), (ex, ey),
                                                     torch.tensor(dirs, device="cuda"), Cg, US, V, sig,
                                                     bt, p, near_slices=7, tol=1e-10, restart=40)
    torch.cuda.synchronize()
    assert op.status() == 0 and all(conv), (its, rel)
    et, eta, xi = et.cpu().numpy(), eta.cpu().numpy(), xi.cpu().numpy()
    A = O.system_matrix(ob, coll, src, srcx)
    Co = OP.c_matrix(ob, src, cell.kx, cell.ky, ex, ey, z0, m1)
    Qo, _ = OP.q_matrix(ob.k, p, cell.kx, cell.ky, ex, ey, z0, m1, n0)
    et_o, eta_o, xi_o, Aop = OP.periodic_solve_dense(ob, coll, src, ("tsvd", A), f, d, (ex, ey), Co, Qo, p)
    e_et = np.abs(et - et_o).max() / np.abs(et_o).max()

    def residual(et_, eta_, xi_):
        ae = O.near_image_sum(ob, coll, src, eta_, dirs, (ex, ey)).reshape(f.shape)
        r = et_ + ae + OP.btilde_samples(ob, coll, p, xi_[:, :OP.n_harmonics(p)]) - f
        return np.abs(r).max() / np.abs(f).max()

    e_res, e_res_o = residual(et, eta, xi), residual(et_o, eta_o, xi_o)
    print(f"iters {its} relres {rel}  eta~ {e_et:.2e}  residual {e_res:.2e} (oracle's own {e_res_o:.2e})  "
          f"|eta| {np.abs(eta).max():.2e} (oracle {np.abs(eta_o).max():.2e})")
    # two approximate solutions of a system of condition kappa differ by at
    # most about kappa times the sum of their relative residuals (factor 2:
    # max norms)
    kappa = np.linalg.cond(Aop)
    assert e_et < 2 * kappa * (e_res + e_res_o) + 1e-12, kappa
    assert e_res < max(10 * e_res_o, 1e-10)
