"""The periodizing scheme's spherical-wave block B~ (Sec. 4, eq. urep; Sec.
4.1) on the GPU against the oracle's trapezoid-rule B~ (oracle/periodizing.py):
each stored mode block equals the oracle's m = n columns, and the packing
leaves the modes above min(P/2, p) out."""
import numpy as np
import pytest

import oracle as O
import synth
from oracle import periodizing as OP

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _case(name):
    if name == "small":
        wl = synth.small_case(seed=7, k=3.0, M=40, N=32, P=16)
    elif name == "small_trans":
        wl = synth.small_case(seed=11, k=2.0, M=44, N=36, P=20, bc=synth.BC_TRANSMISSION)
    elif name == "smooth":
        wl = synth.config_smooth()
    else:
        wl = synth.config_cup()
    ob = wl.obstacles[0]
    coll, src, srcx = O.geometry(ob)
    return wl, ob, coll


@pytest.mark.parametrize("name,p,rows", [("small", 12, None), ("small_trans", 7, None),
                                         ("smooth", 20, range(4, 216, 9)),
                                         ("cup", 48, range(5, 432, 54))])
def test_btilde_parity(name, p, rows):
    from paper_1506_05083_gb300 import axi
    wl, ob, coll = _case(name)
    op = axi.Operator([axi.spec_from_obstacle(wl.obstacles[0])], prec=axi.PREC_FP64)
    blocks, buf = op.btilde(p)
    torch.cuda.synchronize()
    assert op.status() == 0
    nmax = min(ob.P // 2, p)
    assert len(blocks) == nmax + 1
    q = p + nmax + 2                                  # no aliasing: q > |m - n| for m, n <= p, nmax
    ref = OP.btilde(ob, coll, p, q, modes=range(nmax + 1), rows=rows)
    idx = np.arange(ob.M) if rows is None else np.asarray(rows)
    if ob.bc == synth.BC_TRANSMISSION:
        idx = np.concatenate([idx, ob.M + idx])
    scale = np.abs(ref).max()
    for n in range(nmax + 1):
        got = blocks[n].cpu().numpy().T[idx]          # [rows][l - n]
        want = ref[n][:, OP.btilde_columns(p, n)]
        assert np.abs(want.imag).max() < 1e-13 * scale
        assert np.abs(got - want.real).max() < 1e-12 * scale, n


def _cell(axi, k, d, ex, ey, z0, m1, n0, p):
    return axi.Cell(k * d[0], k * d[1], ex, ey, z0, m1, n0, p)


@pytest.mark.parametrize("name", ["small", "cup"])
def test_q_parity(name):
    """The periodizing rows Q (S and W blocks) against the oracle's q_matrix:
    the same Rayleigh-Bloch modes in the same order and every entry within
    1e-12 of the matrix scale. The cup case has the bench's k, p and N0 with
    fewer wall nodes."""
    from paper_1506_05083_gb300 import axi
    wl, ob, coll = _case(name)
    if name == "small":
        k, ex, ey, z0, m1, n0, p = ob.k, 2.0, 1.7, 1.5, 6, 3, 12
    else:
        period = 13 * 2 * np.pi / ob.k
        k, ex, ey, z0, m1, n0, p = ob.k, period, period, 1.2 + period / 4, 8, 11, 48
    d = np.array([0.36, -0.28, np.sqrt(1 - 0.36**2 - 0.28**2)])
    op = axi.Operator([axi.spec_from_obstacle(wl.obstacles[0])], prec=axi.PREC_FP64)
    cell = _cell(axi, k, d, ex, ey, z0, m1, n0, p)
    Qg = op.q_matrix(cell)
    torch.cuda.synchronize()
    assert op.status() == 0
    Qo, modes = OP.q_matrix(k, p, k * d[0], k * d[1], ex, ey, z0, m1, n0)
    assert np.array_equal(axi.q_modes(cell), modes)
    Q = Qg.cpu().numpy().T
    assert Q.shape == Qo.shape
    assert np.abs(Q - Qo).max() < 1e-12 * np.abs(Qo).max()


@pytest.mark.parametrize("name,m1,pairs", [("small", 4, None), ("cup", 4, [0, 5, 10, 15])])
def test_c_parity(name, m1, pairs):
    """The C block (nine phased ring-source images, the six distant ones in
    the wall pairs' discrepancies) against the oracle's c_matrix, which
    forms all eighteen terms by definition: every entry of the sampled rows
    within 1e-12 of the block scale."""
    from paper_1506_05083_gb300 import axi
    wl, ob, coll = _case(name)
    _, src, _ = O.geometry(ob)
    if name == "small":
        ex, ey, z0 = 2.6, 2.3, 1.6
    else:
        period = 13 * 2 * np.pi / ob.k
        ex, ey, z0 = period, period, 1.2 + period / 4
    d = np.array([0.36, -0.28, np.sqrt(1 - 0.36**2 - 0.28**2)])
    op = axi.Operator([axi.spec_from_obstacle(wl.obstacles[0])], prec=axi.PREC_FP64)
    cell = axi.Cell(ob.k * d[0], ob.k * d[1], ex, ey, z0, m1, 3, 4)
    Cg = op.c_block(cell)
    torch.cuda.synchronize()
    assert op.status() == 0
    Co = OP.c_matrix(ob, src, ob.k * d[0], ob.k * d[1], ex, ey, z0, m1, row_pairs=pairs)
    G = Cg.cpu().numpy().T                                        # [rows][cols]
    nr = m1 * m1
    idx = np.arange(nr) if pairs is None else np.asarray(pairs)
    rows = np.concatenate([b * nr + idx for b in range(8)])
    assert np.abs(G[rows] - Co).max() < 1e-12 * np.abs(Co).max()


def test_periodize_edges():
    """Edges of the periodizing fills: C on the direct-sum path (P = 14 has
    the prime 7, outside the FFT's radices), B~ and Q at degrees 0 and 1, a
    2 x 2 node cell with an empty Rayleigh-Bloch set, and C refused for a
    transmission obstacle."""
    from paper_1506_05083_gb300 import axi
    wl = synth.small_case(seed=7, k=3.0, M=40, N=32, P=14)
    ob = wl.obstacles[0]
    coll, src, _ = O.geometry(ob)
    op = axi.Operator([axi.spec_from_obstacle(wl.obstacles[0])], prec=axi.PREC_FP64)
    kx, ky, ex, ey, z0 = 1.1, -0.7, 2.6, 2.3, 1.6
    cell = axi.Cell(kx, ky, ex, ey, z0, 4, 3, 4)
    Cg = op.c_block(cell).cpu().numpy().T
    Co = OP.c_matrix(ob, src, kx, ky, ex, ey, z0, 4)
    assert np.abs(Cg - Co).max() < 1e-12 * np.abs(Co).max()
    for p in (0, 1):
        blocks, _ = op.btilde(p)
        ref = OP.btilde(ob, coll, p, p + min(ob.P // 2, p) + 2, modes=range(len(blocks)))
        for n, b in enumerate(blocks):
            want = ref[n][:, OP.btilde_columns(p, n)].real
            assert np.abs(b.cpu().numpy().T - want).max() < 1e-12 * np.abs(ref).max()
        c2 = axi.Cell(0.0, 0.0, ex, ey, z0, 2, 0, p)
        rows, cols, nrb = axi.q_shape(c2)
        assert nrb == 1 and rows == 32                   # only kappa = 0 lies within pi * 0
        Qo, _ = OP.q_matrix(ob.k, p, 0.0, 0.0, ex, ey, z0, 2, 0)
        Qg = op.q_matrix(c2).cpu().numpy().T
        assert np.abs(Qg - Qo).max() < 1e-12 * np.abs(Qo).max()
        c3 = axi.Cell(0.5, 0.5, ex, ey, z0, 2, 0, p)      # |kappa| > 0 for every mode: none kept
        assert axi.q_shape(c3)[2] == 0
        Qo3, _ = OP.q_matrix(ob.k, p, 0.5, 0.5, ex, ey, z0, 2, 0)
        assert np.abs(op.q_matrix(c3).cpu().numpy().T - Qo3).max() < 1e-12 * np.abs(Qo3).max()
    torch.cuda.synchronize()
    assert op.status() == 0
    wt = synth.small_case(seed=11, k=2.0, M=44, N=36, P=20, bc=synth.BC_TRANSMISSION)
    opt = axi.Operator([axi.spec_from_obstacle(wt.obstacles[0])], prec=axi.PREC_FP64)
    with pytest.raises(axi.AxiError):
        opt.c_block(cell)


def _prescribed(rng, m, n, s):
    U, _ = np.linalg.qr(rng.normal(size=(m, n)) + 1j * rng.normal(size=(m, n)))
    V, _ = np.linalg.qr(rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n)))
    return (U * s) @ V.conj().T, V


@pytest.mark.parametrize("nrhs", [1, 3, 16, 21])
def test_svd_jacobi_prescribed(nrhs):
    """The one-sided Jacobi SVD of a matrix with prescribed singular values
    (a gap at 1e-13): the values come back, (U Sigma) V^H rebuilds the
    matrix, V is unitary, and the truncated solve equals the oracle's for
    nrhs right-hand sides (groups of up to 16; 21 leaves a ragged group)."""
    from paper_1506_05083_gb300 import axi
    rng = np.random.default_rng(4)
    m, n = 70, 45
    s = np.concatenate([np.logspace(0, -4, 30), np.logspace(-13, -14, n - 30)])
    A, Vt = _prescribed(rng, m, n, s)
    At = torch.tensor(np.ascontiguousarray(A.T), device="cuda")       # column-major view
    V, sigma, sweeps = axi.svd_jacobi(At)
    US = At.cpu().numpy().T
    Vn = V.cpu().numpy().T
    sg = sigma.cpu().numpy()
    assert sweeps < 30
    assert np.abs(np.sort(sg)[::-1] - s).max() < 1e-13
    assert np.abs(US @ Vn.conj().T - A).max() < 1e-13
    assert np.abs(Vn.conj().T @ Vn - np.eye(n)).max() < 1e-13
    B = rng.normal(size=(m, nrhs)) + 1j * rng.normal(size=(m, nrhs))
    X = axi.svd_solve(At, V, sigma, torch.tensor(np.ascontiguousarray(B.T), device="cuda"), cutoff=1e-10)
    Xo, _ = OP.q_pinv_solve(A, B, 1e-10)
    assert np.abs(X.cpu().numpy().T - Xo).max() < 1e-9 * np.abs(Xo).max()


def test_svd_of_q_small_cell():
    """Q^+ for the small cell's periodizing rows: the GPU Jacobi SVD of the
    GPU-filled Q against numpy's SVD of the oracle's Q, and the truncated
    solve at a cutoff inside the spectrum's widest gap."""
    from paper_1506_05083_gb300 import axi
    wl, ob, coll = _case("small")
    d = np.array([0.36, -0.28, np.sqrt(1 - 0.36**2 - 0.28**2)])
    op = axi.Operator([axi.spec_from_obstacle(wl.obstacles[0])], prec=axi.PREC_FP64)
    cell = axi.Cell(ob.k * d[0], ob.k * d[1], 2.0, 1.7, 1.5, 6, 3, 12)
    Qg = op.q_matrix(cell)                                            # [cols][rows]
    Qo, _ = OP.q_matrix(ob.k, 12, ob.k * d[0], ob.k * d[1], 2.0, 1.7, 1.5, 6, 3)
    so = np.linalg.svd(Qo, compute_uv=False)
    V, sigma, sweeps = axi.svd_jacobi(Qg)
    torch.cuda.synchronize()
    sg = np.sort(sigma.cpu().numpy())[::-1]
    assert np.abs(sg - so).max() < 1e-11 * so[0]
    lo, hi = np.searchsorted(-so, -1e-6 * so[0]), np.searchsorted(-so, -1e-12 * so[0])
    gap = lo + int(np.argmax(so[lo:hi - 1] / so[lo + 1:hi]))
    cutoff = np.sqrt(so[gap] * so[gap + 1]) / so[0]
    rng = np.random.default_rng(6)
    B = rng.normal(size=(Qo.shape[0], 2)) + 1j * rng.normal(size=(Qo.shape[0], 2))
    X = axi.svd_solve(Qg, V, sigma, torch.tensor(np.ascontiguousarray(B.T), device="cuda"), cutoff=cutoff)
    Xo, _ = OP.q_pinv_solve(Qo, B, cutoff)
    assert np.abs(X.cpu().numpy().T - Xo).max() < 1e-8 * np.abs(Xo).max()
