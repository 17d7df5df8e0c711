"""Host-side checks of the C ABI (no GPU): the library loads, exports every
declared entry point, and its host logic (geometry, quadrature rule,
validation) agrees with the oracle and rejects bad input."""
import json
import math
import os
import re

import numpy as np
import pytest

import oracle as O
import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def axi():
    from paper_1506_05083_gb300 import axi as A, build
    if not os.path.exists(A.LIB_PATH):
        build.build()
    A.lib()
    return A


def test_exports_every_declared_symbol(axi):
    hdr = open(os.path.join(ROOT, "include", "axi_mfs.h")).read()
    declared = set(re.findall(r"^(?:axi_status|const char \*|size_t)\s*(axi_\w+)\(", hdr, re.M))
    assert len(declared) >= 15
    L = axi.lib()
    for name in declared:
        assert hasattr(L, name), name
    bound = {s[0] for s in axi.SIGNATURES}
    assert declared == bound


@pytest.mark.parametrize("make", [synth.config_sphere, synth.config_smooth, synth.config_cup,
                                  synth.small_case])
def test_geometry_matches_oracle(axi, make):
    ob = make().obstacles[0]
    c1, s1, x1 = axi.geometry(ob.shape, ob.params, ob.M, ob.N, ob.tau)
    c2, s2, x2 = O.geometry(ob)
    assert np.abs(c1 - c2).max() < 1e-14
    assert np.abs(s1 - s2).max() < 1e-14
    assert np.abs(x1 - x2).max() < 1e-14
    assert axi.choose_q(ob.M, ob.N, ob.P, c1, s1) == O.choose_q(ob, c2, s2)


def test_batched_geometry_and_q(axi):
    for ob in synth.config_batched().obstacles:
        c1, s1, x1 = axi.geometry(ob.shape, ob.params, ob.M, ob.N, ob.tau)
        c2, s2, x2 = O.geometry(ob)
        assert np.abs(c1 - c2).max() < 1e-14 and np.abs(x1 - x2).max() < 1e-14
        q1 = axi.choose_q(ob.M, ob.N, ob.P, c1, s1, x1 if ob.bc else None)
        assert q1 == O.choose_q(ob, c2, s2, x2)


@pytest.mark.parametrize("make", [synth.small_case, synth.config_smooth])
def test_fill_subgrid_rule(axi, make):
    """Per-pair sub-grids of the fill (Theorem 1 per ring pair): strides in
    {1, 2, 4} that divide q/2 and keep q/s >= P; pairs with a faster rate
    never get a finer grid; and, checked independently with the oracle's own
    samples, every pair's (q/s)-node trapezoid rule agrees with the q-node
    rule for all modes to 1e-14 of max|A| (the accuracy q was chosen for)."""
    ob = make().obstacles[0]
    coll, src, srcx = O.geometry(ob)
    q = ob.q or O.choose_q(ob, coll, src, srcx)
    s = axi.fill_subgrid(ob.M, ob.N, ob.P, q, coll, src).astype(int)
    assert set(np.unique(s)) <= {1, 2, 4}
    assert np.all((q // 2) % s == 0) and np.all(q // s >= ob.P)
    alpha = O.theorem1_rate(coll[:, 0:1], coll[:, 1:2], src[None, :, 0], src[None, :, 1])
    order = np.argsort(alpha, axis=None)
    assert np.all(np.diff(s.reshape(-1)[order]) >= 0)
    D = ob.P // 2 + 1
    A = O.fill(ob.k, coll, src, q, ob.P, True)
    l = np.arange(q)
    E = np.exp(-2j * math.pi * np.outer(l, np.arange(D)) / q) / q
    err = 0.0
    for m0 in range(0, ob.M, 16):
        g = O.ring_samples(ob.k, coll[m0:m0 + 16], src, q, True)
        sg = s[m0:m0 + 16][:, :, None]
        gs = np.where(l[None, None, :] % sg == 0, g * sg, 0)
        err = max(err, np.abs(np.moveaxis(gs @ E, 2, 0) - A[:, m0:m0 + 16]).max())
    assert err < 1e-14 * np.abs(A).max(), err
    if make is synth.config_smooth:
        assert (s > 1).mean() > 0.5          # most pairs sample on a sub-grid


def _plan(axi, **kw):
    import ctypes as C
    ob = synth.small_case().obstacles[0]
    coll, src, srcx = axi.geometry(ob.shape, ob.params, ob.M, ob.N, ob.tau)
    args = dict(bc=0, M=ob.M, N=ob.N, P=ob.P, q=64, k=ob.k, k_minus=0.0, coll=coll, src=src,
                src_ext=None, prec=0)
    args.update(kw)
    prec = args.pop("prec")
    s = axi.ObstacleSpec(**args)
    arr = (axi._Obstacle * 1)()
    arr[0] = axi._Obstacle(s.bc, s.M, s.N, s.P, s.q, s.k, s.k_minus, axi._ptr(s.coll),
                           axi._ptr(s.src), axi._ptr(s.src_ext) if s.src_ext is not None else None)
    plan = C.c_void_p()
    code = axi.lib().axi_plan_create(arr, 1, prec, C.byref(plan))
    if code == 0:
        nb = C.c_size_t()
        assert axi.lib().axi_plan_workspace_bytes(plan, C.byref(nb)) == 0 and nb.value > 0
        axi.lib().axi_plan_destroy(plan)
    return code


def test_plan_validation(axi):
    assert _plan(axi) == 0
    assert _plan(axi, P=15) == -2                  # P odd
    assert _plan(axi, q=10) == -2                  # q < P
    assert _plan(axi, M=10) == -2                  # M < N
    assert _plan(axi, bc=1) == -1                  # transmission without exterior proxies
    assert _plan(axi, k=-1.0) == -1
    ob = synth.small_case().obstacles[0]
    coll, src, _ = axi.geometry(ob.shape, ob.params, ob.M, ob.N, ob.tau)
    bad = src.copy(); bad[3, 0] = -0.1
    assert _plan(axi, src=bad) == -3               # proxy across the axis
    nan = coll.copy(); nan[2, 1] = float("nan")
    assert _plan(axi, coll=nan) == -3
    assert _plan(axi, prec=7) == -1
    assert _plan(axi, prec=axi.PLAN_FULL_FILL_GRID) == 0
    assert _plan(axi, prec=axi.PREC_SPLIT_BF16 | axi.PLAN_FULL_FILL_GRID) == 0


def test_status_strings(axi):
    for c in range(-8, 1):
        assert axi.lib().axi_status_string(c)


def test_plan_tuning_json(axi):
    """Schedule tuning round-trips as JSON; malformed input and values out of
    range are refused without changing the plan."""
    import ctypes as C
    ob = synth.small_case().obstacles[0]
    coll, src, _ = axi.geometry(ob.shape, ob.params, ob.M, ob.N, ob.tau)
    arr = (axi._Obstacle * 1)()
    arr[0] = axi._Obstacle(0, ob.M, ob.N, ob.P, 64, ob.k, 0.0, axi._ptr(coll), axi._ptr(src), None)
    plan = C.c_void_p()
    L = axi.lib()
    assert L.axi_plan_create(arr, 1, axi.PREC_SPLIT_BF16, C.byref(plan)) == 0
    buf = C.create_string_buffer(256)
    try:
        assert L.axi_plan_get_tuning(plan, buf, 256) == 0
        assert json.loads(buf.value.decode()) == {"next_update": 0, "panel_cluster": 0, "rest_grid": 0,
                                                  "panel_threads": 0, "crit_stream": 0, "fill_chunk_mb": 0,
                                                  "next_cluster": 0, "panel_fixed": 0, "rest_start": 0, "apply_cluster": 0}
        assert L.axi_plan_set_tuning(plan, b'{"panel_cluster": 2, "rest_grid": 1, "other": 7}') == 0
        assert L.axi_plan_get_tuning(plan, buf, 256) == 0
        assert json.loads(buf.value.decode()) == {"next_update": 0, "panel_cluster": 2, "rest_grid": 1,
                                                  "panel_threads": 0, "crit_stream": 0, "fill_chunk_mb": 0,
                                                  "next_cluster": 0, "panel_fixed": 0, "rest_start": 0, "apply_cluster": 0}
        for bad in (b'{"panel_cluster": 3}', b'{"rest_grid": 5}', b'{"crit_stream": 2}', b'{"fill_chunk_mb": -1}', b'{"apply_cluster": 3}', b'{"next_cluster": 3}', b'{"rest_start": 2}', b'{"panel_fixed": 3}', b'{"panel_threads": 64}', b'{"next_update": 5}', b'panel_cluster: 1', b'{"rest_grid" 1}'):
            assert L.axi_plan_set_tuning(plan, bad) == -1
        assert json.loads(buf.value.decode())["panel_cluster"] == 2
        assert L.axi_plan_get_tuning(plan, buf, 8) == -1          # buffer too small
    finally:
        L.axi_plan_destroy(plan)


def test_q_shape_and_modes_host():
    """The periodizing rows' host logic (no GPU): the Rayleigh-Bloch set and
    its order equal the oracle's enumeration, the shape follows, and
    out-of-range cells are refused."""
    from paper_1506_05083_gb300 import axi
    from oracle import periodizing as OP
    period = 13 * 2 * math.pi / 25.0
    for (kx, ky, ex, ey, z0, m1, n0, p) in ((1.0, -0.8, 2.0, 1.7, 1.5, 6, 3, 12),
                                            (25 * 0.36, -25 * 0.28, period, period, 2.0, 32, 11, 48),
                                            (0.0, 0.0, 1.0, 3.0, 0.7, 2, 0, 0)):
        cell = axi.Cell(kx, ky, ex, ey, z0, m1, n0, p)
        modes = OP.rb_modes(kx, ky, ex, ey, n0)
        assert np.array_equal(axi.q_modes(cell), modes)
        assert axi.q_shape(cell) == (8 * m1 * m1, (p + 1) ** 2 + 2 * len(modes), len(modes))
    for bad in (axi.Cell(0, 0, 1, 1, 1, 7, 3, 4), axi.Cell(0, 0, 1, 1, 1, 66, 3, 4),
                axi.Cell(0, 0, -1, 1, 1, 6, 3, 4), axi.Cell(0, 0, 1, 1, 1, 6, 3, 256)):
        with pytest.raises(axi.AxiError):
            axi.q_shape(bad)


def test_svd_arguments_refused_on_host():
    """axi_svd_jacobi and axi_svd_solve check their arguments before any
    device work: null pointers, m < n, short leading dimensions, a zero
    sweep budget and misaligned buffers are AXI_ERR_ARG (-1) without a GPU."""
    import ctypes as C
    from paper_1506_05083_gb300 import axi
    L = axi.lib()
    p16 = C.c_void_p(1 << 20)                     # aligned stand-ins, never dereferenced
    sw = C.c_int32()
    assert L.axi_svd_jacobi(None, 8, 4, 8, p16, 4, p16, 1e-15, 10, C.byref(sw), None) == -1
    assert L.axi_svd_jacobi(p16, 3, 4, 8, p16, 4, p16, 1e-15, 10, C.byref(sw), None) == -1   # m < n
    assert L.axi_svd_jacobi(p16, 8, 4, 7, p16, 4, p16, 1e-15, 10, C.byref(sw), None) == -1   # lda < m
    assert L.axi_svd_jacobi(p16, 8, 4, 8, p16, 3, p16, 1e-15, 10, C.byref(sw), None) == -1   # ldv < n
    assert L.axi_svd_jacobi(p16, 8, 4, 8, p16, 4, p16, 1e-15, 0, C.byref(sw), None) == -1    # no sweeps
    assert L.axi_svd_jacobi(C.c_void_p((1 << 20) + 8), 8, 4, 8, p16, 4, p16, 1e-15, 10,
                            C.byref(sw), None) == -1                                        # misaligned
    assert L.axi_svd_solve(p16, p16, p16, 8, 4, 8, 4, 1e-10, p16, 8, 0, p16, 4, p16, None) == -1
    assert L.axi_svd_solve(p16, p16, p16, 8, 4, 8, 4, 1e-10, p16, 7, 1, p16, 4, p16, None) == -1


def test_iter_entries_refused_on_host():
    """The dense C eta product and the eq. iter combine check their arguments
    before any device work (AXI_ERR_ARG = -1, AXI_ERR_WORKSPACE = -4), and the
    product's workspace size is host arithmetic: the cup's C (8192 x 64800)
    with 16 vectors takes 19 column slices of 8192 x 16 partial sums."""
    import ctypes as C
    from paper_1506_05083_gb300 import axi
    L = axi.lib()
    nb = C.c_size_t()
    assert L.axi_matvec_workspace_bytes(8192, 64800, 16, C.byref(nb)) == 0
    assert nb.value == 19 * 16 * 8192 * 16
    assert L.axi_matvec_workspace_bytes(300, 50, 4, C.byref(nb)) == 0 and nb.value == 0
    assert L.axi_matvec_workspace_bytes(300, 50, 17, C.byref(nb)) == -1
    assert L.axi_matvec_workspace_bytes(0, 50, 1, C.byref(nb)) == -1
    p16 = C.c_void_p(1 << 20)                     # aligned stand-ins, never dereferenced
    bad = C.c_void_p((1 << 20) + 8)
    mv = L.axi_matvec_c128
    assert mv(None, 8, 8, 4, p16, 4, 1, p16, 8, None, 0, None) == -1
    assert mv(p16, 7, 8, 4, p16, 4, 1, p16, 8, None, 0, None) == -1            # lda < rows
    assert mv(p16, 8, 8, 4, p16, 3, 1, p16, 8, None, 0, None) == -1            # ldx < cols
    assert mv(p16, 8, 8, 4, p16, 4, 0, p16, 8, None, 0, None) == -1            # no vectors
    assert mv(p16, 8, 8, 4, p16, 4, 17, p16, 8, None, 0, None) == -1           # too many
    assert mv(bad, 8, 8, 4, p16, 4, 1, p16, 8, None, 0, None) == -1            # misaligned
    assert mv(p16, 300, 300, 1000, p16, 1000, 3, p16, 300, None, 0, None) == -4  # no workspace
    cb = L.axi_iter_combine
    # packed B~ of rows 40, P 16, p 8: modes 0..8 of widths 9..1 -> 45 columns
    assert cb(2, 40, 16, 8, p16, p16, p16, 45 * 40 - 1, p16, 81, p16, None) == -1   # short B~
    assert cb(2, 40, 16, 8, p16, p16, p16, 45 * 40, p16, 80, p16, None) == -1       # ldd < 81
    assert cb(2, 40, 1537, 8, p16, p16, p16, 1 << 30, p16, 81, p16, None) == -1     # P too large
    assert cb(2, 40, 16, 256, p16, p16, p16, 1 << 30, p16, 257 * 257, p16, None) == -1   # p > 255
    assert cb(2, 40, 16, 8, bad, p16, p16, 45 * 40, p16, 81, p16, None) == -1       # misaligned g
    assert cb(2, 40, 16, 8, p16, p16, None, 45 * 40, p16, 81, p16, None) == -1      # no B~


def test_noalloc_arguments_refused_on_host():
    """axi_apply_operator_noalloc refuses a null operator, null buffers and an
    empty batch (AXI_ERR_ARG = -1) before it asks CUDA for the current
    device; the device check itself (an operator built on another GPU than
    the current one, or a stream of another device) needs two GPUs."""
    import ctypes as C
    from paper_1506_05083_gb300 import axi
    L = axi.lib()
    p16 = C.c_void_p(1 << 20)                     # stand-ins, never dereferenced
    fn = L.axi_apply_operator_noalloc
    assert fn(None, 0, 1, p16, p16, None, None) == -1
    assert fn(p16, 0, 1, None, p16, None, None) == -1
    assert fn(p16, 0, 1, p16, None, None, None) == -1
    assert fn(p16, 0, 0, p16, p16, None, None) == -1


def test_gmres_host_state_without_a_gpu():
    """The GMRES driver's host side needs no device: the workspace size is
    (restart + 1) basis blocks, one more block and small scalars per wave
    (256-byte aligned pieces); create refuses a short or misaligned buffer
    (AXI_ERR_WORKSPACE = -4) and bad arguments (-1); a fresh state reports
    no steps, residual 1 and not converged; destroy releases it. The
    vector scaling refuses null or misaligned buffers and does nothing for
    an empty count."""
    import ctypes as C
    from paper_1506_05083_gb300 import axi
    L = axi.lib()
    nb = C.c_size_t()
    n, W, m = 1000, 3, 8
    assert L.axi_gmres_workspace_bytes(n, W, m, C.byref(nb)) == 0
    a256 = lambda b: (b + 255) // 256 * 256                                  # noqa: E731
    vec = 16 * n * W
    assert nb.value == a256(vec * (m + 1)) + a256(vec) + 2 * a256(16 * W * (m + 1)) + a256(8 * W)
    assert L.axi_gmres_workspace_bytes(n, W, 0, C.byref(nb)) == -1
    assert L.axi_gmres_workspace_bytes(n, 0, m, C.byref(nb)) == -1
    L.axi_gmres_workspace_bytes(n, W, m, C.byref(nb))
    base = C.c_void_p(1 << 24)                    # aligned stand-in, never dereferenced here
    g = C.c_void_p()
    assert L.axi_gmres_create(n, W, m, 100, 1e-12, base, nb.value - 1, C.byref(g)) == -4
    assert L.axi_gmres_create(n, W, m, 100, 1e-12, C.c_void_p((1 << 24) + 16), nb.value, C.byref(g)) == -4
    assert L.axi_gmres_create(n, W, m, 0, 1e-12, base, nb.value, C.byref(g)) == -1
    assert L.axi_gmres_create(n, W, m, 100, -1.0, base, nb.value, C.byref(g)) == -1
    assert L.axi_gmres_create(n, W, m, 100, 1e-12, base, nb.value, C.byref(g)) == 0 and g.value
    its, rel, conv = (C.c_int32 * W)(), (C.c_double * W)(), (C.c_int32 * W)()
    assert L.axi_gmres_result(g, its, rel, conv) == 0
    assert list(its) == [0] * W and list(rel) == [1.0] * W and list(conv) == [0] * W
    need, din, dout = C.c_int32(), C.c_void_p(), C.c_void_p()
    assert L.axi_gmres_iterate(g, None, base, C.byref(need), C.byref(din), C.byref(dout), None) == -1
    assert L.axi_gmres_destroy(g) == 0
    assert L.axi_vec_scale(4, 2.0, None, None) == -1
    assert L.axi_vec_scale(4, 2.0, C.c_void_p((1 << 20) + 8), None) == -1
    assert L.axi_vec_scale(0, 2.0, C.c_void_p(1 << 20), None) == 0
