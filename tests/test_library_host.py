"""CPU checks of the C-ABI library: it loads, exports every declared entry point, validates
arguments on the host, and its host-side rational approximation matches the oracle."""
import os
import re

import numpy as np
import pytest

from oracle import tables

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1612_04846_gb300 import build_lib, bura
    build_lib.build(verbose=False)
    return bura


def _declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(bura_[a-z_0-9]+)\s*\(", txt))
    return names


def test_library_exports_every_declared_symbol(lib):
    import ctypes
    L = ctypes.CDLL(lib.LIB_PATH)
    declared = _declared_symbols()
    assert {"bura_setup", "bura_solve", "bura_destroy", "bura_rational"} <= declared
    for name in sorted(declared):
        assert hasattr(L, name), name
    assert set(lib.EXPORTED) >= declared


def test_default_options_and_strerror(lib):
    o = lib.bura_default_options()
    assert o.precision == lib.BURA_PREC_MIXED and o.smoother_degree == 2 and o.max_iters > 0
    for code in range(0, -9, -1):
        assert lib.bura_strerror(code) != "unknown status"
    assert lib.bura_strerror(-99) == "unknown status"


@pytest.mark.parametrize("shape,alpha,k", [((0, 5), 0.5, 5), ((5, 5), 0.0, 5), ((5, 5), 1.0, 5),
                                           ((5, 5), 0.5, 0), ((5, 5), 0.5, 13), ((5, 5, 5, 5), 0.5, 5)])
def test_setup_rejects_bad_arguments_on_the_host(lib, shape, alpha, k):
    with pytest.raises(lib.BuraError) as ei:
        lib.bura_setup(shape, alpha, k)
    assert ei.value.code == lib.BURA_EINVAL


@pytest.mark.parametrize("field,value", [("coarse_kernel", -1), ("coarse_kernel", 5), ("cluster_size", 3),
                                         ("cluster_size", 32), ("smoother_degree", 0), ("inner_rtol", 1.0),
                                         ("unscaled", 2), ("unscaled", -1), ("tma_wait_cycles", -1)])
def test_setup_rejects_bad_options_on_the_host(lib, field, value):
    o = lib.bura_default_options()
    assert o.coarse_kernel == lib.BURA_COARSE_AUTO and o.cluster_size == 0
    setattr(o, field, value)
    with pytest.raises(lib.BuraError) as ei:
        lib.bura_setup((31, 31), 0.5, 5, options=o)
    assert ei.value.code == lib.BURA_EINVAL


def test_batch_arguments_on_the_host(lib):
    """bura_solve_batch: an empty batch is a no-op; null arrays and a negative count are rejected before
    any CUDA call."""
    import ctypes as C
    assert lib.bura_solve_batch([], [], [], 1e-6) == []
    L = lib._lib()
    st = (C.c_int * 1)()
    assert L.bura_solve_batch(None, None, None, 1, 1e-6, 1, st) == lib.BURA_EINVAL
    assert L.bura_solve_batch(None, None, None, -1, 1e-6, 1, st) == lib.BURA_EINVAL
    P = C.c_void_p
    nulls = (P * 1)()
    assert L.bura_solve_batch(nulls, nulls, nulls, 1, 1e-6, 1, st) == lib.BURA_EINVAL


def test_server_and_retarget_arguments_on_the_host(lib):
    """Defaults of the solve server and the argument checks that return before any CUDA call."""
    import ctypes as C
    o = lib.bura_server_default_options()
    assert o.workers == 8 and o.mem_budget == 0
    assert o.plan.precision == lib.BURA_PREC_MIXED and o.plan.smoother_degree == 2
    L = lib._lib()
    srv = C.c_void_p()
    assert L.bura_server_create(C.byref(o), None) == lib.BURA_EINVAL
    o.workers = -1
    assert L.bura_server_create(C.byref(o), C.byref(srv)) == lib.BURA_EINVAL
    req = lib.bura_request()
    rid = C.c_ulonglong()
    assert L.bura_server_submit(None, C.byref(req), C.byref(rid)) == lib.BURA_EINVAL
    info = lib.bura_request_info()
    assert L.bura_server_wait(None, 1, 0.0, C.byref(info)) == lib.BURA_EINVAL
    st = lib.bura_server_stats()
    assert L.bura_server_get_stats(None, C.byref(st)) == lib.BURA_EINVAL
    assert L.bura_server_destroy(None) == lib.BURA_OK
    assert L.bura_retarget(None, 0.5) == lib.BURA_EINVAL
    nulls = (C.c_void_p * 2)()
    assert L.bura_solve_chain(nulls, 2, None, None, 1e-6, None) == lib.BURA_EINVAL
    assert L.bura_solve_chain(nulls, 0, None, None, 1e-6, None) == lib.BURA_EINVAL


def test_setup_rejects_nonpositive_coefficients(lib):
    from paper_1612_04846_gb300 import workloads as W
    faces = list(W.constant_faces((4, 5)))
    faces[0] = faces[0].copy()
    faces[0][1, 2] = 0.0
    with pytest.raises(lib.BuraError) as ei:
        lib.bura_setup((5, 4), 0.5, 3, faces=faces)
    assert ei.value.code == lib.BURA_EINVAL


def test_setup_rejects_oversized_grid(lib):
    with pytest.raises(lib.BuraError) as ei:
        lib.bura_setup((2048, 2048, 64), 0.5, 5)
    assert ei.value.code == lib.BURA_ERANGE


@pytest.mark.parametrize("alpha,k", [(a, k) for a in (0.1, 0.25, 0.5, 0.75, 0.9) for k in (1, 3, 5, 7, 9, 10)])
def test_library_rational_matches_oracle(lib, alpha, k):
    """The library's double-precision Remez (factored form + Newton) reproduces the oracle's
    multi-precision Algorithm 1.  What the solve uses is the function r(t) = t sum_j c_j/(t - d_j)
    on the spectrum: it must agree with the oracle's to 2e-15 absolute on [0, 1].  The coefficients
    themselves are ill-conditioned functions of r (a change of r by one rounding unit moves them by
    about eps/E relative), so they are compared to 1e-11 + 4e-17/E relative."""
    try:
        ref = tables.entry(alpha, k)
    except KeyError:
        pytest.skip("no oracle table entry")
    c, d, E = lib.bura_rational(alpha, k)
    assert abs(E - ref["E"]) <= 1e-11 * ref["E"] + 2e-16
    assert d[0] == 0.0
    rtol = 1e-11 + 4e-17 / ref["E"]
    for a, b in zip(c, ref["c"]):
        assert abs(a - b) <= rtol * abs(b)
    for a, b in zip(d[1:], ref["d"][1:]):
        assert abs(a - b) <= rtol * abs(b)
    t = np.concatenate([np.logspace(-40, 0, 2000), np.linspace(0.001, 1, 1000)])

    def r(cc, dd):
        return t * sum(cj / (t - dj) for cj, dj in zip(cc, dd))

    assert np.max(np.abs(r(c, d) - r(ref["c"], ref["d"]))) <= 2e-15


@pytest.mark.parametrize("alpha", [0.37, 0.13])
def test_library_rational_off_the_warm_start_grid_matches_live_oracle(lib, alpha):
    """alpha off the library's warm-start grid (multiples of 0.05) goes through the continuation from the
    nearest grid state; r(t) must still agree with the oracle's multi-precision Algorithm 1 (run live)
    to 2e-15 on [0, 1]."""
    pytest.importorskip("mpmath")
    from oracle.remez import bura
    k = 5
    ref = bura(alpha, k).floats()
    c, d, E = lib.bura_rational(alpha, k)
    assert abs(E - ref["E"]) <= 1e-11 * ref["E"]
    t = np.concatenate([np.logspace(-40, 0, 2000), np.linspace(0.001, 1, 1000)])

    def r(cc, dd):
        return t * sum(cj / (t - dj) for cj, dj in zip(cc, dd))

    assert np.max(np.abs(r(c, d) - r(ref["c"], ref["d"]))) <= 2e-15


def test_library_rational_edge_alphas(lib):
    """Outside the tabulated alphas: positivity, ordering, c_0 = E and the Stahl asymptotics."""
    import math
    for alpha in (0.02, 0.05, 0.95, 0.98):
        for k in (1, 6, 12):
            c, d, E = lib.bura_rational(alpha, k)
            assert np.all(c > 0) and d[0] == 0 and np.all(np.diff(d) < 0)
            assert abs(c[0] - E) <= 1e-12 * E
            if k >= 6:
                g = 1 - alpha
                stahl = 4 ** (1 + g) * math.sin(math.pi * g) * math.exp(-2 * math.pi * math.sqrt(g * k))
                assert 0.6 < stahl / E < 1.8, (alpha, k, stahl, E)


def test_library_rational_rejects_bad_input(lib):
    for a, k in ((0.0, 5), (1.0, 5), (0.5, 0), (0.5, 13)):
        with pytest.raises(lib.BuraError) as ei:
            lib.bura_rational(a, k)
        assert ei.value.code == lib.BURA_EINVAL


@pytest.mark.parametrize("c,d,code", [([1.0, 0.0], [0.0, -1.0], "EINVAL"), ([1.0, 1.0], [0.0, 0.5], "EINVAL"),
                                      ([1.0, float("nan")], [0.0, -1.0], "EINVAL"), ([], [], "EINVAL"),
                                      ([1.0] * 14, [-1.0] * 14, "ERANGE")])
def test_setup_shifts_rejects_bad_weights_and_shifts_on_the_host(lib, c, d, code):
    """bura_setup_shifts (the partial-fraction form of a quadrature, eq. (BonitoPasciak)): positive weights,
    non-positive shifts and at most BURA_MAX_K + 1 systems, checked before any CUDA call."""
    with pytest.raises(lib.BuraError) as ei:
        lib.bura_setup_shifts((31, 31), c, d)
    assert ei.value.code == getattr(lib, "BURA_" + code)


def test_setup_shifts_rejects_the_unscaled_option(lib):
    o = lib.bura_default_options()
    o.unscaled = 1
    with pytest.raises(lib.BuraError) as ei:
        lib.bura_setup_shifts((31, 31), [1.0], [-0.5], options=o)
    assert ei.value.code == lib.BURA_EINVAL


def test_sum_and_wait_budget_arguments_on_the_host(lib):
    import ctypes as C
    L = lib._lib()
    P = C.c_void_p
    nulls = (P * 1)()
    assert L.bura_solve_sum(None, 1, None, None, 1e-6, None) == lib.BURA_EINVAL
    assert L.bura_solve_sum(nulls, 0, None, None, 1e-6, None) == lib.BURA_EINVAL
    assert L.bura_solve_sum(nulls, 1, P(16), P(32), 1e-6, None) == lib.BURA_EINVAL  # a null plan
    assert L.bura_set_tma_wait_cycles(None, 100) == lib.BURA_EINVAL


@pytest.mark.parametrize("shape,var", [((31, 31), False), ((1023, 1023), False), ((7, 5, 3), False),
                                       ((15, 9, 7), True), ((33, 17), True)])
def test_scale_matches_the_oracle_gershgorin_bound(lib, shape, var):
    """bura_scale: Lambda of eq. (algebraic) equals the oracle's max absolute row sum of Atilde."""
    from oracle import operators
    from paper_1612_04846_gb300 import workloads as W
    nps = tuple(reversed(shape))
    faces = W.block_lognormal_faces(nps, 2, 1e-2, 1.0, 3) if var else None
    _, lam = operators.scaled_matrix(nps, faces)
    assert lib.bura_scale(shape, faces) == pytest.approx(lam, rel=1e-14)


@pytest.mark.parametrize("alpha,kp", [(0.25, 0.5), (0.5, 1.0 / 3.0), (0.75, 0.7), (0.5, 1.0)])
def test_bp15_nodes_match_the_oracle(lib, alpha, kp):
    """bura_quadrature_bp15 gives the oracle's weights and shifts of eq. (BonitoPasciak) (1e-14), in the
    same order l = -m..M, and reports the node count when the capacity is short."""
    from oracle import quadrature
    lam = 8.0 * 1024 ** 2
    c, d = lib.bura_quadrature_bp15(alpha, kp, lam)
    co, do = quadrature.bp15_shifts(alpha, kp, lam)
    assert len(c) == len(co)
    np.testing.assert_allclose(c, co, rtol=1e-14)
    np.testing.assert_allclose(d, do, rtol=1e-14)
    import ctypes as C
    n = C.c_int()
    buf = np.zeros(2)
    rc = lib._lib().bura_quadrature_bp15(alpha, kp, lam, 2, lib._hptr(buf), lib._hptr(buf.copy()), C.byref(n))
    assert rc == lib.BURA_ERANGE and n.value == len(co)


def _csr(A):
    return A.indptr, A.indices, A.data


@pytest.mark.parametrize("case", ["unsymmetric", "no_diagonal", "negative_diagonal", "bad_column", "nan",
                                  "bad_offsets", "negative_lambda_min"])
def test_setup_csr_rejects_bad_matrices_on_the_host(lib, case):
    """bura_setup_csr checks the structure (offsets, columns, finite values, a positive diagonal in every
    row) and the symmetry of the matrix before any CUDA call."""
    import scipy.sparse as sp
    from oracle import operators
    A = operators.fd_matrix((5, 4)).tocsr().astype(np.float64)
    A.sort_indices()
    rp, ci, va = A.indptr.copy(), A.indices.copy(), A.data.copy()
    lam = 0.0
    if case == "unsymmetric":
        va[1] *= 2.0
    elif case == "no_diagonal":
        B = A.tolil()
        B[3, 3] = 0.0
        B = B.tocsr()
        B.eliminate_zeros()
        rp, ci, va = B.indptr, B.indices, B.data
    elif case == "negative_diagonal":
        va[np.where(ci[: rp[1]] == 0)[0][0]] = -1.0
    elif case == "bad_column":
        ci = ci.copy()
        ci[-1] = 99
    elif case == "nan":
        va[0] = float("nan")
    elif case == "bad_offsets":
        rp = rp.copy()
        rp[-1] += 1
    elif case == "negative_lambda_min":
        lam = -1.0
    with pytest.raises(lib.BuraError) as ei:
        lib.bura_setup_csr(rp, ci, va, 0.5, 5, lambda_min=lam)
    assert ei.value.code == lib.BURA_EINVAL


@pytest.mark.parametrize("case", ["3d", "faces", "csr"])
def test_fdiag_coarse_kernel_rejected_off_2d_constant_grids_on_the_host(lib, case):
    """BURA_COARSE_FDIAG (the exact sine-eigenbasis solve of a coarse level) exists for 2-D constant-
    coefficient grids only: 3-D grids, face coefficients and sparse matrices are rejected before any
    CUDA call."""
    o = lib.bura_default_options()
    o.coarse_kernel = lib.BURA_COARSE_FDIAG
    with pytest.raises(lib.BuraError) as ei:
        if case == "3d":
            lib.bura_setup((7, 7, 7), 0.5, 5, options=o)
        elif case == "faces":
            from paper_1612_04846_gb300 import workloads as W
            lib.bura_setup((7, 7), 0.5, 5, faces=W.block_lognormal_faces((7, 7), 2, 0.1, 1.0, 1), options=o)
        else:
            from oracle import operators
            A = operators.fd_matrix((5, 4)).tocsr().astype(np.float64)
            A.sort_indices()
            lib.bura_setup_csr(A.indptr, A.indices, A.data, 0.5, 5, options=o)
    assert ei.value.code == lib.BURA_EINVAL
