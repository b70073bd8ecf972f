"""GPU parity of the CUDA path (through the C ABI) against the oracle.

Tolerances (written out per test):
  * operator apply (FP64): 1e-14 relative;
  * FP64 solve: ||u - u_r|| / ||u_r|| <= 1e-10 with u_r the exact BURA value of eq. (Rgeneral);
  * mixed FP32/FP64 solve at tol: ||u - u_r|| / ||u_r|| <= tol.
The library's stopping rule bounds ||u - u_r|| by tol * ||f|| and ||u_r|| >= (1 - E) ||f|| on these
operators (spec(A) in (0,1]), so the solve tolerance is the parity tolerance.
"""
import numpy as np
import pytest

from oracle import direct, exact, operators, tables
from paper_1612_04846_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)


@pytest.fixture(scope="module")
def lib():
    from paper_1612_04846_gb300 import build_lib, bura
    build_lib.build(verbose=False)
    return bura


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _opts(lib, precision, **kw):
    o = lib.bura_default_options()
    o.precision = precision
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def _np_shape(shape):
    return tuple(reversed(shape))  # (nx, ny[, nz]) -> numpy (.., ny, nx)


def _solve(lib, shape, alpha, k, f, tol, precision, faces=None, **kw):
    plan = lib.bura_setup(shape, alpha, k, faces=faces, options=_opts(lib, precision, **kw))
    try:
        fd = torch.from_numpy(f).cuda()
        ud = torch.zeros_like(fd)
        rc = lib.bura_solve(plan, fd, ud, tol)
        torch.cuda.synchronize()
        st = lib.bura_get_stats(plan)
        c, d, E = lib.bura_get_rational(plan, k)
        return ud.cpu().numpy(), st, rc, (c, d, E)
    finally:
        lib.bura_destroy(plan)


# ------------------------------------------------------------------ the multi-shift operator
@pytest.mark.parametrize("shape,var", [((31, 31), False), ((64, 64), False), ((17, 9), False), ((1, 1), False),
                                       ((7, 7, 7), False), ((15, 9, 7), False), ((15, 15, 15), True),
                                       ((33, 17), True), ((5, 1, 3), True)])
def test_apply_shifted_matches_sparse_operator(lib, shape, var):
    """y_j = (A - d_j I) x_j (FP64 kernel) equals the oracle's assembled scaled matrix (1e-14)."""
    k = 5
    nps = _np_shape(shape)
    faces = W.block_lognormal_faces(nps, 2, 1e-2, 1.0, 11) if var else None
    plan = lib.bura_setup(shape, 0.5, k, faces=faces, options=_opts(lib, lib.BURA_PREC_FP64))
    try:
        A, _ = operators.scaled_matrix(nps, faces)
        c, d, _ = lib.bura_get_rational(plan, k)
        N = A.shape[0]
        rng = np.random.default_rng(5)
        X = rng.standard_normal((k + 1, N))
        Y = torch.zeros((k + 1, N), dtype=torch.float64, device="cuda")
        lib.bura_apply_shifted(plan, torch.from_numpy(X).cuda(), Y)
        Y = Y.cpu().numpy()
        for j in range(k + 1):
            ref = A @ X[j] - d[j] * X[j]
            assert _rel(Y[j], ref) < 1e-14, j
    finally:
        lib.bura_destroy(plan)


# ------------------------------------------------------------------ FP64 path
@pytest.mark.parametrize("shape,alpha,k", [((64, 64), 0.5, 5), ((63, 63), 0.25, 7), ((127, 127), 0.75, 7),
                                           ((31, 31), 0.1, 9), ((33, 17), 0.9, 6), ((255, 255), 0.5, 8)])
def test_fp64_solve_matches_exact_bura_2d(lib, shape, alpha, k):
    nps = _np_shape(shape)
    f = W.rhs_uniform(nps, 0)
    u, st, rc, (c, d, E) = _solve(lib, shape, alpha, k, f, 1e-11, lib.BURA_PREC_FP64)
    assert rc == lib.BURA_OK
    ref = tables.entry(alpha, k)
    ur = exact.bura_value(nps, f, ref["c"], ref["d"])
    assert _rel(u, ur) <= 1e-10, (st, _rel(u, ur))
    assert st["err_bound"] <= 1e-11 * 1.0001


@pytest.mark.parametrize("shape", [(15, 15, 15), (31, 31, 31), (7, 15, 31)])
def test_fp64_solve_matches_exact_bura_3d(lib, shape):
    nps = _np_shape(shape)
    f = W.rhs_normal(nps, 3)
    u, st, rc, _ = _solve(lib, shape, 0.5, 9, f, 1e-11, lib.BURA_PREC_FP64)
    assert rc == lib.BURA_OK
    ref = tables.entry(0.5, 9)
    assert _rel(u, exact.bura_value(nps, f, ref["c"], ref["d"])) <= 1e-10


@pytest.mark.parametrize("shape,alpha,k", [((15, 15, 15), 0.5, 9), ((31, 15), 0.25, 5)])
def test_fp64_solve_variable_coefficients_matches_sparse_direct(lib, shape, alpha, k):
    nps = _np_shape(shape)
    faces = W.block_lognormal_faces(nps, 4, 1e-2, 1.0, 2)
    f = W.rhs_normal(nps, 4)
    u, st, rc, _ = _solve(lib, shape, alpha, k, f, 1e-11, lib.BURA_PREC_FP64, faces=faces)
    assert rc == lib.BURA_OK
    ref = tables.entry(alpha, k)
    A, _ = operators.scaled_matrix(nps, faces)
    assert _rel(u, direct.bura_sparse(A, f, ref["c"], ref["d"])) <= 1e-10


def test_fp64_each_system_matches(lib):
    """bura_solve_systems: every v_j = (A - d_j I)^{-1} f separately (FP64, 1e-9 relative each)."""
    shape, alpha, k = (63, 63), 0.5, 5
    nps = _np_shape(shape)
    f = W.rhs_uniform(nps, 9)
    plan = lib.bura_setup(shape, alpha, k, options=_opts(lib, lib.BURA_PREC_FP64))
    try:
        V = torch.zeros((k + 1, f.size), dtype=torch.float64, device="cuda")
        lib.bura_solve_systems(plan, torch.from_numpy(f).cuda(), V, 1e-11)
        V = V.cpu().numpy()
        c, d, _ = lib.bura_get_rational(plan, k)
        ref = exact.bura_components(nps, f, d)
        for j in range(k + 1):
            # ||e_j|| <= ||r_j|| / (lambda_lo - d_j) <= tol ||f|| / (K c_j) and ||v_j|| >= ||f|| / (1 - d_j)
            assert _rel(V[j], ref[j]) <= 1e-11 * (1 - d[j]) / ((k + 1) * c[j]) + 1e-12, j
    finally:
        lib.bura_destroy(plan)


@pytest.mark.parametrize("kind,csize", [("CLUSTER", 0), ("CLUSTER", 2), ("CLUSTER", 8), ("CTA", 0), ("NONE", 0)])
@pytest.mark.parametrize("shape,var", [((255, 255), False), ((31, 31, 31), True), ((127, 63), False)])
def test_fp64_solve_each_coarse_kernel(lib, kind, csize, shape, var):
    """The three ways of running the small levels (one thread-block cluster over L2-resident vectors,
    one CTA over shared memory, grid kernels down to the coarsest level) all converge to the BURA
    value; the profile names the coarse kernel that ran."""
    nps = _np_shape(shape)
    alpha, k = 0.5, 7
    faces = W.block_lognormal_faces(nps, 4, 1e-2, 1.0, 5) if var else None
    f = W.rhs_normal(nps, 6)
    o = _opts(lib, lib.BURA_PREC_FP64, coarse_kernel=getattr(lib, "BURA_COARSE_" + kind), cluster_size=csize)
    plan = lib.bura_setup(shape, alpha, k, faces=faces, options=o)
    try:
        lib.bura_set_profiling(plan, True)
        fd = torch.from_numpy(f).cuda()
        ud = torch.zeros_like(fd)
        assert lib.bura_solve(plan, fd, ud, 1e-11) == lib.BURA_OK
        torch.cuda.synchronize()
        names = {e["name"] for e in lib.bura_get_profile(plan)}
        u = ud.cpu().numpy()
    finally:
        lib.bura_destroy(plan)
    ref = tables.entry(alpha, k)
    if var:
        A, _ = operators.scaled_matrix(nps, faces)
        ur = direct.bura_sparse(A, f, ref["c"], ref["d"])
    else:
        ur = exact.bura_value(nps, f, ref["c"], ref["d"])
    assert _rel(u, ur) <= 1e-10
    has_cluster = any(n.startswith("coarse_cluster") for n in names)
    has_cta = any(n.startswith("coarse_cycle") for n in names)
    assert (has_cluster, has_cta) == (kind == "CLUSTER", kind == "CTA"), names


@pytest.mark.parametrize("shape,k", [((255, 255), 7), ((127, 63), 7), ((31, 31), 7), ((20, 13), 7), ((1, 1), 7),
                                     ((127, 127), 2), ((63, 31), 9)])
def test_fp64_solve_fdiag_coarse_kernel(lib, shape, k):
    """The exact coarse solve by fast diagonalization (the sine eigenbasis of the 5-point operator, per
    axis the eigenpairs of the three-point matrix of Sec. 4.1) converges to the BURA value at 1e-10.
    Where the whole grid is the exact level (31^2, the unrefinable 20 x 13, one point) the preconditioner
    is (A - d_j I)^{-1} itself, so every system converges in a single PCG iteration.  k = 2 and 9 (3 and 10
    systems) leave padding lanes in the 16-byte chunks of the FP64 layout."""
    nps = _np_shape(shape)
    alpha = 0.5
    f = W.rhs_normal(nps, 6)
    o = _opts(lib, lib.BURA_PREC_FP64, coarse_kernel=lib.BURA_COARSE_FDIAG)
    plan = lib.bura_setup(shape, alpha, k, options=o)
    try:
        lib.bura_set_profiling(plan, True)
        fd = torch.from_numpy(f).cuda()
        ud = torch.zeros_like(fd)
        assert lib.bura_solve(plan, fd, ud, 1e-11) == lib.BURA_OK
        torch.cuda.synchronize()
        names = {e["name"] for e in lib.bura_get_profile(plan)}
        st = lib.bura_get_stats(plan)
        u = ud.cpu().numpy()
    finally:
        lib.bura_destroy(plan)
    ref = tables.entry(alpha, k)
    assert _rel(u, exact.bura_value(nps, f, ref["c"], ref["d"])) <= 1e-10
    assert any(n.startswith("coarse_fdiag") for n in names), names
    if max(shape) <= 31:
        assert list(st["shift_iters"]) == [1] * (k + 1), st["shift_iters"]


@pytest.mark.parametrize("shape", [(63, 63), (50, 37), (127, 127), (1023, 1023)])
def test_mixed_solve_fdiag_coarse_kernel(lib, shape):
    """The FP32 fast-diagonalization coarse solve inside the mixed path (the default for 2-D constant
    coefficients) meets the solve tolerance against the exact BURA value; when the whole grid is the
    exact level (at most 63 points per axis in FP32) each inner solve needs at most two PCG iterations
    (FP32 rounding of the inverse)."""
    nps = _np_shape(shape)
    alpha, k, tol = 0.25, 7, 1e-6
    f = W.rhs_uniform(nps, 4)
    u, st, rc, (c, d, E) = _solve(lib, shape, alpha, k, f, tol, lib.BURA_PREC_MIXED,
                                  coarse_kernel=lib.BURA_COARSE_FDIAG)
    assert rc == lib.BURA_OK
    ref = tables.entry(alpha, k)
    assert _rel(u, exact.bura_value(nps, f, ref["c"], ref["d"])) <= tol
    if max(shape) <= 63:
        assert st["iters"] <= 2 * st["outer"], (st["iters"], st["outer"])


# ------------------------------------------------------------------ mixed path
@pytest.mark.parametrize("sweeps", ["AUTO", "GRID"])
@pytest.mark.parametrize("shape,alpha,k,tol", [((64, 64), 0.5, 5, 1e-6), ((127, 127), 0.25, 7, 1e-6),
                                               ((255, 255), 0.75, 7, 1e-6), ((127, 127), 0.5, 7, 1e-8),
                                               ((31, 31, 31), 0.5, 9, 1e-6), ((1023, 255), 0.5, 3, 1e-7),
                                               ((257, 1023), 0.25, 10, 1e-6), ((1023, 511), 0.5, 12, 1e-6)])
def test_mixed_solve_within_tolerance(lib, shape, alpha, k, tol, sweeps):
    """Mixed path with the TMA-staged tile sweeps (AUTO: FP32 2-D constant-coefficient levels with at
    least one 32x16 tile per SM; ragged last tiles on every shape here) and with grid-stride sweeps
    only.  k = 3, 7, 10, 12 give 4, 8, 12 and 16 FP32 values per point (1 to 4 chunks of 16 bytes)."""
    nps = _np_shape(shape)
    f = W.rhs_uniform(nps, 1)
    u, st, rc, _ = _solve(lib, shape, alpha, k, f, tol, lib.BURA_PREC_MIXED,
                          sweeps=getattr(lib, "BURA_SWEEP_" + sweeps))
    assert rc == lib.BURA_OK
    ref = tables.entry(alpha, k)
    err = _rel(u, exact.bura_value(nps, f, ref["c"], ref["d"]))
    assert err <= tol, (err, st)


@pytest.mark.parametrize("mode", [0, 2])
@pytest.mark.parametrize("shape,alpha,k", [((1023, 1023), 0.5, 7), ((255, 255), 0.25, 3), ((511, 255), 0.75, 10),
                                           ((127, 63), 0.5, 12), ((383, 129), 0.9, 7), ((1023, 255), 0.25, 1)])
def test_fused_post_smoothing_matches_two_sweeps(lib, shape, alpha, k, mode):
    """The prolongation and both post-smoothing steps as one sweep (mode 0: TMA tiles, the first step
    recomputed on a one-point halo of every tile; mode 2: y-marching strips of 124 columns, the vertical
    neighbours in registers) against the same as two sweeps.  Every point gets the same operations, but r.z is summed in another grouping, so its
    FP32 partial sums differ; beta reaches the kernels as an FP32 copy, which mostly absorbs that, not
    always.  A preconditioner fault would change the iteration counts or the iterates at the solve
    tolerance: both must agree, the solutions to 1e-8 (observed: bit-identical or within 1e-9), and both
    meet the oracle.  k = 1, 3, 7, 10, 12 give 4, 4, 8, 12 and 16 FP32 values per point (16 on 3-D tensor
    maps); every grid has ragged last tiles and strips."""
    nps = _np_shape(shape)
    f = W.rhs_uniform(nps, 5)
    tol = 1e-6
    u1, st1, rc1, _ = _solve(lib, shape, alpha, k, f, tol, lib.BURA_PREC_MIXED, post_smooth_split=mode)
    u2, st2, rc2, _ = _solve(lib, shape, alpha, k, f, tol, lib.BURA_PREC_MIXED, post_smooth_split=1)
    assert rc1 == lib.BURA_OK and rc2 == lib.BURA_OK
    assert st1["iters"] == st2["iters"] and st1["outer"] == st2["outer"]
    assert _rel(u1, u2) <= 1e-8
    ref = tables.entry(alpha, k)
    ur = exact.bura_value(nps, f, ref["c"], ref["d"])
    assert _rel(u1, ur) <= tol and _rel(u2, ur) <= tol


def test_mixed_variable_3d_within_tolerance(lib):
    shape = (31, 31, 31)
    nps = _np_shape(shape)
    faces = W.block_lognormal_faces(nps, 8, 1e-2, 1.0, 2)
    f = W.rhs_normal(nps, 3)
    u, st, rc, _ = _solve(lib, shape, 0.5, 9, f, 1e-6, lib.BURA_PREC_MIXED, faces=faces)
    assert rc == lib.BURA_OK
    ref = tables.entry(0.5, 9)
    A, _ = operators.scaled_matrix(nps, faces)
    assert _rel(u, direct.bura_sparse(A, f, ref["c"], ref["d"])) <= 1e-6


@pytest.mark.parametrize("shape,alpha,k,tol,var", [((127, 127), 0.25, 7, 1e-6, False), ((255, 255), 0.75, 7, 1e-6, False),
                                                   ((127, 127), 0.5, 7, 1e-9, False), ((31, 31, 31), 0.5, 9, 1e-6, True),
                                                   ((1023, 1023), 0.75, 7, 1e-6, False)])
def test_mixed_double_float_refinement(lib, shape, alpha, k, tol, var):
    """BURA_REFINE_DF: the refinement accumulator as FP32 pairs (about 48 bits), residual and weighted
    sum in double-float arithmetic.  Same tolerance as the FP64 refinement; bura_solve_systems reads
    the same pairs (each v_j against the exact (A - d_j I)^{-1} f for constant coefficients)."""
    nps = _np_shape(shape)
    faces = W.block_lognormal_faces(nps, 8, 1e-2, 1.0, 2) if var else None
    f = W.rhs_uniform(nps, 4)
    u, st, rc, _ = _solve(lib, shape, alpha, k, f, tol, lib.BURA_PREC_MIXED, faces=faces, refine=lib.BURA_REFINE_DF)
    assert rc == lib.BURA_OK
    ref = tables.entry(alpha, k)
    if var:
        A, _ = operators.scaled_matrix(nps, faces)
        ur = direct.bura_sparse(A, f, ref["c"], ref["d"])
    else:
        ur = exact.bura_value(nps, f, ref["c"], ref["d"])
    assert _rel(u, ur) <= tol, st
    if not var and shape[0] <= 255:
        plan = lib.bura_setup(shape, alpha, k, options=_opts(lib, lib.BURA_PREC_MIXED, refine=lib.BURA_REFINE_DF))
        try:
            V = torch.zeros((k + 1, f.size), dtype=torch.float64, device="cuda")
            assert lib.bura_solve_systems(plan, torch.from_numpy(f).cuda(), V, tol) == lib.BURA_OK
            V = V.cpu().numpy()
            c, d, _ = lib.bura_get_rational(plan, k)
        finally:
            lib.bura_destroy(plan)
        comp = exact.bura_components(nps, f, d)
        for j in range(k + 1):
            # ||e_j|| <= ||r_j|| / (lambda_lo - d_j) <= tol ||f|| / (K c_j), ||v_j|| >= ||f|| / (1 - d_j)
            assert _rel(V[j], comp[j]) <= tol * (1 - d[j]) / ((k + 1) * c[j]) + 1e-12, j


# ------------------------------------------------------------------ full size of the bench workload
@pytest.mark.parametrize("alpha", [0.25, 0.5, 0.75])
def test_full_size_1023_mixed_and_fp64(lib, alpha):
    """The bench workload (2D 1023^2, k = 7, f ~ U[-1,1] seed 1): every output against the exact
    BURA value from the sine transform, mixed at 1e-6 and FP64 at 1e-10."""
    shape, k = (1023, 1023), 7
    nps = _np_shape(shape)
    f = W.rhs_uniform(nps, 1)
    ref = tables.entry(alpha, k)
    ur = exact.bura_value(nps, f, ref["c"], ref["d"])
    u, st, rc, _ = _solve(lib, shape, alpha, k, f, 1e-6, lib.BURA_PREC_MIXED)
    assert rc == lib.BURA_OK and _rel(u, ur) <= 1e-6, st
    u, st, rc, _ = _solve(lib, shape, alpha, k, f, 1e-11, lib.BURA_PREC_FP64)
    assert rc == lib.BURA_OK and _rel(u, ur) <= 1e-10, st


# ------------------------------------------------------------------ method-level properties
def test_bura_error_bound_against_exact_fractional(lib):
    """Lemma l:BURAerror (gamma = 1): ||u - A^{-alpha} f||_A <= E ||f||_{A^{-1}} + solver error."""
    shape, alpha, k = (127, 127), 0.5, 6
    nps = _np_shape(shape)
    f = W.rhs_uniform(nps, 7)
    u, st, rc, (c, d, E) = _solve(lib, shape, alpha, k, f, 1e-10, lib.BURA_PREC_FP64)
    A, _ = operators.scaled_matrix(nps)
    diff = u - exact.fractional(nps, f, alpha)
    lhs = np.sqrt(diff @ (A @ diff))
    rhs = E * np.sqrt(f @ exact.apply_function(nps, f, lambda lam: 1.0 / lam))
    assert lhs <= rhs * (1 + 1e-6)


def test_host_entry_point_equals_device_entry_point(lib):
    shape, alpha, k = (127, 127), 0.5, 5
    nps = _np_shape(shape)
    f = W.rhs_uniform(nps, 2)
    plan = lib.bura_setup(shape, alpha, k, options=_opts(lib, lib.BURA_PREC_MIXED))
    try:
        uh = np.zeros_like(f)
        lib.bura_solve_host(plan, f, uh, 1e-6)
        fd = torch.from_numpy(f).cuda()
        ud = torch.zeros_like(fd)
        lib.bura_solve(plan, fd, ud, 1e-6)
        torch.cuda.synchronize()
        assert np.array_equal(uh, ud.cpu().numpy())  # deterministic reductions: bitwise equal
    finally:
        lib.bura_destroy(plan)


def test_zero_rhs_and_single_point(lib):
    for shape in ((1, 1), (2, 2), (1, 5, 1)):
        nps = _np_shape(shape)
        for prec in (lib.BURA_PREC_FP64, lib.BURA_PREC_MIXED):
            u, st, rc, _ = _solve(lib, shape, 0.5, 3, np.zeros(int(np.prod(shape))), 1e-8, prec)
            assert rc == lib.BURA_OK and np.all(u == 0)
            f = W.rhs_uniform(nps, 3)
            u, st, rc, _ = _solve(lib, shape, 0.5, 3, f, 1e-9, prec)
            ref = tables.entry(0.5, 3)
            A, _ = operators.scaled_matrix(nps)
            assert _rel(u, direct.bura_dense(A, f, ref["c"], ref["d"])) <= 1e-9


def test_iteration_cap_reports_enoconv(lib):
    shape = (127, 127)
    f = W.rhs_uniform(_np_shape(shape), 4)
    u, st, rc, _ = _solve(lib, shape, 0.5, 5, f, 1e-12, lib.BURA_PREC_FP64, max_iters=1)
    assert rc == lib.BURA_ENOCONV and st["iters"] == 1


def test_smallest_and_largest_tabulated_k(lib):
    shape = (63, 63)
    nps = _np_shape(shape)
    f = W.rhs_uniform(nps, 5)
    for k in (1, 10):
        u, st, rc, _ = _solve(lib, shape, 0.5, k, f, 1e-11, lib.BURA_PREC_FP64)
        ref = tables.entry(0.5, k)
        assert rc == lib.BURA_OK and _rel(u, exact.bura_value(nps, f, ref["c"], ref["d"])) <= 1e-10


def test_full_size_3d_variable_coefficients(lib):
    """The 3D workload (255^3 interior, 7-point -div(a grad u) with a log-uniform in [1e-2, 1] on 8^3
    blocks, alpha = 0.5, k = 9, f ~ N(0,1), mixed precision, tol 1e-6).  No closed form exists, so the
    oracle's own sparse operator checks every system's residual r_j = f - (A - d_j I) v_j, and the
    rigorous bound ||u - u_r|| <= sum_j c_j ||r_j|| / (lambda_lo - d_j) with lambda_lo = min(a) times the
    closed-form smallest eigenvalue of the constant-coefficient operator (the quadratic form of A is
    at least min(a) times that of the unit-coefficient operator, face by face) must be <= tol ||f||.
    u itself must equal sum_j c_j v_j."""
    shape, alpha, k, tol = (255, 255, 255), 0.5, 9, 1e-6
    nps = _np_shape(shape)
    faces = W.block_lognormal_faces(nps, 8, 1e-2, 1.0, 2)
    f = W.rhs_normal(nps, 3)
    plan = lib.bura_setup(shape, alpha, k, faces=faces, options=_opts(lib, lib.BURA_PREC_MIXED))
    try:
        fd = torch.from_numpy(f).cuda()
        V = torch.zeros((k + 1, f.size), dtype=torch.float64, device="cuda")
        assert lib.bura_solve_systems(plan, fd, V, tol) == lib.BURA_OK
        ud = torch.zeros_like(fd)
        assert lib.bura_solve(plan, fd, ud, tol) == lib.BURA_OK
        torch.cuda.synchronize()
        c, d, E = lib.bura_get_rational(plan, k)
        V = V.cpu().numpy()
        u = ud.cpu().numpy()
    finally:
        lib.bura_destroy(plan)
    A, _ = operators.scaled_matrix(nps, faces)
    amin = min(float(a.min()) for a in faces)
    lam_lo = amin * float(exact.eigenvalues(nps).min())
    fn = np.linalg.norm(f)
    bound = 0.0
    for j in range(k + 1):
        rj = f - (A @ V[j] - d[j] * V[j])
        bound += c[j] * np.linalg.norm(rj) / (lam_lo - d[j])
    assert bound <= tol * fn, bound / fn
    usum = sum(c[j] * V[j] for j in range(k + 1))
    assert _rel(u, usum) <= 1e-12


@pytest.mark.parametrize("n,k,var", [(127, k, v) for v in (False, True) for k in (3, 7, 9, 12)]
                         + [(255, 7, False), (255, 12, False), (255, 3, True)])
def test_staged_3d_sweeps_every_chunk_count(lib, n, k, var):
    """The 3-D FP32 sweeps staged in shared memory (the levels at least 127 points wide) for 1, 2, 3 and
    4 chunks of four systems a point (k = 3, 7, 9, 12), constant and variable coefficients, on 127^3: a
    16 x 8 x 128 work item leaves ragged tiles on every axis (127 = 7 * 16 + 15 = 15 * 8 + 7 < 128); on
    255^3 every column of tiles is two work items along z (128 + 127 planes), so the second item starts
    from the plane below it.  Constant coefficients: within tol of the exact BURA value (eq. (exacalg)).
    Variable coefficients (log-uniform in [1e-2, 1] on 8^3 blocks): the rigorous bound of every system's
    residual, computed with the oracle's sparse operator as in the 255^3 test, within tol ||f||."""
    shape, alpha, tol = (n, n, n), 0.5, 1e-6
    nps = _np_shape(shape)
    f = W.rhs_normal(nps, 11)
    ref = tables.entry(alpha, k)
    if not var:
        u, st, rc, _ = _solve(lib, shape, alpha, k, f, tol, lib.BURA_PREC_MIXED)
        assert rc == lib.BURA_OK
        assert _rel(u, exact.bura_value(nps, f, ref["c"], ref["d"])) <= tol, st
        return
    faces = W.block_lognormal_faces(nps, 8, 1e-2, 1.0, 2)
    plan = lib.bura_setup(shape, alpha, k, faces=faces, options=_opts(lib, lib.BURA_PREC_MIXED))
    try:
        fd = torch.from_numpy(f).cuda()
        V = torch.zeros((k + 1, f.size), dtype=torch.float64, device="cuda")
        assert lib.bura_solve_systems(plan, fd, V, tol) == lib.BURA_OK
        torch.cuda.synchronize()
        c, d, _ = lib.bura_get_rational(plan, k)
        V = V.cpu().numpy()
    finally:
        lib.bura_destroy(plan)
    A, _ = operators.scaled_matrix(nps, faces)
    lam_lo = min(float(a.min()) for a in faces) * float(exact.eigenvalues(nps).min())
    bound = sum(c[j] * np.linalg.norm(f - (A @ V[j] - d[j] * V[j])) / (lam_lo - d[j]) for j in range(k + 1))
    assert bound <= tol * np.linalg.norm(f), bound / np.linalg.norm(f)


@pytest.mark.parametrize("kind", ["CTA", "FDIAG"])
@pytest.mark.parametrize("precision,tol", [("MIXED", 1e-6), ("FP64", 1e-10)])
def test_plan_set_up_after_a_larger_coarse_cta_solves_both(lib, precision, tol, kind):
    """A coarse kernel's shared-memory limit belongs to the kernel, not to a plan: a plan set up later
    with a smaller coarse CTA (31^2: three levels, ~134 KB; or a smaller fast-diagonalization level) must
    not lower the limit under an earlier plan whose CTA holds its whole hierarchy (63x31: four levels,
    ~187 KB; or the 63x31 exact level).  Both plans are solved after both are set up, the larger first."""
    probs = [((63, 31), 0.25, 9), ((31, 31), 0.5, 5)]
    prec = getattr(lib, "BURA_PREC_" + precision)
    plans = []
    try:
        for shape, alpha, k in probs:
            o = _opts(lib, prec, coarse_kernel=getattr(lib, "BURA_COARSE_" + kind))
            plans.append(lib.bura_setup(shape, alpha, k, options=o))
        for i, (shape, alpha, k) in enumerate(probs):
            nps = _np_shape(shape)
            f = W.rhs_uniform(nps, 30 + i)
            fd = torch.from_numpy(f).cuda()
            ud = torch.zeros_like(fd)
            assert lib.bura_solve(plans[i], fd, ud, tol) == lib.BURA_OK
            torch.cuda.synchronize()
            ref = tables.entry(alpha, k)
            assert _rel(ud.cpu().numpy(), exact.bura_value(nps, f, ref["c"], ref["d"])) <= tol, shape
    finally:
        for p in plans:
            lib.bura_destroy(p)
