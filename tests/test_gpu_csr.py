"""GPU parity of the sparse (CSR) operator kind against the oracle's sparse LU.

The matrices: the oracle's 5-point finite-difference matrix, the stiffness matrix of P1 finite elements
on a tetrahedral mesh of the unit cube with the paper's half-cube coefficient jump (Sec. 5.4), and a
randomly perturbed SPD matrix with an irregular sparsity pattern.  The library receives the unscaled
matrices and scales them itself (eq. (algebraic)); the oracle's reference is
u_r = sum_j c_j (A - d_j I)^{-1} f by sparse LU of every shifted system (eq. (Rgeneral)).
Tolerances: operator apply 1e-14 (FP64), FP64 solve 1e-10, mixed solve tol, all relative l2.
"""
import numpy as np
import pytest
import scipy.sparse as sp

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


def _random_spd(n, seed):
    """A symmetric matrix with a random pattern (about 9 entries per row), made SPD by a dominant diagonal."""
    rng = np.random.default_rng(seed)
    m = 4 * n
    r = rng.integers(0, n, m)
    c = rng.integers(0, n, m)
    v = -rng.uniform(0.1, 1.0, m)
    R = sp.coo_matrix((v, (r, c)), shape=(n, n)).tocsr()
    R = R + R.T
    R.setdiag(0.0)
    R.eliminate_zeros()
    d = np.asarray(abs(R).sum(axis=1)).ravel() + rng.uniform(0.05, 0.5, n)
    return (R + sp.diags(d)).tocsr()


def _matrix(kind):
    if kind == "fd2d":
        return operators.fd_matrix((31, 31)).tocsr()
    if kind == "p1_halfcube":
        return W.p1_matrix(15, W.half_cube_field(1e-3)).tocsr()
    return _random_spd(2000, 7)


def _lmin(A):
    return float(np.linalg.eigvalsh(A.toarray())[0])


@pytest.mark.parametrize("kind", ["fd2d", "p1_halfcube", "random"])
def test_csr_apply_shifted_matches_the_matrix(lib, kind):
    """y_j = (A - d_j I) x_j (FP64, A = Atilde / Lambda) against scipy's product (1e-14)."""
    At = _matrix(kind)
    As, lam = operators.scaled_csr(At)
    k = 5
    o = lib.bura_default_options()
    o.precision = lib.BURA_PREC_FP64
    plan = lib.bura_setup_csr(At.indptr, At.indices, At.data, 0.5, k, options=o)
    try:
        assert lib.bura_get_stats(plan)["Lambda"] == pytest.approx(lam, rel=1e-14)
        c, d, _ = lib.bura_get_rational(plan, k)
        X = np.random.default_rng(3).standard_normal((k + 1, At.shape[0]))
        Y = torch.zeros((k + 1, At.shape[0]), dtype=torch.float64, device="cuda")
        lib.bura_apply_shifted(plan, torch.from_numpy(X).cuda(), Y)
        Y = Y.cpu().numpy()
        for j in range(k + 1):
            ref = As @ X[j] - d[j] * X[j]
            assert _rel(Y[j], ref) < 1e-14, j
    finally:
        lib.bura_destroy(plan)


@pytest.mark.parametrize("precision,tol,bound", [(0, 1e-11, 1e-10), (1, 1e-6, 1e-6)])
@pytest.mark.parametrize("kind,alpha,k", [("fd2d", 0.5, 7), ("p1_halfcube", 0.25, 5), ("random", 0.75, 6)])
def test_csr_solve_matches_sparse_direct(lib, precision, tol, bound, kind, alpha, k):
    """The BURA solve with the sparse operator (lambda_min given, so the solver's error bound applies)
    against sparse LU of every shifted system."""
    At = _matrix(kind)
    As, lam = operators.scaled_csr(At)
    o = lib.bura_default_options()
    o.precision = precision
    plan = lib.bura_setup_csr(At.indptr, At.indices, At.data, alpha, k, lambda_min=_lmin(At), options=o)
    try:
        f = W.rhs_uniform((At.shape[0],), 11)
        fd = torch.from_numpy(f).cuda()
        ud = torch.zeros_like(fd)
        assert lib.bura_solve(plan, fd, ud, tol) == lib.BURA_OK
        torch.cuda.synchronize()
        st = lib.bura_get_stats(plan)
    finally:
        lib.bura_destroy(plan)
    e = tables.entry(alpha, k)
    ur = direct.bura_sparse(As, f, e["c"], e["d"])
    assert _rel(ud.cpu().numpy(), ur) <= bound
    assert 0 <= st["err_bound"] <= tol


def test_csr_relative_residual_rule_without_lambda_min(lib):
    """Without a lambda_min bound every system stops at ||r_j|| <= tol ||f||: the residuals of the
    computed systems meet it (checked with the oracle's matrix), and err_bound reports -1."""
    At = _matrix("p1_halfcube")
    As, _ = operators.scaled_csr(At)
    k, tol = 5, 1e-8
    o = lib.bura_default_options()
    o.precision = lib.BURA_PREC_FP64
    plan = lib.bura_setup_csr(At.indptr, At.indices, At.data, 0.5, k, options=o)
    try:
        f = W.rhs_normal((At.shape[0],), 12)
        fd = torch.from_numpy(f).cuda()
        V = torch.zeros((k + 1, f.size), dtype=torch.float64, device="cuda")
        assert lib.bura_solve_systems(plan, fd, V, tol) == lib.BURA_OK
        torch.cuda.synchronize()
        c, d, _ = lib.bura_get_rational(plan, k)
        st = lib.bura_get_stats(plan)
        V = V.cpu().numpy()
    finally:
        lib.bura_destroy(plan)
    for j in range(k + 1):
        assert np.linalg.norm(f - (As @ V[j] - d[j] * V[j])) <= tol * np.linalg.norm(f) * (1 + 1e-6)
    assert st["err_bound"] == -1.0


def test_csr_p1_finite_elements_full_bound_at_63(lib):
    """P1 finite elements on 63^3 interior vertices with the half-cube jump mu = 1e-3 (Sec. 5.4), mixed
    precision, tol 1e-6: lambda_min >= mu h^3 lambda_min(7-point FD) (the stiffness is h^3 times the FD
    matrix for a = 1 and the quadratic form is monotone in a), and the oracle's sparse matrix checks the
    rigorous bound sum_j c_j ||r_j|| / (lambda_lo - d_j) <= tol ||f||."""
    n, mu, alpha, k, tol = 63, 1e-3, 0.5, 7, 1e-6
    At = W.p1_matrix(n, W.half_cube_field(mu)).tocsr()
    As, lam = operators.scaled_csr(At)
    h = 1.0 / (n + 1)
    lmin = mu * h ** 3 * float(exact.eigenvalues((n, n, n)).min()) * exact.gershgorin((n, n, n))
    plan = lib.bura_setup_csr(At.indptr, At.indices, At.data, alpha, k, lambda_min=lmin)
    try:
        f = W.rhs_normal((At.shape[0],), 13)
        fd = torch.from_numpy(f).cuda()
        V = torch.zeros((k + 1, f.size), dtype=torch.float64, device="cuda")
        assert lib.bura_solve_systems(plan, fd, V, tol) == lib.BURA_OK
        ud = torch.zeros_like(fd)
        assert lib.bura_solve(plan, fd, ud, tol) == lib.BURA_OK
        torch.cuda.synchronize()
        c, d, _ = lib.bura_get_rational(plan, k)
        V = V.cpu().numpy()
        u = ud.cpu().numpy()
    finally:
        lib.bura_destroy(plan)
    lam_lo = lmin / lam
    bound = sum(c[j] * np.linalg.norm(f - (As @ V[j] - d[j] * V[j])) / (lam_lo - d[j]) for j in range(k + 1))
    assert bound <= tol * np.linalg.norm(f)
    assert _rel(u, sum(c[j] * V[j] for j in range(k + 1))) <= 1e-12
