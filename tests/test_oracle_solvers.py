"""Pins of the oracle's operators and exact solvers (CPU only)."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import direct, exact, operators, tables
from paper_1612_04846_gb300 import workloads as W


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("shape", [(1, 1), (2, 3), (5, 4), (7, 7), (3, 4, 5), (2, 2, 2)])
def test_constant_operator_spectrum_is_closed_form(shape):
    """The assembled scaled 5-/7-point matrix has the separable sine spectrum (Sec. 5.1, 5.3)
    and lies in (0, 1] (Assumption aa1)."""
    A, Lam = operators.scaled_matrix(shape)
    assert Lam == pytest.approx(exact.gershgorin(shape), rel=1e-15)
    ev = np.sort(np.linalg.eigvalsh(A.toarray()))
    assert np.max(np.abs(ev - np.sort(exact.eigenvalues(shape).ravel()))) < 1e-14
    assert ev[0] > 0 and ev[-1] <= 1 + 1e-15


def test_2d_operator_is_the_papers_kronecker_form():
    """Sec. 5.3: Atilde = h^-2 tridiag(-I, tridiag(-1,4,-1), -I) and A = h^2 Atilde / 8 for n >= 3."""
    n = 6
    h = 1.0 / (n + 1)
    T = sp.diags([-1, 4, -1], [-1, 0, 1], shape=(n, n))
    I = sp.identity(n)
    off = sp.diags([1, 1], [-1, 1], shape=(n, n))
    At = (sp.kron(I, T) - sp.kron(off, I)) / h ** 2
    A, Lam = operators.scaled_matrix((n, n))
    assert Lam == pytest.approx(8 / h ** 2)
    assert abs(A - At * h ** 2 / 8).max() < 1e-14


def test_variable_operator_quadratic_form_and_symmetry():
    """x^T Atilde x = sum over faces a_F (x_P - x_Q)^2 / h^2 (with x = 0 on the boundary);
    the matrix is symmetric and reduces to the constant one for a = 1."""
    shape = (4, 5, 6)
    faces = W.block_lognormal_faces(shape, 2, 1e-2, 1.0, 7)
    At = operators.fd_matrix(shape, faces)
    assert abs(At - At.T).max() == 0
    rng = np.random.default_rng(0)
    for _ in range(3):
        x = rng.standard_normal(At.shape[0])
        assert x @ (At @ x) == pytest.approx(operators.quadratic_form(shape, faces, x), rel=1e-13)
    assert abs(operators.fd_matrix(shape, W.constant_faces(shape)) - operators.fd_matrix(shape)).max() == 0


def test_block_faces_are_constant_inside_blocks():
    """Faces inside one coefficient block share its value (block boundaries at x = b/blocks)."""
    shape = (15, 15, 15)  # h = 1/16, blocks of 4 cells
    ax, ay, az = W.block_lognormal_faces(shape, 4, 1e-2, 1.0, 2)
    assert len(np.unique(ax)) <= 64 and len(np.unique(az)) <= 64
    assert ax.min() >= 1e-2 and ax.max() <= 1.0


@pytest.mark.parametrize("shape", [(5, 4), (3, 4, 5), (6, 6)])
def test_dst_fractional_matches_dense_eigh(shape):
    """eq. (exacalg): the DST eigenbasis and a dense eigendecomposition give the same A^-alpha f."""
    A, _ = operators.scaled_matrix(shape)
    f = W.rhs_uniform(shape, 1)
    for alpha in (0.25, 0.5, 0.75):
        assert _rel(exact.fractional(shape, f, alpha), direct.fractional_dense(A, f, alpha)) < 1e-13


@pytest.mark.parametrize("shape", [(31, 31), (7, 7, 7), (9, 6)])
def test_dst_bura_matches_sparse_direct(shape):
    """eq. (Rgeneral): sum_j c_j (A - d_j I)^{-1} f by DST equals k+1 sparse LU solves."""
    e = tables.entry(0.5, 5)
    A, _ = operators.scaled_matrix(shape)
    f = W.rhs_uniform(shape, 2)
    assert _rel(exact.bura_value(shape, f, e["c"], e["d"]), direct.bura_sparse(A, f, e["c"], e["d"])) < 1e-12


@pytest.mark.parametrize("alpha,k", [(0.25, 5), (0.5, 5), (0.75, 5), (0.5, 7)])
def test_partial_fractions_equal_nested_form(alpha, k):
    """eq. (simplified): t^{-1} P(t)/Q(t) = sum c_j/(t - d_j), so Q(A)^{-1} P(A) A^{-1} f equals the
    partial-fraction sum (both forms of the BURA solution, on a tiny dense matrix)."""
    e = tables.entry(alpha, k)
    shape = (3, 4)
    A, _ = operators.scaled_matrix(shape)
    f = W.rhs_uniform(shape, 3)
    u_pf = direct.bura_dense(A, f, e["c"], e["d"])
    u_nested = direct.bura_nested_dense(A, f, e["p"], e["q"])
    assert _rel(u_pf, u_nested) < 1e-9


@pytest.mark.parametrize("alpha,k", [(0.25, 7), (0.5, 5), (0.75, 7)])
def test_bura_error_bound_lemma(alpha, k):
    """Lemma l:BURAerror with gamma = 1, beta = 1: ||u_r - u||_A <= E ||f||_{A^{-1}}, and per mode
    (u_r - u)_i = (r(lambda_i) - lambda_i^{1-alpha}) / lambda_i * f_i in the eigenbasis."""
    e = tables.entry(alpha, k)
    shape = (63, 63)
    f = W.rhs_uniform(shape, 4)
    A, _ = operators.scaled_matrix(shape)
    u = exact.fractional(shape, f, alpha)
    ur = exact.bura_value(shape, f, e["c"], e["d"])
    diff = ur - u
    lhs = np.sqrt(diff @ (A @ diff))
    finv = exact.apply_function(shape, f, lambda lam: 1.0 / lam)
    rhs = e["E"] * np.sqrt(f @ finv)
    assert lhs <= rhs * (1 + 1e-10)
    assert lhs >= 0.05 * rhs  # the bound is not vacuous for white-noise f


def test_positive_coefficients_keep_the_sum_stable():
    """Remark rm:aaa: with c_j > 0 and d_j <= 0 the partial-fraction value at eigenvalue lambda
    is a sum of positive terms; on the scaled 2D spectrum it stays within E/lambda of lambda^-alpha."""
    e = tables.entry(0.5, 7)
    lam = np.sort(exact.eigenvalues((127, 127)).ravel())
    terms = np.stack([cj / (lam - dj) for cj, dj in zip(e["c"], e["d"])])
    assert np.all(terms > 0)
    val = terms.sum(axis=0)
    assert np.all(np.abs(val - lam ** -0.5) <= e["E"] / lam * (1 + 1e-12))


@pytest.mark.parametrize("shape", [(31, 31), (7, 7, 7), (9, 6)])
def test_dst_components_match_sparse_direct(shape):
    """eq. (Rgeneral), eq. (exacalg): every component v_j = (A - d_j I)^{-1} f of the DST eigenbasis
    equals the sparse LU solve of that shifted system, and sum_j c_j v_j is the exact BURA value.
    A slip in one shift (a sign of d_j, a dropped system) fails the per-component check."""
    e = tables.entry(0.5, 7)
    A, _ = operators.scaled_matrix(shape)
    f = W.rhs_uniform(shape, 5)
    comp = exact.bura_components(shape, f, e["d"])
    ref = direct.shifted_solves_sparse(A, f, e["d"])
    assert comp.shape == ref.shape == (len(e["d"]), int(np.prod(shape)))
    for j in range(len(e["d"])):
        assert _rel(comp[j], ref[j]) < 1e-12, j
    total = sum(float(cj) * vj for cj, vj in zip(e["c"], comp))
    assert _rel(total, exact.bura_value(shape, f, e["c"], e["d"])) < 1e-13


@pytest.mark.parametrize("n", [3, 7])
def test_p1_constant_coefficient_is_the_7_point_matrix(n):
    """P1 finite elements on the tetrahedra around each cube's main diagonal (Sec. 5.4's element type):
    with a = 1 the stiffness matrix is h^3 times the 7-point finite-difference matrix."""
    h = 1.0 / (n + 1)
    A = W.p1_matrix(n)
    assert abs(A - h ** 3 * operators.fd_matrix((n, n, n))).max() < 1e-15


def test_p1_variable_coefficient_is_spd_and_monotone():
    """With a piecewise-constant a (the paper's half cube scaled by mu): symmetric, an M-matrix (off-diagonal
    entries <= 0, row sums >= 0), and its quadratic form lies between mu and 1 times the a = 1 form."""
    n, mu = 7, 1e-3
    A = W.p1_matrix(n, W.half_cube_field(mu))
    A1 = W.p1_matrix(n)
    assert abs(A - A.T).max() == 0
    B = A.tocoo()
    assert np.all(B.data[B.row != B.col] <= 0)
    assert np.all(np.asarray(A.sum(axis=1)).ravel() >= -1e-15)
    rng = np.random.default_rng(1)
    for _ in range(3):
        x = rng.standard_normal(n ** 3)
        q, q1 = x @ (A @ x), x @ (A1 @ x)
        assert mu * q1 * (1 - 1e-12) <= q <= q1 * (1 + 1e-12)
