"""Pins of the oracle's same-method CPU solve (oracle/pcg.py, oracle/cpu_pcg.c): one multigrid-
preconditioned CG per shifted system, u = sum_j c_j (A - d_j I)^{-1} f (eq. (Rgeneral), Sec. 2.2).

It is pinned to the other oracle paths, which rest on independent arithmetic: sparse LU of every shifted
system (variable coefficients), the DST eigenbasis (eq. (exacalg), constant coefficients) and a dense
eigendecomposition for the spectral bounds.  A wrong stencil weight, shift sign or face index changes
the converged answer and fails these; the preconditioner itself only changes the iteration counts.
"""
import numpy as np
import pytest

from oracle import direct, exact, operators, pcg, tables
from paper_1612_04846_gb300 import workloads as W


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("shape,blocks", [((15, 15, 15), 2), ((7, 5, 3), 2), ((33, 17), 4), ((31, 31), 8)])
def test_variable_coefficients_match_sparse_direct(shape, blocks):
    """Variable coefficients (no closed form): PCG to 1e-13 equals k+1 sparse LU solves to 1e-10."""
    e = tables.entry(0.5, 5)
    faces = W.block_lognormal_faces(shape, blocks, 1e-2, 1.0, 7)
    A, _ = operators.scaled_matrix(shape, faces)
    f = W.rhs_normal(shape, 3)
    u, V, its = pcg.bura_pcg(shape, f, e["c"], e["d"], faces, components=True)
    assert _rel(u, direct.bura_sparse(A, f, e["c"], e["d"])) < 1e-10
    ref = direct.shifted_solves_sparse(A, f, e["d"])
    for j in range(len(e["d"])):
        assert _rel(V[j], ref[j]) < 1e-10, j
    assert all(i > 0 for i in its)


@pytest.mark.parametrize("shape", [(31, 31), (9, 6), (7, 7, 7), (64, 64)])
def test_constant_coefficients_match_the_sine_transform(shape):
    """Constant coefficients: PCG equals the exact BURA value of the DST eigenbasis (1e-10), including
    a grid that does not coarsen (9 x 6: one level, dense coarse solve) and 64^2 (Jacobi coarse sweeps)."""
    e = tables.entry(0.25, 7)
    f = W.rhs_uniform(shape, 4)
    u, its = pcg.bura_pcg(shape, f, e["c"], e["d"])
    assert _rel(u, exact.bura_value(shape, f, e["c"], e["d"])) < 1e-10


@pytest.mark.parametrize("shape,var", [((31, 31), False), ((15, 9, 7), True), ((33, 17), True), ((1, 1), False)])
def test_gershgorin_and_lower_bound(shape, var):
    """Lambda from the faces equals the assembled matrix's max row sum; lambda_low is below lambda_min
    of the scaled matrix (dense eigenvalues) and equals it for constant coefficients."""
    faces = W.block_lognormal_faces(shape, 2, 1e-2, 1.0, 9) if var else None
    A, lam = operators.scaled_matrix(shape, faces)
    assert pcg.gershgorin(shape, faces) == pytest.approx(lam, rel=1e-14)
    lmin = float(np.linalg.eigvalsh(A.toarray())[0])
    lo = pcg.lambda_low(shape, faces)
    assert lo <= lmin * (1 + 1e-12)
    if not var:
        assert lo == pytest.approx(lmin, rel=1e-10)


def test_solve_tolerances_meet_the_target():
    """With the per-system targets the partial-fraction value is within tol ||f|| of the exact one, and
    the targets split the budget: sum_j c_j rtol_j / (lambda_lo - d_j) = tol when none is capped at 1."""
    shape, tol = (63, 63), 1e-6
    e = tables.entry(0.75, 7)
    f = W.rhs_uniform(shape, 5)
    rt = pcg.solve_tolerances(shape, e["c"], e["d"], tol)
    lo = pcg.lambda_low(shape)
    assert sum(cj * r / (lo - dj) for cj, dj, r in zip(e["c"], e["d"], rt)) == pytest.approx(tol, rel=1e-12)
    u, _ = pcg.bura_pcg(shape, f, e["c"], e["d"], rtol=rt)
    ur = exact.bura_value(shape, f, e["c"], e["d"])
    assert np.linalg.norm(u - ur) <= tol * np.linalg.norm(f)


def test_threads_do_not_change_the_answer():
    shape = (31, 31, 31)
    e = tables.entry(0.5, 5)
    faces = W.block_lognormal_faces(shape, 4, 1e-2, 1.0, 2)
    f = W.rhs_normal(shape, 6)
    u1, it1 = pcg.bura_pcg(shape, f, e["c"], e["d"], faces, threads=1)
    u4, it4 = pcg.bura_pcg(shape, f, e["c"], e["d"], faces, threads=4)
    assert it1 == it4 and _rel(u4, u1) < 1e-12
