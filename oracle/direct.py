"""Direct solves for any SPD operator (oracle).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

* ``bura_sparse``: u_r = sum_j c_j (A - d_j I)^{-1} f (eq. (Rgeneral), Sec. 2.2),
  each shifted system solved by a sparse LU factorisation (SuperLU).
* ``fractional_dense`` / ``bura_dense``: A = W D W^T by a dense symmetric
  eigendecomposition (eq. (exacalg), Sec. 1.1), for tiny matrices only.
* ``bura_nested_dense``: the same u_r written as r(A) A^{-1} f with r = P/Q in the
  monomial form of eq. (eq1bua), evaluated as Q(A)^{-1} P(A) A^{-1} f; agrees
  with the partial-fraction form exactly in exact arithmetic (eq. (simplified)).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

__all__ = ["bura_sparse", "shifted_solves_sparse", "fractional_dense", "bura_dense", "bura_nested_dense"]


def shifted_solves_sparse(A, f, d):
    """v_j = (A - d_j I)^{-1} f for every d_j, by sparse LU; shape (len(d), N)."""
    A = sp.csc_matrix(A)
    I = sp.identity(A.shape[0], format="csc")
    out = []
    for dj in d:
        lu = spla.splu((A - float(dj) * I).tocsc())
        out.append(lu.solve(np.asarray(f, dtype=np.float64)))
    return np.stack(out)


def bura_sparse(A, f, c, d):
    v = shifted_solves_sparse(A, f, d)
    return sum(float(cj) * vj for cj, vj in zip(c, v))


def fractional_dense(A, f, alpha):
    lam, W = sla.eigh(np.asarray(A.todense() if sp.issparse(A) else A))
    return W @ (lam ** (-float(alpha)) * (W.T @ f))


def bura_dense(A, f, c, d):
    lam, W = sla.eigh(np.asarray(A.todense() if sp.issparse(A) else A))
    phi = sum(float(cj) / (lam - float(dj)) for cj, dj in zip(c, d))
    return W @ (phi * (W.T @ f))


def bura_nested_dense(A, f, p, q):
    """Q(A)^{-1} P(A) A^{-1} f with P, Q given by monomial coefficients (ascending)."""
    M = np.asarray(A.todense() if sp.issparse(A) else A, dtype=np.float64)
    n = M.shape[0]

    def poly(coef):
        out = np.zeros((n, n))
        for cval in reversed([float(x) for x in coef]):  # Horner
            out = out @ M + cval * np.eye(n)
        return out

    F = np.linalg.solve(M, f)
    return np.linalg.solve(poly(q), poly(p) @ F)
