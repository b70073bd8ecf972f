"""Scaled finite-difference matrices A = Atilde / Lambda (oracle).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Atilde is the standard finite-difference matrix of -div(a grad u) on the
uniform interior grid of the unit square/cube with homogeneous Dirichlet data,
lexicographic ordering with x fastest (Sec. 5.3: for a = 1 in 2D this is
h^{-2} tridiag(-I, tridiag(-1,4,-1), -I)).  Lambda is the Gershgorin bound
max_i sum_j |Atilde_ij| >= lambda_max, so that the spectrum of A lies in (0,1]
(eq. (algebraic) and Assumption 1.1 "aa1", Sec. 1.2).

Face-coefficient convention (arrays in C order, x fastest):
  grid shape (nz, ny, nx) in 3D, (ny, nx) in 2D, with h_x = 1/(nx+1) etc.;
  ax has shape (..., nx+1): ax[..., i] is a on the x-face between interior
  nodes i-1 and i (i = 0 and i = nx are the faces to the boundary nodes);
  ay has shape (..., ny+1, nx), az has shape (nz+1, ny, nx) likewise.
  Row of node P:  (Atilde u)_P = sum over its faces F of a_F (u_P - u_nb(F)) / h_F^2,
  with u_nb = 0 on the boundary.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

__all__ = ["fd_matrix", "scaled_matrix", "constant_faces", "quadratic_form", "scaled_csr"]


def constant_faces(shape):
    """Face arrays of a == 1 for a grid of the given (.., ny, nx) shape."""
    shape = tuple(shape)
    d = len(shape)
    out = []
    for ax in range(d):  # ax = 0 is the slowest axis
        s = list(shape)
        s[ax] += 1
        out.append(np.ones(s))
    return tuple(reversed(out))  # (ax, ay[, az]) = faces normal to x, y, z


def fd_matrix(shape, faces=None):
    """Unscaled Atilde (CSR) for interior grid ``shape`` = (ny, nx) or (nz, ny, nx)."""
    shape = tuple(int(n) for n in shape)
    d = len(shape)
    if faces is None:
        faces = constant_faces(shape)
    N = int(np.prod(shape))
    idx = np.arange(N).reshape(shape)
    rows, cols, vals = [], [], []
    diag = np.zeros(shape)
    # faces[0] is normal to x (the last array axis), faces[1] to y, faces[2] to z
    for fdir in range(d):
        axis = d - 1 - fdir
        n = shape[axis]
        h2 = (1.0 / (n + 1)) ** 2
        a = np.asarray(faces[fdir], dtype=np.float64)
        exp_shape = list(shape)
        exp_shape[axis] += 1
        if a.shape != tuple(exp_shape):
            raise ValueError("face array %d has shape %s, expected %s" % (fdir, a.shape, tuple(exp_shape)))
        lo = np.take(a, np.arange(n), axis=axis)        # face between node i-1 and i
        hi = np.take(a, np.arange(1, n + 1), axis=axis)  # face between node i and i+1
        diag += (lo + hi) / h2
        # coupling between node i and i+1 through face i+1 (interior faces only)
        if n > 1:
            left = np.take(idx, np.arange(n - 1), axis=axis).ravel()
            right = np.take(idx, np.arange(1, n), axis=axis).ravel()
            w = np.take(a, np.arange(1, n), axis=axis).ravel() / h2
            rows += [left, right]
            cols += [right, left]
            vals += [-w, -w]
    rows.append(idx.ravel())
    cols.append(idx.ravel())
    vals.append(diag.ravel())
    A = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(N, N))
    A.sum_duplicates()
    return A


def scaled_matrix(shape, faces=None):
    """(A, Lambda) with A = Atilde / Lambda and Lambda = max absolute row sum of Atilde."""
    At = fd_matrix(shape, faces)
    Lam = float(np.max(np.asarray(abs(At).sum(axis=1)).ravel()))
    return (At / Lam).tocsr(), Lam


def quadratic_form(shape, faces, x):
    """x^T Atilde x written face by face: sum_F a_F (x_P - x_Q)^2 / h_F^2 (x = 0 outside)."""
    shape = tuple(shape)
    d = len(shape)
    x = np.asarray(x, dtype=np.float64).reshape(shape)
    total = 0.0
    for fdir in range(d):
        axis = d - 1 - fdir
        n = shape[axis]
        h2 = (1.0 / (n + 1)) ** 2
        pad = [(0, 0)] * d
        pad[axis] = (1, 1)
        xp = np.pad(x, pad)  # zero Dirichlet values on both sides
        diff = np.diff(xp, axis=axis)  # n+1 faces along this axis
        total += float(np.sum(np.asarray(faces[fdir]) * diff * diff)) / h2
    return total


def scaled_csr(A):
    """(A / Lambda, Lambda) for an assembled SPD matrix, Lambda its max absolute row sum (eq. (algebraic))."""
    Lam = float(np.max(np.asarray(abs(A).sum(axis=1)).ravel()))
    return (A / Lam).tocsr(), Lam
