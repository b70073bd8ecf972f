"""Seeded synthetic inputs shared by the tests, smoke() and bench.py.

This module holds input generation only: grids, right-hand sides and
face-coefficient fields.  It contains none of the solver's arithmetic and
imports nothing from the rest of the package, so both the CUDA path's tests
and the oracle can consume the same arrays.

Face-coefficient convention (x fastest, C order), as the C ABI documents:
  2D grid (ny, nx):     ax (ny, nx+1), ay (ny+1, nx)
  3D grid (nz, ny, nx): ax (nz, ny, nx+1), ay (nz, ny+1, nx), az (nz+1, ny, nx)
  ax[..., i] is the coefficient on the x-face between interior nodes i-1 and i.
"""
from __future__ import annotations

import itertools

import numpy as np
import scipy.sparse as sp

__all__ = ["rhs_uniform", "rhs_normal", "block_lognormal_faces", "constant_faces", "checkerboard_rhs", "p1_matrix",
           "half_cube_field"]


def rhs_uniform(shape, seed):
    """f i.i.d. uniform on [-1, 1] (PCG64 with the given seed), float64, flattened."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.uniform(-1.0, 1.0, size=int(np.prod(shape)))


def rhs_normal(shape, seed):
    """f i.i.d. N(0, 1) (PCG64 with the given seed), float64, flattened."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.standard_normal(size=int(np.prod(shape)))


def checkerboard_rhs(shape):
    """+1 where (x-1/2)(y-1/2) > 0 and -1 elsewhere on the interior nodes of a 2D grid."""
    ny, nx = shape
    x = np.arange(1, nx + 1) / (nx + 1)
    y = np.arange(1, ny + 1) / (ny + 1)
    s = (x[None, :] - 0.5) * (y[:, None] - 0.5)
    return np.where(s > 0, 1.0, -1.0).ravel()


def constant_faces(shape, value=1.0):
    shape = tuple(int(n) for n in shape)
    d = len(shape)
    out = []
    for fdir in range(d):
        axis = d - 1 - fdir
        s = list(shape)
        s[axis] += 1
        out.append(np.full(s, float(value)))
    return tuple(out)


def block_lognormal_faces(shape, blocks, lo, hi, seed):
    """Face coefficients of a(x) piecewise constant on blocks^d equal blocks of the unit
    cube/square, log-uniform in [lo, hi] (PCG64 seed).  Each face takes the value of a at
    its midpoint; the block of a coordinate x is min(floor(blocks * x), blocks - 1).
    """
    shape = tuple(int(n) for n in shape)
    d = len(shape)
    rng = np.random.Generator(np.random.PCG64(seed))
    field = np.exp(rng.uniform(np.log(lo), np.log(hi), size=(blocks,) * d))
    faces = []
    for fdir in range(d):
        axis = d - 1 - fdir
        coords = []
        for ax2, n in enumerate(shape):
            h = 1.0 / (n + 1)
            if ax2 == axis:
                xs = (np.arange(n + 1) + 0.5) * h  # face midpoints between nodes i-1 and i
            else:
                xs = (np.arange(n) + 1.0) * h      # node coordinates
            coords.append(np.minimum((xs * blocks).astype(np.int64), blocks - 1))
        mesh = np.meshgrid(*coords, indexing="ij")
        faces.append(field[tuple(mesh)])
    return tuple(faces)


# ---------------------------------------------------------------------- P1 finite-element matrices
# The assembled stiffness matrix is an input of the sparse solve (like the face coefficients of the grid
# operators): the matrix of the paper's 3-D tests, Sec. 5.4.
def _kuhn_element_matrices():
    """Stiffness matrices G G^T |T| of the six tetrahedra of the unit cube that share its main diagonal
    (vertices 0, e_a, e_a + e_b, (1,1,1) for every ordering (a, b, c) of the axes), for a = 1 and h = 1.
    G holds the gradients of the four barycentric functions: the rows of J^-1 and minus their sum."""
    mats, verts = [], []
    for perm in itertools.permutations(range(3)):
        v = np.zeros((4, 3))
        for m in range(1, 4):
            v[m] = v[m - 1]
            v[m, perm[m - 1]] = 1.0
        J = (v[1:] - v[0]).T  # columns: edge vectors from vertex 0, so x = v0 + J (l1, l2, l3)
        Ginv = np.linalg.inv(J)  # row m-1: gradient of the barycentric function of vertex m
        G = np.vstack([-Ginv.sum(axis=0), Ginv])
        vol = abs(np.linalg.det(J)) / 6.0
        mats.append(vol * G @ G.T)
        verts.append(v.astype(np.int64))
    return mats, verts


def p1_matrix(n, field=None):
    """Stiffness matrix (CSR) of continuous piecewise-linear finite elements for -div(a grad u) on the
    unit cube with homogeneous Dirichlet data (the operator of the paper's 3-D tests, Sec. 5.4, with the
    coefficient a = a(x) I piecewise constant).  Mesh: (n+1)^3 cubes of side h = 1/(n+1), each cut into
    the six tetrahedra around its main diagonal; unknowns are the n^3 interior vertices, numbered
    x fastest.  field: None (a = 1) or an array of shape (b, b, b) indexed [z, y, x] giving a on the b^3
    equal blocks of the cube; a tetrahedron takes the value of the block holding its centroid.
    With a = 1 this is h^3 times the 7-point finite-difference matrix."""
    n = int(n)
    h = 1.0 / (n + 1)
    mats, verts = _kuhn_element_matrices()
    c = np.arange(n + 1)
    cz, cy, cx = np.meshgrid(c, c, c, indexing="ij")
    cz, cy, cx = cz.ravel(), cy.ravel(), cx.ravel()
    rows, cols, vals = [], [], []
    for Ke, v in zip(mats, verts):
        # grid coordinates (0..n+1) of the four vertices of this tetrahedron in every cube
        px = cx[:, None] + v[None, :, 0]
        py = cy[:, None] + v[None, :, 1]
        pz = cz[:, None] + v[None, :, 2]
        if field is None:
            a = np.ones(cx.size)
        else:
            fld = np.asarray(field, dtype=np.float64)
            b = fld.shape[0]
            cen = (np.stack([px, py, pz], axis=-1).mean(axis=1)) * h  # centroids, (x, y, z)
            blk = np.minimum((cen * b).astype(np.int64), b - 1)
            a = fld[blk[:, 2], blk[:, 1], blk[:, 0]]
        inside = (px >= 1) & (px <= n) & (py >= 1) & (py <= n) & (pz >= 1) & (pz <= n)
        idx = ((pz - 1) * n + (py - 1)) * n + (px - 1)
        for r in range(4):
            for s in range(4):
                m = inside[:, r] & inside[:, s]
                rows.append(idx[m, r])
                cols.append(idx[m, s])
                vals.append(a[m] * Ke[r, s] * h)  # |T| = h^3 |T_1|, gradients scale by 1/h
    N = n ** 3
    A = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(N, N))
    A.sum_duplicates()
    A.eliminate_zeros()
    return A


def half_cube_field(mu, b=2):
    """Block field of the paper's heterogeneous 3-D test: a = mu on the half x < 1/2, a = 1 elsewhere."""
    fld = np.ones((b, b, b))
    fld[:, :, : b // 2] = float(mu)
    return fld
