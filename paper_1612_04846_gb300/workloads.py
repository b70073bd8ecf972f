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

import numpy as np

__all__ = ["rhs_uniform", "rhs_normal", "block_lognormal_faces", "constant_faces", "checkerboard_rhs"]


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
