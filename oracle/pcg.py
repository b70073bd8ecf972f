"""Same-method CPU solve: one multigrid-preconditioned CG per shifted system (oracle).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

u = sum_j c_j (A - d_j I)^{-1} f (eq. (Rgeneral), Sec. 2.2), every shifted system solved on its own by
PCG in FP64 to a relative residual rtol (1e-13 by default), with a geometric multigrid V-cycle as the
preconditioner; the C code is oracle/cpu_pcg.c (OpenMP over the two slowest grid axes), compiled here with
the host compiler into oracle/_build/.  This is both the oracle of the variable-coefficient operators,
which have no closed form, and the timed same-method CPU baseline.

Shapes follow the other oracle modules: ``shape`` = (ny, nx) or (nz, ny, nx), faces (ax, ay[, az]) in
numpy C order (x fastest) or None for a = 1; Lambda is the max absolute row sum of Atilde
(eq. (algebraic)), computed by ``gershgorin`` from the faces.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

__all__ = ["gershgorin", "lambda_low", "solve_tolerances", "bura_pcg", "build", "max_threads"]

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cpu_pcg.c")
_LIB = os.path.join(_HERE, "_build", "libcpu_pcg.so")
_handle = None


def build(force=False):
    """Compile cpu_pcg.c (gcc -O2 -fopenmp) if the library is missing or older than the source."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    tmp = _LIB + ".tmp%d" % os.getpid()
    subprocess.run(["gcc", "-std=c99", "-O2", "-fopenmp", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"], check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _lib():
    global _handle
    if _handle is None:
        build()
        L = C.CDLL(_LIB)
        dp = C.POINTER(C.c_double)
        L.op_bura_solve.argtypes = [C.c_int, C.POINTER(C.c_int), dp, dp, dp, C.c_double, C.c_int, dp, dp, dp, dp, dp,
                                    dp, C.c_int, C.POINTER(C.c_int), C.c_int]
        L.op_bura_solve.restype = C.c_int
        L.op_max_threads.argtypes = []
        L.op_max_threads.restype = C.c_int
        _handle = L
    return _handle


def max_threads():
    """Threads the OpenMP runtime uses by default on this host."""
    return int(_lib().op_max_threads())


def gershgorin(shape, faces=None):
    """max_P sum_Q |Atilde_PQ| from the face coefficients (a = 1 when faces is None)."""
    shape = tuple(int(n) for n in shape)
    d = len(shape)
    total = np.zeros(shape)
    for fdir in range(d):
        axis = d - 1 - fdir
        n = shape[axis]
        h2 = (1.0 / (n + 1)) ** 2
        if faces is None:
            s = list(shape)
            s[axis] += 1
            a = np.ones(s)
        else:
            a = np.asarray(faces[fdir], dtype=np.float64)
        lo = np.take(a, np.arange(n), axis=axis)
        hi = np.take(a, np.arange(1, n + 1), axis=axis)
        idx = [1] * d
        idx[axis] = n
        i = np.arange(n).reshape(idx)
        # diagonal lo + hi, and the off-diagonal couplings to the interior neighbours
        total = total + (lo + hi + np.where(i > 0, lo, 0.0) + np.where(i < n - 1, hi, 0.0)) / h2
    return float(total.max())


def _ptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def lambda_low(shape, faces=None):
    """A lower bound on lambda_min(A): the smallest face coefficient times lambda_min of the scaled
    constant-coefficient operator (sum over the axes of 4 sin^2(pi h / 2) / h^2, divided by Lambda)."""
    lam = gershgorin(shape, faces)
    lc = sum(4.0 * np.sin(np.pi / (2.0 * (n + 1))) ** 2 * (n + 1) ** 2 for n in shape) / lam
    amin = 1.0 if faces is None else min(float(np.min(a)) for a in faces)
    return amin * lc


def solve_tolerances(shape, c, d, tol, faces=None):
    """Relative residual targets rtol_j with sum_j c_j ||r_j|| / (lambda_lo - d_j) <= tol ||f||: the
    partial-fraction value then lies within tol ||f|| of the exact one (each system's error is at most
    ||r_j|| / (lambda_min - d_j), and the K systems share the budget equally)."""
    lo = lambda_low(shape, faces)
    K = len(c)
    return [min(1.0, tol * (lo - float(dj)) / (K * float(cj))) for cj, dj in zip(c, d)]


def bura_pcg(shape, f, c, d, faces=None, rtol=1e-13, max_iter=1000, threads=0, components=False):
    """u = sum_j c_j (A - d_j I)^{-1} f by PCG per system; returns (u, iterations per system) or, with
    components, (u, V, iterations) with V[j] = (A - d_j I)^{-1} f.  rtol: one relative residual target
    for every system, or a sequence of K targets."""
    shape = tuple(int(n) for n in shape)
    dim = len(shape)
    n = (C.c_int * 3)(*(list(reversed(shape)) + [1] * (3 - dim)))
    f = np.ascontiguousarray(f, dtype=np.float64).ravel()
    N = f.size
    c = np.ascontiguousarray(c, dtype=np.float64)
    d = np.ascontiguousarray(d, dtype=np.float64)
    K = c.size
    keep = []
    fp = [None, None, None]
    if faces is not None:
        for a in range(dim):
            arr = np.ascontiguousarray(faces[a], dtype=np.float64)
            keep.append(arr)
            fp[a] = _ptr(arr)
    lam = gershgorin(shape, faces)
    u = np.zeros(N)
    V = np.zeros((K, N)) if components else None
    its = (C.c_int * K)()
    rt = np.ascontiguousarray(np.broadcast_to(np.asarray(rtol, dtype=np.float64), (K,)))
    rc = _lib().op_bura_solve(dim, n, fp[0], fp[1], fp[2], lam, K, _ptr(c), _ptr(d), _ptr(f), _ptr(u),
                              _ptr(V) if components else None, _ptr(rt), int(max_iter), its, int(threads))
    if rc != 0:
        raise RuntimeError("oracle PCG failed (%d)" % rc)
    return (u, V, list(its)) if components else (u, list(its))
