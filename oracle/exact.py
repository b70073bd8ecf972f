"""Closed-form eigenbasis solutions on constant-coefficient grids (oracle).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

For a = 1 on a uniform Dirichlet grid the matrix Atilde is a Kronecker sum of
1D matrices h^{-2} tridiag(-1,2,-1), whose eigenpairs are
(4 h^{-2} sin^2(i pi h / 2), sin(i j pi h)) (Sec. 5.1, with the 1D scaling undone);
the orthonormal eigenvector matrix is the type-I discrete sine transform.
Every function of A is then W phi(D) W^T f (eq. (exacalg), Sec. 1.1):
  * exact solution          u   = A^{-alpha} f                    (phi = lambda^-alpha)
  * exact BURA value        u_r = sum_j c_j (A - d_j I)^{-1} f    (phi = sum c_j/(lambda-d_j),
                                                                    eq. (Rgeneral), Sec. 2.2)
A = Atilde / Lambda with Lambda = max absolute row sum of Atilde (eq. (algebraic)).
"""
from __future__ import annotations

import numpy as np
import scipy.fft as sfft

__all__ = ["gershgorin", "eigenvalues", "apply_function", "fractional", "bura_value", "bura_components",
           "multistep_value", "multistep_error", "energy_ratio", "product_error_on_interval",
           "reconstruction_ratio"]


def gershgorin(shape):
    """max_i sum_j |Atilde_ij| for a = 1: each axis adds 2/h^2 plus 1/h^2 per interior neighbour."""
    lam = 0.0
    for n in shape:
        h2 = (1.0 / (n + 1)) ** 2
        lam += (2.0 + min(n - 1, 2)) / h2
    return lam


def eigenvalues(shape):
    """Eigenvalues of the scaled A on the grid, as an array of the grid's shape."""
    shape = tuple(int(n) for n in shape)
    lam = np.zeros(shape)
    d = len(shape)
    for axis, n in enumerate(shape):
        h = 1.0 / (n + 1)
        i = np.arange(1, n + 1)
        mu = 4.0 / h ** 2 * np.sin(i * np.pi * h / 2) ** 2
        s = [1] * d
        s[axis] = n
        lam = lam + mu.reshape(s)
    return lam / gershgorin(shape)


def apply_function(shape, f, phi):
    """W phi(Lambda) W^T f with W the orthonormal DST-I on every axis."""
    shape = tuple(int(n) for n in shape)
    F = sfft.dstn(np.asarray(f, dtype=np.float64).reshape(shape), type=1, norm="ortho")
    F *= phi(eigenvalues(shape))
    return sfft.idstn(F, type=1, norm="ortho").ravel()


def fractional(shape, f, alpha):
    """Exact u = A^{-alpha} f."""
    return apply_function(shape, f, lambda lam: lam ** (-float(alpha)))


def bura_value(shape, f, c, d):
    """Exact u_r = sum_j c_j (A - d_j I)^{-1} f (every shifted system solved exactly)."""
    c = [float(v) for v in c]
    d = [float(v) for v in d]
    return apply_function(shape, f, lambda lam: sum(cj / (lam - dj) for cj, dj in zip(c, d)))


def bura_components(shape, f, d):
    """The k+1 exact solutions v_j = (A - d_j I)^{-1} f, shape (k+1, N)."""
    return np.stack([apply_function(shape, f, lambda lam, dj=float(dj): 1.0 / (lam - dj)) for dj in d])


def multistep_value(shape, f, steps):
    """Multi-step BURA value (Sec. "Multi-step BURA approximation"): u_0 = f and
    u_i = r_{alpha_i}(A) A^{-1} u_{i-1}, each step the exact BURA value of its (c, d), steps in order of
    application; approximates A^{-(alpha_1 + ... + alpha_n)} f."""
    u = np.asarray(f, dtype=np.float64)
    for c, d in steps:
        u = bura_value(shape, u, c, d)
    return u


def multistep_error(shape, steps, alpha):
    """E_{alpha_1..alpha_n}(k,k;1) of eq. (multi-step error): the largest |prod_i r_i(t) / t^(n-1) -
    t^(1-alpha)| over the eigenvalues t of A, with r_i(t) = t sum_j c_j/(t - d_j) (eq. (simplified))."""
    lam = eigenvalues(shape).ravel()
    prod = np.ones_like(lam)
    for c, d in steps:
        prod *= lam * sum(float(cj) / (lam - float(dj)) for cj, dj in zip(c, d))
    n = len(steps)
    return float(np.max(np.abs(prod / lam ** (n - 1) - lam ** (1.0 - float(alpha)))))


def energy_ratio(shape, f, u, alpha):
    """||u - A^{-alpha} f||_A / ||f||_{A^{-1}}, the error measure of eq. (errorU)."""
    e = np.asarray(u, dtype=np.float64) - fractional(shape, f, alpha)
    ea = float(e @ apply_function(shape, e, lambda lam: lam))
    fa = float(np.asarray(f) @ apply_function(shape, f, lambda lam: 1.0 / lam))
    return (ea / fa) ** 0.5


def _r_of_t(c, d, t):
    """r(t) = t sum_j c_j/(t - d_j) (eq. (simplified)), continued by r(0) = c_0 where d_0 = 0."""
    t = np.asarray(t, dtype=np.float64)
    out = np.zeros_like(t)
    for cj, dj in zip(c, d):
        cj, dj = float(cj), float(dj)
        out += cj if dj == 0.0 else cj * t / (t - dj)
    return out


def product_error_on_interval(steps, t):
    """|r_1(t) r_2(t) ... - t| on the points t of [0, 1]: the two-step residual of the f-reconstruction
    (Sec. "1D and 3D numerical tests", E_{1-alpha,alpha}(k,k;2) is its maximum over [0, 1])."""
    prod = np.ones_like(np.asarray(t, dtype=np.float64))
    for c, d in steps:
        prod = prod * _r_of_t(c, d, t)
    return np.abs(prod - np.asarray(t))


def reconstruction_ratio(shape, f, steps):
    """||f_r - f|| / ||A^{-1} f|| with f_r = A u_2, u_2 the two-step value of steps (eq. (3D error))."""
    u2 = multistep_value(shape, f, steps)
    fr = apply_function(shape, u2, lambda lam: lam)
    return float(np.linalg.norm(fr - f) / np.linalg.norm(apply_function(shape, f, lambda lam: 1.0 / lam)))
