"""Pins of the oracle's Bonito-Pasciak quadrature (the paper's comparison method, [BP15]).

  * The paper takes u_Q with k' = 1/3 at h = 2^-10 as its reference solution and states an O(1e-7) error.
    Reading: near the bottom of the spectrum, where a smooth solution lives, the scalar quadrature error
    is about 8e-7; the discontinuous checkerboard right-hand side (eq. (checkerboard)) also excites the
    top of the spectrum, where the upper truncation is coarser, and its relative l2 error on 1023^2 is
    1.0-2.4e-6 for alpha = 0.25 .. 0.75.  Pinned: below 5e-6 (and the scalar error at lambda = 20 below
    1e-6).
  * The number of shifted systems M + m + 1 is at least k_Q + 1, k_Q = pi^2 / (4 alpha (1 - alpha) k'^2).
  * The quadrature converges as k' decreases (exponentially in 1/k').
A wrong sign in an exponent or a dropped Lambda^(alpha-1) breaks the first pin by orders of magnitude.
"""
import math

import numpy as np
import pytest

from oracle import exact, quadrature
from paper_1612_04846_gb300 import workloads as W


@pytest.mark.parametrize("alpha", [0.25, 0.5, 0.75])
def test_reference_solution_error_is_order_1e7(alpha):
    shape = (1023, 1023)
    f = W.checkerboard_rhs(shape)
    uq = quadrature.bp15_value(shape, f, alpha, 1.0 / 3.0)
    u = exact.fractional(shape, f, alpha)
    err = float(np.linalg.norm(uq - u) / np.linalg.norm(u))
    assert err < 5e-6, err
    lam = 20.0 / exact.gershgorin(shape)  # the scaled operator's smallest eigenvalues are near this
    c, d = quadrature.bp15_shifts(alpha, 1.0 / 3.0, exact.gershgorin(shape))
    q = sum(cj / (lam - dj) for cj, dj in zip(c, d))
    assert abs(q * lam ** alpha - 1.0) < 1e-6


@pytest.mark.parametrize("alpha,kp", [(0.25, 0.5), (0.5, 1.0 / 3.0), (0.75, 0.7)])
def test_system_count(alpha, kp):
    m, M = quadrature.bp15_counts(alpha, kp)
    kq = math.pi ** 2 / (4.0 * alpha * (1.0 - alpha) * kp ** 2)
    assert M + m + 1 >= kq + 1
    c, d = quadrature.bp15_shifts(alpha, kp, 8.0)
    assert len(c) == len(d) == M + m + 1 and all(x > 0 for x in c) and all(x < 0 for x in d)


def test_error_decreases_with_kprime():
    shape, alpha = (127, 127), 0.5
    f = W.rhs_uniform(shape, 9)
    u = exact.fractional(shape, f, alpha)
    errs = [float(np.linalg.norm(quadrature.bp15_value(shape, f, alpha, kp) - u) / np.linalg.norm(u))
            for kp in (1.0, 0.7, 0.5, 1.0 / 3.0)]
    assert all(a > b for a, b in zip(errs, errs[1:])), errs
    assert errs[-1] < 1e-4 and errs[0] > 1e-2
