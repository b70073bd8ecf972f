"""Pins of the oracle's Bonito-Pasciak quadrature (the paper's comparison method, [BP15]).

  * Without truncation the sinc sum is exact: with l running far beyond (m, M) the weights and shifts give
    lambda^-alpha to 1e-11 over the whole scaled spectrum of the 1023^2 operator (a wrong power of Lambda,
    a sign or the step 2k' fails this by orders of magnitude).
  * The printed truncation (m, M) has the quadrature's O(e^(-pi^2 / (2k'))) error at the bottom of the
    spectrum (unscaled lambda = 2 pi^2, the Laplacian's smallest eigenvalue on the unit square): between
    0.3 and 3 times e^(-pi^2 / (2k')) at k' = 1/3.  Toward the top it is larger: the terms that resolve an
    eigenvalue lambda (unscaled) sit near l = -ln(lambda) / (2k'), so the m large-shift terms leave a tail
    there; at lambda = Lambda = 8.4e6 (h = 2^-10) the relative error is about 1e-2 for alpha = 0.75.

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


@pytest.mark.parametrize("alpha", [0.25, 0.5, 0.75])
def test_untruncated_sinc_sum_is_exact(alpha):
    shape = (1023, 1023)
    Lam = exact.gershgorin(shape)
    lam = np.geomspace(float(exact.eigenvalues(shape).min()), 1.0, 60)
    c, d = quadrature.bp15_shifts(alpha, 1.0 / 3.0, Lam, counts=(300, 300))
    q = sum(cj / (lam - dj) for cj, dj in zip(c, d))
    assert np.max(np.abs(q * lam ** alpha - 1.0)) < 1e-11


@pytest.mark.parametrize("alpha", [0.25, 0.5, 0.75])
def test_printed_truncation_error_bottom_and_top_of_the_spectrum(alpha):
    kp = 1.0 / 3.0
    shape = (1023, 1023)
    Lam = exact.gershgorin(shape)
    c, d = quadrature.bp15_shifts(alpha, kp, Lam)
    est = math.exp(-math.pi ** 2 / (2 * kp))
    lo = 2 * math.pi ** 2 / Lam
    e_lo = abs(sum(cj / (lo - dj) for cj, dj in zip(c, d)) * lo ** alpha - 1.0)
    assert 0.3 * est <= e_lo <= 3 * est, (e_lo, est)
    e_hi = abs(sum(cj / (1.0 - dj) for cj, dj in zip(c, d)) - 1.0)
    assert e_hi > 10 * e_lo
    if alpha == 0.75:
        assert 5e-3 < e_hi < 5e-2
