"""Pins of the oracle's multi-step BURA (Sec. "Multi-step BURA approximation") against the paper.

  * eq. (general 2-step error): E_{a1 a2} <= E_{a2} k(A)^{a1} + E_{a1} k(A)^{a2} + E_{a1} E_{a2} k(A), with
    k(A) <= 1 / Lambda_1 since the spectrum is scaled into (0, 1];
  * the top eigenvector Psi_N: the error ratio is about E_{a1} + E_{a2} - E_{a1} E_{a2} (the residuals are
    -E_{ai} at t = 1, Lemma BURA_caracter), because Lambda_N is close to 1;
  * for any f the ratio ||u_n - A^{-alpha} f||_A / ||f||_{A^{-1}} is at most E_{a1..an} (the argument of
    Lemma l:BURAerror with the multi-step error function).
  * the f-reconstruction (Sec. "1D and 3D numerical tests"): |r_{1-alpha}(t) r_alpha(t) - t| on [0, 1]
    reaches its largest value E_{1-alpha} + E_alpha - E_{1-alpha} E_alpha at t = 1 only (eq. (3D error final),
    stated sharp for k = 5, 7), and ||f_r - f|| / ||A^{-1} f|| stays below it.
A dropped cross term, a wrong power of t or a sign slip breaks one of these.
"""
import numpy as np
import pytest
import scipy.fft as sfft

from oracle import exact, tables
from paper_1612_04846_gb300 import workloads as W


def _steps(alphas, k):
    return [(tables.entry(a, k)["c"], tables.entry(a, k)["d"]) for a in alphas]


@pytest.mark.parametrize("shape", [(63, 63), (127, 127), (31, 31, 31)])
@pytest.mark.parametrize("alphas", [(0.25, 0.25), (0.25, 0.5), (0.5, 0.25)])
def test_two_step_error_obeys_the_paper_bound(shape, alphas):
    k = 7
    e12 = exact.multistep_error(shape, _steps(alphas, k), sum(alphas))
    E1, E2 = tables.entry(alphas[0], k)["E"], tables.entry(alphas[1], k)["E"]
    kappa = 1.0 / float(np.min(exact.eigenvalues(shape)))
    bound = E2 * kappa ** alphas[0] + E1 * kappa ** alphas[1] + E1 * E2 * kappa
    assert 0 < e12 <= bound, (e12, bound)


@pytest.mark.parametrize("alphas", [(0.25, 0.25), (0.25, 0.5)])
def test_top_eigenvector_ratio_is_about_e1_plus_e2_minus_e1e2(alphas):
    shape, k = (127, 127), 7
    F = np.zeros(shape)
    F[-1, -1] = 1.0
    psi = sfft.idstn(F, type=1, norm="ortho").ravel()  # eigenvector of the largest eigenvalue
    u2 = exact.multistep_value(shape, psi, _steps(alphas, k))
    ratio = exact.energy_ratio(shape, psi, u2, sum(alphas))
    E1, E2 = tables.entry(alphas[0], k)["E"], tables.entry(alphas[1], k)["E"]
    lam_n = float(np.max(exact.eigenvalues(shape)))
    assert lam_n > 0.999
    assert abs(ratio - (E1 + E2 - E1 * E2)) <= 0.02 * (E1 + E2), (ratio, E1 + E2 - E1 * E2)


@pytest.mark.parametrize("alphas", [(0.25, 0.25), (0.1, 0.25, 0.25)])
def test_energy_ratio_is_bounded_by_the_multistep_error(alphas):
    shape, k = (63, 63), 7
    steps = _steps(alphas, k)
    f = W.rhs_uniform(shape, 21)
    u = exact.multistep_value(shape, f, steps)
    ratio = exact.energy_ratio(shape, f, u, sum(alphas))
    assert 0 < ratio <= exact.multistep_error(shape, steps, sum(alphas)) * (1 + 1e-9)


def test_one_step_is_the_bura_value():
    shape, k = (31, 31), 5
    f = W.rhs_uniform(shape, 3)
    ref = tables.entry(0.5, k)
    assert np.array_equal(exact.multistep_value(shape, f, [(ref["c"], ref["d"])]),
                          exact.bura_value(shape, f, ref["c"], ref["d"]))


@pytest.mark.parametrize("alpha", [0.25, 0.5, 0.75])
@pytest.mark.parametrize("k", [5, 7])
def test_reconstruction_residual_peaks_at_one(alpha, k):
    steps = _steps((alpha, 1.0 - alpha), k)
    t = np.concatenate([[0.0], np.logspace(-14, 0, 20001)])
    res = exact.product_error_on_interval(steps, t)
    E1, E2 = tables.entry(alpha, k)["E"], tables.entry(1.0 - alpha, k)["E"]
    assert abs(res[-1] - (E1 + E2 - E1 * E2)) <= 1e-9 * (E1 + E2)
    assert int(np.argmax(res)) == len(t) - 1
    assert np.max(res[t < 0.8]) < res[-1]


@pytest.mark.parametrize("shape", [(63, 63), (15, 15, 15)])
def test_reconstruction_ratio_within_the_paper_bound(shape):
    alpha, k = 0.25, 7
    steps = _steps((alpha, 1.0 - alpha), k)
    f = W.rhs_uniform(shape, 41)
    ratio = exact.reconstruction_ratio(shape, f, steps)
    E1, E2 = tables.entry(alpha, k)["E"], tables.entry(1.0 - alpha, k)["E"]
    assert 0 < ratio <= E1 + E2 - E1 * E2
