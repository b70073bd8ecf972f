"""Bonito-Pasciak sinc quadrature of A^{-alpha} (the comparison method of the paper, [BP15]).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The quadrature of the paper's comparison section (from [BP15, Remark 3.1]) approximates
Atilde^{-alpha} f by
    u_Q = (2 k' sin(pi alpha) / pi) sum_{l=-m}^{M} e^{2(alpha-1) l k'} (e^{-2 l k'} I + Atilde)^{-1} f,
    m = ceil(pi^2 / (4 alpha k'^2)),  M = ceil(pi^2 / (4 (1 - alpha) k'^2)),
every term a positive diagonal shift of Atilde.  With the scaled A = Atilde / Lambda (eq. (algebraic))
this is the partial-fraction form sum_l c_l (A - d_l I)^{-1} f of A^{-alpha} f with
    d_l = -e^{-2 l k'} / Lambda,   c_l = (2 k' sin(pi alpha) / pi) e^{2(alpha-1) l k'} Lambda^(alpha-1),
so it runs on the same multi-shift solve as the BURA value (M + m + 1 shifted systems).
"""
from __future__ import annotations

import math

import numpy as np

from . import exact

__all__ = ["bp15_counts", "bp15_shifts", "bp15_value"]


def bp15_counts(alpha, kprime):
    """(m, M) of the quadrature; M + m + 1 shifted systems."""
    m = math.ceil(math.pi ** 2 / (4.0 * alpha * kprime ** 2))
    M = math.ceil(math.pi ** 2 / (4.0 * (1.0 - alpha) * kprime ** 2))
    return m, M


def bp15_shifts(alpha, kprime, Lam, counts=None):
    """Weights c_l and shifts d_l (l = -m .. M) of u_Q for the scaled operator A = Atilde / Lam; counts
    (m, M) overrides the truncation of the printed formula (used to check the untruncated sum)."""
    m, M = bp15_counts(alpha, kprime) if counts is None else counts
    pre = 2.0 * kprime * math.sin(math.pi * alpha) / math.pi
    c, d = [], []
    for l in range(-m, M + 1):
        c.append(pre * math.exp(2.0 * (alpha - 1.0) * l * kprime) * Lam ** (alpha - 1.0))
        d.append(-math.exp(-2.0 * l * kprime) / Lam)
    return c, d


def bp15_value(shape, f, alpha, kprime):
    """u_Q, the quadrature approximation of A^{-alpha} f (A scaled, constant coefficients)."""
    c, d = bp15_shifts(alpha, kprime, exact.gershgorin(shape))
    return exact.apply_function(shape, f, lambda lam: sum(cj / (lam - dj) for cj, dj in zip(c, d)))
