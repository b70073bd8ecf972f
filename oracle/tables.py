"""Lookup of the oracle-generated BURA coefficient table (oracle).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

``tests/golden/bura_oracle_table.json`` is written by
``tests/golden/make_bura_table.py``, which calls only ``oracle.remez.bura``
(Algorithm 1, Sec. 3.2).  Reading the table lets machines without mpmath use
the oracle's coefficients.  Values are stored as 30-digit decimal strings.
"""
from __future__ import annotations

import json
import os

_PATH = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "tests", "golden",
                     "bura_oracle_table.json")
_CACHE = None


def _table():
    global _CACHE
    if _CACHE is None:
        with open(_PATH) as fh:
            _CACHE = json.load(fh)
    return _CACHE


def available():
    return sorted((v["alpha"], v["k"]) for v in _table().values())


def entry(alpha, k):
    """Dict with float lists c, d (d_0 = 0 first), zeta, p, q, eta and float E."""
    key = "%.4f/%d" % (float(alpha), int(k))
    raw = _table().get(key)
    if raw is None:
        raise KeyError("no oracle table entry for alpha=%g k=%d" % (alpha, k))
    out = {"alpha": raw["alpha"], "k": raw["k"], "E": float(raw["E"])}
    for name in ("c", "d", "zeta", "p", "q", "eta"):
        out[name] = [float(x) for x in raw[name]]
    out["raw"] = raw
    return out
