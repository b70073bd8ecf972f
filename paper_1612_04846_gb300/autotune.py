"""A table of tuned solver options per problem class (grid, k), built with the library's autotuner.

bura_autotune (C ABI) times the candidate option sets of one class on the GPU and returns the fastest;
this module keeps the results as a JSON table keyed by the grid and k, and looks options up for new
problems (host bookkeeping only: the timing and the solves run in the library).
"""
from __future__ import annotations

import json
import os

from . import bura

__all__ = ["tune", "save", "load", "options_for"]

_FIELDS = [name for name, _ in bura.bura_options._fields_]


def _key(shape, k):
    return "x".join(str(int(n)) for n in shape) + ":%d" % int(k)


def tune(classes, alpha=0.5, tol=1e-6, trials=3, base=None):
    """classes: iterable of (shape, k).  Returns {key: {"grid", "k", "ms", "options"}}."""
    table = {}
    for shape, k in classes:
        best, ms = bura.bura_autotune(shape, alpha, k, tol=tol, trials=trials, base=base)
        table[_key(shape, k)] = {"grid": [int(n) for n in shape], "k": int(k), "alpha": float(alpha),
                                 "ms": ms, "options": {f: getattr(best, f) for f in _FIELDS}}
    return table


def save(table, path):
    tmp = path + ".tmp%d" % os.getpid()
    with open(tmp, "w") as fh:
        json.dump(table, fh, indent=1, sort_keys=True)
    os.replace(tmp, path)


def load(path):
    with open(path) as fh:
        return json.load(fh)


def options_for(table, shape, k, base=None):
    """bura_options of the tuned class (shape, k), or the defaults (or base) if the class is not in the table."""
    o = base if base is not None else bura.bura_default_options()
    ent = table.get(_key(shape, k))
    if ent is not None:
        for f, v in ent["options"].items():
            setattr(o, f, v)
    return o
