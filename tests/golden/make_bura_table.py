"""Write tests/golden/bura_oracle_table.json from the oracle's Remez (Algorithm 1).

Every value in the table comes from ``oracle.remez.bura`` and nothing else.
Tests, smoke() and bench.py read the table instead of re-running the
multi-precision Remez (mpmath is not installed on every machine that runs them).

Usage:  python tests/golden/make_bura_table.py [--k K1-K2] [alpha ...]   (merges into the file;
        default k = 1..10)
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import mpmath as mp  # noqa: E402

from oracle.remez import bura  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "bura_oracle_table.json")
ALPHAS = [0.1, 0.25, 0.5, 0.75, 0.9]
KMAX = 10


def entry(res):
    s = lambda v: mp.nstr(v, 30, strip_zeros=False)  # noqa: E731
    return {"alpha": res.alpha, "k": res.k, "E": s(res.E),
            "c": [s(v) for v in res.c], "d": [s(v) for v in res.d],
            "zeta": [s(v) for v in res.zeta],
            "p": [s(v) for v in res.p], "q": [s(v) for v in res.q],
            "eta": [s(v) for v in res.eta]}


def main(alphas, kmin, kmax):
    table = {}
    if os.path.exists(OUT):
        with open(OUT) as fh:
            table = json.load(fh)
    for a in alphas:
        for k in range(kmin, kmax + 1):
            t0 = time.time()
            res = bura(a, k)
            table["%.4f/%d" % (a, k)] = entry(res)
            print("alpha=%g k=%d E=%s (%.1fs)" % (a, k, mp.nstr(res.E, 10), time.time() - t0), flush=True)
            # re-read and merge so that parallel runs for different alphas do not clobber each other
            cur = {}
            if os.path.exists(OUT):
                with open(OUT) as fh:
                    cur = json.load(fh)
            cur.update({key: v for key, v in table.items() if key.startswith("%.4f/" % a)})
            with open(OUT + ".tmp%d" % os.getpid(), "w") as fh:
                json.dump(dict(sorted(cur.items())), fh, indent=1)
            os.replace(OUT + ".tmp%d" % os.getpid(), OUT)


if __name__ == "__main__":
    args = sys.argv[1:]
    kmin, kmax = 1, KMAX
    if args and args[0] == "--k":
        lo, hi = args[1].split("-")
        kmin, kmax = int(lo), int(hi)
        args = args[2:]
    al = [float(x) for x in args] or ALPHAS
    main(al, kmin, kmax)
