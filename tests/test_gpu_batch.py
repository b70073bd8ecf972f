"""Batched solves (bura_solve_batch) on the GPU, through the C ABI.

Problems of different grids, alpha and k are solved concurrently by worker threads with their own
streams.  Each result must be bit-for-bit the result of the same plan solved alone (the plan owns its
buffers and its reductions run in a fixed order), and must match the oracle's exact BURA value within
the solve tolerance (the same parity bar as the single-problem tests).
"""
import numpy as np
import pytest

from oracle import exact, tables
from paper_1612_04846_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)


@pytest.fixture(scope="module")
def lib():
    from paper_1612_04846_gb300 import build_lib, bura
    build_lib.build(verbose=False)
    return bura


def _problems(seed, n):
    """n problems: grids from {31^2, 63^2, 127^2, 63x31, 255^2}, alpha from the oracle table's values,
    k in 5..9, f ~ U[-1, 1] (seeded)."""
    rng = np.random.default_rng(seed)
    shapes = [(31, 31), (63, 63), (127, 127), (63, 31), (255, 255)]
    out = []
    for i in range(n):
        shape = shapes[rng.integers(len(shapes))]
        alpha = float(rng.choice([0.1, 0.25, 0.5, 0.75, 0.9]))
        k = int(rng.integers(5, 10))
        out.append((shape, alpha, k, W.rhs_uniform(tuple(reversed(shape)), 100 + i)))
    return out


@pytest.mark.parametrize("precision,tol,nworkers", [("MIXED", 1e-6, 4), ("MIXED", 1e-8, 16), ("FP64", 1e-10, 8)])
def test_batch_equals_single_solves_and_oracle(lib, precision, tol, nworkers):
    probs = _problems(7, 12)
    plans, fs, us = [], [], []
    try:
        for shape, alpha, k, f in probs:
            o = lib.bura_default_options()
            o.precision = getattr(lib, "BURA_PREC_" + precision)
            plans.append(lib.bura_setup(shape, alpha, k, options=o))
            fs.append(torch.from_numpy(f).cuda())
            us.append(torch.zeros_like(fs[-1]))
        st = lib.bura_solve_batch(plans, fs, us, tol, nworkers)
        torch.cuda.synchronize()
        assert st == [lib.BURA_OK] * len(probs)
        batch = [u.cpu().numpy() for u in us]
        # the same plans, one at a time
        for i, (shape, alpha, k, f) in enumerate(probs):
            u1 = torch.zeros_like(fs[i])
            assert lib.bura_solve(plans[i], fs[i], u1, tol) == lib.BURA_OK
            torch.cuda.synchronize()
            assert np.array_equal(u1.cpu().numpy(), batch[i]), (i, shape, alpha, k)
            ref = tables.entry(alpha, k)
            ur = exact.bura_value(tuple(reversed(shape)), f, ref["c"], ref["d"])
            err = float(np.linalg.norm(batch[i] - ur) / np.linalg.norm(ur))
            assert err <= tol, (i, shape, alpha, k, err)
    finally:
        for p in plans:
            lib.bura_destroy(p)


def test_batch_rejects_a_plan_listed_twice(lib):
    plan = lib.bura_setup((31, 31), 0.5, 5)
    try:
        f = torch.ones(31 * 31, dtype=torch.float64, device="cuda")
        u = torch.zeros_like(f)
        v = torch.zeros_like(f)
        with pytest.raises(lib.BuraError) as ei:
            lib.bura_solve_batch([plan, plan], [f, f], [u, v], 1e-6, 2)
        assert ei.value.code == lib.BURA_EINVAL
    finally:
        lib.bura_destroy(plan)
