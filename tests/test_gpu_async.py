"""The device-driven solve (the whole solve one captured graph, decisions taken by controller kernels)
and the captured batch, through the C ABI.

  * bura_solve_async enqueues without waiting; several plans queued on one stream and waited for give
    the results of bura_solve bit for bit, and the oracle's exact BURA value within tol;
  * the captured solve equals the host-driven one (per-kernel profiling turns the host driver on) up to
    the solve tolerance, with the same outcome (status, iteration counts within one);
  * the statuses a solve reports: a zero right-hand side, an iteration cap (BURA_ENOCONV);
  * a BuraBatch (one graph over all problems) run twice equals single solves bit for bit and the oracle.
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


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _opts(lib, precision, **kw):
    o = lib.bura_default_options()
    o.precision = precision
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def _ur(shape, f, alpha, k):
    e = tables.entry(alpha, k)
    return exact.bura_value(tuple(reversed(shape)), f, e["c"], e["d"])


@pytest.mark.parametrize("precision,tol", [(0, 1e-10), (1, 1e-6), (1, 1e-9)])
def test_async_solves_on_one_stream(lib, precision, tol):
    cases = [((127, 127), 0.25, 7), ((63, 63), 0.5, 5), ((255, 255), 0.75, 9)]
    plans, fs, us = [], [], []
    stream = torch.cuda.Stream()
    try:
        for i, (shape, alpha, k) in enumerate(cases):
            plans.append(lib.bura_setup(shape, alpha, k, options=_opts(lib, precision)))
            fs.append(torch.from_numpy(W.rhs_uniform(tuple(reversed(shape)), 40 + i)).cuda())
            us.append(torch.zeros_like(fs[-1]))
        torch.cuda.synchronize()
        for p, f, u in zip(plans, fs, us):
            assert lib.bura_solve_async(p, f, u, tol, stream) == lib.BURA_OK
        for p in plans:
            assert lib.bura_solve_wait(p) == lib.BURA_OK
        stream.synchronize()
        for i, (shape, alpha, k) in enumerate(cases):
            u1 = torch.zeros_like(fs[i])
            assert lib.bura_solve(plans[i], fs[i], u1, tol) == lib.BURA_OK
            torch.cuda.synchronize()
            assert np.array_equal(u1.cpu().numpy(), us[i].cpu().numpy()), i
            assert _rel(us[i].cpu().numpy(), _ur(shape, fs[i].cpu().numpy(), alpha, k)) <= tol
            st = lib.bura_get_stats(plans[i])
            assert st["iters"] > 0 and st["launches"] > 0 and 0 <= st["err_bound"] <= tol
    finally:
        for p in plans:
            lib.bura_destroy(p)


@pytest.mark.parametrize("precision,tol", [(0, 1e-10), (1, 1e-6)])
@pytest.mark.parametrize("shape,var", [((255, 255), False), ((31, 31, 31), True)])
def test_captured_solve_matches_the_host_driven_solve(lib, precision, tol, shape, var):
    nps = tuple(reversed(shape))
    faces = W.block_lognormal_faces(nps, 8, 1e-2, 1.0, 2) if var else None
    f = torch.from_numpy(W.rhs_uniform(nps, 41)).cuda()
    plan = lib.bura_setup(shape, 0.5, 7, faces=faces, options=_opts(lib, precision))
    try:
        u1 = torch.zeros_like(f)
        assert lib.bura_solve(plan, f, u1, tol) == lib.BURA_OK
        torch.cuda.synchronize()
        s1 = lib.bura_get_stats(plan)
        lib.bura_set_profiling(plan, 1)  # per-kernel timing drives the solve from the host
        u2 = torch.zeros_like(f)
        assert lib.bura_solve(plan, f, u2, tol) == lib.BURA_OK
        torch.cuda.synchronize()
        s2 = lib.bura_get_stats(plan)
        lib.bura_set_profiling(plan, 0)
    finally:
        lib.bura_destroy(plan)
    a, b = u1.cpu().numpy(), u2.cpu().numpy()
    assert _rel(a, b) <= 2 * tol
    assert s1["outer"] == s2["outer"] and abs(s1["iters"] - s2["iters"]) <= 1


@pytest.mark.parametrize("precision", [0, 1])
def test_statuses_of_the_captured_solve(lib, precision):
    shape = (63, 63)
    plan = lib.bura_setup(shape, 0.5, 7, options=_opts(lib, precision))
    try:
        z = torch.zeros(63 * 63, dtype=torch.float64, device="cuda")
        u = torch.full_like(z, 7.0)
        assert lib.bura_solve(plan, z, u, 1e-6) == lib.BURA_OK
        torch.cuda.synchronize()
        assert float(u.abs().max()) == 0.0
    finally:
        lib.bura_destroy(plan)
    plan = lib.bura_setup(shape, 0.5, 7, options=_opts(lib, precision, max_iters=1, max_outer=1))
    try:
        f = torch.from_numpy(W.rhs_uniform((63, 63), 42)).cuda()
        u = torch.zeros_like(f)
        assert lib.bura_solve(plan, f, u, 1e-10) == lib.BURA_ENOCONV
        assert lib.bura_solve_async(plan, f, u, 1e-10) == lib.BURA_OK
        assert lib.bura_solve_wait(plan) == lib.BURA_ENOCONV
    finally:
        lib.bura_destroy(plan)


def test_captured_batch_runs_twice_and_equals_single_solves(lib):
    rng = np.random.default_rng(9)
    shapes = [(31, 31), (63, 63), (127, 127), (63, 31), (255, 255)]
    probs, plans, fs, us = [], [], [], []
    try:
        for i in range(14):
            shape = shapes[rng.integers(len(shapes))]
            alpha = float(rng.choice([0.1, 0.25, 0.5, 0.75, 0.9]))
            k = int(rng.integers(5, 10))
            prec = int(rng.integers(2))
            probs.append((shape, alpha, k))
            plans.append(lib.bura_setup(shape, alpha, k, options=_opts(lib, prec)))
            fs.append(torch.from_numpy(W.rhs_uniform(tuple(reversed(shape)), 200 + i)).cuda())
            us.append(torch.zeros_like(fs[-1]))
        batch = lib.BuraBatch(plans, fs, us, 1e-8, branches=5)
        try:
            for rep in range(2):
                for u in us:
                    u.zero_()
                batch.run()
                assert batch.wait() == [lib.BURA_OK] * len(plans)
                torch.cuda.synchronize()
            got = [u.cpu().numpy() for u in us]
        finally:
            batch.close()
        for i, (shape, alpha, k) in enumerate(probs):
            u1 = torch.zeros_like(fs[i])
            assert lib.bura_solve(plans[i], fs[i], u1, 1e-8) == lib.BURA_OK
            torch.cuda.synchronize()
            assert np.array_equal(u1.cpu().numpy(), got[i]), i
            assert _rel(got[i], _ur(shape, fs[i].cpu().numpy(), alpha, k)) <= 1e-8
    finally:
        for p in plans:
            lib.bura_destroy(p)
