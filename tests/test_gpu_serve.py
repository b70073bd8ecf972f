"""bura_retarget and the solve server (bura_server_*) on the GPU, through the C ABI.

A retargeted plan must give exactly the result of a plan set up at the new alpha (same tables, same
captured graph, deterministic reductions); the server's results must equal direct solves of the same
requests bit for bit, whichever resident plan served them, and meet the oracle at the tolerance.
"""
import numpy as np
import pytest

from oracle import direct, exact, operators, tables
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


def _np_shape(shape):
    return tuple(reversed(shape))


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _reference(shape, alpha, k, f, faces):
    ref = tables.entry(alpha, k)
    nps = _np_shape(shape)
    if faces is None:
        return exact.bura_value(nps, f, ref["c"], ref["d"])
    A, _ = operators.scaled_matrix(nps, faces)
    return direct.bura_sparse(A, f, ref["c"], ref["d"])


def _direct(lib, shape, alpha, k, f, tol, faces=None, options=None):
    plan = lib.bura_setup(shape, alpha, k, faces=faces, options=options)
    try:
        u = np.zeros_like(f)
        rc = lib.bura_solve_host(plan, f, u, tol)
        return u, rc
    finally:
        lib.bura_destroy(plan)


@pytest.mark.parametrize("shape,var,precision,refine", [((255, 255), False, "MIXED", "FP64"),
                                                        ((127, 127), False, "FP64", "FP64"),
                                                        ((15, 15, 15), True, "MIXED", "FP64"),
                                                        ((255, 255), False, "MIXED", "DF")])
def test_retarget_equals_a_fresh_plan(lib, shape, var, precision, refine):
    nps = _np_shape(shape)
    faces = W.block_lognormal_faces(nps, 4, 1e-2, 1.0, 2) if var else None
    f = W.rhs_uniform(nps, 11)
    o = lib.bura_default_options()
    o.precision = getattr(lib, "BURA_PREC_" + precision)
    o.refine = getattr(lib, "BURA_REFINE_" + refine)
    tol = 1e-10 if precision == "FP64" else 1e-6
    k = 7
    plan = lib.bura_setup(shape, 0.25, k, faces=faces, options=o)
    try:
        u0 = np.zeros_like(f)
        assert lib.bura_solve_host(plan, f, u0, tol) == lib.BURA_OK
        for alpha in (0.75, 0.5):
            lib.bura_retarget(plan, alpha)
            u = np.zeros_like(f)
            assert lib.bura_solve_host(plan, f, u, tol) == lib.BURA_OK
            uf, rc = _direct(lib, shape, alpha, k, f, tol, faces, o)
            assert rc == lib.BURA_OK
            assert np.array_equal(u, uf), alpha
            c, d, E = lib.bura_get_rational(plan, k)
            ref = tables.entry(alpha, k)
            assert np.allclose(c, ref["c"], rtol=1e-9) and np.allclose(d, ref["d"], rtol=1e-9)
            assert _rel(u, _reference(shape, alpha, k, f, faces)) <= tol
    finally:
        lib.bura_destroy(plan)


def _requests():
    """16 requests over 6 classes (grid, field, k), several alphas per class, 2-D and 3-D, constant and
    block log-normal coefficients (two fields)."""
    rng = np.random.default_rng(3)
    fields = {1: W.block_lognormal_faces(_np_shape((15, 15, 15)), 4, 1e-2, 1.0, 2),
              2: W.block_lognormal_faces(_np_shape((31, 15)), 4, 1e-2, 1.0, 5)}
    classes = [((63, 63), None, 0, 5), ((127, 127), None, 0, 7), ((31, 31, 31), None, 0, 9),
               ((15, 15, 15), 1, 1, 6), ((31, 15), 2, 2, 8), ((63, 31), None, 0, 7)]
    out = []
    for i in range(16):
        shape, fid, field, k = classes[i % len(classes)] if i < 12 else classes[rng.integers(len(classes))]
        alpha = float(rng.choice([0.1, 0.25, 0.5, 0.75, 0.9]))
        f = W.rhs_uniform(_np_shape(shape), 200 + i)
        out.append((shape, fields.get(fid), field, alpha, k, f))
    return out


def test_server_results_equal_direct_solves_and_oracle(lib):
    tol = 1e-6
    reqs = _requests()
    srv = lib.BuraServer(workers=4)
    try:
        ids, us = [], []
        for shape, faces, field, alpha, k, f in reqs:
            u = np.zeros_like(f)
            us.append(u)
            ids.append(srv.submit(shape, alpha, k, f, u, tol, faces=faces, field=field))
        infos = [srv.wait(i) for i in ids]
        st = srv.stats()
    finally:
        srv.close()
    assert all(inf["status"] == lib.BURA_OK for inf in infos), infos
    assert st["submitted"] == st["completed"] == len(reqs)
    assert st["builds"] >= 6 and st["builds"] + st["retargets"] + st["reuses"] == len(reqs)
    assert st["retargets"] + st["reuses"] >= 1
    for (shape, faces, field, alpha, k, f), u, inf in zip(reqs, us, infos):
        ud, rc = _direct(lib, shape, alpha, k, f, tol, faces)
        assert rc == lib.BURA_OK
        assert np.array_equal(u, ud), (shape, alpha, k, inf)
        assert _rel(u, _reference(shape, alpha, k, f, faces)) <= tol
        assert inf["total_ms"] >= inf["service_ms"] >= 0


def test_server_memory_budget_evicts_idle_plans(lib):
    """A budget of 1.1 plans of the larger class: each switch of class evicts the idle plan of the other
    class, and the results stay those of direct solves."""
    tol = 1e-6
    probe = lib.bura_setup((255, 255), 0.5, 7)
    one = lib.bura_get_stats(probe)["device_bytes"]
    lib.bura_destroy(probe)
    assert one > 0
    srv = lib.BuraServer(workers=1, mem_budget=int(one * 1.1))
    reqs = [((255, 255), 0.5, 7), ((255, 127), 0.25, 7), ((255, 255), 0.75, 7), ((255, 127), 0.5, 7)]
    try:
        outs = []
        for i, (shape, alpha, k) in enumerate(reqs):
            f = W.rhs_uniform(_np_shape(shape), 300 + i)
            u = np.zeros_like(f)
            rid = srv.submit(shape, alpha, k, f, u, tol)
            inf = srv.wait(rid)
            outs.append((shape, alpha, k, f, u, inf))
        st = srv.stats()
    finally:
        srv.close()
    assert st["evictions"] >= 3 and st["resident_plans"] == 1 and st["resident_bytes"] <= st["mem_budget"]
    for shape, alpha, k, f, u, inf in outs:
        assert inf["status"] == lib.BURA_OK and inf["built"] == 1
        ud, rc = _direct(lib, shape, alpha, k, f, tol)
        assert np.array_equal(u, ud)


def test_server_wait_timeout_and_unknown_id(lib):
    srv = lib.BuraServer(workers=2)
    try:
        f = W.rhs_uniform(_np_shape((127, 127)), 7)
        u = np.zeros_like(f)
        rid = srv.submit((127, 127), 0.5, 5, f, u, 1e-6)
        first = srv.wait(rid, timeout=0.0)
        info = first if first is not None else srv.wait(rid, timeout=60.0)
        assert info is not None and info["status"] == lib.BURA_OK
        with pytest.raises(lib.BuraError) as ei:
            srv.wait(rid)  # forgotten once reported
        assert ei.value.code == lib.BURA_EINVAL
        with pytest.raises(lib.BuraError):
            srv.submit((127, 127), 1.5, 5, f, u, 1e-6)
    finally:
        srv.close()
