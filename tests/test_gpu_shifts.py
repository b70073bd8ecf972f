"""GPU parity of the caller-given partial-fraction sums (through the C ABI) against the oracle.

  * the sinc quadrature of the paper's comparison method [BP15] (eq. (BonitoPasciak), Sec. 5.3) on the
    multi-shift solve: bura_quadrature_bp15 nodes, bura_setup_shifts, and bura_solve_sum when the nodes
    need more than one plan; the oracle is oracle.quadrature.bp15_value (DST eigenbasis);
  * the unscaled option: utilde = Lambda^-alpha u for Atilde^alpha utilde = ftilde (eq. (algebraic));
  * sums of BURA solves of several plans;
  * failure detection: a TMA wait budget shorter than a copy makes the solve return BURA_ETIMEOUT, and
    the same plan solves correctly again with the default budget.
Tolerances: FP64 1e-10 relative, mixed at the solve tolerance (||u_Q|| >= ||f|| on spec(A) in (0,1]).
"""
import numpy as np
import pytest

from oracle import exact, quadrature, tables
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


def _chunks(c, d, size):
    return [(c[i:i + size], d[i:i + size]) for i in range(0, len(c), size)]


@pytest.mark.parametrize("precision,tol,bound", [(0, 1e-11, 1e-10), (1, 1e-6, 1e-6)])
@pytest.mark.parametrize("alpha,kp", [(0.5, 1.0), (0.5, 0.7), (0.25, 0.8)])
def test_bp15_quadrature_matches_oracle(lib, precision, tol, bound, alpha, kp):
    """eq. (BonitoPasciak): the library's quadrature nodes solved on the multi-shift MG-PCG (split over
    plans of at most BURA_MAX_K + 1 systems, summed by bura_solve_sum) equal the oracle's u_Q."""
    shape = (255, 255)
    f = W.rhs_uniform(shape, 21)
    lam = lib.bura_scale(shape)
    c, d = lib.bura_quadrature_bp15(alpha, kp, lam)
    plans = [lib.bura_setup_shifts(shape, cc, dd, options=_opts(lib, precision))
             for cc, dd in _chunks(c, d, lib.BURA_MAX_K + 1)]
    try:
        fd = torch.from_numpy(f).cuda()
        ud = torch.zeros_like(fd)
        rc = lib.bura_solve_sum(plans, fd, ud, tol)
        torch.cuda.synchronize()
        assert rc == lib.BURA_OK
        uq = quadrature.bp15_value(shape, f, alpha, kp)
        err = _rel(ud.cpu().numpy(), uq)
        assert err <= bound, (err, len(c), len(plans))
        # the plan keeps its systems sorted by descending shift; E is 0 for caller-given shifts
        c0, d0, E0 = lib.bura_get_rational(plans[0], len(_chunks(c, d, lib.BURA_MAX_K + 1)[0][0]) - 1)
        assert E0 == 0.0 and np.all(np.diff(d0) <= 0)
    finally:
        for p in plans:
            lib.bura_destroy(p)


def test_bp15_plan_rejects_retarget(lib):
    plan = lib.bura_setup_shifts((31, 31), [1.0, 2.0], [-0.1, 0.0])
    try:
        with pytest.raises(lib.BuraError) as ei:
            lib.bura_retarget(plan, 0.5)
        assert ei.value.code == lib.BURA_EINVAL
    finally:
        lib.bura_destroy(plan)


@pytest.mark.parametrize("precision,tol,bound", [(0, 1e-11, 1e-10), (1, 1e-6, 1e-6)])
def test_unscaled_option_returns_the_unscaled_solution(lib, precision, tol, bound):
    """eq. (algebraic): Atilde = Lambda A, so Atilde^-alpha ftilde = Lambda^-alpha A^-alpha ftilde; with
    opt.unscaled the solve returns Lambda^-alpha u_r (u_r the exact BURA value), and u_r itself without."""
    shape, alpha, k = (127, 127), 0.5, 7
    f = W.rhs_uniform(shape, 22)
    e = tables.entry(alpha, k)
    ur = exact.bura_value(shape, f, e["c"], e["d"])
    lam = exact.gershgorin(shape)
    fd = torch.from_numpy(f).cuda()
    for unscaled, ref in ((0, ur), (1, lam ** -alpha * ur)):
        plan = lib.bura_setup(shape, alpha, k, options=_opts(lib, precision, unscaled=unscaled))
        try:
            ud = torch.zeros_like(fd)
            assert lib.bura_solve(plan, fd, ud, tol) == lib.BURA_OK
            torch.cuda.synchronize()
            assert _rel(ud.cpu().numpy(), ref) <= bound
            if unscaled:  # after a retarget the scale follows the new alpha
                lib.bura_retarget(plan, 0.25)
                assert lib.bura_solve(plan, fd, ud, tol) == lib.BURA_OK
                torch.cuda.synchronize()
                e2 = tables.entry(0.25, k)
                ref2 = lam ** -0.25 * exact.bura_value(shape, f, e2["c"], e2["d"])
                assert _rel(ud.cpu().numpy(), ref2) <= bound
        finally:
            lib.bura_destroy(plan)


def test_solve_sum_of_bura_plans(lib):
    """bura_solve_sum of two BURA plans is the sum of their exact BURA values (FP64, 1e-10)."""
    shape, k = (63, 63), 5
    f = W.rhs_uniform(shape, 23)
    plans = [lib.bura_setup(shape, a, k, options=_opts(lib, 0)) for a in (0.25, 0.75)]
    try:
        fd = torch.from_numpy(f).cuda()
        ud = torch.zeros_like(fd)
        assert lib.bura_solve_sum(plans, fd, ud, 1e-11) == lib.BURA_OK
        torch.cuda.synchronize()
        ref = sum(exact.bura_value(shape, f, tables.entry(a, k)["c"], tables.entry(a, k)["d"]) for a in (0.25, 0.75))
        assert _rel(ud.cpu().numpy(), ref) <= 1e-10
        with pytest.raises(lib.BuraError) as ei:  # f and u alias: the second term would read a written u
            lib.bura_solve_sum(plans, fd, fd, 1e-11)
        assert ei.value.code == lib.BURA_EINVAL
    finally:
        for p in plans:
            lib.bura_destroy(p)


def test_tma_wait_budget_times_out_and_the_plan_recovers(lib):
    """Failure detection of the TMA-staged sweeps: with a wait budget of 200 SM clocks (far below the
    latency of one tile copy) the waits give up, the kernels drain their copies in flight under the
    default budget and record a fault, and the solve returns BURA_ETIMEOUT; with the default budget the
    same plan then solves to the oracle's value."""
    shape, alpha, k, tol = (255, 255), 0.5, 7, 1e-6
    f = W.rhs_uniform(shape, 24)
    e = tables.entry(alpha, k)
    ur = exact.bura_value(shape, f, e["c"], e["d"])
    plan = lib.bura_setup(shape, alpha, k, options=_opts(lib, lib.BURA_PREC_MIXED))
    try:
        fd = torch.from_numpy(f).cuda()
        ud = torch.zeros_like(fd)
        assert lib.bura_solve(plan, fd, ud, tol) == lib.BURA_OK  # captures the PCG graph
        torch.cuda.synchronize()
        lib.bura_set_tma_wait_cycles(plan, 200)
        with pytest.raises(lib.BuraError) as ei:
            lib.bura_solve(plan, fd, ud, tol)
        assert ei.value.code == lib.BURA_ETIMEOUT
        torch.cuda.synchronize()
        lib.bura_set_tma_wait_cycles(plan, 0)
        ud.zero_()
        assert lib.bura_solve(plan, fd, ud, tol) == lib.BURA_OK
        torch.cuda.synchronize()
        assert _rel(ud.cpu().numpy(), ur) <= tol
    finally:
        lib.bura_destroy(plan)
