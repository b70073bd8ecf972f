"""Multi-step BURA through bura_solve_chain on the GPU (Sec. "Multi-step BURA approximation").

Each step is a BURA solve meeting tol relative to its input; a step's error then passes through the
later steps' r_j(A) A^{-1}, of norm at most lambda_min^{-alpha_j}.  The chain must match the oracle's
exact multi-step value within that bound, and its error against A^{-alpha} f in the ratio of
eq. (errorU) must stay within E_{alpha_1..alpha_n} of eq. (multi-step error).
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


@pytest.mark.parametrize("shape,alphas,precision,tol", [((63, 63), (0.25, 0.25), "FP64", 1e-11),
                                                        ((127, 127), (0.1, 0.25, 0.25), "FP64", 1e-11),
                                                        ((255, 255), (0.25, 0.5), "MIXED", 1e-7),
                                                        ((31, 31, 31), (0.25, 0.25), "MIXED", 1e-7)])
def test_chain_matches_the_multistep_oracle(lib, shape, alphas, precision, tol):
    k = 7
    nps = tuple(reversed(shape))
    f = W.rhs_uniform(nps, 17)
    o = lib.bura_default_options()
    o.precision = getattr(lib, "BURA_PREC_" + precision)
    plans = [lib.bura_setup(shape, a, k, options=o) for a in alphas]
    try:
        fd = torch.from_numpy(f).cuda()
        ud = torch.zeros_like(fd)
        assert lib.bura_solve_chain(plans, fd, ud, tol) == lib.BURA_OK
        torch.cuda.synchronize()
        u = ud.cpu().numpy()
    finally:
        for p in plans:
            lib.bura_destroy(p)
    steps = [(tables.entry(a, k)["c"], tables.entry(a, k)["d"]) for a in alphas]
    ref = exact.multistep_value(nps, f, steps)
    lam_min = float(np.min(exact.eigenvalues(nps)))
    alpha = sum(alphas)
    # step i's error (<= tol times its input, whose norm is <= lam_min^-(alpha_1+..+alpha_{i-1}) ||f||)
    # grows by at most lam_min^-(alpha_{i+1}+..+alpha_n) afterwards; ||ref|| >= ||f||
    bound = tol * len(alphas) * lam_min ** (-(alpha - min(alphas)))
    err = float(np.linalg.norm(u - ref) / np.linalg.norm(ref))
    assert err <= bound, (err, bound)
    ratio = exact.energy_ratio(nps, f, u, alpha)
    assert ratio <= exact.multistep_error(nps, steps, alpha) * (1 + 1e-6) + bound


def test_f_reconstruction_on_a_variable_3d_operator(lib):
    """Sec. "1D and 3D numerical tests": with no exact solution, f_r = A u_2 (u_2 the two-step chain at
    alpha and 1 - alpha) must satisfy ||f_r - f|| / ||A^{-1} f|| <= E_{1-alpha} + E_alpha - E_{1-alpha} E_alpha
    (eq. (3D error final)).  A u_2 comes from the plan's shifted operator (system 0, d_0 = 0) and A^{-1} f
    from system 0 of bura_solve_systems, all through the library."""
    shape, alpha, k, tol = (31, 31, 31), 0.25, 7, 1e-11
    nps = tuple(reversed(shape))
    faces = W.block_lognormal_faces(nps, 8, 1e-2, 1.0, 2)
    f = W.rhs_normal(nps, 3)
    o = lib.bura_default_options()
    o.precision = lib.BURA_PREC_FP64
    plans = [lib.bura_setup(shape, a, k, faces=faces, options=o) for a in (alpha, 1.0 - alpha)]
    try:
        N = f.size
        fd = torch.from_numpy(f).cuda()
        u = torch.zeros_like(fd)
        assert lib.bura_solve_chain(plans, fd, u, tol) == lib.BURA_OK
        X = torch.zeros((k + 1, N), dtype=torch.float64, device="cuda")
        X[0] = u
        Y = torch.zeros_like(X)
        lib.bura_apply_shifted(plans[0], X, Y)
        V = torch.zeros_like(X)
        lib.bura_solve_systems(plans[0], fd, V, tol)
        torch.cuda.synchronize()
        fr, v0 = Y[0].cpu().numpy(), V[0].cpu().numpy()
    finally:
        for p in plans:
            lib.bura_destroy(p)
    ratio = float(np.linalg.norm(fr - f) / np.linalg.norm(v0))
    E1, E2 = tables.entry(alpha, k)["E"], tables.entry(1.0 - alpha, k)["E"]
    assert 0 < ratio <= (E1 + E2 - E1 * E2) * (1 + 1e-6), (ratio, E1 + E2 - E1 * E2, E1 * E2)
