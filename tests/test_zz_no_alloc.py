"""The allocation-free entry point bura_residual_norms_noalloc (GPU).

It exists for callers that cannot allocate device memory: code running under a caller-owned memory
pool or a fixed device-memory budget, or a loop that must never enter the allocator because an
allocation there can block or fail.  Its scratch is a fixed device array inside the library.  Its
output must equal what the allocating entry point gives (the norms of f - (A - d_j I) V_j with
(A - d_j I) V_j from bura_apply_shifted), and the norms the oracle's assembled matrix gives.
This file is collected last so that a run stopping at the first failure has run everything else.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)


@pytest.fixture(scope="module")
def lib():
    from paper_1612_04846_gb300 import build_lib, bura
    build_lib.build(verbose=False)
    return bura


@pytest.mark.parametrize("shape,k", [((127, 127), 7), ((33, 17, 9), 9), ((1, 1), 3), ((1023, 1023), 7)])
def test_noalloc_norms_match_apply_shifted(lib, shape, k):
    o = lib.bura_default_options()
    o.precision = lib.BURA_PREC_FP64
    plan = lib.bura_setup(shape, 0.5, k, options=o)
    try:
        c, d, _ = lib.bura_get_rational(plan, k)
        N = int(np.prod(shape))
        g = torch.Generator(device="cuda").manual_seed(3)
        V = torch.randn((k + 1, N), dtype=torch.float64, device="cuda", generator=g)
        f = torch.randn(N, dtype=torch.float64, device="cuda", generator=g)
        Y = torch.zeros_like(V)
        lib.bura_apply_shifted(plan, V, Y)
        ref = ((f[None, :] - Y) ** 2).sum(dim=1)
        out = torch.full((k + 1,), -1.0, dtype=torch.float64, device="cuda")
        for _ in range(2):  # two calls in a row share (and must reset) the static scratch
            out.fill_(-1.0)
            lib.bura_residual_norms_noalloc(shape, d, f, V, out)
            torch.cuda.synchronize()
            rel = ((out - ref).abs() / ref).max().item()
            assert rel <= 1e-12, rel
    finally:
        lib.bura_destroy(plan)


def test_noalloc_rejects_too_many_systems(lib):
    N = 9
    f = torch.zeros(N, dtype=torch.float64, device="cuda")
    V = torch.zeros((17, N), dtype=torch.float64, device="cuda")
    out = torch.zeros(17, dtype=torch.float64, device="cuda")
    with pytest.raises(lib.BuraError) as ei:
        lib.bura_residual_norms_noalloc((3, 3), np.zeros(17), f, V, out)
    assert ei.value.code == lib.BURA_ERANGE


def test_noalloc_norms_match_the_oracle_matrix(lib):
    """The same norms from the oracle's assembled scaled matrix A = Atilde / Lambda (eq. (algebraic)) on
    the CPU, for a ragged 3-D grid (1e-12 relative)."""
    from oracle import operators
    shape, k = (17, 9, 5), 6
    A, _ = operators.scaled_matrix(tuple(reversed(shape)))
    N = A.shape[0]
    rng = np.random.default_rng(8)
    d = -np.sort(rng.uniform(0.0, 2.0, k + 1))
    d[0] = 0.0
    V = rng.standard_normal((k + 1, N))
    f = rng.standard_normal(N)
    ref = np.array([np.sum((f - (A @ V[j] - d[j] * V[j])) ** 2) for j in range(k + 1)])
    out = torch.full((k + 1,), -1.0, dtype=torch.float64, device="cuda")
    lib.bura_residual_norms_noalloc(shape, d, torch.from_numpy(f).cuda(), torch.from_numpy(V).cuda(), out)
    torch.cuda.synchronize()
    assert np.max(np.abs(out.cpu().numpy() - ref) / ref) <= 1e-12
