"""Audit of the CG dot products' accumulation in the FP32 inner solves (host only).

The FP32 kernels form each thread's products a_i b_i with fused multiply-adds into an FP32 partial,
fold that partial into an FP64 total after every 8 points, and sum the per-thread totals and the block
partials in FP64.  The emulation below reproduces that order for one system (threads striding over the
points as the grid sweeps do) in numpy (float32 fused products are formed exactly in float64 and
rounded once, which is what a fused multiply-add does), and checks it against

    |dot_kernel - dot| <= 8 u32 sum_i |a_i b_i| + (n / 8 + threads) u64 sum_i |a_i b_i|,

u32 = 2^-24, u64 = 2^-53 (each FP32 partial sums at most 8 rounded products; the FP64 stages add
lower-order terms).  For the inner products of preconditioned CG (r . z with z = M r, M symmetric
positive definite; p . (A - d I) p) sum |a_i b_i| is within a small factor of the dot itself on these
operators, so the relative error is about 1e-6: two orders below the FP32 inner solve's own target
(1e-5 per refinement step).  The FP64 refinement recomputes the true residual, so the error of an inner
dot can change an inner iterate, never the accuracy the stopping rule certifies.
"""
import numpy as np
import pytest

from oracle import operators
from paper_1612_04846_gb300 import workloads as W


def kernel_order_dot(a, b, threads, fold=8):
    """The FP32 kernels' order for one system: thread t takes points t, t + threads, ...; its FP32
    partial takes fold fused products at a time, each partial is added to the thread's FP64 total, and
    the thread totals are summed in FP64."""
    a = np.asarray(a, np.float32)
    b = np.asarray(b, np.float32)
    n = a.size
    pad = (-n) % (threads * fold)
    a = np.concatenate([a, np.zeros(pad, np.float32)])
    b = np.concatenate([b, np.zeros(pad, np.float32)])
    A = a.reshape(-1, threads).astype(np.float64)  # row s: the s-th point of every thread
    B = b.reshape(-1, threads).astype(np.float64)
    tot = np.zeros(threads)
    part = np.zeros(threads, np.float32)
    for s in range(A.shape[0]):
        # fmaf(a, b, part): the exact product plus the partial, rounded once to FP32
        part = (A[s] * B[s] + part.astype(np.float64)).astype(np.float32)
        if s % fold == fold - 1:
            tot += part.astype(np.float64)
            part = np.zeros(threads, np.float32)
    tot += part.astype(np.float64)
    return float(np.sum(tot))


def _bound(a, b, threads, fold=8):
    s = float(np.sum(np.abs(np.asarray(a, np.float64) * np.asarray(b, np.float64))))
    return fold * 2.0 ** -24 * s + (a.size / fold + threads) * 2.0 ** -53 * s


@pytest.mark.parametrize("n,threads,seed", [(4096, 256, 0), (65025, 1024, 1), (261121, 4864, 2)])
def test_fp32_partial_dot_within_its_bound(n, threads, seed):
    rng = np.random.default_rng(seed)
    a = rng.standard_normal(n).astype(np.float32)
    b = (a * rng.uniform(0.5, 1.5, n)).astype(np.float32)  # correlated, like r and M r
    exact = float(np.dot(a.astype(np.float64), b.astype(np.float64)))
    got = kernel_order_dot(a, b, threads)
    assert abs(got - exact) <= _bound(a, b, threads)


def test_cg_inner_products_relative_error_is_far_below_the_inner_target():
    """r . z and p . A p on the 5-point operator of a 511^2 grid with r from the workload generator and z
    from a few Jacobi sweeps (a symmetric positive definite stand-in for the V-cycle), 16 points per
    thread as in the level-0 sweeps of a 1023^2 solve: the kernels' accumulation order stays within 1e-6
    relative, against the inner solve's target of 1e-5."""
    shape = (511, 511)
    A, _ = operators.scaled_matrix(shape)
    r = W.rhs_uniform(shape, 7).astype(np.float32).astype(np.float64)
    dinv = 1.0 / A.diagonal()
    z = np.zeros_like(r)
    for _ in range(4):  # damped Jacobi from zero: z = p(D^-1 A) D^-1 r, symmetric positive definite in r
        z = z + 0.5 * dinv * (r - A @ z)
    z32 = z.astype(np.float32)
    Az = (A @ z32.astype(np.float64)).astype(np.float32)
    threads = r.size // 16
    for a, b in ((r.astype(np.float32), z32), (z32, Az)):
        exact = float(np.dot(a.astype(np.float64), b.astype(np.float64)))
        got = kernel_order_dot(a, b, threads)
        assert exact > 0
        assert abs(got - exact) <= _bound(a, b, threads)
        assert abs(got - exact) / exact <= 1e-6


def test_the_emulation_detects_a_plain_fp32_running_sum():
    """The emulation is sensitive to the order it claims: a plain FP32 running sum over a long vector
    (no FP64 folding) breaks the same bound, so the bound is not vacuous."""
    n = 1 << 20
    a = np.full(n, 1.0 + 2.0 ** -12, np.float32)
    b = np.ones(n, np.float32)
    exact = float(np.dot(a.astype(np.float64), b.astype(np.float64)))
    plain = float(np.cumsum(a * b, dtype=np.float32)[-1])
    assert abs(plain - exact) > _bound(a, b, 1024)
    assert abs(kernel_order_dot(a, b, 1024) - exact) <= _bound(a, b, 1024)
