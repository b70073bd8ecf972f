"""Thin ctypes binding of the C ABI in include/bura.h (argument marshalling only).

Every function has the name of its C entry point.  Device buffers are passed as
torch CUDA tensors (their data_ptr()), host buffers as numpy arrays, and streams as
torch.cuda.Stream objects or raw cudaStream_t integers.  Nothing here computes: the
solver runs in libbura.so, and importing this module fails loudly if the library is
missing (there is no CPU fallback).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libbura.so")

BURA_MAX_K = 12
BURA_OK, BURA_EINVAL, BURA_ENOMEM, BURA_EREMEZ = 0, -1, -2, -3
BURA_ENOTSPD, BURA_ENOCONV, BURA_ETIMEOUT, BURA_ECUDA, BURA_ERANGE = -4, -5, -6, -7, -8
BURA_COEF_CONSTANT, BURA_COEF_FACES = 0, 1
BURA_PREC_FP64, BURA_PREC_MIXED = 0, 1
BURA_COARSE_AUTO, BURA_COARSE_CLUSTER, BURA_COARSE_CTA, BURA_COARSE_NONE, BURA_COARSE_FDIAG = 0, 1, 2, 3, 4
BURA_SWEEP_AUTO, BURA_SWEEP_GRID = 0, 1
BURA_REFINE_FP64, BURA_REFINE_DF = 0, 1


class bura_grid(C.Structure):
    _fields_ = [("dim", C.c_int), ("n", C.c_int * 3), ("coef_kind", C.c_int)]


class bura_options(C.Structure):
    _fields_ = [("precision", C.c_int), ("smoother_degree", C.c_int), ("smoother_ratio", C.c_double),
                ("max_iters", C.c_int), ("max_outer", C.c_int), ("inner_rtol", C.c_double),
                ("coarse_degree", C.c_int), ("block_points", C.c_int), ("blocks_per_sm", C.c_int),
                ("coarse_kernel", C.c_int), ("cluster_size", C.c_int), ("sweeps", C.c_int),
                ("refine", C.c_int), ("tma_stages", C.c_int), ("post_smooth_split", C.c_int),
                ("unscaled", C.c_int), ("tma_wait_cycles", C.c_longlong), ("smoother_bf16", C.c_int)]


class bura_csr(C.Structure):
    _fields_ = [("n", C.c_int), ("nnz", C.c_longlong), ("row_ptr", C.POINTER(C.c_int)), ("col", C.POINTER(C.c_int)),
                ("val", C.POINTER(C.c_double)), ("lambda_min", C.c_double)]


class bura_stats(C.Structure):
    _fields_ = [("Lambda", C.c_double), ("E", C.c_double), ("k", C.c_int), ("levels", C.c_int),
                ("iters", C.c_int), ("outer", C.c_int), ("shift_iters", C.c_int * (BURA_MAX_K + 1)),
                ("rel_res", C.c_double * (BURA_MAX_K + 1)), ("err_bound", C.c_double),
                ("lambda_lo", C.c_double), ("launches", C.c_longlong), ("device_bytes", C.c_size_t)]

    def to_dict(self):
        k = self.k
        return {"Lambda": self.Lambda, "E": self.E, "k": k, "levels": self.levels, "iters": self.iters,
                "outer": self.outer, "shift_iters": list(self.shift_iters)[: k + 1],
                "rel_res": list(self.rel_res)[: k + 1], "err_bound": self.err_bound, "lambda_lo": self.lambda_lo,
                "launches": self.launches, "device_bytes": self.device_bytes}


class bura_server_options(C.Structure):
    _fields_ = [("workers", C.c_int), ("mem_budget", C.c_size_t), ("plan", bura_options)]


class bura_request(C.Structure):
    _fields_ = [("grid", bura_grid), ("faces", C.POINTER(C.POINTER(C.c_double))), ("field", C.c_ulonglong),
                ("alpha", C.c_double), ("k", C.c_int), ("tol", C.c_double), ("f", C.POINTER(C.c_double)),
                ("u", C.POINTER(C.c_double))]


class bura_request_info(C.Structure):
    _fields_ = [("status", C.c_int), ("built", C.c_int), ("retargeted", C.c_int), ("iters", C.c_int),
                ("outer", C.c_int), ("err_bound", C.c_double), ("queue_ms", C.c_double), ("service_ms", C.c_double),
                ("total_ms", C.c_double)]

    def to_dict(self):
        return {n: getattr(self, n) for n, _ in self._fields_}


class bura_server_stats(C.Structure):
    _fields_ = [("submitted", C.c_longlong), ("completed", C.c_longlong), ("builds", C.c_longlong),
                ("retargets", C.c_longlong), ("reuses", C.c_longlong), ("evictions", C.c_longlong),
                ("resident_plans", C.c_int), ("resident_bytes", C.c_size_t), ("mem_budget", C.c_size_t)]

    def to_dict(self):
        return {n: getattr(self, n) for n, _ in self._fields_}


class bura_kernel_prof(C.Structure):
    _fields_ = [("name", C.c_char_p), ("launches", C.c_longlong), ("ms", C.c_double), ("bytes", C.c_double)]


class BuraError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        msg = "%s failed: %s (%d)" % (where, _lib().bura_strerror(code).decode(), code)
        if code in (BURA_ECUDA, BURA_ENOMEM):
            msg += " [%s]" % _lib().bura_last_cuda_error().decode()
        super().__init__(msg)


_LIB = None


def _lib():
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("libbura.so is not built (run __graft_entry__.build()); there is no CPU fallback")
        L = C.CDLL(LIB_PATH)
        P = C.c_void_p
        D = C.c_double
        I = C.c_int
        dp = C.POINTER(C.c_double)
        L.bura_default_options.argtypes = [C.POINTER(bura_options)]
        L.bura_default_options.restype = None
        L.bura_rational.argtypes = [D, I, dp, dp, dp]
        L.bura_setup.argtypes = [C.POINTER(bura_grid), C.POINTER(dp), D, I, C.POINTER(bura_options),
                                 C.POINTER(P)]
        L.bura_solve.argtypes = [P, P, P, D, P]
        L.bura_solve_host.argtypes = [P, dp, dp, D, P]
        L.bura_solve_async.argtypes = [P, P, P, D, P]
        L.bura_solve_wait.argtypes = [P]
        L.bura_batch_create.argtypes = [C.POINTER(P), C.POINTER(P), C.POINTER(P), I, D, I, C.POINTER(P)]
        L.bura_batch_run.argtypes = [P, P]
        L.bura_batch_wait.argtypes = [P, C.POINTER(I)]
        L.bura_batch_destroy.argtypes = [P]
        L.bura_autotune.argtypes = [C.POINTER(bura_grid), C.POINTER(dp), D, I, C.POINTER(bura_options), D, I,
                                    C.POINTER(bura_options), dp]
        L.bura_solve_systems.argtypes = [P, P, P, D, P]
        L.bura_apply_shifted.argtypes = [P, P, P, P]
        L.bura_get_rational.argtypes = [P, dp, dp, dp]
        L.bura_get_stats.argtypes = [P, C.POINTER(bura_stats)]
        L.bura_destroy.argtypes = [P]
        L.bura_residual_norms_noalloc.argtypes = [C.POINTER(bura_grid), I, dp, P, P, P, P]
        L.bura_solve_batch.argtypes = [C.POINTER(P), C.POINTER(P), C.POINTER(P), I, D, I, C.POINTER(I)]
        L.bura_set_profiling.argtypes = [P, I]
        L.bura_get_profile.argtypes = [P, I, C.POINTER(bura_kernel_prof), C.POINTER(I)]
        L.bura_retarget.argtypes = [P, D]
        L.bura_solve_chain.argtypes = [C.POINTER(P), I, P, P, D, P]
        L.bura_setup_shifts.argtypes = [C.POINTER(bura_grid), C.POINTER(dp), I, dp, dp, C.POINTER(bura_options),
                                        C.POINTER(P)]
        L.bura_solve_sum.argtypes = [C.POINTER(P), I, P, P, D, P]
        L.bura_scale.argtypes = [C.POINTER(bura_grid), C.POINTER(dp), dp]
        L.bura_setup_csr.argtypes = [C.POINTER(bura_csr), D, I, C.POINTER(bura_options), C.POINTER(P)]
        L.bura_quadrature_bp15.argtypes = [D, D, D, I, dp, dp, C.POINTER(I)]
        L.bura_set_tma_wait_cycles.argtypes = [P, C.c_longlong]
        L.bura_server_default_options.argtypes = [C.POINTER(bura_server_options)]
        L.bura_server_default_options.restype = None
        L.bura_server_create.argtypes = [C.POINTER(bura_server_options), C.POINTER(P)]
        L.bura_server_submit.argtypes = [P, C.POINTER(bura_request), C.POINTER(C.c_ulonglong)]
        L.bura_server_wait.argtypes = [P, C.c_ulonglong, D, C.POINTER(bura_request_info)]
        L.bura_server_get_stats.argtypes = [P, C.POINTER(bura_server_stats)]
        L.bura_server_destroy.argtypes = [P]
        L.bura_strerror.argtypes = [I]
        L.bura_strerror.restype = C.c_char_p
        L.bura_last_cuda_error.argtypes = []
        L.bura_last_cuda_error.restype = C.c_char_p
        for name in ("bura_rational", "bura_setup", "bura_solve", "bura_solve_host", "bura_solve_systems",
                     "bura_apply_shifted", "bura_get_rational", "bura_get_stats", "bura_destroy",
                     "bura_set_profiling", "bura_get_profile", "bura_residual_norms_noalloc",
                     "bura_solve_batch", "bura_retarget", "bura_solve_chain", "bura_setup_shifts", "bura_solve_sum",
                     "bura_set_tma_wait_cycles", "bura_scale", "bura_quadrature_bp15", "bura_setup_csr", "bura_solve_async",
                     "bura_solve_wait", "bura_batch_create", "bura_batch_run", "bura_batch_wait", "bura_batch_destroy",
                     "bura_autotune", "bura_server_create", "bura_server_submit",
                     "bura_server_wait", "bura_server_get_stats", "bura_server_destroy"):
            getattr(L, name).restype = I
        _LIB = L
    return _LIB


def _check(rc, where, allow=()):
    if rc != BURA_OK and rc not in allow:
        raise BuraError(rc, where)
    return rc


def _dptr(t):
    """Device pointer of a contiguous float64 torch CUDA tensor."""
    if not (t.is_cuda and t.is_contiguous() and str(t.dtype) == "torch.float64"):
        raise ValueError("expected a contiguous float64 CUDA tensor")
    return C.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        return C.c_void_p(0)
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


def _hptr(a):
    if not (isinstance(a, np.ndarray) and a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]):
        raise ValueError("expected a C-contiguous float64 numpy array")
    return a.ctypes.data_as(C.POINTER(C.c_double))


def bura_default_options():
    o = bura_options()
    _lib().bura_default_options(C.byref(o))
    return o


def bura_strerror(code):
    return _lib().bura_strerror(int(code)).decode()


def bura_rational(alpha, k):
    """(c, d, E) of the library's BURA of t^(1-alpha), k+1 coefficients each."""
    c = np.zeros(k + 1)
    d = np.zeros(k + 1)
    E = C.c_double()
    _check(_lib().bura_rational(float(alpha), int(k), _hptr(c), _hptr(d), C.byref(E)), "bura_rational")
    return c, d, E.value


def _faces_arg(faces, keep):
    if faces is None:
        return None
    arr = (C.POINTER(C.c_double) * len(faces))()
    for i, a in enumerate(faces):
        a = np.ascontiguousarray(a, dtype=np.float64)
        keep.append(a)
        arr[i] = _hptr(a)
    keep.append(arr)
    return C.cast(arr, C.POINTER(C.POINTER(C.c_double)))


def bura_setup(shape, alpha, k, faces=None, options=None):
    """Plan for an interior grid ``shape`` = (nx, ny) or (nx, ny, nz).

    faces: None (a = 1) or a tuple of float64 arrays (ax, ay[, az]) with the shapes of
    include/bura.h (numpy C order (nz, ny, nx+1) etc.).  Returns an opaque plan handle.
    """
    g = _grid_of(shape, faces)
    keep = []
    fptr = _faces_arg(faces, keep)
    opt = options if options is not None else bura_default_options()
    plan = C.c_void_p()
    _check(_lib().bura_setup(C.byref(g), fptr, float(alpha), int(k), C.byref(opt), C.byref(plan)), "bura_setup")
    return plan


def bura_setup_shifts(shape, c, d, faces=None, options=None):
    """Plan for u = sum_j c[j] (A - d[j] I)^{-1} f with caller-given weights c > 0 and shifts d <= 0."""
    g = _grid_of(shape, faces)
    keep = []
    fptr = _faces_arg(faces, keep)
    c = np.ascontiguousarray(c, dtype=np.float64)
    d = np.ascontiguousarray(d, dtype=np.float64)
    if c.shape != d.shape or c.ndim != 1:
        raise ValueError("c and d must be 1-D arrays of one length")
    opt = options if options is not None else bura_default_options()
    plan = C.c_void_p()
    _check(_lib().bura_setup_shifts(C.byref(g), fptr, int(c.size), _hptr(c), _hptr(d), C.byref(opt), C.byref(plan)),
           "bura_setup_shifts")
    return plan


def bura_setup_csr(indptr, indices, data, alpha, k, lambda_min=0.0, options=None):
    """Plan for the sparse SPD matrix Atilde given by its CSR arrays (row offsets, columns, values; e.g. a
    scipy.sparse.csr_matrix's indptr, indices, data).  lambda_min: a lower bound on its smallest
    eigenvalue, or 0."""
    rp = np.ascontiguousarray(indptr, dtype=np.int32)
    ci = np.ascontiguousarray(indices, dtype=np.int32)
    va = np.ascontiguousarray(data, dtype=np.float64)
    A = bura_csr()
    A.n = int(rp.size - 1)
    A.nnz = int(ci.size)
    A.row_ptr = rp.ctypes.data_as(C.POINTER(C.c_int))
    A.col = ci.ctypes.data_as(C.POINTER(C.c_int))
    A.val = _hptr(va)
    A.lambda_min = float(lambda_min)
    opt = options if options is not None else bura_default_options()
    plan = C.c_void_p()
    _check(_lib().bura_setup_csr(C.byref(A), float(alpha), int(k), C.byref(opt), C.byref(plan)), "bura_setup_csr")
    return plan


def bura_scale(shape, faces=None):
    """Lambda of the grid's operator (host only)."""
    g = _grid_of(shape, faces)
    keep = []
    fptr = _faces_arg(faces, keep)
    lam = C.c_double()
    _check(_lib().bura_scale(C.byref(g), fptr, C.byref(lam)), "bura_scale")
    return lam.value


def bura_quadrature_bp15(alpha, kprime, Lam):
    """(c, d) of the [BP15] sinc quadrature for the scaled operator (host only)."""
    n = C.c_int()
    rc = _lib().bura_quadrature_bp15(float(alpha), float(kprime), float(Lam), 0, None, None, C.byref(n))
    if rc not in (BURA_OK, BURA_ERANGE):
        raise BuraError(rc, "bura_quadrature_bp15")
    c = np.zeros(n.value)
    d = np.zeros(n.value)
    _check(_lib().bura_quadrature_bp15(float(alpha), float(kprime), float(Lam), n.value, _hptr(c), _hptr(d),
                                       C.byref(n)), "bura_quadrature_bp15")
    return c, d


def bura_solve_sum(plans, f, u, tol, stream=None):
    """u = the sum of the plans' partial-fraction solves of f (device float64 tensors f, u)."""
    P = C.c_void_p
    pa = (P * max(len(plans), 1))(*[C.cast(p, P) for p in plans])
    return _check(_lib().bura_solve_sum(pa, int(len(plans)), _dptr(f), _dptr(u), float(tol), _stream(stream)),
                  "bura_solve_sum", allow=(BURA_ENOCONV,))


def bura_set_tma_wait_cycles(plan, cycles):
    """Budget of the TMA ring waits of later solves of the plan (0: the default)."""
    return _check(_lib().bura_set_tma_wait_cycles(plan, int(cycles)), "bura_set_tma_wait_cycles")


def bura_solve(plan, f, u, tol, stream=None):
    """u = sum_j c_j (A - d_j I)^{-1} f on the device (torch float64 CUDA tensors); returns the status."""
    return _check(_lib().bura_solve(plan, _dptr(f), _dptr(u), float(tol), _stream(stream)), "bura_solve",
                  allow=(BURA_ENOCONV,))


def bura_solve_async(plan, f, u, tol, stream=None):
    """Enqueue u = sum_j c_j (A - d_j I)^{-1} f without waiting (device float64 tensors)."""
    return _check(_lib().bura_solve_async(plan, _dptr(f), _dptr(u), float(tol), _stream(stream)), "bura_solve_async")


def bura_solve_wait(plan):
    """Status of the plan's last solve (waits for it); raises on an error other than BURA_ENOCONV."""
    return _check(_lib().bura_solve_wait(plan), "bura_solve_wait", allow=(BURA_ENOCONV,))


def bura_solve_batch(plans, fs, us, tol, nworkers=0):
    """Solve len(plans) independent problems concurrently (device float64 tensors fs[i], us[i]).
    Returns the list of per-problem statuses; raises on an error other than BURA_ENOCONV."""
    n = len(plans)
    if len(fs) != n or len(us) != n:
        raise ValueError("plans, fs and us must have the same length")
    P = C.c_void_p
    pa = (P * max(n, 1))(*[C.cast(p, P) for p in plans])
    fa = (P * max(n, 1))(*[_dptr(t) for t in fs])
    ua = (P * max(n, 1))(*[_dptr(t) for t in us])
    st = (C.c_int * max(n, 1))()
    _check(_lib().bura_solve_batch(pa, fa, ua, int(n), float(tol), int(nworkers), st), "bura_solve_batch",
           allow=(BURA_ENOCONV,))
    return list(st)[:n]


def bura_autotune(shape, alpha, k, tol=1e-6, trials=3, faces=None, base=None):
    """(best bura_options, median ms) over the library's candidate option sets for this problem class."""
    g = _grid_of(shape, faces)
    keep = []
    fptr = _faces_arg(faces, keep)
    b = base if base is not None else bura_default_options()
    best = bura_options()
    ms = C.c_double()
    _check(_lib().bura_autotune(C.byref(g), fptr, float(alpha), int(k), C.byref(b), float(tol), int(trials),
                                C.byref(best), C.byref(ms)), "bura_autotune")
    return best, ms.value


class BuraBatch:
    """bura_batch_create / _run / _wait / _destroy: a batch of (plan, f, u) captured once as one graph."""

    def __init__(self, plans, fs, us, tol, branches=0):
        n = len(plans)
        if len(fs) != n or len(us) != n or n == 0:
            raise ValueError("plans, fs and us must have the same nonzero length")
        P = C.c_void_p
        self._keep = (list(fs), list(us))
        pa = (P * n)(*[C.cast(p, P) for p in plans])
        fa = (P * n)(*[_dptr(t) for t in fs])
        ua = (P * n)(*[_dptr(t) for t in us])
        self.n = n
        self.b = C.c_void_p()
        _check(_lib().bura_batch_create(pa, fa, ua, int(n), float(tol), int(branches), C.byref(self.b)),
               "bura_batch_create")

    def run(self, stream=None):
        return _check(_lib().bura_batch_run(self.b, _stream(stream)), "bura_batch_run")

    def wait(self):
        st = (C.c_int * self.n)()
        _check(_lib().bura_batch_wait(self.b, st), "bura_batch_wait", allow=(BURA_ENOCONV,))
        return list(st)

    def close(self):
        if self.b is not None:
            _lib().bura_batch_destroy(self.b)
            self.b = None


def bura_solve_chain(plans, f, u, tol, stream=None):
    """Multi-step BURA: the plans' BURA solves applied in order to f (device float64 tensors f, u)."""
    P = C.c_void_p
    pa = (P * max(len(plans), 1))(*[C.cast(p, P) for p in plans])
    return _check(_lib().bura_solve_chain(pa, int(len(plans)), _dptr(f), _dptr(u), float(tol), _stream(stream)),
                  "bura_solve_chain", allow=(BURA_ENOCONV,))


def bura_retarget(plan, alpha):
    """Move the plan to another alpha (new rational approximation and shift tables, same hierarchy)."""
    return _check(_lib().bura_retarget(plan, float(alpha)), "bura_retarget")


def _grid_of(shape, faces):
    g = bura_grid()
    g.dim = len(shape)
    for i, n in enumerate(shape[:3]):
        g.n[i] = int(n)
    g.coef_kind = BURA_COEF_CONSTANT if faces is None else BURA_COEF_FACES
    return g


def bura_server_default_options():
    o = bura_server_options()
    _lib().bura_server_default_options(C.byref(o))
    return o


def bura_server_create(options=None):
    opt = options if options is not None else bura_server_default_options()
    srv = C.c_void_p()
    _check(_lib().bura_server_create(C.byref(opt), C.byref(srv)), "bura_server_create")
    return srv


def bura_server_submit(srv, req):
    """Queue a filled bura_request; returns its id.  The arrays it points to must stay alive until
    bura_server_wait reports it done (BuraServer keeps them)."""
    rid = C.c_ulonglong()
    _check(_lib().bura_server_submit(srv, C.byref(req), C.byref(rid)), "bura_server_submit")
    return rid.value


def bura_server_wait(srv, rid, timeout=-1.0):
    """The request's bura_request_info as a dict once done; None if not done within timeout seconds."""
    info = bura_request_info()
    rc = _check(_lib().bura_server_wait(srv, C.c_ulonglong(rid), float(timeout), C.byref(info)),
                "bura_server_wait", allow=(BURA_ETIMEOUT,))
    return None if rc == BURA_ETIMEOUT else info.to_dict()


def bura_server_get_stats(srv):
    st = bura_server_stats()
    _check(_lib().bura_server_get_stats(srv, C.byref(st)), "bura_server_get_stats")
    return st.to_dict()


def bura_server_destroy(srv):
    return _check(_lib().bura_server_destroy(srv), "bura_server_destroy")


class BuraServer:
    """The solve server with host numpy arrays: submit() keeps f, u and the faces alive until wait()."""

    def __init__(self, workers=0, mem_budget=0, options=None):
        o = bura_server_default_options()
        o.workers = int(workers)
        o.mem_budget = int(mem_budget)
        if options is not None:
            o.plan = options
        self.srv = bura_server_create(o)
        self._keep = {}

    def submit(self, shape, alpha, k, f, u, tol, faces=None, field=0):
        req = bura_request()
        req.grid = _grid_of(shape, faces)
        keep = [f, u]
        if faces is not None:
            arr = (C.POINTER(C.c_double) * len(faces))()
            for i, a in enumerate(faces):
                a = np.ascontiguousarray(a, dtype=np.float64)
                keep.append(a)
                arr[i] = _hptr(a)
            keep.append(arr)
            req.faces = C.cast(arr, C.POINTER(C.POINTER(C.c_double)))
        req.field = int(field)
        req.alpha = float(alpha)
        req.k = int(k)
        req.tol = float(tol)
        req.f = _hptr(f)
        req.u = _hptr(u)
        rid = bura_server_submit(self.srv, req)
        self._keep[rid] = (keep, req)
        return rid

    def wait(self, rid, timeout=-1.0):
        info = bura_server_wait(self.srv, rid, timeout)
        if info is not None:
            self._keep.pop(rid, None)
        return info

    def stats(self):
        return bura_server_get_stats(self.srv)

    def close(self):
        if self.srv is not None:
            bura_server_destroy(self.srv)
            self.srv = None
            self._keep.clear()


def bura_solve_host(plan, f, u, tol, stream=None):
    """Same with host numpy arrays (copies inside the call)."""
    return _check(_lib().bura_solve_host(plan, _hptr(f), _hptr(u), float(tol), _stream(stream)),
                  "bura_solve_host", allow=(BURA_ENOCONV,))


def bura_solve_systems(plan, f, V, tol, stream=None):
    """The k+1 solutions (A - d_j I)^{-1} f into the (k+1, N) float64 CUDA tensor V."""
    return _check(_lib().bura_solve_systems(plan, _dptr(f), _dptr(V), float(tol), _stream(stream)),
                  "bura_solve_systems", allow=(BURA_ENOCONV,))


def bura_apply_shifted(plan, x, y, stream=None):
    """y_j = (A - d_j I) x_j for (k+1, N) float64 CUDA tensors."""
    return _check(_lib().bura_apply_shifted(plan, _dptr(x), _dptr(y), _stream(stream)), "bura_apply_shifted")


def bura_get_rational(plan, k):
    c = np.zeros(k + 1)
    d = np.zeros(k + 1)
    E = C.c_double()
    _check(_lib().bura_get_rational(plan, _hptr(c), _hptr(d), C.byref(E)), "bura_get_rational")
    return c, d, E.value


def bura_get_stats(plan):
    st = bura_stats()
    _check(_lib().bura_get_stats(plan, C.byref(st)), "bura_get_stats")
    return st.to_dict()


def bura_set_profiling(plan, enable):
    return _check(_lib().bura_set_profiling(plan, int(bool(enable))), "bura_set_profiling")


def bura_get_profile(plan, max_entries=64):
    """List of dicts {name, launches, ms, bytes} of the timed fine-level kernels."""
    arr = (bura_kernel_prof * max_entries)()
    n = C.c_int()
    _check(_lib().bura_get_profile(plan, max_entries, arr, C.byref(n)), "bura_get_profile")
    return [{"name": arr[i].name.decode(), "launches": arr[i].launches, "ms": arr[i].ms, "bytes": arr[i].bytes}
            for i in range(n.value)]


def bura_residual_norms_noalloc(shape, d, f, V, rr, stream=None):
    """rr[j] = ||f - (A - d_j I) V_j||^2 for the constant-coefficient grid `shape`, allocating nothing.

    d: host numpy array of the shifts; f (N), V (len(d), N) and rr (len(d)) are float64 CUDA tensors.
    """
    g = bura_grid()
    g.dim = len(shape)
    for i, n in enumerate(shape[:3]):
        g.n[i] = int(n)
    g.coef_kind = BURA_COEF_CONSTANT
    d = np.ascontiguousarray(d, dtype=np.float64)
    return _check(_lib().bura_residual_norms_noalloc(C.byref(g), int(d.size), _hptr(d), _dptr(f), _dptr(V),
                                                     _dptr(rr), _stream(stream)), "bura_residual_norms_noalloc")


def bura_destroy(plan):
    return _check(_lib().bura_destroy(plan), "bura_destroy")


EXPORTED = ["bura_default_options", "bura_rational", "bura_setup", "bura_solve", "bura_solve_host",
            "bura_solve_systems", "bura_apply_shifted", "bura_get_rational", "bura_get_stats", "bura_destroy",
            "bura_strerror", "bura_set_profiling", "bura_get_profile", "bura_residual_norms_noalloc",
            "bura_last_cuda_error", "bura_solve_batch", "bura_retarget", "bura_solve_chain", "bura_setup_shifts",
            "bura_solve_sum", "bura_set_tma_wait_cycles", "bura_scale", "bura_quadrature_bp15", "bura_setup_csr",
            "bura_solve_async", "bura_solve_wait", "bura_batch_create", "bura_batch_run", "bura_batch_wait",
            "bura_batch_destroy", "bura_autotune", "bura_server_default_options",
            "bura_server_create", "bura_server_submit", "bura_server_wait", "bura_server_get_stats",
            "bura_server_destroy"]
