"""Thin ctypes binding of libcpgn.so (include/cpgn.h), same call names.

Argument marshalling only: torch tensors are passed as raw device pointers
plus shapes; every step runs in the library's CUDA kernels.  The library is
loaded on first use; if it is missing the call raises (there is no CPU
fallback).  All device work is enqueued on torch's current CUDA stream.
"""
from __future__ import annotations

import ctypes
import itertools
import os
import threading
import weakref

import torch

from . import build as _build

MAX_ORDER = 8

CP_OK, CP_ERR_ARG, CP_ERR_CUDA, CP_ERR_NOMEM, CP_ERR_UNSUPPORTED = 0, 1, 2, 3, 4
CP_ERR_NOT_SPD, CP_ERR_NONFINITE, CP_ERR_BREAKDOWN, CP_ERR_TIMEOUT, CP_WARN_CG_MAXIT = 5, 6, 7, 8, 9
CP_F32, CP_F64 = 0, 1
CP_PREC_FP64, CP_PREC_BF16X3, CP_PREC_RESIDUAL = 0, 1, 2
PREC = {"fp64": CP_PREC_FP64, "bf16x3": CP_PREC_BF16X3, "residual": CP_PREC_RESIDUAL}
CP_REG_IDENTITY, CP_REG_DIAG = 0, 1
REG = {"identity": CP_REG_IDENTITY, "diag": CP_REG_DIAG}

SYMBOLS = ("cp_status_string", "cp_create", "cp_destroy", "cp_set_stream", "cp_workspace_size",
           "cp_mttkrp_all", "cp_gradient", "cp_gn_matvec", "cp_gn_step", "cp_gn_solve", "cp_als_sweep",
           "cp_residual", "cp_residual_sums", "cp_residual_tensor", "cp_hosvd", "cp_tucker_expand", "cp_gn_solve_batched", "cp_gn_matvec_noalloc",
           "cp_batch_plan_create", "cp_batch_plan_launch", "cp_batch_plan_results", "cp_batch_plan_threads", "cp_batch_plan_order",
           "cp_batch_plan_configure", "cp_batch_plan_destroy", "cp_probe_grid_barrier", "cp_probe_fp64_fma")


class cp_desc(ctypes.Structure):
    _fields_ = [("order", ctypes.c_int), ("rank", ctypes.c_int), ("dims", ctypes.c_int64 * MAX_ORDER),
                ("x_dtype", ctypes.c_int), ("x_version", ctypes.c_uint64)]


class cp_gn_params(ctypes.Structure):
    _fields_ = [("eps_cg", ctypes.c_double), ("cg_max_iter", ctypes.c_int), ("lam", ctypes.c_double),
                ("lam_lo", ctypes.c_double), ("lam_hi", ctypes.c_double), ("mu", ctypes.c_double),
                ("lam_dir", ctypes.c_int), ("lam_fixed", ctypes.c_int), ("reg", ctypes.c_int), ("prec", ctypes.c_int),
                ("cg_fp32", ctypes.c_int), ("want_residual", ctypes.c_int),
                ("stop_stationarity", ctypes.c_double), ("spin_limit", ctypes.c_int64),
                ("armijo_c", ctypes.c_double), ("armijo_beta", ctypes.c_double), ("armijo_max", ctypes.c_int)]


class cp_gn_stats(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("cg_iters", ctypes.c_int), ("stopped", ctypes.c_int),
                ("grad_norm_sum", ctypes.c_double), ("m_norm_sum", ctypes.c_double),
                ("update_norm_sum", ctypes.c_double), ("factor_norm_sum", ctypes.c_double),
                ("lam_used", ctypes.c_double), ("cg_rnorm", ctypes.c_double), ("rel_residual", ctypes.c_double),
                ("entry_residual", ctypes.c_double), ("mttkrp_ms", ctypes.c_double), ("pcg_ms", ctypes.c_double), ("step_ms", ctypes.c_double),
                ("kernel_launches", ctypes.c_int), ("cg_blocks", ctypes.c_int), ("step", ctypes.c_double),
                ("f_entry", ctypes.c_double), ("ls_trials", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class cp_solve_opts(ctypes.Structure):
    _fields_ = [("max_iters", ctypes.c_int), ("target_residual", ctypes.c_double),
                ("target_stationarity", ctypes.c_double), ("refine_below", ctypes.c_double),
                ("refine_prec", ctypes.c_int), ("residual_every", ctypes.c_int)]


class cp_solve_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("iters", ctypes.c_int), ("iters_refined", ctypes.c_int),
                ("cg_iters_total", ctypes.c_int), ("converged", ctypes.c_int), ("stationarity", ctypes.c_double),
                ("rel_residual", ctypes.c_double), ("lam", ctypes.c_double), ("mttkrp_ms", ctypes.c_double),
                ("pcg_ms", ctypes.c_double), ("device_ms", ctypes.c_double), ("kernel_launches", ctypes.c_longlong),
                ("cg_blocks", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lock = threading.Lock()
_lib = None


class cp_batch_problem(ctypes.Structure):
    _fields_ = [("dims", ctypes.c_int64 * 3), ("rank", ctypes.c_int), ("X", ctypes.c_void_p),
                ("A", ctypes.c_void_p * 3), ("lam", ctypes.c_double), ("lam_lo", ctypes.c_double),
                ("lam_hi", ctypes.c_double), ("mu", ctypes.c_double), ("reg", ctypes.c_int),
                ("lam_fixed", ctypes.c_int), ("armijo_c", ctypes.c_double), ("armijo_beta", ctypes.c_double),
                ("armijo_max", ctypes.c_int)]


class cp_batch_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("iters", ctypes.c_int), ("cg_iters_total", ctypes.c_int),
                ("converged", ctypes.c_int), ("cg_breakdowns", ctypes.c_int), ("rel_residual", ctypes.c_double),
                ("lam", ctypes.c_double), ("ls_backtracks", ctypes.c_int)]


class CPError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        super().__init__(f"{where}: {status_string(status)} ({status})")


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """Load libcpgn.so.  Raises if it is missing (no fallback)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(_build.LIB):
            if build_if_missing:
                _build.build()
            else:
                raise RuntimeError(f"libcpgn.so not built ({_build.LIB}); run __graft_entry__.build()")
        L = ctypes.CDLL(_build.LIB)
        vp, i, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
        pd = ctypes.POINTER(cp_desc)
        L.cp_status_string.argtypes = [i]
        L.cp_status_string.restype = ctypes.c_char_p
        L.cp_create.argtypes = [ctypes.POINTER(vp), i]
        L.cp_destroy.argtypes = [vp]
        L.cp_set_stream.argtypes = [vp, vp]
        L.cp_workspace_size.argtypes = [vp, pd, i, ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(ctypes.c_size_t)]
        L.cp_mttkrp_all.argtypes = [vp, pd, vp, vp, vp, i]
        L.cp_gradient.argtypes = [vp, pd, vp, vp, vp, i, ctypes.POINTER(d), ctypes.POINTER(d)]
        L.cp_gn_matvec.argtypes = [vp, pd, vp, vp, vp, d, i, vp, i]
        L.cp_gn_step.argtypes = [vp, pd, vp, vp, ctypes.POINTER(cp_gn_params), ctypes.POINTER(cp_gn_stats)]
        L.cp_gn_solve.argtypes = [vp, pd, vp, vp, ctypes.POINTER(cp_gn_params), ctypes.POINTER(cp_solve_opts),
                                  ctypes.POINTER(cp_solve_result)]
        L.cp_als_sweep.argtypes = [vp, pd, vp, vp, d, i, ctypes.POINTER(d)]
        L.cp_residual.argtypes = [vp, pd, vp, vp, ctypes.POINTER(d)]
        L.cp_residual_sums.argtypes = [vp, pd, vp, vp, ctypes.POINTER(d), ctypes.POINTER(d)]
        L.cp_residual_tensor.argtypes = [vp, pd, vp, vp, vp, ctypes.POINTER(d), ctypes.POINTER(d)]
        L.cp_hosvd.argtypes = [vp, pd, vp, ctypes.POINTER(i), vp, vp, ctypes.POINTER(i)]
        L.cp_tucker_expand.argtypes = [vp, i, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(i), i, vp, vp, vp]
        L.cp_gn_matvec_noalloc.argtypes = [pd, vp, vp, d, vp, vp]
        L.cp_gn_solve_batched.argtypes = [vp, i, ctypes.POINTER(cp_batch_problem), d, i, i, d,
                                          ctypes.POINTER(cp_batch_result)]
        L.cp_batch_plan_create.argtypes = [vp, i, ctypes.POINTER(cp_batch_problem), d, i, i, d, i,
                                           ctypes.POINTER(vp)]
        L.cp_batch_plan_launch.argtypes = [vp, vp]
        L.cp_batch_plan_results.argtypes = [vp, vp, ctypes.POINTER(cp_batch_result)]
        L.cp_batch_plan_threads.argtypes = [vp, ctypes.POINTER(i)]
        L.cp_batch_plan_order.argtypes = [vp, ctypes.POINTER(i)]
        L.cp_batch_plan_configure.argtypes = [vp, i, i]
        L.cp_batch_plan_destroy.argtypes = [vp]
        L.cp_probe_grid_barrier.argtypes = [i, i, i, i, ctypes.POINTER(d)]
        L.cp_probe_fp64_fma.argtypes = [i, ctypes.POINTER(d)]
        for name in SYMBOLS:
            if name != "cp_status_string":
                getattr(L, name).restype = ctypes.c_int
        _lib = L
        return L


def status_string(s: int) -> str:
    return load().cp_status_string(int(s)).decode()


def _check(s, where, ok=(CP_OK,)):
    if s not in ok:
        raise CPError(s, where)
    return s


# --------------------------------------------------------------------- marshalling

def make_desc(shape, rank, x_dtype, version=0) -> cp_desc:
    d = cp_desc()
    d.order = len(shape)
    d.rank = int(rank)
    for k, s in enumerate(shape):
        d.dims[k] = int(s)
    d.x_dtype = CP_F32 if x_dtype == torch.float32 else CP_F64
    d.x_version = int(version)
    return d


def _ptr_array(tensors):
    arr = (ctypes.c_void_p * len(tensors))()
    for k, t in enumerate(tensors):
        arr[k] = t.data_ptr()
    return arr


def _check_factor(t, rows, rank, name):
    if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous() and tuple(t.shape) == (rows, rank)):
        raise ValueError(f"{name}: expected contiguous CUDA float64 tensor of shape ({rows}, {rank})")


def _check_outputs(outs, shape, rank, name, device):
    """Caller-supplied outputs: one contiguous float64 (s_n, R) tensor per mode
    on `device` (the library cannot see the size of a device buffer)."""
    if len(outs) != len(shape):
        raise ValueError(f"{name}: need one output per mode")
    for n, t in enumerate(outs):
        _check_factor(t, shape[n], rank, f"{name}[{n}]")
        if t.device != device:
            raise ValueError(f"{name}[{n}] is on {t.device}, expected {device}")


def _check_x(X):
    if not (X.is_cuda and X.dtype in (torch.float32, torch.float64) and X.is_contiguous()):
        raise ValueError("X: expected a contiguous CUDA float32/float64 tensor")


class XVersions:
    """Version stamps for the library's cache of the bf16 split of X, which it
    keys by X's address, size, dtype and the descriptor's x_version.  A tensor
    gets a new stamp whenever the object at its address is not the one seen
    there last, or torch's in-place version counter of it has moved, or
    bump() is called; stamps come from one counter, so a stamp is never reused
    (a new tensor that the caching allocator places at a freed address can
    never match the old tensor's cached split)."""

    def __init__(self):
        self._seen = {}
        self._next = itertools.count(1)

    @staticmethod
    def _inplace(X):
        try:
            return X._version
        except RuntimeError:  # inference-mode tensors keep no version counter
            return None

    def stamp(self, X) -> int:
        ptr = X.data_ptr()
        seen = self._seen.get(ptr)
        tv = self._inplace(X)
        if seen is not None and seen[0]() is X and seen[1] == tv:
            return seen[2]
        ver = next(self._next)
        self._seen[ptr] = (weakref.ref(X), tv, ver)
        return ver

    def bump(self, X) -> int:
        ver = next(self._next)
        self._seen[X.data_ptr()] = (weakref.ref(X), self._inplace(X), ver)
        return ver


class Handle:
    """Owns a cp_handle bound to a CUDA device; work goes to torch's current stream."""

    def __init__(self, device=None):
        L = load()
        dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        self.device = dev.index if dev.index is not None else torch.cuda.current_device()
        h = ctypes.c_void_p()
        _check(L.cp_create(ctypes.byref(h), self.device), "cp_create")
        self.h = h
        self._xv = XVersions()

    def close(self):
        if getattr(self, "h", None):
            load().cp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _bind_stream(self):
        load().cp_set_stream(self.h, ctypes.c_void_p(torch.cuda.current_stream(self.device).cuda_stream))

    def desc(self, X, rank):
        _check_x(X)
        if X.device.index != self.device:
            raise ValueError(f"X is on {X.device}, the handle on cuda:{self.device}")
        return make_desc(X.shape, rank, X.dtype, self._xv.stamp(X))

    def bump_version(self, X):
        """Declare that the contents of X changed (invalidates the split cache).
        Changes made through torch in place, and new tensors, are detected
        without it; writes that bypass torch (a raw pointer, another library)
        need it."""
        self._xv.bump(X)


def _factors(X, A):
    if len(A) != X.dim():
        raise ValueError("need one factor per mode")
    R = A[0].shape[1]
    for n, a in enumerate(A):
        _check_factor(a, X.shape[n], R, f"A[{n}]")
        if a.device != X.device:
            raise ValueError(f"A[{n}] is on {a.device}, X on {X.device}")
    return R


def cp_workspace_size(h: Handle, X, rank, prec="fp64"):
    d = h.desc(X, rank)
    b, sb = ctypes.c_size_t(), ctypes.c_size_t()
    _check(load().cp_workspace_size(h.h, ctypes.byref(d), PREC[prec], ctypes.byref(b), ctypes.byref(sb)),
           "cp_workspace_size")
    return b.value, sb.value


def cp_mttkrp_all(h: Handle, X, A, M=None, prec="fp64"):
    R = _factors(X, A)
    if M is None:
        M = [torch.empty_like(a) for a in A]
    _check_outputs(M, X.shape, R, "M", X.device)
    h._bind_stream()
    d = h.desc(X, R)
    _check(load().cp_mttkrp_all(h.h, ctypes.byref(d), X.data_ptr(), _ptr_array(A), _ptr_array(M), PREC[prec]),
           "cp_mttkrp_all")
    return M


def cp_gradient(h: Handle, X, A, G=None, prec="fp64"):
    R = _factors(X, A)
    if G is None:
        G = [torch.empty_like(a) for a in A]
    _check_outputs(G, X.shape, R, "G", X.device)
    h._bind_stream()
    d = h.desc(X, R)
    N = X.dim()
    gn, mn = (ctypes.c_double * N)(), (ctypes.c_double * N)()
    _check(load().cp_gradient(h.h, ctypes.byref(d), X.data_ptr(), _ptr_array(A), _ptr_array(G), PREC[prec],
                              gn, mn), "cp_gradient")
    return G, list(gn), list(mn)


def cp_gn_matvec(h: Handle, A, W, lam, Q=None, grams=None, reg="identity", prec="fp64"):
    """Q = (J^T J + lam D) W with D = I (reg="identity") or diag(J^T J)
    (reg="diag"); grams: optional (N, R, R) float64 CUDA tensor of the Gram
    matrices A^(n)^T A^(n); prec "fp64" or the mixed CG's FP32 arithmetic
    ("bf16x3" / "residual")."""
    R = A[0].shape[1]
    shape = [a.shape[0] for a in A]
    for n in range(len(A)):
        _check_factor(A[n], shape[n], R, f"A[{n}]")
        _check_factor(W[n], shape[n], R, f"W[{n}]")
    if len(W) != len(A):
        raise ValueError("need one W per factor")
    for n in range(len(A)):
        if A[n].device != A[0].device or W[n].device != A[0].device:
            raise ValueError("A and W must be on one device")
    if A[0].device.index != h.device:
        raise ValueError(f"A is on {A[0].device}, the handle on cuda:{h.device}")
    if grams is not None:
        if not (grams.is_cuda and grams.dtype == torch.float64 and grams.is_contiguous()
                and tuple(grams.shape) == (len(A), R, R) and grams.device == A[0].device):
            raise ValueError(f"grams: expected a contiguous CUDA float64 tensor of shape ({len(A)}, {R}, {R})")
    if Q is None:
        Q = [torch.empty_like(a) for a in A]
    _check_outputs(Q, shape, R, "Q", A[0].device)
    h._bind_stream()
    d = make_desc(shape, R, torch.float64)
    _check(load().cp_gn_matvec(h.h, ctypes.byref(d), _ptr_array(A), grams.data_ptr() if grams is not None else None,
                               _ptr_array(W), float(lam), REG[reg], _ptr_array(Q), PREC[prec]), "cp_gn_matvec")
    return Q


def gn_params(lam, lam_lo, lam_hi, mu=2.0, eps_cg=1e-3, cg_max_iter=250, prec="fp64", cg_fp32=None,
              lam_dir=0, lam_fixed=False, want_residual=False, stop_stationarity=0.0, spin_limit=0,
              reg="identity", armijo_c=0.0, armijo_beta=0.5, armijo_max=10):
    """reg: "identity" damps by lam I, "diag" by lam diag(J^T J) (then lam is
    dimensionless); armijo_c > 0 turns on step-size control by Armijo's
    condition (backtracking by armijo_beta, at most armijo_max reductions)."""
    p = cp_gn_params()
    p.eps_cg, p.cg_max_iter = float(eps_cg), int(cg_max_iter)
    p.lam, p.lam_lo, p.lam_hi, p.mu = float(lam), float(lam_lo), float(lam_hi), float(mu)
    p.lam_dir, p.lam_fixed = int(lam_dir), int(bool(lam_fixed))
    p.reg = REG[reg]
    p.prec = PREC[prec]
    p.cg_fp32 = int(prec in ("bf16x3", "residual")) if cg_fp32 is None else int(bool(cg_fp32))
    p.want_residual = int(bool(want_residual))
    p.stop_stationarity = float(stop_stationarity)
    p.spin_limit = int(spin_limit)
    p.armijo_c, p.armijo_beta, p.armijo_max = float(armijo_c), float(armijo_beta), int(armijo_max)
    return p


def cp_gn_step(h: Handle, X, A, params: cp_gn_params, check=True):
    """One GN iteration; A (list of float64 CUDA tensors) is updated in place.
    Returns (status, stats dict); params.lam / lam_dir advance in place."""
    R = _factors(X, A)
    h._bind_stream()
    d = h.desc(X, R)
    st = cp_gn_stats()
    s = load().cp_gn_step(h.h, ctypes.byref(d), X.data_ptr(), _ptr_array(A), ctypes.byref(params), ctypes.byref(st))
    if check:
        _check(s, "cp_gn_step", ok=(CP_OK, CP_WARN_CG_MAXIT))
    return s, st.as_dict()


def solve_opts(max_iters=200, target_residual=0.0, target_stationarity=0.0, refine_below=0.0, residual_every=0,
               refine_prec="residual"):
    o = cp_solve_opts()
    o.max_iters, o.target_residual, o.target_stationarity = int(max_iters), float(target_residual), \
        float(target_stationarity)
    o.refine_below, o.residual_every = float(refine_below), int(residual_every)
    o.refine_prec = PREC[refine_prec]
    return o


def cp_gn_solve(h: Handle, X, A, params: cp_gn_params, opts: cp_solve_opts, check=True):
    R = _factors(X, A)
    h._bind_stream()
    d = h.desc(X, R)
    res = cp_solve_result()
    s = load().cp_gn_solve(h.h, ctypes.byref(d), X.data_ptr(), _ptr_array(A), ctypes.byref(params),
                           ctypes.byref(opts), ctypes.byref(res))
    if check:
        _check(s, "cp_gn_solve")
    return s, res.as_dict()


def cp_als_sweep(h: Handle, X, A, lam=0.0, prec="fp64", want_residual=True):
    R = _factors(X, A)
    h._bind_stream()
    d = h.desc(X, R)
    r = ctypes.c_double(-1.0)
    _check(load().cp_als_sweep(h.h, ctypes.byref(d), X.data_ptr(), _ptr_array(A), float(lam), PREC[prec],
                               ctypes.byref(r) if want_residual else None), "cp_als_sweep")
    return r.value


def cp_residual(h: Handle, X, A):
    R = _factors(X, A)
    h._bind_stream()
    d = h.desc(X, R)
    r = ctypes.c_double()
    _check(load().cp_residual(h.h, ctypes.byref(d), X.data_ptr(), _ptr_array(A), ctypes.byref(r)), "cp_residual")
    return r.value


def cp_residual_sums(h: Handle, X, A):
    """(||X - [[A]]||_F^2, ||X||_F^2) in FP64."""
    R = _factors(X, A)
    h._bind_stream()
    d = h.desc(X, R)
    e, x = ctypes.c_double(), ctypes.c_double()
    _check(load().cp_residual_sums(h.h, ctypes.byref(d), X.data_ptr(), _ptr_array(A), ctypes.byref(e),
                                   ctypes.byref(x)), "cp_residual_sums")
    return e.value, x.value


def cp_residual_tensor(h: Handle, X, A, E=None, sums_only=False):
    """E = X - [[A]] in FP64 (a CUDA tensor shaped like X) by the residual-form
    gradient's reconstruction; returns (E, sum E^2, ||X||^2).  sums_only: no E
    (returned as None), the two sums alone."""
    R = _factors(X, A)
    if sums_only:
        E = None
    else:
        if E is None:
            E = torch.empty(X.shape, dtype=torch.float64, device=X.device)
        if not (E.is_cuda and E.dtype == torch.float64 and E.is_contiguous() and E.shape == X.shape
                and E.device == X.device):
            raise ValueError("E: expected a contiguous CUDA float64 tensor shaped like X")
    h._bind_stream()
    d = h.desc(X, R)
    e, x = ctypes.c_double(), ctypes.c_double()
    _check(load().cp_residual_tensor(h.h, ctypes.byref(d), X.data_ptr(), _ptr_array(A),
                                     E.data_ptr() if E is not None else None, ctypes.byref(e), ctypes.byref(x)),
           "cp_residual_tensor")
    return E, e.value, x.value


def cp_hosvd(h: Handle, X, ranks):
    """Truncated HoSVD (Tucker compression): returns (U list of (s_n, r_n)
    float64 CUDA tensors with orthonormal columns, core float64 CUDA tensor of
    shape ranks, iteration counts)."""
    ranks = [int(r) for r in ranks]
    if len(ranks) != X.dim():
        raise ValueError("one rank per mode")
    U = [torch.empty((s, r), dtype=torch.float64, device=X.device) for s, r in zip(X.shape, ranks)]
    core = torch.empty(ranks, dtype=torch.float64, device=X.device)
    h._bind_stream()
    d = h.desc(X, 1)
    rk = (ctypes.c_int * len(ranks))(*ranks)
    it = (ctypes.c_int * len(ranks))()
    _check(load().cp_hosvd(h.h, ctypes.byref(d), X.data_ptr(), rk, _ptr_array(U), core.data_ptr(), it), "cp_hosvd")
    return U, core, list(it)


def cp_tucker_expand(h: Handle, U, B):
    """A_n = U_n B_n (float64 CUDA tensors): the CP factors of X from the CP
    factors B of the Tucker core."""
    if len(U) != len(B):
        raise ValueError("one B per U")
    R = B[0].shape[1]
    for n, (u, b) in enumerate(zip(U, B)):
        _check_factor(u, u.shape[0], u.shape[1], f"U[{n}]")
        _check_factor(b, u.shape[1], R, f"B[{n}]")
        if u.device.index != h.device or b.device.index != h.device:
            raise ValueError("U and B must be on the handle's device")
    A = [torch.empty((u.shape[0], R), dtype=torch.float64, device=u.device) for u in U]
    h._bind_stream()
    N = len(U)
    dims = (ctypes.c_int64 * N)(*[u.shape[0] for u in U])
    rk = (ctypes.c_int * N)(*[u.shape[1] for u in U])
    _check(load().cp_tucker_expand(h.h, N, dims, rk, R, _ptr_array(U), _ptr_array(B), _ptr_array(A)),
           "cp_tucker_expand")
    return A


def _batch_array(problems, device: int):
    n = len(problems)
    arr = (cp_batch_problem * max(n, 1))()
    for k, q in enumerate(problems):
        X, A = q["X"], q["A"]
        if X.dtype != torch.float32 or not X.is_cuda or X.dim() != 3 or not X.is_contiguous():
            raise ValueError("batched: X must be a contiguous 3-D float32 CUDA tensor")
        if X.device.index != device:
            raise ValueError(f"batched: problem {k} is on {X.device}, the handle on cuda:{device}")
        R = A[0].shape[1]
        for m in range(3):
            _check_factor(A[m], X.shape[m], R, f"A[{m}]")
            if A[m].device != X.device:
                raise ValueError(f"batched: problem {k}, A[{m}] is on {A[m].device}, X on {X.device}")
        arr[k].dims = (ctypes.c_int64 * 3)(*X.shape)
        arr[k].rank = R
        arr[k].X = X.data_ptr()
        arr[k].A = (ctypes.c_void_p * 3)(*[a.data_ptr() for a in A])
        arr[k].lam, arr[k].lam_lo, arr[k].lam_hi, arr[k].mu = q["lam"], q["lam_lo"], q["lam_hi"], q.get("mu", 2.0)
        arr[k].reg = REG[q.get("reg", "identity")]
        arr[k].lam_fixed = int(bool(q.get("lam_fixed", False)))
        arr[k].armijo_c = float(q.get("armijo_c", 0.0))
        arr[k].armijo_beta = float(q.get("armijo_beta", 0.5))
        arr[k].armijo_max = int(q.get("armijo_max", 10))
    return arr


_BATCH_KEYS = ("status", "iters", "cg_iters_total", "converged", "cg_breakdowns", "rel_residual", "lam",
               "ls_backtracks")


def cp_gn_solve_batched(h: Handle, problems, eps_cg=1e-3, cg_max_iter=250, max_iters=200, target_residual=1e-6):
    """Solve many small order-3 problems in one persistent launch.  problems: list of
    dicts with X (float32 CUDA, 3-D), A (three float64 CUDA (s_n, R) tensors, updated in
    place), lam, lam_lo, lam_hi, mu, and optionally reg ("identity" / "diag"),
    lam_fixed, armijo_c, armijo_beta, armijo_max.  Returns a list of result dicts."""
    n = len(problems)
    arr = _batch_array(problems, h.device)
    res = (cp_batch_result * max(n, 1))()
    h._bind_stream()
    _check(load().cp_gn_solve_batched(h.h, n, arr, eps_cg, cg_max_iter, max_iters, target_residual, res),
           "cp_gn_solve_batched")
    return [{k2: getattr(res[k], k2) for k2 in _BATCH_KEYS} for k in range(n)]


class BatchPlan:
    """A reusable batched solve (cp_batch_plan_*): created once (with the
    autotuner's choice of block size), then launched -- asynchronously, on the
    handle's stream, capturable into a CUDA graph -- and read back."""

    def __init__(self, h: Handle, problems, eps_cg=1e-3, cg_max_iter=250, max_iters=200, target_residual=1e-6,
                 autotune=True):
        self.h, self.n = h, len(problems)
        self._keep = problems  # the plan holds their device pointers
        arr = _batch_array(problems, h.device)
        p = ctypes.c_void_p()
        h._bind_stream()
        _check(load().cp_batch_plan_create(h.h, self.n, arr, eps_cg, cg_max_iter, max_iters, target_residual,
                                           int(bool(autotune)), ctypes.byref(p)), "cp_batch_plan_create")
        self.p = p

    @property
    def threads(self):
        t = ctypes.c_int()
        _check(load().cp_batch_plan_threads(self.p, ctypes.byref(t)), "cp_batch_plan_threads")
        return t.value

    @property
    def order(self):
        """0: problems taken in the given order, 1: largest work first."""
        o = ctypes.c_int()
        _check(load().cp_batch_plan_order(self.p, ctypes.byref(o)), "cp_batch_plan_order")
        return o.value

    def configure(self, threads, order):
        """Fix the block size (128, 256 or 384) and the problem order (0 or 1) of later launches."""
        _check(load().cp_batch_plan_configure(self.p, int(threads), int(order)), "cp_batch_plan_configure")

    def launch(self):
        """Enqueue one solve of every problem on torch's current stream (no synchronisation)."""
        self.h._bind_stream()
        _check(load().cp_batch_plan_launch(self.h.h, self.p), "cp_batch_plan_launch")

    def results(self):
        res = (cp_batch_result * self.n)()
        self.h._bind_stream()
        _check(load().cp_batch_plan_results(self.h.h, self.p, res), "cp_batch_plan_results")
        return [{k2: getattr(res[k], k2) for k2 in _BATCH_KEYS} for k in range(self.n)]

    def close(self):
        if self.p:
            load().cp_batch_plan_destroy(self.p)
            self.p = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def cp_gn_matvec_noalloc(A, W, lam, Q):
    """Q = (J^T J + lam I) W without any device allocation (static scratch in
    the library; order <= 4, rank <= 64).  Q must be preallocated by the
    caller; work goes to torch's current stream on the current device."""
    R = A[0].shape[1]
    shape = [a.shape[0] for a in A]
    if len(W) != len(A) or len(Q) != len(A):
        raise ValueError("need one W and one Q per factor")
    dev = torch.device("cuda", torch.cuda.current_device())
    for n in range(len(A)):
        for name, t in (("A", A[n]), ("W", W[n]), ("Q", Q[n])):
            _check_factor(t, shape[n], R, f"{name}[{n}]")
            if t.device != dev:
                raise ValueError(f"{name}[{n}] is on {t.device}; the call runs on the current device {dev}")
    d = make_desc(shape, R, torch.float64)
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    _check(load().cp_gn_matvec_noalloc(ctypes.byref(d), _ptr_array(A), _ptr_array(W), float(lam), _ptr_array(Q),
                                       st), "cp_gn_matvec_noalloc")
    return Q


def cp_probe_grid_barrier(device: int, blocks: int, threads: int = 512, iters: int = 20000) -> float:
    """Device time of one grid barrier of the persistent CG kernel's kind, in
    microseconds, with `blocks` co-resident blocks of `threads` threads."""
    us = ctypes.c_double()
    _check(load().cp_probe_grid_barrier(int(device), int(blocks), int(threads), int(iters), ctypes.byref(us)),
           "cp_probe_grid_barrier")
    return us.value


def cp_probe_fp64_fma(device: int) -> float:
    """Measured FP64 FMA rate of the device in TFLOP/s (2 flops per FMA)."""
    t = ctypes.c_double()
    _check(load().cp_probe_fp64_fma(int(device), ctypes.byref(t)), "cp_probe_fp64_fma")
    return t.value
