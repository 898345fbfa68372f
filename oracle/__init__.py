"""Plain FP64 CPU oracle for Gauss-Newton CP decomposition.

TEST INFRASTRUCTURE ONLY.  This package is the independent checker of the
CUDA library in ``paper_1910_12331_gb300``.  It shares no code with it and
must only be imported by ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py``.  The product path never imports it.

The arithmetic lives in ``cpgn_oracle.c`` (plain C loops in double
precision, OpenMP over independent outer indices); this module compiles it
with gcc into ``_liboracle.so`` beside the source and exposes numpy-facing
wrappers.  Factor matrices are passed as Python lists of ``(s_n, R)``
float64 arrays; the wrappers pack them the way the C code expects.

Parity status of each routine (pins live in ``tests/test_oracle_pins.py``):
  gram / gamma          pinned (numpy A^T A products, Eq. (2.2)/(3.3) identities)
  mttkrp_def / _dt      pinned (brute-force einsum of the definition, rank-1
                        closed form, zero gradient at an exact decomposition,
                        Strassen and classical matmul-tensor decompositions)
  gradient              pinned (explicit Jacobian J^T r, finite differences)
  precond_inv           pinned ((Gamma + lam D) P_inv = I, D = I or diag(Gamma))
  matvec                pinned (explicit Jacobian (J^T J + lam D) v with
                        D = I or diag(J^T J), null directions of the scaling
                        indeterminacy)
  pcg                   pinned (dense solve of the explicit normal equations,
                        both dampings; with diag(J^T J) the step commutes with
                        the column rescaling of the CP model)
  lambda_next           pinned (hand-derived sequence, golden fixture)
  gn_step               pinned (exact recovery of exact-rank tensors)
  gn_step_ls            pinned (Armijo's condition holds at the accepted step and
                        fails at the one before, monotone objective, the full
                        step is taken near an exact decomposition, constant lambda)
  residual              pinned (numpy reconstruction, zero at exact factors)
  unfold_gram / sym_eig / mode_product_t / hosvd
                        pinned (numpy products and eigenvalues, eigen-equation and
                        orthonormality, exact recovery of a tensor of low
                        multilinear rank, the HoSVD error bounds, the split of
                        the CP error of an expanded core)
  residual_tensor       pinned (numpy reconstruction, zero at exact factors, its
                        squared sum is the residual's numerator)
  als_sweep             pinned (monotone objective, zero mode gradient)
  The lambda thresholds, mu and the collinearity/noise recipe are chosen
  conventions: "parity unpinned" beyond the rule itself.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cpgn_oracle.c")
_LIB = os.path.join(_HERE, "_liboracle.so")
_lock = threading.Lock()
_lib = None

MAXN = 8
OK, ERR_ARG, ERR_NOT_SPD, ERR_BREAKDOWN, WARN_CG_MAXIT = 0, 1, 5, 7, 9
# damping of the CG system (Section 3.2): lam I or lam diag(J^T J)
REG_IDENTITY, REG_DIAG = 0, 1


class _Desc(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int), ("R", ctypes.c_int), ("dims", ctypes.c_int64 * MAXN)]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (portable flags: runs on x86 and Arm)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-o", _LIB + ".tmp", _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(_LIB + ".tmp", _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            P = ctypes.POINTER
            d = P(_Desc)
            dp = P(ctypes.c_double)
            lib.orc_gram.argtypes = [d, dp, dp]
            lib.orc_gamma.argtypes = [d, dp, dp]
            lib.orc_mttkrp_def.argtypes = [d, dp, dp, dp]
            lib.orc_mttkrp_dt.argtypes = [d, dp, dp, dp]
            lib.orc_mttkrp_row.argtypes = [d, dp, dp, ctypes.c_int, ctypes.c_int64, dp]
            lib.orc_gradient.argtypes = [d, dp, dp, dp, dp, dp]
            lib.orc_precond_inv.argtypes = [ctypes.c_int, dp, ctypes.c_double, ctypes.c_int, dp]
            lib.orc_precond_inv.restype = ctypes.c_int
            lib.orc_matvec.argtypes = [d, dp, dp, dp, ctypes.c_double, ctypes.c_int, dp]
            lib.orc_pcg.argtypes = [d, dp, dp, dp, ctypes.c_double, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                    ctypes.c_int, dp, P(ctypes.c_int), dp]
            lib.orc_pcg.restype = ctypes.c_int
            lib.orc_lambda_next.argtypes = [dp, P(ctypes.c_int), ctypes.c_double, ctypes.c_double,
                                            ctypes.c_double]
            lib.orc_gn_step.argtypes = [d, dp, dp, dp, P(ctypes.c_int), ctypes.c_double, ctypes.c_double,
                                        ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                        ctypes.c_int, ctypes.c_int, dp]
            lib.orc_gn_step.restype = ctypes.c_int
            lib.orc_gn_step_ls.argtypes = [d, dp, dp, dp, P(ctypes.c_int), ctypes.c_double, ctypes.c_double,
                                           ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                           ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                           ctypes.c_int, dp]
            lib.orc_gn_step_ls.restype = ctypes.c_int
            lib.orc_gn_solve.argtypes = [d, dp, dp, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                         ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_double,
                                         ctypes.c_int, ctypes.c_int, ctypes.c_int, dp]
            lib.orc_gn_solve.restype = ctypes.c_int
            lib.orc_set_threads.argtypes = [ctypes.c_int]
            lib.orc_set_threads.restype = None
            lib.orc_residual.argtypes = [d, dp, dp]
            lib.orc_residual_tensor.argtypes = [d, dp, dp, dp]
            lib.orc_unfold_gram.argtypes = [d, dp, ctypes.c_int, dp]
            lib.orc_unfold_gram.restype = None
            lib.orc_sym_eig.argtypes = [ctypes.c_int, dp, dp, dp]
            lib.orc_sym_eig.restype = None
            lib.orc_mode_product_t.argtypes = [ctypes.c_int, P(ctypes.c_int64), dp, ctypes.c_int, ctypes.c_int, dp,
                                               dp]
            lib.orc_mode_product_t.restype = None
            lib.orc_residual_tensor.restype = None
            lib.orc_residual.restype = ctypes.c_double
            lib.orc_als_sweep.argtypes = [d, dp, dp, ctypes.c_double]
            lib.orc_als_sweep.restype = ctypes.c_int
            _lib = lib
    return _lib


# ------------------------------------------------------------------ marshalling

def _desc(dims, R):
    d = _Desc()
    d.N = len(dims)
    d.R = int(R)
    for i, s in enumerate(dims):
        d.dims[i] = int(s)
    return d


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _pack(mats):
    return np.ascontiguousarray(np.concatenate([np.asarray(m, dtype=np.float64).reshape(-1) for m in mats]))


def _unpack(buf, dims, R):
    out, off = [], 0
    for s in dims:
        out.append(buf[off:off + s * R].reshape(s, R).copy())
        off += s * R
    return out


def _x64(X):
    # exact upcast of the same bytes the GPU reads
    return np.ascontiguousarray(np.asarray(X), dtype=np.float64)


# --------------------------------------------------------------------- routines

def gram(A):
    dims, R = [a.shape[0] for a in A], A[0].shape[1]
    S = np.zeros((len(A), R, R))
    _load().orc_gram(ctypes.byref(_desc(dims, R)), _ptr(_pack(A)), _ptr(S))
    return S


def gamma(S):
    N, R = S.shape[0], S.shape[1]
    G = np.zeros((N, N, R, R))
    _load().orc_gamma(ctypes.byref(_desc([1] * N, R)), _ptr(np.ascontiguousarray(S)), _ptr(G))
    return G


def mttkrp(X, A, method: str = "def"):
    """All-mode MTTKRP; method 'def' (definition) or 'dt' (dimension tree)."""
    X = _x64(X)
    dims, R = list(X.shape), A[0].shape[1]
    Mbuf = np.zeros(sum(dims) * R)
    fn = _load().orc_mttkrp_def if method == "def" else _load().orc_mttkrp_dt
    fn(ctypes.byref(_desc(dims, R)), _ptr(X), _ptr(_pack(A)), _ptr(Mbuf))
    return _unpack(Mbuf, dims, R)


def mttkrp_row(X, A, n: int, i: int):
    X = _x64(X)
    dims, R = list(X.shape), A[0].shape[1]
    out = np.zeros(R)
    _load().orc_mttkrp_row(ctypes.byref(_desc(dims, R)), _ptr(X), _ptr(_pack(A)), int(n), int(i), _ptr(out))
    return out


def gradient(A, Gam, M):
    dims, R = [a.shape[0] for a in A], A[0].shape[1]
    Gbuf = np.zeros(sum(dims) * R)
    gn = np.zeros(MAXN)
    _load().orc_gradient(ctypes.byref(_desc(dims, R)), _ptr(_pack(A)), _ptr(np.ascontiguousarray(Gam)),
                         _ptr(_pack(M)), _ptr(Gbuf), _ptr(gn))
    return _unpack(Gbuf, dims, R), gn[:len(dims)].copy()


def precond_inv(Gnn, lam, reg: int = REG_IDENTITY):
    R = Gnn.shape[0]
    P = np.zeros((R, R))
    st = _load().orc_precond_inv(R, _ptr(np.ascontiguousarray(Gnn, dtype=np.float64)), float(lam), int(reg),
                                 _ptr(P))
    return P, st


def matvec(A, Gam, W, lam, reg: int = REG_IDENTITY):
    dims, R = [a.shape[0] for a in A], A[0].shape[1]
    Q = np.zeros(sum(dims) * R)
    _load().orc_matvec(ctypes.byref(_desc(dims, R)), _ptr(_pack(A)), _ptr(np.ascontiguousarray(Gam)),
                       _ptr(_pack(W)), float(lam), int(reg), _ptr(Q))
    return _unpack(Q, dims, R)


def pcg(A, Gam, G, lam, eps_cg, maxit, beta_kind: int = 0, reg: int = REG_IDENTITY):
    dims, R = [a.shape[0] for a in A], A[0].shape[1]
    V = np.zeros(sum(dims) * R)
    it = ctypes.c_int(0)
    rn = np.zeros(1)
    st = _load().orc_pcg(ctypes.byref(_desc(dims, R)), _ptr(_pack(A)), _ptr(np.ascontiguousarray(Gam)),
                         _ptr(_pack(G)), float(lam), int(reg), float(eps_cg), int(maxit), int(beta_kind), _ptr(V),
                         ctypes.byref(it), _ptr(rn))
    return _unpack(V, dims, R), it.value, float(rn[0]), st


def lambda_next(lam, direction, lo, hi, mu):
    l = np.array([lam], dtype=np.float64)
    dr = ctypes.c_int(int(direction))
    _load().orc_lambda_next(_ptr(l), ctypes.byref(dr), float(lo), float(hi), float(mu))
    return float(l[0]), dr.value


def gn_step(X, A, lam, direction, lam_lo, lam_hi, mu, eps_cg, maxit, beta_kind=0, use_dt=False,
            reg=REG_IDENTITY):
    """One CP-GN iteration (Algorithm 1).  Returns (A_new, lam, dir, stats, status);
    stats = dict(grad_norm_sum, update_norm_sum, lam_used, cg_iters, cg_rnorm, m_norm_sum)."""
    X = _x64(X)
    dims, R = list(X.shape), A[0].shape[1]
    Abuf = _pack(A)
    l = np.array([lam], dtype=np.float64)
    dr = ctypes.c_int(int(direction))
    stats = np.zeros(6)
    st = _load().orc_gn_step(ctypes.byref(_desc(dims, R)), _ptr(X), _ptr(Abuf), _ptr(l), ctypes.byref(dr),
                             float(lam_lo), float(lam_hi), float(mu), float(eps_cg), int(maxit),
                             int(beta_kind), int(bool(use_dt)), int(reg), _ptr(stats))
    keys = ("grad_norm_sum", "update_norm_sum", "lam_used", "cg_iters", "cg_rnorm", "m_norm_sum")
    s = dict(zip(keys, stats.tolist()))
    s["cg_iters"] = int(s["cg_iters"])
    return _unpack(Abuf, dims, R), float(l[0]), dr.value, s, st


def gn_step_ls(X, A, lam, direction, lam_lo, lam_hi, mu, eps_cg, maxit, use_dt=False, reg=REG_IDENTITY,
               lam_fixed=False, armijo_c=0.0, armijo_beta=0.5, armijo_max=10):
    """One CP-GN iteration with a constant lambda (lam_fixed) and/or Armijo
    step-size control (armijo_c > 0).  Returns (A_new, lam, dir, stats, status);
    stats as gn_step plus step (t applied), f0 (1/2 ||X - [[A]]||^2 at entry, -1
    without the line search) and trials."""
    X = _x64(X)
    dims, R = list(X.shape), A[0].shape[1]
    Abuf = _pack(A)
    l = np.array([lam], dtype=np.float64)
    dr = ctypes.c_int(int(direction))
    stats = np.zeros(9)
    st = _load().orc_gn_step_ls(ctypes.byref(_desc(dims, R)), _ptr(X), _ptr(Abuf), _ptr(l), ctypes.byref(dr),
                                float(lam_lo), float(lam_hi), float(mu), float(eps_cg), int(maxit),
                                int(bool(use_dt)), int(reg), int(bool(lam_fixed)), float(armijo_c),
                                float(armijo_beta), int(armijo_max), _ptr(stats))
    keys = ("grad_norm_sum", "update_norm_sum", "lam_used", "cg_iters", "cg_rnorm", "m_norm_sum", "step", "f0",
            "trials")
    s = dict(zip(keys, stats.tolist()))
    s["cg_iters"], s["trials"] = int(s["cg_iters"]), int(s["trials"])
    return _unpack(Abuf, dims, R), float(l[0]), dr.value, s, st


def gn_solve(X, A, lam0, lam_lo, lam_hi, mu, eps_cg, maxit, target, max_gn, use_dt=True, reg=REG_IDENTITY):
    """Algorithm 1 until the entry point of an iteration has
    sum||G||/sum||M|| <= target (no update there) or max_gn updates.
    Returns (A_new, status, dict(updates, cg_iters, stationarity, converged, lam))."""
    X = _x64(X)
    dims, R = list(X.shape), A[0].shape[1]
    Abuf = _pack(A)
    out = np.zeros(5)
    st = _load().orc_gn_solve(ctypes.byref(_desc(dims, R)), _ptr(X), _ptr(Abuf), float(lam0), float(lam_lo),
                              float(lam_hi), float(mu), float(eps_cg), int(maxit), float(target), int(max_gn),
                              int(bool(use_dt)), int(reg), _ptr(out))
    info = {"updates": int(out[0]), "cg_iters": int(out[1]), "stationarity": float(out[2]),
            "converged": bool(out[3]), "lam": float(out[4])}
    return _unpack(Abuf, dims, R), st, info


def set_threads(n: int) -> None:
    """Threads of the oracle's OpenMP loops from now on."""
    _load().orc_set_threads(int(n))


def residual(X, A):
    X = _x64(X)
    dims, R = list(X.shape), A[0].shape[1]
    return float(_load().orc_residual(ctypes.byref(_desc(dims, R)), _ptr(X), _ptr(_pack(A))))


def residual_tensor(X, A):
    """E = X - [[A]] element by element in FP64 (same shape as X)."""
    X = _x64(X)
    dims, R = list(X.shape), A[0].shape[1]
    E = np.empty(X.shape, dtype=np.float64)
    _load().orc_residual_tensor(ctypes.byref(_desc(dims, R)), _ptr(X), _ptr(_pack(A)), _ptr(E))
    return E


def unfold_gram(X, n):
    """S = X_(n) X_(n)^T (FP64)."""
    X = _x64(X)
    dims = list(X.shape)
    S = np.empty((dims[n], dims[n]))
    _load().orc_unfold_gram(ctypes.byref(_desc(dims, 1)), _ptr(X), int(n), _ptr(S))
    return S


def sym_eig(S):
    """Cyclic Jacobi eigen-decomposition: (w decreasing, V with eigenvector columns)."""
    s = S.shape[0]
    A = np.ascontiguousarray(S, dtype=np.float64).copy()
    w, V = np.empty(s), np.empty((s, s))
    _load().orc_sym_eig(int(s), _ptr(A), _ptr(w), _ptr(V))
    return w, V


def mode_product_t(T, n, U):
    """T x_n U^T (U: s_n x r)."""
    T = np.ascontiguousarray(T, dtype=np.float64)
    dims = list(T.shape)
    r = U.shape[1]
    out = list(dims)
    out[n] = r
    Y = np.empty(out)
    d = (ctypes.c_int64 * len(dims))(*dims)
    _load().orc_mode_product_t(len(dims), d, _ptr(T), int(n), int(r), _ptr(np.ascontiguousarray(U, np.float64)),
                               _ptr(Y))
    return Y


def hosvd(X, ranks):
    """Truncated higher-order SVD (Tucker compression): U_n = the eigenvectors of
    X_(n) X_(n)^T of the ranks[n] largest eigenvalues; core = X x_1 U_1^T ... x_N U_N^T.
    Returns (U list, core, eigenvalue lists)."""
    X = _x64(X)
    U, W = [], []
    for n in range(X.ndim):
        w, V = sym_eig(unfold_gram(X, n))
        U.append(np.ascontiguousarray(V[:, :ranks[n]]))
        W.append(w)
    core = X
    for n in range(X.ndim):
        core = mode_product_t(core, n, U[n])
    return U, core, W


def als_sweep(X, A, lam=0.0):
    X = _x64(X)
    dims, R = list(X.shape), A[0].shape[1]
    Abuf = _pack(A)
    st = _load().orc_als_sweep(ctypes.byref(_desc(dims, R)), _ptr(X), _ptr(Abuf), float(lam))
    return _unpack(Abuf, dims, R), st


def default_lambda(A, lo_ratio=1e-7, hi_ratio=1e-1):
    """The lambda thresholds used by this project (a chosen convention, the
    paper gives none): tau = mean_n trace(Gamma^(n,n)) / R at the starting
    point, lambda_hi = hi_ratio * tau, lambda_lo = lo_ratio * tau."""
    G = gamma(gram(A))
    N, R = G.shape[0], G.shape[2]
    tau = float(np.mean([np.trace(G[n, n]) for n in range(N)]) / R)
    return hi_ratio * tau, lo_ratio * tau
