"""Parity of the plain FP64 CUDA path (through the C ABI) with the FP64 oracle.

Tolerance: 1e-12 relative to the largest magnitude of each result for the
FP64 path (MTTKRP, gradient, matvec, residual, per-step GN update with a
fixed CG iteration count, ALS sweep)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL = 1e-12

SHAPES = [((5, 7, 9), 3), ((6, 5, 4, 7), 4), ((8, 6), 3), ((20, 20, 20), 5), ((37, 70, 45), 67),
          ((3, 4, 2, 3, 2), 2), ((1, 9, 1), 2), ((33, 1, 65), 1), ((130, 3, 97), 9)]


@pytest.fixture(scope="module")
def env():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1910_12331_gb300 import api

    api.load(build_if_missing=True)
    h = api.Handle(0)
    yield torch, api, h
    h.close()


def _factors(dims, R, seed):
    rng = np.random.default_rng(seed)
    return [rng.standard_normal((s, R)) for s in dims]


def _tensor(dims, seed):
    return np.random.default_rng(seed + 7).standard_normal(dims)


def _dev(torch, arrs):
    return [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in arrs]


def _update(A_new, A_old):
    """V = A_new - A_old per mode (A_new: CUDA tensors or arrays)."""
    return [(a.cpu().numpy() if hasattr(a, "cpu") else a) - a0 for a, a0 in zip(A_new, A_old)]


def _relerr(got, ref):
    scale = max(np.abs(r).max() for r in ref)
    return max(np.abs(g - r).max() for g, r in zip(got, ref)) / scale


@pytest.mark.parametrize("dims,R", SHAPES)
@pytest.mark.parametrize("xdt", ["f64", "f32"])
def test_mttkrp_fp64(env, orc, dims, R, xdt):
    torch, api, h = env
    A = _factors(dims, R, 1)
    X = _tensor(dims, 1).astype(np.float64 if xdt == "f64" else np.float32)
    M = api.cp_mttkrp_all(h, torch.from_numpy(X).cuda(), _dev(torch, A), prec="fp64")
    ref = orc.mttkrp(X, A, "def")
    assert _relerr([m.cpu().numpy() for m in M], ref) <= TOL


@pytest.mark.parametrize("dims,R", SHAPES[:6])
def test_gradient_fp64(env, orc, dims, R):
    torch, api, h = env
    A = _factors(dims, R, 2)
    X = _tensor(dims, 2)
    G, gn, mn = api.cp_gradient(h, torch.from_numpy(X).cuda(), _dev(torch, A), prec="fp64")
    Gam = orc.gamma(orc.gram(A))
    M = orc.mttkrp(X, A)
    Gr, gnr = orc.gradient(A, Gam, M)
    # G cancels near the optimum; measure against the scale of M (and A Gamma)
    scale = max(np.abs(m).max() for m in M)
    err = max(np.abs(g.cpu().numpy() - r).max() for g, r in zip(G, Gr)) / scale
    assert err <= TOL
    np.testing.assert_allclose(gn, gnr, rtol=1e-10)
    np.testing.assert_allclose(mn, [np.linalg.norm(m) for m in M], rtol=1e-12)


@pytest.mark.parametrize("dims,R", SHAPES[:6])
@pytest.mark.parametrize("lam", [0.0, 0.25])
def test_matvec_fp64(env, orc, dims, R, lam):
    torch, api, h = env
    A = _factors(dims, R, 3)
    W = _factors(dims, R, 4)
    Q = api.cp_gn_matvec(h, _dev(torch, A), _dev(torch, W), lam)
    ref = orc.matvec(A, orc.gamma(orc.gram(A)), W, lam)
    assert _relerr([q.cpu().numpy() for q in Q], ref) <= TOL


@pytest.mark.parametrize("dims,R", SHAPES)
def test_residual_fp64(env, orc, dims, R):
    torch, api, h = env
    A = _factors(dims, R, 5)
    X = _tensor(dims, 5)
    r = api.cp_residual(h, torch.from_numpy(X).cuda(), _dev(torch, A))
    assert abs(r - orc.residual(X, A)) <= 1e-12 * orc.residual(X, A)


def test_residual_exact_zero(env, orc):
    torch, api, h = env
    from paper_1910_12331_gb300 import datagen

    p = datagen.workload("exact20", seed=0)
    r = api.cp_residual(h, torch.from_numpy(p["X"]).cuda(), _dev(torch, p["truth"]))
    assert r <= 1e-15


@pytest.mark.parametrize("dims,R,k", [((20, 20, 20), 5, 5), ((6, 5, 4, 7), 4, 7), ((37, 70, 45), 9, 4),
                                      ((8, 6), 3, 3)])
@pytest.mark.parametrize("cg_fp32", [False])
def test_gn_step_fixed_cg(env, orc, dims, R, k, cg_fp32):
    """One GN step from an identical state with a fixed CG iteration count."""
    torch, api, h = env
    A = _factors(dims, R, 6)
    X = _tensor(dims, 6)
    hi, lo = orc.default_lambda(A)
    Ad = _dev(torch, A)
    params = api.gn_params(hi, lo, hi, eps_cg=0.0, cg_max_iter=k, cg_fp32=cg_fp32)
    s, st = api.cp_gn_step(h, torch.from_numpy(X).cuda(), Ad, params)
    Ao, lam_o, dir_o, so, sto = orc.gn_step(X, A, hi, 0, lo, hi, 2.0, 0.0, k)
    assert st["cg_iters"] == so["cg_iters"] == k
    assert s == sto == api.CP_WARN_CG_MAXIT
    # the per-step update V itself (not A + V, which would hide an error in V behind |A|)
    assert _relerr(_update(Ad, A), _update(Ao, A)) <= TOL
    assert abs(st["grad_norm_sum"] - so["grad_norm_sum"]) <= TOL * so["grad_norm_sum"]
    assert params.lam == lam_o and params.lam_dir == dir_o


@pytest.mark.parametrize("dims,R,k", [((20, 20, 20), 5, 5), ((6, 5, 4, 7), 4, 7), ((37, 70, 45), 9, 4),
                                      ((8, 6), 3, 3), ((150, 120, 90), 12, 6)])
def test_gn_step_fixed_cg_fp32(env, orc, dims, R, k):
    """FP32 CG vectors (FP64 gradient, FP32 Gamma and preconditioner): the
    same k iterations as the FP64 oracle.  Each of the k steps rounds the
    vectors and the matrices to FP32 (2^-24) and the preconditioned system at
    lambda_hi has a condition number below 1e2 here, so the direction agrees
    to 1e2 * k * 2^-24 * (a few) < 1e-4."""
    torch, api, h = env
    A = _factors(dims, R, 6)
    X = _tensor(dims, 6)
    hi, lo = orc.default_lambda(A)
    Ad = _dev(torch, A)
    params = api.gn_params(hi, lo, hi, eps_cg=0.0, cg_max_iter=k, cg_fp32=True)
    s, st = api.cp_gn_step(h, torch.from_numpy(X).cuda(), Ad, params)
    Ao, _, _, so, sto = orc.gn_step(X, A, hi, 0, lo, hi, 2.0, 0.0, k)
    assert st["cg_iters"] == so["cg_iters"] == k
    assert s == sto == api.CP_WARN_CG_MAXIT
    d_gpu = [a.cpu().numpy() - a0 for a, a0 in zip(Ad, A)]
    d_orc = [a - a0 for a, a0 in zip(Ao, A)]
    assert _relerr(d_gpu, d_orc) <= 1e-4


@pytest.mark.parametrize("dims,R,k", [((20, 20, 20), 5, 5), ((6, 5, 4, 7), 4, 7), ((37, 70, 45), 9, 4),
                                      ((8, 6), 3, 3), ((130, 3, 97), 9, 3)])
def test_gn_step_diag_damping(env, orc, dims, R, k):
    """Damping by lam diag(J^T J) (Section 3.2): one FP64 GN step with k CG
    iterations against the oracle's step with the same damping."""
    torch, api, h = env
    A = _factors(dims, R, 16)
    X = _tensor(dims, 16)
    lam, lo, hi = 0.05, 1e-7, 0.1
    Ad = _dev(torch, A)
    params = api.gn_params(lam, lo, hi, eps_cg=0.0, cg_max_iter=k, reg="diag")
    s, st = api.cp_gn_step(h, torch.from_numpy(X).cuda(), Ad, params)
    Ao, lam_o, dir_o, so, sto = orc.gn_step(X, A, lam, 0, lo, hi, 2.0, 0.0, k, reg=orc.REG_DIAG)
    assert st["cg_iters"] == so["cg_iters"] == k
    assert s == sto == api.CP_WARN_CG_MAXIT
    got = [a.cpu().numpy() for a in Ad]
    assert _relerr(_update(got, A), _update(Ao, A)) <= TOL
    assert abs(st["grad_norm_sum"] - so["grad_norm_sum"]) <= TOL * so["grad_norm_sum"]
    assert st["lam_used"] == lam and params.lam == lam_o and params.lam_dir == dir_o
    # the damping option is honoured: lam I gives another step
    Ai, _, _, _, _ = orc.gn_step(X, A, lam, 0, lo, hi, 2.0, 0.0, k)
    assert _relerr(got, Ai) > 1e-6


@pytest.mark.parametrize("dims,R,k", [((20, 20, 20), 5, 5), ((150, 120, 90), 12, 6)])
def test_gn_step_diag_damping_cg_fp32(env, orc, dims, R, k):
    """The same with FP32 CG vectors; tolerance as for the FP32 CG step with
    lam I (the damped system at lam = 0.1 is as well conditioned)."""
    torch, api, h = env
    A = _factors(dims, R, 17)
    X = _tensor(dims, 17)
    lam, lo, hi = 0.1, 1e-7, 0.1
    Ad = _dev(torch, A)
    params = api.gn_params(lam, lo, hi, eps_cg=0.0, cg_max_iter=k, cg_fp32=True, reg="diag")
    s, st = api.cp_gn_step(h, torch.from_numpy(X).cuda(), Ad, params)
    Ao, _, _, so, sto = orc.gn_step(X, A, lam, 0, lo, hi, 2.0, 0.0, k, reg=orc.REG_DIAG)
    assert st["cg_iters"] == so["cg_iters"] == k
    assert s == sto == api.CP_WARN_CG_MAXIT
    d_gpu = [a.cpu().numpy() - a0 for a, a0 in zip(Ad, A)]
    d_orc = [a - a0 for a, a0 in zip(Ao, A)]
    assert _relerr(d_gpu, d_orc) <= 1e-4


def test_gn_step_damping_kind_rejected(env):
    torch, api, h = env
    A = _factors((5, 6, 7), 2, 18)
    X = torch.from_numpy(_tensor((5, 6, 7), 18)).cuda()
    Ad = _dev(torch, A)
    params = api.gn_params(0.1, 1e-7, 0.1)
    params.reg = 2
    s, _ = api.cp_gn_step(h, X, Ad, params, check=False)
    assert s == api.CP_ERR_ARG
    np.testing.assert_array_equal(Ad[0].cpu().numpy(), A[0])  # nothing ran


def test_gn_solve_diag_damping_recovery(env, orc):
    """Algorithm 1 with the varying lam applied to lam diag(J^T J) (lam between
    1e-7 and 0.1, dimensionless) recovers the 20^3 rank-5 exact decompositions."""
    torch, api, h = env
    from paper_1910_12331_gb300 import datagen

    for seed in range(4):
        p = datagen.workload("exact20", seed=seed)
        Ad = _dev(torch, p["init"])
        params = api.gn_params(0.1, 1e-7, 0.1, reg="diag")
        opts = api.solve_opts(max_iters=100, target_residual=1e-10)
        _, res = api.cp_gn_solve(h, torch.from_numpy(p["X"]).cuda(), Ad, params, opts)
        assert res["converged"] == 1 and res["rel_residual"] <= 1e-10


def test_gn_step_tolerance_stop(env, orc):
    torch, api, h = env
    from paper_1910_12331_gb300 import datagen

    p = datagen.workload("exact20", seed=2)
    hi, lo = orc.default_lambda(p["init"])
    Ad = _dev(torch, p["init"])
    params = api.gn_params(hi, lo, hi, eps_cg=1e-3, cg_max_iter=250)
    _, st = api.cp_gn_step(h, torch.from_numpy(p["X"]).cuda(), Ad, params)
    Ao, _, _, so, _ = orc.gn_step(p["X"], p["init"], hi, 0, lo, hi, 2.0, 1e-3, 250)
    assert st["cg_iters"] == so["cg_iters"]
    assert _relerr(_update(Ad, p["init"]), _update(Ao, p["init"])) <= TOL


def test_gn_exact_recovery(env, orc):
    """Algorithm 1 on the GPU recovers 20^3 rank-5 exact decompositions to r <= 1e-10."""
    torch, api, h = env
    from paper_1910_12331_gb300 import datagen

    for seed in range(4):
        p = datagen.workload("exact20", seed=seed)
        hi, lo = orc.default_lambda(p["init"])
        Ad = _dev(torch, p["init"])
        params = api.gn_params(hi, lo, hi)
        opts = api.solve_opts(max_iters=100, target_residual=1e-10)
        _, res = api.cp_gn_solve(h, torch.from_numpy(p["X"]).cuda(), Ad, params, opts)
        assert res["converged"] == 1 and res["rel_residual"] <= 1e-10
        assert orc.residual(p["X"], [a.cpu().numpy() for a in Ad]) <= 1e-10


@pytest.mark.parametrize("dims,R,lam", [((8, 7, 6), 3, 0.0), ((6, 5, 4, 7), 4, 0.3), ((30, 41, 12), 7, 0.0)])
def test_als_sweep_fp64(env, orc, dims, R, lam):
    torch, api, h = env
    A = _factors(dims, R, 8)
    X = _tensor(dims, 8)
    Ad = _dev(torch, A)
    r = api.cp_als_sweep(h, torch.from_numpy(X).cuda(), Ad, lam=lam)
    Ao, st = orc.als_sweep(X, A, lam)
    assert _relerr([a.cpu().numpy() for a in Ad], Ao) <= 1e-10
    assert abs(r - orc.residual(X, Ao)) <= 1e-10


# --------------------------------------------------------------- error paths

def test_nonfinite_reported(env):
    torch, api, h = env
    dims, R = (6, 5, 4), 2
    X = torch.from_numpy(_tensor(dims, 9)).cuda()
    X[1, 2, 3] = float("nan")
    Ad = _dev(torch, _factors(dims, R, 9))
    params = api.gn_params(1.0, 1e-6, 1.0)
    s, _ = api.cp_gn_step(h, X, Ad, params, check=False)
    assert s == api.CP_ERR_NONFINITE


def test_not_spd_reported(env):
    torch, api, h = env
    dims, R = (6, 5, 4), 3
    A = _factors(dims, R, 10)
    A[1][:, 2] = 0.0  # a zero column: Gamma^(n,n) (n != 1) has a zero row, its pivot is exactly 0
    X = torch.from_numpy(_tensor(dims, 10)).cuda()
    params = api.gn_params(0.0, 0.0, 0.0, lam_fixed=True)
    s, _ = api.cp_gn_step(h, X, _dev(torch, A), params, check=False)
    assert s == api.CP_ERR_NOT_SPD


def test_barrier_timeout_reported(env):
    """A spin limit of one poll makes a grid barrier give up: the kernel returns
    CP_ERR_TIMEOUT through the status word and the context stays usable."""
    torch, api, h = env
    dims, R = (200, 180, 160), 8
    X = torch.from_numpy(_tensor(dims, 11)).cuda()
    A = _factors(dims, R, 11)
    params = api.gn_params(1.0, 1e-6, 1.0, eps_cg=0.0, cg_max_iter=50, spin_limit=1)
    s, _ = api.cp_gn_step(h, X, _dev(torch, A), params, check=False)
    assert s == api.CP_ERR_TIMEOUT
    # the context still works
    r = api.cp_residual(h, X, _dev(torch, A))
    assert np.isfinite(r)


def test_argument_errors(env):
    torch, api, h = env
    import ctypes

    dims, R = (4, 5, 6), 2
    X = torch.from_numpy(_tensor(dims, 12)).cuda()
    A = _dev(torch, _factors(dims, R, 12))
    L = api.load()
    d = h.desc(X, R)
    # output aliases an input
    arr = api._ptr_array(A)
    assert L.cp_mttkrp_all(h.h, ctypes.byref(d), X.data_ptr(), arr, arr, 0) == api.CP_ERR_ARG
    d.order = 9
    M = [torch.empty_like(a) for a in A]
    assert L.cp_mttkrp_all(h.h, ctypes.byref(d), X.data_ptr(), arr, api._ptr_array(M), 0) == api.CP_ERR_ARG
    d = h.desc(X, R)
    d.rank = 0
    assert L.cp_mttkrp_all(h.h, ctypes.byref(d), X.data_ptr(), arr, api._ptr_array(M), 0) == api.CP_ERR_ARG
