"""GPU parity of the API branches that the other files leave out: the CUDA-core
reconstruction of the residual tensor at R > 64, the tensor-core
reconstruction with an FP64 X, the bf16x3 ALS sweep, cp_gn_solve with the
FP64 refinement and with residual_every, calls on a non-default CUDA stream,
cp_workspace_size, the matvec's FP32 arithmetic and diagonal damping through
the C ABI, and order 8 (the largest order the header allows).

Tolerances (each from the arithmetic of its result):
- FP64 results: 1e-12 of the largest entry (the update V of a GN step
  relative to max |V|).
- bf16x3 MTTKRP: TOL_BF16X3 = 2e-5 of max |M| (two-part bf16 splits, 2^-16
  per part, FP32 accumulation; the same bound as tests/test_gpu_tc.py).
- residual-form gradient: 5 TOL_BF16X3 of max |G| (the split error of the
  MTTKRP of E scales with E; the reconstruction of E itself is exact to far
  below that).
- FP32 matvec: A, W and Gamma are rounded to FP32 (2^-24 each) and every
  product and sum rounds at 2^-24.  The longest chain of sums behind an
  entry of Q is the s_p rows of Y^(p) = A^(p)T W^(p) followed by the (N + 1) R
  terms of Q, so each entry is within 2 (max_p s_p + (N + 1) R + 4) 2^-24 of
  the same matvec evaluated on |A|, |W| and |Gamma| (the sum of the term
  magnitudes), the standard bound for recursive summation.
- bf16x3 ALS sweep: each mode update is M^(n) Gamma^(n)^-1 with M^(n) to
  TOL_BF16X3 max |M^(n)|, so the update carries at most
  cond(Gamma^(n)) TOL_BF16X3 relative error, and the later modes of the sweep
  see it once more; 10 cond TOL_BF16X3 bounds the whole sweep."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL = 1e-12
TOL_BF16X3 = 2e-5


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


def _dev(torch, arrs):
    return [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in arrs]


def _host(ts):
    return [t.cpu().numpy() for t in ts]


def _relerr(got, ref):
    scale = max(np.abs(r).max() for r in ref)
    return max(np.abs(g - r).max() for g, r in zip(got, ref)) / scale


def _near_exact(dims, R, seed, eps, xdt=np.float32):
    """X = [[T]] + noise, A = T + eps-perturbation: a point near the optimum
    where G = A Gamma - M cancels to |G| << |M|."""
    from tests import cpref

    rng = np.random.default_rng(seed)
    T = [rng.standard_normal((s, R)) for s in dims]
    X = cpref.reconstruct(T)
    X = (X + 1e-6 * np.linalg.norm(X) / np.sqrt(X.size) * rng.standard_normal(dims)).astype(xdt)
    A = [t + eps * rng.standard_normal(t.shape) for t in T]
    return X, A


def _oracle_grad(orc, X, A):
    M = orc.mttkrp(X, A, "def")
    G, gn = orc.gradient(A, orc.gamma(orc.gram(A)), M)
    return G, gn, M


# ------------------------------------------------ residual tensor: both kernels, both X types

@pytest.mark.parametrize("dims,R", [((130, 9, 140), 80), ((70, 6, 90), 100), ((20, 7, 5, 33), 72)])
@pytest.mark.parametrize("eps", [1e-6, None])
def test_residual_gradient_cuda_core_reconstruction(env, orc, dims, R, eps):
    """R > 64: the residual tensor comes from the CUDA-core kernel (extended
    FP32 arithmetic, rank loop in chunks of 32); near the optimum and far from it."""
    torch, api, h = env
    if eps is None:
        rng = np.random.default_rng(41)
        A = [rng.standard_normal((s, R)) for s in dims]
        X = rng.standard_normal(dims).astype(np.float32)
    else:
        X, A = _near_exact(dims, R, 42, eps)
    G, gn, _ = api.cp_gradient(h, torch.from_numpy(X).cuda(), _dev(torch, A), prec="residual")
    Go, gno, _ = _oracle_grad(orc, X, A)
    assert _relerr(_host(G), Go) <= 5 * TOL_BF16X3
    np.testing.assert_allclose(gn, gno, rtol=5 * TOL_BF16X3)


@pytest.mark.parametrize("dims,R,eps", [((130, 9, 140), 50, 1e-6), ((37, 70, 45), 13, None), ((40, 6, 8, 36), 20, 1e-5)])
def test_residual_gradient_fp64_x(env, orc, dims, R, eps):
    """The tensor-core reconstruction with an FP64 X (the subtraction from x
    in FP64, X read element by element under row and column bounds)."""
    torch, api, h = env
    if eps is None:
        rng = np.random.default_rng(43)
        A = [rng.standard_normal((s, R)) for s in dims]
        X = rng.standard_normal(dims)
    else:
        X, A = _near_exact(dims, R, 44, eps, np.float64)
    G, gn, _ = api.cp_gradient(h, torch.from_numpy(X).cuda(), _dev(torch, A), prec="residual")
    Go, gno, _ = _oracle_grad(orc, X, A)
    assert _relerr(_host(G), Go) <= 5 * TOL_BF16X3
    np.testing.assert_allclose(gn, gno, rtol=5 * TOL_BF16X3)


# ------------------------------------------------ ALS at bf16x3

@pytest.mark.parametrize("dims,R", [((60, 50, 70), 8), ((130, 9, 140), 20), ((12, 10, 9, 11), 5)])
def test_als_sweep_bf16x3(env, orc, dims, R):
    """One ALS sweep (Section 2.2) with the mode-by-mode tensor-core MTTKRP."""
    torch, api, h = env
    rng = np.random.default_rng(45)
    A = [rng.standard_normal((s, R)) for s in dims]
    X = rng.standard_normal(dims).astype(np.float32)
    Ad = _dev(torch, A)
    r = api.cp_als_sweep(h, torch.from_numpy(X).cuda(), Ad, 0.0, prec="bf16x3")
    Ao, _ = orc.als_sweep(X, A, 0.0)
    # cond(Gamma^(n)) along the oracle's own sweep
    cur = [a.copy() for a in A]
    cond = 1.0
    for n in range(len(A)):
        Gam = orc.gamma(orc.gram(cur))
        cond = max(cond, np.linalg.cond(Gam[n, n]))
        cur[n] = Ao[n]
    err = _relerr(_host(Ad), Ao)
    assert err <= 10 * cond * TOL_BF16X3, (err, cond)
    ro = orc.residual(X, Ao)
    assert abs(r - ro) <= 10 * cond * TOL_BF16X3 * ro


# ------------------------------------------------ cp_gn_solve options

def test_solve_refine_fp64(env, orc):
    """bf16x3 gradient, switching to the plain FP64 gradient (refine_prec =
    fp64) below stationarity 3e-5: the end state is stationary to 1e-8 by the
    oracle's FP64 gradient."""
    torch, api, h = env
    from paper_1910_12331_gb300 import datagen

    p = datagen.make_problem((48, 40, 36), 6, "normal", None, 1e-6, np.float32, seed=11)
    hi, lo = orc.default_lambda(p["init"])
    Ad = _dev(torch, p["init"])
    params = api.gn_params(hi, lo, hi, prec="bf16x3")
    opts = api.solve_opts(max_iters=200, target_stationarity=1e-8, refine_below=3e-5, refine_prec="fp64")
    _, res = api.cp_gn_solve(h, torch.from_numpy(p["X"]).cuda(), Ad, params, opts)
    assert res["converged"] == 1 and res["iters_refined"] >= 1
    A = _host(Ad)
    _, gn, M = _oracle_grad(orc, p["X"], A)
    assert gn.sum() / sum(np.linalg.norm(m) for m in M) <= 1.01e-8


@pytest.mark.parametrize("every", [1, 3])
def test_solve_residual_every(env, orc, every):
    """residual_every = k evaluates the direct residual after every k-th
    update; the last one reported equals the oracle's residual at the factors
    it was taken at (the solve is stopped right after such an update)."""
    torch, api, h = env
    from paper_1910_12331_gb300 import datagen

    p = datagen.workload("exact20", seed=1)
    hi, lo = orc.default_lambda(p["init"])
    X = torch.from_numpy(p["X"]).cuda()
    Ad = _dev(torch, p["init"])
    params = api.gn_params(hi, lo, hi)
    opts = api.solve_opts(max_iters=2 * every, residual_every=every)
    _, res = api.cp_gn_solve(h, X, Ad, params, opts)
    assert res["iters"] == 2 * every
    ro = orc.residual(p["X"], _host(Ad))
    assert abs(res["rel_residual"] - ro) <= 1e-12 * ro


# ------------------------------------------------ a non-default stream

def test_calls_on_side_stream(env, orc):
    """Every call enqueues on the handle's stream (torch's current stream in
    the binding): the same results on a side stream as on the oracle."""
    torch, api, h = env
    dims, R = (37, 70, 45), 9
    rng = np.random.default_rng(46)
    A = [rng.standard_normal((s, R)) for s in dims]
    X = rng.standard_normal(dims)
    X32 = X.astype(np.float32)
    side = torch.cuda.Stream()
    hi, lo = orc.default_lambda(A)
    with torch.cuda.stream(side):
        Xd, X32d = torch.from_numpy(X).cuda(), torch.from_numpy(X32).cuda()
        Ad = _dev(torch, A)
        M = api.cp_mttkrp_all(h, Xd, Ad, prec="fp64")
        Mt = api.cp_mttkrp_all(h, X32d, Ad, prec="bf16x3")
        G, _, _ = api.cp_gradient(h, X32d, Ad, prec="residual")
        As = _dev(torch, A)
        params = api.gn_params(hi, lo, hi, eps_cg=0.0, cg_max_iter=4)
        api.cp_gn_step(h, Xd, As, params)
        side.synchronize()
    Mo = orc.mttkrp(X, A, "def")
    assert _relerr(_host(M), Mo) <= TOL
    assert _relerr(_host(Mt), orc.mttkrp(X32, A, "def")) <= TOL_BF16X3
    Go, _, _ = _oracle_grad(orc, X32, A)
    assert _relerr(_host(G), Go) <= 5 * TOL_BF16X3
    Ao, _, _, _, _ = orc.gn_step(X, A, hi, 0, lo, hi, 2.0, 0.0, 4)
    V = [a - a0 for a, a0 in zip(_host(As), A)]
    Vo = [a - a0 for a, a0 in zip(Ao, A)]
    assert _relerr(V, Vo) <= TOL


# ------------------------------------------------ workspace query

def test_workspace_size_bounds_allocation(env):
    """cp_workspace_size is an upper bound of what a handle allocates: the
    device memory a fresh handle takes for a residual-form gradient, after the
    modules are loaded, stays below the reported bytes plus one allocation
    granule per buffer."""
    torch, api, h = env
    dims, R = (200, 60, 180), 40
    rng = np.random.default_rng(47)
    X = torch.from_numpy(rng.standard_normal(dims).astype(np.float32)).cuda()
    A = _dev(torch, [rng.standard_normal((s, R)) for s in dims])
    sizes = {p: api.cp_workspace_size(h, X, R, p) for p in ("fp64", "bf16x3", "residual")}
    assert 0 < sizes["fp64"][0] <= sizes["bf16x3"][0] <= sizes["residual"][0]
    assert sizes["fp64"][1] == sizes["residual"][1] == 0
    assert sizes["bf16x3"][1] >= 4 * X.numel()  # two bf16 planes of X
    G = [torch.empty_like(a) for a in A]  # outputs allocated before the measurement
    api.cp_gradient(h, X, A, G, prec="residual")  # modules loaded
    torch.cuda.synchronize()
    h2 = api.Handle(0)
    free0 = torch.cuda.mem_get_info()[0]
    api.cp_gradient(h2, X, A, G, prec="residual")
    torch.cuda.synchronize()
    used = free0 - torch.cuda.mem_get_info()[0]
    h2.close()
    assert used <= sizes["residual"][0] + 32 * (2 << 20), (used, sizes["residual"][0])


# ------------------------------------------------ matvec through the C ABI: FP32 arithmetic, damping, Grams

@pytest.mark.parametrize("dims,R", [((37, 70, 45), 13), ((6, 5, 4, 7), 4), ((30, 20), 9)])
@pytest.mark.parametrize("reg", ["identity", "diag"])
def test_matvec_fp64_damping_and_grams(env, orc, dims, R, reg):
    torch, api, h = env
    rng = np.random.default_rng(48)
    A = [rng.standard_normal((s, R)) for s in dims]
    W = [rng.standard_normal((s, R)) for s in dims]
    lam = 0.3
    Ad, Wd = _dev(torch, A), _dev(torch, W)
    Q = api.cp_gn_matvec(h, Ad, Wd, lam, reg=reg)
    ref = orc.matvec(A, orc.gamma(orc.gram(A)), W, lam, reg=orc.REG_DIAG if reg == "diag" else orc.REG_IDENTITY)
    assert _relerr(_host(Q), ref) <= TOL
    grams = torch.from_numpy(np.stack(orc.gram(A))).cuda()
    Qg = api.cp_gn_matvec(h, Ad, Wd, lam, grams=grams, reg=reg)
    assert _relerr(_host(Qg), ref) <= TOL


@pytest.mark.parametrize("dims,R", [((37, 70, 45), 13), ((400, 400, 400), 50), ((6, 5, 4, 7), 4)])
@pytest.mark.parametrize("reg", ["identity", "diag"])
def test_matvec_fp32_arithmetic(env, orc, dims, R, reg):
    """The matvec in the FP32 arithmetic of the mixed CG, against the FP64
    oracle, within the FP32 rounding bound of its sums."""
    torch, api, h = env
    rng = np.random.default_rng(49)
    A = [rng.standard_normal((s, R)) for s in dims]
    W = [rng.standard_normal((s, R)) for s in dims]
    lam = 0.25
    kind = orc.REG_DIAG if reg == "diag" else orc.REG_IDENTITY
    Q = _host(api.cp_gn_matvec(h, _dev(torch, A), _dev(torch, W), lam, reg=reg, prec="bf16x3"))
    Gam = orc.gamma(orc.gram(A))
    ref = orc.matvec(A, Gam, W, lam, reg=kind)
    # the same matvec on |A|, |W|, |Gamma|: the sum of the magnitudes of every term
    Aa, Wa = [np.abs(a) for a in A], [np.abs(w) for w in W]
    mag = orc.matvec(Aa, orc.gamma(orc.gram(Aa)), Wa, lam, reg=kind)
    N = len(dims)
    bound = 2 * (max(dims) + (N + 1) * R + 4) * 2.0 ** -24
    for q, r, m in zip(Q, ref, mag):
        assert np.all(np.abs(q - r) <= bound * m + 1e-300)
    assert _relerr(Q, ref) > 1e-12  # it really ran in FP32


# ------------------------------------------------ order 8

DIMS8, R8 = (3, 2, 3, 2, 2, 3, 2, 3), 3


def test_order8_mttkrp_fp64_and_bf16x3(env, orc):
    torch, api, h = env
    rng = np.random.default_rng(50)
    A = [rng.standard_normal((s, R8)) for s in DIMS8]
    X = rng.standard_normal(DIMS8)
    Ad = _dev(torch, A)
    M = api.cp_mttkrp_all(h, torch.from_numpy(X).cuda(), Ad, prec="fp64")
    Mo = orc.mttkrp(X, A, "def")
    assert _relerr(_host(M), Mo) <= TOL
    X32 = X.astype(np.float32)
    Mt = api.cp_mttkrp_all(h, torch.from_numpy(X32).cuda(), Ad, prec="bf16x3")
    assert _relerr(_host(Mt), orc.mttkrp(X32, A, "def")) <= TOL_BF16X3


def test_order8_gn_step_and_residual_gradient(env, orc):
    torch, api, h = env
    rng = np.random.default_rng(51)
    A = [rng.standard_normal((s, R8)) for s in DIMS8]
    X = rng.standard_normal(DIMS8)
    hi, lo = orc.default_lambda(A)
    Ad = _dev(torch, A)
    params = api.gn_params(hi, lo, hi, eps_cg=0.0, cg_max_iter=3)
    s, st = api.cp_gn_step(h, torch.from_numpy(X).cuda(), Ad, params)
    Ao, lam_o, dir_o, so, sto = orc.gn_step(X, A, hi, 0, lo, hi, 2.0, 0.0, 3)
    assert s == sto == api.CP_WARN_CG_MAXIT and st["cg_iters"] == 3
    V = [a - a0 for a, a0 in zip(_host(Ad), A)]
    Vo = [a - a0 for a, a0 in zip(Ao, A)]
    assert _relerr(V, Vo) <= TOL
    assert abs(st["grad_norm_sum"] - so["grad_norm_sum"]) <= TOL * so["grad_norm_sum"]
    X32 = X.astype(np.float32)
    G, _, _ = api.cp_gradient(h, torch.from_numpy(X32).cuda(), _dev(torch, A), prec="residual")
    Go, _, _ = _oracle_grad(orc, X32, A)
    assert _relerr(_host(G), Go) <= 5 * TOL_BF16X3
    r = api.cp_residual(h, torch.from_numpy(X).cuda(), _dev(torch, A))
    assert abs(r - orc.residual(X, A)) <= TOL * orc.residual(X, A)
