"""Parity of the tcgen05 bf16x3 MTTKRP (through the C ABI) with the FP64 oracle.

The split products carry about 2^-16 relative error each; the bound used here,
max |M_gpu - M_oracle| <= TOL_BF16X3 * max |M_oracle| per call, was set from
measurement and holds with margin on these shapes, which cover
ragged i-blocks and k-chunks, several k-groups, several rank tiles, orders 2-5."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL_BF16X3 = 2e-5

SHAPES = [((37, 70, 45), 13), ((20, 20, 20), 5), ((130, 3, 140), 64), ((300, 5, 520), 20), ((6, 5, 4, 7), 4),
          ((50, 70), 9), ((40, 30, 50), 100), ((3, 4, 2, 3, 2), 2), ((129, 9, 127), 50), ((64, 33, 8), 1)]


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


def _problem(dims, R, seed, xdt=np.float32):
    rng = np.random.default_rng(seed)
    A = [rng.standard_normal((s, R)) for s in dims]
    X = rng.standard_normal(dims).astype(xdt)
    return X, A


@pytest.mark.parametrize("dims,R", SHAPES)
def test_mttkrp_bf16x3(env, orc, dims, R):
    torch, api, h = env
    X, A = _problem(dims, R, 1)
    Ad = [torch.from_numpy(a).cuda() for a in A]
    M = api.cp_mttkrp_all(h, torch.from_numpy(X).cuda(), Ad, prec="bf16x3")
    ref = orc.mttkrp(X, A, "def")
    errs = [np.abs(m.cpu().numpy() - r).max() / np.abs(r).max() for m, r in zip(M, ref)]
    print("bf16x3 rel err per mode", dims, R, ["%.2e" % e for e in errs])
    assert max(errs) <= TOL_BF16X3


def test_mttkrp_bf16x3_fp64_input_and_cache(env, orc):
    """FP64 X takes the same path (split once, cached by pointer/version); a
    version bump after changing X re-splits it."""
    torch, api, h = env
    X, A = _problem((33, 17, 40), 7, 2, np.float64)
    Xd = torch.from_numpy(X).cuda()
    Ad = [torch.from_numpy(a).cuda() for a in A]
    M1 = [m.cpu().numpy() for m in api.cp_mttkrp_all(h, Xd, Ad, prec="bf16x3")]
    ref = orc.mttkrp(X, A)
    assert max(np.abs(m - r).max() / np.abs(r).max() for m, r in zip(M1, ref)) <= TOL_BF16X3
    Xd.mul_(2.0)
    h.bump_version(Xd)
    M2 = [m.cpu().numpy() for m in api.cp_mttkrp_all(h, Xd, Ad, prec="bf16x3")]
    for a, b in zip(M1, M2):
        np.testing.assert_allclose(b, 2.0 * a, rtol=1e-6, atol=1e-6 * np.abs(a).max())


def test_mttkrp_bf16x3_new_tensor_at_freed_address(env, orc):
    """The split of X is cached by address, size, dtype and version: a new
    tensor that the caching allocator places where a freed one lived gets its
    own split (the binding's version stamps), not the stale one."""
    torch, api, h = env
    X1, A = _problem((48, 20, 36), 5, 8)
    X2, _ = _problem((48, 20, 36), 5, 9)
    Ad = [torch.from_numpy(a).cuda() for a in A]
    Xd = torch.from_numpy(X1).cuda()
    ptr = Xd.data_ptr()
    api.cp_mttkrp_all(h, Xd, Ad, prec="bf16x3")
    del Xd
    Xd = torch.from_numpy(X2).cuda()
    M = [m.cpu().numpy() for m in api.cp_mttkrp_all(h, Xd, Ad, prec="bf16x3")]
    ref = orc.mttkrp(X2, A)
    assert max(np.abs(m - r).max() / np.abs(r).max() for m, r in zip(M, ref)) <= TOL_BF16X3
    print("same address reused:", Xd.data_ptr() == ptr)


def test_mttkrp_bf16x3_exact_gradient_invariant(env):
    """At an exact decomposition M^(n) = A^(n) Gamma^(n): checked at 256^3, R=32,
    a size the oracle cannot brute-force, through the invariant alone."""
    torch, api, h = env
    from paper_1910_12331_gb300 import datagen

    p = datagen.workload("loss256", seed=0)
    Xd = torch.from_numpy(p["X"]).cuda()
    Ad = [torch.from_numpy(a).cuda() for a in p["truth"]]
    M = api.cp_mttkrp_all(h, Xd, Ad, prec="bf16x3")
    for n in range(3):
        G = torch.ones(32, 32, dtype=torch.float64, device="cuda")
        for m in range(3):
            if m != n:
                G *= Ad[m].T @ Ad[m]
        ref = Ad[n] @ G
        err = ((M[n] - ref).abs().max() / ref.abs().max()).item()
        assert err <= 3 * TOL_BF16X3, err


def _near_exact(dims, R, seed, eps):
    rng = np.random.default_rng(seed)
    T = [rng.standard_normal((s, R)) for s in dims]
    from tests import cpref

    X = cpref.reconstruct(T).astype(np.float32)
    A = [t + eps * rng.standard_normal(t.shape) for t in T]
    return X, A


@pytest.mark.parametrize("dims,R,eps", [((37, 70, 45), 6, 1e-6), ((30, 20, 24, 10), 5, 1e-5), ((130, 9, 140), 20, 1e-7)])
def test_gradient_residual_mode_near_optimum(env, orc, dims, R, eps):
    """G = -E_(n) P^(n) (E formed in double-float): near the optimum its error
    is far below the bf16x3 error of A Gamma - M; measured against sum|M|."""
    torch, api, h = env
    X, A = _near_exact(dims, R, 3, eps)
    Ad = [torch.from_numpy(a).cuda() for a in A]
    Xd = torch.from_numpy(X).cuda()
    Gr, gn, mn = api.cp_gradient(h, Xd, Ad, prec="residual")
    Gam = orc.gamma(orc.gram(A))
    M = orc.mttkrp(X, A)
    Go, gno = orc.gradient(A, Gam, M)
    msum = sum(np.linalg.norm(m) for m in M)
    err = sum(np.linalg.norm(g.cpu().numpy() - o) for g, o in zip(Gr, Go)) / msum
    Gb, _, _ = api.cp_gradient(h, Xd, Ad, prec="bf16x3")
    err_b = sum(np.linalg.norm(g.cpu().numpy() - o) for g, o in zip(Gb, Go)) / msum
    print("residual-mode gradient err", err, "bf16x3 err", err_b, "stationarity", sum(gno) / msum)
    stat = sum(gno) / msum
    # the error scales with |E|, i.e. with the stationarity, at the bf16x3 rate
    assert err <= 3 * TOL_BF16X3 * stat + 1e-12
    assert err < err_b / 10
    np.testing.assert_allclose(mn, [np.linalg.norm(m) for m in M], rtol=1e-9)


@pytest.mark.parametrize("dims,R", [((130, 9, 140), 16), ((130, 9, 140), 33), ((130, 9, 140), 48), ((130, 9, 140), 49),
                                    ((130, 9, 140), 50), ((140, 130, 150), 64), ((30, 20, 24, 10), 57), ((50, 70), 64)])
def test_gradient_residual_mode_ranks(env, orc, dims, R):
    """The residual tensor on the tensor cores covers ranks up to 64 (four
    16-column K-steps): the residual-form gradient near the optimum stays at
    the bf16x3 rate times the stationarity, for every rank count."""
    torch, api, h = env
    X, A = _near_exact(dims, R, 4, 1e-6)
    Gr, _, _ = api.cp_gradient(h, torch.from_numpy(X).cuda(), [torch.from_numpy(a).cuda() for a in A], prec="residual")
    Gam = orc.gamma(orc.gram(A))
    M = orc.mttkrp(X, A)
    Go, gno = orc.gradient(A, Gam, M)
    msum = sum(np.linalg.norm(m) for m in M)
    err = sum(np.linalg.norm(g.cpu().numpy() - o) for g, o in zip(Gr, Go)) / msum
    assert err <= 3 * TOL_BF16X3 * (sum(gno) / msum) + 1e-12


@pytest.mark.parametrize("R,rank", [(50, 48), (50, 49), (64, 56), (64, 63), (49, 48), (40, 35), (64, None), (50, None)])
def test_residual_exact_rank(env, orc, R, rank):
    """At an exact factorisation the residual tensor is only the FP32
    rounding of X, so the step's entry residual equals the oracle's; one
    nonzero rank column probes each 16-column K-step of the reconstruction on
    its own (a missing piece product would show at 1e-3)."""
    torch, api, h = env
    dims = (130, 9, 140)
    rng = np.random.default_rng(3)
    T = [rng.standard_normal((s, R)) for s in dims]
    if rank is not None:
        for t in T:
            t[:, np.arange(R) != rank] = 0.0
    from tests import cpref

    X = cpref.reconstruct(T).astype(np.float32)
    params = api.gn_params(1.0, 1e-9, 1.0, eps_cg=0.0, cg_max_iter=0, prec="residual", cg_fp32=True, lam_fixed=True)
    _, st = api.cp_gn_step(h, torch.from_numpy(X).cuda(), [torch.from_numpy(t.copy()).cuda() for t in T], params,
                           check=False)
    r = orc.residual(X, T)
    assert abs(st["entry_residual"] - r) <= 1e-3 * r


def test_residual_gradient_call_to_call_identical(env):
    """The residual tensor on the tensor cores is deterministic: repeated
    calls on one input (many CTAs, many runs per CTA, R = 50) are bit-identical."""
    torch, api, h = env
    rng = np.random.default_rng(21)
    dims, R = (384, 96, 320), 50
    A = [torch.from_numpy(rng.standard_normal((s, R))).cuda() for s in dims]
    X = torch.from_numpy(rng.standard_normal(dims).astype(np.float32)).cuda()
    ref = None
    for _ in range(8):
        G, _, _ = api.cp_gradient(h, X, A, prec="residual")
        g = [x.cpu().numpy() for x in G]
        if ref is None:
            ref = g
        else:
            for a, b in zip(g, ref):
                assert np.array_equal(a, b)


def test_gradient_residual_mode_far(env, orc):
    torch, api, h = env
    X, A = _problem((37, 70, 45), 13, 5)
    Gr, _, _ = api.cp_gradient(h, torch.from_numpy(X).cuda(), [torch.from_numpy(a).cuda() for a in A], prec="residual")
    Go, _ = orc.gradient(A, orc.gamma(orc.gram(A)), orc.mttkrp(X, A))
    M = orc.mttkrp(X, A)
    scale = max(np.abs(m).max() for m in M)
    assert max(np.abs(g.cpu().numpy() - o).max() for g, o in zip(Gr, Go)) / scale <= 5 * TOL_BF16X3


def test_step_entry_residual(env, orc):
    torch, api, h = env
    X, A = _near_exact((40, 30, 50), 7, 6, 1e-4)
    Ad = [torch.from_numpy(a).cuda() for a in A]
    params = api.gn_params(1e-3, 1e-9, 1e-3, prec="residual", cg_fp32=True)
    _, st = api.cp_gn_step(h, torch.from_numpy(X).cuda(), Ad, params)
    r = orc.residual(X, A)
    assert abs(st["entry_residual"] - r) <= 1e-6 * r


def test_mixed_solve_reaches_fp64_stationarity(env, orc):
    """The mixed path (bf16x3 gradient, FP32 CG, residual-tensor refinement)
    meets sum|G|/sum|M| <= 1e-8 as judged by the FP64 oracle's gradient."""
    torch, api, h = env
    from paper_1910_12331_gb300 import datagen

    p = datagen.make_problem((48, 40, 36), 6, "normal", None, 1e-6, np.float32, seed=11)
    hi, lo = orc.default_lambda(p["init"])
    Ad = [torch.from_numpy(a.copy()).cuda() for a in p["init"]]
    params = api.gn_params(hi, lo, hi, prec="bf16x3")
    opts = api.solve_opts(max_iters=200, target_stationarity=1e-8, refine_below=3e-5)
    _, res = api.cp_gn_solve(h, torch.from_numpy(p["X"]).cuda(), Ad, params, opts)
    assert res["converged"] == 1 and res["iters_refined"] >= 1
    A = [a.cpu().numpy() for a in Ad]
    M = orc.mttkrp(p["X"], A)
    _, gn = orc.gradient(A, orc.gamma(orc.gram(A)), M)
    assert gn.sum() / sum(np.linalg.norm(m) for m in M) <= 2e-8


@pytest.mark.parametrize("dims,R,prec", [((130, 40, 70), 9, "bf16x3"), ((300, 60, 200), 24, "bf16x3"),
                                         ((300, 60, 200), 24, "residual")])
def test_mixed_solve_bit_reproducible(env, orc, dims, R, prec):
    """Every device reduction that feeds a decision has a fixed order (the
    gradient norms included): two solves from the same state give identical
    factors and iteration counts, bit for bit."""
    torch, api, h = env
    from paper_1910_12331_gb300 import datagen

    p = datagen.make_problem(dims, R, "normal", 0.5, 1e-6, np.float32, seed=12)
    hi, lo = orc.default_lambda(p["init"])
    X = torch.from_numpy(p["X"]).cuda()
    outs = []
    for _ in range(2):
        Ad = [torch.from_numpy(a.copy()).cuda() for a in p["init"]]
        params = api.gn_params(hi, lo, hi, prec=prec)
        opts = api.solve_opts(max_iters=12, target_stationarity=0.0, refine_below=3e-5)
        _, res = api.cp_gn_solve(h, X, Ad, params, opts)
        outs.append(([a.cpu().numpy() for a in Ad], res["cg_iters_total"], res["iters"]))
    (A1, c1, i1), (A2, c2, i2) = outs
    assert c1 == c2 and i1 == i2
    for a, b in zip(A1, A2):
        assert np.array_equal(a, b)
