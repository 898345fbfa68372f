"""The batched solver (many small order-3 problems, one persistent launch):
one-step parity with the FP64 oracle at a fixed CG count, convergence of a
mixed batch checked by the oracle's residual, and argument checks."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


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


@pytest.fixture(scope="module")
def orc():
    import oracle

    oracle.build()
    return oracle


def _prob(torch, orc, dims, R, seed, noise=1e-8):
    from paper_1910_12331_gb300 import datagen

    p = datagen.make_problem(dims, R, "normal", None, noise, np.float32, seed=seed)
    hi, lo = orc.default_lambda(p["init"])
    return p, dict(X=torch.from_numpy(p["X"]).cuda(), A=[torch.from_numpy(a.copy()).cuda() for a in p["init"]],
                   lam=hi, lam_lo=lo, lam_hi=hi, mu=2.0)


@pytest.mark.parametrize("k", [1, 4])
def test_one_step_matches_oracle(env, orc, k):
    """One GN iteration with exactly k CG iterations (eps_cg = 0) from the same
    state as the oracle's step: FP32 vectors vs FP64, so the bound is FP32-level."""
    torch, api, h = env
    cases = [((17, 23, 19), 4, 1), ((40, 16, 33), 7, 2), ((24, 24, 24), 12, 3)]
    probs, data = [], []
    for dims, R, seed in cases:
        p, q = _prob(torch, orc, dims, R, seed)
        probs.append(q)
        data.append(p)
    res = api.cp_gn_solve_batched(h, probs, eps_cg=0.0, cg_max_iter=k, max_iters=1, target_residual=0.0)
    for p, q, r in zip(data, probs, res):
        assert r["status"] == 0 and r["iters"] == 1 and r["cg_iters_total"] == k
        A_ref, _, _, st, _ = orc.gn_step(p["X"], [a.copy() for a in p["init"]], q["lam"], 0, q["lam_lo"],
                                         q["lam_hi"], 2.0, 0.0, k, 0, False)
        for a, a0, b in zip(q["A"], p["init"], A_ref):
            d_gpu = a.cpu().numpy() - a0
            d_ref = b - a0
            assert np.linalg.norm(d_gpu - d_ref) <= 2e-4 * np.linalg.norm(d_ref) + 1e-12


def test_batch_converges(env, orc):
    """A batch of uneven sizes and ranks reaches r <= 1e-6; the oracle's FP64
    residual of the returned factors confirms it."""
    torch, api, h = env
    rng = np.random.default_rng(5)
    probs, data = [], []
    for s in range(10):
        dims = tuple(int(v) for v in rng.integers(16, 49, size=3))
        R = int(rng.integers(3, 9))
        p, q = _prob(torch, orc, dims, R, 100 + s)
        probs.append(q)
        data.append(p)
    res = api.cp_gn_solve_batched(h, probs, eps_cg=1e-3, cg_max_iter=250, max_iters=200, target_residual=1e-6)
    conv = [r for r in res if r["converged"]]
    assert len(conv) >= 8, res
    for p, q, r in zip(data, probs, res):
        assert r["status"] in (0,)
        if r["converged"]:
            rr = orc.residual(p["X"], [a.cpu().numpy() for a in q["A"]])
            assert rr <= 1.2e-6, (rr, r)


def test_argument_checks(env, orc):
    torch, api, h = env
    p, q = _prob(torch, orc, (10, 11, 12), 40, 1)
    with pytest.raises(api.CPError):  # rank above the batched limit
        api.cp_gn_solve_batched(h, [q])
    p, q = _prob(torch, orc, (250, 250, 250), 32, 1)
    with pytest.raises(api.CPError):  # shared memory above the per-block limit
        api.cp_gn_solve_batched(h, [q])
    assert api.cp_gn_solve_batched(h, []) == []


def _batch(torch, orc, count, seed0):
    rng = np.random.default_rng(seed0)
    probs = []
    for k in range(count):
        dims = tuple(int(x) for x in rng.integers(16, 49, size=3))
        R = int(rng.integers(4, 13))
        _, q = _prob(torch, orc, dims, R, seed0 + k)
        probs.append(q)
    return probs


def _snapshot(probs):
    return [[a.clone() for a in q["A"]] for q in probs]


def _restore(probs, snap):
    for q, s in zip(probs, snap):
        for a, b in zip(q["A"], s):
            a.copy_(b)


def test_plan_matches_one_shot(env, orc):
    """A plan (block size 256, no autotuning) launches the same kernel as the
    one-shot call: identical factors and results, bit for bit."""
    torch, api, h = env
    probs = _batch(torch, orc, 12, 500)
    snap = _snapshot(probs)
    r1 = api.cp_gn_solve_batched(h, probs, eps_cg=1e-3, cg_max_iter=100, max_iters=30, target_residual=1e-6)
    a1 = _snapshot(probs)
    _restore(probs, snap)
    plan = api.BatchPlan(h, probs, eps_cg=1e-3, cg_max_iter=100, max_iters=30, target_residual=1e-6, autotune=False)
    assert plan.threads == 256
    plan.launch()
    r2 = plan.results()
    plan.close()
    assert r1 == r2
    for x, y in zip(a1, _snapshot(probs)):
        for a, b in zip(x, y):
            assert torch.equal(a, b)


def test_plan_graph_replay(env, orc):
    """A plan launch captured in a CUDA graph and replayed from the same
    factors gives the same factors and results as a direct launch."""
    torch, api, h = env
    probs = _batch(torch, orc, 10, 600)
    snap = _snapshot(probs)
    plan = api.BatchPlan(h, probs, eps_cg=1e-3, cg_max_iter=100, max_iters=30, target_residual=1e-6, autotune=False)
    plan.launch()
    r_direct = plan.results()
    a_direct = _snapshot(probs)
    _restore(probs, snap)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        plan.launch()
    _restore(probs, snap)  # capture does not run the kernel; start the replay from the initial factors
    torch.cuda.synchronize()
    g.replay()
    torch.cuda.synchronize()
    r_graph = plan.results()
    plan.close()
    assert r_graph == r_direct
    for x, y in zip(a_direct, _snapshot(probs)):
        for a, b in zip(x, y):
            assert torch.equal(a, b)


# Shapes that reach every branch of the kernel: each register bucket of the rank sums (R <= 8, 16, 24, 32),
# third sides from under one warp to eight warps' worth (256), odd row counts (the two-row MTTKRP's tail),
# odd R (the register tiles' second column absent) and a rank above a side.
_VARIANT_CASES = [((17, 23, 19), 4, 11), ((9, 5, 3), 2, 12), ((16, 17, 256), 16, 13), ((45, 33, 70), 21, 14),
                  ((30, 31, 100), 28, 15), ((61, 20, 47), 13, 16), ((6, 40, 33), 9, 17)]


@pytest.mark.parametrize("threads", [128, 256, 384])
@pytest.mark.parametrize("order", [0, 1])
def test_every_variant_matches_oracle(env, orc, threads, order):
    """Each block size and problem order, fixed by cp_batch_plan_configure: one GN
    iteration with exactly three CG iterations from the oracle's state, per problem
    against the oracle's FP64 step (FP32 vectors, so an FP32-level bound)."""
    torch, api, h = env
    k = 3
    data, probs = [], []
    for dims, R, seed in _VARIANT_CASES:
        p, q = _prob(torch, orc, dims, R, seed)
        data.append(p)
        probs.append(q)
    plan = api.BatchPlan(h, probs, eps_cg=0.0, cg_max_iter=k, max_iters=1, target_residual=0.0, autotune=False)
    plan.configure(threads, order)
    assert plan.threads == threads and plan.order == order
    plan.launch()
    res = plan.results()
    plan.close()
    for p, q, r in zip(data, probs, res):
        assert r["status"] == 0 and r["iters"] == 1 and r["cg_iters_total"] == k
        A_ref, _, _, st, _ = orc.gn_step(p["X"], [a.copy() for a in p["init"]], q["lam"], 0, q["lam_lo"],
                                         q["lam_hi"], 2.0, 0.0, k, 0, False)
        for a, a0, b in zip(q["A"], p["init"], A_ref):
            d_gpu = a.cpu().numpy() - a0
            d_ref = b - a0
            assert np.linalg.norm(d_gpu - d_ref) <= 2e-4 * np.linalg.norm(d_ref) + 1e-12


def test_plan_configure_rejects_bad_arguments(env, orc):
    torch, api, h = env
    _, q = _prob(torch, orc, (8, 9, 10), 3, 5)
    plan = api.BatchPlan(h, [q], eps_cg=1e-3, cg_max_iter=10, max_iters=2, target_residual=1e-6, autotune=False)
    for threads, order in ((64, 0), (512, 0), (256, 2), (256, -1)):
        with pytest.raises(api.CPError):
            plan.configure(threads, order)
    assert plan.threads == 256 and plan.order == 0
    plan.close()


def test_plan_autotune(env, orc):
    """The autotuner times the block sizes on a scratch copy of the factors:
    the caller's factors are untouched by plan creation, the pick is one of
    the variants, and the tuned plan solves the batch."""
    torch, api, h = env
    probs = _batch(torch, orc, 16, 700)
    snap = _snapshot(probs)
    plan = api.BatchPlan(h, probs, eps_cg=1e-3, cg_max_iter=250, max_iters=200, target_residual=1e-6, autotune=True)
    for x, y in zip(snap, _snapshot(probs)):
        for a, b in zip(x, y):
            assert torch.equal(a, b)
    assert plan.threads in (128, 256, 384)
    plan.launch()
    res = plan.results()
    plan.close()
    assert sum(r["converged"] for r in res) >= 14
    for q, r in zip(probs, res):
        if r["converged"]:
            rr = orc.residual(q["X"].cpu().numpy(), [a.cpu().numpy() for a in q["A"]])
            assert rr <= 1.2e-6
