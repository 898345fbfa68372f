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
