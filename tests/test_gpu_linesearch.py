"""Step-size control by Armijo's condition and the damping variants (Section
3.2's lambda diag(J^T J), constant lambda) in cp_gn_step and the batched
solver, against the oracle's GN step with the same options.

Tolerances: the FP64 step as the other FP64 tests (the applied update t V to
1e-12 of its largest entry, the entry objective to 1e-12); the batched
solver's FP32 vectors to its one-step bound (2e-4 of the update's norm).  The
step length t is an exact decision; the cases are chosen with a clear margin
(the full step raises f by 40%, the half step lowers it by 17%)."""
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


def _dev(torch, arrs):
    return [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in arrs]


def _armijo_case(orc):
    """6x5x7 random tensor, R = 4, after two plain GN steps at constant
    lambda = 1e-4: the full third step raises the objective (84.75 -> 121.76),
    Armijo's condition accepts t = 1/2 (70.17)."""
    rng = np.random.default_rng(0)
    dims, R = (6, 5, 7), 4
    X = rng.standard_normal(dims)
    A = [rng.standard_normal((s, R)) for s in dims]
    for _ in range(2):
        A, _, _, _, _ = orc.gn_step_ls(X, A, 1e-4, 0, 1e-9, 1.0, 2.0, 1e-10, 60, lam_fixed=True)
    return X, A


@pytest.mark.parametrize("reg", ["identity", "diag"])
def test_gn_step_armijo_matches_oracle(env, orc, reg):
    torch, api, h = env
    X, A = _armijo_case(orc)
    k = 12
    kind = orc.REG_DIAG if reg == "diag" else orc.REG_IDENTITY
    lam = 1e-4
    Ad = _dev(torch, A)
    params = api.gn_params(lam, 1e-9, 1.0, eps_cg=0.0, cg_max_iter=k, prec="fp64", lam_fixed=True, reg=reg,
                           armijo_c=1e-4, armijo_beta=0.5, armijo_max=10)
    s, st = api.cp_gn_step(h, torch.from_numpy(X).cuda(), Ad, params)
    Ao, lam_o, _, so, sto = orc.gn_step_ls(X, A, lam, 0, 1e-9, 1.0, 2.0, 0.0, k, reg=kind, lam_fixed=True,
                                           armijo_c=1e-4, armijo_beta=0.5, armijo_max=10)
    assert s == sto and st["cg_iters"] == so["cg_iters"] == k
    assert st["step"] == so["step"] and st["ls_trials"] == so["trials"], (st["step"], so["step"])
    assert abs(st["f_entry"] - so["f0"]) <= 1e-12 * so["f0"]
    V = [a.cpu().numpy() - a0 for a, a0 in zip(Ad, A)]
    Vo = [a - a0 for a, a0 in zip(Ao, A)]
    scale = max(np.abs(v).max() for v in Vo)
    assert max(np.abs(v - vo).max() for v, vo in zip(V, Vo)) <= 1e-12 * scale
    assert params.lam == lam_o == lam  # constant lambda
    if reg == "identity":
        assert st["step"] == 0.5


def test_gn_step_armijo_full_step_and_fp32(env, orc):
    """Near an exact decomposition the full step is taken (one trial), also
    with the mixed path's FP32 CG and residual-form gradient."""
    torch, api, h = env
    from paper_1910_12331_gb300 import datagen

    p = datagen.workload("exact20", seed=0)
    rng = np.random.default_rng(5)
    A = [a + 1e-4 * rng.standard_normal(a.shape) for a in p["truth"]]
    X32 = p["X"].astype(np.float32)
    hi, lo = orc.default_lambda(A)
    for prec in ("fp64", "residual"):
        Ad = _dev(torch, A)
        params = api.gn_params(1e-3 * hi, lo, hi, eps_cg=1e-3, cg_max_iter=100, prec=prec, lam_fixed=True,
                               armijo_c=1e-4)
        X = torch.from_numpy(p["X"] if prec == "fp64" else X32).cuda()
        _, st = api.cp_gn_step(h, X, Ad, params)
        assert st["step"] == 1.0 and st["ls_trials"] == 1, (prec, st)


def test_gn_step_armijo_argument_checks(env):
    torch, api, h = env
    rng = np.random.default_rng(1)
    A = _dev(torch, [rng.standard_normal((s, 2)) for s in (4, 5, 6)])
    X = torch.from_numpy(rng.standard_normal((4, 5, 6))).cuda()
    for c, beta, mx in [(1.5, 0.5, 3), (-0.1, 0.5, 3), (1e-4, 1.0, 3), (1e-4, 0.0, 3), (1e-4, 0.5, -1)]:
        params = api.gn_params(0.1, 1e-6, 1.0, armijo_c=c, armijo_beta=beta, armijo_max=mx)
        s, _ = api.cp_gn_step(h, X, A, params, check=False)
        assert s == api.CP_ERR_ARG


def _batched_prob(torch, X, A, lam, **kw):
    q = dict(X=torch.from_numpy(np.ascontiguousarray(X, dtype=np.float32)).cuda(), A=_dev(torch, A), lam=lam,
             lam_lo=1e-9, lam_hi=1.0, mu=2.0)
    q.update(kw)
    return q


@pytest.mark.parametrize("opts", [dict(reg="diag"), dict(lam_fixed=True), dict(lam_fixed=True, armijo_c=1e-4)])
def test_batched_one_step_options(env, orc, opts):
    """One batched GN iteration with each option, against the oracle's step on
    the same FP32-stored tensor (FP32 vectors: the one-step bound 2e-4)."""
    torch, api, h = env
    X, A = _armijo_case(orc)
    X = X.astype(np.float32)
    k, lam = 12, (0.05 if opts.get("reg") == "diag" else 1e-4)
    q = _batched_prob(torch, X, A, lam, **opts)
    res = api.cp_gn_solve_batched(h, [q], eps_cg=0.0, cg_max_iter=k, max_iters=1, target_residual=0.0)[0]
    assert res["status"] == 0 and res["iters"] == 1 and res["cg_iters_total"] == k
    kind = orc.REG_DIAG if opts.get("reg") == "diag" else orc.REG_IDENTITY
    Ao, lam_o, _, so, _ = orc.gn_step_ls(X, A, lam, 0, 1e-9, 1.0, 2.0, 0.0, k, reg=kind,
                                         lam_fixed=opts.get("lam_fixed", False), armijo_c=opts.get("armijo_c", 0.0))
    if "armijo_c" in opts:
        assert so["step"] == 0.5 and res["ls_backtracks"] == 1
    d_gpu = [a.cpu().numpy() - a0 for a, a0 in zip(q["A"], A)]
    d_ref = [b - a0 for b, a0 in zip(Ao, A)]
    num = np.sqrt(sum(np.sum((x - y) ** 2) for x, y in zip(d_gpu, d_ref)))
    den = np.sqrt(sum(np.sum(y ** 2) for y in d_ref))
    assert num <= 2e-4 * den, num / den
    assert res["lam"] == lam_o or not opts.get("lam_fixed")


def test_batched_armijo_converges_where_plain_gn_stalls(env, orc):
    """The mixed batch of the benchmark's recipe (sides 16..96, ranks 4..24,
    1e-8 noise), solved with and without Armijo's condition: the line search
    loses no more than one problem plain GN solves (its backtracks are
    reported)."""
    torch, api, h = env
    from paper_1910_12331_gb300 import datagen

    probs = datagen.batched_problems(128, seed=0)
    def mk(armijo):
        out = []
        for p in probs:
            hi, lo = orc.default_lambda(p["init"])
            q = dict(X=torch.from_numpy(p["X"]).cuda(), A=_dev(torch, [a.copy() for a in p["init"]]), lam=hi,
                     lam_lo=lo, lam_hi=hi, mu=2.0)
            if armijo:
                q.update(armijo_c=1e-4, armijo_beta=0.5, armijo_max=10)
            out.append(q)
        return out
    plain = api.cp_gn_solve_batched(h, mk(False), 1e-3, 250, 200, 1e-6)
    ls = api.cp_gn_solve_batched(h, mk(True), 1e-3, 250, 200, 1e-6)
    n_plain = sum(r["converged"] for r in plain)
    n_ls = sum(r["converged"] for r in ls)
    print("converged: plain", n_plain, "armijo", n_ls, "backtracks", sum(r["ls_backtracks"] for r in ls))
    assert n_ls >= n_plain - 1
