"""The CP loss autograd Function: forward and hand-written backward (fused
MTTKRP) against the FP64 oracle, finite differences, torch.autograd.gradcheck
and an einsum autograd reference of the same loss."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1910_12331_gb300 import api, autograd

    api.load(build_if_missing=True)
    h = api.Handle(0)
    yield torch, autograd, h
    h.close()


@pytest.fixture(scope="module")
def orc():
    import oracle

    oracle.build()
    return oracle


def _problem(torch, dims, R, seed, xdt):
    rng = np.random.default_rng(seed)
    A = [rng.standard_normal((s, R)) for s in dims]
    X = rng.standard_normal(dims).astype(xdt)
    return X, A


def _oracle_grad(orc, X, A):
    M = orc.mttkrp(X, A)
    G, _ = orc.gradient(A, orc.gamma(orc.gram(A)), M)
    return G, M


def _einsum_loss(torch, X, A):
    letters = "abcdefgh"[: X.dim()]
    spec = ",".join(l + "z" for l in letters) + "->" + letters
    return ((X.double() - torch.einsum(spec, *A)) ** 2).sum()


@pytest.mark.parametrize("dims,R", [((12, 9, 10), 4), ((7, 5, 6, 4), 3), ((40, 30, 50), 16)])
def test_forward_and_fp64_backward_match_oracle(env, orc, dims, R):
    torch, ag, h = env
    X, A = _problem(torch, dims, R, 1, np.float64)
    Xd = torch.from_numpy(X).cuda()
    Ad = [torch.from_numpy(a).cuda().requires_grad_() for a in A]
    loss = ag.cp_loss(Xd, Ad, prec="fp64", handle=h)
    r = orc.residual(X, A)
    ref = r * r * float((X.astype(np.float64) ** 2).sum())
    assert abs(loss.item() - ref) <= 1e-12 * ref
    loss.backward()
    G, M = _oracle_grad(orc, X, A)
    scale = sum(np.linalg.norm(m) for m in M)
    for a, g in zip(Ad, G):
        assert np.linalg.norm(a.grad.cpu().numpy() - 2.0 * g) <= 1e-12 * 2.0 * scale


def test_backward_bf16x3_bound(env, orc):
    torch, ag, h = env
    dims, R = (64, 48, 80), 8
    X, A = _problem(torch, dims, R, 2, np.float32)
    Xd = torch.from_numpy(X).cuda()
    Ad = [torch.from_numpy(a).cuda().requires_grad_() for a in A]
    ag.cp_loss(Xd, Ad, prec="bf16x3", handle=h).backward()
    G, M = _oracle_grad(orc, X, A)
    for a, g, m in zip(Ad, G, M):
        # error relative to ||M^(n)|| (the gradient is a difference of O(||M||) terms)
        assert np.linalg.norm(a.grad.cpu().numpy() - 2.0 * g) <= 2e-5 * 2.0 * np.linalg.norm(m)


def test_finite_differences(env):
    torch, ag, h = env
    dims, R = (6, 5, 7), 3
    X, A = _problem(torch, dims, R, 3, np.float64)
    Xd = torch.from_numpy(X).cuda()
    Ad = [torch.from_numpy(a).cuda().requires_grad_() for a in A]
    ag.cp_loss(Xd, Ad, prec="fp64", handle=h).backward()
    rng = np.random.default_rng(4)
    eps = 1e-5
    for _ in range(3):
        D = [rng.standard_normal(a.shape) for a in A]
        plus = ag.cp_loss(Xd, [torch.from_numpy(a + eps * d).cuda() for a, d in zip(A, D)], prec="fp64", handle=h)
        minus = ag.cp_loss(Xd, [torch.from_numpy(a - eps * d).cuda() for a, d in zip(A, D)], prec="fp64", handle=h)
        fd = (plus.item() - minus.item()) / (2 * eps)
        an = sum(float((a.grad.cpu().numpy() * d).sum()) for a, d in zip(Ad, D))
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(an))


def test_gradcheck(env):
    torch, ag, h = env
    X, A = _problem(torch, (4, 3, 5), 2, 5, np.float64)
    Xd = torch.from_numpy(X).cuda()
    Ad = tuple(torch.from_numpy(a).cuda().requires_grad_() for a in A)
    # the FP64 MTTKRP accumulates rows with atomics: a repeated backward may differ in the last bits
    assert torch.autograd.gradcheck(lambda *f: ag.cp_loss(Xd, list(f), prec="fp64", handle=h), Ad, eps=1e-6,
                                    atol=1e-6, rtol=1e-6, nondet_tol=1e-10)


def test_matches_einsum_autograd(env):
    torch, ag, h = env
    X, A = _problem(torch, (20, 24, 18), 5, 6, np.float32)
    Xd = torch.from_numpy(X).cuda()
    A1 = [torch.from_numpy(a).cuda().requires_grad_() for a in A]
    A2 = [torch.from_numpy(a).cuda().requires_grad_() for a in A]
    l1 = ag.cp_loss(Xd, A1, prec="fp64", handle=h)
    l2 = _einsum_loss(torch, Xd, A2)
    l1.backward()
    l2.backward()
    assert abs(l1.item() - l2.item()) <= 1e-10 * l2.item()
    for a, b in zip(A1, A2):
        assert torch.allclose(a.grad, b.grad, rtol=1e-9, atol=1e-9 * b.grad.abs().max().item())


def test_argument_checks(env):
    torch, ag, h = env
    X = torch.zeros(3, 4, 5, device="cuda")
    with pytest.raises(ValueError):
        ag.cp_loss(X, [torch.zeros(3, 2, device="cuda", dtype=torch.float32)] * 3, handle=h)
    with pytest.raises(ValueError):
        ag.cp_loss(X.cpu(), [torch.zeros(3, 2, dtype=torch.float64)] * 3, handle=h)


@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
def test_loss256_full_size(env, orc, prec):
    """The loss workload at its stated size: 256^3 FP32 tensor from rank-32
    N(0,1) factors, gradients at the (non-optimal) seeded start.  The forward
    against the oracle's residual (1e-12); the backward against the oracle's
    FP64 dimension-tree gradient 2 (A Gamma - M) (1e-12 of ||M^(n)|| in FP64,
    2e-5 with the bf16x3 MTTKRP) and against central differences of the FP64
    loss along random directions (relative 1e-6: at h = 1e-4 the truncation h^2 |f'''| / 6 is about
    2e-8 relative (1.5e-6 measured at h = 1e-3) and the cancellation 1e-16 |f| / h about 1e-10)."""
    torch, ag, h = env
    from paper_1910_12331_gb300 import datagen

    p = datagen.workload("loss256", seed=0)
    X, A = p["X"], p["init"]
    Xd = torch.from_numpy(X).cuda()
    Ad = [torch.from_numpy(a.copy()).cuda().requires_grad_() for a in A]
    loss = ag.cp_loss(Xd, Ad, prec=prec, handle=h)
    X64 = X.astype(np.float64)
    r = orc.residual(X64, A)
    ref = r * r * float(np.sum(X64 * X64))
    assert abs(loss.item() - ref) <= 1e-12 * ref
    loss.backward()
    M = orc.mttkrp(X64, A, "dt")
    G, _ = orc.gradient(A, orc.gamma(orc.gram(A)), M)
    tol = 1e-12 if prec == "fp64" else 2e-5
    for a, g, m in zip(Ad, G, M):
        assert np.linalg.norm(a.grad.cpu().numpy() - 2.0 * g) <= tol * 2.0 * np.linalg.norm(m)
    if prec == "fp64":
        rng = np.random.default_rng(9)
        eps = 1e-4
        for _ in range(2):
            D = [rng.standard_normal(a.shape) for a in A]
            fp = orc.residual(X64, [a + eps * d for a, d in zip(A, D)]) ** 2 * float(np.sum(X64 * X64))
            fm = orc.residual(X64, [a - eps * d for a, d in zip(A, D)]) ** 2 * float(np.sum(X64 * X64))
            fd = (fp - fm) / (2 * eps)
            an = sum(float((a.grad.cpu().numpy() * d).sum()) for a, d in zip(Ad, D))
            assert abs(fd - an) <= 1e-6 * abs(an), (fd, an)
