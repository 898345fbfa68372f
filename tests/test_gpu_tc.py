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
