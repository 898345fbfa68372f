"""The residual tensor E = X - [[A]] itself, element by element, against the
oracle's FP64 E (cp_residual_tensor: the reconstruction the residual-form
gradient uses, written out in FP64).

Bounds, per element (i, m, k) with m the index of the middle modes:
- tensor cores (R <= 64): 2^-38.5 R sigma tau, sigma and tau the powers of two
  at or above max_r |a^(1)_ir w_m[r]| and max_r |a^(N)_kr| (the error-free
  slice products: five bf16 pieces per operand, the pairs of levels 2..6,
  levels 2-4 accumulated exactly), doubled here because the kernel takes
  sigma from FP32 row maxima, plus 2^-50 |x| for the final FP64 subtraction;
- CUDA cores (R > 64): 2^-44 R B with B = sum_r max_i |a^(1)_ir| max_m |w_m[r]|
  max_k |a^(N)_kr| (at least the bound B of every tile): the leading products
  are summed against an offset sigma <= 9 B, so each part a fused
  multiply-add drops is below 2^-24 sigma and is recovered exactly into an FP32
  low accumulator of at most R such parts, whose own rounding is then below
  2^-24 R 2^-24 sigma <= 2^-44 R B.  (Measured: 2^-35 of max |[[A]]| at
  R = 80 with Gaussian factors.)"""
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


def _pow2_ceil(v):
    """Smallest power of two >= v (elementwise, v > 0)."""
    m, e = np.frexp(v)
    return np.where(m == 0.5, np.ldexp(1.0, e - 1), np.ldexp(1.0, e))


def _uv(A):
    """u = rows (i, m) of A^(1) * w_m (s1*mid x R) and v = A^(N)."""
    R = A[0].shape[1]
    W = np.ones((1, R))
    for a in A[1:-1]:
        W = (W[:, None, :] * a[None, :, :]).reshape(-1, R)
    U = (A[0][:, None, :] * W[None, :, :]).reshape(-1, R)
    return U, A[-1]


def _tc_bound(X, A):
    U, V = _uv(A)
    R = A[0].shape[1]
    sig = _pow2_ceil(np.maximum(np.abs(U).max(axis=1), 2.0 ** -100))
    tau = np.where(np.abs(V).max(axis=1) > 0, _pow2_ceil(np.maximum(np.abs(V).max(axis=1), 1e-300)), 1.0)
    Xm = np.asarray(X, dtype=np.float64).reshape(U.shape[0], V.shape[0])
    return 2.0 * 2.0 ** -38.5 * R * sig[:, None] * tau[None, :] + 2.0 ** -50 * np.abs(Xm)


def _check_tc(api, h, torch, orc, X, A):
    Xd = torch.from_numpy(X).cuda()
    Ad = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in A]
    E, sq_err, sq_x = api.cp_residual_tensor(h, Xd, Ad)
    Eg = E.cpu().numpy()
    Eo = orc.residual_tensor(X, A)
    bound = _tc_bound(X, A)
    diff = np.abs(Eg - Eo).reshape(bound.shape)
    worst = float((diff / bound).max())
    assert worst <= 1.0, worst
    # the squared sums (E rounded to FP32 in the kernel's sum)
    assert abs(sq_err - np.sum(Eo * Eo)) <= 1e-6 * np.sum(Eo * Eo) + 1e-300
    assert abs(sq_x - np.sum(np.asarray(X, np.float64) ** 2)) <= 1e-6 * np.sum(np.asarray(X, np.float64) ** 2)
    return Eg, worst


@pytest.mark.parametrize("dims,R,xdt", [((130, 9, 140), 50, np.float32), ((37, 70, 45), 13, np.float32),
                                        ((20, 7, 5, 33), 64, np.float32), ((50, 70), 9, np.float32),
                                        ((64, 33, 8), 1, np.float32), ((130, 9, 140), 20, np.float64),
                                        ((3, 4, 2, 3, 2), 16, np.float32), ((257, 3, 385), 33, np.float32)])
def test_residual_tensor_tensor_cores(env, orc, dims, R, xdt):
    """Random factors and tensor: every column chunk (ragged last chunk, s_N not
    a multiple of 4 so X read without tensor copies, FP64 X), orders 2-5."""
    torch, api, h = env
    rng = np.random.default_rng(71)
    A = [rng.standard_normal((s, R)) for s in dims]
    X = rng.standard_normal(dims).astype(xdt)
    _check_tc(api, h, torch, orc, X, A)


@pytest.mark.parametrize("R", [50, 64, 7])
def test_residual_tensor_near_optimum(env, orc, R):
    """X = [[T]] + 1e-6 noise and A = T + 1e-7 perturbation: |E| ~ 1e-6 |X|,
    where the cancellation is, and E still within the absolute bound."""
    torch, api, h = env
    from tests import cpref

    dims = (130, 9, 140)
    rng = np.random.default_rng(72)
    T = [rng.standard_normal((s, R)) for s in dims]
    X0 = cpref.reconstruct(T)
    X = (X0 + 1e-6 * np.linalg.norm(X0) / np.sqrt(X0.size) * rng.standard_normal(dims)).astype(np.float32)
    A = [t + 1e-7 * rng.standard_normal(t.shape) for t in T]
    Eg, worst = _check_tc(api, h, torch, orc, X, A)
    print("near optimum, R", R, "worst / bound", worst, "|E| max", np.abs(Eg).max())


def test_residual_tensor_call_to_call_identical(env):
    torch, api, h = env
    rng = np.random.default_rng(73)
    dims, R = (384, 96, 320), 50
    A = [torch.from_numpy(rng.standard_normal((s, R))).cuda() for s in dims]
    X = torch.from_numpy(rng.standard_normal(dims).astype(np.float32)).cuda()
    E1, s1, _ = api.cp_residual_tensor(h, X, A)
    E1 = E1.clone()
    for _ in range(3):
        E2, s2, _ = api.cp_residual_tensor(h, X, A)
        assert torch.equal(E1, E2) and s1 == s2


@pytest.mark.parametrize("dims,R", [((130, 9, 140), 80), ((70, 6, 90), 100)])
def test_residual_tensor_cuda_cores(env, orc, dims, R):
    torch, api, h = env
    rng = np.random.default_rng(74)
    A = [rng.standard_normal((s, R)) for s in dims]
    X = rng.standard_normal(dims).astype(np.float32)
    E, _, _ = api.cp_residual_tensor(h, torch.from_numpy(X).cuda(), [torch.from_numpy(a).cuda() for a in A])
    Eo = orc.residual_tensor(X, A)
    W = np.ones((1, R))
    for a in A[1:-1]:
        W = (W[:, None, :] * a[None, :, :]).reshape(-1, R)
    B = float(np.sum(np.abs(A[0]).max(axis=0) * np.abs(W).max(axis=0) * np.abs(A[-1]).max(axis=0)))
    err = np.abs(E.cpu().numpy() - Eo).max()
    print("CUDA-core reconstruction, R", R, "error / bound", err / (2.0 ** -44 * R * B))
    assert err <= 2.0 ** -44 * R * B


@pytest.mark.parametrize("which", ["init", "truth"])
def test_residual_tensor_full_size_collinear400(env, orc, which):
    """The 400^3 R = 50 collinear workload the benchmark solves: E at the
    starting point (|E| ~ |X|) and at the generating factors (E = the 1e-6
    noise plus the FP32 rounding of X), element by element."""
    torch, api, h = env
    from paper_1910_12331_gb300 import datagen

    p = datagen.workload("collinear400", seed=0)
    Eg, worst = _check_tc(api, h, torch, orc, p["X"], p[which])
    print("collinear400", which, "worst / bound", worst)
    del Eg
    torch.cuda.empty_cache()
