"""Tucker compression ahead of CP (Section 1; the complexity comparison of
Section 3.5 assumes it): cp_hosvd against the oracle's truncated HoSVD, and
cp_tucker_expand.

The bases are unique up to a rotation within each subspace, so the test
compares the projectors U_n U_n^T and the reconstruction X^ = G x_1 U_1 ...
x_N U_N (both unique), plus the invariants: orthonormal columns and ||G||_F.
Tolerance: the GPU's orthogonal iteration stops at a subspace residual of
1e-12 ||S_n V||, so with the eigen-gaps of these tensors (the noise is 1e-3 of
the signal or less) the projectors agree to about 1e-12 / gap; 1e-9 is
written below."""
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


def _expand(core, U):
    Xh = core
    for n, u in enumerate(U):
        Xh = np.moveaxis(np.tensordot(u, Xh, axes=(1, n)), 0, n)
    return Xh


@pytest.mark.parametrize("dims,ranks,noise,xdt", [((37, 45, 29), (5, 7, 4), 1e-3, np.float32),
                                                  ((70, 33, 41), (9, 3, 12), 1e-4, np.float64),
                                                  ((12, 9, 14, 10), (3, 4, 2, 5), 1e-3, np.float32),
                                                  ((65, 40), (6, 6), 0.0, np.float64),
                                                  ((20, 30, 25), (20, 1, 25), 1e-3, np.float64)])
def test_hosvd_matches_oracle(env, orc, dims, ranks, noise, xdt):
    """Several 32-row Gram tiles and a ragged last tile (70, 65), orders 2-4,
    FP32 and FP64 X, a rank-1 mode and full-rank modes (r_n = s_n)."""
    torch, api, h = env
    from paper_1910_12331_gb300 import datagen

    X, _ = datagen.tucker_tensor(dims, ranks, noise=noise, seed=3, dtype=xdt)
    U, core, iters = api.cp_hosvd(h, torch.from_numpy(X).cuda(), ranks)
    Ug = [u.cpu().numpy() for u in U]
    Gg = core.cpu().numpy()
    Uo, Go, _ = orc.hosvd(X, ranks)
    for n, (u, uo) in enumerate(zip(Ug, Uo)):
        assert np.abs(u.T @ u - np.eye(ranks[n])).max() <= 1e-13, n
        assert np.abs(u @ u.T - uo @ uo.T).max() <= 1e-9, (n, iters)
    Xh, Xho = _expand(Gg, Ug), _expand(Go, Uo)
    assert np.abs(Xh - Xho).max() <= 1e-9 * np.abs(Xho).max()
    assert abs(np.linalg.norm(Gg) - np.linalg.norm(Go)) <= 1e-12 * np.linalg.norm(Go)
    print(dims, ranks, "iterations", iters)


def test_hosvd_exact_multilinear_rank_reproduces_x(env):
    """Without noise the truncated HoSVD reproduces X (to FP64 rounding), and
    each U_n spans the generating Q_n."""
    torch, api, h = env
    from paper_1910_12331_gb300 import datagen

    X, Q = datagen.tucker_tensor((50, 38, 44), (6, 5, 7), seed=4)
    U, core, _ = api.cp_hosvd(h, torch.from_numpy(X).cuda(), (6, 5, 7))
    Ug = [u.cpu().numpy() for u in U]
    assert np.abs(_expand(core.cpu().numpy(), Ug) - X).max() <= 1e-12 * np.abs(X).max()
    for u, q in zip(Ug, Q):
        assert np.abs(u @ u.T - q @ q.T).max() <= 1e-11


def test_hosvd_core_cp_and_expansion(env, orc):
    """CP of the core by cp_gn_solve, expanded by cp_tucker_expand: A_n = U_n B_n
    (against numpy's product), and the squared error of [[A]] splits into the
    compression error plus the core's CP error (orthogonal projection)."""
    torch, api, h = env
    from paper_1910_12331_gb300 import datagen

    p = datagen.make_problem((60, 50, 70), 6, noise=1e-3, dtype=np.float64, seed=5)
    X = torch.from_numpy(p["X"]).cuda()
    U, core, _ = api.cp_hosvd(h, X, (6, 6, 6))
    # start: the generating factors' coordinates in the bases, perturbed
    rng = np.random.default_rng(6)
    B0 = [u.cpu().numpy().T @ a for u, a in zip(U, p["truth"])]
    B = [torch.from_numpy(b + 1e-2 * np.abs(b).max() * rng.standard_normal(b.shape)).cuda() for b in B0]
    hi, lo = orc.default_lambda([b.cpu().numpy() for b in B])
    params = api.gn_params(hi, lo, hi, eps_cg=1e-3, cg_max_iter=100, prec="fp64")
    api.cp_gn_solve(h, core, B, params, api.solve_opts(max_iters=60))
    A = api.cp_tucker_expand(h, U, B)
    for a, u, b in zip(A, U, B):
        ref = u.cpu().numpy() @ b.cpu().numpy()
        assert np.abs(a.cpu().numpy() - ref).max() <= 1e-14 * np.abs(ref).max() * 6
    e_full, x2 = api.cp_residual_sums(h, X, A)
    e_core, g2 = api.cp_residual_sums(h, core, B)
    e_comp = x2 - g2
    assert abs(e_full - (e_comp + e_core)) <= 1e-9 * x2
    assert np.sqrt(e_full / x2) <= 2e-3  # the 1e-3 noise, recovered through the compressed problem


@pytest.mark.parametrize("which", ["truth", "none"])
def test_hosvd_full_size_collinear400(env, which):
    """The 400^3 R = 50 collinear workload compressed to 50^3 (its multilinear
    rank, plus the 1e-6 noise): orthonormal bases, ||X - X^||^2 = ||X||^2 -
    ||G||^2 at the noise level, and the generating factors inside the spans."""
    torch, api, h = env
    from paper_1910_12331_gb300 import datagen

    p = datagen.workload("collinear400", seed=0)
    X = torch.from_numpy(p["X"]).cuda()
    U, core, iters = api.cp_hosvd(h, X, (50, 50, 50))
    x2 = float(torch.sum(X.double() ** 2))
    g2 = float(torch.sum(core ** 2))
    rel = np.sqrt(max(x2 - g2, 0.0) / x2)
    print("collinear400 compression error", rel, "iterations", iters)
    assert rel <= 3e-6  # noise 1e-6 plus the FP32 storage of X
    for u, a in zip(U, p["truth"]):
        uu = u.cpu().numpy()
        assert np.abs(uu.T @ uu - np.eye(50)).max() <= 1e-12
        resid = a - uu @ (uu.T @ a)
        assert np.linalg.norm(resid) <= 1e-5 * np.linalg.norm(a)
    del X, core, U
    torch.cuda.empty_cache()


def test_hosvd_argument_checks(env):
    torch, api, h = env
    X = torch.zeros((6, 5, 4), dtype=torch.float64, device="cuda")
    for ranks in [(7, 2, 2), (0, 2, 2)]:  # rank above the side, rank 0
        with pytest.raises(api.CPError) as e:
            api.cp_hosvd(h, X, ranks)
        assert e.value.status == api.CP_ERR_ARG
    with pytest.raises(api.CPError) as e:
        api.cp_hosvd(h, X, (2, 2, 2))  # X = 0: no r-dimensional dominant subspace
    assert e.value.status == api.CP_ERR_NOT_SPD
    # the handle stays usable
    Y = torch.from_numpy(np.random.default_rng(7).standard_normal((6, 5, 4))).cuda()
    U, core, _ = api.cp_hosvd(h, Y, (2, 2, 2))
    assert torch.isfinite(core).all()
