"""The seeded input generator does what its recipe says: the synthetic tensors
of Section 5 (Gaussian or uniform factors, exact rank plus relative noise),
column collinearity, the batched problem mix, and reproducible bytes."""
import numpy as np
import pytest

from paper_1910_12331_gb300 import datagen


@pytest.mark.parametrize("s,R,c", [(40, 7, 0.9), (25, 25, 0.5), (400, 50, 0.9), (10, 3, 0.0)])
def test_collinear_factor_cosines_and_norms(s, R, c):
    A = datagen.draw_factor(datagen._rng(3, 1), s, R, "normal", c if c > 0 else None)
    if c > 0:
        norms = np.linalg.norm(A, axis=0)
        np.testing.assert_allclose(norms, np.sqrt(s), rtol=1e-12)
        cos = (A.T @ A) / np.outer(norms, norms)
        off = cos[~np.eye(R, dtype=bool)]
        np.testing.assert_allclose(off, c, atol=1e-12)


def test_collinear_needs_rank_at_most_side():
    with pytest.raises(ValueError):
        datagen.draw_factor(datagen._rng(0, 1), 5, 6, "normal", 0.9)


def test_distributions():
    rng = datagen._rng(1, 1)
    u = datagen.draw_factor(rng, 2000, 4, "uniform01")
    assert u.min() >= 0.0 and u.max() < 1.0 and abs(u.mean() - 0.5) < 0.02
    v = datagen.draw_factor(rng, 2000, 4, "uniform11")
    assert v.min() >= -1.0 and v.max() < 1.0 and abs(v.mean()) < 0.03
    g = datagen.draw_factor(rng, 20000, 2, "normal")
    assert abs(g.mean()) < 0.03 and abs(g.std() - 1.0) < 0.03
    with pytest.raises(ValueError):
        datagen.draw_factor(rng, 3, 2, "cauchy")


def test_full_tensor_is_sum_of_outer_products():
    rng = np.random.default_rng(0)
    A = [rng.standard_normal((s, 3)) for s in (4, 5, 2, 3)]
    X = datagen.full_tensor(A)
    ref = np.zeros((4, 5, 2, 3))
    for r in range(3):
        ref += np.multiply.outer(np.multiply.outer(np.multiply.outer(A[0][:, r], A[1][:, r]), A[2][:, r]), A[3][:, r])
    np.testing.assert_allclose(X, ref, rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("eta", [0.0, 1e-8, 1e-4, 0.3])
def test_noise_level_exact(eta):
    p = datagen.make_problem((9, 8, 7), 3, "normal", None, eta, np.float64, seed=5)
    X0 = datagen.full_tensor(p["truth"])
    rel = np.linalg.norm(p["X"] - X0) / np.linalg.norm(X0)
    assert abs(rel - eta) <= 1e-9 * max(eta, 1e-300) + (0.0 if eta else 1e-16)


def test_seeds_streams_and_storage():
    a = datagen.make_problem((6, 5, 4), 2, "normal", None, 1e-6, np.float32, seed=11)
    b = datagen.make_problem((6, 5, 4), 2, "normal", None, 1e-6, np.float32, seed=11)
    c = datagen.make_problem((6, 5, 4), 2, "normal", None, 1e-6, np.float32, seed=12)
    assert a["X"].dtype == np.float32 and a["X"].flags["C_CONTIGUOUS"]
    assert a["X"].tobytes() == b["X"].tobytes()
    assert a["X"].tobytes() != c["X"].tobytes()
    for t, i in zip(a["truth"], a["init"]):
        assert t.dtype == np.float64 and i.dtype == np.float64
        assert not np.array_equal(t, i)  # the start comes from its own stream
    # the FP32 tensor is the rounding of the FP64 one
    p64 = datagen.make_problem((6, 5, 4), 2, "normal", None, 1e-6, np.float64, seed=11)
    np.testing.assert_array_equal(a["X"], p64["X"].astype(np.float32))


def test_workload_table():
    expect = {"exact20": ((20, 20, 20), 5, np.float64), "collinear400": ((400, 400, 400), 50, np.float32),
              "uniform120x4": ((120, 120, 120, 120), 40, np.float32), "loss256": ((256, 256, 256), 32, np.float32)}
    for name, (dims, R, dt) in expect.items():
        cfg = datagen.WORKLOADS[name]
        assert tuple(cfg["dims"]) == dims and cfg["R"] == R and cfg["dtype"] == dt, name
    assert datagen.WORKLOADS["collinear400"]["collinearity"] == 0.9
    assert datagen.WORKLOADS["collinear400"]["noise"] == 1e-6
    assert datagen.WORKLOADS["uniform120x4"]["dist"] == "uniform01"
    assert datagen.WORKLOADS["uniform120x4"]["noise"] == 1e-4
    p = datagen.workload("exact20", seed=0)
    assert p["X"].shape == (20, 20, 20) and p["X"].dtype == np.float64
    np.testing.assert_array_equal(p["X"], datagen.full_tensor(p["truth"]))  # no noise


def test_batched_problem_mix():
    probs = datagen.batched_problems(count=64, seed=3)
    assert len(probs) == 64
    sides = np.array([p["X"].shape for p in probs])
    ranks = np.array([p["truth"][0].shape[1] for p in probs])
    assert sides.min() >= 16 and sides.max() <= 96 and ranks.min() >= 4 and ranks.max() <= 24
    assert len(set(map(tuple, sides))) > 32  # uneven sizes
    for p in probs[:4]:
        assert p["X"].dtype == np.float32 and p["X"].ndim == 3
        X0 = datagen.full_tensor(p["truth"])
        rel = np.linalg.norm(p["X"].astype(np.float64) - X0) / np.linalg.norm(X0)
        assert rel < 1e-6  # 1e-8 noise plus the FP32 rounding of X
    again = datagen.batched_problems(count=4, seed=3)
    for p, q in zip(probs[:4], again):
        assert p["X"].tobytes() == q["X"].tobytes()


def test_tucker_tensor_recipe():
    """Exact multilinear rank: every unfolding has rank r_n, its column space is
    spanned by the orthonormal Q_n; the noise is the stated relative level;
    seeds reproduce the bytes."""
    X, Q = datagen.tucker_tensor((9, 8, 7), (3, 4, 2), seed=5)
    for n, (q, r) in enumerate(zip(Q, (3, 4, 2))):
        np.testing.assert_allclose(q.T @ q, np.eye(r), atol=1e-14)
        Xn = np.moveaxis(X, n, 0).reshape(X.shape[n], -1)
        sv = np.linalg.svd(Xn, compute_uv=False)
        assert sv[r - 1] > 1e-3 * sv[0] and (len(sv) == r or sv[r] < 1e-12 * sv[0])
        np.testing.assert_allclose(q @ (q.T @ Xn), Xn, atol=1e-12 * np.abs(Xn).max())
    Xe, _ = datagen.tucker_tensor((9, 8, 7), (3, 4, 2), noise=1e-3, seed=5)
    assert abs(np.linalg.norm(Xe - X) / np.linalg.norm(X) - 1e-3) < 1e-12
    X2, _ = datagen.tucker_tensor((9, 8, 7), (3, 4, 2), seed=5)
    assert X.tobytes() == X2.tobytes()
