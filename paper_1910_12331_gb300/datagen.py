"""Seeded synthetic inputs for CP decomposition (Section 5, "tensors made by
random matrices" / "by Gaussian matrices", and the matrix multiplication tensor).

This module holds no step of the method: it draws factor matrices, builds the
exact-rank tensor X = [[A^(1), ..., A^(N)]] with numpy's ``einsum``, adds
noise, and returns plain numpy arrays.  Both the CUDA library's tests and the
CPU oracle read the very same bytes it returns.

Recipe (the parts the paper does not fix are conventions of this project):
  * factors: N(0,1), uniform(0,1) or uniform(-1,1) entries (Section 5);
  * column collinearity c: A = sqrt(s) Q L^T with Q an orthonormal basis of an
    s x R Gaussian draw and L L^T = (1-c) I + c 1 1^T, so that every pair of
    columns has cosine exactly c and every column has norm sqrt(s);
  * noise eta: X = X0 + eta ||X0||_F E / ||E||_F with E i.i.d. N(0,1);
  * the starting point is drawn from the factor distribution (without
    collinearity) with an independent stream of the same seed;
  * tensors are generated in float64 and cast to the storage dtype.
"""
from __future__ import annotations

import string

import numpy as np

DISTS = ("normal", "uniform01", "uniform11")


def _rng(seed: int, stream: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence([int(seed), int(stream)])))


def draw_factor(rng: np.random.Generator, s: int, R: int, dist: str = "normal",
                collinearity: float | None = None) -> np.ndarray:
    if collinearity is not None and collinearity > 0.0:
        if R > s:
            raise ValueError("collinear factors need R <= s")
        Q, _ = np.linalg.qr(rng.standard_normal((s, R)))
        C = (1.0 - collinearity) * np.eye(R) + collinearity * np.ones((R, R))
        L = np.linalg.cholesky(C)
        return np.sqrt(s) * Q @ L.T
    if dist == "normal":
        return rng.standard_normal((s, R))
    if dist == "uniform01":
        return rng.uniform(0.0, 1.0, (s, R))
    if dist == "uniform11":
        return rng.uniform(-1.0, 1.0, (s, R))
    raise ValueError(f"unknown distribution {dist!r}")


def full_tensor(factors) -> np.ndarray:
    """Dense [[A^(1), ..., A^(N)]] via numpy.einsum (float64)."""
    N = len(factors)
    letters = string.ascii_lowercase[:N]
    spec = ",".join(f"{c}z" for c in letters) + "->" + letters
    return np.einsum(spec, *factors, optimize=True)


def add_noise(rng: np.random.Generator, X: np.ndarray, eta: float) -> np.ndarray:
    if eta <= 0.0:
        return X
    E = rng.standard_normal(X.shape)
    return X + eta * np.linalg.norm(X) * E / np.linalg.norm(E)


def make_problem(dims, R, dist="normal", collinearity=None, noise=0.0, dtype=np.float32, seed=0,
                 init_dist=None):
    """Returns dict(X, truth, init): X stored in ``dtype``; truth and init are
    lists of float64 (s_n, R) arrays."""
    rng_f = _rng(seed, 1)
    truth = [draw_factor(rng_f, int(s), int(R), dist, collinearity) for s in dims]
    X = full_tensor(truth)
    X = add_noise(_rng(seed, 2), X, noise)
    rng_i = _rng(seed, 3)
    init = [draw_factor(rng_i, int(s), int(R), init_dist or dist) for s in dims]
    return {"X": np.ascontiguousarray(X.astype(dtype)), "truth": truth, "init": init}


# Workloads (sizes and distributions of the paper's synthetic experiments and of
# the benchmark configurations of this project).
WORKLOADS = {
    # order-3 20^3 exact rank-5 Gaussian tensor, FP64, no noise
    "exact20": dict(dims=(20, 20, 20), R=5, dist="normal", noise=0.0, dtype=np.float64),
    # order-3 400^3 FP32, rank-50 Gaussian factors with collinearity 0.9, 1e-6 noise
    "collinear400": dict(dims=(400, 400, 400), R=50, dist="normal", collinearity=0.9, noise=1e-6,
                         dtype=np.float32),
    # order-4 120^4 FP32, rank-40 uniform(0,1) factors, 1e-4 noise
    "uniform120x4": dict(dims=(120, 120, 120, 120), R=40, dist="uniform01", noise=1e-4, dtype=np.float32),
    # order-3 256^3 FP32, rank-32 Gaussian factors (loss/gradient workload)
    "loss256": dict(dims=(256, 256, 256), R=32, dist="normal", noise=0.0, dtype=np.float32),
}


def workload(name: str, seed: int = 0, **overrides):
    cfg = dict(WORKLOADS[name])
    cfg.update(overrides)
    return make_problem(seed=seed, **cfg)


def batched_problems(count=512, side_range=(16, 96), rank_range=(4, 24), noise=1e-8, seed=0,
                     dtype=np.float32):
    """Many independent order-3 problems with sides and ranks drawn uniformly
    (inclusive ranges), Gaussian factors plus relative noise."""
    rng = _rng(seed, 7)
    probs = []
    for k in range(count):
        dims = tuple(int(v) for v in rng.integers(side_range[0], side_range[1] + 1, size=3))
        R = int(rng.integers(rank_range[0], rank_range[1] + 1))
        probs.append(make_problem(dims, R, "normal", None, noise, dtype, seed=seed * 100003 + k))
    return probs


def tucker_tensor(dims, ranks, noise=0.0, seed=0, dtype=np.float64):
    """X = G x_1 Q_1 ... x_N Q_N with Q_n an orthonormal basis of an s_n x r_n
    Gaussian draw and G an N(0,1) core: a tensor of exact multilinear rank
    `ranks`, plus relative noise eta as in `add_noise`.  Returns (X, Q list)."""
    rng = _rng(seed, 21)
    Q = [np.linalg.qr(rng.standard_normal((int(s), int(r))))[0] for s, r in zip(dims, ranks)]
    X = rng.standard_normal(tuple(int(r) for r in ranks))
    for n, q in enumerate(Q):
        X = np.moveaxis(np.tensordot(q, X, axes=(1, n)), 0, n)
    if noise:
        X = add_noise(rng, X, noise)
    return np.ascontiguousarray(X.astype(dtype)), Q


def matmul_tensor(n: int) -> np.ndarray:
    """Order-3 unfolding of t_{ijklmn} = delta_lm delta_ik delta_nj (Section 5):
    T[(i,j), (k,l), (m,n)] with pair index a*n + b; c_ij = sum T a_kl b_mn."""
    T = np.zeros((n * n, n * n, n * n))
    for i in range(n):
        for j in range(n):
            for l in range(n):
                T[i * n + j, i * n + l, l * n + j] = 1.0
    return T


def likelihood_problems(n_problems=100, ranks=range(3, 10), starts=5, side=4, dist="uniform11", seed=0,
                        dtype=np.float32):
    """The convergence-likelihood study of Section 5: for every rank R, n_problems
    exact rank-R order-3 tensors of side `side` from factors of `dist`, each with
    `starts` starting points drawn from the same distribution.  Returns a list of
    dicts (X, truth, init, rank, problem, start) in the order rank, problem, start."""
    out = []
    for R in ranks:
        for q in range(n_problems):
            rng_f = _rng(seed * 1000003 + R * 1009 + q, 11)
            truth = [draw_factor(rng_f, side, int(R), dist) for _ in range(3)]
            X = np.ascontiguousarray(full_tensor(truth).astype(dtype))
            for st in range(starts):
                rng_i = _rng(seed * 1000003 + R * 1009 + q, 100 + st)
                init = [draw_factor(rng_i, side, int(R), dist) for _ in range(3)]
                out.append({"X": X, "truth": truth, "init": init, "rank": int(R), "problem": q, "start": st})
    return out
