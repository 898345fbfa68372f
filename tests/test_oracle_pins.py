"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

None of these compares the oracle with itself: every expected value comes from
an independent construction (explicit Jacobian of Eq. (3.1), numpy einsum of a
definition, closed forms, exact decompositions, finite differences, dense
solves).  Sizes keep the whole file to seconds.
"""
import os

import numpy as np
import pytest

from tests import cpref
from paper_1910_12331_gb300 import datagen

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

SHAPES = [((5, 7, 9), 3), ((6, 5, 4, 7), 4), ((8, 6), 3), ((3, 4, 2, 3, 2), 2),
          ((2, 3, 2, 2, 3, 2, 2, 2), 2)]  # the largest order, 8


def _rand_factors(dims, R, seed):
    rng = np.random.default_rng(seed)
    return [rng.standard_normal((s, R)) for s in dims]


def _rand_tensor(dims, seed):
    return np.random.default_rng(seed + 1000).standard_normal(dims)


# ----------------------------------------------------------------- Gram, Gamma

@pytest.mark.parametrize("dims,R", SHAPES)
def test_gram_gamma(orc, dims, R):
    A = _rand_factors(dims, R, 1)
    S = orc.gram(A)
    for n, a in enumerate(A):
        np.testing.assert_allclose(S[n], a.T @ a, rtol=1e-13, atol=1e-13)
    G = orc.gamma(S)
    N = len(dims)
    for n in range(N):
        for p in range(N):
            ref = np.ones((R, R))
            for m in range(N):
                if m not in (n, p):
                    ref = ref * (A[m].T @ A[m])
            np.testing.assert_allclose(G[n, p], ref, rtol=1e-13)
            np.testing.assert_array_equal(G[n, p], G[p, n])      # symmetric in (n, p)
            np.testing.assert_allclose(G[n, p], G[n, p].T, rtol=1e-13)  # each block symmetric


def test_gamma_order2_all_ones(orc):
    A = _rand_factors((5, 6), 3, 2)
    G = orc.gamma(orc.gram(A))
    np.testing.assert_array_equal(G[0, 1], np.ones((3, 3)))
    np.testing.assert_allclose(G[0, 0], A[1].T @ A[1], rtol=1e-14)


# ---------------------------------------------------------------------- MTTKRP

def _einsum_mttkrp(X, A, n):
    """M^(n) = X_(n) P^(n) written as one einsum over the definition."""
    N = X.ndim
    letters = "abcdefgh"[:N]
    ins = [letters] + [f"{letters[m]}z" for m in range(N) if m != n]
    spec = ",".join(ins) + f"->{letters[n]}z"
    return np.einsum(spec, X, *[A[m] for m in range(N) if m != n], optimize=True)


@pytest.mark.parametrize("dims,R", SHAPES)
@pytest.mark.parametrize("method", ["def", "dt"])
def test_mttkrp_definition(orc, dims, R, method):
    A = _rand_factors(dims, R, 3)
    X = _rand_tensor(dims, 3)
    M = orc.mttkrp(X, A, method)
    for n in range(len(dims)):
        ref = _einsum_mttkrp(X, A, n)
        np.testing.assert_allclose(M[n], ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())


@pytest.mark.parametrize("dims,R", SHAPES[:2])
def test_mttkrp_row(orc, dims, R):
    A = _rand_factors(dims, R, 4)
    X = _rand_tensor(dims, 4)
    M = orc.mttkrp(X, A)
    for n in range(len(dims)):
        for i in (0, dims[n] - 1):
            np.testing.assert_allclose(orc.mttkrp_row(X, A, n, i), M[n][i], rtol=1e-13, atol=1e-13)


def test_mttkrp_rank1_closed_form(orc):
    """All-ones factors: M^(n)_{i r} = sum of the mode-n slice i of X."""
    dims = (4, 6, 5)
    X = _rand_tensor(dims, 5)
    A = [np.ones((s, 2)) for s in dims]
    M = orc.mttkrp(X, A, "dt")
    for n in range(3):
        axes = tuple(m for m in range(3) if m != n)
        sums = X.sum(axis=axes)
        np.testing.assert_allclose(M[n], np.stack([sums, sums], 1), rtol=1e-13)


@pytest.mark.parametrize("dims,R", [((7, 8, 9), 4), ((5, 4, 6, 3), 3)])
def test_mttkrp_exact_decomposition(orc, dims, R):
    """For X = [[A]] the normal equations hold exactly: M^(n) = A^(n) Gamma^(n),
    and <X, X> = <M^(n), A^(n)> for every mode n."""
    A = _rand_factors(dims, R, 6)
    X = cpref.reconstruct(A)
    M = orc.mttkrp(X, A, "dt")
    for n in range(len(dims)):
        Gam = np.ones((R, R))
        for m in range(len(dims)):
            if m != n:
                Gam *= A[m].T @ A[m]
        np.testing.assert_allclose(M[n], A[n] @ Gam, rtol=1e-12, atol=1e-12 * np.abs(M[n]).max())
        assert abs(np.sum(M[n] * A[n]) - np.sum(X * X)) <= 1e-12 * np.sum(X * X)


@pytest.mark.parametrize("perm", [(1, 0, 2, 3), (3, 2, 1, 0), (2, 0, 3, 1), (0, 3, 1, 2)])
def test_mttkrp_mode_permutation_equivariance(orc, perm):
    """M^(n) depends on which factor multiplies which mode, not on the order
    the modes are stored in: permuting X's modes and the factor list permutes
    the outputs.  The dimension tree treats the first, middle and last modes
    differently, so this exercises each of its index paths."""
    dims, R = (5, 4, 6, 3), 3
    A = _rand_factors(dims, R, 31)
    X = _rand_tensor(dims, 31)
    M = orc.mttkrp(X, A, "dt")
    Xp = np.ascontiguousarray(np.transpose(X, perm))
    Mp = orc.mttkrp(Xp, [A[q] for q in perm], "dt")
    for k, q in enumerate(perm):
        np.testing.assert_allclose(Mp[k], M[q], rtol=1e-12, atol=1e-12 * np.abs(M[q]).max())


# ---------------------------------------------------------------- matmul tensor

def test_strassen_golden(orc):
    C, Af, Bf = cpref.load_strassen(os.path.join(GOLDEN, "strassen_2x2.txt"))
    T = datagen.matmul_tensor(2)
    # the fixture itself: it is an exact rank-7 decomposition of the tensor
    np.testing.assert_array_equal(cpref.reconstruct([C, Af, Bf]), T)
    # the tensor multiplies matrices (c_ij = sum_l a_il b_lj)
    rng = np.random.default_rng(0)
    a, b = rng.standard_normal((2, 2)), rng.standard_normal((2, 2))
    c = np.einsum("xyz,y,z->x", T, a.reshape(-1), b.reshape(-1)).reshape(2, 2)
    np.testing.assert_allclose(c, a @ b, rtol=1e-14)
    A = [C, Af, Bf]
    assert orc.residual(T, A) == 0.0
    Gam = orc.gamma(orc.gram(A))
    M = orc.mttkrp(T, A, "dt")
    G, gn = orc.gradient(A, Gam, M)
    assert np.all(gn == 0.0)  # entries are small integers: exact arithmetic
    # classical algorithm, rank 8: product (i,l,j) -> c_ij += a_il b_lj
    Cc, Ac, Bc = np.zeros((4, 8)), np.zeros((4, 8)), np.zeros((4, 8))
    r = 0
    for i in range(2):
        for j in range(2):
            for l in range(2):
                Cc[2 * i + j, r] = Ac[2 * i + l, r] = Bc[2 * l + j, r] = 1.0
                r += 1
    assert orc.residual(T, [Cc, Ac, Bc]) == 0.0
    # a perturbed Strassen factor has a non-zero residual and gradient
    A2 = [C.copy(), Af.copy(), Bf.copy()]
    A2[1][0, 0] += 1.0
    assert orc.residual(T, A2) > 0.1


# -------------------------------------------------------------------- gradient

@pytest.mark.parametrize("dims,R", [((20, 20, 20), 5), ((4, 3, 5, 2), 3)])
def test_gradient_is_jacobian_transpose_residual(orc, dims, R):
    """G = J_r^T r (Section 3: gradient of phi) with J_r the explicit Jacobian of
    Eq. (3.1) and r = X - [[A]]; checked at a random (non-stationary) point."""
    A = _rand_factors(dims, R, 7)
    X = _rand_tensor(dims, 7)
    Gam = orc.gamma(orc.gram(A))
    M = orc.mttkrp(X, A, "dt")
    G, gn = orc.gradient(A, Gam, M)
    J = cpref.jacobian(A)
    r = (X - cpref.reconstruct(A)).reshape(-1)
    ref = J.T @ r
    got = cpref.pack(G)
    np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())
    np.testing.assert_allclose(gn, [np.linalg.norm(g) for g in cpref.unpack(ref, dims, R)], rtol=1e-12)


@pytest.mark.parametrize("dims,R", [((9, 7, 8), 4), ((5, 4, 6, 3), 3), ((10, 12), 5)])
def test_gradient_residual_form(orc, dims, R):
    """Eq. (2.3)'s gradient in residual form: A^(n) Gamma^(n,n) - M^(n) equals
    -MTTKRP(X - [[A]])^(n), because [[A]]_(n) P^(n) = A^(n) Gamma^(n,n)."""
    A = _rand_factors(dims, R, 17)
    X = _rand_tensor(dims, 17)
    G, _ = orc.gradient(A, orc.gamma(orc.gram(A)), orc.mttkrp(X, A))
    E = X - cpref.reconstruct(A)
    ME = orc.mttkrp(E, A)
    for g, me in zip(G, ME):
        np.testing.assert_allclose(g, -me, rtol=1e-11, atol=1e-11 * np.abs(me).max())


def test_gradient_finite_differences(orc):
    dims, R = (6, 5, 7), 3
    A = _rand_factors(dims, R, 8)
    X = _rand_tensor(dims, 8)
    Gam = orc.gamma(orc.gram(A))
    G, _ = orc.gradient(A, Gam, orc.mttkrp(X, A, "def"))
    rng = np.random.default_rng(9)
    h = 1e-5
    for _ in range(3):
        D = [rng.standard_normal(a.shape) for a in A]
        fp = cpref.objective(X, [a + h * d for a, d in zip(A, D)])
        fm = cpref.objective(X, [a - h * d for a, d in zip(A, D)])
        fd = (fp - fm) / (2 * h)
        an = sum(float(np.sum(g * d)) for g, d in zip(G, D))
        assert abs(fd - an) <= 1e-7 * max(1.0, abs(an))


# ------------------------------------------------------------ preconditioner

def test_precond_inverse(orc):
    A = _rand_factors((9, 8, 7), 5, 10)
    Gam = orc.gamma(orc.gram(A))
    for lam in (0.0, 1e-3, 10.0):
        P, st = orc.precond_inv(Gam[0, 0], lam)
        assert st == orc.OK
        np.testing.assert_allclose((Gam[0, 0] + lam * np.eye(5)) @ P, np.eye(5), atol=1e-12)
        np.testing.assert_allclose(P, P.T, rtol=1e-12, atol=1e-14)


def test_precond_not_spd(orc):
    G = np.ones((3, 3))  # rank one: singular
    _, st = orc.precond_inv(G, 0.0)
    assert st == orc.ERR_NOT_SPD
    _, st = orc.precond_inv(-np.eye(2), 0.5)
    assert st == orc.ERR_NOT_SPD


# ----------------------------------------------------------------------- matvec

@pytest.mark.parametrize("dims,R", [((20, 20, 20), 5), ((4, 3, 5, 2), 3), ((5, 6), 2), ((2, 2, 3, 2, 2, 2, 2, 2), 2)])
@pytest.mark.parametrize("lam", [0.0, 0.37])
def test_matvec_explicit_jacobian(orc, dims, R, lam):
    """Q = (J^T J + lam I) w with J formed explicitly (Eq. (3.1)); checks the
    Hessian blocks of Eq. (3.2) and the contractions of Eq. (3.4)."""
    A = _rand_factors(dims, R, 11)
    W = _rand_factors(dims, R, 12)
    Gam = orc.gamma(orc.gram(A))
    Q = orc.matvec(A, Gam, W, lam)
    J = cpref.jacobian(A)
    w = cpref.pack(W)
    ref = J.T @ (J @ w) + lam * w
    np.testing.assert_allclose(cpref.pack(Q), ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())


def test_matvec_listing_einsums(orc):
    """Listing 1's einsum strings evaluated by numpy on the same inputs."""
    dims, R = (6, 7, 5), 4
    A = _rand_factors(dims, R, 13)
    W = _rand_factors(dims, R, 14)
    Gam = orc.gamma(orc.gram(A))
    Q = orc.matvec(A, Gam, W, 0.0)
    for n in range(3):
        U = np.zeros((dims[n], R))
        for p in range(3):
            if n == p:
                U += np.einsum("rz,kz->kr", Gam[n, p], W[p])
            else:
                U += np.einsum("kz,lr,rz,lz->kr", A[n], A[p], Gam[n, p], W[p])
        np.testing.assert_allclose(Q[n], U, rtol=1e-12, atol=1e-12 * np.abs(U).max())


def test_matvec_symmetric_psd_nullspace(orc):
    dims, R = (7, 6, 5), 3
    A = _rand_factors(dims, R, 15)
    Gam = orc.gamma(orc.gram(A))
    U = _rand_factors(dims, R, 16)
    V = _rand_factors(dims, R, 17)
    HU = orc.matvec(A, Gam, U, 0.0)
    HV = orc.matvec(A, Gam, V, 0.0)
    uhv = sum(float(np.sum(u * h)) for u, h in zip(U, HV))
    vhu = sum(float(np.sum(v * h)) for v, h in zip(V, HU))
    assert abs(uhv - vhu) <= 1e-12 * abs(uhv)
    assert sum(float(np.sum(v * h)) for v, h in zip(V, HV)) > 0
    # scaling indeterminacy (Section 3.2): d/dt [[a1 (1+t), a2/(1+t), a3]] = 0
    D = [np.zeros_like(a) for a in A]
    D[0][:, 1] = A[0][:, 1]
    D[1][:, 1] = -A[1][:, 1]
    HD = orc.matvec(A, Gam, D, 0.0)
    scale = max(np.abs(h).max() for h in HU)
    assert max(np.abs(h).max() for h in HD) <= 1e-12 * scale


@pytest.mark.parametrize("dims,R", [((7, 6, 5, 4), 3), ((9, 8), 4), ((6, 5, 7), 5)])
def test_matvec_quadratic_form_from_grams(orc, dims, R):
    """<W, (J^T J + lam I) W> from R x R quantities only: lam ||W||^2 +
    sum_n <W^(n)T W^(n), Gamma^(n,n)> + sum_n <Y^(n)T, T^(n)>, Y^(p) = A^(p)T W^(p),
    T^(n) = sum_{p != n} Gamma^(n,p) * Y^(p) (the curvature of a CG step without
    forming Q)."""
    A = _rand_factors(dims, R, 51)
    W = _rand_factors(dims, R, 52)
    lam = 0.3
    Gam = orc.gamma(orc.gram(A))
    N = len(dims)
    direct = sum(float(np.sum(w * q)) for w, q in zip(W, orc.matvec(A, Gam, W, lam)))
    Y = [a.T @ w for a, w in zip(A, W)]
    T = [sum(Gam[n, p] * Y[p] for p in range(N) if p != n) for n in range(N)]
    grams = lam * sum(float(np.sum(w * w)) for w in W) + sum(float(np.sum((w.T @ w) * Gam[n, n]))
                                                            for n, w in enumerate(W))
    grams += sum(float(np.sum(Y[n].T * T[n])) for n in range(N))
    assert abs(grams - direct) <= 1e-12 * abs(direct)


# -------------------------------------------------------------------------- PCG

@pytest.mark.parametrize("dims,R,lam", [((5, 4, 6), 3, 1e-2), ((4, 3, 3, 2), 2, 0.5)])
def test_pcg_solves_normal_equations(orc, dims, R, lam):
    """CP-CG (Algorithm 2) driven to a tiny tolerance equals the dense solve of
    (J^T J + lam I) v = -g, within the N s R iteration bound of Section 3.4."""
    A = _rand_factors(dims, R, 18)
    X = _rand_tensor(dims, 18)
    Gam = orc.gamma(orc.gram(A))
    G, _ = orc.gradient(A, Gam, orc.mttkrp(X, A))
    V, iters, rn, st = orc.pcg(A, Gam, G, lam, 1e-13, 10000)
    assert st == orc.OK
    J = cpref.jacobian(A)
    H = J.T @ J + lam * np.eye(J.shape[1])
    ref = np.linalg.solve(H, -cpref.pack(G))
    np.testing.assert_allclose(cpref.pack(V), ref, rtol=1e-8, atol=1e-9 * np.abs(ref).max())
    # finite termination: N s R iterations already reach the solution up to rounding
    n_unknowns = sum(dims) * R
    Vn, it_n, _, _ = orc.pcg(A, Gam, G, lam, 0.0, n_unknowns)
    assert it_n == n_unknowns
    np.testing.assert_allclose(cpref.pack(Vn), ref, rtol=1e-7, atol=1e-8 * np.abs(ref).max())


def test_pcg_fixed_iterations_and_warning(orc):
    dims, R = (6, 5, 4), 3
    A = _rand_factors(dims, R, 19)
    X = _rand_tensor(dims, 19)
    Gam = orc.gamma(orc.gram(A))
    G, _ = orc.gradient(A, Gam, orc.mttkrp(X, A))
    V, iters, _, st = orc.pcg(A, Gam, G, 1e-3, 0.0, 4)
    assert iters == 4 and st == orc.WARN_CG_MAXIT
    # one CG step from V=0 is the preconditioned steepest-descent step
    V1, it1, _, _ = orc.pcg(A, Gam, G, 1e-3, 0.0, 1)
    Z = [g @ orc.precond_inv(Gam[n, n], 1e-3)[0] for n, g in enumerate(G)]
    Rr = [-g for g in G]
    Zr = [-z for z in Z]
    HZ = orc.matvec(A, Gam, Zr, 1e-3)
    alpha = sum(np.sum(r * z) for r, z in zip(Rr, Zr)) / sum(np.sum(z * h) for z, h in zip(Zr, HZ))
    for v, z in zip(V1, Zr):
        np.testing.assert_allclose(v, alpha * z, rtol=1e-12, atol=1e-15)


def test_pcg_printed_beta_differs(orc):
    """The ratio printed for beta in Algorithm 2 differs from standard PCG; the
    oracle keeps both (beta_kind) and the library follows standard PCG."""
    dims, R = (6, 5, 4), 3
    A = _rand_factors(dims, R, 20)
    X = _rand_tensor(dims, 20)
    Gam = orc.gamma(orc.gram(A))
    G, _ = orc.gradient(A, Gam, orc.mttkrp(X, A))
    Vs, _, _, _ = orc.pcg(A, Gam, G, 1e-2, 0.0, 3, 0)
    Vp, _, _, _ = orc.pcg(A, Gam, G, 1e-2, 0.0, 3, 1)
    assert max(np.abs(a - b).max() for a, b in zip(Vs, Vp)) > 1e-6


# ------------------------------------------------- diagonal damping (Section 3.2)

def _diag_damping(J):
    return np.diag(np.diag(J.T @ J))


@pytest.mark.parametrize("dims,R", [((6, 5, 7), 3), ((4, 3, 5, 2), 3), ((5, 6), 2)])
def test_matvec_diag_damping_explicit_jacobian(orc, dims, R):
    """Q = (J^T J + lam diag(J^T J)) w with J formed explicitly (Eq. (3.1))."""
    A = _rand_factors(dims, R, 41)
    W = _rand_factors(dims, R, 42)
    Gam = orc.gamma(orc.gram(A))
    J = cpref.jacobian(A)
    w = cpref.pack(W)
    lam = 0.37
    ref = J.T @ (J @ w) + lam * (_diag_damping(J) @ w)
    got = cpref.pack(orc.matvec(A, Gam, W, lam, orc.REG_DIAG))
    np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())
    # the two dampings differ exactly by lam (diag(J^T J) - I) w
    ident = cpref.pack(orc.matvec(A, Gam, W, lam, orc.REG_IDENTITY))
    np.testing.assert_allclose(got - ident, lam * (_diag_damping(J) - np.eye(len(w))) @ w, rtol=1e-10,
                               atol=1e-12 * np.abs(ref).max())


def test_precond_diag_damping(orc):
    A = _rand_factors((9, 8, 7), 5, 43)
    Gam = orc.gamma(orc.gram(A))
    B = Gam[1, 1]
    for lam in (0.0, 1e-3, 10.0):
        P, st = orc.precond_inv(B, lam, orc.REG_DIAG)
        assert st == orc.OK
        np.testing.assert_allclose((B + lam * np.diag(np.diag(B))) @ P, np.eye(5), atol=1e-12)
    # an indefinite matrix stays rejected
    _, st = orc.precond_inv(np.array([[1.0, 2.0], [2.0, 1.0]]), 0.5, orc.REG_DIAG)
    assert st == orc.ERR_NOT_SPD


@pytest.mark.parametrize("dims,R,lam", [((5, 4, 6), 3, 1e-2), ((4, 3, 3, 2), 2, 0.5)])
def test_pcg_diag_damping_solves_normal_equations(orc, dims, R, lam):
    A = _rand_factors(dims, R, 44)
    X = _rand_tensor(dims, 44)
    Gam = orc.gamma(orc.gram(A))
    G, _ = orc.gradient(A, Gam, orc.mttkrp(X, A))
    V, _, _, st = orc.pcg(A, Gam, G, lam, 1e-13, 10000, 0, orc.REG_DIAG)
    assert st == orc.OK
    J = cpref.jacobian(A)
    ref = np.linalg.solve(J.T @ J + lam * _diag_damping(J), -cpref.pack(G))
    np.testing.assert_allclose(cpref.pack(V), ref, rtol=1e-8, atol=1e-9 * np.abs(ref).max())


def test_diag_damping_is_folded_gamma_diagonal(orc):
    """lam diag(J^T J) touches only the diagonal of each Gamma^(n,n): the damped
    preconditioner, matvec and CG equal the undamped ones (lam = 0) on Gamma
    with Gamma^(n,n)_{rr} replaced by (1 + lam) Gamma^(n,n)_{rr}, the form in
    which the library applies it."""
    dims, R, lam = (6, 7, 5, 4), 3, 0.3
    A = _rand_factors(dims, R, 46)
    W = _rand_factors(dims, R, 47)
    X = _rand_tensor(dims, 46)
    Gam = orc.gamma(orc.gram(A))
    Gd = Gam.copy()
    for n in range(len(dims)):
        Gd[n, n][np.diag_indices(R)] += lam * np.diag(Gam[n, n])
    for q, qd in zip(orc.matvec(A, Gam, W, lam, orc.REG_DIAG), orc.matvec(A, Gd, W, 0.0)):
        np.testing.assert_allclose(q, qd, rtol=1e-13, atol=1e-13 * np.abs(q).max())
    for n in range(len(dims)):
        np.testing.assert_allclose(orc.precond_inv(Gam[n, n], lam, orc.REG_DIAG)[0],
                                   orc.precond_inv(Gd[n, n], 0.0)[0], rtol=1e-12, atol=1e-15)
    G, _ = orc.gradient(A, Gam, orc.mttkrp(X, A))
    V, _, _, _ = orc.pcg(A, Gam, G, lam, 0.0, 6, 0, orc.REG_DIAG)
    Vd, _, _, _ = orc.pcg(A, Gd, G, 0.0, 0.0, 6)
    for v, vd in zip(V, Vd):
        np.testing.assert_allclose(v, vd, rtol=1e-10, atol=1e-12 * np.abs(v).max())


def test_gn_step_diag_damping_commutes_with_column_scaling(orc):
    """The CP model is unchanged by A^(1) c, A^(2) / c (column scaling, Section
    3.2).  The map is linear in the unknowns, J(phi(A)) = J(A) S^-1, so the
    system damped by diag(J^T J), its block-Jacobi preconditioner and every CG
    iterate transform covariantly: a GN step from the rescaled point is the
    rescaled GN step.  Damping by lam I breaks this."""
    dims, R = (7, 6, 5), 3
    A = _rand_factors(dims, R, 45)
    X = _rand_tensor(dims, 45)
    c = np.array([3.0, 0.7, 1.9])
    Ac = [A[0] * c, A[1] / c, A[2].copy()]
    np.testing.assert_allclose(cpref.reconstruct(Ac), cpref.reconstruct(A), rtol=1e-12, atol=1e-12)

    def step(F, reg):
        out, _, _, _, st = orc.gn_step(X, F, 0.05, 0, 1e-3, 1.0, 2.0, 0.0, 6, reg=reg)
        assert st == orc.WARN_CG_MAXIT
        return out

    new = step(A, orc.REG_DIAG)
    newc = step(Ac, orc.REG_DIAG)
    for got, ref in zip(newc, [new[0] * c, new[1] / c, new[2]]):
        np.testing.assert_allclose(got, ref, rtol=1e-9, atol=1e-10 * np.abs(ref).max())
    new = step(A, orc.REG_IDENTITY)
    newc = step(Ac, orc.REG_IDENTITY)
    dev = max(np.abs(g - r).max() / np.abs(r).max() for g, r in zip(newc, [new[0] * c, new[1] / c, new[2]]))
    assert dev > 1e-4


# ------------------------------------------------------------------ lambda rule

def test_lambda_schedule_golden(orc):
    for lam0, lo, hi, mu, seq in cpref.load_lambda_golden(os.path.join(GOLDEN, "lambda_schedule.txt")):
        lam, d = lam0, 0
        got = []
        for _ in seq:
            got.append(lam)
            lam, d = orc.lambda_next(lam, d, lo, hi, mu)
        np.testing.assert_allclose(got, seq, rtol=1e-15)


# ---------------------------------------------------------------------- GN step

def test_gn_exact_recovery(orc):
    """Algorithm 1 recovers exact rank-5 decompositions of 20^3 Gaussian tensors
    to relative residual <= 1e-10 (Section 5.3's exact-CP setting)."""
    converged = 0
    for seed in range(4):
        p = datagen.workload("exact20", seed=seed)
        X, A = p["X"], p["init"]
        hi, lo = orc.default_lambda(A)
        lam, d = hi, 0
        r = 1.0
        for _ in range(100):
            A, lam, d, s, st = orc.gn_step(X, A, lam, d, lo, hi, 2.0, 1e-3, 250)
            assert st in (orc.OK, orc.WARN_CG_MAXIT)
            r = orc.residual(X, A)
            if r <= 1e-10:
                break
        converged += r <= 1e-10
    assert converged == 4


def test_gn_step_stats(orc):
    p = datagen.workload("exact20", seed=1)
    X, A = p["X"], p["init"]
    Gam = orc.gamma(orc.gram(A))
    M = orc.mttkrp(X, A)
    _, gn = orc.gradient(A, Gam, M)
    A1, lam, d, s, st = orc.gn_step(X, A, 1.0, 0, 1e-3, 1.0, 2.0, 0.0, 5)
    assert s["cg_iters"] == 5 and st == orc.WARN_CG_MAXIT
    assert abs(s["grad_norm_sum"] - gn.sum()) <= 1e-12 * gn.sum()
    assert s["lam_used"] == 1.0 and lam == 0.5 and d == 0
    V, _, _, _ = orc.pcg(A, Gam, orc.gradient(A, Gam, M)[0], 1.0, 0.0, 5)
    for a1, a, v in zip(A1, A, V):
        np.testing.assert_allclose(a1, a + v, rtol=1e-13, atol=1e-14)


# --------------------------------------------------------------------- residual

def test_residual(orc):
    dims, R = (9, 8, 7), 4
    A = _rand_factors(dims, R, 21)
    X0 = cpref.reconstruct(A)
    assert orc.residual(X0, A) <= 1e-15
    E = np.random.default_rng(22).standard_normal(dims)
    eta = 1e-3
    X = X0 + eta * np.linalg.norm(X0) * E / np.linalg.norm(E)
    r = orc.residual(X, A)
    ref = np.linalg.norm(X - X0) / np.linalg.norm(X)
    assert abs(r - ref) <= 1e-12 * ref
    assert abs(r - eta) <= 2e-3 * eta
    B = _rand_factors(dims, R, 23)
    ref = np.linalg.norm(X - cpref.reconstruct(B)) / np.linalg.norm(X)
    assert abs(orc.residual(X, B) - ref) <= 1e-13 * ref


# -------------------------------------------------------------------------- ALS

def test_als_monotone_and_normal_equations(orc):
    """ALS decreases the objective monotonically (Section 1) and, right after
    mode n is updated, its gradient block vanishes (the normal equations)."""
    dims, R = (8, 7, 6), 3
    X = _rand_tensor(dims, 24)
    A = _rand_factors(dims, R, 25)
    f_prev = cpref.objective(X, A)
    for _ in range(8):
        A, st = orc.als_sweep(X, A)
        assert st == orc.OK
        f = cpref.objective(X, A)
        assert f <= f_prev * (1 + 1e-14)
        f_prev = f
        # the last mode was updated last: its gradient block is zero
        Gam = orc.gamma(orc.gram(A))
        G, gn = orc.gradient(A, Gam, orc.mttkrp(X, A))
        Mn = np.linalg.norm(orc.mttkrp(X, A)[2])
        assert gn[2] <= 1e-12 * Mn


def test_als_regularised(orc):
    """With lam > 0 the mode update solves A (Gamma + lam I) = M."""
    dims, R = (6, 5, 7), 3
    X = _rand_tensor(dims, 26)
    A = _rand_factors(dims, R, 27)
    lam = 0.3
    A1, _ = orc.als_sweep(X, A, lam)
    # mode 0 was updated with the original factors of modes 1, 2
    Gam0 = (A[1].T @ A[1]) * (A[2].T @ A[2])
    M0 = _einsum_mttkrp(X, A, 0)
    np.testing.assert_allclose(A1[0] @ (Gam0 + lam * np.eye(R)), M0, rtol=1e-11, atol=1e-12)


def test_gn_solve_is_the_step_loop_with_algorithm1_test(orc):
    """The oracle's solve is Algorithm 1's loop: the same factors, bit for bit,
    as repeated single steps stopped at the first entry point whose
    sum||G||/sum||M|| meets the target; and it recovers the exact 20^3 rank-5
    decomposition (r <= 1e-10)."""
    from paper_1910_12331_gb300 import datagen

    p = datagen.workload("exact20", seed=0)
    hi, lo = orc.default_lambda(p["init"])
    target = 1e-12
    A_s, st, info = orc.gn_solve(p["X"], p["init"], hi, lo, hi, 2.0, 1e-3, 250, target, 100)
    assert st == orc.OK and info["converged"]
    A, lam, d, n, cg = [a.copy() for a in p["init"]], hi, 0, 0, 0
    while True:
        M = orc.mttkrp(p["X"], A, "dt")
        _, gn = orc.gradient(A, orc.gamma(orc.gram(A)), M)
        if gn.sum() <= target * sum(np.linalg.norm(m) for m in M):
            break
        A, lam, d, s, _ = orc.gn_step(p["X"], A, lam, d, lo, hi, 2.0, 1e-3, 250, use_dt=True)
        n, cg = n + 1, cg + s["cg_iters"]
    assert info["updates"] == n and info["cg_iters"] == cg
    for a, b in zip(A_s, A):
        assert np.array_equal(a, b)
    assert orc.residual(p["X"], A_s) <= 1e-10


def test_residual_tensor_definition(orc):
    """E = X - [[A]] element by element: equal to numpy's reconstruction from
    the definition (tests/cpref.py), zero at an exact decomposition, and its
    squared sum over ||X||^2 is the squared relative residual."""
    from tests import cpref

    rng = np.random.default_rng(61)
    for dims, R in [((5, 4, 6), 3), ((3, 4, 2, 5), 2), ((7, 9), 4)]:
        A = [rng.standard_normal((s, R)) for s in dims]
        X = rng.standard_normal(dims)
        E = orc.residual_tensor(X, A)
        np.testing.assert_allclose(E, X - cpref.reconstruct(A), rtol=0, atol=1e-13)
        r = orc.residual(X, A)
        assert abs(np.sum(E * E) / np.sum(X * X) - r * r) <= 1e-13 * r * r
        assert np.abs(orc.residual_tensor(cpref.reconstruct(A), A)).max() <= 1e-13


def _armijo_case(orc):
    """A 6x5x7 random tensor, R = 4, after two plain GN steps at a constant
    lambda = 1e-4: the full third step raises the objective (84.75 -> 121.76)."""
    rng = np.random.default_rng(0)
    dims, R = (6, 5, 7), 4
    X = rng.standard_normal(dims)
    A = [rng.standard_normal((s, R)) for s in dims]
    for _ in range(2):
        A, _, _, _, _ = orc.gn_step_ls(X, A, 1e-4, 0, 1e-9, 1.0, 2.0, 1e-10, 60, lam_fixed=True)
    return X, A


def test_armijo_condition_at_the_accepted_step(orc):
    """Section 5's step-size control by Armijo's condition: the step taken is
    the first t in 1, 1/2, 1/4, ... with f(A + tV) <= f(A) + c t <grad f, V>,
    checked with numpy's objective (tests/cpref.py) and the oracle's pinned
    gradient; the trial before it fails the condition; f decreases."""
    from tests import cpref

    X, A = _armijo_case(orc)
    c = 1e-4
    A_full, _, _, _, _ = orc.gn_step_ls(X, A, 1e-4, 0, 1e-9, 1.0, 2.0, 1e-10, 60, lam_fixed=True)
    A_ls, lam, _, s, st = orc.gn_step_ls(X, A, 1e-4, 0, 1e-9, 1.0, 2.0, 1e-10, 60, lam_fixed=True, armijo_c=c)
    assert st in (orc.OK, orc.WARN_CG_MAXIT) and lam == 1e-4  # constant lambda
    V = [af - a for af, a in zip(A_full, A)]  # the full GN direction
    G, _ = orc.gradient(A, orc.gamma(orc.gram(A)), orc.mttkrp(X, A))
    slope = sum(float(np.sum(g * v)) for g, v in zip(G, V))
    f0 = cpref.objective(X, A)
    assert abs(s["f0"] - f0) <= 1e-12 * f0 and slope < 0
    t = s["step"]
    assert t == 0.5 and s["trials"] == 2
    for a_ls, a, v in zip(A_ls, A, V):
        np.testing.assert_allclose(a_ls, a + t * v, rtol=0, atol=1e-12)
    assert cpref.objective(X, A_ls) <= f0 + c * t * slope
    assert cpref.objective(X, [a + 2 * t * v for a, v in zip(A, V)]) > f0 + c * 2 * t * slope
    assert cpref.objective(X, A_ls) < f0


def test_armijo_full_step_near_exact_decomposition(orc):
    """Close to an exact decomposition the GN step is nearly a Newton step and
    the full step meets Armijo's condition at once."""
    from paper_1910_12331_gb300 import datagen

    p = datagen.workload("exact20", seed=0)
    rng = np.random.default_rng(5)
    A = [a + 1e-4 * rng.standard_normal(a.shape) for a in p["truth"]]
    _, _, _, s, st = orc.gn_step_ls(p["X"], A, 1e-6, 0, 1e-9, 1.0, 2.0, 1e-10, 100, lam_fixed=True, armijo_c=1e-4)
    assert st in (orc.OK, orc.WARN_CG_MAXIT) and s["step"] == 1.0 and s["trials"] == 1


def test_armijo_off_is_the_plain_step(orc):
    """armijo_c = 0 and a varying lambda: bit for bit the plain GN step."""
    X, A = _armijo_case(orc)
    A1, l1, d1, s1, st1 = orc.gn_step(X, A, 0.3, 0, 1e-3, 1.0, 2.0, 1e-3, 50)
    A2, l2, d2, s2, st2 = orc.gn_step_ls(X, A, 0.3, 0, 1e-3, 1.0, 2.0, 1e-3, 50)
    assert st1 == st2 and l1 == l2 and d1 == d2 and s2["step"] == 1.0
    for a, b in zip(A1, A2):
        assert np.array_equal(a, b)


# ------------------------------------------------ Tucker / HoSVD (compression ahead of CP, for R < s)

def _tucker_tensor(dims, ranks, seed, noise=0.0):
    """X = G x_1 Q_1 ... x_N Q_N with orthonormal Q_n (s_n x r_n) and a random core:
    a tensor of exact multilinear rank `ranks` (plus optional noise)."""
    rng = np.random.default_rng(seed)
    Q = [np.linalg.qr(rng.standard_normal((s, r)))[0] for s, r in zip(dims, ranks)]
    X = rng.standard_normal(ranks)
    for n, q in enumerate(Q):
        X = np.moveaxis(np.tensordot(q, X, axes=(1, n)), 0, n)
    if noise:
        X = X + noise * rng.standard_normal(dims)
    return X, Q


def test_unfold_gram_and_jacobi_eigen(orc):
    rng = np.random.default_rng(80)
    X = rng.standard_normal((5, 6, 7, 4))
    for n in range(4):
        Xn = np.moveaxis(X, n, 0).reshape(X.shape[n], -1)
        S = orc.unfold_gram(X, n)
        np.testing.assert_allclose(S, Xn @ Xn.T, rtol=0, atol=1e-12 * np.abs(S).max())
        w, V = orc.sym_eig(S)
        np.testing.assert_allclose(w, np.sort(np.linalg.eigvalsh(S))[::-1], rtol=0, atol=1e-12 * w[0])
        np.testing.assert_allclose(V.T @ V, np.eye(len(w)), atol=1e-13)
        np.testing.assert_allclose(S @ V, V * w, atol=1e-12 * w[0])


def test_mode_product_definition(orc):
    rng = np.random.default_rng(81)
    T = rng.standard_normal((4, 5, 6))
    U = rng.standard_normal((5, 3))
    np.testing.assert_allclose(orc.mode_product_t(T, 1, U), np.einsum("ijk,ja->iak", T, U), atol=1e-13)


def test_hosvd_exact_multilinear_rank(orc):
    """A tensor of multilinear rank (3, 4, 2) is reproduced exactly by its
    truncated HoSVD, and the U_n span the generating subspaces."""
    X, Q = _tucker_tensor((9, 8, 7), (3, 4, 2), 82)
    U, core, _ = orc.hosvd(X, (3, 4, 2))
    Xh = core
    for n, u in enumerate(U):
        Xh = orc.mode_product_t(Xh, n, u.T)  # x_n U_n
    np.testing.assert_allclose(Xh, X, atol=1e-12 * np.abs(X).max())
    for u, q in zip(U, Q):
        np.testing.assert_allclose(u @ u.T, q @ q.T, atol=1e-12)


def test_hosvd_error_bounds(orc):
    """De Lathauwer, De Moor and Vandewalle (2000): the truncated HoSVD error
    satisfies max_n sum_{i > r_n} lambda_i^(n) <= ||X - X^||^2 <=
    sum_n sum_{i > r_n} lambda_i^(n), lambda^(n) the eigenvalues of X_(n) X_(n)^T."""
    X, _ = _tucker_tensor((8, 9, 10), (3, 3, 4), 83, noise=0.05)
    ranks = (3, 3, 4)
    U, core, W = orc.hosvd(X, ranks)
    Xh = core
    for n, u in enumerate(U):
        Xh = orc.mode_product_t(Xh, n, u.T)
    err = float(np.sum((X - Xh) ** 2))
    tails = [float(np.sum(w[r:])) for w, r in zip(W, ranks)]
    assert max(tails) * (1 - 1e-10) <= err <= sum(tails) * (1 + 1e-10)


def test_cp_of_the_core_splits_the_error(orc):
    """With orthonormal U_n, a CP model B of the core expanded to A_n = U_n B_n
    has ||X - [[A]]||^2 = ||X - X^||^2 + ||core - [[B]]||^2 (Pythagoras in the
    subspace), which is what makes CP on the compressed core exact."""
    from tests import cpref

    X, _ = _tucker_tensor((9, 8, 7), (4, 4, 3), 84, noise=0.1)
    ranks = (4, 4, 3)
    U, core, _ = orc.hosvd(X, ranks)
    Xh = core
    for n, u in enumerate(U):
        Xh = orc.mode_product_t(Xh, n, u.T)
    rng = np.random.default_rng(85)
    B = [rng.standard_normal((r, 3)) for r in ranks]
    A = [u @ b for u, b in zip(U, B)]
    lhs = 2 * cpref.objective(X, A)
    rhs = float(np.sum((X - Xh) ** 2)) + 2 * cpref.objective(core, B)
    assert abs(lhs - rhs) <= 1e-12 * lhs
