"""The arithmetic of the tensor-core reconstruction of the residual tensor
(error-free bf16 slice products on fixed power-of-two grids), emulated in
NumPy on the CPU: the premises the kernel relies on hold, and the scheme's
error stays within its stated bound.

Scheme (per slice m): u_ir = a1_ir w_r and v_kr are scaled by powers of two
sigma_i >= max_r |u_ir|, tau_k >= max_r |v_kr| and cut into six pieces on the
grids 2^-8s (round to nearest, remainder to the next piece); the level sums
D_L = sum_{s+t=L} sum_r u_s v_t for L = 2..7 are combined in double-float.
The FP32 steps of the kernel's cutting of u (hi/lo double-float input) are
emulated with float32 arithmetic; the pieces of v are cut in FP64."""
import numpy as np
import pytest

f32 = np.float32


def _pow2_ceil(v):
    v = np.maximum(np.asarray(v, dtype=np.float64), 2.0 ** -100)
    return 2.0 ** np.ceil(np.log2(v))


def _cut_df(h, l):
    """Six pieces of the double-float value h + l (|h| <= 1), FP32 steps."""
    h, l = h.astype(f32), l.astype(f32)
    out = []
    for s in (1, 2, 3):
        g = f32(2.0 ** (8 * s))
        q = (np.rint(h * g) / g).astype(f32)
        out.append(q)
        h = (h - q).astype(f32)
    hh = (h + l).astype(f32)
    z = (hh - h).astype(f32)
    ll = ((h - (hh - z)) + (l - z)).astype(f32)
    g = f32(2.0 ** 32)
    q = (np.rint(hh * g) / g).astype(f32)
    out.append(q)
    hh = ((hh - q) + ll).astype(f32)
    for s in (5, 6):
        g = f32(2.0 ** (8 * s))
        q = (np.rint(hh * g) / g).astype(f32)
        out.append(q)
        hh = (hh - q).astype(f32)
    return out


def _cut_fp64(x):
    out = []
    for s in range(1, 7):
        g = 2.0 ** (8 * s)
        q = np.rint(x * g) / g
        out.append(q)
        x = x - q
    return out


def _is_bf16(x):
    b = np.asarray(x, dtype=f32).view(np.uint32)
    return bool(np.all((b & 0xFFFF) == 0))


@pytest.mark.parametrize("s1,sN,R,collinear", [(48, 40, 50, False), (40, 56, 64, False), (32, 32, 50, True),
                                               (24, 20, 7, False), (64, 64, 1, False)])
def test_reconstruction_scheme(s1, sN, R, collinear):
    rng = np.random.default_rng(s1 * 1000 + R)
    A1 = rng.standard_normal((s1, R))
    AN = rng.standard_normal((sN, R))
    w = rng.standard_normal(R)
    if collinear:  # columns with cosine ~0.9 (all products of one sign dominate the sums)
        A1 = np.abs(A1) + 2.0
        AN = np.abs(AN) + 2.0
        w = np.abs(w) + 1.0
    U = A1 * w
    uh = U.astype(f32)
    ul = (U - uh.astype(np.float64)).astype(f32)
    sig = _pow2_ceil(np.abs(uh).max(axis=1)).astype(f32)
    pu = _cut_df(uh / sig[:, None], ul / sig[:, None])
    tau = _pow2_ceil(np.abs(AN).max(axis=1))
    pv = _cut_fp64(AN / tau[:, None])
    # every piece is an exact bf16 value (at most 8 significant bits)
    assert all(_is_bf16(p) for p in pu)
    assert all(_is_bf16(p.astype(f32)) and np.array_equal(p.astype(f32).astype(np.float64), p) for p in pv)
    levels = []
    for L in range(2, 8):
        D = np.zeros((s1, sN))
        for s in range(1, 7):
            t = L - s
            if 1 <= t <= 6:
                D += pu[s - 1].astype(np.float64) @ pv[t - 1].T
        units = D * 2.0 ** (8 * L)
        # integers on the level's grid, below 2^23: exact in the FP32 accumulator at every partial sum
        assert np.array_equal(units, np.rint(units))
        assert np.abs(units).max() < 2.0 ** 23
        assert np.array_equal(D.astype(f32).astype(np.float64), D)
        levels.append(D.astype(f32))
    # double-float combination as in the epilogue, then the reconstruction error against FP64
    D2, D3, D4, D5, D6, D7 = levels
    small = (((D7 + D6) + D5) + D4).astype(f32)
    h = (D2 + D3).astype(f32)
    z = (h - D2).astype(f32)
    l = ((D2 - (h - z)) + (D3 - z)).astype(f32)
    l = (l + small).astype(f32)
    rec = (h.astype(np.float64) + l.astype(np.float64)) * (sig[:, None].astype(np.float64) * tau[None, :])
    exact = U @ AN.T
    # the dropped piece pairs and remainders stay below 2^-46 R sigma tau; the FP32 additions of the small
    # levels (|D4| <~ 2^-16 R) add up to 2^-24 of that: total below 2^-39 R sigma tau
    bound = 2.0 ** -39 * R * (sig[:, None].astype(np.float64) * tau[None, :])
    assert np.all(np.abs(rec - exact) <= bound)
