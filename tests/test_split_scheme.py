"""CPU emulation of the operand splits of the tensor-core MTTKRP, on the very
inputs of the GPU bf16x3 tests: where the 2e-5 tolerance of those tests comes
from.

The library splits every operand value v into bf16 parts v = v_hi + v_lo + d,
v_hi = RN_bf16(v), v_lo = RN_bf16(v - v_hi), so |d| <= 2^-8 |v - v_hi| <= 2^-16 |v|
(bf16 keeps 8 significant bits; round to nearest errs by at most 2^-8 of the
value).  Each bf16 x bf16 product is exact in the FP32 accumulator (16
significant bits).
  mode 1 (GEMM-Y, three products x_hi b_hi + x_lo b_hi + x_hi b_lo, b = a^(N)
  split from FP64, times w_m rounded to FP32): a term x b w carries at most
  3 * 2^-16 + 2^-24 of relative error (d_x, d_b, the dropped x_lo b_lo, w).
  mode N (GEMM-Z, all four products of u = fl32(fl32(a^(1)) fl32(w_m)) and x):
  at most 2 * 2^-16 + 3 * 2^-24.
  middle modes: c_m = sum_i a^(1)_i (x_m A^(N))_i with the GEMM-Y products and
  the FP32 A^(1) rows: at most 3 * 2^-16 + 2^-24 again.
The emulation accumulates in FP64, so it isolates these representation errors
(the kernel's FP32 accumulation adds about 1e-6 more).  The checks: every entry
within its bound times the sum of |terms|, and the largest error below half of
the GPU tests' tolerance (2e-5 of max |M|), so that tolerance keeps at least a
factor 2 for the FP32 accumulation."""
import numpy as np
import pytest

TOL_BF16X3 = 2e-5  # the tolerance of the GPU bf16x3 MTTKRP tests
U = 2.0 ** -16      # representation bound of a two-part bf16 split
E32 = 2.0 ** -24


def bf16_rn(v):
    """Round to the nearest bf16 value (8 significant bits, ties to even)."""
    v = np.asarray(v, dtype=np.float64)
    m, e = np.frexp(v)
    return np.ldexp(np.rint(np.ldexp(m, 8)), e - 8)


def split(v):
    hi = bf16_rn(v)
    return hi, bf16_rn(v - hi)


def f32(v):
    return np.asarray(v, dtype=np.float32).astype(np.float64)


def _problem(dims, R, seed):
    rng = np.random.default_rng(seed)
    A = [rng.standard_normal((s, R)) for s in dims]
    X = rng.standard_normal(dims).astype(np.float32)
    return X, A


def _middle_weights(A, dims):
    mids = dims[1:-1]
    R = A[0].shape[1]
    W = np.ones((int(np.prod(mids)) if mids else 1, R))
    if mids:
        idx = np.indices(mids).reshape(len(mids), -1)
        for q, ix in enumerate(idx):
            W = W * A[1 + q][ix]
    return W


def emulate(X, A):
    """(emulated M, exact M, sum of |terms|) per mode, FP64 accumulation."""
    dims = X.shape
    N = len(dims)
    X3 = X.reshape(dims[0], -1, dims[-1]).astype(np.float64)
    xh, xl = split(X3)
    W = _middle_weights(A, dims)
    Wf = f32(W)
    bh, bl = split(A[-1])
    A1f = f32(A[0])
    out = []
    # mode 1: M1[i] = sum_m w_m * (X_m A^(N))[i]
    DY = np.einsum("imk,kr->imr", xh, bh) + np.einsum("imk,kr->imr", xl, bh) + np.einsum("imk,kr->imr", xh, bl)
    DYx = np.einsum("imk,kr->imr", X3, A[-1])
    M1 = np.einsum("mr,imr->ir", Wf, DY)
    M1x = np.einsum("mr,imr->ir", W, DYx)
    S1 = np.einsum("mr,imk,kr->ir", np.abs(W), np.abs(X3), np.abs(A[-1]))
    out.append((M1, M1x, S1))
    # middle modes: c_m = colsum(A^(1) * Y_m), times the other middle factors
    mids = dims[1:-1]
    if mids:
        c = np.einsum("ir,imr->mr", A1f, DY)
        cx = np.einsum("ir,imr->mr", A[0], DYx)
        cs = np.einsum("ir,imk,kr->mr", np.abs(A[0]), np.abs(X3), np.abs(A[-1]))
        idx = np.indices(mids).reshape(len(mids), -1)
        for q in range(len(mids)):
            other = np.ones_like(W)
            for q2, ix in enumerate(idx):
                if q2 != q:
                    other = other * A[1 + q2][ix]
            Mq, Mqx, Sq = (np.zeros((mids[q], W.shape[1])) for _ in range(3))
            np.add.at(Mq, idx[q], c * other)
            np.add.at(Mqx, idx[q], cx * other)
            np.add.at(Sq, idx[q], cs * np.abs(other))
            out.append((Mq, Mqx, Sq))
    # mode N: M^(N)[k] = sum_m sum_i u_{m,i} x_{i,m,k}, u = fl32(A1f * Wf)
    MN = np.zeros((dims[-1], W.shape[1]))
    for m in range(X3.shape[1]):
        uh, ul = split(f32(A1f * Wf[m]))
        MN += (xh[:, m, :] + xl[:, m, :]).T @ (uh + ul)
    MNx = np.einsum("imk,ir,mr->kr", X3, A[0], W)
    SN = np.einsum("imk,ir,mr->kr", np.abs(X3), np.abs(A[0]), np.abs(W))
    out.append((MN, MNx, SN))
    return out


SHAPES = [((37, 70, 45), 13), ((20, 20, 20), 5), ((130, 3, 140), 64), ((300, 5, 520), 20), ((6, 5, 4, 7), 4),
          ((50, 70), 9), ((40, 30, 50), 100), ((3, 4, 2, 3, 2), 2), ((129, 9, 127), 50), ((64, 33, 8), 1)]


@pytest.mark.parametrize("dims,R", SHAPES)
def test_split_representation_error(dims, R):
    X, A = _problem(dims, R, 1)
    res = emulate(X, A)
    N = len(dims)
    bounds = [3 * U + E32] + [3 * U + E32] * (N - 2) + [2 * U + 3 * E32]
    worst = 0.0
    for n, ((M, Mx, S), bnd) in enumerate(zip(res, bounds)):
        err = np.abs(M - Mx)
        assert np.all(err <= bnd * S * (1 + 1e-6) + 1e-300), (dims, R, n)
        worst = max(worst, err.max() / np.abs(Mx).max())
    assert worst <= TOL_BF16X3 / 2, (dims, R, worst)


def test_split_parts():
    """The premises: hi and lo are bf16 values (8 significant bits), the split
    error is at most 2^-16 |v|, and a bf16 x bf16 product is exact in FP32."""
    rng = np.random.default_rng(5)
    v = rng.standard_normal(100000) * np.exp(rng.uniform(-20, 20, 100000))
    hi, lo = split(v)
    for part in (hi, lo):
        m, _ = np.frexp(part)
        assert np.all(np.ldexp(m, 8) == np.rint(np.ldexp(m, 8)))
    assert np.all(np.abs(v - hi - lo) <= U * np.abs(v))
    p = hi[:-1] * hi[1:]
    assert np.all(f32(p) == p)
