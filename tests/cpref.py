"""Independent numpy constructions used to pin the oracle (tests only).

These build the objects of Section 3 from their definitions -- the Jacobian
tensor of Eq. (3.1) as an explicit matrix, the CP reconstruction, the
objective of Eq. (2.3) -- so that the oracle's structured formulas (Gamma
products, reassociated matvec, dimension tree) are checked against something
other than themselves.
"""
import string

import numpy as np


def reconstruct(A):
    N = len(A)
    letters = string.ascii_lowercase[:N]
    return np.einsum(",".join(f"{c}z" for c in letters) + "->" + letters, *A)


def objective(X, A):
    """f = 1/2 ||X - [[A]]||_F^2 (Eq. (2.3))."""
    D = np.asarray(X, dtype=np.float64) - reconstruct(A)
    return 0.5 * float(np.sum(D * D))


def jacobian(A):
    """Explicit matrix form of the Jacobian tensor of Eq. (3.1):
    J[e, (n, k, r)] = -(prod_{m != n} a^(m)_{i_m r}) delta_{i_n k}, rows e over
    the tensor entries in C order, columns over (mode n, row k, column r) in
    the packed factor order."""
    dims = [a.shape[0] for a in A]
    R = A[0].shape[1]
    N = len(A)
    total = int(np.prod(dims))
    cols = sum(dims) * R
    J = np.zeros((total, cols))
    idx = np.indices(dims).reshape(N, -1)  # multi-index of every entry, C order
    off = 0
    for n in range(N):
        for r in range(R):
            prod = np.ones(total)
            for m in range(N):
                if m != n:
                    prod *= A[m][idx[m], r]
            J[np.arange(total), off + idx[n] * R + r] = -prod
        off += dims[n] * R
    return J


def pack(mats):
    return np.concatenate([np.asarray(m, dtype=np.float64).reshape(-1) for m in mats])


def unpack(v, dims, R):
    out, off = [], 0
    for s in dims:
        out.append(v[off:off + s * R].reshape(s, R))
        off += s * R
    return out


def load_strassen(path):
    """Parse tests/golden/strassen_2x2.txt -> (C, A, B) each 4 x 7."""
    mats = {}
    rank = None
    with open(path) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            head, *rest = line.split(None, 1)
            if head == "strassen":
                rank = int(rest[0])
                continue
            rows = [list(map(float, part.split())) for part in rest[0].split("|")]
            mats[head] = np.array(rows)
    assert all(m.shape == (4, rank) for m in mats.values())
    return mats["C"], mats["A"], mats["B"]


def load_lambda_golden(path):
    cases = []
    with open(path) as fh:
        lines = [l.strip() for l in fh if l.strip() and not l.startswith("#")]
    for k in range(0, len(lines), 2):
        lam0, lo, hi, mu = map(float, lines[k].split())
        seq = list(map(float, lines[k + 1].split()))
        cases.append((lam0, lo, hi, mu, seq))
    return cases
