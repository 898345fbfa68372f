"""The allocation-free matvec entry point (cp_gn_matvec_noalloc).

It exists for callers that cannot call cudaMalloc -- code under a fixed,
pre-reserved device-memory budget, inside an allocator callback, or in a
serving loop that must not allocate after start-up -- and keeps its scratch
in a static device array of the library.  This file checks, through the C
ABI, that two calls in a row give the same result as the handle-based
cp_gn_matvec within the FP64 tolerance of the other tests, and that shapes
beyond the static scratch are refused.  It is collected last on purpose."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL = 1e-12


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


def _mats(torch, dims, R, seed):
    rng = np.random.default_rng(seed)
    return [torch.from_numpy(rng.standard_normal((s, R))).cuda() for s in dims]


def _relerr(a, b):
    scale = max(x.abs().max().item() for x in b)
    return max((x - y).abs().max().item() for x, y in zip(a, b)) / scale


@pytest.mark.parametrize("dims,R", [((37, 70, 45), 13), ((6, 5, 4, 7), 4), ((300, 120, 80), 64), ((9, 11), 3)])
def test_noalloc_matches_handle_matvec_twice(env, dims, R):
    torch, api, h = env
    A = _mats(torch, dims, R, 1)
    Q = [torch.full_like(a, float("nan")) for a in A]
    for call, (seed, lam) in enumerate([(2, 0.0), (3, 0.75)]):
        W = _mats(torch, dims, R, seed)
        ref = api.cp_gn_matvec(h, A, W, lam)
        api.cp_gn_matvec_noalloc(A, W, lam, Q)
        torch.cuda.synchronize()
        err = _relerr(Q, ref)
        assert err <= TOL, (call, err)


def test_noalloc_rejects_beyond_static_scratch(env):
    torch, api, h = env
    L = api.load()
    for dims, R in [((4, 4, 4), 65), ((3, 3, 3, 3, 3), 2)]:
        A = _mats(torch, dims, R, 4)
        Q = [torch.empty_like(a) for a in A]
        d = api.make_desc(dims, R, torch.float64)
        s = L.cp_gn_matvec_noalloc(ctypes.byref(d), api._ptr_array(A), api._ptr_array(A), 0.0, api._ptr_array(Q), None)
        assert s == api.CP_ERR_UNSUPPORTED
