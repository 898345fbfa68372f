"""CPU checks of the C-ABI library: it builds, loads, and exports every call the
header declares; host-side logic that needs no GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?\w+\**\s+\**(cp_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_1910_12331_gb300 import build

    build.build()
    return ctypes.CDLL(build.LIB)


def test_header_declares_calls():
    names = _declared()
    for n in ("cp_mttkrp_all", "cp_gn_matvec", "cp_gn_step", "cp_als_sweep", "cp_residual"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_names_match_header():
    from paper_1910_12331_gb300 import api

    assert set(api.SYMBOLS) <= set(_declared())


def test_status_strings(lib):
    lib.cp_status_string.restype = ctypes.c_char_p
    assert lib.cp_status_string(0) == b"CP_OK"
    assert lib.cp_status_string(8) == b"CP_ERR_TIMEOUT"
    assert lib.cp_status_string(123) == b"CP_UNKNOWN_STATUS"


def test_null_arguments_rejected_without_gpu(lib):
    # argument checks run before any CUDA call
    lib.cp_mttkrp_all.restype = ctypes.c_int
    assert lib.cp_mttkrp_all(None, None, None, None, None, 0) == 1
    lib.cp_residual.restype = ctypes.c_int
    assert lib.cp_residual(None, None, None, None, None) == 1
    lib.cp_create.restype = ctypes.c_int
    assert lib.cp_create(None, 0) == 1


def test_batch_plan_arguments_rejected_without_gpu(lib):
    """The plan entry points check their arguments before any CUDA call."""
    vp = ctypes.c_void_p
    lib.cp_batch_plan_create.restype = ctypes.c_int
    lib.cp_batch_plan_create.argtypes = [vp, ctypes.c_int, vp, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                         ctypes.c_double, ctypes.c_int, ctypes.POINTER(vp)]
    out = vp()
    assert lib.cp_batch_plan_create(None, 4, None, 1e-3, 10, 10, 1e-6, 0, ctypes.byref(out)) == 1
    assert out.value is None
    for name in ("cp_batch_plan_launch", "cp_batch_plan_results"):
        f = getattr(lib, name)
        f.restype = ctypes.c_int
        assert f(None, None, None) == 1 if name == "cp_batch_plan_results" else f(None, None) == 1
    lib.cp_batch_plan_threads.restype = ctypes.c_int
    lib.cp_batch_plan_threads.argtypes = [vp, ctypes.POINTER(ctypes.c_int)]
    t = ctypes.c_int(-1)
    assert lib.cp_batch_plan_threads(None, ctypes.byref(t)) == 1 and t.value == -1
    lib.cp_batch_plan_configure.restype = ctypes.c_int
    lib.cp_batch_plan_configure.argtypes = [vp, ctypes.c_int, ctypes.c_int]
    assert lib.cp_batch_plan_configure(None, 256, 0) == 1
    lib.cp_batch_plan_destroy.restype = ctypes.c_int
    assert lib.cp_batch_plan_destroy(None) == 1


def test_noalloc_matvec_degenerate_arguments_rejected(lib):
    """cp_gn_matvec_noalloc takes no handle and checks every argument before
    its first CUDA call: order < 2, rank < 1, an empty mode, null factor
    pointers, an output that aliases an input or another output, and a
    negative or non-finite lambda are CP_ERR_ARG; order or rank beyond the
    static scratch is CP_ERR_UNSUPPORTED.  (Skipped where a GPU is visible:
    the fake device addresses must never reach a kernel.)"""
    import torch

    if torch.cuda.is_available():
        pytest.skip("argument checks only; fake device pointers")
    from paper_1910_12331_gb300 import api

    hdr = open(os.path.join(ROOT, "include", "cpgn.h")).read()
    max_order = int(re.search(r"#define CP_NOALLOC_MAX_ORDER (\d+)", hdr).group(1))
    max_rank = int(re.search(r"#define CP_NOALLOC_MAX_RANK (\d+)", hdr).group(1))
    vp = ctypes.c_void_p
    f = lib.cp_gn_matvec_noalloc
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.POINTER(api.cp_desc), vp, vp, ctypes.c_double, vp, vp]

    def ptrs(*vals):
        arr = (ctypes.c_void_p * len(vals))()
        for k, v in enumerate(vals):
            arr[k] = v
        return arr

    def call(dims, R, lam=0.5, A=None, W=None, Q=None):
        d = api.make_desc(dims, R, torch.float64)
        n = len(dims)
        A = A if A is not None else ptrs(*[0x1000 + 0x100 * k for k in range(n)])
        W = W if W is not None else ptrs(*[0x2000 + 0x100 * k for k in range(n)])
        Q = Q if Q is not None else ptrs(*[0x3000 + 0x100 * k for k in range(n)])
        return f(ctypes.byref(d), A, W, lam, Q, None)

    assert f(None, None, None, 0.0, None, None) == api.CP_ERR_ARG
    assert call((5,), 2) == api.CP_ERR_ARG                       # order 1
    assert call((5, 6, 7), 0) == api.CP_ERR_ARG                  # rank 0
    assert call((5, 0, 7), 2) == api.CP_ERR_ARG                  # empty mode
    assert call((5, 6, 7), 2, A=ptrs(0x1000, 0, 0x1200)) == api.CP_ERR_ARG           # null factor
    assert call((5, 6, 7), 2, Q=ptrs(0x3000, 0x1100, 0x3200)) == api.CP_ERR_ARG      # Q aliases A
    assert call((5, 6, 7), 2, Q=ptrs(0x3000, 0x2000, 0x3200)) == api.CP_ERR_ARG      # Q aliases W
    assert call((5, 6, 7), 2, Q=ptrs(0x3000, 0x3000, 0x3200)) == api.CP_ERR_ARG      # Q[0] is Q[1]
    assert call((5, 6, 7), 2, lam=-1.0) == api.CP_ERR_ARG
    assert call((5, 6, 7), 2, lam=float("nan")) == api.CP_ERR_ARG
    assert call((5, 6, 7), 2, lam=float("inf")) == api.CP_ERR_ARG
    assert call((3,) * (max_order + 1), 2) == api.CP_ERR_UNSUPPORTED
    assert call((5, 6, 7), max_rank + 1) == api.CP_ERR_UNSUPPORTED


def test_struct_layouts_match_header():
    """The ctypes mirrors of the header structs have the C sizes (checked with gcc)."""
    import subprocess
    import tempfile

    from paper_1910_12331_gb300 import api

    prog = r"""
#include <stdio.h>
#include "cpgn.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu %zu\n", sizeof(cp_desc), sizeof(cp_gn_params), sizeof(cp_gn_stats),
         sizeof(cp_solve_opts), sizeof(cp_solve_result), sizeof(cp_batch_problem), sizeof(cp_batch_result));
  return 0;
}
"""
    with tempfile.TemporaryDirectory() as d:
        src, exe = os.path.join(d, "s.c"), os.path.join(d, "s")
        open(src, "w").write(prog)
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), src, "-o", exe], check=True)
        sizes = list(map(int, subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()))
    mine = [ctypes.sizeof(c) for c in (api.cp_desc, api.cp_gn_params, api.cp_gn_stats, api.cp_solve_opts,
                                       api.cp_solve_result, api.cp_batch_problem, api.cp_batch_result)]
    assert sizes == mine


def test_struct_field_offsets_match_header():
    """Every field of every ctypes mirror sits at the C offset of the header's
    field of the same name (offsetof, compiled with gcc)."""
    import subprocess
    import tempfile

    from paper_1910_12331_gb300 import api

    structs = (api.cp_desc, api.cp_gn_params, api.cp_gn_stats, api.cp_solve_opts, api.cp_solve_result,
               api.cp_batch_problem, api.cp_batch_result)
    lines = [f'  printf("%zu\\n", offsetof({c.__name__}, {f}));' for c in structs for f, _ in c._fields_]
    prog = "#include <stdio.h>\n#include <stddef.h>\n#include \"cpgn.h\"\nint main(void) {\n" + \
        "\n".join(lines) + "\n  return 0;\n}\n"
    with tempfile.TemporaryDirectory() as d:
        src, exe = os.path.join(d, "o.c"), os.path.join(d, "o")
        open(src, "w").write(prog)
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), src, "-o", exe], check=True)
        offs = list(map(int, subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()))
    mine = [getattr(c, f).offset for c in structs for f, _ in c._fields_]
    names = [f"{c.__name__}.{f}" for c in structs for f, _ in c._fields_]
    assert [n for n, a, b in zip(names, offs, mine) if a != b] == []
    assert len(offs) == len(mine)


def test_split_cache_version_stamps():
    """The binding's x_version stamps (the library caches the bf16 split of X
    by address, size, dtype and stamp): same tensor unchanged -> same stamp;
    in-place change, explicit bump, or another tensor at a freed address ->
    a stamp never used before."""
    import gc

    import torch

    from paper_1910_12331_gb300 import api

    xv = api.XVersions()
    X = torch.zeros(64, 64)
    s1 = xv.stamp(X)
    assert xv.stamp(X) == s1
    X.mul_(2.0)                      # in place through torch
    s2 = xv.stamp(X)
    assert s2 != s1 and xv.stamp(X) == s2
    s3 = xv.bump(X)                  # a write torch cannot see
    assert s3 not in (s1, s2) and xv.stamp(X) == s3
    Y = torch.ones(64, 64)
    sy = xv.stamp(Y)
    assert sy not in (s1, s2, s3)
    # a new tensor at the freed address of an old one gets a new stamp
    ptr = X.data_ptr()
    del X
    gc.collect()
    used = {s1, s2, s3, sy}
    for _ in range(50):
        Z = torch.empty(64, 64)
        sz = xv.stamp(Z)
        assert sz not in used
        used.add(sz)
        if Z.data_ptr() == ptr:
            break
        del Z
    # a view at the same address is another object: a new stamp (a re-split, never a stale hit)
    W = Y.view(4096)
    assert xv.stamp(W) not in used
    with torch.inference_mode():
        I = torch.zeros(8)
    si = xv.stamp(I)
    assert xv.stamp(I) == si


def test_binding_rejects_bad_outputs_and_devices():
    """The binding checks what the library cannot see: the shape, dtype,
    layout and device of every caller-supplied output (a wrong-sized device
    buffer would be written out of bounds), and that factors sit on X's
    device and X on the handle's."""
    import torch

    from paper_1910_12331_gb300 import api

    class T:  # the attributes the validators read, on a chosen device
        def __init__(self, shape, dev=0, dtype=torch.float64, contiguous=True):
            self.shape, self.dtype, self.is_cuda = tuple(shape), dtype, True
            self.device = torch.device("cuda", dev)
            self._c = contiguous

        def is_contiguous(self):
            return self._c

        def dim(self):
            return len(self.shape)

    shape, R = (5, 6, 7), 3
    ok = [T((s, R)) for s in shape]
    api._check_outputs(ok, shape, R, "G", torch.device("cuda", 0))
    bad_cases = [
        [T((5, R)), T((6, R))],                                          # one missing
        [T((5, R)), T((6, R + 1)), T((7, R))],                           # wrong rank
        [T((5, R)), T((7, R)), T((7, R))],                               # wrong rows
        [T((5, R)), T((6, R), dtype=torch.float32), T((7, R))],          # wrong dtype
        [T((5, R)), T((6, R), contiguous=False), T((7, R))],             # not contiguous
        [T((5, R)), T((6, R), dev=1), T((7, R))],                        # another device
    ]
    for outs in bad_cases:
        with pytest.raises(ValueError):
            api._check_outputs(outs, shape, R, "G", torch.device("cuda", 0))
    X = T(shape)
    X.dtype = torch.float32
    assert api._factors(X, ok) == R
    with pytest.raises(ValueError):
        api._factors(X, [T((5, R)), T((6, R), dev=1), T((7, R))])
    with pytest.raises(ValueError):
        api._factors(X, ok[:2])
    h = object.__new__(api.Handle)  # a handle record without a device context
    h.device, h._xv, h.h = 0, api.XVersions(), None
    with pytest.raises(ValueError):
        h.desc(T(shape, dev=1, dtype=torch.float32), R)
