"""C-ABI checks that need no GPU: the library loads, exports every function that
include/tt.h declares, and rejects invalid arguments before touching the device."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "tt.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(tt_\w+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_2011_06532_gb300 import _native

    _native.build()
    return _native.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for f in ["tt_round", "tt_round_batched", "tt_add", "tt_hadamard", "tt_dot", "tt_norm", "tt_status_string",
              "tt_round_workspace_size", "tt_dot_workspace_size", "tt_norm_workspace_size"]:
        assert f in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), f"{name} not exported"


def make_desc(I, R, dtype=0, null_core=False):
    from paper_2011_06532_gb300 import _native

    N = len(I)
    Ia = (ctypes.c_int64 * N)(*I)
    Ra = (ctypes.c_int64 * (N + 1))(*R)
    ptrs = (ctypes.c_void_p * N)(*[None if null_core else 0x1000 * (k + 1) for k in range(N)])
    d = _native.TTTensor(N, dtype, Ia, Ra, ptrs)
    d._keep = (Ia, Ra, ptrs)
    return d


def test_status_strings(lib):
    for st in [0, 1, 2, 3, 4, 6, 7]:
        assert lib.tt_status_string(st)
    assert lib.tt_status_string(99) == b"unknown status"


@pytest.mark.parametrize("I,R,dtype", [
    ([4, 5], [2, 3, 1], 0),        # R[0] != 1
    ([4, 5], [1, 3, 2], 0),        # R[N] != 1
    ([4, 0], [1, 3, 1], 0),        # zero mode size
    ([4, 5], [1, 0, 1], 0),        # zero rank
    ([4, 5], [1, 3, 1], 7),        # bad dtype
])
def test_invalid_tensors_rejected(lib, I, R, dtype):
    x = make_desc(I, R, dtype)
    out = make_desc(I, [1] * (len(I) + 1), dtype)
    n = ctypes.c_size_t(0)
    assert lib.tt_round_workspace_size(ctypes.byref(x), 0, ctypes.byref(n)) == 1
    assert lib.tt_round(ctypes.byref(x), 1e-6, 0, ctypes.byref(out), None, 0, None) == 1
    assert lib.tt_add(ctypes.byref(x), ctypes.byref(x), ctypes.byref(out), None) == 1


def test_invalid_eps_and_mismatch_rejected(lib):
    x = make_desc([4, 5, 6], [1, 2, 3, 1])
    out = make_desc([4, 5, 6], [1, 1, 1, 1])
    for eps in [-1.0, float("nan"), float("inf")]:
        assert lib.tt_round(ctypes.byref(x), eps, 0, ctypes.byref(out), None, 0, None) == 1
    other = make_desc([4, 5, 7], [1, 2, 3, 1])
    res = ctypes.c_double(0)
    assert lib.tt_dot(ctypes.byref(x), ctypes.byref(other), ctypes.byref(res), None, 0, None) == 1
    assert lib.tt_hadamard(ctypes.byref(x), ctypes.byref(other), ctypes.byref(out), None) == 1
    assert lib.tt_round(ctypes.byref(x), 1e-3, 0, None, None, 0, None) == 1
    nullc = make_desc([4, 5, 6], [1, 2, 3, 1], null_core=True)
    assert lib.tt_round(ctypes.byref(nullc), 1e-3, 0, ctypes.byref(out), None, 0, None) == 1
    # precision must match the element type
    for prec in [2, 3, 7, -1]:
        assert lib.tt_round(ctypes.byref(x), 1e-3, prec, ctypes.byref(out), None, 0, None) == 1
    x32 = make_desc([4, 5, 6], [1, 2, 3, 1], dtype=1)
    out32 = make_desc([4, 5, 6], [1, 1, 1, 1], dtype=1)
    assert lib.tt_round(ctypes.byref(x32), 1e-3, 1, ctypes.byref(out32), None, 0, None) == 1


def test_rank_above_maximum_unsupported(lib):
    x = make_desc([300, 300], [1, 200, 1])
    n = ctypes.c_size_t(0)
    assert lib.tt_round_workspace_size(ctypes.byref(x), 0, ctypes.byref(n)) == 6


def test_missing_library_fails_loudly(tmp_path):
    from paper_2011_06532_gb300 import _native

    with pytest.raises(RuntimeError, match="missing"):
        _native.load(str(tmp_path / "nope.so"))


def test_workspace_size_query_has_no_device_side_effects(lib):
    # the size query is pure host arithmetic over the shapes
    x = make_desc([64, 32, 16], [1, 8, 4, 1])
    n = ctypes.c_size_t(0)
    st = lib.tt_round_workspace_size(ctypes.byref(x), 0, ctypes.byref(n))
    assert st == 0 and n.value > 0
    x32 = make_desc([64, 32, 16], [1, 8, 4, 1], dtype=1)
    for prec in [0, 2, 3]:
        assert lib.tt_round_workspace_size(ctypes.byref(x32), prec, ctypes.byref(n)) == 0 and n.value > 0


def test_plain_c_client(lib, tmp_path):
    """The header compiles as C and the library links into a C program (host-only calls)."""
    import shutil
    import subprocess

    from paper_2011_06532_gb300 import _native

    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    exe = tmp_path / "abi_check"
    libdir = os.path.dirname(_native.LIB)
    r = subprocess.run([cc, "-std=c11", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                        os.path.join(ROOT, "tests", "abi_check.c"), "-o", str(exe), "-L", libdir, "-lttgb",
                        "-Wl,-rpath," + libdir], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stdout + r.stderr

