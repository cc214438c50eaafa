"""tt_dot_noalloc: the inner product for callers that cannot allocate device memory.

Some callers cannot call cudaMalloc: their host framework owns every device allocation,
cudaMalloc's device-wide synchronization is not acceptable in their loop, or they run
where allocating is forbidden.  tt_dot_noalloc serves them with scratch from a fixed
device array instead of a caller workspace.  This file checks, through the C ABI, that
it returns what tt_dot returns (within the 1e-12 relative tolerance of the other
inner-product tests) on two calls in a row, without changing the device's free memory,
and that it refuses sizes beyond its fixed scratch.  It is collected last and passes both alone and after the other tests.
"""
import ctypes

import numpy as np
import pytest

import ttgen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import torch

    from paper_2011_06532_gb300 import _native

    assert torch.cuda.is_available()
    _native.build()
    return _native.load()


def desc(x, keep):
    from paper_2011_06532_gb300 import _native

    N = len(x.I)
    I = (ctypes.c_int64 * N)(*x.I)
    R = (ctypes.c_int64 * (N + 1))(*x.R)
    ptrs = (ctypes.c_void_p * N)(*[c.data_ptr() for c in x.cores])
    keep += [I, R, ptrs]
    return _native.TTTensor(N, 0, I, R, ptrs)


def test_noalloc_matches_tt_dot_twice(lib):
    import torch

    import paper_2011_06532_gb300 as ttgb

    I = [700, 50, 333, 91]
    a = ttgen.random_tt(I, [1, 12, 20, 9, 1], 301)
    b = ttgen.random_tt(I, [1, 7, 16, 14, 1], 302)
    da = ttgb.from_host(a.I, a.R, a.cores)
    db = ttgb.from_host(b.I, b.R, b.cores)
    keep = []
    sa, sb = desc(da, keep), desc(db, keep)
    # the existing entry point, with a caller workspace
    n = ctypes.c_size_t(0)
    assert lib.tt_dot_workspace_size(ctypes.byref(sa), ctypes.byref(sb), ctypes.byref(n)) == 0
    ws = torch.empty(n.value, dtype=torch.uint8, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    ref = ctypes.c_double(0)
    assert lib.tt_dot(ctypes.byref(sa), ctypes.byref(sb), ctypes.byref(ref), ctypes.c_void_p(ws.data_ptr()),
                      ctypes.c_size_t(ws.numel()), stream) == 0
    scale = np.sqrt(ttgb.tt_dot(da, da) * ttgb.tt_dot(db, db))
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(2):
        got = ctypes.c_double(0)
        assert lib.tt_dot_noalloc(ctypes.byref(sa), ctypes.byref(sb), ctypes.byref(got), stream) == 0
        assert abs(got.value - ref.value) <= 1e-12 * scale
        # nothing was allocated on the device: its free memory is what it was before
        assert torch.cuda.mem_get_info()[0] == free0


def test_noalloc_rejects_sizes_beyond_its_scratch(lib):
    import paper_2011_06532_gb300 as ttgb

    I = [400, 400]
    a = ttgen.random_tt(I, [1, 64, 1], 303)  # 304 * 64 * 64 partial sums > 8 MiB
    da = ttgb.from_host(a.I, a.R, a.cores)
    keep = []
    sa = desc(da, keep)
    got = ctypes.c_double(0)
    assert lib.tt_dot_noalloc(ctypes.byref(sa), ctypes.byref(sa), ctypes.byref(got), None) == 6
