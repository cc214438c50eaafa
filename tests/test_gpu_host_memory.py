"""tt_round on cores in pinned host memory (read and written by the kernels over the host
link): bit-identical to the rounding of the same cores in device memory, and against the
oracle; unregistered host memory is refused before anything runs."""
import ctypes

import numpy as np
import pytest

import ttgen
from ttgen import TT

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gpu():
    import torch

    import paper_2011_06532_gb300 as ttgb

    assert torch.cuda.is_available()
    ttgb.build()
    return ttgb


@pytest.mark.parametrize("prec,dtype,tol", [("fp64", "f64", 1e-12), ("fp32x2", "f32", 1e-6)])
def test_host_cores_match_device_cores(gpu, orc, prec, dtype, tol):
    import torch

    tdt = torch.float64 if dtype == "f64" else torch.float32
    Y, Yp = ttgen.perturbed_pair([700, 1300, 4099, 900], 6, 2011065600)
    X = orc.tt_add(Y, Yp)
    ref, _ = orc.tt_round(X, 1e-6)
    dX = gpu.from_host(X.I, X.R, X.cores, dtype=tdt)
    hX = gpu.DeviceTT(list(X.I), list(X.R), [c.cpu().pin_memory() for c in dX.cores])
    y_dev = gpu.tt_round(dX, 1e-6, precision=prec)
    y_host = gpu.tt_round(hX, 1e-6, precision=prec)
    assert all(c.device.type == "cpu" and c.is_pinned() for c in y_host.cores)
    assert y_host.R == y_dev.R == ref.R
    for a, b in zip(y_host.cores, y_dev.cores):
        assert torch.equal(a, b.cpu())
    got = TT(list(y_host.I), list(y_host.R), [c.double().numpy() for c in y_host.cores])
    assert orc.rel_err(got, ref) <= tol
    # mixed: host input, device output
    out = [torch.empty(s, dtype=tdt, device="cuda") for s in dX.core_sizes()]
    y_mix = gpu.tt_round(hX, 1e-6, out=out, precision=prec)
    for a, b in zip(y_mix.cores, y_dev.cores):
        assert torch.equal(a, b)


def test_unregistered_host_memory_refused(gpu):
    import torch

    from paper_2011_06532_gb300 import _native

    lib = _native.load()
    I, R = [64, 32], [1, 4, 1]
    plain = [np.zeros(R[n] * I[n] * R[n + 1]) for n in range(2)]  # ordinary (pageable) host arrays
    dev = [torch.zeros(R[n] * I[n] * R[n + 1], dtype=torch.float64, device="cuda") for n in range(2)]

    def desc(ptrs):
        Ia = (ctypes.c_int64 * 2)(*I)
        Ra = (ctypes.c_int64 * 3)(*R)
        pa = (ctypes.c_void_p * 2)(*ptrs)
        d = _native.TTTensor(2, 0, Ia, Ra, pa)
        d._keep = (Ia, Ra, pa)
        return d

    n = ctypes.c_size_t(0)
    xd = desc([c.data_ptr() for c in dev])
    assert lib.tt_round_workspace_size(ctypes.byref(xd), 0, ctypes.byref(n)) == 0
    ws = torch.empty(n.value, dtype=torch.uint8, device="cuda")
    args = (ctypes.c_void_p(ws.data_ptr()), ctypes.c_size_t(ws.numel()), None)
    xh = desc([a.ctypes.data for a in plain])
    od = desc([c.data_ptr() for c in dev])
    assert lib.tt_round(ctypes.byref(xh), 1e-6, 0, ctypes.byref(od), *args) == 1
    oh = desc([a.ctypes.data for a in plain])
    assert lib.tt_round(ctypes.byref(xd), 1e-6, 0, ctypes.byref(oh), *args) == 1
    # the same call on device memory runs
    assert lib.tt_round(ctypes.byref(xd), 1e-6, 0, ctypes.byref(od), *args) == 0
    torch.cuda.synchronize()
