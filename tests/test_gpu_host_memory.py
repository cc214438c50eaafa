"""Cores in pinned host memory (read and written by the kernels over the host link):
tt_round bit-identical to the rounding of the same cores in device memory, and against the
oracle; inner product and norm likewise; unregistered host memory is refused by every
compute entry point before anything runs."""
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


def test_ops_on_pinned_host_cores(gpu):
    import torch

    A = ttgen.random_tt([300, 200, 300], [1, 5, 4, 1], 2011065601)
    B = ttgen.random_tt([300, 200, 300], [1, 3, 6, 1], 2011065602)
    dA = gpu.from_host(A.I, A.R, A.cores)
    dB = gpu.from_host(B.I, B.R, B.cores)
    hA = gpu.DeviceTT(list(A.I), list(A.R), [c.cpu().pin_memory() for c in dA.cores])
    hB = gpu.DeviceTT(list(B.I), list(B.R), [c.cpu().pin_memory() for c in dB.cores])
    assert gpu.tt_dot(hA, hB) == gpu.tt_dot(dA, dB)
    assert gpu.tt_norm(hA) == gpu.tt_norm(dA)


def test_unregistered_host_memory_refused_everywhere(gpu):
    import torch

    from paper_2011_06532_gb300 import _native

    lib = _native.load()
    I, R = [64, 32], [1, 4, 1]
    plain = [np.zeros(R[n] * I[n] * R[n + 1]) for n in range(2)]
    dev = [torch.zeros(R[n] * I[n] * R[n + 1], dtype=torch.float64, device="cuda") for n in range(2)]

    def desc(ptrs):
        Ia = (ctypes.c_int64 * 2)(*I)
        Ra = (ctypes.c_int64 * 3)(*R)
        pa = (ctypes.c_void_p * 2)(*ptrs)
        d = _native.TTTensor(2, 0, Ia, Ra, pa)
        d._keep = (Ia, Ra, pa)
        return d

    xh, xd = desc([a.ctypes.data for a in plain]), desc([c.data_ptr() for c in dev])
    out = desc([c.data_ptr() for c in dev])
    res = ctypes.c_double(0)
    ws = torch.empty(1 << 20, dtype=torch.uint8, device="cuda")
    wsa = (ctypes.c_void_p(ws.data_ptr()), ctypes.c_size_t(ws.numel()), None)
    assert lib.tt_add(ctypes.byref(xh), ctypes.byref(xd), ctypes.byref(out), None) == 1
    assert lib.tt_hadamard(ctypes.byref(xd), ctypes.byref(xh), ctypes.byref(out), None) == 1
    assert lib.tt_dot(ctypes.byref(xh), ctypes.byref(xd), ctypes.byref(res), *wsa) == 1
    assert lib.tt_dot_noalloc(ctypes.byref(xd), ctypes.byref(xh), ctypes.byref(res), None) == 1
    assert lib.tt_norm(ctypes.byref(xh), ctypes.byref(res), *wsa) == 1
    xs = (_native.TTTensor * 1)(xh)
    outs = (_native.TTTensor * 1)(out)
    eps = (ctypes.c_double * 1)(1e-6)
    assert lib.tt_round_batched(1, xs, eps, 0, outs, *wsa) == 1
    # the same sum on device memory runs (its output has the summed ranks 8)
    big = [torch.zeros(8 * 64, dtype=torch.float64, device="cuda"), torch.zeros(8 * 32, dtype=torch.float64, device="cuda")]
    assert lib.tt_add(ctypes.byref(xd), ctypes.byref(xd), ctypes.byref(desc([c.data_ptr() for c in big])), None) == 0
    torch.cuda.synchronize()

