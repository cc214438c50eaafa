"""GPU parity of the batched form (a10): every member of an uneven batch against its own
oracle rounding (ranks identical; rel. error <= 1e-12 in FP64, <= 1e-6 in fp32x2), and the
asynchronous batch captured in a CUDA graph and replayed gives bit-identical results.
Members follow the batched recipe (N, I_n, r uniform; X = Y + Y' with formal ranks 2r) at
reduced mode sizes so the oracle finishes in seconds; full-size members of the 512-tensor
recipe are checked against the FP64 GPU path (oracle-verified in test_gpu_round.py)."""
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


def uneven_batch(count, seed, max_I=256):
    out = []
    for t in range(count):
        u = ttgen.uniforms(22, seed, 1 << 21, t)
        N = ttgen.uniform_int(u[0], 2, 8)
        r = ttgen.uniform_int(u[1], 2, 12)
        I = [ttgen.uniform_int(u[2 + n], 8, max_I) for n in range(N)]
        Y, Yp = ttgen.perturbed_pair(I, r, seed + 31 * t, stream=t)
        out.append((Y, Yp))
    return out


def down(y) -> TT:
    import paper_2011_06532_gb300 as ttgb

    return TT(list(y.I), list(y.R), ttgb.to_host(y))


@pytest.mark.parametrize("prec,dtype,tol", [("fp64", "f64", 1e-12), ("fp32x2", "f32", 1e-6)])
def test_uneven_batch_matches_oracle(gpu, orc, prec, dtype, tol):
    import torch

    tdt = torch.float64 if dtype == "f64" else torch.float32
    pairs = uneven_batch(40, 2011065404)
    Xs = [orc.tt_add(Y, Yp) for Y, Yp in pairs]
    dxs = [gpu.from_host(X.I, X.R, X.cores, dtype=tdt) for X in Xs]
    outs = gpu.tt_round_batched(dxs, [1e-6] * len(dxs), precision=prec)
    for X, o in zip(Xs, outs):
        ref, _ = orc.tt_round(X, 1e-6)
        got = down(o)
        assert got.R == ref.R
        assert orc.rel_err(got, ref) <= tol


def test_graph_captured_batch_replays_identically(gpu):
    import torch

    pairs = uneven_batch(24, 2011065405)
    dxs = []
    for Y, Yp in pairs:
        dxs.append(gpu.tt_add(gpu.from_host(Y.I, Y.R, Y.cores, dtype=torch.float32),
                              gpu.from_host(Yp.I, Yp.R, Yp.cores, dtype=torch.float32)))
    ref = gpu.Batch(dxs, [1e-6] * len(dxs), "fp32x2").run()
    b = gpu.Batch(dxs, [1e-6] * len(dxs), "fp32x2")
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        b.enqueue(s)  # first use creates the slot streams outside the capture
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        b.enqueue(s)
    for _ in range(2):
        for o in b.outs:
            for c in o:
                c.zero_()
        b.ranks_dev.zero_()
        g.replay()
        torch.cuda.synchronize()
        got = b.outputs()
        for r, o in zip(ref, got):
            assert r.R == o.R
            for cr, co in zip(r.cores, o.cores):
                assert torch.equal(cr, co)


def test_full_size_members_against_fp64_path(gpu):
    import torch

    def neg_first(x):
        c = [t.clone() for t in x.cores]
        c[0] = -c[0]
        return gpu.DeviceTT(list(x.I), list(x.R), c)

    shapes = ttgen.batched_shapes()
    sizes = [sum(I) * r * r for I, r in shapes]
    picks = [0, 1, 2, int(np.argmin(sizes)), int(np.argmax(sizes))]
    xs64, xs32 = [], []
    for t in picks:
        (Y, Yp), eps = ttgen.batched_member(t)
        x = gpu.tt_add(gpu.from_host(Y.I, Y.R, Y.cores), gpu.from_host(Yp.I, Yp.R, Yp.cores))
        xs64.append(x)
        xs32.append(gpu.DeviceTT(list(x.I), list(x.R), [c.float() for c in x.cores]))
    out64 = gpu.tt_round_batched(xs64, [1e-6] * len(picks), precision="fp64")
    out32 = gpu.tt_round_batched(xs32, [1e-6] * len(picks), precision="fp32x2")
    for t, a, b in zip(picks, out64, out32):
        assert a.R == b.R, t
        # the Y + Y' construction comes back to the rank of Y (capped by the mode sizes)
        _, r = shapes[t]
        assert max(a.R) <= r
        d = gpu.tt_add(gpu.DeviceTT(list(b.I), list(b.R), [c.double() for c in b.cores]), neg_first(a))
        assert gpu.tt_norm(d) <= 1e-6 * gpu.tt_norm(a)
