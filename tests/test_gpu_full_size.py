"""GPU parity against the FP64 CPU oracle at the sizes that are benchmarked.

Every case compares the CUDA path (through the C ABI, in the launch configuration the
benchmark times: default plans, the library's own tt_add forming the sums) with an
oracle rounding of the same seeded input, computed in spawned worker processes (see
oracle_pool.py; one large-mode oracle rounding is ~1.2e11 flops of single-threaded C).
Ranks must be identical element by element; the error ||Y_gpu - Y_orc|| / ||Y_orc|| is
measured by the oracle's orthonormalization norm of the difference TT (Sec. 3.2.4) and
must stay within 1e-12 in FP64 and 1e-6 in the FP32-storage forms (Alg. 2, Ensure
clause, with the tolerances of the mixed and batched forms).

  * the large-mode workload at full size: N=10, I_n=65536, formal ranks 32 (4.33 GB), and
    the same tensor split into two shards of 32768 slices per core and rounded by
    tt_round_sharded (two threads of this process, one stream each, exchanging through a
    host all-gather), its slices put back together against the same oracle rounding;
  * the paper's Model 1 (Sec. 4.2, Table 2): N=50, I_n=2000, Y = 2X - X with X of rank
    25 (formal ranks 50), in FP64 at eps=1e-8 and fp32x2 at eps=1e-6;
  * the decaying-spectrum construction at N=50 (formal ranks 64, eps=1e-5) with I_n=1024,
    in fp32x2 and FP64;
  * members 0..15, the largest and the smallest of the full-size 512-tensor batched
    recipe, rounded as one batch in fp32x2 and in FP64.

The FP32-storage inputs are the FP32 roundings of the FP64 tensors the oracle rounds, so
the reported error includes the input quantisation.  Each test runs every precision of its
workload on the GPU first and then submits all its error measurements to the pool at once,
so that they run side by side.
"""
import numpy as np
import pytest

import ttgen
from tests import oracle_pool
from ttgen import TT

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL_MIXED = 1e-6


@pytest.fixture(scope="module")
def gpu():
    import torch

    import paper_2011_06532_gb300 as ttgb

    assert torch.cuda.is_available()
    ttgb.build()
    return ttgb


@pytest.fixture(scope="module")
def pool():
    return oracle_pool.get_pool()


def down(y) -> TT:
    import paper_2011_06532_gb300 as ttgb

    return TT(list(y.I), list(y.R), ttgb.to_host(y))


def release(gpu):
    import torch

    gpu._ws_cache.clear()
    torch.cuda.empty_cache()


def as32(gpu, x):
    return gpu.DeviceTT(list(x.I), list(x.R), [c.float() for c in x.cores])


def test_large_modes_full_size_fp64(gpu, pool):
    Y, Yp = oracle_pool.large_modes_input()
    X = gpu.tt_add(gpu.from_host(Y.I, Y.R, Y.cores), gpu.from_host(Yp.I, Yp.R, Yp.cores))
    del Y, Yp
    got = down(gpu.tt_round(X, oracle_pool.LARGE_MODES["eps"]))
    del X
    release(gpu)
    ref = pool.get("large_modes")
    assert got.R == ref.R == [1] + [16] * 9 + [1], (got.R, ref.R)
    err = pool.rel_err_async(got, ref).get(1500)
    assert err <= TOL64, err


def test_large_modes_full_size_sharded(gpu, pool):
    import threading

    import torch

    from tests.test_gpu_sharded import HostGather, gather_slices

    Y, Yp = oracle_pool.large_modes_input()
    X = gpu.tt_add(gpu.from_host(Y.I, Y.R, Y.cores), gpu.from_host(Yp.I, Yp.R, Yp.cores))
    del Y, Yp
    world, I_global, R = 2, list(X.I), list(X.R)
    shards = []
    for r in range(world):
        cores, I = [], []
        for n in range(X.N):
            b, e = gpu.shard_range(X.I[n], world, r)
            # core n as (R[n+1], I[n], R[n]) in C order holds entry (a, i, b) at [b, i, a]
            cores.append(X.cores[n].view(X.R[n + 1], X.I[n], X.R[n])[:, b:e, :].contiguous().view(-1))
            I.append(e - b)
        shards.append(gpu.DeviceTT(I, R, cores))
    del X
    torch.cuda.synchronize()
    g = HostGather(world)
    out = [None] * world

    def work(r):
        try:
            s = torch.cuda.Stream()
            y = gpu.tt_round_sharded(shards[r], oracle_pool.LARGE_MODES["eps"], I_global, r, world, g.fn(r),
                                     stream=s)
            s.synchronize()
            out[r] = TT(list(y.I), list(y.R), gpu.to_host(y))
        except gpu.TTError as e:
            out[r] = e
        except BaseException as e:  # noqa: BLE001 -- reported below
            out[r] = e
            g.bar.abort()

    threads = [threading.Thread(target=work, args=(r,)) for r in range(world)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    del shards
    release(gpu)
    for p in out:
        if isinstance(p, BaseException):
            raise p
    assert g.calls == [2 * len(I_global)] * world
    got = gather_slices(out, I_global)
    ref = pool.get("large_modes")
    assert got.R == ref.R == [1] + [16] * 9 + [1], (got.R, ref.R)
    err = pool.rel_err_async(got, ref).get(1500)
    assert err <= TOL64, err


def test_paper_model1(gpu, pool):
    import torch

    X = oracle_pool.model1_x()
    runs = []
    for prec, eps, tol, dt in (("fp64", 1e-8, TOL64, torch.float64), ("fp32x2", 1e-6, TOL_MIXED, torch.float32)):
        dX = gpu.from_host(X.I, X.R, X.cores, dtype=dt)
        two = gpu.DeviceTT(list(X.I), list(X.R), [2.0 * dX.cores[0]] + dX.cores[1:])
        neg = gpu.DeviceTT(list(X.I), list(X.R), [-dX.cores[0]] + dX.cores[1:])
        Y = gpu.tt_add(two, neg)  # Y = 2X - X (Sec. 4.2), formal ranks 50
        runs.append((prec, eps, tol, down(gpu.tt_round(Y, eps, precision=prec))))
        del dX, two, neg, Y
        release(gpu)
    pending = []
    for prec, eps, tol, got in runs:
        ref = pool.get("model1_%g" % eps)
        assert got.R == ref.R == ttgen.uniform_ranks(oracle_pool.MODEL1["N"], oracle_pool.MODEL1["r"]), (prec, got.R)
        pending.append((prec, tol, pool.rel_err_async(got, ref)))
    for prec, tol, p in pending:
        err = p.get(1500)
        assert err <= tol, (prec, err)


def test_decaying_N50(gpu, pool):
    terms = oracle_pool.decaying_terms()
    X = gpu.from_host(terms[0].I, terms[0].R, terms[0].cores)
    for T in terms[1:]:
        X = gpu.tt_add(X, gpu.from_host(T.I, T.R, T.cores))
    del terms
    runs = []
    for prec, tol in (("fp32x2", TOL_MIXED), ("fp64", TOL64)):
        x = X if prec == "fp64" else as32(gpu, X)
        runs.append((prec, tol, down(gpu.tt_round(x, oracle_pool.DECAYING["eps"], precision=prec))))
        del x
    del X
    release(gpu)
    ref = pool.get("decaying")
    assert max(ref.R) < 64  # the threshold cuts the decaying spectra (to ranks near 48)
    pending = []
    for prec, tol, got in runs:
        assert got.R == ref.R, (prec, got.R, ref.R)
        pending.append((prec, tol, pool.rel_err_async(got, ref)))
    for prec, tol, p in pending:
        err = p.get(1500)
        assert err <= tol, (prec, err)


def test_batched_recipe_subset_full_size(gpu, pool):
    import torch

    members = oracle_pool.batched_subset()
    xs = []
    for t in members:
        (Y, Yp), _ = ttgen.batched_member(t)
        xs.append(gpu.tt_add(gpu.from_host(Y.I, Y.R, Y.cores), gpu.from_host(Yp.I, Yp.R, Yp.cores)))
        del Y, Yp
    torch.cuda.synchronize()
    gots = {}
    for prec in ("fp32x2", "fp64"):
        batch = xs if prec == "fp64" else [as32(gpu, x) for x in xs]
        outs = gpu.tt_round_batched(batch, [1e-6] * len(batch), precision=prec)
        gots[prec] = [down(o) for o in outs]
        del batch, outs
        release(gpu)
    del xs
    release(gpu)
    pending = []
    for i, t in enumerate(members):
        ref = pool.get("batched_%d" % t)
        for prec, tol in (("fp32x2", TOL_MIXED), ("fp64", TOL64)):
            got = gots[prec][i]
            assert got.R == ref.R, (t, prec, got.R, ref.R)
            pending.append((t, prec, tol, pool.rel_err_async(got, ref)))
    bad = {}
    for t, prec, tol, p in pending:
        e = p.get(1500)
        if not e <= tol:
            bad[(t, prec)] = e
    assert not bad, bad
