"""GPU parity of sharded rounding: one tensor distributed over W shards, each owning a
contiguous range of the slices of every core (the 1 x P x 1 distribution of Sec. 3.1), each
tall-skinny QR of Alg. 6 reduced across the shards by an all-gather of the shards' triangular
factors and a tree that every shard factors alike (TSQR, Sec. 3.3).

The shards run as threads of this process on the one GPU, each on its own CUDA stream,
exchanging through a host all-gather (a barrier between the threads): the library
synchronizes its stream before every all-gather, so no kernel ever waits on another.  The
shards' result slices, put back together, must have the oracle's ranks element by element
and lie within 1e-12 (FP64) or 1e-6 (fp32x2) of the oracle's rounding of the whole tensor;
every shard must report the same ranks and make the same 2N all-gathers.
"""
import threading

import numpy as np
import pytest

import ttgen
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


class HostGather:
    """All-gather between the shard threads: every thread deposits its payload, waits for
    the others, copies all of them in rank order, and waits again before the next round."""

    def __init__(self, world: int):
        self.world = world
        self.parts = [None] * world
        self.calls = [0] * world
        self.bar = threading.Barrier(world, timeout=300)

    def fn(self, rank: int):
        def f(send, recv):
            self.calls[rank] += 1
            self.parts[rank] = send.copy()
            self.bar.wait()
            recv[:] = np.concatenate(self.parts)
            self.bar.wait()

        return f


def shard_of(gpu, x: TT, world: int, rank: int) -> TT:
    """Slices shard_range(I_n, world, rank) of every core of x."""
    cores, I = [], []
    for n in range(x.N):
        b, e = gpu.shard_range(x.I[n], world, rank)
        cores.append(np.asfortranarray(x.core3(n)[:, b:e, :]).ravel(order="F"))
        I.append(e - b)
    return TT(I, list(x.R), cores)


def gather_slices(parts, I) -> TT:
    """The whole tensor from its shards' result slices (ranks equal on every shard)."""
    R = parts[0].R
    cores = []
    for n in range(len(I)):
        c = np.concatenate([p.core3(n) for p in parts], axis=1)
        cores.append(np.asfortranarray(c).ravel(order="F"))
    return TT(list(I), list(R), cores)


def run_sharded(gpu, x: TT, eps, world, precision="fp64", eps_of=None, edit=None):
    """Rounds x over `world` shard threads; returns (per-shard TT or exception, gather)."""
    import torch

    dt = torch.float64 if precision == "fp64" else torch.float32
    g = HostGather(world)
    out = [None] * world

    def work(r):
        try:
            s = torch.cuda.Stream()
            part = shard_of(gpu, x, world, r)
            if edit is not None:
                edit(r, part)
            with torch.cuda.stream(s):
                xs = gpu.from_host(part.I, part.R, part.cores, dtype=dt)
                y = gpu.tt_round_sharded(xs, eps_of(r) if eps_of else eps, x.I, r, world, g.fn(r),
                                         precision=precision, stream=s)
                s.synchronize()
                out[r] = TT(list(y.I), list(y.R), gpu.to_host(y))
        except gpu.TTError as e:
            out[r] = e  # the library's status: the shards left the all-gathers in step
        except BaseException as e:  # noqa: BLE001 -- compared by the test
            out[r] = e
            g.bar.abort()  # a shard that fails outside the library releases the others

    threads = [threading.Thread(target=work, args=(r,)) for r in range(world)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    return out, g


def check_parity(orc, x: TT, eps, parts, tol, ref=None):
    for p in parts:
        if isinstance(p, BaseException):
            raise p
    assert all(p.R == parts[0].R for p in parts), [p.R for p in parts]
    got = gather_slices(parts, x.I)
    if ref is None:
        ref, _ = orc.tt_round(x, eps)
    assert got.R == ref.R, (got.R, ref.R)
    err = orc.rel_err(got, ref)
    assert err <= tol, err
    return got


def decaying_tt(I, r, seed, rate=0.5):
    x = ttgen.random_tt(I, ttgen.uniform_ranks(len(I), r), seed)
    for n in range(len(I) - 1):
        c = x.core3(n) * (rate ** np.arange(r))[None, None, :]
        x.cores[n] = np.asfortranarray(c).ravel(order="F")
    return x


CASES = {
    # (tensor, eps, world sizes)
    "small_workload": (lambda orc: orc.tt_add(*ttgen.config_small()[0]), 1e-6, (2, 3)),
    "many_tiles": (lambda orc: orc.tt_add(*ttgen.perturbed_pair([4099] * 4, 16, 2011065400)), 1e-8, (2, 4)),
    "decaying": (lambda orc: decaying_tt([300, 257, 411, 190, 64], 12, 131), 1e-4, (3,)),
    "wide_slabs": (lambda orc: ttgen.random_tt([3, 4, 5, 3], [1, 3, 6, 4, 1], 132), 1e-10, (3,)),
    "uneven_ranks": (lambda orc: ttgen.random_tt([600, 700, 500, 400], [1, 48, 64, 40, 1], 133), 1e-10, (2,)),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_sharded_fp64_vs_oracle(gpu, orc, case):
    make, eps, worlds = CASES[case]
    x = make(orc)
    ref, _ = orc.tt_round(x, eps)
    for world in worlds:
        parts, g = run_sharded(gpu, x, eps, world)
        check_parity(orc, x, eps, parts, TOL64, ref)
        assert g.calls == [2 * x.N] * world, g.calls


def test_sharded_fp32x2_vs_oracle(gpu, orc):
    Y, Yp = ttgen.perturbed_pair([4099] * 4, 16, 2011065400)
    X = orc.tt_add(Y, Yp)
    X = TT(list(X.I), list(X.R), [c.astype(np.float32).astype(np.float64) for c in X.cores])
    parts, _ = run_sharded(gpu, X, 1e-6, 3, precision="fp32x2")
    check_parity(orc, X, 1e-6, parts, TOL_MIXED)


def test_one_shard_is_tt_round(gpu, orc):
    X = orc.tt_add(*ttgen.config_small()[0])
    parts, g = run_sharded(gpu, X, 1e-6, 1)
    whole = gpu.tt_round(gpu.from_host(X.I, X.R, X.cores), 1e-6)
    assert parts[0].R == whole.R and g.calls == [0]
    for a, b in zip(parts[0].cores, gpu.to_host(whole)):
        assert np.array_equal(a, b)


def test_nonfinite_slab_fails_on_every_shard(gpu, orc):
    X = orc.tt_add(*ttgen.config_small()[0])

    def poison(r, part):
        if r == 1:
            part.cores[2][5] = np.nan

    parts, g = run_sharded(gpu, X, 1e-6, 3, edit=poison)
    assert all(isinstance(p, gpu.TTError) and p.status == 4 for p in parts), parts
    assert g.calls == [2 * X.N] * 3, g.calls


def test_disagreeing_arguments_stop_after_the_handshake(gpu, orc):
    X = orc.tt_add(*ttgen.config_small()[0])
    parts, g = run_sharded(gpu, X, 1e-6, 2, eps_of=lambda r: 1e-6 if r == 0 else 1e-5)
    assert all(isinstance(p, gpu.TTError) and p.status == 1 for p in parts), parts
    assert g.calls == [1, 1]
