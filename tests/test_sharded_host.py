"""Host side of sharded rounding, without a GPU.

* tt_shard_range: the slabs of the 1 x P x 1 distribution (Sec. 3.1) tile every mode, in
  rank order, with lengths that differ by at most one.
* Two gloo ranks (one process each) call tt_round_sharded through the C ABI with the
  torch.distributed all-gather adapter.  Their cores are ordinary host memory, which no
  kernel may read, so every shard fails its own checks: the library must still make the
  first all-gather (the handshake) and nothing after it, every shard must send its status
  and the digest of the arguments all shards share (equal digests for equal arguments,
  different ones when a shard passes another eps), and every shard must return the same
  status.  An all-gather that raises returns TT_ERR_COMM on every shard.
* The sharded workspace query (host planning) checks the shard's range and sizes the
  shard-level trees on top of the local plan.
"""
import ctypes
import json
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
I_GLOBAL = [10, 7, 9]
RANKS = [1, 3, 4, 1]


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_shard_ranges_tile_every_mode():
    import paper_2011_06532_gb300 as ttgb

    for I in (1, 2, 7, 10, 31, 4099, 65536):
        for world in range(1, min(I, 9) + 1):
            ranges = [ttgb.shard_range(I, world, r) for r in range(world)]
            assert ranges[0][0] == 0 and ranges[-1][1] == I
            assert all(ranges[r][1] == ranges[r + 1][0] for r in range(world - 1))
            lens = [e - b for b, e in ranges]
            assert min(lens) >= 1 and max(lens) - min(lens) <= 1
    for bad in ((5, 0, 0), (5, 6, 0), (5, 2, 2), (5, 2, -1), (5000, 1025, 0)):
        with pytest.raises(ttgb.TTError) as e:
            ttgb.shard_range(*bad)
        assert e.value.status == 1


def _desc(I, R, arrays):
    from paper_2011_06532_gb300 import _native

    N = len(I)
    Ia = (ctypes.c_int64 * N)(*I)
    Ra = (ctypes.c_int64 * (N + 1))(*R)
    ptrs = (ctypes.c_void_p * N)(*[a.ctypes.data for a in arrays])
    d = _native.TTTensor(N, 0, Ia, Ra, ptrs)
    d._keep = (Ia, Ra, ptrs, arrays)
    return d


def _headers(recv, world):
    per = len(recv) // world
    out = []
    for p in range(world):
        chunk = recv[p * per: p * per + 16].tobytes()
        status, seq = np.frombuffer(chunk[:8], dtype=np.int32)
        check = int(np.frombuffer(chunk[8:16], dtype=np.uint64)[0])
        out.append({"status": int(status), "seq": int(seq), "check": check, "bytes": per})
    return out


def _rank_main(rank, world, port, outdir, eps_by_rank, raise_in_gather):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import paper_2011_06532_gb300 as ttgb
    from paper_2011_06532_gb300 import _native

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    lib = _native.load()
    I = [e - b for b, e in (ttgb.shard_range(i, world, rank) for i in I_GLOBAL)]
    x = _desc(I, RANKS, [np.zeros(RANKS[n] * I[n] * RANKS[n + 1]) for n in range(len(I))])
    out = _desc(I, [1] * len(RANKS), [np.zeros(RANKS[n] * I[n] * RANKS[n + 1]) for n in range(len(I))])
    seen = []
    inner = ttgb.dist_allgather()

    def fn(send, recv):
        inner(send, recv)
        seen.append(recv.copy())
        if raise_in_gather:
            raise RuntimeError("planted all-gather failure")

    g = ttgb._Gather(fn, world)
    Ig = (ctypes.c_int64 * len(I_GLOBAL))(*I_GLOBAL)
    sh = _native.TTShard(rank, world, Ig, g.c, None)
    st = lib.tt_round_sharded(ctypes.byref(x), eps_by_rank[rank], 0, ctypes.byref(sh), ctypes.byref(out), None, 0,
                              None)
    dist.barrier()
    with open(os.path.join(outdir, f"r{rank}.json"), "w") as f:
        json.dump({"status": st, "calls": len(seen), "headers": [_headers(r, world) for r in seen],
                   "raised": g.error is not None}, f)
    dist.destroy_process_group()


def _run(tmp_path, eps_by_rank, raise_in_gather=False):
    import torch.multiprocessing as mp

    mp.spawn(_rank_main, args=(2, free_port(), str(tmp_path), eps_by_rank, raise_in_gather), nprocs=2, join=True)
    return [json.load(open(os.path.join(tmp_path, f"r{r}.json"))) for r in range(2)]


def test_handshake_agrees_on_status_and_digest(tmp_path):
    res = _run(tmp_path, [1e-6, 1e-6])
    for r in res:
        assert r["status"] == 1 and r["calls"] == 1
        hs = r["headers"][0]
        assert [h["status"] for h in hs] == [1, 1] and [h["seq"] for h in hs] == [0, 0]
        assert hs[0]["bytes"] == 16  # the handshake carries the header only
        assert hs[0]["check"] == hs[1]["check"] != 0
    assert res[0]["headers"] == res[1]["headers"]


def test_handshake_digest_differs_with_eps(tmp_path):
    res = _run(tmp_path, [1e-6, 1e-5])
    for r in res:
        assert r["status"] == 1 and r["calls"] == 1
        hs = r["headers"][0]
        assert hs[0]["check"] != hs[1]["check"]


def test_failed_all_gather_is_comm_error_on_every_shard(tmp_path):
    res = _run(tmp_path, [1e-6, 1e-6], raise_in_gather=True)
    for r in res:
        assert r["status"] == 7 and r["calls"] == 1 and r["raised"]


def test_sharded_workspace_query_on_the_host():
    # planning is host logic: the query answers without a GPU, rejects a tensor that is not
    # this shard's range, and a sharded plan needs at least what the local slab's own
    # rounding does (the local leaves and trees) plus the shard-level trees
    import paper_2011_06532_gb300 as ttgb
    from paper_2011_06532_gb300 import _native

    lib = _native.load()
    I_glob, R, world = [4099, 300, 4099], [1, 16, 24, 1], 3
    Ig = (ctypes.c_int64 * 3)(*I_glob)
    cb = _native.ALLGATHER_FN(lambda s, r, n, c: 1)
    for rank in range(world):
        I = [e - b for b, e in (ttgb.shard_range(i, world, rank) for i in I_glob)]
        x = _desc(I, R, [np.zeros(1)] * 3)
        sh = _native.TTShard(rank, world, Ig, cb, None)
        n_sh, n_loc = ctypes.c_size_t(0), ctypes.c_size_t(0)
        assert lib.tt_round_sharded_workspace_size(ctypes.byref(x), 1, ctypes.byref(sh), ctypes.byref(n_sh)) == 0
        assert lib.tt_round_workspace_size(ctypes.byref(x), 1, ctypes.byref(n_loc)) == 0
        assert n_sh.value > n_loc.value > 0
        wrong = _desc([i + 1 for i in I], R, [np.zeros(1)] * 3)
        assert lib.tt_round_sharded_workspace_size(ctypes.byref(wrong), 1, ctypes.byref(sh), ctypes.byref(n_sh)) == 1
    bad = _native.TTShard(world, world, Ig, cb, None)  # rank out of range
    assert lib.tt_round_sharded_workspace_size(ctypes.byref(x), 1, ctypes.byref(bad), ctypes.byref(n_sh)) == 1


def _adapter_main(rank, world, port, outdir):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import paper_2011_06532_gb300 as ttgb

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    fn = ttgb.dist_allgather()
    send = (np.arange(24, dtype=np.uint8) * (rank + 1)).astype(np.uint8)
    recv = np.zeros(24 * world, dtype=np.uint8)
    fn(send, recv)
    with open(os.path.join(outdir, f"a{rank}.json"), "w") as f:
        json.dump(recv.tolist(), f)
    dist.destroy_process_group()


def test_dist_allgather_orders_payloads_by_rank(tmp_path):
    # the adapter the sharded rounding calls: every rank receives every payload, rank p's
    # at offset p * bytes
    import torch.multiprocessing as mp

    world = 3
    mp.spawn(_adapter_main, args=(world, free_port(), str(tmp_path)), nprocs=world, join=True)
    want = np.concatenate([(np.arange(24, dtype=np.uint8) * (p + 1)).astype(np.uint8) for p in range(world)])
    for r in range(world):
        got = np.array(json.load(open(os.path.join(tmp_path, f"a{r}.json"))), dtype=np.uint8)
        assert np.array_equal(got, want)
