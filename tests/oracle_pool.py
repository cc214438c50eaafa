"""A pool of oracle processes for the full-size parity tests.

The FP64 oracle is single-threaded C; at the benchmarked sizes one rounding takes a
minute or more (the large-mode workload: ~1.2e11 flops).  The full-size tests therefore
submit their oracle roundings, and the error measurements against them, to worker
processes started with the "spawn" method (a forked child of a process that has used
CUDA can hang).  Workers import only numpy, ttgen and the oracle.

Jobs are submitted when test collection finishes (see conftest.py), so they run while
the other GPU tests do; the tests collect the results by name.
"""
from __future__ import annotations

import multiprocessing
import os
from typing import Dict, List, Sequence, Tuple

import numpy as np

# --------------------------------------------------------------------------------------
# workloads (components drawn by ttgen, arithmetic by the oracle)
# --------------------------------------------------------------------------------------

LARGE_MODES = dict(I=65536, N=10, r=16, seed=2011065302, eps=1e-8)
MODEL1 = dict(I=2000, N=50, r=25, seed=2011065306)
DECAYING = dict(I=1024, N=50, seed=2011065303, eps=1e-5)


def batched_subset() -> List[int]:
    """Members 0..15 of the 512-tensor batched recipe plus its largest and smallest."""
    import ttgen

    def size(I, r):
        R = [1] + [2 * r] * (len(I) - 1) + [1]
        return sum(R[n] * I[n] * R[n + 1] for n in range(len(I)))

    sizes = [size(I, r) for I, r in ttgen.batched_shapes()]
    out = list(range(16))
    for t in (int(np.argmax(sizes)), int(np.argmin(sizes))):
        if t not in out:
            out.append(t)
    return out


def large_modes_input():
    """X = Y + Y' of the large-mode workload as components (Y, Y')."""
    import ttgen

    return ttgen.perturbed_pair([LARGE_MODES["I"]] * LARGE_MODES["N"], LARGE_MODES["r"], LARGE_MODES["seed"])


def model1_x():
    """The random rank-25 TT X of the paper's Model 1 (Y = 2X - X is formed by each side)."""
    import ttgen

    N, I, r = MODEL1["N"], MODEL1["I"], MODEL1["r"]
    return ttgen.random_tt([I] * N, ttgen.uniform_ranks(N, r), MODEL1["seed"])


def decaying_terms():
    import ttgen

    return ttgen.decaying_terms(DECAYING["N"], DECAYING["I"], DECAYING["seed"])


# --------------------------------------------------------------------------------------
# jobs (run in the workers)
# --------------------------------------------------------------------------------------

def _as_tuple(x) -> Tuple[list, list, list]:
    return (list(x.I), list(x.R), x.cores)


def job_large_modes():
    import oracle

    Y, Yp = large_modes_input()
    X = oracle.tt_add(Y, Yp)
    del Y, Yp
    ref, _ = oracle.tt_round(X, LARGE_MODES["eps"])
    return _as_tuple(ref)


def job_model1(eps: float):
    import oracle

    X = model1_x()
    Y = oracle.tt_add(oracle.scale_first(X, 2.0), oracle.scale_first(X, -1.0))
    del X
    ref, _ = oracle.tt_round(Y, eps)
    return _as_tuple(ref)


def job_decaying():
    import oracle

    terms = decaying_terms()
    X = terms[0]
    for T in terms[1:]:
        X = oracle.tt_add(X, T)
    del terms
    ref, _ = oracle.tt_round(X, DECAYING["eps"])
    return _as_tuple(ref)


def job_batched_member(t: int):
    import oracle
    import ttgen

    (Y, Yp), eps = ttgen.batched_member(t)
    X = oracle.tt_add(Y, Yp)
    del Y, Yp
    ref, _ = oracle.tt_round(X, eps)
    return _as_tuple(ref)


def job_rel_err(got: Tuple[list, list, list], ref: Tuple[list, list, list]) -> float:
    import oracle
    from ttgen import TT

    return oracle.rel_err(TT(*got), TT(*ref))


def _job_plan() -> Dict[str, tuple]:
    """Every oracle rounding the full-size tests need, largest first."""
    import ttgen

    jobs = {}
    shapes = ttgen.batched_shapes()

    def member_cost(t):
        I, r = shapes[t]
        return sum(i for i in I) * (2 * r) ** 3

    members = sorted(batched_subset(), key=member_cost, reverse=True)
    # the largest members and the N=50 workloads dominate: start them first
    order = [("decaying", (job_decaying, ())), ("batched_%d" % members[0], (job_batched_member, (members[0],))),
             ("large_modes", (job_large_modes, ())), ("model1_1e-08", (job_model1, (1e-8,))),
             ("model1_1e-06", (job_model1, (1e-6,)))]
    order += [("batched_%d" % t, (job_batched_member, (t,))) for t in members[1:]]
    for name, spec in order:
        jobs[name] = spec
    return jobs


# --------------------------------------------------------------------------------------
# pool handle used by the tests
# --------------------------------------------------------------------------------------

class OraclePool:
    def __init__(self, workers: int):
        import oracle

        oracle.build()  # compile once here, not in every worker
        ctx = multiprocessing.get_context("spawn")
        self.pool = ctx.Pool(workers)
        self.results = {}

    def submit_plan(self):
        for name, (fn, args) in _job_plan().items():
            self.results[name] = self.pool.apply_async(fn, args)

    def get(self, name: str, timeout: float = 1500.0):
        from ttgen import TT

        return TT(*self.results[name].get(timeout))

    def rel_err_async(self, got, ref):
        return self.pool.apply_async(job_rel_err, (_as_tuple(got), _as_tuple(ref)))

    def close(self):
        self.pool.terminate()
        self.pool.join()


def default_workers() -> int:
    # leave cores to the test process, which draws the same inputs for the GPU meanwhile
    n = os.cpu_count() or 2
    return max(1, min(12, n - 4))


_POOL = None


def start() -> OraclePool:
    global _POOL
    if _POOL is None:
        _POOL = OraclePool(default_workers())
        _POOL.submit_plan()
    return _POOL


def get_pool() -> OraclePool:
    return start()


def stop() -> None:
    global _POOL
    if _POOL is not None:
        _POOL.close()
        _POOL = None


def names(seq: Sequence[int]) -> List[str]:
    return ["batched_%d" % t for t in seq]
