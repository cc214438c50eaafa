#!/usr/bin/env python3
"""TT-rounding throughput on GB300.

Default workload (the plain-FP64 large-mode case): X = Y + Y', Y a random rank-16 TT
with N = 10 modes of size I_n = 65536 (entries N(0,1)/sqrt(I_n R_{n-1})), Y' = 0.5 Y
+ 1e-9 Z taken core-wise, so X has formal ranks 32 (4.33 GB of FP64 cores) and is
rounded at eps = 1e-8 back to ranks 16.  One step = one full TT rounding (both sweeps,
every core) through the C ABI, inputs resident in HBM.  Inputs exceed L2 (129 MB), so
no flush is needed between steps.

  python bench.py [--gpus N --steps K --warmup W]          # this library
  python bench.py --impl reference [...]                    # the FP64 CPU oracle

Multi-GPU (torchrun): every rank rounds its own independent TT (seed + rank), no data
collective; value = all ranks' rounds / max-over-ranks time ("weak" scaling).
Prints one JSON line on rank 0.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "TT-rounds/sec and HBM GB/s, mixed+batched vs plain FP64 on GB300 at rel err ≤1e-6"
N_MODES, I_MODE, RANK, EPS = 10, 65536, 16, 1e-8
SEED = 2011065302
# FP64 pipe of GB300: 152 SMs x 2 FP64 FMA per clock x 2 flop x 2.07 GHz (nominal 1.25 TFLOP/s)
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12


def parse_args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--modes", type=int, default=I_MODE, help="mode size I_n (default: the full 65536)")
    p.add_argument("--variants", type=int, default=1,
                   help="1: also time the mixed-precision and batched forms (N=1 only), 0: skip")
    p.add_argument("--batch", type=int, default=512, help="tensors of the batched recipe timed in the variants")
    p.add_argument("--chunk", type=int, default=64, help="batched-recipe tensors resident at once")
    return p.parse_args()


# --------------------------------------------------------------------------------------
# multi-rank plumbing (one process per GPU; the ranks share no data, only the clock)
# --------------------------------------------------------------------------------------

def rank_seed(rank):
    """Seed of rank r's independent TT (rank 0 rounds the single-GPU workload)."""
    return SEED + 7919 * rank


def max_over_ranks(x, dist, device):
    """Largest x over the ranks (the job's time is its slowest rank's); x itself without dist."""
    if dist is None:
        return float(x)
    import torch

    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(world, steps, ms):
    """Whole-job rounds per second: every rank rounded `steps` TTs in the slowest rank's ms."""
    return world * steps / (ms / 1e3)


def workload_desc(I):
    return (f"plain-FP64 TT rounding, N={N_MODES}, I_n={I}, X = Y + (0.5Y + 1e-9Z) with rank-{RANK} Y, Z "
            f"(formal ranks {2 * RANK}), eps={EPS:g}")


def tt_bytes(I, R, es):
    return sum(R[n] * I[n] * R[n + 1] for n in range(len(I))) * es


# --------------------------------------------------------------------------------------
# flop model (Sec. 3.5: TSQR 2mb^2, TRMM push, TSQR-Apply-Q 4mbc), per kernel class
# --------------------------------------------------------------------------------------

def flops_by_kernel(I, R, L):
    """Algorithmic flops of one rounding, split like the library's kernel classes.
    R: input ranks, L: output ranks."""
    N = len(I)
    K = [1] * (N + 1)
    for n in range(N - 1, 0, -1):
        K[n] = min(R[n], I[n] * K[n + 1])
    f = {"s1_leaf": 0.0, "s2_leaf": 0.0, "s2_out": 0.0}
    for n in range(N - 1, 0, -1):  # sweep 1: QR of H(X_n)^T (m = I K_{n+1} rows, b = R_n) + push of R_{n+1}
        m, b = I[n] * K[n + 1], R[n]
        f["s1_leaf"] += 2.0 * m * b * b + (m * b * R[n + 1] if n < N - 1 else 0.0)
    for n in range(N - 1):  # sweep 2
        if n >= 1:
            f["s2_leaf"] += 4.0 * (I[n] * K[n + 1]) * R[n] * L[n]  # apply Q_n to S^T
        else:
            f["s2_leaf"] += 1.0 * I[0] * K[1] * R[1]  # push into core 0
        f["s2_leaf"] += 2.0 * (L[n] * I[n]) * K[n + 1] ** 2  # QR of V(Y_n)
        f["s2_out"] += 4.0 * (L[n] * I[n]) * K[n + 1] * L[n + 1]  # Q' U_hat
    f["s2_leaf"] += 4.0 * (I[N - 1] * 1) * R[N - 1] * L[N - 1]  # last core
    return f


def source_hash():
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2011_06532_gb300", "csrc")
    for f in sorted(os.listdir(d)):
        h.update(open(os.path.join(d, f), "rb").read())
    return h.hexdigest()[:16]


def read_traffic(kernel):
    """DRAM bytes per launch from the committed ncu summary, if taken on the current sources."""
    path = os.path.join(ROOT, "profiles", f"{kernel}_fp64_large_modes.txt")
    if not os.path.exists(path):
        return None
    vals = {}
    for line in open(path):
        if ":" in line:
            k, v = line.split(":", 1)
            vals[k.strip()] = v.strip()
    if vals.get("source_sha") != source_hash():
        return None
    try:
        return float(vals["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


# --------------------------------------------------------------------------------------
# clocks
# --------------------------------------------------------------------------------------

class ClockSampler:
    def __init__(self, index):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={index}", f"--query-gpu={q}", "--format=csv,noheader",
                                       "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        rows = []
        for line in open(self.f.name):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1].split()[0]), float(parts[2].split()[0]), parts[5:9]))
            except ValueError:
                continue
        os.unlink(self.f.name)
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for _, _, r in rows for k in range(4) if r[k].lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


# --------------------------------------------------------------------------------------
# CPU oracle (baseline / reference arm)
# --------------------------------------------------------------------------------------

def host_cpu():
    """Model name and logical core count of this host (where the oracle runs)."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if model is None:
        try:
            for line in open("/proc/cpuinfo"):
                if line.lower().startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
        except OSError:
            pass
    import platform

    return {"model": model or platform.processor() or platform.machine(), "hardware_concurrency": os.cpu_count()}


def oracle_sample_time(I_sample, seed):
    import oracle
    import ttgen

    Y, Yp = ttgen.perturbed_pair([I_sample] * N_MODES, RANK, seed)
    X = oracle.tt_add(Y, Yp)
    t0 = time.perf_counter()
    oracle.tt_round(X, EPS)
    return time.perf_counter() - t0


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    total = args.steps + args.warmup
    # per-step sample sized so the whole run stays within a few minutes (cost is linear in I_n)
    I_sample = max(512, min(8192, int(65536 * 120.0 / (max(total, 1) * 115.0)) // 512 * 512))
    times = []
    for k in range(total):
        t = oracle_sample_time(I_sample, SEED)
        if k >= args.warmup:
            times.append(t)
    t_step = sum(times) / len(times)
    value = (I_sample / args.modes) / t_step
    sample = f"oracle tt_round of the same construction with I_n={I_sample} per step, scaled by {I_sample}/{args.modes}"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "TT-rounds/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_step * 1e3 * args.modes / I_sample,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_desc(args.modes), "N": N_MODES, "I": args.modes, "formal_rank": 2 * RANK,
                       "eps": EPS, "seed": SEED},
            "cpu_baseline": {"value": value, "unit": "TT-rounds/s", "cores": 1, "kind": "oracle", "sample": sample,
                             "host": host_cpu()},
            "e2e": {"value": value, "unit": "TT-rounds/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------------------
# variants: the mixed-precision and batched forms beside plain FP64, same box, same run
# --------------------------------------------------------------------------------------

def _time(fn, reps=2):
    import torch

    fn()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(reps):
        fn()
    torch.cuda.synchronize()
    return (time.perf_counter() - t0) / reps


def run_variants(args):
    """Decaying-spectrum workload (N=50, I_n=16384, formal ranks 64, eps=1e-5) in fp64,
    fp32x2 and fp32, and the first `args.batch` tensors of the 512-tensor batched recipe
    (N in 4..20, I_n in 64..4096, ranks 2r with r in 4..48, eps=1e-6): a loop of FP64
    roundings against graph-captured batches in FP64, fp32x2 and fp32."""
    import torch

    import paper_2011_06532_gb300 as ttgb
    import ttgen

    out = {}

    def neg_first(x):
        c = [t.clone() for t in x.cores]
        c[0] = -c[0]
        return ttgb.DeviceTT(list(x.I), list(x.R), c)

    def as64(x):
        return ttgb.DeviceTT(list(x.I), list(x.R), [c.double() for c in x.cores])

    # ---- mixed precision on the decaying-spectrum workload
    terms = ttgen.decaying_terms(50, 16384, ttgen.BASE_SEED + 3)
    X = ttgb.from_host(terms[0].I, terms[0].R, terms[0].cores)
    for T in terms[1:]:
        X = ttgb.tt_add(X, ttgb.from_host(T.I, T.R, T.cores))
    del terms
    X32 = ttgb.DeviceTT(list(X.I), list(X.R), [c.float() for c in X.cores])
    res = {}
    y64 = ttgb.tt_round(X, 1e-5)
    t64 = _time(lambda: ttgb.tt_round(X, 1e-5))
    res["fp64"] = {"tt_rounds_per_s": 1.0 / t64, "ms": t64 * 1e3, "ranks_max": max(y64.R)}
    n64 = ttgb.tt_norm(y64)
    for prec in ("fp32x2", "fp32"):
        ttgb._ws_cache.clear()
        torch.cuda.empty_cache()
        y = ttgb.tt_round(X32, 1e-5, precision=prec)
        t = _time(lambda: ttgb.tt_round(X32, 1e-5, precision=prec))
        err = ttgb.tt_norm(ttgb.tt_add(as64(y), neg_first(y64))) / n64
        res[prec] = {"tt_rounds_per_s": 1.0 / t, "ms": t * 1e3, "rel_err_vs_fp64": err, "ranks_equal": y.R == y64.R,
                     "speedup_vs_fp64": t64 / t}
    out["decaying_N50_I16384_eps1e-5"] = res
    del X, X32, y64
    ttgb._ws_cache.clear()
    torch.cuda.empty_cache()

    # ---- batched recipe: the whole 512-tensor recipe in chunks (its FP64 form, 290 GB, does
    # not fit in HBM at once): per chunk a loop of FP64 roundings, one graph-captured FP64
    # batch, and graph-captured batches in fp32x2 and fp32; times summed over the chunks
    out["batched_%d" % args.batch] = run_batched_recipe(args)
    torch.cuda.empty_cache()
    out["hadamard_pipeline"] = run_pipeline(args)
    out["paper_model1"] = run_model1(args)
    out["small_N6_I32_R10"] = run_small(args)
    return out


def run_small(args):
    """The small workload (N=6, I_n=32, formal ranks 10 -> 5, eps=1e-6, FP64): one rounding at
    a time (launch- and latency-bound: each call queues one small launch per leaf phase, tree
    level and cut, and synchronizes once for the ranks) and 512 copies rounded as one
    graph-captured batch."""
    import torch

    import paper_2011_06532_gb300 as ttgb
    import ttgen

    (Y, Yp), eps = ttgen.config_small()
    X = ttgb.tt_add(ttgb.from_host(Y.I, Y.R, Y.cores), ttgb.from_host(Yp.I, Yp.R, Yp.cores))
    y = ttgb.tt_round(X, eps)
    t1 = _time(lambda: ttgb.tt_round(X, eps), reps=200)
    copies = 512
    xs = [ttgb.DeviceTT(list(X.I), list(X.R), [c.clone() for c in X.cores]) for _ in range(copies)]
    b = ttgb.Batch(xs, [eps] * copies, "fp64")
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        b.enqueue(s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        b.enqueue(s)
    tb = _time(g.replay, reps=5)
    same = all(o.R == y.R for o in b.outputs())
    del b, g, xs
    torch.cuda.empty_cache()
    return {"ranks": y.R, "single_tt_rounds_per_s": 1.0 / t1, "single_ms": t1 * 1e3,
            "graph_batch": {"copies": copies, "tt_rounds_per_s": copies / tb, "ms": tb * 1e3, "ranks_equal": same}}


def run_batched_recipe(args):
    """The first args.batch tensors of the batched recipe, args.chunk at a time (inputs drawn on
    the device with the recipe's shapes; timing only).  Per chunk: a Python loop of FP64
    tt_round calls (each synchronizes the host), one graph-captured FP64 batch (isolates the
    gain from concurrency), then graph-captured fp32x2 and fp32 batches (the precision gain
    on top).  Ranks of every batched form are compared with the FP64 loop's."""
    import torch

    import paper_2011_06532_gb300 as ttgb
    import ttgen

    shapes = ttgen.batched_shapes()[: args.batch]
    tot = {"fp64_loop": 0.0, "fp64_graph": 0.0, "fp32x2_graph": 0.0, "fp32_graph": 0.0}
    tuned = None
    equal = {k: True for k in tot if k != "fp64_loop"}
    gb32 = 0.0

    def graph_time(xs, prec):
        b = ttgb.Batch(xs, [1e-6] * len(xs), prec)
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            b.enqueue(s)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            b.enqueue(s)
        t = _time(g.replay, reps=1)
        outs = b.outputs()
        del b, g
        return t, outs

    for c0 in range(0, len(shapes), args.chunk):
        X64 = []
        for t, (I, r) in enumerate(shapes[c0:c0 + args.chunk]):
            (I_, R, Y), (_, _, Yp) = ttgen.device_perturbed_pair(I, r, ttgen.BASE_SEED + 4 + 97 * (c0 + t))
            X64.append(ttgb.tt_add(ttgb.DeviceTT(I_, R, Y), ttgb.DeviceTT(I_, R, Yp)))
            del Y, Yp
        torch.cuda.synchronize()
        t = _time(lambda: [ttgb.tt_round(x, 1e-6) for x in X64], reps=1)
        tot["fp64_loop"] += t
        ref = [ttgb.tt_round(x, 1e-6).R for x in X64]
        ttgb._ws_cache.clear()
        t, outs = graph_time(X64, "fp64")
        tot["fp64_graph"] += t
        equal["fp64_graph"] &= all(a == o.R for a, o in zip(ref, outs))
        del outs
        X32 = [ttgb.DeviceTT(x.I, x.R, [c.float() for c in x.cores]) for x in X64]
        gb32 += sum(x.nbytes() for x in X32) / 1e9
        del X64
        torch.cuda.empty_cache()
        for prec in ("fp32x2", "fp32"):
            t, outs = graph_time(X32, prec)
            tot[prec + "_graph"] += t
            equal[prec + "_graph"] &= all(a == o.R for a, o in zip(ref, outs))
            del outs
            torch.cuda.empty_cache()
            if prec == "fp32x2" and c0 == 0:
                # the autotuner's batch policy on the first chunk (tt_autotune_batched)
                b = ttgb.Batch(X32, [1e-6] * len(X32), prec)
                t0 = time.perf_counter()
                b.autotune()
                tune_s = time.perf_counter() - t0
                del b
                t2, outs = graph_time(X32, prec)
                caps = sorted({int(ln.split()[7]) for ln in ttgb.tune_export().splitlines()
                               if ln and not ln.startswith("#") and int(ln.split()[7]) < int(ln.split()[2])})
                tuned = {"tensors": len(X32), "ms_default": t * 1e3, "ms_tuned": t2 * 1e3, "tuning_s": tune_s,
                         "leaf_cap": caps[0] if caps else None,
                         "ranks_equal": all(a == o.R for a, o in zip(ref, outs))}
                del outs
                ttgb.tune_clear()
                torch.cuda.empty_cache()
        del X32
        torch.cuda.empty_cache()
    n = len(shapes)
    res = {"tensors": n, "chunk": args.chunk, "input_gb_fp32": gb32, "first_chunk_fp32x2_autotuned": tuned}
    for k, v in tot.items():
        res[k] = {"tts_per_s": n / v, "ms": v * 1e3}
        if k != "fp64_loop":
            res[k].update({"speedup_vs_fp64_loop": tot["fp64_loop"] / v, "ranks_equal": equal[k]})
        if k.startswith("fp32"):
            res[k]["speedup_vs_fp64_graph"] = tot["fp64_graph"] / v
    return res


def run_model1(args):
    """The paper's TT Model 1 (Sec. 4, synthetic models: N=50 modes of size 2000, ranks 50
    halved by the rounding), built the paper's way, Y = 2X - X with X a random rank-25 TT
    (here via tt_add of two scaled copies), rounded at eps = 1e-8 (the paper states no
    tolerance; any value between rounding error and the 25th singular value halves the
    ranks).  Its single-node timing (Table 3: 9.2 s on one Skylake core, 0.27 s on 40) is
    context for this row, not a ratio of the headline."""
    import torch

    import paper_2011_06532_gb300 as ttgb
    import ttgen

    N, I, r = 50, 2000, 25
    _, R, X = ttgen.device_random_tt([I] * N, ttgen.uniform_ranks(N, r), ttgen.BASE_SEED + 6)
    two = ttgb.DeviceTT([I] * N, R, [2.0 * X[0]] + X[1:])
    neg = ttgb.DeviceTT([I] * N, R, [-X[0]] + X[1:])
    Y = ttgb.tt_add(two, neg)
    del two, neg, X
    res = {"N": N, "I": I, "formal_rank": 2 * r, "eps": 1e-8, "input_gb_fp64": Y.nbytes() / 1e9,
           "paper_seconds": {"1 Skylake core": 9.2, "40 Skylake cores": 0.27}}
    y = ttgb.tt_round(Y, 1e-8)
    t = _time(lambda: ttgb.tt_round(Y, 1e-8), reps=3)
    ttgb.trace(True)
    ttgb.tt_round(Y, 1e-8)
    torch.cuda.synchronize()
    tr = ttgb.trace_read()
    ttgb.trace(False)
    res["fp64"] = {"ms": t * 1e3, "ranks_max": max(y.R), "ranks_halved": max(y.R) == r,
                   "kernel_ms": {k: round(v[1], 3) for k, v in tr.items() if v[0]},
                   "launches": sum(v[0] for v in tr.values())}
    Y32 = ttgb.DeviceTT(list(Y.I), list(Y.R), [c.float() for c in Y.cores])
    ttgb._ws_cache.clear()
    torch.cuda.empty_cache()
    y32 = ttgb.tt_round(Y32, 1e-6, precision="fp32x2")
    t32 = _time(lambda: ttgb.tt_round(Y32, 1e-6, precision="fp32x2"), reps=3)
    res["fp32x2_eps1e-6"] = {"ms": t32 * 1e3, "ranks_max": max(y32.R)}
    del Y, Y32, y, y32
    ttgb._ws_cache.clear()
    torch.cuda.empty_cache()
    return res


def _round_supported(I, r, precision):
    """Whether tt_round plans a TT of modes I and uniform rank r (host-side size query)."""
    import ctypes

    import paper_2011_06532_gb300 as ttgb
    from paper_2011_06532_gb300 import _native

    N = len(I)
    R = [1] + [r] * (N - 1) + [1]
    Ia, Ra = (ctypes.c_int64 * N)(*I), (ctypes.c_int64 * (N + 1))(*R)
    ptrs = (ctypes.c_void_p * N)(*([1] * N))  # never dereferenced by the size query
    d = _native.TTTensor(N, 1, Ia, Ra, ptrs)
    n = ctypes.c_size_t(0)
    return _native.load().tt_round_workspace_size(ctypes.byref(d), ttgb.PRECISIONS[precision], ctypes.byref(n)) == 0


def run_pipeline(args):
    """Hadamard pipeline (N=30, I_n=1024): Z = A o B, Y = round(Z, 1e-6), <Y, Z>, ||Y||.
    Pair 0 (ranks 8 x 8 -> 64) in FP64 and fp32x2; then every pair of the 64-pair recipe
    whose product rank is within the supported maximum, with the roundings as one batch."""
    import torch

    import paper_2011_06532_gb300 as ttgb
    import ttgen

    res = {}

    def neg_first(x):
        c = [t.clone() for t in x.cores]
        c[0] = -c[0]
        return ttgb.DeviceTT(list(x.I), list(x.R), c)

    A, B = ttgen.hadamard_pair(0)
    runs = {}
    for prec, dt in (("fp64", torch.float64), ("fp32x2", torch.float32)):
        dA = ttgb.from_host(A.I, A.R, A.cores, dtype=dt)
        dB = ttgb.from_host(B.I, B.R, B.cores, dtype=dt)

        def step():
            Z = ttgb.tt_hadamard(dA, dB)
            Y = ttgb.tt_round(Z, 1e-6, precision=prec)
            return Y, ttgb.tt_dot(Y, Z), ttgb.tt_norm(Y)

        out = step()
        t = _time(step, reps=2)
        runs[prec] = out
        res[prec] = {"ms": t * 1e3, "pipelines_per_s": 1.0 / t, "ranks_max": max(out[0].R)}
    (y64, d64, n64), (y32, d32, n32) = runs["fp64"], runs["fp32x2"]
    y32d = ttgb.DeviceTT(list(y32.I), list(y32.R), [c.double() for c in y32.cores])
    res["fp32x2"].update({
        "speedup_vs_fp64": res["fp64"]["ms"] / res["fp32x2"]["ms"],
        "rel_err_Y_vs_fp64": ttgb.tt_norm(ttgb.tt_add(y32d, neg_first(y64))) / n64,
        "rel_err_dot_vs_fp64": abs(d32 - d64) / abs(d64), "ranks_equal": y32.R == y64.R})
    del runs, y64, y32, y32d
    torch.cuda.empty_cache()
    # the batch of supported pairs (inputs drawn on the device; timing only)
    shapes = ttgen.hadamard_pair_shapes()
    pairs = [p for p, (ra, rb) in enumerate(shapes) if _round_supported([1024] * 30, ra * rb, "fp32x2")]
    N, I = 30, 1024
    Zs = []
    for p in pairs:
        ra, rb = shapes[p]
        _, Ra, ca = ttgen.device_random_tt([I] * N, ttgen.uniform_ranks(N, ra), ttgen.BASE_SEED + 5 + 2 * p)
        _, Rb, cb = ttgen.device_random_tt([I] * N, ttgen.uniform_ranks(N, rb), ttgen.BASE_SEED + 6 + 2 * p)
        a = ttgb.DeviceTT([I] * N, Ra, [c.float() for c in ca])
        b = ttgb.DeviceTT([I] * N, Rb, [c.float() for c in cb])
        Zs.append((a, b))
        del ca, cb

    def batch_step():
        Z = [ttgb.tt_hadamard(a, b) for a, b in Zs]
        Y = ttgb.Batch(Z, [1e-6] * len(Z), "fp32x2").run()
        return [(ttgb.tt_dot(y, z), ttgb.tt_norm(y)) for y, z in zip(Y, Z)]

    t = _time(batch_step, reps=1)
    res["batch_fp32x2"] = {"pairs": len(pairs), "of_recipe_pairs": len(shapes), "ms": t * 1e3,
                           "pipelines_per_s": len(pairs) / t,
                           "note": "pairs whose product rank tt_round does not place are skipped"}
    del Zs
    torch.cuda.empty_cache()
    return res


# --------------------------------------------------------------------------------------
# this library
# --------------------------------------------------------------------------------------

def run_ours(args):
    import numpy as np
    import torch

    import paper_2011_06532_gb300 as ttgb
    import ttgen

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    ttgb.build()
    dev = torch.device("cuda", local)
    seed = rank_seed(rank)
    I = [args.modes] * N_MODES
    Y, Yp = ttgen.perturbed_pair(I, RANK, seed)
    dY = ttgb.from_host(Y.I, Y.R, Y.cores, device=dev)
    dYp = ttgb.from_host(Yp.I, Yp.R, Yp.cores, device=dev)
    X = ttgb.tt_add(dY, dYp)  # formal ranks 32, built by the library's own sum kernel
    del dY, dYp
    torch.cuda.synchronize()
    in_bytes = X.nbytes()
    stream = torch.cuda.current_stream()

    for _ in range(args.warmup):
        out = ttgb.tt_round(X, EPS)
    torch.cuda.synchronize()
    L = out.R

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    # ---------------- device-resident timed region ----------------
    clocks = ClockSampler(local)
    barrier()
    ttgb.trace(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        out = ttgb.tt_round(X, EPS)
    e1.record(stream)
    barrier()
    ttgb.trace(False)
    ms = max_over_ranks(e0.elapsed_time(e1), dist, dev)
    clk = clocks.stop()
    tr = ttgb.trace_read()
    launches = sum(v[0] for v in tr.values())
    out_bytes = out.nbytes()

    # ---------------- end to end through the API, host buffers ----------------
    # Inputs and outputs in pinned host memory.  (1) tt_round on the host cores directly:
    # its kernels read each input core once and write each output core once over the
    # host link (NVLink-C2C on GB300), inside the timed region.  (2) For comparison, the
    # same with explicit staging copies host -> device -> host around a device rounding.
    hX = [c.to("cpu").pin_memory() for c in X.cores]
    hOut = [torch.empty(s, dtype=torch.float64).pin_memory() for s in X.core_sizes()]
    hXt = ttgb.DeviceTT(X.I, X.R, hX)
    ttgb.tt_round(hXt, EPS, out=hOut)  # warm-up of the host-memory path
    barrier()
    e2, e3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e2.record(stream)
    h2d = d2h = 0
    for _ in range(args.steps):
        y = ttgb.tt_round(hXt, EPS, out=hOut)
        h2d += sum(c.numel() * 8 for c in hX)
        d2h += sum(c.numel() * 8 for c in y.cores)
    e3.record(stream)
    barrier()
    ms_e2e = max_over_ranks(e2.elapsed_time(e3), dist, dev)
    dX = [torch.empty_like(c) for c in X.cores]
    barrier()
    e4, e5 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e4.record(stream)
    for _ in range(args.steps):
        for dc, hc in zip(dX, hX):
            dc.copy_(hc, non_blocking=True)
        y = ttgb.tt_round(ttgb.DeviceTT(X.I, X.R, dX), EPS)
        for k, c in enumerate(y.cores):
            hOut[k][: c.numel()].copy_(c, non_blocking=True)
    e5.record(stream)
    barrier()
    ms_copy = max_over_ranks(e4.elapsed_time(e5), dist, dev)

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return

    rounds_per_s = job_rate(world, args.steps, ms)
    fl = flops_by_kernel(I, X.R, L)
    dom = max(("s1_leaf", "s2_leaf", "s2_out"), key=lambda k: tr[k][1])
    n_dom, ms_dom = tr[dom]
    flops_per_launch = fl[dom] * args.steps / max(n_dom, 1)
    achieved = fl[dom] * args.steps / (ms_dom / 1e3) / 1e12 if ms_dom > 0 else None
    traffic = read_traffic(dom)

    # CPU baseline: the oracle on a bounded sample (1/8 of the slices), one thread
    cpu = None
    if world == 1:
        I_s = min(8192, args.modes)
        t_cpu = oracle_sample_time(I_s, SEED)
        cpu = {"value": (I_s / args.modes) / t_cpu, "unit": "TT-rounds/s", "cores": 1, "kind": "oracle",
               "sample": f"oracle tt_round of the same construction with I_n={I_s} ({t_cpu:.1f} s), "
                         f"scaled by {I_s}/{args.modes} (cost is linear in I_n)", "host": host_cpu()}

    variants = None
    if world == 1 and args.variants:
        del X, dX, hX, hOut
        ttgb._ws_cache.clear()
        torch.cuda.empty_cache()
        variants = run_variants(args)

    alg_bytes = 2 * in_bytes + out_bytes  # two reads of the input cores, one write of the output
    line = {
        "metric": METRIC, "value": rounds_per_s, "unit": "TT-rounds/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_desc(args.modes), "N": N_MODES, "I": args.modes, "formal_rank": 2 * RANK,
                   "eps": EPS, "seed": SEED, "output_ranks": L, "input_bytes": in_bytes,
                   "l2": "inputs larger than L2 (no flush)", "parallelism": "one independent TT per rank"},
        "hbm_gbs": alg_bytes * rounds_per_s / world / 1e9,
        "roofline": {"bound": "alu", "kernel": dom, "achieved": achieved, "peak": FP64_PEAK_TFLOPS,
                     "unit": "TFLOP/s", "frac": (achieved / FP64_PEAK_TFLOPS) if achieved else None,
                     "traffic": traffic, "flops_per_launch": flops_per_launch,
                     "ms_per_launch": ms_dom / max(n_dom, 1),
                     "peak_note": "FP64 pipe: 152 SMs x 2 FMA/clk x 2 x 2.07 GHz"},
        "kernel_ms_per_step": {k: v[1] / args.steps for k, v in tr.items() if v[0]},
        "cpu_baseline": cpu,
        "e2e": {"value": job_rate(world, args.steps, ms_e2e), "unit": "TT-rounds/s",
                "h2d_bytes_per_step": h2d // args.steps, "d2h_bytes_per_step": d2h // args.steps,
                "path": "tt_round on pinned host cores (kernels read inputs and write outputs over the host link)",
                "staged_copies": {"value": job_rate(world, args.steps, ms_copy), "unit": "TT-rounds/s",
                                  "path": "host->device copies, device tt_round, device->host copies"}},
        "gpu_launches": launches,
        "clocks": clk,
        "variants": variants,
    }
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def main():
    args = parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
