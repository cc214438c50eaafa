"""TT arithmetic on one NVIDIA GB300 (sm_103a): rounding, sum, Hadamard, inner product, norm.

Thin Python binding over the C ABI of include/tt.h (libttgb.so).  It only marshals
arguments: device memory and streams come from PyTorch, every step of every
operation runs in the library's own CUDA kernels.  There is no CPU fallback: a
missing library or a machine without CUDA raises.

A tensor is a ``DeviceTT``: mode sizes I, ranks R and a list of 1-D CUDA tensors,
core n holding R[n]*I[n]*R[n+1] elements, entry (a, i, b) at a + R[n]*(i + I[n]*b)
(Sec. 3.1's vec-oriented order).  float64 cores compute in FP64; float32 cores
stream and run the per-slab Householder work in FP32 with FP64 small factors.
"""
from __future__ import annotations

import ctypes
import dataclasses
from typing import List, Optional, Sequence

import torch

from . import _native
from ._native import build  # noqa: F401  (re-export)

__all__ = ["DeviceTT", "Batch", "build", "tt_round", "tt_round_batched", "tt_add", "tt_hadamard", "tt_dot", "tt_norm",
           "tt_orthonormalize", "tt_round_hadamard", "tt_round_sharded", "shard_range", "dist_allgather", "TTError",
           "from_host", "to_host", "trace", "trace_read"]

_DTYPES = {torch.float64: 0, torch.float32: 1}
# tt_precision: "default" (fp64 for float64 cores, fp32x2 for float32), "fp64", "fp32x2", "fp32"
PRECISIONS = {"default": 0, "fp64": 1, "fp32x2": 2, "fp32": 3}
# tt_order: "rlr" (right-to-left orthonormalization, truncation from the left; Alg. 2) or "lrl"
ORDERS = {"rlr": 0, "lrl": 1}
SIDES = {"right": 0, "left": 1}


class TTError(RuntimeError):
    def __init__(self, status: int, what: str):
        msg = _native.load().tt_status_string(status).decode()
        super().__init__(f"{what}: status {status} ({msg})")
        self.status = status


@dataclasses.dataclass
class DeviceTT:
    I: List[int]
    R: List[int]
    cores: List[torch.Tensor]

    @property
    def N(self) -> int:
        return len(self.I)

    @property
    def dtype(self) -> torch.dtype:
        return self.cores[0].dtype

    def core_sizes(self) -> List[int]:
        return [self.R[n] * self.I[n] * self.R[n + 1] for n in range(self.N)]

    def nbytes(self) -> int:
        return sum(s * self.cores[0].element_size() for s in self.core_sizes())


class _Desc:
    """Keeps the ctypes arrays of one tt_tensor descriptor alive."""

    def __init__(self, I: Sequence[int], R: Sequence[int], cores: Sequence[torch.Tensor], dtype: torch.dtype):
        N = len(I)
        self.I = (ctypes.c_int64 * N)(*I)
        self.R = (ctypes.c_int64 * (N + 1))(*R)
        self.ptrs = (ctypes.c_void_p * N)(*[c.data_ptr() for c in cores])
        self.s = _native.TTTensor(N, _DTYPES[dtype], self.I, self.R, self.ptrs)

    @property
    def ref(self):
        return ctypes.byref(self.s)

    def ranks(self) -> List[int]:
        return [int(v) for v in self.R]


def _check(status: int, what: str):
    if status != 0:
        raise TTError(status, what)


def _stream(stream: Optional[torch.cuda.Stream]):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _cuda_device(x: DeviceTT) -> torch.device:
    """The device a call on x runs on (the current one when x's cores are pinned host memory)."""
    return x.cores[0].device if x.cores[0].is_cuda else torch.device("cuda", torch.cuda.current_device())


def _validate(x: DeviceTT, host_ok: bool = False):
    ok = (lambda c: c.is_cuda or (c.device.type == "cpu" and c.is_pinned())) if host_ok else (lambda c: c.is_cuda)
    if not x.cores or any(not ok(c) for c in x.cores):
        raise ValueError("cores must be CUDA tensors" + (" or pinned host tensors" if host_ok else ""))
    if any(c.dtype != x.cores[0].dtype for c in x.cores) or x.cores[0].dtype not in _DTYPES:
        raise ValueError("cores must all be float64 or all float32")
    for n, c in enumerate(x.cores):
        if not c.is_contiguous() or c.numel() < x.R[n] * x.I[n] * x.R[n + 1]:
            raise ValueError(f"core {n} is too small or not contiguous")


_ws_cache: dict = {}


def _workspace(nbytes: int, device) -> torch.Tensor:
    key = (str(device),)
    buf = _ws_cache.get(key)
    if buf is None or buf.numel() < nbytes:
        buf = torch.empty(max(nbytes, 256), dtype=torch.uint8, device=device)
        _ws_cache[key] = buf
    return buf


def round_workspace_size(x: DeviceTT, precision: str = "default") -> int:
    lib = _native.load()
    d = _Desc(x.I, x.R, x.cores, x.dtype)
    n = ctypes.c_size_t(0)
    _check(lib.tt_round_workspace_size(d.ref, PRECISIONS[precision], ctypes.byref(n)), "tt_round_workspace_size")
    return int(n.value)


def tt_round(x: DeviceTT, eps: float, stream=None, out: Optional[List[torch.Tensor]] = None,
             workspace: Optional[torch.Tensor] = None, precision: str = "default", order: str = "rlr") -> DeviceTT:
    """TT rounding (Alg. 2 / Alg. 6): returns Y with ||X - Y|| <= eps ||X||.

    precision: "default", "fp64" (float64 cores), "fp32x2" or "fp32" (float32 cores).
    order: "rlr" (right-to-left orthonormalization, then truncation from the left, as in
    Alg. 2) or "lrl" (the mirror ordering, Sec. 4.3.2).
    Cores (of x and of out) may be CUDA tensors or pinned host tensors; the kernels read
    and write pinned host cores directly over the host link.  Without `out`, the result
    cores are allocated where x's are."""
    _validate(x, host_ok=True)
    if out is not None:
        _validate(DeviceTT(list(x.I), list(x.R), list(out)), host_ok=True)
    lib = _native.load()
    dev = _cuda_device(x)
    prec = PRECISIONS[precision]
    od = ORDERS[order]
    d = _Desc(x.I, x.R, x.cores, x.dtype)
    n = ctypes.c_size_t(0)
    if od == 0:
        _check(lib.tt_round_workspace_size(d.ref, prec, ctypes.byref(n)), "tt_round_workspace_size")
    else:
        _check(lib.tt_round_ordered_workspace_size(d.ref, prec, od, ctypes.byref(n)),
               "tt_round_ordered_workspace_size")
    ws = workspace if workspace is not None else _workspace(int(n.value), dev)
    if out is None:
        if x.cores[0].is_cuda:
            out = [torch.empty(s, dtype=x.dtype, device=dev) for s in x.core_sizes()]
        else:
            out = [torch.empty(s, dtype=x.dtype, pin_memory=True) for s in x.core_sizes()]
    o = _Desc(x.I, [1] * (x.N + 1), out, x.dtype)
    if od == 0:
        _check(lib.tt_round(d.ref, float(eps), prec, o.ref, ctypes.c_void_p(ws.data_ptr()),
                            ctypes.c_size_t(ws.numel()), _stream(stream)), "tt_round")
    else:
        _check(lib.tt_round_ordered(d.ref, float(eps), prec, od, o.ref, ctypes.c_void_p(ws.data_ptr()),
                                    ctypes.c_size_t(ws.numel()), _stream(stream)), "tt_round_ordered")
    R = o.ranks()
    cores = [out[k][: R[k] * x.I[k] * R[k + 1]] for k in range(x.N)]
    return DeviceTT(list(x.I), R, cores)


def tt_orthonormalize(x: DeviceTT, side: str = "right", precision: str = "default", stream=None) -> DeviceTT:
    """Orthonormalization with explicit factors (Alg. 1 / Alg. 5): side "right" makes
    H(Y_n) row-orthonormal for n >= 2 (the scale in core 1), "left" makes V(Y_n)
    column-orthonormal for n <= N-1 (the scale in core N).  Queued on the stream."""
    _validate(x)
    lib = _native.load()
    dev = x.cores[0].device
    prec = PRECISIONS[precision]
    sd = SIDES[side]
    d = _Desc(x.I, x.R, x.cores, x.dtype)
    n = ctypes.c_size_t(0)
    _check(lib.tt_orthonormalize_workspace_size(d.ref, prec, sd, ctypes.byref(n)), "tt_orthonormalize_workspace_size")
    ws = _workspace(int(n.value), dev)
    out = [torch.empty(s, dtype=x.dtype, device=dev) for s in x.core_sizes()]
    o = _Desc(x.I, [1] * (x.N + 1), out, x.dtype)
    _check(lib.tt_orthonormalize(d.ref, prec, sd, o.ref, ctypes.c_void_p(ws.data_ptr()), ctypes.c_size_t(ws.numel()),
                                 _stream(stream)), "tt_orthonormalize")
    R = o.ranks()
    return DeviceTT(list(x.I), R, [out[k][: R[k] * x.I[k] * R[k + 1]] for k in range(x.N)])


def autotune(x: DeviceTT, eps: float, precision: str = "default", stream=None) -> DeviceTT:
    """Tunes the leaves and tile rows of x's core classes for single roundings (timing
    complete roundings on the GPU, see tt_autotune) and returns the last rounding of x.
    Later plans of this process use the recorded choices."""
    _validate(x)
    lib = _native.load()
    dev = x.cores[0].device
    prec = PRECISIONS[precision]
    d = _Desc(x.I, x.R, x.cores, x.dtype)
    n = ctypes.c_size_t(0)
    _check(lib.tt_autotune_workspace_size(d.ref, prec, ctypes.byref(n)), "tt_autotune_workspace_size")
    ws = torch.empty(max(int(n.value), 256), dtype=torch.uint8, device=dev)
    out = [torch.empty(s, dtype=x.dtype, device=dev) for s in x.core_sizes()]
    o = _Desc(x.I, [1] * (x.N + 1), out, x.dtype)
    _check(lib.tt_autotune(d.ref, float(eps), prec, o.ref, ctypes.c_void_p(ws.data_ptr()), ctypes.c_size_t(ws.numel()),
                           _stream(stream)), "tt_autotune")
    R = o.ranks()
    return DeviceTT(list(x.I), R, [out[k][: R[k] * x.I[k] * R[k + 1]] for k in range(x.N)])


def tune_export() -> str:
    """The tile table as text (one "prec ctx I R0 R1 K0 K1 P Tt" line per entry)."""
    lib = _native.load()
    n = ctypes.c_size_t(0)
    _check(lib.tt_tune_export(None, 0, ctypes.byref(n)), "tt_tune_export")
    buf = ctypes.create_string_buffer(int(n.value))
    _check(lib.tt_tune_export(buf, ctypes.c_size_t(n.value), ctypes.byref(n)), "tt_tune_export")
    return buf.value.decode()


def tune_import(text: str) -> None:
    """Adds the entries of a text written by tune_export to the tile table."""
    _check(_native.load().tt_tune_import(text.encode()), "tt_tune_import")


def tune_clear() -> None:
    """Empties the tile table: plans go back to the built-in choices."""
    _check(_native.load().tt_tune_clear(), "tt_tune_clear")


def tune_generation() -> int:
    return int(_native.load().tt_tune_generation())


class Batch:
    """A prepared batch: descriptors, output buffers and workspace of a list of tensors.

    run() rounds the whole batch synchronously; enqueue() queues it without a host
    synchronization (ranks stay on the device), so it can be captured in a CUDA graph;
    ranks() / outputs() read the results after the queued work has finished."""

    def __init__(self, xs: Sequence[DeviceTT], eps: Sequence[float], precision: str = "default"):
        for x in xs:
            _validate(x)
        lib = _native.load()
        self.xs = list(xs)
        self.eps = (ctypes.c_double * max(len(xs), 1))(*[float(v) for v in eps])
        self.prec = PRECISIONS[precision]
        dev = xs[0].cores[0].device
        self.descs = [_Desc(x.I, x.R, x.cores, x.dtype) for x in xs]
        self.outs = [[torch.empty(s, dtype=x.dtype, device=dev) for s in x.core_sizes()] for x in xs]
        self.odescs = [_Desc(x.I, [1] * (x.N + 1), o, x.dtype) for x, o in zip(xs, self.outs)]
        self.arr_in = (_native.TTTensor * len(xs))(*[d.s for d in self.descs])
        self.arr_out = (_native.TTTensor * len(xs))(*[d.s for d in self.odescs])
        n = ctypes.c_size_t(0)
        _check(lib.tt_round_batched_workspace_size(len(xs), self.arr_in, self.prec, ctypes.byref(n)),
               "tt_round_batched_workspace_size")
        self.ws = torch.empty(max(int(n.value), 256), dtype=torch.uint8, device=dev)
        self.gen = tune_generation()
        self.ranks_dev = torch.zeros(sum(x.N + 1 for x in xs), dtype=torch.int32, device=dev)
        self.status_dev = torch.zeros(len(xs), dtype=torch.int32, device=dev)

    def _resize(self) -> None:
        # plans (and so workspace sizes) follow the tile table
        if self.gen == tune_generation():
            return
        n = ctypes.c_size_t(0)
        _check(_native.load().tt_round_batched_workspace_size(len(self.xs), self.arr_in, self.prec, ctypes.byref(n)),
               "tt_round_batched_workspace_size")
        if self.ws.numel() < int(n.value):
            self.ws = torch.empty(int(n.value), dtype=torch.uint8, device=self.ws.device)
        self.gen = tune_generation()

    def autotune(self, stream=None) -> None:
        """Tunes one leaf/tile policy for the members of this batch (tt_autotune_batched);
        later runs and enqueues of any batch with these member shapes use it."""
        lib = _native.load()
        n = ctypes.c_size_t(0)
        _check(lib.tt_autotune_batched_workspace_size(len(self.xs), self.arr_in, self.prec, ctypes.byref(n)),
               "tt_autotune_batched_workspace_size")
        ws = torch.empty(max(int(n.value), 256), dtype=torch.uint8, device=self.ws.device)
        _check(lib.tt_autotune_batched(len(self.xs), self.arr_in, self.eps, self.prec, self.arr_out,
                                       ctypes.c_void_p(ws.data_ptr()), ctypes.c_size_t(ws.numel()), _stream(stream)),
               "tt_autotune_batched")
        del ws
        self._resize()

    def run(self, stream=None) -> List[DeviceTT]:
        self._resize()
        lib = _native.load()
        _check(lib.tt_round_batched(len(self.xs), self.arr_in, self.eps, self.prec, self.arr_out,
                                    ctypes.c_void_p(self.ws.data_ptr()), ctypes.c_size_t(self.ws.numel()),
                                    _stream(stream)), "tt_round_batched")
        res = []
        for k, x in enumerate(self.xs):
            R = [int(self.arr_out[k].R[i]) for i in range(x.N + 1)]
            res.append(DeviceTT(list(x.I), R, [self.outs[k][n][: R[n] * x.I[n] * R[n + 1]] for n in range(x.N)]))
        return res

    def enqueue(self, stream=None) -> None:
        self._resize()
        lib = _native.load()
        _check(lib.tt_round_batched_async(len(self.xs), self.arr_in, self.eps, self.prec, self.arr_out,
                                          ctypes.c_void_p(self.ranks_dev.data_ptr()),
                                          ctypes.c_void_p(self.status_dev.data_ptr()),
                                          ctypes.c_void_p(self.ws.data_ptr()), ctypes.c_size_t(self.ws.numel()),
                                          _stream(stream)), "tt_round_batched_async")

    def outputs(self) -> List[DeviceTT]:
        status = self.status_dev.tolist()
        for st in status:
            _check(st, "tt_round_batched_async")
        ranks = self.ranks_dev.tolist()
        res, off = [], 0
        for k, x in enumerate(self.xs):
            R = ranks[off: off + x.N + 1]
            off += x.N + 1
            res.append(DeviceTT(list(x.I), R, [self.outs[k][n][: R[n] * x.I[n] * R[n + 1]] for n in range(x.N)]))
        return res


def tt_round_batched(xs: Sequence[DeviceTT], eps: Sequence[float], stream=None,
                     precision: str = "default") -> List[DeviceTT]:
    """Rounds several independent tensors with one call (spread over internal streams)."""
    if not xs:
        return []
    return Batch(xs, eps, precision).run(stream)


def tt_add(a: DeviceTT, b: DeviceTT, stream=None) -> DeviceTT:
    """Summation (Sec. 3.2.1); ranks add."""
    _validate(a)
    _validate(b)
    lib = _native.load()
    N = a.N
    R = [1] + [a.R[n] + b.R[n] for n in range(1, N)] + [1] if N > 1 else [1, 1]
    dev = a.cores[0].device
    out = [torch.empty(R[n] * a.I[n] * R[n + 1], dtype=a.dtype, device=dev) for n in range(N)]
    da, db = _Desc(a.I, a.R, a.cores, a.dtype), _Desc(b.I, b.R, b.cores, b.dtype)
    o = _Desc(a.I, R, out, a.dtype)
    _check(lib.tt_add(da.ref, db.ref, o.ref, _stream(stream)), "tt_add")
    return DeviceTT(list(a.I), o.ranks(), out)


def tt_hadamard(a: DeviceTT, b: DeviceTT, stream=None) -> DeviceTT:
    """Hadamard product (Sec. 3.2.2); ranks multiply."""
    _validate(a)
    _validate(b)
    lib = _native.load()
    N = a.N
    R = [a.R[n] * b.R[n] for n in range(N + 1)]
    dev = a.cores[0].device
    out = [torch.empty(R[n] * a.I[n] * R[n + 1], dtype=a.dtype, device=dev) for n in range(N)]
    da, db = _Desc(a.I, a.R, a.cores, a.dtype), _Desc(b.I, b.R, b.cores, b.dtype)
    o = _Desc(a.I, R, out, a.dtype)
    _check(lib.tt_hadamard(da.ref, db.ref, o.ref, _stream(stream)), "tt_hadamard")
    return DeviceTT(list(a.I), o.ranks(), out)


def shard_range(I: int, world: int, rank: int):
    """Slices [begin, end) of a mode of size I owned by shard `rank` of `world` (the 1 x P x 1
    distribution of Sec. 3.1): begin = floor(rank I / world)."""
    lib = _native.load()
    b, e = ctypes.c_int64(0), ctypes.c_int64(0)
    _check(lib.tt_shard_range(int(I), int(world), int(rank), ctypes.byref(b), ctypes.byref(e)), "tt_shard_range")
    return int(b.value), int(e.value)


class _Gather:
    """ctypes adapter of a Python all-gather fn(send, recv) over uint8 numpy views of the
    library's host buffers; an exception raised by fn becomes status TT_ERR_COMM in the
    library and is raised again after the call."""

    def __init__(self, fn, world: int):
        import numpy as np

        self.fn, self.world, self.error = fn, world, None

        def cb(send, recv, nbytes, ctx):
            try:
                s = np.ctypeslib.as_array((ctypes.c_ubyte * nbytes).from_address(send))
                r = np.ctypeslib.as_array((ctypes.c_ubyte * (nbytes * self.world)).from_address(recv))
                self.fn(s, r)
                return 0
            except BaseException as e:  # noqa: BLE001 -- reported after the call
                if self.error is None:
                    self.error = e
                return 1

        self.c = _native.ALLGATHER_FN(cb)


def dist_allgather(group=None):
    """An all-gather for tt_round_sharded over a torch.distributed process group: the payload
    is gathered as a uint8 tensor (host tensors for gloo, tensors of the current CUDA device
    for NCCL) in rank order."""
    import torch.distributed as dist

    def fn(send, recv):
        world = dist.get_world_size(group)
        t = torch.from_numpy(send.copy())
        if dist.get_backend(group) == "nccl":
            t = t.cuda()
        parts = [torch.empty_like(t) for _ in range(world)]
        dist.all_gather(parts, t, group=group)
        recv[:] = torch.cat(parts).cpu().numpy()

    return fn


def tt_round_sharded(x: DeviceTT, eps: float, I_global: Sequence[int], rank: int, world: int, allgather,
                     precision: str = "default", stream=None, workspace: Optional[torch.Tensor] = None) -> DeviceTT:
    """TT rounding (Alg. 2 / Alg. 6) of a tensor distributed over `world` shards: x is shard
    `rank`, holding slices shard_range(I_global[n], world, rank) of every core.  Every shard
    calls this with the same eps, precision, I_global and ranks; allgather(send, recv) gathers
    the bytes of send (uint8 numpy array) from every shard into recv (world times longer, in
    rank order), e.g. dist_allgather().  Returns this shard's slices of the rounded tensor
    (ranks equal on every shard).  The workspace is this call's own (shards on threads of one
    process do not share one)."""
    _validate(x)
    lib = _native.load()
    dev = x.cores[0].device
    prec = PRECISIONS[precision]
    d = _Desc(x.I, x.R, x.cores, x.dtype)
    g = _Gather(allgather, world)
    Ig = (ctypes.c_int64 * x.N)(*[int(v) for v in I_global])
    sh = _native.TTShard(int(rank), int(world), Ig, g.c, None)
    n = ctypes.c_size_t(0)
    _check(lib.tt_round_sharded_workspace_size(d.ref, prec, ctypes.byref(sh), ctypes.byref(n)),
           "tt_round_sharded_workspace_size")
    ws = workspace if workspace is not None else torch.empty(max(int(n.value), 256), dtype=torch.uint8, device=dev)
    out = [torch.empty(s, dtype=x.dtype, device=dev) for s in x.core_sizes()]
    o = _Desc(x.I, [1] * (x.N + 1), out, x.dtype)
    st = lib.tt_round_sharded(d.ref, float(eps), prec, ctypes.byref(sh), o.ref, ctypes.c_void_p(ws.data_ptr()),
                              ctypes.c_size_t(ws.numel()), _stream(stream))
    if g.error is not None:
        raise TTError(st, "tt_round_sharded (all-gather)") from g.error
    _check(st, "tt_round_sharded")
    R = o.ranks()
    return DeviceTT(list(x.I), R, [out[k][: R[k] * x.I[k] * R[k + 1]] for k in range(x.N)])


def tt_round_hadamard(a: DeviceTT, b: DeviceTT, eps: float, stream=None, precision: str = "default") -> DeviceTT:
    """round(A o B, eps) without forming the Hadamard product (its entries are formed
    where the rounding reads them); same result as tt_round(tt_hadamard(a, b), eps)."""
    _validate(a)
    _validate(b)
    lib = _native.load()
    dev = a.cores[0].device
    prec = PRECISIONS[precision]
    da, db = _Desc(a.I, a.R, a.cores, a.dtype), _Desc(b.I, b.R, b.cores, b.dtype)
    n = ctypes.c_size_t(0)
    _check(lib.tt_round_hadamard_workspace_size(da.ref, db.ref, prec, ctypes.byref(n)),
           "tt_round_hadamard_workspace_size")
    ws = _workspace(int(n.value), dev)
    Rz = [a.R[k] * b.R[k] for k in range(a.N + 1)]
    out = [torch.empty(Rz[k] * a.I[k] * Rz[k + 1], dtype=a.dtype, device=dev) for k in range(a.N)]
    o = _Desc(a.I, [1] * (a.N + 1), out, a.dtype)
    _check(lib.tt_round_hadamard(da.ref, db.ref, float(eps), prec, o.ref, ctypes.c_void_p(ws.data_ptr()),
                                 ctypes.c_size_t(ws.numel()), _stream(stream)), "tt_round_hadamard")
    R = o.ranks()
    return DeviceTT(list(a.I), R, [out[k][: R[k] * a.I[k] * R[k + 1]] for k in range(a.N)])


def tt_dot(a: DeviceTT, b: DeviceTT, stream=None) -> float:
    """Inner product <A, B> (Sec. 3.2.3); cores may be CUDA tensors or pinned host tensors."""
    _validate(a, host_ok=True)
    _validate(b, host_ok=True)
    lib = _native.load()
    da, db = _Desc(a.I, a.R, a.cores, a.dtype), _Desc(b.I, b.R, b.cores, b.dtype)
    n = ctypes.c_size_t(0)
    _check(lib.tt_dot_workspace_size(da.ref, db.ref, ctypes.byref(n)), "tt_dot_workspace_size")
    ws = _workspace(int(n.value), _cuda_device(a))
    res = ctypes.c_double(0.0)
    _check(lib.tt_dot(da.ref, db.ref, ctypes.byref(res), ctypes.c_void_p(ws.data_ptr()), ctypes.c_size_t(ws.numel()),
                      _stream(stream)), "tt_dot")
    return float(res.value)


def tt_norm(x: DeviceTT, stream=None) -> float:
    """Norm through orthonormalization (Sec. 3.2.4); cores may be CUDA or pinned host tensors."""
    _validate(x, host_ok=True)
    lib = _native.load()
    d = _Desc(x.I, x.R, x.cores, x.dtype)
    n = ctypes.c_size_t(0)
    _check(lib.tt_norm_workspace_size(d.ref, ctypes.byref(n)), "tt_norm_workspace_size")
    ws = _workspace(int(n.value), _cuda_device(x))
    res = ctypes.c_double(0.0)
    _check(lib.tt_norm(d.ref, ctypes.byref(res), ctypes.c_void_p(ws.data_ptr()), ctypes.c_size_t(ws.numel()),
                       _stream(stream)), "tt_norm")
    return float(res.value)


def trace(enable: bool) -> None:
    """Start (reset counters, bracket launches with CUDA events) or stop kernel tracing."""
    _check(_native.load().tt_trace(1 if enable else 0), "tt_trace")


def trace_read() -> dict:
    """{kernel class: (launches, device milliseconds)} since the last trace(True)."""
    lib = _native.load()
    out = {}
    for k, name in enumerate(_native.KERNEL_KINDS):
        n = ctypes.c_int64(0)
        ms = ctypes.c_double(0.0)
        _check(lib.tt_trace_read(k, ctypes.byref(n), ctypes.byref(ms)), "tt_trace_read")
        out[name] = (int(n.value), float(ms.value))
    return out


def from_host(I: Sequence[int], R: Sequence[int], cores: Sequence, dtype=torch.float64, device="cuda") -> DeviceTT:
    """Upload host cores (numpy arrays or tensors) to the GPU."""
    dev_cores = [torch.as_tensor(c).to(device=device, dtype=dtype).contiguous() for c in cores]
    return DeviceTT(list(map(int, I)), list(map(int, R)), dev_cores)


def to_host(x: DeviceTT):
    """Cores back to the host as float64 numpy arrays."""
    return [c.detach().to("cpu", torch.float64).numpy() for c in x.cores]
