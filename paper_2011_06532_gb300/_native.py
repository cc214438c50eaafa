"""Build and load the CUDA library libttgb.so (sm_103a), in-tree.

The library is compiled from csrc/*.cu with nvcc, one object per translation unit
in parallel, then linked into paper_2011_06532_gb300/_build/libttgb.so.  Nothing
is installed into site-packages.
"""
from __future__ import annotations

import concurrent.futures
import ctypes
import os
import shutil
import subprocess

_HERE = os.path.dirname(os.path.abspath(__file__))
_ROOT = os.path.dirname(_HERE)
CSRC = os.path.join(_HERE, "csrc")
INCLUDE = os.path.join(_ROOT, "include")
BUILD = os.path.join(_HERE, "_build")
LIB = os.path.join(BUILD, "libttgb.so")
SOURCES = ["tt_round.cu", "tt_ops.cu", "tt_api.cu", "tt_tune.cu", "tt_orth.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libttgb.so")


def _deps_mtime() -> float:
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INCLUDE, "tt.h")]
    return max(os.path.getmtime(f) for f in files)


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile every translation unit for sm_103a and link libttgb.so; returns its path."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= _deps_mtime():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    common = [nvcc, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE]

    def compile_one(src):
        obj = os.path.join(BUILD, src.replace(".cu", ".o"))
        cmd = [*common, "-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        if verbose:
            print(r.stdout + r.stderr)
        return obj

    with concurrent.futures.ThreadPoolExecutor(len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = LIB + f".tmp{os.getpid()}"
    r = subprocess.run([nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


class TTTensor(ctypes.Structure):
    _fields_ = [
        ("N", ctypes.c_int32),
        ("dtype", ctypes.c_int32),
        ("I", ctypes.POINTER(ctypes.c_int64)),
        ("R", ctypes.POINTER(ctypes.c_int64)),
        ("cores", ctypes.POINTER(ctypes.c_void_p)),
    ]


# int (*)(const void *send, void *recv, size_t bytes, void *ctx)
ALLGATHER_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)


class TTShard(ctypes.Structure):
    _fields_ = [
        ("rank", ctypes.c_int32),
        ("world_size", ctypes.c_int32),
        ("I_global", ctypes.POINTER(ctypes.c_int64)),
        ("allgather", ALLGATHER_FN),
        ("ctx", ctypes.c_void_p),
    ]


EXPORTS = [
    "tt_round_workspace_size", "tt_round", "tt_round_batched", "tt_add", "tt_hadamard",
    "tt_dot_workspace_size", "tt_dot", "tt_norm_workspace_size", "tt_norm", "tt_status_string",
    "tt_trace", "tt_trace_read", "tt_dot_noalloc", "tt_round_batched_workspace_size", "tt_round_batched_async",
    "tt_autotune_workspace_size", "tt_autotune", "tt_autotune_batched_workspace_size", "tt_autotune_batched",
    "tt_tune_export", "tt_tune_import", "tt_tune_clear", "tt_tune_generation",
    "tt_round_ordered_workspace_size", "tt_round_ordered", "tt_orthonormalize_workspace_size", "tt_orthonormalize",
    "tt_round_hadamard_workspace_size", "tt_round_hadamard",
    "tt_shard_range", "tt_round_sharded_workspace_size", "tt_round_sharded",
]
KERNEL_KINDS = ["s1_leaf", "tree_factor", "tree_apply", "s2_leaf", "s2_out", "svd", "add", "hadamard", "dot", "misc"]

_lib = None


def load(path: str | None = None):
    """Load libttgb.so (it must have been built); raises if it is missing."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB
    if not os.path.exists(p):
        raise RuntimeError(f"{p} is missing: run paper_2011_06532_gb300.build() (or __graft_entry__.build()) first")
    lib = ctypes.CDLL(p)
    T = ctypes.POINTER(TTTensor)
    vp, sz = ctypes.c_void_p, ctypes.POINTER(ctypes.c_size_t)
    dp = ctypes.POINTER(ctypes.c_double)
    sigs = {
        "tt_round_workspace_size": [T, ctypes.c_int, sz],
        "tt_round": [T, ctypes.c_double, ctypes.c_int, T, vp, ctypes.c_size_t, vp],
        "tt_round_batched": [ctypes.c_int32, T, dp, ctypes.c_int, T, vp, ctypes.c_size_t, vp],
        "tt_round_batched_workspace_size": [ctypes.c_int32, T, ctypes.c_int, sz],
        "tt_round_batched_async": [ctypes.c_int32, T, dp, ctypes.c_int, T, vp, vp, vp, ctypes.c_size_t, vp],
        "tt_add": [T, T, T, vp],
        "tt_hadamard": [T, T, T, vp],
        "tt_dot_workspace_size": [T, T, sz],
        "tt_dot": [T, T, dp, vp, ctypes.c_size_t, vp],
        "tt_dot_noalloc": [T, T, dp, vp],
        "tt_norm_workspace_size": [T, sz],
        "tt_norm": [T, dp, vp, ctypes.c_size_t, vp],
        "tt_autotune_workspace_size": [T, ctypes.c_int, sz],
        "tt_autotune": [T, ctypes.c_double, ctypes.c_int, T, vp, ctypes.c_size_t, vp],
        "tt_autotune_batched_workspace_size": [ctypes.c_int32, T, ctypes.c_int, sz],
        "tt_autotune_batched": [ctypes.c_int32, T, dp, ctypes.c_int, T, vp, ctypes.c_size_t, vp],
        "tt_tune_export": [ctypes.c_char_p, ctypes.c_size_t, sz],
        "tt_tune_import": [ctypes.c_char_p],
        "tt_tune_clear": [],
        "tt_round_ordered_workspace_size": [T, ctypes.c_int, ctypes.c_int, sz],
        "tt_round_ordered": [T, ctypes.c_double, ctypes.c_int, ctypes.c_int, T, vp, ctypes.c_size_t, vp],
        "tt_orthonormalize_workspace_size": [T, ctypes.c_int, ctypes.c_int, sz],
        "tt_orthonormalize": [T, ctypes.c_int, ctypes.c_int, T, vp, ctypes.c_size_t, vp],
        "tt_round_hadamard_workspace_size": [T, T, ctypes.c_int, sz],
        "tt_round_hadamard": [T, T, ctypes.c_double, ctypes.c_int, T, vp, ctypes.c_size_t, vp],
        "tt_shard_range": [ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(ctypes.c_int64),
                           ctypes.POINTER(ctypes.c_int64)],
        "tt_round_sharded_workspace_size": [T, ctypes.c_int, ctypes.POINTER(TTShard), sz],
        "tt_round_sharded": [T, ctypes.c_double, ctypes.c_int, ctypes.POINTER(TTShard), T, vp, ctypes.c_size_t, vp],
    }
    for name, args in sigs.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = ctypes.c_int
    lib.tt_trace.argtypes = [ctypes.c_int]
    lib.tt_trace.restype = ctypes.c_int
    lib.tt_trace_read.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_double)]
    lib.tt_trace_read.restype = ctypes.c_int
    lib.tt_tune_generation.argtypes = []
    lib.tt_tune_generation.restype = ctypes.c_uint64
    lib.tt_status_string.argtypes = [ctypes.c_int]
    lib.tt_status_string.restype = ctypes.c_char_p
    if path is None:
        _lib = lib
    return lib
