"""FP64 CPU oracle for TT arithmetic -- TEST INFRASTRUCTURE ONLY.

Only tests/, ``__graft_entry__.smoke()`` and the CPU-baseline leg of bench.py
may import this package.  The CUDA library never imports, links or calls it,
and the two share no code: the oracle is plain C (oracle.c, no BLAS) behind a
ctypes wrapper, and inputs reach it only through the seeded generators in
``ttgen``.

Every function follows a passage of Al Daas, Ballard, Benner, "Parallel
Algorithms for Tensor Train Arithmetic" (arXiv 2011.06532), cited in oracle.c:
  qr          Householder QR (local QR of Alg. 1 / Alg. 2)
  svd         one-sided Jacobi SVD (the SVD of Alg. 2, taken of the R factor)
  tt_round    Alg. 2, TT rounding (right-to-left orthonormalization, then
              left-to-right delta-truncation, delta = eps ||X|| / sqrt(N-1))
  tt_orth_right  Alg. 1
  tt_orth_left   the mirror of Alg. 1 (left-orthonormalization, Sec. 3.4)
  tt_round_lrl   TT rounding in the LRL ordering (Sec. 3.4, Sec. 4.3.2)
  tt_norm     Sec. 3.2.4, norm through orthonormalization
  tt_dot      Sec. 3.2.3, Eq. innerprodsum (and its two-multiplication form)
  tt_add      Sec. 3.2.1;  tt_hadamard  Sec. 3.2.2
  tt_full / tt_svd  brute-force helpers for tiny tensors.
All are pinned by tests/test_oracle_pins.py; none is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from typing import Optional, Tuple

import numpy as np

from ttgen import TT, core_sizes, from_flat

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lib = None

_i64p = ctypes.POINTER(ctypes.c_int64)
_f64p = ctypes.POINTER(ctypes.c_double)


def build(force: bool = False, extra_flags=(), out_path: Optional[str] = None) -> str:
    """Compile oracle.c with gcc into a shared library; returns its path."""
    out = out_path or _LIB_PATH
    os.makedirs(os.path.dirname(out), exist_ok=True)
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(_SRC):
        tmp = out + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm", *extra_flags]
        subprocess.run(cmd, check=True)
        os.replace(tmp, out)
    return out


def _bind(lib):
    sig = {
        "orc_qr": [ctypes.c_int64, ctypes.c_int64, _f64p, _f64p, _f64p],
        "orc_svd": [ctypes.c_int64, ctypes.c_int64, _f64p, _f64p, _f64p, _f64p],
        "orc_tt_orth_right": [ctypes.c_int64, _i64p, _i64p, _f64p, _i64p, _f64p],
        "orc_tt_orth_left": [ctypes.c_int64, _i64p, _i64p, _f64p, _i64p, _f64p],
        "orc_tt_norm": [ctypes.c_int64, _i64p, _i64p, _f64p, _f64p],
        "orc_tt_round": [ctypes.c_int64, _i64p, _i64p, _f64p, ctypes.c_double, _i64p, _f64p, _f64p, _f64p, _f64p],
        "orc_tt_round_lrl": [ctypes.c_int64, _i64p, _i64p, _f64p, ctypes.c_double, _i64p, _f64p, _f64p, _f64p,
                             _f64p],
        "orc_tt_add": [ctypes.c_int64, _i64p, _i64p, _f64p, _i64p, _f64p, _i64p, _f64p],
        "orc_tt_hadamard": [ctypes.c_int64, _i64p, _i64p, _f64p, _i64p, _f64p, _i64p, _f64p],
        "orc_tt_dot": [ctypes.c_int64, _i64p, _i64p, _f64p, _i64p, _f64p, _f64p],
        "orc_tt_dot_two_step": [ctypes.c_int64, _i64p, _i64p, _f64p, _i64p, _f64p, _f64p],
        "orc_tt_full": [ctypes.c_int64, _i64p, _i64p, _f64p, _f64p],
        "orc_tt_svd": [ctypes.c_int64, _i64p, _f64p, ctypes.c_double, _i64p, _f64p],
    }
    for name, args in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = ctypes.c_int
    return lib


def load(path: Optional[str] = None):
    """Load (building first if needed) the oracle library."""
    global _lib
    if path is not None:
        return _bind(ctypes.CDLL(path))
    if _lib is None:
        _lib = _bind(ctypes.CDLL(build()))
    return _lib


class OracleError(RuntimeError):
    pass


def _chk(st: int, what: str):
    if st != 0:
        raise OracleError(f"{what} failed with status {st}")


def _p64(a: np.ndarray):
    return a.ctypes.data_as(_f64p)


def _pi(a: np.ndarray):
    return a.ctypes.data_as(_i64p)


def _tt_args(x: TT):
    I = np.ascontiguousarray(x.I, dtype=np.int64)
    R = np.ascontiguousarray(x.R, dtype=np.int64)
    flat = np.ascontiguousarray(x.flat(), dtype=np.float64)
    return I, R, flat


# --------------------------------------------------------------------------------------
# matrix kernels
# --------------------------------------------------------------------------------------

def qr(A: np.ndarray, lib=None) -> Tuple[np.ndarray, np.ndarray]:
    """Economy Householder QR of a 2-D array: A = Q R (Q m x k, R k x b)."""
    lib = lib or load()
    A = np.asfortranarray(A, dtype=np.float64)
    m, b = A.shape
    k = min(m, b)
    Q = np.zeros((m, k), order="F")
    R = np.zeros((k, b), order="F")
    _chk(lib.orc_qr(m, b, _p64(A), _p64(Q), _p64(R)), "orc_qr")
    return Q, R


def svd(B: np.ndarray, lib=None) -> Tuple[np.ndarray, np.ndarray, np.ndarray]:
    """Thin one-sided Jacobi SVD: B = U diag(S) V^T, S non-increasing."""
    lib = lib or load()
    B = np.asfortranarray(B, dtype=np.float64)
    m, n = B.shape
    k = min(m, n)
    U = np.zeros((m, k), order="F")
    S = np.zeros(k)
    V = np.zeros((n, k), order="F")
    _chk(lib.orc_svd(m, n, _p64(B), _p64(U), _p64(S), _p64(V)), "orc_svd")
    return U, S, V


# --------------------------------------------------------------------------------------
# TT operations
# --------------------------------------------------------------------------------------

class RoundInfo:
    def __init__(self, nrm: float, delta: float, tails: np.ndarray):
        self.nrm = nrm
        self.delta = delta
        self.tails = tails

    def __repr__(self):
        return f"RoundInfo(nrm={self.nrm!r}, delta={self.delta!r}, tails={self.tails!r})"


def tt_round(x: TT, eps: float, lib=None) -> Tuple[TT, RoundInfo]:
    """Alg. 2.  Returns the rounded TT and (||X||, delta, per-cut discarded tails)."""
    lib = lib or load()
    I, R, flat = _tt_args(x)
    Ro = np.zeros(x.N + 1, dtype=np.int64)
    out = np.zeros_like(flat)
    nrm = np.zeros(1)
    delta = np.zeros(1)
    tails = np.zeros(max(x.N - 1, 1))
    _chk(lib.orc_tt_round(x.N, _pi(I), _pi(R), _p64(flat), float(eps), _pi(Ro), _p64(out), _p64(nrm), _p64(delta),
                          _p64(tails)), "orc_tt_round")
    return from_flat(x.I, Ro, out), RoundInfo(float(nrm[0]), float(delta[0]), tails[: max(x.N - 1, 0)])


def tt_round_lrl(x: TT, eps: float, lib=None) -> Tuple[TT, RoundInfo]:
    """TT rounding in the LRL ordering (Sec. 3.4, Sec. 4.3.2): left-orthonormalization,
    then truncation from right to left.  tails[n-1] is the cut between cores n-1 and n."""
    lib = lib or load()
    I, R, flat = _tt_args(x)
    Ro = np.zeros(x.N + 1, dtype=np.int64)
    out = np.zeros_like(flat)
    nrm = np.zeros(1)
    delta = np.zeros(1)
    tails = np.zeros(max(x.N - 1, 1))
    _chk(lib.orc_tt_round_lrl(x.N, _pi(I), _pi(R), _p64(flat), float(eps), _pi(Ro), _p64(out), _p64(nrm),
                              _p64(delta), _p64(tails)), "orc_tt_round_lrl")
    return from_flat(x.I, Ro, out), RoundInfo(float(nrm[0]), float(delta[0]), tails[: max(x.N - 1, 0)])


def tt_orth_left(x: TT, lib=None) -> TT:
    """Left-orthonormalization (the mirror of Alg. 1): V(Y_n) has orthonormal columns
    for n < N-1 and the tensor is unchanged."""
    lib = lib or load()
    I, R, flat = _tt_args(x)
    Ro = np.zeros(x.N + 1, dtype=np.int64)
    out = np.zeros_like(flat)
    _chk(lib.orc_tt_orth_left(x.N, _pi(I), _pi(R), _p64(flat), _pi(Ro), _p64(out)), "orc_tt_orth_left")
    return from_flat(x.I, Ro, out)


def tt_orth_right(x: TT, lib=None) -> TT:
    lib = lib or load()
    I, R, flat = _tt_args(x)
    Ro = np.zeros(x.N + 1, dtype=np.int64)
    out = np.zeros_like(flat)
    _chk(lib.orc_tt_orth_right(x.N, _pi(I), _pi(R), _p64(flat), _pi(Ro), _p64(out)), "orc_tt_orth_right")
    return from_flat(x.I, Ro, out)


def tt_norm(x: TT, lib=None) -> float:
    lib = lib or load()
    I, R, flat = _tt_args(x)
    out = np.zeros(1)
    _chk(lib.orc_tt_norm(x.N, _pi(I), _pi(R), _p64(flat), _p64(out)), "orc_tt_norm")
    return float(out[0])


def _binary_shapes(a: TT, b: TT):
    if list(a.I) != list(b.I):
        raise ValueError("mode sizes differ")


def tt_add(a: TT, b: TT, lib=None) -> TT:
    lib = lib or load()
    _binary_shapes(a, b)
    I, Ra, fa = _tt_args(a)
    _, Rb, fb = _tt_args(b)
    N = a.N
    if N == 1:
        Ro = [1, 1]
    else:
        Ro = [1] + [int(Ra[n] + Rb[n]) for n in range(1, N)] + [1]
    out = np.zeros(sum(core_sizes(a.I, Ro)))
    Rout = np.zeros(N + 1, dtype=np.int64)
    _chk(lib.orc_tt_add(N, _pi(I), _pi(Ra), _p64(fa), _pi(Rb), _p64(fb), _pi(Rout), _p64(out)), "orc_tt_add")
    return from_flat(a.I, Rout, out)


def tt_hadamard(a: TT, b: TT, lib=None) -> TT:
    lib = lib or load()
    _binary_shapes(a, b)
    I, Ra, fa = _tt_args(a)
    _, Rb, fb = _tt_args(b)
    Ro = [int(Ra[n] * Rb[n]) for n in range(a.N + 1)]
    out = np.zeros(sum(core_sizes(a.I, Ro)))
    Rout = np.zeros(a.N + 1, dtype=np.int64)
    _chk(lib.orc_tt_hadamard(a.N, _pi(I), _pi(Ra), _p64(fa), _pi(Rb), _p64(fb), _pi(Rout), _p64(out)),
         "orc_tt_hadamard")
    return from_flat(a.I, Rout, out)


def tt_dot(a: TT, b: TT, two_step: bool = False, lib=None) -> float:
    lib = lib or load()
    _binary_shapes(a, b)
    I, Ra, fa = _tt_args(a)
    _, Rb, fb = _tt_args(b)
    out = np.zeros(1)
    fn = lib.orc_tt_dot_two_step if two_step else lib.orc_tt_dot
    _chk(fn(a.N, _pi(I), _pi(Ra), _p64(fa), _pi(Rb), _p64(fb), _p64(out)), "orc_tt_dot")
    return float(out[0])


def tt_full(x: TT, lib=None) -> np.ndarray:
    """Full tensor as an N-d array (index order i_1, ..., i_N; Fortran layout)."""
    lib = lib or load()
    I, R, flat = _tt_args(x)
    total = int(np.prod(x.I))
    out = np.zeros(total)
    _chk(lib.orc_tt_full(x.N, _pi(I), _pi(R), _p64(flat), _p64(out)), "orc_tt_full")
    return out.reshape(tuple(x.I), order="F")


def tt_svd(full: np.ndarray, eps: float, lib=None) -> TT:
    """TT-SVD of a full tensor with the rounding's delta rule (brute-force helper)."""
    lib = lib or load()
    I = np.ascontiguousarray(full.shape, dtype=np.int64)
    data = np.ascontiguousarray(full.ravel(order="F"), dtype=np.float64)
    N = len(I)
    Ro = np.zeros(N + 1, dtype=np.int64)
    out = np.zeros(data.size * max(1, int(np.max(I)) ** 2))
    _chk(lib.orc_tt_svd(N, _pi(I), _p64(data), float(eps), _pi(Ro), _p64(out)), "orc_tt_svd")
    return from_flat(list(full.shape), Ro, out)


def scale_first(x: TT, s: float) -> TT:
    """Copy of x with its first core multiplied by s (so the tensor is scaled by s)."""
    cores = [c.copy() for c in x.cores]
    cores[0] = cores[0] * s
    return TT(list(x.I), list(x.R), cores)


def rel_err(y: TT, ref: TT, lib=None) -> float:
    """||y - ref|| / ||ref||, the difference formed as a TT sum and measured by the
    orthonormalization norm (Sec. 3.2.4: more accurate for small norms)."""
    lib = lib or load()
    d = tt_add(y.astype(np.float64), scale_first(ref, -1.0), lib=lib)
    nref = tt_norm(ref, lib=lib)
    nd = tt_norm(d, lib=lib)
    if nref == 0.0:
        return 0.0 if nd == 0.0 else float("inf")
    return nd / nref
