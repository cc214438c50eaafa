"""Seeded synthetic TT inputs shared by the oracle tests, the GPU tests and bench.py.

This module holds random-number generation, a plain TT container and the
workload recipes (which random cores to draw, with which shapes and scalings).
It holds none of the method's arithmetic: TT sums, Hadamard products, rounding
and norms are computed by each side (the oracle, the CUDA library) with its own
code.  Recipes therefore return the *components* of each workload (e.g. Y and
Y' for X = Y + Y'); the consumer forms the sum with its own ``tt_add``.

Random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random
numbers: as easy as 1, 2, 3", SC'11), implemented here from its published
definition, followed by the Box-Muller transform in FP64 on the host.  Each
counter value yields two 53-bit uniforms and hence two normals.  Key =
(seed mod 2^32, stream), counter = (pair index lo, pair index hi, core index,
0).  The paper draws "random TT" tensors without naming a distribution (Sec.
4.2); entries here are i.i.d. N(0,1) / sqrt(I_n R_{n-1}).
"""
from __future__ import annotations

import dataclasses
from typing import List, Sequence

import numpy as np

_M0 = np.uint64(0xD2511F53)
_M1 = np.uint64(0xCD9E8D57)
_W0 = np.uint32(0x9E3779B9)
_W1 = np.uint32(0xBB67AE85)
_MASK32 = np.uint64(0xFFFFFFFF)


def philox4x32_10(ctr: np.ndarray, key: Sequence[int]) -> np.ndarray:
    """Philox4x32 with 10 rounds.

    ctr: uint32 array of shape (n, 4); key: two 32-bit integers.
    Returns a uint32 array of shape (n, 4).
    """
    c = np.asarray(ctr, dtype=np.uint32)
    c0 = c[:, 0].astype(np.uint64)
    c1 = c[:, 1].astype(np.uint64)
    c2 = c[:, 2].astype(np.uint64)
    c3 = c[:, 3].astype(np.uint64)
    k0 = np.uint32(key[0] & 0xFFFFFFFF)
    k1 = np.uint32(key[1] & 0xFFFFFFFF)
    with np.errstate(over="ignore"):
        for rnd in range(10):
            if rnd:
                k0 = np.uint32((int(k0) + int(_W0)) & 0xFFFFFFFF)
                k1 = np.uint32((int(k1) + int(_W1)) & 0xFFFFFFFF)
            p0 = _M0 * c0
            p1 = _M1 * c2
            hi0, lo0 = p0 >> np.uint64(32), p0 & _MASK32
            hi1, lo1 = p1 >> np.uint64(32), p1 & _MASK32
            c0, c1, c2, c3 = (hi1 ^ c1 ^ np.uint64(k0), lo1, hi0 ^ c3 ^ np.uint64(k1), lo0)
    return np.stack([c0, c1, c2, c3], axis=1).astype(np.uint32)


def _normal_pairs(p0: int, p1: int, seed: int, stream: int, core: int, out: np.ndarray) -> None:
    """Fills out[2*p0 : 2*p1] with the normals of counter values p0..p1-1."""
    idx = np.arange(p0, p1, dtype=np.uint64)
    ctr = np.empty((p1 - p0, 4), dtype=np.uint32)
    ctr[:, 0] = (idx & _MASK32).astype(np.uint32)
    ctr[:, 1] = (idx >> np.uint64(32)).astype(np.uint32)
    ctr[:, 2] = np.uint32(core & 0xFFFFFFFF)
    ctr[:, 3] = 0
    r = philox4x32_10(ctr, (seed & 0xFFFFFFFF, stream & 0xFFFFFFFF)).astype(np.uint64)
    a = (r[:, 0] << np.uint64(32)) | r[:, 1]
    b = (r[:, 2] << np.uint64(32)) | r[:, 3]
    u1 = ((a >> np.uint64(11)).astype(np.float64) + 1.0) * (2.0 ** -53)  # (0, 1]
    u2 = (b >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)  # [0, 1)
    rad = np.sqrt(-2.0 * np.log(u1))
    th = 2.0 * np.pi * u2
    out[2 * p0:2 * p1:2] = rad * np.cos(th)
    out[2 * p0 + 1:2 * p1:2] = rad * np.sin(th)


_CHUNK = 1 << 19


def normals(count: int, seed: int, stream: int, core: int) -> np.ndarray:
    """`count` standard normals (FP64) for one (seed, stream, core) triple.

    Large requests are split by counter range over host threads; the values do
    not depend on the split.
    """
    pairs = (count + 1) // 2
    z = np.empty(2 * pairs, dtype=np.float64)
    bounds = [(p, min(p + _CHUNK, pairs)) for p in range(0, pairs, _CHUNK)]
    if len(bounds) <= 1:
        for p0, p1 in bounds:
            _normal_pairs(p0, p1, seed, stream, core, z)
    else:
        import concurrent.futures
        import os

        with concurrent.futures.ThreadPoolExecutor(min(len(bounds), os.cpu_count() or 1)) as ex:
            list(ex.map(lambda b: _normal_pairs(b[0], b[1], seed, stream, core, z), bounds))
    return z[:count]


@dataclasses.dataclass
class TT:
    """A TT tensor on the host: N cores, core n is R[n] x I[n] x R[n+1].

    Each core is a flat 1-D array; entry (a, i, b) of core n sits at
    a + R[n] * (i + I[n] * b) (first rank fastest, then the mode index).
    """

    I: List[int]
    R: List[int]
    cores: List[np.ndarray]

    @property
    def N(self) -> int:
        return len(self.I)

    def core3(self, n: int) -> np.ndarray:
        """Core n as an (R[n], I[n], R[n+1]) view (Fortran order)."""
        return self.cores[n].reshape((self.R[n], self.I[n], self.R[n + 1]), order="F")

    def flat(self) -> np.ndarray:
        return np.concatenate([c.ravel() for c in self.cores])

    @property
    def nbytes(self) -> int:
        return sum(c.nbytes for c in self.cores)

    def astype(self, dtype) -> "TT":
        return TT(list(self.I), list(self.R), [np.ascontiguousarray(c, dtype=dtype) for c in self.cores])


def core_sizes(I: Sequence[int], R: Sequence[int]) -> List[int]:
    return [int(R[n]) * int(I[n]) * int(R[n + 1]) for n in range(len(I))]


def from_flat(I: Sequence[int], R: Sequence[int], flat: np.ndarray) -> TT:
    cores, off = [], 0
    for s in core_sizes(I, R):
        cores.append(np.array(flat[off:off + s], copy=True))
        off += s
    return TT(list(map(int, I)), list(map(int, R)), cores)


def random_tt(I: Sequence[int], R: Sequence[int], seed: int, stream: int = 0) -> TT:
    """Random TT with entries N(0,1)/sqrt(I_n R_{n-1}) (FP64)."""
    I = [int(x) for x in I]
    R = [int(x) for x in R]
    assert len(R) == len(I) + 1 and R[0] == 1 and R[-1] == 1
    cores = []
    for n in range(len(I)):
        cnt = R[n] * I[n] * R[n + 1]
        cores.append(normals(cnt, seed, stream, n) / np.sqrt(I[n] * R[n]))
    return TT(I, R, cores)


def uniform_ranks(N: int, r: int) -> List[int]:
    return [1] + [r] * (N - 1) + [1]


# --------------------------------------------------------------------------------------
# Workload recipes.  Each returns components; the consumer sums them with its own tt_add.
# --------------------------------------------------------------------------------------

BASE_SEED = 2011065300


def perturbed_pair(I: Sequence[int], r: int, seed: int, stream: int = 0):
    """(Y, Y') with Y a random rank-r TT and Y' = 0.5 Y + 1e-9 Z taken core-wise.

    Core-wise reading: Y'_1 = 0.5 Y_1 + 1e-9 Z_1 and Y'_n = Y_n + 1e-9 Z_n for
    n >= 2, Z an independent rank-r TT drawn with seed + 1000.  Y' stays rank r
    and is close to 0.5 Y, so X = Y + Y' has formal ranks 2r and numerical
    ranks r (plus perturbation terms of order 1e-18).
    """
    N = len(I)
    R = uniform_ranks(N, r)
    Y = random_tt(I, R, seed, stream)
    Z = random_tt(I, R, seed + 1000, stream)
    cores = []
    for n in range(N):
        scale = 0.5 if n == 0 else 1.0
        cores.append(scale * Y.cores[n] + 1e-9 * Z.cores[n])
    return Y, TT(list(Y.I), list(R), cores)


def config_small(seed: int = BASE_SEED + 1):
    """N=6, I_n=32, rank-5 Y, formal ranks 10 after X = Y + Y'; eps = 1e-6."""
    return perturbed_pair([32] * 6, 5, seed), 1e-6


def config_large_modes(I: int = 65536, seed: int = BASE_SEED + 2):
    """N=10, I_n=65536, rank-16 Y, formal ranks 32; eps = 1e-8."""
    return perturbed_pair([I] * 10, 16, seed), 1e-8


def decaying_terms(N: int, I: int, seed: int, r: int = 16, terms: int = 4, stream: int = 0):
    """Components T_0..T_{terms-1} of the decaying-spectrum workload.

    Each T_j is a random rank-r TT whose interior cores have V-unfolding
    G diag(d_k), d_k = 10^(-k/8) / nu (k = 0..r-1, nu makes rms(d) = 1), and whose
    first core is scaled by 10^(-2j).  Summed (by the consumer) they give formal
    ranks terms*r with cut spectra close to 10^(-m/8), m = 0..terms*r-1.
    """
    R = uniform_ranks(N, r)
    d = 10.0 ** (-np.arange(r) / 8.0)
    d = d / np.sqrt(np.mean(d * d))
    out = []
    for j in range(terms):
        T = random_tt([I] * N, R, seed + 7 * j, stream)
        for n in range(N):
            c = T.core3(n)
            if 0 < n < N - 1:
                c = c * d[None, None, :]
            if n == 0:
                c = c * 10.0 ** (-2 * j)
            T.cores[n] = np.asfortranarray(c).ravel(order="F")
        out.append(T)
    return out


def config_decaying(N: int = 50, I: int = 16384, seed: int = BASE_SEED + 3):
    return decaying_terms(N, I, seed), 1e-5


def uniforms(count: int, seed: int, stream: int, core: int) -> np.ndarray:
    """`count` uniforms in [0, 1) with 53 random bits each."""
    pairs = (count + 1) // 2
    idx = np.arange(pairs, dtype=np.uint64)
    ctr = np.empty((pairs, 4), dtype=np.uint32)
    ctr[:, 0] = (idx & _MASK32).astype(np.uint32)
    ctr[:, 1] = (idx >> np.uint64(32)).astype(np.uint32)
    ctr[:, 2] = np.uint32(core & 0xFFFFFFFF)
    ctr[:, 3] = np.uint32(1)
    out = philox4x32_10(ctr, (seed & 0xFFFFFFFF, stream & 0xFFFFFFFF)).astype(np.uint64)
    u = np.empty(2 * pairs, dtype=np.float64)
    u[0::2] = (((out[:, 0] << np.uint64(32)) | out[:, 1]) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
    u[1::2] = (((out[:, 2] << np.uint64(32)) | out[:, 3]) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
    return u[:count]


def uniform_int(u: float, lo: int, hi: int) -> int:
    """Map a uniform in [0, 1) to an integer uniform on {lo, ..., hi}."""
    return lo + min(hi - lo, int(u * (hi - lo + 1)))


def batched_shapes(count: int = 512, seed: int = BASE_SEED + 4):
    """Per-TT (I list, r) for the batched workload: N ~ U{4..20}, I_n ~ U{64..4096},
    r ~ U{4..48} (doubled later by Y + Y')."""
    shapes = []
    for t in range(count):
        u = uniforms(22, seed, 1 << 20, t)
        N = uniform_int(u[0], 4, 20)
        r = uniform_int(u[1], 4, 48)
        shapes.append(([uniform_int(u[2 + n], 64, 4096) for n in range(N)], r))
    return shapes


def batched_member(t: int, count: int = 512, seed: int = BASE_SEED + 4):
    Is, r = batched_shapes(count, seed)[t]
    return perturbed_pair(Is, r, seed + 17, stream=t), 1e-6


def device_random_tt(I: Sequence[int], R: Sequence[int], seed: int, device="cuda"):
    """Random TT cores drawn on the GPU with torch's seeded Philox generator, for timing
    runs whose inputs are too large to draw on the host in reasonable time.  Entries are
    N(0,1)/sqrt(I_n R_{n-1}) like random_tt, but the values differ from the host
    generator's, so these inputs are never used where the oracle is compared.
    Returns (I, R, cores) with cores as flat float64 CUDA tensors."""
    import torch

    gen = torch.Generator(device=device)
    gen.manual_seed(seed)
    I = [int(x) for x in I]
    R = [int(x) for x in R]
    cores = [torch.randn(R[n] * I[n] * R[n + 1], generator=gen, device=device, dtype=torch.float64)
             / float(np.sqrt(I[n] * R[n])) for n in range(len(I))]
    return I, R, cores


def device_perturbed_pair(I: Sequence[int], r: int, seed: int, device="cuda"):
    """Device-drawn (Y, Y') of the perturbed-pair recipe (see perturbed_pair)."""
    N = len(I)
    R = uniform_ranks(N, r)
    _, _, Y = device_random_tt(I, R, seed, device)
    _, _, Z = device_random_tt(I, R, seed + 1000, device)
    Yp = [(0.5 if n == 0 else 1.0) * Y[n] + 1e-9 * Z[n] for n in range(N)]
    return (list(I), R, Y), (list(I), R, Yp)


def hadamard_pair_shapes(count: int = 64, seed: int = BASE_SEED + 5):
    """(r_A, r_B) per pair of the Hadamard pipeline recipe: U{4..12} each, pair 0 fixed 8 x 8."""
    out = [(8, 8)]
    for p in range(1, count):
        u = uniforms(2, seed, 1 << 22, p)
        out.append((uniform_int(u[0], 4, 12), uniform_int(u[1], 4, 12)))
    return out


def hadamard_pair(p: int, N: int = 30, I: int = 1024, count: int = 64, seed: int = BASE_SEED + 5):
    """Random TTs A_p, B_p (N modes of size I) with the ranks of hadamard_pair_shapes;
    the pipeline forms Z = A o B, rounds it, then takes <Y, Z> and ||Y||."""
    ra, rb = hadamard_pair_shapes(count, seed)[p]
    A = random_tt([I] * N, uniform_ranks(N, ra), seed + 2 * p, stream=1)
    B = random_tt([I] * N, uniform_ranks(N, rb), seed + 2 * p + 1, stream=2)
    return A, B
