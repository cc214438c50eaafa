"""GPU parity of the rounding of a Hadamard product formed on the fly (Sec. 3.2.2 followed by
Alg. 2): tt_round_hadamard(A, B) against the oracle's tt_round(tt_hadamard(A, B)), ranks
identical and relative error <= 1e-12 in FP64 (<= 1e-6 in fp32x2), and in FP64 bit for bit
the library's own tt_hadamard followed by tt_round (the same products, the same kernels).
"""
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


def down(y) -> TT:
    import paper_2011_06532_gb300 as ttgb

    return TT(list(y.I), list(y.R), ttgb.to_host(y))


def f32_exact(x: TT) -> TT:
    return TT(list(x.I), list(x.R), [c.astype(np.float32).astype(np.float64) for c in x.cores])


CASES = [
    # (N, I, ra, rb, eps)
    (6, 48, 8, 8, 1e-6),
    (5, 300, 5, 7, 1e-8),
    (4, 2000, 9, 6, 1e-10),
    (8, 512, 8, 8, 1e-6),
]


@pytest.mark.parametrize("N,I,ra,rb,eps", CASES)
def test_fused_fp64_vs_oracle_and_unfused(gpu, orc, N, I, ra, rb, eps):
    A = ttgen.random_tt([I] * N, ttgen.uniform_ranks(N, ra), 500 + N * ra, stream=1)
    B = ttgen.random_tt([I] * N, ttgen.uniform_ranks(N, rb), 600 + N * rb, stream=2)
    ref, _ = orc.tt_round(orc.tt_hadamard(A, B), eps)
    dA, dB = gpu.from_host(A.I, A.R, A.cores), gpu.from_host(B.I, B.R, B.cores)
    y = gpu.tt_round_hadamard(dA, dB, eps)
    got = down(y)
    assert got.R == ref.R, (got.R, ref.R)
    assert orc.rel_err(got, ref) <= 1e-12
    unfused = gpu.tt_round(gpu.tt_hadamard(dA, dB), eps)
    assert unfused.R == y.R
    for a, b in zip(unfused.cores, y.cores):
        assert bool((a == b).all())


def test_fused_fp32x2_vs_oracle(gpu, orc):
    import torch

    N, I = 8, 512
    A = f32_exact(ttgen.random_tt([I] * N, ttgen.uniform_ranks(N, 8), 701, stream=1))
    B = f32_exact(ttgen.random_tt([I] * N, ttgen.uniform_ranks(N, 8), 702, stream=2))
    ref, _ = orc.tt_round(orc.tt_hadamard(A, B), 1e-6)
    dA = gpu.from_host(A.I, A.R, A.cores, dtype=torch.float32)
    dB = gpu.from_host(B.I, B.R, B.cores, dtype=torch.float32)
    got = down(gpu.tt_round_hadamard(dA, dB, 1e-6, precision="fp32x2"))
    assert got.R == ref.R
    assert orc.rel_err(got, ref) <= 1e-6


def test_fused_pipeline_pair_below_fp32_range(gpu, orc):
    # the Hadamard pipeline's norm leaves the FP32 range (||A o B|| ~ I^(-N/2)): the fused
    # rounding carries it by the same exponent rescaling as the unfused one
    import torch

    N, I = 40, 128
    A = f32_exact(ttgen.random_tt([I] * N, ttgen.uniform_ranks(N, 4), ttgen.BASE_SEED + 11, stream=1))
    B = f32_exact(ttgen.random_tt([I] * N, ttgen.uniform_ranks(N, 4), ttgen.BASE_SEED + 12, stream=2))
    ref, _ = orc.tt_round(orc.tt_hadamard(A, B), 1e-6)
    for prec, dt, tol in (("fp64", torch.float64, 1e-12), ("fp32x2", torch.float32, 1e-6)):
        dA = gpu.from_host(A.I, A.R, A.cores, dtype=dt)
        dB = gpu.from_host(B.I, B.R, B.cores, dtype=dt)
        got = down(gpu.tt_round_hadamard(dA, dB, 1e-6, precision=prec))
        assert got.R == ref.R
        assert orc.rel_err(got, ref) <= tol, prec


def test_fused_single_core_and_shape_errors(gpu, orc):
    A = TT([7], [1, 1], [np.arange(7.0)])
    B = TT([7], [1, 1], [np.arange(7.0) + 1])
    got = down(gpu.tt_round_hadamard(gpu.from_host(A.I, A.R, A.cores), gpu.from_host(B.I, B.R, B.cores), 0.1))
    assert got.R == [1, 1] and np.array_equal(got.cores[0], A.cores[0] * B.cores[0])
    C = ttgen.random_tt([7, 5], [1, 2, 1], 9)
    D = ttgen.random_tt([7, 6], [1, 2, 1], 10)
    with pytest.raises(gpu.TTError) as e:
        gpu.tt_round_hadamard(gpu.from_host(C.I, C.R, C.cores), gpu.from_host(D.I, D.R, D.cores), 0.1)
    assert e.value.status == 1
