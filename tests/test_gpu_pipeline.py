"""GPU parity of the TT-arithmetic pipeline: Z = A o B (Hadamard, Sec. 3.2.2), Y = round(Z,
1e-6) (Alg. 2), then <Y, Z> (Sec. 3.2.3) and ||Y|| (Sec. 3.2.4), in FP64 and in the fp32x2
mixed form.  Against the oracle at reduced mode sizes (ranks identical; Y within 1e-12 in
FP64 and 1e-6 in fp32x2; inner product and norm likewise relative); at the full size of
pair 0 (N=30, I_n=1024, ranks 8 x 8 = 64) the fp32x2 pipeline is checked against the FP64
GPU pipeline (oracle-verified at reduced sizes).  The reduced-size cases include the
recipe's largest product rank (12 x 12 = 144).

With unit-norm factors the product's norm is about I^(-N/2) (2^-150 at the full size,
2^-140 in the range test), below the FP32 range: the FP32-storage forms must carry it
through their power-of-two rescaling of the pushed factors and of the inner-product
contractions."""
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
    """The same TT with every core entry rounded to FP32, so that FP32 storage holds the
    oracle's input exactly (only the FP32 product cores of the Hadamard step round)."""
    return TT(list(x.I), list(x.R), [c.astype(np.float32).astype(np.float64) for c in x.cores])


def supported_pairs(k):
    # the first k pairs of the recipe plus its largest product rank (12 x 12 = 144)
    shapes = ttgen.hadamard_pair_shapes()
    big = max(range(len(shapes)), key=lambda p: shapes[p][0] * shapes[p][1])
    return sorted(set(list(range(k)) + [big]))


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32x2", 1e-6)])
def test_pipeline_reduced_size_vs_oracle(gpu, orc, prec, tol):
    import torch

    dt = torch.float64 if prec == "fp64" else torch.float32
    for p in supported_pairs(3):
        A, B = ttgen.hadamard_pair(p, N=6, I=48)
        if prec != "fp64":
            A, B = f32_exact(A), f32_exact(B)
        Z = orc.tt_hadamard(A, B)
        Y, _ = orc.tt_round(Z, 1e-6)
        dot_ref, nrm_ref = orc.tt_dot(Y, Z), orc.tt_norm(Y)
        dZ = gpu.tt_hadamard(gpu.from_host(A.I, A.R, A.cores, dtype=dt), gpu.from_host(B.I, B.R, B.cores, dtype=dt))
        if prec == "fp64":
            assert [np.array_equal(a, b) for a, b in zip(gpu.to_host(dZ), Z.cores)] == [True] * Z.N
        dY = gpu.tt_round(dZ, 1e-6, precision=prec)
        got = down(dY)
        assert got.R == Y.R
        assert orc.rel_err(got, Y) <= tol
        # FP64: the scalars to the plain-FP64 bar itself; the FP32-storage forms carry
        # the FP32 rounding of the stored cores into them, so they get a factor 10
        stol = tol if prec == "fp64" else tol * 10
        assert abs(gpu.tt_dot(dY, dZ) - dot_ref) <= stol * abs(dot_ref)
        assert abs(gpu.tt_norm(dY) - nrm_ref) <= stol * nrm_ref


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32x2", 1e-6), ("fp32", 1e-3)])
def test_pipeline_norm_below_fp32_range_vs_oracle(gpu, orc, prec, tol):
    import torch

    N, I = 40, 128
    A = ttgen.random_tt([I] * N, ttgen.uniform_ranks(N, 4), ttgen.BASE_SEED + 11, stream=1)
    B = ttgen.random_tt([I] * N, ttgen.uniform_ranks(N, 4), ttgen.BASE_SEED + 12, stream=2)
    A, B = f32_exact(A), f32_exact(B)
    Z = orc.tt_hadamard(A, B)
    Y, _ = orc.tt_round(Z, 1e-6)
    nrm_ref, dot_ref = orc.tt_norm(Y), orc.tt_dot(Y, Z)
    assert 0 < nrm_ref < 2.0 ** -126  # the tensor itself lies below the FP32 range
    dt = torch.float64 if prec == "fp64" else torch.float32
    dZ = gpu.tt_hadamard(gpu.from_host(A.I, A.R, A.cores, dtype=dt), gpu.from_host(B.I, B.R, B.cores, dtype=dt))
    dY = gpu.tt_round(dZ, 1e-6, precision=prec)
    got = down(dY)
    assert all(np.isfinite(c).all() for c in got.cores)
    if prec != "fp32":
        assert got.R == Y.R
        assert orc.rel_err(got, Y) <= tol
    else:
        # plain FP32 may pick different ranks at this eps; it must stay within its accuracy
        assert orc.rel_err(got, Z) <= 1e-6 + tol
    assert abs(gpu.tt_norm(dY) - nrm_ref) <= 10 * tol * nrm_ref
    assert abs(gpu.tt_dot(dY, dZ) - dot_ref) <= 10 * tol * abs(dot_ref)


def test_pipeline_full_size_pair0(gpu):
    import torch

    def neg_first(x):
        c = [t.clone() for t in x.cores]
        c[0] = -c[0]
        return gpu.DeviceTT(list(x.I), list(x.R), c)

    A, B = ttgen.hadamard_pair(0)
    A, B = f32_exact(A), f32_exact(B)
    res = {}
    for prec, dt in [("fp64", torch.float64), ("fp32x2", torch.float32)]:
        dZ = gpu.tt_hadamard(gpu.from_host(A.I, A.R, A.cores, dtype=dt), gpu.from_host(B.I, B.R, B.cores, dtype=dt))
        dY = gpu.tt_round(dZ, 1e-6, precision=prec)
        res[prec] = (dY, gpu.tt_dot(dY, dZ), gpu.tt_norm(dY))
    (y64, d64, n64), (y32, d32, n32) = res["fp64"], res["fp32x2"]
    assert y64.R == y32.R and max(y64.R) == 64
    y32d = gpu.DeviceTT(list(y32.I), list(y32.R), [c.double() for c in y32.cores])
    assert gpu.tt_norm(gpu.tt_add(y32d, neg_first(y64))) <= 1e-6 * n64
    assert abs(d32 - d64) <= 1e-6 * abs(d64)
    assert abs(n32 - n64) <= 1e-6 * n64
