"""GPU parity of the feeder operations (sum, Hadamard, inner product, norm) against
the FP64 oracle: sum and Hadamard are copies/products of input entries and must be
bit-exact; the inner product and norm agree to 1e-12 relative."""
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


def up(ttgb, x, dtype=None):
    import torch

    return ttgb.from_host(x.I, x.R, x.cores, dtype=dtype or torch.float64)


SHAPES = [([7, 5, 9, 4], [1, 3, 4, 2, 1], [1, 2, 5, 3, 1]), ([11], [1, 1], [1, 1]), ([300, 257], [1, 6, 1], [1, 4, 1]),
          ([64, 33, 17, 90, 5], [1, 8, 12, 7, 9, 1], [1, 5, 6, 11, 4, 1])]


@pytest.mark.parametrize("I,Ra,Rb", SHAPES)
def test_add_hadamard_bitexact(gpu, orc, I, Ra, Rb):
    a = ttgen.random_tt(I, Ra, 201)
    b = ttgen.random_tt(I, Rb, 202)
    for op_g, op_o in [(gpu.tt_add, orc.tt_add), (gpu.tt_hadamard, orc.tt_hadamard)]:
        got = op_g(up(gpu, a), up(gpu, b))
        ref = op_o(a, b)
        assert got.R == ref.R
        for cg, cr in zip(gpu.to_host(got), ref.cores):
            assert np.array_equal(cg, cr)


@pytest.mark.parametrize("I,Ra,Rb", SHAPES)
def test_dot_and_norm(gpu, orc, I, Ra, Rb):
    a = ttgen.random_tt(I, Ra, 203)
    b = ttgen.random_tt(I, Rb, 204)
    ref = orc.tt_dot(a, b)
    got = gpu.tt_dot(up(gpu, a), up(gpu, b))
    scale = np.sqrt(orc.tt_dot(a, a) * orc.tt_dot(b, b))
    assert abs(got - ref) <= 1e-12 * scale
    nref = orc.tt_norm(a)
    assert abs(gpu.tt_norm(up(gpu, a)) - nref) <= 1e-12 * nref


def test_dot_large_modes(gpu, orc):
    I = [20000, 3000, 20000]
    a = ttgen.random_tt(I, [1, 16, 16, 1], 205)
    b = ttgen.random_tt(I, [1, 8, 24, 1], 206)
    ref = orc.tt_dot(a, b)
    scale = np.sqrt(orc.tt_dot(a, a) * orc.tt_dot(b, b))
    assert abs(gpu.tt_dot(up(gpu, a), up(gpu, b)) - ref) <= 1e-12 * scale
    assert abs(gpu.tt_norm(up(gpu, a)) - orc.tt_norm(a)) <= 1e-12 * orc.tt_norm(a)


def test_norm_of_small_difference(gpu, orc):
    # Sec. 3.2.4: the orthonormalization norm does not cancel
    x = ttgen.random_tt([50, 40, 30], [1, 6, 5, 1], 207)
    d = orc.tt_add(x, orc.scale_first(x, -(1 + 1e-10)))
    ref = orc.tt_norm(d)
    # both sides carry an absolute error of order u ||x||, i.e. ~u/1e-10 relative to ||d||;
    # the inner-product route would lose all digits here (sqrt(u) ||x|| >> ||d||)
    assert abs(gpu.tt_norm(up(gpu, d)) - ref) <= 1e-4 * ref
