"""GPU parity: the CUDA TT rounding (through the C ABI) against the FP64 CPU oracle.

Ranks must be identical element by element; tensors agree to 1e-12 relative in FP64
(measured as ||Y_gpu - Y_orc|| / ||Y_orc|| with the oracle's orthonormalization norm
of the difference TT, Sec. 3.2.4).  Inputs are the seeded components from ttgen; each
side forms sums with its own tt_add.
"""
import numpy as np
import pytest

import ttgen
from ttgen import TT

pytestmark = pytest.mark.gpu

TOL64 = 1e-12


@pytest.fixture(scope="module")
def gpu():
    import torch

    import paper_2011_06532_gb300 as ttgb

    assert torch.cuda.is_available()
    ttgb.build()
    return ttgb


def up(ttgb, x: TT, dtype=None):
    import torch

    return ttgb.from_host(x.I, x.R, x.cores, dtype=dtype or torch.float64)


def down(y) -> TT:
    import paper_2011_06532_gb300 as ttgb

    return TT(list(y.I), list(y.R), ttgb.to_host(y))


def check_round(gpu, orc, x: TT, eps: float, tol=TOL64):
    ref, info = orc.tt_round(x, eps)
    out = gpu.tt_round(up(gpu, x), eps)
    got = down(out)
    assert got.R == ref.R, f"ranks {got.R} vs oracle {ref.R}"
    err = orc.rel_err(got, ref)
    assert err <= tol, f"rel err {err:.3e}"
    return got, ref, err


def decaying_tt(I, r, seed, rate=0.5):
    N = len(I)
    x = ttgen.random_tt(I, ttgen.uniform_ranks(N, r), seed)
    for n in range(N - 1):
        c = x.core3(n) * (rate ** np.arange(r))[None, None, :]
        x.cores[n] = np.asfortranarray(c).ravel(order="F")
    return x


def test_small_workload_parity(gpu, orc):
    (Y, Yp), eps = ttgen.config_small()
    X = orc.tt_add(Y, Yp)
    got, ref, err = check_round(gpu, orc, X, eps)
    assert got.R == [1, 5, 5, 5, 5, 5, 1]


def test_small_workload_with_gpu_sum(gpu, orc):
    # X formed on the device with the library's own tt_add
    (Y, Yp), eps = ttgen.config_small()
    dx = gpu.tt_add(up(gpu, Y), up(gpu, Yp))
    ref, _ = orc.tt_round(orc.tt_add(Y, Yp), eps)
    got = down(gpu.tt_round(dx, eps))
    assert got.R == ref.R
    assert orc.rel_err(got, ref) <= TOL64


@pytest.mark.parametrize("seed", [1, 2, 3, 4])
@pytest.mark.parametrize("eps", [1e-1, 1e-4, 1e-10])
def test_random_decaying_parity(gpu, orc, seed, eps):
    shapes = {1: [5, 7, 6, 4, 8], 2: [40, 3, 30], 3: [2, 9, 9, 2], 4: [64, 50, 70, 33, 20, 9]}
    x = decaying_tt(shapes[seed], 7 if seed != 4 else 12, 100 + seed)
    check_round(gpu, orc, x, eps)


def test_n2_and_wide_unfoldings(gpu, orc):
    check_round(gpu, orc, decaying_tt([30, 20], 9, 7), 1e-3)
    x = ttgen.random_tt([2, 3, 3, 2], [1, 5, 7, 5, 1], 94)  # every cut capped by the dimensions
    got, _, _ = check_round(gpu, orc, x, 1e-14)
    assert got.R == [1, 2, 6, 2, 1]


def test_eps_zero_keeps_numerical_rank(gpu, orc):
    x = ttgen.random_tt([3, 4, 3], [1, 3, 3, 1], 95)
    check_round(gpu, orc, x, 0.0)


def test_zero_tensor(gpu, orc):
    x = TT([6, 5, 4], [1, 3, 2, 1], [np.zeros(18), np.zeros(30), np.zeros(8)])
    out = gpu.tt_round(up(gpu, x), 1e-6)
    got = down(out)
    assert got.R == [1, 1, 1, 1]
    # Alg. 2 keeps U(:, 1) of a zero unfolding (a unit vector) and pushes Sigma = 0 on:
    # the first core is a unit column, the tensor is exactly zero
    assert abs(np.linalg.norm(got.cores[0]) - 1.0) < 1e-15
    assert np.all(orc.tt_full(got) == 0)
    ref, _ = orc.tt_round(x, 1e-6)
    assert ref.R == got.R and abs(np.linalg.norm(ref.cores[0]) - 1.0) < 1e-15


def test_single_core_copies(gpu, orc):
    x = TT([9], [1, 1], [np.arange(9.0)])
    got = down(gpu.tt_round(up(gpu, x), 0.3))
    assert got.R == [1, 1] and np.array_equal(got.cores[0], x.cores[0])


def test_x_plus_x_rounds_to_2x(gpu, orc):
    x = ttgen.random_tt([17, 9, 23, 5], [1, 4, 6, 3, 1], 96)
    xx = orc.tt_add(x, x)
    got = down(gpu.tt_round(up(gpu, xx), 1e-10))
    assert got.R == x.R
    assert orc.rel_err(got, orc.scale_first(x, 2.0)) <= TOL64


def test_many_tiles_and_ragged_tails(gpu, orc):
    # I = 4099 slices: several leaves per SM pair, ragged last tile of every leaf
    (Y, Yp), eps = ttgen.perturbed_pair([4099, 4099, 4099, 4099], 16, 2011065400), 1e-8
    X = orc.tt_add(Y, Yp)
    got, ref, err = check_round(gpu, orc, X, eps)
    assert got.R == [1, 16, 16, 16, 1]


def test_deterministic(gpu, orc):
    (Y, Yp), eps = ttgen.config_small()
    X = up(gpu, orc.tt_add(Y, Yp))
    a = gpu.tt_round(X, eps)
    b = gpu.tt_round(X, eps)
    assert a.R == b.R
    for ca, cb in zip(a.cores, b.cores):
        assert (ca == cb).all()


@pytest.mark.parametrize("core,value", [(0, np.nan), (1, np.nan), (2, np.inf), (3, -np.inf)])
def test_nonfinite_input_returns_numerical_status(gpu, orc, core, value):
    # A non-finite entry written on the host into one input core: the rounding runs to
    # the end (no kernel waits on a value) and reports TT_ERR_NUMERICAL.
    x = ttgen.random_tt([20, 30, 25, 10], [1, 4, 6, 5, 1], 97)
    x.cores[core] = x.cores[core].copy()
    x.cores[core][7] = value
    with pytest.raises(gpu.TTError) as e:
        gpu.tt_round(up(gpu, x), 1e-6)
    assert e.value.status == 4
    # the library stays usable afterwards
    ok = ttgen.random_tt([20, 30, 25, 10], [1, 4, 6, 5, 1], 98)
    check_round(gpu, orc, ok, 1e-6)
