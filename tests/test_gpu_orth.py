"""GPU parity of orthonormalization (Alg. 1 / Alg. 5 and the left-hand mirror) and of the
LRL ordering of rounding (Sec. 3.4, Sec. 4.3.2), through the C ABI, against the FP64
oracle.

Orthonormal factors are unique only up to signs (Eq. nonunique), so the checks compare
what is unique: the ranks (element by element), the represented tensor (relative error of
the difference, by the oracle's orthonormalization norm), the norm carried by the end
core, and the orthonormality of every other core (Sec. 2.3 definitions).
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


def right_orth_err(y: TT):
    e = 0.0
    for n in range(1, y.N):
        H = y.cores[n].reshape((y.R[n], -1), order="F")
        e = max(e, np.abs(H @ H.T - np.eye(y.R[n])).max())
    return e


def left_orth_err(y: TT):
    e = 0.0
    for n in range(y.N - 1):
        V = y.cores[n].reshape((y.R[n] * y.I[n], y.R[n + 1]), order="F")
        e = max(e, np.abs(V.T @ V - np.eye(y.R[n + 1])).max())
    return e


CASES = {
    "small": lambda: ttgen.random_tt([5, 7, 6, 4, 8], [1, 3, 5, 4, 2, 1], 401),
    "wide_caps": lambda: ttgen.random_tt([2, 3, 3, 2], [1, 5, 7, 5, 1], 402),
    "many_tiles": lambda: ttgen.random_tt([4099, 300, 4099], [1, 16, 24, 1], 403),
    "rank40": lambda: ttgen.random_tt([700, 900, 500, 60], [1, 40, 40, 30, 1], 404),
}


@pytest.mark.parametrize("side", ["right", "left"])
@pytest.mark.parametrize("case", sorted(CASES))
def test_orthonormalize_fp64_vs_oracle(gpu, orc, side, case):
    x = CASES[case]()
    ref = orc.tt_orth_right(x) if side == "right" else orc.tt_orth_left(x)
    got = down(gpu.tt_orthonormalize(up(gpu, x), side=side))
    assert got.R == ref.R, (got.R, ref.R)
    assert orc.rel_err(got, x) <= TOL64
    nrm = orc.tt_norm(x)
    end = got.cores[0] if side == "right" else got.cores[-1]
    assert abs(np.linalg.norm(end) - nrm) <= TOL64 * nrm
    assert (right_orth_err(got) if side == "right" else left_orth_err(got)) < 1e-13


@pytest.mark.parametrize("side", ["right", "left"])
def test_orthonormalize_fp32x2(gpu, orc, side):
    import torch

    x = CASES["many_tiles"]()
    x = TT(list(x.I), list(x.R), [c.astype(np.float32).astype(np.float64) for c in x.cores])
    got = down(gpu.tt_orthonormalize(up(gpu, x, torch.float32), side=side, precision="fp32x2"))
    ref = orc.tt_orth_right(x) if side == "right" else orc.tt_orth_left(x)
    assert got.R == ref.R
    assert orc.rel_err(got, x) <= 1e-6
    assert (right_orth_err(got) if side == "right" else left_orth_err(got)) < 1e-6


def test_orthonormalize_zero_and_single_core(gpu, orc):
    z = TT([6, 5, 4], [1, 3, 2, 1], [np.zeros(18), np.zeros(30), np.zeros(8)])
    for side in ("right", "left"):
        got = down(gpu.tt_orthonormalize(up(gpu, z), side=side))
        assert np.all(orc.tt_full(got) == 0)
        assert (right_orth_err(got) if side == "right" else left_orth_err(got)) < 1e-14
    one = TT([9], [1, 1], [np.arange(9.0)])
    got = down(gpu.tt_orthonormalize(up(gpu, one), side="left"))
    assert got.R == [1, 1] and np.array_equal(got.cores[0], one.cores[0])


def decaying_tt(I, r, seed, rate=0.5):
    N = len(I)
    x = ttgen.random_tt(I, ttgen.uniform_ranks(N, r), seed)
    for n in range(N - 1):
        c = x.core3(n) * (rate ** np.arange(r))[None, None, :]
        x.cores[n] = np.asfortranarray(c).ravel(order="F")
    return x


def lrl_cases():
    (Y, Yp), eps = ttgen.config_small()
    yield "small_workload", (Y, Yp), eps
    yield "many_tiles", ttgen.perturbed_pair([4099, 4099, 4099, 4099], 16, 2011065400), 1e-8
    for seed, eps in [(1, 1e-1), (2, 1e-4), (3, 1e-10)]:
        shapes = {1: [5, 7, 6, 4, 8], 2: [40, 3, 30], 3: [64, 50, 70, 33, 20, 9]}
        yield f"decaying{seed}", decaying_tt(shapes[seed], 7 if seed != 3 else 12, 110 + seed), eps


@pytest.mark.parametrize("name,spec,eps", list(lrl_cases()), ids=[c[0] for c in lrl_cases()])
def test_round_lrl_fp64_vs_oracle(gpu, orc, name, spec, eps):
    X = orc.tt_add(*spec) if isinstance(spec, tuple) else spec
    ref, _ = orc.tt_round_lrl(X, eps)
    got = down(gpu.tt_round(up(gpu, X), eps, order="lrl"))
    assert got.R == ref.R, (got.R, ref.R)
    assert orc.rel_err(got, ref) <= TOL64
    assert right_orth_err(got) < 1e-12  # truncated from the right: H(Y_n) row-orthonormal


def test_round_lrl_fp32x2_vs_oracle(gpu, orc):
    import torch

    Y, Yp = ttgen.perturbed_pair([4099, 4099, 4099, 4099], 16, 2011065400)
    X = orc.tt_add(Y, Yp)
    ref, _ = orc.tt_round_lrl(X, 1e-6)
    got = down(gpu.tt_round(up(gpu, X, torch.float32), 1e-6, precision="fp32x2", order="lrl"))
    assert got.R == ref.R
    assert orc.rel_err(got, ref) <= 1e-6


def test_round_orderings_both_meet_the_bound(gpu, orc):
    # RLR and LRL differ by O(delta) but both satisfy the Ensure clause of Alg. 2
    X = decaying_tt([30, 40, 35, 20], 10, 120)
    eps = 1e-3
    for order in ("rlr", "lrl"):
        got = down(gpu.tt_round(up(gpu, X), eps, order=order))
        assert orc.rel_err(got, X) <= eps * (1 + 1e-10)
