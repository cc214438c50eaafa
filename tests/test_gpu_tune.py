"""GPU checks of the tile autotuner: tuning a single rounding and a batch leaves results
within the parity bar of the oracle (ranks identical; 1e-12 in FP64, 1e-6 in fp32x2),
records one entry per core class in the right context, and the tuned plans that later
calls pick up give the same ranks and stay within the bar."""
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
    ttgb.tune_clear()
    yield ttgb
    ttgb.tune_clear()


def down(y) -> TT:
    import paper_2011_06532_gb300 as ttgb

    return TT(list(y.I), list(y.R), ttgb.to_host(y))


def table(gpu):
    rows = [ln.split() for ln in gpu.tune_export().splitlines() if ln and not ln.startswith("#")]
    return [tuple(int(v) for v in r) for r in rows]


def test_autotune_single_rounding(gpu, orc):
    import torch

    Y, Yp = ttgen.perturbed_pair([3000, 1500, 2048, 900, 3000], 8, 2011065500)
    X = orc.tt_add(Y, Yp)
    ref, _ = orc.tt_round(X, 1e-6)
    dx = gpu.from_host(X.I, X.R, X.cores, dtype=torch.float64)
    gpu.tune_clear()
    y = gpu.autotune(dx, 1e-6, precision="fp64")
    got = down(y)
    assert got.R == ref.R and orc.rel_err(got, ref) <= 1e-12
    rows = table(gpu)
    # one entry per core class (here every core is its own class), FP64, single-rounding context
    assert len(rows) == X.N and all(r[0] == 1 and r[1] == 0 for r in rows)
    assert sorted(r[2] for r in rows) == sorted(X.I)
    # the tuned plans are what later calls use
    y2 = down(gpu.tt_round(dx, 1e-6, precision="fp64"))
    assert y2.R == ref.R and orc.rel_err(y2, ref) <= 1e-12
    assert abs(gpu.tt_norm(dx) - orc.tt_norm(X)) <= 1e-12 * orc.tt_norm(X)


def test_autotune_batch(gpu, orc):
    import torch

    from tests.test_gpu_batched import uneven_batch

    pairs = uneven_batch(24, 2011065501, max_I=2048)
    Xs = [orc.tt_add(Y, Yp) for Y, Yp in pairs]
    refs = [orc.tt_round(X, 1e-6)[0] for X in Xs]
    dxs = [gpu.from_host(X.I, X.R, X.cores, dtype=torch.float32) for X in Xs]
    gpu.tune_clear()
    b = gpu.Batch(dxs, [1e-6] * len(dxs), "fp32x2")
    b.autotune()
    rows = table(gpu)
    assert rows and all(r[0] == 2 and r[1] == 1 for r in rows)
    # a single P cap for the whole batch: every entry's P is min(cap, I)
    caps = {r[7] for r in rows if r[7] < r[2]}
    assert len(caps) <= 1
    for outs in (b.run(), None):
        if outs is None:
            b.enqueue()
            torch.cuda.synchronize()
            outs = b.outputs()
        for ref, o in zip(refs, outs):
            got = down(o)
            assert got.R == ref.R
            assert orc.rel_err(got, ref) <= 1e-6
    # batch entries do not touch single roundings
    y = down(gpu.tt_round(dxs[0], 1e-6, precision="fp32x2"))
    assert y.R == refs[0].R and orc.rel_err(y, refs[0]) <= 1e-6
