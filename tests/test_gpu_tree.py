"""GPU parity of the TSQR tree shapes: nodes that factor their children's triangles in one
interleaved pass (fan-in 4 up to rank 79, 3 up to 93), nodes that take short children one
by one (leaves holding fewer rows than the rank), binary trees at higher ranks (117; and
144, where the leaves' carried tile block and the SVD's rotation accumulator move to global
memory, as the Hadamard products of rank-12 TTs need), and applies split over column
chunks -- each against the oracle (ranks
identical, relative error <= 1e-12 in FP64, <= 1e-6 in fp32x2)."""
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


CASES = [
    # (I, R, eps): what the shape exercises
    ([64, 50, 64], [1, 32, 8, 1], 1e-6),          # 50 one-slice leaves of 8 rows < 32: short children, then full ones
    ([3000, 2500, 3000], [1, 24, 24, 1], 1e-6),   # fan-in 4, interleaved nodes at every level
    ([2000, 1800, 2000], [1, 60, 60, 1], 1e-6),   # fan-in 4 at rank 60
    ([900, 700, 900], [1, 80, 80, 1], 1e-6),      # fan-in 3 at rank 80, apply in column chunks
    ([5000, 37, 5000], [1, 40, 40, 1], 0.0),      # wide middle core (37 slices of 40 rows), eps = 0
    ([300, 260, 300], [1, 100, 100, 1], 1e-6),    # rank 100: leaf buffers spilled to the global scratch
    ([240, 200, 240], [1, 117, 117, 1], 1e-6),    # rank 117: shared memory holds the leaf tile only
    ([150, 130, 150], [1, 144, 144, 1], 1e-6),    # rank 144: carried tile block and SVD V in global memory
]


@pytest.mark.parametrize("I,R,eps", CASES)
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32x2", 1e-6)])
def test_tree_shapes_vs_oracle(gpu, orc, I, R, eps, prec, tol):
    import numpy as np
    import torch

    X = ttgen.random_tt(I, R, 2011065700 + sum(I) + R[1])
    if prec != "fp64":
        X = TT(list(X.I), list(X.R), [c.astype(np.float32).astype(np.float64) for c in X.cores])
    ref, _ = orc.tt_round(X, eps)
    dt = torch.float64 if prec == "fp64" else torch.float32
    y = gpu.tt_round(gpu.from_host(X.I, X.R, X.cores, dtype=dt), eps, precision=prec)
    got = down(y)
    assert got.R == ref.R
    assert orc.rel_err(got, ref) <= tol
