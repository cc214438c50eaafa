"""The algorithmic flop count behind bench.py's roofline numerator agrees with the paper's
cost of TT rounding (Sec. 3.5): one more interior core of uniform input rank R and output
rank L adds I R (3 R^2 + 6 R L + 4 L^2) flops -- 3 I R^3 for the orthogonalization (QR of
H(X_n)^T and the triangular push), 6 I R^2 L for the sweep-2 apply of Q_n and the QR of
V(Y_n), 4 I R L^2 for forming the output core."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def total(N, I, R, L):
    import bench

    f = bench.flops_by_kernel([I] * N, [1] + [R] * (N - 1) + [1], [1] + [L] * (N - 1) + [1])
    return sum(f.values())


@pytest.mark.parametrize("I,R,L", [(65536, 32, 16), (1000, 10, 7), (4096, 64, 48), (2000, 50, 25)])
def test_interior_core_cost_matches_the_paper(I, R, L):
    assert total(8, I, R, L) - total(7, I, R, L) == I * R * (3 * R * R + 6 * R * L + 4 * L * L)


def test_headline_flops_per_rounding():
    # the headline workload: N = 10, I = 65536, formal ranks 32 rounded to 16
    assert total(10, 65536, 32, 16) == pytest.approx(1.2086e11, rel=1e-3)
