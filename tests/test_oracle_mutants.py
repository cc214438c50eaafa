"""Planted mistakes: every plausible slip in the oracle must fail at least one pin.

Each mutant is oracle.c with one textual change (a dropped term, a wrong sign,
a transposed operand, an off-by-one, a misplaced block), compiled into its own
library under a temporary directory.  The battery below uses only truths that
do not come from the oracle: brute-force slice products, numpy's LAPACK SVD,
and invariants the paper states.  The unmodified oracle must pass the battery;
every mutant must fail it.  All mutants keep every memory access in bounds.
"""
import os
import shutil
import subprocess
import sys

import numpy as np
import pytest

import oracle
import ttgen
from ttgen import TT

SRC = os.path.join(os.path.dirname(oracle.__file__), "oracle.c")

MUTANTS = {
    "push_dropped": ("    memcpy(P, T, sizeof(double) * (size_t)(M * k));\n    w->r[n] = k;",
                     "    (void)T;\n    w->r[n] = k;"),
    "push_transposed": ("s += P[row + M * a] * R[a2 + k * a];", "s += P[row + M * a] * R[a + k * a2];"),
    "delta_without_sqrt": ("core_size(w.I, w.r, 0), 1);\n  double delta = eps * nrm / sqrt((double)(N - 1));",
                           "core_size(w.I, w.r, 0), 1);\n  double delta = eps * nrm;"),
    "rank_rule_strict": ("if (t[l] <= d2) {", "if (t[l] < d2) {"),
    "rank_off_by_one": ("      L = l;\n      break;", "      L = l < k ? l + 1 : l;\n      break;"),
    "house_tau_sign": ("tau[j] = (beta - alpha) / beta;", "tau[j] = (alpha - beta) / beta;"),
    "jacobi_rotation_sign": ("bq[r] = s * x + c * y;", "bq[r] = -s * x + c * y;"),
    "jacobi_v_not_accumulated": ("vq[r] = s * x + c * y;", "vq[r] = y;"),
    "sigma_not_pushed": ("T[l + L * col] = S[l] * s;", "T[l + L * col] = s;"),
    "u_transposed": ("s += Q[row + m * j] * Ur[j + k * l];", "s += Q[row + m * j] * Ur[l + k * j];"),
    "hadamard_kron_order": ("Z[(p * rb0 + q) + r0 * (i + In * (s * rb1 + t))]",
                            "Z[(q * ra0 + p) + r0 * (i + In * (s * rb1 + t))]"),
    "add_block_misplaced": ("i64 row_shift = (n == 0) ? 0 : ra0;", "i64 row_shift = 0;"),
    "dot_sum_dropped": ("Wn[q + qy * s] += acc;", "Wn[q + qy * s] = acc;"),
    "left_push_transposed": ("s += R[a2 + k * a] * H[a + b * col];", "s += R[a + k * a2] * H[a + b * col];"),
    "lrl_norm_of_first_core": ("double nrm = norm2_pairwise(w.c[N - 1], core_size(w.I, w.r, N - 1), 1);",
                               "double nrm = norm2_pairwise(w.c[0], core_size(w.I, w.r, 0), 1);"),
    "lrl_sigma_not_pushed": ("T[row + M * l] = S[l] * s2;", "T[row + M * l] = s2;"),
    "lrl_u_transposed": ("for (i64 j = 0; j < k; ++j) s += Q[col + m * j] * Ur[j + k * l];\n          Xn[l + L * col]",
                         "for (i64 j = 0; j < k; ++j) s += Q[col + m * j] * Ur[l + k * j];\n          Xn[l + L * col]"),
}


def entry(x: TT, idx):
    v = np.ones((1, 1))
    for n, i in enumerate(idx):
        v = v @ x.core3(n)[:, i, :]
    return v[0, 0]


def full(x: TT):
    out = np.zeros(tuple(x.I))
    for idx in np.ndindex(*x.I):
        out[idx] = entry(x, idx)
    return out


def numpy_tt_svd_ranks_and_full(f, eps):
    """TT-SVD through numpy's LAPACK SVD, with the same delta rule (brute force)."""
    N = f.ndim
    delta = eps * np.linalg.norm(f) / np.sqrt(N - 1)
    C = f.reshape(f.shape[0], -1, order="F")
    ranks, r = [1], 1
    cores = []
    for n in range(N - 1):
        C = C.reshape(r * f.shape[n], -1, order="F")
        U, S, Vt = np.linalg.svd(C, full_matrices=False)
        tail = np.concatenate([np.cumsum((S ** 2)[::-1])[::-1], [0.0]])
        L = next(l for l in range(1, len(S) + 1) if tail[l] <= delta ** 2)
        cores.append(U[:, :L])
        C = S[:L, None] * Vt[:L]
        r = L
        ranks.append(L)
    ranks.append(1)
    # rebuild the full tensor from the numpy factors
    T = np.ones((1, 1))
    for n, U in enumerate(cores):
        T = (T @ U.reshape(T.shape[1], -1, order="F")).reshape(-1, U.shape[1], order="F") if n else U
    T = T @ C
    return ranks, T.reshape(f.shape, order="F")


def decaying_tt(I, r, seed, rate=0.5):
    N = len(I)
    x = ttgen.random_tt(I, ttgen.uniform_ranks(N, r), seed)
    for n in range(N - 1):
        c = x.core3(n) * (rate ** np.arange(r))[None, None, :]
        x.cores[n] = np.asfortranarray(c).ravel(order="F")
    return x


def battery(lib):
    """Returns a list of failed check names (empty when everything holds)."""
    failed = []
    rng = np.random.default_rng(2024)

    A = rng.standard_normal((30, 6))
    Q, R = oracle.qr(A, lib=lib)
    if not (np.abs(Q @ R - A).max() < 1e-12 and np.abs(Q.T @ Q - np.eye(6)).max() < 1e-12):
        failed.append("qr")

    s = np.array([5.0, 2.0, 1.0, 0.5, 1e-3, 1e-6, 1e-9, 1e-12])
    U0 = np.linalg.qr(rng.standard_normal((12, 8)))[0]
    V0 = np.linalg.qr(rng.standard_normal((8, 8)))[0]
    B = (U0 * s) @ V0.T
    try:
        U, S, V = oracle.svd(B, lib=lib)
        if not (np.allclose(S, s, rtol=1e-10, atol=1e-14) and np.abs((U * S) @ V.T - B).max() < 1e-12):
            failed.append("svd")
    except oracle.OracleError:
        failed.append("svd")

    I = [2, 3, 4, 3]
    x = ttgen.random_tt(I, [1, 2, 3, 2, 1], 5)
    y = ttgen.random_tt(I, [1, 3, 2, 4, 1], 6)
    fx, fy = full(x), full(y)
    if np.abs(full(oracle.tt_add(x, y, lib=lib)) - (fx + fy)).max() > 1e-12:
        failed.append("add")
    if np.abs(full(oracle.tt_hadamard(x, y, lib=lib)) - fx * fy).max() > 1e-12:
        failed.append("hadamard")
    if abs(oracle.tt_dot(x, y, lib=lib) - np.sum(fx * fy)) > 1e-12:
        failed.append("dot")

    for seed, eps in [(1, 1e-3), (2, 1e-1), (3, 1e-6)]:
        xt = decaying_tt([3, 4, 5, 4, 3], 6, 80 + seed)
        f = full(xt)
        try:
            yt, _ = oracle.tt_round(xt, eps, lib=lib)
        except oracle.OracleError:
            failed.append(f"round{seed}")
            continue
        ranks, fref = numpy_tt_svd_ranks_and_full(f, eps)
        ok = yt.R == ranks and np.abs(full(yt) - fref).max() < 1e-11 * np.linalg.norm(f)
        ok = ok and np.linalg.norm(full(yt) - f) <= eps * np.linalg.norm(f) * (1 + 1e-9)
        if not ok:
            failed.append(f"round{seed}")

    # left-orthonormalization and the LRL ordering: the TT-SVD of the mode-reversed tensor
    xl = ttgen.random_tt([4, 3, 5, 3], [1, 3, 4, 2, 1], 9)
    fl = full(xl)
    yl = oracle.tt_orth_left(xl, lib=lib)
    if np.abs(full(yl) - fl).max() > 1e-12 * np.linalg.norm(fl):
        failed.append("orth_left")
    for seed, eps in [(1, 1e-3), (2, 1e-1)]:
        xt = decaying_tt([3, 4, 5, 4, 3], 6, 90 + seed)
        f = full(xt)
        try:
            yt, _ = oracle.tt_round_lrl(xt, eps, lib=lib)
        except oracle.OracleError:
            failed.append(f"lrl{seed}")
            continue
        g = np.transpose(f, axes=tuple(range(f.ndim - 1, -1, -1)))
        ranks, fref = numpy_tt_svd_ranks_and_full(g, eps)
        fref = np.transpose(fref, axes=tuple(range(f.ndim - 1, -1, -1)))
        ok = yt.R == ranks[::-1] and np.abs(full(yt) - fref).max() < 1e-11 * np.linalg.norm(f)
        if not ok:
            failed.append(f"lrl{seed}")

    z = TT([3, 4, 2], [1, 2, 3, 1], [np.zeros(6), np.zeros(24), np.zeros(6)])
    try:
        if oracle.tt_round(z, 1e-6, lib=lib)[0].R != [1, 1, 1, 1]:
            failed.append("zero")
    except oracle.OracleError:
        failed.append("zero")
    return failed


@pytest.fixture(scope="module")
def mutant_dir(tmp_path_factory):
    return tmp_path_factory.mktemp("mutants")


def test_unmodified_oracle_passes_battery():
    assert battery(oracle.load()) == []


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, mutant_dir):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site for {name} not unique"
    d = mutant_dir / name
    d.mkdir()
    shutil.copy(SRC, d / "orig.c")
    (d / "oracle.c").write_text(src.replace(old, new))
    so = str(d / "liboracle.so")
    subprocess.run(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-o", so, str(d / "oracle.c"), "-lm"], check=True)
    # run the battery in a child process so that a mutant can never disturb this one
    code = ("import sys, oracle, tests.test_oracle_mutants as t; "
            f"f = t.battery(oracle.load({so!r})); print('FAILED', f); sys.exit(0 if f else 3)")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", code], cwd=root, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, f"planted mistake {name} was not caught: {r.stdout[-500:]} {r.stderr[-500:]}"
