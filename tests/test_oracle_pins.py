"""Pins for the FP64 CPU oracle: each check ties it to something other than itself.

Sources of truth used here (never the oracle's own formula retyped):
  * hand-worked examples (tests/golden/hand_examples.json, each cited);
  * closed forms (rank-1 exp, rank-2 sin, rank-1 inner products);
  * brute force on tiny full tensors (entry-by-entry slice products, Sec. 2.1);
  * textbook identities (QR vs Cholesky of A^T A, SVD reconstruction,
    Eckart-Young for N = 2 through numpy's LAPACK SVD);
  * invariants the paper states (orthonormality definitions of Sec. 2.3, the
    Ensure clause of Alg. 2, norm identities of Sec. 2.3 and 3.2.4, gauge
    freedom Eq. nonunique, ranks of sums and Hadamard products).
"""
import json
import os

import numpy as np
import pytest

import ttgen
from ttgen import TT

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "hand_examples.json")))


def entry(x: TT, idx):
    """X(i_1..i_N) as the product of slices X_1(i_1) ... X_N(i_N) (Sec. 2.1)."""
    v = np.ones((1, 1))
    for n, i in enumerate(idx):
        v = v @ x.core3(n)[:, i, :]
    return v[0, 0]


def full_by_entries(x: TT):
    out = np.zeros(tuple(x.I))
    for idx in np.ndindex(*x.I):
        out[idx] = entry(x, idx)
    return out


def rand_orth(rng, m, k):
    q, r = np.linalg.qr(rng.standard_normal((m, k)))
    return q * np.sign(np.diag(r))


# ----------------------------------------------------------------------------------
# generator
# ----------------------------------------------------------------------------------

def test_philox_known_answers():
    # Known-answer vectors published with the Random123 reference implementation.
    k = ttgen.philox4x32_10
    assert list(k(np.zeros((1, 4), np.uint32), (0, 0))[0]) == [0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8]
    assert list(k(np.full((1, 4), 0xFFFFFFFF, np.uint32), (0xFFFFFFFF, 0xFFFFFFFF))[0]) == [
        0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD]
    ctr = np.array([[0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344]], np.uint32)
    assert list(k(ctr, (0xA4093822, 0x299F31D0))[0]) == [0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1]


def test_normals_moments():
    z = ttgen.normals(400000, 11, 0, 0)
    assert abs(z.mean()) < 0.01 and abs(z.std() - 1) < 0.01


# ----------------------------------------------------------------------------------
# Householder QR
# ----------------------------------------------------------------------------------

def test_qr_hand_example(orc):
    g = GOLD["qr_3x2"]
    Q, R = orc.qr(np.array(g["A"]))
    np.testing.assert_allclose(np.abs(R), np.array(g["abs_R"]), rtol=0, atol=1e-14)


@pytest.mark.parametrize("m,b", [(40, 7), (7, 7), (5, 9), (300, 32), (1, 4)])
def test_qr_factorization(orc, m, b):
    rng = np.random.default_rng(m * 100 + b)
    A = rng.standard_normal((m, b))
    Q, R = orc.qr(A)
    k = min(m, b)
    assert Q.shape == (m, k) and R.shape == (k, b)
    assert np.abs(Q @ R - A).max() <= 1e-14 * max(1, np.abs(A).max()) * np.sqrt(m)
    assert np.abs(Q.T @ Q - np.eye(k)).max() <= 1e-14 * np.sqrt(m)
    assert np.all(np.tril(R, -1) == 0)


def test_qr_matches_cholesky_of_gram(orc):
    # textbook: for full-rank A, R = D chol(A^T A)^T with D = diag(+-1)
    rng = np.random.default_rng(3)
    A = rng.standard_normal((60, 9))
    _, R = orc.qr(A)
    C = np.linalg.cholesky(A.T @ A).T
    D = np.sign(np.diag(R))
    np.testing.assert_allclose(D[:, None] * R, C, rtol=1e-12, atol=1e-12)


def test_qr_rank_deficient_q_is_orthonormal(orc):
    rng = np.random.default_rng(4)
    A = rng.standard_normal((50, 3)) @ rng.standard_normal((3, 8))  # rank 3, 8 columns
    Q, R = orc.qr(A)
    assert np.abs(Q.T @ Q - np.eye(8)).max() < 1e-13
    assert np.abs(Q @ R - A).max() < 1e-13


# ----------------------------------------------------------------------------------
# one-sided Jacobi SVD
# ----------------------------------------------------------------------------------

def test_svd_hand_example(orc):
    g = GOLD["svd_2x2"]
    _, S, _ = orc.svd(np.array(g["B"]))
    np.testing.assert_allclose(S, g["sigma"], rtol=1e-15)


@pytest.mark.parametrize("m,n", [(30, 12), (12, 12), (8, 20)])
def test_svd_known_spectrum(orc, m, n):
    rng = np.random.default_rng(m + 7 * n)
    k = min(m, n)
    s = np.sort(10.0 ** rng.uniform(-12, 2, size=k))[::-1]
    U0, V0 = rand_orth(rng, m, k), rand_orth(rng, n, k)
    B = (U0 * s) @ V0.T
    U, S, V = orc.svd(B)
    # relative accuracy for the well-resolved values, absolute u*||B|| for the rest
    err = np.abs(S - s)
    assert np.all(err <= 1e-13 * s + 1e-15 * s[0] * 10)
    assert np.abs(U.T @ U - np.eye(k)).max() < 1e-12
    assert np.abs(V.T @ V - np.eye(k)).max() < 1e-12
    assert np.abs((U * S) @ V.T - B).max() < 1e-13 * s[0]


def test_svd_matches_lapack_and_special_cases(orc):
    rng = np.random.default_rng(5)
    B = rng.standard_normal((25, 10))
    np.testing.assert_allclose(orc.svd(B)[1], np.linalg.svd(B, compute_uv=False), rtol=1e-13)
    u, v = rng.standard_normal(9), rng.standard_normal(6)
    S = orc.svd(np.outer(u, v))[1]  # rank 1
    assert abs(S[0] - np.linalg.norm(u) * np.linalg.norm(v)) < 1e-13 * S[0]
    assert np.all(S[1:] < 1e-14 * S[0])
    d = np.array([0.5, 3.0, 2.0, 7.0])  # diagonal, unsorted -> sorted values
    np.testing.assert_allclose(orc.svd(np.diag(d))[1], np.sort(d)[::-1], rtol=1e-15)


# ----------------------------------------------------------------------------------
# TT basic operations against brute force
# ----------------------------------------------------------------------------------

SMALL_SHAPES = [([3, 4, 2], [1, 2, 3, 1]), ([2, 3, 4, 3], [1, 2, 3, 2, 1]), ([5], [1, 1]), ([4, 3], [1, 3, 1])]


@pytest.mark.parametrize("I,R", SMALL_SHAPES)
def test_full_matches_slice_products(orc, I, R):
    x = ttgen.random_tt(I, R, 21)
    np.testing.assert_allclose(orc.tt_full(x), full_by_entries(x), rtol=1e-14, atol=1e-15)


@pytest.mark.parametrize("I,R", SMALL_SHAPES)
def test_add_hadamard_dot_bruteforce(orc, I, R):
    x = ttgen.random_tt(I, R, 31)
    R2 = [1] + [r + 1 for r in R[1:-1]] + [1]
    y = ttgen.random_tt(I, R2, 32)
    fx, fy = full_by_entries(x), full_by_entries(y)
    s = orc.tt_add(x, y)
    h = orc.tt_hadamard(x, y)
    if len(I) > 1:
        assert s.R == [1] + [a + b for a, b in zip(R[1:-1], R2[1:-1])] + [1]  # ranks add (Sec. 3.2.1)
    assert h.R == [a * b for a, b in zip(R, R2)]  # ranks multiply (Sec. 3.2.2)
    np.testing.assert_allclose(full_by_entries(s), fx + fy, rtol=1e-13, atol=1e-14)
    np.testing.assert_allclose(full_by_entries(h), fx * fy, rtol=1e-13, atol=1e-15)
    ref = float(np.sum(fx * fy))
    assert abs(orc.tt_dot(x, y) - ref) <= 1e-13 * max(1.0, abs(ref))
    assert abs(orc.tt_dot(x, y, two_step=True) - ref) <= 1e-13 * max(1.0, abs(ref))


def test_dot_rank1_hand_example(orc):
    g = GOLD["tt_inner_rank1"]
    mk = lambda vs: TT([len(v) for v in vs], [1] * (len(vs) + 1), [np.array(v, float) for v in vs])
    assert orc.tt_dot(mk(g["x"]), mk(g["y"])) == g["dot"]


def test_hadamard_with_ones_is_dot(orc):
    I = [4, 5, 3, 2]
    x = ttgen.random_tt(I, [1, 3, 2, 2, 1], 41)
    y = ttgen.random_tt(I, [1, 2, 4, 3, 1], 42)
    ones = TT(I, [1] * 5, [np.ones(i) for i in I])
    a = orc.tt_dot(orc.tt_hadamard(x, y), ones)
    assert abs(a - orc.tt_dot(x, y)) < 1e-13 * max(1, abs(a))


def test_dot_two_step_matches_recurrence_larger(orc):
    I = [40, 30, 20, 10]
    x = ttgen.random_tt(I, [1, 6, 7, 5, 1], 43)
    y = ttgen.random_tt(I, [1, 4, 9, 3, 1], 44)
    a, b = orc.tt_dot(x, y), orc.tt_dot(x, y, two_step=True)
    assert abs(a - b) < 1e-13 * max(1, abs(a))


# ----------------------------------------------------------------------------------
# orthonormalization and norm
# ----------------------------------------------------------------------------------

def test_right_orth_invariants(orc):
    I = [4, 6, 5, 3, 4]
    x = ttgen.random_tt(I, [1, 3, 5, 4, 2, 1], 51)
    y = orc.tt_orth_right(x)
    for n in range(1, x.N):
        H = y.cores[n].reshape((y.R[n], -1), order="F")
        assert np.abs(H @ H.T - np.eye(y.R[n])).max() < 1e-13  # Sec. 2.3 definition
    f = full_by_entries(x)
    np.testing.assert_allclose(full_by_entries(y), f, rtol=1e-12, atol=1e-14)  # Eq. nonunique
    assert abs(np.linalg.norm(y.cores[0]) - np.linalg.norm(f)) < 1e-13 * np.linalg.norm(f)  # Sec. 2.3
    assert abs(orc.tt_norm(x) - np.linalg.norm(f)) < 1e-13 * np.linalg.norm(f)


def test_left_orth_invariants(orc):
    # the mirror of Alg. 1 (Sec. 3.4): V(Y_n) has orthonormal columns for n < N-1 (Sec. 2.3),
    # the tensor is unchanged (Eq. nonunique) and ||X|| = ||Y_N||_F (Sec. 2.3, Sec. 3.2.4)
    I = [4, 6, 5, 3, 4]
    x = ttgen.random_tt(I, [1, 3, 5, 4, 2, 1], 53)
    y = orc.tt_orth_left(x)
    assert left_orth_err(y) < 1e-13
    f = full_by_entries(x)
    np.testing.assert_allclose(full_by_entries(y), f, rtol=1e-12, atol=1e-14)
    assert abs(np.linalg.norm(y.cores[-1]) - np.linalg.norm(f)) < 1e-13 * np.linalg.norm(f)
    # wide unfoldings: the first cut is capped by R_0 I_0 = 2
    z = orc.tt_orth_left(ttgen.random_tt([2, 3, 3, 2], [1, 5, 7, 5, 1], 54))
    assert z.R == [1, 2, 6, 5, 1]


def test_norm_ortho_accurate_for_small_norm(orc):
    # Sec. 3.2.4: the orthonormalization norm avoids the cancellation of <X,X>.
    x = ttgen.random_tt([8, 9, 7, 6], [1, 4, 5, 3, 1], 52)
    h = 1e-10
    d = orc.tt_add(x, orc.scale_first(x, -(1 + h)))  # exactly -h * X up to rounding of (1+h)
    expect = h * orc.tt_norm(x)
    assert abs(orc.tt_norm(d) - expect) < 1e-4 * expect


# ----------------------------------------------------------------------------------
# rounding (Alg. 2)
# ----------------------------------------------------------------------------------

def decaying_tt(I, r, seed, rate=0.5):
    """Random TT whose interior cores have columns scaled by rate^k (so truncation bites)."""
    N = len(I)
    x = ttgen.random_tt(I, ttgen.uniform_ranks(N, r), seed)
    for n in range(N - 1):
        c = x.core3(n) * (rate ** np.arange(r))[None, None, :]
        x.cores[n] = np.asfortranarray(c).ravel(order="F")
    return x


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


def test_round_hand_example_n2(orc):
    g = GOLD["round_matrix_n2"]
    A = np.array(g["A"])
    x = TT([3, 3], [1, 3, 1], [np.eye(3).ravel(order="F"), A.ravel(order="F")])  # X = I * A
    for case in g["cases"]:
        y, _ = orc.tt_round(x, case["eps"])
        assert y.R == case["ranks"]


@pytest.mark.parametrize("seed", [1, 2, 3])
@pytest.mark.parametrize("eps", [1e-1, 1e-3, 1e-8])
def test_round_matches_tt_svd_bruteforce(orc, seed, eps):
    I = [3, 4, 5, 4, 3] if seed != 2 else [6, 5, 6, 4]
    x = decaying_tt(I, 6, 60 + seed)
    f = full_by_entries(x)
    y, info = orc.tt_round(x, eps)
    z = orc.tt_svd(f, eps)
    assert y.R == z.R
    fy = full_by_entries(y)
    np.testing.assert_allclose(fy, full_by_entries(z), rtol=0, atol=1e-12 * np.linalg.norm(f))
    # Ensure clause of Alg. 2 and the exact error identity of nested orthogonal projections
    err = np.linalg.norm(fy - f)
    assert err <= eps * np.linalg.norm(f) * (1 + 1e-12) + 1e-14
    tails = float(np.sum(info.tails))
    if tails > 1e-20 * np.linalg.norm(f) ** 2:
        assert abs(err ** 2 - tails) <= 1e-8 * tails + 1e-26
    assert left_orth_err(y) < 1e-13


def reversed_tt_svd(f, eps):
    """Right-to-left TT-SVD of the full tensor f, through numpy's LAPACK SVD: the
    textbook left-to-right TT-SVD (sequential truncated SVDs of the unfoldings, same
    delta rule) of f with its modes in reverse order, then the modes put back."""
    g = np.transpose(f, axes=tuple(range(f.ndim - 1, -1, -1)))
    N = g.ndim
    delta = eps * np.linalg.norm(g) / np.sqrt(N - 1)
    C = g.reshape(g.shape[0], -1, order="F")
    ranks, r, Us = [1], 1, []
    for n in range(N - 1):
        C = C.reshape(r * g.shape[n], -1, order="F")
        U, S, Vt = np.linalg.svd(C, full_matrices=False)
        tail = np.concatenate([np.cumsum((S ** 2)[::-1])[::-1], [0.0]])
        L = next(l for l in range(1, len(S) + 1) if tail[l] <= delta ** 2)
        Us.append(U[:, :L])
        C = S[:L, None] * Vt[:L]
        r = L
        ranks.append(L)
    ranks.append(1)
    T = Us[0]
    for U in Us[1:]:
        T = (T @ U.reshape(T.shape[1], -1, order="F")).reshape(-1, U.shape[1], order="F")
    T = (T @ C).reshape(g.shape, order="F")
    return ranks[::-1], np.transpose(T, axes=tuple(range(N - 1, -1, -1)))


@pytest.mark.parametrize("seed", [1, 2, 3])
@pytest.mark.parametrize("eps", [1e-1, 1e-3, 1e-8])
def test_round_lrl_matches_reversed_tt_svd_bruteforce(orc, seed, eps):
    # LRL ordering (Sec. 3.4, Sec. 4.3.2): left-orthonormalization, then truncation from
    # the right; in exact arithmetic the TT-SVD of the mode-reversed tensor
    I = [3, 4, 5, 4, 3] if seed != 2 else [6, 5, 6, 4]
    x = decaying_tt(I, 6, 60 + seed)
    f = full_by_entries(x)
    y, info = orc.tt_round_lrl(x, eps)
    ranks, fref = reversed_tt_svd(f, eps)
    assert y.R == ranks
    fy = full_by_entries(y)
    np.testing.assert_allclose(fy, fref, rtol=0, atol=1e-12 * np.linalg.norm(f))
    err = np.linalg.norm(fy - f)
    assert err <= eps * np.linalg.norm(f) * (1 + 1e-12) + 1e-14  # Ensure clause of Alg. 2
    tails = float(np.sum(info.tails))
    if tails > 1e-20 * np.linalg.norm(f) ** 2:
        assert abs(err ** 2 - tails) <= 1e-8 * tails + 1e-26
    assert right_orth_err(y) < 1e-13  # truncation from the right leaves H(Y_n) row-orthonormal
    assert abs(info.nrm - np.linalg.norm(f)) < 1e-13 * np.linalg.norm(f)


def test_round_lrl_x_plus_x_and_n2(orc):
    x = ttgen.random_tt([5, 4, 6, 3], [1, 3, 4, 2, 1], 72)
    y, _ = orc.tt_round_lrl(orc.tt_add(x, x), 1e-10)
    assert y.R == x.R
    np.testing.assert_allclose(full_by_entries(y), 2 * full_by_entries(x), atol=1e-13)
    # N = 2: the Eckart-Young truncation of the matrix, whichever the ordering
    rng = np.random.default_rng(8)
    U0, V0 = rand_orth(rng, 20, 8), rand_orth(rng, 15, 8)
    s = 2.0 ** -np.arange(8)
    A = (U0 * s) @ V0.T
    xm = TT([20, 15], [1, 8, 1], [U0.ravel(order="F"), (s[:, None] * V0.T).ravel(order="F")])
    ym, _ = orc.tt_round_lrl(xm, 0.05)
    Ua, Sa, Vta = np.linalg.svd(A)
    delta = 0.05 * np.linalg.norm(A)
    tail = np.cumsum((Sa ** 2)[::-1])[::-1]
    L = next(l for l in range(1, len(Sa) + 1) if (tail[l] if l < len(Sa) else 0.0) <= delta ** 2)
    assert ym.R[1] == L
    np.testing.assert_allclose(full_by_entries(ym), (Ua[:, :L] * Sa[:L]) @ Vta[:L], atol=1e-13)


def test_round_n2_is_eckart_young(orc):
    rng = np.random.default_rng(7)
    U0, V0 = rand_orth(rng, 20, 8), rand_orth(rng, 15, 8)
    s = 2.0 ** -np.arange(8)
    A = (U0 * s) @ V0.T
    # X = U0 (diag(s) V0^T): core 1 is 1 x 20 x 8, core 2 is 8 x 15 x 1
    x = TT([20, 15], [1, 8, 1], [U0.ravel(order="F"), (s[:, None] * V0.T).ravel(order="F")])
    eps = 0.05
    y, _ = orc.tt_round(x, eps)
    Ua, Sa, Vta = np.linalg.svd(A)
    delta = eps * np.linalg.norm(A)
    tail = np.cumsum((Sa ** 2)[::-1])[::-1]
    L = next(l for l in range(1, len(Sa) + 1) if (tail[l] if l < len(Sa) else 0.0) <= delta ** 2)
    assert y.R[1] == L
    best = (Ua[:, :L] * Sa[:L]) @ Vta[:L]
    np.testing.assert_allclose(full_by_entries(y), best, atol=1e-13)


def test_round_x_plus_x_is_2x_same_ranks(orc):
    x = ttgen.random_tt([5, 4, 6, 3], [1, 3, 4, 2, 1], 71)
    y, _ = orc.tt_round(orc.tt_add(x, x), 1e-10)
    assert y.R == x.R
    np.testing.assert_allclose(full_by_entries(y), 2 * full_by_entries(x), atol=1e-13)


def test_round_2x_minus_x_recovers_ranks(orc):
    # Sec. 4.2: Y = 2X - X has doubled ranks; rounding brings them back.
    I = [7, 6, 8, 5, 6]
    x = ttgen.random_tt(I, [1, 3, 4, 4, 2, 1], 72)
    yy = orc.tt_add(orc.scale_first(x, 2.0), orc.scale_first(x, -1.0))
    assert yy.R == [1, 6, 8, 8, 4, 1]
    y, _ = orc.tt_round(yy, 1e-9)
    assert y.R == x.R
    assert orc.rel_err(y, x) < 1e-13


def grid_tt(fn_cores, N, n):
    xs = np.linspace(0.0, 1.0, n)
    return fn_cores(xs, N), xs


def exp_tt(xs, N):
    # rank 1: exp(sum x_i) = prod exp(x_i)
    return TT([len(xs)] * N, [1] * (N + 1), [np.exp(xs) for _ in range(N)])


def sin_tt(xs, N):
    # rank 2: [sin s, cos s] advanced by sin(a+b) = sin a cos b + cos a sin b
    n = len(xs)
    cores = []
    for k in range(N):
        s, c = np.sin(xs), np.cos(xs)
        if k == 0:
            cores.append(np.concatenate([s, c]))  # (1, n, 2): [sin x, cos x]
        elif k == N - 1:
            # [sin(S+x); cos(S+x)] -> sin(S+x) = sin S cos x + cos S sin x
            core = np.zeros((2, n, 1))
            core[0, :, 0] = c
            core[1, :, 0] = s
            cores.append(core.ravel(order="F"))
        else:
            core = np.zeros((2, n, 2))
            core[0, :, 0] = c   # sin(S+x) <- sin S cos x
            core[1, :, 0] = s   #          + cos S sin x
            core[0, :, 1] = -s  # cos(S+x) <- -sin S sin x
            core[1, :, 1] = c   #          + cos S cos x
            cores.append(core.ravel(order="F"))
    return TT([n] * N, [1] + [2] * (N - 1) + [1], cores)


@pytest.mark.parametrize("kind,rank", [("exp", 1), ("sin", 2)])
def test_round_closed_forms(orc, kind, rank):
    N, n = 5, 6
    x, xs = grid_tt(exp_tt if kind == "exp" else sin_tt, N, n)
    infl = orc.tt_add(x, x)  # formal ranks doubled
    y, _ = orc.tt_round(infl, 1e-12)
    assert y.R == [1] + [rank] * (N - 1) + [1]
    rng = np.random.default_rng(8)
    for _ in range(50):
        idx = tuple(int(v) for v in rng.integers(0, n, size=N))
        S = sum(xs[i] for i in idx)
        ref = 2 * (np.exp(S) if kind == "exp" else np.sin(S))
        assert abs(entry(y, idx) - ref) < 1e-13 * max(1.0, abs(ref)) * 4


def test_round_gauge_invariance(orc):
    rng = np.random.default_rng(9)
    x = decaying_tt([5, 6, 4, 5], 5, 91)
    y0, _ = orc.tt_round(x, 1e-3)
    # insert M and M^{-1} between cores 1 and 2 (Eq. nonunique)
    M = rng.standard_normal((5, 5)) + 3 * np.eye(5)
    c1 = x.core3(1)
    c2 = x.core3(2)
    c1n = np.einsum("aib,bc->aic", c1, M)
    c2n = np.einsum("cb,bid->cid", np.linalg.inv(M), c2)
    xg = TT(list(x.I), list(x.R), [x.cores[0], np.asfortranarray(c1n).ravel(order="F"),
                                    np.asfortranarray(c2n).ravel(order="F"), x.cores[3]])
    y1, _ = orc.tt_round(xg, 1e-3)
    assert y1.R == y0.R
    assert orc.rel_err(y1, y0) < 1e-12


def test_round_zero_tensor(orc):
    x = TT([3, 4, 2], [1, 2, 3, 1], [np.zeros(6), np.zeros(24), np.zeros(6)])
    y, info = orc.tt_round(x, 1e-6)
    assert y.R == [1, 1, 1, 1] and info.nrm == 0.0
    assert np.all(full_by_entries(y) == 0.0)


def test_round_n1_and_eps0(orc):
    x = TT([7], [1, 1], [np.arange(7.0)])
    y, _ = orc.tt_round(x, 0.5)
    assert y.R == [1, 1] and np.array_equal(y.cores[0], x.cores[0])
    # eps = 0 keeps everything that is not exactly zero; ranks capped by the dimensions
    x = ttgen.random_tt([2, 3, 2], [1, 4, 4, 1], 93)
    y, _ = orc.tt_round(x, 0.0)
    assert y.R == [1, 2, 2, 1]
    assert orc.rel_err(y, x) < 1e-14


def test_round_wide_unfoldings_cap_ranks(orc):
    x = ttgen.random_tt([2, 3, 3, 2], [1, 5, 7, 5, 1], 94)
    y, _ = orc.tt_round(x, 1e-14)
    assert y.R == [1, 2, 6, 2, 1]  # caps min(prod I_left, prod I_right): 2, 6, 2
    np.testing.assert_allclose(full_by_entries(y), full_by_entries(x), atol=1e-13)


def test_round_small_workload_recovers_rank(orc):
    (Y, Yp), eps = ttgen.config_small()
    X = orc.tt_add(Y, Yp)
    assert X.R == [1] + [10] * 5 + [1]
    out, info = orc.tt_round(X, eps)
    assert out.R == [1] + [5] * 5 + [1]
    assert orc.rel_err(out, X) <= eps
    # Ensure clause: the discarded mass is far below the budget for this input
    assert np.sqrt(np.sum(info.tails)) <= eps * info.nrm


def test_cost_model_constants():
    g = GOLD["cost_model"]
    c = lambda R, L: (3 * R * R + 6 * R * L + 4 * L * L) / R ** 2
    assert c(50, 25) == g["halved_constant"]
    assert c(50, 0) == g["min_constant"] and c(50, 50) == g["max_constant"]
    model1 = 48 * 50 * 2000 * 50 * 8 + 2 * 2000 * 50 * 8
    assert model1 == g["model1_bytes"]
