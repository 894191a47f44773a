"""Pins of the CPU oracle against what the paper and the mathematics fix.

These run without a GPU. They check the oracle against library routines
(NumPy matmul, SciPy's Hankel constructor, sliding-window views), exact
integer arithmetic, closed forms, invariants and the paper's printed counts,
and they show that plausible mistakes planted in a copy of the oracle's loop
are caught.
"""
import json
import os
from fractions import Fraction

import numpy as np
import pytest

import cov_workloads as wl
from oracle import algorithm1, combinations as cb, exact

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------------------------
# Library brute force: X built with NumPy's sliding-window view (column stack,
# Eq. 2.1) and R = X X^H / K with NumPy's matmul.
# ----------------------------------------------------------------------------
def brute_force(A, P, Q, mean=True):
    A = np.asarray(A, np.complex128)
    W = np.lib.stride_tricks.sliding_window_view(A, (P, Q))  # [p, q, i, j]
    X = W.transpose(0, 1, 3, 2).reshape(-1, P * Q).T          # x[i + P j]
    R = X @ X.conj().T
    return R / X.shape[1] if mean else R


def rel_err(X, Y):
    return float(np.linalg.norm(X - Y) / max(np.linalg.norm(Y), 1e-300))


SMALL_SHAPES = [(N, M, P, Q) for N in (1, 2, 3, 5, 7) for M in (1, 2, 4, 6)
                for P in range(1, N + 1) for Q in range(1, M + 1)]


@pytest.mark.parametrize("N,M,P,Q", SMALL_SHAPES)
def test_oracle_matches_numpy_bruteforce(oracle_mod, N, M, P, Q):
    for seed in (0, 1, 2):
        A = wl.complex_normal((N, M), 1000 + seed)
        R = oracle_mod.cov_window(A, P, Q)
        assert rel_err(R, brute_force(A, P, Q)) < 1e-14
        Rs = oracle_mod.cov_window(A, P, Q, mean=False)
        assert rel_err(Rs, brute_force(A, P, Q, mean=False)) < 1e-14


def test_oracle_exhaustive_up_to_10x10(oracle_mod):
    # every shape N, M <= 10 and every window P <= N, Q <= M, three seeds
    for N in range(1, 11):
        for M in range(1, 11):
            for seed in (0, 1, 2):
                A = wl.complex_normal((N, M), 2000 + 100 * N + 10 * M + seed)
                for P in range(1, N + 1):
                    for Q in range(1, M + 1):
                        assert rel_err(oracle_mod.cov_window(A, P, Q), brute_force(A, P, Q)) < 1e-14, \
                            (N, M, P, Q, seed)


def test_oracle_matches_bruteforce_medium(oracle_mod):
    A = wl.complex_normal((40, 33), 7)
    for P, Q in ((8, 8), (5, 11), (13, 2)):
        assert rel_err(oracle_mod.cov_window(A, P, Q), brute_force(A, P, Q)) < 1e-13


# ----------------------------------------------------------------------------
# Exact integer arithmetic.
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("N,M,P,Q", [(6, 5, 2, 3), (7, 7, 3, 3), (9, 4, 4, 2), (5, 8, 5, 1)])
def test_integer_inputs_exact(oracle_mod, N, M, P, Q):
    A = wl.integer_valued((N, M), 2285 + N * M)
    are = [[int(v) for v in row] for row in A.real]
    aim = [[int(v) for v in row] for row in A.imag]
    Cre, Cim = exact.window_sum_exact(are, aim, P, Q)
    S = oracle_mod.cov_window(A, P, Q, mean=False)
    assert np.array_equal(S.real, np.array(Cre, float))
    assert np.array_equal(S.imag, np.array(Cim, float))
    R = oracle_mod.cov_window(A, P, Q, mean=True)
    K = (N - P + 1) * (M - Q + 1)
    # the exact mean (Fractions) rounded once to FP64 is what an exact sum
    # followed by one IEEE division by K gives
    Fre, Fim = exact.covariance_exact(are, aim, P, Q, mean=True)
    for row_f, row_c in zip(Fre, Cre):
        assert row_f == [Fraction(v, K) for v in row_c]
    assert np.array_equal(R.real, np.array([[float(v) for v in row] for row in Fre]))
    assert np.array_equal(R.imag, np.array([[float(v) for v in row] for row in Fim]))
    Sre, Sim = exact.covariance_exact(are, aim, P, Q, mean=False)
    assert (Sre, Sim) == (Cre, Cim)


@pytest.mark.parametrize("N,M,P,Q", [(6, 5, 2, 3), (8, 9, 3, 4), (10, 4, 10, 1)])
def test_exact_window_sum_matches_integer_bruteforce(N, M, P, Q):
    # NumPy int64 products of the explicitly built window matrix: exact
    A = wl.integer_valued((N, M), 77 + N * M)
    W = np.lib.stride_tricks.sliding_window_view(A, (P, Q)).transpose(0, 1, 3, 2)
    X = W.reshape(-1, P * Q).T
    Xr, Xi = X.real.astype(np.int64), X.imag.astype(np.int64)
    want_re = Xr @ Xr.T + Xi @ Xi.T         # Re(x_a conj(x_b))
    want_im = Xi @ Xr.T - Xr @ Xi.T         # Im(x_a conj(x_b))
    Cre, Cim = exact.window_sum_exact([[int(v) for v in r] for r in A.real],
                                      [[int(v) for v in r] for r in A.imag], P, Q)
    assert np.array_equal(np.array(Cre, dtype=np.int64), want_re)
    assert np.array_equal(np.array(Cim, dtype=np.int64), want_im)


# ----------------------------------------------------------------------------
# Closed forms.
# ----------------------------------------------------------------------------
def test_constant_input(oracle_mod):
    A = np.full((9, 7), 3 + 4j)
    for P, Q in ((1, 1), (3, 2), (9, 7), (4, 5)):
        R = oracle_mod.cov_window(A, P, Q)
        assert np.array_equal(R, np.full((P * Q, P * Q), 25.0 + 0j))


def test_single_exponential_is_rank_one(oracle_mod):
    c, om, nu = 0.7 - 1.3j, 0.9, -2.1
    A = wl.single_exponential(23, 19, c, om, nu)
    for P, Q in ((4, 3), (6, 6), (1, 5)):
        i = np.arange(P * Q) % P
        j = np.arange(P * Q) // P
        v = np.exp(1j * (om * i + nu * j))
        want = abs(c) ** 2 * np.outer(v, v.conj())
        assert rel_err(oracle_mod.cov_window(A, P, Q), want) < 3e-15 * 10


def test_window_1x1_is_mean_power(oracle_mod):
    A = wl.complex_normal((11, 13), 5)
    R = oracle_mod.cov_window(A, 1, 1)
    assert R.shape == (1, 1)
    assert abs(R[0, 0] - np.mean(np.abs(A) ** 2)) < 1e-14 * np.mean(np.abs(A) ** 2)
    assert R[0, 0].imag == 0.0


def test_full_window_is_outer_product(oracle_mod):
    A = wl.integer_valued((4, 3), 9)
    v = A.flatten(order="F")  # column stack, Eq. 2.1
    assert np.array_equal(oracle_mod.cov_window(A, 4, 3), np.outer(v, v.conj()))


def test_one_dimensional_case_is_hankel_product(oracle_mod):
    from scipy.linalg import hankel
    a = wl.complex_normal((37,), 11)
    for P in (1, 5, 12, 37):
        H = hankel(a[:P], a[P - 1:])      # H[i, k] = a[i + k]
        want = H @ H.conj().T / H.shape[1]
        got = oracle_mod.cov_window(a[:, None], P, 1)
        assert rel_err(got, want) < 1e-14


# ----------------------------------------------------------------------------
# Invariants.
# ----------------------------------------------------------------------------
def test_hermitian_and_psd(oracle_mod):
    A = wl.complex_normal((30, 26), 17)
    for P, Q in ((5, 5), (8, 3), (2, 9)):
        R = oracle_mod.cov_window(A, P, Q)
        assert np.array_equal(R, R.conj().T)
        assert np.all(R.diagonal().imag == 0)
        lam = np.linalg.eigvalsh(R)
        assert lam.min() >= -1e-12 * np.linalg.norm(R, 2)


def test_scaling_modulation_conjugation_transpose(oracle_mod):
    A = wl.complex_normal((17, 21), 23)
    P, Q = 4, 6
    R = oracle_mod.cov_window(A, P, Q)
    c = 1.5 - 0.25j
    assert rel_err(oracle_mod.cov_window(c * A, P, Q), abs(c) ** 2 * R) < 1e-14
    om, nu = 0.3, -1.1
    mod = wl.single_exponential(17, 21, 1.0, om, nu)
    i = np.arange(P * Q) % P
    j = np.arange(P * Q) // P
    Dg = np.diag(np.exp(1j * (om * i + nu * j)))
    assert rel_err(oracle_mod.cov_window(A * mod, P, Q), Dg @ R @ Dg.conj().T) < 1e-13
    assert np.array_equal(oracle_mod.cov_window(A.conj(), P, Q), R.conj())
    # transposing A and swapping P, Q permutes x: x^T[j + Q i] = x[i + P j]
    perm = np.array([(a // Q) + P * (a % Q) for a in range(P * Q)])
    RT = oracle_mod.cov_window(A.T, Q, P)
    assert rel_err(RT, R[np.ix_(perm, perm)]) < 1e-14


def test_element_and_threads_bit_identical(oracle_mod):
    A = wl.complex_normal((20, 18), 31)
    P, Q = 5, 4
    R1 = oracle_mod.cov_window(A, P, Q, threads=1)
    R4 = oracle_mod.cov_window(A, P, Q, threads=4)
    assert np.array_equal(R1, R4)
    rng = np.random.default_rng(0)
    for _ in range(40):
        a, b = (int(v) for v in rng.integers(0, P * Q, 2))
        assert oracle_mod.cov_element(A, P, Q, a, b) == R1[a, b]


# ----------------------------------------------------------------------------
# The paper's counts and the two theorems of Section 4.
# ----------------------------------------------------------------------------
def test_paper_printed_counts():
    with open(os.path.join(GOLDEN, "paper_counts.json")) as f:
        g = json.load(f)
    for e in g["unique_combinations"]:
        assert cb.n_unique_combinations(e["P"], e["Q"]) == e["count"]
        assert len(cb.unique_combinations(e["P"], e["Q"])) == e["count"]
    for e in g["sm_over_um_hat"]:
        assert cb.sm_over_um_hat(e["N"], e["M"], e["P"], e["Q"]) == Fraction(e["value"])


def test_sm_naive_against_the_printed_ratio_and_a_count():
    # Eq. 4.1 over the upper bound of Eq. 4.7 is the ratio of Eq. 4.8, and the
    # paper prints its value 45.125 for N = M = 32, P = Q = 13 (Eq. 4.9)
    with open(os.path.join(GOLDEN, "paper_counts.json")) as f:
        g = json.load(f)
    for e in g["sm_over_um_hat"]:
        N, M, P, Q = e["N"], e["M"], e["P"], e["Q"]
        assert Fraction(cb.sm_naive(N, M, P, Q)) / cb.um_hat(N, M, P, Q) == Fraction(e["value"])
    for N, M, P, Q in ((20, 20, 8, 8), (64, 64, 8, 8), (37, 11, 5, 9), (1024, 1024, 16, 16)):
        assert Fraction(cb.sm_naive(N, M, P, Q)) / cb.um_hat(N, M, P, Q) == \
            cb.sm_over_um_hat(N, M, P, Q)

    # a count of the multiplications that forming every outer product x x^H
    # makes, over the positions Section 4.1 counts (N - P down, M - Q right)
    class Counted:
        n = 0

        def __init__(self, v):
            self.v = v

        def __mul__(self, other):
            Counted.n += 1
            return Counted(self.v * other.v)

        def conjugate(self):
            return Counted(self.v.conjugate())

    for N, M, P, Q in ((5, 4, 2, 2), (6, 7, 3, 2), (4, 4, 1, 3)):
        Counted.n = 0
        A = wl.complex_normal((N, M), 5)
        for p in range(N - P):
            for q in range(M - Q):
                x = np.array([Counted(complex(A[p + a % P, q + a // P])) for a in range(P * Q)],
                             dtype=object)
                np.outer(x, np.conjugate(x))
        assert Counted.n == cb.sm_naive(N, M, P, Q)


@pytest.mark.parametrize("N,M,P,Q", [(64, 64, 8, 8), (1024, 1024, 16, 16),
                                     (2048, 512, 32, 32), (256, 256, 12, 12),
                                     (37, 11, 5, 9), (9, 9, 9, 9)])
def test_um_closed_form(N, M, P, Q):
    assert cb.um_closed_form(N, M, P, Q) == cb.um_enumerated(N, M, P, Q)
    assert cb.um_enumerated(N, M, P, Q) <= cb.um_hat(N, M, P, Q)


def test_um_of_the_workloads():
    assert cb.um_enumerated(64, 64, 8, 8) == 410_656
    assert cb.um_enumerated(1024, 1024, 16, 16) == 496_775_296
    assert cb.um_enumerated(2048, 512, 32, 32) == 2_001_920_512


@pytest.mark.parametrize("P,Q", [(p, q) for p in range(1, 8) for q in range(1, 8)])
def test_collision_freedom_and_coverage(P, Q):
    seen = {}
    total = 0
    for dr, dc in cb.unique_combinations(P, Q):
        idx = cb.write_indices(P, Q, dr, dc)
        assert len(idx) == cb.eta(P, Q, dr, dc)
        total += len(idx)
        for ab in idx:
            assert ab not in seen, (ab, seen.get(ab), (dr, dc))   # Section 4.2
            seen[ab] = (dr, dc)
            assert cb.combination_of_index(P, *ab) == (dr, dc)
    D = P * Q
    assert total == D * (D + 1) // 2                              # Eq. 4.22
    assert set(seen) == cb.upper_triangle(P, Q)                   # Section 4.3


@pytest.mark.parametrize("N,M,P,Q", [(5, 6, 2, 3), (6, 6, 3, 3), (7, 4, 3, 2), (4, 4, 4, 4),
                                     (6, 5, 1, 5), (5, 7, 5, 2)])
def test_algorithm1_equals_definition(oracle_mod, N, M, P, Q):
    A = wl.complex_normal((N, M), 3 * N + M)
    got = algorithm1.covariance_algorithm1(A, P, Q)
    assert rel_err(got, oracle_mod.cov_window(A, P, Q)) < 1e-14
    Ai = wl.integer_valued((N, M), 77 + N)
    assert np.array_equal(algorithm1.covariance_algorithm1(Ai, P, Q, mean=False),
                          oracle_mod.cov_window(Ai, P, Q, mean=False))


# ----------------------------------------------------------------------------
# Planted mistakes: a Python copy of the oracle's loop, with one mistake at a
# time, must fail at least one of the pins above.
# ----------------------------------------------------------------------------
def py_window(A, P, Q, mistake=None):
    A = np.asarray(A, np.complex128)
    N, M = A.shape
    D = P * Q
    S = np.zeros((D, D), np.complex128)
    p_hi = N - P + (0 if mistake == "paper_limits" else 1)
    q_hi = M - Q + (0 if mistake == "paper_limits" else 1)
    for p in range(p_hi):
        for q in range(q_hi):
            if mistake == "row_stack":
                x = [A[p + a // Q, q + a % Q] for a in range(D)]
            else:
                x = [A[p + a % P, q + a // P] for a in range(D)]
            for a in range(D):
                for b in range(a, D):
                    ar, ai = x[a].real, x[a].imag
                    br, bi = x[b].real, x[b].imag
                    if mistake == "no_conj":
                        S[a, b] += complex(ar * br - ai * bi, ai * br + ar * bi)
                    elif mistake == "conj_first":
                        S[a, b] += complex(ar * br + ai * bi, ar * bi - ai * br)
                    else:
                        S[a, b] += complex(ar * br + ai * bi, ai * br - ar * bi)
    K = (N - P + 1) * (M - Q + 1)
    if mistake == "wrong_K":
        K = (N - P) * (M - Q) or 1
    R = S / K
    R = np.triu(R) + np.conj(np.triu(R, 1)).T
    R[np.diag_indices(D)] = R.diagonal().real
    return R


def pins_pass(fn) -> bool:
    A = wl.complex_normal((6, 5), 99)
    if rel_err(fn(A, 3, 2), brute_force(A, 3, 2)) > 1e-13:
        return False
    if not np.array_equal(fn(np.full((5, 6), 3 + 4j), 2, 3), np.full((6, 6), 25 + 0j)):
        return False
    return True


def test_planted_mistakes_are_caught(oracle_mod):
    A = wl.complex_normal((6, 5), 5)
    assert np.array_equal(py_window(A, 3, 2), oracle_mod.cov_window(A, 3, 2))
    assert pins_pass(py_window)
    for mistake in ("no_conj", "conj_first", "row_stack", "paper_limits", "wrong_K"):
        assert not pins_pass(lambda A, P, Q, m=mistake: py_window(A, P, Q, m)), mistake


# ----------------------------------------------------------------------------
# The adjoint: finite differences in FP64.
# ----------------------------------------------------------------------------
def _loss(oracle_mod, A, T, P, Q):
    R = oracle_mod.cov_window(A, P, Q)
    return float(np.sum(np.abs(R - T) ** 2))


@pytest.mark.parametrize("N,M,P,Q", [(16, 16, 4, 4), (7, 9, 3, 2), (5, 5, 5, 5)])
def test_backward_matches_finite_differences(oracle_mod, N, M, P, Q):
    A = wl.complex_normal((N, M), 40 + N)
    T = oracle_mod.cov_window(wl.complex_normal((N, M), 5000 + N), P, Q)
    G = 2.0 * (oracle_mod.cov_window(A, P, Q) - T)      # dL/dR for ||R - T||_F^2
    dA = oracle_mod.cov_backward(A, G, P, Q)
    h = 1e-6
    fd = np.zeros((N, M), np.complex128)
    for n in range(N):
        for m in range(M):
            for unit in (1.0, 1j):
                E = np.zeros((N, M), np.complex128)
                E[n, m] = unit * h
                d = (_loss(oracle_mod, A + E, T, P, Q) - _loss(oracle_mod, A - E, T, P, Q)) / (2 * h)
                fd[n, m] += d * (1.0 if unit == 1.0 else 1j)
    assert rel_err(dA, fd) < 1e-7


def test_backward_of_linear_functional(oracle_mod):
    # L = Re <G, R> is linear in R, so dL/dA from the oracle must reproduce the
    # exact change of L along a random direction E (a second-order Taylor term
    # remains: L is quadratic in A).
    A = wl.complex_normal((9, 8), 61)
    P, Q = 3, 4
    G = wl.complex_normal((P * Q, P * Q), 62)
    E = wl.complex_normal((9, 8), 63)
    dA = oracle_mod.cov_backward(A, G, P, Q)

    def L(X):
        return float(np.real(np.sum(np.conj(G) * oracle_mod.cov_window(X, P, Q))))

    t = 1e-4
    d = (L(A + t * E) - L(A - t * E)) / (2 * t)
    assert abs(d - float(np.real(np.sum(np.conj(dA) * E)))) < 1e-8 * max(1.0, abs(d))


# ----------------------------------------------------------------------------
# Planted mistakes in the adjoint: a NumPy copy of the oracle's adjoint, with
# one mistake at a time, must fail the finite-difference pin (a Hermitian G)
# or the linear-functional pin (a general G).
# ----------------------------------------------------------------------------
def py_backward(A, G, P, Q, mistake=None):
    A = np.asarray(A, np.complex128)
    N, M = A.shape
    K = (N - P + 1) * (M - Q + 1)
    if mistake == "g_only":
        H = 2.0 * G / K                       # drops the Hermitian part of G
    elif mistake == "no_K":
        H = G + G.conj().T
    else:
        H = (G + G.conj().T) / K
    dA = np.zeros((N, M), np.complex128)
    for p in range(N - P + 1):
        for q in range(M - Q + 1):
            x = A[p:p + P, q:q + Q].flatten(order="F")
            y = H @ (x.conj() if mistake == "conj_x" else x)
            if mistake == "transposed_h":
                y = H.T @ x
            dA[p:p + P, q:q + Q] += y.reshape((P, Q), order="F")
    return dA


def adjoint_pins_pass(oracle_mod, backward) -> bool:
    N, M, P, Q = 5, 6, 2, 3
    A = wl.complex_normal((N, M), 71)
    # finite differences of ||R - T||_F^2 (G = 2 (R - T), Hermitian)
    T = oracle_mod.cov_window(wl.complex_normal((N, M), 72), P, Q)
    G = 2.0 * (oracle_mod.cov_window(A, P, Q) - T)
    dA = backward(A, G, P, Q)
    h = 1e-6
    fd = np.zeros((N, M), np.complex128)
    for n in range(N):
        for m in range(M):
            for unit in (1.0, 1j):
                E = np.zeros((N, M), np.complex128)
                E[n, m] = unit * h
                d = (_loss(oracle_mod, A + E, T, P, Q) - _loss(oracle_mod, A - E, T, P, Q)) / (2 * h)
                fd[n, m] += d * (1.0 if unit == 1.0 else 1j)
    if rel_err(dA, fd) >= 1e-7:
        return False
    # L = Re <G, R> for a general G, along a random direction
    G = wl.complex_normal((P * Q, P * Q), 75)
    E = wl.complex_normal((N, M), 76)
    dA = backward(A, G, P, Q)

    def L(X):
        return float(np.real(np.sum(np.conj(G) * oracle_mod.cov_window(X, P, Q))))

    t = 1e-4
    d = (L(A + t * E) - L(A - t * E)) / (2 * t)
    return abs(d - float(np.real(np.sum(np.conj(dA) * E)))) < 1e-8 * max(1.0, abs(d))


def test_planted_adjoint_mistakes_are_caught(oracle_mod):
    A = wl.complex_normal((6, 5), 73)
    G = wl.complex_normal((6, 6), 74)
    assert rel_err(py_backward(A, G, 3, 2), oracle_mod.cov_backward(A, G, 3, 2)) < 1e-14
    assert adjoint_pins_pass(oracle_mod, oracle_mod.cov_backward)
    assert adjoint_pins_pass(oracle_mod, py_backward)
    for mistake in ("g_only", "no_K", "conj_x", "transposed_h"):
        assert not adjoint_pins_pass(oracle_mod,
                                     lambda A, G, P, Q, m=mistake: py_backward(A, G, P, Q, m)), mistake


# ----------------------------------------------------------------------------
# The Gram form of Eq. 2.2 (oracle/gram.py), the full-size reference.
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("N,M,P,Q", [s for s in SMALL_SHAPES if s[0] * s[1] >= 6])
def test_gram_form_matches_window_loop_and_bruteforce(oracle_mod, N, M, P, Q):
    from oracle.gram import cov_gram
    A = wl.complex_normal((N, M), 3000 + N * M)
    R = oracle_mod.cov_window(A, P, Q)
    for g in (1, 2, 0):  # one window row per group, two, the default
        G = cov_gram(A, P, Q, rows_per_group=g)
        assert rel_err(G, R) < 1e-14
        assert rel_err(G, brute_force(A, P, Q)) < 1e-14
        assert np.array_equal(G, G.conj().T)
    assert rel_err(cov_gram(A, P, Q, mean=False), brute_force(A, P, Q, mean=False)) < 1e-14


def test_gram_form_medium_and_workload_shaped(oracle_mod):
    from oracle.gram import cov_gram
    A = wl.complex_normal((40, 33), 7)
    for P, Q in ((8, 8), (5, 11), (13, 2), (40, 33), (1, 1)):
        assert rel_err(cov_gram(A, P, Q, rows_per_group=3), oracle_mod.cov_window(A, P, Q)) < 1e-14
    # the SAR-like recipe (sum of exponentials plus noise), smaller
    S, _ = wl.sar_like(48, 40, 2, dtype="c128")
    assert rel_err(cov_gram(S, 12, 10), oracle_mod.cov_window(S, 12, 10)) < 1e-14


@pytest.mark.parametrize("N,M,P,Q", [(30, 20, 4, 3), (30, 20, 7, 7), (30, 20, 30, 20),
                                     (17, 9, 1, 1), (12, 25, 6, 12)])
def test_gram_form_integer_inputs_bit_exact(oracle_mod, N, M, P, Q):
    # every partial sum of Gaussian integers is an exact integer in FP64, so
    # any summation order gives the exact sum and one IEEE division by K
    from oracle.gram import cov_gram
    A = wl.integer_valued((N, M), 4000 + N + M)
    for g in (1, 5, 0):
        assert np.array_equal(cov_gram(A, P, Q, rows_per_group=g), oracle_mod.cov_window(A, P, Q))
        assert np.array_equal(cov_gram(A, P, Q, mean=False, rows_per_group=g),
                              oracle_mod.cov_window(A, P, Q, mean=False))


def test_gram_form_closed_forms():
    from oracle.gram import cov_gram
    for P, Q in ((1, 1), (3, 2), (9, 7), (4, 5)):
        assert np.array_equal(cov_gram(np.full((9, 7), 3 + 4j), P, Q),
                              np.full((P * Q, P * Q), 25.0 + 0j))
    c, om, nu = 0.7 - 0.2j, 0.9, -2.1
    A = wl.single_exponential(20, 16, c, om, nu)
    P, Q = 5, 4
    v = np.array([np.exp(1j * (om * (a % P) + nu * (a // P))) for a in range(P * Q)])
    assert rel_err(cov_gram(A, P, Q), abs(c) ** 2 * np.outer(v, v.conj())) < 1e-14


# ----------------------------------------------------------------------------
# The Capon spectrum (oracle/capon.py), the downstream use of R (Section 2.3).
# ----------------------------------------------------------------------------
def test_capon_closed_forms():
    from oracle.capon import capon_spectrum, steering_vectors
    P, Q = 4, 3
    D = P * Q
    rng = np.random.default_rng(5)
    A = steering_vectors(P, Q, rng.uniform(-np.pi, np.pi, 9), rng.uniform(-np.pi, np.pi, 9))
    assert np.allclose(np.abs(A) ** 2, 1.0)
    # white noise: P = (s2 + d) / ||a||^2 with d = loading * trace / D = loading * s2
    s2 = 2.5
    for loading in (0.0, 0.1):
        got = capon_spectrum(s2 * np.eye(D), A, loading)
        assert np.allclose(got, (s2 * (1 + loading)) / D, rtol=1e-13)
    # one source plus noise, Sherman-Morrison:
    # a^H (v v^H + s2 I)^{-1} a = (||a||^2 - |v^H a|^2 / (s2 + ||v||^2)) / s2
    v = steering_vectors(P, Q, [0.7], [-1.3])[0] * (1.5 - 0.5j)
    R = np.outer(v, v.conj()) + s2 * np.eye(D)
    got = capon_spectrum(R, A)
    na = np.sum(np.abs(A) ** 2, axis=1)
    va = A @ v.conj()                       # v^H a_f, conjugated: |.| is the same
    want = s2 / (na - np.abs(va) ** 2 / (s2 + np.vdot(v, v).real))
    assert np.allclose(got, want, rtol=1e-12)
    # the peak is at the source's own steering vector
    grid = steering_vectors(P, Q, np.linspace(-np.pi, np.pi, 41)[:-1].repeat(40),
                            np.tile(np.linspace(-np.pi, np.pi, 41)[:-1], 40))
    spec = capon_spectrum(R, np.vstack([grid, v / np.linalg.norm(v) * np.sqrt(D)]))
    assert np.argmax(spec) == len(spec) - 1


def test_capon_scaling_and_batch():
    from oracle.capon import capon_spectrum, steering_vectors
    P, Q = 3, 5
    rng = np.random.default_rng(9)
    X = rng.standard_normal((P * Q, 40)) + 1j * rng.standard_normal((P * Q, 40))
    R = X @ X.conj().T / 40
    A = steering_vectors(P, Q, rng.uniform(-3, 3, 6), rng.uniform(-3, 3, 6))
    p1 = capon_spectrum(R, A, 0.05)
    assert np.all(p1 > 0)
    assert np.allclose(capon_spectrum(3.0 * R, A, 0.05), 3.0 * p1, rtol=1e-12)
    both = capon_spectrum(np.stack([R, 2 * R]), A, 0.05)
    assert np.allclose(both[0], p1, rtol=1e-14) and np.allclose(both[1], 2 * p1, rtol=1e-12)
    # a planted mistake (a^H R a instead of a^H R^{-1} a) fails the closed form
    bad = 1.0 / np.einsum("fd,de,fe->f", A.conj(), 2.5 * np.eye(P * Q), A).real
    assert not np.allclose(bad, 2.5 / (P * Q))
