"""The regroupings the CUDA path computes by, checked on the CPU against the oracle.

Each kernel family evaluates the estimate in a different order from the plain
window loop of Eq. 2.1-2.2; the identities that make those orders equal are
restated here in plain NumPy and held to the oracle:

* the combination / box-sum form (Section 3): combination (dr, dc) owns the
  outputs of a diagonal segment, and each owned output is a box sum of the
  combination's product image; the walk (Section 3.3) moves the box;
* the dense GEMM form: R from the real Gram matrix of Y = [Re X; Im X];
* the split-precision operand formats of the GEMM form (TF32 hi/lo, BF16
  hi/mid/lo) and the error of the products they keep;
* the stencil form of the adjoint: dA as a sum over combinations of
  class-dependent weights times shifted A;
* the strip form of the aperture batch (Section 2.3): the apertures side by
  side share one product image per combination over their strip, column sums
  walked down it and window sums slid along each aperture's output columns
  give every aperture's R blocks.

No GPU is needed; integer inputs make the sums exact, so those comparisons are
bit for bit.
"""
import numpy as np
import pytest

import cov_workloads as wl
from oracle import combinations as cb


def rel_err(X, Y):
    return float(np.linalg.norm(X - Y) / max(np.linalg.norm(Y), 1e-300))


def owned_outputs(P, Q, dr, dc):
    """The outputs combination (dr, dc) owns, as window offsets (i, j) of the
    first element: i in [max(0, -dr), P-1-max(0, dr)], j in [0, Q-1-dc]."""
    return [(i, j) for j in range(0, Q - dc) for i in range(max(0, -dr), P - max(0, dr))]


def box_sum(A, P, Q, dr, dc, i, j):
    """Sum of Pi[n][m] = A[n][m] conj(A[n+dr][m+dc]) over the box
    n in [i, i+N-P], m in [j, j+M-Q]."""
    N, M = A.shape
    a = A[i:i + N - P + 1, j:j + M - Q + 1]
    b = A[i + dr:i + dr + N - P + 1, j + dc:j + dc + M - Q + 1]
    return (a * np.conj(b)).sum()


BOX_SHAPES = [(6, 7, 2, 3), (7, 7, 3, 3), (9, 5, 4, 2), (5, 8, 5, 1), (8, 8, 1, 4), (10, 11, 4, 5)]


@pytest.mark.parametrize("N,M,P,Q", BOX_SHAPES)
def test_owned_outputs_are_the_written_indices(N, M, P, Q):
    # Section 4.2-4.3: the segments of the unique combinations cover the upper
    # triangle once; the owned ranges above are those segments.
    seen = set()
    for dr, dc in cb.unique_combinations(P, Q):
        mine = {(i + P * j, (i + dr) + P * (j + dc)) for i, j in owned_outputs(P, Q, dr, dc)}
        assert mine == set(cb.write_indices(P, Q, dr, dc))
        assert not (mine & seen)
        seen |= mine
    assert seen == cb.upper_triangle(P, Q)


@pytest.mark.parametrize("N,M,P,Q", BOX_SHAPES)
def test_box_sum_identity_exact(oracle_mod, N, M, P, Q):
    A = wl.integer_valued((N, M), 500 + 7 * N + M)
    S = oracle_mod.cov_window(A, P, Q, mean=False)
    for dr, dc in cb.unique_combinations(P, Q):
        for i, j in owned_outputs(P, Q, dr, dc):
            a, b = i + P * j, (i + dr) + P * (j + dc)
            assert box_sum(A, P, Q, dr, dc, i, j) == S[a, b], (dr, dc, i, j)


@pytest.mark.parametrize("N,M,P,Q", [(9, 8, 4, 3), (7, 10, 3, 5)])
def test_walk_moves_the_box(N, M, P, Q):
    # Section 3.3: one step down the diagonal adds the product row entering the
    # box and removes the one leaving it; a step to the next segment does the
    # same with columns. Exact on integer inputs.
    A = wl.integer_valued((N, M), 41 + N)
    for dr, dc in cb.unique_combinations(P, Q):
        own = set(owned_outputs(P, Q, dr, dc))
        Pi = np.zeros((N, M), np.complex128)
        for n in range(max(0, -dr), min(N, N - dr)):
            for m in range(0, M - dc):
                Pi[n, m] = A[n, m] * np.conj(A[n + dr, m + dc])
        for i, j in own:
            O = box_sum(A, P, Q, dr, dc, i, j)
            if (i + 1, j) in own:
                down = O + Pi[i + N - P + 1, j:j + M - Q + 1].sum() - Pi[i, j:j + M - Q + 1].sum()
                assert down == box_sum(A, P, Q, dr, dc, i + 1, j)
            if (i, j + 1) in own:
                right = O + Pi[i:i + N - P + 1, j + M - Q + 1].sum() - Pi[i:i + N - P + 1, j].sum()
                assert right == box_sum(A, P, Q, dr, dc, i, j + 1)


# ----------------------------------------------------------------------------
# Dense form: R = (B11 + B22) + i (B21 - B12) with B = Y Y^T, Y = [Re X; Im X].
# ----------------------------------------------------------------------------
def windows(A, P, Q):
    W = np.lib.stride_tricks.sliding_window_view(np.asarray(A), (P, Q))
    return W.transpose(0, 1, 3, 2).reshape(-1, P * Q).T          # x[i + P j]


@pytest.mark.parametrize("N,M,P,Q", [(12, 10, 3, 4), (16, 16, 4, 4), (9, 20, 5, 2)])
def test_real_gram_form(oracle_mod, N, M, P, Q):
    A = wl.complex_normal((N, M), 60 + N)
    X = windows(A, P, Q)
    D, K = X.shape
    Y = np.concatenate([X.real, X.imag], axis=0)
    B = Y @ Y.T
    R = ((B[:D, :D] + B[D:, D:]) + 1j * (B[D:, :D] - B[:D, D:])) / K
    assert rel_err(R, oracle_mod.cov_window(A, P, Q)) < 1e-14
    Ai = wl.integer_valued((N, M), 61 + N)
    Xi = windows(Ai, P, Q)
    Yi = np.concatenate([Xi.real, Xi.imag], axis=0)
    Bi = Yi @ Yi.T
    Si = (Bi[:D, :D] + Bi[D:, D:]) + 1j * (Bi[D:, :D] - Bi[:D, D:])
    assert np.array_equal(Si, oracle_mod.cov_window(Ai, P, Q, mean=False))


# ----------------------------------------------------------------------------
# Split operand formats. RN-even to BF16 (8 significant bits) and
# round-half-away to TF32 (11 significant bits), restated on FP32 bit patterns.
# ----------------------------------------------------------------------------
def rn_bf16(x):
    u = np.asarray(x, np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32)


def rna_tf32(x):
    u = np.asarray(x, np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x1000) & 0xFFFFE000
    return u.astype(np.uint32).view(np.float32)


def significant_bits(v):
    """Bits between the leading and the trailing one of each FP32 value's significand."""
    m, e = np.frexp(np.asarray(v, np.float64))
    out = np.zeros(m.shape, np.int64)
    nz = m != 0
    mi = np.abs(np.ldexp(m[nz], 24)).astype(np.int64)
    tz = np.zeros(mi.shape, np.int64)
    t = mi.copy()
    while np.any((t & 1) == 0):
        z = (t & 1) == 0
        tz += z
        t = np.where(z, t >> 1, t)
    out[nz] = 24 - tz
    return out


def fp32_samples(n, seed):
    rng = np.random.default_rng(seed)
    mag = np.exp(rng.uniform(-20.0, 20.0, n))
    return (rng.choice([-1.0, 1.0], n) * mag).astype(np.float32)


def test_bf16_three_way_split_is_exact():
    x = fp32_samples(200_000, 11)
    hi = rn_bf16(x)
    r1 = (x - hi).astype(np.float32)
    mid = rn_bf16(r1)
    r2 = (r1 - mid).astype(np.float32)
    lo = rn_bf16(r2)
    for part in (hi, mid, lo):
        assert significant_bits(part).max() <= 8
    # each remainder is exact in FP32 and the three parts add up to x
    x64 = x.astype(np.float64)
    assert np.array_equal(hi.astype(np.float64) + r1.astype(np.float64), x64)
    assert np.array_equal(mid.astype(np.float64) + r2.astype(np.float64), r1.astype(np.float64))
    assert np.array_equal(hi.astype(np.float64) + mid + lo.astype(np.float64), x64)


def test_bf16x3_six_products_error():
    x = fp32_samples(100_000, 12)
    y = fp32_samples(100_000, 13)

    def split(v):
        h = rn_bf16(v)
        m = rn_bf16((v - h).astype(np.float32))
        lo = rn_bf16((v - h - m).astype(np.float32))
        return [p.astype(np.float64) for p in (h, m, lo)]

    (xh, xm, xl), (yh, ym, yl) = split(x), split(y)
    exact = x.astype(np.float64) * y.astype(np.float64)
    six = xh * yh + (xh * ym + xm * yh) + (xm * ym + xh * yl + xl * yh)
    rel = np.abs(six - exact) / np.abs(exact)
    assert rel.max() < 2.0 ** -21
    # without the terms of order 2^-16 the error is far larger
    three = xh * yh + (xh * ym + xm * yh)
    assert (np.abs(three - exact) / np.abs(exact)).max() > 2.0 ** -18


def test_tf32x3_split_and_three_products_error():
    x = fp32_samples(100_000, 14)
    y = fp32_samples(100_000, 15)

    def split(v):
        h = rna_tf32(v)
        lo = rna_tf32((v - h).astype(np.float32))
        return h, lo

    (xh, xl), (yh, yl) = split(x), split(y)
    for part in (xh, xl, yh, yl):
        assert significant_bits(part).max() <= 11
    # the first remainder is exact in FP32
    assert np.array_equal(xh.astype(np.float64) + (x - xh).astype(np.float64), x.astype(np.float64))
    xh, xl, yh, yl = (v.astype(np.float64) for v in (xh, xl, yh, yl))
    exact = x.astype(np.float64) * y.astype(np.float64)
    three = xh * yh + (xh * yl + xl * yh)
    assert (np.abs(three - exact) / np.abs(exact)).max() < 2.0 ** -19
    one = xh * yh
    assert (np.abs(one - exact) / np.abs(exact)).max() > 2.0 ** -12


# ----------------------------------------------------------------------------
# Stencil form of the adjoint: with H = (G + G^H)/K,
#   dA[n][m] = sum_{(dr,dc)} T_(dr,dc)(n, m) A[n+dr][m+dc],
#   T_(dr,dc)(n, m) = sum of H[a][a + (dr,dc)] over the offsets a = (ia, ja)
#   that a valid window places on (n, m): ia in [max(0, n-(N-P)), min(P-1, n)],
#   ja likewise, with the partner a + (dr, dc) inside the window.
# ----------------------------------------------------------------------------
def stencil_weight(H, N, M, P, Q, dr, dc, n, m):
    t = 0j
    for ja in range(max(0, m - (M - Q)), min(Q - 1, m) + 1):
        if not 0 <= ja + dc < Q:
            continue
        for ia in range(max(0, n - (N - P)), min(P - 1, n) + 1):
            if 0 <= ia + dr < P:
                t += H[ia + P * ja, (ia + dr) + P * (ja + dc)]
    return t


def row_class(n, N, P):
    """2P-1 classes: the P-1 top fringe rows, the inner rows, the P-1 bottom ones."""
    if n < P - 1:
        return n
    if n <= N - P:
        return P - 1
    return P - 1 + n - (N - P)


def class_row(c, N, P):
    return c if c <= P - 1 else (N - P) + c - (P - 1)


@pytest.mark.parametrize("N,M,P,Q", [(8, 9, 3, 4), (11, 7, 4, 2), (6, 6, 1, 3), (9, 9, 5, 5)])
def test_stencil_adjoint_identity(oracle_mod, N, M, P, Q):
    A = wl.complex_normal((N, M), 90 + N)
    G = wl.complex_normal((P * Q, P * Q), 91 + M)
    K = (N - P + 1) * (M - Q + 1)
    H = (G + G.conj().T) / K
    dA = np.zeros((N, M), np.complex128)
    for dr in range(-(P - 1), P):
        for dc in range(-(Q - 1), Q):
            for n in range(N):
                for m in range(M):
                    t = stencil_weight(H, N, M, P, Q, dr, dc, n, m)
                    if t != 0:
                        assert 0 <= n + dr < N and 0 <= m + dc < M
                        dA[n, m] += t * A[n + dr, m + dc]
    assert rel_err(dA, oracle_mod.cov_backward(A, G, P, Q)) < 1e-13


@pytest.mark.parametrize("N,M,P,Q", [(8, 9, 3, 4), (12, 10, 4, 5)])
def test_stencil_weights_depend_on_the_class_only(N, M, P, Q):
    # with N >= 2P-1 and M >= 2Q-1 the admissible offsets of (n, m) are set by
    # its row class and column class alone: (2P-1)(2Q-1) tables per combination
    G = wl.complex_normal((P * Q, P * Q), 7)
    H = G + G.conj().T
    for dr in range(-(P - 1), P):
        for dc in range(-(Q - 1), Q):
            for n in range(N):
                for m in range(M):
                    rep = stencil_weight(H, N, M, P, Q, dr, dc, class_row(row_class(n, N, P), N, P),
                                         class_row(row_class(m, M, Q), M, Q))
                    assert stencil_weight(H, N, M, P, Q, dr, dc, n, m) == rep


@pytest.mark.parametrize("H,W,ap,step,P,Q", [(64, 80, (25, 25), (10, 10), 10, 10),
                                             (47, 51, (20, 17), (9, 5), 4, 3),
                                             (30, 70, (12, 30), (3, 7), 5, 9),
                                             (20, 40, (20, 20), (2, 2), 16, 4)])
def test_strip_of_apertures(oracle_mod, H, W, ap, step, P, Q):
    """Apertures of one row of apertures, side by side in a strip of at most 64
    columns: per combination (dr, dc) the products over the strip are formed
    once, column sums over the Hb = ap_n - P + 1 box rows are walked down the
    output rows (entering row added, leaving row subtracted), and aperture
    k's output (s, j) is the sum of the Wd = ap_m - Q + 1 column sums from
    column k * step_c + j, slid along j. The blocks (j, j + dc) and their
    conjugate mirrors then fill each aperture's R exactly (integer input)."""
    A = wl.integer_valued((H, W), 77 + H)
    an, am = ap
    sr, sc = step
    nr, nc = (H - an) // sr + 1, (W - am) // sc + 1
    G = max(1, min(nc, 1 + (64 - am) // sc))
    Hb, Wd, D = an - P + 1, am - Q + 1, P * Q
    formed = 0
    for a in range(nr):
        for g0 in range(0, nc, G):
            Gc = min(G, nc - g0)
            Sw = (Gc - 1) * sc + am
            S = A[a * sr:a * sr + an, g0 * sc:g0 * sc + Sw]
            Rs = np.zeros((Gc, D, D), dtype=complex)
            for dc in range(Q):
                for dr in (range(P) if dc == 0 else range(-(P - 1), P)):
                    i0, I = max(0, -dr), P - abs(dr)
                    rows = Hb + I - 1
                    # the strip's product image, once per combination
                    Pi = S[i0:i0 + rows, :Sw - dc] * np.conj(S[i0 + dr:i0 + dr + rows, dc:Sw])
                    formed += Pi.size
                    V = np.zeros((I, Sw - dc), dtype=complex)
                    V[0] = Pi[:Hb].sum(axis=0)
                    for s in range(1, I):
                        V[s] = V[s - 1] + Pi[s - 1 + Hb] - Pi[s - 1]
                    for k in range(Gc):
                        for s in range(I):
                            v = V[s, k * sc:k * sc + Wd + Q - dc - 1]
                            w = v[:Wd].sum()
                            for j in range(Q - dc):
                                if j:
                                    w = w + v[j - 1 + Wd] - v[j - 1]
                                i = i0 + s
                                Rs[k, i + P * j, i + dr + P * (j + dc)] = w
                                Rs[k, i + dr + P * (j + dc), i + P * j] = np.conj(w)
            for k in range(Gc):
                sub = A[a * sr:a * sr + an, (g0 + k) * sc:(g0 + k) * sc + am]
                want = oracle_mod.cov_window(sub, P, Q, mean=False)
                assert np.array_equal(Rs[k], want), (a, g0 + k)
    per_aperture = nr * nc * sum((an - abs(dr)) * (am - dc) for dc in range(Q)
                                 for dr in (range(P) if dc == 0 else range(-(P - 1), P)))
    if G > 1:
        assert formed < per_aperture  # products shared by the apertures of a strip
