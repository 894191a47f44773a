"""Counting and indexing of the combination decomposition (Sections 3-4).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

All indices are 0-based. The paper is 1-based (Section 2.2); the readings used
here are:

* x[i + P*j] = window element (i, j)  (Eq. 2.1, shifted to 0-based);
* a combination is Delta = (dr, dc) = (r2 - r1, c2 - c1)  (Eq. 3.1), the first
  element being the one that is not conjugated;
* mu(Delta) = (N - |dr|)(M - |dc|)  (Eq. 3.5 read with absolute values: the
  closed forms of Eq. 4.4-4.6 only hold that way).
"""
from __future__ import annotations

from fractions import Fraction
from typing import List, Set, Tuple


def unique_combinations(P: int, Q: int) -> List[Tuple[int, int]]:
    """UC of Eq. 3.3: {0<=dr<=P-1, 0<=dc<=Q-1} u {-(P-1)<=dr<=-1, 1<=dc<=Q-1}."""
    out = [(dr, dc) for dc in range(Q) for dr in range(P)]
    out += [(dr, dc) for dc in range(1, Q) for dr in range(-(P - 1), 0)]
    return out


def n_unique_combinations(P: int, Q: int) -> int:
    """|UC| = PQ + (P-1)(Q-1)  (Eq. 3.4)."""
    return P * Q + (P - 1) * (Q - 1)


def mu(N: int, M: int, dr: int, dc: int) -> int:
    """Distinct products of one combination (Eq. 3.5, with |dr|, |dc|)."""
    return (N - abs(dr)) * (M - abs(dc))


def um_enumerated(N: int, M: int, P: int, Q: int) -> int:
    """UM = sum over UC of mu  (Eq. 3.6 / 4.3), by enumeration."""
    return sum(mu(N, M, dr, dc) for dr, dc in unique_combinations(P, Q))


def um_closed_form(N: int, M: int, P: int, Q: int) -> Fraction:
    """UM from Eq. 4.6 (UM_1 of Eq. 4.4 plus UM_2 of Eq. 4.5)."""
    um1 = Fraction(P, 2) * (2 * N - (P - 1)) * Fraction(Q, 2) * (2 * M - (Q - 1))
    um2 = Fraction(P - 1, 2) * (2 * N - P) * Fraction(Q - 1, 2) * (2 * M - Q)
    return um1 + um2


def um_hat(N: int, M: int, P: int, Q: int) -> Fraction:
    """The upper bound of Eq. 4.7."""
    return 2 * Fraction(P, 2) * (2 * N - (P - 1)) * Fraction(Q, 2) * (2 * M - (Q - 1))


def sm_naive(N: int, M: int, P: int, Q: int) -> int:
    """Multiplications of the naive serial algorithm, Eq. 4.1 (the paper counts
    (N-P)(M-Q) window positions there)."""
    return (N - P) * (M - Q) * P * P * Q * Q


def sm_over_um_hat(N: int, M: int, P: int, Q: int) -> Fraction:
    """The ratio of Eq. 4.8."""
    num = Fraction((N - P) * (M - Q) * P * Q)
    den = 2 * (N - Fraction(P - 1, 2)) * (M - Fraction(Q - 1, 2))
    return num / den


def eta(P: int, Q: int, dr: int, dc: int) -> int:
    """Output indices of one combination, Eq. 3.8."""
    return (P - abs(dr)) * (Q - abs(dc))


def initial_write_index(P: int, dr: int, dc: int) -> Tuple[int, int]:
    """Eq. 3.7 restated 0-based: with the window at its initial placement the
    pair sits on the window's top and left borders, so the first element is at
    window row max(0, -dr), column 0 and the second at row max(0, dr),
    column dc."""
    a0 = max(0, -dr)
    b0 = max(0, dr) + P * dc
    return a0, b0


def write_indices(P: int, Q: int, dr: int, dc: int) -> List[Tuple[int, int]]:
    """Indices (a, b) of R written by combination (dr, dc): the initial index
    shifted by +1 for each step of the window upward and by +P for each step
    leftward (Section 3.3, Fig. 2): P-|dr| steps by Q-|dc| steps."""
    a0, b0 = initial_write_index(P, dr, dc)
    return [(a0 + s + P * t, b0 + s + P * t)
            for t in range(Q - abs(dc)) for s in range(P - abs(dr))]


def upper_triangle(P: int, Q: int) -> Set[Tuple[int, int]]:
    D = P * Q
    return {(a, b) for a in range(D) for b in range(a, D)}


def combination_of_index(P: int, a: int, b: int) -> Tuple[int, int]:
    """The combination that owns output (a, b): the distance of the pair of
    window elements that index names."""
    return (b % P - a % P, b // P - a // P)
