"""Exact rational stationary distribution of a tiny PBN (n <= 4).

TEST INFRASTRUCTURE ONLY.  Solves pi P = pi, sum pi = 1 (Sec. 2.1) with Python
Fractions by Gaussian elimination, for networks whose perturbation and
selection probabilities are given as exact rationals.  This is a different
method (direct linear solve, exact arithmetic) from the FP64 power iteration
of exact.py, so the two check each other.
"""
from __future__ import annotations

from fractions import Fraction
from itertools import product


def _fn_value(tt: int, parents, s: int) -> int:
    idx = 0
    for m, v in enumerate(parents):
        idx |= ((s >> v) & 1) << m
    return (tt >> idx) & 1


def transition_matrix(n, functions, p: Fraction, mode: int):
    """functions[i] = list of (parents, truth_table, Fraction prob)."""
    S = 1 << n
    P = [[Fraction(0)] * S for _ in range(S)]
    for s in range(S):
        # probability that node i's function part yields 1
        q = []
        for i in range(n):
            qi = Fraction(0)
            for par, tt, c in functions[i]:
                if _fn_value(tt, par, s):
                    qi += c
            q.append(qi)
        for s2 in range(S):
            if mode == 0:
                pr = Fraction(1)
                for i in range(n):
                    bit = (s2 >> i) & 1
                    flip = bit != ((s >> i) & 1)
                    p_one = p * (1 - ((s >> i) & 1)) + (1 - p) * q[i]
                    pr *= p_one if bit else (1 - p_one)
                P[s][s2] = pr
            else:
                fpart = Fraction(1)
                for i in range(n):
                    bit = (s2 >> i) & 1
                    fpart *= q[i] if bit else (1 - q[i])
                pr = (1 - p) ** n * fpart
                g = s ^ s2
                if g:
                    h = bin(g).count("1")
                    pr += p ** h * (1 - p) ** (n - h)
                P[s][s2] = pr
    return P


def stationary(P):
    S = len(P)
    # rows: (P^T - I) pi = 0 with the last equation replaced by sum pi = 1
    A = [[P[j][i] - (1 if i == j else 0) for j in range(S)] for i in range(S)]
    b = [Fraction(0)] * S
    A[-1] = [Fraction(1)] * S
    b[-1] = Fraction(1)
    # Gaussian elimination with exact pivots
    for col in range(S):
        piv = next(r for r in range(col, S) if A[r][col] != 0)
        A[col], A[piv] = A[piv], A[col]
        b[col], b[piv] = b[piv], b[col]
        inv = 1 / A[col][col]
        A[col] = [v * inv for v in A[col]]
        b[col] *= inv
        for r in range(S):
            if r != col and A[r][col] != 0:
                f = A[r][col]
                A[r] = [a - f * c for a, c in zip(A[r], A[col])]
                b[r] -= f * b[col]
    return b


def three_node_functions():
    """The hand-built 3-node PBN of pbn_synth.three_node with exact rationals."""
    return [
        [((1, 2), 0b1000, Fraction(1))],
        [((0,), 0b01, Fraction(3, 4)), ((2,), 0b10, Fraction(1, 4))],
        [((0, 1), 0b1110, Fraction(1))],
    ]
