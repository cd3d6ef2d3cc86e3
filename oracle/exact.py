"""Exact steady-state distribution of a small PBN with perturbations.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Runs FP64 power iteration pi <- pi P of the DTMC underlying a PBN (Sec.
2.1-2.2) from the uniform distribution until the L1 change drops below a
tolerance; an ergodic DTMC's limiting distribution does not depend on the
start (Sec. 2.1).  State index s = sum_i v_i 2^i.  For n <= 12 the full
2^n x 2^n transition matrix P is built; for 13 <= n <= 16 each step is taken
without forming P, from the product form of its rows (ProductStep below).
Pins: tests/test_oracle_sim.py, tests/test_oracle_exact_large.py.

The probabilities are the quantised ones the simulation realises exactly:
perturbation probability P32/2^32 and function probabilities
(T_j - T_{j-1})/2^32 (see oracle.c for the definition of P32 and T_j).  This
module recomputes that quantisation in Python on its own, so that comparing it
with the C simulator checks both.
"""
from __future__ import annotations

import math

import numpy as np

TWO32 = 4294967296


def _llround_pos(x: float) -> int:
    q = math.floor(x)
    if x - q >= 0.5:
        q += 1
    return int(q)


def perturb_threshold(p: float) -> int:
    return max(0, min(_llround_pos(p * 4294967296.0), TWO32 - 1))


def category_probabilities(net):
    """Returns (p_pert, probs) where probs[f] = P(category of f) unconditionally
    (u uniform on [0, 2^32)), and p_pert = P32 / 2^32."""
    P32 = perturb_threshold(net.p)
    span = TWO32 - P32
    probs = np.zeros(net.n_functions, dtype=np.float64)
    for i in range(net.n):
        f0, f1 = int(net.fn_offset[i]), int(net.fn_offset[i + 1])
        S = 0.0
        prev = P32
        for f in range(f0, f1):
            S += float(net.select_prob[f])
            if f == f1 - 1:
                T = TWO32
            else:
                q = min(max(_llround_pos(float(span) * S), 0), span)
                T = min(P32 + q, TWO32 - 1)
            probs[f] = (T - prev) / TWO32
            prev = T
    return P32 / TWO32, probs


def function_values(net, states: np.ndarray) -> np.ndarray:
    """vals[s, f] = value of function f on state s (truth-table lookup)."""
    S = len(states)
    vals = np.zeros((S, net.n_functions), dtype=np.uint8)
    for f in range(net.n_functions):
        par = net.parents_of(f)
        idx = np.zeros(S, dtype=np.int64)
        for m, v in enumerate(par):
            idx |= ((states >> int(v)) & 1) << m
        words = np.asarray(net.tt_of(f), dtype=np.int64)
        vals[:, f] = (words[idx >> 5] >> (idx & 31)) & 1
    return vals


def transition_matrix(net, mode: int = 0) -> np.ndarray:
    """Dense P for n <= 12.  mode 0: per-node perturbation; mode 1: global
    (s XOR gamma when gamma != 0, functions otherwise)."""
    n = net.n
    if n > 12:
        raise ValueError("dense transition matrix only for n <= 12")
    S = 1 << n
    states = np.arange(S, dtype=np.int64)
    p_e, probs = category_probabilities(net)
    vals = function_values(net, states)
    # q[s, i] = P(next value of node i is 1 | s) for the function part
    qf = np.zeros((S, n), dtype=np.float64)
    for i in range(n):
        for f in net.functions_of(i):
            qf[:, i] += probs[f] * vals[:, f]
    bits = ((states[:, None] >> np.arange(n)[None, :]) & 1).astype(np.float64)

    def product_rows(q):
        R = np.ones((S, 1), dtype=np.float64)
        for i in range(n):
            V = np.stack([1.0 - q[:, i], q[:, i]], axis=1)  # [S, 2]
            R = (V[:, :, None] * R[:, None, :]).reshape(S, -1)
        return R

    if mode == 0:
        q = p_e * (1.0 - bits) + qf
        return product_rows(q)
    # global: conditional on no perturbation the function of node i is chosen
    # with probability probs[f] / (1 - p_e)
    qc = qf / (1.0 - p_e) if p_e < 1.0 else qf
    P = (1.0 - p_e) ** n * product_rows(qc)
    h = np.array([bin(x).count("1") for x in range(S)], dtype=np.int64)
    flip = np.where(h > 0, p_e ** h * (1.0 - p_e) ** (n - h), 0.0)  # by XOR pattern
    P += flip[states[:, None] ^ states[None, :]]
    return P


def stationary_power(P: np.ndarray, tol: float = 1e-14, max_iter: int = 2_000_000):
    """FP64 power iteration from the uniform distribution.  Returns (pi, iters)."""
    S = P.shape[0]
    pi = np.full(S, 1.0 / S)
    for it in range(1, max_iter + 1):
        nxt = pi @ P
        delta = float(np.abs(nxt - pi).sum())
        pi = nxt
        if delta < tol:
            return pi, it
    raise RuntimeError("power iteration did not converge")


def soi_mask(n: int, soi) -> np.ndarray:
    states = np.arange(1 << n, dtype=np.int64)
    m = np.ones(1 << n, dtype=bool)
    for v, val in zip(soi.nodes, soi.values):
        m &= ((states >> int(v)) & 1) == int(val)
    return m


def steady_state_probability(net, soi, mode: int = 0, tol: float = 1e-14):
    P = transition_matrix(net, mode)
    pi, _ = stationary_power(P, tol)
    return float(pi[soi_mask(net.n, soi)].sum()), pi


# ---------------------------------------------------------------------------
# 13 <= n <= 16: the transition matrix is never formed
# ---------------------------------------------------------------------------
#
# Given the current state s, the nodes' next values are independent (Sec. 2.2:
# each node is perturbed or draws its own function, independently), so row s
# of P is a product measure over the nodes:
#     P(s, s') = prod_i q_i(s)^{s'_i} (1 - q_i(s))^{1 - s'_i},
# q_i(s) = P(node i is 1 after the step | s).  Split the nodes into a low
# half A (index a = s' mod 2^h) and a high half B (b = s' div 2^h); the row
# factors as P(s, a + 2^h b) = RA[s, a] RB[s, b], with RA and RB the product
# measures of the two halves.  Hence one step of the chain,
#     (pi P)(a + 2^h b) = sum_s pi(s) RA[s, a] RB[s, b] = (RB^T diag(pi) RA)[b, a],
# is one matrix product of a 2^(n-h) x 2^n and a 2^n x 2^h matrix: the 4^n
# terms of the row-by-row expansion, summed by a library matmul.  RA and RB
# (2^n x 2^h doubles each, 134 MB at n = 16) do not change between steps.
#
# GLOBAL reading: with probability (1 - p)^n no node is perturbed and every
# node draws a function with the conditional probabilities probs/(1 - p);
# otherwise the state becomes s XOR gamma for a nonzero pattern gamma of
# independent Bernoulli(p) bits.  The first part is a product measure as
# above, scaled by (1 - p)^n; the second is the n independent bit-flip
# channels applied one node at a time, minus their gamma = 0 term.


def _half_rows(q: np.ndarray, nodes) -> np.ndarray:
    """R[s, c] = prod_{m} q[s, nodes[m]]^{c_m} (1 - q[s, nodes[m]])^{1 - c_m},
    c = sum_m c_m 2^m (nodes in ascending order)."""
    S = q.shape[0]
    R = np.ones((S, 1), dtype=np.float64)
    for i in nodes:
        V = np.stack([1.0 - q[:, i], q[:, i]], axis=1)     # [S, 2]: value 0, value 1
        R = (V[:, :, None] * R[:, None, :]).reshape(S, -1)  # node i becomes the top bit
    return R


def _one_probabilities(net, mode: int):
    """(q, p_e): q[s, i] = P(node i is 1 after one step | state s) given that
    the functions are applied (GLOBAL: conditional on no perturbation), and
    the quantised perturbation probability p_e."""
    n = net.n
    S = 1 << n
    states = np.arange(S, dtype=np.int64)
    p_e, probs = category_probabilities(net)
    vals = function_values(net, states)
    qf = np.zeros((S, n), dtype=np.float64)
    for i in range(n):
        for f in net.functions_of(i):
            qf[:, i] += probs[f] * vals[:, f]
    if mode == 0:
        bits = ((states[:, None] >> np.arange(n)[None, :]) & 1).astype(np.float64)
        return p_e * (1.0 - bits) + qf, p_e
    return (qf / (1.0 - p_e) if p_e < 1.0 else qf), p_e


def _flip_channels(pi: np.ndarray, n: int, p: float) -> np.ndarray:
    """sum_gamma pi(s' XOR gamma) prod_i p^{gamma_i} (1-p)^{1-gamma_i}: node i's
    bit flipped with probability p, independently, one node after another."""
    out = pi.copy()
    for i in range(n):
        v = out.reshape(-1, 2, 1 << i)
        out = ((1.0 - p) * v + p * v[:, ::-1, :]).reshape(-1)
    return out


class ProductStep:
    """One step pi -> pi P of a PBN's chain for n <= 16 without forming P."""

    def __init__(self, net, mode: int = 0):
        n = net.n
        if n > 16:
            raise ValueError("implicit transition step only for n <= 16")
        self.n, self.mode = n, mode
        q, self.p_e = _one_probabilities(net, mode)
        self.h = n // 2
        self.RA = _half_rows(q, range(self.h))
        self.RB = _half_rows(q, range(self.h, n))
        self.no_pert = (1.0 - self.p_e) ** n

    def __call__(self, pi: np.ndarray) -> np.ndarray:
        fn_part = (self.RB.T @ (pi[:, None] * self.RA)).reshape(-1)
        if self.mode == 0:
            return fn_part
        return self.no_pert * fn_part + (_flip_channels(pi, self.n, self.p_e) - self.no_pert * pi)


def stationary_implicit(net, mode: int = 0, tol: float = 1e-14, max_iter: int = 200_000):
    """FP64 power iteration pi <- pi P from the uniform distribution with the
    implicit step (any n <= 16).  Returns (pi, iters)."""
    step = ProductStep(net, mode)
    S = 1 << net.n
    pi = np.full(S, 1.0 / S)
    for it in range(1, max_iter + 1):
        nxt = step(pi)
        delta = float(np.abs(nxt - pi).sum())
        pi = nxt
        if delta < tol:
            return pi, it
    raise RuntimeError("power iteration did not converge")


def steady_state_probability_any(net, soi, mode: int = 0, tol: float = 1e-14):
    """Exact steady-state probability of the state of interest: the dense
    matrix for n <= 12, the implicit step for 13 <= n <= 16."""
    if net.n <= 12:
        return steady_state_probability(net, soi, mode, tol)
    pi, _ = stationary_implicit(net, mode, tol)
    return float(pi[soi_mask(net.n, soi)].sum()), pi
