"""Pins of the exact solver's implicit step for 13 <= n <= 16 (oracle/exact.py:
ProductStep, stationary_implicit), the FP64 power iteration of Sec. 2.1 on
networks whose 2^n x 2^n transition matrix is never formed.

  * it equals the dense matrix's step pi P (n = 10..12, both perturbation
    readings of Sec. 2.2) and converges to the same stationary distribution;
  * sum pi = 1 and pi > 0 (p > 0 makes the chain ergodic, Sec. 2.2) at n = 14;
  * an all-identity network has the uniform law at n = 16 (both readings:
    every node flips with probability p and otherwise keeps its value);
  * a 16-node network made of five disjoint copies of the hand-built 3-node
    PBN (exact rational golden) and one identity node has, under the per-node
    reading, the product of the copies' exact laws and 1/2.  Copies sit on
    nodes (0,1,2), (3,4,5), (6,7,8), ...: the third straddles the split of
    the nodes into the two halves of the implicit step, and the copies are
    permuted within themselves so that parents point both up and down.
"""
import json
import os

import numpy as np
import pytest

import pbn_synth as S
from oracle import exact as E

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.mark.parametrize("n", [10, 11, 12])
@pytest.mark.parametrize("mode", [0, 1])
def test_implicit_step_equals_dense(n, mode):
    net = S.random_pbn(300 + n, n, (1, 3), (1, 4), "fair", "uniform", 0.05)
    P = E.transition_matrix(net, mode)
    step = E.ProductStep(net, mode)
    rng = np.random.default_rng(n)
    for _ in range(3):
        pi = rng.random(1 << n)
        pi /= pi.sum()
        a, b = pi @ P, step(pi)
        assert np.max(np.abs(a - b)) <= 1e-15 * max(1.0, np.max(np.abs(a))) + 1e-17
    # a point mass: the step returns row s of P itself
    s = int(rng.integers(1 << n))
    e = np.zeros(1 << n)
    e[s] = 1.0
    assert np.max(np.abs(step(e) - P[s])) <= 1e-15
    pd, _ = E.stationary_power(P)
    pim, _ = E.stationary_implicit(net, mode)
    assert np.max(np.abs(pd - pim)) <= 1e-12 * np.max(pd)


@pytest.mark.parametrize("mode", [0, 1])
def test_sum_one_and_positive_n14(mode):
    net = S.random_pbn(414, 14, (1, 3), (1, 3), "biased", "uniform", 0.05)
    pi, it = E.stationary_implicit(net, mode)
    assert abs(pi.sum() - 1.0) < 1e-12
    assert np.all(pi > 0.0)
    # pi is a fixed point of the step
    step = E.ProductStep(net, mode)
    assert np.abs(step(pi) - pi).sum() < 1e-13


@pytest.mark.parametrize("mode", [0, 1])
def test_all_identity_uniform_n16(mode):
    net = S.all_identity(16, 0.05)
    pi, it = E.stationary_implicit(net, mode)
    assert np.max(np.abs(pi - 2.0 ** -16)) < 1e-18
    # from a point mass the law after t steps is the product over nodes of
    # (1 + lam^t)/2 for the starting value and (1 - lam^t)/2 for the other,
    # lam = 1 - 2p (under GLOBAL the flip pattern gamma, zero included, has
    # the same product law, since no perturbation leaves the state unchanged)
    step = E.ProductStep(net, mode)
    p_e = E.perturb_threshold(0.05) / 2.0 ** 32
    s0 = 12345
    x = np.zeros(1 << 16)
    x[s0] = 1.0
    states = np.arange(1 << 16, dtype=np.int64)
    for t in range(1, 9):
        x = step(x)
        lam = (1.0 - 2.0 * p_e) ** t
        same = 16 - np.array([bin(int(v)).count("1") for v in (states ^ s0)])
        expect = ((1.0 + lam) / 2.0) ** same * ((1.0 - lam) / 2.0) ** (16 - same)
        assert np.max(np.abs(x - expect)) < 1e-15


def _three_node_blocks():
    """Five copies of the hand-built 3-node PBN on nodes 3b..3b+2, node v_j of
    copy b placed at 3b + perm_b[j], plus an identity node 15."""
    perms = [(0, 1, 2), (2, 0, 1), (1, 2, 0), (2, 1, 0), (0, 2, 1)]
    base = S.three_node(1.0 / 16)
    fns = [None] * 16
    for b, perm in enumerate(perms):
        place = [3 * b + perm[j] for j in range(3)]
        for j in range(3):
            fl = []
            for f in base.functions_of(j):
                par = [place[int(v)] for v in base.parents_of(f)]
                fl.append((par, int(base.truth_table[f]), float(base.select_prob[f])))
            fns[place[j]] = fl
    fns[15] = [([15], 0b10, 1.0)]
    return S.from_lists(16, fns, 1.0 / 16, "three-node-x5"), perms


def test_product_of_three_node_copies_n16():
    net, perms = _three_node_blocks()
    with open(os.path.join(GOLDEN, "three_node.json")) as f:
        g = json.load(f)
    pi3 = np.array([a / b for a, b in g["per_node"]["pi_num_den"]])
    states = np.arange(1 << 16, dtype=np.int64)
    expect = np.full(1 << 16, 0.5)
    for b, perm in enumerate(perms):
        idx = np.zeros(1 << 16, dtype=np.int64)
        for j in range(3):
            idx |= ((states >> (3 * b + perm[j])) & 1) << j
        expect *= pi3[idx]
    pi, it = E.stationary_implicit(net, 0)
    assert abs(pi.sum() - 1.0) < 1e-12
    assert np.max(np.abs(pi - expect)) < 1e-13 * np.max(expect) + 1e-18
    # marginal of one straddling copy's v0 equals the golden P(v0 = 1)
    soi = S.StateOfInterest([6 + perms[2][0]], [1])
    assert abs(pi[E.soi_mask(16, soi)].sum() - g["per_node"]["p_v0_1"]) < 1e-12


def test_any_size_entry_point():
    net = S.random_pbn(7, 13, (1, 2), (1, 3), "fair", "uniform", 0.1)
    soi = S.StateOfInterest([0, 5], [1, 0])
    prob, pi = E.steady_state_probability_any(net, soi, 0)
    assert 0.0 < prob < 1.0 and abs(pi.sum() - 1.0) < 1e-12
    small = S.random_pbn(7, 9, (1, 2), (1, 3), "fair", "uniform", 0.1)
    a, _ = E.steady_state_probability_any(small, soi, 1)
    b, _ = E.steady_state_probability(small, soi, 1)
    assert a == b


def _golden16():
    with open(os.path.join(GOLDEN, "exact_n16.json")) as f:
        return json.load(f)


def test_golden_n16_reproduces():
    """tests/golden/exact_n16.json is what its committed script computes."""
    import importlib.util
    spec = importlib.util.spec_from_file_location("make_exact_n16", os.path.join(GOLDEN, "make_exact_n16.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    fresh, g = mod.compute(), _golden16()
    for name in ("per_node", "global"):
        assert abs(fresh[name]["prob"] - g[name]["prob"]) < 1e-13


@pytest.mark.parametrize("mode,name", [(0, "per_node"), (1, "global")])
def test_oracle_within_r_of_exact_n16(orc, mode, name):
    """Alg. GR + Alg. 3 on the 16-node network: the estimate lies within r of
    the exact answer with frequency at least s over 40 seeds (Sec. 3.1)."""
    net, soi, cfg = S.exact_config(16)
    exact_p = _golden16()[name]["prob"]
    hits = 0
    for sd in range(40):
        o = orc.estimate_two_state(net, soi, seed=sd, mode=mode, omega=cfg["omega"], psi0=cfg["psi0"],
                                   rhat=cfg["rhat"], r=cfg["r"], s=cfg["s"], eps=cfg["eps"])
        assert o["status"] == 0, o
        assert o["N"] <= o["sample_size"] and o["M"] <= o["psi"]
        hits += abs(o["prob"] - exact_p) < cfg["r"]
    assert hits / 40 >= cfg["s"]
