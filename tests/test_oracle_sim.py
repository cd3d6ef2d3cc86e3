"""Pins of the oracle's simulator and exact solver (Sec. 2.1-2.2).

* one-step transition law: from every start state the empirical distribution
  of the next state matches the exact transition matrix built independently
  by oracle/exact.py (chi-square), for both perturbation readings;
* exact solver: power iteration agrees with an eigen/linear solve and with the
  exact rational solve of the hand-built 3-node PBN (golden file);
* invariants: sum pi = 1, pi > 0, ergodicity under the global reading, uniform
  stationary law of identity networks, the periodic all-NOT counter-example of
  the per-node reading;
* long-run frequencies of the simulator match the exact answer.
"""
import json
import os

import numpy as np
import pytest
import scipy.stats as st

import pbn_synth as S
from oracle import exact

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "three_node.json")


def _one_step_counts(orc, net, mode, s, reps, omega=1024, seed=11):
    """Counts of next states from start state s over reps*omega transitions."""
    counts = np.zeros(1 << net.n, dtype=np.int64)
    bits = np.array([(s >> i) & 1 for i in range(net.n)], dtype=np.uint8)
    w = (1 << np.arange(net.n)).astype(np.int64)
    for t in range(reps):
        states = np.tile(bits, (omega, 1))
        nxt, _ = orc.simulate(net, mode, seed, states, t0=1000 + 7 * t + s * 100003, steps=1, record=False)
        idx = (nxt.astype(np.int64) * w).sum(axis=1)
        counts += np.bincount(idx, minlength=1 << net.n)
    return counts


def _chi2_pvalue(counts, probs):
    total = counts.sum()
    exp = probs * total
    keep = exp >= 5
    o = np.append(counts[keep], counts[~keep].sum())
    e = np.append(exp[keep], exp[~keep].sum())
    if e[-1] < 5:  # fold the small remainder into the largest cell
        j = np.argmax(e[:-1]); o[j] += o[-1]; e[j] += e[-1]; o = o[:-1]; e = e[:-1]
    # cells the exact law gives probability 0 must never occur
    assert counts[probs == 0].sum() == 0
    return st.chisquare(o, e).pvalue


NETS = [
    ("three-node", lambda: S.three_node(1 / 16)),
    ("random-n4", lambda: S.random_pbn(123, 4, (1, 3), (1, 3), "fair", "uniform", 0.05)),
    ("random-n5-k0", lambda: S.from_lists(5, [
        [((), 1, 0.3), ((1, 2), 0b0110, 0.7)],
        [((0, 3, 4), 0b10010110, 1.0)],
        [((2,), 0b01, 0.5), ((4, 0), 0b1000, 0.25), ((1,), 0b10, 0.25)],
        [((0, 1, 2, 3, 4), 0x96696996, 1.0)],
        [((3,), 0b10, 0.9), ((), 0, 0.1)]], 0.1)),
]


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("name,make", NETS)
def test_one_step_law_matches_exact_matrix(orc, name, make, mode):
    net = make()
    assert orc.validate(net) == 0
    P = exact.transition_matrix(net, mode)
    pmin = 1.0
    for s in range(1 << net.n):
        c = _one_step_counts(orc, net, mode, s, reps=12)
        pmin = min(pmin, _chi2_pvalue(c, P[s]))
    # 2^n independent tests; a correct simulator fails this with prob ~1e-5
    assert pmin > 1e-6 / (1 << net.n), pmin


def test_exact_rows_are_distributions():
    for mode in (0, 1):
        for _, make in NETS:
            P = exact.transition_matrix(make(), mode)
            assert np.all(P >= 0)
            np.testing.assert_allclose(P.sum(axis=1), 1.0, rtol=0, atol=1e-13)


@pytest.mark.parametrize("mode", [0, 1])
def test_three_node_golden(mode):
    gold = json.load(open(GOLDEN))["per_node" if mode == 0 else "global"]
    net = S.three_node(1 / 16)
    P = exact.transition_matrix(net, mode)
    pi, _ = exact.stationary_power(P)
    np.testing.assert_allclose(pi, gold["pi"], rtol=1e-12, atol=0)
    assert abs(pi.sum() - 1.0) < 1e-13
    assert abs(pi[1::2].sum() - gold["p_v0_1"]) < 1e-12


def test_power_iteration_matches_linear_solve():
    for mode in (0, 1):
        net = S.random_pbn(5, 8, (1, 3), (1, 3), "fair", "uniform", 0.02)
        P = exact.transition_matrix(net, mode)
        pi, _ = exact.stationary_power(P)
        w, v = np.linalg.eig(P.T)
        k = np.argmin(np.abs(w - 1.0))
        ref = np.real(v[:, k]); ref = ref / ref.sum()
        np.testing.assert_allclose(pi, ref, rtol=1e-9, atol=1e-15)
        assert np.all(pi > 0)


def _is_primitive(P):
    """Irreducible and aperiodic: some power of the 0/1 pattern is all positive."""
    A = (P > 0).astype(np.float64)
    M = A.copy()
    for _ in range(2 * P.shape[0]):
        if np.all(M > 0):
            return True
        M = np.minimum(M @ A, 1.0)
    return False


def test_global_reading_is_ergodic_for_n_ge_2():
    for seed in range(6):
        net = S.random_pbn(seed, 2 + seed % 4, (1, 3), (1, 3), "fair", "uniform", 0.01)
        assert _is_primitive(exact.transition_matrix(net, 1))
    # the all-NOT network is ergodic under the global reading as well
    assert _is_primitive(exact.transition_matrix(S.all_not(3, 0.05), 1))


def test_per_node_reading_can_be_periodic():
    """Under the per-node reading every node of the all-NOT network flips at
    every step whether or not it is perturbed, so the chain has period 2: the
    ergodicity claim of Sec. 2.2 holds for the global reading only."""
    P = exact.transition_matrix(S.all_not(3, 0.05), 0)
    for s in range(8):
        assert P[s, s ^ 7] == pytest.approx(1.0, abs=1e-15)
    assert not _is_primitive(P)


def test_identity_network_uniform():
    for mode in (0, 1):
        net = S.all_identity(5, 0.03)
        pi, _ = exact.stationary_power(exact.transition_matrix(net, mode))
        np.testing.assert_allclose(pi, 1 / 32, rtol=1e-10)


def test_long_run_frequency_matches_exact(orc):
    """Time average of the simulated indicator vs the exact stationary
    probability of the tiny workload network; tolerance from batch means."""
    net, soi, _ = S.tiny_config()
    for mode in (0, 1):
        exact_p, _ = exact.steady_state_probability(net, soi, mode)
        omega, steps, burn = 64, 6000, 500
        st0 = orc.init_states(net, 3, omega)
        _, ind = orc.simulate(net, mode, 3, st0, 0, steps, soi)
        x = ind[:, burn:].astype(np.float64)
        chain_means = x.mean(axis=1)
        est = chain_means.mean()
        se = chain_means.std(ddof=1) / np.sqrt(omega)
        assert abs(est - exact_p) < 5 * se + 1e-4, (mode, est, exact_p, se)


def test_uniform_digit_layout(orc):
    """u of a chain is assembled from bit (chain % 32) of the 32 digit words,
    most significant digit first; digit words come from blocks b = 0..7."""
    seed, node, t, chain = 0x1234567890, 17, (5 << 32) + 99, 70
    key = [seed & 0xFFFFFFFF, seed >> 32]
    words = []
    for b in range(8):
        words += list(orc.philox4x32_10([node, t & 0xFFFFFFFF, (t >> 32) | (b << 24), chain >> 5], key))
    u = 0
    for d in range(32):
        u |= ((int(words[d]) >> (chain & 31)) & 1) << (31 - d)
    assert orc.uniform(seed, node, t, chain) == u


def test_uniforms_are_uniform(orc):
    rng = np.random.default_rng(0)
    us = np.array([orc.uniform(7, int(rng.integers(50)), int(rng.integers(1 << 40)), int(rng.integers(4096)))
                   for _ in range(20000)], dtype=np.float64) / 2.0 ** 32
    assert st.kstest(us, "uniform").pvalue > 1e-4


def test_quantisation_thresholds(orc):
    assert orc.perturb_threshold(0.0) == 0
    assert orc.perturb_threshold(1 / 16) == 1 << 28
    assert orc.perturb_threshold(0.01) == 42949673
    net = S.random_pbn(9, 30, (1, 4), (1, 3), "fair", "uniform", 0.001)
    thr = orc.select_thresholds(net).astype(np.int64)
    P32 = orc.perturb_threshold(net.p)
    p_e, probs = exact.category_probabilities(net)
    assert p_e == P32 / 2 ** 32
    for i in range(net.n):
        fs = list(net.functions_of(i))
        prev = P32
        for f in fs:
            assert thr[f] >= prev
            assert probs[f] == (thr[f] - prev) / 2 ** 32
            prev = thr[f]
        assert thr[fs[-1]] == 1 << 32
        assert abs(sum(probs[f] for f in fs) + p_e - 1.0) < 1e-15
