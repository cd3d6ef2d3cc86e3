"""Pins of the oracle's sequential two-state driver (Sec. 3.1, Alg. 1): the
stopping rule, an independent replay of the final window, exact answers within
r, and the paper's check of the parallel method against the sequential one
(Sec. 5.1: estimates of the same property within 2r of each other)."""
import numpy as np
import pytest

import pbn_synth as S
from oracle import exact

KW = dict(m0=0, n0=1024, eps=1e-10, r=0.01, s=0.95)


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("chain", [0, 37])
def test_stopping_rule_and_replay(orc, mode, chain):
    net, soi, _ = S.tiny_config()
    out = orc.estimate_two_state_seq(net, soi, seed=5, mode=mode, chain=chain, **KW)
    assert out["status"] == 0
    L, N, M = out["length"], out["N"], out["M"]
    assert M + N <= L
    # alpha, beta come from the last N positions of the round (N before it is
    # recomputed), the estimate from the last N positions after it
    W = out["ab_window"]
    assert W <= L and sum(out["n4"]) == W - 1
    assert out["prob"] == out["ones"] / N
    c = out["n4"]
    assert out["alpha"] == c[1] / (c[0] + c[1]) and out["beta"] == c[2] / (c[2] + c[3])
    # replay chain `chain` with the simulator and recount both windows
    st0 = orc.init_states(net, 5, 1, chain0=chain)
    _, ind = orc.simulate(net, mode, 5, st0, 0, L, soi, chain0=chain)
    x = ind[0].astype(np.int64)
    assert out["ones"] == int(x[L - N:L].sum())
    pairs = 2 * x[L - W:L - 1] + x[L - W + 1:L]
    assert [int((pairs == v).sum()) for v in range(4)] == c


def test_rounds_grow_the_trajectory_to_m_plus_n(orc):
    """Every round extends to the recomputed M + N, so the final length is the
    M + N of the round before the last (or the initial m0 + n0)."""
    net = S.identity_node(0.02)
    soi = S.StateOfInterest([0], [1])
    out = orc.estimate_two_state_seq(net, soi, seed=1, **KW)
    assert out["status"] == 0 and out["rounds"] >= 2
    assert out["length"] > KW["m0"] + KW["n0"]


def _hit_rate(orc, net, soi, target, seeds, **kw):
    hits = 0
    for sd in seeds:
        out = orc.estimate_two_state_seq(net, soi, seed=sd, **kw)
        assert out["status"] == 0
        hits += abs(out["prob"] - target) < kw["r"]
    return hits / len(seeds)


def test_identity_node_within_r(orc):
    assert _hit_rate(orc, S.identity_node(0.1), S.StateOfInterest([0], [1]), 0.5, range(20), **KW) >= 0.8


def test_constant_node_within_r(orc):
    net = S.constant_node(0.05)
    p_eff = orc.perturb_threshold(0.05) / 2 ** 32
    assert _hit_rate(orc, net, S.StateOfInterest([0], [1]), 1 / (1 + p_eff), range(20), **KW) >= 0.8


@pytest.mark.parametrize("mode", [0, 1])
def test_tiny_workload_within_r_of_exact(orc, mode):
    net, soi, _ = S.tiny_config()
    target, _ = exact.steady_state_probability(net, soi, mode)
    assert _hit_rate(orc, net, soi, target, range(20), mode=mode, **KW) >= 0.8


def test_parallel_agrees_with_sequential(orc):
    """Sec. 5.1's correctness check: the two estimates of one property differ
    by less than 2r (expected with probability about 0.95)."""
    net, soi, _ = S.tiny_config()
    close = 0
    seeds = range(20)
    for sd in seeds:
        seq = orc.estimate_two_state_seq(net, soi, seed=sd, **KW)
        par = orc.estimate_two_state(net, soi, omega=8, seed=1000 + sd, psi0=256, rhat=1.1, r=KW["r"], s=KW["s"])
        assert seq["status"] == 0 and par["status"] == 0
        close += abs(seq["prob"] - par["prob"]) < 2 * KW["r"]
    assert close / len(seeds) >= 0.85


# ---------------------------------------------------------------- Alg. 2

@pytest.mark.parametrize("mode", [0, 1])
def test_skart_seq_bookkeeping_and_replay(orc, mode):
    net, soi, _ = S.tiny_config()
    out = orc.estimate_skart_seq(net, soi, seed=4, H_star=0.1, relative=True, mode=mode)
    assert out["status"] == 0
    k, b, d = out["kappa"], out["batches"], out["spacer"]
    assert out["psi"] == d * k and out["length"] == k * (b + d) and out["sample_size"] == k * b
    assert out["H"] <= 0.1 * abs(out["mean"])
    assert out["ci_lo"] <= out["mean"] <= out["ci_hi"]
    st0 = orc.init_states(net, 4, 1)
    _, ind = orc.simulate(net, mode, 4, st0, 0, out["length"], soi)
    x = ind[0, d * k:d * k + k * b].astype(np.float64)
    assert out["mean"] == pytest.approx(x.reshape(b, k).mean(axis=1).mean(), rel=1e-12)


def test_skart_seq_covers_a_known_mean(orc):
    """Identity node: the stationary mean of the indicator is exactly 1/2."""
    net, soi = S.identity_node(0.1), S.StateOfInterest([0], [1])
    covered = 0
    seeds = range(20)
    for sd in seeds:
        out = orc.estimate_skart_seq(net, soi, seed=sd, H_star=0.02, relative=False)
        assert out["status"] == 0 and out["H"] <= 0.02
        covered += out["ci_lo"] <= 0.5 <= out["ci_hi"]
    assert covered / len(seeds) >= 0.8


def test_skart_parallel_agrees_with_sequential(orc):
    net, soi = S.identity_node(0.1), S.StateOfInterest([0], [1])
    close = 0
    seeds = range(15)
    for sd in seeds:
        seq = orc.estimate_skart_seq(net, soi, seed=sd, H_star=0.02, relative=False)
        par = orc.estimate_skart(net, soi, omega=16, seed=500 + sd, H_star=0.02, relative=False, psi0=256, rhat=1.1)
        assert seq["status"] == 0 and par["status"] == 0
        close += abs(seq["mean"] - par["mean"]) < 2 * 0.02
    assert close / len(seeds) >= 0.85
