"""Whole-method pins of the oracle drivers: Alg. GR followed by Alg. 3
(two-state, Sec. 4.2) or Alg. 4 (Skart, Sec. 4.3).  The estimate must lie
within the requested precision r of the exact steady-state probability with
about the requested confidence s (Sec. 3.1, Sec. 5.1's correctness check)."""
import numpy as np
import pytest

import pbn_synth as S
from oracle import exact


def _within_r_fraction(orc, net, soi, exact_p, seeds, **kw):
    hits = 0
    for sd in seeds:
        out = orc.estimate_two_state(net, soi, seed=sd, **kw)
        assert out["status"] == 0, out
        assert out["N"] <= out["sample_size"]
        assert out["M"] <= out["psi"]
        hits += abs(out["prob"] - exact_p) < kw["r"]
    return hits / len(seeds)


@pytest.mark.parametrize("mode", [0, 1])
def test_identity_node_two_state(orc, mode):
    net = S.identity_node(0.1)
    soi = S.StateOfInterest([0], [1])
    frac = _within_r_fraction(orc, net, soi, 0.5, range(20), omega=8, psi0=256, rhat=1.1,
                              r=0.01, s=0.95, eps=1e-10, mode=mode)
    assert frac >= 0.8


def test_identity_node_alpha_beta(orc):
    out = orc.estimate_two_state(S.identity_node(0.1), S.StateOfInterest([0], [1]), omega=16, seed=3,
                                 psi0=256, rhat=1.1, r=0.005, s=0.95)
    p_eff = orc.perturb_threshold(0.1) / 2 ** 32
    # alpha, beta estimate p with binomial error on ~N/2 transitions each
    se = np.sqrt(p_eff * (1 - p_eff) / (out["sample_size"] / 2))
    assert abs(out["alpha"] - p_eff) < 5 * se
    assert abs(out["beta"] - p_eff) < 5 * se


def test_constant_node_two_state(orc):
    net = S.constant_node(0.05)
    soi = S.StateOfInterest([0], [1])
    p_eff = orc.perturb_threshold(0.05) / 2 ** 32
    frac = _within_r_fraction(orc, net, soi, 1 / (1 + p_eff), range(20), omega=8, psi0=256, rhat=1.1,
                              r=0.01, s=0.95, eps=1e-10, mode=0)
    assert frac >= 0.8


@pytest.mark.parametrize("mode", [0, 1])
def test_tiny_workload_within_r_of_exact(orc, mode):
    net, soi, cfg = S.tiny_config()
    exact_p, _ = exact.steady_state_probability(net, soi, mode)
    frac = _within_r_fraction(orc, net, soi, exact_p, range(20), omega=cfg["omega"], psi0=1024,
                              rhat=cfg["rhat"], r=cfg["r"], s=cfg["s"], eps=cfg["eps"], mode=mode)
    assert frac >= 0.8


def test_three_node_two_state(orc):
    import json, os
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "three_node.json")))
    net = S.three_node(1 / 16)
    soi = S.StateOfInterest([0], [1])
    frac = _within_r_fraction(orc, net, soi, gold["per_node"]["p_v0_1"], range(12), omega=32, psi0=512,
                              rhat=1.05, r=0.01, s=0.95, eps=1e-10, mode=0)
    assert frac >= 0.75


def test_skart_identity_node(orc):
    """Mean 1/2 exactly; relative precision 0.05 -> the CI covers 1/2 in most runs."""
    net = S.identity_node(0.2)
    soi = S.StateOfInterest([0], [1])
    covered = 0
    for sd in range(12):
        out = orc.estimate_skart(net, soi, omega=16, seed=sd, H_star=0.05, relative=True, alpha=0.05,
                                 psi0=256, rhat=1.1)
        assert out["status"] == 0, out
        assert out["H"] <= 0.05 * abs(out["mean"]) + 1e-15
        assert out["batches"] % 16 == 0        # p = ceil(p/omega) omega (Alg. 4)
        covered += out["ci_lo"] <= 0.5 <= out["ci_hi"]
    assert covered >= 9


def test_skart_tiny_workload(orc):
    net, soi, cfg = S.tiny_config()
    exact_p, _ = exact.steady_state_probability(net, S.StateOfInterest([3], [1]), 0)
    out = orc.estimate_skart(net, S.StateOfInterest([3], [1]), omega=8, seed=5, H_star=0.01, relative=False,
                             alpha=0.05, psi0=1024, rhat=1.1)
    assert out["status"] == 0
    assert abs(out["mean"] - exact_p) < 3 * out["H"]


def test_constant_node_alpha_beta_not_swapped(orc):
    """Constant-1 node, per-node reading: alpha = 1 (0 -> 1 always), beta = p."""
    out = orc.estimate_two_state(S.constant_node(0.05), S.StateOfInterest([0], [1]), omega=16, seed=4,
                                 psi0=256, rhat=1.1, r=0.005, s=0.95, mode=0)
    assert out["alpha"] == 1.0
    assert abs(out["beta"] - 0.05) < 0.01


@pytest.mark.parametrize("mode", [0, 1])
def test_periodic_chain_is_not_converged(orc, mode):
    """NOT node: under both perturbation readings the node flips at every
    step, so the indicator alternates.  Every chain then has psi/2 ones in
    each window: B = 0 and R-hat = sqrt(1 - 1/psi) exactly (Alg. GR), every
    transition is 0->1 or 1->0 (alpha = beta = 1), and Alg. 3 cannot size a
    sample: PBN_ERR_NOT_CONVERGED."""
    omega, psi0 = 8, 64
    out = orc.estimate_two_state(S.not_node(0.05), S.StateOfInterest([0], [1]), omega=omega, seed=3, psi0=psi0,
                                 rhat=1.1, r=0.01, s=0.95, mode=mode)
    assert out["status"] == 5
    assert out["rhat"] == pytest.approx(np.sqrt(1 - 1 / psi0), rel=1e-15)
    half = omega * (psi0 - 1) // 2
    assert out["n4"] == [0, half, half, 0]
