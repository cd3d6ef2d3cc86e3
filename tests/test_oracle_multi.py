"""Pins of the oracle's multi-property driver (Sec. 4.2, last part: q
properties abstracted from the same trajectories).  It must reduce to Alg. 3
for one property, abstract every property from the very chains the simulator
produces, satisfy the stopping rule for every property, and estimate each
property within r of its exact steady-state probability."""
import numpy as np
import pytest

import pbn_synth as S
from oracle import exact

KW = dict(omega=8, psi0=256, rhat=1.1, r=0.01, s=0.95, eps=1e-10)
RUN_KEYS = ("prob", "rhat", "alpha", "beta", "psi", "gr_psi", "length", "sample_size", "M", "N", "ones", "n4",
            "gr_rounds", "ts_rounds", "status")


def _tiny_props():
    net, soi, _ = S.tiny_config()
    return net, [soi, S.StateOfInterest([5], [0]), S.StateOfInterest([1, 2], [1, 1])]


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_one_property_is_alg3(orc, mode, seed):
    net, props = _tiny_props()
    single = orc.estimate_two_state(net, props[0], seed=seed, mode=mode, **KW)
    multi = orc.estimate_two_state_multi(net, props[:1], seed=seed, mode=mode, **KW)
    for k in RUN_KEYS:
        assert multi[k] == single[k], k
    p = multi["properties"][0]
    for k in ("prob", "alpha", "beta", "M", "N", "ones", "n4"):
        assert p[k] == single[k], k


@pytest.mark.parametrize("seed", [3, 4])
def test_repeated_property_changes_nothing(orc, seed):
    net, props = _tiny_props()
    single = orc.estimate_two_state(net, props[1], seed=seed, **KW)
    multi = orc.estimate_two_state_multi(net, [props[1]] * 3, seed=seed, **KW)
    for k in RUN_KEYS:
        assert multi[k] == single[k], k
    for p in multi["properties"]:
        assert p["prob"] == single["prob"] and p["n4"] == single["n4"]


@pytest.mark.parametrize("mode", [0, 1])
def test_complementary_properties_split_the_window(orc, mode):
    net, _ = _tiny_props()
    a, b = S.StateOfInterest([3], [1]), S.StateOfInterest([3], [0])
    out = orc.estimate_two_state_multi(net, [a, b], seed=9, mode=mode, **KW)
    assert out["status"] == 0
    pa, pb = out["properties"]
    assert pa["ones"] + pb["ones"] == out["sample_size"]
    assert abs(pa["prob"] + pb["prob"] - 1.0) < 1e-15
    # n01 of one property is n10 of the other, and n00 / n11 swap
    assert pa["n4"] == [pb["n4"][3], pb["n4"][2], pb["n4"][1], pb["n4"][0]]


@pytest.mark.parametrize("mode", [0, 1])
def test_every_property_abstracts_the_same_trajectories(orc, mode):
    """Replay the chains with the simulator and count every property's ones
    in the final window independently."""
    net, props = _tiny_props()
    out = orc.estimate_two_state_multi(net, props, seed=11, mode=mode, **KW)
    assert out["status"] == 0
    L, psi = out["length"], out["psi"]
    st0 = orc.init_states(net, 11, KW["omega"])
    for m, soi in enumerate(props):
        _, ind = orc.simulate(net, mode, 11, st0, 0, L, soi)
        assert out["properties"][m]["ones"] == int(ind[:, psi:L].sum()), m


def test_stopping_rule_holds_for_every_property(orc):
    net, props = _tiny_props()
    for seed in range(5):
        out = orc.estimate_two_state_multi(net, props, seed=seed, **KW)
        assert out["status"] == 0
        assert out["rhat"] < KW["rhat"]
        for p in out["properties"]:
            assert p["N"] <= out["sample_size"]
            assert p["M"] <= out["psi"]
            assert p["rhat"] < KW["rhat"]
        # the burn-in is the largest M or the Gelman-Rubin psi
        assert out["psi"] in [out["gr_psi"]] + [p["M"] for p in out["properties"]]


@pytest.mark.parametrize("mode", [0, 1])
def test_each_property_within_r_of_exact(orc, mode):
    net, props = _tiny_props()
    exact_p = [exact.steady_state_probability(net, soi, mode)[0] for soi in props]
    hits = np.zeros(len(props))
    seeds = range(20)
    for sd in seeds:
        out = orc.estimate_two_state_multi(net, props, seed=sd, mode=mode, **KW)
        assert out["status"] == 0
        hits += [abs(p["prob"] - e) < KW["r"] for p, e in zip(out["properties"], exact_p)]
    assert (hits / len(seeds) >= 0.8).all(), hits
