"""Whole-method check of the CUDA path against exact answers above the dense
solver's reach: on the 16-node network of pbn_synth.exact_config (p = 0.05),
pbn_estimate_two_state (Alg. GR then Alg. 3, Sec. 4.2) equals the oracle's
estimate_two_state decision by decision for every seed, and its estimate lies
within r of the exact steady-state probability (FP64 power iteration over all
65536 states, tests/golden/exact_n16.json) with frequency at least s over 40
seeds, under both perturbation readings of Sec. 2.2."""
import json
import os

import pytest

import oracle
import pbn_synth as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    from paper_1508_07828_gb300 import _build
    _build.build()
    import paper_1508_07828_gb300 as P
    return P


@pytest.mark.parametrize("mode,name", [(0, "per_node"), (1, "global")])
def test_n16_within_r_and_equal_to_oracle(P, mode, name):
    with open(os.path.join(os.path.dirname(__file__), "golden", "exact_n16.json")) as f:
        exact_p = json.load(f)[name]["prob"]
    net, soi, cfg = S.exact_config(16)
    N = P.pbn_load(net)
    kw = dict(omega=cfg["omega"], psi0=cfg["psi0"], rhat=cfg["rhat"], r=cfg["r"], s=cfg["s"], eps=cfg["eps"])
    hits = 0
    for sd in range(40):
        o = oracle.estimate_two_state(net, soi, seed=sd, mode=mode, **kw)
        g = P.pbn_estimate_two_state(N, soi, seed=sd, mode=mode, **kw)
        assert o["status"] == 0
        for k in ("psi", "gr_psi", "length", "sample_size", "ones", "gr_rounds", "ts_rounds", "M", "N"):
            assert g[k] == o[k], (sd, k, g[k], o[k])
        assert g["n4"] == o["n4"]
        assert g["prob"] == o["prob"] and g["alpha"] == o["alpha"] and g["beta"] == o["beta"]
        assert g["rhat"] == pytest.approx(o["rhat"], rel=1e-12)
        hits += abs(g["prob"] - exact_p) < cfg["r"]
    assert hits / 40 >= cfg["s"]
