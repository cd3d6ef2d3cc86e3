"""Predictor functions with more than five inputs on the GPU (truth tables of
several words, looked up chain by chain by a warp): trajectories bit-exact
against the oracle under both schedules, every staging and both perturbation
readings; the estimate drivers and the engine on such networks."""
import numpy as np
import pytest

import oracle
import pbn_synth as S
from test_oracle_wide_tt import _parity_majority_net

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    from paper_1508_07828_gb300 import _build
    _build.build()
    import paper_1508_07828_gb300 as P
    return P


def _wide_random(n=300, seed=41):
    return S.random_pbn(seed, n, (1, 4), (2, 9), "biased", "powerlaw", 0.01, f"wide-k9-n{n}")


def _check_trajectories(P, net, soi, omega, seed, mode, chunks, **launch):
    N = P.pbn_load(net)
    total = sum(chunks)
    cs = P.ChainSet(N, omega, bits_cap=total)
    P.pbn_init_chains(cs, seed, mode)
    for k in chunks:
        P.pbn_run_chains(cs, k, seed, mode, soi, **launch)
    ref, ind = oracle.simulate(net, mode, seed, oracle.init_states(net, seed, omega), 0, total, soi)
    assert np.array_equal(cs.states_numpy(), ref)
    assert np.array_equal(cs.indicator_numpy(0, total), ind)


@pytest.mark.parametrize("schedule", ["fused", "select_ahead"])
@pytest.mark.parametrize("mode", [0, 1])
def test_parity_majority_bit_exact(P, schedule, mode):
    net = _parity_majority_net()
    net.p = 0.02  # perturbations on, so the chains wander
    _check_trajectories(P, net, S.StateOfInterest([0, 1], [1, 0]), 70, 9, mode, [33, 20], schedule=schedule)


@pytest.mark.parametrize("schedule", ["fused", "select_ahead"])
@pytest.mark.parametrize("staging", ["auto", "smem", "global", "tiles"])
def test_random_wide_network_bit_exact(P, schedule, staging):
    if schedule == "select_ahead" and staging == "tiles":
        pytest.skip("select-ahead takes whole tables or global reads")
    net = _wide_random()
    assert np.diff(net.par_offset).max() >= 8
    for mode in (0, 1):
        _check_trajectories(P, net, S.StateOfInterest([1, 2, 3], [1, 0, 1]), 40, 13, mode, [17, 9],
                            schedule=schedule, staging=staging)


def test_wide_networks_run_one_thread_per_item(P):
    N = P.pbn_load(_wide_random())
    cs = P.ChainSet(N, 64)
    P.pbn_init_chains(cs, 1)
    with pytest.raises(P.PbnError) as e:
        P.pbn_run_chains(cs, 3, 1, schedule="fused", threads_per_item=2)
    assert e.value.status == P.PBN_ERR_UNSUPPORTED


def test_estimate_on_wide_network_matches_oracle(P):
    net = _wide_random(n=60, seed=5)
    soi = S.StateOfInterest([0, 4], [1, 1])
    kw = dict(omega=64, psi0=256, rhat=1.05, r=0.02)
    o = oracle.estimate_two_state(net, soi, seed=3, **kw)
    assert o["status"] == 0
    g = P.pbn_estimate_two_state(P.pbn_load(net), soi, seed=3, **kw)
    for k in ("psi", "gr_psi", "length", "sample_size", "ones", "n4", "prob", "alpha", "beta", "M", "N",
              "gr_rounds", "ts_rounds"):
        assert g[k] == o[k], k


def test_engine_on_wide_network_matches_alone(P):
    net = _wide_random(n=60, seed=5)
    soi = S.StateOfInterest([0, 4], [1, 1])
    N = P.pbn_load(net)
    kw = dict(omega=64, seed=3, psi0=256, rhat=1.05, r=0.02)
    alone = P.pbn_estimate_two_state(N, soi, **kw)
    eng = P.Engine()
    eng.submit_two_state(N, soi, tag=1, **kw)
    eng.submit_two_state(P.pbn_load(S.mid_config()[0]), S.mid_config()[1], tag=2, omega=256, seed=4, psi0=256,
                         rhat=1.05, r=0.01)
    res = {r["tag"]: r for r in eng.run()}
    eng.close()
    assert res[1]["status"] == 0
    for k in ("prob", "length", "ones", "n4", "M", "N", "psi"):
        assert res[1]["report"][k] == alone[k], k
