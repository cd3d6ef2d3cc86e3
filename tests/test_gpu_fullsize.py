"""Parity at the full sizes of the measured workloads, in the launch
configuration the driver uses: sampled chains replayed one by one by the
oracle (the oracle can simulate any single chain from its global index), and
properties that hold at any size for the whole-query statistics."""
import numpy as np
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


def _sampled_chains(omega, rng, k):
    picks = {0, omega - 1, omega // 2, 31, 32}
    picks |= set(int(x) for x in rng.integers(0, omega, size=k))
    return sorted(c for c in picks if c < omega)


def _replay_and_compare(P, net, soi, omega, seed, length, rng, k=3, **launch):
    N = P.pbn_load(net)
    cs = P.ChainSet(N, omega, bits_cap=length)
    P.pbn_init_chains(cs, seed)
    P.pbn_run_chains(cs, length, seed, P.PER_NODE, soi, **launch)
    states = cs.states_numpy()
    bits = cs.indicator_numpy(0, length)
    for c in _sampled_chains(omega, rng, k):
        st0 = oracle.init_states(net, seed, 1, chain0=c)
        ref, ind = oracle.simulate(net, 0, seed, st0, 0, length, soi, chain0=c)
        assert np.array_equal(states[c], ref[0]), c
        assert np.array_equal(bits[c], ind[0]), c
    return cs


def test_mid_workload_full_query(P):
    """The bench query (n = 100, 1024 chains, two-state r = 0.005): the report
    satisfies the method's invariants, and chains run to the query's length
    match the oracle chain by chain."""
    net, soi, cfg = S.mid_config()
    N = P.pbn_load(net)
    rep = P.pbn_estimate_two_state(N, soi, omega=cfg["omega"], seed=1_000_000, psi0=1024, rhat=cfg["rhat"],
                                   r=cfg["r"], s=cfg["s"], eps=cfg["eps"])
    n = rep["length"] - rep["psi"]
    assert sum(rep["n4"]) == cfg["omega"] * (n - 1)
    assert rep["sample_size"] == cfg["omega"] * n >= rep["N"]
    assert rep["M"] <= rep["psi"]
    assert rep["prob"] == rep["ones"] / (cfg["omega"] * n)
    assert rep["alpha"] == rep["n4"][1] / (rep["n4"][0] + rep["n4"][1])
    rng = np.random.default_rng(0)
    _replay_and_compare(P, net, soi, cfg["omega"], 1_000_000, rep["length"], rng)


def test_large_workload_sampled_chains(P):
    """n = 2000 scale-free, 16384 chains, the driver's automatic launch shape
    (and the other staging modes)."""
    net, nodes, cfg = S.large_config()
    soi = S.StateOfInterest(nodes, np.ones(10, dtype=np.uint8))
    rng = np.random.default_rng(1)
    _replay_and_compare(P, net, soi, cfg["omega"], 77, 60, rng, k=2)
    _replay_and_compare(P, net, soi, cfg["omega"], 78, 12, rng, k=1, staging="tiles")


def test_large_workload_skart(P):
    """Skart on the large network at relative precision 0.01: the target of
    the 10-node state of interest is chain 0's state after a burn-in (from
    the oracle), so the pattern has mass.  Checks the stopping rule, the
    parallel batch layout p = ceil(p/omega) omega (Alg. 4), and agreement with
    an independent two-state estimate of the same probability."""
    net, nodes, cfg = S.large_config()
    st, _ = oracle.simulate(net, 0, 5, oracle.init_states(net, 5, 1), 0, 1024, None, record=False)
    soi = S.StateOfInterest(nodes, st[0][nodes])
    N = P.pbn_load(net)
    omega = 4096
    sk = P.pbn_estimate_skart(N, soi, omega=omega, seed=9, H_star=cfg["rel"], relative=True, alpha=0.05, psi0=256,
                              rhat=1.05, max_length=1 << 19)
    assert sk["H"] <= cfg["rel"] * abs(sk["mean"])
    assert sk["batches"] % omega == 0 and sk["sample_size"] == sk["kappa"] * sk["batches"]
    assert sk["ci_lo"] <= sk["mean"] <= sk["ci_hi"]
    # two estimates, each within about H of the truth at 95%: their difference
    # has a standard deviation near 0.72 H, so 4 H is more than 5 of them
    ts = P.pbn_estimate_two_state(N, soi, omega=omega, seed=10, psi0=256, rhat=1.05, r=sk["H"], s=0.95,
                                  max_length=1 << 20)
    assert abs(ts["prob"] - sk["mean"]) < 4 * sk["H"], (ts["prob"], sk["mean"], sk["H"])


def test_wide_workload_sampled_chains(P):
    """n = 4096 with about 400 KB of function records, too many for shared
    memory: the automatic launch reads them from global memory; TMA tiles
    streamed through shared memory give the same chains."""
    net, nodes, cfg = S.wide_config()
    soi = S.StateOfInterest(nodes, np.ones(10, dtype=np.uint8))
    rng = np.random.default_rng(2)
    _replay_and_compare(P, net, soi, cfg["omega"], 91, 24, rng, k=1)
    _replay_and_compare(P, net, soi, cfg["omega"], 92, 8, rng, k=1, staging="tiles")


@pytest.mark.parametrize("schedule", ["fused", "select_ahead"])
def test_mid_workload_schedules_sampled_chains(P, schedule):
    """The mid network's 1024 chains over 2500 steps (three select-ahead
    chunks, the last one ragged) under both schedules."""
    net, soi, cfg = S.mid_config()
    rng = np.random.default_rng(3)
    _replay_and_compare(P, net, soi, cfg["omega"], 4242, 2500, rng, k=2, schedule=schedule)


def test_large_network_skart_several_batches_per_chain(P):
    """Alg. GR + Alg. 4 on the large network (n = 2000 scale-free) with 256
    chains, so that every chain holds several batches (p = ceil(p/omega)
    omega from 1280) and the randomness test and the lag-1 factor act on
    within-chain neighbours at this size.  The chains are replayed to the
    query's final length; the oracle's batch-means statistics on the
    replayed bitstream give the report's mean, variance, interval and
    half-width (1e-12 relative; skewness and correlation 1e-12 absolute), the
    randomness test passes on the accepted layout, and sampled chains match
    the oracle chain by chain."""
    net, nodes, cfg = S.large_config()
    st, _ = oracle.simulate(net, 0, 5, oracle.init_states(net, 5, 1), 0, 1024, None, record=False)
    soi = S.StateOfInterest(nodes[:2], st[0][nodes[:2]])
    N = P.pbn_load(net)
    omega, seed = 256, 11
    sk = P.pbn_estimate_skart(N, soi, omega=omega, seed=seed, H_star=0.05, relative=True, alpha=0.05, psi0=256,
                              rhat=1.05, max_length=1 << 18)
    bpc = sk["batches"] // omega
    assert bpc >= 2 and sk["batches"] % omega == 0
    kappa, start, L = sk["kappa"], sk["psi"], sk["length"]
    cs = P.ChainSet(N, omega, bits_cap=L)
    P.pbn_init_chains(cs, seed)
    P.pbn_run_chains(cs, L, seed, P.PER_NODE, soi)
    x = cs.indicator_numpy(start, kappa * bpc)
    means = x.reshape(omega, bpc, kappa).mean(axis=2).reshape(-1)
    ci = oracle.skart_ci(means, omega, bpc, 0.05)
    for k in ("mean", "var", "ci_lo", "ci_hi", "H"):
        assert sk[k] == pytest.approx(ci[k], rel=1e-12, abs=1e-15), k
    for k in ("skew", "phi"):
        assert sk[k] == pytest.approx(ci[k], rel=0, abs=1e-12), k
    if sk["ci_rounds"] == 1:
        # the interval was taken on the layout the randomness test accepted
        spaced_ok, _ = oracle.vonneumann_pass(means, omega, bpc, sk["spacer"], 0.2)
        assert spaced_ok
    states = cs.states_numpy()
    full = cs.indicator_numpy(0, L)
    for c in (0, 137, omega - 1):
        st0 = oracle.init_states(net, seed, 1, chain0=c)
        ref, ind = oracle.simulate(net, 0, seed, st0, 0, L, soi, chain0=c)
        assert np.array_equal(states[c], ref[0]), c
        assert np.array_equal(full[c], ind[0]), c
