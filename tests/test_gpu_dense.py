"""The dense class of the paper's sweep (Sec. 5.1, density 150-300: 12-16
functions of 10-15 inputs per node) on the CUDA path: trajectories and
indicator bitstreams bit-exact against the oracle under both perturbation
readings (the fused kernel's variant for nodes with more than 8 functions),
whole queries equal to the oracle's, sampled chains of a sweep-sized model,
and the schedules and the engine that do not take such networks refuse them
with PBN_ERR_UNSUPPORTED."""
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


def _dense(n=16, seed=1616):
    return S.random_pbn(seed, n, (12, 16), (10, min(15, n)), "biased", "uniform", 0.05, f"dense-n{n}")


NETS = [
    ("dense-n16", _dense(), S.StateOfInterest([0, 7], [1, 0]), 70),
    ("dense-n14-k14", _dense(14, 1414), S.StateOfInterest([0, 3], [1, 0]), 33),
    ("sweep-dense-n80", *S.sweep_config(80, "dense"), 40),
    ("mixed-l", S.random_pbn(99, 24, (1, 16), (2, 15), "fair", "uniform", 0.02), S.StateOfInterest([2], [1]), 64),
]


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("name,net,soi,omega", NETS, ids=[x[0] for x in NETS])
def test_dense_trajectories_bit_exact(P, name, net, soi, omega, mode):
    seed = 4242 + omega
    N = P.pbn_load(net)
    chunks = [37, 20]
    cs = P.ChainSet(N, omega, bits_cap=sum(chunks))
    P.pbn_init_chains(cs, seed, mode)
    ref = oracle.init_states(net, seed, omega)
    assert np.array_equal(cs.states_numpy(), ref)
    t0 = 0
    for k in chunks:
        P.pbn_run_chains(cs, k, seed, mode, soi)
        ref, ind = oracle.simulate(net, mode, seed, ref, t0, k, soi)
        assert np.array_equal(cs.states_numpy(), ref), (name, t0)
        assert np.array_equal(cs.indicator_numpy(t0, k), ind), (name, t0)
        t0 += k


def test_select_ahead_and_engine_refuse_dense(P):
    net = _dense()
    N = P.pbn_load(net)
    cs = P.ChainSet(N, 64, bits_cap=8)
    P.pbn_init_chains(cs, 1)
    with pytest.raises(P.PbnError) as e:
        P.pbn_run_chains(cs, 8, 1, P.PER_NODE, S.StateOfInterest([0], [1]), schedule="select_ahead")
    assert e.value.status == P.PBN_ERR_UNSUPPORTED
    # the automatic schedule takes the fused kernel instead
    P.pbn_run_chains(cs, 8, 1, P.PER_NODE, S.StateOfInterest([0], [1]))
    eng = P.Engine()
    with pytest.raises(P.PbnError) as e:
        eng.submit_two_state(N, S.StateOfInterest([0], [1]), omega=64, seed=1, psi0=256, r=0.01)
    assert e.value.status == P.PBN_ERR_UNSUPPORTED
    eng.close()


@pytest.mark.parametrize("mode", [0, 1])
def test_dense_query_equals_oracle(P, mode):
    net = _dense(14, 1414)
    soi = S.StateOfInterest([0, 3], [1, 0])
    N = P.pbn_load(net)
    kw = dict(omega=64, psi0=256, rhat=1.05, r=0.01, s=0.95, eps=1e-10)
    for seed in (1, 2):
        o = oracle.estimate_two_state(net, soi, seed=seed, mode=mode, **kw)
        g = P.pbn_estimate_two_state(N, soi, seed=seed, mode=mode, **kw)
        assert o["status"] == 0
        for k in ("psi", "gr_psi", "length", "sample_size", "ones", "gr_rounds", "ts_rounds", "M", "N"):
            assert g[k] == o[k], (seed, k)
        assert g["n4"] == o["n4"] and g["prob"] == o["prob"]
        assert g["alpha"] == o["alpha"] and g["beta"] == o["beta"]
        assert g["rhat"] == pytest.approx(o["rhat"], rel=1e-12)


def test_sweep_sized_dense_model_sampled_chains(P):
    """A sweep model of the dense class (n = 500, about 7000 functions and
    16 MB of truth tables, read from global memory) with 2048 chains in the
    launch shape the sweep uses: sampled chains replayed one by one by the
    oracle."""
    net, soi = S.sweep_config(500, "dense")
    N = P.pbn_load(net)
    omega, steps, seed = 2048, 24, 31337
    cs = P.ChainSet(N, omega, bits_cap=steps)
    P.pbn_init_chains(cs, seed)
    P.pbn_run_chains(cs, steps, seed, P.PER_NODE, soi)
    states, bits = cs.states_numpy(), cs.indicator_numpy(0, steps)
    for c in (0, 31, 32, 1000, omega - 1):
        st0 = oracle.init_states(net, seed, 1, chain0=c)
        ref, ind = oracle.simulate(net, 0, seed, st0, 0, steps, soi, chain0=c)
        assert np.array_equal(states[c], ref[0]), c
        assert np.array_equal(bits[c], ind[0]), c


@pytest.mark.parametrize("staging", ["tiles", "global"])
def test_dense_staging_modes_bit_exact(P, staging):
    """The dense variant with its function records streamed through shared
    memory as TMA tiles (several per step) or read from global memory: the
    same chains as the oracle."""
    net, soi = S.sweep_config(200, "dense")
    assert net.n_functions > 1536  # more than one tile of records
    N = P.pbn_load(net)
    omega, steps, seed = 64, 9, 515
    cs = P.ChainSet(N, omega, bits_cap=steps)
    P.pbn_init_chains(cs, seed)
    P.pbn_run_chains(cs, steps, seed, P.PER_NODE, soi, staging=staging)
    ref, ind = oracle.simulate(net, 0, seed, oracle.init_states(net, seed, omega), 0, steps, soi)
    assert np.array_equal(cs.states_numpy(), ref)
    assert np.array_equal(cs.indicator_numpy(0, steps), ind)
