"""Several properties from the same trajectories (Sec. 4.2, last part) on the
GPU: every property's indicator bitstream bit-exact against the oracle's
simulator under both schedules, one property reducing to the single-property
driver, and the multi-property driver matching the oracle's decision by
decision."""
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


def _props_of(net):
    rng = np.random.default_rng(net.n)
    props = [S.random_soi(rng, net.n, 1, 4) for _ in range(3)]
    props.append(S.StateOfInterest([0, 0], [1, 0]))  # names node 0 twice: never holds
    return props


NETS = [("tiny", S.tiny_config()[0], 8), ("mid", S.mid_config()[0], 70),
        ("k0-mix", S.from_lists(5, [[((), 1, 0.3), ((1, 2), 0b0110, 0.7)], [((0, 3, 4), 0b10010110, 1.0)],
                                    [((2,), 0b01, 0.5), ((4, 0), 0b1000, 0.25), ((1,), 0b10, 0.25)],
                                    [((0, 1, 2, 3, 4), 0x96696996, 1.0)], [((3,), 0b10, 0.9), ((), 0, 0.1)]], 0.1),
         33),
        ("scalefree-300", S.random_pbn(5, 300, (1, 4), (2, 5), "biased", "powerlaw", 0.01), 64)]


@pytest.mark.parametrize("schedule", ["fused", "select_ahead"])
@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("name,net,omega", NETS, ids=[x[0] for x in NETS])
def test_every_property_bitstream_bit_exact(P, name, net, omega, mode, schedule):
    props = _props_of(net)
    N = P.pbn_load(net)
    chunks = [37, 1100] if schedule == "select_ahead" else [37, 60]
    total = sum(chunks)
    cs = P.ChainSet(N, omega, bits_cap=total, n_props=len(props))
    P.pbn_init_chains(cs, 21, mode)
    for k in chunks:
        P.pbn_run_chains(cs, k, 21, mode, props=props, schedule=schedule)
    st0 = oracle.init_states(net, 21, omega)
    for m, soi in enumerate(props):
        ref, ind = oracle.simulate(net, mode, 21, st0, 0, total, soi)
        assert np.array_equal(cs.indicator_numpy(0, total, prop=m), ind), (name, m)
    assert np.array_equal(cs.states_numpy(), ref)
    assert not cs.indicator_numpy(0, total, prop=3).any()


def test_one_property_is_the_single_driver(P):
    net, soi, _ = S.mid_config()
    N = P.pbn_load(net)
    kw = dict(omega=256, seed=5, psi0=512, rhat=1.05, r=0.01)
    single = P.pbn_estimate_two_state(N, soi, **kw)
    multi = P.pbn_estimate_two_state_multi(N, [soi], **kw)
    for k in ("prob", "rhat", "alpha", "beta", "psi", "gr_psi", "length", "sample_size", "M", "N", "ones", "n4",
              "gr_rounds", "ts_rounds"):
        assert multi[k] == single[k], k
    p = multi["properties"][0]
    for k in ("prob", "alpha", "beta", "M", "N", "ones", "n4"):
        assert p[k] == single[k], k


@pytest.mark.parametrize("case", ["tiny", "tiny-global", "mid-small"])
def test_multi_driver_matches_oracle(P, case):
    if case.startswith("tiny"):
        net, soi, _ = S.tiny_config()
        props = [soi, S.StateOfInterest([5], [0]), S.StateOfInterest([1, 2], [1, 1])]
        kw = dict(omega=8, psi0=256, rhat=1.1, r=0.01)
    else:
        net, soi, _ = S.mid_config()
        props = [soi, S.StateOfInterest([7], [1]), S.StateOfInterest([3, 9, 11], [0, 1, 1])]
        kw = dict(omega=64, psi0=512, rhat=1.05, r=0.01)
    mode = 1 if case.endswith("global") else 0
    N = P.pbn_load(net)
    for seed in (1, 2):
        o = oracle.estimate_two_state_multi(net, props, seed=seed, mode=mode, **kw)
        assert o["status"] == 0
        g = P.pbn_estimate_two_state_multi(N, props, seed=seed, mode=mode, **kw)
        for k in ("psi", "gr_psi", "length", "sample_size", "gr_rounds", "ts_rounds"):
            assert g[k] == o[k], k
        assert g["rhat"] == pytest.approx(o["rhat"], rel=1e-12)
        for gp, op in zip(g["properties"], o["properties"]):
            for k in ("prob", "alpha", "beta", "M", "N", "ones", "n4"):
                assert gp[k] == op[k], k
            assert gp["rhat"] == pytest.approx(op["rhat"], rel=1e-12)
