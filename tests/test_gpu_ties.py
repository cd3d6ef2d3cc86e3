"""Ties in the category draw (Sec. 2.2's draw of a uniform against the
category bounds, compared digit by digit, four digits per Philox block).  A
lane whose digits so far equal a bound's stays undecided until a later block
breaks the tie, and the warp runs further blocks while any lane of its items
is tied.  Covered here, bit-exact against the oracle: networks whose
neighbouring bounds share their first 8 digits (a selection probability below
2^-8, so that a lane is tied with two bounds at once), nodes with up to 8
functions (the out-of-line item variant) and a perturbation bound far from
zero, in the fused kernel with one thread per item and in the batched
engine."""
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


def close_bounds_net(n=48, seed=808, p=0.001):
    """Every third node has three functions with selection probabilities
    (0.5, 0.0005, 0.4995): its two thresholds lie about 2^21 apart, so most
    lanes tied with one after 8 digits are tied with both.  The other nodes
    have one or two functions of probability 0.3 / 0.7."""
    rng = np.random.default_rng(seed)
    fns = []
    for i in range(n):
        probs = [0.5, 0.0005, 0.4995] if i % 3 == 0 else ([1.0] if i % 3 == 1 else [0.3, 0.7])
        fl = []
        for c in probs:
            k = int(rng.integers(1, 5))
            par = [int(x) for x in rng.choice(n, size=k, replace=False)]
            tt = int(rng.integers(0, 1 << (1 << k)))
            fl.append((par, tt, c))
        fns.append(fl)
    return S.from_lists(n, fns, p, "close-bounds")


@pytest.mark.parametrize("mode", [0, 1])
def test_close_bounds_bit_exact(P, mode):
    net = close_bounds_net()
    soi = S.StateOfInterest([0, 3], [1, 0])
    N = P.pbn_load(net)
    omega, seed = 2000, 77
    cs = P.ChainSet(N, omega, bits_cap=60)
    P.pbn_init_chains(cs, seed)
    ref = oracle.init_states(net, seed, omega)
    t0 = 0
    for k in (31, 29):
        P.pbn_run_chains(cs, k, seed, mode, soi, threads_per_item=1)
        ref, ind = oracle.simulate(net, mode, seed, ref, t0, k, soi)
        assert np.array_equal(cs.states_numpy(), ref), t0
        assert np.array_equal(cs.indicator_numpy(t0, k), ind), t0
        t0 += k


def test_many_functions_bit_exact(P):
    """1-8 functions per node (bounds up to 8, the out-of-line item variant)
    and p = 0.05 (bound 0 far from zero): one thread per item."""
    net = S.random_pbn(606, 200, (1, 8), (2, 5), "biased", "uniform", 0.05)
    soi = S.StateOfInterest([5], [1])
    N = P.pbn_load(net)
    omega, seed = 1000, 4
    cs = P.ChainSet(N, omega, bits_cap=50)
    P.pbn_init_chains(cs, seed)
    P.pbn_run_chains(cs, 50, seed, P.PER_NODE, soi, threads_per_item=1)
    ref, ind = oracle.simulate(net, 0, seed, oracle.init_states(net, seed, omega), 0, 50, soi)
    assert np.array_equal(cs.states_numpy(), ref)
    assert np.array_equal(cs.indicator_numpy(0, 50), ind)


def test_engine_close_bounds_equals_oracle(P):
    net = close_bounds_net()
    soi = S.StateOfInterest([0, 3], [1, 0])
    kw = dict(omega=256, seed=22, psi0=256, rhat=1.05, r=0.01)
    eng = P.Engine()
    eng.submit_two_state(P.pbn_load(net), soi, tag=0, **kw)
    g = eng.run()[0]["report"]
    eng.close()
    o = oracle.estimate_two_state(net, soi, **kw)
    assert o["status"] == 0
    for key in ("psi", "gr_psi", "length", "sample_size", "ones", "gr_rounds", "ts_rounds", "M", "N"):
        assert g[key] == o[key], key
    assert g["prob"] == o["prob"]
