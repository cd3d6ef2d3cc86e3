"""Balanced fused launches (more chain groups than SMs, not a whole multiple):
phase 1 runs the SMs that carry one group more for fewer steps, phase 2
finishes those groups spread over all SMs.  Every chain still takes its own
transitions in order (Sec. 2.2), so states and indicator bitstreams must equal
the oracle's bit for bit, and equal those of the one-launch shape
(groups_per_block given explicitly, which keeps a single launch)."""
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


@pytest.fixture(scope="module")
def sms():
    import torch
    return torch.cuda.get_device_properties(0).multi_processor_count


def _groups(R, q, rem):
    return q * R + rem


def _run(P, net, soi, omega, seed, mode, chunks, **launch):
    N = P.pbn_load(net)
    cs = P.ChainSet(N, omega, bits_cap=sum(chunks))
    P.pbn_init_chains(cs, seed, mode)
    states = []
    for k in chunks:
        P.pbn_run_chains(cs, k, seed, mode, soi, **launch)
        states.append(cs.states_numpy().copy())
    return cs, states


# (q, share of SMs that carry q + 1 groups, ragged chains in the last group,
# nodes, threads per CTA).  One-warp CTAs make a group's items take more than
# one round, so that q and q + 1 groups differ in step cost and the launch is
# split; the default CTA of the 18-node network covers every item in one
# round (one launch: nothing to balance).
SHAPES = [(1, 3, 5, 18, 32), (3, None, 0, 18, 32), (2, 2, 17, 24, 32), (1, 3, 0, 18, 0)]


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("shape", SHAPES, ids=[f"q{s[0]}-n{s[3]}-t{s[4]}" for s in SHAPES])
def test_balanced_launches_bit_exact(P, sms, shape, mode):
    q, div, ragged, n, threads = shape
    # q = 3 with 56 of 152 SMs one group over: the 16384-chain workload
    rem = (56 * sms) // 152 if div is None else sms // div
    G = _groups(sms, q, rem)
    omega = 32 * G - ragged
    net = S.random_pbn(31 + q, n, (1, 4), (1, 5), "biased", "powerlaw", 0.01)
    soi = S.StateOfInterest([0, 3, 7], [1, 0, 1])
    seed = 0xBA1 + q
    chunks = [64, 77]  # each call long enough to be split into two phases
    launch = dict(threads_per_block=threads) if threads else {}
    cs, states = _run(P, net, soi, omega, seed, mode, chunks, **launch)
    ref = oracle.init_states(net, seed, omega)
    t0 = 0
    inds = []
    for k, got in zip(chunks, states):
        ref, ind = oracle.simulate(net, mode, seed, ref, t0, k, soi)
        inds.append(ind)
        assert np.array_equal(got, ref), (q, t0)
        t0 += k
    assert np.array_equal(cs.indicator_numpy(0, t0), np.concatenate(inds, axis=1))
    # the one-launch shape gives the same chains
    gpb = -(-G // sms)
    one, s1 = _run(P, net, soi, omega, seed, mode, chunks, groups_per_block=gpb, **launch)
    assert np.array_equal(s1[-1], states[-1])
    assert np.array_equal(one.indicator_numpy(0, t0), cs.indicator_numpy(0, t0))
    assert P.pbn_take_device_status() == 0


def test_balanced_launches_several_properties(P, sms):
    """Two recorded properties through the two phases (bitstream columns of
    phase 2 start at its step offset)."""
    G = _groups(sms, 1, sms // 2)
    omega = 32 * G
    net = S.random_pbn(41, 20, (1, 3), (2, 4), "fair", "uniform", 0.02)  # one-warp CTAs: 1 vs 2 rounds
    props = [S.StateOfInterest([0, 1], [1, 1]), S.StateOfInterest([5], [0])]
    N = P.pbn_load(net)
    cs = P.ChainSet(N, omega, bits_cap=100, n_props=2)
    P.pbn_init_chains(cs, 9, 0)
    P.pbn_run_chains(cs, 100, 9, 0, props=props, threads_per_block=32)
    init = oracle.init_states(net, 9, omega)
    for m, soi in enumerate(props):
        ref, ind = oracle.simulate(net, 0, 9, init, 0, 100, soi)
        assert np.array_equal(cs.indicator_numpy(0, 100, prop=m), ind)
    assert np.array_equal(cs.states_numpy(), ref)
