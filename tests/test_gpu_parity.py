"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Bit-exact: initial states, trajectories (states after every launch), the
indicator bitstream, exact integer sums (G&R S1/S2, transition counts, batch
sums).  FP64 statistics: R-hat, alpha, beta to 1e-12 relative (both sides
form them from the same integers; alpha and beta are single correctly
rounded divisions and must agree exactly), M and N exactly unless the value
before ceil lies within 1e-12 relative of an integer, Skart statistics to
1e-12 (relative for the mean, variance and interval, absolute for the
skewness and lag-1 correlation; moments are formed differently on the two
sides: exact shifted integer moments on the GPU, two-pass FP64 over means in
the oracle).
"""
import math

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


def _nets():
    big_l = S.random_pbn(77, 10, (8, 8), (0, 5), "fair", "uniform", 0.05, "l8")
    return [
        ("tiny", *S.tiny_config()[:2], 8),
        ("three-node", S.three_node(1 / 16), S.StateOfInterest([0, 2], [1, 0]), 40),
        ("mid", *S.mid_config()[:2], 70),
        ("scalefree-300", S.random_pbn(5, 300, (1, 4), (2, 5), "biased", "powerlaw", 0.001),
         S.StateOfInterest(np.arange(10), [1, 0] * 5), 64),
        ("k0-mix", S.from_lists(5, [
            [((), 1, 0.3), ((1, 2), 0b0110, 0.7)],
            [((0, 3, 4), 0b10010110, 1.0)],
            [((2,), 0b01, 0.5), ((4, 0), 0b1000, 0.25), ((1,), 0b10, 0.25)],
            [((0, 1, 2, 3, 4), 0x96696996, 1.0)],
            [((3,), 0b10, 0.9), ((), 0, 0.1)]], 0.1), S.StateOfInterest([3], [1]), 33),
        ("identity-p0.3", S.identity_node(0.3), S.StateOfInterest([0], [1]), 32),
        ("p0", S.random_pbn(8, 20, (1, 3), (1, 4), "fair", "uniform", 0.0), S.StateOfInterest([1, 2], [0, 1]), 31),
        ("l8", big_l, S.StateOfInterest([0, 5], [1, 1]), 35),
        ("high-p", S.random_pbn(9, 12, (1, 3), (1, 3), "fair", "uniform", 0.4), S.StateOfInterest([4], [0]), 96),
    ]


NETS = _nets()


def _gpu_run(P, net, soi, omega, seed, mode, chunks, **launch):
    N = P.pbn_load(net)
    total = sum(chunks)
    cs = P.ChainSet(N, omega, bits_cap=total)
    P.pbn_init_chains(cs, seed, mode)
    init = cs.states_numpy().copy()
    states = []
    for k in chunks:
        P.pbn_run_chains(cs, k, seed, mode, soi, **launch)
        states.append(cs.states_numpy().copy())
    return cs, init, states


@pytest.mark.parametrize("schedule", ["fused", "select_ahead"])
@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("name,net,soi,omega", NETS, ids=[x[0] for x in NETS])
def test_trajectories_bit_exact(P, name, net, soi, omega, mode, schedule):
    seed = 0xC0FFEE + omega
    chunks = [50, 27]
    cs, init, states = _gpu_run(P, net, soi, omega, seed, mode, chunks, schedule=schedule)
    ref = oracle.init_states(net, seed, omega)
    assert np.array_equal(init, ref)
    t0 = 0
    inds = []
    for k, got in zip(chunks, states):
        ref, ind = oracle.simulate(net, mode, seed, ref, t0, k, soi)
        inds.append(ind)
        assert np.array_equal(got, ref), (name, t0)
        t0 += k
    assert np.array_equal(cs.indicator_numpy(0, t0), np.concatenate(inds, axis=1))


LAUNCHES = [dict(groups_per_block=2), dict(groups_per_block=3, threads_per_block=64), dict(threads_per_block=32),
            dict(threads_per_item=1, blocks_per_round=1), dict(threads_per_item=1, blocks_per_round=2),
            dict(threads_per_item=2), dict(threads_per_item=4), dict(threads_per_item=4, groups_per_block=2),
            dict(threads_per_item=2, threads_per_block=96)]


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("launch", LAUNCHES, ids=[str(x) for x in LAUNCHES])
def test_launch_shape_does_not_change_results(P, launch, mode):
    net, soi = S.mid_config()[:2]
    a, _, sa = _gpu_run(P, net, soi, 200, 3, mode, [40])
    b, _, sb = _gpu_run(P, net, soi, 200, 3, mode, [40], **launch)
    assert np.array_equal(sa[-1], sb[-1])
    assert np.array_equal(a.indicator_numpy(0, 40), b.indicator_numpy(0, 40))


@pytest.mark.parametrize("launch", [dict(threads_per_item=1, blocks_per_round=1), dict(threads_per_item=2),
                                    dict(threads_per_item=4)], ids=["t1b1", "t2", "t4"])
@pytest.mark.parametrize("name", ["k0-mix", "l8", "scalefree-300", "high-p"])
def test_item_thread_variants_bit_exact(P, name, launch):
    net, soi, omega = next((x[1], x[2], x[3]) for x in NETS if x[0] == name)
    for mode in (0, 1):
        cs, init, states = _gpu_run(P, net, soi, omega, 77, mode, [33], **launch)
        ref, ind = oracle.simulate(net, mode, 77, oracle.init_states(net, 77, omega), 0, 33, soi)
        assert np.array_equal(states[-1], ref)
        assert np.array_equal(cs.indicator_numpy(0, 33), ind)


@pytest.mark.parametrize("gpb", [0, 3])
@pytest.mark.parametrize("name", ["k0-mix", "l8", "scalefree-300", "high-p", "three-node"])
def test_resident_apply_with_more_functions_bit_exact(P, name, gpb):
    """The select-ahead schedule with one thread per item asked for: the
    register-resident apply, with its path for nodes of more than two
    functions (up to eight in l8), one or three chain groups per CTA, both
    perturbation readings, a call that spans two chunks: the oracle's chains."""
    net, soi, omega = next((x[1], x[2], x[3]) for x in NETS if x[0] == name)
    for mode in (0, 1):
        cs, init, states = _gpu_run(P, net, soi, 3 * omega, 41, mode, [37, 2100], schedule="select_ahead",
                                    threads_per_item=1, groups_per_block=gpb)
        ref = oracle.init_states(net, 41, 3 * omega)
        t0, inds = 0, []
        for k, got in zip([37, 2100], states):
            ref, ind = oracle.simulate(net, mode, 41, ref, t0, k, soi)
            inds.append(ind)
            assert np.array_equal(got, ref), (name, mode, t0)
            t0 += k
        assert np.array_equal(cs.indicator_numpy(0, t0), np.concatenate(inds, axis=1))


@pytest.mark.parametrize("schedule", ["fused", "select_ahead"])
def test_max_nodes_and_max_soi(P, schedule):
    net = S.random_pbn(31, 4096, (1, 2), (0, 5), "biased", "uniform", 0.002)
    soi = S.StateOfInterest(np.arange(0, 4096, 128), np.arange(32) % 2)
    cs, init, states = _gpu_run(P, net, soi, 33, 17, 0, [6], schedule=schedule)
    ref0 = oracle.init_states(net, 17, 33)
    ref, ind = oracle.simulate(net, 0, 17, ref0, 0, 6, soi)
    assert np.array_equal(states[-1], ref)
    assert np.array_equal(cs.indicator_numpy(0, 6), ind)


SA_LAUNCHES = [dict(groups_per_block=2), dict(groups_per_block=3, threads_per_block=64), dict(threads_per_block=32),
               dict(staging="smem"), dict(staging="global"),
               dict(groups_per_block=7, threads_per_block=1024, threads_per_item=4),
               dict(groups_per_block=7, threads_per_block=512, threads_per_item=1),
               dict(threads_per_item=1), dict(threads_per_item=2), dict(threads_per_item=2, staging="global"),
               dict(threads_per_item=4, groups_per_block=3, threads_per_block=64),
               dict(groups_per_block=4), dict(groups_per_block=4, staging="smem")]


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("launch", SA_LAUNCHES, ids=[str(x) for x in SA_LAUNCHES])
def test_select_ahead_launch_shapes(P, launch, mode):
    """The select-ahead schedule with several groups per CTA, fewer threads
    than items, and either staging: the fused schedule's chains."""
    net, soi = S.mid_config()[:2]
    a, _, sa = _gpu_run(P, net, soi, 200, 3, mode, [40], schedule="fused")
    b, _, sb = _gpu_run(P, net, soi, 200, 3, mode, [40], schedule="select_ahead", **launch)
    assert np.array_equal(sa[-1], sb[-1])
    assert np.array_equal(a.indicator_numpy(0, 40), b.indicator_numpy(0, 40))


@pytest.mark.parametrize("mode", [0, 1])
def test_select_ahead_chunks_and_calls(P, mode):
    """Select-ahead chunks of 1024 steps: calls of 1, 1023, 1025 and 2100
    steps (chunk edges inside and at the ends of calls) against the oracle."""
    net, soi = next((x[1], x[2]) for x in NETS if x[0] == "k0-mix")
    chunks = [1, 1023, 1025, 2100]
    cs, init, states = _gpu_run(P, net, soi, 45, 99, mode, chunks, schedule="select_ahead")
    ref = oracle.init_states(net, 99, 45)
    t0, inds = 0, []
    for k, got in zip(chunks, states):
        ref, ind = oracle.simulate(net, mode, 99, ref, t0, k, soi)
        inds.append(ind)
        assert np.array_equal(got, ref), t0
        t0 += k
    assert np.array_equal(cs.indicator_numpy(0, t0), np.concatenate(inds, axis=1))


def test_select_ahead_refuses_tiles(P):
    net, soi = S.mid_config()[:2]
    with pytest.raises(P.PbnError) as e:
        _gpu_run(P, net, soi, 64, 3, 0, [4], schedule="select_ahead", staging="tiles")
    assert e.value.status == P.PBN_ERR_UNSUPPORTED


def test_gelman_rubin_parity(P):
    net, soi = S.mid_config()[:2]
    omega, T = 96, 600
    cs, _, _ = _gpu_run(P, net, soi, omega, 21, 0, [T])
    ind = cs.indicator_numpy(0, T)
    for start, psi in [(100, 256), (300, 300), (0, 37)]:
        g = P.pbn_gelman_rubin(cs, start, psi)
        c = ind[:, start:start + psi].astype(np.int64).sum(axis=1)
        assert g["S1"] == int(c.sum()) and g["S2"] == int((c * c).sum())
        r = oracle.gelman_rubin(ind, start, psi)
        if math.isinf(r):
            assert math.isinf(g["rhat"])
        else:
            assert g["rhat"] == pytest.approx(r, rel=1e-12)


def test_two_state_parity(P):
    net, soi = S.mid_config()[:2]
    omega, T = 70, 900
    cs, _, _ = _gpu_run(P, net, S.StateOfInterest([0], [1]), omega, 23, 0, [T])
    ind = cs.indicator_numpy(0, T)
    for start, length in [(10, 800), (0, 900), (555, 33), (5, 1)]:
        t = P.pbn_two_state(cs, start, length, 1e-10, 0.005, 0.95)
        n4 = oracle.transition_counts(ind, start, length)
        assert [t["n00"], t["n01"], t["n10"], t["n11"]] == list(n4)
        assert t["ones"] == int(ind[:, start:start + length].sum())
        if n4[1] == 0 or n4[2] == 0:
            assert t["status"] == 6
            continue
        a = n4[1] / (n4[0] + n4[1]); b = n4[2] / (n4[2] + n4[3])
        assert t["alpha"] == a and t["beta"] == b
        rc, M, N = oracle.two_state_MN(a, b, 1e-10, 0.005, 0.95)
        assert t["N"] == N and t["M"] == M


def test_skart_statistics_parity(P):
    net, soi = S.mid_config()[:2]
    omega, T = 64, 700
    cs, _, _ = _gpu_run(P, net, S.StateOfInterest([1], [1]), omega, 29, 0, [T])
    ind = cs.indicator_numpy(0, T).astype(np.float64)
    for start, kappa, bpc, spacer in [(20, 3, 40, 0), (0, 10, 7, 1), (100, 1, 600, 3), (33, 64, 1, 0)]:
        g = P.pbn_skart(cs, start, kappa, bpc, spacer, 0.05, 0.20)
        seg = ind[:, start:start + kappa * bpc].reshape(omega, bpc, kappa)
        means = seg.mean(axis=2).reshape(-1)
        ci = oracle.skart_ci(means, omega, bpc, 0.05)
        for k in ("mean", "var", "skew", "phi", "A", "H", "ci_lo", "ci_hi"):
            assert g[k] == pytest.approx(ci[k], rel=1e-10, abs=1e-13), k
        ok, stat = oracle.vonneumann_pass(means, omega, bpc, spacer, 0.20)
        assert bool(g["vn_pass"]) == ok
        assert g["vn_stat"] == pytest.approx(stat, rel=1e-10, abs=1e-13)


def _cmp_two_state(g, o):
    for k in ("psi", "gr_psi", "length", "sample_size", "ones", "gr_rounds", "ts_rounds"):
        assert g[k] == o[k], k
    assert g["n4"] == o["n4"]
    assert g["prob"] == o["prob"]
    assert g["alpha"] == o["alpha"] and g["beta"] == o["beta"]
    assert g["M"] == o["M"] and g["N"] == o["N"]
    assert g["rhat"] == pytest.approx(o["rhat"], rel=1e-12)


@pytest.mark.parametrize("case", ["tiny", "identity", "three-node", "mid-small", "tiny-global"])
def test_estimate_two_state_matches_oracle(P, case):
    if case.startswith("tiny"):
        net, soi, cfg = S.tiny_config()
        kw = dict(omega=8, psi0=1024, rhat=1.1, r=0.01)
    elif case == "identity":
        net, soi, kw = S.identity_node(0.1), S.StateOfInterest([0], [1]), dict(omega=8, psi0=256, rhat=1.1, r=0.01)
    elif case == "three-node":
        net, soi, kw = S.three_node(1 / 16), S.StateOfInterest([0], [1]), dict(omega=32, psi0=512, rhat=1.05, r=0.01)
    else:
        net, soi, _ = S.mid_config()
        kw = dict(omega=64, psi0=512, rhat=1.05, r=0.01)
    mode = 1 if case.endswith("global") else 0
    for seed in (1, 2):
        o = oracle.estimate_two_state(net, soi, seed=seed, mode=mode, **kw)
        assert o["status"] == 0
        g = P.pbn_estimate_two_state(P.pbn_load(net), soi, seed=seed, mode=mode, **kw)
        _cmp_two_state(g, o)


@pytest.mark.parametrize("case", ["identity", "tiny", "mid-relative", "tiny-multibatch", "three-node-multibatch",
                                  "identity-correlated"])
def test_estimate_skart_matches_oracle(P, case):
    """Alg. GR + Alg. 4 end to end, GPU vs oracle: every decision (kappa, the
    batch count, the spacer, the rounds of each loop) and length exactly, the
    FP64 statistics to 1e-10 relative.  The multi-batch cases keep omega small
    (80 or more batches per chain), so the randomness test on within-chain
    spaced batch means and the lag-1 correlation act on real data."""
    if case == "identity":
        net, soi, kw = S.identity_node(0.2), S.StateOfInterest([0], [1]), dict(omega=16, psi0=256, rhat=1.1,
                                                                              H_star=0.05, relative=True)
    elif case == "tiny":
        net, soi, _ = S.tiny_config()
        soi = S.StateOfInterest([3], [1])
        kw = dict(omega=8, psi0=1024, rhat=1.1, H_star=0.01, relative=False)
    elif case == "mid-relative":
        net, soi, _ = S.mid_config()
        kw = dict(omega=1024, psi0=1024, rhat=1.05, H_star=0.05, relative=True)
    elif case == "tiny-multibatch":
        net, soi, _ = S.tiny_config()
        kw = dict(omega=16, psi0=512, rhat=1.1, H_star=0.004, relative=False)
    elif case == "three-node-multibatch":
        net, soi = S.three_node(1 / 16), S.StateOfInterest([0, 1], [1, 0])
        kw = dict(omega=4, psi0=256, rhat=1.1, H_star=0.003, relative=False)
    else:
        # batch means of single values of a sticky chain (lag-1 correlation
        # near 1 - 2p): the randomness test fails, the spacer steps up and the
        # batch size grows by sqrt 2 several times before it passes
        net, soi = S.identity_node(0.02), S.StateOfInterest([0], [1])
        kw = dict(omega=8, psi0=256, rhat=1.1, H_star=0.02, relative=False)
    o = oracle.estimate_skart(net, soi, seed=5, alpha=0.05, **kw)
    assert o["status"] == 0
    if case.endswith("multibatch"):
        assert o["batches"] // kw["omega"] >= 80 and o["rand_rounds"] >= 1
    if case == "identity-correlated":
        assert o["rand_rounds"] > 10 and o["spacer"] > 0 and o["kappa"] > 16
    g = P.pbn_estimate_skart(P.pbn_load(net), soi, seed=5, alpha=0.05, **kw)
    for k in ("psi", "length", "kappa", "batches", "spacer", "sample_size", "gr_rounds", "rand_rounds", "ci_rounds"):
        assert g[k] == o[k], k
    # mean, variance, CI and half-width to 1e-12 relative; skewness and lag-1
    # correlation to 1e-12 absolute (their relative error grows where they are
    # near 0: both sides reach them through cancelling central-moment sums)
    for k in ("mean", "ci_lo", "ci_hi", "H", "var"):
        assert g[k] == pytest.approx(o[k], rel=1e-12, abs=1e-15), k
    for k in ("skew", "phi"):
        assert g[k] == pytest.approx(o[k], rel=0, abs=1e-12), k


def _tiles(net):
    """Number of 1536-record TMA tiles of a network (functions in processing order)."""
    per = np.diff(net.fn_offset)
    return int(np.ceil(per.sum() / 1536))


@pytest.mark.parametrize("staging", ["smem", "tiles", "global"])
@pytest.mark.parametrize("name,n,fr", [("scalefree-300", 300, (1, 4)), ("multi-tile-1200", 1200, (1, 4)),
                                       ("multi-tile-4096", 4096, (1, 2))])
def test_staging_modes_bit_exact(P, staging, name, n, fr):
    """Whole tables in shared memory, TMA tiles streamed per step, or global
    reads: the same trajectories (checked against the oracle)."""
    net = S.random_pbn(n, n, fr, (2, 5), "biased", "powerlaw", 0.002)
    if name.startswith("multi"):
        assert _tiles(net) >= 2
    soi = S.StateOfInterest([1, 2, 3], [1, 0, 1])
    omega, steps = 40, 5
    try:
        cs, _, states = _gpu_run(P, net, soi, omega, 13, 0, [steps], staging=staging)
    except P.PbnError as e:
        # whole tables that do not fit shared memory are refused, not silently staged otherwise
        assert staging == "smem" and e.status == P.PBN_ERR_UNSUPPORTED
        return
    ref, ind = oracle.simulate(net, 0, 13, oracle.init_states(net, 13, omega), 0, steps, soi)
    assert np.array_equal(states[-1], ref)
    assert np.array_equal(cs.indicator_numpy(0, steps), ind)
    assert P.pbn_take_device_status() == 0


def test_tiles_global_mode_many_steps(P):
    """TMA tiles over many steps (the double-buffered tile sequence wraps
    across steps) and the global perturbation reading."""
    net = S.random_pbn(77, 1500, (1, 4), (2, 5), "biased", "powerlaw", 0.01)
    soi = S.StateOfInterest([0], [1])
    a, _, sa = _gpu_run(P, net, soi, 100, 5, 1, [37, 12], staging="tiles")
    b, _, sb = _gpu_run(P, net, soi, 100, 5, 1, [37, 12], staging="global")
    assert np.array_equal(sa[-1], sb[-1])
    assert np.array_equal(a.indicator_numpy(0, 49), b.indicator_numpy(0, 49))
