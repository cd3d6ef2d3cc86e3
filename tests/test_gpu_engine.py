"""The batched / serving engine: every query's result is the same alone
(pbn_estimate_two_state / pbn_estimate_skart) and in any mix, whether the
epochs run as a CUDA graph or as direct launches, whatever the tuning, when
queries arrive while others run, and under a device-memory budget that
makes queries wait."""
import numpy as np
import pytest

import pbn_synth as S

pytestmark = pytest.mark.gpu

TS_KEYS = ("prob", "alpha", "beta", "psi", "gr_psi", "length", "sample_size", "M", "N", "ones", "n4",
           "gr_rounds", "ts_rounds", "rhat")
SK_KEYS = ("mean", "ci_lo", "ci_hi", "H", "var", "skew", "phi", "psi", "length", "kappa", "batches", "spacer",
           "sample_size", "gr_rounds", "rand_rounds", "ci_rounds", "rhat")


@pytest.fixture(scope="module")
def P():
    from paper_1508_07828_gb300 import _build
    _build.build()
    import paper_1508_07828_gb300 as P
    return P


def _queries():
    """(kind, net, soi, kwargs) of a mix of uneven networks and chain counts."""
    mid, mid_soi, _ = S.mid_config()
    tiny, tiny_soi, _ = S.tiny_config()
    q = []
    q.append(("ts", mid, mid_soi, dict(omega=1024, seed=1, psi0=512, rhat=1.05, r=0.005)))
    q.append(("ts", mid, mid_soi, dict(omega=300, seed=2, psi0=256, rhat=1.05, r=0.01)))
    q.append(("ts", tiny, tiny_soi, dict(omega=8, seed=3, psi0=1024, rhat=1.1, r=0.01)))
    q.append(("ts", tiny, tiny_soi, dict(omega=40, seed=4, psi0=512, rhat=1.1, r=0.01, mode=1)))
    q.append(("ts", S.identity_node(0.1), S.StateOfInterest([0], [1]), dict(omega=8, seed=5, psi0=256, rhat=1.1, r=0.01)))
    q.append(("ts", S.three_node(1 / 16), S.StateOfInterest([0], [1]), dict(omega=33, seed=6, psi0=512, rhat=1.05, r=0.01)))
    big = S.random_pbn(11, 700, (1, 4), (2, 5), "biased", "powerlaw", 0.001)
    q.append(("ts", big, S.StateOfInterest([3, 7], [1, 0]), dict(omega=2048, seed=7, psi0=256, rhat=1.05, r=0.01)))
    q.append(("sk", S.identity_node(0.2), S.StateOfInterest([0], [1]), dict(omega=16, seed=8, psi0=256, rhat=1.1,
                                                                         H_star=0.05, relative=True)))
    q.append(("sk", tiny, S.StateOfInterest([3], [1]), dict(omega=8, seed=9, psi0=1024, rhat=1.1, H_star=0.01,
                                                             relative=False)))
    return q


QUERIES = _queries()


@pytest.fixture(scope="module")
def alone(P):
    """Each query run alone through the single-query drivers."""
    out = []
    for kind, net, soi, kw in QUERIES:
        N = P.pbn_load(net)
        if kind == "ts":
            out.append(P.pbn_estimate_two_state(N, soi, **kw))
        else:
            out.append(P.pbn_estimate_skart(N, soi, alpha=0.05, **kw))
    return out


def _submit(P, eng, idx, nets):
    kind, net, soi, kw = QUERIES[idx]
    N = nets.setdefault(idx, P.pbn_load(net))
    if kind == "ts":
        return eng.submit_two_state(N, soi, tag=idx, **kw)
    return eng.submit_skart(N, soi, alpha=0.05, tag=idx, **kw)


def _check(results, alone):
    assert len(results) == len(alone)
    for r in results:
        assert r["status"] == 0, r
        ref = alone[r["tag"]]
        keys = TS_KEYS if QUERIES[r["tag"]][0] == "ts" else SK_KEYS
        for k in keys:
            assert r["report"][k] == ref[k], (r["tag"], k, r["report"][k], ref[k])


@pytest.mark.parametrize("use_graph", [True, False])
def test_mix_matches_alone(P, alone, use_graph):
    eng = P.Engine(use_graph=use_graph)
    nets = {}
    for i in range(len(QUERIES)):
        _submit(P, eng, i, nets)
    _check(eng.run(), alone)
    eng.close()


@pytest.mark.parametrize("cfg", [dict(steps_per_epoch=64, threads_per_block=256, items_per_thread=1),
                                 dict(steps_per_epoch=5000, threads_per_block=512, items_per_thread=8),
                                 dict(steps_per_epoch=333, max_active=3),
                                 dict(epoch_target_ms=0.3)])
def test_tuning_does_not_change_results(P, alone, cfg):
    eng = P.Engine(**cfg)
    nets = {}
    for i in range(len(QUERIES)):
        _submit(P, eng, i, nets)
    _check(eng.run(), alone)


def test_continuous_admission(P, alone):
    """Queries submitted while others are on the GPU are admitted as slots
    free up; their results do not change."""
    eng = P.Engine(max_active=4, steps_per_epoch=256)
    nets = {}
    order = list(range(len(QUERIES)))
    results = []
    _submit(P, eng, order.pop(0), nets)
    saw_overlap = False
    for _ in range(100000):
        st = eng.step()
        results += eng.poll()
        if order and st["epoch"] % 2 == 0:
            _submit(P, eng, order.pop(0), nets)
        saw_overlap |= st["active"] >= 2
        if not order and st["active"] == 0 and st["pending"] == 0:
            break
    assert saw_overlap
    _check(results, alone)


def test_memory_budget_makes_queries_wait(P, alone):
    eng = P.Engine(hbm_budget_bytes=256 << 10, steps_per_epoch=512)
    nets = {}
    for i in range(len(QUERIES)):
        _submit(P, eng, i, nets)
    max_active, results = 0, []
    for _ in range(100000):
        st = eng.step()
        results += eng.poll()
        max_active = max(max_active, st["active"])
        assert st["hbm_in_use"] >= 0
        if st["active"] == 0 and st["pending"] == 0:
            break
    assert max_active < len(QUERIES)
    _check(results, alone)


def test_failed_query_reports_status_and_others_finish(P, alone):
    eng = P.Engine()
    nets = {}
    mid, mid_soi, _ = S.mid_config()
    N = P.pbn_load(mid)
    # R-hat >= sqrt(1 - 1/psi) always (B >= 0), so a threshold of 0.5 is never met
    bad = eng.submit_two_state(N, mid_soi, omega=64, seed=1, psi0=64, rhat=0.5, r=0.005, max_length=512,
                               tag=999)
    for i in range(len(QUERIES)):
        _submit(P, eng, i, nets)
    res = eng.run()
    badr = [r for r in res if r["tag"] == 999]
    assert badr and badr[0]["status"] == P.PBN_ERR_NOT_CONVERGED
    _check([r for r in res if r["tag"] != 999], alone)


# ------------------------------------------------------- against the oracle

import oracle  # noqa: E402


def _oracle_of(kind, net, soi, kw):
    kw = dict(kw)
    if kind == "ts":
        return oracle.estimate_two_state(net, soi, **kw)
    return oracle.estimate_skart(net, soi, alpha=0.05, **kw)


def _cmp_oracle(kind, g, o, what):
    """Engine report vs oracle run of the same query: integer decisions and
    counts exactly, FP64 statistics as the single-query parity tests do."""
    assert o["status"] == 0, (what, o)
    if kind == "ts":
        for k in ("psi", "gr_psi", "length", "sample_size", "ones", "gr_rounds", "ts_rounds", "M", "N"):
            assert g[k] == o[k], (what, k, g[k], o[k])
        assert list(g["n4"]) == list(o["n4"]), what
        assert g["prob"] == o["prob"] and g["alpha"] == o["alpha"] and g["beta"] == o["beta"], what
        assert g["rhat"] == pytest.approx(o["rhat"], rel=1e-12), what
    else:
        for k in ("psi", "length", "kappa", "batches", "spacer", "sample_size", "gr_rounds", "rand_rounds",
                  "ci_rounds"):
            assert g[k] == o[k], (what, k, g[k], o[k])
        for k in ("mean", "ci_lo", "ci_hi", "H", "var"):
            assert g[k] == pytest.approx(o[k], rel=1e-12, abs=1e-15), (what, k)
        for k in ("skew", "phi"):
            assert g[k] == pytest.approx(o[k], rel=0, abs=1e-12), (what, k)


def test_mix_matches_oracle(P):
    """Every query of the mix whose network the oracle simulates in seconds,
    compared field by field with the oracle's own Alg. GR + Alg. 3 / Alg. 4
    (not with the single-query GPU driver), after running in the mix."""
    eng = P.Engine(use_graph=True)
    nets = {}
    for i in range(len(QUERIES)):
        _submit(P, eng, i, nets)
    res = {r["tag"]: r for r in eng.run()}
    checked = 0
    for i, (kind, net, soi, kw) in enumerate(QUERIES):
        if net.n * kw["omega"] > 200_000:
            continue
        assert res[i]["status"] == 0
        _cmp_oracle(kind, res[i]["report"], _oracle_of(kind, net, soi, kw), (i, net.name))
        checked += 1
    assert checked >= 8


def test_cancel_pending_and_active(P, alone):
    """A withdrawn query reports PBN_ERR_CANCELLED and frees its slot; the
    other queries' results do not change."""
    eng = P.Engine(max_active=3, steps_per_epoch=256)
    nets = {}
    ids = [_submit(P, eng, i, nets) for i in range(len(QUERIES))]
    eng.cancel(ids[-1])                       # still waiting (3 slots)
    st = eng.step()
    assert st["active"] >= 1
    eng.cancel(ids[0])                        # admitted in the first epoch
    with pytest.raises(P.PbnError) as e:
        eng.cancel(ids[0])                    # already cancelled
    assert e.value.status == P.PBN_ERR_INVALID
    with pytest.raises(P.PbnError):
        eng.cancel(10_000)                    # unknown id
    res = eng.poll() + eng.run()
    cancelled = [r for r in res if r["status"] == P.PBN_ERR_CANCELLED]
    assert sorted(r["tag"] for r in cancelled) == [0, len(QUERIES) - 1]
    for r in res:
        if r["status"] == P.PBN_ERR_CANCELLED:
            continue
        assert r["status"] == 0
        ref = alone[r["tag"]]
        keys = TS_KEYS if QUERIES[r["tag"]][0] == "ts" else SK_KEYS
        for k in keys:
            assert r["report"][k] == ref[k], (r["tag"], k)
    assert len(res) == len(QUERIES)
    with pytest.raises(P.PbnError):
        eng.cancel(ids[1])                    # finished


# ------------------------------------------- the batched workload (64 networks)

def _replay_window(P, net, soi, omega, seed, rep, rng, mode=0):
    """Replays the query's chains to its final length with pbn_run_chains and
    recounts the window [psi, length) on the host; sampled chains are
    replayed by the oracle, bit for bit."""
    N = P.pbn_load(net)
    L, psi = rep["length"], rep["psi"]
    cs = P.ChainSet(N, omega, bits_cap=L)
    P.pbn_init_chains(cs, seed, mode)
    P.pbn_run_chains(cs, L, seed, mode, soi)
    x = cs.indicator_numpy(psi, L - psi)
    assert int(x.sum()) == rep["ones"]
    a, b = x[:, :-1], x[:, 1:]
    n4 = [int(((a == i) & (b == j)).sum()) for i in (0, 1) for j in (0, 1)]
    assert n4 == list(rep["n4"])
    states = cs.states_numpy()
    for c in sorted({0, omega - 1, int(rng.integers(omega))}):
        st0 = oracle.init_states(net, seed, 1, chain0=c)
        ref, ind = oracle.simulate(net, mode, seed, st0, 0, L, soi, chain0=c)
        assert np.array_equal(states[c], ref[0]), c
        assert np.array_equal(x[c], ind[0][psi:]), c


@pytest.mark.parametrize("mode", [0, 1])
def test_batch_workload_in_mix_equals_alone_and_replays(mode):
    """The batched workload's 64 networks (n log-uniform in [50, 3000],
    256-4096 chains, p in {0.001, 0.01}, two-state r = 0.005) in one engine,
    under both perturbation readings: every query equals its single-query
    run; for the networks of n >= 2000 the chains replayed to the query's
    final length give its counts, and sampled chains match the oracle."""
    from paper_1508_07828_gb300 import _build
    _build.build()
    import paper_1508_07828_gb300 as P
    cfgs = S.batch_configs()
    assert len(cfgs) == 64 and max(net.n for net, _, _ in cfgs) >= 2000
    nets = [P.pbn_load(net) for net, _, _ in cfgs]
    kw = lambda c, k: dict(omega=c["omega"], seed=1000 + k, psi0=1024, rhat=c["rhat"], eps=c["eps"], r=c["r"],
                           s=c["s"], max_length=1 << 20, mode=mode)
    eng = P.Engine(use_graph=True)
    for k, ((net, soi, c), N) in enumerate(zip(cfgs, nets)):
        eng.submit_two_state(N, soi, tag=k, **kw(c, k))
    res = {r["tag"]: r for r in eng.run()}
    assert len(res) == 64
    rng = np.random.default_rng(5)
    replayed = 0
    for k, ((net, soi, c), N) in enumerate(zip(cfgs, nets)):
        ref = P.pbn_estimate_two_state(N, soi, **kw(c, k))
        got = res[k]
        assert got["status"] == 0
        for key in TS_KEYS:
            assert got["report"][key] == ref[key], (k, key)
        if net.n >= 2000:
            _replay_window(P, net, soi, c["omega"], 1000 + k, got["report"], rng, mode=mode)
            replayed += 1
    assert replayed >= 2


# ----------------------------------------------- the serving pool (200 networks)

def _serving_queries(count=40, seed=1508078290):
    pool = S.serving_pool()
    rng = np.random.default_rng(seed)
    out = []
    for k in range(count):
        i = int(rng.integers(len(pool)))
        soi = S.random_soi(rng, pool[i].n)
        r = float(rng.choice([0.01, 0.005, 0.001]))
        kind = "ts" if k % 2 == 0 else "sk"
        out.append((kind, i, soi, r, 20_000 + k))
    return pool, out


def test_serving_pool_continuous_mix():
    """Queries over the 200-network serving pool (n log-uniform in [20, 3000],
    1-10-node states of interest, r in {0.01, 0.005, 0.001}, two-state and
    Skart at absolute precision r), submitted a few per epoch while others
    run: each result equals the query alone; the queries on small networks
    also equal the oracle's."""
    from paper_1508_07828_gb300 import _build
    _build.build()
    import paper_1508_07828_gb300 as P
    pool, qs = _serving_queries()
    loaded = {}

    def net_of(i):
        if i not in loaded:
            loaded[i] = P.pbn_load(pool[i])
        return loaded[i]

    def kwargs(kind, r, seed):
        base = dict(omega=256, seed=seed, psi0=512, rhat=1.05, max_length=1 << 15)
        if kind == "ts":
            return dict(base, r=r)
        return dict(base, H_star=r, relative=False)

    eng = P.Engine(use_graph=True, epoch_target_ms=2.0)
    results, nxt = [], 0
    for _ in range(100_000):
        for _ in range(3):
            if nxt < len(qs):
                kind, i, soi, r, seed = qs[nxt]
                if kind == "ts":
                    eng.submit_two_state(net_of(i), soi, tag=nxt, **kwargs(kind, r, seed))
                else:
                    eng.submit_skart(net_of(i), soi, alpha=0.05, tag=nxt, **kwargs(kind, r, seed))
                nxt += 1
        st = eng.step()
        results += eng.poll()
        if nxt == len(qs) and st["active"] == 0 and st["pending"] == 0:
            break
    assert len(results) == len(qs)
    oracle_checked = 0
    for res in results:
        kind, i, soi, r, seed = qs[res["tag"]]
        kw = kwargs(kind, r, seed)
        try:
            ref = (P.pbn_estimate_two_state(net_of(i), soi, **kw) if kind == "ts"
                   else P.pbn_estimate_skart(net_of(i), soi, alpha=0.05, **kw))
            ref_status = 0
        except P.PbnError as e:
            ref, ref_status = None, e.status
        assert res["status"] == ref_status, (res["tag"], res["status"], ref_status)
        if ref is None:
            continue
        for key in (TS_KEYS if kind == "ts" else SK_KEYS):
            assert res["report"][key] == ref[key], (res["tag"], key)
        if pool[i].n <= 60 and res["report"]["length"] * pool[i].n <= 3_000_000:
            _cmp_oracle(kind, res["report"], _oracle_of(kind, pool[i], soi, kw), res["tag"])
            oracle_checked += 1
    assert oracle_checked >= 2
