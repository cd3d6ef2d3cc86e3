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
                                 dict(steps_per_epoch=333, max_active=3)])
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
