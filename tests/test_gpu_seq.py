"""The sequential control runs on the GPU (Sec. 3.1 Alg. 1, Sec. 3.2 Alg. 2):
chain 0 of the seed's family, decision by decision equal to the oracle's
sequential drivers."""
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


def _case(name):
    if name.startswith("tiny"):
        net, soi, _ = S.tiny_config()
        return net, soi, dict(m0=0, n0=1024, r=0.01)
    if name == "identity":
        return S.identity_node(0.1), S.StateOfInterest([0], [1]), dict(m0=0, n0=512, r=0.01)
    if name == "three-node":
        return S.three_node(1 / 16), S.StateOfInterest([0], [1]), dict(m0=100, n0=256, r=0.01)
    net, soi, _ = S.mid_config()
    return net, soi, dict(m0=0, n0=4096, r=0.02)


@pytest.mark.parametrize("name", ["tiny", "tiny-global", "identity", "three-node", "mid"])
def test_alg1_matches_oracle(P, name):
    net, soi, kw = _case(name)
    mode = 1 if name.endswith("global") else 0
    N = P.pbn_load(net)
    for seed in (1, 2):
        o = oracle.estimate_two_state_seq(net, soi, seed=seed, mode=mode, **kw)
        assert o["status"] == 0
        g = P.pbn_estimate_two_state_seq(N, soi, seed=seed, mode=mode, **kw)
        for k in ("prob", "alpha", "beta", "M", "N", "length", "ones", "n4", "ab_window", "rounds"):
            assert g[k] == o[k], (name, k, g[k], o[k])


@pytest.mark.parametrize("name", ["identity", "tiny", "tiny-global"])
def test_alg2_matches_oracle(P, name):
    if name == "identity":
        net, soi, kw = S.identity_node(0.1), S.StateOfInterest([0], [1]), dict(H_star=0.02, relative=False)
    else:
        net, soi, _ = S.tiny_config()
        kw = dict(H_star=0.1, relative=True)
    mode = 1 if name.endswith("global") else 0
    N = P.pbn_load(net)
    for seed in (3, 4):
        o = oracle.estimate_skart_seq(net, soi, seed=seed, mode=mode, alpha=0.05, **kw)
        assert o["status"] == 0
        g = P.pbn_estimate_skart_seq(N, soi, seed=seed, mode=mode, alpha=0.05, **kw)
        for k in ("psi", "length", "kappa", "batches", "spacer", "sample_size", "rand_rounds", "ci_rounds"):
            assert g[k] == o[k], (name, k)
        for k in ("mean", "ci_lo", "ci_hi", "H", "var", "skew", "phi"):
            assert g[k] == pytest.approx(o[k], rel=1e-10, abs=1e-13), (name, k)
