"""Pins of the oracle on the dense class of the paper's sweep (Sec. 5.1:
density D(G) 150-300, here 12-16 predictor functions of 10-15 parents per
node, truth tables of 32-1024 words): the recipe's density, the one-step
law from given states (every node's next value and the joint law of four
nodes, against probabilities computed here from the truth tables and the
quantised selection probabilities), and the whole method within r of the
exact answer on a 14-node dense network."""
import numpy as np
import pytest
import scipy.stats as st

import pbn_synth as S
from oracle import exact


def _dense(n=16, seed=1616):
    return S.random_pbn(seed, n, (12, 16), (10, min(15, n)), "biased", "uniform", 0.05, f"dense-n{n}")


def test_recipe_density_in_the_dense_class():
    for n in (80, 200):
        net, soi = S.sweep_config(n, "dense")
        assert 150 <= net.density() <= 300, (n, net.density())
        ks = np.diff(net.par_offset)
        assert ks.min() >= 10 and ks.max() == 15
        assert np.diff(net.fn_offset).max() == 16 and np.diff(net.fn_offset).min() == 12
    net = _dense()
    assert 150 <= net.density() <= 300


def _next_one_probabilities(net, s, mode):
    """P(node i is 1 after one step | state s), from the quantised category
    probabilities and the truth tables (Sec. 2.2), for both readings."""
    n = net.n
    p_e, probs = exact.category_probabilities(net)
    vals = exact.function_values(net, np.array([s], dtype=np.int64))[0]
    qf = np.zeros(n)
    for i in range(n):
        for f in net.functions_of(i):
            qf[i] += probs[f] * vals[f]
    bits = np.array([(s >> i) & 1 for i in range(n)], dtype=np.float64)
    if mode == 0:
        return p_e * (1.0 - bits) + qf, None
    qc = qf / (1.0 - p_e)
    none = (1.0 - p_e) ** n
    # GLOBAL: no perturbation with probability (1-p)^n (functions, conditional
    # probabilities qc); else s XOR gamma over the nonzero patterns gamma
    q = none * qc + p_e * (1.0 - bits) + ((1.0 - p_e) - none) * bits
    return q, (qc, none, p_e, bits)


def _joint_probabilities(q, extra, nodes, mode):
    """Law of the next values of `nodes` (cell index sum_m a_m 2^m)."""
    k = len(nodes)
    cells = np.arange(1 << k)
    a = ((cells[:, None] >> np.arange(k)[None, :]) & 1).astype(np.float64)
    if mode == 0:
        qa = q[nodes]
        return np.prod(a * qa + (1 - a) * (1 - qa), axis=1)
    qc, none, p_e, bits = extra
    qa, sa = qc[nodes], bits[nodes]
    fn_part = none * np.prod(a * qa + (1 - a) * (1 - qa), axis=1)
    x = np.abs(a - sa)            # gamma restricted to the nodes
    g = np.prod(x * p_e + (1 - x) * (1 - p_e), axis=1)
    g[np.all(x == 0, axis=1)] -= none  # gamma = 0 is the no-perturbation case
    return fn_part + g


@pytest.mark.parametrize("mode", [0, 1])
def test_one_step_law_of_a_dense_network(orc, mode):
    net = _dense()
    assert orc.validate(net) == 0
    omega = 1 << 15
    rng = np.random.default_rng(mode)
    nodes = [0, 5, 9, 15]
    zmax, pmin = 0.0, 1.0
    for s in [0, (1 << 16) - 1] + [int(x) for x in rng.integers(0, 1 << 16, size=4)]:
        bits = np.array([(s >> i) & 1 for i in range(net.n)], dtype=np.uint8)
        nxt, _ = orc.simulate(net, mode, 5 + s, np.tile(bits, (omega, 1)), t0=77, steps=1, record=False)
        q, extra = _next_one_probabilities(net, s, mode)
        freq = nxt.mean(axis=0)
        sd = np.sqrt(np.maximum(q * (1 - q), 1e-12) / omega)
        zmax = max(zmax, float(np.max(np.abs(freq - q) / sd)))
        # nodes whose next value is certain never take the other one
        assert np.all(nxt[:, q == 0.0] == 0) and np.all(nxt[:, q == 1.0] == 1)
        cell = (nxt[:, nodes].astype(np.int64) << np.arange(len(nodes))).sum(axis=1)
        counts = np.bincount(cell, minlength=1 << len(nodes))
        probs = _joint_probabilities(q, extra, nodes, mode)
        keep = probs * omega >= 5
        o = np.append(counts[keep], counts[~keep].sum())
        e = np.append(probs[keep] * omega, probs[~keep].sum() * omega)
        if e[-1] < 5:
            o, e = o[:-1], e[:-1]
            e *= o.sum() / e.sum()
        pmin = min(pmin, st.chisquare(o, e).pvalue)
    assert zmax < 5.5, zmax
    assert pmin > 1e-6, pmin


def test_whole_method_within_r_on_a_dense_network(orc):
    """Alg. GR + Alg. 3 on a 14-node dense network: within r of the exact
    answer (FP64 power iteration with the implicit step) at frequency >= s."""
    net = _dense(14, 1414)
    soi = S.StateOfInterest([0, 3], [1, 0])
    exact_p, _ = exact.steady_state_probability_any(net, soi, 0)
    hits = 0
    for sd in range(20):
        o = orc.estimate_two_state(net, soi, omega=64, seed=sd, psi0=256, rhat=1.05, r=0.01, s=0.95, eps=1e-10)
        assert o["status"] == 0, o
        hits += abs(o["prob"] - exact_p) < 0.01
    assert hits / 20 >= 0.95
