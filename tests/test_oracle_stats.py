"""Pins of the oracle's statistics: Gelman & Rubin (Sec. 4.1), the two-state
Markov chain formulas (Sec. 3.1, Alg. 1 line 8), the normal and Student-t
quantiles, skewness, transition counts and the Skart pieces (Sec. 3.2)."""
import math

import numpy as np
import pytest
import scipy.stats as st


# ---------------------------------------------------------------- G&R ------

def _rhat_closed_form(x, start, psi):
    """R-hat from the integer sums S1 = sum c_i, S2 = sum c_i^2 of the chains'
    ones counts: an algebraic reduction of Alg. GR for 0/1 values."""
    c = x[:, start:start + psi].astype(np.int64).sum(axis=1)
    w = len(c)
    S1, S2 = int(c.sum()), int((c * c).sum())
    W = (psi * S1 - S2) / (w * psi * (psi - 1))
    B = (w * S2 - S1 * S1) / (w * (w - 1) * psi)
    if W <= 0:
        return math.inf
    return math.sqrt(((1 - 1 / psi) * W + B / psi) / W)


def _rhat_numpy(x, start, psi):
    seg = x[:, start:start + psi].astype(np.float64)
    mu = seg.mean(axis=1)
    s2 = seg.var(axis=1, ddof=1)
    W = s2.mean()
    B = psi * mu.var(ddof=1)
    return math.sqrt(((1 - 1 / psi) * W + B / psi) / W)


@pytest.mark.parametrize("omega,psi,q", [(8, 64, 0.3), (33, 1000, 0.02), (256, 17, 0.5)])
def test_gelman_rubin_matches_closed_form_and_numpy(orc, omega, psi, q):
    rng = np.random.default_rng(omega * psi)
    # chains with different means so B is not ~0
    means = rng.uniform(q / 2, min(1.0, 1.5 * q), size=omega)
    x = (rng.random((omega, 2 * psi + 5)) < means[:, None]).astype(np.uint8)
    r = orc.gelman_rubin(x, psi, psi)
    assert r == pytest.approx(_rhat_closed_form(x, psi, psi), rel=1e-13)
    assert r == pytest.approx(_rhat_numpy(x, psi, psi), rel=1e-12)


def test_gelman_rubin_iid_near_one_and_separated_large(orc):
    rng = np.random.default_rng(1)
    x = (rng.random((64, 20000)) < 0.3).astype(np.uint8)
    assert abs(orc.gelman_rubin(x, 10000, 10000) - 1.0) < 0.01
    y = np.zeros((8, 2000), dtype=np.uint8)
    y[:4] = (rng.random((4, 2000)) < 0.9)
    y[4:] = (rng.random((4, 2000)) < 0.1)
    # B ~ psi var(mu) dominates W: R-hat ~ sqrt(B/(psi W)) ~ 1.7
    assert orc.gelman_rubin(y, 1000, 1000) > 1.5


def test_gelman_rubin_degenerate_within_zero(orc):
    x = np.ones((4, 100), dtype=np.uint8)
    assert math.isinf(orc.gelman_rubin(x, 50, 50))


# ----------------------------------------------------- two-state ----------

def test_norm_ppf_matches_scipy(orc):
    for q in [1e-12, 1e-6, 0.01, 0.2, 0.5, 0.8, 0.975, 0.995, 1 - 1e-9]:
        assert orc.norm_ppf(q) == pytest.approx(st.norm.ppf(q), rel=1e-13, abs=1e-15)
    assert orc.norm_ppf(0.975) == pytest.approx(1.959963984540054, rel=1e-15)


@pytest.mark.parametrize("dof", [1, 2, 5, 29, 127, 1023, 16383, 1e6])
def test_t_ppf_matches_scipy(orc, dof):
    for q in [0.005, 0.025, 0.1, 0.9, 0.975, 0.995]:
        assert orc.t_ppf(q, dof) == pytest.approx(st.t.ppf(q, dof), rel=1e-11)


def test_identity_node_closed_forms(orc):
    """Identity node (v0 := v0) flips only when perturbed: alpha = beta = p.
    At p = 0.01, eps = 1e-10, s = 0.95: M = ceil(1105.43) = 1106 and
    N = ceil(950761.06) = 950762 for r = 0.01; N = 3803045 for r = 0.005."""
    rc, M, N = orc.two_state_MN(0.01, 0.01, 1e-10, 0.01, 0.95)
    assert rc == 0 and M == 1106 and N == 950762
    rc, M, N = orc.two_state_MN(0.01, 0.01, 1e-10, 0.005, 0.95)
    assert N == 3803045
    rc, M, N = orc.two_state_MN(0.1, 0.1, 1e-10, 0.01, 0.95)
    assert (M, N) == (101, 86433)


def test_constant_node_closed_forms(orc):
    """Constant-1 node under the per-node reading: from 0 the node becomes 1
    whether or not it is perturbed (alpha = 1); from 1 it drops to 0 only when
    perturbed (beta = p).  With beta = p = 0.01 and r = 0.01: M = 5, N = 370."""
    rc, M, N = orc.two_state_MN(1.0, 0.01, 1e-10, 0.01, 0.95)
    assert rc == 0 and (M, N) == (5, 370)


def test_two_state_formula_against_independent_evaluation(orc):
    rng = np.random.default_rng(2)
    z = st.norm.ppf(0.975)
    for _ in range(200):
        a, b = rng.uniform(1e-4, 0.9, size=2)
        rc, M, N = orc.two_state_MN(a, b, 1e-10, 0.005, 0.95)
        Mr = math.log(1e-10 * (a + b) / max(a, b)) / math.log(abs(1 - a - b))
        Nr = a * b * (2 - a - b) / (a + b) ** 3 * z * z / 0.005 ** 2
        if abs(Nr - round(Nr)) > 1e-6 * Nr:
            assert N == math.ceil(Nr)
        if abs(Mr - round(Mr)) > 1e-9 * max(1, Mr):
            assert M == max(0, math.ceil(Mr))


def test_two_state_edge_cases(orc):
    assert orc.two_state_MN(0.0, 0.3, 1e-10, 0.01, 0.95)[0] != 0
    assert orc.two_state_MN(0.3, 0.0, 1e-10, 0.01, 0.95)[0] != 0
    rc, M, N = orc.two_state_MN(0.4, 0.6, 1e-10, 0.01, 0.95)  # |1-a-b| = 0
    assert rc == 0 and M == 0
    assert orc.two_state_MN(1.0, 1.0, 1e-10, 0.01, 0.95)[0] == 5


def test_transition_counts_bruteforce(orc):
    rng = np.random.default_rng(3)
    x = (rng.random((7, 300)) < 0.4).astype(np.uint8)
    n4 = orc.transition_counts(x, 13, 200)
    ref = np.zeros(4, dtype=np.int64)
    for c in range(7):
        for j in range(13, 13 + 199):
            ref[2 * x[c, j] + x[c, j + 1]] += 1
    assert list(n4) == list(ref)


# ------------------------------------------------------------ Skart --------

def test_skewness_matches_scipy(orc):
    rng = np.random.default_rng(4)
    for K in (3, 10, 1000):
        v = rng.exponential(size=K)
        assert orc.skewness(v) == pytest.approx(st.skew(v), rel=1e-12)
    assert orc.skewness(np.ones(10)) == 0.0


def test_vonneumann_detects_correlation(orc):
    rng = np.random.default_rng(5)
    # the test has size 0.20 on iid data
    passes = [orc.vonneumann_pass(rng.normal(size=500), 1, 500, 0)[0] for _ in range(400)]
    assert 0.74 <= np.mean(passes) <= 0.86
    ar = np.zeros(2000)
    for j in range(1, 2000):
        ar[j] = 0.5 * ar[j - 1] + rng.normal()
    ok, c = orc.vonneumann_pass(ar, 1, 2000, 0)
    assert not ok and c > 0.3
    # one batch per chain: no within-chain pairs, passes by construction
    assert orc.vonneumann_pass(ar[:64], 64, 1, 0)[0]


def test_vonneumann_single_chain_is_textbook(orc):
    """With one chain the pooled statistic reduces to von Neumann's
    C = 1 - sum (x_{j+1}-x_j)^2 / (2 sum (x - mean)^2)."""
    rng = np.random.default_rng(6)
    x = rng.normal(size=50)
    ok, c = orc.vonneumann_pass(x, 1, 50, 0)
    ref = 1 - np.sum(np.diff(x) ** 2) / (2 * np.sum((x - x.mean()) ** 2))
    assert c == pytest.approx(ref, rel=1e-13)


def test_skart_ci_reduces_to_student_t(orc):
    """Symmetric means (zero skewness) and no within-chain pairs: the CI is
    the plain Student-t interval mean +- t_{1-a/2,K-1} S/sqrt(K)."""
    v = np.array([0.1, 0.2, 0.3, 0.4, 0.5, 0.6, 0.7])
    o = orc.skart_ci(v, 7, 1, 0.05)
    half = st.t.ppf(0.975, 6) * v.std(ddof=1) / np.sqrt(7)
    assert o["skew"] == pytest.approx(0.0, abs=1e-15)
    assert o["H"] == pytest.approx(half, rel=1e-11)
    assert o["ci_lo"] == pytest.approx(v.mean() - half, rel=1e-11)


def test_skart_ci_coverage_iid():
    """Skewness-adjusted t interval covers the mean of iid batch means at
    about the nominal rate."""
    import oracle
    rng = np.random.default_rng(7)
    hits = 0
    for _ in range(400):
        v = rng.binomial(20, 0.1, size=64) / 20.0
        o = oracle.skart_ci(v, 64, 1, 0.1)
        hits += o["ci_lo"] <= 0.1 <= o["ci_hi"]
    assert 0.85 <= hits / 400 <= 0.95


def _two_state_batch_means(rng, a, b, chains, batches, kappa):
    """Batch means of stationary two-state Markov chains (0 -> 1 with
    probability a, 1 -> 0 with probability b), generated directly from the
    transition law, chain-major as the Skart statistics take them."""
    pi1 = a / (a + b)
    x = (rng.random(chains) < pi1).astype(np.int64)
    sums = np.zeros((chains, batches))
    for j in range(batches):
        acc = np.zeros(chains)
        for _ in range(kappa):
            u = rng.random(chains)
            x = np.where(x == 1, (u >= b).astype(np.int64), (u < a).astype(np.int64))
            acc += x
        sums[:, j] = acc
    return sums / kappa


def test_skart_ci_on_a_correlated_chain_with_exact_variance():
    """Batch means of a two-state chain, whose autocovariance is exact:
    gamma_h = pi (1 - pi) rho^h with rho = 1 - a - b, so the variance of a
    mean of kappa consecutive values is gamma_0 / kappa (1 + 2 sum_h
    (1 - h / kappa) rho^h), tending to the asymptotic variance
    pi (1 - pi) (2 - a - b) / (a + b) over kappa.  The CI statistics (batch
    variance, lag-1 factor A, skewness-adjusted t interval, Sec. 3.2) must
    recover that variance and cover pi at about the nominal rate."""
    import oracle
    a, b, kappa, omega, bpc, reps = 0.05, 0.15, 100, 32, 4, 240
    pi1 = a / (a + b)
    rho = 1 - a - b
    h = np.arange(1, kappa)
    var_mean = pi1 * (1 - pi1) / kappa * (1 + 2 * np.sum((1 - h / kappa) * rho ** h))
    asym = pi1 * (1 - pi1) * (2 - a - b) / (a + b)
    # the sum in closed form: kappa var = asym - 2 gamma_0 rho (1 - rho^kappa) / (kappa (1 - rho)^2)
    g0 = pi1 * (1 - pi1)
    assert math.isclose(kappa * var_mean, asym - 2 * g0 * rho * (1 - rho ** kappa) / (kappa * (1 - rho) ** 2),
                        rel_tol=1e-12)
    rng = np.random.default_rng(11)
    means = _two_state_batch_means(rng, a, b, omega * reps, bpc, kappa)
    raw, est, hits = [], [], 0
    for r in range(reps):
        m = means[r * omega:(r + 1) * omega].reshape(-1)
        o = oracle.skart_ci(m, omega, bpc, 0.1)
        raw.append(o["var"])
        est.append(o["A"] * o["var"])
        hits += o["ci_lo"] <= pi1 <= o["ci_hi"]
    # the batch-mean variance against the exact value (standard error of the
    # average over replications about 0.6%; measured 1.003); the lag-1 factor
    # A = (1 + phi) / (1 - phi) only inflates it a little here, since batches
    # of 100 steps are nearly uncorrelated (measured 1.04)
    assert abs(np.mean(raw) / var_mean - 1) < 0.03
    assert 1.0 <= np.mean(est) / var_mean < 1.08
    assert 0.84 <= hits / reps <= 0.96
