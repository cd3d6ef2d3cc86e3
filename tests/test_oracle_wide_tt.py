"""Pins of the oracle for predictor functions with more than five parents,
whose truth tables span several 32-bit words (bit j of a table is bit j % 32 of
word j / 32): closed forms (parity, majority) under deterministic dynamics,
and the one-step transition law against the exact matrix."""
import numpy as np
import pytest

import pbn_synth as S
from oracle import exact
from test_oracle_sim import _chi2_pvalue, _one_step_counts


def _parity_majority_net():
    """n = 10, p = 0, one function per node: v0 = parity(v1..v9) (9 parents,
    512-bit table), v1 = majority(v2..v9) (8 parents, 256-bit table), and
    v_i = v_{(i+1) % 10} for i >= 2."""
    par9 = list(range(1, 10))
    parity = [bin(j).count("1") & 1 for j in range(1 << 9)]
    par8 = list(range(2, 10))
    majority = [int(bin(j).count("1") >= 5) for j in range(1 << 8)]
    fns = [[(par9, parity, 1.0)], [(par8, majority, 1.0)]]
    fns += [[(((i + 1) % 10,), 0b10, 1.0)] for i in range(2, 10)]
    return S.from_lists(10, fns, 0.0, "parity-majority")


def test_tables_are_word_ranges():
    net = _parity_majority_net()
    assert list(np.diff(net.tt_offset)) == [16, 8] + [1] * 8
    # bit 511 of the parity table: 9 ones -> 1, in word 15, bit 31
    assert (int(net.tt_of(0)[15]) >> 31) & 1 == 1


@pytest.mark.parametrize("mode", [0, 1])
def test_deterministic_closed_forms(orc, mode):
    net = _parity_majority_net()
    assert orc.validate(net) == 0
    omega, steps = 64, 25
    st = orc.init_states(net, 3, omega).astype(np.int64)
    for t in range(steps):
        nxt, _ = orc.simulate(net, mode, 3, st.astype(np.uint8), t, 1, record=False)
        want = np.empty_like(st)
        want[:, 0] = st[:, 1:10].sum(axis=1) & 1
        want[:, 1] = (st[:, 2:10].sum(axis=1) >= 5).astype(np.int64)
        for i in range(2, 10):
            want[:, i] = st[:, (i + 1) % 10]
        assert np.array_equal(nxt.astype(np.int64), want), t
        st = nxt.astype(np.int64)


def _wide_random():
    return S.random_pbn(77, 7, (1, 3), (4, 7), "fair", "uniform", 0.05, "wide-n7")


@pytest.mark.parametrize("mode", [0, 1])
def test_one_step_law_with_wide_tables(orc, mode):
    net = _wide_random()
    ks = np.diff(net.par_offset)
    assert ks.max() >= 6 and orc.validate(net) == 0
    P = exact.transition_matrix(net, mode)
    pmin = 1.0
    for s in range(0, 1 << net.n, 9):
        c = _one_step_counts(orc, net, mode, s, reps=10)
        pmin = min(pmin, _chi2_pvalue(c, P[s]))
    assert pmin > 1e-6 / 15, pmin


def test_validation_rejects_bad_tables(orc):
    net = _wide_random()
    bad = S.PBN(n=net.n, fn_offset=net.fn_offset, par_offset=net.par_offset, parents=net.parents,
                truth_table=net.truth_table, select_prob=net.select_prob, p=net.p,
                tt_offset=np.arange(net.n_functions + 1, dtype=np.int32),
                tt_words=net.truth_table.copy())
    assert orc.validate(bad) != 0
