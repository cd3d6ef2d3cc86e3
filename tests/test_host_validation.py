"""Malformed inputs are refused on the host, before any device work (so these
run without a GPU): pbn_load's validation of the network (structure,
probabilities, limits) and the drivers' validation of a query.  Each returns
its status code with a message from pbn_last_error."""
import math
import types

import numpy as np
import pytest

import pbn_synth as S


@pytest.fixture(scope="module")
def P():
    from paper_1508_07828_gb300 import _build
    _build.build()
    import paper_1508_07828_gb300 as P
    return P


def _net(**over):
    """A valid 3-node network (the hand-built one), with fields replaced."""
    base = S.three_node(1 / 16)
    d = dict(n=base.n, fn_offset=base.fn_offset.copy(), par_offset=base.par_offset.copy(),
             parents=base.parents.copy(), truth_table=base.truth_table.copy(),
             select_prob=base.select_prob.copy(), p=base.p, tt_offset=None, tt_words=None)
    d.update(over)
    return types.SimpleNamespace(**d)


def _status(P, net):
    with pytest.raises(P.PbnError) as e:
        P.pbn_load(net)
    assert str(e.value).split(":", 1)[1].strip()  # a message says why
    return e.value.status


def test_structure_is_checked(P):
    assert _status(P, _net(n=0, fn_offset=np.zeros(1, np.int32))) == P.PBN_ERR_INVALID
    fo = _net().fn_offset.copy()
    fo[-1] += 1  # does not span the functions
    assert _status(P, _net(fn_offset=fo)) == P.PBN_ERR_INVALID
    par = _net().parents.copy()
    par[0] = 3  # node 3 of a 3-node network
    assert _status(P, _net(parents=par)) == P.PBN_ERR_INVALID
    par[0] = -1
    assert _status(P, _net(parents=par)) == P.PBN_ERR_INVALID
    fo = _net().fn_offset.copy()
    fo[1] = fo[0]  # node 0 without a predictor function
    assert _status(P, _net(fn_offset=fo)) == P.PBN_ERR_INVALID


def test_offsets_are_checked_before_reading_through_them(P):
    """Offsets that stay inside [0, F] at both ends but would lead a later
    node or function past the arrays' ends are refused first (3 nodes,
    4 functions, 6 parents)."""
    assert _status(P, _net(fn_offset=np.array([0, 3, 5, 4], np.int32))) == P.PBN_ERR_INVALID
    assert _status(P, _net(fn_offset=np.array([0, 2, 1, 4], np.int32))) == P.PBN_ERR_INVALID
    # function 0 claims 7 parents of the 6, function 1 then goes backwards
    assert _status(P, _net(par_offset=np.array([0, 7, 3, 4, 6], np.int32))) == P.PBN_ERR_INVALID
    assert _status(P, _net(par_offset=np.array([1, 2, 3, 4, 6], np.int32))) == P.PBN_ERR_INVALID
    wide = _net()
    wide.tt_offset = np.array([0, 2, 1, 3, 4], np.int32)
    wide.tt_words = np.zeros(4, np.uint32)
    assert _status(P, wide) == P.PBN_ERR_INVALID


def test_array_lengths_are_checked_by_the_binding(P):
    """The function count passed to pbn_load is the arrays' own, and arrays
    shorter or longer than the counts imply are refused before the call."""
    base = _net()
    assert _status(P, _net(select_prob=base.select_prob[:3])) == P.PBN_ERR_INVALID
    assert _status(P, _net(truth_table=base.truth_table[:3])) == P.PBN_ERR_INVALID
    assert _status(P, _net(par_offset=base.par_offset[:4])) == P.PBN_ERR_INVALID
    assert _status(P, _net(fn_offset=np.array([0, 1, 3, 4, 4], np.int32))) == P.PBN_ERR_INVALID
    assert _status(P, _net(parents=base.parents[:5])) == P.PBN_ERR_INVALID
    wide = _net()
    wide.tt_offset = np.arange(5, dtype=np.int32)
    wide.tt_words = np.zeros(3, np.uint32)
    assert _status(P, wide) == P.PBN_ERR_INVALID


def test_state_of_interest_lengths_are_checked_by_the_binding(P):
    """pbn_soi carries one size for its two arrays: nodes and values of
    different lengths are refused before any call."""
    for nodes, values in (([0, 1], [1]), ([0], [1, 0])):
        with pytest.raises(P.PbnError) as e:
            P.SoiArg(types.SimpleNamespace(nodes=np.array(nodes), values=np.array(values)))
        assert e.value.status == P.PBN_ERR_INVALID


def test_statistics_windows_and_parameters_are_checked(P):
    """The statistics entry points check the window against the recorded
    positions and their parameters before any device work (here a chain set
    whose device pointers are never dereferenced)."""
    import ctypes
    L = P.lib()
    ch = P.Chains(64, 16, 16, 1000, 100, 900)  # omega 64; positions 100 .. 899 recorded, capacity 1000
    out = ctypes.c_void_p(16)
    cases = [
        (L.pbn_gelman_rubin, (ctypes.byref(ch), 99, 100, out, None), P.PBN_ERR_INVALID),    # before bits_base
        (L.pbn_gelman_rubin, (ctypes.byref(ch), 800, 101, out, None), P.PBN_ERR_INVALID),   # past the length
        (L.pbn_gelman_rubin, (ctypes.byref(ch), 100, 1, out, None), P.PBN_ERR_INVALID),     # psi < 2
        (L.pbn_two_state, (ctypes.byref(ch), 100, 0, 1e-10, 0.01, 0.95, out, None), P.PBN_ERR_INVALID),
        (L.pbn_two_state, (ctypes.byref(ch), 100, 50, 1e-10, 0.01, 1.0, out, None), P.PBN_ERR_INVALID),
        (L.pbn_skart, (ctypes.byref(ch), 100, 0, 1, 0, 0.05, 0.2, out, None), P.PBN_ERR_INVALID),
        (L.pbn_skart, (ctypes.byref(ch), 100, 10, 81, 0, 0.05, 0.2, out, None), P.PBN_ERR_INVALID),
        (L.pbn_skart, (ctypes.byref(ch), 100, (1 << 30) + 1, 1, 0, 0.05, 0.2, out, None), P.PBN_ERR_UNSUPPORTED),
        (L.pbn_skart, (ctypes.byref(ch), 100, 1 << 30, (1 << 32) + 1, 0, 0.05, 0.2, out, None),
         P.PBN_ERR_UNSUPPORTED),
        (L.pbn_skart_static, (ctypes.byref(ch), 100, 10, 81, 0, 0.05, 0.2, out, None), P.PBN_ERR_INVALID),
        (L.pbn_skart_static, (ctypes.byref(ch), 100, 1, 1 << 13, 0, 0.05, 0.2, out, None), P.PBN_ERR_UNSUPPORTED),
        # kappa above 2^30 is beyond the build's limits, as in pbn_skart
        (L.pbn_skart_static, (ctypes.byref(ch), 100, (1 << 30) + 1, 1, 0, 0.05, 0.2, out, None),
         P.PBN_ERR_UNSUPPORTED),
        # a batch count whose product with omega overflows 64 bits is refused by capacity
        (L.pbn_skart_static, (ctypes.byref(ch), 100, 1, 1 << 62, 0, 0.05, 0.2, out, None), P.PBN_ERR_UNSUPPORTED),
    ]
    for fn, args, want in cases:
        assert fn(*args) == want, (fn.__name__, args[1:4])
        assert L.pbn_last_error().decode()


def _networks_of_every_recipe():
    yield S.three_node(1 / 16)
    yield S.identity_node(0.01)
    yield S.constant_node(0.01)
    yield S.all_identity(12, 0.01)
    yield S.tiny_config()[0]
    yield S.mid_config()[0]
    yield S.large_config()[0]
    yield S.wide_config()[0]
    for n in (80, 100, 200, 500, 1000, 2000):
        for density in ("sparse", "in-between"):
            yield S.sweep_config(n, density)[0]
    for net, _, _ in S.batch_configs():
        yield net
    yield from S.serving_pool()


def test_every_synthetic_recipe_passes_validation(P):
    """Every network the tests and the bench stage passes pbn_load's checks:
    without a GPU the call fails only at the device copy (PBN_ERR_CUDA), with
    one it loads."""
    count = 0
    for net in _networks_of_every_recipe():
        try:
            P.pbn_load(net).close()
        except P.PbnError as e:
            assert e.status == P.PBN_ERR_CUDA, (getattr(net, "name", "?"), str(e))
        count += 1
    assert count > 270


def test_probabilities_are_checked(P):
    for p in (float("nan"), -0.1, 1.0, 1.5):
        assert _status(P, _net(p=p)) == P.PBN_ERR_INVALID, p
    c = _net().select_prob.copy()
    c[1] = math.nan
    assert _status(P, _net(select_prob=c)) == P.PBN_ERR_INVALID
    c = _net().select_prob.copy()
    c[1] += 0.01  # node 1's probabilities no longer sum to 1
    assert _status(P, _net(select_prob=c)) == P.PBN_ERR_INVALID
    c = _net().select_prob.copy()
    c[1], c[2] = 1.25, -0.25  # sums to 1, but not probabilities
    assert _status(P, _net(select_prob=c)) == P.PBN_ERR_INVALID


def test_limits_are_checked(P):
    big = S.random_pbn(1, 4097, (1, 1), (1, 1), "fair", "uniform", 0.01)  # PBN_MAX_NODES + 1
    assert _status(P, big) == P.PBN_ERR_UNSUPPORTED
    many = S.from_lists(1, [[((0,), 0b10, 1 / 17)] * 17], 0.01)  # PBN_MAX_FUNCTIONS_PER_NODE + 1 functions
    assert _status(P, many) == P.PBN_ERR_UNSUPPORTED
    # PBN_MAX_PARENTS + 1 inputs
    wide = S.random_pbn(3, 18, (1, 1), (16, 16), "fair", "uniform", 0.01)
    assert _status(P, wide) == P.PBN_ERR_UNSUPPORTED
    # a 6-input function without a multi-word table
    six = _net(par_offset=np.array([0, 6, 7, 8, 10], np.int32),
               parents=np.array([1, 2, 0, 1, 2, 0, 0, 2, 0, 1], np.int32))
    six.tt_offset = None
    assert _status(P, six) == P.PBN_ERR_INVALID


def test_query_without_network_is_refused(P):
    """A query on no network is refused before anything is launched (the C
    entry point, stream NULL)."""
    import ctypes
    soi = P.SoiArg(S.StateOfInterest([0], [1]))
    out = P.TwoStateReport()
    q = P.TwoStateQuery(8, 64, 1.05, 1e-10, 0.01, 0.95, 1 << 20, 1, 0, soi.struct)
    assert P.lib().pbn_estimate_two_state(None, ctypes.byref(q), ctypes.byref(out), None) == P.PBN_ERR_INVALID
    assert P.lib().pbn_last_error().decode()


@pytest.mark.gpu
@pytest.mark.parametrize("bad", [dict(omega=1), dict(psi0=1), dict(r=0.0), dict(r=math.nan), dict(s=1.0),
                                 dict(eps=0.0), dict(max_length=100), dict(rhat=0.0), dict(mode=7)],
                         ids=lambda d: next(iter(d)))
def test_query_parameters_are_checked(P, bad):
    """Parameters out of range fail the query with PBN_ERR_INVALID."""
    N = P.pbn_load(_net())
    kw = dict(omega=8, seed=1, psi0=64, r=0.01)
    kw.update(bad)
    with pytest.raises(P.PbnError) as e:
        P.pbn_estimate_two_state(N, S.StateOfInterest([0], [1]), **kw)
    assert e.value.status == P.PBN_ERR_INVALID


@pytest.mark.gpu
def test_state_of_interest_is_checked(P):
    N = P.pbn_load(_net())
    for soi in (S.StateOfInterest([3], [1]), S.StateOfInterest([0], [2]), S.StateOfInterest([], [])):
        with pytest.raises(P.PbnError) as e:
            P.pbn_estimate_two_state(N, soi, omega=8, seed=1, psi0=64, r=0.01)
        assert e.value.status == P.PBN_ERR_INVALID
