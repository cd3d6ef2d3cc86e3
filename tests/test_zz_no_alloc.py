"""pbn_skart_static: the Skart statistics entry point for callers that cannot
let the library allocate device memory (their program owns all device memory
through its own allocator, or cannot afford the stall of an allocation).  It
must give what pbn_skart gives, call after call, while reusing one fixed
array inside the library.  This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    from paper_1508_07828_gb300 import _build
    _build.build()
    import paper_1508_07828_gb300 as P
    return P


def _chains(P, omega=96, T=900):
    import pbn_synth as S
    net, _, _ = S.mid_config()
    N = P.pbn_load(net)
    cs = P.ChainSet(N, omega, bits_cap=T)
    P.pbn_init_chains(cs, 41)
    P.pbn_run_chains(cs, T, 41, P.PER_NODE, S.StateOfInterest([0, 3], [1, 1]))
    return N, cs


def _same(a, b):
    for k in ("mean", "var", "skew", "phi", "A", "H", "ci_lo", "ci_hi", "vn_stat"):
        assert a[k] == pytest.approx(b[k], rel=1e-10, abs=1e-13), k
    assert a["vn_pass"] == b["vn_pass"] and a["batches"] == b["batches"]


def test_static_matches_allocating_entry_point_twice_in_a_row(P):
    N, cs = _chains(P)
    # consecutive calls with different batch layouts: no call may see what an
    # earlier one left in the shared array.  Small after large and the same
    # batch count with another kappa leave stale sums exactly where a read
    # past the call's own batches would find them.
    layouts = [(100, 8, 80, 1), (50, 3, 250, 0), (100, 8, 80, 1), (60, 6, 100, 2), (60, 7, 100, 2),
               (100, 8, 80, 1)]
    for start, kappa, bpc, spacer in layouts:
        got = P.pbn_skart_static(cs, start, kappa, bpc, spacer, 0.05, 0.20)
        ref = P.pbn_skart(cs, start, kappa, bpc, spacer, 0.05, 0.20)
        _same(got, ref)


def test_static_rejects_more_batches_than_its_capacity(P):
    N, cs = _chains(P, omega=1024, T=8)
    lib = P.lib()
    out = np.zeros(ctypes.sizeof(P.SkartResult), dtype=np.uint8)
    cap = 1 << 18
    bpc = cap // 1024 + 1
    rc = lib.pbn_skart_static(ctypes.byref(cs.c), 0, 1, bpc, 0, 0.05, 0.2, ctypes.c_void_p(out.ctypes.data),
                              ctypes.c_void_p(0))
    assert rc == P.PBN_ERR_UNSUPPORTED
    assert b"capacity" in lib.pbn_last_error()
