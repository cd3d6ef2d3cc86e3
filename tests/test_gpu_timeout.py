"""A bounded device-side wait that runs out: a TMA tile that is never issued
(test hook PBN_TEST_STALL_FIRST_TILE=1, read when the library loads) makes
the fused simulation kernel give up after its 1 s limit, record
PBN_ERR_TIMEOUT in the device status word and return; the host reads the
status, a driver query reading results after such a launch fails with
PBN_ERR_TIMEOUT, and the CUDA context stays usable.  The same hook keeps the
register-resident apply kernel's first bulk copy from being issued: its
producer gives up on that step after 1 s, issues nothing more, and the
launch ends with the same status."""
import os
import subprocess
import sys
import textwrap

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.abspath(os.path.join(os.path.dirname(__file__), ".."))

CHILD = textwrap.dedent("""
    import sys
    sys.path.insert(0, {root!r})
    import numpy as np
    import torch
    import pbn_synth as S
    import paper_1508_07828_gb300 as P
    # tables of about 380 KB, streamed through shared memory as TMA tiles
    net = S.random_pbn(3, 4096, (4, 8), (2, 4), "biased", "uniform", 0.01)
    soi = S.StateOfInterest([0], [1])
    N = P.pbn_load(net)
    cs = P.ChainSet(N, 64, bits_cap=16)
    P.pbn_init_chains(cs, 1)
    P.pbn_run_chains(cs, 4, 1, P.PER_NODE, soi, staging="tiles", schedule="fused")
    torch.cuda.synchronize()
    st = P.pbn_take_device_status()
    assert st == P.PBN_ERR_TIMEOUT, st
    assert P.pbn_take_device_status() == 0          # cleared
    # a stalled launch queued ahead of a query on the same stream: the query's
    # first result read also reads the status word and fails the query
    P.pbn_run_chains(cs, 4, 1, P.PER_NODE, soi, staging="tiles", schedule="fused")
    try:
        P.pbn_estimate_two_state(N, soi, omega=64, seed=2, psi0=64, r=0.05, max_length=256)
        raise SystemExit("expected a timeout")
    except P.PbnError as e:
        assert e.status == P.PBN_ERR_TIMEOUT, e
    assert P.pbn_take_device_status() == 0          # the failed query cleared it
    # the context is still usable: untiled launches and plain torch work
    P.pbn_run_chains(cs, 4, 1, P.PER_NODE, soi, staging="global")
    torch.cuda.synchronize()
    assert P.pbn_take_device_status() == 0
    x = torch.arange(10, device="cuda").sum().item()
    assert x == 45
    print("timeout path ok")
""")


def test_stalled_tile_times_out_and_context_survives():
    from paper_1508_07828_gb300 import _build
    _build.build()
    env = dict(os.environ, PBN_TEST_STALL_FIRST_TILE="1")
    r = subprocess.run([sys.executable, "-c", CHILD.format(root=ROOT)], env=env, capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "timeout path ok" in r.stdout


CHILD_RESIDENT = textwrap.dedent("""
    import sys
    sys.path.insert(0, {root!r})
    import torch
    import pbn_synth as S
    import paper_1508_07828_gb300 as P
    net, soi, cfg = S.mid_config()
    N = P.pbn_load(net)
    cs = P.ChainSet(N, 64, bits_cap=64)
    P.pbn_init_chains(cs, 1)
    # one select-ahead chunk: select_kernel, then the register-resident apply
    P.pbn_run_chains(cs, 40, 1, P.PER_NODE, soi, schedule="select_ahead")
    torch.cuda.synchronize()
    st = P.pbn_take_device_status()
    assert st == P.PBN_ERR_TIMEOUT, st
    assert P.pbn_take_device_status() == 0
    # the context is still usable: the fused schedule and plain torch work
    P.pbn_run_chains(cs, 4, 1, P.PER_NODE, soi, schedule="fused")
    torch.cuda.synchronize()
    assert P.pbn_take_device_status() == 0
    assert torch.arange(10, device="cuda").sum().item() == 45
    print("resident timeout path ok")
""")


def test_stalled_bulk_copy_times_out_and_context_survives():
    from paper_1508_07828_gb300 import _build
    _build.build()
    env = dict(os.environ, PBN_TEST_STALL_FIRST_TILE="1")
    r = subprocess.run([sys.executable, "-c", CHILD_RESIDENT.format(root=ROOT)], env=env, capture_output=True,
                       text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "resident timeout path ok" in r.stdout
