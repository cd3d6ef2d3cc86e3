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


_SHIM = r"""
#define _GNU_SOURCE
#include <dlfcn.h>
#include <stddef.h>
static volatile long g_calls = 0;
long shim_calls(void) { return g_calls; }
void shim_reset(void) { g_calls = 0; }
#define FWD(name, params, args)                                   \
  int name params {                                               \
    static int (*real) params = 0;                                \
    if (!real) real = (int (*) params)dlsym(RTLD_NEXT, #name);    \
    __sync_fetch_and_add(&g_calls, 1);                            \
    return real args;                                             \
  }
FWD(cudaMalloc, (void **p, size_t n), (p, n))
FWD(cudaMallocAsync, (void **p, size_t n, void *s), (p, n, s))
FWD(cudaMallocManaged, (void **p, size_t n, unsigned f), (p, n, f))
FWD(cudaMallocHost, (void **p, size_t n), (p, n))
FWD(cudaHostAlloc, (void **p, size_t n, unsigned f), (p, n, f))
FWD(cudaMallocPitch, (void **p, size_t *pitch, size_t w, size_t h), (p, pitch, w, h))
FWD(cudaMallocFromPoolAsync, (void **p, size_t n, void *pool, void *s), (p, n, pool, s))
"""

_CHILD = r"""
import ctypes, json, sys
sys.path.insert(0, sys.argv[1])
shim = ctypes.CDLL(sys.argv[2])
shim.shim_calls.restype = ctypes.c_long
import torch
from paper_1508_07828_gb300 import _build
import paper_1508_07828_gb300 as P
import pbn_synth as S
net, _, _ = S.mid_config()
N = P.pbn_load(net)
cs = P.ChainSet(N, 96, bits_cap=900)
P.pbn_init_chains(cs, 41)
P.pbn_run_chains(cs, 900, 41, P.PER_NODE, S.StateOfInterest([0, 3], [1, 1]))
out = torch.zeros(ctypes.sizeof(P.SkartResult), dtype=torch.uint8, device="cuda")
stream = torch.cuda.Stream()          # a stream pbn_skart has never seen
torch.cuda.synchronize()
L = P.lib()
args = lambda: (ctypes.byref(cs.c), 100, 8, 80, 1, 0.05, 0.2, ctypes.c_void_p(out.data_ptr()),
                ctypes.c_void_p(stream.cuda_stream))
shim.shim_reset()
rc1 = L.pbn_skart_static(*args())
rc2 = L.pbn_skart_static(*args())
torch.cuda.synchronize()
static_calls = shim.shim_calls()
rc3 = L.pbn_skart(*args())            # the allocating entry point on the same fresh stream
torch.cuda.synchronize()
print(json.dumps({"rc": [rc1, rc2, rc3], "static_calls": static_calls,
                  "allocating_calls": shim.shim_calls() - static_calls}))
"""


def test_static_entry_point_calls_no_allocator(P, tmp_path):
    """In a fresh process whose CUDA runtime allocation calls are counted (a
    shim preloaded in front of the runtime), two calls of pbn_skart_static on
    a stream the library has never seen make no allocation call, while
    pbn_skart on the same stream does (which shows that the count sees the
    library's calls)."""
    import json
    import os
    import subprocess
    import sys
    src, shim = tmp_path / "shim.c", tmp_path / "libshim.so"
    src.write_text(_SHIM)
    subprocess.check_call(["gcc", "-O1", "-shared", "-fPIC", "-o", str(shim), str(src), "-ldl"])
    child = tmp_path / "child.py"
    child.write_text(_CHILD)
    root = os.path.abspath(os.path.join(os.path.dirname(__file__), ".."))
    env = dict(os.environ, LD_PRELOAD=str(shim))
    r = subprocess.run([sys.executable, str(child), root, str(shim)], env=env, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    d = json.loads(r.stdout.strip().splitlines()[-1])
    assert d["rc"] == [0, 0, 0], d
    assert d["static_calls"] == 0, d
    assert d["allocating_calls"] > 0, d
