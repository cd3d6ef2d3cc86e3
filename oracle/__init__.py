"""CPU oracle of the parallel PBN steady-state method.

TEST INFRASTRUCTURE ONLY.  The tests, `__graft_entry__.smoke()` and the
`cpu_baseline` / reference legs of `bench.py` are the only callers.  The CUDA
product path neither imports nor links anything here, and nothing here
imports the product package.

`oracle.c` is a plain, single-threaded C implementation (simulation, Gelman &
Rubin, two-state Markov chain, Skart); `exact.py` computes exact stationary
distributions of small networks by FP64 power iteration.  This module builds
`oracle.c` with gcc and wraps it with ctypes.

Parity status per function (what pins it; see tests/test_oracle_*.py):
  philox4x32_10      cuRAND's host Philox4_32_10 generator (library outputs)
  simulate/init      exact one-step transition law of exact.py (chi-square),
                     exact stationary distributions, hand-built 3-node PBN
  exact (n <= 16)    dense step = implicit step at n = 10..12; uniform law and
                     its closed-form transient on all-identity networks; the
                     product of five exact 3-node laws at n = 16
  gelman_rubin       closed form from integer sums; numpy; R-hat -> 1 on iid
  two_state_MN       closed forms on the identity / constant node
  norm_ppf, t_ppf    scipy.stats norm.ppf / t.ppf
  skewness           scipy.stats.skew
  estimate_two_state exact answers on small networks (within r), up to n = 16
  estimate_two_state_seq
                     Alg. 1 on one chain: the stopping rule, an independent
                     replay of the final window, exact answers within r,
                     agreement with the parallel driver within 2r
  estimate_skart_seq Alg. 2 with the placeholder constants of estimate_skart:
                     an independent recount of its batch means, coverage on
                     processes with a known mean; parity unpinned like Alg. 4
  estimate_two_state_multi
                     reduces to estimate_two_state for one property and for
                     repeated copies of it; complementary properties sum to 1
                     exactly; exact answers on small networks (within r)
  estimate_skart     coverage on processes with a known mean; its constants
                     (skewness threshold, test size, spacer limit, growth
                     factors) are placeholders: parity unpinned.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

PER_NODE = 0
GLOBAL = 1


def build(force: bool = False) -> str:
    """Compile oracle.c into oracle/liboracle.so (plain -O2, single thread)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-ffp-contract=off", "-shared", "-fPIC",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Net(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("F", ctypes.c_int32),
                ("fn_offset", ctypes.c_void_p), ("par_offset", ctypes.c_void_p),
                ("parents", ctypes.c_void_p), ("tt_offset", ctypes.c_void_p), ("tt_words", ctypes.c_void_p),
                ("select_prob", ctypes.c_void_p), ("p", ctypes.c_double)]


class _TwoStateRun(ctypes.Structure):
    _fields_ = [("omega", ctypes.c_int64), ("psi0", ctypes.c_int64), ("rhat_threshold", ctypes.c_double),
                ("max_length", ctypes.c_int64), ("mode", ctypes.c_int32), ("seed", ctypes.c_uint64),
                ("eps", ctypes.c_double), ("r", ctypes.c_double), ("s", ctypes.c_double),
                ("prob", ctypes.c_double), ("rhat", ctypes.c_double), ("alpha", ctypes.c_double),
                ("beta", ctypes.c_double), ("psi", ctypes.c_int64), ("gr_psi", ctypes.c_int64),
                ("length", ctypes.c_int64), ("sample_size", ctypes.c_int64), ("M", ctypes.c_int64),
                ("N", ctypes.c_int64), ("n4", ctypes.c_int64 * 4), ("ones", ctypes.c_int64),
                ("gr_rounds", ctypes.c_int32), ("ts_rounds", ctypes.c_int32), ("status", ctypes.c_int32)]


class _SkartRun(ctypes.Structure):
    _fields_ = [("omega", ctypes.c_int64), ("psi0", ctypes.c_int64), ("rhat_threshold", ctypes.c_double),
                ("max_length", ctypes.c_int64), ("mode", ctypes.c_int32), ("seed", ctypes.c_uint64),
                ("H_star", ctypes.c_double), ("relative", ctypes.c_int32), ("alpha", ctypes.c_double),
                ("mean", ctypes.c_double), ("ci_lo", ctypes.c_double), ("ci_hi", ctypes.c_double),
                ("H", ctypes.c_double), ("var", ctypes.c_double), ("skew", ctypes.c_double),
                ("phi", ctypes.c_double), ("rhat", ctypes.c_double),
                ("psi", ctypes.c_int64), ("length", ctypes.c_int64), ("kappa", ctypes.c_int64),
                ("batches", ctypes.c_int64), ("spacer", ctypes.c_int64), ("sample_size", ctypes.c_int64),
                ("gr_rounds", ctypes.c_int32), ("rand_rounds", ctypes.c_int32), ("ci_rounds", ctypes.c_int32),
                ("status", ctypes.c_int32)]


class _SkartCI(ctypes.Structure):
    _fields_ = [(k, ctypes.c_double) for k in ("mean", "var", "skew", "phi", "A", "H", "ci_lo", "ci_hi")]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            vp, i32, i64, u64, dbl = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
            L.orc_philox4x32_10.argtypes = [vp, vp, vp]
            L.orc_validate.argtypes = [vp]
            L.orc_perturb_threshold.argtypes = [dbl]; L.orc_perturb_threshold.restype = ctypes.c_uint32
            L.orc_select_thresholds.argtypes = [vp, vp]
            L.orc_uniform.argtypes = [u64, i32, u64, i64]; L.orc_uniform.restype = ctypes.c_uint32
            L.orc_init_states.argtypes = [vp, u64, i64, vp]
            L.orc_simulate.argtypes = [vp, i32, u64, i64, u64, i64, vp, vp, vp, i32, vp, i64]
            L.orc_simulate_from.argtypes = [vp, i32, u64, i64, i64, u64, i64, vp, vp, vp, i32, vp, i64]
            L.orc_init_states_from.argtypes = [vp, u64, i64, i64, vp]
            L.orc_gelman_rubin.argtypes = [vp, i64, i64, i64, i64]; L.orc_gelman_rubin.restype = dbl
            L.orc_norm_ppf.argtypes = [dbl]; L.orc_norm_ppf.restype = dbl
            L.orc_t_ppf.argtypes = [dbl, dbl]; L.orc_t_ppf.restype = dbl
            L.orc_two_state_MN.argtypes = [dbl, dbl, dbl, dbl, dbl, vp, vp]
            L.orc_transition_counts.argtypes = [vp, i64, i64, i64, i64, vp]
            L.orc_estimate_two_state.argtypes = [vp, vp, vp, i32, vp]
            L.orc_estimate_two_state_multi.argtypes = [vp, i32, vp, vp, vp, vp, vp]
            L.orc_estimate_two_state_seq.argtypes = [vp, vp, vp, i32, vp]
            L.orc_estimate_skart_seq.argtypes = [vp, vp, vp, i32, vp]
            L.orc_skewness.argtypes = [vp, i64]; L.orc_skewness.restype = dbl
            L.orc_vonneumann_pass.argtypes = [vp, i64, i64, i64, dbl, vp]
            L.orc_skart_ci_from_means.argtypes = [vp, i64, i64, dbl, vp]
            L.orc_estimate_skart.argtypes = [vp, vp, vp, i32, vp]
            _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


class NetHandle:
    """Keeps the contiguous arrays alive for the C struct."""

    def __init__(self, net):
        self.fn_offset = np.ascontiguousarray(net.fn_offset, dtype=np.int32)
        self.par_offset = np.ascontiguousarray(net.par_offset, dtype=np.int32)
        self.parents = np.ascontiguousarray(net.parents if len(net.parents) else np.zeros(1, np.int32), dtype=np.int32)
        self.tt_offset = np.ascontiguousarray(net.tt_offset, dtype=np.int32)
        self.tt_words = np.ascontiguousarray(net.tt_words, dtype=np.uint32)
        self.select_prob = np.ascontiguousarray(net.select_prob, dtype=np.float64)
        self.n = int(net.n)
        self.s = _Net(self.n, int(self.fn_offset[-1]), self.fn_offset.ctypes.data, self.par_offset.ctypes.data,
                      self.parents.ctypes.data, self.tt_offset.ctypes.data, self.tt_words.ctypes.data,
                      self.select_prob.ctypes.data,
                      float(net.p))

    @property
    def ref(self):
        return ctypes.byref(self.s)


def philox4x32_10(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def validate(net) -> int:
    h = NetHandle(net)
    return int(lib().orc_validate(h.ref))


def perturb_threshold(p: float) -> int:
    return int(lib().orc_perturb_threshold(float(p)))


def select_thresholds(net) -> np.ndarray:
    h = NetHandle(net)
    thr = np.zeros(net.n_functions, dtype=np.uint64)
    lib().orc_select_thresholds(h.ref, _ptr(thr))
    return thr


def uniform(seed: int, node: int, t: int, chain: int) -> int:
    return int(lib().orc_uniform(seed, node, t, chain))


def init_states(net, seed: int, omega: int, chain0: int = 0) -> np.ndarray:
    """Initial states of chains chain0 .. chain0+omega-1 as uint8 [omega, n]."""
    h = NetHandle(net)
    st = np.zeros((omega, net.n), dtype=np.uint8)
    lib().orc_init_states_from(h.ref, seed, chain0, omega, _ptr(st))
    return st


def simulate(net, mode: int, seed: int, states: np.ndarray, t0: int, steps: int, soi=None, record=True,
             chain0: int = 0):
    """Advance states (uint8 [omega, n], modified copy returned) of chains
    chain0 .. chain0+omega-1 by `steps` transitions starting at transition
    index t0.  Returns (states, ind) with ind uint8 [omega, steps] (indicator
    of the state of interest after each transition) or None."""
    h = NetHandle(net)
    st = np.ascontiguousarray(states, dtype=np.uint8).copy()
    omega = st.shape[0]
    if soi is None:
        nodes = np.zeros(1, np.int32); vals = np.zeros(1, np.uint8); k = 0
    else:
        nodes = np.ascontiguousarray(soi.nodes, dtype=np.int32); vals = np.ascontiguousarray(soi.values, dtype=np.uint8)
        k = len(nodes)
    ind = np.zeros((omega, steps), dtype=np.uint8) if record else None
    rc = lib().orc_simulate_from(h.ref, mode, seed, chain0, omega, t0, steps, _ptr(st), _ptr(nodes), _ptr(vals),
                                 k, _ptr(ind) if record else None, steps)
    if rc:
        raise RuntimeError(f"orc_simulate failed: {rc}")
    return st, ind


def gelman_rubin(x: np.ndarray, start: int, psi: int) -> float:
    x = np.ascontiguousarray(x, dtype=np.uint8)
    return float(lib().orc_gelman_rubin(_ptr(x), x.shape[0], x.shape[1], start, psi))


def norm_ppf(q: float) -> float:
    return float(lib().orc_norm_ppf(q))


def t_ppf(q: float, dof: float) -> float:
    return float(lib().orc_t_ppf(q, dof))


def two_state_MN(alpha, beta, eps, r, s):
    M = ctypes.c_int64(); N = ctypes.c_int64()
    rc = lib().orc_two_state_MN(alpha, beta, eps, r, s, ctypes.byref(M), ctypes.byref(N))
    return rc, int(M.value), int(N.value)


def transition_counts(x: np.ndarray, start: int, length: int) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.uint8)
    out = np.zeros(4, dtype=np.int64)
    lib().orc_transition_counts(_ptr(x), x.shape[0], x.shape[1], start, length, _ptr(out))
    return out


def skewness(v) -> float:
    v = np.ascontiguousarray(v, dtype=np.float64)
    return float(lib().orc_skewness(_ptr(v), len(v)))


def vonneumann_pass(means: np.ndarray, omega: int, bpc: int, d: int, alpha_ran: float = 0.2):
    m = np.ascontiguousarray(means, dtype=np.float64)
    stat = ctypes.c_double()
    ok = lib().orc_vonneumann_pass(_ptr(m), omega, bpc, d, alpha_ran, ctypes.byref(stat))
    return bool(ok), float(stat.value)


def skart_ci(means: np.ndarray, omega: int, bpc: int, alpha: float) -> dict:
    m = np.ascontiguousarray(means, dtype=np.float64)
    o = _SkartCI()
    lib().orc_skart_ci_from_means(_ptr(m), omega, bpc, alpha, ctypes.byref(o))
    return {k: getattr(o, k) for k, _ in _SkartCI._fields_}


def _soi_arrays(soi):
    return (np.ascontiguousarray(soi.nodes, dtype=np.int32), np.ascontiguousarray(soi.values, dtype=np.uint8))


def estimate_two_state(net, soi, omega, seed, psi0=1024, rhat=1.05, eps=1e-10, r=0.005, s=0.95,
                       mode=PER_NODE, max_length=1 << 26) -> dict:
    """Alg. GR then Alg. 3 (parallel two-state Markov chain approach)."""
    h = NetHandle(net)
    nodes, vals = _soi_arrays(soi)
    run = _TwoStateRun()
    run.omega, run.psi0, run.rhat_threshold, run.max_length = omega, psi0, rhat, max_length
    run.mode, run.seed, run.eps, run.r, run.s = mode, seed, eps, r, s
    rc = lib().orc_estimate_two_state(h.ref, _ptr(nodes), _ptr(vals), len(nodes), ctypes.byref(run))
    out = {k: getattr(run, k) for k, _ in _TwoStateRun._fields_ if k != "n4"}
    out["n4"] = list(run.n4)
    out["status"] = rc
    return out


class _TwoStateSeqRun(ctypes.Structure):
    _fields_ = [("m0", ctypes.c_int64), ("n0", ctypes.c_int64), ("max_length", ctypes.c_int64),
                ("mode", ctypes.c_int32), ("seed", ctypes.c_uint64), ("chain", ctypes.c_int64),
                ("eps", ctypes.c_double), ("r", ctypes.c_double), ("s", ctypes.c_double),
                ("prob", ctypes.c_double), ("alpha", ctypes.c_double), ("beta", ctypes.c_double),
                ("M", ctypes.c_int64), ("N", ctypes.c_int64), ("length", ctypes.c_int64), ("ones", ctypes.c_int64),
                ("n4", ctypes.c_int64 * 4), ("ab_window", ctypes.c_int64), ("rounds", ctypes.c_int32),
                ("status", ctypes.c_int32)]


def estimate_two_state_seq(net, soi, seed, m0=0, n0=1024, eps=1e-10, r=0.005, s=0.95, mode=PER_NODE, chain=0,
                           max_length=1 << 30) -> dict:
    """Alg. 1 (sequential two-state Markov chain approach) on chain `chain`
    of the seed's family."""
    h = NetHandle(net)
    nodes, vals = _soi_arrays(soi)
    run = _TwoStateSeqRun()
    run.m0, run.n0, run.max_length, run.mode, run.seed, run.chain = m0, n0, max_length, mode, seed, chain
    run.eps, run.r, run.s = eps, r, s
    rc = lib().orc_estimate_two_state_seq(h.ref, _ptr(nodes), _ptr(vals), len(nodes), ctypes.byref(run))
    out = {k: getattr(run, k) for k, _ in _TwoStateSeqRun._fields_ if k != "n4"}
    out["n4"] = list(run.n4)
    out["status"] = rc
    return out


class _Property(ctypes.Structure):
    _fields_ = [("prob", ctypes.c_double), ("alpha", ctypes.c_double), ("beta", ctypes.c_double),
                ("rhat", ctypes.c_double), ("M", ctypes.c_int64), ("N", ctypes.c_int64), ("ones", ctypes.c_int64),
                ("n4", ctypes.c_int64 * 4)]


MAX_PROPERTIES = 8


def estimate_two_state_multi(net, sois, omega, seed, psi0=1024, rhat=1.05, eps=1e-10, r=0.005, s=0.95,
                             mode=PER_NODE, max_length=1 << 26) -> dict:
    """Several properties from the same trajectories (Sec. 4.2, last part):
    common chains, Alg. GR over every property, extension by the smallest
    deficit, burn-in by the largest M.  Returns the common run fields (whose
    per-property fields repeat property 0) and "properties": one dict each."""
    h = NetHandle(net)
    q = len(sois)
    nodes = np.ascontiguousarray(np.concatenate([np.asarray(x.nodes) for x in sois]), dtype=np.int32)
    vals = np.ascontiguousarray(np.concatenate([np.asarray(x.values) for x in sois]), dtype=np.uint8)
    sizes = np.ascontiguousarray([len(x.nodes) for x in sois], dtype=np.int32)
    run = _TwoStateRun()
    run.omega, run.psi0, run.rhat_threshold, run.max_length = omega, psi0, rhat, max_length
    run.mode, run.seed, run.eps, run.r, run.s = mode, seed, eps, r, s
    props = (_Property * MAX_PROPERTIES)()
    rc = lib().orc_estimate_two_state_multi(h.ref, q, _ptr(nodes), _ptr(vals), _ptr(sizes), ctypes.byref(run),
                                            ctypes.byref(props))
    out = {k: getattr(run, k) for k, _ in _TwoStateRun._fields_ if k != "n4"}
    out["n4"] = list(run.n4)
    out["status"] = rc
    out["properties"] = [dict({k: getattr(props[m], k) for k, _ in _Property._fields_ if k != "n4"},
                              n4=list(props[m].n4)) for m in range(q)]
    return out


def estimate_skart(net, soi, omega, seed, H_star, relative=True, alpha=0.05, psi0=1024, rhat=1.05,
                   mode=PER_NODE, max_length=1 << 26) -> dict:
    """Alg. GR then Alg. 4 (parallel Skart)."""
    h = NetHandle(net)
    nodes, vals = _soi_arrays(soi)
    run = _SkartRun()
    run.omega, run.psi0, run.rhat_threshold, run.max_length = omega, psi0, rhat, max_length
    run.mode, run.seed, run.H_star, run.relative, run.alpha = mode, seed, H_star, int(relative), alpha
    rc = lib().orc_estimate_skart(h.ref, _ptr(nodes), _ptr(vals), len(nodes), ctypes.byref(run))
    out = {k: getattr(run, k) for k, _ in _SkartRun._fields_}
    out["status"] = rc
    return out


def estimate_skart_seq(net, soi, seed, H_star, relative=True, alpha=0.05, mode=PER_NODE, max_length=1 << 30) -> dict:
    """Alg. 2 (sequential Skart) on chain 0 of the seed's family; "psi" is the
    skipped zeta = d kappa and "batches" the final p'."""
    h = NetHandle(net)
    nodes, vals = _soi_arrays(soi)
    run = _SkartRun()
    run.omega, run.psi0, run.rhat_threshold, run.max_length = 1, 0, 0.0, max_length
    run.mode, run.seed, run.H_star, run.relative, run.alpha = mode, seed, H_star, int(relative), alpha
    rc = lib().orc_estimate_skart_seq(h.ref, _ptr(nodes), _ptr(vals), len(nodes), ctypes.byref(run))
    out = {k: getattr(run, k) for k, _ in _SkartRun._fields_}
    out["status"] = rc
    return out
