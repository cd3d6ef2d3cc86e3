"""Python binding of libpbn_gb300.so, the C-ABI GB300 engine for parallel
approximate steady-state analysis of probabilistic Boolean networks.

Argument marshalling only: every step of the method runs in the library's
CUDA kernels.  PyTorch provides device memory (tensors whose data pointers are
passed through the ABI) and the current CUDA stream.  The binding fails loudly
when the compiled library is missing; there is no CPU path.

Entry points keep the C names (see include/pbn.h): pbn_load, pbn_init_chains,
pbn_run_chains, pbn_gelman_rubin, pbn_two_state, pbn_skart,
pbn_estimate_two_state, pbn_estimate_skart.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpbn_gb300.so")

PBN_OK = 0
PBN_ERR_INVALID = 1
PBN_ERR_OOM = 2
PBN_ERR_CUDA = 3
PBN_ERR_TIMEOUT = 4
PBN_ERR_NOT_CONVERGED = 5
PBN_ERR_INSUFFICIENT = 6
PBN_ERR_UNSUPPORTED = 7
PBN_ERR_CANCELLED = 8
PER_NODE = 0
GLOBAL = 1
MAX_SOI = 32


class PbnError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"pbn status {status}: {msg}")
        self.status = status


# ----------------------------------------------------------- ABI structures

c_i32, c_i64, c_u32, c_u64, c_dbl, c_vp = (ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32, ctypes.c_uint64,
                                           ctypes.c_double, ctypes.c_void_p)


class NetworkDesc(ctypes.Structure):
    _fields_ = [("n", c_i32), ("n_functions", c_i32), ("fn_offset", c_vp), ("par_offset", c_vp),
                ("parents", c_vp), ("truth_table", c_vp), ("select_prob", c_vp), ("p", c_dbl),
                ("tt_offset", c_vp), ("tt_words", c_vp)]


class NetInfo(ctypes.Structure):
    _fields_ = [("n", c_i32), ("n_functions", c_i32), ("perturb_threshold", c_u32), ("table_bytes", c_i64)]


class Soi(ctypes.Structure):
    _fields_ = [("size", c_i32), ("nodes", c_vp), ("values", c_vp)]


class Chains(ctypes.Structure):
    _fields_ = [("omega", c_i64), ("state", c_vp), ("bits", c_vp), ("bits_cap", c_i64), ("bits_base", c_i64),
                ("length", c_i64)]


class RunCfg(ctypes.Structure):
    _fields_ = [("seed", c_u64), ("perturb_mode", c_i32), ("soi", Soi), ("groups_per_block", c_i32),
                ("threads_per_block", c_i32), ("threads_per_item", c_i32), ("blocks_per_round", c_i32),
                ("staging", c_i32), ("schedule", c_i32), ("n_props", c_i32), ("props", c_vp)]


class GrResult(ctypes.Structure):
    _fields_ = [("rhat", c_dbl), ("W", c_dbl), ("B", c_dbl), ("sigma2", c_dbl), ("S1", c_u64), ("S2_lo", c_u64),
                ("S2_hi", c_u64)]


class TwoStateResult(ctypes.Structure):
    _fields_ = [("n00", c_i64), ("n01", c_i64), ("n10", c_i64), ("n11", c_i64), ("ones", c_i64),
                ("alpha", c_dbl), ("beta", c_dbl), ("prob", c_dbl), ("M", c_i64), ("N", c_i64),
                ("status", c_i32), ("pad", c_i32)]


class SkartResult(ctypes.Structure):
    _fields_ = [(k, c_dbl) for k in ("mean", "var", "skew", "phi", "A", "H", "ci_lo", "ci_hi", "vn_stat")] + \
               [("vn_pass", c_i32), ("pad", c_i32), ("batches", c_i64)]


class TwoStateQuery(ctypes.Structure):
    _fields_ = [("omega", c_i64), ("psi0", c_i64), ("rhat_threshold", c_dbl), ("eps", c_dbl), ("r", c_dbl),
                ("s", c_dbl), ("max_length", c_i64), ("seed", c_u64), ("perturb_mode", c_i32), ("soi", Soi)]


class TwoStateReport(ctypes.Structure):
    _fields_ = [("prob", c_dbl), ("rhat", c_dbl), ("alpha", c_dbl), ("beta", c_dbl), ("psi", c_i64),
                ("gr_psi", c_i64), ("length", c_i64), ("sample_size", c_i64), ("M", c_i64), ("N", c_i64),
                ("ones", c_i64), ("n4", c_i64 * 4), ("gr_rounds", c_i32), ("ts_rounds", c_i32),
                ("chain_node_updates", c_i64), ("device_ms", c_dbl), ("sim_ms", c_dbl), ("sim_launches", c_i64),
                ("kernel_launches", c_i64), ("sim_items", c_i64), ("d2h_bytes", c_i64), ("apply_ms", c_dbl),
                ("apply_launches", c_i64)]


class TwoStateSeqQuery(ctypes.Structure):
    _fields_ = [("m0", c_i64), ("n0", c_i64), ("eps", c_dbl), ("r", c_dbl), ("s", c_dbl), ("max_length", c_i64),
                ("seed", c_u64), ("perturb_mode", c_i32), ("soi", Soi)]


class TwoStateSeqReport(ctypes.Structure):
    _fields_ = [("prob", c_dbl), ("alpha", c_dbl), ("beta", c_dbl), ("M", c_i64), ("N", c_i64), ("length", c_i64),
                ("ones", c_i64), ("n4", c_i64 * 4), ("ab_window", c_i64), ("rounds", c_i32),
                ("chain_node_updates", c_i64), ("device_ms", c_dbl), ("sim_ms", c_dbl), ("sim_launches", c_i64),
                ("kernel_launches", c_i64), ("d2h_bytes", c_i64)]


class PropertyResult(ctypes.Structure):
    _fields_ = [("prob", c_dbl), ("alpha", c_dbl), ("beta", c_dbl), ("rhat", c_dbl), ("M", c_i64), ("N", c_i64),
                ("ones", c_i64), ("n4", c_i64 * 4)]


class SkartQuery(ctypes.Structure):
    _fields_ = [("omega", c_i64), ("psi0", c_i64), ("rhat_threshold", c_dbl), ("H_star", c_dbl),
                ("relative", c_i32), ("alpha", c_dbl), ("max_length", c_i64), ("seed", c_u64),
                ("perturb_mode", c_i32), ("soi", Soi)]


class SkartReport(ctypes.Structure):
    _fields_ = [(k, c_dbl) for k in ("mean", "ci_lo", "ci_hi", "H", "var", "skew", "phi", "rhat")] + \
               [(k, c_i64) for k in ("psi", "length", "kappa", "batches", "spacer", "sample_size")] + \
               [("gr_rounds", c_i32), ("rand_rounds", c_i32), ("ci_rounds", c_i32),
                ("chain_node_updates", c_i64), ("device_ms", c_dbl), ("sim_ms", c_dbl), ("sim_launches", c_i64),
                ("kernel_launches", c_i64), ("sim_items", c_i64), ("d2h_bytes", c_i64), ("apply_ms", c_dbl),
                ("apply_launches", c_i64)]


class EngineCfg(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", c_i64), ("max_active", c_i32), ("steps_per_epoch", c_i32),
                ("threads_per_block", c_i32), ("items_per_thread", c_i32), ("use_graph", c_i32),
                ("epoch_target_ms", c_dbl)]


class EngineQuery(ctypes.Structure):
    _fields_ = [("net", c_vp), ("method", c_i32), ("two_state", TwoStateQuery), ("skart", SkartQuery), ("tag", c_u64)]


class EngineResult(ctypes.Structure):
    _fields_ = [("id", c_i64), ("tag", c_u64), ("method", c_i32), ("status", c_i32), ("two_state", TwoStateReport),
                ("skart", SkartReport), ("submit_epoch", c_i64), ("admit_epoch", c_i64), ("finish_epoch", c_i64)]


class EngineStats(ctypes.Structure):
    _fields_ = [("epoch", c_i64), ("active", c_i32), ("pending", c_i32), ("finished", c_i64), ("updates", c_i64),
                ("epoch_ms", c_dbl), ("hbm_in_use", c_i64), ("steps_per_epoch", c_i32),
                ("threads_per_block", c_i32), ("items_per_thread", c_i32), ("kernel_launches", c_i32),
                ("sim_ms", c_dbl), ("sim_items", c_i64), ("d2h_bytes", c_i64), ("tuning", c_i32), ("pad", c_i32)]


METHOD_TWO_STATE = 0
METHOD_SKART = 1

_lock = threading.Lock()
_lib = None


def lib():
    """The loaded C-ABI library (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise ImportError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() "
                                  "(the CUDA extension is required; there is no CPU path)")
            L = ctypes.CDLL(LIB_PATH)
            P = ctypes.POINTER
            L.pbn_load.argtypes = [P(NetworkDesc), P(c_vp)]
            L.pbn_free.argtypes = [c_vp]
            L.pbn_free.restype = None
            L.pbn_net_get_info.argtypes = [c_vp, P(NetInfo)]
            L.pbn_init_chains.argtypes = [c_vp, P(RunCfg), P(Chains), c_vp]
            L.pbn_run_chains.argtypes = [c_vp, P(RunCfg), P(Chains), c_i64, c_vp]
            L.pbn_balance_phases.argtypes = [c_i32, c_i32, c_i32, c_i32, c_i32, c_i32, c_i64, P(c_i32), P(c_i32)]
            L.pbn_gelman_rubin.argtypes = [P(Chains), c_i64, c_i64, c_vp, c_vp]
            L.pbn_two_state.argtypes = [P(Chains), c_i64, c_i64, c_dbl, c_dbl, c_dbl, c_vp, c_vp]
            L.pbn_skart.argtypes = [P(Chains), c_i64, c_i64, c_i64, c_i64, c_dbl, c_dbl, c_vp, c_vp]
            L.pbn_skart_static.argtypes = [P(Chains), c_i64, c_i64, c_i64, c_i64, c_dbl, c_dbl, c_vp, c_vp]
            L.pbn_estimate_two_state.argtypes = [c_vp, P(TwoStateQuery), P(TwoStateReport), c_vp]
            L.pbn_estimate_two_state_multi.argtypes = [c_vp, P(TwoStateQuery), c_i32, c_vp, P(TwoStateReport),
                                                       P(PropertyResult), c_vp]
            L.pbn_estimate_two_state_seq.argtypes = [c_vp, P(TwoStateSeqQuery), P(TwoStateSeqReport), c_vp]
            L.pbn_estimate_skart_seq.argtypes = [c_vp, P(SkartQuery), P(SkartReport), c_vp]
            L.pbn_estimate_skart.argtypes = [c_vp, P(SkartQuery), P(SkartReport), c_vp]
            L.pbn_engine_create.argtypes = [P(EngineCfg), c_vp, P(c_vp)]
            L.pbn_engine_destroy.argtypes = [c_vp]
            L.pbn_engine_destroy.restype = None
            L.pbn_engine_submit.argtypes = [c_vp, P(EngineQuery), P(c_i64)]
            L.pbn_engine_step.argtypes = [c_vp, P(EngineStats)]
            L.pbn_engine_poll.argtypes = [c_vp, c_vp, c_i32, P(c_i32)]
            L.pbn_engine_cancel.argtypes = [c_vp, c_i64]
            L.pbn_take_device_status.argtypes = [P(c_i32)]
            L.pbn_last_error.restype = ctypes.c_char_p
            L.pbn_status_string.restype = ctypes.c_char_p
            L.pbn_status_string.argtypes = [ctypes.c_int]
            _lib = L
    return _lib


def _check(rc):
    if rc != PBN_OK:
        raise PbnError(rc, lib().pbn_last_error().decode())


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("a CUDA device is required")
    return torch


def _stream(stream=None):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return c_vp(s.cuda_stream)


def _as_struct(cls, obj):
    return {k: (list(getattr(obj, k)) if k == "n4" else getattr(obj, k)) for k, _ in cls._fields_ if k != "pad"}


# ------------------------------------------------------------------ network

def _network_counts(n: int, a: dict, n_parents: int) -> int:
    """The function count F to pass to pbn_load with the host arrays `a`
    (numpy arrays or host tensors): the entries of select_prob.  pbn_load
    reads every array up to the length that n and F imply, so arrays of any
    other length are refused here."""
    F = len(a["select_prob"])
    sizes = [("fn_offset", n + 1), ("truth_table", F), ("par_offset", F + 1)]
    if "tt_offset" in a:
        sizes.append(("tt_offset", F + 1))
    for name, want in sizes:
        if len(a[name]) != want:
            raise PbnError(PBN_ERR_INVALID, f"{name} has {len(a[name])} entries, {want} expected "
                                            f"(n = {n}, {F} functions)")
    ends = [("parents", "par_offset", n_parents)]
    if "tt_offset" in a:
        ends.append(("tt_words", "tt_offset", len(a["tt_words"])))
    for name, off, have in ends:
        if int(a[off][-1]) > have:
            raise PbnError(PBN_ERR_INVALID, f"{name} has {have} entries, {off}[-1] = {int(a[off][-1])}")
    return F


class Network:
    """A PBN staged on the device (owns the pbn_net handle)."""

    def __init__(self, net):
        self._arrays = dict(
            fn_offset=np.ascontiguousarray(net.fn_offset, dtype=np.int32),
            par_offset=np.ascontiguousarray(net.par_offset, dtype=np.int32),
            parents=np.ascontiguousarray(net.parents if len(net.parents) else np.zeros(1, np.int32), dtype=np.int32),
            truth_table=np.ascontiguousarray(net.truth_table, dtype=np.uint32),
            select_prob=np.ascontiguousarray(net.select_prob, dtype=np.float64))
        wide = getattr(net, "tt_offset", None) is not None
        if wide:
            self._arrays["tt_offset"] = np.ascontiguousarray(net.tt_offset, dtype=np.int32)
            self._arrays["tt_words"] = np.ascontiguousarray(net.tt_words, dtype=np.uint32)
        a = self._arrays
        n, F = int(net.n), _network_counts(int(net.n), a, len(net.parents))
        desc = NetworkDesc(n, F, a["fn_offset"].ctypes.data, a["par_offset"].ctypes.data,
                           a["parents"].ctypes.data, a["truth_table"].ctypes.data, a["select_prob"].ctypes.data,
                           float(net.p), a["tt_offset"].ctypes.data if wide else None,
                           a["tt_words"].ctypes.data if wide else None)
        h = c_vp()
        _check(lib().pbn_load(ctypes.byref(desc), ctypes.byref(h)))
        self.handle = h
        self.n = n
        self.n_functions = F

    def info(self) -> dict:
        o = NetInfo()
        _check(lib().pbn_net_get_info(self.handle, ctypes.byref(o)))
        return _as_struct(NetInfo, o)

    def close(self):
        if getattr(self, "handle", None):
            lib().pbn_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pbn_load(net) -> Network:
    return Network(net)


def pbn_load_pinned(host_arrays: dict, n: int, p: float) -> Network:
    """Stage a network whose CSR arrays are pinned host tensors (keys
    fn_offset, par_offset, parents, truth_table, select_prob, and optionally
    tt_offset, tt_words): pbn_load then copies them to the device from
    page-locked memory."""
    self = Network.__new__(Network)
    self._arrays = host_arrays
    a = host_arrays
    F = _network_counts(int(n), a, len(a["parents"]))
    desc = NetworkDesc(int(n), F, a["fn_offset"].data_ptr(), a["par_offset"].data_ptr(),
                       a["parents"].data_ptr(), a["truth_table"].data_ptr(), a["select_prob"].data_ptr(), float(p),
                       a["tt_offset"].data_ptr() if "tt_offset" in a else None,
                       a["tt_words"].data_ptr() if "tt_words" in a else None)
    h = c_vp()
    _check(lib().pbn_load(ctypes.byref(desc), ctypes.byref(h)))
    self.handle = h
    self.n = int(n)
    self.n_functions = F
    return self


class SoiArg:
    def __init__(self, soi):
        if soi is None:
            self.nodes = np.zeros(1, np.int32); self.values = np.zeros(1, np.uint8); self.size = 0
        else:
            self.nodes = np.ascontiguousarray(soi.nodes, dtype=np.int32).reshape(-1)
            self.values = np.ascontiguousarray(soi.values, dtype=np.uint8).reshape(-1)
            if len(self.values) != len(self.nodes):  # the C call reads `size` entries of each
                raise PbnError(PBN_ERR_INVALID, f"state of interest: {len(self.nodes)} nodes, "
                                                f"{len(self.values)} values")
            self.size = len(self.nodes)
        self.struct = Soi(self.size, self.nodes.ctypes.data, self.values.ctypes.data)


class PropsArg:
    """Several states of interest as a pbn_soi array (keeps the host arrays alive)."""

    def __init__(self, sois):
        self.items = [SoiArg(x) for x in (sois or [])]
        self.array = (Soi * max(1, len(self.items)))(*[x.struct for x in self.items])
        self.count = len(self.items)
        self.ptr = ctypes.cast(self.array, c_vp).value if self.count else None


# ------------------------------------------------------------------- chains

class ChainSet:
    """omega chains of one network in caller-owned device memory (torch
    tensors): bit-sliced states [G, n] and indicator bitstreams
    [n_props * G, cap] (property m in rows m*G .. m*G+G-1)."""

    def __init__(self, network: Network, omega: int, bits_cap: int = 0, bits_base: int = 0, n_props: int = 1):
        torch = _torch()
        self.network = network
        self.omega = int(omega)
        self.G = (self.omega + 31) // 32
        self.n_props = int(n_props)
        self.state = torch.zeros((self.G, network.n), dtype=torch.int32, device="cuda")
        self.bits = torch.zeros((self.n_props * self.G, max(bits_cap, 1)), dtype=torch.int32,
                                device="cuda") if bits_cap else None
        self.c = Chains(self.omega, self.state.data_ptr(), self.bits.data_ptr() if self.bits is not None else None,
                        int(bits_cap), int(bits_base), 0)

    @property
    def length(self) -> int:
        return int(self.c.length)

    def states_numpy(self) -> np.ndarray:
        """Node values as uint8 [omega, n] (unpacked from the bit-sliced words)."""
        w = self.state.cpu().numpy().view(np.uint32)
        lanes = np.arange(32, dtype=np.uint32)
        bits = ((w[:, None, :] >> lanes[None, :, None]) & 1).astype(np.uint8)  # [G, 32, n]
        return bits.reshape(self.G * 32, -1)[: self.omega]

    def set_states(self, states: np.ndarray):
        """Pack uint8 [omega, n] node values into the bit-sliced layout."""
        torch = _torch()
        st = np.zeros((self.G * 32, self.network.n), dtype=np.uint64)
        st[: self.omega] = states
        st = st.reshape(self.G, 32, -1)
        w = (st << np.arange(32, dtype=np.uint64)[None, :, None]).sum(axis=1).astype(np.uint32)
        self.state.copy_(torch.from_numpy(w.view(np.int32)))

    def indicator_numpy(self, start: int, length: int, prop: int = 0) -> np.ndarray:
        """Indicator bits uint8 [omega, length] of property `prop` at positions
        start .. start+length-1."""
        col = start - int(self.c.bits_base)
        w = self.bits[prop * self.G:(prop + 1) * self.G, col:col + length].cpu().numpy().view(np.uint32)
        lanes = np.arange(32, dtype=np.uint32)
        b = ((w[:, None, :] >> lanes[None, :, None]) & 1).astype(np.uint8)  # [G, 32, len]
        return b.reshape(self.G * 32, length)[: self.omega]


STAGING = {"auto": 0, "smem": 1, "tiles": 2, "global": 3}
SCHEDULE = {"auto": 0, "fused": 1, "select_ahead": 2}


def _cfg(seed, mode, soi_arg, groups_per_block=0, threads_per_block=0, threads_per_item=0, blocks_per_round=0,
         staging="auto", schedule="auto", props_arg=None):
    return RunCfg(int(seed), int(mode), soi_arg.struct, int(groups_per_block), int(threads_per_block),
                  int(threads_per_item), int(blocks_per_round), STAGING[staging], SCHEDULE[schedule],
                  props_arg.count if props_arg else 0, props_arg.ptr if props_arg else None)


def pbn_balance_phases(G: int, R: int, gpb: int, T: int, threads: int, n: int, k: int):
    """The balanced split of one fused call (host arithmetic only): None for
    one launch, else two launches, each a list of two segments
    (CTAs, first group, groups, steps, step offset)."""
    out = (c_i32 * 20)()
    split = c_i32()
    _check(lib().pbn_balance_phases(int(G), int(R), int(gpb), int(T), int(threads), int(n), int(k), out,
                                    ctypes.byref(split)))
    if not split.value:
        return None
    v = list(out)
    return [[tuple(v[10 * l + 5 * q:10 * l + 5 * q + 5]) for q in range(2)] for l in range(2)]


def pbn_take_device_status() -> int:
    """Read and clear the device status word (0 or PBN_ERR_TIMEOUT)."""
    v = c_i32()
    _check(lib().pbn_take_device_status(ctypes.byref(v)))
    return v.value


def pbn_init_chains(chains: ChainSet, seed: int, mode: int = PER_NODE, stream=None):
    soi = SoiArg(None)
    cfg = _cfg(seed, mode, soi)
    _check(lib().pbn_init_chains(chains.network.handle, ctypes.byref(cfg), ctypes.byref(chains.c), _stream(stream)))


def pbn_run_chains(chains: ChainSet, steps: int, seed: int, mode: int = PER_NODE, soi=None,
                   groups_per_block: int = 0, threads_per_block: int = 0, threads_per_item: int = 0,
                   blocks_per_round: int = 0, staging: str = "auto", schedule: str = "auto", props=None,
                   stream=None):
    """Extend every chain by `steps` transitions, recording the indicator of
    `soi`, or of each of `props` (a list of states of interest, one bitstream
    each: chains.n_props must match)."""
    soi_arg = SoiArg(soi)
    props_arg = PropsArg(props) if props else None
    if props_arg and props_arg.count != chains.n_props:
        raise ValueError(f"{props_arg.count} properties for a chain set with {chains.n_props} bitstreams")
    cfg = _cfg(seed, mode, soi_arg, groups_per_block, threads_per_block, threads_per_item, blocks_per_round, staging,
               schedule, props_arg)
    _check(lib().pbn_run_chains(chains.network.handle, ctypes.byref(cfg), ctypes.byref(chains.c), int(steps),
                                _stream(stream)))


def _device_result(cls, call):
    torch = _torch()
    buf = torch.zeros(ctypes.sizeof(cls), dtype=torch.uint8, device="cuda")
    call(c_vp(buf.data_ptr()))
    host = buf.cpu().numpy().tobytes()
    return cls.from_buffer_copy(host)


def pbn_gelman_rubin(chains: ChainSet, start: int, psi: int, stream=None) -> dict:
    r = _device_result(GrResult, lambda p: _check(lib().pbn_gelman_rubin(
        ctypes.byref(chains.c), int(start), int(psi), p, _stream(stream))))
    out = _as_struct(GrResult, r)
    out["S2"] = (r.S2_hi << 64) | r.S2_lo
    return out


def pbn_two_state(chains: ChainSet, start: int, length: int, eps: float, r: float, s: float, stream=None) -> dict:
    res = _device_result(TwoStateResult, lambda p: _check(lib().pbn_two_state(
        ctypes.byref(chains.c), int(start), int(length), float(eps), float(r), float(s), p, _stream(stream))))
    return _as_struct(TwoStateResult, res)


def pbn_skart(chains: ChainSet, start: int, kappa: int, batches_per_chain: int, spacer: int, alpha_ci: float,
              alpha_ran: float = 0.20, stream=None) -> dict:
    res = _device_result(SkartResult, lambda p: _check(lib().pbn_skart(
        ctypes.byref(chains.c), int(start), int(kappa), int(batches_per_chain), int(spacer), float(alpha_ci),
        float(alpha_ran), p, _stream(stream))))
    return _as_struct(SkartResult, res)


def pbn_skart_static(chains: ChainSet, start: int, kappa: int, batches_per_chain: int, spacer: int,
                     alpha_ci: float, alpha_ran: float = 0.20, stream=None) -> dict:
    """pbn_skart for callers that cannot allocate device memory: the batch
    sums live in a fixed array inside the library (see include/pbn.h), so the
    call allocates nothing.  Calls that overlap on the GPU share that array
    and must be serialised by the caller."""
    res = _device_result(SkartResult, lambda p: _check(lib().pbn_skart_static(
        ctypes.byref(chains.c), int(start), int(kappa), int(batches_per_chain), int(spacer), float(alpha_ci),
        float(alpha_ran), p, _stream(stream))))
    return _as_struct(SkartResult, res)


def pbn_estimate_two_state(network: Network, soi, omega: int, seed: int, psi0: int = 1024, rhat: float = 1.05,
                           eps: float = 1e-10, r: float = 0.005, s: float = 0.95, mode: int = PER_NODE,
                           max_length: int = 1 << 26, stream=None) -> dict:
    """Alg. GR then Alg. 3 end to end; returns the report as a dict."""
    soi_arg = SoiArg(soi)
    q = TwoStateQuery(int(omega), int(psi0), float(rhat), float(eps), float(r), float(s), int(max_length), int(seed),
                      int(mode), soi_arg.struct)
    out = TwoStateReport()
    _check(lib().pbn_estimate_two_state(network.handle, ctypes.byref(q), ctypes.byref(out), _stream(stream)))
    return _as_struct(TwoStateReport, out)


def pbn_estimate_two_state_seq(network: Network, soi, seed: int, m0: int = 0, n0: int = 1024, eps: float = 1e-10,
                               r: float = 0.005, s: float = 0.95, mode: int = PER_NODE, max_length: int = 1 << 30,
                               stream=None) -> dict:
    """Alg. 1 (sequential two-state Markov chain approach) on chain 0 of the
    seed's family: the control run of the parallel method."""
    soi_arg = SoiArg(soi)
    q = TwoStateSeqQuery(int(m0), int(n0), float(eps), float(r), float(s), int(max_length), int(seed), int(mode),
                         soi_arg.struct)
    out = TwoStateSeqReport()
    _check(lib().pbn_estimate_two_state_seq(network.handle, ctypes.byref(q), ctypes.byref(out), _stream(stream)))
    return _as_struct(TwoStateSeqReport, out)


def pbn_estimate_two_state_multi(network: Network, sois, omega: int, seed: int, psi0: int = 1024, rhat: float = 1.05,
                                 eps: float = 1e-10, r: float = 0.005, s: float = 0.95, mode: int = PER_NODE,
                                 max_length: int = 1 << 26, stream=None) -> dict:
    """Several properties from the same trajectories (Sec. 4.2, last part);
    returns the common report with "properties": one dict per property."""
    props_arg = PropsArg(sois)
    q = TwoStateQuery(int(omega), int(psi0), float(rhat), float(eps), float(r), float(s), int(max_length), int(seed),
                      int(mode), SoiArg(None).struct)
    out = TwoStateReport()
    each = (PropertyResult * max(1, props_arg.count))()
    _check(lib().pbn_estimate_two_state_multi(network.handle, ctypes.byref(q), props_arg.count, props_arg.ptr,
                                              ctypes.byref(out), each, _stream(stream)))
    rep = _as_struct(TwoStateReport, out)
    rep["properties"] = [_as_struct(PropertyResult, each[m]) for m in range(props_arg.count)]
    return rep


def pbn_estimate_skart(network: Network, soi, omega: int, seed: int, H_star: float, relative: bool = True,
                       alpha: float = 0.05, psi0: int = 1024, rhat: float = 1.05, mode: int = PER_NODE,
                       max_length: int = 1 << 26, stream=None) -> dict:
    """Alg. GR then Alg. 4 end to end; returns the report as a dict."""
    soi_arg = SoiArg(soi)
    q = SkartQuery(int(omega), int(psi0), float(rhat), float(H_star), int(bool(relative)), float(alpha),
                   int(max_length), int(seed), int(mode), soi_arg.struct)
    out = SkartReport()
    _check(lib().pbn_estimate_skart(network.handle, ctypes.byref(q), ctypes.byref(out), _stream(stream)))
    return _as_struct(SkartReport, out)


def pbn_estimate_skart_seq(network: Network, soi, seed: int, H_star: float, relative: bool = True,
                           alpha: float = 0.05, mode: int = PER_NODE, max_length: int = 1 << 30,
                           stream=None) -> dict:
    """Alg. 2 (sequential Skart) on chain 0 of the seed's family."""
    soi_arg = SoiArg(soi)
    q = SkartQuery(1, 0, 0.0, float(H_star), int(bool(relative)), float(alpha), int(max_length), int(seed),
                   int(mode), soi_arg.struct)
    out = SkartReport()
    _check(lib().pbn_estimate_skart_seq(network.handle, ctypes.byref(q), ctypes.byref(out), _stream(stream)))
    return _as_struct(SkartReport, out)


# ------------------------------------------------------------------ engine

class Engine:
    """Batched / served queries (pbn_engine_* in include/pbn.h): queries of
    uneven size advance together, one persistent simulation launch and one
    batched statistics launch per epoch, admitted as slots and the
    device-memory budget allow."""

    def __init__(self, hbm_budget_bytes: int = 0, max_active: int = 0, steps_per_epoch: int = 0,
                 threads_per_block: int = 0, items_per_thread: int = 0, use_graph: bool = True,
                 epoch_target_ms: float = 0.0, stream=None):
        cfg = EngineCfg(int(hbm_budget_bytes), int(max_active), int(steps_per_epoch), int(threads_per_block),
                        int(items_per_thread), int(bool(use_graph)), float(epoch_target_ms))
        h = c_vp()
        _check(lib().pbn_engine_create(ctypes.byref(cfg), _stream(stream), ctypes.byref(h)))
        self.handle = h
        self._nets = {}

    def submit_two_state(self, network: Network, soi, omega: int, seed: int, psi0: int = 1024, rhat: float = 1.05,
                         eps: float = 1e-10, r: float = 0.005, s: float = 0.95, mode: int = PER_NODE,
                         max_length: int = 1 << 26, tag: int = 0) -> int:
        soi_arg = SoiArg(soi)
        q = EngineQuery()
        q.net = network.handle
        q.method = METHOD_TWO_STATE
        q.two_state = TwoStateQuery(int(omega), int(psi0), float(rhat), float(eps), float(r), float(s),
                                    int(max_length), int(seed), int(mode), soi_arg.struct)
        q.tag = int(tag)
        qid = c_i64()
        _check(lib().pbn_engine_submit(self.handle, ctypes.byref(q), ctypes.byref(qid)))
        self._nets[qid.value] = network
        return qid.value

    def submit_skart(self, network: Network, soi, omega: int, seed: int, H_star: float, relative: bool = True,
                     alpha: float = 0.05, psi0: int = 1024, rhat: float = 1.05, mode: int = PER_NODE,
                     max_length: int = 1 << 26, tag: int = 0) -> int:
        soi_arg = SoiArg(soi)
        q = EngineQuery()
        q.net = network.handle
        q.method = METHOD_SKART
        q.skart = SkartQuery(int(omega), int(psi0), float(rhat), float(H_star), int(bool(relative)), float(alpha),
                             int(max_length), int(seed), int(mode), soi_arg.struct)
        q.tag = int(tag)
        qid = c_i64()
        _check(lib().pbn_engine_submit(self.handle, ctypes.byref(q), ctypes.byref(qid)))
        self._nets[qid.value] = network
        return qid.value

    def step(self) -> dict:
        st = EngineStats()
        _check(lib().pbn_engine_step(self.handle, ctypes.byref(st)))
        return _as_struct(EngineStats, st)

    def poll(self, max_results: int = 256) -> list:
        buf = (EngineResult * max_results)()
        n = c_i32()
        _check(lib().pbn_engine_poll(self.handle, ctypes.cast(buf, c_vp), int(max_results), ctypes.byref(n)))
        out = []
        for k in range(n.value):
            r = buf[k]
            d = {"id": r.id, "tag": r.tag, "method": r.method, "status": r.status,
                 "submit_epoch": r.submit_epoch, "admit_epoch": r.admit_epoch, "finish_epoch": r.finish_epoch}
            d["report"] = _as_struct(TwoStateReport if r.method == METHOD_TWO_STATE else SkartReport,
                                     r.two_state if r.method == METHOD_TWO_STATE else r.skart)
            self._nets.pop(r.id, None)
            out.append(d)
        return out

    def cancel(self, qid: int) -> None:
        """Withdraw a waiting or active query; its result arrives with status
        PBN_ERR_CANCELLED."""
        _check(lib().pbn_engine_cancel(self.handle, int(qid)))

    def run(self, max_epochs: int = 1_000_000) -> list:
        """Step until nothing is active or waiting; returns all results."""
        results = []
        for _ in range(max_epochs):
            st = self.step()
            results += self.poll()
            if st["active"] == 0 and st["pending"] == 0:
                break
        return results

    def close(self):
        if getattr(self, "handle", None):
            lib().pbn_engine_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
