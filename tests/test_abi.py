"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
function that include/pbn.h declares (no compute calls here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.abspath(os.path.join(os.path.dirname(__file__), ".."))
HEADER = os.path.join(ROOT, "include", "pbn.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*(pbn_[a-z_0-9]+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("pbn_load", "pbn_free", "pbn_run_chains", "pbn_gelman_rubin", "pbn_two_state", "pbn_skart",
                     "pbn_init_chains", "pbn_estimate_two_state", "pbn_estimate_skart", "pbn_last_error"):
        assert required in names


def test_library_loads_and_exports_every_declared_symbol():
    from paper_1508_07828_gb300 import _build
    path = _build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings_and_error_channel():
    from paper_1508_07828_gb300 import _build
    lib = ctypes.CDLL(_build.build())
    lib.pbn_status_string.restype = ctypes.c_char_p
    lib.pbn_last_error.restype = ctypes.c_char_p
    assert lib.pbn_status_string(0) == b"ok"
    assert b"not converged" in lib.pbn_status_string(5)
    # NULL arguments are rejected on the host without touching the device
    assert lib.pbn_load(None, None) == 1
    assert b"NULL" in lib.pbn_last_error()
    assert lib.pbn_status_string(8) == b"cancelled"
    # cancelling on no engine is refused on the host
    lib.pbn_engine_cancel.argtypes = [ctypes.c_void_p, ctypes.c_int64]
    assert lib.pbn_engine_cancel(None, 3) == 1
    assert b"NULL" in lib.pbn_last_error()


STRUCTS = {
    "NetworkDesc": ("pbn_network_desc", ["n", "n_functions", "fn_offset", "par_offset", "parents", "truth_table",
                                         "select_prob", "p", "tt_offset", "tt_words"]),
    "NetInfo": ("pbn_net_info", ["n", "n_functions", "perturb_threshold", "table_bytes"]),
    "Soi": ("pbn_soi", ["size", "nodes", "values"]),
    "Chains": ("pbn_chains", ["omega", "state", "bits", "bits_cap", "bits_base", "length"]),
    "RunCfg": ("pbn_run_cfg", ["seed", "perturb_mode", "soi", "groups_per_block", "threads_per_block",
                               "threads_per_item", "blocks_per_round", "staging", "schedule", "n_props", "props"]),
    "GrResult": ("pbn_gr_result", ["rhat", "W", "B", "sigma2", "S1", "S2_lo", "S2_hi"]),
    "TwoStateResult": ("pbn_two_state_result", ["n00", "n01", "n10", "n11", "ones", "alpha", "beta", "prob", "M",
                                                "N", "status"]),
    "SkartResult": ("pbn_skart_result", ["mean", "var", "skew", "phi", "A", "H", "ci_lo", "ci_hi", "vn_stat",
                                         "vn_pass", "batches"]),
    "TwoStateQuery": ("pbn_two_state_query", ["omega", "psi0", "rhat_threshold", "eps", "r", "s", "max_length",
                                              "seed", "perturb_mode", "soi"]),
    "TwoStateReport": ("pbn_two_state_report", ["prob", "rhat", "alpha", "beta", "psi", "gr_psi", "length",
                                                "sample_size", "M", "N", "ones", "n4", "gr_rounds", "ts_rounds",
                                                "chain_node_updates", "device_ms", "sim_ms", "sim_launches",
                                                "kernel_launches", "sim_items", "d2h_bytes", "apply_ms",
                                                "apply_launches"]),
    "TwoStateSeqQuery": ("pbn_two_state_seq_query", ["m0", "n0", "eps", "r", "s", "max_length", "seed",
                                                     "perturb_mode", "soi"]),
    "TwoStateSeqReport": ("pbn_two_state_seq_report", ["prob", "alpha", "beta", "M", "N", "length", "ones", "n4",
                                                       "ab_window", "rounds", "chain_node_updates", "device_ms",
                                                       "sim_ms", "sim_launches", "kernel_launches", "d2h_bytes"]),
    "PropertyResult": ("pbn_property_result", ["prob", "alpha", "beta", "rhat", "M", "N", "ones", "n4"]),
    "SkartQuery": ("pbn_skart_query", ["omega", "psi0", "rhat_threshold", "H_star", "relative", "alpha",
                                       "max_length", "seed", "perturb_mode", "soi"]),
    "SkartReport": ("pbn_skart_report", ["mean", "ci_lo", "ci_hi", "H", "var", "skew", "phi", "rhat", "psi",
                                         "length", "kappa", "batches", "spacer", "sample_size", "gr_rounds",
                                         "rand_rounds", "ci_rounds", "chain_node_updates", "device_ms", "sim_ms",
                                         "sim_launches", "kernel_launches", "sim_items", "d2h_bytes", "apply_ms",
                                         "apply_launches"]),
    "EngineCfg": ("pbn_engine_cfg", ["hbm_budget_bytes", "max_active", "steps_per_epoch", "threads_per_block",
                                     "items_per_thread", "use_graph", "epoch_target_ms"]),
    "EngineQuery": ("pbn_engine_query", ["net", "method", "two_state", "skart", "tag"]),
    "EngineResult": ("pbn_engine_result", ["id", "tag", "method", "status", "two_state", "skart", "submit_epoch",
                                           "admit_epoch", "finish_epoch"]),
    "EngineStats": ("pbn_engine_stats", ["epoch", "active", "pending", "finished", "updates", "epoch_ms",
                                         "hbm_in_use", "steps_per_epoch", "threads_per_block", "items_per_thread",
                                         "kernel_launches", "sim_ms", "sim_items", "d2h_bytes", "tuning"]),
}


def test_binding_structs_match_the_c_layout(tmp_path):
    """Every ctypes mirror has the size and field offsets that a C compiler
    gives the structs of include/pbn.h."""
    import subprocess
    import paper_1508_07828_gb300 as P
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "pbn.h"', "int main(void) {"]
    for py, (cname, fields) in STRUCTS.items():
        lines.append(f'printf("{py} SIZEOF %zu\\n", sizeof({cname}));')
        for f in fields:
            lines.append(f'printf("{py} {f} %zu\\n", offsetof({cname}, {f}));')
    lines += ["return 0; }"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    out = subprocess.check_output([str(exe)], text=True).split("\n")
    for line in filter(None, out):
        py, field, value = line.split()
        cls = getattr(P, py)
        if field == "SIZEOF":
            assert ctypes.sizeof(cls) == int(value), (py, value)
        else:
            assert getattr(cls, field).offset == int(value), (py, field, value)
