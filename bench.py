#!/usr/bin/env python
"""Throughput of the parallel steady-state method on one GB300: batched
against plain.

One step = one pass of the batched workload: 64 independent PBNs (n
log-uniform in [50, 3000], 256-4096 chains log-uniform, 2 functions per node,
2-5 parents, p in {0.001, 0.01}), each a whole query of the hot path: chain
initialisation, the Gelman & Rubin burn-in (Alg. GR, R-hat < 1.05) and the
parallel two-state Markov chain approach (Alg. 3, r = 0.005, s = 0.95,
eps = 1e-10) up to the estimate.  The batched form runs all 64 queries in the
engine (one persistent simulation launch per epoch under a captured CUDA
graph, autotuned); the plain form runs the same 64 queries (same seeds, the
same chain-node updates) one network at a time through
pbn_estimate_two_state.  The metric is chain-node updates per second (the sum
of omega x chain length x n over the step's time) with the p50/p99 query
latency beside it; `value` is the batched form's, `plain` the loop's.

Timing: CUDA events on the current stream around every step (the engine and
the drivers synchronise their streams, so the events bracket the whole job),
W warm-up steps first (they also settle the engine's autotuner); L2 is
flushed (a 256 MB write) between timed steps, outside the events.  `e2e`
repeats the batched step through the C ABI with the 64 networks' CSR arrays
in pinned host memory, staged on the device inside the timed region, and the
results read back on the host.

--impl reference times the CPU oracle (single-threaded C) on bounded samples
of the same workload: all chains of all 64 networks for a fixed number of
transitions per step.  --mid measures the single mid-size query (n = 100,
1024 chains) instead; the default line carries it as `mid_query`.

Multi-GPU: the queries are independent, so N ranks run N replicas of the
workload (weak scaling); ranks only meet at the barriers and the final
max-over-ranks of the timed region.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "chain-node updates/s"
WORKLOAD = "mid-n100-omega1024-two-state-r0.005"
BATCH_WORKLOAD = "batched-64nets-n50-3000-omega256-4096-two-state-r0.005"
PSI0 = 1024


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--mid", action="store_true",
                    help="the single mid-size query (n = 100, 1024 chains) as the bench line")
    ap.add_argument("--mid-steps", type=int, default=40, help="mid-size queries timed for the default line's mid_query")
    ap.add_argument("--sim-only", choices=["mid", "large", "wide"], default=None,
                    help="time the simulation kernel alone on a workload (kernel benchmark / profiling case)")
    ap.add_argument("--sim-steps", type=int, default=1024, help="transitions per launch in --sim-only")
    ap.add_argument("--threads-per-item", type=int, default=0)
    ap.add_argument("--blocks-per-round", type=int, default=0)
    ap.add_argument("--groups-per-block", type=int, default=0)
    ap.add_argument("--staging", choices=["auto", "smem", "tiles", "global"], default="auto",
                    help="where the function table sits during a --sim-only launch")
    ap.add_argument("--schedule", choices=["auto", "fused", "select_ahead"], default="auto",
                    help="step schedule of a --sim-only launch")
    ap.add_argument("--batched", action="store_true",
                    help="64 networks of uneven size: the engine vs the plain one-query-at-a-time loop")
    ap.add_argument("--serve", action="store_true", help="Poisson arrivals over a pool of 200 networks")
    ap.add_argument("--skart-large", action="store_true",
                    help="Alg. GR + Alg. 4 (Skart) on the large network: n = 2000, 16384 chains, relative 0.01")
    ap.add_argument("--seq", action="store_true",
                    help="sequential Alg. 1 on one chain against the parallel query (speed-up, speed-up E)")
    ap.add_argument("--seq-runs", type=int, default=3, help="sequential/parallel pairs of --seq")
    ap.add_argument("--seq-r", type=float, default=1e-4,
                    help="precision r of the --seq comparison (the paper's experiments use 1e-4)")
    ap.add_argument("--sweep", action="store_true", help="the paper's n x density sweep at precision --seq-r")
    ap.add_argument("--sweep-omega", type=int, default=2048)
    ap.add_argument("--sweep-seq-max-n", type=int, default=100)
    ap.add_argument("--sweep-classes", default="sparse,in-between,dense", help="density classes of --sweep")
    ap.add_argument("--sweep-seq-classes", default="sparse",
                    help="classes whose smallest models also run the sequential Alg. 1 (minutes per model otherwise)")
    ap.add_argument("--multi", type=int, default=0,
                    help="Q properties from the same trajectories against Q separate queries (mid workload)")
    ap.add_argument("--rates", default="50,200,1000,2000", help="arrival rates (queries/s) for --serve")
    ap.add_argument("--queries", type=int, default=1000, help="queries per rate for --serve")
    ap.add_argument("--epoch-ms", type=float, default=6.0,
                    help="--serve: the engine's latency bound per epoch (pbn_engine_cfg.epoch_target_ms)")
    ap.add_argument("--max-length", type=int, default=1 << 20)
    return ap.parse_args()


def workload():
    import pbn_synth as S
    net, soi, cfg = S.mid_config()
    return net, soi, cfg


def config_dict(cfg, net):
    return {"workload": WORKLOAD, "nodes": int(net.n), "functions": int(net.n_functions), "chains": cfg["omega"],
            "p": net.p, "rhat_threshold": cfg["rhat"], "r": cfg["r"], "s": cfg["s"], "eps": cfg["eps"],
            "psi0": PSI0, "state_of_interest": "nodes 0-4 = (1,0,1,1,0)", "perturbation": "per-node",
            "l2": "flushed between timed steps (256 MB write)"}


# ------------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi every 50 ms from start() to stop(); only the samples taken
    between mark_begin() and mark_end() (the timed region) are summarised."""
    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None
        self.t0 = self.t1 = None

    def mark_begin(self):
        self.t0 = time.time()

    def mark_end(self):
        self.t1 = time.time()

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        import datetime
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 10:
                continue
            try:
                ts = datetime.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                rows.append((ts, float(parts[2]), float(parts[3]), parts[6:10]))
            except ValueError:
                continue
        os.unlink(self.path)
        inside = [r for r in rows if self.t0 is not None and self.t1 is not None and self.t0 <= r[0] <= self.t1]
        window = "timed region"
        if not inside and rows:  # region shorter than the sampling period: the nearest sample
            mid = 0.5 * ((self.t0 or rows[0][0]) + (self.t1 or rows[-1][0]))
            inside = [min(rows, key=lambda r: abs(r[0] - mid))]
            window = "nearest sample"
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in inside:
            for name, v in zip(names, r[3]):
                if v.lower() in ("active", "1", "yes"):
                    reasons.add(name)
        sm = [r[1] for r in inside]
        smax = [r[2] for r in inside]
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm), "window": window}


# -------------------------------------------------------------- roofline

def draw_ops_per_item(net) -> np.ndarray:
    """Integer operations of the category draw of one (node, chain group)
    item, per node, in expectation:
      Philox4x32-10 blocks: 40 ops each (10 rounds x (2 wide multiplies +
        2 three-input XORs)); blocks needed so that no lane of 32 is still tied
        with one of the node's L category bounds: 1 + sum_b>=1 of
        1 - (1 - min(1, L 2^-4b))^32;
      digit comparison: 3 ops per bound per digit (4 digits per block)."""
    ops = np.zeros(net.n)
    for i in range(net.n):
        L = len(list(net.functions_of(i)))
        blocks = 1.0 + sum(1.0 - (1.0 - min(1.0, L * 2.0 ** (-4 * b))) ** 32 for b in range(1, 8))
        ops[i] = blocks * (40 + 4 * 3 * L)
    return ops


def apply_ops_per_item(net) -> np.ndarray:
    """Integer operations of the state update of one item, per node, in
    expectation: for each function some lane selects (probability
    1 - (1 - c)^32) 2 ops per truth-table leaf, 1 per multiplexer and 1 load
    per parent (3 * 2^k - 1 + k); combine and store: 2 ops."""
    ops = np.full(net.n, 2.0)
    for i in range(net.n):
        for f in net.functions_of(i):
            k = int(net.par_offset[f + 1] - net.par_offset[f])
            c = float(net.select_prob[f])
            ops[i] += (1.0 - (1.0 - c) ** 32) * (3 * (1 << k) - 1 + k)
    return ops


def algorithmic_ops_per_item(net) -> np.ndarray:
    """Whole step: the draw plus the update (the fused kernel does both)."""
    return draw_ops_per_item(net) + apply_ops_per_item(net)


def alu_peak_tops(device_index):
    """Issue-rate peak: SMs x 4 schedulers x 32 lanes x max SM clock."""
    import torch
    sms = torch.cuda.get_device_properties(device_index).multi_processor_count
    mhz = None
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        mhz = float(peaks.get("sm_max_mhz"))
    except Exception:
        pass
    src = "MEASURED_PEAKS.json sm_max_mhz"
    if not mhz:
        try:
            out = subprocess.check_output(["nvidia-smi", f"--id={device_index}", "--query-gpu=clocks.max.sm",
                                           "--format=csv,noheader,nounits"], text=True)
            mhz = float(out.strip().splitlines()[0]); src = "nvidia-smi clocks.max.sm"
        except Exception:
            mhz = 2070.0; src = "nominal 2070 MHz"
    return sms * 4 * 32 * mhz * 1e6 / 1e12, sms, mhz, src


# ------------------------------------------------------------- CPU oracle

def oracle_sample(net, soi, omega, target_s=12.0):
    """Times the oracle simulating all `omega` chains of the workload network
    for a number of transitions calibrated to about target_s seconds."""
    import oracle
    oracle.build()
    st = oracle.init_states(net, 99, omega)
    t = time.perf_counter()
    oracle.simulate(net, 0, 99, st, 0, 2, soi)
    per_step = (time.perf_counter() - t) / 2
    steps = max(2, int(target_s / max(per_step, 1e-6)))
    t = time.perf_counter()
    oracle.simulate(net, 0, 99, st, 2, steps, soi)
    dt = time.perf_counter() - t
    upd = omega * steps * net.n
    return upd / dt, steps, dt


def _oracle_worker(job):
    """One host process of oracle_all_cores: its share of the chains for a
    fixed number of transitions; returns the seconds the simulation took."""
    net, omega_w, steps, soi = job
    import oracle
    st = oracle.init_states(net, 99, omega_w)
    t = time.perf_counter()
    oracle.simulate(net, 0, 99, st, 0, steps, soi)
    return time.perf_counter() - t


def oracle_all_cores(net, soi, omega, rate_one_core, target_s=8.0):
    """The same oracle on every host core at once: the chains split over
    os.cpu_count() processes (spawned, so none inherits a CUDA context), each
    simulating its share for a number of transitions sized to about target_s
    seconds at the one-core rate.  Throughput = all updates / slowest share."""
    import multiprocessing as mp
    cores = os.cpu_count() or 1
    omega_w = max(1, omega // cores)
    steps = max(2, int(target_s * rate_one_core / (omega_w * net.n)))
    with mp.get_context("spawn").Pool(cores) as pool:
        times = pool.map(_oracle_worker, [(net, omega_w, steps, soi)] * cores)
    upd = cores * omega_w * steps * net.n
    return upd / max(times), cores, steps, omega_w, max(times)


# ------------------------------------------------------------------- arms

def reduce_over_ranks(slowest, summed, world, device):
    """Whole-job figures of N replicas: the timed durations as their maximum
    over the ranks (the job ends with its slowest replica), the units of work
    as their sum.  One rank: the values themselves."""
    slowest = [float(x) for x in slowest]
    summed = [float(x) for x in summed]
    if world <= 1:
        return slowest, summed
    import torch
    import torch.distributed as dist
    t = torch.tensor(slowest, dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    u = torch.tensor(summed, dtype=torch.float64, device=device)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return [float(x) for x in t], [float(x) for x in u]


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def run_reference(args):
    """The oracle (single-threaded C) on bounded samples of the batched
    workload: each step advances all chains of all 64 networks by T
    transitions, T sized so that the whole run takes about two minutes."""
    world, rank, local = dist_setup()
    if rank != 0:
        return
    import oracle
    oracle.build()
    cfgs = batch_workload()
    per_step_s = min(4.0, 120.0 / max(args.steps + args.warmup, 1))
    rate, _, _ = oracle_batch_sample(cfgs, target_s=1.0)
    work = sum(net.n * c["omega"] for net, _, c in cfgs)
    T = max(1, int(per_step_s * rate / work))
    states = [oracle.init_states(net, 7, c["omega"]) for net, _, c in cfgs]
    t0 = 0

    def step():
        nonlocal t0
        for i, (net, soi, c) in enumerate(cfgs):
            states[i], _ = oracle.simulate(net, 0, 7, states[i], t0, T, soi)
        t0 += T

    for _ in range(args.warmup):
        step()
    times = []
    for _ in range(args.steps):
        t = time.perf_counter()
        step()
        times.append(time.perf_counter() - t)
    upd = work * T
    value = upd * len(times) / sum(times)
    sample = f"oracle simulation of all chains of all {len(cfgs)} networks for {T} transitions per step"
    line = {"metric": METRIC, "value": value, "unit": "updates/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
            "config": batch_config_dict(cfgs), "impl": "reference",
            "cpu_baseline": {"value": value, "unit": "updates/s", "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def run_mid(args):
    """The mid-size query as the bench line (--mid): n = 100, 1024 chains,
    Alg. GR + Alg. 3 at r = 0.005, one query per step."""
    import torch
    world, rank, local = dist_setup()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", init_method="env://")
    from paper_1508_07828_gb300 import _build
    _build.build()
    import paper_1508_07828_gb300 as P

    net, soi, cfg = workload()
    omega = cfg["omega"]
    N = P.pbn_load(net)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    q = dict(omega=omega, psi0=PSI0, rhat=cfg["rhat"], eps=cfg["eps"], r=cfg["r"], s=cfg["s"])
    seed0 = 1_000_000 * (rank + 1)

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    clocks = ClockSampler(local)
    clocks.start()  # sampling runs before the timed region begins
    for w in range(args.warmup):
        P.pbn_estimate_two_state(N, soi, seed=seed0 + 900_000 + w, **q)
    barrier()
    clocks.mark_begin()
    times, reports = [], []
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for k in range(args.steps):
        flush.zero_()
        ev0.record(stream)
        rep = P.pbn_estimate_two_state(N, soi, seed=seed0 + k, **q)
        ev1.record(stream)
        ev1.synchronize()
        times.append(ev0.elapsed_time(ev1))
        reports.append(rep)
    barrier()
    clocks.mark_end()
    clk = clocks.stop()

    # e2e: host CSR arrays in pinned memory -> pbn_load -> query -> result on the host
    host = {k: torch.from_numpy(np.ascontiguousarray(getattr(net, k))).pin_memory()
            for k in ("fn_offset", "par_offset", "parents", "truth_table", "select_prob")}
    h2d = int(sum(v.numel() * v.element_size() for v in host.values()))
    e2e_times, e2e_upd, e2e_d2h = [], 0, 0
    barrier()
    for k in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t = time.perf_counter()
        Nk = P.pbn_load_pinned(host, net.n, net.p)
        rep = P.pbn_estimate_two_state(Nk, soi, seed=seed0 + k, **q)
        torch.cuda.synchronize()
        e2e_times.append(time.perf_counter() - t)
        Nk.close()
        e2e_upd += rep["chain_node_updates"]
        e2e_d2h += rep["d2h_bytes"]
    barrier()

    total_ms = sum(times)
    upd = sum(r["chain_node_updates"] for r in reports)
    e2e_s = sum(e2e_times)
    (total_ms, e2e_s), (upd_all, e2e_upd_all) = reduce_over_ranks([total_ms, e2e_s], [upd, e2e_upd], world, "cuda")
    if rank != 0:
        return

    value = upd_all / (total_ms / 1e3)
    # roofline of the dominant simulation kernel: algorithmic integer ops per
    # launch over its event-timed launch durations in the timed region.  The
    # select-ahead schedule (chosen for this chain count) splits a step into
    # select_kernel (category draws) and apply_kernel (state updates, the
    # longer of the two); the fused schedule runs sim_kernel alone.
    sim_ms = sum(r["sim_ms"] for r in reports)
    sim_launches = sum(r["sim_launches"] for r in reports)
    apply_ms = sum(r["apply_ms"] for r in reports)
    apply_launches = sum(r["apply_launches"] for r in reports)
    items = sum(r["sim_items"] for r in reports)
    groups_steps = items / net.n
    peak, sms, mhz, peak_src = alu_peak_tops(local)
    if apply_launches:
        kernel, k_ms, k_launches = "apply_resident_kernel", apply_ms, apply_launches
        ops_per_group_step = float(apply_ops_per_item(net).sum())
        other = {"select_kernel": {"achieved": float(draw_ops_per_item(net).sum()) * groups_steps /
                                   ((sim_ms - apply_ms) / 1e3) / 1e12, "ms": sim_ms - apply_ms,
                                   "launches": sim_launches - apply_launches}}
    else:
        kernel, k_ms, k_launches = "sim_kernel", sim_ms, sim_launches
        ops_per_group_step = float(algorithmic_ops_per_item(net).sum())
        other = {}
    achieved = ops_per_group_step * groups_steps / (k_ms / 1e3) / 1e12
    # DRAM bytes per launch of the dominant kernel, from the ncu capture of
    # apply_resident_kernel on this workload (256 steps x 32 groups: 6599680
    # bytes read, 0 written; cold caches, as ncu replays a launch): 806 bytes
    # per (group, step), the category words, scaled to the average launch
    traffic = None
    if apply_launches:
        traffic = 6599680.0 / (256 * 32) * groups_steps / max(apply_launches, 1)
    lat = sorted(times)
    line = {"metric": METRIC, "value": value, "unit": "updates/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": config_dict(cfg, net),
            "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                           "mean": float(np.mean(lat))},
            "queries_per_s": args.steps * world / (total_ms / 1e3),
            "roofline": {"bound": "alu", "kernel": kernel, "achieved": achieved, "peak": peak,
                         "unit": "Tops/s", "frac": achieved / peak, "traffic": traffic,
                         "peak_source": f"issue rate {sms} SMs x 128 lanes x {mhz:.0f} MHz ({peak_src})",
                         "kernel_share_of_step": k_ms / total_ms, "sim_share_of_step": sim_ms / total_ms,
                         "ops_per_update": ops_per_group_step / net.n / 32,
                         "launches": k_launches, "avg_launch_ms": k_ms / max(k_launches, 1),
                         "ns_per_transition": 1e6 * sim_ms / max(groups_steps / ((omega + 31) // 32), 1),
                         "other_kernels": other},
            "clocks": clk,
            "e2e": {"value": e2e_upd_all / e2e_s, "unit": "updates/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": e2e_d2h // max(args.steps, 1)},
            "gpu_launches": int(sum(r["kernel_launches"] for r in reports)),
            "query": {"mean_length": float(np.mean([r["length"] for r in reports])),
                      "mean_sample_size": float(np.mean([r["sample_size"] for r in reports])),
                      "mean_prob": float(np.mean([r["prob"] for r in reports]))}}
    if world == 1 and not args.no_cpu_baseline:
        v, steps, dt = oracle_sample(net, soi, omega)
        line["cpu_baseline"] = {"value": v, "unit": "updates/s", "cores": 1, "kind": "oracle",
                                "sample": f"oracle simulation of all {omega} chains for {steps} transitions "
                                          f"({dt:.1f} s)"}
        va, cores, steps_a, omega_w, dta = oracle_all_cores(net, soi, omega, v)
        line["cpu_baseline_all_cores"] = {"value": va, "unit": "updates/s", "cores": cores, "kind": "oracle",
                                          "sample": f"{cores} processes, {omega_w} chains each, {steps_a} "
                                                    f"transitions ({dta:.1f} s)"}
    print(json.dumps(line))


def batch_workload():
    import pbn_synth as S
    return S.batch_configs()


def batch_config_dict(cfgs):
    ns = [int(net.n) for net, _, _ in cfgs]
    oms = [int(c["omega"]) for _, _, c in cfgs]
    return {"workload": BATCH_WORKLOAD, "networks": len(cfgs), "nodes": f"log-uniform [50, 3000] ({min(ns)}-{max(ns)})",
            "chains": f"log-uniform [256, 4096] ({min(oms)}-{max(oms)})", "functions_per_node": 2,
            "parents": "2-5", "p": "0.001 or 0.01", "rhat_threshold": 1.05, "r": 0.005, "s": 0.95, "eps": 1e-10,
            "psi0": PSI0, "state_of_interest": "5 random nodes and values per network", "perturbation": "per-node",
            "total_nodes": int(sum(ns)), "total_chains": int(sum(oms)),
            "l2": "flushed between timed steps (256 MB write)"}


def _batch_kw(c, seed, max_length):
    return dict(omega=c["omega"], seed=seed, psi0=PSI0, rhat=c["rhat"], eps=c["eps"], r=c["r"], s=c["s"],
                max_length=max_length)


def oracle_batch_sample(cfgs, target_s=12.0):
    """Times the oracle on a bounded sample of the batched workload: all
    chains of all 64 networks advanced by T transitions each, T calibrated to
    about target_s seconds.  Returns (updates/s, T, seconds)."""
    import oracle
    oracle.build()
    states = [oracle.init_states(net, 99, c["omega"]) for net, _, c in cfgs]
    t = time.perf_counter()
    for (net, soi, c), st in zip(cfgs, states):
        oracle.simulate(net, 0, 99, st, 0, 1, soi)
    per = time.perf_counter() - t
    T = max(1, int(round(target_s / max(per, 1e-6))))
    t = time.perf_counter()
    upd = 0
    for (net, soi, c), st in zip(cfgs, states):
        oracle.simulate(net, 0, 99, st, 1, T, soi)
        upd += c["omega"] * T * net.n
    dt = time.perf_counter() - t
    return upd / dt, T, dt


def _oracle_batch_worker(job):
    """One host process of oracle_batch_all_cores: its networks' chains for T
    transitions; returns (updates, seconds)."""
    items, T = job
    import oracle
    t = time.perf_counter()
    upd = 0
    for net, soi, omega in items:
        st = oracle.init_states(net, 99, omega)
        oracle.simulate(net, 0, 99, st, 0, T, soi)
        upd += omega * T * net.n
    return upd, time.perf_counter() - t


def oracle_batch_all_cores(cfgs, rate_one_core, target_s=8.0):
    """The same oracle on every host core at once: the 64 networks dealt
    over os.cpu_count() spawned processes (largest first, to the least
    loaded), T transitions each, sized to about target_s seconds.
    Throughput = all updates / the slowest process."""
    import multiprocessing as mp
    cores = os.cpu_count() or 1
    work = sorted(((net.n * c["omega"], net, soi, c["omega"]) for net, soi, c in cfgs), key=lambda x: -x[0])
    total = sum(w for w, *_ in work)
    T = max(1, int(target_s * rate_one_core * cores / max(total, 1)))
    bins = [[] for _ in range(cores)]
    load = [0] * cores
    for w, net, soi, om in work:
        k = int(np.argmin(load))
        bins[k].append((net, soi, om))
        load[k] += w
    jobs = [(b, T) for b in bins if b]
    with mp.get_context("spawn").Pool(len(jobs)) as pool:
        res = pool.map(_oracle_batch_worker, jobs)
    upd = sum(u for u, _ in res)
    slowest = max(t for _, t in res)
    return upd / slowest, len(jobs), T, slowest


def measure_mid(P, torch, steps, warmup, seed0, flush):
    """The mid-size query (n = 100, 1024 chains, two-state r = 0.005), one
    query per step, CUDA events around each: throughput and latency."""
    net, soi, cfg = workload()
    N = P.pbn_load(net)
    q = dict(omega=cfg["omega"], psi0=PSI0, rhat=cfg["rhat"], eps=cfg["eps"], r=cfg["r"], s=cfg["s"])
    stream = torch.cuda.current_stream()
    for w in range(warmup):
        P.pbn_estimate_two_state(N, soi, seed=seed0 + 900_000 + w, **q)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    times, upd, apply_ms, apply_launches, items = [], 0, 0.0, 0, 0
    for k in range(steps):
        flush.zero_()
        ev0.record(stream)
        rep = P.pbn_estimate_two_state(N, soi, seed=seed0 + k, **q)
        ev1.record(stream)
        ev1.synchronize()
        times.append(ev0.elapsed_time(ev1))
        upd += rep["chain_node_updates"]
        apply_ms += rep["apply_ms"]
        apply_launches += rep["apply_launches"]
        items += rep["sim_items"]
    N.close()
    out = {"workload": WORKLOAD, "value": upd / (sum(times) / 1e3), "unit": "updates/s", "steps": steps,
           "latency_ms": _percentiles(times)}
    if apply_launches:
        ops = float(apply_ops_per_item(net).sum()) * items / net.n
        out["apply_resident_kernel_tops"] = ops / (apply_ms / 1e3) / 1e12
    return out


def run_ours(args):
    """The default line: the batched workload, engine against the plain loop."""
    import torch
    world, rank, local = dist_setup()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", init_method="env://")
    from paper_1508_07828_gb300 import _build
    _build.build()
    import paper_1508_07828_gb300 as P

    cfgs = batch_workload()
    nets = [P.pbn_load(net) for net, _, _ in cfgs]
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    seed_base = 1_000_000 * (rank + 1)
    seed_of = lambda step, k: seed_base + 1000 * step + k
    ml = args.max_length

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    eng = P.Engine(use_graph=True)

    def batched_step(step, networks=None):
        """All 64 queries through the engine; returns (updates, per-query
        latencies in ms, engine stats summed, reports by tag)."""
        networks = networks or nets
        t0 = time.perf_counter()
        for k, ((net, soi, c), N) in enumerate(zip(cfgs, networks)):
            eng.submit_two_state(N, soi, tag=k, **_batch_kw(c, seed_of(step, k), ml))
        agg = {"epochs": 0, "sim_ms": 0.0, "sim_items": 0, "launches": 0, "d2h": 0, "epoch_ms": 0.0}
        lat, reps = [], {}
        while True:
            st = eng.step()
            agg["epochs"] += 1
            agg["sim_ms"] += st["sim_ms"]
            agg["sim_items"] += st["sim_items"]
            agg["launches"] += st["kernel_launches"]
            agg["d2h"] += st["d2h_bytes"]
            agg["epoch_ms"] += st["epoch_ms"]
            for r in eng.poll():
                lat.append(1e3 * (time.perf_counter() - t0))
                reps[r["tag"]] = r
            if st["active"] == 0 and st["pending"] == 0:
                break
        bad = [k for k, r in reps.items() if r["status"] != 0]
        if bad or len(reps) != len(cfgs):
            raise RuntimeError(f"batched step {step}: queries {bad} failed or missing")
        upd = sum(r["report"]["chain_node_updates"] for r in reps.values())
        return upd, lat, agg, reps, st

    def plain_step(step):
        t0 = time.perf_counter()
        lat, upd, launches = [], 0, 0
        for k, ((net, soi, c), N) in enumerate(zip(cfgs, nets)):
            r = P.pbn_estimate_two_state(N, soi, **_batch_kw(c, seed_of(step, k), ml))
            upd += r["chain_node_updates"]
            launches += r["kernel_launches"]
            lat.append(1e3 * (time.perf_counter() - t0))
        return upd, lat, launches

    def timed(fn, *a):
        flush.zero_()
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        out = fn(*a)
        ev1.record(stream)
        ev1.synchronize()
        return ev0.elapsed_time(ev1), out

    clocks = ClockSampler(local)
    clocks.start()  # sampling runs before the timed region begins
    for w in range(args.warmup):
        batched_step(10_000 + w)
        plain_step(10_000 + w)
    # the engine's autotuner times one live epoch per candidate; the timed
    # steps start once it has chosen
    for w in range(64):
        if not batched_step(20_000 + w)[4]["tuning"]:
            break
    barrier()
    clocks.mark_begin()
    b_ms, b_upd, b_lat, b_launch = [], 0, [], 0
    sim_ms, ops, sim_items, epochs, epoch_ms = 0.0, 0.0, 0, 0, 0.0
    ops_per_item = [float(algorithmic_ops_per_item(net).sum()) / net.n for net, _, _ in cfgs]
    for k in range(args.steps):
        ms, (upd, lat, agg, reps, st) = timed(batched_step, k)
        b_ms.append(ms)
        b_upd += upd
        b_lat += lat
        b_launch += agg["launches"]
        sim_ms += agg["sim_ms"]
        sim_items += agg["sim_items"]
        epochs += agg["epochs"]
        epoch_ms += agg["epoch_ms"]
        ops += sum(ops_per_item[t] * r["report"]["sim_items"] for t, r in reps.items())
    tuned = {key: st[key] for key in ("steps_per_epoch", "threads_per_block", "items_per_thread")}
    p_ms, p_upd, p_lat, p_launch = [], 0, [], 0
    for k in range(args.steps):
        ms, (upd, lat, launches) = timed(plain_step, k)
        p_ms.append(ms)
        p_upd += upd
        p_lat += lat
        p_launch += launches
    barrier()
    clocks.mark_end()
    clk = clocks.stop()

    # e2e: the 64 networks' CSR arrays in pinned host memory, staged on the
    # device inside the timed region; results read on the host
    host = []
    h2d = 0
    for net, _, _ in cfgs:
        arr = {key: torch.from_numpy(np.ascontiguousarray(getattr(net, key))).pin_memory()
               for key in ("fn_offset", "par_offset", "parents", "truth_table", "select_prob")}
        h2d += int(sum(v.numel() * v.element_size() for v in arr.values()))
        host.append((arr, net.n, net.p))
    e2e_s, e2e_upd, e2e_d2h = 0.0, 0, 0
    barrier()
    for k in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t = time.perf_counter()
        staged = [P.pbn_load_pinned(a, n, pp) for a, n, pp in host]
        upd, lat, agg, reps, _ = batched_step(k, staged)
        torch.cuda.synchronize()
        e2e_s += time.perf_counter() - t
        e2e_upd += upd
        e2e_d2h += agg["d2h"]
        for Nk in staged:
            Nk.close()
    barrier()
    eng.close()

    total_ms, plain_ms = sum(b_ms), sum(p_ms)
    (total_ms, plain_ms, e2e_s), (upd_all, p_upd_all, e2e_upd_all) = reduce_over_ranks(
        [total_ms, plain_ms, e2e_s], [b_upd, p_upd, e2e_upd], world, "cuda")
    if rank != 0:
        return
    value = upd_all / (total_ms / 1e3)
    plain_value = p_upd_all / (plain_ms / 1e3)
    peak, sms, mhz, peak_src = alu_peak_tops(local)
    achieved = ops / (sim_ms / 1e3) / 1e12 if sim_ms > 0 else None
    line = {"metric": METRIC, "value": value, "unit": "updates/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": batch_config_dict(cfgs),
            "latency_ms": _percentiles(b_lat),
            "queries_per_s": len(cfgs) * args.steps * world / (total_ms / 1e3),
            "plain": {"value": plain_value, "unit": "updates/s", "ms_per_step": plain_ms / args.steps,
                      "latency_ms": _percentiles(p_lat),
                      "queries_per_s": len(cfgs) * args.steps * world / (plain_ms / 1e3),
                      "form": "one pbn_estimate_two_state per network, in order", "gpu_launches": p_launch},
            "speedup_vs_plain": value / plain_value, "same_updates": b_upd == p_upd,
            "engine": {"epochs_per_step": epochs / args.steps, "tuned": tuned,
                       "device_ms_per_step": epoch_ms / args.steps},
            "roofline": {"bound": "alu", "kernel": "batch_sim_kernel", "achieved": achieved, "peak": peak,
                         "unit": "Tops/s", "frac": (achieved / peak) if achieved else None, "traffic": None,
                         "peak_source": f"issue rate {sms} SMs x 128 lanes x {mhz:.0f} MHz ({peak_src})",
                         "kernel_share_of_step": sim_ms / total_ms,
                         "launches": epochs, "avg_launch_ms": sim_ms / max(epochs, 1),
                         "ops_per_update": ops / max(sim_items, 1) / 32,
                         "items_per_launch": sim_items / max(epochs, 1)},
            "clocks": clk,
            "e2e": {"value": e2e_upd_all / e2e_s, "unit": "updates/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": e2e_d2h // max(args.steps, 1)},
            "gpu_launches": int(b_launch)}
    if world == 1:
        line["mid_query"] = measure_mid(P, torch, args.mid_steps, 3, 5_000_000, flush)
    if world == 1 and not args.no_cpu_baseline:
        v, T, dt = oracle_batch_sample(cfgs)
        line["cpu_baseline"] = {"value": v, "unit": "updates/s", "cores": 1, "kind": "oracle",
                                "sample": f"oracle simulation of all chains of all {len(cfgs)} networks for {T} "
                                          f"transitions ({dt:.1f} s)"}
        va, procs, Ta, dta = oracle_batch_all_cores(cfgs, v)
        line["cpu_baseline_all_cores"] = {"value": va, "unit": "updates/s", "cores": procs, "kind": "oracle",
                                          "sample": f"{procs} processes, the networks dealt between them, {Ta} "
                                                    f"transitions each ({dta:.1f} s)"}
    print(json.dumps(line))


def run_sim_only(args):
    """The simulation kernel alone: omega chains advanced by --sim-steps
    transitions per launch, CUDA events around each launch."""
    import torch
    import pbn_synth as S
    from paper_1508_07828_gb300 import _build
    _build.build()
    import paper_1508_07828_gb300 as P
    torch.cuda.set_device(0)
    if args.sim_only == "mid":
        net, soi, cfg = workload()
        omega = cfg["omega"]
    else:
        net, nodes, cfg = S.large_config() if args.sim_only == "large" else S.wide_config()
        soi = S.StateOfInterest(nodes, np.ones(len(nodes), dtype=np.uint8))
        omega = cfg["omega"]
    N = P.pbn_load(net)
    steps = args.sim_steps
    cs = P.ChainSet(N, omega, bits_cap=steps)
    P.pbn_init_chains(cs, 5)
    launch = dict(threads_per_item=args.threads_per_item, blocks_per_round=args.blocks_per_round,
                  groups_per_block=args.groups_per_block, staging=args.staging, schedule=args.schedule)
    stream = torch.cuda.current_stream()

    def one():
        cs.c.bits_base = cs.c.length
        P.pbn_run_chains(cs, steps, 5, P.PER_NODE, soi, **launch)

    for _ in range(args.warmup):
        one()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for a, b in ev:
        a.record(stream)
        one()
        b.record(stream)
    torch.cuda.synchronize()
    ms = [a.elapsed_time(b) for a, b in ev]
    upd = omega * steps * net.n
    ops = algorithmic_ops_per_item(net).sum() * ((omega + 31) // 32) * steps
    peak, sms, mhz, src = alu_peak_tops(0)
    achieved = ops / (np.mean(ms) / 1e3) / 1e12
    print(json.dumps({"mode": "sim-only", "workload": args.sim_only, "nodes": int(net.n), "chains": omega,
                      "functions": int(net.n_functions), "table_bytes": 16 * int(net.n_functions),
                      "steps_per_launch": steps, "launches": args.steps, "ms_per_launch": float(np.mean(ms)),
                      "ms_min": float(np.min(ms)), "updates_per_s": upd / (np.mean(ms) / 1e3),
                      "ns_per_transition": 1e6 * float(np.mean(ms)) / steps,
                      "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tops/s",
                                   "frac": achieved / peak},
                      "launch": launch}))


def run_skart_large(args):
    """The large workload end to end: n = 2000 scale-free network, 16384
    chains, Gelman & Rubin (R-hat < 1.05) then Skart at relative precision
    0.01 on nodes 0..9.  Their target values are chain 0's state after 1024
    transitions of the GPU path itself, so the pattern has mass."""
    import torch
    import pbn_synth as S
    from paper_1508_07828_gb300 import _build
    _build.build()
    import paper_1508_07828_gb300 as P
    torch.cuda.set_device(0)
    net, nodes, cfg = S.large_config()
    N = P.pbn_load(net)
    cs = P.ChainSet(N, 32, bits_cap=1)
    P.pbn_init_chains(cs, 5)
    P.pbn_run_chains(cs, 1024, 5, P.PER_NODE, None)
    soi = S.StateOfInterest(nodes, cs.states_numpy()[0][nodes])
    kw = dict(omega=cfg["omega"], H_star=cfg["rel"], relative=True, alpha=cfg["alpha"], psi0=PSI0, rhat=cfg["rhat"])
    P.pbn_estimate_skart(N, soi, seed=1, **kw)  # warm-up
    rows = []
    for k in range(max(1, min(args.steps, 5))):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = P.pbn_estimate_skart(N, soi, seed=10 + k, **kw)
        dt = time.perf_counter() - t0
        rows.append(dict(seconds=dt, updates_per_s=r["chain_node_updates"] / dt, length=r["length"],
                         psi=r["psi"], sample_size=r["sample_size"], batches=r["batches"], kappa=r["kappa"],
                         mean=r["mean"], ci=[r["ci_lo"], r["ci_hi"]], H=r["H"], sim_share=r["sim_ms"] / r["device_ms"]))
    print(json.dumps({"mode": "skart-large", "workload": "large-n2000-omega16384-skart-rel0.01",
                      "functions": int(net.n_functions), "runs": rows,
                      "median_seconds": float(np.median([x["seconds"] for x in rows])),
                      "median_updates_per_s": float(np.median([x["updates_per_s"] for x in rows]))}))


def _percentiles(x):
    x = np.asarray(x, dtype=np.float64)
    return {"p50": float(np.percentile(x, 50)), "p99": float(np.percentile(x, 99)), "mean": float(x.mean())}


def run_batched(args):
    """64 independent networks (n log-uniform in [50, 3000], 256-4096
    chains, p in {0.001, 0.01}, two-state at r = 0.005): the engine (one
    persistent launch per epoch, CUDA graph, autotuned) against the plain
    loop of one pbn_estimate_two_state per network, same seeds."""
    import torch
    import pbn_synth as S
    from paper_1508_07828_gb300 import _build
    _build.build()
    import paper_1508_07828_gb300 as P
    torch.cuda.set_device(0)
    cfgs = S.batch_configs()
    nets = [P.pbn_load(net) for net, _, _ in cfgs]
    kw = lambda c, k: dict(omega=c["omega"], seed=1000 + k, psi0=PSI0, rhat=c["rhat"], eps=c["eps"], r=c["r"],
                           s=c["s"], max_length=args.max_length)

    def plain():
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        lat, upd, ok = [], 0, 0
        for k, ((net, soi, c), N) in enumerate(zip(cfgs, nets)):
            try:
                r = P.pbn_estimate_two_state(N, soi, **kw(c, k))
                upd += r["chain_node_updates"]
                ok += 1
            except P.PbnError:
                pass
            lat.append(time.perf_counter() - t0)
        return time.perf_counter() - t0, upd, ok, lat

    def batched():
        eng = P.Engine(use_graph=True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k, ((net, soi, c), N) in enumerate(zip(cfgs, nets)):
            eng.submit_two_state(N, soi, tag=k, **kw(c, k))
        upd, ok, lat, epochs, ms = 0, 0, [], 0, 0.0
        while True:
            st = eng.step()
            epochs += 1
            ms += st["epoch_ms"]
            for r in eng.poll():
                lat.append(time.perf_counter() - t0)
                upd += r["report"]["chain_node_updates"]
                ok += r["status"] == 0
            if st["active"] == 0 and st["pending"] == 0:
                break
        wall = time.perf_counter() - t0
        eng.close()
        return wall, upd, ok, lat, epochs, st

    # warm-up runs let the engine's autotuner settle (its choice persists
    # for later engines of the process)
    for _ in range(max(1, args.warmup)):
        batched()
    plain()
    pw, pu, pok, plat = plain()
    bw, bu, bok, blat, epochs, st = batched()
    print(json.dumps({"mode": "batched", "networks": len(cfgs), "config": "64 nets, n log-uniform [50,3000], "
                      "chains log-uniform [256,4096], p in {0.001,0.01}, two-state r=0.005",
                      "plain": {"seconds": pw, "updates_per_s": pu / pw, "queries_ok": pok,
                                "latency_s": _percentiles(plat)},
                      "batched": {"seconds": bw, "updates_per_s": bu / bw, "queries_ok": bok, "epochs": epochs,
                                  "latency_s": _percentiles(blat),
                                  "tuned": {k: st[k] for k in ("steps_per_epoch", "threads_per_block",
                                                               "items_per_thread")}},
                      "speedup": pw / bw, "same_updates": pu == bu}))


def run_multi(args):
    """Several properties from the same trajectories (Sec. 4.2, last part) on
    the mid-size workload: one pbn_estimate_two_state_multi against the loop
    of one pbn_estimate_two_state per property, same seeds, wall time with
    the device synchronised on both sides."""
    import torch
    import pbn_synth as S
    from paper_1508_07828_gb300 import _build
    _build.build()
    import paper_1508_07828_gb300 as P
    torch.cuda.set_device(0)
    net, soi, cfg = workload()
    rng = np.random.default_rng(S.BASE_SEED + 6)
    props = [soi] + [S.random_soi(rng, net.n, 1, 5) for _ in range(args.multi - 1)]
    N = P.pbn_load(net)
    kw = dict(omega=cfg["omega"], psi0=PSI0, rhat=cfg["rhat"], eps=cfg["eps"], r=cfg["r"], s=cfg["s"],
              max_length=args.max_length)

    def separate(seed):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        reps = [P.pbn_estimate_two_state(N, x, seed=seed, **kw) for x in props]
        return time.perf_counter() - t0, reps

    def together(seed):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rep = P.pbn_estimate_two_state_multi(N, props, seed=seed, **kw)
        return time.perf_counter() - t0, rep

    for k in range(max(1, args.warmup)):
        separate(k)
        together(k)
    ts, tm, upd_s, upd_m = [], [], 0, 0
    for k in range(args.steps):
        dt, reps = separate(100 + k)
        ts.append(dt)
        upd_s += sum(r["chain_node_updates"] for r in reps)
        dt, rep = together(100 + k)
        tm.append(dt)
        upd_m += rep["chain_node_updates"]
    print(json.dumps({"mode": "multi", "workload": WORKLOAD, "properties": len(props),
                      "separate": {"seconds_per_query_set": float(np.median(ts)), "chain_node_updates": upd_s},
                      "together": {"seconds_per_query_set": float(np.median(tm)), "chain_node_updates": upd_m,
                                   "length": rep["length"], "psi": rep["psi"]},
                      "speedup": float(np.median(ts) / np.median(tm)),
                      "simulation_saved": 1.0 - upd_m / max(upd_s, 1)}))


def run_seq(args):
    """The paper's speed-up (Sec. 5.1) on one GPU: the sequential Alg. 1 on
    one chain against the parallel Alg. GR + Alg. 3 on the bench workload's
    chains, same property and precision; E = speed-up x parallel sample size /
    sequential sample size removes the effect of the sample sizes drawn."""
    import torch
    from paper_1508_07828_gb300 import _build
    _build.build()
    import paper_1508_07828_gb300 as P
    torch.cuda.set_device(0)
    net, soi, cfg = workload()
    N = P.pbn_load(net)
    r = args.seq_r
    par_kw = dict(omega=cfg["omega"], psi0=PSI0, rhat=cfg["rhat"], eps=cfg["eps"], r=r, s=cfg["s"],
                  max_length=args.max_length)
    seq_kw = dict(m0=0, n0=PSI0, eps=cfg["eps"], r=r, s=cfg["s"])

    def timed(fn):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rep = fn()
        return time.perf_counter() - t0, rep

    timed(lambda: P.pbn_estimate_two_state(N, soi, seed=1, **par_kw))
    timed(lambda: P.pbn_estimate_two_state_seq(N, soi, seed=1, **seq_kw))
    rows = []
    for k in range(args.seq_runs):
        tp, rp = timed(lambda: P.pbn_estimate_two_state(N, soi, seed=100 + k, **par_kw))
        ts, rs = timed(lambda: P.pbn_estimate_two_state_seq(N, soi, seed=200 + k, **seq_kw))
        sp = ts / tp
        rows.append({"t_par_s": tp, "t_seq_s": ts, "size_par": rp["sample_size"], "size_seq": rs["N"],
                     "len_seq": rs["length"], "prob_par": rp["prob"], "prob_seq": rs["prob"], "speedup": sp,
                     "speedup_E": sp * rp["sample_size"] / rs["N"]})
    med = lambda key: float(np.median([r[key] for r in rows]))
    agree = float(np.mean([abs(x["prob_par"] - x["prob_seq"]) < 2 * r for x in rows]))
    print(json.dumps({"mode": "seq-vs-par", "workload": WORKLOAD.replace("r0.005", f"r{r:g}"), "runs": len(rows),
                      "chains": cfg["omega"], "r": r,
                      "t_par_s": med("t_par_s"), "t_seq_s": med("t_seq_s"), "speedup": med("speedup"),
                      "speedup_E": med("speedup_E"), "size_par": med("size_par"), "size_seq": med("size_seq"),
                      "seq_length": med("len_seq"), "agreement_within_2r": agree}))


def run_sweep(args):
    """The paper's sweep (Sec. 5.1) in shape: n in {80, 100, 200, 500, 1000,
    2000} x density classes (sparse ~10, in-between 50-100; synthetic models
    from pbn_synth.sweep_config), two-state at precision r (1e-4 in the
    paper) with --sweep-omega chains; for n <= --sweep-seq-max-n also the
    sequential Alg. 1 (speed-up and speed-up E).  One JSON line per model."""
    import torch
    import pbn_synth as S
    from paper_1508_07828_gb300 import _build
    _build.build()
    import paper_1508_07828_gb300 as P
    torch.cuda.set_device(0)
    r = args.seq_r
    for density in [d for d in args.sweep_classes.split(",") if d in S.DENSITY_CLASSES]:
        for n in (80, 100, 200, 500, 1000, 2000):
            net, soi = S.sweep_config(n, density)
            N = P.pbn_load(net)
            kw = dict(omega=args.sweep_omega, psi0=PSI0, rhat=1.05, eps=1e-10, r=r, s=0.95,
                      max_length=args.max_length)
            row = {"mode": "sweep", "n": n, "density_class": density, "density": round(net.density(), 1),
                   "functions": int(net.n_functions), "chains": args.sweep_omega, "r": r}
            try:
                P.pbn_estimate_two_state(N, soi, seed=1, **dict(kw, r=0.01))  # warm-up
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                rep = P.pbn_estimate_two_state(N, soi, seed=2, **kw)
                tp = time.perf_counter() - t0
                row.update({"t_par_s": tp, "length": rep["length"], "sample_size": rep["sample_size"],
                            "prob": rep["prob"], "updates_per_s": rep["chain_node_updates"] / tp})
                if n <= args.sweep_seq_max_n and density in args.sweep_seq_classes.split(","):
                    t0 = time.perf_counter()
                    sq = P.pbn_estimate_two_state_seq(N, soi, seed=3, m0=0, n0=PSI0, eps=1e-10, r=r, s=0.95)
                    ts = time.perf_counter() - t0
                    sp = ts / tp
                    row.update({"t_seq_s": ts, "seq_size": sq["N"], "prob_seq": sq["prob"], "speedup": sp,
                                "speedup_E": sp * rep["sample_size"] / sq["N"],
                                "within_2r": abs(sq["prob"] - rep["prob"]) < 2 * r})
            except P.PbnError as e:
                row["error"] = str(e)
            print(json.dumps(row), flush=True)


def run_serve(args):
    """Serving: queries arrive as a Poisson process; each names a random
    network of the 200-network pool (n log-uniform in [20, 3000]), a state
    of interest of 1-10 nodes, r in {0.01, 0.005, 0.001} and the two-state or
    the Skart stopping rule (half each; Skart at absolute precision r), 1024
    chains.  The engine admits them while others run (continuous batching);
    the baseline serves the same arrival trace one query at a time."""
    import torch
    import pbn_synth as S
    from paper_1508_07828_gb300 import _build
    _build.build()
    import paper_1508_07828_gb300 as P
    torch.cuda.set_device(0)
    pool = S.serving_pool()
    nets = [P.pbn_load(n) for n in pool]
    rng = np.random.default_rng(1508078284)
    out = {"mode": "serve", "pool": len(pool), "queries_per_rate": args.queries, "rates": []}

    def submit(eng, q, tag):
        i, soi, r, seed, kind = q
        kw = dict(omega=1024, seed=seed, psi0=PSI0, rhat=1.05, max_length=args.max_length, tag=tag)
        if kind == "ts":
            eng.submit_two_state(nets[i], soi, r=r, **kw)
        else:
            eng.submit_skart(nets[i], soi, H_star=r, relative=False, alpha=0.05, **kw)

    def alone(q):
        i, soi, r, seed, kind = q
        kw = dict(omega=1024, seed=seed, psi0=PSI0, rhat=1.05, max_length=args.max_length)
        if kind == "ts":
            return P.pbn_estimate_two_state(nets[i], soi, r=r, **kw)
        return P.pbn_estimate_skart(nets[i], soi, H_star=r, relative=False, alpha=0.05, **kw)

    # the engine's autotuner settles on a short warm-up trace
    eng = P.Engine(use_graph=True)
    for k in range(16):
        i = int(rng.integers(len(pool)))
        submit(eng, (i, S.random_soi(rng, pool[i].n), 0.01, 5000 + k, "ts" if k % 2 else "sk"), k)
    eng.run()
    eng.close()
    for rate in [float(x) for x in args.rates.split(",")]:
        arrivals = np.cumsum(rng.exponential(1.0 / rate, size=args.queries))
        qs = []
        for k in range(args.queries):
            i = int(rng.integers(len(pool)))
            qs.append((i, S.random_soi(rng, pool[i].n), float(rng.choice([0.01, 0.005, 0.001])), 10_000 + k,
                       "ts" if rng.random() < 0.5 else "sk"))
        # engine, continuous batching, epochs bounded for latency
        eng = P.Engine(use_graph=True, epoch_target_ms=args.epoch_ms)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        nxt, lat, upd, done, ok = 0, [], 0, 0, 0
        while done < len(qs):
            now = time.perf_counter() - t0
            while nxt < len(qs) and arrivals[nxt] <= now:
                submit(eng, qs[nxt], nxt)
                nxt += 1
            st = eng.step()
            for res in eng.poll():
                lat.append(time.perf_counter() - t0 - arrivals[res["tag"]])
                rep = res["report"]
                upd += rep["chain_node_updates"]
                ok += res["status"] == 0
                done += 1
            if st["active"] == 0 and st["pending"] == 0 and nxt < len(qs):
                time.sleep(max(0.0, min(0.001, arrivals[nxt] - (time.perf_counter() - t0))))
        wall = time.perf_counter() - t0
        eng.close()
        # baseline: the same trace served one query at a time
        t0 = time.perf_counter()
        blat, bupd, free_at, bok = [], 0, 0.0, 0
        for k, q in enumerate(qs):
            start = max(free_at, arrivals[k])
            wait = start - (time.perf_counter() - t0)
            if wait > 0:
                time.sleep(wait)
            try:
                rep = alone(q)
                bupd += rep["chain_node_updates"]
                bok += 1
            except P.PbnError:
                pass
            free_at = time.perf_counter() - t0
            blat.append(free_at - arrivals[k])
        bwall = time.perf_counter() - t0
        out["rates"].append({"rate_per_s": rate,
                             "engine": {"latency_s": _percentiles(lat), "queries_per_s": len(qs) / wall,
                                        "updates_per_s": upd / wall, "ok": ok},
                             "one_at_a_time": {"latency_s": _percentiles(blat), "queries_per_s": len(qs) / bwall,
                                               "updates_per_s": bupd / bwall, "ok": bok}})
        print(json.dumps(out["rates"][-1]), file=sys.stderr, flush=True)
    print(json.dumps(out))


def main():
    args = parse()
    if args.sim_only:
        run_sim_only(args)
        return
    if args.multi:
        run_multi(args)
        return
    if args.seq:
        run_seq(args)
        return
    if args.sweep:
        run_sweep(args)
        return
    if args.batched:
        run_batched(args)
        return
    if args.skart_large:
        return run_skart_large(args)
    if args.serve:
        run_serve(args)
        return
    if args.impl == "reference":
        run_reference(args)
    elif args.mid:
        run_mid(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
