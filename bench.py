#!/usr/bin/env python
"""Benchmark of the explorer: unique states/s and time-to-optimal-config.

One step = one ``mc_min_time`` query of the large workload (C3 at G=36:
P=8 compute units, WG in 2^0..2^9, TS in 2^0..2^5, FREE dispatch, cost
U{1..16} per (WG, TS) from splitmix64 seed 2305091303, 128-bit packed
states; 1,072,924,481 reachable states, closed form) with iterative
threshold lowering and no pruning -- each check explores like an exhaustive
verifier and stops at its first counterexample level, and the last check
(T_min - 1, which holds) explores every reachable state.  A step covers
every stage of the path: the WG/TS selects, level expansion, visited-set
inserts, the property on terminals, the min-reduction and threshold
refinement, and the witness trace.

Output: one JSON line (rank 0).  ``value`` = unique states explored per
second of device time with the model resident in HBM; ``e2e`` = the same
metric through the public C-ABI calls from host buffers (create, query,
destroy); ``roofline`` = the exploration kernel's algorithmic bytes per
launch over its event-timed duration against the measured HBM copy peak,
beside its probe rate against the random 32-byte read+CAS rate measured in
the same run; ``cpu_baseline`` = the CPU oracle on a bounded sample of the
same workload.  The default run adds ``secondary`` (the medium workload C2
at G=80, 64-bit keys), ``batched`` (256 uneven instances in one batch
against the same queries one at a time) and ``served`` (Poisson arrivals of
large-model queries at two rates, against the same arrivals served one at a
time through the single-model calls).

``--impl reference`` times the CPU oracle instead (the method's plain CPU
restatement) on bounded samples of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time
from dataclasses import dataclass, field

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2305_09130_gb300 import pe_workloads as PW  # noqa: E402
from paper_2305_09130_gb300 import workloads as W  # noqa: E402


@dataclass
class Workload:
    make: object                 # () -> ModelSpec
    desc: str
    dtype: str                   # key width the path computes in
    expect: tuple = None         # (T_min, WG, TS) of mc_min_time, from the closed form / the oracle
    cpu_T: int = None            # CPU baseline: oracle check(T) with pruning (None: check(T_min - 1) unpruned)
    ref_T: int = None            # reference arm: oracle check(T) with pruning per step
    tune: dict = field(default_factory=dict)   # autotuner space (option -> candidates)
    traffic: str = None          # committed ncu DRAM-traffic summary for roofline.traffic


WORKLOADS = {
    "c3_star": Workload(
        lambda: W.c3_star(),
        "c3_star: G=36, P=8, WG 2^0..2^9, TS 2^0..2^5, FREE dispatch, cost U{1..16} per (WG, TS) "
        "(splitmix64 seed 2305091303), speed 1, 128-bit packed states; 1,072,924,481 reachable states "
        "(closed form), widest level 193,344,684",
        "u128", expect=(1, 512, 2), cpu_T=30, ref_T=16,
        tune={"probe_scheme": ["split", "one_call", "cas_first", "cas_clear"], "stage_chunk": [128, 192],
              "load_factor_pct": [15, 25]},
        traffic="explore_kernel_c3star_traffic.txt"),
    "c2_star": Workload(
        lambda: W.c2_star(),
        "c2_star: G=80, P=4, WG 2^0..2^8, TS 2^0..2^4, FREE dispatch, cost ceil(WG/TS)*4+WG+2*TS, "
        "speeds U{1..3} (splitmix64 seed 2305091302), 64-bit packed states; 10,385,335 reachable states",
        "u64", expect=(96, 8, 4), cpu_T=None, ref_T=300,
        tune={"probe_scheme": ["split", "one_call", "cas_first", "cas_clear"], "load_factor_pct": [10, 15],
              "stage_chunk": [128, 192]},
        traffic="explore_kernel_c2star_traffic.txt"),
    "c2": Workload(
        lambda: W.c2(rule=W.GREEDY),
        "c2: G=1024, P=4, WG 2^0..2^8, TS 2^0..2^4, GREEDY, cost ceil(WG/TS)*4+WG+2*TS, speeds U{1..3} "
        "(splitmix64 seed 2305091302), 64-bit keys (deep, narrow levels)", "u64",
        tune={"probe_scheme": ["split", "one_call"]}),
    "c3": Workload(
        lambda: W.c3(rule=W.GREEDY),
        "c3: G=4096, P=8, WG 2^0..2^9, TS 2^0..2^5, GREEDY, cost U{1..16} (splitmix64 seed "
        "2305091303), 128-bit keys", "u128", tune={"probe_scheme": ["split", "one_call"]}),
    "c3_star_g24": Workload(
        lambda: W.c3(G=24, rule=W.FREE, key_bits=128),
        "c3 at G=24: P=8, WG 2^0..2^9, TS 2^0..2^5, FREE, cost U{1..16} (seed 2305091303), "
        "128-bit keys (a reduced C3* for profiling: 63,885,179 states)", "u128",
        tune={"probe_scheme": ["split", "one_call"]}),
}
DEFAULT_WORKLOAD = "c3_star"
METRIC = "unique states/sec"
UNIT = "states/s"
FALLBACK_HBM_GBS = 6800.0
KERNEL_SRCS = [os.path.join(ROOT, "paper_2305_09130_gb300", "csrc", f)
               for f in ("mc_explore.cuh", "mc_device.cuh", "mc_internal.h")]
PROFILES = os.path.join(ROOT, "profiles")


# ---------------------------------------------------------------- distributed helpers
def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def dist_init(world: int, use_cuda: bool):
    if world <= 1:
        return None
    import torch.distributed as dist
    if not dist.is_initialized():
        dist.init_process_group(backend="nccl" if use_cuda else "gloo")
    return dist


def reduce_scalar(x: float, op: str, device=None) -> float:
    """max or sum of a scalar over all ranks (identity with one rank)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return x
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


def barrier(device=None):
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        if device is not None:
            dist.barrier(device_ids=[device.index])
        else:
            dist.barrier()


# ---------------------------------------------------------------- clocks during the timed region
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    NAMES = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="clocks", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.25)

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        self.proc.wait()
        sm, mx, reasons = [], [], set()
        with open(self.path) as f:
            for line in f:
                cols = [c.strip() for c in line.split(",")]
                if len(cols) < 9:
                    continue
                try:
                    sm.append(float(cols[1]))
                    mx.append(float(cols[2]))
                except ValueError:
                    continue
                for name, val in zip(self.NAMES, cols[5:9]):
                    if val.lower() == "active":
                        reasons.add(name)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------- roofline inputs
def measured_hbm_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return FALLBACK_HBM_GBS, "fallback"


def algorithmic_bytes_per_state(P: int, key_words: int) -> int:
    """Per unique state: P random 32-byte bucket reads (a FREE state is
    generated once per unit, in-degree ~ P), one 32-byte sector written back
    for its slot, its key written to and read back from the frontier log, and
    its 4-byte parent index."""
    return 32 * P + 32 + 2 * 8 * key_words + 4


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    for path in KERNEL_SRCS:
        with open(path, "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def read_traffic_file(path: str) -> dict:
    fields = {}
    with open(path) as f:
        for line in f:
            if ":" in line and not line.startswith("#"):
                k, v = line.split(":", 1)
                fields[k.strip()] = v.strip()
    return fields


def ncu_traffic_per_launch(path: str, load_factor_pct: int, probe_scheme: str, states_per_launch: float):
    """DRAM bytes per exploration launch from a committed ncu summary, or
    None when the summary is missing, was taken on another kernel source, or
    holds no capture at this visited-set load factor and probe scheme
    ("split" or "one_call").  A summary taken on the benchmarked launches
    gives ``dram_bytes_per_launch_lf<LF>_<scheme>``; one taken on a smaller
    case of the same kernel gives ``dram_bytes_per_state_lf<LF>_<scheme>``, scaled
    here by the states one launch processes (the traffic of this DRAM-bound
    kernel grows with the states it inserts)."""
    try:
        fields = read_traffic_file(path)
        if fields.get("kernel_source_sha256_16") != kernel_source_hash():
            return None
        key = f"dram_bytes_per_launch_lf{int(load_factor_pct)}_{probe_scheme}"
        if key in fields:
            return float(fields[key])
        key = f"dram_bytes_per_state_lf{int(load_factor_pct)}_{probe_scheme}"
        if key in fields:
            return float(fields[key]) * states_per_launch
        return None
    except (OSError, KeyError, ValueError):
        return None


# ---------------------------------------------------------------- arms
def cpu_baseline_sample(spec, wl: Workload, t_min: int) -> dict:
    """The oracle as it stands on a bounded sample of the workload: a pruned
    check(T) (the states of time <= T) or, for a workload the oracle finishes
    in seconds, the holding check check(T_min - 1) without pruning."""
    from oracle import oracle as O
    O.build()
    t0 = time.perf_counter()
    if wl.cpu_T is None:
        r = O.check(spec, t_min - 1, prune=False, early_exit=True)
        what = f"check(T_min-1={t_min - 1}) without pruning"
    else:
        r = O.check(spec, wl.cpu_T, prune=True, early_exit=False)
        what = f"check(T={wl.cpu_T}) with pruning (every state of time <= {wl.cpu_T})"
    dt = time.perf_counter() - t0
    return {"value": r["states"] / dt, "unit": UNIT, "cores": 1, "host_cores": os.cpu_count(),
            "kind": "oracle",
            "sample": f"oracle DFS (std::unordered_set) over {what} of {spec.name}: {r['states']} states "
                      f"in {dt:.2f} s, single thread on a host with {os.cpu_count()} cores"}


def run_reference(args):
    rank, world, _local = dist_env()
    if rank != 0:
        return 0
    from oracle import oracle as O
    O.build()
    wl = WORKLOADS[args.workload or DEFAULT_WORKLOAD]
    spec = wl.make()
    T = wl.ref_T if wl.ref_T is not None else 16

    def step():
        t0 = time.perf_counter()
        r = O.check(spec, T, prune=True, early_exit=False)
        return r["states"], time.perf_counter() - t0

    for _ in range(args.warmup):
        step()
    states = 0
    secs = 0.0
    for _ in range(args.steps):
        s, dt = step()
        states += s
        secs += dt
    value = states / secs
    sample = (f"each step: oracle DFS over check(T={T}) of {spec.name} with pruning (every state of time "
              f"<= {T}), {states // max(args.steps, 1)} states, single thread on a host with "
              f"{os.cpu_count()} cores")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 * secs / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": wl.dtype, "data": "synthetic",
            "config": {"workload": wl.desc, "sample": sample},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "host_cores": os.cpu_count(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0},
            "gpu_launches": 0}
    print(json.dumps(line), flush=True)
    return 0


def measure_single(args, name: str, steps: int, warmup: int, device, stream, local: int,
                   cpu_baseline: bool, random_roofline: bool) -> dict:
    """One workload's line: `steps` timed mc_min_time (or mc_count_states)
    queries on a resident model, the exploration kernel's roofline, the end
    to end rate through the C-ABI from host buffers, and optionally the CPU
    oracle on a bounded sample."""
    import torch

    from paper_2305_09130_gb300 import autotune as AT
    from paper_2305_09130_gb300 import mc

    wl = WORKLOADS[name]
    spec = wl.make()
    # visited-set load factor and probe scheme from the autotuner (outside
    # the timed region; every candidate must return the same answer) unless
    # fixed on the command line; launch shape at the occupancy maximum
    space, fixed = {}, {}
    for k, cands in wl.tune.items():
        if k == "load_factor_pct" and args.load_factor:
            fixed[k] = args.load_factor
        elif k == "probe_scheme" and args.probe_scheme != "tune":
            fixed[k] = mc.PROBE[args.probe_scheme]
        else:
            space[k] = [mc.PROBE[c] for c in cands] if k == "probe_scheme" else list(cands)
    if args.load_factor and "load_factor_pct" not in fixed:
        fixed["load_factor_pct"] = args.load_factor
    if args.probe_scheme not in ("tune",) and "probe_scheme" not in fixed:
        fixed["probe_scheme"] = mc.PROBE[args.probe_scheme]
    if args.no_log_tags:
        fixed["no_log_tags"] = 1
    if args.engine != "auto":
        fixed["engine"] = mc.ENGINE[args.engine]
    if args.stage_chunk:
        space.pop("stage_chunk", None)
        fixed["stage_chunk"] = args.stage_chunk
    if args.unit_threads:
        fixed["unit_threads"] = args.unit_threads

    def tune_measure(c):
        m = mc.mc_model_create(spec, mc.mc_options_default(search=args.mode, prune=args.prune, timing=1,
                                                           **fixed, **c),
                               allocator="torch")
        run = (lambda: mc.mc_count_states(m)) if args.query == "count" else (lambda: mc.mc_min_time(m, trace=False))
        run()
        best = math.inf
        for _ in range(3):
            mc.mc_reset_stats(m)
            ans = run()
            best = min(best, mc.mc_get_stats(m)["explore_ms"])
        mc.mc_model_destroy(m)
        torch.cuda.empty_cache()
        return best, ans
    tuned = AT.tune(tune_measure, space, reps=1) if space else {"options": {}}
    chosen = {**fixed, **tuned["options"]}
    opts = mc.mc_options_default(search=args.mode, prune=args.prune, timing=1, **chosen)
    model = mc.mc_model_create(spec, opts, allocator="torch", stream=stream)
    mc.mc_reserve(model)
    layout = mc.mc_model_layout(model)
    scheme = {v: k for k, v in mc.PROBE.items()}[layout["probe_scheme"]]
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=device)  # > 129 MB of L2

    def flush_l2(k):
        with torch.cuda.stream(stream):
            flush.fill_(k & 0xFF)

    if args.query == "count":
        def query():
            return {"states": mc.mc_count_states(model), "checks": 1, "t_min": None, "wg": None,
                    "ts": None, "t_ini": None}
    else:
        # the witness's trace is walked on the device and read back with the
        # headers in every step; the timed steps skip building the Python
        # list of its keys (host work after the library's read-back, which
        # the events would count while the stream idles); the end-to-end arm
        # builds it
        def query():
            return mc.mc_min_time(model, trace=False)

    ref = None
    for w in range(warmup):
        flush_l2(w)
        ref = query()
    if wl.expect and args.query == "min_time":
        if (ref["t_min"], ref["wg"], ref["ts"]) != wl.expect:
            raise SystemExit(f"wrong result on {name}: {ref} != {wl.expect}")
    if args.query == "count" and spec.rule == W.FREE and ref["states"] != layout["state_bound"]:
        raise SystemExit(f"wrong count {ref['states']} != {layout['state_bound']}")

    mc.mc_reset_stats(model)
    torch.cuda.synchronize()
    barrier(device)
    sampler = ClockSampler(local)
    sampler.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    wall0 = time.perf_counter()
    for k in range(steps):
        flush_l2(k)
        ev[k][0].record(stream)
        r = query()
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    barrier(device)
    clocks = sampler.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    st = mc.mc_get_stats(model)
    dev_ms = sum(step_ms)
    states_local = st["states"]
    dev_ms_max = reduce_scalar(dev_ms, "max", device)
    states_all = reduce_scalar(states_local, "sum", device)
    value = states_all / (dev_ms_max / 1000.0)

    # roofline of the exploration kernel (events on the model's stream)
    bps = algorithmic_bytes_per_state(spec.P, layout["key_words"])
    launches = st["explore_launches"]
    states_per_launch = st["states"] / max(launches, 1)
    achieved = bps * st["states"] / (st["explore_ms"] / 1000.0) / 1e9
    peak, peak_kind = measured_hbm_peak()
    traffic = (ncu_traffic_per_launch(os.path.join(PROFILES, wl.traffic), layout_lf(opts), scheme,
                                      states_per_launch)
               if wl.traffic and args.query == "min_time" else None)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": traffic,
                "algorithmic_bytes_per_launch": bps * states_per_launch,
                "bytes_per_state": bps, "states_per_launch": states_per_launch,
                "avg_launch_ms": st["explore_ms"] / max(launches, 1),
                "kernel": (f"explore_kernel<u{64 * layout['key_words']}, tile {1 << (spec.P - 1).bit_length()}, "
                           f"{'FREE' if spec.rule == W.FREE else 'GREEDY'}, {scheme} insert>"
                           if layout["engine"] == mc.ENGINE["level"] else
                           f"cfg_kernel<u{64 * layout['key_words']}> ({layout['unit_threads']} threads per "
                           f"configuration)"),
                "peak_source": f"{peak_kind} HBM copy bandwidth (MEASURED_PEAKS.json hbm_gbs)"
                               if peak_kind == "measured" else "fallback 6.8 TB/s",
                "launch_timing": "CUDA events on the model's stream, one pair around each query's chained "
                                 "exploration launches (gaps between them included), over the timed steps"}
    if wl.traffic:
        roofline["traffic_source"] = (f"profiles/{wl.traffic}: dram__bytes_read.sum + dram__bytes_write.sum "
                                      f"per exploration launch from ncu (null when the kernel source changed "
                                      f"since the capture)")
    gpu_launches = st["explore_launches"] + st["other_launches"]
    # random-access ceilings (outside the timed region): random 32-byte sector
    # reads and reads followed by a CAS over a buffer far larger than L2, and
    # reads over one the size of this model's visited set (L2-resident when
    # it fits)
    if random_roofline:
        table_bytes = layout["table_slots"] * 8 * layout["key_words"]
        hbm = mc.mc_measure_random_access(64 << 30, 200_000_000, 0)
        hbm_cas = mc.mc_measure_random_access(64 << 30, 200_000_000, 1)
        hbm_cas_only = mc.mc_measure_random_access(64 << 30, 200_000_000, 2)
        l2 = mc.mc_measure_random_access(max(table_bytes, 1 << 20), 200_000_000, 0)
        l2_cas = mc.mc_measure_random_access(max(table_bytes, 1 << 20), 200_000_000, 1)
        l2_cas_only = mc.mc_measure_random_access(max(table_bytes, 1 << 20), 200_000_000, 2)
        explore_s = st["explore_ms"] / 1000.0
        probes = spec.P * st["states"] / explore_s
        # the rate of a kernel that did nothing but its visited-set accesses,
        # at the measured random-access rates: P bucket reads and about one
        # CAS per unique state (split, one call), P CAS (CAS first), P + 1
        # CAS (CAS first with clearing: the expanded state's own slot)
        def states_ceiling(read, read_cas, cas_only):
            if scheme in ("cas_first", "cas_clear"):
                return cas_only["sectors_per_s"] / (spec.P + (1 if scheme == "cas_clear" else 0))
            return 1.0 / (spec.P / read["sectors_per_s"] + 1.0 / read_cas["sectors_per_s"])
        ceiling = states_ceiling(hbm, hbm_cas, hbm_cas_only)
        ceiling_table = states_ceiling(l2, l2_cas, l2_cas_only)
        if scheme in ("cas_first", "cas_clear"):
            per_state = spec.P + (1 if scheme == "cas_clear" else 0)
            note = (f"{per_state} random CAS per unique state (one per generated successor"
                    f"{', one clearing the expanded state' if scheme == 'cas_clear' else ''}); "
                    f"ceiling = CAS rate / {per_state}, over 64 GiB and over a buffer of the visited set's size")
        else:
            note = ("P random 32-byte bucket reads per unique state (one per generated successor) and about "
                    "one CAS; ceiling = 1 / (P / read rate + 1 / read+CAS rate), over 64 GiB and over a "
                    "buffer of the visited set's size (L2-resident when it fits)")
        roofline["random_access"] = {
            "hbm_64GiB_sector_reads_per_s": hbm["sectors_per_s"],
            "hbm_64GiB_sector_read_cas_per_s": hbm_cas["sectors_per_s"],
            "hbm_64GiB_cas_per_s": hbm_cas_only["sectors_per_s"],
            "table_sized_sector_reads_per_s": l2["sectors_per_s"],
            "table_sized_sector_read_cas_per_s": l2_cas["sectors_per_s"],
            "table_sized_cas_per_s": l2_cas_only["sectors_per_s"],
            "table_bytes": table_bytes,
            "probe_scheme": scheme,
            "kernel_probes_per_s": probes,
            "frac_of_hbm_64GiB": probes / (hbm_cas_only if scheme in ("cas_first", "cas_clear")
                                           else hbm)["sectors_per_s"],
            "frac_of_table_sized": probes / l2["sectors_per_s"],
            "states_per_s_ceiling_hbm": ceiling,
            "kernel_states_per_s": st["states"] / explore_s,
            "frac_of_states_ceiling_hbm": (st["states"] / explore_s) / ceiling,
            "states_per_s_ceiling_table_sized": ceiling_table,
            "frac_of_states_ceiling_table_sized": (st["states"] / explore_s) / ceiling_table,
            "note": note}
        if traffic:
            roofline["random_access"]["dram_bytes_per_state"] = traffic / states_per_launch

    # end to end through the public C-ABI from host buffers, as a C caller
    # makes the calls: create (H2D of the model arrays through pinned
    # staging), query, read results, destroy; the library's own allocator and
    # no kernel timing
    e2e_opts = mc.mc_options_default(search=args.mode, prune=args.prune, **chosen)
    retention = int(args.pool_retention_gib * (1 << 30)) if args.pool_retention_gib else None
    if retention is not None:
        mc.mc_set_pool_retention(retention)
    e2e_s = []
    h2d = d2h = 0
    for k in range(steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        m2 = mc.mc_model_create(spec, e2e_opts, allocator=None, stream=stream)
        if args.query == "count":
            r2 = {"t_min": None}
            mc.mc_count_states(m2)
        else:
            r2 = mc.mc_min_time(m2, trace=True)
        s2 = mc.mc_get_stats(m2)
        mc.mc_model_destroy(m2)
        e2e_s.append(time.perf_counter() - t0)
        h2d += s2["h2d_bytes"]
        d2h += s2["d2h_bytes"]
        assert r2["t_min"] == r["t_min"]
    e2e_total = reduce_scalar(sum(e2e_s), "max", device)
    e2e_value = states_all / e2e_total
    if retention is not None:
        mc.mc_set_pool_retention(1 << 30)
    mc.mc_release_cached()

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "ms_per_step": dev_ms_max / steps,
        "dtype": wl.dtype,
        "config": {"workload": wl.desc,
                   "query": (f"mc_min_time search={args.mode} prune={int(args.prune)} early_exit=1 "
                             f"(iterative threshold lowering from the simulated T_ini)"
                             if args.query == "min_time" else "mc_count_states (every reachable state)"),
                   "l2": "flushed between steps (256 MiB write, untimed)",
                   "trace": ("walked on the device and read back in every step; the Python list of its keys "
                             "is built in the end-to-end arm only") if args.query == "min_time" else None,
                   "autotuned": tuned["options"], "autotune_ms": tuned.get("timings", {}),
                   "options_fixed": fixed,
                   "probe_scheme": scheme,
                   "load_factor_pct": layout_lf(opts),
                   "visited_set_bytes": layout["table_slots"] * 8 * layout["key_words"],
                   "frontier_log_bytes": layout["log_capacity"] * (8 * layout["key_words"] + 4),
                   "states_per_step": states_local / steps,
                   "checks_per_step": r["checks"]},
        "time_to_optimal_config_ms": dev_ms_max / steps,
        "result": {"t_min": r["t_min"], "wg": r["wg"], "ts": r["ts"], "t_ini": r["t_ini"],
                   "expected": list(wl.expect) if wl.expect else None},
        "roofline": roofline,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d // steps,
                "d2h_bytes_per_step": d2h // steps,
                "ms_per_step": 1000.0 * e2e_total / steps,
                "pool_retention_bytes": retention if retention is not None else 1 << 30},
        "gpu_launches": gpu_launches,
        "clocks": clocks,
        "wall_s_timed_region": wall,
    }
    mc.mc_model_destroy(model)
    del flush
    torch.cuda.empty_cache()
    if cpu_baseline and args.query == "min_time":
        line["cpu_baseline"] = cpu_baseline_sample(spec, wl, r["t_min"])
    return line


def layout_lf(opts) -> int:
    return int(opts.load_factor_pct)


def run_ours(args):
    import torch

    rank, world, local = dist_env()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device (there is no CPU fallback)")
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    dist_init(world, True)
    stream = torch.cuda.Stream(device)
    name = args.workload or DEFAULT_WORKLOAD
    default_run = args.workload is None
    first = rank == 0 and world == 1
    line = measure_single(args, name, args.steps, args.warmup, device, stream, local,
                          cpu_baseline=first and not args.no_cpu_baseline,
                          random_roofline=not args.no_random_roofline)
    out = {"metric": METRIC, "value": line["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": line["ms_per_step"], "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": line["dtype"],
           "data": "synthetic (seeded model description; no dataset)"}
    out.update({k: v for k, v in line.items() if k not in out})
    out["config"]["parallelism"] = f"replicas x{world}" if world > 1 else "single GPU"
    if default_run and not args.no_extras:
        # the medium workload beside the headline; then the batched and
        # served forms against one query at a time
        sec = measure_single(args, "c2_star", min(args.steps, 20), args.warmup, device, stream, local,
                             cpu_baseline=False, random_roofline=not args.no_random_roofline)
        out["secondary"] = {"c2_star": {k: sec[k] for k in ("value", "unit", "ms_per_step", "dtype", "config",
                                                            "result", "roofline", "e2e", "clocks")}}
        out["gpu_launches"] += sec["gpu_launches"]
        if first:
            out["batched"] = measure_c4(args, device, local, steps=min(args.steps, 10), warmup=args.warmup)
            out["served"] = measure_c5(args, local, rates=[100.0, 1000.0], queries=args.served_queries)
            out["swarm"] = measure_swarm(args, local)
    if rank == 0:
        print(json.dumps(out), flush=True)
    return 0


def percentile(xs, q):
    xs = sorted(xs)
    if not xs:
        return None
    k = min(len(xs) - 1, max(0, int(round(q / 100.0 * (len(xs) - 1)))))
    return xs[k]


def swarm_searches(spec, walks: int, searches: int):
    """The exact T_min, then `searches` swarm searches with consecutive
    seeds (after one warm-up search)."""
    from paper_2305_09130_gb300 import mc

    m = mc.mc_model_create(spec, mc.mc_options_default(timing=1))
    t_min = mc.mc_min_time(m, trace=False)["t_min"]
    mc.mc_swarm(m, 1, walks, max_rounds=2, trace=False)  # warm-up
    runs = [mc.mc_swarm(m, 2305091300 + k, walks, max_rounds=64, trace=True) for k in range(searches)]
    mc.mc_model_destroy(m)
    return t_min, runs


def swarm_summary(t_min, runs) -> dict:
    return {
        "runs_per_s": sum(r["walks"] for r in runs) / (sum(r["total_ms"] for r in runs) / 1000.0),
        "t_min_exact": t_min,
        "searches": [{"first_trail_ms": r["first_trail_ms"], "total_ms": r["total_ms"], "rounds": r["rounds"],
                      "first_time": r["first_time"], "best_time": r["best_time"],
                      "first_trail_optimality": t_min / r["first_time"],
                      "final_optimality": t_min / r["best_time"], "wg": r["wg"], "ts": r["ts"]} for r in runs],
    }


def measure_swarm(args, local: int) -> dict:
    """The default line's swarm object (Section 5, Table 1's last columns):
    five searches each on C2 at G=80 and on C3 literal, with the first
    trail's time and optimality against the exact T_min."""
    out = {"walks_per_round": args.swarm_walks,
           "stop": "after the first round without a run at or below best - 1 (at most 64 rounds)"}
    sampler = ClockSampler(local)
    sampler.start()
    for name in ("c2_star", "c3"):
        wl = WORKLOADS[name]
        t_min, runs = swarm_searches(wl.make(), args.swarm_walks, 5)
        out[name] = {"workload": wl.desc, **swarm_summary(t_min, runs)}
    out["clocks"] = sampler.stop()
    return out


def run_swarm(args):
    """Swarm search (Section 5) on a workload: rounds of random runs on the
    GPU, the first trail's time and optimality against the exact T_min, as in
    the paper's Table 1 (first trail, optimality of the first trail)."""
    import torch

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    wl = WORKLOADS[args.workload or DEFAULT_WORKLOAD]
    spec = wl.make()
    t_min, runs = swarm_searches(spec, args.swarm_walks, args.steps)
    walks = args.swarm_walks
    best = runs[-1]
    line = {
        "metric": "swarm search: random runs per second, first-trail time and optimality",
        "value": sum(r["walks"] for r in runs) / (sum(r["total_ms"] for r in runs) / 1000.0),
        "unit": "runs/s", "n_gpus": 1, "steps": args.steps, "warmup": 1,
        "ms_per_step": sum(r["total_ms"] for r in runs) / len(runs), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": wl.dtype, "data": "synthetic",
        "config": {"workload": wl.desc, "walks_per_round": walks,
                   "stop": "after the first round without a run at or below best - 1 (at most 64 rounds)"},
        "t_min_exact": t_min,
        "runs": [{"first_trail_ms": r["first_trail_ms"], "total_ms": r["total_ms"], "rounds": r["rounds"],
                  "first_time": r["first_time"], "best_time": r["best_time"],
                  "first_trail_optimality": t_min / r["first_time"],
                  "final_optimality": t_min / r["best_time"], "wg": r["wg"], "ts": r["ts"]} for r in runs],
        "trace_states": len(best["trace"]),
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


PE_WORKLOADS = {
    # name: (spec factory, description, expected (t_min, wg, ts) from the oracle
    #        (tests/golden/pe_oracle_expected.json), T of the oracle's bounded sample)
    "pe_abstract": (lambda: PW.pe_abstract(16, P=4, np_=4, gmt=1),
                    "PE-level model of the abstract kernel (Listings 2, 8): size 16, 4 units x 4 PEs, "
                    "GMT 1, WG and TS in {2, 4, 8}; every PE mark, barrier arrival, release, dispatch "
                    "and clock tick interleaved; 37,040,200 reachable states over 1,295 BFS levels",
                    (38, 4, 8), 6),
    "pe_minimum": (lambda: PW.pe_minimum(64, P=4, np_=4, gmt=2),
                   "PE-level model of the Minimum kernel (Listings 10-15): size 64, 4 units x 4 PEs, "
                   "GMT 2, WG and TS in 2^1..2^5; 3,178,678 reachable states over 3,859 BFS levels",
                   (17, 4, 4), 17),
}


def run_pe(args):
    """The processing-element level model: one step = one mc_pe_min_time (a
    full exploration for T_min, the certificate check at T_min - 1 and the
    counterexample check at T_min), or one mc_pe_count_states."""
    import torch

    from paper_2305_09130_gb300 import mc

    rank, world, local = dist_env()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device (there is no CPU fallback)")
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    dist_init(world, True)
    spec = PE_WORKLOADS[args.workload][0]()
    desc = PE_WORKLOADS[args.workload][1]
    # the tile that expands one state and the grid, from the autotuner (every
    # candidate must give the same answer); outside the timed region
    from paper_2305_09130_gb300 import autotune as AT
    fd, cache = tempfile.mkstemp(suffix=".json")
    os.close(fd)
    tuned = AT.tune_pe(spec, "count" if args.query == "count" else "min_time",
                       space={"lanes_per_state": [8, 16, 32], "blocks_per_sm": [0, 2, 3]}, reps=1, path=cache)
    os.unlink(cache)
    opts = mc.mc_options_default(timing=1, **tuned["options"])
    stream = torch.cuda.Stream(device)
    model = mc.mc_pe_model_create(spec, opts, stream=stream.cuda_stream)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=device)

    def flush_l2(k):
        with torch.cuda.stream(stream):
            flush.fill_(k & 0xFF)

    if args.query == "count":
        def query(m):
            return {"states": mc.mc_pe_count_states(m), "t_min": None, "wg": None, "ts": None, "checks": 1}
    else:
        def query(m):
            return mc.mc_pe_min_time(m, trace=True)
    ref = None
    for w in range(args.warmup):  # the first warm-up also grows the buffers to fit
        flush_l2(w)
        ref = query(model)
    lay = mc.mc_pe_model_layout(model)
    expect = PE_WORKLOADS[args.workload][2]
    if args.query == "min_time" and (ref["t_min"], ref["wg"], ref["ts"]) != expect:
        raise SystemExit(f"wrong result {ref} != {expect}")
    mc.mc_pe_reset_stats(model)
    torch.cuda.synchronize()
    barrier(device)
    sampler = ClockSampler(local)
    sampler.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    for k in range(args.steps):
        flush_l2(k)
        ev[k][0].record(stream)
        r = query(model)
        ev[k][1].record(stream)
        assert r["t_min"] == ref["t_min"]
    torch.cuda.synchronize()
    barrier(device)
    clocks = sampler.stop()
    st = mc.mc_pe_get_stats(model)
    dev_ms = sum(a.elapsed_time(b) for a, b in ev)
    dev_ms_max = reduce_scalar(dev_ms, "max", device)
    states_all = reduce_scalar(st["states"], "sum", device)
    value = states_all / (dev_ms_max / 1000.0)
    # per unique state: one 32-byte bucket probe per generated successor, one
    # 32-byte slot write-back, the 16-byte key written to and read back from
    # the frontier log, the 4-byte parent index
    probes_per_state = st["probes"] / max(st["states"], 1)
    bps = 32 * probes_per_state + 32 + 2 * 16 + 4
    launches = st["explore_launches"]
    achieved = bps * st["states"] / (st["explore_ms"] / 1000.0) / 1e9
    peak, peak_kind = measured_hbm_peak()
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": None, "bytes_per_state": bps, "probes_per_state": probes_per_state,
                "algorithmic_bytes_per_launch": bps * st["states"] / max(launches, 1),
                "avg_launch_ms": st["explore_ms"] / max(launches, 1),
                "levels_per_launch": st["device_steps"] / max(launches, 1),
                "kernel": f"pe_explore_kernel<tile {lay['tile']}>",
                "peak_source": f"{peak_kind} HBM copy bandwidth"}
    # end to end through the public C-ABI from host buffers
    e2e_s, h2d, d2h = [], 0, 0
    big = dict(tuned["options"], log_capacity=lay["log_capacity"],
               table_log2=lay["table_slots"].bit_length() - 1)
    for k in range(args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        m2 = mc.mc_pe_model_create(spec, mc.mc_options_default(**big), stream=stream.cuda_stream)
        r2 = query(m2)
        s2 = mc.mc_pe_get_stats(m2)
        mc.mc_pe_model_destroy(m2)
        e2e_s.append(time.perf_counter() - t0)
        h2d += s2["h2d_bytes"]
        d2h += s2["d2h_bytes"]
        assert r2["t_min"] == ref["t_min"]
    e2e_total = reduce_scalar(sum(e2e_s), "max", device)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": dev_ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u128",
        "data": "synthetic (model description from the kernels' listings; no dataset)",
        "config": {"workload": desc,
                   "query": "mc_pe_min_time (full pass, check(T_min-1), check(T_min)), prune=1 early_exit=1"
                   if args.query == "min_time" else "mc_pe_count_states",
                   "l2": "flushed between steps (256 MiB write, untimed)",
                   "autotuned": tuned["options"],
                   "states_per_step": st["states"] / args.steps},
        "time_to_optimal_config_ms": dev_ms_max / args.steps,
        "result": {"t_min": ref["t_min"], "wg": ref["wg"], "ts": ref["ts"]},
        "roofline": roofline,
        "e2e": {"value": states_all / e2e_total, "unit": UNIT, "h2d_bytes_per_step": h2d // args.steps,
                "d2h_bytes_per_step": d2h // args.steps, "ms_per_step": 1000.0 * e2e_total / args.steps},
        "gpu_launches": st["explore_launches"],
        "clocks": clocks,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        from oracle import oracle as O
        O.build()
        T = PE_WORKLOADS[args.workload][3]
        t0 = time.perf_counter()
        rs = O.pe_check(spec, T, prune=True, early_exit=False)
        dt = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": rs["states"] / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": f"oracle BFS (std::unordered_set) over check(T={T}) of the same "
                                          f"model with pruning: {rs['states']} states in {dt:.2f} s, "
                                          f"single thread"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    mc.mc_pe_model_destroy(model)
    return 0


C4_DESC = ("c4: 256 instances, G=2^U{6..12}, P in {2,4,8}, WG 2^0..2^8, TS 2^0..2^4, cost U{1..16}, "
           "speeds U{1..3} (splitmix64 seed 2305091304), GREEDY; half mc_min_time, half mc_check at "
           "round(U[0.8,1.2] x T_min)")
C5_DESC = ("c5: min-time queries on G=4096, P=8, WG 2^0..2^9, TS 2^0..2^5, cost U{1..16} (new splitmix64 "
           "seed per query), GREEDY, 128-bit keys; Poisson arrivals (splitmix64 seed 2305091305)")


def measure_c4(args, device, local: int, steps: int, warmup: int) -> dict:
    """Batched queries: 256 uneven models (G = 2^U{6..12}, P in {2,4,8}, WG
    2^0..2^8, TS 2^0..2^4, cost U{1..16}, speeds U{1..3}, GREEDY), half
    min-time and half check at round(U[0.8,1.2] x T_min), answered by one
    mc_batch_run, against the same queries one at a time on the single-model
    calls."""
    import torch

    from paper_2305_09130_gb300 import autotune as AT
    from paper_2305_09130_gb300 import mc

    specs = W.c4_instances(256)
    probe = mc.mc_batch_create(specs)
    optima0 = [r["time"] for r in mc.mc_batch_run(probe, [("min_time", None)] * len(specs))]
    mc.mc_batch_destroy(probe)
    queries0 = [("min_time", None) if sp.meta["query"] else
                ("check", round(t * sp.meta["t_frac_milli"] / 1000)) for sp, t in zip(specs, optima0)]
    if args.engine != "auto":  # fixed on the command line: no tuning
        fixed = {"engine": mc.ENGINE[args.engine]}
        if args.unit_threads:
            fixed["unit_threads"] = args.unit_threads
        tuned = {"options": fixed, "timings": {}}
    else:
        tuned = AT.tune_batch(specs, queries0, space=[AT.BATCH_LEVEL_SPACE, AT.BATCH_CONFIG_SPACE],
                              reps=1, cache={}, path=os.path.join(tempfile.gettempdir(), "mc_autotune_c4.json"))
    opts = mc.mc_options_default(timing=1, **tuned["options"])
    stream = torch.cuda.Stream(device)
    batch = mc.mc_batch_create(specs, opts, stream=stream)
    # the check thresholds are fractions of each instance's optimum: take the
    # optima from an untimed all-min-time run
    optima = [r["time"] for r in mc.mc_batch_run(batch, [("min_time", None)] * len(specs))]
    queries = [("min_time", None) if sp.meta["query"] else
               ("check", round(t * sp.meta["t_frac_milli"] / 1000)) for sp, t in zip(specs, optima)]
    for _ in range(warmup):
        ref = mc.mc_batch_run(batch, queries)
    torch.cuda.synchronize()
    st0 = mc.mc_batch_get_stats(batch)
    sampler = ClockSampler(local)
    sampler.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    states = 0
    for k in range(steps):
        ev[k][0].record(stream)
        res = mc.mc_batch_run(batch, queries)
        ev[k][1].record(stream)
        states += sum(r["states"] for r in res)
        assert [r["status"] for r in res] == [0] * len(res)
        assert [(r["time"], r["states"]) for r in res] == [(r["time"], r["states"]) for r in ref]
    torch.cuda.synchronize()
    clocks = sampler.stop()
    bst = mc.mc_batch_get_stats(batch)
    mc.mc_batch_destroy(batch)
    batch_ms = [a.elapsed_time(b) for a, b in ev]
    dev_ms = sum(batch_ms)
    value = states / (dev_ms / 1000.0)

    # one query at a time on the single-model entry points (models created
    # untimed, with the library's default launch shape -- the batch's tuned
    # options suit its own launch, not a lone query); latency of query k when
    # all arrive together = sum of the service times of queries 0..k
    seq_opts = mc.mc_options_default(timing=1)
    models = [mc.mc_model_create(sp.with_key_bits(128), seq_opts, stream=stream) for sp in specs]
    for m in models:
        mc.mc_reserve(m)
    service = []
    seq_states = 0
    for m, (kind, T), rb in zip(models, queries, ref):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        r = mc.mc_min_time(m, trace=False) if kind == "min_time" else mc.mc_check(m, T, trace=False)
        b.record(stream)
        b.synchronize()
        service.append(a.elapsed_time(b))
        seq_states += r["states"]
        assert r["states"] == rb["states"]
    for m in models:
        mc.mc_model_destroy(m)
    seq_total = sum(service)
    cum, acc = [], 0.0
    for x in service:
        acc += x
        cum.append(acc)
    return {
        "workload": C4_DESC,
        "query": "one mc_batch_run per step",
        "autotuned_options": tuned["options"], "autotune_ms": tuned["timings"],
        "steps": steps, "ms_per_batch": dev_ms / steps, "states_per_s": value,
        "states_per_batch": states / steps,
        "kernels_per_batch": ((bst["explore_launches"] + bst["other_launches"])
                              - (st0["explore_launches"] + st0["other_launches"])) / steps,
        "graph_replays_per_batch": (bst["graph_launches"] - st0["graph_launches"]) / steps,
        "query_latency_ms_p50": percentile(batch_ms, 50), "query_latency_ms_p99": percentile(batch_ms, 99),
        "sequential": {"options": "library defaults (single-model explorer, load factor 25%)",
                       "ms_total": seq_total, "states_per_s": seq_states / (seq_total / 1000.0),
                       "service_ms_p50": percentile(service, 50), "service_ms_p99": percentile(service, 99),
                       "latency_all_arrive_together_ms_p50": percentile(cum, 50),
                       "latency_all_arrive_together_ms_p99": percentile(cum, 99)},
        "speedup_vs_sequential": seq_total / (dev_ms / steps),
        "clocks": clocks,
    }


def c5_query(k: int):
    return W.c3(G=4096, rule=W.GREEDY, seed=2305091305 * 1000003 + k, key_bits=128)


def poisson_arrivals(rng, rate: float, n: int):
    out, t = [], 0.0
    for _ in range(n):
        u = (rng.next() >> 11) / float(1 << 53)
        t += -math.log(1.0 - u) / rate
        out.append(t)
    return out


def wait_until(t0: float, t: float, poll=None):
    """Sleep until perf_counter() - t0 >= t (the last 0.3 ms spinning)."""
    while True:
        left = t - (time.perf_counter() - t0)
        if left <= 0:
            return
        if poll:
            poll()
        if left > 0.0006:
            time.sleep(min(left - 0.0003, 0.0002 if poll else left - 0.0003))


def measure_c5(args, local: int, rates, queries: int) -> dict:
    """Served queries: Poisson arrivals of min-time queries on models drawn as
    the large single query (G=4096, P=8, WG 2^0..2^9, TS 2^0..2^5, cost
    U{1..16} with a new seed per query, GREEDY, 128-bit keys), at each rate,
    answered by the request loop (mc_server_*), against the same arrival
    stream served one query at a time through the single-model calls
    (mc_model_create, mc_min_time, mc_model_destroy), each started at its
    arrival or when the previous one finished."""
    import torch

    from paper_2305_09130_gb300 import mc

    rng = W.SplitMix64(2305091305)
    free_b, _tot = torch.cuda.mem_get_info()
    pool = int(min(free_b * 0.6, 120 << 30))
    srv = mc.mc_server_create(slots=args.slots, pool_bytes=pool)
    opts = mc.mc_options_default()
    for k in range(3):  # warm the library's allocator and staging
        m = mc.mc_model_create(c5_query(10_000_000 + k), opts, allocator=None)
        mc.mc_min_time(m, trace=False)
        mc.mc_model_destroy(m)
    sweep = []
    qid = 0
    for rate in rates:
        n = queries if queries else int(min(10000, max(2000, rate * args.c5_seconds)))
        arrivals = poisson_arrivals(rng, rate, n)
        specs = [c5_query(qid + k) for k in range(n)]
        qid += n
        # served
        got = {}

        def poll():
            for r in mc.mc_server_poll(srv, wait_ms=0):
                got[r["ticket"]] = r
        sampler = ClockSampler(local)
        sampler.start()
        t0 = time.perf_counter()
        for k in range(n):
            wait_until(t0, arrivals[k], poll)
            mc.mc_server_submit(srv, specs[k], "min_time")
        while len(got) < n:
            for r in mc.mc_server_poll(srv, wait_ms=20):
                got[r["ticket"]] = r
            if time.perf_counter() - t0 > arrivals[-1] + 600:
                raise SystemExit(f"served run at {rate}/s did not finish: {mc.mc_server_status(srv)}")
        clocks = sampler.stop()
        res = [got[t] for t in sorted(got)]
        assert all(r["status"] == 0 for r in res)
        lat = [1000.0 * (r["done_s"] - r["submit_s"]) for r in res]
        span = max(r["done_s"] for r in res) - min(r["submit_s"] for r in res)
        # one at a time, the same arrival stream in real time
        seq_lat, seq_res = [], []
        sampler2 = ClockSampler(local)
        sampler2.start()
        t0 = time.perf_counter()
        for k in range(n):
            wait_until(t0, arrivals[k])
            m = mc.mc_model_create(specs[k], opts, allocator=None)
            rr = mc.mc_min_time(m, trace=False)
            mc.mc_model_destroy(m)
            seq_lat.append(1000.0 * (time.perf_counter() - t0 - arrivals[k]))
            seq_res.append(rr)
        seq_span = time.perf_counter() - t0 - arrivals[0]
        clocks2 = sampler2.stop()
        # every served result equals the one-at-a-time result of the same query
        mism = sum(1 for a, b in zip(res, seq_res)
                   if (a["time"], a["states"], a["wg"], a["ts"]) != (b["t_min"], b["states"], b["wg"], b["ts"]))
        sweep.append({
            "rate_per_s": rate, "queries": n,
            "served": {"throughput_qps": n / span, "latency_ms_p50": percentile(lat, 50),
                       "latency_ms_p99": percentile(lat, 99), "latency_ms_max": max(lat),
                       "states_per_s": sum(r["states"] for r in res) / span,
                       "ran_alone": sum(r["path"] == "alone" for r in res), "clocks": clocks},
            "one_at_a_time": {"throughput_qps": n / seq_span, "latency_ms_p50": percentile(seq_lat, 50),
                              "latency_ms_p99": percentile(seq_lat, 99), "latency_ms_max": max(seq_lat),
                              "states_per_s": sum(r["states"] for r in seq_res) / seq_span,
                              "clocks": clocks2},
            "results_differ": mism,
        })
    status = mc.mc_server_status(srv)
    mc.mc_server_destroy(srv)
    mc.mc_release_cached()
    return {"workload": C5_DESC, "slots": args.slots, "pool_bytes": pool,
            "query": "mc_min_time (search SINGLE, library default options) per request",
            "one_at_a_time": "the same arrival stream replayed in real time; each query starts at its arrival "
                             "or when the previous one finished and runs mc_model_create, mc_min_time, "
                             "mc_model_destroy (library allocator); latency from arrival to result",
            "sweep": sweep, "device_loop_launches": status["launches"]}


def run_c4(args):
    import torch

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    b = measure_c4(args, device, local, steps=args.steps, warmup=args.warmup)
    line = {"metric": METRIC, "value": b["states_per_s"], "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": b["ms_per_batch"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u128", "data": "synthetic (seeded model descriptions)",
            "config": {"workload": C4_DESC}, "batched": b, "clocks": b["clocks"]}
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def run_c5(args):
    import torch

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    rates = [float(x) for x in args.rates.split(",")]
    s = measure_c5(args, local, rates, queries=args.c5_queries)
    top = s["sweep"][-1]
    line = {"metric": "served queries: throughput with p50/p99 latency", "value": top["served"]["throughput_qps"],
            "unit": "queries/s", "n_gpus": 1, "steps": len(rates), "warmup": 0, "ms_per_step": None,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u128",
            "data": "synthetic (seeded model per query)", "config": {"workload": C5_DESC}, "served": s,
            "clocks": top["served"]["clocks"]}
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def main(argv=None):
    p = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--mode", choices=["single", "lower", "bisect"], default="lower")
    p.add_argument("--prune", type=int, default=0)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--pool-retention-gib", type=float, default=64.0,
                   help="end-to-end arm: device memory the library's pool keeps between models "
                        "(mc_set_pool_retention, as a server creating and destroying models sets it; "
                        "0 = the library default, 1 GiB)")
    p.add_argument("--no-random-roofline", action="store_true")
    p.add_argument("--no-extras", action="store_true",
                   help="default run: skip the secondary, batched and served objects")
    p.add_argument("--load-factor", type=int, default=0,
                   help="visited-set load factor in percent (0: the autotuner picks it)")
    p.add_argument("--probe-scheme", choices=["tune", "auto", "split", "one_call", "cas_first", "cas_clear"], default="tune",
                   help="visited-set insert of the exploration kernel (tune: the autotuner picks it)")
    p.add_argument("--no-log-tags", action="store_true",
                   help="untagged frontier log: blocks write their entries before they arrive at a level")
    p.add_argument("--engine", choices=["auto", "level", "config"], default="auto",
                   help="single-model explorer: level-synchronous or one block per configuration "
                        "(auto: by the model's widest configuration level)")
    p.add_argument("--stage-chunk", type=int, default=0,
                   help="level engine: winners staged per warp before a flush (0: the autotuner picks it)")
    p.add_argument("--unit-threads", type=int, default=0,
                   help="configuration engine: threads per block (0: from the model, or the tuner's pick)")
    p.add_argument("--rates", default="10,30,100,300,1000", help="c5 arrival rates (queries/s)")
    p.add_argument("--slots", type=int, default=512, help="c5 requests on the device at once")
    p.add_argument("--c5-seconds", type=float, default=100.0,
                   help="c5: queries per rate = min(10000, max(2000, rate x this)) unless --c5-queries")
    p.add_argument("--c5-queries", type=int, default=0, help="c5 queries per rate (0: from --c5-seconds)")
    p.add_argument("--served-queries", type=int, default=2000, help="default run: queries per served rate")
    p.add_argument("--workload", choices=sorted(WORKLOADS) + ["c4", "c5"] + sorted(PE_WORKLOADS),
                   default=None,
                   help="one workload alone (default: the c3_star line with the c2_star, batched and "
                        "served objects)")
    p.add_argument("--query", choices=["min_time", "count", "swarm"], default="min_time")
    p.add_argument("--swarm-walks", type=int, default=1 << 20, help="random runs per swarm round")
    args = p.parse_args(argv)
    if args.warmup < 3:
        p.error("--warmup must be >= 3")
    if args.impl == "reference":
        if args.workload not in (None,) + tuple(WORKLOADS):
            p.error("--impl reference times the oracle on a single-model workload")
        return run_reference(args)
    if args.workload == "c4":
        return run_c4(args)
    if args.query == "swarm":
        return run_swarm(args)
    if args.workload == "c5":
        return run_c5(args)
    if args.workload in PE_WORKLOADS:
        return run_pe(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
