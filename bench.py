#!/usr/bin/env python
"""Benchmark of the explorer: unique states/s and time-to-optimal-config.

One step = one ``mc_min_time`` query of the medium workload (C2 at G=80:
P=4 compute units, WG in 2^0..2^8, TS in 2^0..2^4, FREE dispatch, formula
cost, per-unit speeds U{1..3} from splitmix64 seed 2305091302; 10,385,335
reachable states) with iterative threshold lowering and no pruning -- each
check explores like an exhaustive verifier and stops at its first
counterexample level, and the last check (T_min - 1, which holds) explores
every reachable state.  A step covers every stage of the path: the WG/TS
selects, level expansion, visited-set inserts, the property on terminals,
the min-reduction and threshold refinement, and the witness trace.

Output: one JSON line (rank 0).  ``value`` = unique states explored per
second of device time with the model resident in HBM; ``e2e`` = the same
metric through the public C-ABI calls from host buffers (create, query,
destroy); ``roofline`` = the exploration kernel's algorithmic bytes per
launch over its event-timed duration against the measured HBM copy peak;
``cpu_baseline`` = the CPU oracle on a bounded sample of the same workload.

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

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2305_09130_gb300 import pe_workloads as PW  # noqa: E402
from paper_2305_09130_gb300 import workloads as W  # noqa: E402

WORKLOADS = {
    # name: (spec factory, description)
    "c2_star": (lambda: W.c2_star(), None),
    "c3_star": (lambda: W.c3_star(),
                "c3_star: G=36, P=8, WG 2^0..2^9, TS 2^0..2^5, FREE, cost U{1..16} (splitmix64 seed "
                "2305091303), 128-bit keys; 1,072,924,481 reachable states"),
    "c2": (lambda: W.c2(rule=W.GREEDY),
           "c2: G=1024, P=4, WG 2^0..2^8, TS 2^0..2^4, GREEDY, cost ceil(WG/TS)*4+WG+2*TS, speeds U{1..3} "
           "(splitmix64 seed 2305091302), 64-bit keys (deep, narrow levels)"),
    "c3": (lambda: W.c3(rule=W.GREEDY),
           "c3: G=4096, P=8, WG 2^0..2^9, TS 2^0..2^5, GREEDY, cost U{1..16} (splitmix64 seed "
           "2305091303), 128-bit keys"),
    "c3_star_g24": (lambda: W.c3(G=24, rule=W.FREE, key_bits=128),
                    "c3 at G=24: P=8, WG 2^0..2^9, TS 2^0..2^5, FREE, cost U{1..16} (seed 2305091303), "
                    "128-bit keys (a reduced C3* for profiling)"),
}
METRIC = "unique states/sec"
UNIT = "states/s"
WORKLOAD = ("c2_star: G=80, P=4, WG 2^0..2^8, TS 2^0..2^4, FREE dispatch, cost ceil(WG/TS)*4+WG+2*TS, "
            "speeds U{1..3} (splitmix64 seed 2305091302); 10,385,335 reachable states")
REFERENCE_SAMPLE_T = 300     # pruned check of the same model: ~0.74M states
FALLBACK_HBM_GBS = 6800.0
KERNEL_SRCS = [os.path.join(ROOT, "paper_2305_09130_gb300", "csrc", f)
               for f in ("mc_kernels.cu", "mc_device.cuh", "mc_internal.h")]
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "explore_kernel_c2star_traffic.txt")


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


def ncu_traffic_per_launch(load_factor_pct: int, probe_scheme: str):
    """dram bytes per exploration launch from the committed ncu summary, or
    None when the summary is missing, was taken on another kernel source, or
    holds no capture at this visited-set load factor and probe scheme
    ("split" or "one_call")."""
    try:
        fields = {}
        with open(TRAFFIC_FILE) as f:
            for line in f:
                if ":" in line and not line.startswith("#"):
                    k, v = line.split(":", 1)
                    fields[k.strip()] = v.strip()
        if fields.get("kernel_source_sha256_16") != kernel_source_hash():
            return None
        return float(fields[f"dram_bytes_per_launch_lf{int(load_factor_pct)}_{probe_scheme}"])
    except (OSError, KeyError, ValueError):
        return None


# ---------------------------------------------------------------- arms
def cpu_baseline_sample(spec, t_min: int) -> dict:
    """The oracle as it stands on the holding check check(T_min - 1) of the
    workload without pruning: a full DFS over every reachable state."""
    from oracle import oracle as O
    O.build()
    t0 = time.perf_counter()
    r = O.check(spec, t_min - 1, prune=False, early_exit=True)
    dt = time.perf_counter() - t0
    return {"value": r["states"] / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"oracle DFS (std::unordered_set) over check(T_min-1={t_min - 1}) of c2_star "
                      f"without pruning: {r['states']} states in {dt:.2f} s, single thread"}


def run_reference(args):
    rank, world, _local = dist_env()
    if rank != 0:
        return 0
    from oracle import oracle as O
    O.build()
    spec = W.c2_star()

    def step():
        t0 = time.perf_counter()
        r = O.check(spec, REFERENCE_SAMPLE_T, prune=True, early_exit=False)
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
    sample = (f"each step: oracle DFS over check(T={REFERENCE_SAMPLE_T}) of c2_star with pruning, "
              f"{states // max(args.steps, 1)} states, single thread")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 * secs / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": sample},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0},
            "gpu_launches": 0}
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import torch

    from paper_2305_09130_gb300 import mc

    rank, world, local = dist_env()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device (there is no CPU fallback)")
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    dist_init(world, True)
    spec = WORKLOADS[args.workload][0]()
    workload = WORKLOADS[args.workload][1] or WORKLOAD
    # visited-set load factor (C2 at G=80) and probe scheme from the
    # autotuner (outside the timed region; every candidate must return the
    # same answer) unless fixed on the command line; launch shape at the
    # occupancy maximum, which the tuner also picks for this kernel
    from paper_2305_09130_gb300 import autotune as AT

    space, fixed = {}, {}
    if args.load_factor:
        fixed["load_factor_pct"] = args.load_factor
    elif args.workload == "c2_star":
        space["load_factor_pct"] = [10, 15]
    if args.no_log_tags:
        fixed["no_log_tags"] = 1
    if args.probe_scheme == "tune":
        space["probe_scheme"] = [mc.PROBE["split"], mc.PROBE["one_call"]]
    else:
        fixed["probe_scheme"] = mc.PROBE[args.probe_scheme]

    def lf_measure(c):
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
        return best, ans
    tuned = AT.tune(lf_measure, space, reps=1) if space else {"options": {}}
    chosen = {**fixed, **tuned["options"]}
    opts = mc.mc_options_default(search=args.mode, prune=args.prune, timing=1, **chosen)
    stream = torch.cuda.Stream(device)
    model = mc.mc_model_create(spec, opts, allocator="torch", stream=stream)
    mc.mc_reserve(model)
    layout = mc.mc_model_layout(model)
    scheme = "split" if layout["probe_scheme"] == mc.PROBE["split"] else "one_call"
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=device)  # > 129 MB of L2

    def flush_l2(k):
        with torch.cuda.stream(stream):
            flush.fill_(k & 0xFF)

    if args.query == "count":
        def query():
            return {"states": mc.mc_count_states(model), "checks": 1, "t_min": None, "wg": None,
                    "ts": None, "t_ini": None}
    else:
        def query():
            return mc.mc_min_time(model, trace=True)

    ref = None
    for w in range(args.warmup):
        flush_l2(w)
        ref = query()
    if args.workload == "c2_star" and args.query == "min_time":
        expect = (96, 8, 4)  # T_min and (WG, TS) of this workload, from the oracle
        if (ref["t_min"], ref["wg"], ref["ts"]) != expect:
            raise SystemExit(f"wrong result {ref} != {expect}")
    if args.query == "count" and spec.rule == W.FREE and ref["states"] != layout["state_bound"]:
        raise SystemExit(f"wrong count {ref['states']} != {layout['state_bound']}")

    mc.mc_reset_stats(model)
    torch.cuda.synchronize()
    barrier(device)
    sampler = ClockSampler(local)
    sampler.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    wall0 = time.perf_counter()
    for k in range(args.steps):
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
    achieved = bps * st["states"] / (st["explore_ms"] / 1000.0) / 1e9
    peak, peak_kind = measured_hbm_peak()
    traffic = (ncu_traffic_per_launch(opts.load_factor_pct, scheme)
               if (args.workload, args.query) == ("c2_star", "min_time") else None)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": traffic,
                "algorithmic_bytes_per_launch": bps * st["states"] / max(launches, 1),
                "bytes_per_state": bps, "states_per_launch": st["states"] / max(launches, 1),
                "avg_launch_ms": st["explore_ms"] / max(launches, 1),
                "kernel": f"explore_kernel<u{64 * layout['key_words']}, tile {1 << (spec.P - 1).bit_length()}, "
                          f"{'FREE' if spec.rule == W.FREE else 'GREEDY'}, {scheme} insert>",
                "peak_source": f"{peak_kind} HBM copy bandwidth (MEASURED_PEAKS.json hbm_gbs)"
                               if peak_kind == "measured" else "fallback 6.8 TB/s"}
    gpu_launches = st["explore_launches"] + st["other_launches"]
    # random-access ceilings (outside the timed region): random 32-byte sector
    # reads over a buffer far larger than L2, and over one the size of this
    # model's visited set (L2-resident when it fits)
    if not args.no_random_roofline:
        table_bytes = layout["table_slots"] * 8 * layout["key_words"]
        hbm = mc.mc_measure_random_access(64 << 30, 200_000_000, 0)
        hbm_cas = mc.mc_measure_random_access(64 << 30, 200_000_000, 1)
        l2 = mc.mc_measure_random_access(max(table_bytes, 1 << 20), 200_000_000, 0)
        probes = spec.P * st["states"] / (st["explore_ms"] / 1000.0)
        roofline["random_access"] = {
            "hbm_64GiB_sector_reads_per_s": hbm["sectors_per_s"],
            "hbm_64GiB_sector_read_cas_per_s": hbm_cas["sectors_per_s"],
            "table_sized_sector_reads_per_s": l2["sectors_per_s"],
            "table_bytes": table_bytes,
            "kernel_probe_reads_per_s": probes,
            "frac_of_table_sized": probes / l2["sectors_per_s"],
            "note": "one 32-byte bucket read per generated successor (P per state)"}

    # end to end through the public C-ABI from host buffers, as a C caller
    # makes the calls: create (H2D of the model arrays through pinned
    # staging), query, read results, destroy; the library's own allocator and
    # no kernel timing
    e2e_opts = mc.mc_options_default(search=args.mode, prune=args.prune, **chosen)
    e2e_s = []
    h2d = d2h = 0
    for k in range(args.steps):
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

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": dev_ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u64",
        "data": "synthetic (seeded model description; no dataset)",
        "config": {"workload": workload,
                   "query": (f"mc_min_time search={args.mode} prune={int(args.prune)} early_exit=1 "
                             f"(iterative threshold lowering from the simulated T_ini)"
                             if args.query == "min_time" else "mc_count_states (every reachable state)"),
                   "l2": "flushed between steps (256 MiB write, untimed)",
                   "autotuned": tuned["options"], "autotune_ms": tuned.get("timings", {}),
                   "options_fixed": fixed,
                   "probe_scheme": scheme,
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                   "states_per_step": states_local / args.steps,
                   "checks_per_step": r["checks"]},
        "time_to_optimal_config_ms": dev_ms_max / args.steps,
        "result": {"t_min": r["t_min"], "wg": r["wg"], "ts": r["ts"], "t_ini": r["t_ini"]},
        "roofline": roofline,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d // args.steps,
                "d2h_bytes_per_step": d2h // args.steps,
                "ms_per_step": 1000.0 * e2e_total / args.steps},
        "gpu_launches": gpu_launches,
        "clocks": clocks,
        "wall_s_timed_region": wall,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline and args.workload == "c2_star" \
            and args.query == "min_time":
        line["cpu_baseline"] = cpu_baseline_sample(spec, r["t_min"])
    if rank == 0:
        print(json.dumps(line), flush=True)
    mc.mc_model_destroy(model)
    return 0


def percentile(xs, q):
    xs = sorted(xs)
    if not xs:
        return None
    k = min(len(xs) - 1, max(0, int(round(q / 100.0 * (len(xs) - 1)))))
    return xs[k]


def run_swarm(args):
    """Swarm search (Section 5) on a workload: rounds of random runs on the
    GPU, the first trail's time and optimality against the exact T_min, as in
    the paper's Table 1 (first trail, optimality of the first trail)."""
    import torch

    from paper_2305_09130_gb300 import mc

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    spec = WORKLOADS[args.workload][0]()
    m = mc.mc_model_create(spec, mc.mc_options_default(timing=1))
    t_min = mc.mc_min_time(m, trace=False)["t_min"]
    walks = args.swarm_walks
    mc.mc_swarm(m, 1, walks, max_rounds=2, trace=False)  # warm-up
    runs = []
    for k in range(args.steps):
        runs.append(mc.mc_swarm(m, 2305091300 + k, walks, max_rounds=64, trace=True))
    best = runs[-1]
    line = {
        "metric": "swarm search: random runs per second, first-trail time and optimality",
        "value": sum(r["walks"] for r in runs) / (sum(r["total_ms"] for r in runs) / 1000.0),
        "unit": "runs/s", "n_gpus": 1, "steps": args.steps, "warmup": 1,
        "ms_per_step": sum(r["total_ms"] for r in runs) / len(runs), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": WORKLOADS[args.workload][1] or WORKLOAD, "walks_per_round": walks,
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


def run_c4(args):
    """Batched queries: 256 uneven models (G = 2^U{6..12}, P in {2,4,8}, WG
    2^0..2^8, TS 2^0..2^4, cost U{1..16}, speeds U{1..3}, GREEDY), half
    min-time and half check at round(U[0.8,1.2] x T_min), answered by one
    persistent launch, against the same queries one at a time."""
    import torch

    from paper_2305_09130_gb300 import mc

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    dist_init(world, True)
    specs = W.c4_instances(256)
    from paper_2305_09130_gb300 import autotune as AT
    probe = mc.mc_batch_create(specs)
    optima0 = [r["time"] for r in mc.mc_batch_run(probe, [("min_time", None)] * len(specs))]
    mc.mc_batch_destroy(probe)
    queries0 = [("min_time", None) if sp.meta["query"] else
                ("check", round(t * sp.meta["t_frac_milli"] / 1000)) for sp, t in zip(specs, optima0)]
    tuned = AT.tune_batch(specs, queries0, space={"blocks_per_sm": [0, 1, 2], "load_factor_pct": [25, 50]},
                          reps=1, cache={}, path=os.path.join(tempfile.gettempdir(), "mc_autotune_c4.json"))
    opts = mc.mc_options_default(timing=1, **tuned["options"])
    stream = torch.cuda.Stream(device)
    batch = mc.mc_batch_create(specs, opts, stream=stream)
    # the check thresholds are fractions of each instance's optimum: take the
    # optima from an untimed all-min-time run
    optima = [r["time"] for r in mc.mc_batch_run(batch, [("min_time", None)] * len(specs))]
    queries = [("min_time", None) if sp.meta["query"] else
               ("check", round(t * sp.meta["t_frac_milli"] / 1000)) for sp, t in zip(specs, optima)]
    for _ in range(args.warmup):
        ref = mc.mc_batch_run(batch, queries)
    torch.cuda.synchronize()
    barrier(device)
    sampler = ClockSampler(local)
    sampler.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    states = 0
    for k in range(args.steps):
        ev[k][0].record(stream)
        res = mc.mc_batch_run(batch, queries)
        ev[k][1].record(stream)
        states += sum(r["states"] for r in res)
        assert [r["status"] for r in res] == [0] * len(res)
        assert [(r["time"], r["states"]) for r in res] == [(r["time"], r["states"]) for r in ref]
    torch.cuda.synchronize()
    barrier(device)
    clocks = sampler.stop()
    batch_ms = [a.elapsed_time(b) for a, b in ev]
    dev_ms = sum(batch_ms)
    dev_ms_max = reduce_scalar(dev_ms, "max", device)
    states_all = reduce_scalar(states, "sum", device)
    value = states_all / (dev_ms_max / 1000.0)

    # one query at a time on the single-model entry points (models created
    # untimed, with the library's default launch shape -- the batch's tuned
    # options suit its lockstep steps, not a lone query); latency of query k
    # when all arrive together = sum of the service times of queries 0..k
    seq_opts = mc.mc_options_default(timing=1)
    models = [mc.mc_model_create(sp.with_key_bits(128), seq_opts, stream=stream) for sp in specs]
    for m in models:
        mc.mc_reserve(m)
    service = []
    seq_states = 0
    for m, (kind, T) in zip(models, queries):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        r = mc.mc_min_time(m, trace=False) if kind == "min_time" else mc.mc_check(m, T, trace=False)
        b.record(stream)
        b.synchronize()
        service.append(a.elapsed_time(b))
        seq_states += r["states"]
    seq_total = sum(service)
    cum, acc = [], 0.0
    for x in service:
        acc += x
        cum.append(acc)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": dev_ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u128", "data": "synthetic (seeded model descriptions)",
        "config": {"workload": "c4: 256 instances, G=2^U{6..12}, P in {2,4,8}, WG 2^0..2^8, TS 2^0..2^4, "
                               "cost U{1..16}, speeds U{1..3} (splitmix64 seed 2305091304), GREEDY; "
                               "half mc_min_time, half mc_check at round(U[0.8,1.2] x T_min)",
                   "query": "one mc_batch_run per step (one persistent launch)",
                   "autotuned_options": tuned["options"], "autotune_ms": tuned["timings"],
                   "sequential_options": "library defaults (occupancy-maximum grid, load factor 25%)",
                   "states_per_step": states / args.steps},
        "batched": {"ms_per_batch": dev_ms_max / args.steps, "states_per_s": value,
                    "query_latency_ms_p50": percentile(batch_ms, 50),
                    "query_latency_ms_p99": percentile(batch_ms, 99)},
        "sequential": {"ms_total": seq_total, "states_per_s": seq_states / (seq_total / 1000.0),
                       "service_ms_p50": percentile(service, 50), "service_ms_p99": percentile(service, 99),
                       "latency_all_arrive_together_ms_p50": percentile(cum, 50),
                       "latency_all_arrive_together_ms_p99": percentile(cum, 99)},
        "speedup_vs_sequential": seq_total / (dev_ms_max / args.steps),
        "gpu_launches": args.steps, "clocks": clocks,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def run_c5(args):
    """Served queries: Poisson arrivals of min-time queries on models drawn as
    the large single query (G=4096, P=8, WG 2^0..2^9, TS 2^0..2^5, cost
    U{1..16} with a new seed per query, GREEDY, 128-bit keys), at each rate of
    --rates, answered by the request loop (mc_server_*), against the same
    arrivals served one query at a time on the single-model entry point."""
    import torch

    from paper_2305_09130_gb300 import mc

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    rates = [float(x) for x in args.rates.split(",")]
    rng = W.SplitMix64(2305091305)
    free_b, _tot = torch.cuda.mem_get_info()
    pool = int(min(free_b * 0.6, 120 << 30))
    srv = mc.mc_server_create(slots=args.slots, pool_bytes=pool)

    def make_query(k):
        return W.c3(G=4096, rule=W.GREEDY, seed=2305091305 * 1000003 + k, key_bits=128)

    # one-query-at-a-time service times on a sample of the same query stream:
    # end to end as a caller of the single-model API sees it (create the
    # model from host arrays, mc_min_time, read the result, destroy; the
    # library's own pooled allocator, its fastest path), and the
    # exploration's device time alone
    sample = [make_query(10_000_000 + k) for k in range(args.c5_sample)]
    for sp in sample[:3]:  # warm the allocator and the library
        m = mc.mc_model_create(sp, allocator=None)
        mc.mc_min_time(m, trace=False)
        mc.mc_model_destroy(m)
    service, service_dev, service_states = [], [], []
    for sp in sample:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        m = mc.mc_model_create(sp, allocator=None)
        r = mc.mc_min_time(m, trace=False)
        mc.mc_model_destroy(m)
        service.append(time.perf_counter() - t0)
        service_states.append(r["states"])
        m = mc.mc_model_create(sp)
        mc.mc_reserve(m)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record()
        mc.mc_min_time(m, trace=False)
        b.record()
        b.synchronize()
        service_dev.append(a.elapsed_time(b) / 1000.0)
        mc.mc_model_destroy(m)

    sweep = []
    qid = 0
    for rate in rates:
        n = int(min(args.c5_queries, max(20, rate * args.c5_seconds)))
        arrivals, t = [], 0.0
        for _ in range(n):
            u = (rng.next() >> 11) / float(1 << 53)
            t += -math.log(1.0 - u) / rate
            arrivals.append(t)
        specs = [make_query(qid + k) for k in range(n)]
        qid += n
        got = {}
        sampler = ClockSampler(local)
        sampler.start()
        t0 = time.perf_counter()
        for k in range(n):
            while time.perf_counter() - t0 < arrivals[k]:
                for r in mc.mc_server_poll(srv, wait_ms=0):
                    got[r["ticket"]] = r
                time.sleep(0.0002)
            mc.mc_server_submit(srv, specs[k], "min_time")
        while len(got) < n:
            for r in mc.mc_server_poll(srv, wait_ms=20):
                got[r["ticket"]] = r
            if time.perf_counter() - t0 > arrivals[-1] + 600:
                raise SystemExit(f"served run at {rate}/s did not finish: {mc.mc_server_status(srv)}")
        clocks = sampler.stop()
        res = list(got.values())
        assert all(r["status"] == 0 for r in res)
        lat = [1000.0 * (r["done_s"] - r["submit_s"]) for r in res]
        first = min(r["submit_s"] for r in res)
        last = max(r["done_s"] for r in res)
        # the same arrivals served FIFO one at a time, service times cycling
        # through the measured sample (end to end; and device time only)
        def fifo(times):
            clock, out = 0.0, []
            for k, a in enumerate(arrivals):
                clock = max(clock, a) + times[k % len(times)]
                out.append(1000.0 * (clock - a))
            return clock, out

        clock, seq_lat = fifo(service)
        clock_dev, seq_lat_dev = fifo(service_dev)
        sweep.append({
            "rate_per_s": rate, "queries": n,
            "served": {"throughput_qps": n / (last - first), "latency_ms_p50": percentile(lat, 50),
                       "latency_ms_p99": percentile(lat, 99),
                       "states_per_s": sum(r["states"] for r in res) / (last - first),
                       "ran_alone": sum(r["path"] == "alone" for r in res)},
            "sequential": {"throughput_qps": n / (clock - arrivals[0]) if clock > arrivals[0] else None,
                           "latency_ms_p50": percentile(seq_lat, 50), "latency_ms_p99": percentile(seq_lat, 99)},
            "sequential_device_only": {
                "throughput_qps": n / (clock_dev - arrivals[0]) if clock_dev > arrivals[0] else None,
                "latency_ms_p50": percentile(seq_lat_dev, 50), "latency_ms_p99": percentile(seq_lat_dev, 99)},
            "clocks": clocks,
        })
    status = mc.mc_server_status(srv)
    mc.mc_server_destroy(srv)
    top = sweep[-1]
    line = {
        "metric": "served queries: throughput with p50/p99 latency", "value": top["served"]["throughput_qps"],
        "unit": "queries/s", "n_gpus": 1, "steps": len(rates), "warmup": 0,
        "ms_per_step": None, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "u128", "data": "synthetic (seeded model per query)",
        "config": {"workload": "c5: min-time queries on G=4096, P=8, WG 2^0..2^9, TS 2^0..2^5, "
                               "cost U{1..16} (new splitmix64 seed per query), GREEDY, 128-bit keys; "
                               "Poisson arrivals", "slots": args.slots, "pool_bytes": pool,
                   "sequential_service_ms_mean": 1000.0 * sum(service) / len(service),
                   "sequential_device_ms_mean": 1000.0 * sum(service_dev) / len(service_dev),
                   "sequential_sample": len(service),
                   "note": "sequential latencies: the same arrival times served FIFO one at a time, with "
                           "service times cycling through the measured single-query sample; 'sequential' "
                           "times each query end to end through the single-model C-ABI (create, "
                           "mc_min_time, destroy), as the served latency is measured from submit to "
                           "result; 'sequential_device_only' counts the exploration's device time alone"},
        "sweep": sweep, "device_loop_launches": status["launches"], "clocks": top["clocks"],
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def main(argv=None):
    p = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=100)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--mode", choices=["single", "lower", "bisect"], default="lower")
    p.add_argument("--prune", type=int, default=0)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-random-roofline", action="store_true")
    p.add_argument("--load-factor", type=int, default=0,
                   help="visited-set load factor in percent (0: the autotuner picks it for c2_star)")
    p.add_argument("--probe-scheme", choices=["tune", "auto", "split", "one_call"], default="tune",
                   help="visited-set insert of the exploration kernel (tune: the autotuner picks it)")
    p.add_argument("--no-log-tags", action="store_true",
                   help="untagged frontier log: blocks write their entries before they arrive at a level")
    p.add_argument("--rates", default="10,30,100,300,1000", help="c5 arrival rates (queries/s)")
    p.add_argument("--slots", type=int, default=512, help="c5 requests on the device at once")
    p.add_argument("--c5-seconds", type=float, default=10.0, help="c5 arrivals per rate span")
    p.add_argument("--c5-queries", type=int, default=10000, help="c5 queries per rate at most")
    p.add_argument("--c5-sample", type=int, default=48, help="c5 single-query service sample")
    p.add_argument("--workload", choices=sorted(WORKLOADS) + ["c4", "c5"] + sorted(PE_WORKLOADS),
                   default="c2_star",
                   help="profiling aid; the benchmark line is c2_star")
    p.add_argument("--query", choices=["min_time", "count", "swarm"], default="min_time")
    p.add_argument("--swarm-walks", type=int, default=1 << 20, help="random runs per swarm round")
    args = p.parse_args(argv)
    if args.warmup < 3:
        p.error("--warmup must be >= 3")
    if args.impl == "reference":
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
