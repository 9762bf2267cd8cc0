"""Autotuner for the explorer's launch and table parameters, with a JSON cache.

The knobs are the runtime options of ``mc_options``, searched per engine:

* the level-synchronous engine: threads per block, blocks per SM (the
  persistent grid), the visited-set load factor, the probe scheme of the
  insert (split: pick a slot from the fetched bucket and issue every CAS of
  the round before resolving any; one call: the general insert per
  proposal), the frontier chunk a warp stages before it copies its winners
  out, and the lanes per state;
* the configuration engine (one block per configuration): threads per block
  and lanes per state;
* batches: the engine, and per engine the grid and load factor, or the
  threads per block and lanes per state;
* the processing-element level model: the lanes that expand one state (a
  quarter, half or whole warp) and the grid.

A
candidate is timed on the real query through the C-ABI (CUDA events recorded
by the library around its kernels), every candidate must return the same
answer as the default options (a tuning run never trades correctness), and
the fastest wins.  Results are cached per workload signature -- dispatch
rule, compute units, key width, domain sizes and the magnitude of the state
bound -- so models of the same shape reuse them.

Cache file: ``$MC_AUTOTUNE_CACHE`` or ``./mc_autotune.json``.
"""
from __future__ import annotations

import itertools
import json
import math
import os
import time
from typing import Callable, Dict, List, Optional, Sequence

DEFAULT_SPACE = {
    "threads_per_block": [128, 256],
    "blocks_per_sm": [0, 2, 3],
    "load_factor_pct": [25, 50],
    "probe_scheme": [1, 2, 3],  # mc_probe_scheme: split, one call, CAS first
}
KNOBS = tuple(DEFAULT_SPACE) + ("engine", "stage_chunk", "unit_threads", "lanes_per_state")
# per engine (mc_engine: 1 level-synchronous, 2 one block per configuration)
LEVEL_SPACE = {
    "engine": [1],
    "blocks_per_sm": [0, 2],
    "load_factor_pct": [25, 50],
    "probe_scheme": [1, 2, 3, 4],  # split, one call, CAS first, CAS first with clearing
    "stage_chunk": [64, 128, 192],
}
CONFIG_SPACE = {
    "engine": [2],
    "unit_threads": [0, 128, 256, 512],
    "lanes_per_state": [0, 16],
}
BATCH_LEVEL_SPACE = {"engine": [1], "blocks_per_sm": [0, 1, 2], "load_factor_pct": [25, 50]}
BATCH_CONFIG_SPACE = {"engine": [2], "unit_threads": [0, 256, 512], "lanes_per_state": [0, 8]}


def cache_path() -> str:
    return os.environ.get("MC_AUTOTUNE_CACHE", os.path.join(os.getcwd(), "mc_autotune.json"))


def load_cache(path: Optional[str] = None) -> dict:
    path = path or cache_path()
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def save_cache(cache: dict, path: Optional[str] = None) -> None:
    path = path or cache_path()
    tmp = f"{path}.tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def signature(layout: dict, spec, query: str, batch: int = 1) -> str:
    """Shape of a workload as far as the knobs care."""
    bound = max(1, int(layout.get("state_bound", 1)))
    return (f"{query}|rule{spec.rule}|P{spec.P}|k{layout['key_bits']}|a{len(spec.wg_values)}"
            f"|b{len(spec.ts_values)}|L{layout['max_level']}|S2^{int(math.log2(bound))}|n{batch}")


def candidates(space=None) -> List[dict]:
    """Every combination of a space's values; a list of spaces gives the
    union of their candidates (one space per engine)."""
    space = space or DEFAULT_SPACE
    if isinstance(space, (list, tuple)):
        out, seen = [], set()
        for sp in space:
            for c in candidates(sp):
                key = json.dumps(c, sort_keys=True)
                if key not in seen:
                    seen.add(key)
                    out.append(c)
        return out
    names = [k for k in KNOBS if k in space] + sorted(k for k in space if k not in KNOBS)
    return [dict(zip(names, vals)) for vals in itertools.product(*(space[k] for k in names))]


def pick(timings: Dict[str, float]) -> str:
    """Key of the fastest candidate (ties: the first in sorted order)."""
    return min(sorted(timings), key=lambda k: timings[k])


def tune(measure: Callable[[dict], tuple], space=None, reps: int = 3) -> dict:
    """Generic search: ``measure(opts) -> (ms, answer)``.  Candidates whose
    answer differs from the first candidate's are rejected."""
    timings, answers, cands = {}, {}, candidates(space)
    reference = None
    for c in cands:
        key = json.dumps(c, sort_keys=True)
        best = math.inf
        for _ in range(reps):
            try:
                ms, ans = measure(c)
            except RuntimeError:  # options the library refuses for this model
                best = math.inf
                break
            if reference is None:
                reference = ans
            if ans != reference:
                best = math.inf
                break
            best = min(best, ms)
        if best < math.inf:
            timings[key] = best
            answers[key] = ans
    if not timings:
        raise RuntimeError("no candidate reproduced the reference answer")
    win = pick(timings)
    return {"options": json.loads(win), "ms": timings[win], "timings": timings}


# ---------------------------------------------------------------- GPU front ends
def tune_query(spec, query: str = "min_time", T: Optional[int] = None, space=None, reps: int = 3,
               cache: Optional[dict] = None, path: Optional[str] = None) -> dict:
    """Tune the single-model query on `spec` ("count", "check" with T, or
    "min_time") and record the winner in the cache."""
    from . import mc

    mc.load()
    lay = mc.mc_model_layout(mc.mc_model_create(spec, allocator=None))
    sig = signature(lay, spec, query)
    cache = load_cache(path) if cache is None else cache
    if space is None:  # both engines where the configuration engine takes the model
        space = [LEVEL_SPACE] + ([CONFIG_SPACE] if lay["engine"] == mc.ENGINE["config"] else [])

    def measure(c):
        m = mc.mc_model_create(spec, mc.mc_options_default(timing=1, **c))
        run = {"count": lambda: mc.mc_count_states(m),
               "check": lambda: mc.mc_check(m, T, trace=False),
               "min_time": lambda: mc.mc_min_time(m, trace=False)}[query]
        run()
        mc.mc_reset_stats(m)
        ans = run()
        ms = mc.mc_get_stats(m)["explore_ms"]
        mc.mc_model_destroy(m)
        if isinstance(ans, dict):
            ans = {k: v for k, v in ans.items() if k != "trace"}
        return ms, ans

    out = tune(measure, space, reps)
    cache[sig] = {"options": out["options"], "ms": out["ms"], "when": time.time()}
    save_cache(cache, path)
    return {"signature": sig, **out}


def tune_batch(specs, queries, space=None, reps: int = 2, cache: Optional[dict] = None,
               path: Optional[str] = None) -> dict:
    """Tune one batched launch of `queries` on `specs`."""
    from . import mc

    mc.load()
    # the lockstep kernel has one block size and one probe scheme; the
    # configuration engine is tried where it takes every instance
    if space is None:
        space = [BATCH_LEVEL_SPACE, BATCH_CONFIG_SPACE]
    elif isinstance(space, dict):
        space = {k: v for k, v in space.items() if k not in ("threads_per_block", "probe_scheme")}
    lay = mc.mc_model_layout(mc.mc_model_create(specs[0].with_key_bits(128), allocator=None))
    sig = signature(lay, specs[0], "batch", len(specs))
    cache = load_cache(path) if cache is None else cache

    def measure(c):
        b = mc.mc_batch_create(specs, mc.mc_options_default(timing=1, **c))
        mc.mc_batch_run(b, queries)
        t0 = mc.mc_batch_get_stats(b)["explore_ms"]
        res = mc.mc_batch_run(b, queries)
        ms = mc.mc_batch_get_stats(b)["explore_ms"] - t0
        mc.mc_batch_destroy(b)
        return ms, [(r["status"], r["time"], r["states"], r["key"]) for r in res]

    out = tune(measure, space, reps)
    cache[sig] = {"options": out["options"], "ms": out["ms"], "when": time.time()}
    save_cache(cache, path)
    return {"signature": sig, **out}


PE_SPACE = {
    "lanes_per_state": [8, 16, 32],
    "blocks_per_sm": [0, 1, 2],
}


def tune_pe(spec, query: str = "min_time", space=None, reps: int = 2, cache: Optional[dict] = None,
            path: Optional[str] = None) -> dict:
    """Tune the PE-level model's query ("count" or "min_time"): lanes per
    state (the warp tile that expands one state) and the persistent grid.
    Candidates whose tile cannot hold the model's successors are skipped."""
    from . import mc

    mc.load()
    space = dict(space or PE_SPACE)
    probe = mc.mc_pe_model_create(spec, stream=0)
    lay = mc.mc_pe_model_layout(probe)
    lanes = spec.P * lay["mask_bits"] + spec.P + 1
    fits = lambda t: -(-lanes // t) <= (1 if t >= 32 else 2 if t == 16 else 3)
    space["lanes_per_state"] = [t for t in space.get("lanes_per_state", [0]) if t == 0 or fits(t)]
    sig = (f"pe|{query}|P{spec.P}|m{lay['mask_bits']}|a{spec.a}|b{spec.b}|L{lay['max_level']}"
           f"|k{lay['used_bits']}")
    cache = load_cache(path) if cache is None else cache
    grown = {}

    def measure(c):
        m = mc.mc_pe_model_create(spec, mc.mc_options_default(timing=1, **c, **grown))
        run = {"count": lambda: mc.mc_pe_count_states(m),
               "min_time": lambda: mc.mc_pe_min_time(m, trace=False)}[query]
        run()
        if not grown:  # later candidates start at the grown buffer sizes
            L = mc.mc_pe_model_layout(m)
            grown.update(log_capacity=L["log_capacity"], table_log2=L["table_slots"].bit_length() - 1)
        mc.mc_pe_reset_stats(m)
        ans = run()
        ms = mc.mc_pe_get_stats(m)["explore_ms"]
        mc.mc_pe_model_destroy(m)
        return ms, ans

    out = tune(measure, space, reps)
    cache[sig] = {"options": out["options"], "ms": out["ms"], "when": time.time()}
    save_cache(cache, path)
    return {"signature": sig, **out}


def options_for(spec, query: str = "min_time", batch: int = 1, path: Optional[str] = None,
                **overrides):
    """mc_options for `spec`: the cached winner for its signature (if any)
    with `overrides` applied on top."""
    from . import mc

    lay = mc.mc_model_layout(mc.mc_model_create(spec if batch == 1 else spec.with_key_bits(128),
                                                allocator=None))
    hit = load_cache(path).get(signature(lay, spec, "batch" if batch > 1 else query, batch))
    opts = dict(hit["options"]) if hit else {}
    opts.update(overrides)
    return mc.mc_options_default(**opts)
