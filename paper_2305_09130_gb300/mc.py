"""Python binding of the explorer's C-ABI (include/mc.h).

Argument marshalling only: every function forwards to the function of the
same name in ``libmcgpu.so``; every step of a query runs in the library's
CUDA kernels.  PyTorch supplies device memory (the caching allocator, through
``mc_set_allocator``) and the stream.  There is no CPU fallback: if the
library is missing or no CUDA device is usable, the calls raise.
"""
from __future__ import annotations

import atexit
import ctypes as C
import os
import threading
import weakref
from typing import Optional

from . import build as _build

MC_OK = 0
MC_ERR_INVAL = -1
MC_ERR_NOMEM = -2
MC_ERR_TABLE_FULL = -3
MC_ERR_FRONTIER = -4
MC_ERR_TIMEOUT = -5
MC_ERR_CUDA = -6
MC_ERR_OVERFLOW = -7
MC_FREE, MC_GREEDY = 0, 1
SEARCH = {"single": 0, "lower": 1, "bisect": 2}
PROBE = {"auto": 0, "split": 1, "one_call": 2, "cas_first": 3, "cas_clear": 4}  # mc_probe_scheme
ENGINE = {"auto": 0, "level": 1, "config": 2}  # mc_engine
NO_LIMIT = (1 << 64) - 1

U32P = C.POINTER(C.c_uint32)


class McModelDesc(C.Structure):
    _fields_ = [("n_wg", C.c_uint32), ("n_ts", C.c_uint32), ("P", C.c_uint32),
                ("wg_values", U32P), ("ts_values", U32P), ("n_workgroups", U32P),
                ("cost", U32P), ("speed", U32P), ("rule", C.c_uint32), ("key_bits", C.c_uint32)]


class McOptions(C.Structure):
    _fields_ = [("prune", C.c_uint32), ("early_exit", C.c_uint32), ("search", C.c_uint32),
                ("refine", C.c_uint32), ("sim_seed", C.c_uint64), ("sim_walks", C.c_uint32),
                ("load_factor_pct", C.c_uint32), ("table_log2", C.c_uint32),
                ("threads_per_block", C.c_uint32), ("blocks_per_sm", C.c_uint32),
                ("max_probes", C.c_uint32), ("log_capacity", C.c_uint64),
                ("barrier_timeout_ns", C.c_uint64), ("debug_barrier_extra", C.c_uint32),
                ("timing", C.c_uint32), ("lanes_per_state", C.c_uint32),
                ("probe_scheme", C.c_uint32), ("no_log_tags", C.c_uint32), ("engine", C.c_uint32),
                ("unit_threads", C.c_uint32), ("stage_chunk", C.c_uint32)]


class McCheckResult(C.Structure):
    _fields_ = [("holds", C.c_uint32), ("levels", C.c_uint32), ("states", C.c_uint64),
                ("cex_time", C.c_uint64), ("cex_wg_index", C.c_uint32),
                ("cex_ts_index", C.c_uint32), ("cex_wg", C.c_uint32), ("cex_ts", C.c_uint32),
                ("cex_level", C.c_uint32), ("key_words", C.c_uint32),
                ("cex_key", C.c_uint64 * 2)]


class McMinResult(C.Structure):
    _fields_ = [("t_min", C.c_uint64), ("t_ini", C.c_uint64), ("wg_index", C.c_uint32),
                ("ts_index", C.c_uint32), ("wg", C.c_uint32), ("ts", C.c_uint32),
                ("states", C.c_uint64), ("checks", C.c_uint32), ("level", C.c_uint32),
                ("witness_key", C.c_uint64 * 2)]


class McLayout(C.Structure):
    _fields_ = [("key_bits", C.c_uint32), ("key_words", C.c_uint32), ("used_bits", C.c_uint32),
                ("P", C.c_uint32), ("n_bits", C.c_uint32), ("ts_bits", C.c_uint32),
                ("wg_bits", C.c_uint32), ("ts_shift", C.c_uint32), ("wg_shift", C.c_uint32),
                ("max_level", C.c_uint32), ("n_shift", C.c_uint32 * 16),
                ("table_slots", C.c_uint64), ("log_capacity", C.c_uint64),
                ("max_width", C.c_uint64), ("state_bound", C.c_uint64),
                ("device_bytes", C.c_uint64), ("probe_scheme", C.c_uint32), ("log_tag_bits", C.c_uint32),
                ("engine", C.c_uint32), ("unit_threads", C.c_uint32), ("unit_width", C.c_uint64)]


class McSwarmResult(C.Structure):
    _fields_ = [("best_time", C.c_uint64), ("first_time", C.c_uint64), ("wg_index", C.c_uint32),
                ("ts_index", C.c_uint32), ("wg", C.c_uint32), ("ts", C.c_uint32), ("rounds", C.c_uint32),
                ("key_words", C.c_uint32), ("walks", C.c_uint64), ("best_walk", C.c_uint64),
                ("first_trail_ms", C.c_double), ("total_ms", C.c_double)]


class McStats(C.Structure):
    _fields_ = [("explore_launches", C.c_uint64), ("other_launches", C.c_uint64),
                ("states", C.c_uint64), ("h2d_bytes", C.c_uint64), ("d2h_bytes", C.c_uint64),
                ("explore_ms", C.c_double), ("device_steps", C.c_uint64), ("probes", C.c_uint64),
                ("graph_launches", C.c_uint64)]


class McQuery(C.Structure):
    _fields_ = [("kind", C.c_uint32), ("reserved", C.c_uint32), ("T", C.c_uint64)]


class McBatchResult(C.Structure):
    _fields_ = [("status", C.c_int32), ("kind", C.c_uint32), ("holds", C.c_uint32),
                ("levels", C.c_uint32), ("states", C.c_uint64), ("checks", C.c_uint32),
                ("level", C.c_uint32), ("time", C.c_uint64), ("t_ini", C.c_uint64),
                ("wg_index", C.c_uint32), ("ts_index", C.c_uint32), ("wg", C.c_uint32),
                ("ts", C.c_uint32), ("key", C.c_uint64 * 2)]


MC_QUERY_CHECK, MC_QUERY_MIN_TIME = 0, 1


class McServerConfig(C.Structure):
    _fields_ = [("slots", C.c_uint32), ("reserved0", C.c_uint32), ("pool_bytes", C.c_uint64),
                ("idle_ns", C.c_uint64), ("solo_states", C.c_uint64), ("reserved", C.c_uint64 * 3)]


class McServerResult(C.Structure):
    _fields_ = [("ticket", C.c_uint64), ("result", McBatchResult), ("submit_s", C.c_double),
                ("admit_s", C.c_double), ("done_s", C.c_double), ("path", C.c_uint32),
                ("reserved", C.c_uint32)]

class McPeModelDesc(C.Structure):
    _fields_ = [("n_wg", C.c_uint32), ("n_ts", C.c_uint32), ("P", C.c_uint32),
                ("wg_values", C.POINTER(C.c_uint32)), ("ts_values", C.POINTER(C.c_uint32)),
                ("n_workgroups", C.POINTER(C.c_uint32)), ("pes", C.POINTER(C.c_uint32)),
                ("prog_off", C.POINTER(C.c_uint32)), ("seg_ticks", C.POINTER(C.c_uint32)),
                ("seg_pes", C.POINTER(C.c_uint32))]


class McPeLayout(C.Structure):
    _fields_ = [("used_bits", C.c_uint32), ("P", C.c_uint32), ("wg_bits", C.c_uint32),
                ("ts_bits", C.c_uint32), ("level_bits", C.c_uint32), ("unit_bits", C.c_uint32),
                ("n_bits", C.c_uint32), ("pc_bits", C.c_uint32), ("mask_bits", C.c_uint32),
                ("tile", C.c_uint32), ("wg_shift", C.c_uint32), ("ts_shift", C.c_uint32),
                ("level_shift", C.c_uint32), ("max_level", C.c_uint32),
                ("unit_shift", C.c_uint32 * 8), ("max_steps", C.c_uint64),
                ("table_slots", C.c_uint64), ("log_capacity", C.c_uint64),
                ("device_bytes", C.c_uint64)]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)

_lib = None
_lock = threading.Lock()
_live = weakref.WeakSet()


@atexit.register
def _destroy_live_models():
    # free device buffers while PyTorch (the allocator behind them) is alive
    for m in list(_live):
        try:
            if isinstance(m, PeModel):
                mc_pe_model_destroy(m)
            else:
                mc_model_destroy(m)
        except Exception:
            pass


class MCError(RuntimeError):
    def __init__(self, code: int, where: str, detail: str = ""):
        self.code = code
        msg = f"{where}: {mc_strerror(code)} ({code})"
        if detail:
            msg += f": {detail}"
        super().__init__(msg)


def library_path() -> str:
    return _build.LIB


def load(build: bool = True):
    """Load libmcgpu.so, building it first when missing or stale."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if build:
            _build.build()
        if not os.path.exists(_build.LIB):
            raise RuntimeError(f"CUDA library missing: {_build.LIB}")
        L = C.CDLL(_build.LIB)
        P = C.c_void_p
        sig = {
            "mc_options_default": (None, [C.POINTER(McOptions)]),
            "mc_model_create": (C.c_int, [C.POINTER(McModelDesc), C.POINTER(McOptions), C.POINTER(P)]),
            "mc_model_destroy": (None, [P]),
            "mc_set_options": (C.c_int, [P, C.POINTER(McOptions)]),
            "mc_set_stream": (C.c_int, [P, P]),
            "mc_set_allocator": (C.c_int, [P, ALLOC_FN, FREE_FN, P]),
            "mc_reserve": (C.c_int, [P]),
            "mc_model_layout": (C.c_int, [P, C.POINTER(McLayout)]),
            "mc_check": (C.c_int, [P, C.c_uint64, C.POINTER(McCheckResult), C.POINTER(P)]),
            "mc_min_time": (C.c_int, [P, C.POINTER(McMinResult), C.POINTER(P)]),
            "mc_count_states": (C.c_int, [P, C.POINTER(C.c_uint64)]),
            "mc_simulate": (C.c_int, [P, C.c_uint64, C.c_uint32, C.POINTER(C.c_uint64)]),
            "mc_swarm": (C.c_int, [P, C.c_uint64, C.c_uint32, C.c_uint32, C.POINTER(McSwarmResult),
                                   C.POINTER(P)]),
            "mc_last_widths": (C.c_int, [P, C.POINTER(C.c_uint64), C.c_uint32, C.POINTER(C.c_uint32)]),
            "mc_get_stats": (C.c_int, [P, C.POINTER(McStats)]),
            "mc_batch_create": (C.c_int, [C.POINTER(McModelDesc), C.c_uint32, C.POINTER(McOptions),
                                          C.POINTER(P)]),
            "mc_batch_destroy": (None, [P]),
            "mc_batch_set_stream": (C.c_int, [P, P]),
            "mc_batch_set_allocator": (C.c_int, [P, ALLOC_FN, FREE_FN, P]),
            "mc_batch_device_bytes": (C.c_int, [P, C.POINTER(C.c_uint64)]),
            "mc_batch_run": (C.c_int, [P, C.POINTER(McQuery), C.POINTER(McBatchResult)]),
            "mc_batch_trace": (C.c_int, [P, C.c_uint32, C.POINTER(C.c_uint64), C.c_uint32,
                                         C.POINTER(C.c_uint32)]),
            "mc_batch_get_stats": (C.c_int, [P, C.POINTER(McStats)]),
            "mc_batch_last_error": (C.c_char_p, [P]),
            "mc_server_create": (C.c_int, [C.POINTER(McServerConfig), C.POINTER(McOptions), C.POINTER(P)]),
            "mc_server_submit": (C.c_int, [P, C.POINTER(McModelDesc), C.POINTER(McQuery),
                                           C.POINTER(C.c_uint64)]),
            "mc_server_poll": (C.c_int, [P, C.POINTER(McServerResult), C.c_uint32, C.POINTER(C.c_uint32),
                                         C.c_uint32]),
            "mc_server_status": (C.c_int, [P, C.POINTER(C.c_uint32), C.POINTER(C.c_uint32),
                                           C.POINTER(C.c_uint64)]),
            "mc_server_destroy": (None, [P]),
            "mc_measure_random_access": (C.c_int, [C.c_uint64, C.c_uint64, C.c_int,
                                                   C.POINTER(C.c_double), C.POINTER(C.c_double)]),
            "mc_check_noalloc": (C.c_int, [C.POINTER(McModelDesc), C.c_uint64, C.c_uint32, C.c_uint32,
                                           P, C.POINTER(McCheckResult)]),
            "mc_reset_stats": (C.c_int, [P]),
            "mc_pe_model_create": (C.c_int, [C.POINTER(McPeModelDesc), C.POINTER(McOptions),
                                             C.POINTER(P)]),
            "mc_pe_model_destroy": (None, [P]),
            "mc_pe_set_stream": (C.c_int, [P, P]),
            "mc_pe_model_layout": (C.c_int, [P, C.POINTER(McPeLayout)]),
            "mc_pe_check": (C.c_int, [P, C.c_uint64, C.POINTER(McCheckResult), C.POINTER(P)]),
            "mc_pe_min_time": (C.c_int, [P, C.POINTER(McMinResult), C.POINTER(P)]),
            "mc_pe_count_states": (C.c_int, [P, C.POINTER(C.c_uint64)]),
            "mc_pe_last_widths": (C.c_int, [P, C.POINTER(C.c_uint64), C.c_uint32,
                                            C.POINTER(C.c_uint32)]),
            "mc_pe_get_stats": (C.c_int, [P, C.POINTER(McStats)]),
            "mc_pe_reset_stats": (C.c_int, [P]),
            "mc_pe_last_error": (C.c_char_p, [P]),
            "mc_trace_length": (C.c_int, [P]),
            "mc_trace_key_words": (C.c_uint32, [P]),
            "mc_trace_states": (C.POINTER(C.c_uint64), [P]),
            "mc_trace_free": (None, [P]),
            "mc_strerror": (C.c_char_p, [C.c_int]),
            "mc_release_cached": (C.c_int, []),
            "mc_set_pool_retention": (C.c_int, [C.c_uint64]),
            "mc_last_error": (C.c_char_p, [P]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
        return L


def mc_release_cached():
    """Give back the library's cached device blocks and pinned host blocks."""
    rc = load(build=False).mc_release_cached()
    if rc != MC_OK:
        raise MCError(rc, "mc_release_cached")


def mc_set_pool_retention(nbytes: int):
    """Bytes of freed device memory the library's pools keep for later models
    (1 GiB by default); see mc_set_pool_retention in mc.h."""
    rc = load(build=False).mc_set_pool_retention(int(nbytes))
    if rc != MC_OK:
        raise MCError(rc, "mc_set_pool_retention")


def mc_strerror(code: int) -> str:
    return load(build=False).mc_strerror(code).decode() if _lib else f"error {code}"


_OPTION_FIELDS = frozenset(f[0] for f in McOptions._fields_ if f[0] != "reserved")


def mc_options_default(**overrides) -> McOptions:
    o = McOptions()
    load().mc_options_default(C.byref(o))
    for k, v in overrides.items():
        if k not in _OPTION_FIELDS:  # ctypes would keep an unknown name as a plain attribute
            raise TypeError(f"unknown mc_options field {k!r}")
        if k == "search" and isinstance(v, str):
            v = SEARCH[v]
        if k == "probe_scheme" and isinstance(v, str):
            v = PROBE[v]
        if k == "engine" and isinstance(v, str):
            v = ENGINE[v]
        setattr(o, k, int(v))
    return o


class Model:
    """Owns an ``mc_model*``; destroyed with ``mc_model_destroy``."""

    def __init__(self, handle: int, spec=None):
        self.handle = C.c_void_p(handle)
        self.spec = spec
        self._callbacks = None
        self._layout = None
        _live.add(self)

    def __del__(self):
        try:
            mc_model_destroy(self)
        except Exception:
            pass

    def _check(self, rc: int, where: str):
        if rc != MC_OK:
            detail = ""
            if self.handle:
                detail = load(build=False).mc_last_error(self.handle).decode()
            raise MCError(rc, where, detail)


def _u32(xs):
    return (C.c_uint32 * len(xs))(*[int(x) for x in xs])


def mc_model_create(spec, options: Optional[McOptions] = None, allocator: Optional[str] = "torch",
                    stream=None) -> Model:
    """Create a model from a ``workloads.ModelSpec`` (or any object with the
    same fields).  ``allocator``: "torch" (PyTorch caching allocator),
    "cuda" (the library's own stream-ordered pool) or None (same as "cuda")."""
    L = load()
    arrs = (_u32(spec.wg_values), _u32(spec.ts_values), _u32(spec.n_workgroups), _u32(spec.cost),
            _u32(spec.speed))
    d = McModelDesc(len(spec.wg_values), len(spec.ts_values), spec.P, arrs[0], arrs[1], arrs[2],
                    arrs[3], arrs[4], spec.rule, getattr(spec, "key_bits", 0))
    h = C.c_void_p()
    rc = L.mc_model_create(C.byref(d), C.byref(options) if options is not None else None, C.byref(h))
    if rc != MC_OK:
        raise MCError(rc, "mc_model_create")
    m = Model(h.value, spec)
    if allocator == "torch":
        mc_set_allocator(m, "torch")
    if stream is not None:
        mc_set_stream(m, stream)
    return m


def mc_model_destroy(model: Model):
    if model.handle and model.handle.value:
        load(build=False).mc_model_destroy(model.handle)
        model.handle = C.c_void_p()


def mc_set_options(model: Model, options: McOptions):
    model._check(load().mc_set_options(model.handle, C.byref(options)), "mc_set_options")


def mc_set_stream(model: Model, stream):
    """``stream``: a torch.cuda.Stream, a raw cudaStream_t int, or None."""
    raw = getattr(stream, "cuda_stream", stream)
    model._check(load().mc_set_stream(model.handle, C.c_void_p(raw or 0)), "mc_set_stream")


def mc_set_allocator(model: Model, kind: str = "torch"):
    """Route the model's device allocations through PyTorch's caching allocator."""
    if kind != "torch":
        raise ValueError("only the 'torch' allocator can be installed from Python")
    import torch

    device = torch.cuda.current_device()

    def _alloc(nbytes, stream, _ctx):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), device, int(stream or 0))
        except Exception:
            return None

    def _free(ptr, _nbytes, _stream, _ctx):
        torch.cuda.caching_allocator_delete(int(ptr))

    cbs = (ALLOC_FN(_alloc), FREE_FN(_free))
    model._callbacks = cbs
    model._check(load().mc_set_allocator(model.handle, cbs[0], cbs[1], None), "mc_set_allocator")


def mc_reserve(model: Model):
    model._check(load().mc_reserve(model.handle), "mc_reserve")


def mc_model_layout(model: Model) -> dict:
    lay = McLayout()
    model._check(load().mc_model_layout(model.handle, C.byref(lay)), "mc_model_layout")
    out = {k: getattr(lay, k) for k, _t in McLayout._fields_ if k not in ("n_shift", "reserved")}
    out["n_shift"] = list(lay.n_shift[: lay.P])
    model._layout = out
    return out


def _take_trace(h: C.c_void_p):
    if not h.value:
        return None
    L = load(build=False)
    n = L.mc_trace_length(h)
    w = L.mc_trace_key_words(h)
    ptr = L.mc_trace_states(h)
    words = [ptr[k] for k in range(n * w)]
    L.mc_trace_free(h)
    if w == 1:
        return words
    return [words[2 * k] | (words[2 * k + 1] << 64) for k in range(n)]


def mc_check(model: Model, T: int, trace: bool = True) -> dict:
    r = McCheckResult()
    h = C.c_void_p()
    rc = load().mc_check(model.handle, int(T) & NO_LIMIT, C.byref(r), C.byref(h) if trace else None)
    model._check(rc, "mc_check")
    out = {"holds": bool(r.holds), "states": r.states, "levels": r.levels}
    if not r.holds:
        key = r.cex_key[0] | (r.cex_key[1] << 64)
        out.update(cex_time=r.cex_time, cex_i=r.cex_wg_index, cex_j=r.cex_ts_index, cex_wg=r.cex_wg,
                   cex_ts=r.cex_ts, cex_level=r.cex_level, cex_key=key)
        if trace:
            out["trace"] = _take_trace(h)
    return out


def mc_min_time(model: Model, trace: bool = True) -> dict:
    r = McMinResult()
    h = C.c_void_p()
    rc = load().mc_min_time(model.handle, C.byref(r), C.byref(h) if trace else None)
    model._check(rc, "mc_min_time")
    out = {"t_min": r.t_min, "t_ini": r.t_ini, "i": r.wg_index, "j": r.ts_index, "wg": r.wg,
           "ts": r.ts, "states": r.states, "checks": r.checks, "level": r.level,
           "witness_key": r.witness_key[0] | (r.witness_key[1] << 64)}
    if trace:
        out["trace"] = _take_trace(h)
    return out


def mc_count_states(model: Model) -> int:
    v = C.c_uint64()
    model._check(load().mc_count_states(model.handle, C.byref(v)), "mc_count_states")
    return v.value


def mc_simulate(model: Model, seed: int, walks: int = 1) -> int:
    v = C.c_uint64()
    model._check(load().mc_simulate(model.handle, int(seed) & NO_LIMIT, int(walks), C.byref(v)),
                 "mc_simulate")
    return v.value


def mc_swarm(model: Model, seed: int, walks_per_round: int, max_rounds: int = 64,
             trace: bool = True) -> dict:
    r = McSwarmResult()
    h = C.c_void_p()
    model._check(load().mc_swarm(model.handle, int(seed) & NO_LIMIT, int(walks_per_round),
                                 int(max_rounds), C.byref(r), C.byref(h) if trace else None), "mc_swarm")
    out = {k: getattr(r, k) for k, _t in McSwarmResult._fields_}
    out["i"], out["j"] = out.pop("wg_index"), out.pop("ts_index")
    if trace:
        out["trace"] = _take_trace(h)
    return out


def mc_last_widths(model: Model, cap: int = 1 << 16) -> list:
    buf = (C.c_uint64 * cap)()
    n = C.c_uint32()
    model._check(load().mc_last_widths(model.handle, buf, cap, C.byref(n)), "mc_last_widths")
    return list(buf[: min(n.value, cap)])


def mc_get_stats(model: Model) -> dict:
    """Counters since the last mc_reset_stats (mc_stats in mc.h).  With
    ``timing=1`` ``explore_ms`` is the CUDA-event time of the exploration
    kernels, one window around each query's chained launches; the windows'
    events are read here, not while a query runs."""
    st = McStats()
    model._check(load().mc_get_stats(model.handle, C.byref(st)), "mc_get_stats")
    return {k: getattr(st, k) for k, _t in McStats._fields_}


def mc_reset_stats(model: Model):
    model._check(load().mc_reset_stats(model.handle), "mc_reset_stats")


def mc_check_noalloc(spec, T: int, prune: bool = True, early_exit: bool = True, stream=None) -> dict:
    """mc_check for callers that cannot allocate device memory: the library's
    static scratch array holds every buffer (models up to
    MC_NOALLOC_SCRATCH_BYTES of scratch).  Same fields as mc_check, no trace."""
    arrs = (_u32(spec.wg_values), _u32(spec.ts_values), _u32(spec.n_workgroups), _u32(spec.cost),
            _u32(spec.speed))
    d = McModelDesc(len(spec.wg_values), len(spec.ts_values), spec.P, arrs[0], arrs[1], arrs[2],
                    arrs[3], arrs[4], spec.rule, getattr(spec, "key_bits", 0))
    raw = getattr(stream, "cuda_stream", stream)
    r = McCheckResult()
    rc = load().mc_check_noalloc(C.byref(d), int(T) & NO_LIMIT, int(prune), int(early_exit),
                                 C.c_void_p(raw or 0), C.byref(r))
    if rc != MC_OK:
        raise MCError(rc, "mc_check_noalloc")
    out = {"holds": bool(r.holds), "states": r.states, "levels": r.levels}
    if not r.holds:
        out.update(cex_time=r.cex_time, cex_i=r.cex_wg_index, cex_j=r.cex_ts_index, cex_wg=r.cex_wg,
                   cex_ts=r.cex_ts, cex_level=r.cex_level,
                   cex_key=r.cex_key[0] | (r.cex_key[1] << 64))
    return out


def mc_measure_random_access(buffer_bytes: int, accesses: int, op: int = 0) -> dict:
    """Random 32-byte sector reads (op 0), read + CAS (op 1) or CAS alone
    (op 2) per second over a buffer of buffer_bytes on the current device."""
    rate = C.c_double()
    ms = C.c_double()
    rc = load().mc_measure_random_access(int(buffer_bytes), int(accesses), int(op), C.byref(rate),
                                         C.byref(ms))
    if rc != MC_OK:
        raise MCError(rc, "mc_measure_random_access")
    return {"sectors_per_s": rate.value, "ms": ms.value, "gbs_32b": rate.value * 32 / 1e9}


class Batch:
    """Owns an ``mc_batch*`` (many models answered by one launch)."""

    def __init__(self, handle: int, specs):
        self.handle = C.c_void_p(handle)
        self.specs = specs
        self._callbacks = None
        self._keep = None
        _live.add(self)

    def __del__(self):
        try:
            mc_batch_destroy(self)
        except Exception:
            pass

    def _check(self, rc: int, where: str):
        if rc != MC_OK:
            detail = load(build=False).mc_batch_last_error(self.handle).decode() if self.handle else ""
            raise MCError(rc, where, detail)


def _descs(specs):
    keep = []
    arr = (McModelDesc * len(specs))()
    for k, spec in enumerate(specs):
        a = (_u32(spec.wg_values), _u32(spec.ts_values), _u32(spec.n_workgroups), _u32(spec.cost),
             _u32(spec.speed))
        keep.append(a)
        arr[k] = McModelDesc(len(spec.wg_values), len(spec.ts_values), spec.P, a[0], a[1], a[2], a[3],
                             a[4], spec.rule, 128)
    return arr, keep


def mc_batch_create(specs, options: Optional[McOptions] = None, allocator: Optional[str] = "torch",
                    stream=None) -> Batch:
    L = load()
    arr, keep = _descs(specs)
    h = C.c_void_p()
    rc = L.mc_batch_create(arr, len(specs), C.byref(options) if options is not None else None,
                           C.byref(h))
    if rc != MC_OK:
        raise MCError(rc, "mc_batch_create")
    b = Batch(h.value, list(specs))
    if allocator == "torch":
        import torch

        device = torch.cuda.current_device()

        def _alloc(nbytes, strm, _ctx):
            try:
                return torch.cuda.caching_allocator_alloc(int(nbytes), device, int(strm or 0))
            except Exception:
                return None

        def _free(ptr, _nbytes, _strm, _ctx):
            torch.cuda.caching_allocator_delete(int(ptr))

        b._callbacks = (ALLOC_FN(_alloc), FREE_FN(_free))
        b._check(L.mc_batch_set_allocator(b.handle, b._callbacks[0], b._callbacks[1], None),
                 "mc_batch_set_allocator")
    if stream is not None:
        raw = getattr(stream, "cuda_stream", stream)
        b._check(L.mc_batch_set_stream(b.handle, C.c_void_p(raw or 0)), "mc_batch_set_stream")
    return b


def mc_batch_destroy(batch: Batch):
    if batch.handle and batch.handle.value:
        load(build=False).mc_batch_destroy(batch.handle)
        batch.handle = C.c_void_p()


def mc_batch_device_bytes(batch: Batch) -> int:
    v = C.c_uint64()
    batch._check(load().mc_batch_device_bytes(batch.handle, C.byref(v)), "mc_batch_device_bytes")
    return v.value


def mc_batch_run(batch: Batch, queries) -> list:
    """queries: list of ("check", T) or ("min_time", None); one per model."""
    n = len(batch.specs)
    q = (McQuery * n)()
    for k, (kind, T) in enumerate(queries):
        q[k] = McQuery(MC_QUERY_MIN_TIME if kind == "min_time" else MC_QUERY_CHECK, 0,
                       int(T or 0) & NO_LIMIT)
    res = (McBatchResult * n)()
    batch._check(load().mc_batch_run(batch.handle, q, res), "mc_batch_run")
    return [_batch_result(r) for r in res]


def mc_batch_trace(batch: Batch, i: int) -> list:
    n = C.c_uint32()
    L = load()
    batch._check(L.mc_batch_trace(batch.handle, i, None, 0, C.byref(n)), "mc_batch_trace")
    buf = (C.c_uint64 * (2 * max(n.value, 1)))()
    batch._check(L.mc_batch_trace(batch.handle, i, buf, n.value, C.byref(n)), "mc_batch_trace")
    return [buf[2 * k] | (buf[2 * k + 1] << 64) for k in range(n.value)]


def mc_batch_get_stats(batch: Batch) -> dict:
    st = McStats()
    batch._check(load().mc_batch_get_stats(batch.handle, C.byref(st)), "mc_batch_get_stats")
    return {k: getattr(st, k) for k, _t in McStats._fields_}


def _batch_result(r) -> dict:
    return {"status": r.status, "kind": "min_time" if r.kind == 1 else "check", "holds": bool(r.holds),
            "levels": r.levels, "states": r.states, "checks": r.checks, "level": r.level,
            "time": r.time, "t_ini": r.t_ini, "i": r.wg_index, "j": r.ts_index, "wg": r.wg, "ts": r.ts,
            "key": r.key[0] | (r.key[1] << 64)}


class Server:
    """Owns an ``mc_server*`` (a request loop over a persistent device loop)."""

    def __init__(self, handle: int):
        self.handle = C.c_void_p(handle)
        _live.add(self)

    def __del__(self):
        try:
            mc_server_destroy(self)
        except Exception:
            pass


def mc_server_create(slots: int, pool_bytes: int, options: Optional[McOptions] = None,
                     idle_ns: int = 0, solo_states: int = 0) -> Server:
    """solo_states: requests that find the server idle and whose state bound
    is at most this run alone on the single-model explorer (0: the library's
    default, 1: never)."""
    cfg = McServerConfig(int(slots), 0, int(pool_bytes), int(idle_ns), int(solo_states))
    h = C.c_void_p()
    rc = load().mc_server_create(C.byref(cfg), C.byref(options) if options is not None else None,
                                 C.byref(h))
    if rc != MC_OK:
        raise MCError(rc, "mc_server_create")
    return Server(h.value)


def mc_server_submit(server: Server, spec, kind: str, T: Optional[int] = None) -> int:
    arr, keep = _descs([spec])
    q = McQuery(MC_QUERY_MIN_TIME if kind == "min_time" else MC_QUERY_CHECK, 0, int(T or 0) & NO_LIMIT)
    t = C.c_uint64()
    rc = load().mc_server_submit(server.handle, arr, C.byref(q), C.byref(t))
    if rc != MC_OK:
        raise MCError(rc, "mc_server_submit")
    return t.value


def mc_server_poll(server: Server, cap: int = 1024, wait_ms: int = 0) -> list:
    buf = (McServerResult * cap)()
    n = C.c_uint32()
    rc = load().mc_server_poll(server.handle, buf, cap, C.byref(n), int(wait_ms))
    if rc != MC_OK:
        raise MCError(rc, "mc_server_poll")
    out = []
    for k in range(n.value):
        r = buf[k]
        d = _batch_result(r.result)
        d.update(ticket=r.ticket, submit_s=r.submit_s, admit_s=r.admit_s, done_s=r.done_s,
                 path={0: "loop", 1: "alone", 2: "config"}.get(r.path, "loop"))
        out.append(d)
    return out


def mc_server_status(server: Server) -> dict:
    q, r, l = C.c_uint32(), C.c_uint32(), C.c_uint64()
    fatal = load().mc_server_status(server.handle, C.byref(q), C.byref(r), C.byref(l))
    return {"queued": q.value, "running": r.value, "launches": l.value, "fatal": fatal}


def mc_server_destroy(server: Server):
    if server.handle and server.handle.value:
        load(build=False).mc_server_destroy(server.handle)
        server.handle = C.c_void_p()


def decode_key(layout: dict, key: int):
    """(i, j, n) of a packed state, i/j 1-based (0 = not selected yet)."""
    i = (key >> layout["wg_shift"]) & ((1 << layout["wg_bits"]) - 1)
    j = (key >> layout["ts_shift"]) & ((1 << layout["ts_bits"]) - 1)
    mask = (1 << layout["n_bits"]) - 1
    n = tuple((key >> s) & mask for s in layout["n_shift"])
    return i, j, n


# ---------------------------------------------------------------- PE-level model
class PeModel(Model):
    """Owns an ``mc_pe_model*``; destroyed with ``mc_pe_model_destroy``."""

    def __del__(self):
        try:
            mc_pe_model_destroy(self)
        except Exception:
            pass

    def _check(self, rc: int, where: str):
        if rc != MC_OK:
            detail = ""
            if self.handle:
                detail = load(build=False).mc_pe_last_error(self.handle).decode()
            raise MCError(rc, where, detail)


def mc_pe_model_create(spec, options: Optional[McOptions] = None, stream=None) -> PeModel:
    """Create a PE-level model from a ``pe_workloads.PeSpec``."""
    L = load()
    off, ticks, pes = spec.flat()
    arrs = (_u32(spec.wg_values), _u32(spec.ts_values), _u32(spec.n_workgroups), _u32(spec.pes),
            _u32(off), _u32(ticks), _u32(pes))
    d = McPeModelDesc(spec.a, spec.b, spec.P, *arrs)
    h = C.c_void_p()
    rc = L.mc_pe_model_create(C.byref(d), C.byref(options) if options is not None else None, C.byref(h))
    if rc != MC_OK:
        raise MCError(rc, "mc_pe_model_create")
    m = PeModel(h.value, spec)
    if stream is None:
        import torch

        if torch.cuda.is_available():
            stream = torch.cuda.current_stream().cuda_stream
    if stream is not None:
        m._check(L.mc_pe_set_stream(m.handle, C.c_void_p(int(stream))), "mc_pe_set_stream")
    return m


def mc_pe_model_destroy(model: PeModel):
    if model.handle and model.handle.value:
        load(build=False).mc_pe_model_destroy(model.handle)
        model.handle = C.c_void_p()
    _live.discard(model)


def mc_pe_model_layout(model: PeModel) -> dict:
    lay = McPeLayout()
    model._check(load().mc_pe_model_layout(model.handle, C.byref(lay)), "mc_pe_model_layout")
    out = {k: getattr(lay, k) for k, _t in McPeLayout._fields_ if k != "unit_shift"}
    out["unit_shift"] = list(lay.unit_shift[: lay.P])
    return out


def mc_pe_check(model: PeModel, T: int, trace: bool = True) -> dict:
    r = McCheckResult()
    h = C.c_void_p()
    rc = load().mc_pe_check(model.handle, int(T) & NO_LIMIT, C.byref(r), C.byref(h) if trace else None)
    model._check(rc, "mc_pe_check")
    out = {"holds": bool(r.holds), "states": r.states, "levels": r.levels}
    if not r.holds:
        out.update(cex_time=r.cex_time, cex_i=r.cex_wg_index, cex_j=r.cex_ts_index, cex_wg=r.cex_wg,
                   cex_ts=r.cex_ts, cex_level=r.cex_level, cex_key=r.cex_key[0] | (r.cex_key[1] << 64))
        if trace:
            out["trace"] = _take_trace(h)
    return out


def mc_pe_min_time(model: PeModel, trace: bool = True) -> dict:
    r = McMinResult()
    h = C.c_void_p()
    rc = load().mc_pe_min_time(model.handle, C.byref(r), C.byref(h) if trace else None)
    model._check(rc, "mc_pe_min_time")
    out = {"t_min": r.t_min, "i": r.wg_index, "j": r.ts_index, "wg": r.wg, "ts": r.ts,
           "states": r.states, "checks": r.checks, "level": r.level,
           "witness_key": r.witness_key[0] | (r.witness_key[1] << 64)}
    if trace:
        out["trace"] = _take_trace(h)
    return out


def mc_pe_count_states(model: PeModel) -> int:
    v = C.c_uint64()
    model._check(load().mc_pe_count_states(model.handle, C.byref(v)), "mc_pe_count_states")
    return v.value


def mc_pe_last_widths(model: PeModel, cap: int = 1 << 16) -> list:
    buf = (C.c_uint64 * cap)()
    n = C.c_uint32()
    model._check(load().mc_pe_last_widths(model.handle, buf, cap, C.byref(n)), "mc_pe_last_widths")
    return list(buf[: min(n.value, cap)])


def mc_pe_get_stats(model: PeModel) -> dict:
    st = McStats()
    model._check(load().mc_pe_get_stats(model.handle, C.byref(st)), "mc_pe_get_stats")
    return {k: getattr(st, k) for k, _t in McStats._fields_}


def mc_pe_reset_stats(model: PeModel):
    model._check(load().mc_pe_reset_stats(model.handle), "mc_pe_reset_stats")


def decode_pe_key(layout: dict, key: int) -> dict:
    """Fields of a packed PE-level state: i, j (1-based, 0 = not selected),
    level, and per unit (n, busy, pc, mask)."""
    f = lambda shift, bits: (key >> shift) & ((1 << bits) - 1)
    units = []
    M, pcb = layout["mask_bits"], layout["pc_bits"]
    for shift in layout["unit_shift"]:
        u = f(shift, layout["unit_bits"])
        units.append((u >> (M + pcb + 1), (u >> (M + pcb)) & 1, (u >> M) & ((1 << pcb) - 1),
                      u & ((1 << M) - 1)))
    return {"i": f(layout["wg_shift"], layout["wg_bits"]), "j": f(layout["ts_shift"], layout["ts_bits"]),
            "level": f(layout["level_shift"], layout["level_bits"]), "units": units}
