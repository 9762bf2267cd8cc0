"""ctypes binding of the CPU oracle (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg use this module.  It builds ``oracle/liboracle.so`` from ``oracle.cpp``
with the host C++ compiler and exposes:

* ``check(spec, T, prune, early_exit)`` -- the over-time property
  G(FIN -> time > T) of Section 4, Step 2, with the counting rules stated in
  ``oracle.cpp``;
* ``count(spec)`` -- every reachable state;
* ``simulate(spec, seed, walks)`` -- T_ini from random runs (Section 4,
  Step 3: a simulation gives the initial bound);
* ``min_time(spec, search, ...)`` -- Step 3 (search for T_min) and Step 4
  (the configuration of the last counterexample);
* ``walk(spec, seed, w)`` and ``swarm(spec, seed, walks, rounds)`` -- the
  random runs and the swarm search of Section 5;
* ``pe_check``, ``pe_count``, ``pe_min_time`` -- the same queries on the
  processing-element level model (``oracle_pe.cpp``).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
SRCS = [os.path.join(HERE, "oracle.cpp"), os.path.join(HERE, "oracle_pe.cpp")]
LIB = os.path.join(HERE, "liboracle.so")
NO_LIMIT = (1 << 64) - 1
SEARCH = {"single": 0, "lower": 1, "bisect": 2}

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/liboracle.so (host code only)."""
    stale = not os.path.exists(LIB) or any(os.path.getmtime(LIB) < os.path.getmtime(s) for s in SRCS)
    if force or stale:
        tmp = LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", *SRCS, "-o", tmp])
        os.replace(tmp, LIB)
    return LIB


class OrModel(C.Structure):
    _fields_ = [("a", C.c_uint32), ("b", C.c_uint32), ("P", C.c_uint32), ("rule", C.c_uint32),
                ("N", C.POINTER(C.c_uint32)), ("cost", C.POINTER(C.c_uint32)),
                ("speed", C.POINTER(C.c_uint32))]


class OrCheck(C.Structure):
    _fields_ = [("holds", C.c_uint32), ("levels", C.c_uint32), ("states", C.c_uint64),
                ("cex_time", C.c_uint64), ("cex_i", C.c_uint32), ("cex_j", C.c_uint32),
                ("cex_level", C.c_uint32), ("pad", C.c_uint32), ("cex_n", C.c_uint32 * 16)]


class OrMin(C.Structure):
    _fields_ = [("t_min", C.c_uint64), ("t_ini", C.c_uint64), ("states", C.c_uint64),
                ("checks", C.c_uint32), ("i", C.c_uint32), ("j", C.c_uint32),
                ("level", C.c_uint32), ("n", C.c_uint32 * 16)]


class OrPeModel(C.Structure):
    _fields_ = [("a", C.c_uint32), ("b", C.c_uint32), ("P", C.c_uint32),
                ("N", C.POINTER(C.c_uint32)), ("pes", C.POINTER(C.c_uint32)),
                ("prog_off", C.POINTER(C.c_uint32)), ("seg_ticks", C.POINTER(C.c_uint32)),
                ("seg_pes", C.POINTER(C.c_uint32))]


class OrPeCheck(C.Structure):
    _fields_ = [("holds", C.c_uint32), ("levels", C.c_uint32), ("states", C.c_uint64),
                ("cex_time", C.c_uint64), ("cex_i", C.c_uint32), ("cex_j", C.c_uint32),
                ("cex_level", C.c_uint32), ("pad", C.c_uint32)]


class OrPeMin(C.Structure):
    _fields_ = [("t_min", C.c_uint64), ("states", C.c_uint64), ("checks", C.c_uint32),
                ("i", C.c_uint32), ("j", C.c_uint32), ("level", C.c_uint32)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(LIB)
            L.oracle_check.argtypes = [C.POINTER(OrModel), C.c_uint64, C.c_int, C.c_int,
                                       C.POINTER(OrCheck), C.POINTER(C.c_uint64), C.c_uint32]
            L.oracle_count.argtypes = [C.POINTER(OrModel), C.POINTER(C.c_uint64)]
            L.oracle_simulate.argtypes = [C.POINTER(OrModel), C.c_uint64, C.c_uint32,
                                          C.POINTER(C.c_uint64)]
            L.oracle_min_time.argtypes = [C.POINTER(OrModel), C.c_int, C.c_int, C.c_int, C.c_int,
                                          C.c_uint64, C.c_uint32, C.POINTER(OrMin)]
            L.oracle_walk.argtypes = [C.POINTER(OrModel), C.c_uint64, C.c_uint64, C.POINTER(C.c_uint64),
                                      C.POINTER(C.c_uint32), C.POINTER(C.c_uint32)]
            L.oracle_pe_check.argtypes = [C.POINTER(OrPeModel), C.c_uint64, C.c_int, C.c_int,
                                          C.POINTER(OrPeCheck), C.POINTER(C.c_uint64), C.c_uint32]
            L.oracle_pe_count.argtypes = [C.POINTER(OrPeModel), C.POINTER(C.c_uint64)]
            L.oracle_pe_min_time.argtypes = [C.POINTER(OrPeModel), C.c_int, C.c_int, C.c_int,
                                             C.POINTER(OrPeMin)]
            for f in (L.oracle_check, L.oracle_count, L.oracle_simulate, L.oracle_min_time,
                      L.oracle_walk, L.oracle_pe_check, L.oracle_pe_count, L.oracle_pe_min_time):
                f.restype = C.c_int
            _lib = L
    return _lib


def _model(spec):
    arr = lambda xs: (C.c_uint32 * len(xs))(*xs)
    keep = (arr(spec.n_workgroups), arr(spec.cost), arr(spec.speed))
    m = OrModel(spec.a, spec.b, spec.P, spec.rule, keep[0], keep[1], keep[2])
    return m, keep


def check(spec, T: int, prune: bool = True, early_exit: bool = True, widths: int = 0) -> dict:
    m, _keep = _model(spec)
    r = OrCheck()
    w = (C.c_uint64 * max(widths, 1))()
    rc = lib().oracle_check(C.byref(m), T & NO_LIMIT, int(prune), int(early_exit), C.byref(r),
                            w if widths else None, widths)
    if rc != 0:
        raise ValueError(f"oracle_check failed ({rc})")
    out = {"holds": bool(r.holds), "states": r.states, "levels": r.levels}
    if not r.holds:
        out.update(cex_time=r.cex_time, cex_i=r.cex_i, cex_j=r.cex_j, cex_level=r.cex_level,
                   cex_n=list(r.cex_n[: spec.P]))
    if widths:
        out["widths"] = list(w[: r.levels])
    return out


def count(spec) -> int:
    m, _keep = _model(spec)
    out = C.c_uint64()
    if lib().oracle_count(C.byref(m), C.byref(out)) != 0:
        raise ValueError("oracle_count failed")
    return out.value


def simulate(spec, seed: int, walks: int = 1) -> int:
    m, _keep = _model(spec)
    out = C.c_uint64()
    if lib().oracle_simulate(C.byref(m), seed & NO_LIMIT, walks, C.byref(out)) != 0:
        raise ValueError("oracle_simulate failed")
    return out.value


def walk(spec, seed: int, w: int):
    """(time, i, j) of random run number w of `seed` (Section 5's swarm runs)."""
    m, _keep = _model(spec)
    t, i, j = C.c_uint64(), C.c_uint32(), C.c_uint32()
    if lib().oracle_walk(C.byref(m), seed & NO_LIMIT, w, C.byref(t), C.byref(i), C.byref(j)) != 0:
        raise ValueError("oracle_walk failed")
    return t.value, i.value, j.value


def swarm(spec, seed: int, walks_per_round: int, max_rounds: int) -> dict:
    """Section 5's swarm search over the same runs: round 0 takes the least
    terminal time of its runs; each later round looks for a run ending at or
    below (best - 1) and the search stops after a round that finds none."""
    bound = None
    out = {"rounds": 0, "walks": 0}
    for r in range(max_rounds):
        base = r * walks_per_round
        found = None
        for k in range(walks_per_round):
            t, i, j = walk(spec, seed, base + k)
            if (bound is None or t <= bound) and (found is None or (t, k) < found[:2]):
                found = (t, k, i, j)
        out["rounds"] = r + 1
        out["walks"] += walks_per_round
        if found is None:
            break
        out.update(best_time=found[0], best_walk=base + found[1], i=found[2], j=found[3])
        if r == 0:
            out["first_time"] = found[0]
        bound = found[0] - 1
    return out


def min_time(spec, search: str = "single", prune: bool = True, early_exit: bool = True,
             refine: bool = True, seed: int = 2305091300, walks: int = 1) -> dict:
    m, _keep = _model(spec)
    r = OrMin()
    rc = lib().oracle_min_time(C.byref(m), SEARCH[search], int(prune), int(early_exit),
                               int(refine), seed & NO_LIMIT, walks, C.byref(r))
    if rc != 0:
        raise ValueError(f"oracle_min_time failed ({rc})")
    return {"t_min": r.t_min, "t_ini": r.t_ini, "states": r.states, "checks": r.checks,
            "i": r.i, "j": r.j, "level": r.level, "n": list(r.n[: spec.P])}


# ---------------------------------------------------------------- PE-level model
def _pe_model(spec):
    arr = lambda xs: (C.c_uint32 * max(1, len(xs)))(*xs)
    off, ticks, pes = spec.flat()
    keep = (arr(spec.n_workgroups), arr(spec.pes), arr(off), arr(ticks), arr(pes))
    return OrPeModel(spec.a, spec.b, spec.P, *keep), keep


def pe_check(spec, T: int, prune: bool = True, early_exit: bool = True, widths: int = 0) -> dict:
    """G(FIN -> time > T) on the processing-element level model."""
    m, _keep = _pe_model(spec)
    r = OrPeCheck()
    w = (C.c_uint64 * max(widths, 1))()
    rc = lib().oracle_pe_check(C.byref(m), T & NO_LIMIT, int(prune), int(early_exit), C.byref(r),
                               w if widths else None, widths)
    if rc != 0:
        raise ValueError(f"oracle_pe_check failed ({rc})")
    out = {"holds": bool(r.holds), "states": r.states, "levels": r.levels}
    if not r.holds:
        out.update(cex_time=r.cex_time, cex_i=r.cex_i, cex_j=r.cex_j, cex_level=r.cex_level)
    if widths:
        out["widths"] = list(w[: r.levels])
    return out


def pe_count(spec) -> int:
    m, _keep = _pe_model(spec)
    out = C.c_uint64()
    if lib().oracle_pe_count(C.byref(m), C.byref(out)) != 0:
        raise ValueError("oracle_pe_count failed")
    return out.value


def pe_min_time(spec, prune: bool = True, early_exit: bool = True, refine: bool = True) -> dict:
    m, _keep = _pe_model(spec)
    r = OrPeMin()
    if lib().oracle_pe_min_time(C.byref(m), int(prune), int(early_exit), int(refine), C.byref(r)) != 0:
        raise ValueError("oracle_pe_min_time failed")
    return {"t_min": r.t_min, "states": r.states, "checks": r.checks, "i": r.i, "j": r.j,
            "level": r.level}
