"""Brute-force enumeration of every schedule of a tiny model (test helper).

Independent of the oracle's graph search: it walks the tree of ALL paths
(every WG choice, every TS choice, every sequence of dispatch decisions)
without any visited set, and collects what each path passes through.  The
state set, the level of each state and the terminal times fall out of the
paths themselves, so a mistake in the oracle's successor function, level
rule, pruning or counterexample choice shows up as a mismatch.

Exponential: use only for P <= 3 and N <= 6.
"""
from __future__ import annotations

FREE, GREEDY = 0, 1


def _paths(spec):
    """Yield every maximal path as a list of states (i, j, n-tuple); i, j are
    1-based, 0 = not yet selected."""
    P = spec.P
    zero = (0,) * P
    for i in range(1, spec.a + 1):
        for j in range(1, spec.b + 1):
            cfg = (i - 1) * spec.b + (j - 1)
            N = spec.n_workgroups[cfg]
            t = [spec.cost[cfg] * spec.speed[c] for c in range(P)]
            prefix = [(0, 0, zero), (i, 0, zero), (i, j, zero)]

            def rec(n, path):
                done = sum(n)
                if done == N:
                    yield path
                    return
                clocks = [n[c] * t[c] for c in range(P)]
                if spec.rule == FREE:
                    units = range(P)
                else:
                    mn = min(clocks)
                    units = [c for c in range(P) if clocks[c] == mn]
                for c in units:
                    m = list(n)
                    m[c] += 1
                    m = tuple(m)
                    yield from rec(m, path + [(i, j, m)])

            yield from rec(zero, prefix)


def state_time(spec, s):
    i, j, n = s
    if i == 0 or j == 0:
        return 0
    cfg = (i - 1) * spec.b + (j - 1)
    return max(n[c] * spec.cost[cfg] * spec.speed[c] for c in range(spec.P))


def enumerate_model(spec):
    """Return (levels, terminals): levels maps state -> path position (the
    same for every path through it, which the enumeration asserts), and
    terminals maps each terminal state -> model time."""
    levels = {}
    terminals = {}
    for path in _paths(spec):
        for pos, s in enumerate(path):
            if levels.setdefault(s, pos) != pos:
                raise AssertionError(f"state {s} reached at two path lengths")
        last = path[-1]
        terminals[last] = state_time(spec, last)
    return levels, terminals


def schedules(spec):
    """Terminal model time of every complete schedule, as (i, j, time) per path."""
    out = []
    for path in _paths(spec):
        i, j, _n = path[-1]
        out.append((i - 1, j - 1, state_time(spec, path[-1])))
    return out


def brute_check(spec, T, prune=True, early_exit=True):
    """The check of the over-time property by brute force: kept states are
    reachable states whose max clock is <= T (with pruning), the first level
    holding a terminal with time <= T stops the count (with early exit), and
    the counterexample is the smallest (time, i, j, n) there."""
    levels, terminals = enumerate_model(spec)
    kept = {s: l for s, l in levels.items() if not prune or state_time(spec, s) <= T}
    viol = {s: kept[s] for s in terminals if s in kept and terminals[s] <= T}
    out = {}
    if viol:
        first = min(viol.values())
        cands = [(terminals[s], s[0] - 1, s[1] - 1, tuple(s[2])) for s, l in viol.items()
                 if l == first]
        best = min(cands)
        out.update(holds=False, cex_time=best[0], cex_i=best[1], cex_j=best[2],
                   cex_n=list(best[3]), cex_level=first)
        last = first if early_exit else max(kept.values())
    else:
        out["holds"] = True
        last = max(kept.values())
    out["states"] = sum(1 for l in kept.values() if l <= last)
    out["levels"] = last + 1
    return out
