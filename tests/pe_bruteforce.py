"""Brute-force breadth-first enumeration of the processing-element level model.

A third, deliberately plain implementation of the transition relation (the
CPU oracle and the CUDA path are the other two), used to pin the oracle on
tiny models.  States are Python tuples; nothing is packed.

The model (Listings 3-9, processes ``host``, ``device``, ``unit``, ``pex``,
``barrier``, ``clock``), as read for this project:

* ``s0`` selects WG (level 1), then TS (level 2): configuration (i, j) with
  every unit idle and N_ij work-groups left to hand out.
* A unit that is idle while work-groups are left may take the next one (the
  device's ``dev_u ! go`` is received by any unit waiting for it): it starts
  the configuration's program at its first step with no PE marked.
* A program step is a clock tick of a work segment or a local barrier.  In
  either, each participating PE marks itself once, in any order: in a tick it
  reports ``NRP_work++`` and waits for ``time`` to change (Listing 8,
  ``long_work``), at a barrier it sends ``done`` to the ``barrier`` process
  (Listing 7).  When all participants of a barrier are marked, the barrier
  releases them (one step: the unit moves to its next program step).
* The clock ticks (``time++``, Listing 9) when every busy unit is in a tick
  step with all of its participants marked and no unit is idle while
  work-groups are left; every busy unit then moves to its next step.
* A unit whose program ends becomes idle.  FIN holds when no work-group is
  left and every unit is idle; its model time is the number of ticks.
"""
from __future__ import annotations

from typing import Dict, List, Tuple


def steps_of(program):
    out = []
    for ticks, m in program:
        if ticks == 0:
            out.append(("B", m))
        else:
            out.extend([("W", m)] * ticks)
    return out


def program_ticks(program) -> int:
    return sum(t for t, _m in program)


class PeModel:
    def __init__(self, spec):
        self.spec = spec
        self.P = spec.P
        self.steps = [steps_of(p) for p in spec.programs]

    def initial(self, i, j):
        P = self.P
        return (i, j, (0,) * P, (0,) * P, (0,) * P, (0,) * P, 0)

    def successors(self, s) -> List[tuple]:
        if s == ("s0",):
            return [("wg", i) for i in range(self.spec.a)]
        if s[0] == "wg":
            return [self.initial(s[1], j) for j in range(self.spec.b)]
        i, j, n, busy, pc, mask, t = s
        cfg = i * self.spec.b + j
        steps = self.steps[cfg]
        S = len(steps)
        left = self.spec.n_workgroups[cfg] - sum(n)
        out = []
        for c in range(self.P):
            if busy[c]:
                kind, m = steps[pc[c]]
                for e in range(m):
                    if not mask[c] >> e & 1:
                        mk = list(mask)
                        mk[c] |= 1 << e
                        out.append((i, j, n, busy, pc, tuple(mk), t))
                if kind == "B" and mask[c] == (1 << m) - 1:
                    p2, b2, m2 = list(pc), list(busy), list(mask)
                    p2[c] += 1
                    m2[c] = 0
                    if p2[c] == S:
                        b2[c], p2[c] = 0, 0
                    out.append((i, j, n, tuple(b2), tuple(p2), tuple(m2), t))
            elif left > 0:
                n2, b2, p2, m2 = list(n), list(busy), list(pc), list(mask)
                n2[c] += 1
                b2[c], p2[c], m2[c] = 1, 0, 0
                out.append((i, j, tuple(n2), tuple(b2), tuple(p2), tuple(m2), t))
        any_busy = any(busy)
        idle_waiting = left > 0 and not all(busy)
        ready = all(steps[pc[c]][0] == "W" and mask[c] == (1 << steps[pc[c]][1]) - 1
                    for c in range(self.P) if busy[c])
        if any_busy and ready and not idle_waiting:
            b2, p2, m2 = list(busy), list(pc), list(mask)
            for c in range(self.P):
                if busy[c]:
                    p2[c] += 1
                    m2[c] = 0
                    if p2[c] == S:
                        b2[c], p2[c] = 0, 0
            out.append((i, j, n, tuple(b2), tuple(p2), tuple(m2), t + 1))
        return out

    def is_fin(self, s) -> bool:
        if len(s) != 7:
            return False
        i, j, n, busy, _pc, _mask, _t = s
        return sum(n) == self.spec.n_workgroups[i * self.spec.b + j] and not any(busy)

    @staticmethod
    def time(s) -> int:
        return s[6] if len(s) == 7 else 0


def enumerate_levels(spec) -> List[List[tuple]]:
    """Every reachable state, level by level; asserts that no state is
    reachable at two different depths (the graph is layered)."""
    M = PeModel(spec)
    depth: Dict[tuple, int] = {("s0",): 0}
    levels = [[("s0",)]]
    while levels[-1]:
        nxt = []
        d = len(levels)
        for s in levels[-1]:
            for u in M.successors(s):
                if u in depth:
                    assert depth[u] == d, ("state reached at two depths", u, depth[u], d)
                    continue
                depth[u] = d
                nxt.append(u)
        levels.append(nxt)
    levels.pop()
    return levels


def brute_check(spec, T: int, prune: bool = True, early_exit: bool = True) -> dict:
    """Level-synchronous check of G(FIN -> time > T), counted like the
    explorer: states of the explored levels (up to the first level holding a
    violating terminal with early exit), the minimum (time, i, j) over that
    level's violating terminals as the counterexample."""
    M = PeModel(spec)
    seen = {("s0",)}
    frontier = [("s0",)]
    states, level, first = 1, 0, None
    best_all = None
    while frontier:
        nxt = []
        for s in frontier:
            for u in M.successors(s):
                if prune and M.time(u) > T:
                    continue
                if u not in seen:
                    seen.add(u)
                    nxt.append(u)
        if not nxt:
            break
        level += 1
        states += len(nxt)
        viol = [(M.time(u), u[0], u[1]) for u in nxt if M.is_fin(u) and M.time(u) <= T]
        if viol:
            v = min(viol)
            best_all = v if best_all is None else min(best_all, v)
            if first is None:
                first = (level, v)
            if early_exit:
                return {"holds": False, "states": states, "levels": level + 1, "cex_time": v[0],
                        "cex_i": v[1], "cex_j": v[2], "cex_level": level}
        frontier = nxt
    if first is None:
        return {"holds": True, "states": states, "levels": level + 1}
    lv, v = first
    return {"holds": False, "states": states, "levels": level + 1, "cex_time": v[0], "cex_i": v[1],
            "cex_j": v[2], "cex_level": lv}


def fin_times(spec) -> Dict[Tuple[int, int], set]:
    """Model times of every reachable FIN state, per configuration."""
    out: Dict[Tuple[int, int], set] = {}
    M = PeModel(spec)
    for lv in enumerate_levels(spec):
        for s in lv:
            if M.is_fin(s):
                out.setdefault((s[0], s[1]), set()).add(M.time(s))
    return out
