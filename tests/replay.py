"""Replay of a counterexample trace against the model's rules (test helper).

A trace is valid when it starts at s0, selects a WG index, then a TS index
(Listing 3), then dispatches one work-group per step to a unit the rule
allows (FREE: any unit; GREEDY: a unit whose clock is minimal), and ends in a
terminal state (all N_ij work-groups dispatched, Listing 4) whose model time
satisfies the requested bound.  The trace's parent choices are racy on the
GPU, so traces are checked by replay rather than compared.
"""
from __future__ import annotations


def decode(layout, key):
    i = (key >> layout["wg_shift"]) & ((1 << layout["wg_bits"]) - 1)
    j = (key >> layout["ts_shift"]) & ((1 << layout["ts_bits"]) - 1)
    mask = (1 << layout["n_bits"]) - 1
    n = [(key >> s) & mask for s in layout["n_shift"]]
    return i, j, n


def replay(spec, layout, keys, time_ok):
    """Return the terminal's (time, i, j, n); raise AssertionError on any
    invalid step.  time_ok(t) decides whether the final time is acceptable."""
    P = spec.P
    states = [decode(layout, k) for k in keys]
    assert states[0] == (0, 0, [0] * P), states[0]
    i1, j1, n1 = states[1]
    assert j1 == 0 and n1 == [0] * P and 1 <= i1 <= spec.a, states[1]
    i2, j2, n2 = states[2]
    assert i2 == i1 and 1 <= j2 <= spec.b and n2 == [0] * P, states[2]
    cfg = (i1 - 1) * spec.b + (j2 - 1)
    t = [spec.cost[cfg] * spec.speed[c] for c in range(P)]
    N = spec.n_workgroups[cfg]
    prev = n2
    for (i, j, n) in states[3:]:
        assert (i, j) == (i1, j2)
        diff = [n[c] - prev[c] for c in range(P)]
        assert sorted(diff) == [0] * (P - 1) + [1], (prev, n)
        c = diff.index(1)
        assert sum(prev) < N
        if spec.rule == 1:
            clocks = [prev[u] * t[u] for u in range(P)]
            assert clocks[c] == min(clocks), (prev, c)
        prev = n
    assert sum(prev) == N, "trace does not end in a terminal state"
    time = max(prev[c] * t[c] for c in range(P))
    assert time_ok(time), time
    return time, i1 - 1, j2 - 1, prev
