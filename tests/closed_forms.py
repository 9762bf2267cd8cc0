"""Closed forms of the model's state counts and minimal times (test helper).

These follow from the scheduling semantics of Listings 3-9 by counting, not
by search, so they pin the oracle (and, through it, the CUDA path) at sizes
brute force cannot reach.

FREE (any compute unit takes the next work-group):
  * the states of a configuration with N work-groups are the vectors
    n in N^P with sum(n) <= N, so there are C(N+P, P) of them, and
    C(k+P-1, P-1) of them at level k+2 (sum(n) = k);
  * the minimal model time is the N-th smallest element of the multiset
    { m * t_c : m >= 1, c < P } (N identical jobs on uniform machines:
    the k-th smallest completion time is the best makespan for k jobs).

GREEDY (only the unit whose clock is smallest takes the next work-group):
  * the next job always starts at the smallest unused start time of the
    multiset S = { m * t_c : m >= 0, c < P }; so after k jobs every start
    below tau (the (k+1)-th smallest element of S) is used and x of the
    `tie` units whose next start equals tau were served in any order:
    C(tie, x) states at level k+2, with x = k - #{s in S : s < tau};
  * its minimal time takes the committed starts below the N-th smallest
    start tau_N and gives the x remaining jobs to the fastest tied units.
"""
from __future__ import annotations

from bisect import bisect_left, bisect_right
from math import comb


def unit_times(spec, cfg):
    return [spec.cost[cfg] * spec.speed[c] for c in range(spec.P)]


def free_count(spec) -> int:
    return 1 + spec.a + sum(comb(N + spec.P, spec.P) for N in spec.n_workgroups)


def free_widths(spec):
    n_max = max(spec.n_workgroups)
    w = [1, spec.a]
    for k in range(n_max + 1):
        w.append(sum(comb(k + spec.P - 1, spec.P - 1) for N in spec.n_workgroups if N >= k))
    return w


def free_tmin_cfg(spec, cfg) -> int:
    N = spec.n_workgroups[cfg]
    t = unit_times(spec, cfg)
    ends = sorted(m * tc for tc in t for m in range(1, N + 1))
    return ends[N - 1]


def _starts(spec, cfg, upto):
    t = unit_times(spec, cfg)
    return sorted((m * t[c], c) for c in range(spec.P) for m in range(upto + 1))


def greedy_cfg_widths(spec, cfg):
    """Level widths C(tie, x) of one configuration for k = 0..N."""
    N = spec.n_workgroups[cfg]
    values = [s for s, _c in _starts(spec, cfg, N + 1)]
    out = []
    for k in range(N + 1):
        tau = values[k]
        below = bisect_left(values, tau)
        tie = bisect_right(values, tau) - below
        out.append(comb(tie, k - below))
    return out


def greedy_level_width(spec, cfg, k) -> int:
    return greedy_cfg_widths(spec, cfg)[k]


def greedy_count(spec) -> int:
    return 1 + spec.a + sum(sum(greedy_cfg_widths(spec, cfg)) for cfg in range(spec.a * spec.b))


def greedy_widths(spec):
    n_max = max(spec.n_workgroups)
    w = [1, spec.a] + [0] * (n_max + 1)
    for cfg in range(spec.a * spec.b):
        for k, x in enumerate(greedy_cfg_widths(spec, cfg)):
            w[2 + k] += x
    return w


def greedy_tmin_cfg(spec, cfg) -> int:
    N = spec.n_workgroups[cfg]
    t = unit_times(spec, cfg)
    starts = _starts(spec, cfg, N)
    tau = starts[N - 1][0]
    committed = [(s, c) for s, c in starts if s < tau]
    x = N - len(committed)
    tied = sorted(t[c] for s, c in starts if s == tau)
    finish = max([s + t[c] for s, c in committed] + [tau + tied[x - 1]])
    return finish


def tmin(spec):
    """(T_min, sorted list of (i, j) reaching it)."""
    f = free_tmin_cfg if spec.rule == 0 else greedy_tmin_cfg
    per = {(cfg // spec.b, cfg % spec.b): f(spec, cfg) for cfg in range(spec.a * spec.b)}
    best = min(per.values())
    return best, sorted(k for k, v in per.items() if v == best)


def count(spec) -> int:
    return free_count(spec) if spec.rule == 0 else greedy_count(spec)


def widths(spec):
    return free_widths(spec) if spec.rule == 0 else greedy_widths(spec)
