"""Seeded synthetic model descriptions (the inputs of every query).

This module produces what a user hands to ``mc_model_create``: the tuning
parameter domains (work-group sizes WG and tile sizes TS, chosen by the
nondeterministic ``select`` of the process ``main``, Listing 3), the number of
work-groups N_ij of each configuration, the per-work-group cost table and the
per-compute-unit speed factors.  It holds none of the explorer's arithmetic:
no transition rule, no clock, no property.  Both the CUDA path and the CPU
oracle consume these arrays; neither imports the other.

Readings of the paper used here (where it is silent or inconsistent):

* Number of work-groups: ``N = ceil(G / WG)`` (at least 1).  The paper prints
  ``WGs = size / (WG * TS)`` (Listing 3) but its Table 1 contradicts that
  formula; the host program of Listing 11 pads the global size to a multiple
  of WG, so every work-group is full.
* Cost of one work-group: ``ceil(WG/TS)*4 + WG + 2*TS`` -- global loads of the
  tile loop of Listing 2, one local operation per work item, tile set-up.  The
  ceiling keeps at least one global load when TS > WG.
* Random draws use splitmix64 (Steele, Lea and Flood, OOPSLA 2014):
  ``x % range + lo`` for a value in ``[lo, lo + range)``.

Sizes of the named workloads:

* ``c1``: G=64, P=2, WG in {1,2,4,8,16}, TS in {1,2,4}, speed 1 (8,763
  reachable states under FREE, 579 under GREEDY).
* ``c2``: G=1024, P=4, WG in 2^0..2^8, TS in 2^0..2^4, formula cost, speeds
  U{1..3} (seed 2305091302).  ``c2_star`` is the same with G=80 under FREE
  (10,385,335 reachable states).
* ``c3``: G=4096, P=8, WG in 2^0..2^9, TS in 2^0..2^5, cost U{1..16} per
  (WG, TS) (seed 2305091303), speed 1, 128-bit keys.  ``c3_star`` is the same
  with G=36 under FREE (1,072,924,481 reachable states).
* ``c4_instances``: 256 uneven instances for batched runs (seed 2305091304).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List

MASK64 = (1 << 64) - 1
SPLITMIX_GAMMA = 0x9E3779B97F4A7C15

FREE = 0
GREEDY = 1


def splitmix64_mix(z: int) -> int:
    """The splitmix64 output function (Steele, Lea, Flood 2014)."""
    z &= MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return z ^ (z >> 31)


class SplitMix64:
    """Sequential splitmix64: the k-th output (k >= 0) is mix(seed + (k+1)*gamma)."""

    def __init__(self, seed: int):
        self.state = seed & MASK64

    def next(self) -> int:
        self.state = (self.state + SPLITMIX_GAMMA) & MASK64
        return splitmix64_mix(self.state)

    def uniform(self, lo: int, hi: int) -> int:
        """Integer in [lo, hi] as ``x % (hi - lo + 1) + lo``."""
        return self.next() % (hi - lo + 1) + lo


@dataclass
class ModelSpec:
    """One model: the arrays ``mc_model_desc`` carries, plus a name.

    ``n_workgroups`` and ``cost`` are row-major ``[i][j]`` over
    ``wg_values[i]``, ``ts_values[j]``.
    """

    name: str
    P: int
    wg_values: List[int]
    ts_values: List[int]
    n_workgroups: List[int]
    cost: List[int]
    speed: List[int]
    rule: int = FREE
    key_bits: int = 0
    G: int = 0
    meta: dict = field(default_factory=dict)

    @property
    def a(self) -> int:
        return len(self.wg_values)

    @property
    def b(self) -> int:
        return len(self.ts_values)

    def with_rule(self, rule: int) -> "ModelSpec":
        return ModelSpec(self.name, self.P, list(self.wg_values), list(self.ts_values),
                         list(self.n_workgroups), list(self.cost), list(self.speed),
                         rule, self.key_bits, self.G, dict(self.meta))

    def with_key_bits(self, key_bits: int) -> "ModelSpec":
        m = self.with_rule(self.rule)
        m.key_bits = key_bits
        return m


def n_workgroups_for(G: int, wg: int) -> int:
    """Work-groups for global size G at work-group size wg: ceil(G/wg), >= 1."""
    return max(1, -(-G // wg))


def formula_cost(wg: int, ts: int) -> int:
    """Per-work-group time of the abstract kernel (Listing 2): ceil(WG/TS)
    global-memory tile loads of 4 units each, WG local operations, 2*TS for
    the tile set-up."""
    return -(-wg // ts) * 4 + wg + 2 * ts


def from_formula(name: str, G: int, P: int, wg_values, ts_values, speed, rule) -> ModelSpec:
    n = [n_workgroups_for(G, wg) for wg in wg_values for _ts in ts_values]
    cost = [formula_cost(wg, ts) for wg in wg_values for ts in ts_values]
    return ModelSpec(name, P, list(wg_values), list(ts_values), n, cost, list(speed),
                     rule, 0, G)


def pow2_range(lo_exp: int, hi_exp: int) -> List[int]:
    return [1 << e for e in range(lo_exp, hi_exp + 1)]


def c1(rule: int = FREE) -> ModelSpec:
    """Tiny plain query: G=64, P=2, WG {1,2,4,8,16}, TS {1,2,4}, speed 1."""
    return from_formula("c1", 64, 2, [1, 2, 4, 8, 16], [1, 2, 4], [1, 1], rule)


def tiny(rule: int = FREE) -> ModelSpec:
    """G=8, P=2, WG {1,2}, TS {1,2}, speeds (1,3)."""
    return from_formula("tiny", 8, 2, [1, 2], [1, 2], [1, 3], rule)


def c2(G: int = 1024, rule: int = GREEDY, seed: int = 2305091302) -> ModelSpec:
    """Medium query: P=4, WG 2^0..2^8, TS 2^0..2^4, formula cost, speed U{1..3}."""
    rng = SplitMix64(seed)
    speed = [rng.uniform(1, 3) for _ in range(4)]
    m = from_formula("c2" if G == 1024 else f"c2_G{G}", G, 4, pow2_range(0, 8),
                     pow2_range(0, 4), speed, rule)
    m.meta["seed"] = seed
    return m


def c2_star(rule: int = FREE) -> ModelSpec:
    """C2 at G=80 under FREE: 10,385,335 reachable states."""
    m = c2(G=80, rule=rule)
    m.name = "c2_star"
    return m


def c3(G: int = 4096, rule: int = GREEDY, seed: int = 2305091303, key_bits: int = 128) -> ModelSpec:
    """Large query: P=8, WG 2^0..2^9, TS 2^0..2^5, cost U{1..16}, speed 1."""
    rng = SplitMix64(seed)
    wg = pow2_range(0, 9)
    ts = pow2_range(0, 5)
    cost = [rng.uniform(1, 16) for _ in range(len(wg) * len(ts))]
    n = [n_workgroups_for(G, w) for w in wg for _t in ts]
    m = ModelSpec("c3" if G == 4096 else f"c3_G{G}", 8, wg, ts, n, cost, [1] * 8, rule,
                  key_bits, G)
    m.meta["seed"] = seed
    return m


def c3_star(rule: int = FREE) -> ModelSpec:
    """C3 at G=36 under FREE with forced 128-bit keys: 1,072,924,481 states."""
    m = c3(G=36, rule=rule, key_bits=128)
    m.name = "c3_star"
    return m


def c4_instances(count: int = 256, seed: int = 2305091304, rule: int = GREEDY) -> List[ModelSpec]:
    """Uneven instances for batched runs: G = 2^U{6..12}, P in {2,4,8},
    WG 2^0..2^8, TS 2^0..2^4, cost U{1..16} per (WG, TS), speeds U{1..3}.

    Each instance also carries ``meta['t_frac_milli']``: a draw U{800..1200}
    that a batched driver turns into a check threshold round(frac * T_min),
    and ``meta['query']``: 0 = check, 1 = min-time (50/50).
    """
    rng = SplitMix64(seed)
    out = []
    wg = pow2_range(0, 8)
    ts = pow2_range(0, 4)
    for k in range(count):
        G = 1 << rng.uniform(6, 12)
        P = (2, 4, 8)[rng.uniform(0, 2)]
        cost = [rng.uniform(1, 16) for _ in range(len(wg) * len(ts))]
        speed = [rng.uniform(1, 3) for _ in range(P)]
        n = [n_workgroups_for(G, w) for w in wg for _t in ts]
        m = ModelSpec(f"c4_{k}", P, wg, ts, n, cost, speed, rule, 0, G)
        m.meta["query"] = rng.uniform(0, 1)
        m.meta["t_frac_milli"] = rng.uniform(800, 1200)
        out.append(m)
    return out


def random_small(seed: int, P: int, a: int, b: int, n_max: int, cost_max: int = 9,
                 speed_max: int = 3, rule: int = FREE, key_bits: int = 0) -> ModelSpec:
    """A small random model for parity sweeps: N_ij U{1..n_max}, cost U{1..cost_max},
    speeds U{1..speed_max}; WG/TS values are 2^i, 2^j (informative only)."""
    rng = SplitMix64(seed)
    n = [rng.uniform(1, n_max) for _ in range(a * b)]
    cost = [rng.uniform(1, cost_max) for _ in range(a * b)]
    speed = [rng.uniform(1, speed_max) for _ in range(P)]
    return ModelSpec(f"rand_{seed}", P, pow2_range(0, a - 1), pow2_range(0, b - 1), n, cost,
                     speed, rule, key_bits, 0, {"seed": seed})


NAMED = {
    "tiny": tiny,
    "c1": c1,
    "c2": c2,
    "c2_star": c2_star,
    "c3": c3,
    "c3_star": c3_star,
}
