"""Seeded synthetic inputs of the processing-element level model.

The processing-element (PE) level model keeps what the cost-table model folds
away: every compute unit runs a work-group as NWE processing elements (the
processes ``pex`` of Listing 8 and ``barrier`` of Listing 7), each PE reports
every tick of its ``long_work`` to the ``clock`` process (Listing 9), and
the unit's local barrier waits for all of its PEs.  What a user hands to
``mc_pe_model_create`` is, per configuration (WG index i, TS index j):

* ``n_workgroups``: the work-groups N_ij the device hands out;
* ``pes``: NWE_ij, the PEs each unit runs the work-group on (1..8);
* a *program*: the segments every PE of a unit executes for one work-group,
  each either a work segment of ``ticks`` clock ticks in which ``seg_pes``
  PEs report once per tick, or a local barrier (``ticks == 0``) that
  ``seg_pes`` PEs arrive at before the unit releases them.

This module builds those arrays from the kernels the paper models.  It holds
none of the explorer's arithmetic (no transition, no clock, no property).

Readings of the paper used here (where it is silent or inconsistent):

* ``long_work(gt, tz)`` lasts ``gt * tz + 1`` ticks: it leaves its loop once
  ``time > start_time + gt * tz`` and ``start_time`` is the time it began
  (Listing 8 sets ``start_time`` before every call but the global-memory one
  of the second and later iterations; the stale value is read as a slip).
* Abstract kernel (Listings 2 and 8): N = size / WG work-groups (one element
  per work item), NWE = min(WG, NP); a PE serves ceil(WG / NP) work items one
  after another (the unit re-activates it, Listing 6); each item runs
  size / TS iterations of [global load: long_work(GMT, TS); barrier; local
  work: long_work(1, TS); barrier], then stores its result: long_work(GMT, 1).
  WG and TS range over 2^1 .. 2^(n-1) for size = 2^n (``select`` in main,
  Listing 3).  With one unit of four PEs and GMT = 1 the minimum over this
  domain at size 8 is 44 at TS = 4, WG = 4 -- the first row of Table 1.
* Minimum kernel (Listings 10-15): N = ceil(size / (WG * TS)) work-groups,
  NWE = min(WG, NP); a PE maps ceil(WG / NP) slices of TS elements, each
  element a global read of GMT + 1 ticks, with no barrier in between; then
  one barrier, and PE 0 alone reduces the unit's NWE local minima (NWE - 1
  ticks) and writes the result to global memory (GMT ticks).  The reduction
  is taken per work-group as in the OpenCL kernel (Listing 10).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Sequence, Tuple

# A segment: (ticks, pes).  ticks == 0 is a local barrier.
Segment = Tuple[int, int]


@dataclass
class PeSpec:
    """One PE-level model: the arrays ``mc_pe_model_desc`` carries.

    Per-configuration arrays are row-major ``[i][j]`` over ``wg_values[i]``,
    ``ts_values[j]``; ``programs[cfg]`` is the segment list of that
    configuration.
    """

    name: str
    P: int
    wg_values: List[int]
    ts_values: List[int]
    n_workgroups: List[int]
    pes: List[int]
    programs: List[List[Segment]]
    meta: dict = field(default_factory=dict)

    @property
    def a(self) -> int:
        return len(self.wg_values)

    @property
    def b(self) -> int:
        return len(self.ts_values)

    def flat(self):
        """(prog_off[a*b + 1], seg_ticks[], seg_pes[]) as the C-ABI takes them."""
        off, ticks, pes = [0], [], []
        for prog in self.programs:
            for t, m in prog:
                ticks.append(t)
                pes.append(m)
            off.append(len(ticks))
        return off, ticks, pes


def _pow2_domain(size: int) -> List[int]:
    n = size.bit_length() - 1
    return [size >> (n - i) for i in range(1, n)]


def abstract_program(size: int, wg: int, ts: int, np_: int, gmt: int) -> List[Segment]:
    nwe = min(wg, np_)
    items = -(-wg // np_)
    one_item: List[Segment] = []
    for _ in range(size // ts):
        one_item += [(gmt * ts + 1, nwe), (0, nwe), (ts + 1, nwe), (0, nwe)]
    one_item.append((gmt + 1, nwe))
    return one_item * items


def pe_abstract(size: int, P: int = 1, np_: int = 4, gmt: int = 1,
                wg_values: Sequence[int] = (), ts_values: Sequence[int] = ()) -> PeSpec:
    """The abstract kernel of Listings 2 and 8 on P units of np_ PEs."""
    wg = list(wg_values) or _pow2_domain(size)
    ts = list(ts_values) or _pow2_domain(size)
    n, pes, progs = [], [], []
    for w in wg:
        for t in ts:
            n.append(max(1, size // w))
            pes.append(min(w, np_))
            progs.append(abstract_program(size, w, t, np_, gmt))
    return PeSpec(f"pe_abstract_s{size}_P{P}_np{np_}_g{gmt}", P, wg, ts, n, pes, progs,
                  {"size": size, "NP": np_, "GMT": gmt, "kernel": "abstract"})


def minimum_program(wg: int, ts: int, np_: int, gmt: int) -> List[Segment]:
    nwe = min(wg, np_)
    items = -(-wg // np_)
    prog: List[Segment] = [(ts * (gmt + 1), nwe)] * items
    prog.append((0, nwe))
    if nwe > 1:
        prog.append((nwe - 1, 1))
    prog.append((gmt, 1))
    return prog


def pe_minimum(size: int, P: int = 2, np_: int = 4, gmt: int = 2,
               wg_values: Sequence[int] = (), ts_values: Sequence[int] = ()) -> PeSpec:
    """The Minimum kernel of Listings 10-15 on P units of np_ PEs."""
    wg = list(wg_values) or _pow2_domain(size)
    ts = list(ts_values) or _pow2_domain(size)
    n, pes, progs = [], [], []
    for w in wg:
        for t in ts:
            n.append(max(1, -(-size // (w * t))))
            pes.append(min(w, np_))
            progs.append(minimum_program(w, t, np_, gmt))
    return PeSpec(f"pe_minimum_s{size}_P{P}_np{np_}_g{gmt}", P, wg, ts, n, pes, progs,
                  {"size": size, "NP": np_, "GMT": gmt, "kernel": "minimum"})


def table1_row1() -> PeSpec:
    """Table 1's platform (one device, one unit, four PEs) at size 8, GMT 1."""
    m = pe_abstract(8, P=1, np_=4, gmt=1)
    m.name = "pe_table1_size8"
    return m


NAMED = {
    "pe_table1_size8": table1_row1,
}
