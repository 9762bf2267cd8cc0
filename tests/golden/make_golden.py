"""Write tests/golden/oracle_expected.json from the CPU oracle alone.

The GPU parity tests read these values for the workloads whose oracle runs
take longer than a test should (C2 at G=80 under FREE: 10,385,335 states).
Every number here comes from oracle/ (no value from the CUDA path).

    python tests/golden/make_golden.py
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle import oracle as O  # noqa: E402
from paper_2305_09130_gb300 import workloads as W  # noqa: E402

SEED = 2305091300


def min_time_cases(spec, cases):
    out = {}
    for search, prune in cases:
        t = time.time()
        r = O.min_time(spec, search=search, prune=prune, early_exit=True, refine=True, seed=SEED,
                       walks=1)
        r["oracle_seconds"] = round(time.time() - t, 2)
        out[f"{search}/prune{int(prune)}"] = r
        print(spec.name, search, prune, r, flush=True)
    return out


def main():
    gold = {"seed": SEED}
    spec = W.c2_star()
    t = time.time()
    gold["c2_star"] = {"count": O.count(spec), "count_seconds": round(time.time() - t, 2),
                       "min_time": min_time_cases(spec, [("single", True), ("lower", True),
                                                         ("bisect", True), ("lower", False)])}
    spec = W.c2(rule=W.GREEDY)
    gold["c2_greedy"] = {"count": O.count(spec),
                         "min_time": min_time_cases(spec, [("single", True), ("lower", False)])}
    spec = W.c3(rule=W.GREEDY)
    gold["c3_greedy"] = {"count": O.count(spec),
                         "min_time": min_time_cases(spec, [("single", True)])}
    with open(os.path.join(HERE, "oracle_expected.json"), "w") as f:
        json.dump(gold, f, indent=1, sort_keys=True)
        f.write("\n")


if __name__ == "__main__":
    main()
