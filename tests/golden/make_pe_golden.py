"""Write tests/golden/pe_oracle_expected.json from the CPU oracle alone.

The GPU parity tests of the processing-element level model read these
values for the workloads whose oracle runs take minutes.  Every number here
comes from oracle/ (no value from the CUDA path).

    python tests/golden/make_pe_golden.py
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle import oracle as O  # noqa: E402
from paper_2305_09130_gb300 import pe_workloads as PW  # noqa: E402

WORKLOADS = {
    "pe_abstract_s16_P4": lambda: PW.pe_abstract(16, P=4, np_=4, gmt=1),
    "pe_minimum_s64_P4": lambda: PW.pe_minimum(64, P=4, np_=4, gmt=2),
}


def main():
    gold = {}
    for name, make in WORKLOADS.items():
        spec = make()
        t = time.time()
        full = O.pe_check(spec, (1 << 64) - 1, prune=False, early_exit=False, widths=1 << 20)
        secs = round(time.time() - t, 1)
        mt = O.pe_min_time(spec, prune=True, early_exit=True, refine=True)
        gold[name] = {"count": full["states"], "levels": full["levels"], "widths": full["widths"],
                      "count_seconds": secs, "min_time": mt}
        print(name, full["states"], full["levels"], secs, mt, flush=True)
    with open(os.path.join(HERE, "pe_oracle_expected.json"), "w") as f:
        json.dump(gold, f, sort_keys=True)
        f.write("\n")


if __name__ == "__main__":
    main()
