"""The ctypes mirrors of the C structs (paper_2305_09130_gb300/mc.py) have the
layout the C compiler gives the structs of include/mc.h and include/mc_pe.h:
a C99 program prints sizeof and offsetof for every field, and the Python side
must agree field by field (no GPU needed)."""
import ctypes as C
import os
import subprocess

import pytest

from paper_2305_09130_gb300 import build as B
from paper_2305_09130_gb300 import mc

PAIRS = [
    ("mc_model_desc", mc.McModelDesc), ("mc_options", mc.McOptions),
    ("mc_check_result", mc.McCheckResult), ("mc_min_result", mc.McMinResult),
    ("mc_layout", mc.McLayout), ("mc_swarm_result", mc.McSwarmResult), ("mc_stats", mc.McStats),
    ("mc_query", mc.McQuery), ("mc_batch_result", mc.McBatchResult),
    ("mc_server_config", mc.McServerConfig), ("mc_server_result", mc.McServerResult),
    ("mc_pe_model_desc", mc.McPeModelDesc), ("mc_pe_layout", mc.McPeLayout),
]


def python_layout(cls):
    return [("sizeof", C.sizeof(cls))] + [(name, getattr(cls, name).offset) for name, *_ in cls._fields_]


def test_ctypes_structs_match_the_c_headers(tmp_path):
    if not os.path.exists(B.INCLUDE):
        pytest.skip("headers missing")
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "mc.h"', '#include "mc_pe.h"',
             "int main(void) {"]
    for cname, cls in PAIRS:
        lines.append(f'  printf("{cname} sizeof %zu\\n", sizeof({cname}));')
        for name, *_ in cls._fields_:
            lines.append(f'  printf("{cname} {name} %zu\\n", offsetof({cname}, {name}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = str(tmp_path / "layout")
    subprocess.check_call(["gcc", "-std=c99", "-Wall", "-Werror", "-I", B.INCLUDE, str(src), "-o", exe])
    out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split("\n")
    got = {}
    for line in out:
        if line:
            cname, field, value = line.split()
            got.setdefault(cname, []).append((field, int(value)))
    for cname, cls in PAIRS:
        assert got[cname] == python_layout(cls), cname
