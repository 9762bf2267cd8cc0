"""The boundary is a C-ABI: a plain C99 program (tests/c_abi/min_time_c1.c)
includes include/mc.h and include/mc_pe.h, links against libmcgpu.so and runs
a query.  Without a GPU it must get MC_ERR_CUDA back (no CPU fallback); on a
GB300 it must get T_min = 80 at WG 16, TS 4 for the tiny model."""
import os
import subprocess

import pytest

from paper_2305_09130_gb300 import build as B

HERE = os.path.dirname(os.path.abspath(__file__))


def compile_program(tmp_path):
    lib = B.build()
    exe = str(tmp_path / "min_time_c1")
    subprocess.check_call(["gcc", "-std=c99", "-Wall", "-Werror", "-I", B.INCLUDE,
                           os.path.join(HERE, "c_abi", "min_time_c1.c"), "-o", exe,
                           "-L", os.path.dirname(lib), "-lmcgpu", "-Wl,-rpath," + os.path.dirname(lib)])
    return exe


def test_c_program_builds_and_fails_loudly_without_a_gpu(tmp_path):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    r = subprocess.run([compile_program(tmp_path)], capture_output=True, text=True)
    assert r.returncode == 3, r.stdout + r.stderr


@pytest.mark.gpu
def test_c_program_answers_on_the_gpu(tmp_path):
    r = subprocess.run([compile_program(tmp_path)], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "T_min 80 at WG 16 TS 4" in r.stdout
