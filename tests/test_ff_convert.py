"""The FP64 <-> float-float conversions that the float-float kernels run on the GPU
(integer operations on the bit patterns, csrc/ff.cuh), compiled for the host from the same
header and checked against the FP64 route: the split bit for bit, the join within one unit
in the last place of the correctly rounded sum, over random values, arbitrary finite bit
patterns and the range edges (zero, subnormal, overflowing and infinite values)."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2112_04167_gb300", "csrc")


def _nvcc():
    for c in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    return None


def test_ff_conversions_match_fp64_route(tmp_path):
    nvcc = _nvcc()
    if nvcc is None:
        pytest.skip("nvcc not available")
    exe = str(tmp_path / "ff_convert_check")
    subprocess.run([nvcc, "-std=c++17", "-O2", "-x", "cu", "-I", CSRC,
                    os.path.join(HERE, "native", "ff_convert_check.cu"), "-o", exe],
                   check=True, capture_output=True, timeout=300)
    r = subprocess.run([exe, "1000000"], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "split_mismatch 0 join_mismatch 0" in r.stdout
