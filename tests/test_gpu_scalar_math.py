"""The Newton-Raphson FP64 reciprocal and reciprocal square root used in the kernels'
scalar chains agree with CUDA's 1/x and 1/sqrt(x) to within 2 ulps over 2^20 arguments
spanning 2^-580 .. 2^579 (both signs for the reciprocal)."""
import os
import re
import subprocess

import pytest

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def test_newton_rcp_rsqrt_within_2_ulp(tmp_path):
    exe = str(tmp_path / "nr_check")
    subprocess.run(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17",
                    "-I", os.path.join(ROOT, "paper_2011_06532_gb300", "csrc"), "-I", os.path.join(ROOT, "include"),
                    os.path.join(HERE, "nr_check.cu"), "-o", exe], check=True)
    out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout
    m = re.search(r"max_ulp_rcp (\S+) max_ulp_rsqrt (\S+) err (.*)", out)
    assert m, out
    assert m.group(3).strip() == "no error"
    assert float(m.group(1)) <= 2 and float(m.group(2)) <= 2, out
