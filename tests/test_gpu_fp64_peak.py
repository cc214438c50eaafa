"""The FP64 FMA rate of the GPU the tests run on (tests/fp64_peak.cu), the measured
counterpart of the unit-count peak (SMs x 2 FP64 FMA per clock x 2 flops x clock) that the
FP64 kernels' roofline fractions use.  Prints the rate; checks it is within 15 % of the
unit-count figure at the maximum SM clock (the probe reports what the FP64 pipe delivers)."""
import os
import re
import subprocess

import pytest

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


def test_fp64_fma_rate(tmp_path):
    exe = str(tmp_path / "fp64_peak")
    subprocess.run(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3", os.path.join(HERE, "fp64_peak.cu"),
                    "-o", exe], check=True)
    out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout
    m = re.search(r"fp64_tflops (\S+) sms (\d+) ms (\S+) err (.*)", out)
    assert m, out
    assert m.group(4).strip() == "no error"
    tflops, sms = float(m.group(1)), int(m.group(2))
    print(out.strip())
    unit_count = sms * 2 * 2 * 2.07e9 / 1e12
    assert 0.85 * unit_count <= tflops <= 1.05 * unit_count, (tflops, unit_count)
