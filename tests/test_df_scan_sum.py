"""Host build of the FP64 alpha sweep's double-float spectral sum
(qbvm_dfsum.cuh, the arithmetic the sweep kernel runs per term; the device's
approximate reciprocal replaced by the quotient) against long double
(tests/native/df_scan_sum_check.cu): sums of Re 1/(d_{2m} + tau Lambda) over
the even frequencies of Section 3.3, on a wide input set and on the ranges of
the 512-instance sweep workload.  Needs nvcc, no GPU."""
import os
import re
import shutil
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_double_float_scan_sum_error_bounds():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    with tempfile.TemporaryDirectory() as d:
        exe = os.path.join(d, "df_scan_sum_check")
        src = os.path.join(ROOT, "tests", "native", "df_scan_sum_check.cu")
        inc = os.path.join(ROOT, "paper_2107_06381_gb300", "csrc")
        subprocess.run([nvcc, "-O2", "-std=c++17", "-I", inc, "-x", "cu", "-o", exe, src], check=True,
                       capture_output=True)
        res = subprocess.run([exe], capture_output=True, text=True)
    assert res.returncode == 0, res.stdout + res.stderr
    val = {(s, k.strip()): float(v)
           for s, k, v in re.findall(r"^\[(\w+)\] (max [^\n]*?) ([0-9.e+-]+)$", res.stdout, re.M)}
    for s in ("wide", "sweep"):
        # a sum to 2^-42 of the sum of its terms' magnitudes (measured 6.2e-14, 4.4e-14)
        assert val[(s, "max |err| / sum|terms|")] <= 2.0 ** -42, res.stdout
        # each term to 2^-42 of its scale (measured 6.3e-14, 5.9e-14)
        assert val[(s, "max term err / max(|term|, (|Re d| + tau Lambda) / |z|^2)")] <= 2.0 ** -42, res.stdout
        # FP64 summation of the same terms keeps more digits where they cancel;
        # the check reports both so the gap stays visible
        assert val[(s, "max |err| / |sum| in FP64")] <= val[(s, "max |err| / |sum|")]
    # over the sweep workload's ranges a mode's sum stays within 1e-8 of itself
    # (measured 1.5e-9, FP64 6.6e-11)
    assert val[("sweep", "max |err| / |sum|")] <= 1e-8, res.stdout
