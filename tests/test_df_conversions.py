"""Host build of the integer-pipe FP64 <-> FP32 conversions used by the
refinement kernels, checked bit for bit against the hardware casts
(tests/native/df_convert_check.cu).  Needs nvcc, no GPU."""
import os
import shutil
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_split_and_join_match_hardware_casts():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    with tempfile.TemporaryDirectory() as d:
        exe = os.path.join(d, "df_convert_check")
        src = os.path.join(ROOT, "tests", "native", "df_convert_check.cu")
        inc = os.path.join(ROOT, "paper_2107_06381_gb300", "csrc")
        subprocess.run([nvcc, "-O2", "-std=c++17", "-I", inc, "-x", "cu", "-o", exe, src], check=True,
                       capture_output=True)
        res = subprocess.run([exe], capture_output=True, text=True)
        assert res.returncode == 0, res.stdout + res.stderr
        assert "mismatches 0, join mismatches 0" in res.stdout
