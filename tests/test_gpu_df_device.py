"""Device build of the FP64 <-> double-float conversions (tests/native/
df_convert_check_gpu.cu): the FP64-add join used by the final conversion of
the refinement, the integer-pipe join and the split, bit for bit against the
hardware operations on the GPU."""
import os
import shutil
import subprocess
import tempfile

import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_device_joins_and_split_match_hardware():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    with tempfile.TemporaryDirectory() as d:
        exe = os.path.join(d, "df_convert_check_gpu")
        src = os.path.join(ROOT, "tests", "native", "df_convert_check_gpu.cu")
        inc = os.path.join(ROOT, "paper_2107_06381_gb300", "csrc")
        subprocess.run([nvcc, "-O3", "-std=c++17", "-gencode", "arch=compute_103a,code=sm_103a", "-I", inc,
                        "-o", exe, src], check=True, capture_output=True)
        res = subprocess.run([exe], capture_output=True, text=True, timeout=120)
        assert res.returncode == 0, res.stdout + res.stderr
        assert "dadd-join mismatches 0, int-join mismatches 0, split mismatches 0" in res.stdout
