"""bench.py on the host: the reference arm's JSON line (the CPU FP64 oracle,
runnable without a GPU), the operation and byte model the roofline divides
by, and the freshness of the recorded DRAM traffic."""
import json
import math
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
import bhcp_inputs as bi  # noqa: E402


def test_reference_arm_line():
    """One step of the oracle on 255^2 x 256 (two full solves): the line carries
    every key of the contract, and its config equals the GPU arm's."""
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0"],
                         cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads([ln for ln in out.stdout.splitlines() if ln.startswith("{")][-1])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC and line["unit"] == bench.UNIT
    assert line["higher_is_better"] is True and line["dtype"] == "f64" and line["steps"] == 1
    assert line["value"] > 0 and line["ms_per_step"] > 0
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"] and cb["sample"]
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"], "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}

    class A:
        rhs = "general"
        gpus = 1
    want = bench.headline_config(A, bench.workload().grid, 2, "replicas1")
    assert line["config"] == want


def test_kernel_model_of_the_headline_passes():
    """Algorithmic bytes and FP64 operations per launch on 255^2 x 256: a DST
    pass reads and writes every value once (16 B per unknown); the time solve
    reads F and its Step (b) table and writes y."""
    grid = bi.Grid(2, (256, 256), 1.0, 0.1, 256)
    nt, Nx = grid.nt, grid.Nx
    byts, ops = bench.kernel_model("dst_y", grid, "general")
    assert byts == 16 * nt * Nx
    # 2 pre-processing + half of a length-256 complex FFT + separation + prefix sum
    assert ops == pytest.approx((2 + bench._fft_ops(8) / 2 + 2) * nt * Nx)
    byts, ops = bench.kernel_model("time_solve", grid, "general")
    assert byts == 8 * (nt * Nx + nt * Nx) + 16 * (nt // 2) * Nx
    byts_d, _ = bench.kernel_model("time_solve", grid, "delta")
    assert byts_d == byts - 8 * (nt - 1) * Nx            # the delta right-hand side reads one level
    assert bench.kernel_model("residual_df", grid, "general") == (None, None)
    assert bench.flop_budget("dst_x", grid) == pytest.approx(22 * nt * Nx)
    assert bench.flop_budget("time_solve", grid) == pytest.approx((10 * math.log2(nt) + 21) * nt * Nx)


def test_recorded_traffic_matches_the_tile_sources():
    """The DRAM traffic bench.py reports beside the roofline was captured on the
    present sources of the DST and time-solve tiles (else it reports null)."""
    assert bench.PROFILED_TRAFFIC["sources"] == bench.traffic_source_hash()
    assert set(bench.PROFILED_TRAFFIC["bytes"]) == {"dst_x", "dst_y", "time_solve"}
