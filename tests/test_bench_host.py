"""Host-side checks of the benchmark: the reference arm (the FP64 oracle,
with its own bootstrap of the smooth vectors) runs on the CPU and prints the
contract's JSON line, and the byte and operation counts of the roofline are
the stated formulas."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


@pytest.mark.parametrize("smooth", ["bootstrap", "relaxed"])
def test_reference_arm_prints_the_contract_line(smooth):
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--grid", "32",
                        "--steps", "1", "--warmup", "0", "--smooth", smooth],
                       capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["higher_is_better"] is False
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "scaling", "config",
              "cpu_baseline", "e2e", "dtype", "data"):
        assert k in line, k
    assert line["value"] > 0 and line["unit"] == "ms/RHS"
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert ("bootstrap" in line["config"]["workload"]) == (smooth == "bootstrap")


def test_roofline_counts():
    lv = {"n0": 1000, "nnz0": 9000, "n1": 250, "npv1": 4000}
    K = 32
    assert bench.algorithmic_bytes("spmv_cg", lv, K, 4) == 9000 * 12 + 4 * 1001 + 1000 * K * 4 + 1000 * K * 8
    assert bench.alu_ops("spmv_cg", lv, K) == 9000 * K * 11 + 1000 * K * 14
    assert bench.alu_ops("restrict_l0", lv, K) is None
    assert bench.ALU_PEAK_OPS == pytest.approx(152 * 128 * 2.07e9)


def test_whole_job_value_is_per_rhs_over_all_ranks():
    assert bench.whole_job_ms_per_rhs(1000.0, 5, 32, 1) == pytest.approx(1000.0 / 5 / 32)
    assert bench.whole_job_ms_per_rhs(1000.0, 5, 32, 4) == pytest.approx(1000.0 / 5 / 128)
