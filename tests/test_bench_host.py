"""Host-side checks of the benchmark: the reference arm (the FP64 oracle on
the host cores, with its own bootstrap of the smooth vectors) runs on the
CPU and prints the contract's JSON line, and the byte and operation counts
of the roofline are the stated formulas."""
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
                        "--steps", "1", "--warmup", "0", "--smooth", smooth, "--cpu-sample-s", "1",
                        "--cpu-cores", "2"],
                       capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["higher_is_better"] is False
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "scaling", "config",
              "cpu_baseline", "e2e", "dtype", "data"):
        assert k in line, k
    assert line["value"] > 0 and line["unit"] == "ms/RHS"
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == line["value"] and cb["cores"] == 2
    assert cb["one_core_ms_per_rhs"] > 0 and cb["cpu"]
    assert ("bootstrap" in line["config"]["workload"]) == (smooth == "bootstrap")


def test_reference_arm_other_workload():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--config", "1",
                        "--grid", "24", "--steps", "1", "--warmup", "0", "--cpu-sample-s", "0.5",
                        "--cpu-cores", "1"],
                       capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert "poisson5 24x24" in line["config"]["workload"] and line["cpu_baseline"]["cores"] == 1


LV = {"n0": 1000, "nnz0": 9000, "n1": 250, "npv1": 4000}
K = 32
n, nnz, n1, npv, rp = 1000, 9000, 250, 4000, 4 * 1001


def test_roofline_counts_double_float_mode():
    """The float32 cycle with double-float CG: what each level-0 kernel reads
    and writes once (the first pre-sweep folded into the scaled matrix)."""
    ab = lambda k: bench.algorithmic_bytes(k, LV, K, "df")  # noqa: E731
    # col + (hi, lo) values, rowptr, p float read, q (hi, lo) written
    assert ab("spmv_cg") == nnz * 12 + rp + n * K * 4 + n * K * 8
    # q (hi, lo) read, r (hi, lo) read and written
    assert ab("cg_update") == 3 * n * K * 8
    # z and p read, p written; after every second iteration also p_{k-1} and x (hi, lo) read
    # and x written: 12 and 32 bytes per row and column, 22 per launch on average
    assert ab("cg_direction") == n * K * 22
    # col + float values, rowptr, D^-1, f = r_hi, u, r_lo read, z written
    assert ab("smooth_l0") == nnz * 8 + rp + n * 4 + 4 * n * K * 4
    # scaled matrix, f read once, P, fc and uc written, D_c^-1 read
    assert ab("restrict_l0") == nnz * 8 + rp + n * K * 4 + npv * 4 + n1 * (2 * K * 4 + 4)
    # P, uc read, f read, u written, D^-1 read
    assert ab("prolong_l0") == npv * 4 + n1 * K * 4 + 2 * n * K * 4 + n * 4
    assert ab("coarse_levels") is None
    assert bench.alu_ops("spmv_cg", LV, K) == 9000 * K * 11 + 1000 * K * 14
    assert bench.alu_ops("restrict_l0", LV, K) is None
    assert bench.ALU_PEAK_OPS == pytest.approx(152 * 128 * 2.07e9)


def test_roofline_counts_float64_and_fp64_cg_modes():
    ab = lambda k, m: bench.algorithmic_bytes(k, LV, K, m)  # noqa: E731
    assert ab("spmv_cg", "f64") == ab("spmv_cg", "f32c_f64") == nnz * 12 + rp + 2 * n * K * 8
    # x, r read and written, p, q read, u0 stored (cycle width), f0 = fl32(r) in the float32 cycle
    assert ab("cg_update", "f64") == 6 * n * K * 8 + n * 8 + n * K * 8
    assert ab("cg_update", "f32c_f64") == 6 * n * K * 8 + n * 8 + n * K * 4 + n * K * 4
    assert ab("cg_direction", "f64") == n * K * 24 and ab("cg_direction", "f32c_f64") == n * K * 20
    assert ab("smooth_l0", "f64") == nnz * 12 + rp + n * 8 + 3 * n * K * 8
    assert ab("smooth_l0", "f32c_f64") == nnz * 8 + rp + n * 4 + n * K * 20
    assert ab("restrict_l0", "f64") == nnz * 12 + rp + 2 * n * K * 8 + npv * 8 + n1 * (2 * K * 8 + 8)
    assert ab("prolong_l0", "f32c_f64") == npv * 4 + n1 * K * 4 + 2 * n * K * 4


def test_double_float_counts_at_the_headline_size():
    """At 1024^2 with 32 columns the update moves 805 MB (not the 1.9 GB of
    the earlier count that still stored x and u0) and the post-smoother
    621 MB."""
    lv = {"n0": 1048576, "nnz0": 9424900, "n1": 262144, "npv1": 4194304}
    assert bench.algorithmic_bytes("cg_update", lv, 32, "df") == 805306368
    assert bench.algorithmic_bytes("smooth_l0", lv, 32, "df") == pytest.approx(621e6, rel=0.01)


def test_whole_job_value_is_per_rhs_over_all_ranks():
    assert bench.whole_job_ms_per_rhs(1000.0, 5, 32, 1) == pytest.approx(1000.0 / 5 / 32)
    assert bench.whole_job_ms_per_rhs(1000.0, 5, 32, 4) == pytest.approx(1000.0 / 5 / 128)


def test_restriction_by_r_counts():
    """With R = P^T (I - A D^-1) (one pre-sweep) the level-0 restriction reads
    R once (pattern offsets and coarse starts, 4-byte columns, values per
    entry), f once, D_c^-1 once, and writes fc and uc."""
    nagg, ent, rs = 250, 250 * 36, 4
    lv = dict(LV, nagg1=nagg, rf_entries=ent, rf_rs=rs)
    for mode, w in (("df", 4), ("f32c_f64", 4), ("f64", 8)):
        assert bench.algorithmic_bytes("restrict_l0", lv, K, mode) == (
            8 * (nagg + 1) + ent * (4 + rs * w) + n * K * w + n1 * (2 * K * w + w))
    # without R the CSR count stands
    assert bench.algorithmic_bytes("restrict_l0", dict(lv, rf_entries=0), K, "df") == \
        bench.algorithmic_bytes("restrict_l0", LV, K, "df")
    # at 1024^2, 32 columns, aggregates of 16 with 4 x 4 blocks of a 9-point stencil
    # (36 halo rows each): 248 MB, against 299 MB for the CSR form
    big = {"n0": 1048576, "nnz0": 9424900, "n1": 262144, "npv1": 4194304, "nagg1": 65536,
           "rf_entries": 65536 * 36, "rf_rs": 4}
    assert bench.algorithmic_bytes("restrict_l0", big, 32, "df") == pytest.approx(248e6, rel=0.01)
