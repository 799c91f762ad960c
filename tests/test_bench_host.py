"""Host logic of the benchmark (no GPU): the algorithmic byte and flop counts
behind the roofline, and the source-hash check that voids a stale ncu
traffic figure."""
import os
import shutil

import pytest

import bench


def test_spmm_algorithmic_bytes():
    """One read of the CSR (values and column indices), the row offsets, X read
    and Y written: the 1e6 x 5e5 FP32 case at b = 8 is 135,963,516 bytes."""
    assert bench.spmm_bytes(1_000_000, 500_000, 12_495_439, 8, 4) == 135_963_516
    assert bench.spmm_bytes(10, 5, 20, 1, 8) == 20 * 12 + 44 + 2 * 8 * 5


def test_kernel_hash_sees_only_the_named_functions(tmp_path, monkeypatch):
    src_dir = tmp_path / "paper_1408_5535_gb300" / "csrc"
    src_dir.mkdir(parents=True)
    orig = os.path.join(bench.ROOT, "paper_1408_5535_gb300", "csrc", "k_small.cu")
    shutil.copy(orig, src_dir / "k_small.cu")
    h0 = bench.kernel_source_sha256("k_small.cu", bench.JACOBI_FUNCS)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.kernel_source_sha256("k_small.cu", bench.JACOBI_FUNCS) == h0
    text = (src_dir / "k_small.cu").read_text()
    (src_dir / "k_small.cu").write_text("// an unrelated comment\n" + text)
    assert bench.kernel_source_sha256("k_small.cu", bench.JACOBI_FUNCS) == h0
    edited = text.replace("__device__ inline void rot_params(double app",
                          "__device__ inline void rot_params(double  app", 1)
    assert edited != text
    (src_dir / "k_small.cu").write_text(edited)
    assert bench.kernel_source_sha256("k_small.cu", bench.JACOBI_FUNCS) != h0
    assert bench.kernel_source_sha256("k_small.cu", ["no_such_kernel"]) is None


def test_measured_traffic_is_voided_by_a_source_change(tmp_path, monkeypatch):
    assert bench.measured_traffic("k_small.cu", bench.JACOBI_FUNCS, "jacobi_fp32_targets_grid32.txt",
                                  "dram_bytes_per_call") == 133376.0
    (tmp_path / "profiles").mkdir()
    shutil.copy(os.path.join(bench.ROOT, "profiles", "jacobi_fp32_targets_grid32.txt"), tmp_path / "profiles")
    src_dir = tmp_path / "paper_1408_5535_gb300" / "csrc"
    src_dir.mkdir(parents=True)
    text = open(os.path.join(bench.ROOT, "paper_1408_5535_gb300", "csrc", "k_small.cu")).read()
    (src_dir / "k_small.cu").write_text(text.replace("const double h = x * (y * y);", "const double h = (y * y) * x;"))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.measured_traffic("k_small.cu", bench.JACOBI_FUNCS, "jacobi_fp32_targets_grid32.txt",
                                  "dram_bytes_per_call") is None
    assert bench.measured_traffic("k_small.cu", bench.JACOBI_FUNCS, "missing.txt", "dram_bytes_per_call") is None


def test_roofline_of_the_projected_eigensolve_class():
    prof = {"n_class": [10, 0, 0, 0, 0, 300] + [0] * 6, "t_class_ms": [1.0, 0, 0, 0, 0, 60.0] + [0] * 6,
            "jacobi_calls": 200, "jacobi_dim_sum": 200 * 27, "jacobi_rotations": 200 * 700, "spmm_c_width": 4,
            "iters_stage1_fp32": 0}
    r = bench.roofline_for(None, prof, 5, 6761.6, "measured")
    flops = 18.0 * 27 * 700
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    assert r["flops_per_solve_call"] == pytest.approx(flops)
    assert r["achieved"] == pytest.approx(flops / 0.3e-3 / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    assert r["launches_per_call"] == pytest.approx(1.5)


def test_roofline_of_an_fp32_class_is_bandwidth():
    """FP32 classes (mixed stage 1): the counted algorithmic bytes over the
    class's device time, against the measured HBM rate."""
    b = bench.spmm_bytes(1000, 500, 4000, 4, 4)
    prof = {"n_class": [0] * 6 + [10, 0, 0, 0, 0, 0], "t_class_ms": [0.0] * 6 + [2.0, 0, 0, 0, 0, 0],
            "class_flops": [0.0] * 6 + [10 * 4 * 4000 * 4.0] + [0.0] * 5,
            "class_bytes": [0.0] * 6 + [10.0 * b] + [0.0] * 5, "jacobi_calls": 0}
    r = bench.roofline_for(None, prof, 6, 6761.6, "measured")
    assert r["bound"] == "hbm" and r["bytes_per_launch"] == b
    assert r["achieved"] == pytest.approx(b / 0.2e-3 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / 6761.6)


def test_roofline_of_an_fp64_class_is_the_fp64_pipe():
    """FP64 classes: counted algorithmic flops over the class's device time,
    against GB300's FP64 peak (they lie far above its FP64 ridge)."""
    prof = {"n_class": [0, 4, 0, 0, 0, 0] + [0] * 6, "t_class_ms": [0.0, 8.0, 0, 0, 0, 0] + [0.0] * 6,
            "class_flops": [0.0, 4 * 8.8e8, 0, 0, 0, 0] + [0.0] * 6,
            "class_bytes": [0.0, 4 * 2.4e8, 0, 0, 0, 0] + [0.0] * 6, "jacobi_calls": 0}
    r = bench.roofline_for(None, prof, 1, 6761.6, "measured")
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    assert r["achieved"] == pytest.approx(4 * 8.8e8 / 8e-3 / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / 1.25)
    assert r["flops_per_launch"] == pytest.approx(8.8e8)


def test_oracle_samples_are_scaled_by_the_recorded_iterations():
    import argparse
    ns = argparse.Namespace(workload="c3", grid=64, sigma_log=1.0, k=20, block=8, precond="none")
    gi = bench.golden_iters(ns)
    assert gi and gi > 0
    v, est, total, gold = bench._scaled(ns, 20, {"seconds": 10.0, "iters": 5, "finished": False}, 999)
    assert gold and total == gi and est == pytest.approx(10.0 / 5 * gi) and v == pytest.approx(20 / est)
    v, est, total, gold = bench._scaled(ns, 20, {"seconds": 10.0, "iters": 5, "finished": True}, 999)
    assert est == 10.0
