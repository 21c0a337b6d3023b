"""Host logic of bench.py that shapes the reported line: precision tokens, the roofline arithmetic of
the FP64 product and of the FP32 defect, and the rule that a recorded DRAM traffic is used only while
the captured kernel source is unchanged."""
import hashlib
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


@pytest.fixture(scope="module")
def bench():
    saved = sys.argv
    sys.argv = ["bench.py"]
    try:
        import bench as b
    finally:
        sys.argv = saved
    return b


def test_precision_tokens(bench):
    assert bench.split_precision("f64") == ("f64", "f64")
    assert bench.split_precision("bf16") == ("bf16", "f64")
    assert bench.split_precision("bf16+f32d") == ("bf16", "f32")
    assert bench.split_precision("f32+f32d") == ("f32", "f32")
    for bad in ("fp16", "bf16+f64d", "bf16+", "+f32d"):
        with pytest.raises(ValueError):
            bench.split_precision(bad)
    assert bench.dtype_label("f64") == "f64"
    assert "f32 V-cycle defects" in bench.dtype_label("bf16+f32d")
    assert "bf16 cell inverses" in bench.dtype_label("bf16+f32d")
    assert "defects" not in bench.dtype_label("bf16")


def _prof(ms, launches, nbytes):
    return {"ms": ms, "launches": launches, "bytes": nbytes}


def test_defect_roofline_arithmetic(bench):
    # 10 launches of 180 MB in 0.5 ms: 50 us per launch, 3.6 TB/s
    r = {"finest": {"defect_f32": _prof(0.5, 10, 10 * 180e6)}}
    rl = bench.defect_roofline(r, None, 7200.0, "test peak", "no_such_workload")
    assert rl["bound"] == "hbm" and rl["unit"] == "GB/s"
    assert rl["avg_launch_us"] == pytest.approx(50.0)
    assert rl["bytes_per_launch"] == pytest.approx(180e6)
    assert rl["achieved"] == pytest.approx(3600.0)
    assert rl["frac"] == pytest.approx(0.5)
    assert rl["traffic"] is None
    assert bench.defect_roofline({"finest": {"defect_f32": _prof(0.0, 0, 0.0)}}, None, 7200.0, "", "x") is None


def test_fp64_product_roofline_arithmetic(bench):
    # 2 nnz flop per launch: nnz = 1e8 in 100 us is 2 TFLOP/s, against a 1.25 TFLOP/s pipe
    r = {"finest": {"jacobian_spmv": _prof(1.0, 10, 10 * 8.0e8)}}
    rl = bench.spmv_roofline(r, None, [{"nnz": int(1e8)}], 1.25, "no_such_workload")
    assert rl["bound"] == "alu" and rl["unit"] == "TFLOP/s"
    assert rl["avg_launch_us"] == pytest.approx(100.0)
    assert rl["achieved"] == pytest.approx(2.0)
    assert rl["frac"] == pytest.approx(1.6)
    assert rl["hbm_gbs_algorithmic"] == pytest.approx(8000.0)


def test_recorded_traffic_needs_the_captured_source(bench, tmp_path, monkeypatch):
    src = tmp_path / "kernel.cu"
    src.write_text("// captured source\n")
    sha = hashlib.sha256(src.read_bytes()).hexdigest()
    (tmp_path / "profiles").mkdir()
    rec = {"captures": [{"workload": "w", "precision": "f32", "kernel": "k", "source": "kernel.cu",
                         "source_sha256": sha, "dram_bytes_read": 100.0, "dram_bytes_write": 20.0,
                         "profile": "profiles/k.md"}]}
    (tmp_path / "profiles" / "roofline_traffic.json").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.recorded_traffic("w", "k")["per_launch_bytes"] == 120.0
    assert bench.recorded_traffic("w", "k", "f32")["per_launch_bytes"] == 120.0
    assert bench.recorded_traffic("w", "k", "bf16") is None
    assert bench.recorded_traffic("other", "k") is None
    src.write_text("// changed source\n")
    assert bench.recorded_traffic("w", "k") is None


def test_committed_traffic_records_name_existing_profiles(bench):
    rec = json.load(open(os.path.join(ROOT, "profiles", "roofline_traffic.json")))
    for e in rec["captures"]:
        assert os.path.exists(os.path.join(ROOT, e["profile"])), e["profile"]
        assert os.path.exists(os.path.join(ROOT, e["source"])), e["source"]
        assert e["dram_bytes_read"] > 0 and e["dram_bytes_write"] >= 0


def test_headline_is_a_conforming_mixed_run(bench):
    """The headline never comes from the FP32-defect run, however fast it is."""
    res = {"f64": {"ms_per_solve": 90.0}, "f32": {"ms_per_solve": 70.0}, "bf16": {"ms_per_solve": 60.0},
           "bf16+f32d": {"ms_per_solve": 40.0}}
    assert bench.pick_head(res) == "bf16"
    res["f32"]["ms_per_solve"] = 50.0
    assert bench.pick_head(res) == "f32"
    assert bench.pick_head({"f64": {"ms_per_solve": 1.0}, "bf16+f32d": {"ms_per_solve": 0.5}}) == "f64"


def test_full_workload_dofs_match_the_level_table(bench):
    """(k+1)(d R + n_p C) of the obstacle channels: the per-config DoF counts of the workloads."""
    import synth
    expect = {"c1_2d_k1": 5956, "c2_2d_k2": 536448, "c3_3d_k1": 962208, "c4_2d_k1": 90112, "c5_3d_k1": 7459392}
    for name, n in expect.items():
        assert bench.full_workload_dofs(synth.WORKLOADS[name]) == n


def test_cpu_baseline_scaling(bench):
    import synth
    o1 = {"threads": 1, "solve_s": [8.0, 9.0, 10.0], "iters": [11, 11, 11], "sweep_s": [0.2, 0.1, 0.3],
          "setup_s": 50.0, "sizes": {"n_dofs": 1000, "n_cells": 10, "n_local": 170, "n_levels": 2}}
    on = dict(o1, threads=15, solve_s=[4.0, 5.0, 6.0])
    e = bench.cpu_baseline_entry(o1, on, 8000, 80, 12, synth.WORKLOADS["c3_3d_k1"])
    assert e["value"] == pytest.approx(9.0 * 8)
    assert e["cores"] == 1 and e["kind"] == "oracle"
    assert e["one_thread"]["sweep_s_scaled"] == pytest.approx(0.2 * 8)
    assert e["all_threads"]["solve_s_scaled"] == pytest.approx(5.0 * 8)
    assert e["all_threads"]["threads"] == 15
