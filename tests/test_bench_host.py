"""Host-side logic of bench.py (no GPU): the kernel-variant decoding reported with the
roofline, the algorithmic byte counts, the peak lookup, and the DRAM-traffic record's
freshness check (a record taken on another source of the kernel must not be reported)."""
import hashlib
import json
import os

import pytest

torch = pytest.importorskip("torch")
import bench  # noqa: E402


def test_variant_names_decode_the_option_encoding():
    assert bench.variant_names(None) is None and bench.variant_names(-1) is None
    v = bench.variant_names(0 + 4 * 3 + 16 * 3 + 64)
    assert v["row_r2c"] == "k_row_r2c<float, 8>"
    assert v["col_matvec"] == "k_col<float, 4, 2>"
    assert v["row_c2r_combine"] == "k_row_c2r<float, 4, 1>"
    assert v["col_q4"] is True and v["code"] == 124
    v = bench.variant_names(2 + 4 * 1 + 16 * 2)
    assert v["row_r2c"] == "k_row_r2c_w<float>"
    assert v["col_matvec"] == "k_col_matvec_par<float, 8>"
    assert v["row_c2r_combine"] == "k_row_combine_w<float>"
    assert v["col_q4"] is False
    v = bench.variant_names(3 + 4 * 3 + 16 * 2 + 256)
    assert v["col_matvec"] == "k_col_pair<N>" and v["row_r2c"] == "k_row_r2c<float, 4>"
    assert v["row_c2r_combine"] == "k_row_combine_w<float>" and v["code"] == 303
    v = bench.variant_names(3 + 4 * 3 + 16 * 3 + 256 + 512)
    assert v["col_matvec"] == "k_col_pair<N>" and v["row_c2r_combine"] == "k_comb_pair<M/2>"
    assert bench.variant_names(3 + 4 * 3 + 16 * 3 + 1792)["row_r2c"] == "k_row_r2c_pair<M/2>"


def test_algorithmic_bytes():
    P, T = 1024 * 1024, 4
    assert bench.algorithmic_bytes("col_matvec", P, T, 2) == 16 * P  # 4.2 MB in, 12.6 MB out
    assert bench.algorithmic_bytes("row_c2r_combine", P, T, 2) == 36 * P
    assert bench.algorithmic_bytes("residual", P, T, 2) == 52 * P
    assert bench.algorithmic_bytes("gmres_dots", P, T, 2) == 12 * P
    assert bench.algorithmic_bytes("nonexistent", P, T, 2) is None


def test_peaks_read_the_measured_file_or_fall_back():
    v, src = bench.peaks()
    if os.path.exists(os.path.join(bench.ROOT, "MEASURED_PEAKS.json")):
        assert src == "measured" and v > 1000
    else:
        assert src == "fallback" and v == 6800.0


def test_traffic_record_is_reported_only_for_the_current_source(tmp_path, monkeypatch):
    src = tmp_path / "kernel.cu"
    src.write_text("__global__ void k() {}\n")
    sha = hashlib.sha256(src.read_bytes()).hexdigest()[:16]
    (tmp_path / "profiles").mkdir()
    rec = {"col_matvec": {"bytes_per_launch": 123, "size": 1024, "source": "kernel.cu",
                          "source_sha": sha}}
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.traffic_for("col_matvec", 1024) == 123
    assert bench.traffic_for("col_matvec", 2048) is None      # other size
    assert bench.traffic_for("residual", 1024) is None        # no record
    src.write_text("__global__ void k() { /* changed */ }\n")
    assert bench.traffic_for("col_matvec", 1024) is None      # source changed since


def test_reference_arm_line_describes_the_region_it_timed():
    # the reference arm (the CPU oracle on all host cores): its steps x ms_per_step must fit
    # in the wall time of the run, its config must be the benchmark's own, and its core count
    # the processes it used
    import subprocess
    import sys
    import time
    t0 = time.time()
    out = subprocess.run([sys.executable, os.path.join(bench.ROOT, "bench.py"), "--impl",
                          "reference", "--steps", "2", "--warmup", "1", "--size", "64"],
                         capture_output=True, text=True, timeout=300, check=True).stdout
    wall = time.time() - t0
    line = json.loads(out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["steps"] == 2 and line["warmup"] == 1
    assert line["steps"] * line["ms_per_step"] / 1000.0 <= wall
    assert line["config"] == bench.workload_config(64, 1)
    assert line["cpu_baseline"]["cores"] == bench.host_cores()
    assert line["value"] > 0 and line["e2e"]["value"] == line["value"]


def test_extrapolation_counts_every_residual_and_matvec():
    counts = dict(newton=13, halvings=7, gmres=91, cycles=13)
    # 21 residual evaluations, 91 + 0 + 13 matvecs
    assert bench.extrapolate(1.0, 2.0, 3.0, counts) == 1.0 + 21 * 2.0 + 104 * 3.0
