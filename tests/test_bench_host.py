"""Host logic of bench.py that needs no GPU: the hash-checked DRAM traffic
record of the dominant kernel and the fit's phase clocks per LM iteration."""
import hashlib
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _write_record(root, src_text: str, recorded_text: str, nbytes: int):
    os.makedirs(os.path.join(root, "profiles"))
    os.makedirs(os.path.join(root, "src"))
    with open(os.path.join(root, "src", "k.cu"), "w") as f:
        f.write(src_text)
    h = hashlib.sha256(recorded_text.encode()).hexdigest()[:16]
    rec = {"k_lm_fit": {"source": "src/k.cu", "source_sha256_16": h, "bytes_per_launch": nbytes}}
    with open(os.path.join(root, "profiles", "traffic.json"), "w") as f:
        json.dump(rec, f)


def test_traffic_record_used_only_while_the_source_matches(tmp_path, monkeypatch):
    import bench
    root = str(tmp_path / "same")
    _write_record(root, "kernel v1", "kernel v1", 1234)
    monkeypatch.setattr(bench, "ROOT", root)
    rec = bench._traffic_record()
    assert rec["k_lm_fit"]["bytes_per_launch"] == 1234

    root2 = str(tmp_path / "changed")
    _write_record(root2, "kernel v2", "kernel v1", 1234)
    monkeypatch.setattr(bench, "ROOT", root2)
    assert bench._traffic_record() == {}            # the counters belong to another source


def test_traffic_record_missing_or_broken_file(tmp_path, monkeypatch):
    import bench
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench._traffic_record() == {}
    os.makedirs(tmp_path / "profiles")
    (tmp_path / "profiles" / "traffic.json").write_text("{not json")
    assert bench._traffic_record() == {}


def test_fit_phases_per_lm_iteration():
    import bench
    st = {"lm_iters": 2000, "lm_passes": 1900, "fit_refinements": 500, "fit_fallbacks": 3,
          "fit_pass_ms": 10.0, "fit_reduce_ms": 8.0, "fit_solve_ms": 20.0, "fit_factor_ms": 15.0,
          "fit_subst_ms": 3.0}
    ph = bench._fit_phases(st)
    assert ph["lm_iters"] == 2000 and ph["passes"] == 1900
    assert ph["refinements"] == 500 and ph["fp64_fallbacks"] == 3
    us = ph["us_per_lm_iter"]
    assert us["pixel_pass"] == pytest.approx(5.0)        # 10 ms / 2000 solves
    assert us["chi2_decision_reduction"] == pytest.approx(4.0)
    assert us["solve_total"] == pytest.approx(10.0)
    assert us["damped_solve"] == pytest.approx(7.5)
    assert us["post_solve_checks"] == pytest.approx(1.5)
    # no fit ran: no division by zero
    zero = dict(st, lm_iters=0, fit_pass_ms=0.0)
    assert bench._fit_phases(zero)["us_per_lm_iter"]["pixel_pass"] == 0.0


def test_rooflines_from_algorithmic_work():
    """Each kernel class's achieved rate is the method's algorithmic work over
    its event-timed launch time, against the measured peak of its bound."""
    import bench
    m = {"N": 1024 * 1024,
         "kernels": {"k_lm_fit": {"launches": 10, "total_ms": 100.0}, "k_sub_h": {"launches": 10, "total_ms": 3.0},
                     "k_sub_v_argmax": {"launches": 10, "total_ms": 1.0},
                     "k_smooth_h": {"launches": 10, "total_ms": 4.0},
                     "k_smooth_v_argmax": {"launches": 10, "total_ms": 4.0},
                     "k_argmax_abs": {"launches": 2, "total_ms": 0.01}},
         "prof": {"fit_flops": 4e12, "fit_pass_ms": 40.0, "fit_ex2": 1e11, "sub_bytes": 8e9, "sub_flops": 4e10,
                  "smooth_flops": 8e10, "smooth_iters": 100}}
    alu = {"fp32_fma_tflops": 76.0, "fp32_fma2_tflops": 80.0, "ex2_gops": 10000.0}
    r = bench.rooflines(m, {"hbm_gbs": 6800.0}, alu)
    f = r["k_lm_fit"]
    assert f["peak"] == 80.0 and f["achieved"] == pytest.approx(40.0) and f["frac"] == pytest.approx(0.5)
    assert f["pixel_pass_only"]["achieved"] == pytest.approx(100.0)
    assert f["ex2"]["achieved_gops"] == pytest.approx(1000.0) and f["ex2"]["frac"] == pytest.approx(0.1)
    s = r["k_sub_h+k_sub_v_argmax"]
    assert s["achieved"] == pytest.approx(2000.0) and s["frac"] == pytest.approx(2000.0 / 6800.0)
    sm = r["k_smooth_h+k_smooth_v_argmax"]
    assert sm["achieved"] == pytest.approx(10.0) and sm["hbm_gbs"] == pytest.approx(4.0 * 1024 * 1024 * 100 / 8e-3 / 1e9)
    assert r["k_argmax_abs"]["achieved"] == pytest.approx(4.0 * 1024 * 1024 * 2 / 1e-5 / 1e9)


def test_fft_update_roofline_and_absent_classes():
    """The FFT residual update's rate is 124 N bytes per update over its
    event time; classes that did not launch get no entry (no division by
    zero)."""
    import bench
    m = {"N": 1024 * 1024,
         "kernels": {"k_lm_fit": {"launches": 10, "total_ms": 100.0}, "k_sub_h": {"launches": 0, "total_ms": 0.0},
                     "k_sub_v_argmax": {"launches": 0, "total_ms": 0.0},
                     "subtraction (FFT)": {"launches": 10, "total_ms": 0.5}},
         "prof": {"fit_flops": 4e12, "fit_pass_ms": 40.0, "fit_ex2": 1e11, "sub_bytes": 0.0, "sub_flops": 0.0,
                  "smooth_flops": 0.0, "smooth_iters": 0}}
    alu = {"fp32_fma_tflops": 76.0, "fp32_fma2_tflops": 80.0, "ex2_gops": 10000.0}
    r = bench.rooflines(m, {"hbm_gbs": 6800.0}, alu)
    assert "k_sub_h+k_sub_v_argmax" not in r and "k_smooth_h+k_smooth_v_argmax" not in r
    f = r["subtraction (FFT)"]
    assert f["achieved"] == pytest.approx(124.0 * 1024 * 1024 * 10 / 5e-4 / 1e9)
    assert f["us_per_update"] == pytest.approx(50.0)
