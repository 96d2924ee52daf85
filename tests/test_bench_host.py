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
