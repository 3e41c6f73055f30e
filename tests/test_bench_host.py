"""Host logic of bench.py (CPU): the sweep-kernel naming rule matches the library's launcher,
committed traffic numbers are looked up by source hash, and job rates use the max over ranks."""
import os
import re

import numpy as np

import bench
import mdp_synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _constant(path, name):
    with open(os.path.join(ROOT, path)) as f:
        m = re.search(r"constexpr\s+int\s+" + name + r"\s*=\s*(\d+)\s*;", f.read())
    assert m, name
    return int(m.group(1))


def test_window_rule_matches_the_library():
    ring = _constant("paper_2211_04299_gb300/csrc/sweep.cu", "WIN_RING")
    nb = _constant("paper_2211_04299_gb300/csrc/sweep.cu", "WIN_NB")
    assert bench.WIN_SPAN_MAX == (ring - 2 * nb) // 2
    assert bench.WIN_MIN_S == 4 * nb


def test_sweep_kernel_names():
    banded = mdp_synth.ell_banded(5000, 4, 8, 300, 40, 0.9, seed=1, val_dtype=np.float32)
    uniform = mdp_synth.ell_uniform(5000, 4, 8, 0.9, seed=2, val_dtype=np.float32)
    wide = mdp_synth.ell_banded(9000, 6, 8, 1800, 10, 0.9, seed=3, val_dtype=np.float32)
    small = mdp_synth.ell_banded(900, 4, 8, 100, 10, 0.9, seed=4, val_dtype=np.float32)
    dense = mdp_synth.tiny_random(50, 2, seed=5, kind="dense")
    assert bench.sweep_kernel_name(banded) == "sweep_ell_window_kernel"
    assert bench.sweep_kernel_name(uniform) == "sweep_ell_warp_kernel"
    assert bench.sweep_kernel_name(wide) == "sweep_ell_warp_kernel"   # reach above 1792
    assert bench.sweep_kernel_name(small) == "sweep_ell_warp_kernel"  # S below 4 steps
    assert bench.sweep_kernel_name(dense) == "sweep_dense_tma_kernel"


def test_traffic_lookup_needs_the_current_source_hash(tmp_path, monkeypatch):
    entry = {"k": {"dram_bytes_per_launch": 123.0, "source_hash": bench.source_hash()},
             "old": {"dram_bytes_per_launch": 5.0, "source_hash": "0000000000000000"}}
    (tmp_path / "profiles").mkdir()
    import json
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps(entry))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "source_hash", lambda: entry["k"]["source_hash"])
    assert bench.traffic_for("k") == 123.0
    assert bench.traffic_for("old") is None
    assert bench.traffic_for("missing") is None


def test_job_rate_single_rank():
    assert abs(bench.job_rate(20, 2.0, 1) - 10.0) < 1e-12


def test_both_arms_share_the_config_object():
    """The oracle arm's line carries the same config keys and values as the GPU arm's (the
    GPU arm adds nothing else to config), with the CPU model and core count beside it."""
    import argparse
    args = argparse.Namespace(config=2, S=bench.S_, forcing_c=0.0, precond_block=0, gpus=1,
                              steps=2, warmup=0)
    syn = mdp_synth.dense_dirichlet(64, 8, 0.1, bench.GAMMA, seed=1)
    cfg = dict(bench.config_fields(args, syn), parallelism="replicas x1")
    line = bench.reference_line(args, 0.5, 4.0, cfg, "sample")
    assert line["config"] == cfg
    for key in ("S", "A", "gamma", "tol", "alpha", "restart", "workload"):
        assert key in cfg
    assert line["cpu_baseline"]["cpu"] and line["cpu_baseline"]["cores"] >= 1
    assert line["ms_per_step"] == 2000.0
