"""Host logic of bench.py, no GPU: the reference arm's JSON line (the FP64 oracle timed on
the host cores, on a smaller sample than the benchmark's so that the test stays short) and
the kernel-source hash that ties the stored DRAM-traffic figure to the code it was taken
on (comments do not count, code does)."""
import argparse
import contextlib
import io
import json
import os
import shutil

import pytest

import bench


def test_reference_arm_prints_one_complete_line(monkeypatch):
    monkeypatch.setattr(bench, "CPU_SAMPLE_SCALE", 12)
    args = argparse.Namespace(steps=2, warmup=3, scale=14, seed=0, eps=1e-8, gpus=1, workload="rmat",
                              allocator="torch")
    out = io.StringIO()
    with contextlib.redirect_stdout(out):
        bench.run_reference(args)
    lines = [l for l in out.getvalue().splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC
    assert d["value"] > 0 and d["unit"] == "edges/s" and d["higher_is_better"] is True
    assert d["steps"] == 2 and d["warmup"] == 3 and d["n_gpus"] == 1
    # the value is the sample's draws over the measured seconds per step, and the seconds
    # per step are what was measured (no extrapolation)
    draws = 16 << 12
    assert d["value"] == pytest.approx(draws / (d["ms_per_step"] / 1e3))
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] >= 1 and "scale 12" in d["cpu_baseline"]["sample"]
    assert d["cpu_baseline"]["nproc"] >= 1 and "cpu_model" in d["cpu_baseline"]
    assert d["e2e"] == {"value": d["value"], "unit": "edges/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    # the same configuration object as the GPU arm's
    assert d["config"] == bench.workload_config(args)
    assert d["config"]["workload"].startswith("rmat_scale14")


def test_parity_block_counts_near_ties_and_flags_mismatches():
    import numpy as np

    rng = np.random.default_rng(0)
    ref = rng.random(1000)
    ref[[10, 11]] = 0.999999999, 0.9999999995  # a near tie at the top
    out = {"psi": ref, "m_unique": 77, "iters": 5}
    order = np.lexsort((np.arange(ref.size), -ref))[:100]
    out["top_ids"] = order
    gpu_top = order.copy()
    i, j = list(order).index(10), list(order).index(11)
    gpu_top[i], gpu_top[j] = gpu_top[j], gpu_top[i]
    b = bench.parity_block(ref * (1 + 1e-9), (gpu_top, None), out, 77)
    assert b["rel_l1_ok"] and b["rel_l1"] == pytest.approx(1e-9, rel=1e-3)
    assert not b["top100_equal"] and b["top100_equal_up_to_near_ties"] and b["near_tie_swaps"] == 2
    assert b["m_unique_equal"]
    bad = order.copy()
    bad[0], bad[50] = bad[50], bad[0]
    b = bench.parity_block(ref, (bad, None), out, 78)
    assert not b["top100_equal_up_to_near_ties"] and not b["m_unique_equal"]


def test_oracle_memory_guard():
    assert bench.oracle_bytes(1 << 25, 16 << 25) > 20 * 2**30
    avail = bench.host_available_bytes()
    assert avail is None or avail > 0


def test_kernel_hash_follows_code_not_comments(tmp_path, monkeypatch):
    for p in bench.KERNEL_SOURCES:
        os.makedirs(tmp_path / os.path.dirname(p), exist_ok=True)
        shutil.copy(os.path.join(bench.ROOT, p), tmp_path / p)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    base = bench.kernel_sha()
    target = tmp_path / bench.KERNEL_SOURCES[0]
    text = target.read_text()
    target.write_text("// a new comment line\n\n" + text.replace("\n", "\n  \n", 1))
    assert bench.kernel_sha() == base  # comments and blank lines are not code
    target.write_text(text + "\nconstexpr int kAnotherConstant = 1;\n")
    assert bench.kernel_sha() != base
