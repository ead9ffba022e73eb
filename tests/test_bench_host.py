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
    assert d["value"] > 0 and d["unit"] == "s" and d["higher_is_better"] is False
    assert d["steps"] == 2 and d["warmup"] == 3 and d["n_gpus"] == 1
    assert d["ms_per_step"] == pytest.approx(d["value"] * 1e3)
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] >= 1 and "scale 12" in d["cpu_baseline"]["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["config"]["workload"].startswith("rmat_scale14")


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
