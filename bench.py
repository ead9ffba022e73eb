#!/usr/bin/env python3
"""Benchmark of the Power-psi hot path on GB300.

One step = the whole path on one synthetic graph: psi_graph_create (validate, renumber,
sort + merge duplicates, CSR, sigma/c/d, tile schedule), psi_solve (Power-psi to
eps = 1e-8 on the psi-tolerance eps_t/N, FP32 series + FP64 refinement, final psi) and
psi_topk (k = 100).  Default workload: R-MAT scale 25 (N = 2^25), edge factor 16,
(a, b, c) = (.57, .19, .19), random relabel, lambda, mu ~ LogNormal(0, 1.5) clipped to
[1e-3, 1e3] -- a synthetic stand-in for the paper's social graphs.

``value`` is the whole-path throughput in input edges per second (edge draws of the
workload x ranks / seconds per step) with inputs resident in HBM; ``ms_per_step`` is the
step time behind it.  ``e2e`` is the same step through the C ABI from pinned host buffers
(H2D of edges and rates, D2H of the top-k inside the timed region).  After the timed
steps the oracle solves the same graph on the host cores: its time is ``cpu_baseline``
and the comparison of its psi with the GPU's is ``parity``.  ``--impl reference`` times the
FP64 CPU oracle alone, one bounded sample of the workload per step.  Multi-GPU runs are
replicas (one independent graph per rank, weak scaling).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import platform
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Power-ψ time-to-L1<1e-8 and GTEPS/iter at N=2^25; % of HBM peak"
FALLBACK_HBM_GBS = 6800.0
# DRAM bytes per launch of the FP32 series step (k_spmv + fix-up) from one ncu capture,
# valid only while the kernel sources hash to `sha`.
NCU_TRAFFIC = {"sha": "ded6a86fa40ec657", "bytes_per_launch": 2461379255,
               "note": "k_spmv<float,EpiSeries,32> (tile 2048, 28672 entries in shared memory, tiles claimed at run "
                       "time) DRAM read + write on R-MAT scale 23 (one capture: 622.2 MB = 0.938 x the "
                       "kernel's own bytes), scaled to the scale-25 launch by its kernel bytes (2.624 GB)"}
KERNEL_SOURCES = ["paper_2206_09960_gb300/csrc/spmv.cuh", "paper_2206_09960_gb300/csrc/common.cuh"]
CPU_SAMPLE_SCALE = 20
ONE_THREAD_SCALE = 18
UNIT = "edges/s"


def kernel_sha() -> str:
    """Hash of the kernel sources' code: whole-line comments and blank lines are left out,
    so that editing a comment does not retire the stored traffic figure."""
    h = hashlib.sha256()
    for p in KERNEL_SOURCES:
        with open(os.path.join(ROOT, p), encoding="utf-8") as fh:
            for line in fh:
                t = line.strip()
                if t and not t.startswith("//"):
                    h.update(t.encode() + b"\n")
    return h.hexdigest()[:16]


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return FALLBACK_HBM_GBS, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(self.dev)], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    mx.append(float(parts[2]))
                except ValueError:
                    continue
                for name, v in zip(names, parts[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(name)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def host_info():
    """Host cores and CPU model of the machine the oracle runs on."""
    model = ""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    return {"nproc": os.cpu_count(), "cpu_model": model or platform.processor() or platform.machine()}


def oracle_seconds(w, eps, threads=None):
    """The oracle as it stands on workload `w`: canonicalise + build A, B explicitly +
    Algorithm 2 to eps on the psi-tolerance + the top-100 ranking.  Returns (seconds,
    oracle output, threads used)."""
    import oracle

    if threads:
        oracle.set_threads(threads)
    used = oracle.num_threads()
    t = time.perf_counter()
    out = oracle.solve(w["n"], w["follower"], w["leader"], w["lam"], w["mu"], eps=eps, tol_mode=oracle.TOL_PSI)
    out["top_ids"], out["top_vals"] = oracle.topk(out["psi"], 100)
    sec = time.perf_counter() - t
    if threads:
        oracle.set_threads(os.cpu_count() or 1)
    return sec, out, used


def sampled_cpu_baseline(cases, scale, sample, threads=None):
    """The oracle as it stands (canonicalise, explicit A/B, Algorithm 2, top-100) on a bounded
    sample of a secondary workload: `cases` are (workload dict, eps, tol_mode) solved one
    after another on the host cores; the line's value is their seconds times `scale` (the
    sample's share of the workload), stated in `sample`."""
    import oracle

    if threads:
        oracle.set_threads(threads)
    used = oracle.num_threads()
    t = time.perf_counter()
    for w, eps, tol in cases:
        out = oracle.solve(w["n"], w["follower"], w["leader"], w["lam"], w["mu"], eps=eps, tol_mode=tol)
        oracle.topk(out["psi"], 100)
    sec = time.perf_counter() - t
    if threads:
        oracle.set_threads(os.cpu_count() or 1)
    return {"value": sec * scale, "unit": "s", "cores": used, "kind": "oracle", "sample": sample,
            "measured_s": sec, "scaled_by": scale}


def oracle_bytes(n, draws):
    """Host memory the oracle needs for a graph: the sort keys (8 B per draw), both explicit
    CSR copies of A and B (two ids and four FP64 values per edge) and its per-user vectors."""
    return 8 * draws + 40 * draws + 64 * n


def host_available_bytes():
    """MemAvailable, capped by the cgroup's memory limit (None if neither is readable)."""
    avail = None
    try:
        with open("/proc/meminfo") as fh:
            for line in fh:
                if line.startswith("MemAvailable:"):
                    avail = int(line.split()[1]) * 1024
    except OSError:
        pass
    for path in ("/sys/fs/cgroup/memory.max", "/sys/fs/cgroup/memory/memory.limit_in_bytes"):
        try:
            with open(path) as fh:
                v = fh.read().strip()
            if v.isdigit():
                used = 0
                for upath in ("/sys/fs/cgroup/memory.current", "/sys/fs/cgroup/memory/memory.usage_in_bytes"):
                    if os.path.exists(upath):
                        with open(upath) as fh:
                            used = int(fh.read().strip() or 0)
                        break
                room = int(v) - used
                avail = room if avail is None else min(avail, room)
        except (OSError, ValueError):
            pass
    return avail


def parity_block(gpu_psi, gpu_top, out, m_unique_gpu, tol=1e-6):
    """psi of the GPU against the oracle's on the same graph: relative L1 (Eq. 12's psi, the
    spec measure), relative L2 (the paper's Eq. 23), the top-100 ids (a swap of two
    users whose oracle values differ by less than tol relative to them counts as a near
    tie, not a mismatch) and the unique edge count (bit-exact)."""
    import numpy as np

    ref = out["psi"]
    rel_l1 = float(np.abs(gpu_psi - ref).sum() / np.abs(ref).sum())
    rel_l2 = float(np.linalg.norm(gpu_psi - ref) / np.linalg.norm(ref))
    ids_g = np.asarray(gpu_top[0])
    ids_o = np.asarray(out["top_ids"])
    exact = bool(np.array_equal(ids_g, ids_o))
    swaps = [(int(a), int(b)) for a, b in zip(ids_g, ids_o) if a != b]
    near = len(swaps)
    ok = all(abs(ref[a] - ref[b]) <= tol * max(abs(ref[a]), abs(ref[b])) for a, b in swaps)
    return {"rel_l1": rel_l1, "rel_l2": rel_l2, "tol_rel_l1": tol, "rel_l1_ok": rel_l1 <= tol,
            "top100_equal": exact, "top100_equal_up_to_near_ties": bool(ok), "near_tie_swaps": near,
            "m_unique_equal": int(out["m_unique"]) == int(m_unique_gpu),
            "psi_sum_gpu": float(gpu_psi.sum()), "psi_sum_oracle": float(ref.sum()),
            "oracle": f"FP64, same graph and stop rule, {int(out['iters'])} steps"}


def host_placement(buf):
    """Where a pinned host buffer lives relative to the GPU: the NUMA nodes of its pages (from
    /proc/self/numa_maps), the GPU's NUMA node and the host's node count (Linux only)."""
    import glob

    out = {"host_numa_nodes": len(glob.glob("/sys/devices/system/node/node[0-9]*"))}
    try:
        bus = subprocess.run(["nvidia-smi", "--query-gpu=pci.bus_id", "--format=csv,noheader", "-i",
                              os.environ.get("LOCAL_RANK", "0")], capture_output=True, text=True,
                             timeout=10).stdout.strip().lower()
        tail = bus[-12:] if bus else ""
        for d in glob.glob("/sys/bus/pci/devices/*"):
            if tail and d.lower().endswith(tail[-7:]):
                with open(os.path.join(d, "numa_node")) as fh:
                    out["gpu_numa_node"] = int(fh.read().strip())
    except (OSError, ValueError, subprocess.SubprocessError):
        pass
    try:
        addr = buf.data_ptr()
        with open("/proc/self/numa_maps") as fh:
            for line in fh:
                start = int(line.split()[0], 16)
                if start <= addr < start + buf.numel() * buf.element_size():
                    out["buffer_pages"] = " ".join(t for t in line.split() if t.startswith("N") and "=" in t)
                    break
    except (OSError, ValueError):
        pass
    return out


def host_quiesce(limit_s=60.0, quiet_s=2.0):
    """Waits (at most limit_s) until the kernel's background memory compaction has been idle
    for quiet_s: compaction that a previous process's memory churn set off was measured
    stalling DMA from pinned host memory (copies of the same buffer taking 2-8x longer),
    which is not this library's transfer.  Returns the seconds waited and the compaction
    counters moved meanwhile (Linux; nothing to wait for elsewhere)."""
    keys = ("compact_daemon_migrate_scanned", "compact_daemon_free_scanned", "compact_isolated", "pgmigrate_success")

    def counters():
        d = {}
        try:
            with open("/proc/vmstat") as fh:
                for line in fh:
                    k, v = line.split()
                    if k in keys:
                        d[k] = int(v)
        except OSError:
            pass
        return d

    t0 = time.perf_counter()
    first = last = counters()
    if not first:
        return 0.0, {}
    still = 0.0
    while time.perf_counter() - t0 < limit_s and still < quiet_s:
        time.sleep(0.5)
        now = counters()
        still = still + 0.5 if now == last else 0.0
        last = now
    return time.perf_counter() - t0, {k: last[k] - first[k] for k in last if last[k] != first[k]}


def pinned_h2d_gbs(h, d, stream, reps=3):
    """Host-to-device bandwidth of one pinned input buffer (GB/s), timed with CUDA events."""
    import torch

    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    d.copy_(h, non_blocking=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(reps):
        d.copy_(h, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    return h.numel() * h.element_size() * reps / (e0.elapsed_time(e1) / 1e3) / 1e9


def run_reference(args):
    """The reference arm: the FP64 oracle alone on the host cores.  Each step is one bounded
    sample of the workload -- the whole path (canonicalise, build, Algorithm 2, ranking) on
    an R-MAT graph of the same recipe at scale CPU_SAMPLE_SCALE -- and the value is that
    sample's edge draws per second, the unit of the GPU arm."""
    import psigen

    ws, rank, _ = dist_env()
    if rank != 0:
        return
    w = psigen.workload("rmat", seed=args.seed, scale=min(CPU_SAMPLE_SCALE, args.scale))
    draws = int(w["follower"].size)
    times = []
    threads = 1
    for i in range(args.warmup + args.steps):
        sec, _, threads = oracle_seconds(w, args.eps)
        if i >= args.warmup:
            times.append(sec)
    sec = statistics.mean(times)
    v = draws / sec
    sample = (f"whole path of the oracle (canonicalise, explicit A/B, Algorithm 2 to eps={args.eps:g} on eps_t/N, "
              f"top-100) on R-MAT scale {min(CPU_SAMPLE_SCALE, args.scale)} of the same recipe ({draws} edge draws) "
              f"per step, {threads} threads")
    cpu = {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample}
    cpu.update(host_info())
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": sec * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": workload_config(args),
            "cpu_baseline": cpu,
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_batch(args, S=64, plain_sample=8):
    """64 activity scenarios (lambda, mu ~ LogNormal(0, 1) each) on one R-MAT graph (default
    scale 22, edge factor 16): one batched solve against the plain form (one graph and one
    solve per scenario, timed on `plain_sample` scenarios and scaled to S)."""
    import numpy as np
    import torch

    import psigen
    import paper_2206_09960_gb300 as psi

    scale = 22 if args.scale == 25 else args.scale
    psi.load(build_if_missing=False)
    n = 1 << scale
    f, l = psigen.rmat_graph(scale, 16, *psigen.RMAT_ABC, args.seed, relabel=True)
    lam = np.stack([psigen.lognormal_rates(n, 0.0, 1.0, 1e-3, 1e3, args.seed * 1000 + q, 301) for q in range(S)])
    mu = np.stack([psigen.lognormal_rates(n, 0.0, 1.0, 1e-3, 1e3, args.seed * 1000 + q, 302) for q in range(S)])
    f_d, l_d = torch.from_numpy(f).cuda(), torch.from_numpy(l).cuda()
    lam_d, mu_d = torch.from_numpy(lam).cuda(), torch.from_numpy(mu).cuda()
    stream = torch.cuda.current_stream()

    def timed(fn, reps):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        outs = [fn() for _ in range(reps)]
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3 / reps, outs[-1]

    def batched(profile=False):
        with psi.Batch(n, f_d, l_d, lam_d, mu_d, stream=stream, profile=profile) as b:
            status, infos = b.solve(args.eps, 100000)
            st = b.stats()
        return status, infos, st

    def plain():
        infos = []
        for q in range(plain_sample):
            with psi.Graph(n, f_d, l_d, lam_d[q], mu_d[q], stream=stream) as g:
                infos.append(g.solve(args.eps, 100000))
        return infos

    clocks = Clocks(torch.cuda.current_device())
    clocks.start()
    t_batch, (status, infos, st) = timed(batched, args.steps)
    clk = clocks.stop()
    _, pinfo, _ = batched(profile=True)
    t_plain, pinfos = timed(plain, 1)
    # series product of the batch: 4 B per nonzero, the compulsory read of every gathered
    # user's 64-value row, and per row mu, 1/sigma, s (read and write) and the new term for
    # each scenario
    step_ms = pinfo[0]["spmv_ms"] / max(pinfo[0]["spmv_timed"], 1)
    alg = 4 * st["m_unique"] + 4 * (st["n_rows"] + 1) + 4 * S * st["n_gathered"] + 28 * S * st["n_rows"]
    peak, peak_kind = measured_peaks()
    roofline = {"bound": "hbm", "achieved": alg / step_ms / 1e6, "peak": peak, "unit": "GB/s",
                "frac": alg / step_ms / 1e6 / peak, "traffic": None, "peak_kind": peak_kind,
                "kernel": "k_spmm_claims<EpiSeriesS> + fix-up (batched FP32 series step, chunks claimed at run time)",
                "alg_bytes_per_launch": alg, "avg_launch_ms": step_ms, "launches_timed": pinfo[0]["spmv_timed"]}
    t_plain_all = t_plain * S / plain_sample
    solve_batch = infos[0]["ms"] / 1e3
    solve_plain = sum(i["ms"] for i in pinfos) / 1e3 * S / plain_sample
    line = {"metric": "batched Power-psi: 64 activity scenarios on one graph, time to L1<1e-8 for all",
            "value": t_batch, "unit": "s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "higher_is_better": False, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"rmat_scale{scale}_ef16_64_scenarios_lognormal1", "n": n, "scenarios": S,
                       "m_unique": st["m_unique"], "eps": args.eps},
            "status": status, "iters_max": max(i["iters"] for i in infos),
            "iters_mean": sum(i["iters"] for i in infos) / S,
            "batch_solve_s": solve_batch, "plain_s_for_64": t_plain_all, "plain_solve_s_for_64": solve_plain,
            "speedup_total": t_plain_all / t_batch, "speedup_solve": solve_plain / solve_batch,
            "plain_sample": plain_sample, "clocks": clk, "roofline": roofline}
    if not args.no_cpu_baseline:  # one scenario of the 64 through the oracle, scaled by 64
        import oracle

        w0 = dict(n=n, follower=f, leader=l, lam=lam[0], mu=mu[0])
        line["cpu_baseline"] = sampled_cpu_baseline(
            [(w0, args.eps, oracle.TOL_PSI)], S, f"scenario 0 of {S} on the same graph, oracle solve to eps, "
                                               f"times {S}")
    print(json.dumps(line), flush=True)


def multi_roofline(st, solve_s, iters):
    """Whole-solve roofline of the independent-graph object: every step reads each graph's
    column indices and per-user vectors once (4M + 32N per step while the graph steps,
    averaged over the graphs' step counts), divided by the solve time; the replayed CUDA
    graphs leave no per-launch timing."""
    peak, peak_kind = measured_peaks()
    mean_steps = sum(iters) / len(iters)
    alg = (4 * st["m_unique"] + 32 * st["n"]) * mean_steps
    return {"bound": "hbm", "achieved": alg / solve_s / 1e9, "peak": peak, "unit": "GB/s",
            "frac": alg / solve_s / 1e9 / peak, "traffic": None, "peak_kind": peak_kind,
            "kernel": "whole solve (series products, confirming steps, stop tests, final product)",
            "alg_bytes_per_solve": alg, "solve_ms": solve_s * 1e3}


def run_multi(args, G=256, plain_sample=32):
    """256 independent Chung-Lu graphs (N ~ U{1000..100000}, 12 draws per user, exponent
    2.1, lambda, mu ~ LogNormal(0, 1)) built and solved together in one object (psi_multi,
    steps replayed from a CUDA graph), against the plain form (one graph object and solve per
    graph, timed on `plain_sample` graphs and scaled by their share of the edges)."""
    import numpy as np
    import torch

    import psigen
    import paper_2206_09960_gb300 as psi

    psi.load(build_if_missing=False)
    w = psigen.multi_workload(G, seed=args.seed)
    n_g, m_g = w["n_g"], w["m_g"]
    dev = [torch.from_numpy(np.ascontiguousarray(w[k])).cuda() for k in ("follower", "leader", "lam", "mu")]
    stream = torch.cuda.current_stream()

    def timed(fn, reps):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        outs = [fn() for _ in range(reps)]
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3 / reps, outs[-1]

    def together():
        with psi.Multi(n_g, m_g, *dev, stream=stream) as mg:
            status, infos = mg.solve(args.eps, 100000)
            ids, _ = mg.topk(100)
            st = mg.stats()
        return status, infos, st

    eo = np.concatenate([[0], np.cumsum(m_g)])
    no = np.concatenate([[0], np.cumsum(n_g)])
    sample = list(range(0, G, max(1, G // plain_sample)))[:plain_sample]

    def plain():
        infos = []
        for q in sample:
            with psi.Graph(int(n_g[q]), dev[0][eo[q]:eo[q + 1]], dev[1][eo[q]:eo[q + 1]], dev[2][no[q]:no[q + 1]],
                           dev[3][no[q]:no[q + 1]], stream=stream) as g:
                infos.append(g.solve(args.eps, 100000))
                g.topk(100)
        return infos

    launches0 = psi._binding.load().psi_kernel_launches()
    clocks = Clocks(torch.cuda.current_device())
    clocks.start()
    t_multi, (status, infos, st) = timed(together, args.steps)
    clk = clocks.stop()
    if args.profile_solve:  # one more solve of the built object inside a profiler range (for ncu)
        with psi.Multi(n_g, m_g, *dev, stream=stream) as mg:
            mg.solve(args.eps, 100000)
            torch.cuda.synchronize()
            torch.cuda.profiler.start()
            mg.solve(args.eps, 100000)
            torch.cuda.synchronize()
            torch.cuda.profiler.stop()
    launches = (psi._binding.load().psi_kernel_launches() - launches0) / (args.warmup + args.steps)
    t_plain, pinfos = timed(plain, 1)
    share = float(m_g[sample].sum()) / float(m_g.sum())
    t_plain_all = t_plain / share
    solve_multi = infos[0]["ms"] / 1e3
    solve_plain = sum(i["ms"] for i in pinfos) / 1e3 / share
    iters = [i["iters"] for i in infos]
    line = {"metric": "independent graphs: 256 Chung-Lu graphs, build + Power-psi to L1<1e-8 + top-100 for all",
            "value": t_multi, "unit": "s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "higher_is_better": False, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "256 Chung-Lu graphs, N~U{1000..100000}, 12 draws/user, gamma 2.1, lognormal1",
                       "n_total": int(n_g.sum()), "m_unique": st["m_unique"], "eps": args.eps},
            "status": status, "iters_min": min(iters), "iters_max": max(iters), "iters_mean": sum(iters) / G,
            "multi_solve_s": solve_multi, "plain_s_for_256": t_plain_all, "plain_solve_s_for_256": solve_plain,
            "speedup_total": t_plain_all / t_multi, "speedup_solve": solve_plain / solve_multi,
            "plain_sample": len(sample), "gpu_launches": launches, "build_ms": st["build_ms"], "clocks": clk,
            "spmv_tile": st["spmv_tile"],
            "roofline": multi_roofline(st, solve_multi, iters)}
    if not args.no_cpu_baseline:  # every 32nd graph through the oracle, scaled by its share of the edges
        import oracle

        cases, m_s = [], 0
        for q in range(0, G, 32):
            cases.append((dict(n=int(n_g[q]), follower=w["follower"][eo[q]:eo[q + 1]],
                               leader=w["leader"][eo[q]:eo[q + 1]], lam=w["lam"][no[q]:no[q + 1]],
                               mu=w["mu"][no[q]:no[q + 1]]), args.eps, oracle.TOL_PSI))
            m_s += int(m_g[q])
        line["cpu_baseline"] = sampled_cpu_baseline(
            cases, float(m_g.sum()) / max(m_s, 1), f"{len(cases)} of {G} graphs (every 32nd), oracle solve "
                                                   "to eps each, scaled by their share of the edge draws")
    print(json.dumps(line), flush=True)


def run_pagerank(args, alpha=0.85, eps=1e-9):
    """The comparison of the paper's Table IV on the benchmark graph: PageRank's power method
    (Eq. 22, pi-tolerance eps) against Power-psi with heterogeneous activity and with the
    homogeneous activity lambda = 0.15, mu = 0.85 that reduces psi to PageRank (both on the
    s-tolerance eps, the paper's setting), all on one graph handle, solve times only."""
    import numpy as np
    import torch

    import psigen
    import paper_2206_09960_gb300 as psi

    psi.load(build_if_missing=False)
    w = psigen.workload("rmat", seed=args.seed, scale=args.scale)
    n = w["n"]
    dev = [torch.from_numpy(np.ascontiguousarray(w[k])).cuda() for k in ("follower", "leader", "lam", "mu")]
    hom = [torch.full((n,), 0.15, dtype=torch.float64, device="cuda"),
           torch.full((n,), 0.85, dtype=torch.float64, device="cuda")]
    stream = torch.cuda.current_stream()

    def timed(fn):
        res = None
        ts = []
        for rep in range(args.warmup + args.steps):
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            res = fn()
            e1.record(stream)
            torch.cuda.synchronize()
            if rep >= args.warmup:
                ts.append(e0.elapsed_time(e1) / 1e3)
        return sum(ts) / len(ts), res

    out = {}
    clocks = Clocks(torch.cuda.current_device())
    clocks.start()
    with psi.Graph(n, dev[0], dev[1], dev[2], dev[3], tol_mode="s_abs", stream=stream, profile=True) as g:
        out["psi_heterogeneous"] = timed(lambda: g.solve(eps, 100000))
        out["pagerank"] = timed(lambda: g.pagerank(alpha, eps, 100000)[1])
        st = g.stats()
    with psi.Graph(n, dev[0], dev[1], hom[0], hom[1], tol_mode="s_abs", stream=stream) as g:
        out["psi_homogeneous"] = timed(lambda: g.solve(eps, 100000))
        psi_h = g.scores()
        pi, _ = g.pagerank(alpha, eps, 100000)
        diff = float((psi_h - pi).abs().sum() / pi.abs().sum())
    clk = clocks.stop()
    pinfo = out["pagerank"][1]
    step_ms = pinfo["spmv_ms"] / max(pinfo["spmv_timed"], 1)
    alg = 4 * st["m_unique"] + 32 * n
    peak, peak_kind = measured_peaks()
    roofline = {"bound": "hbm", "achieved": alg / step_ms / 1e6, "peak": peak, "unit": "GB/s",
                "frac": alg / step_ms / 1e6 / peak, "traffic": None, "peak_kind": peak_kind,
                "kernel": "k_spmv<float,EpiSeries> + k_fixup (PageRank step of Eq. 22 in series form)",
                "alg_bytes_per_launch": alg, "avg_launch_ms": step_ms, "launches_timed": pinfo["spmv_timed"]}
    line = {"metric": "Table IV comparison: solve time of PageRank (Eq. 22) and Power-psi at eps=1e-9",
            "value": out["psi_heterogeneous"][0], "unit": "s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "higher_is_better": False, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"rmat_scale{args.scale}_ef16_a.57_b.19_c.19_relabel_lognormal1.5", "n": n,
                       "alpha": alpha, "eps": eps, "tolerance": "s-tolerance (psi), pi-tolerance (PageRank)"},
            "psi_heterogeneous_s": out["psi_heterogeneous"][0],
            "psi_heterogeneous_iters": out["psi_heterogeneous"][1]["iters"],
            "pagerank_s": out["pagerank"][0], "pagerank_iters": out["pagerank"][1]["iters"],
            "psi_homogeneous_s": out["psi_homogeneous"][0],
            "psi_homogeneous_iters": out["psi_homogeneous"][1]["iters"],
            "homogeneous_psi_vs_pagerank_rel_l1": diff, "clocks": clk, "roofline": roofline}
    if not args.no_cpu_baseline:  # the heterogeneous Power-psi solve on a scale-20 graph of the recipe
        import oracle

        ws = psigen.workload("rmat", seed=args.seed, scale=20)
        line["cpu_baseline"] = sampled_cpu_baseline(
            [(ws, eps, oracle.TOL_S_ABS)], float(n) / ws["n"],
            "R-MAT scale 20 of the same recipe (2^-5 of the edges), oracle Power-psi to the same eps on the "
            "s-tolerance, scaled by the edge ratio 32")
    print(json.dumps(line), flush=True)


# Node and edge counts of the paper's Table III graphs (Konect DBLP, HepPh, Facebook,
# Twitter) and its CPU times for Power-NF and Power-psi with heterogeneous rates (eps = 1e-9;
# another machine and the real graphs: context only).
TABLE3 = [("dblp", 12_591, 49_743, 17.805, 0.029), ("hepph", 34_546, 421_578, 272.358, 0.622),
          ("facebook", 63_731, 817_035, 1764.226, 0.307), ("twitter", 465_017, 834_797, 14526.039, 0.634)]
# and its Table IV times with homogeneous rates (lambda = 0.15, mu = 0.85): PageRank's power
# method, Power-NF and Power-psi
TABLE4 = {"dblp": (0.023, 20.775, 0.034), "hepph": (0.361, 360.769, 0.908), "facebook": (0.308, 2253.302, 0.454),
          "twitter": (0.584, 17411.146, 0.806)}


def run_powernf(args, eps=1e-9, sample=64):
    """The paper's Tables III and IV on stand-ins of its four graphs: Chung-Lu (gamma = 2.1)
    graphs with the same node and edge-draw counts and rates U(0, 1) (Sec. V's heterogeneous
    case), then the same graphs with lambda = 0.15, mu = 0.85 (the homogeneous case, with
    PageRank's power method at alpha = 0.85 and pi-tolerance eps beside).  Power-NF
    (Algorithm 1, every origin, per-origin p-tolerance eps) against Power-psi (Algorithm 2,
    FP64, s-tolerance eps) on the same graph handle, solve times only, and the largest psi
    difference between the two.  The oracle's Algorithm 1 runs on a few
    origins of every graph (parity, one by one), and on `sample` random origins of the
    largest for the CPU baseline."""
    import numpy as np
    import torch

    import oracle
    import psigen
    import paper_2206_09960_gb300 as psi

    psi.load(build_if_missing=False)
    stream = torch.cuda.current_stream()

    def timed(fn, reps, warm):
        res = None
        ts = []
        for rep in range(warm + reps):
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            res = fn()
            e1.record(stream)
            torch.cuda.synchronize()
            if rep >= warm:
                ts.append(e0.elapsed_time(e1) / 1e3)
        return sum(ts) / len(ts), res

    clocks = Clocks(torch.cuda.current_device())
    clocks.start()
    rows, hom_rows = [], []
    cpu = None
    for name, n, draws, paper_nf, paper_psi in TABLE3:
        f, l = psigen.chung_lu_graph(n, 2.1, draws, args.seed)
        lam = psigen.uniform_rates(n, 0.0, 1.0, args.seed, psigen.STREAM_LAMBDA)
        mu = psigen.uniform_rates(n, 0.0, 1.0, args.seed, psigen.STREAM_MU)
        dev = [torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in (f, l, lam, mu)]
        with psi.Graph(n, *dev, precision="fp64", tol_mode="s_abs", stream=stream) as g:
            st = g.stats()
            # Power-NF once (the first graph also warms the kernels up); Power-psi as a step
            t_nf, (nf_psi, nf) = timed(lambda: g.power_nf(eps, 100000), 1, 1 if not rows else 0)
            t_ps, pinfo = timed(lambda: g.solve(eps, 100000), args.steps, args.warmup)
            ps = g.scores()
            diff = float(((nf_psi - ps).abs() / ps.abs().clamp_min(1.0 / n)).max())
            nf_host = nf_psi.cpu().numpy()
        followers = np.bincount(l, minlength=n)
        top = np.argsort(-followers, kind="stable")[:4]
        t0 = time.perf_counter()
        with oracle.Model(n, f, l, lam, mu) as m:
            ref, _ = m.power_nf(eps, origins=top)
            t_top = time.perf_counter() - t0
            t1 = time.perf_counter()
            m.power_psi(eps, oracle.TOL_S_ABS)
            t_opsi = time.perf_counter() - t1
            if name == TABLE3[-1][0] and not args.no_cpu_baseline:
                pick = (psigen.uniform(args.seed, 77, sample) * n).astype(np.int64)
                t2 = time.perf_counter()
                m.power_nf(eps, origins=pick)
                t_s = time.perf_counter() - t2
                cpu = {"value": t_s * n / sample, "unit": "s", "cores": 1, "kind": "oracle",
                       "sample": f"the oracle's Algorithm 1 on {sample} origins drawn uniformly from the {n} of "
                                 f"the {name} stand-in, scaled by {n}/{sample}",
                       "measured_s": t_s, "scaled_by": n / sample}
        parity = float(np.max(np.abs(nf_host[top] - ref) / np.maximum(np.abs(ref), 1.0 / n)))
        # Table IV: the same graph with homogeneous rates, where psi is PageRank with alpha = 0.85
        hom = [torch.full((n,), v, dtype=torch.float64, device="cuda") for v in (0.15, 0.85)]
        with psi.Graph(n, dev[0], dev[1], *hom, precision="fp64", tol_mode="s_abs", stream=stream) as g:
            h_nf, (h_nf_psi, h_nf_info) = timed(lambda: g.power_nf(eps, 100000), 1, 0)
            h_ps, h_pinfo = timed(lambda: g.solve(eps, 100000), args.steps, args.warmup)
            h_pr, (h_pi, h_prinfo) = timed(lambda: g.pagerank(0.85, eps, 100000), args.steps, args.warmup)
            h_psi = g.scores()
            h_diff = float((h_psi - h_pi).abs().sum() / h_pi.abs().sum())
            h_nfdiff = float(((h_nf_psi - h_psi).abs() / h_psi.abs().clamp_min(1.0 / n)).max())
        hom_rows.append({"workload": f"{name}_standin_homogeneous_0.15_0.85", "pagerank_s": h_pr,
                         "pagerank_iters": h_prinfo["iters"], "power_nf_s": h_nf,
                         "power_nf_matvecs": h_nf_info["spmv_launches"], "power_psi_s": h_ps,
                         "power_psi_iters": h_pinfo["iters"], "psi_vs_pagerank_rel_l1": h_diff,
                         "max_rel_psi_diff_nf_vs_psi": h_nfdiff,
                         "paper_cpu_s": dict(zip(("pagerank", "power_nf", "power_psi"), TABLE4[name]))})
        rows.append({"workload": f"{name}_standin_chunglu_gamma2.1_n{n}_draws{draws}_uniform0-1", "n": n,
                     "edges_drawn": draws, "edges_unique": st["m_unique"], "users_with_leaders": st["n_gathered"],
                     "users_with_followers": st["n_rows"],
                     "power_nf_s": t_nf, "power_nf_matvecs": nf["spmv_launches"], "power_nf_steps_max": nf["iters"],
                     "power_psi_s": t_ps, "power_psi_iters": pinfo["iters"], "nf_over_psi_time": t_nf / t_ps,
                     "max_rel_psi_diff_nf_vs_psi": diff, "oracle_nf_top4_rel_diff": parity,
                     "oracle_nf_top4_s": t_top, "oracle_power_psi_s": t_opsi,
                     "paper_cpu_s": {"power_nf": paper_nf, "power_psi": paper_psi}})
    clk = clocks.stop()
    line = {"metric": "Table III (i) stand-ins: solve time of Power-NF (Algorithm 1) at the Twitter graph's size",
            "value": rows[-1]["power_nf_s"], "unit": "s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "higher_is_better": False, "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "+".join(r["workload"] for r in rows), "eps": eps,
                       "tolerance": "per-origin ||p_t - p_t-1||_1 (Power-NF), ||s_t - s_t-1||_1 (Power-psi)"},
            "cases": rows, "cases_homogeneous": hom_rows, "clocks": clk}
    if cpu is not None:
        line["cpu_baseline"] = cpu
    print(json.dumps(line), flush=True)


def run_warmstart(args, n_train=200, eval_scale=23, train_steps=1500):
    """Train the warm-start network on solves of `n_train` seeded R-MAT graphs of scale 16-20
    (the benchmark's rate law), then time Power-psi to eps on a held-out R-MAT graph of scale
    `eval_scale` from s_0 = c and from the network's start."""
    import numpy as np
    import torch

    import psigen
    import paper_2206_09960_gb300 as psi
    from paper_2206_09960_gb300.warmstart import train, training_rows

    psi.load(build_if_missing=False)
    t0 = time.perf_counter()
    x_parts, t_parts = [], []
    for k in range(n_train):  # generated and solved in chunks to bound host memory
        w = psigen.workload("rmat", seed=1000 + k, scale=16 + k % 5)
        x, t = training_rows([w], rows_per_graph=1 << 14, seed=k)
        x_parts.append(x)
        t_parts.append(t)
    x, t = torch.cat(x_parts), torch.cat(t_parts)
    t_data = time.perf_counter() - t0
    t0 = time.perf_counter()
    model, losses = train(x, t, steps=train_steps, batch=1 << 16, lr=3e-3)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    w = psigen.workload("rmat", seed=7777, scale=eval_scale)
    args_d = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (w["follower"], w["leader"], w["lam"], w["mu"])]
    stream = torch.cuda.current_stream()
    res = {}
    clocks = Clocks(torch.cuda.current_device())
    clocks.start()
    with psi.Graph(w["n"], *args_d, stream=stream) as g:
        n_rows = g.stats()["n_rows"]
        for name in ("cold", "warm"):
            ts, its = [], []
            for rep in range(args.warmup + args.steps):
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                info = g.solve(args.eps, 100000) if name == "cold" else model.solve(g, args.eps, 100000)
                e1.record(stream)
                torch.cuda.synchronize()
                if rep >= args.warmup:
                    ts.append(e0.elapsed_time(e1) / 1e3)
                    its.append(info["iters"])
            res[name] = (statistics.mean(ts), its[-1], info["converged"])
        psi_warm = g.scores().cpu().numpy()
        g.solve(args.eps, 100000)
        psi_cold = g.scores().cpu().numpy()
    # resuming from the solved iterate after every rate moves by ~1% (multiplicative
    # LogNormal(0, 0.01) noise): the start the library also offers (psi_get_iterate -> init_s)
    rng = np.random.default_rng(7778)
    lam2 = w["lam"] * np.exp(0.01 * rng.standard_normal(w["n"]))
    mu2 = w["mu"] * np.exp(0.01 * rng.standard_normal(w["n"]))
    with psi.Graph(w["n"], *args_d, stream=stream) as g:
        g.solve(args.eps, 100000)
        s_prev = g.iterate()
    args_p = [args_d[0], args_d[1], torch.from_numpy(lam2).cuda(), torch.from_numpy(mu2).cuda()]
    with psi.Graph(w["n"], *args_p, stream=stream) as g:
        for name in ("changed_cold", "changed_resume"):
            ts, its = [], []
            for rep in range(args.warmup + args.steps):
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                info = g.solve(args.eps, 100000, s_prev if name == "changed_resume" else None)
                e1.record(stream)
                torch.cuda.synchronize()
                if rep >= args.warmup:
                    ts.append(e0.elapsed_time(e1) / 1e3)
                    its.append(info["iters"])
            res[name] = (statistics.mean(ts), its[-1], info["converged"])
    clk = clocks.stop()
    rel = float(np.abs(psi_warm - psi_cold).sum() / np.abs(psi_cold).sum())
    # the network on tensor cores: one forward pass over the held-out graph's rows and one
    # gradient over a training batch, each timed with CUDA events
    xr = torch.randn(n_rows, 8, device="cuda")
    tr = torch.randn(1 << 16, device="cuda")

    def ev_time(fn, reps=5):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3 / reps

    fwd_s = ev_time(lambda: model.forward(xr))
    grad_s = ev_time(lambda: model.grad(xr[: 1 << 16], tr))
    flop_row = 2 * (8 * 64 + 64 * 64 + 64)  # multiply-adds of the three layers, x2
    with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
        bf16_peak = float(json.load(fh).get("bf16_tflops", 1900.0))
    net = {"bound": "tensor", "achieved": n_rows * flop_row / fwd_s / 1e12, "peak": bf16_peak, "unit": "TFLOP/s",
           "frac": n_rows * flop_row / fwd_s / 1e12 / bf16_peak, "traffic": None, "peak_kind": "measured",
           "kernel": "k_mlp_forward (mma.sync m16n8k16 BF16, FP32 accumulate)", "rows": n_rows,
           "forward_ms": fwd_s * 1e3, "grad_ms_65536_rows": grad_s * 1e3,
           "grad_tflops": 3 * (1 << 16) * flop_row / grad_s / 1e12}
    line = {"metric": "warm start: Power-psi time and steps to L1<1e-8 from the network's s_0 vs s_0 = c",
            "value": res["warm"][0], "unit": "s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "higher_is_better": False, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"train: {n_train} R-MAT graphs scale 16-20; eval: R-MAT scale {eval_scale}",
                       "eps": args.eps, "train_rows": int(x.shape[0]), "train_steps": train_steps},
            "cold_s": res["cold"][0], "cold_iters": res["cold"][1], "warm_s": res["warm"][0],
            "warm_iters": res["warm"][1], "converged": [res["cold"][2], res["warm"][2]],
            "psi_rel_l1_warm_vs_cold": rel,
            "rates_changed_1pct": {"cold_s": res["changed_cold"][0], "cold_iters": res["changed_cold"][1],
                                   "resume_s": res["changed_resume"][0], "resume_iters": res["changed_resume"][1],
                                   "converged": [res["changed_cold"][2], res["changed_resume"][2]]},
            "loss_first": float(np.mean(losses[:10])),
            "loss_last": float(np.mean(losses[-50:])), "data_s": t_data, "train_s": t_train, "clocks": clk,
            "roofline": net}
    print(json.dumps(line), flush=True)


def workload_config(args):
    """The workload's configuration, identical in both arms."""
    return {"workload": f"rmat_scale{args.scale}_ef16_a.57_b.19_c.19_relabel_lognormal1.5",
            "n": 1 << args.scale, "edge_draws": 16 << args.scale, "eps": args.eps,
            "tolerance": "eps_t/N (psi tolerance, B_norm=1)", "topk": 100,
            "l2": "inputs larger than L2 (edge list 8 B x draws)", "parallelism": "replicas"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--scale", type=int, default=25)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--eps", type=float, default=1e-8)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--allocator", default="torch", choices=["torch", "library"],
                    help="device memory of the library: its own stream-ordered pool, or torch's caching allocator")
    ap.add_argument("--profile-solve", action="store_true",
                    help="multi workload: run one extra solve between cudaProfilerStart/Stop (ncu --profile-from-start off)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-check", action="store_true", help="skip the oracle parity check after the timed steps")
    ap.add_argument("--spmv-tile", type=int, default=0, help="fix the product's tile (0: autotuner / rule)")
    ap.add_argument("--spmv-hot", type=int, default=-1,
                    help="fix the series product's shared-memory copy (-1: autotuner's choice)")
    ap.add_argument("--workload", default="rmat", choices=["rmat", "batch", "warmstart", "multi", "pagerank", "powernf"],
                    help="rmat: the single-graph step (default); batch: 64 activity scenarios on one graph; "
                         "warmstart: train the start-vector network and compare steps and time to eps")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.impl == "reference":
        run_reference(args)
        return
    if args.workload == "batch":
        run_batch(args)
        return
    if args.workload == "warmstart":
        run_warmstart(args)
        return
    if args.workload == "multi":
        run_multi(args)
        return
    if args.workload == "pagerank":
        run_pagerank(args)
        return
    if args.workload == "powernf":
        run_powernf(args)
        return

    import numpy as np
    import torch

    import psigen
    import paper_2206_09960_gb300 as psi
    from paper_2206_09960_gb300 import shard

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    psi.load(build_if_missing=False)

    # one independent graph per rank (replicas)
    seed = args.seed + rank
    n = 1 << args.scale
    m0 = 16 << args.scale
    f_h = torch.empty(m0, dtype=torch.int32).pin_memory()
    l_h = torch.empty(m0, dtype=torch.int32).pin_memory()
    psigen.rmat_graph(args.scale, 16, *psigen.RMAT_ABC, seed, relabel=True, out=(f_h.numpy(), l_h.numpy()))
    lam_h = torch.from_numpy(psigen.lognormal_rates(n, 0.0, 1.5, 1e-3, 1e3, seed, psigen.STREAM_LAMBDA)).pin_memory()
    mu_h = torch.from_numpy(psigen.lognormal_rates(n, 0.0, 1.5, 1e-3, 1e3, seed, psigen.STREAM_MU)).pin_memory()
    f_d, l_d, lam_d, mu_d = (x.cuda() for x in (f_h, l_h, lam_h, mu_h))
    ids_d = torch.empty(100, dtype=torch.int32, device="cuda")
    vals_d = torch.empty(100, dtype=torch.float64, device="cuda")
    ids_h = torch.empty(100, dtype=torch.int32).pin_memory()
    vals_h = torch.empty(100, dtype=torch.float64).pin_memory()
    stream = torch.cuda.current_stream()

    alloc = "torch" if args.allocator == "torch" else None

    def step(inputs, ids, vals, profile=False, **kw):
        kw.setdefault("spmv_tile", args.spmv_tile)
        kw.setdefault("spmv_hot", args.spmv_hot)
        with psi.Graph(n, *inputs, profile=profile, stream=stream, allocator=alloc, **kw) as g:
            info = g.solve(args.eps, 100000)
            g.topk(100, ids, vals)
            return info, g.stats()

    def barrier():
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    def max_over_ranks(x):
        return shard.max_over_ranks(x, device="cuda")

    dev_in = (f_d, l_d, lam_d, mu_d)
    host_in = (f_h, l_h, lam_h, mu_h)
    warm_stats = []
    for _ in range(args.warmup):
        warm_stats.append(step(dev_in, ids_d, vals_d)[1])

    # ---- timed region: inputs resident in HBM
    clocks = Clocks(torch.cuda.current_device())
    clocks.start()
    launches0 = psi.psi_kernel_launches()
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    infos, stats, builds_ms = [], None, []
    marks = [e0]
    for _ in range(args.steps):
        info, stats = step(dev_in, ids_d, vals_d, profile=True)
        infos.append(info)
        builds_ms.append(stats["build_ms"])
        m = torch.cuda.Event(enable_timing=True)
        m.record(stream)
        marks.append(m)
    e1.record(stream)
    barrier()
    launches = psi.psi_kernel_launches() - launches0
    clk = clocks.stop()
    step_s = max_over_ranks(e0.elapsed_time(e1) / 1e3 / args.steps)
    steps_ms = [marks[i].elapsed_time(marks[i + 1]) for i in range(args.steps)]

    # ---- the autotuner's pick (made on the first warm-up graph) against the fixed rule
    info_fixed, st_fixed = step(dev_in, ids_d, vals_d, profile=True, autotune=False, spmv_tile=0, spmv_hot=-1)
    tuner = {"tile": stats["spmv_tile"], "hot": stats["spmv_hot"], "tune_ms": warm_stats[0]["tune_ms"],
             "fixed_rule": {"tile": st_fixed["spmv_tile"], "hot": 0,
                            "series_step_ms": info_fixed["spmv_ms"] / max(info_fixed["spmv_timed"], 1),
                            "time_to_eps_s": info_fixed["ms"] / 1e3}}

    # ---- end to end from pinned host buffers (H2D of inputs and D2H of the ranking inside)
    # Two graphs in flight: two host threads, each with its own stream and output buffers,
    # take the steps in turn through the public API, so that one step's upload (on the copy
    # engines) overlaps the previous step's solve.  Every step's copies stay inside the timed
    # region; the value is all steps' edges over the wall time from the first upload to the
    # last ranking read back.  The same steps one after another are the `sequential` record.
    e2e = None
    if not args.no_e2e:
        import threading

        quiesce_s, quiesce_moved = host_quiesce()
        e_streams = [torch.cuda.Stream(), torch.cuda.Stream()]  # not the legacy default stream, which
        # would wait for (and hold up) the other one
        e_out = [(ids_h, vals_h), (torch.empty(100, dtype=torch.int32).pin_memory(),
                                   torch.empty(100, dtype=torch.float64).pin_memory())]

        def host_step(i):
            st_i = e_streams[i]
            tw = time.perf_counter()
            with torch.cuda.stream(st_i):
                with psi.Graph(n, *host_in, stream=st_i, allocator=alloc, spmv_tile=args.spmv_tile,
                               spmv_hot=args.spmv_hot) as g:
                    g.solve(args.eps, 100000)
                    g.topk(100, *e_out[i])
                    bms = g.stats()["build_ms"]
            st_i.synchronize()
            return time.perf_counter() - tw, bms

        for i in (0, 1):  # warm-up of both lanes
            host_step(i)
        def device_allocs():
            return torch.cuda.memory_stats().get("num_device_alloc", 0)

        # sequential: the steps one after another on one stream
        barrier()
        na_seq = device_allocs()
        t0 = time.perf_counter()
        seq_walls, seq_builds = [], []
        for _ in range(args.steps):
            w_, b_ = host_step(0)
            seq_walls.append(w_)
            seq_builds.append(b_)
        barrier()
        seq_s = max_over_ranks((time.perf_counter() - t0) / args.steps)
        na_seq = device_allocs() - na_seq
        # two in flight
        walls = [[], []]
        builds = [[], []]
        errors = []

        def lane(i):
            try:
                for _ in range(args.steps // 2 + (args.steps % 2 if i == 0 else 0)):
                    w_, b_ = host_step(i)
                    walls[i].append(w_)
                    builds[i].append(b_)
            except Exception as exc:  # surfaced below, after both threads end
                errors.append(exc)

        # one untimed round with both lanes in flight, so that the allocator already holds two
        # graphs' worth of device memory when the timed steps start (the sequential warm-up
        # held one)
        warm = [threading.Thread(target=host_step, args=(i,)) for i in (0, 1)]
        for t_ in warm:
            t_.start()
        for t_ in warm:
            t_.join()
        torch.cuda.synchronize()
        barrier()
        na_fl = device_allocs()
        t0 = time.perf_counter()
        threads = [threading.Thread(target=lane, args=(i,)) for i in (0, 1)]
        for t_ in threads:
            t_.start()
        for t_ in threads:
            t_.join()
        torch.cuda.synchronize()
        if errors:
            raise errors[0]
        barrier()
        e2e_s = max_over_ranks((time.perf_counter() - t0) / args.steps)
        na_fl = device_allocs() - na_fl
        h2d_gbs = pinned_h2d_gbs(f_h, f_d, stream)
        placement = host_placement(f_h)
        ms_ = torch.cuda.memory_stats()
        alloc_stats = {k: ms_.get(k) for k in ("num_alloc_retries", "num_device_alloc", "num_device_free")}
        alloc_stats["reserved_gib"] = round(torch.cuda.memory_reserved() / 2**30, 1)
        # new device segments taken while the timed steps ran (a cudaMalloc there is timed)
        alloc_stats["device_allocs_in_timed_steps"] = {"sequential": na_seq, "in_flight": na_fl}
        e2e = {"value": ws * m0 / e2e_s, "unit": UNIT, "h2d_bytes_per_step": int(2 * 4 * m0 + 2 * 8 * n),
               "d2h_bytes_per_step": int(100 * (4 + 8)), "s_per_step": e2e_s, "in_flight": 2,
               "h2d_gbs": h2d_gbs, "host_buffers": placement,
               "steps_wall_ms": [[round(x * 1e3, 3) for x in w] for w in walls],
               "steps_build_ms": [[round(x, 3) for x in b] for b in builds],
               "sequential": {"value": ws * m0 / seq_s, "s_per_step": seq_s,
                              "steps_wall_ms": [round(x * 1e3, 3) for x in seq_walls],
                              "steps_build_ms": [round(x, 3) for x in seq_builds]},
               "torch_allocator": alloc_stats,
               "host_quiesce": {"waited_s": round(quiesce_s, 2), "compaction_counters_moved": quiesce_moved}}

    # ---- roofline of the dominant kernel: the FP32 series step (sparse product + fix-up)
    iters = statistics.mean(i["iters"] for i in infos)
    spmv_launches = sum(i["spmv_timed"] for i in infos)
    spmv_ms = sum(i["spmv_ms"] for i in infos)
    avg_launch_s = spmv_ms / 1e3 / max(spmv_launches, 1)
    m_u, n_rows, n_g = stats["m_unique"], stats["n_rows"], stats["n_gathered"]
    alg_bytes = 4 * m_u + 32 * n  # 4M + 32N: every user's vectors once, every column index once
    kernel_bytes = 4 * m_u + 32 * n_rows + 4 * n_g  # what this kernel has to touch (rows, gathered users)
    peak, peak_kind = measured_peaks()
    achieved = alg_bytes / avg_launch_s / 1e9
    # the stored figure holds only for the kernel sources and the copy size it was taken with
    # (the tile changes the carries and the schedule, a few MB, not the streams or the gathers)
    same_cfg = stats.get("spmv_hot") == 28672
    traffic = NCU_TRAFFIC["bytes_per_launch"] if NCU_TRAFFIC["sha"] == kernel_sha() and same_cfg else None
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic, "peak_kind": peak_kind,
                "kernel": (f"k_spmv<float,EpiSeries,{32 if stats['spmv_hot'] else 8}> + k_fixup "
                           f"(FP32 series step of Eq. 13; {stats['spmv_hot']} entries from shared memory)"),
                "alg_bytes_per_launch": alg_bytes, "alg_bytes_formula": "4*M_unique + 32*N",
                "avg_launch_ms": avg_launch_s * 1e3, "launches_timed": spmv_launches,
                "kernel_bytes_per_launch": kernel_bytes,
                "frac_kernel_bytes": kernel_bytes / avg_launch_s / 1e9 / peak}
    solve_s = statistics.mean(i["ms"] for i in infos) / 1e3
    build_s = statistics.mean(builds_ms) / 1e3

    # ---- the GPU's psi and ranking of the same graph, for the parity check below
    gpu_psi = gpu_top = None
    if rank == 0 and ws == 1 and not args.no_check:
        with psi.Graph(n, *dev_in, stream=stream, allocator=alloc) as g:
            g.solve(args.eps, 100000)
            gpu_psi = g.scores().cpu().numpy()
            ids, vals = g.topk(100)
            gpu_top = (ids.cpu().numpy(), vals.cpu().numpy())

    line = {"metric": METRIC, "value": ws * m0 / step_s, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": step_s * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": workload_config(args),
            "e2e": e2e, "gpu_launches": int(launches), "clocks": clk, "roofline": roofline,
            "precision": "fp32 series terms, fp64 iterate; confirming step and final product in float pairs "
                         "(~48-bit sums) with fp64 row updates; fp64 gap, psi and sum of psi",
            "allocator": args.allocator,
            "graph": {"m_unique": m_u, "n_rows": n_rows, "n_gathered": n_g, "spmv_tile": stats.get("spmv_tile"),
                      "spmv_hot": stats.get("spmv_hot")},
            "autotune": dict(tuner, series_step_ms=avg_launch_s * 1e3),
            "time_to_eps_s": solve_s, "build_s": build_s, "iters": iters,
            "steps_ms": [round(x, 3) for x in steps_ms],
            "steps_build_ms": [round(x, 3) for x in builds_ms],
            "steps_solve_ms": [round(i["ms"], 3) for i in infos],
            "refinements": statistics.mean(i["refinements"] for i in infos),
            "gteps_per_iter": m_u / avg_launch_s / 1e9,
            "gap_psi_bound": infos[-1]["gap_psi_bound"], "gap_scaled": infos[-1]["gap_scaled"],
            "psi_sum": infos[-1]["psi_sum"], "problems_per_s": ws / step_s}

    # ---- after every GPU measurement: the oracle on the same graph (all host cores), which
    # is both the measured CPU baseline and the parity check, plus a one-thread sample
    if rank == 0 and ws == 1 and not (args.no_check and args.no_cpu_baseline):
        del dev_in, f_d, l_d, lam_d, mu_d
        w = {"n": n, "follower": f_h.numpy(), "leader": l_h.numpy(), "lam": lam_h.numpy(), "mu": mu_h.numpy()}
        need = oracle_bytes(n, m0)
        avail = host_available_bytes()
        if avail is not None and avail < 1.5 * need:
            why = f"host memory: {avail / 2**30:.0f} GiB available, the oracle needs ~{need / 2**30:.0f} GiB"
            line["cpu_baseline"] = {"unavailable": why}
            line["parity"] = {"unavailable": why}
        else:
            sec, out, threads = oracle_seconds(w, args.eps)
            cpu = {"value": m0 / sec, "unit": UNIT, "cores": threads, "kind": "oracle",
                   "sample": f"the whole workload (R-MAT scale {args.scale}, {m0} edge draws), one full oracle run: "
                             f"canonicalise, explicit A/B, Algorithm 2 to eps={args.eps:g} on eps_t/N, top-100; "
                             f"{sec:.1f} s on {threads} threads",
                   "seconds": sec, "iters": int(out["iters"])}
            cpu.update(host_info())
            w1 = psigen.workload("rmat", seed=args.seed, scale=min(ONE_THREAD_SCALE, args.scale))
            sec1, _, _ = oracle_seconds(w1, args.eps, threads=1)
            d1 = int(w1["follower"].size)
            cpu["one_thread"] = {"value": d1 / sec1, "unit": UNIT, "cores": 1, "seconds": sec1,
                                 "sample": f"whole oracle path on R-MAT scale {min(ONE_THREAD_SCALE, args.scale)} "
                                           f"of the same recipe ({d1} edge draws), 1 thread"}
            if not args.no_cpu_baseline:
                line["cpu_baseline"] = cpu
            if gpu_psi is not None:
                line["parity"] = parity_block(gpu_psi, gpu_top, out, stats["m_unique"])
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
