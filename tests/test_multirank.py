"""Multi-rank host logic on CPU ranks (torch.distributed, gloo, world size 2): the row
partition balanced by nonzeros, a row-sharded Power-psi iteration with one exchange per
step (allgather of the new s, allreduce of the L1 gap) that must reproduce the single-process
oracle, the max-over-ranks timing of replica runs, and a rank that leaves before an exchange
(the other rank's collective ends with an error within the process-group timeout).  No GPU."""
import os
import socket
import tempfile

import numpy as np
import pytest

import oracle
import psigen
from paper_2206_09960_gb300 import shard


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, fn_name, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    from datetime import timedelta

    import torch.distributed as dist

    # a short timeout: a collective whose peer is gone ends with an error, not a hang
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=timedelta(seconds=20))
    try:
        result = globals()[fn_name](rank, world)
    finally:
        if dist.is_initialized():
            dist.destroy_process_group()
    np.save(os.path.join(out_dir, "%s_%d.npy" % (fn_name, rank)), np.asarray(result, dtype=object),
            allow_pickle=True)


def _run(fn_name, world=2):
    import torch.multiprocessing as mp

    with tempfile.TemporaryDirectory() as d:
        mp.spawn(_worker, args=(world, _free_port(), fn_name, d), nprocs=world, join=True)
        return [np.load(os.path.join(d, "%s_%d.npy" % (fn_name, r)), allow_pickle=True).item() for r in range(world)]


def _transposed_csr(n, f, l):
    order = np.lexsort((f, l))
    rows, cols = l[order], f[order]
    row_ptr = np.concatenate([[0], np.cumsum(np.bincount(rows, minlength=n))]).astype(np.int64)
    return row_ptr, rows, cols


def _sharded_power_psi(rank, world, eps=1e-12, max_iter=10000):
    """Algorithm 2 (psi tolerance, B_norm = 1) with the rows split over the ranks."""
    import torch

    w = psigen.workload("rmat", seed=21, scale=10)
    n = w["n"]
    with oracle.Model(n, w["follower"], w["leader"], w["lam"], w["mu"]) as g:
        f, l = g.edges()
        c, d, sigma = g.vectors()
        lam, mu = g.lam, g.mu
    row_ptr, rows, cols = _transposed_csr(n, f, l)
    plan = shard.make_plan(row_ptr, world, rank)
    lo, hi = plan.rows
    e0, e1 = row_ptr[lo], row_ptr[hi]
    my_rows, my_cols = rows[e0:e1] - lo, cols[e0:e1]
    isig = np.where(sigma > 0, 1.0 / np.where(sigma > 0, sigma, 1.0), 0.0)

    def pull(s):  # G(s) on this rank's rows
        return np.bincount(my_rows, weights=(s * isig)[my_cols], minlength=hi - lo)

    s = c.copy()
    gap, t = 1.0, 0
    while gap / n > eps and t < max_iter:  # Algorithm 2's loop test, gap starting at 1
        s_local = c[lo:hi] + mu[lo:hi] * pull(s)
        gap_local = float(np.abs(s_local - s[lo:hi]).sum())
        s = shard.allgather_rows(torch.from_numpy(s_local), plan).numpy()
        gap = shard.allreduce_sum(gap_local)
        t += 1
    psi_local = (lam[lo:hi] * pull(s) + d[lo:hi]) / n
    psi = shard.allgather_rows(torch.from_numpy(psi_local), plan).numpy()
    return dict(psi=psi, s=s, iters=t, rows=(lo, hi), nnz=int(e1 - e0))


def _replica_timing(rank, world):
    # each rank "times" a different step; the job's step time is the slowest rank's
    return dict(step=shard.max_over_ranks(0.1 + 0.05 * rank), gap=shard.allreduce_sum(1.5 * (rank + 1)))


def _dropped_rank(rank, world):
    """Rank 1 leaves before the exchange of the first step; rank 0 must see an error."""
    import time

    import torch
    import torch.distributed as dist

    plan = shard.ShardPlan(np.array([0, 4, 8]), rank)
    if rank == 1:
        dist.destroy_process_group()
        return dict(left=True)
    t0 = time.monotonic()
    try:
        shard.allgather_rows(torch.ones(4, dtype=torch.float64), plan)
        err = None
    except Exception as e:  # the collective fails: the peer is gone
        err = type(e).__name__
    return dict(left=False, error=err, seconds=time.monotonic() - t0)


def test_partition_balances_nonzeros():
    rng = np.random.default_rng(0)
    deg = rng.zipf(2.0, 5000).clip(max=4000)
    row_ptr = np.concatenate([[0], np.cumsum(deg)])
    for world in (1, 2, 3, 8):
        b = shard.partition_rows(row_ptr, world)
        assert b[0] == 0 and b[-1] == deg.size and np.all(np.diff(b) >= 0)
        work = np.array([row_ptr[b[r + 1]] - row_ptr[b[r]] + (b[r + 1] - b[r]) for r in range(world)])
        share = (row_ptr[-1] + deg.size) / world
        assert work.max() <= share + deg.max() + 1  # at most one row over its share
    # degenerate inputs: no rows, more ranks than rows
    assert list(shard.partition_rows([0], 4)) == [0, 0, 0, 0, 0]
    b = shard.partition_rows([0, 5, 5], 4)
    assert b[0] == 0 and b[-1] == 2 and np.all(np.diff(b) >= 0)
    with pytest.raises(ValueError):
        shard.make_plan([0, 1], 2, 2)


def test_row_sharded_power_psi_matches_oracle():
    res = _run("_sharded_power_psi")
    w = psigen.workload("rmat", seed=21, scale=10)
    ref = oracle.solve(w["n"], w["follower"], w["leader"], w["lam"], w["mu"], eps=1e-12)
    # the two ranks split the rows and the nonzeros, and end with the same vectors
    (lo0, hi0), (lo1, hi1) = res[0]["rows"], res[1]["rows"]
    assert lo0 == 0 and hi0 == lo1 and hi1 == w["n"]
    assert abs(res[0]["nnz"] - res[1]["nnz"]) <= 0.2 * (res[0]["nnz"] + res[1]["nnz"])
    np.testing.assert_array_equal(res[0]["psi"], res[1]["psi"])
    assert res[0]["iters"] == res[1]["iters"]
    # the gap sums round differently from the single sum: allow one step of difference
    assert abs(res[0]["iters"] - ref["iters"]) <= 1
    assert np.abs(res[0]["psi"] - ref["psi"]).sum() / ref["psi"].sum() <= 1e-10


def test_replica_timing_is_the_slowest_rank():
    res = _run("_replica_timing")
    for r in res:
        assert r["step"] == pytest.approx(0.15)
        assert r["gap"] == pytest.approx(4.5)
    assert shard.max_over_ranks(0.3) == 0.3  # a single process is its own maximum


def test_a_dropped_rank_is_an_error_not_a_hang():
    res = _run("_dropped_rank")
    assert res[1]["left"]
    assert res[0]["error"] is not None
    assert res[0]["seconds"] < 60
