"""Multi-process logic on CPU (gloo, world size 2).

bench.py with N > 1 runs one independent replica per GPU (no collective on
the data path): barrier, per-rank timing, the maximum over ranks, and the
whole-job throughput.  These tests run that aggregation with two gloo ranks,
and check the partition reading of the paper's multi-process mode (Sec. 5.2,
footnote: contiguous batches divided among workers) with the oracle: the NLL
and gradient of two contiguous shards add up to the whole dataset's, once the
extended term (sum of yields) is counted once."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch
    import torch.distributed as dist

    import bench
    import datagen
    import oracle
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    try:
        # aggregation used by bench.py: slowest rank wins
        slowest = bench.max_over_ranks(10.0 + rank, dist, "cpu")
        # contiguous shard of a C2-shaped dataset, evaluated by this rank
        w = datagen.c4(toys=1, nu_s_range=(800, 800.001), nu_b_range=(2000, 2000.001))
        cols = w["cols"]
        n = cols.shape[1]
        lo, hi = rank * n // world, (rank + 1) * n // world
        p = [5.02, 0.51, -0.29, 790.0, 2010.0]
        v, g, rc = oracle.nll(w["spec"], p, cols[:, lo:hi])
        t = torch.tensor([v, *g], dtype=torch.float64)
        dist.all_reduce(t)
        q.put((rank, slowest, t.numpy().tolist(), n))
    finally:
        dist.destroy_process_group()


def test_two_rank_aggregation_and_event_partition():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for pr in procs:
        pr.start()
    res = [q.get(timeout=120) for _ in range(2)]
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    import bench
    import datagen
    import oracle
    assert all(r[1] == 11.0 for r in res)          # max over ranks, on every rank
    assert bench.job_throughput(1000, 2, 1.0) == 2e6
    w = datagen.c4(toys=1, nu_s_range=(800, 800.001), nu_b_range=(2000, 2000.001))
    p = [5.02, 0.51, -0.29, 790.0, 2010.0]
    v, g, _ = oracle.nll(w["spec"], p, w["cols"])
    summed = np.array(res[0][2])
    # each shard carried the extended term sum(nu) and d/dnu = +1 once
    summed[0] -= p[3] + p[4]
    summed[4] -= 1.0
    summed[5] -= 1.0
    assert abs(summed[0] - v) <= 1e-12 * abs(v)
    np.testing.assert_allclose(summed[1:], g, rtol=1e-10, atol=1e-8)


class _FakeGraph:
    """Stands in for a Graph on CPU: its 'NLL' is the shard's oracle NLL with
    the extended term weighted as set (no GPU needed)."""

    def __init__(self, spec, cols, p):
        self.spec, self.cols, self.p = spec, cols, p
        self.n_par = len(p)
        self.w = None

    def set_shard_weight(self, w):
        self.w = w

    def nll(self, ev, params, out):
        import oracle
        import torch
        v, g, rc = oracle.nll(self.spec, self.p, self.cols)
        ext = sum(self.p[3:5])
        v = v - ext + self.w * ext                 # extended term weighted
        g = np.array(g)
        g[3:5] += self.w - 1.0
        out.copy_(torch.tensor([v, *g], dtype=torch.float64))


def _shard_worker(rank, world, port, q):
    import torch
    import torch.distributed as dist

    import datagen
    import paper_2003_12875_gb300 as rf
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    try:
        w = datagen.c4(toys=1, nu_s_range=(800, 800.001), nu_b_range=(2000, 2000.001))
        n = w["cols"].shape[1]
        lo, hi = rf.shard_range(n, rank, world)
        p = [5.02, 0.51, -0.29, 790.0, 2010.0]
        G = _FakeGraph(w["spec"], w["cols"][:, lo:hi], p)
        runs = [rf.sharded_nll(G, torch.empty(1, hi - lo), torch.tensor(p), rank).numpy()
                for _ in range(2)]
        q.put((rank, G.w, [r.tolist() for r in runs],
               [r.view(np.int64).tolist() for r in runs]))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_nll_helper_reduces_over_ranks(world):
    """paper_2003_12875_gb300.sharded_nll on gloo ranks: the extended term is
    weighted on rank 0 only, the all-gathered shard values are added in rank
    order, and the result is the whole dataset's NLL and gradient, bit for bit
    the same on every rank and in two runs (oracle shards stand in for the
    GPU)."""
    import datagen
    import oracle
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_shard_worker, args=(r, world, port, q)) for r in range(world)]
    for pr in procs:
        pr.start()
    res = sorted(q.get(timeout=180) for _ in range(world))
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    assert [r[1] for r in res] == [1.0] + [0.0] * (world - 1)
    bits = res[0][3][0]
    for _, _, _, b in res:
        assert b[0] == bits and b[1] == bits        # every rank, both runs
    w = datagen.c4(toys=1, nu_s_range=(800, 800.001), nu_b_range=(2000, 2000.001))
    v, g, rc = oracle.nll(w["spec"], [5.02, 0.51, -0.29, 790.0, 2010.0], w["cols"])
    out = res[0][2][0]
    assert abs(out[0] - v) <= 1e-11 * abs(v)
    np.testing.assert_allclose(out[1:], g, rtol=1e-9, atol=1e-9)


def test_rank_order_sum_is_compensated_and_ordered():
    """rank_order_sum against the exactly rounded sum (math.fsum) on values
    whose plain sum loses everything, and its fixed order: permuting the rows
    may change the bits, repeating the call never does."""
    import math

    import torch

    import paper_2003_12875_gb300 as rf
    rows = torch.tensor([[1e16, 3.0], [1.0, -1e-3], [-1e16, 2.5], [1.0, 7e-4]],
                        dtype=torch.float64)
    got = rf.rank_order_sum(rows).numpy()
    for j in range(2):
        assert got[j] == math.fsum(rows[:, j].tolist())
    plain = 0.0
    for v in rows[:, 0].tolist():
        plain += v
    assert plain == 1.0 and got[0] == 2.0               # the plain sum loses a 1
    r = np.random.default_rng(3).standard_normal((8, 5)) * 10.0 ** np.arange(5)
    t = torch.from_numpy(r)
    a, b = rf.rank_order_sum(t), rf.rank_order_sum(t.clone())
    assert torch.equal(a, b)
    for j in range(5):
        assert abs(float(a[j]) - math.fsum(r[:, j])) <= 4e-16 * np.abs(r[:, j]).sum()
