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
        out = rf.sharded_nll(G, torch.empty(1, hi - lo), torch.tensor(p), rank)
        q.put((rank, G.w, out.numpy().tolist()))
    finally:
        dist.destroy_process_group()


def test_sharded_nll_helper_reduces_over_ranks():
    """paper_2003_12875_gb300.sharded_nll on three gloo ranks: the extended
    term is weighted on rank 0 only and the all-reduced result is the whole
    dataset's NLL and gradient (oracle shards stand in for the GPU)."""
    import datagen
    import oracle
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_shard_worker, args=(r, 3, port, q)) for r in range(3)]
    for pr in procs:
        pr.start()
    res = sorted(q.get(timeout=180) for _ in range(3))
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    assert [r[1] for r in res] == [1.0, 0.0, 0.0]
    w = datagen.c4(toys=1, nu_s_range=(800, 800.001), nu_b_range=(2000, 2000.001))
    v, g, rc = oracle.nll(w["spec"], [5.02, 0.51, -0.29, 790.0, 2010.0], w["cols"])
    for _, _, out in res:
        assert abs(out[0] - v) <= 1e-11 * abs(v)
        np.testing.assert_allclose(out[1:], g, rtol=1e-9, atol=1e-9)
