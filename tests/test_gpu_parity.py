"""GPU parity: the CUDA path through the C-ABI against the FP64 oracle on the
same seeded inputs.  Sizes span several blocks and a ragged tail; the shape
sweep covers empty, tiny and unaligned inputs; tolerances are in _common.py."""
import math

import numpy as np
import pytest
import torch

import datagen
import oracle
from _common import TOL, free_mask, grad_l1, logp_err, rel_nll

pytestmark = pytest.mark.gpu

DEV = "cuda"


@pytest.fixture(scope="module")
def rf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2003_12875_gb300 as rf
    rf.load()
    return rf


def to_dev(w):
    dt = torch.float32 if w["dtype"] == "f32" else torch.float64
    return torch.from_numpy(np.ascontiguousarray(w["cols"])).to(DEV, dt)


def params_dev(p):
    return torch.tensor(np.asarray(p, np.float64), device=DEV)


SMALL = {
    "c1": lambda: datagen.c1(),
    "c2": lambda: datagen.c2(n=200_003),
    "c3": lambda: datagen.c3(n=100_003),
    "c3_noext": lambda: datagen.c3(n=50_001, extended=False),
    "c5": lambda: datagen.c5(3_000, 300_000),
    "johnson": lambda: datagen.johnson_exp(20_011, 80_000),
    "c5_free_p": lambda: _free_p(datagen.c5(3_000, 300_000)),
    "c5_fixed_p": lambda: _fixed_p(datagen.c5(3_000, 300_000), 0.8),
    "prod6": lambda: datagen.prod6(60_011),
}
JIT_ONLY = {"prod6"}  # more than 4 leaves: specialised kernels only
OFF_MIN = {  # gradient checks away from the minimum
    "c1": [0.25, 1.1],
    "c2": [5.05, 0.52, -0.28, 0.21],
    "c3": [0.05, 1.55, -0.48, 0.21, -0.09, 0.055, 0.025, 100_500.0],
    "c3_noext": [0.05, 1.55, -0.48, 0.21, -0.09, 0.055, 0.025],
    "c5": [5.2792, 0.0031, 1.55, 3.1, 5.29, -19.5, 0.5, 3_050.0, 299_000.0],
    "johnson": [4.05, 0.78, -0.45, 1.62, -0.21, 19_800.0, 80_300.0],
    "c5_free_p": [5.2792, 0.0031, 1.55, 3.1, 5.29, -19.5, 0.58, 3_050.0, 299_000.0],
    "c5_fixed_p": [5.2792, 0.0031, 1.55, 3.1, 5.29, -19.5, 0.8, 3_050.0, 299_000.0],
    "prod6": [5.05, 0.62, -1.15, 3.02, 0.41, 1.25, 2.6, 0.28, -0.18, -0.24, 0.18, 0.31,
              0.31, 0.29],
}


def _free_p(w):
    """The C5 model with the ARGUS power p free (general-p form, d/dp)."""
    spec = dict(w["spec"])
    spec["fixed"] = list(spec["fixed"])
    spec["fixed"][6] = False
    return {**w, "spec": spec}


def _fixed_p(w, pval):
    """The C5 model with the ARGUS power fixed at pval != 1/2: the graph is
    compiled with that value, which selects the general-p form without a
    d/dp sum."""
    spec = dict(w["spec"])
    spec["params"] = list(spec["params"])
    spec["params"][6] = pval
    return {**w, "spec": spec}


_cache = {}


def workload(name):
    if name not in _cache:
        w = SMALL[name]()
        p = OFF_MIN[name]
        v, g, sc, rc = oracle.nll_scaled(w["spec"], p, w["cols"].astype(np.float64))
        assert rc == 0
        _cache[name] = (w, p, v, g, sc)
    return _cache[name]


@pytest.mark.parametrize("jit", [True, False])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("name", sorted(SMALL))
def test_nll_and_gradient_match_oracle(rf, name, prec, jit):
    """Both kernel forms: specialised for the graph (NVRTC) and generic."""
    w, p, v, g, sc = workload(name)
    G = rf.Graph(w["spec"], w["dtype"], prec)
    if name in JIT_ONLY and not jit:
        with pytest.raises(rf.RFError):
            G.set_jit(False)
        return
    G.set_jit(jit)
    assert G.uses_jit() == jit
    nll, grad = G.nll(to_dev(w), params_dev(p))
    torch.cuda.synchronize()
    nll = float(nll.item())
    grad = grad.cpu().numpy()
    assert rel_nll(nll, v) <= TOL[prec]["nll"], (nll, v, rel_nll(nll, v))
    err = grad_l1(grad, g, sc, free_mask(w["spec"]))
    assert err.max() <= TOL[prec]["grad"], (err, grad, g)
    fixed = [not f for f in free_mask(w["spec"])]
    assert all(grad[k] == 0.0 for k in range(len(grad)) if fixed[k])
    assert G.status() == 0
    assert G.last_launches() == 2   # prologue + fused kernel


@pytest.mark.parametrize("jit", [True, False])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("name", ["c1", "c2", "c3", "c5", "johnson", "c5_free_p", "c5_fixed_p",
                                  "prod6"])
def test_per_event_log_probability(rf, name, prec, jit):
    if name in JIT_ONLY and not jit:
        pytest.skip("specialised kernels only")
    w, p, *_ = workload(name)
    sub = {**w, "cols": w["cols"][:, :20_011]}
    want, rc = oracle.logp(w["spec"], p, sub["cols"].astype(np.float64))
    G = rf.Graph(w["spec"], w["dtype"], prec)
    G.set_jit(jit)
    got = G.logp(to_dev(sub), params_dev(p)).cpu().numpy()
    err = logp_err(got, want)
    assert err.max() <= TOL[prec]["logp"], (err.max(), int(err.argmax()))


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("n", [0, 1, 3, 4, 5, 7, 8, 9, 31, 32, 33, 1023, 1024, 1025, 100_007])
def test_shape_sweep(rf, n, prec):
    w = datagen.c2(n=n) if n > 0 else {**datagen.c2(n=1), "cols": np.zeros((1, 0))}
    p = OFF_MIN["c2"]
    v, g, sc, rc = oracle.nll_scaled(w["spec"], p, w["cols"])
    G = rf.Graph(w["spec"], "f64", prec)
    nll, grad = G.nll(to_dev(w), params_dev(p))
    nll = float(nll.item())
    if n == 0:
        assert nll == 0.0 and np.all(grad.cpu().numpy() == 0.0)
        return
    assert rel_nll(nll, v) <= TOL[prec]["nll"]
    if prec == "fp32" and n < 200:
        # the FP32 gradient bound is for samples, not single events: one
        # event's d/d lambda is w (x - <x>), which cancels near the mean, and
        # its own size is the whole L1 scale (the same reading as for tiny toys)
        return
    assert grad_l1(grad.cpu().numpy(), g, sc, [True] * 4).max() <= TOL[prec]["grad"]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("n,shift", [(4001, 0), (4000, 1), (4003, 3), (4004, 2), (2, 1),
                                     (200_003, 1)])
def test_unaligned_columns(rf, n, shift, prec):
    """Column bases off the 16-byte grid (a sliced buffer) and column phases
    that differ between observables (n not a multiple of 4): the lane-
    interleaved 32-bit loads, their tail, and (200,003 events) many blocks."""
    w = datagen.c3(n=n)
    p = OFF_MIN["c3"][:7] + [float(n)]
    v, g, sc, rc = oracle.nll_scaled(w["spec"], p, w["cols"].astype(np.float64))
    flat = torch.zeros(3 * n + shift, dtype=torch.float32, device=DEV)
    flat[shift:] = torch.from_numpy(w["cols"].reshape(-1)).to(DEV)
    ev = flat[shift:].view(3, n)
    G = rf.Graph(w["spec"], "f32", prec)
    nll, grad = G.nll(ev, params_dev(p))
    assert rel_nll(float(nll.item()), v) <= TOL[prec]["nll"]
    assert grad_l1(grad.cpu().numpy(), g, sc, [True] * 8).max() <= TOL[prec]["grad"]


@pytest.mark.parametrize("jit", [True, False])
def test_every_launch_configuration(rf, jit):
    w, p, v, g, sc = workload("c5")
    ev = to_dev(w)
    pd = params_dev(p)
    for prec, epts in (("fp32", (4, 8, 16) if jit else (4, 8)), ("fp64", (4,))):
        G = rf.Graph(w["spec"], "f32", prec)
        G.set_jit(jit)
        for block in (64, 128, 256):
            for ept in epts:
                for bps in (1, 2, 3, 4, 6, 8):
                    for mb in ((2, 3, 4) if jit else (2,)):
                        G.set_launch(block=block, ept=ept, blocks_per_sm=bps, min_blocks=mb)
                        nll, grad = G.nll(ev, pd)
                        cfg = (block, ept, bps, mb)
                        assert rel_nll(float(nll.item()), v) <= TOL[prec]["nll"], cfg
                        err = grad_l1(grad.cpu().numpy(), g, sc, free_mask(w["spec"]))
                        assert err.max() <= TOL[prec]["grad"], (cfg, err)


def test_launch_defaults_and_invalid_register_budget(rf):
    w, p, *_ = workload("c2")
    assert rf.Graph(w["spec"], "f64", "fp32").get_launch()["min_blocks"] == 3
    G = rf.Graph(w["spec"], "f64", "fp64")
    assert G.get_launch()["min_blocks"] == 2
    with pytest.raises(rf.RFError):
        G.set_launch(min_blocks=5)
    assert G.get_launch()["min_blocks"] == 2


def test_tuner_picks_a_valid_configuration(rf):
    w, p, v, *_ = workload("c2")
    G = rf.Graph(w["spec"], "f64", "fp32")
    ms = G.tune(to_dev(w), params_dev(p))
    assert ms > 0
    cfg = G.get_launch()
    assert cfg["block"] in (64, 128, 256) and cfg["ept"] in (4, 8, 16)
    assert cfg["min_blocks"] in (2, 3, 4)
    nll, _ = G.nll(to_dev(w), params_dev(p))
    assert rel_nll(float(nll.item()), v) <= TOL["fp32"]["nll"]


def test_tuner_cache_round_trip(rf):
    """A tuned configuration is stored on disk under the graph's kernel,
    precisions, size bucket and device: a second graph of the same model finds
    it and times only that configuration; cache=False times every one."""
    w, p, v, *_ = workload("c2")
    ev, pd = to_dev(w), params_dev(p)
    G = rf.Graph(w["spec"], "f64", "fp32")
    G.tune(ev, pd, refresh=True)
    assert not G.tune_from_cache
    first = G.get_launch()
    H = rf.Graph(w["spec"], "f64", "fp32")
    assert H.tune(ev, pd) > 0
    assert H.tune_from_cache and H.get_launch() == first
    H.tune(ev, pd, cache=False)
    assert not H.tune_from_cache
    nll, _ = H.nll(ev, pd)
    assert rel_nll(float(nll.item()), v) <= TOL["fp32"]["nll"]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_run_to_run_bitwise_determinism(rf, prec):
    w, p, *_ = workload("c5")
    G = rf.Graph(w["spec"], "f32", prec)
    ev, pd = to_dev(w), params_dev(p)
    a = torch.cat(G.nll(ev, pd)).cpu()
    for _ in range(3):
        b = torch.cat(G.nll(ev, pd)).cpu()
        assert torch.equal(a, b)


def test_back_to_back_calls_with_changing_parameters(rf):
    """Calls queued back to back on one stream (each prologue overlaps the
    previous call's event pass): parameters rewritten between calls by a
    device kernel and by a host copy, two graphs interleaved, outputs written
    to separate buffers; every result equals the same call made alone."""
    w, p, *_ = workload("c5")
    G = rf.Graph(w["spec"], "f32", "fp32")
    w2, p2, *_ = workload("c2")
    G2 = rf.Graph(w2["spec"], "f64", "fp32")
    ev, ev2 = to_dev(w), to_dev(w2)
    pts = [np.array(p) * (1.0 + 1e-3 * k * np.array([0, 1, 1, 0, 0, 1, 0, 1, 1]))
           for k in range(4)]
    alone = []
    for q in pts:
        alone.append(torch.cat(G.nll(ev, params_dev(list(q)))).cpu())
    alone2 = torch.cat(G2.nll(ev2, params_dev(p2))).cpu()
    torch.cuda.synchronize()
    pd = params_dev(list(pts[0]))
    pd2 = params_dev(p2)
    outs = [torch.empty(1 + len(p), dtype=torch.float64, device=DEV) for _ in pts]
    out2 = torch.empty(1 + len(p2), dtype=torch.float64, device=DEV)
    for k in range(len(pts)):
        if k == 1:
            pd.copy_(torch.from_numpy(pts[1]).to(DEV))          # device-side update
        elif k == 2:
            pd.copy_(torch.from_numpy(pts[2]), non_blocking=False)  # host copy
        elif k == 3:
            pd.mul_(0).add_(torch.from_numpy(pts[3]).to(DEV))   # two device kernels
        G.nll(ev, pd, out=outs[k])
        G2.nll(ev2, pd2, out=out2)
    torch.cuda.synchronize()
    for k in range(len(pts)):
        assert torch.equal(outs[k].cpu(), alone[k]), k
    assert torch.equal(out2.cpu(), alone2)


@pytest.mark.parametrize("shards", [2, 3])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_sharded_evaluation_adds_up(rf, shards, prec):
    """A dataset split into contiguous shards (the multi-process mode of
    Sec. 5.2): each shard evaluated by its own graph on the GPU, the extended
    term weighted 1 on one shard and 0 on the others, the shards' (NLL,
    gradient) added in rank order with compensation (the reduction every rank
    of sharded_nll runs) -- against the oracle's whole-dataset NLL and
    gradient."""
    w = datagen.c4(toys=1, nu_s_range=(30_000, 30_001), nu_b_range=(90_000, 90_001))
    spec = w["spec"]
    p = [5.03, 0.51, -0.29, 29_500.0, 91_000.0]
    ev = to_dev(w)
    n = ev.shape[1]
    parts = []
    for r in range(shards):
        lo, hi = rf.shard_range(n, r, shards)
        G = rf.Graph(spec, "f64", prec)
        G.set_shard_weight(1.0 if r == 0 else 0.0)
        parts.append(torch.cat(G.nll(ev[:, lo:hi].contiguous(), params_dev(p))))
    total = rf.rank_order_sum(torch.stack(parts)).cpu().numpy()
    v, gref, sc, rc = oracle.nll_scaled(spec, p, w["cols"])
    assert rc == 0
    assert rel_nll(total[0], v) <= TOL[prec]["nll"]
    assert grad_l1(total[1:], gref, sc, [True] * 5).max() <= TOL[prec]["grad"]
    again = rf.rank_order_sum(torch.stack(parts)).cpu().numpy()
    assert np.array_equal(again.view(np.int64), total.view(np.int64))


def test_gradient_against_finite_differences(rf):
    """GPU adjoint vs Richardson differences of the GPU FP64 NLL (<= 1e-4)."""
    w, p, v, g, sc = workload("c2")
    G = rf.Graph(w["spec"], "f64", "fp64")
    ev = to_dev(w)
    _, grad = G.nll(ev, params_dev(p))
    grad = grad.cpu().numpy()
    G32 = rf.Graph(w["spec"], "f64", "fp32")
    _, grad32 = G32.nll(ev, params_dev(p))
    grad32 = grad32.cpu().numpy()
    for j in range(4):
        h = 1e-4 * max(abs(p[j]), 1e-2)

        def f(x):
            q = list(p)
            q[j] = x
            return float(G.nll(ev, params_dev(q), grad=False)[0].item())
        d1 = (f(p[j] + h) - f(p[j] - h)) / (2 * h)
        d2 = (f(p[j] + h / 2) - f(p[j] - h / 2)) / h
        fd = (4 * d2 - d1) / 3
        assert abs(grad[j] - fd) <= 1e-4 * sc[j]
        assert abs(grad32[j] - fd) <= 1e-4 * sc[j]


def test_parameter_domain_errors(rf):
    w, p, *_ = workload("c2")
    G = rf.Graph(w["spec"], "f64", "fp32")
    ev = to_dev(w)
    for bad in ([5.0, -0.5, -0.3, 0.2], [5.0, 0.5, -0.3, 1.5], [5.0, 0.0, -0.3, 0.2]):
        nll, grad = G.nll(ev, params_dev(bad))
        assert math.isinf(float(nll.item())) and float(nll.item()) > 0
        assert torch.isnan(grad).all()
    st = G.status()
    assert st & 1
    assert G.status() == 0          # cleared on read
    # an event where the Chebychev polynomial is negative: non-finite log P
    cheb = {"obs": [(-1.0, 1.0)], "params": [1.5], "fixed": [False],
            "nodes": [{"type": "cheb", "obs": 0, "params": [0]}], "root": 0}
    G2 = rf.Graph(cheb, "f64", "fp64")
    nll, _ = G2.nll(torch.tensor([[-0.9, 0.5]], dtype=torch.float64, device=DEV),
                    params_dev([1.5]))
    assert math.isinf(float(nll.item()))
    assert G2.status() & 2


@pytest.mark.parametrize("jit", [True, False])
def test_zero_fraction_edge(rf, jit):
    """f = 0 and f = 1: a component with coefficient exactly 0.  d/df there
    sums the absent component's P_c/P, which reaches e^50 for events 10 sigma
    from the Gaussian; FP32 evaluation therefore runs such a call's events in
    FP64 and meets the FP32 bounds on every gradient component.  Also the
    per-event log P of such a call."""
    w, p, *_ = workload("c2")
    for f in (0.0, 1.0):
        q = [5.0, 0.5, -0.3, f]
        v, g, sc, rc = oracle.nll_scaled(w["spec"], q, w["cols"])
        want, _ = oracle.logp(w["spec"], q, w["cols"][:, :5003])
        for prec in ("fp64", "fp32"):
            G = rf.Graph(w["spec"], "f64", prec)
            G.set_jit(jit)
            nll, grad = G.nll(to_dev(w), params_dev(q))
            assert rel_nll(float(nll.item()), v) <= TOL[prec]["nll"]
            err = grad_l1(grad.cpu().numpy(), g, sc, [True] * 4)
            assert err.max() <= TOL[prec]["grad"], (f, prec, err)
            got = G.logp(to_dev({**w, "cols": w["cols"][:, :5003]}), params_dev(q))
            assert logp_err(got.cpu().numpy(), want).max() <= TOL[prec]["logp"]


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_six_leaf_toys(rf, prec):
    """Toys of the six-leaf model (three two-observable components): the
    batched NLL and gradient of every toy against the oracle."""
    w = datagen.prod6(40_000)
    spec = w["spec"]
    off = np.array([0, 3_000, 3_001, 9_500, 9_500, 21_000, 40_000], np.int64)
    rng = np.random.default_rng(5)
    pm = np.array(OFF_MIN["prod6"])[None, :] * (1 + 0.01 * rng.standard_normal((6, 14)))
    pm[:, 12:] = [0.3, 0.3]
    want, rc = oracle.nll_batched(spec, w["cols"], off, pm)
    assert rc == 0
    G = rf.Graph(spec, "f32", prec)
    G.bind_events(to_dev(w), 6)
    got = G.nll_batched(torch.from_numpy(off).to(DEV), torch.from_numpy(pm).to(DEV)).cpu().numpy()
    for t in range(6):
        n_t = int(off[t + 1] - off[t])
        if n_t == 0:
            continue
        assert rel_nll(got[t, 0], want[t, 0]) <= TOL[prec]["nll"], (t, got[t, 0], want[t, 0])
        if n_t >= 200:
            _, _, sc, _ = oracle.nll_scaled(spec, pm[t], w["cols"][:, off[t]:off[t + 1]])
            assert grad_l1(got[t, 1:], want[t, 1:], sc, [True] * 14).max() <= TOL[prec]["grad"]


def test_zero_yield_toys_and_ragged_ends(rf):
    """Toys with an exactly zero yield among ordinary toys (FP32 evaluation:
    those toys' events in FP64), and a single dataset whose length leaves a
    ragged head and tail, against the oracle."""
    spec = datagen.gauss_exp_ext_spec()
    w = datagen.c4(toys=24, nu_s_range=(300, 3000), nu_b_range=(500, 5000))
    pm = np.array(w["params_matrix"], np.float64)
    pm[3::4, 3] = 0.0          # signal yield 0 in toys 3, 7, 11, ...
    pm[2::6, 4] = 0.0          # background yield 0 in toys 2, 8, 14, 20
    want, rc = oracle.nll_batched(spec, w["cols"], w["offsets"], pm)
    assert rc == 0
    for prec in ("fp32", "fp64"):
        G = rf.Graph(spec, "f64", prec)
        G.bind_events(to_dev(w), 24)
        got = G.nll_batched(torch.from_numpy(w["offsets"]).to(DEV),
                            torch.from_numpy(pm).to(DEV)).cpu().numpy()
        for t in range(24):
            n_t = int(w["offsets"][t + 1] - w["offsets"][t])
            if n_t == 0:
                continue
            assert rel_nll(got[t, 0], want[t, 0]) <= TOL[prec]["nll"], (prec, t)
            if n_t >= 200:
                _, _, sc, _ = oracle.nll_scaled(spec, pm[t],
                                                w["cols"][:, w["offsets"][t]:w["offsets"][t + 1]])
                assert grad_l1(got[t, 1:], want[t, 1:], sc, [True] * 5).max() <= TOL[prec]["grad"]
    # a single dataset with a zero yield, FP32 columns at an odd offset
    w5 = datagen.c5(2_000, 60_000)
    q = [5.2792, 0.0031, 1.55, 3.1, 5.29, -19.5, 0.5, 0.0, 61_000.0]
    cols = np.ascontiguousarray(w5["cols"][:, 3:60_002])
    v, g, sc, rc = oracle.nll_scaled(w5["spec"], q, cols.astype(np.float64))
    assert rc == 0
    G = rf.Graph(w5["spec"], "f32", "fp32")
    nll, grad = G.nll(torch.from_numpy(cols).to(DEV), params_dev(q))
    assert rel_nll(float(nll.item()), v) <= TOL["fp32"]["nll"]
    assert grad_l1(grad.cpu().numpy(), g, sc, free_mask(w5["spec"])).max() <= TOL["fp32"]["grad"]


def test_autograd_function(rf):
    w, p, v, g, sc = workload("c2")
    G = rf.Graph(w["spec"], "f64", "fp64")
    pt = params_dev(p).requires_grad_(True)
    out = rf.RFNll.apply(pt, to_dev(w), G)
    (2.0 * out).backward()
    assert rel_nll(float(out.item()), v) <= 1e-12
    err = grad_l1(pt.grad.cpu().numpy() / 2.0, g, sc, [True] * 4)
    assert err.max() <= 1e-10


def test_host_buffers_entry_point(rf):
    w, p, v, g, sc = workload("c3")
    G = rf.Graph(w["spec"], "f32", "fp32")
    ev = torch.from_numpy(np.ascontiguousarray(w["cols"])).pin_memory()
    nll, grad = G.nll_host(ev, torch.tensor(p, dtype=torch.float64))
    d_nll, d_grad = G.nll(to_dev(w), params_dev(p))
    # same kernel; a differently aligned host buffer may change the chunking
    assert rel_nll(nll, float(d_nll.item())) <= TOL["fp32"]["nll"]
    assert grad_l1(grad.numpy(), d_grad.cpu().numpy(), sc, [True] * 8).max() <= TOL["fp32"]["grad"]
    assert rel_nll(nll, v) <= TOL["fp32"]["nll"]
    # pageable host memory goes through the staging copy
    nll2, _ = G.nll_host(torch.from_numpy(np.ascontiguousarray(w["cols"])),
                         torch.tensor(p, dtype=torch.float64))
    assert rel_nll(nll2, v) <= TOL["fp32"]["nll"]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_plain_node_by_node_baseline(rf, prec):
    w, p, v, g, sc = workload("c5")
    G = rf.Graph(w["spec"], "f32", prec)
    nll, grad = G.nll_plain(to_dev(w), params_dev(p))
    assert rel_nll(float(nll.item()), v) <= 1e-12        # always FP64
    err = grad_l1(grad.cpu().numpy(), g, sc, free_mask(w["spec"]))
    assert err.max() <= 1e-4                              # central differences
    assert G.last_launches() > 10


def small_toys(t=64):
    return datagen.c4(toys=t, nu_s_range=(20.0, 2000.0), nu_b_range=(50.0, 5000.0))


@pytest.mark.parametrize("jit", [True, False])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("shape", [(256, 2), (64, 1)])
def test_batched_toys_match_oracle_and_single(rf, prec, shape, jit):
    """Every toy against the oracle and against a single-dataset call; two
    launch shapes (2432 and 304 warps over ~95k events, so warp ranges and
    toys cut each other in different places)."""
    w = small_toys()
    pm = w["params_matrix"].copy()
    pm[:, 0] += 0.02
    want, rc = oracle.nll_batched(w["spec"], w["cols"], w["offsets"], pm)
    G = rf.Graph(w["spec"], "f64", prec)
    G.set_jit(jit)
    ev = to_dev(w)
    G.set_launch(block=shape[0], blocks_per_sm=shape[1])
    assert int(G.toy_kernel_hash(), 16) == 0  # no toy kernel before the bind
    assert G.get_toy_launch()["regs_per_thread"] == 0
    G.bind_events(ev, 64)
    assert (int(G.toy_kernel_hash(), 16) != 0) == jit
    assert G.toy_kernel_hash() != G.kernel_hash() or not jit
    tl = G.get_toy_launch()
    assert tl["block"] == shape[0] and tl["events_per_lane"] in (4, 8, 16)
    assert (tl["regs_per_thread"] > 0) == jit
    off = torch.from_numpy(w["offsets"]).to(DEV)
    pmd = torch.from_numpy(pm).to(DEV)
    got = G.nll_batched(off, pmd).cpu().numpy()
    assert G.last_launches() == 3
    for t in range(64):
        b, e = w["offsets"][t], w["offsets"][t + 1]
        _, gref, sc, _ = oracle.nll_scaled(w["spec"], pm[t], w["cols"][:, b:e])
        assert rel_nll(got[t, 0], want[t, 0]) <= TOL[prec]["nll"], t
        assert grad_l1(got[t, 1:], gref, sc, [True] * 5).max() <= TOL[prec]["grad"], t
        single = G.nll(ev[:, b:e].contiguous(), pmd[t].contiguous())
        assert rel_nll(float(single[0].item()), got[t, 0]) <= TOL[prec]["nll"]


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_batched_toys_bulk_copy_form(rf, prec, monkeypatch):
    """The segment kernel's bulk-copy form (per-warp shared-memory stage rings
    filled by cp.async.bulk, RF_TOY_STREAM=bulk at graph compile) against the
    oracle, with hundreds of tiny toys among large ones."""
    monkeypatch.setenv("RF_TOY_STREAM", "bulk")
    w = small_toys(256)
    counts = np.diff(w["offsets"]).copy()
    counts[5:205] = np.arange(200) % 7           # 200 toys of 0..6 events
    off = np.zeros(len(counts) + 1, np.int64)
    np.cumsum(counts, out=off[1:])
    pm = w["params_matrix"].copy()
    pm[:, 0] += 0.01
    want, rc = oracle.nll_batched(w["spec"], w["cols"], off, pm)
    G = rf.Graph(w["spec"], "f64", prec)
    G.bind_events(to_dev(w), len(counts))
    got = G.nll_batched(torch.from_numpy(off).to(DEV), torch.from_numpy(pm).to(DEV)).cpu().numpy()
    assert G.status() == 0
    for t in range(len(counts)):
        assert rel_nll(got[t, 0], want[t, 0]) <= TOL[prec]["nll"], t
        if counts[t] >= 200 or prec == "fp64":
            if counts[t] == 0:
                continue
            b, e = off[t], off[t + 1]
            _, gref, sc, _ = oracle.nll_scaled(w["spec"], pm[t], w["cols"][:, b:e])
            assert grad_l1(got[t, 1:], gref, sc, [True] * 5).max() <= TOL[prec]["grad"], t


def test_batched_empty_and_tiny_toys(rf):
    w = small_toys(8)
    off = w["offsets"].copy()
    # toy 2 empty, toy 5 one event
    counts = np.diff(off)
    counts[2] = 0
    counts[5] = 1
    new_off = np.zeros(9, np.int64)
    np.cumsum(counts, out=new_off[1:])
    pm = w["params_matrix"]
    want, _ = oracle.nll_batched(w["spec"], w["cols"], new_off, pm)
    G = rf.Graph(w["spec"], "f64", "fp64")
    G.bind_events(to_dev(w), 8)
    got = G.nll_batched(torch.from_numpy(new_off).to(DEV),
                        torch.from_numpy(pm).to(DEV)).cpu().numpy()
    np.testing.assert_allclose(got[:, 0], want[:, 0], rtol=1e-12)
    assert got[2, 0] == pm[2, 3] + pm[2, 4]          # extended term only


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_batched_ragged_layouts(rf, prec):
    """Toy layouts that stress the even split of events over warps: 700 toys
    of 0..40 events (many toys per warp range, empty toys inside ranges),
    toys that do not start at event 0 or end at the last bound event, and
    fewer events than warps; each toy against the oracle (NLL and, in FP64,
    every gradient component)."""
    rng = np.random.default_rng(17)
    base = datagen.c4(toys=16, nu_s_range=(500.0, 600.0), nu_b_range=(2000.0, 2100.0))
    cols = base["cols"]
    n = cols.shape[1]
    spec = base["spec"]
    for counts, first in [(rng.integers(0, 41, 700), 0),
                          (rng.integers(0, 41, 700), 123),
                          (np.array([0, 3, 0, 0, 1, 2, 0]), 5),
                          (np.array([n - 10]), 9)]:
        toys = len(counts)
        off = np.zeros(toys + 1, np.int64)
        off[0] = first
        np.cumsum(counts, out=off[1:])
        off[1:] += first
        assert off[-1] <= n
        pm = np.repeat(base["params_matrix"][:1], toys, axis=0)
        pm[:, 0] += rng.uniform(-0.05, 0.05, toys)
        want, _ = oracle.nll_batched(spec, cols, off, pm)
        G = rf.Graph(spec, "f64", prec)
        G.bind_events(torch.from_numpy(cols).to(DEV), toys)
        got = G.nll_batched(torch.from_numpy(off).to(DEV),
                            torch.from_numpy(pm).to(DEV)).cpu().numpy()
        assert G.status() == 0
        for t in range(toys):
            assert rel_nll(got[t, 0], want[t, 0]) <= TOL[prec]["nll"], (toys, t)
            if off[t + 1] > off[t]:
                b, e = off[t], off[t + 1]
                # FP32 gradients of toys under 200 events are not compared:
                # the FP32 error of a single tail event's weight exp(-|dv|)
                # (relative |dv| 2^-23 and the FP32 rounding of x) is not
                # averaged over so few events; FP64 checks every toy
                if prec == "fp64" or e - b >= 200:
                    _, gref, sc, _ = oracle.nll_scaled(spec, pm[t], cols[:, b:e])
                    err = grad_l1(got[t, 1:], gref, sc, [True] * 5)
                    assert err.max() <= TOL[prec]["grad"], (toys, t)
            else:
                assert got[t, 0] == pm[t, 3] + pm[t, 4]


def test_batched_decreasing_offsets_raise_status(rf):
    """A decreasing offset pair is reported through the status word; the
    call reads nothing outside the bound columns and later calls are
    unaffected."""
    w = small_toys(8)
    G = rf.Graph(w["spec"], "f64", "fp64")
    G.bind_events(to_dev(w), 8)
    pmd = torch.from_numpy(w["params_matrix"]).to(DEV)
    bad = w["offsets"].copy()
    bad[3], bad[4] = bad[4], bad[3]
    G.nll_batched(torch.from_numpy(bad).to(DEV), pmd)
    assert G.status() & 2
    good = G.nll_batched(torch.from_numpy(w["offsets"]).to(DEV), pmd).cpu().numpy()
    assert G.status() == 0
    want, _ = oracle.nll_batched(w["spec"], w["cols"], w["offsets"], w["params_matrix"])
    np.testing.assert_allclose(good[:, 0], want[:, 0], rtol=1e-12)


def test_fit_toys_follows_oracle_adam(rf):
    """50 Adam steps per toy, CUDA-graph replayed, against the oracle replaying
    the same updates from its own gradients (16 toys, FP64 evaluation); each
    toy's parameters are moved in units of their starting |theta|."""
    w = small_toys(16)
    pm0 = w["params_matrix"].copy()
    scale = np.maximum(np.abs(pm0), 1.0)
    iters, lr = 50, 1e-2
    G = rf.Graph(w["spec"], "f64", "fp64")
    G.bind_events(to_dev(w), 16)
    pmd = torch.from_numpy(pm0.copy()).to(DEV)
    G.fit_toys(torch.from_numpy(w["offsets"]).to(DEV), pmd,
               torch.from_numpy(scale).to(DEV), iters, lr)
    assert G.last_launches() == 3 * iters
    got = pmd.cpu().numpy()
    for t in range(16):
        b, e = w["offsets"][t], w["offsets"][t + 1]
        th = pm0[t].copy()
        m1, m2 = np.zeros(5), np.zeros(5)
        for it in range(1, iters + 1):
            v, gr, _ = oracle.nll(w["spec"], th, w["cols"][:, b:e])
            assert np.isfinite(v)
            oracle.adam_step(th, gr, scale[t], [1] * 5, m1, m2, it, lr)
        np.testing.assert_allclose(got[t], th, rtol=1e-9, atol=1e-9)
    # the fit lowered the NLL summed over the toys
    before = sum(oracle.nll(w["spec"], pm0[t], w["cols"][:, w["offsets"][t]:w["offsets"][t + 1]],
                            grad=False)[0] for t in range(16))
    after = sum(oracle.nll(w["spec"], got[t], w["cols"][:, w["offsets"][t]:w["offsets"][t + 1]],
                           grad=False)[0] for t in range(16))
    assert after < before


def test_fast_log_accuracy(rf):
    """The library's FP32 log (hardware lg2.approx times ln 2, used for every
    per-event log-density) against an FP64 reference: absolute error within
    2^-21 * ln2 * max(1, |log2 x|) (twice the documented lg2.approx bound),
    the scale of one FP32 rounding of the result; CUDA logf shown beside it."""
    rng = np.random.default_rng(5)
    x = np.concatenate([np.exp(rng.uniform(-80, 80, 400_000)),
                        1.0 + rng.uniform(-1e-3, 1e-3, 100_000),
                        rng.uniform(0.5, 2.0, 200_000),
                        np.array([1.0, 2.0, 0.5, 0.70710677, 1.4142135, 1e-37, 3e38])]
                       ).astype(np.float32)
    yf, yr = rf.check_log(torch.from_numpy(x).to(DEV))
    ref = np.log(x.astype(np.float64))
    bound = 2.0 ** -21 * np.log(2.0) * np.maximum(1.0, np.abs(np.log2(x.astype(np.float64))))
    err_fast = np.abs(yf.cpu().numpy().astype(np.float64) - ref)
    err_cuda = np.abs(yr.cpu().numpy().astype(np.float64) - ref)
    assert np.all(err_fast <= bound), (err_fast / bound).max()
    assert np.all(err_cuda <= bound)
    # special values
    sp = torch.tensor([0.0, -1.0, float("inf"), float("nan")], device=DEV)
    a, _ = rf.check_log(sp)
    a = a.cpu().numpy()
    assert a[0] == -np.inf and np.isnan(a[1]) and a[2] == np.inf and np.isnan(a[3])


def test_double_to_float_rounding_is_exact(rf):
    """FP64 columns evaluated in FP32 are rounded by integer operations; the
    result must equal the hardware round-to-nearest-even bit for bit,
    including halfway cases, carries into the exponent and the fallbacks."""
    rng = np.random.default_rng(11)
    x = np.concatenate([rng.normal(0, 3, 300_000), np.exp(rng.uniform(-100, 100, 300_000)),
                        -np.exp(rng.uniform(-90, 90, 100_000)), rng.uniform(0, 10, 100_000)])
    f = x.astype(np.float32).astype(np.float64)
    ulp = np.spacing(np.abs(x.astype(np.float32))).astype(np.float64)
    halfway = np.concatenate([f + 0.5 * ulp, f - 0.5 * ulp, f + 0.5000001 * ulp])
    special = np.array([0.0, -0.0, 1e-40, -1e-45, 3.4028235677973366e38, 3.5e38, 1e300,
                        np.inf, -np.inf, np.nan, 1.1754943508222875e-38,
                        1.1754942e-38, 2.0 ** -149, 2.0 ** 128 - 2.0 ** 103])
    allx = np.concatenate([x, halfway, special])
    yf, yr = rf.check_d2f(torch.from_numpy(allx).to(DEV))
    a = yf.cpu().numpy().view(np.uint32)
    b = yr.cpu().numpy().view(np.uint32)
    nan = np.isnan(yr.cpu().numpy())
    assert np.array_equal(a[~nan], b[~nan])
    assert np.all(np.isnan(yf.cpu().numpy()[nan]))


def test_microbench_reports_positive_rates(rf):
    r = rf.microbench()
    assert all(v > 0 for v in r.values())
    assert r["fp32_fma"] > r["fp64_fma"]


def test_argus_fixed_p_other_than_one_half_is_a_domain_error(rf):
    """A p fixed at 1/2 when the graph is compiled runs the p = 1/2 form;
    calling it with another value sets the parameter-domain bit (a free p
    takes any p > 0, and so does a p fixed away from 1/2 at compile time)."""
    w, p, *_ = workload("c5")
    G = rf.Graph(w["spec"], "f32", "fp32")
    q = list(p)
    q[6] = 0.7
    nll, grad = G.nll(to_dev(w), params_dev(q))
    assert nll.item() == float("inf") and G.status() & rf.STATUS_PARAM_DOMAIN
    w2, p2, v2, *_ = workload("c5_free_p")
    G2 = rf.Graph(w2["spec"], "f32", "fp64")
    q2 = list(p2)
    for bad in (0.0, -0.2):
        q2[6] = bad
        nll, _ = G2.nll(to_dev(w2), params_dev(q2))
        assert nll.item() == float("inf") and G2.status() & rf.STATUS_PARAM_DOMAIN


@pytest.mark.parametrize("pval", [0.5, 1.3])
def test_argus_free_p_values(rf, pval):
    """Free p away from 1/2, FP64 evaluation: NLL and gradient (d/dp
    included) against the oracle."""
    w, p, *_ = workload("c5_free_p")
    q = list(p)
    q[6] = pval
    v, g, sc, rc = oracle.nll_scaled(w["spec"], q, w["cols"].astype(np.float64))
    assert rc == 0
    G = rf.Graph(w["spec"], "f32", "fp64")
    nll, grad = G.nll(to_dev(w), params_dev(q))
    assert rel_nll(float(nll.item()), v) <= TOL["fp64"]["nll"]
    assert grad_l1(grad.cpu().numpy(), g, sc, free_mask(w["spec"])).max() <= TOL["fp64"]["grad"]
