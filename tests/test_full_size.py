"""Parity at the workloads' full sizes, in the launch configuration bench.py
times (the autotuned one where bench.py tunes), against the FP64 oracle run
on the host cores.

C1 1e4 Gaussian events (FP64), C2 1e6 Gauss+Exp events (FP64 columns, FP64
and FP32 evaluation), C3 1e7 x 3 FP32 columns (FP32 evaluation), C5 1.01e8
FP32 Crystal Ball + ARGUS events (FP32 and FP64 evaluation): whole-dataset
NLL and gradient.  C4, 4096 toys of 1.31e8 events: every toy's NLL, and the
gradients of 64 sampled toys (their L1 scales computed one by one)."""
import numpy as np
import pytest
import torch

import datagen
import oracle
from _common import TOL, free_mask, grad_l1, rel_nll

pytestmark = pytest.mark.gpu

DEV = "cuda"
_data = {}


@pytest.fixture(scope="module")
def rf():
    import paper_2003_12875_gb300 as rf
    rf.load()
    return rf


def full(name):
    if name not in _data:
        _data[name] = getattr(datagen, name)()
    return _data[name]


def to_dev(w):
    dt = torch.float32 if w["dtype"] == "f32" else torch.float64
    return torch.from_numpy(np.ascontiguousarray(w["cols"])).to(DEV, dt)


# C1 at the stated point; the others at their generating values (bench.py's)
POINT = {"c1": [0.25, 1.1]}


@pytest.mark.parametrize("name,prec,tune", [("c1", "fp64", False), ("c1", "fp32", False),
                                            ("c2", "fp64", False), ("c2", "fp32", True),
                                            ("c3", "fp32", True), ("c5", "fp32", True),
                                            ("c5", "fp64", False)])
def test_full_size_nll_and_gradient(rf, name, prec, tune):
    w = full(name)
    p = POINT.get(name, w["spec"]["params"])
    v, g, sc, rc = oracle.nll_scaled(w["spec"], p, w["cols"])
    assert rc == 0
    G = rf.Graph(w["spec"], w["dtype"], prec)
    ev = to_dev(w)
    pd = torch.tensor(np.asarray(p, np.float64), device=DEV)
    if tune:
        G.tune(ev, pd)
    nll, grad = G.nll(ev, pd)
    torch.cuda.synchronize()
    assert rel_nll(float(nll.item()), v) <= TOL[prec]["nll"], (name, prec, G.get_launch())
    err = grad_l1(grad.cpu().numpy(), g, sc, free_mask(w["spec"]))
    assert err.max() <= TOL[prec]["grad"], (name, prec, err)
    assert G.status() == 0


def test_full_size_toy_study(rf):
    w = full("c4")
    G = rf.Graph(w["spec"], "f64", "fp32")
    ev = to_dev(w)
    toys = len(w["offsets"]) - 1
    G.bind_events(ev, toys)
    off = torch.from_numpy(w["offsets"]).to(DEV)
    pm = w["params_matrix"]
    got = G.nll_batched(off, torch.from_numpy(pm).to(DEV)).cpu().numpy()
    want, rc = oracle.nll_batched(w["spec"], w["cols"], w["offsets"], pm)
    assert rc == 0
    assert G.status() == 0
    rel = np.abs(got[:, 0] - want[:, 0]) / np.abs(want[:, 0])
    assert rel.max() <= TOL["fp32"]["nll"], int(rel.argmax())
    rng = np.random.default_rng(4096)
    for t in rng.choice(toys, 64, replace=False):
        b, e = w["offsets"][t], w["offsets"][t + 1]
        _, gref, sc, _ = oracle.nll_scaled(w["spec"], pm[t], w["cols"][:, b:e])
        assert grad_l1(got[t, 1:], gref, sc, [True] * 5).max() <= TOL["fp32"]["grad"], t
