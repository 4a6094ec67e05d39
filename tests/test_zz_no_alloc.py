"""rf_nll_noalloc: the entry point for callers that cannot allocate device
memory (its scratch is a static device array inside the library).  On two
calls in a row (the second reuses the scratch the first one left behind) it
must give the oracle's NLL and gradient within the parity tolerances, and the
same as rf_nll on the same inputs; its largest grid must use every row of the
scratch; and its calls must not change the free device memory.  This file is
collected last on purpose."""
import numpy as np
import pytest
import torch

import datagen
import oracle
from _common import TOL, free_mask, grad_l1, rel_nll

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2003_12875_gb300 as rf
    rf.load()
    return rf


CASES = {
    "c2": (lambda: datagen.c2(n=200_003), [5.05, 0.52, -0.28, 0.21]),
    "c5": (lambda: datagen.c5(3_000, 300_000),
           [5.2792, 0.0031, 1.55, 3.1, 5.29, -19.5, 0.5, 3_050.0, 299_000.0]),
}


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("name", sorted(CASES))
def test_noalloc_matches_oracle_and_rf_nll_on_two_calls(rf, name, prec):
    make, p = CASES[name]
    w = make()
    dt = torch.float32 if w["dtype"] == "f32" else torch.float64
    ev = torch.from_numpy(np.ascontiguousarray(w["cols"])).to("cuda", dt)
    pd = torch.tensor(p, dtype=torch.float64, device="cuda")
    G = rf.Graph(w["spec"], w["dtype"], prec)
    ref_nll, ref_grad = G.nll(ev, pd)
    ref_nll, ref_grad = float(ref_nll.item()), ref_grad.cpu().numpy()
    v, g, scale, rc = oracle.nll_scaled(w["spec"], p, w["cols"].astype(np.float64))
    assert rc == 0
    free = free_mask(w["spec"])
    for call in range(2):
        out = torch.full((1 + len(p),), float("nan"), dtype=torch.float64, device="cuda")
        rf.nll_noalloc(w["spec"], ev, pd, out, w["dtype"], prec)
        got = out.cpu().numpy()
        assert rel_nll(got[0], v) <= TOL[prec]["nll"], (call, got[0], v)
        assert grad_l1(got[1:], g, scale, free).max() <= TOL[prec]["grad"], call
        # and the same evaluation as the graph-owned path
        assert rel_nll(got[0], ref_nll) <= TOL[prec]["nll"], (call, got[0], ref_nll)
        err = grad_l1(got[1:], ref_grad, scale, free)
        assert err.max() <= TOL[prec]["grad"], (call, err)
        assert all(got[1 + k] == 0.0 for k in range(len(p)) if not free[k])


def test_noalloc_full_grid_of_1024_blocks(rf):
    """The largest grid the static scratch holds: 600,000 FP64 events at two
    events per thread fill 1172 blocks of 256 threads, capped at 1024, so every
    row of the scratch (and its group rows) is written and summed."""
    w = datagen.c2(n=600_000)
    p = [5.04, 0.49, -0.31, 0.19]
    ev = torch.from_numpy(w["cols"]).cuda()
    pd = torch.tensor(p, dtype=torch.float64, device="cuda")
    v, g, scale, rc = oracle.nll_scaled(w["spec"], p, w["cols"])
    assert rc == 0
    G = rf.Graph(w["spec"], "f64", "fp64")
    ref_nll, ref_grad = G.nll(ev, pd)
    for call in range(2):
        out = torch.full((5,), float("nan"), dtype=torch.float64, device="cuda")
        rf.nll_noalloc(w["spec"], ev, pd, out, "f64", "fp64", blocks=1024)
        got = out.cpu().numpy()
        assert rel_nll(got[0], v) <= TOL["fp64"]["nll"], (call, got[0], v)
        assert grad_l1(got[1:], g, scale, [True] * 4).max() <= TOL["fp64"]["grad"]
        assert rel_nll(got[0], float(ref_nll.item())) <= TOL["fp64"]["nll"]


def test_noalloc_allocates_no_device_memory(rf):
    """Free device memory is the same before and after ten calls (the first
    call, which loads the module and looks up the scratch, comes before)."""
    w = datagen.c2(n=50_000)
    ev = torch.from_numpy(w["cols"]).cuda()
    pd = torch.tensor([5.0, 0.5, -0.3, 0.2], dtype=torch.float64, device="cuda")
    out = torch.empty(5, dtype=torch.float64, device="cuda")
    rf.nll_noalloc(w["spec"], ev, pd, out, "f64", "fp64")
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(10):
        rf.nll_noalloc(w["spec"], ev, pd, out, "f64", "fp64")
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert np.isfinite(out[0].item())


def test_noalloc_rejects_too_many_blocks(rf):
    w = datagen.c2(n=1000)
    ev = torch.from_numpy(w["cols"]).cuda()
    pd = torch.tensor([5.0, 0.5, -0.3, 0.2], dtype=torch.float64, device="cuda")
    out = torch.empty(5, dtype=torch.float64, device="cuda")
    with pytest.raises(rf.RFError) as ei:
        rf.nll_noalloc(w["spec"], ev, pd, out, "f64", "fp64", blocks=1025)
    assert "1024" in str(ei.value)
    rf.nll_noalloc(w["spec"], ev, pd, out, "f64", "fp64", blocks=1024)
    assert np.isfinite(out[0].item())
