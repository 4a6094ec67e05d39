"""rf_nll_noalloc: the entry point for callers that cannot allocate device
memory (its scratch is a static device array inside the library).  It must
give the same NLL and gradient as rf_nll on the same inputs, on two calls in a
row (the second call reuses the scratch the first one left behind).  This file
is collected last on purpose."""
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
def test_noalloc_matches_rf_nll_on_two_calls(rf, name, prec):
    make, p = CASES[name]
    w = make()
    dt = torch.float32 if w["dtype"] == "f32" else torch.float64
    ev = torch.from_numpy(np.ascontiguousarray(w["cols"])).to("cuda", dt)
    pd = torch.tensor(p, dtype=torch.float64, device="cuda")
    G = rf.Graph(w["spec"], w["dtype"], prec)
    ref_nll, ref_grad = G.nll(ev, pd)
    ref_nll, ref_grad = float(ref_nll.item()), ref_grad.cpu().numpy()
    _, _, scale, rc = oracle.nll_scaled(w["spec"], p, w["cols"].astype(np.float64))
    assert rc == 0
    free = free_mask(w["spec"])
    for call in range(2):
        out = torch.full((1 + len(p),), float("nan"), dtype=torch.float64, device="cuda")
        rf.nll_noalloc(w["spec"], ev, pd, out, w["dtype"], prec)
        got = out.cpu().numpy()
        assert rel_nll(got[0], ref_nll) <= TOL[prec]["nll"], (call, got[0], ref_nll)
        err = grad_l1(got[1:], ref_grad, scale, free)
        assert err.max() <= TOL[prec]["grad"], (call, err)
        assert all(got[1 + k] == 0.0 for k in range(len(p)) if not free[k])


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
