"""Formula leaves (the formula PDFs of Sec. 4) on the GPU against the oracle.

The oracle parses the text itself, walks its tree with forward derivatives and
integrates it by adaptive Gauss-Legendre quadrature; the library translates
the text into the graph's NVRTC-compiled kernels and integrates it by fixed
composite Gauss-Legendre in a normalisation kernel.  Both are compared on the
NLL, the gradient and per-event log P, in FP64 and FP32 evaluation, at sizes
that span many blocks and a ragged tail; plus domain errors, the calls that do
not take formula leaves, back-to-back calls with changing parameters and the
tuner."""
import numpy as np
import pytest
import torch

import datagen
import oracle
from _common import TOL, free_mask, grad_l1, logp_err, rel_nll

pytestmark = pytest.mark.gpu
DEV = "cuda"

GAUSS = "exp(-0.5*((x-p0)/p1)^2)"


@pytest.fixture(scope="module")
def rf():
    import paper_2003_12875_gb300 as rf
    rf.load()
    return rf


def as_formulas(spec, texts):
    s = {**spec, "nodes": [dict(n) for n in spec["nodes"]]}
    for i, t in texts.items():
        s["nodes"][i].update(type="formula", formula=t)
    return s


def bw_exp_spec(nu_s=3000.0, nu_b=7000.0):
    # Breit-Wigner (m, Gamma/2) + exponential, extended, on [0, 10]
    return {"obs": [(0.0, 10.0)], "params": [4.2, 0.6, -0.25, nu_s, nu_b],
            "nodes": [{"type": "formula", "formula": "1/(1+((x-p0)/p1)^2)", "obs": 0,
                       "params": [0, 1]},
                      {"type": "formula", "formula": "exp(p0*x)", "obs": 0, "params": [2]},
                      {"type": "add_ext", "children": [0, 1], "params": [3, 4]}],
            "root": 2}


def poly_gauss_spec():
    # two observables: a skewed bump x^2 exp(-p0 x) + p1 on [0, 8] times a
    # Gaussian written as a formula on [-5, 5]
    return {"obs": [(0.0, 8.0), (-5.0, 5.0)], "params": [1.3, 0.05, 0.2, 1.1],
            "nodes": [{"type": "formula", "formula": "x^2*exp(-p0*x) + p1", "obs": 0,
                       "params": [0, 1]},
                      {"type": "formula", "formula": GAUSS, "obs": 1, "params": [2, 3]},
                      {"type": "prod", "children": [0, 1]}],
            "root": 2}


def data_one(n, seed, lo, hi, dtype):
    r = np.random.default_rng(seed)
    x = np.concatenate([r.normal(4.3, 0.8, n // 2), lo + (hi - lo) * r.random(n - n // 2)])
    x = np.clip(x, lo, hi).astype(dtype)
    r.shuffle(x)
    return x.reshape(1, -1)


def data_two(n, seed, dtype):
    r = np.random.default_rng(seed)
    a = np.clip(r.gamma(3.0, 1 / 1.3, n), 0.0, 8.0)
    b = np.clip(r.normal(0.2, 1.1, n), -5.0, 5.0)
    return np.stack([a, b]).astype(dtype)


CASES = {
    "gauss_exp_as_formulas": (lambda: as_formulas(datagen.gauss_exp_ext_spec(),
                                                  {0: GAUSS, 1: "exp(p0*x)"}),
                              lambda dt: datagen.c4(toys=1)["cols"][:, :30_011].astype(dt),
                              [5.03, 0.52, -0.31, 9_000.0, 21_000.0]),
    "breit_wigner_exp": (bw_exp_spec, lambda dt: data_one(100_003, 7, 0.0, 10.0, dt),
                         [4.25, 0.55, -0.27, 31_000.0, 69_000.0]),
    "two_observable_prod": (poly_gauss_spec, lambda dt: data_two(50_001, 11, dt),
                            [1.25, 0.06, 0.17, 1.05]),
}


@pytest.mark.parametrize("dt", ["f32", "f64"])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("name", sorted(CASES))
def test_formula_models_match_oracle(rf, name, prec, dt):
    make, data, p = CASES[name]
    spec = make()
    cols = data(np.float32 if dt == "f32" else np.float64)
    v, g, sc, rc = oracle.nll_scaled(spec, p, cols.astype(np.float64))
    assert rc == 0
    G = rf.Graph(spec, dt, prec)
    assert G.uses_jit()
    ev = torch.from_numpy(np.ascontiguousarray(cols)).to(DEV)
    pd = torch.tensor(p, dtype=torch.float64, device=DEV)
    nll, grad = G.nll(ev, pd)
    assert G.last_launches() == 3  # normalisation, prologue, fused
    assert rel_nll(float(nll.item()), v) <= TOL[prec]["nll"], (float(nll.item()), v)
    err = grad_l1(grad.cpu().numpy(), g, sc, free_mask(spec))
    assert err.max() <= TOL[prec]["grad"], err
    assert G.status() == 0
    sub = cols[:, :20_011]
    want, _ = oracle.logp(spec, p, sub.astype(np.float64))
    got = G.logp(torch.from_numpy(np.ascontiguousarray(sub)).to(DEV), pd).cpu().numpy()
    assert logp_err(got, want).max() <= TOL[prec]["logp"]


def test_formula_equals_builtin_on_the_gpu(rf):
    """The same model written with formula leaves and with the built-in
    Gaussian and Exponential gives the same FP64 NLL and gradient."""
    spec = datagen.gauss_exp_ext_spec()
    alt = as_formulas(spec, {0: GAUSS, 1: "exp(p0*x)"})
    w = datagen.c4(toys=2)
    ev = torch.from_numpy(w["cols"]).to(DEV)
    pd = torch.tensor([5.02, 0.49, -0.29, 2.0e4, 5.0e4], dtype=torch.float64, device=DEV)
    a, ga = rf.Graph(spec, "f64", "fp64").nll(ev, pd)
    b, gb = rf.Graph(alt, "f64", "fp64").nll(ev, pd)
    assert abs(a.item() - b.item()) <= 1e-12 * abs(a.item())
    _, _, sc, _ = oracle.nll_scaled(spec, pd.cpu().numpy(), w["cols"])
    assert grad_l1(gb.cpu().numpy(), ga.cpu().numpy(), sc, [True] * 5).max() <= 1e-10


@pytest.mark.parametrize("n", [0, 1, 5, 1023, 4097])
def test_formula_small_and_ragged_sizes(rf, n):
    spec = bw_exp_spec()
    cols = data_one(max(n, 1), 3, 0.0, 10.0, np.float64)[:, :n]
    p = [4.1, 0.7, -0.2, 40.0, 60.0]
    v, g, sc, rc = oracle.nll_scaled(spec, p, cols)
    G = rf.Graph(spec, "f64", "fp64")
    nll, grad = G.nll(torch.from_numpy(np.ascontiguousarray(cols)).to(DEV),
                      torch.tensor(p, dtype=torch.float64, device=DEV))
    assert rel_nll(float(nll.item()), v) <= 1e-12
    assert grad_l1(grad.cpu().numpy(), g, sc, [True] * 5).max() <= 1e-10


def test_back_to_back_calls_with_new_parameters(rf):
    """Each call integrates the formula at its own parameters before the
    prologue reads the result."""
    spec = bw_exp_spec()
    cols = data_one(60_000, 5, 0.0, 10.0, np.float32)
    G = rf.Graph(spec, "f32", "fp64")
    ev = torch.from_numpy(cols).to(DEV)
    pts = [[4.0 + 0.05 * k, 0.5 + 0.02 * k, -0.2 - 0.01 * k, 2e4, 4e4] for k in range(6)]
    outs = [G.nll(ev, torch.tensor(q, dtype=torch.float64, device=DEV))[0] for q in pts]
    torch.cuda.synchronize()
    for q, o in zip(pts, outs):
        v, _, _ = oracle.nll(spec, q, cols.astype(np.float64), grad=False)
        assert rel_nll(float(o.item()), v) <= 1e-12


def test_formula_domain_errors(rf):
    # negative density inside the range: +inf and the non-finite bit
    spec = {"obs": [(-1.0, 1.0)], "params": [0.5],
            "nodes": [{"type": "formula", "formula": "1 + p0*x*4", "obs": 0, "params": [0]}],
            "root": 0}
    G = rf.Graph(spec, "f64", "fp64")
    ev = torch.tensor([[-0.9, 0.1, 0.5]], dtype=torch.float64, device=DEV)
    nll, grad = G.nll(ev, torch.tensor([0.5], dtype=torch.float64, device=DEV))
    assert nll.item() == float("inf") and G.status() & rf.STATUS_NONFINITE
    # a non-positive integral: +inf and the parameter-domain bit
    spec["nodes"][0]["formula"] = "x - p0"
    G = rf.Graph(spec, "f64", "fp64")
    ev = torch.tensor([[0.7, 0.9]], dtype=torch.float64, device=DEV)
    nll, grad = G.nll(ev, torch.tensor([0.5], dtype=torch.float64, device=DEV))
    assert nll.item() == float("inf") and G.status() & rf.STATUS_PARAM_DOMAIN
    assert torch.isnan(grad).all()


def test_calls_without_formula_support(rf):
    spec = bw_exp_spec()
    G = rf.Graph(spec, "f64", "fp64")
    with pytest.raises(rf.RFError):
        G.set_jit(False)
    ev = torch.from_numpy(data_one(1000, 1, 0.0, 10.0, np.float64)).to(DEV)
    with pytest.raises(rf.RFError):
        G.bind_events(ev, 4)
    pd = torch.tensor(spec["params"], dtype=torch.float64, device=DEV)
    with pytest.raises(rf.RFError):
        G.nll_plain(ev, pd)
    pm = pd.reshape(1, -1)
    cc = torch.tensor([[3, 4]], dtype=torch.int64, device=DEV)
    off = torch.tensor([0, 7], dtype=torch.int64, device=DEV)
    with pytest.raises(rf.RFError):
        G.generate_toys(pm, cc, off, seed=1)
    out = torch.zeros(1 + len(spec["params"]), dtype=torch.float64, device=DEV)
    with pytest.raises(rf.RFError):
        rf.nll_noalloc(spec, ev, pd, out)


def test_tuner_with_formula_leaves(rf):
    make, data, p = CASES["breit_wigner_exp"]
    spec = make()
    cols = data(np.float32)
    G = rf.Graph(spec, "f32", "fp32")
    ev = torch.from_numpy(cols).to(DEV)
    pd = torch.tensor(p, dtype=torch.float64, device=DEV)
    assert G.tune(ev, pd) > 0
    assert G.get_launch()["min_blocks"] in (2, 3, 4)
    v, _, _ = oracle.nll(spec, p, cols.astype(np.float64), grad=False)
    assert rel_nll(float(G.nll(ev, pd)[0].item()), v) <= TOL["fp32"]["nll"]
