"""Device toy generation (rf_generate_toys) against the oracle's generator:
the same counter-based uniforms (Philox4x64-10, each side its own
implementation) and the same FP64 sampling formulas, so the columns agree
value by value -- within 1e-11 relative in FP64 columns (the two sides' erfc,
erfcinv, log and pow differ in the last bits), and in FP32 columns exactly up
to a rare one-ulp difference when an FP64 value falls next to a rounding
boundary.  Then the loop a toy study runs: events drawn on the device, bound,
evaluated and fitted there."""
import numpy as np
import pytest
import torch

import datagen
import oracle
from _common import TOL

pytestmark = pytest.mark.gpu
DEV = "cuda"


@pytest.fixture(scope="module")
def rf():
    import paper_2003_12875_gb300 as rf
    rf.load()
    return rf


def single(kind, params, lo, hi, fixed=None):
    s = {"obs": [(lo, hi)], "params": list(params),
         "nodes": [{"type": kind, "obs": 0, "params": list(range(len(params)))}], "root": 0}
    if fixed:
        s["fixed"] = fixed
    return s


CASES = [
    ("gauss", [5.0, 0.5], 0.0, 10.0, None),
    ("gauss", [0.3, 1.2], 1.0, 4.0, None),
    ("exp", [-0.3], 0.0, 10.0, None),
    ("exp", [0.8], 0.0, 10.0, None),
    ("cheb", [0.2, -0.1, 0.05, 0.02], -1.0, 1.0, None),
    ("cb", [5.279, 0.003, 1.5, 3.0], 5.20, 5.29, None),
    ("cb", [0.0, 1.0, -1.2, 1.0], -3.0, 12.0, None),
    ("argus", [5.29, -20.0, 0.5], 5.20, 5.29, [True, False, True]),
    ("argus", [5.29, 2.0, 0.5], 5.0, 5.29, [True, False, True]),
    ("johnson", [0.5, 1.3, -0.4, 1.7], -2.0, 3.0, None),
    ("johnson", [0.0, 1.0, 2.5, 0.9], 2.0, 40.0, None),
]


def compare(got, want, f32):
    got = np.asarray(got, np.float64)
    want = np.asarray(want, np.float64)
    assert got.shape == want.shape
    assert np.all(np.isfinite(got))
    if f32:
        g32, w32 = got.astype(np.float32), want.astype(np.float32)
        diff = g32.view(np.int32).astype(np.int64) - w32.view(np.int32).astype(np.int64)
        assert np.abs(diff).max() <= 1
        assert np.count_nonzero(diff) <= max(2, got.size // 10_000)
    else:
        # 1e-11: inverting the Crystal Ball's power-law tail maps a value
        # through exp(G) (pow at n != 1), which multiplies the last-bit
        # differences of the two sides' exp / log by |G| (3e-12 seen)
        rel = np.abs(got - want) / np.maximum(np.abs(want), 1e-300)
        assert rel.max() <= 1e-11, (rel.max(), int(rel.argmax()))


@pytest.mark.parametrize("col", ["f64", "f32"])
@pytest.mark.parametrize("kind,params,lo,hi,fixed", CASES)
def test_leaf_values_match_oracle(rf, kind, params, lo, hi, fixed, col):
    n = 50_000
    spec = single(kind, params, lo, hi, fixed)
    G = rf.Graph(spec, col, "fp64" if col == "f64" else "fp32")
    pm = torch.tensor([params], dtype=torch.float64, device=DEV)
    cc = torch.tensor([[n]], dtype=torch.int64, device=DEV)
    off = torch.tensor([0, n], dtype=torch.int64, device=DEV)
    got = G.generate_toys(pm, cc, off, seed=12875).cpu().numpy()
    assert G.status() == 0
    want, ex, rc = oracle.generate(spec, [params], [[n]], [0, n], seed=12875,
                                   col_f32=(col == "f32"))
    assert rc == 0 and ex == 0
    compare(got, want, col == "f32")


def toy_counts(rng, toys, nu):
    return rng.poisson(nu, size=(toys, len(nu))).astype(np.int64)


def test_extended_model_many_toys(rf):
    """Two components in order within each toy, some toys empty or one-sided,
    a parameter row per toy, the columns larger than the toys need."""
    spec = datagen.gauss_exp_ext_spec()
    rng = np.random.default_rng(5)
    toys = 300
    counts = toy_counts(rng, toys, [40.0, 120.0])
    counts[3] = 0
    counts[4, 0] = 0
    counts[5, 1] = 0
    off = np.concatenate([[0], np.cumsum(counts.sum(1))]).astype(np.int64)
    pm = np.tile(np.array(spec["params"], np.float64), (toys, 1))
    pm[:, 0] += rng.uniform(-0.2, 0.2, toys)
    pm[:, 1] *= rng.uniform(0.8, 1.2, toys)
    pm[:, 2] *= rng.uniform(0.5, 1.5, toys)
    G = rf.Graph(spec, "f64", "fp64")
    n_cap = int(off[-1]) + 17
    got = G.generate_toys(torch.from_numpy(pm).to(DEV), torch.from_numpy(counts).to(DEV),
                          torch.from_numpy(off).to(DEV), seed=99, n_events=n_cap)
    assert G.status() == 0
    want, ex, rc = oracle.generate(spec, pm, counts, off, seed=99, col_f32=False)
    assert rc == 0 and ex == 0
    compare(got.cpu().numpy()[:, :off[-1]], want, False)


def test_argus_p_other_than_one_half_is_not_sampled(rf):
    spec = single("argus", [5.29, -20.0, 0.8], 5.20, 5.29, [True, False, False])
    G = rf.Graph(spec, "f64", "fp64")
    pm = torch.tensor([[5.29, -20.0, 0.8]], dtype=torch.float64, device=DEV)
    ev = G.generate_toys(pm, torch.tensor([[10]], dtype=torch.int64, device=DEV),
                         torch.tensor([0, 10], dtype=torch.int64, device=DEV), seed=3)
    assert G.status() & rf.STATUS_PARAM_DOMAIN
    assert torch.isnan(ev).all()
    assert oracle.generate(spec, [[5.29, -20.0, 0.8]], [[10]], [0, 10], seed=3,
                           col_f32=False)[2] == oracle.EUNSUPPORTED


def test_counts_that_do_not_fill_a_toy(rf):
    spec = datagen.gauss_exp_ext_spec()
    G = rf.Graph(spec, "f64", "fp64")
    counts = torch.tensor([[3, 4], [2, 2]], dtype=torch.int64, device=DEV)
    off = torch.tensor([0, 7, 12], dtype=torch.int64, device=DEV)   # toy 1 owns 5, counts 4
    pm = torch.tensor([spec["params"]] * 2, dtype=torch.float64, device=DEV)
    ev = G.generate_toys(pm, counts, off, seed=1).cpu().numpy()
    assert G.status() & 2
    assert np.all(np.isfinite(ev[0, :11])) and np.isnan(ev[0, 11])


def test_generated_toys_evaluate_and_fit_on_the_device(rf):
    """The toy loop on the GPU: 512 extended Gauss+Exp toys drawn on the
    device at Poisson counts, bound, evaluated in FP32 (against the oracle on
    the oracle's own draw of the same toys) and fitted by Adam."""
    spec = datagen.gauss_exp_ext_spec()
    rng = np.random.default_rng(12875004)
    toys = 512
    nu = np.stack([rng.uniform(200, 2000, toys), rng.uniform(500, 5000, toys)], 1)
    counts = rng.poisson(nu).astype(np.int64)
    off = np.concatenate([[0], np.cumsum(counts.sum(1))]).astype(np.int64)
    pm = np.tile(np.array(spec["params"], np.float64), (toys, 1))
    pm[:, 3:] = counts
    G = rf.Graph(spec, "f64", "fp32")
    ev = G.generate_toys(torch.from_numpy(pm).to(DEV), torch.from_numpy(counts).to(DEV),
                         torch.from_numpy(off).to(DEV), seed=4242)
    G.bind_events(ev, toys)
    start = pm.copy()
    start[:, 0] += 0.05
    offd = torch.from_numpy(off).to(DEV)
    got = G.nll_batched(offd, torch.from_numpy(start).to(DEV)).cpu().numpy()
    cols, ex, rc = oracle.generate(spec, pm, counts, off, seed=4242, col_f32=False)
    assert rc == 0 and ex == 0
    want, rc = oracle.nll_batched(spec, cols, off, start)
    rel = np.abs(got[:, 0] - want[:, 0]) / np.abs(want[:, 0])
    assert rel.max() <= TOL["fp32"]["nll"]
    pmd = torch.from_numpy(start.copy()).to(DEV)
    scale = torch.from_numpy(np.maximum(np.abs(start), 1.0)).to(DEV)
    G.fit_toys(offd, pmd, scale, 50, 1e-2)
    after = G.nll_batched(offd, pmd).cpu().numpy()[:, 0]
    assert after.sum() < got[:, 0].sum()
    assert np.mean(after < got[:, 0]) > 0.9
