"""Pin of the oracle's L1 gradient scale (the denominator of every gradient
parity assertion).

orc_nll_scaled returns, beside the NLL and its gradient, for every parameter
k the scale sum_i |d(-log P_i)/d theta_k| (+1 for a yield, whose extended term
sum(nu) adds 1 to the derivative).  Here that sum is rebuilt without the
oracle: each event's log P_i comes from library densities (scipy.stats
truncated by their CDFs, the same references that pin the oracle's leaves),
its derivative by a Richardson-extrapolated central difference in theta_k,
and the absolute values are summed in numpy.  A slip in the oracle's scale --
a missing absolute value, a dropped 1/P, a derivative taken in the wrong
parameter -- moves it far outside the 1e-10 bound.

Events within 0.05 (in units of the width) of the Crystal Ball's core/tail
junction are left out: log f is only once differentiable there, and a
difference step that straddles the junction loses the O(h^4) accuracy of the
extrapolation.
"""
import math

import numpy as np
import pytest
import scipy.stats as st

import datagen
import oracle

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def trunc_logpdf(kind, th, lo, hi, x):
    """log of the density normalised on [lo, hi], from scipy.stats."""
    if kind == "gauss":
        mu, s = th
        return st.truncnorm((lo - mu) / s, (hi - mu) / s, loc=mu, scale=s).logpdf(x)
    if kind == "exp":
        (lam,) = th
        assert lam < 0
        return st.truncexpon((hi - lo) * -lam, loc=lo, scale=1 / -lam).logpdf(x)
    if kind == "cb":
        m0, s, a, n = th
        assert a > 0
        d = st.crystalball(a, n, loc=m0, scale=s)
        return d.logpdf(x) - np.log(d.cdf(hi) - d.cdf(lo))
    if kind == "argus":
        m0, c, p = th
        assert p == 0.5 and c < 0
        d = st.argus(math.sqrt(-2 * c), loc=0.0, scale=m0)
        return d.logpdf(x) - np.log(d.cdf(min(hi, m0)) - d.cdf(lo))
    raise KeyError(kind)


def event_logp(spec, theta, x):
    """log P_i of a one-observable model whose root is a leaf or an Add of
    two leaves (fraction or extended yields), vectorised over the events."""
    lo, hi = spec["obs"][0]
    nodes, root = spec["nodes"], spec["nodes"][spec["root"]]

    def leaf(i):
        nd = nodes[i]
        return trunc_logpdf(nd["type"], [theta[p] for p in nd["params"]], lo, hi, x)

    if root["type"] not in ("add_frac", "add_ext"):
        return leaf(spec["root"])
    a, b = root["children"]
    la, lb = leaf(a), leaf(b)
    if root["type"] == "add_frac":
        f = theta[root["params"][0]]
        ca, cb = f, 1.0 - f
    else:
        ca, cb = theta[root["params"][0]], theta[root["params"][1]]
    m = np.maximum(la, lb)
    return m + np.log(ca * np.exp(la - m) + cb * np.exp(lb - m))


def independent_scale(spec, theta, x, steps):
    """sum_i |d(-log P_i)/d theta_k| by per-event Richardson differences."""
    theta = np.asarray(theta, np.float64)
    out = np.zeros(len(theta))
    root = spec["nodes"][spec["root"]]
    yields = set(root["params"]) if root["type"] == "add_ext" else set()
    for k, h in enumerate(steps):
        if h is None:
            continue

        def f(v):
            t = theta.copy()
            t[k] = v
            return event_logp(spec, t, x)

        d1 = (f(theta[k] + h) - f(theta[k] - h)) / (2 * h)
        d2 = (f(theta[k] + h / 2) - f(theta[k] - h / 2)) / h
        d = (4 * d2 - d1) / 3
        out[k] = np.sum(np.abs(d)) + (1.0 if k in yields else 0.0)
    return out


def oracle_scale(spec, theta, x):
    _, _, sc, rc = oracle.nll_scaled(spec, theta, x.reshape(1, -1), nthreads=1)
    assert rc == 0
    return sc


def check(spec, theta, x, steps):
    got = oracle_scale(spec, theta, x)
    want = independent_scale(spec, theta, x, steps)
    for k, h in enumerate(steps):
        if h is None:
            continue
        assert want[k] > 0
        assert abs(got[k] - want[k]) <= 1e-10 * want[k], (k, got[k], want[k])


def test_scale_single_gaussian():
    w = datagen.c1(n=400)
    x = w["cols"][0].astype(np.float64)
    theta = [0.31, 1.17]
    check(w["spec"], theta, x, [1e-3 * 1.17, 1e-3 * 1.17])


def test_scale_gauss_exp_fraction():
    w = datagen.c2(n=400)
    x = w["cols"][0].astype(np.float64)
    theta = [5.05, 0.55, -0.27, 0.23]
    check(w["spec"], theta, x, [1e-3 * 0.55, 1e-3 * 0.55, 1e-3 * 0.27, 1e-3])


def test_scale_gauss_exp_extended():
    spec = datagen.gauss_exp_ext_spec(nu_s=120.0, nu_b=280.0)
    w = datagen.c2(n=400)
    x = w["cols"][0].astype(np.float64)
    theta = [4.96, 0.47, -0.32, 131.0, 262.0]
    check(spec, theta, x, [1e-3 * 0.47, 1e-3 * 0.47, 1e-3 * 0.32, 1e-3 * 131.0, 1e-3 * 262.0])


def test_scale_crystal_ball_argus_extended():
    w = datagen.c5(60, 340)
    x = w["cols"][0].astype(np.float64)
    theta = [5.2793, 0.0032, 1.45, 3.2, 5.29, -19.0, 0.5, 65.0, 330.0]
    t = (x - theta[0]) / theta[1]
    x = x[np.abs(t + theta[2]) > 0.05]           # away from the core/tail junction
    assert x.size > 300
    sg = theta[1]
    # ARGUS m0 (the range edge) and p stay as given: neither has a library
    # density to difference against (p) or a smooth neighbourhood (m0 = hi)
    steps = [1e-3 * sg, 1e-3 * sg, 1e-3 * 1.45, 1e-3 * 3.2, None, 1e-3 * 19.0, None,
             1e-3 * 65.0, 1e-3 * 330.0]
    check(w["spec"], theta, x, steps)
