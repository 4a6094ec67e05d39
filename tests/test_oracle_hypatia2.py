"""Pins of the oracle's Hypatia2 leaf and its Bessel function K_nu.

The oracle computes K_nu(z) by adaptive quadrature of its integral
representation and the Hypatia2 log-density with forward-mode derivatives.
Here they are tied to independent sources: scipy.special's Bessel functions,
scipy.stats' generalised hyperbolic distribution (the core, with the tails
moved off the range), the continuity of value and slope where the tails take
over, mpmath quadrature of the density (its normalisation), and Richardson
differences of the log-density and of the normalisation (its derivatives).
"""
import math

import mpmath as mp
import numpy as np
import pytest
import scipy.special as sp
import scipy.stats as st

import oracle

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")

NU_Z = [(0.0, 1.0), (0.5, 0.3), (-2.5, 0.3), (1.7, 12.0), (-0.3, 0.05), (4.2, 80.0),
        (-4.5, 2.0), (3.3, 0.01), (0.9, 400.0)]


def richardson(f, x, h):
    d1 = (f(x + h) - f(x - h)) / (2 * h)
    d2 = (f(x + h / 2) - f(x - h / 2)) / h
    return (4 * d2 - d1) / 3


@pytest.mark.parametrize("nu,z", NU_Z)
def test_besselk_against_scipy(nu, z):
    K, dz, dn, rc = oracle.besselk(nu, z)
    assert rc == 0
    assert abs(K / sp.kv(nu, z) - 1) <= 1e-13
    assert abs(dz / sp.kvp(nu, z) - 1) <= 1e-12
    want = richardson(lambda v: sp.kv(v, z), nu, 1e-3)
    assert abs(dn - want) <= 1e-9 * abs(K) + 1e-9 * abs(want)


TH = [-1.5, 1.2, 0.1, 0.5, 5.0, 2.0, 3.0, 2.5, 4.0]   # lambda zeta beta sigma mu a n a2 n2
LO, HI = 0.0, 10.0


def delta_alpha(lam, zeta, sigma):
    phi = sp.kv(lam + 1, zeta) / sp.kv(lam, zeta)
    return sigma * math.sqrt(zeta / phi), math.sqrt(zeta * phi) / sigma


def logf(th, x):
    v, d, rc = oracle.leaf_logf("hypatia2", th, LO, HI, x)
    assert rc == 0
    return v, d


@pytest.mark.parametrize("th", [TH, [0.8, 2.5, -0.3, 0.7, 4.6, 2.0, 3.0, 2.5, 4.0],
                                [-3.0, 0.4, 0.0, 1.1, 5.2, 2.0, 3.0, 2.5, 4.0]])
def test_core_is_the_generalised_hyperbolic_density(th):
    """Tails moved off the range: log f(x) - log f(x0) equals scipy's
    genhyperbolic log-density difference (p = lambda, a = zeta, b = beta delta,
    loc = mu, scale = delta)."""
    core = list(th)
    core[5] = core[7] = 50.0
    lam, zeta, beta, sigma, mu = th[:5]
    delta, alpha = delta_alpha(lam, zeta, sigma)
    d = st.genhyperbolic(lam, zeta, beta * delta, loc=mu, scale=delta)
    xs = np.linspace(LO + 0.3, HI - 0.3, 17)
    want = d.logpdf(xs) - d.logpdf(xs[8])
    got = np.array([logf(core, x)[0] for x in xs]) - logf(core, xs[8])[0]
    np.testing.assert_allclose(got, want, rtol=0, atol=2e-11)


def test_tails_continue_value_and_slope():
    mu, sigma, a, a2 = TH[4], TH[3], TH[5], TH[7]
    for xj in (mu - a * sigma, mu + a2 * sigma):
        # the jump across the junction, after the slope's share is removed
        eps = 1e-6
        v0, d0 = logf(TH, xj - eps)[0], logf(TH, xj + eps)[0]
        slope = (logf(TH, xj + 3 * eps)[0] - logf(TH, xj - 3 * eps)[0]) / (6 * eps)
        assert abs((d0 - v0) - 2 * eps * slope) <= 1e-9
        h = 1e-4
        left = (logf(TH, xj - h)[0] - logf(TH, xj - 2 * h)[0]) / h
        right = (logf(TH, xj + 2 * h)[0] - logf(TH, xj + h)[0]) / h
        # one-sided slopes h and 2h from the junction: equal up to O(h) curvature
        assert abs(left - right) <= 5e-3 * max(1.0, abs(left))


def test_normalisation_against_mpmath():
    I, dI, rc = oracle.leaf_norm("hypatia2", TH, LO, HI)
    assert rc == 0
    mp.mp.dps = 20
    cuts = [LO, TH[4] - TH[5] * TH[3], TH[4] + TH[7] * TH[3], HI]
    want = float(mp.quad(lambda x: mp.e ** logf(TH, float(x))[0], cuts))
    assert abs(I / want - 1) <= 1e-12


def test_log_density_derivatives_against_richardson():
    for x in (1.2, 3.9, 4.6, 5.3, 6.1, 7.9):   # left tail, core, right tail
        _, d = logf(TH, x)
        for j in range(9):
            def f(v, j=j):
                t = list(TH)
                t[j] = v
                return logf(t, x)[0]
            h = 1e-4 * max(abs(TH[j]), 0.1)
            want = richardson(f, TH[j], h)
            assert abs(d[j] - want) <= 1e-8 * max(1.0, abs(want)), (x, j, d[j], want)


@pytest.mark.slow
@pytest.mark.parametrize("j", [3, 6])
def test_normalisation_derivatives_against_richardson(j):
    I, dI, rc = oracle.leaf_norm("hypatia2", TH, LO, HI)
    assert rc == 0

    def f(v):
        t = list(TH)
        t[j] = v
        return oracle.leaf_norm("hypatia2", t, LO, HI)[0]
    want = richardson(f, TH[j], 1e-3 * abs(TH[j]))
    assert abs(dI[j] - want) <= 1e-7 * abs(I)
