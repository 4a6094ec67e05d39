"""Seeded synthetic inputs for the unbinned-NLL path.

This module only draws events and writes down the five workload models as plain
data.  It holds none of the likelihood arithmetic: no normalisation integral, no
log-likelihood, no gradient.  Both the FP64 oracle and the CUDA path take their
inputs from here and from nowhere else.

Random numbers come from numpy's Philox4x32-10 counter-based generator (Salmon
et al., SC'11).  A large sample is drawn in fixed chunks of ``CHUNK`` events,
chunk ``c`` of seed ``s`` from ``Philox(SeedSequence([s, c]))``, so the data do
not depend on how the work is split.

The paper's own workloads (Fig. 1: "datasets of 100 000 to 300 000 events for
various likelihood models") are not available; these five models stand in for
them.  Sampling methods (the paper's Sec. 3 "Generating Samples" contrasts
accept/reject with dedicated generators; both are used here):
  Gaussian      normal draws, truncated to the range by rejection
  Exponential   inverse CDF of the truncated exponential
  Chebychev     accept/reject against the bound 1 + sum |c_j|
  Crystal Ball  accept/reject of uniform proposals (peak height 1)
  ARGUS (p=1/2) tau ~ Gamma(3/2, rate -c) = (Exp(1) + Z^2/2)/(-c), truncated
                to the range by rejection, m = m0 sqrt(1 - tau)
FP32 columns hold the FP32 rounding of each draw; a draw whose FP32 value
leaves the observable range is rejected and redrawn.
"""
from __future__ import annotations

import math

import numpy as np

CHUNK = 1 << 20
SEEDS = {"c1": 12875001, "c2": 12875002, "c3": 12875003, "c4": 12875004,
         "c5": 12875005, "johnson": 12875006, "prod6": 12875007, "hypatia2": 12875008}


def rng(seed: int, chunk: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(np.random.SeedSequence([seed, chunk])))


# ----------------------------------------------------------------- samplers

def _fill(r, n, draw, dtype, lo, hi):
    """Collect n draws from ``draw(r, k)`` that lie in [lo, hi] after rounding
    to ``dtype``."""
    out = np.empty(n, dtype)
    got = 0
    while got < n:
        need = n - got
        x = draw(r, int(need * 1.25) + 64).astype(dtype)
        x = x[(x >= lo) & (x <= hi)]
        k = min(len(x), need)
        out[got:got + k] = x[:k]
        got += k
    return out


def gauss(r, n, mu, sigma, lo, hi, dtype=np.float64):
    return _fill(r, n, lambda r, k: r.normal(mu, sigma, k), dtype, lo, hi)


def expo(r, n, lam, lo, hi, dtype=np.float64):
    L = hi - lo
    if lam == 0.0:
        return _fill(r, n, lambda r, k: lo + L * r.random(k), dtype, lo, hi)
    span = math.expm1(lam * L)
    return _fill(r, n, lambda r, k: lo + np.log1p(r.random(k) * span) / lam, dtype, lo, hi)


def cheb(r, n, coefs, lo, hi, dtype=np.float64):
    bound = 1.0 + float(np.sum(np.abs(coefs)))

    def draw(r, k):
        x = lo + (hi - lo) * r.random(k)
        u = (2.0 * x - lo - hi) / (hi - lo)
        t_prev, t_cur, shape = np.ones_like(u), u, np.ones_like(u)
        for j, c in enumerate(coefs, start=1):
            if j > 1:
                t_prev, t_cur = t_cur, 2.0 * u * t_cur - t_prev
            shape = shape + c * t_cur
        return x[r.random(k) * bound < shape]
    return _fill(r, n, draw, dtype, lo, hi)


def crystal_ball(r, n, m0, sigma, alpha, nexp, lo, hi, dtype=np.float64):
    a = abs(alpha)
    sgn = 1.0 if alpha >= 0 else -1.0
    big_a = (nexp / a) ** nexp * math.exp(-0.5 * a * a)
    big_b = nexp / a - a

    def draw(r, k):
        x = lo + (hi - lo) * r.random(k)
        t = sgn * (x - m0) / sigma
        in_core = t > -a
        core = np.exp(-0.5 * t * t)
        tail = big_a * np.power(np.where(in_core, big_b + a, big_b - t), -nexp)
        shape = np.where(in_core, core, tail)
        return x[r.random(k) < shape]
    return _fill(r, n, draw, dtype, lo, hi)


def argus_half(r, n, m0, c, lo, hi, dtype=np.float64):
    """ARGUS with p = 1/2 through its Gamma(3/2) form in tau."""
    k_rate = -c
    if not k_rate > 0:
        raise ValueError("argus_half needs c < 0")
    tau_max = 1.0 - (lo / m0) ** 2

    def draw(r, k):
        tau = (r.standard_exponential(k) + 0.5 * r.standard_normal(k) ** 2) / k_rate
        tau = tau[(tau > 0.0) & (tau <= tau_max)]
        m = m0 * np.sqrt(1.0 - tau)
        return m[m < m0]
    out = _fill(r, n, draw, dtype, lo, hi)
    if np.any(out.astype(np.float64) >= m0):  # the open support, after rounding
        raise AssertionError("ARGUS draw at or above the endpoint")
    return out


def johnson_su(r, n, mu, lam, gamma, delta, lo, hi, dtype=np.float64):
    """Johnson SU by its defining transform: gamma + delta asinh((x-mu)/lam)
    is a standard normal, so x = mu + lam sinh((z - gamma)/delta)."""
    return _fill(r, n, lambda r, k: mu + lam * np.sinh((r.standard_normal(k) - gamma) / delta),
                 dtype, lo, hi)


# ----------------------------------------------------------------- workloads
# Each workload returns {"spec", "cols" [n_obs, n], "dtype", "params",
# "fixed", "name"}.  spec["params"] holds the evaluation point.

def _gauss_spec(mu, sigma, lo, hi):
    return {"obs": [(lo, hi)], "params": [mu, sigma], "fixed": [False, False],
            "nodes": [{"type": "gauss", "obs": 0, "params": [0, 1]}], "root": 0}


def c1(n=10_000, seed=SEEDS["c1"]):
    """Single Gaussian on [-10, 10]; events from N(0.3, 1.2); NLL at (0.25, 1.1)."""
    x = _chunked(n, seed, lambda r, k: gauss(r, k, 0.3, 1.2, -10.0, 10.0))
    return {"name": "gauss_1e4_f64", "spec": _gauss_spec(0.25, 1.1, -10.0, 10.0),
            "cols": x.reshape(1, -1), "dtype": "f64"}


def gauss_exp_spec(mu=5.0, sigma=0.5, lam=-0.3, frac=0.2, lo=0.0, hi=10.0):
    return {"obs": [(lo, hi)], "params": [mu, sigma, lam, frac],
            "fixed": [False] * 4,
            "nodes": [{"type": "gauss", "obs": 0, "params": [0, 1]},
                      {"type": "exp", "obs": 0, "params": [2]},
                      {"type": "add_frac", "children": [0, 1], "params": [3]}],
            "root": 2}


def c2(n=1_000_000, seed=SEEDS["c2"]):
    """Gauss(5, 0.5) + Exp(-0.3) on [0, 10], fraction 0.2 on the Gaussian."""
    def draw(r, k):
        sig = r.random(k) < 0.2
        ns = int(sig.sum())
        out = np.empty(k)
        out[sig] = gauss(r, ns, 5.0, 0.5, 0.0, 10.0)
        out[~sig] = expo(r, k - ns, -0.3, 0.0, 10.0)
        return out
    x = _chunked(n, seed, draw)
    return {"name": "gauss_exp_frac_1e6_f64", "spec": gauss_exp_spec(),
            "cols": x.reshape(1, -1), "dtype": "f64"}


CHEB4 = (0.2, -0.1, 0.05, 0.02)


def prod3_spec(nu, extended=True):
    nodes = [{"type": "gauss", "obs": 0, "params": [0, 1]},
             {"type": "exp", "obs": 1, "params": [2]},
             {"type": "cheb", "obs": 2, "params": [3, 4, 5, 6]},
             {"type": "prod", "children": [0, 1, 2]}]
    params = [0.0, 1.5, -0.5, *CHEB4]
    if extended:
        nodes.append({"type": "add_ext", "children": [3], "params": [7]})
        params.append(float(nu))
    return {"obs": [(-8.0, 8.0), (0.0, 10.0), (-1.0, 1.0)], "params": params,
            "fixed": [False] * len(params), "nodes": nodes, "root": len(nodes) - 1}


def c3(n=10_000_000, seed=SEEDS["c3"], extended=True):
    """Gauss(x;0,1.5) x Exp(y;-0.5) x Cheb4(z) with FP32 columns; extended by a
    yield nu (evaluated at nu = n) so that the model has 8 parameters."""
    def draw(r, k):
        return np.stack([gauss(r, k, 0.0, 1.5, -8.0, 8.0, np.float32),
                         expo(r, k, -0.5, 0.0, 10.0, np.float32),
                         cheb(r, k, CHEB4, -1.0, 1.0, np.float32)])
    cols = _chunked(n, seed, draw, ncols=3, dtype=np.float32)
    return {"name": "prod3_1e7_f32", "spec": prod3_spec(n, extended), "cols": cols,
            "dtype": "f32"}


def gauss_exp_ext_spec(mu=5.0, sigma=0.5, lam=-0.3, nu_s=1000.0, nu_b=1000.0):
    return {"obs": [(0.0, 10.0)], "params": [mu, sigma, lam, nu_s, nu_b],
            "fixed": [False] * 5,
            "nodes": [{"type": "gauss", "obs": 0, "params": [0, 1]},
                      {"type": "exp", "obs": 0, "params": [2]},
                      {"type": "add_ext", "children": [0, 1], "params": [3, 4]}],
            "root": 2}


def c4(toys=4096, seed=SEEDS["c4"], nu_s_range=(500.0, 5e4), nu_b_range=(1e3, 1e5)):
    """Toy study: per toy nu_s, nu_b log-uniform, counts Poisson, events from
    Gauss(5, 0.5) + Exp(-0.3) on [0, 10], shuffled within the toy, FP64,
    concatenated by toy.  Start point (per toy): generating shape with mu+0.05,
    yields = the observed counts."""
    r = rng(seed, 0)
    ls, lb = np.log(nu_s_range), np.log(nu_b_range)
    nu_s = np.exp(r.uniform(ls[0], ls[1], toys))
    nu_b = np.exp(r.uniform(lb[0], lb[1], toys))
    n_s = r.poisson(nu_s)
    n_b = r.poisson(nu_b)
    counts = n_s + n_b
    offsets = np.zeros(toys + 1, np.int64)
    np.cumsum(counts, out=offsets[1:])
    x = np.empty(int(offsets[-1]))
    for t in range(toys):
        rt = rng(seed, 1 + t)
        ev = np.concatenate([gauss(rt, int(n_s[t]), 5.0, 0.5, 0.0, 10.0),
                             expo(rt, int(n_b[t]), -0.3, 0.0, 10.0)])
        rt.shuffle(ev)
        x[offsets[t]:offsets[t + 1]] = ev
    start = np.empty((toys, 5))
    start[:, 0] = 5.05
    start[:, 1] = 0.5
    start[:, 2] = -0.3
    start[:, 3] = n_s
    start[:, 4] = n_b
    return {"name": f"toys{toys}_gauss_exp_ext_f64", "spec": gauss_exp_ext_spec(),
            "cols": x.reshape(1, -1), "dtype": "f64", "offsets": offsets,
            "params_matrix": start, "nu_true": np.stack([nu_s, nu_b], 1)}


def cb_argus_spec(nu_s=1e6, nu_b=1e8):
    # params: 0 m0_cb, 1 sigma, 2 alpha, 3 n, 4 m0_argus, 5 c, 6 p, 7 nu_s, 8 nu_b
    return {"obs": [(5.20, 5.29)],
            "params": [5.279, 0.003, 1.5, 3.0, 5.29, -20.0, 0.5, float(nu_s), float(nu_b)],
            "fixed": [False, False, False, False, True, False, True, False, False],
            "nodes": [{"type": "cb", "obs": 0, "params": [0, 1, 2, 3]},
                      {"type": "argus", "obs": 0, "params": [4, 5, 6]},
                      {"type": "add_ext", "children": [0, 1], "params": [7, 8]}],
            "root": 2}


def c5(n_sig=1_000_000, n_bkg=100_000_000, seed=SEEDS["c5"]):
    """Crystal Ball (5.279, 0.003, 1.5, 3) + ARGUS (5.29, -20, 1/2) on
    [5.20, 5.29], FP32 column, exactly n_sig + n_bkg events in a uniformly
    random order (per-chunk hypergeometric split, then a shuffle)."""
    n = n_sig + n_bkg
    nchunks = (n + CHUNK - 1) // CHUNK
    r0 = rng(seed, 0)
    left = np.array([n_sig, n_bkg], np.int64)
    out = np.empty(n, np.float32)
    for c in range(nchunks):
        k = min(CHUNK, n - c * CHUNK)
        split = r0.multivariate_hypergeometric(left, k) if left.sum() > k else left.copy()
        left -= split
        r = rng(seed, 1 + c)
        ev = np.concatenate([
            crystal_ball(r, int(split[0]), 5.279, 0.003, 1.5, 3.0, 5.20, 5.29, np.float32),
            argus_half(r, int(split[1]), 5.29, -20.0, 5.20, 5.29, np.float32)])
        r.shuffle(ev)
        out[c * CHUNK:c * CHUNK + k] = ev
    return {"name": "cb_argus_ext_1.01e8_f32", "spec": cb_argus_spec(n_sig, n_bkg),
            "cols": out.reshape(1, -1), "dtype": "f32"}


def johnson_exp_spec(nu_s=2e4, nu_b=8e4):
    # params: 0 mu, 1 lambda, 2 gamma, 3 delta, 4 exp slope, 5 nu_s, 6 nu_b
    return {"obs": [(0.0, 10.0)],
            "params": [4.0, 0.8, -0.5, 1.6, -0.2, float(nu_s), float(nu_b)],
            "fixed": [False] * 7,
            "nodes": [{"type": "johnson", "obs": 0, "params": [0, 1, 2, 3]},
                      {"type": "exp", "obs": 0, "params": [4]},
                      {"type": "add_ext", "children": [0, 1], "params": [5, 6]}],
            "root": 2}


def johnson_exp(n_sig=20_000, n_bkg=80_000, seed=SEEDS["johnson"]):
    """Extended Johnson SU (4.0, 0.8, -0.5, 1.6) + Exp(-0.2) on [0, 10], FP32
    column, the two blocks shuffled together."""
    r = rng(seed, 0)
    ev = np.concatenate([johnson_su(r, n_sig, 4.0, 0.8, -0.5, 1.6, 0.0, 10.0, np.float32),
                         expo(r, n_bkg, -0.2, 0.0, 10.0, np.float32)])
    r.shuffle(ev)
    return {"name": "johnson_exp_ext_f32", "spec": johnson_exp_spec(n_sig, n_bkg),
            "cols": ev.reshape(1, -1), "dtype": "f32"}


def prod6_spec(f1=0.3, f2=0.3):
    """Six leaves in three two-observable components (x on [0, 10], y on
    [-1, 1]): Gauss(x) Exp(y) + CB(x) Cheb2(y) + Exp(x) Gauss(y), fractions
    f1, f2 on the first two."""
    # params: 0 mu1, 1 sigma1, 2 lambda1 (y), 3 m0, 4 sigma2, 5 alpha, 6 n,
    #         7 c1, 8 c2 (y), 9 lambda3 (x), 10 mu3 (y), 11 sigma3, 12 f1, 13 f2
    return {"obs": [(0.0, 10.0), (-1.0, 1.0)],
            "params": [5.0, 0.6, -1.2, 3.0, 0.4, 1.2, 2.5, 0.3, -0.2, -0.25, 0.2, 0.3,
                       float(f1), float(f2)],
            "fixed": [False] * 14,
            "nodes": [{"type": "gauss", "obs": 0, "params": [0, 1]},
                      {"type": "exp", "obs": 1, "params": [2]},
                      {"type": "prod", "children": [0, 1]},
                      {"type": "cb", "obs": 0, "params": [3, 4, 5, 6]},
                      {"type": "cheb", "obs": 1, "params": [7, 8]},
                      {"type": "prod", "children": [3, 4]},
                      {"type": "exp", "obs": 0, "params": [9]},
                      {"type": "gauss", "obs": 1, "params": [10, 11]},
                      {"type": "prod", "children": [6, 7]},
                      {"type": "add_frac", "children": [2, 5, 8], "params": [12, 13]}],
            "root": 9}


def prod6(n=60_000, seed=SEEDS["prod6"], dtype=np.float32):
    """Events of prod6_spec(): per component its (x, y) pairs drawn from its
    two leaves, 30% / 30% / 40%, shuffled; two columns."""
    r = rng(seed, 0)
    k = r.multinomial(n, [0.3, 0.3, 0.4])
    x = np.concatenate([gauss(r, int(k[0]), 5.0, 0.6, 0.0, 10.0, dtype),
                        crystal_ball(r, int(k[1]), 3.0, 0.4, 1.2, 2.5, 0.0, 10.0, dtype),
                        expo(r, int(k[2]), -0.25, 0.0, 10.0, dtype)])
    y = np.concatenate([expo(r, int(k[0]), -1.2, -1.0, 1.0, dtype),
                        cheb(r, int(k[1]), [0.3, -0.2], -1.0, 1.0, dtype),
                        gauss(r, int(k[2]), 0.2, 0.3, -1.0, 1.0, dtype)])
    perm = r.permutation(n)
    cols = np.stack([x[perm], y[perm]])
    return {"name": "prod6_frac_f32", "spec": prod6_spec(), "cols": np.ascontiguousarray(cols),
            "dtype": "f32" if dtype == np.float32 else "f64"}


def hypatia2_exp_spec(nu_s=2e4, nu_b=3e4):
    """Extended Hypatia2 (lambda, zeta, beta, sigma, mu, a, n, a2, n2) +
    Exponential on [0, 10]."""
    return {"obs": [(0.0, 10.0)],
            "params": [-1.5, 1.2, 0.1, 0.5, 5.0, 2.0, 3.0, 2.5, 4.0, -0.2,
                       float(nu_s), float(nu_b)],
            "fixed": [False] * 12,
            "nodes": [{"type": "hypatia2", "obs": 0, "params": list(range(9))},
                      {"type": "exp", "obs": 0, "params": [9]},
                      {"type": "add_ext", "children": [0, 1], "params": [10, 11]}],
            "root": 2}


def hypatia2_exp(n_sig=20_000, n_bkg=30_000, seed=SEEDS["hypatia2"], dtype=np.float32):
    """Signal from the generalised hyperbolic density that is Hypatia2's core
    (scipy's sampler; the tails are not imposed), kept inside [0, 10], plus
    Exp(-0.2) background, shuffled."""
    import scipy.special as sps
    import scipy.stats as sst
    lam, zeta, beta, sigma, mu = -1.5, 1.2, 0.1, 0.5, 5.0
    delta = sigma * np.sqrt(zeta * sps.kv(lam, zeta) / sps.kv(lam + 1, zeta))
    d = sst.genhyperbolic(lam, zeta, beta * delta, loc=mu, scale=delta)
    r = rng(seed, 0)
    sig = _fill(r, n_sig, lambda r, k: d.rvs(size=k, random_state=r), dtype, 0.0, 10.0)
    ev = np.concatenate([sig, expo(r, n_bkg, -0.2, 0.0, 10.0, dtype)])
    r.shuffle(ev)
    return {"name": "hypatia2_exp_ext", "spec": hypatia2_exp_spec(n_sig, n_bkg),
            "cols": ev.reshape(1, -1), "dtype": "f32" if dtype == np.float32 else "f64"}


def _chunked(n, seed, draw, ncols=1, dtype=np.float64):
    out = np.empty((ncols, n), dtype) if ncols > 1 else np.empty(n, dtype)
    for c in range((n + CHUNK - 1) // CHUNK):
        k = min(CHUNK, n - c * CHUNK)
        block = draw(rng(seed, c), k)
        if ncols > 1:
            out[:, c * CHUNK:c * CHUNK + k] = block
        else:
            out[c * CHUNK:c * CHUNK + k] = block
    return out


WORKLOADS = {"c1": c1, "c2": c2, "c3": c3, "c4": c4, "c5": c5}
