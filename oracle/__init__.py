"""FP64 CPU oracle for the unbinned NLL of a PDF graph -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline /
reference leg import this package.  The product library never does, and the
two share no code.  The arithmetic lives in ``rf_oracle.c`` (plain C, FP64);
this module compiles it with gcc and marshals arguments through ctypes.

A model is the plain-data ``spec`` dict used throughout the repository::

    {"obs": [(lo, hi), ...],          # observable ranges
     "params": [v0, v1, ...],         # parameter values
     "nodes": [{"type": "gauss", "obs": 0, "params": [0, 1]},
               {"type": "add_frac", "children": [0, 1], "params": [2]}, ...],
     "root": index}

Leaf parameter order: gauss (mu, sigma); exp (lambda); cheb (c_1..c_m);
cb (m0, sigma, alpha, n); argus (m0, c, p); johnson (mu, lambda, gamma,
delta); formula (p0 .. p(m-1) of the node's "formula" text in x); hypatia2
(lambda, zeta, beta, sigma, mu, a, n, a2, n2).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_SRC = os.path.join(_HERE, "rf_oracle.c")

TYPES = {"gauss": 1, "exp": 2, "cheb": 3, "cb": 4, "argus": 5, "johnson": 9,
         "formula": 10, "hypatia2": 11, "add_frac": 6, "add_ext": 7, "prod": 8}
MAXCH, MAXNP, MAXPAR = 8, 12, 64
OK, EINVAL, EUNSUPPORTED, EDOMAIN = 0, 1, 2, 3

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile rf_oracle.c into _build/liboracle.so (gcc, FP64, IEEE: no fast
    math, no FMA contraction so x86 and Arm hosts round identically)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= max(os.path.getmtime(_SRC),
                                             os.path.getmtime(os.path.join(_HERE, "rf_oracle.h")))):
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
           "-ffp-contract=off", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


class _Model(C.Structure):
    _fields_ = [("n_nodes", C.c_int32), ("root", C.c_int32),
                ("n_obs", C.c_int32), ("n_par", C.c_int32),
                ("type", C.c_void_p), ("obs", C.c_void_p),
                ("nchild", C.c_void_p), ("child", C.c_void_p),
                ("npar", C.c_void_p), ("par", C.c_void_p),
                ("obs_lo", C.c_void_p), ("obs_hi", C.c_void_p),
                ("expr", C.c_void_p)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_SO)
            dp = C.POINTER(C.c_double)
            L.orc_leaf_logf.argtypes = [C.c_int, dp, C.c_int, C.c_double, C.c_double,
                                        C.c_double, dp, dp]
            L.orc_leaf_norm.argtypes = [C.c_int, dp, C.c_int, C.c_double, C.c_double, dp, dp]
            L.orc_nll.argtypes = [C.POINTER(_Model), dp, dp, C.c_int64, C.c_int64, C.c_int,
                                  dp, dp]
            L.orc_nll_scaled.argtypes = [C.POINTER(_Model), dp, dp, C.c_int64, C.c_int64,
                                         C.c_int, dp, dp, dp]
            L.orc_logp.argtypes = [C.POINTER(_Model), dp, dp, C.c_int64, C.c_int64, dp]
            L.orc_nll_batched.argtypes = [C.POINTER(_Model), dp, C.c_int64,
                                          C.POINTER(C.c_int64), C.c_int32, dp, C.c_int, dp]
            L.orc_adam_step.argtypes = [C.c_int, dp, dp, dp, C.POINTER(C.c_uint8), dp, dp,
                                        C.c_int, C.c_double, C.c_double, C.c_double,
                                        C.c_double]
            L.orc_adam_step.restype = None
            u64p = C.POINTER(C.c_uint64)
            L.orc_philox4x64.argtypes = [u64p, u64p, u64p]
            L.orc_philox4x64.restype = None
            L.orc_erfcinv.argtypes = [C.c_double]
            L.orc_erfcinv.restype = C.c_double
            i64p = C.POINTER(C.c_int64)
            L.orc_generate.argtypes = [C.POINTER(_Model), dp, C.c_int32, i64p, i64p, C.c_uint64,
                                       C.c_int, dp, C.c_int64, i64p]
            L.orc_besselk.argtypes = [C.c_double, C.c_double, dp]
            L.orc_expr_check.argtypes = [C.c_char_p, C.c_int]
            L.orc_expr_logf.argtypes = [C.c_char_p, dp, C.c_int, C.c_double, dp, dp]
            L.orc_expr_norm.argtypes = [C.c_char_p, dp, C.c_int, C.c_double, C.c_double, dp,
                                        dp]
            _lib = L
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


class Model:
    """The oracle's flat-array form of a spec (keeps the arrays alive)."""

    def __init__(self, spec: dict):
        nodes = spec["nodes"]
        N = len(nodes)
        self.n_par = len(spec["params"])
        self.type = np.zeros(N, np.int32)
        self.obs = np.full(N, -1, np.int32)
        self.nchild = np.zeros(N, np.int32)
        self.child = np.full(N * MAXCH, -1, np.int32)
        self.npar = np.zeros(N, np.int32)
        self.par = np.full(N * MAXNP, -1, np.int32)
        for i, nd in enumerate(nodes):
            self.type[i] = TYPES[nd["type"]]
            self.obs[i] = nd.get("obs", -1)
            ch = nd.get("children", [])
            self.nchild[i] = len(ch)
            self.child[i * MAXCH:i * MAXCH + len(ch)] = ch
            ps = nd.get("params", [])
            self.npar[i] = len(ps)
            self.par[i * MAXNP:i * MAXNP + len(ps)] = ps
        self.texts = [nd.get("formula", "").encode() for nd in nodes]
        self.expr = (C.c_char_p * N)(*self.texts)
        rng = np.asarray(spec["obs"], np.float64).reshape(-1, 2)
        self.lo = np.ascontiguousarray(rng[:, 0])
        self.hi = np.ascontiguousarray(rng[:, 1])
        self.n_obs = rng.shape[0]
        self.s = _Model(N, spec.get("root", N - 1), self.n_obs, self.n_par,
                        self.type.ctypes.data, self.obs.ctypes.data,
                        self.nchild.ctypes.data, self.child.ctypes.data,
                        self.npar.ctypes.data, self.par.ctypes.data,
                        self.lo.ctypes.data, self.hi.ctypes.data,
                        C.cast(self.expr, C.c_void_p).value)


def _cols(cols) -> np.ndarray:
    c = np.ascontiguousarray(np.asarray(cols, dtype=np.float64))
    if c.ndim == 1:
        c = c.reshape(1, -1)
    return c


def nll(spec: dict, params, cols, nthreads: int = 0, grad: bool = True):
    """(NLL, gradient or None, return code).  cols: [n_obs, n] (widened to FP64
    exactly when given in FP32)."""
    m = Model(spec)
    c = _cols(cols)
    p = np.ascontiguousarray(np.asarray(params, np.float64))
    out = np.zeros(1)
    g = np.zeros(m.n_par) if grad else None
    rc = lib().orc_nll(C.byref(m.s), _dp(p), _dp(c), c.shape[1], c.shape[1], nthreads,
                       _dp(out), _dp(g) if grad else None)
    return float(out[0]), g, rc


def nll_scaled(spec: dict, params, cols, nthreads: int = 0):
    """(NLL, gradient, L1 gradient scale, return code)."""
    m = Model(spec)
    c = _cols(cols)
    p = np.ascontiguousarray(np.asarray(params, np.float64))
    out = np.zeros(1)
    g = np.zeros(m.n_par)
    sc = np.zeros(m.n_par)
    rc = lib().orc_nll_scaled(C.byref(m.s), _dp(p), _dp(c), c.shape[1], c.shape[1],
                              nthreads, _dp(out), _dp(g), _dp(sc))
    return float(out[0]), g, sc, rc


def logp(spec: dict, params, cols):
    m = Model(spec)
    c = _cols(cols)
    p = np.ascontiguousarray(np.asarray(params, np.float64))
    out = np.zeros(c.shape[1])
    rc = lib().orc_logp(C.byref(m.s), _dp(p), _dp(c), c.shape[1], c.shape[1], _dp(out))
    return out, rc


def leaf_logf(kind: str, theta, lo: float, hi: float, x: float):
    th = np.ascontiguousarray(np.asarray(theta, np.float64))
    lf = np.zeros(1)
    d = np.zeros(max(len(th), 1))
    rc = lib().orc_leaf_logf(TYPES[kind], _dp(th), len(th), lo, hi, x, _dp(lf), _dp(d))
    return float(lf[0]), d[:len(th)], rc


def leaf_norm(kind: str, theta, lo: float, hi: float):
    th = np.ascontiguousarray(np.asarray(theta, np.float64))
    I = np.zeros(1)
    d = np.zeros(max(len(th), 1))
    rc = lib().orc_leaf_norm(TYPES[kind], _dp(th), len(th), lo, hi, _dp(I), _dp(d))
    return float(I[0]), d[:len(th)], rc


def expr_check(text: str, npar: int) -> int:
    return lib().orc_expr_check(text.encode(), npar)


def expr_logf(text: str, theta, x: float):
    """(log f(x), d log f / dp_j, return code) of a formula leaf."""
    th = np.ascontiguousarray(np.asarray(theta, np.float64))
    lf = np.zeros(1)
    d = np.zeros(max(len(th), 1))
    rc = lib().orc_expr_logf(text.encode(), _dp(th) if len(th) else None, len(th), x,
                             _dp(lf), _dp(d))
    return float(lf[0]), d[:len(th)], rc


def expr_norm(text: str, theta, lo: float, hi: float):
    """(I, dI/dp_j, return code) of a formula leaf on [lo, hi]."""
    th = np.ascontiguousarray(np.asarray(theta, np.float64))
    I = np.zeros(1)
    d = np.zeros(max(len(th), 1))
    rc = lib().orc_expr_norm(text.encode(), _dp(th) if len(th) else None, len(th), lo, hi,
                             _dp(I), _dp(d))
    return float(I[0]), d[:len(th)], rc


def nll_batched(spec: dict, cols, offsets, params_matrix, nthreads: int = 0):
    """out[t] = (NLL_t, grad_t...) for toy t on events [offsets[t], offsets[t+1])."""
    m = Model(spec)
    c = _cols(cols)
    off = np.ascontiguousarray(np.asarray(offsets, np.int64))
    pm = np.ascontiguousarray(np.asarray(params_matrix, np.float64))
    toys = len(off) - 1
    out = np.zeros((toys, 1 + m.n_par))
    rc = lib().orc_nll_batched(C.byref(m.s), _dp(c), c.shape[1],
                               off.ctypes.data_as(C.POINTER(C.c_int64)), toys, _dp(pm),
                               nthreads, _dp(out))
    return out, rc


def adam_step(theta, grad, scale, free_mask, m1, m2, t, lr, beta1=0.9, beta2=0.999,
              eps=1e-8):
    """In-place Adam step on FP64 arrays (theta, m1, m2)."""
    fm = np.ascontiguousarray(np.asarray(free_mask, np.uint8))
    g = np.ascontiguousarray(np.asarray(grad, np.float64))
    sc = np.ascontiguousarray(np.asarray(scale, np.float64))
    lib().orc_adam_step(len(theta), _dp(theta), _dp(g), _dp(sc),
                        fm.ctypes.data_as(C.POINTER(C.c_uint8)), _dp(m1), _dp(m2), t, lr,
                        beta1, beta2, eps)


def philox4x64(counter, key):
    """One Philox4x64-10 block (4 uint64) for a 4-word counter and 2-word key."""
    c = (C.c_uint64 * 4)(*[int(x) for x in counter])
    k = (C.c_uint64 * 2)(*[int(x) for x in key])
    o = (C.c_uint64 * 4)()
    lib().orc_philox4x64(c, k, o)
    return [int(x) for x in o]


def besselk(nu: float, z: float):
    """(K_nu(z), dK/dz, dK/dnu, return code) from the oracle's quadrature of
    the integral representation."""
    out = np.zeros(3)
    rc = lib().orc_besselk(float(nu), float(z), _dp(out))
    return float(out[0]), float(out[1]), float(out[2]), rc


def erfcinv(q: float) -> float:
    return float(lib().orc_erfcinv(float(q)))


def generate(spec: dict, params_matrix, comp_counts, offsets, seed: int, col_f32: bool,
             n_events: int | None = None):
    """Toy events drawn by the oracle's generator: (cols [n_obs, n_events] FP64,
    values that exhausted their attempts, return code).  comp_counts [toys, K]."""
    m = Model(spec)
    pm = np.ascontiguousarray(np.asarray(params_matrix, np.float64))
    cc = np.ascontiguousarray(np.asarray(comp_counts, np.int64))
    off = np.ascontiguousarray(np.asarray(offsets, np.int64))
    toys = len(off) - 1
    n = int(off[-1]) if n_events is None else int(n_events)
    cols = np.full((len(spec["obs"]), n), np.nan)
    ex = C.c_int64(0)
    rc = lib().orc_generate(C.byref(m.s), _dp(pm), toys, cc.ctypes.data_as(C.POINTER(C.c_int64)),
                            off.ctypes.data_as(C.POINTER(C.c_int64)), C.c_uint64(seed),
                            1 if col_f32 else 0, _dp(cols), n, C.byref(ex))
    return cols, int(ex.value), rc
