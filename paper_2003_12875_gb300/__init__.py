"""rfgpu -- unbinned negative log-likelihood of a PDF graph on one GB300 GPU.

A thin binding over the C-ABI library ``librfgpu.so`` (include/rf.h): argument
marshalling only.  Every step of the likelihood -- normalisation integrals,
per-event PDFs, the log-sum, the adjoint gradient and the reductions -- runs in
the library's CUDA kernels.  PyTorch provides device memory and streams.  There
is no CPU fallback: without the compiled library (and a GPU) these calls raise.

The model is the plain-data ``spec`` dict (see datagen and oracle)::

    {"obs": [(lo, hi), ...], "params": [...], "fixed": [bool...] (optional),
     "nodes": [{"type": "gauss", "obs": 0, "params": [0, 1]}, ...], "root": i}

Typical use::

    g = Graph(spec, column_dtype="f32", eval_precision="fp32")
    nll, grad = g.nll(events, params)            # events: [n_obs, n] CUDA tensor
    v = RFNll.apply(params, events, g)           # autograd: dv/dparams = grad
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import torch

from . import build as _build

__all__ = ["Graph", "RFNll", "RFError", "load", "microbench", "TYPES", "shard_range",
           "sharded_nll", "rank_order_sum"]

TYPES = {"gauss": 1, "exp": 2, "cheb": 3, "cb": 4, "argus": 5,
         "add_frac": 6, "add_ext": 7, "prod": 8, "johnson": 9, "formula": 10, "hypatia2": 11}
_STATUS = {0: "RF_OK", 1: "RF_EINVAL", 2: "RF_EUNSUPPORTED", 3: "RF_EALIGN",
           4: "RF_ECUDA", 5: "RF_ENOMEM"}
MAX_CHILDREN, MAX_NODE_PARAMS = 8, 12
STATUS_PARAM_DOMAIN, STATUS_NONFINITE = 1, 2
TUNE_NO_CACHE, TUNE_REFRESH = 1, 2


class RFError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_STATUS.get(code, code)}: {msg}")
        self.code = code


class _Node(C.Structure):
    _fields_ = [("type", C.c_int32), ("obs", C.c_int32), ("n_children", C.c_int32),
                ("children", C.c_int32 * MAX_CHILDREN), ("n_params", C.c_int32),
                ("params", C.c_int32 * MAX_NODE_PARAMS), ("formula", C.c_char_p)]


class _Desc(C.Structure):
    _fields_ = [("n_nodes", C.c_int32), ("nodes", C.POINTER(_Node)), ("root", C.c_int32),
                ("n_obs", C.c_int32), ("obs_lo", C.POINTER(C.c_double)),
                ("obs_hi", C.POINTER(C.c_double)), ("n_params", C.c_int32),
                ("param_fixed", C.POINTER(C.c_uint8)), ("column_dtype", C.c_int32),
                ("eval_precision", C.c_int32), ("param_values", C.POINTER(C.c_double))]


class _Launch(C.Structure):
    _fields_ = [("block", C.c_int32), ("ept", C.c_int32), ("blocks_per_sm", C.c_int32),
                ("min_blocks", C.c_int32)]


_lib = None
_lock = threading.Lock()
SYMBOLS = ["rf_graph_validate", "rf_graph_compile", "rf_graph_destroy", "rf_nll",
           "rf_nll_host", "rf_logp", "rf_graph_bind_events", "rf_nll_batched",
           "rf_fit_toys", "rf_nll_plain", "rf_graph_get_launch", "rf_graph_set_launch",
           "rf_graph_tune", "rf_graph_status", "rf_graph_last_launches", "rf_last_error",
           "rf_microbench", "rf_graph_set_jit", "rf_graph_uses_jit", "rf_graph_kernel_regs",
           "rf_jit_check", "rf_check_log", "rf_nll_noalloc", "rf_graph_kernel_hash",
           "rf_check_d2f", "rf_generate_toys", "rf_graph_set_shard_weight",
           "rf_graph_tune_ex", "rf_graph_toy_kernel_hash", "rf_graph_get_toy_launch"]


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load librfgpu.so (building it for sm_103a first if it is missing or
    stale).  torch is imported first so the library binds to torch's CUDA
    runtime."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if build_if_missing:
            _build.build()
        if not os.path.exists(_build.LIB):
            raise ImportError(f"librfgpu.so not built at {_build.LIB}")
        L = C.CDLL(_build.LIB)
        vp, i64, i32, dp = C.c_void_p, C.c_int64, C.c_int32, C.POINTER(C.c_double)
        L.rf_graph_validate.argtypes = [C.POINTER(_Desc)]
        L.rf_graph_compile.argtypes = [C.POINTER(_Desc), C.POINTER(vp)]
        L.rf_graph_destroy.argtypes = [vp]
        L.rf_nll.argtypes = [vp, vp, i64, vp, vp, vp, vp]
        L.rf_nll_host.argtypes = [vp, vp, i64, vp, vp, vp, vp]
        L.rf_logp.argtypes = [vp, vp, i64, vp, vp, vp]
        L.rf_graph_bind_events.argtypes = [vp, vp, i64, i32]
        L.rf_nll_batched.argtypes = [vp, vp, i32, vp, vp, vp]
        L.rf_fit_toys.argtypes = [vp, vp, i32, vp, vp, i32, C.c_double, vp, vp]
        L.rf_generate_toys.argtypes = [vp, vp, vp, vp, i32, C.c_uint64, vp, i64, vp]
        L.rf_graph_set_shard_weight.argtypes = [vp, C.c_double]
        L.rf_nll_plain.argtypes = [vp, vp, i64, vp, vp, vp, vp]
        L.rf_graph_get_launch.argtypes = [vp, C.POINTER(_Launch)]
        L.rf_graph_set_launch.argtypes = [vp, C.POINTER(_Launch)]
        L.rf_graph_tune.argtypes = [vp, vp, i64, vp, vp, dp]
        L.rf_graph_tune_ex.argtypes = [vp, vp, i64, vp, vp, i32, dp, C.POINTER(i32)]
        L.rf_graph_status.argtypes = [vp, C.POINTER(C.c_uint32)]
        L.rf_graph_last_launches.argtypes = [vp]
        L.rf_graph_last_launches.restype = i32
        L.rf_last_error.restype = C.c_char_p
        L.rf_microbench.argtypes = [dp]
        L.rf_graph_set_jit.argtypes = [vp, i32]
        L.rf_graph_uses_jit.argtypes = [vp]
        L.rf_graph_uses_jit.restype = i32
        L.rf_graph_kernel_regs.argtypes = [vp]
        L.rf_graph_kernel_regs.restype = i32
        L.rf_jit_check.argtypes = [C.POINTER(_Desc)]
        L.rf_check_log.argtypes = [vp, vp, vp, i64, vp]
        L.rf_nll_noalloc.argtypes = [C.POINTER(_Desc), vp, i64, vp, vp, vp, i32, vp]
        L.rf_check_d2f.argtypes = [vp, vp, vp, i64, vp]
        L.rf_graph_kernel_hash.argtypes = [vp]
        L.rf_graph_kernel_hash.restype = C.c_uint64
        L.rf_graph_toy_kernel_hash.argtypes = [vp]
        L.rf_graph_toy_kernel_hash.restype = C.c_uint64
        i32p = C.POINTER(C.c_int32)
        L.rf_graph_get_toy_launch.argtypes = [vp, i32p, i32p, i32p]
        for name in SYMBOLS:
            if name not in ("rf_last_error", "rf_graph_last_launches", "rf_graph_uses_jit",
                            "rf_graph_kernel_regs", "rf_graph_kernel_hash",
                            "rf_graph_toy_kernel_hash"):
                getattr(L, name).restype = C.c_int
        _lib = L
    return _lib


def _check(code: int):
    if code != 0:
        raise RFError(code, load().rf_last_error().decode())


def _ptr(t: torch.Tensor | None):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def make_desc(spec: dict, column_dtype: str = "f64", eval_precision: str = "fp64"):
    """Build the C descriptor (and keep its buffers alive in the returned
    tuple)."""
    nodes = spec["nodes"]
    arr = (_Node * len(nodes))()
    texts = [nd["formula"].encode() if "formula" in nd else None for nd in nodes]
    for i, nd in enumerate(nodes):
        arr[i].type = TYPES[nd["type"]]
        arr[i].formula = texts[i]
        arr[i].obs = nd.get("obs", -1)
        ch = nd.get("children", [])
        arr[i].n_children = len(ch)
        for k, c in enumerate(ch):
            arr[i].children[k] = c
        ps = nd.get("params", [])
        arr[i].n_params = len(ps)
        for k, p in enumerate(ps):
            arr[i].params[k] = p
    rng = list(spec["obs"])
    lo = (C.c_double * len(rng))(*[float(r[0]) for r in rng])
    hi = (C.c_double * len(rng))(*[float(r[1]) for r in rng])
    npar = len(spec["params"])
    fixed = spec.get("fixed")
    fx = (C.c_uint8 * max(npar, 1))(*[1 if (fixed and fixed[j]) else 0 for j in range(npar)])
    # the spec's parameter values at compile time (they select forms only,
    # e.g. the general ARGUS form for a p fixed away from 1/2)
    vals = (C.c_double * max(npar, 1))(*[float(v) for v in spec["params"]])
    d = _Desc(len(nodes), arr, spec.get("root", len(nodes) - 1), len(rng), lo, hi, npar,
              fx, 0 if column_dtype == "f32" else 1, 0 if eval_precision == "fp32" else 1,
              vals)
    return d, (arr, lo, hi, fx, texts, vals)


def validate(spec: dict, column_dtype: str = "f64", eval_precision: str = "fp64") -> int:
    """Host-only check of a spec; returns the rf_status code (0 = OK)."""
    d, keep = make_desc(spec, column_dtype, eval_precision)
    return load().rf_graph_validate(C.byref(d))


def jit_check(spec: dict, column_dtype: str = "f64", eval_precision: str = "fp64") -> int:
    """NVRTC-compile the graph's specialised kernels without a GPU; 0 = OK."""
    d, keep = make_desc(spec, column_dtype, eval_precision)
    return load().rf_jit_check(C.byref(d))


def nll_noalloc(spec: dict, events: torch.Tensor, params: torch.Tensor, out: torch.Tensor,
                column_dtype: str = "f64", eval_precision: str = "fp64", blocks: int = 0):
    """rf_nll_noalloc: NLL and gradient with no device allocation by the
    library (its scratch is a static device array).  `out` is a caller-owned
    CUDA float64 tensor [1 + n_params]: out[0] = NLL, out[1:] = gradient."""
    d, keep = make_desc(spec, column_dtype, eval_precision)
    n = events.shape[-1] if events.dim() == 2 else events.numel()
    _check(load().rf_nll_noalloc(C.byref(d), _ptr(events), int(n), _ptr(params), _ptr(out),
                                 C.c_void_p(out.data_ptr() + 8), int(blocks), _stream()))
    return out


def check_d2f(x: torch.Tensor):
    """(library FP64->FP32 rounding, hardware rounding) of a CUDA float64 tensor."""
    x = x.contiguous()
    yf = torch.empty(x.shape, dtype=torch.float32, device=x.device)
    yr = torch.empty_like(yf)
    _check(load().rf_check_d2f(_ptr(x), _ptr(yf), _ptr(yr), x.numel(), _stream()))
    return yf, yr


def check_log(x: torch.Tensor):
    """(library FP32 log, CUDA logf) of a CUDA float32 tensor."""
    x = x.contiguous()
    yf, yr = torch.empty_like(x), torch.empty_like(x)
    _check(load().rf_check_log(_ptr(x), _ptr(yf), _ptr(yr), x.numel(), _stream()))
    return yf, yr


class Graph:
    """A compiled PDF graph on the current CUDA device."""

    def __init__(self, spec: dict, column_dtype: str = "f64", eval_precision: str = "fp64"):
        if column_dtype not in ("f32", "f64") or eval_precision not in ("fp32", "fp64"):
            raise ValueError("column_dtype in {f32, f64}, eval_precision in {fp32, fp64}")
        L = load()
        self.spec = spec
        self.column_dtype = column_dtype
        self.eval_precision = eval_precision
        self.dtype = torch.float32 if column_dtype == "f32" else torch.float64
        self.n_obs = len(spec["obs"])
        self.n_par = len(spec["params"])
        d, keep = make_desc(spec, column_dtype, eval_precision)
        h = C.c_void_p()
        _check(L.rf_graph_compile(C.byref(d), C.byref(h)))
        self._h = h
        self._bound = None
        self.tune_from_cache = False

    def close(self):
        if getattr(self, "_h", None):
            load().rf_graph_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------ checks
    def _events(self, events: torch.Tensor) -> int:
        if not events.is_cuda or events.dtype != self.dtype:
            raise TypeError(f"events must be a CUDA {self.dtype} tensor")
        if not events.is_contiguous():
            raise ValueError("events must be contiguous ([n_obs, n] SoA)")
        n = events.shape[-1] if events.dim() == 2 else events.numel()
        if events.dim() == 2 and events.shape[0] != self.n_obs:
            raise ValueError(f"events must have {self.n_obs} rows (observables)")
        return int(n)

    def _params(self, params: torch.Tensor):
        if not params.is_cuda or params.dtype != torch.float64 or not params.is_contiguous():
            raise TypeError("params must be a contiguous CUDA float64 tensor")
        if params.numel() != self.n_par:
            raise ValueError(f"params must have {self.n_par} entries")

    # ------------------------------------------------------------ calls
    def nll(self, events: torch.Tensor, params: torch.Tensor, grad: bool = True,
            out: torch.Tensor | None = None):
        """(nll [1], grad [P] or None) as CUDA float64 tensors; one fused kernel."""
        n = self._events(events)
        self._params(params)
        if out is None:
            out = torch.empty(1 + self.n_par, dtype=torch.float64, device=events.device)
        _check(load().rf_nll(self._h, _ptr(events), n, _ptr(params), _ptr(out),
                             C.c_void_p(out.data_ptr() + 8) if grad else None, _stream()))
        return out[:1], (out[1:] if grad else None)

    def nll_host(self, events_host: torch.Tensor, params_host: torch.Tensor, grad: bool = True):
        """The same from host tensors (pinned memory recommended): copies in,
        evaluates, copies out, synchronises.  Returns (nll float, grad tensor)."""
        if events_host.is_cuda or params_host.is_cuda:
            raise TypeError("nll_host takes host tensors")
        ev = events_host.contiguous()
        pa = params_host.to(torch.float64).contiguous()
        n = ev.shape[-1] if ev.dim() == 2 else ev.numel()
        o = torch.empty(1, dtype=torch.float64)
        g = torch.empty(self.n_par, dtype=torch.float64) if grad else None
        _check(load().rf_nll_host(self._h, _ptr(ev), int(n), _ptr(pa), _ptr(o),
                                  _ptr(g) if grad else None, _stream()))
        return float(o[0]), g

    def logp(self, events: torch.Tensor, params: torch.Tensor) -> torch.Tensor:
        n = self._events(events)
        self._params(params)
        out = torch.empty(n, dtype=torch.float64, device=events.device)
        _check(load().rf_logp(self._h, _ptr(events), n, _ptr(params), _ptr(out), _stream()))
        return out

    def bind_events(self, events: torch.Tensor, max_toys: int):
        n = self._events(events)
        _check(load().rf_graph_bind_events(self._h, _ptr(events), n, int(max_toys)))
        self._bound = events

    def nll_batched(self, offsets: torch.Tensor, params_matrix: torch.Tensor,
                    out: torch.Tensor | None = None) -> torch.Tensor:
        toys = offsets.numel() - 1
        if offsets.dtype != torch.int64 or not offsets.is_cuda:
            raise TypeError("offsets must be a CUDA int64 tensor")
        if params_matrix.shape != (toys, self.n_par) or params_matrix.dtype != torch.float64:
            raise ValueError("params_matrix must be float64 [toys, n_params]")
        if out is None:
            out = torch.empty(toys, 1 + self.n_par, dtype=torch.float64, device=offsets.device)
        _check(load().rf_nll_batched(self._h, _ptr(offsets), toys, _ptr(params_matrix),
                                     _ptr(out), _stream()))
        return out

    def set_shard_weight(self, w: float):
        """Weight of the extended term in this graph's NLL (1 on exactly one
        shard of a dataset split over processes, 0 on the others)."""
        _check(load().rf_graph_set_shard_weight(self._h, float(w)))

    def generate_toys(self, params_matrix: torch.Tensor, comp_counts: torch.Tensor,
                      offsets: torch.Tensor, seed: int, n_events: int | None = None,
                      out: torch.Tensor | None = None) -> torch.Tensor:
        """Events of toys drawn on the device (rf_generate_toys): params_matrix
        [toys, n_params] FP64, comp_counts [toys, n_comp] int64, offsets
        [toys + 1] int64, all CUDA; returns (or fills) the [n_obs, n_events]
        column tensor of the graph's column type."""
        toys = offsets.numel() - 1
        for t, dt in ((params_matrix, torch.float64), (comp_counts, torch.int64),
                      (offsets, torch.int64)):
            if not t.is_cuda or t.dtype != dt or not t.is_contiguous():
                raise TypeError("generate_toys takes contiguous CUDA tensors "
                                "(FP64 params, int64 counts and offsets)")
        if params_matrix.shape != (toys, self.n_par) or comp_counts.shape[0] != toys:
            raise ValueError("params_matrix [toys, n_params], comp_counts [toys, n_comp]")
        if n_events is None:
            n_events = int(offsets[-1].item())
        if out is None:
            out = torch.empty(self.n_obs, n_events, dtype=self.dtype, device=offsets.device)
        _check(load().rf_generate_toys(self._h, _ptr(params_matrix), _ptr(comp_counts),
                                       _ptr(offsets), toys, C.c_uint64(seed), _ptr(out),
                                       int(n_events), _stream()))
        return out

    def fit_toys(self, offsets: torch.Tensor, params_matrix: torch.Tensor,
                 scale: torch.Tensor, iters: int, lr: float) -> torch.Tensor:
        """Adam on every toy, `iters` CUDA-graph replays; params_matrix is
        updated in place; scale is [toys, n_params] (units of each toy's
        parameters); returns the (NLL, grad) rows of the last evaluation."""
        toys = offsets.numel() - 1
        if scale.shape != (toys, self.n_par) or scale.dtype != torch.float64:
            raise ValueError("scale must be float64 [toys, n_params]")
        out = torch.empty(toys, 1 + self.n_par, dtype=torch.float64, device=offsets.device)
        _check(load().rf_fit_toys(self._h, _ptr(offsets), toys, _ptr(params_matrix),
                                  _ptr(scale), int(iters), float(lr), _ptr(out), _stream()))
        return out

    def nll_plain(self, events: torch.Tensor, params: torch.Tensor, grad: bool = True):
        n = self._events(events)
        self._params(params)
        out = torch.empty(1 + self.n_par, dtype=torch.float64, device=events.device)
        _check(load().rf_nll_plain(self._h, _ptr(events), n, _ptr(params), _ptr(out),
                                   C.c_void_p(out.data_ptr() + 8) if grad else None, _stream()))
        return out[:1], (out[1:] if grad else None)

    def get_launch(self) -> dict:
        c = _Launch()
        _check(load().rf_graph_get_launch(self._h, C.byref(c)))
        return {"block": c.block, "ept": c.ept, "blocks_per_sm": c.blocks_per_sm,
                "min_blocks": c.min_blocks}

    def set_launch(self, block=None, ept=None, blocks_per_sm=None, min_blocks=None):
        cur = self.get_launch()
        c = _Launch(block or cur["block"], ept or cur["ept"],
                    blocks_per_sm or cur["blocks_per_sm"], min_blocks or cur["min_blocks"])
        _check(load().rf_graph_set_launch(self._h, C.byref(c)))

    def tune(self, events: torch.Tensor, params: torch.Tensor, cache: bool = True,
             refresh: bool = False) -> float:
        """Picks the fastest launch configuration (mean ms of one call with it
        returned); the choice is cached on disk unless cache=False, and
        refresh=True times every configuration even on a cache hit."""
        n = self._events(events)
        self._params(params)
        ms, hit = C.c_double(), C.c_int32()
        flags = (0 if cache else TUNE_NO_CACHE) | (TUNE_REFRESH if refresh else 0)
        _check(load().rf_graph_tune_ex(self._h, _ptr(events), n, _ptr(params), _stream(),
                                       flags, C.byref(ms), C.byref(hit)))
        self.tune_from_cache = bool(hit.value)
        return ms.value

    def status(self) -> int:
        v = C.c_uint32()
        _check(load().rf_graph_status(self._h, C.byref(v)))
        return int(v.value)

    def last_launches(self) -> int:
        return int(load().rf_graph_last_launches(self._h))

    def set_jit(self, enable: bool):
        _check(load().rf_graph_set_jit(self._h, 1 if enable else 0))

    def uses_jit(self) -> bool:
        return bool(load().rf_graph_uses_jit(self._h))

    def kernel_regs(self) -> int:
        return int(load().rf_graph_kernel_regs(self._h))

    def kernel_hash(self) -> str:
        return f"{int(load().rf_graph_kernel_hash(self._h)):016x}"

    def toy_kernel_hash(self) -> str:
        return f"{int(load().rf_graph_toy_kernel_hash(self._h)):016x}"

    def get_toy_launch(self) -> dict:
        """The toy segment kernel's block size, events per lane and registers
        per thread (0 before bind_events or with the generic kernels)."""
        b, e, r = C.c_int32(), C.c_int32(), C.c_int32()
        _check(load().rf_graph_get_toy_launch(self._h, C.byref(b), C.byref(e), C.byref(r)))
        return {"block": b.value, "events_per_lane": e.value, "regs_per_thread": r.value}


class RFNll(torch.autograd.Function):
    """NLL as a differentiable function of the parameter tensor: the forward
    launches the fused kernel with its adjoint, backward scales the stored
    gradient (no finite differences)."""

    @staticmethod
    def forward(ctx, params: torch.Tensor, events: torch.Tensor, graph: Graph):
        v, g = graph.nll(events, params.detach(), grad=True)
        ctx.save_for_backward(g)
        return v.reshape(())

    @staticmethod
    def backward(ctx, gout):
        (g,) = ctx.saved_tensors
        return gout * g, None, None


def microbench() -> dict:
    """Measured per-operation throughput (operations/s) on the current GPU,
    and single-warp FP64 latencies (ns per dependent operation)."""
    out = (C.c_double * 24)()
    _check(load().rf_microbench(out))
    keys = ["fp32_fma", "expf", "logf", "rcp_f32", "fp64_fma", "exp_f64", "log_f64", "erf_f64",
            "log_fast_f32", "exp_neg_f32", "rcp_approx_f32", "fp32_fma_packed_x2",
            "fp64_fma_latency_ns_1lane", "fp64_fma_latency_ns_32lanes",
            "exp_f64_latency_ns_1lane", "exp_f64_latency_ns_32lanes",
            "sqrtf", "sqrt_approx_f32", "log2_f64", "exp2_f64", "div_f64", "lg2_approx_f32",
            "ex2_approx_f32", "sqrt_f64"]
    return dict(zip(keys, list(out)))


def shard_range(n_events: int, rank: int, world: int) -> tuple[int, int]:
    """The contiguous event range [lo, hi) of rank `rank` of `world`."""
    return rank * n_events // world, (rank + 1) * n_events // world


def rank_order_sum(parts: torch.Tensor) -> torch.Tensor:
    """Sum of the rows of parts [world, m] in row (rank) order with
    Neumaier's compensation (Neumaier 1974): the result depends only on the
    rows' values and order, never on a collective's internal reduction order,
    so every rank that holds the same rows gets the same bits."""
    s = parts[0].clone()
    c = torch.zeros_like(s)
    for r in range(1, parts.shape[0]):
        x = parts[r]
        t = s + x
        c += torch.where(s.abs() >= x.abs(), (s - t) + x, (x - t) + s)
        s = t
    return s + c


def sharded_nll(graph: "Graph", shard_events: torch.Tensor, params: torch.Tensor,
                rank: int, group=None) -> torch.Tensor:
    """NLL and gradient of a dataset split over the processes of a
    torch.distributed group (the multi-process mode of the paper's Sec. 5.2:
    contiguous batches of the dataset divided among processes).  This rank
    evaluates its contiguous shard with rf_nll (the extended term on rank 0
    only), the ranks' (1 + n_params) values are all-gathered, and every rank
    adds them in rank order with Neumaier compensation (rank_order_sum), so
    all ranks return the same bits, run after run.  Returns [1 + n_params]
    (NLL, gradient) of the whole dataset."""
    import torch.distributed as dist
    graph.set_shard_weight(1.0 if rank == 0 else 0.0)
    out = torch.empty(1 + graph.n_par, dtype=torch.float64, device=shard_events.device)
    graph.nll(shard_events, params, out=out)
    world = dist.get_world_size(group)
    parts = [torch.empty_like(out) for _ in range(world)]
    dist.all_gather(parts, out, group=group)
    return rank_order_sum(torch.stack(parts))
