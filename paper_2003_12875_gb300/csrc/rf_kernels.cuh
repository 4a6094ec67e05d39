// rf_kernels.cuh -- kernel bodies, templated on a Model that supplies the
// per-event computation.  Two kinds of Model exist:
//  * GenericModel<NL>: the leaf types, component membership and gradient
//    masks are read from the RfProgram at run time (uniform branches); it is
//    compiled ahead of time for every leaf count and precision;
//  * a per-graph model emitted by the graph compiler, in which all of these
//    are compile-time constants, compiled with NVRTC for sm_103a when the
//    graph is compiled (see jit.cpp).
// Both use the same leaf functions, prologue, reduction and epilogue.
//
// A Model provides:
//   static constexpr int NL, NCOL;              leaves, columns read
//   static constexpr unsigned long long AMASK;  accumulators in use
//   template <class Real> static void event(const RfProgram&,
//       const EvalConsts<Real, NL>&, const Real (&x)[NL], Real (&q)[NACC])
#pragma once
#include "rf_device.cuh"

namespace rf {

template <int NL>
struct GenericModel {
  static constexpr int NL_ = NL;
  static constexpr int NCOL = NL;
  static constexpr unsigned long long AMASK = ~0ull;

  // leaves -> components -> log-sum-exp -> adjoint weights, into q
  template <typename Real>
  static __device__ __forceinline__ void event(const RfProgram& P,
                                               const EvalConsts<Real, NL>& K,
                                               const Real (&xc)[NL],
                                               Real (&q)[RF_NACC(NL)]) {
    typedef Fn<Real> F;
    Real u[NL], g[NL][RF_LEAF_MAXP];
#pragma unroll
    for (int k = 0; k < NL; ++k) {
      const int col = P.leaf[k].col;
      Real x = xc[0];
#pragma unroll
      for (int c = 1; c < NL; ++c)
        if (col == c) x = xc[c];
      eval_leaf<Real>(P.leaf[k].type, P.leaf[k].gmask, x, K.pc[k], u[k], g[k]);
    }
    Real v[NL], w[NL];
#pragma unroll
    for (int c = 0; c < NL; ++c) {
      v[c] = K.delta[c];
#pragma unroll
      for (int k = 0; k < NL; ++k)
        if (P.leaf[k].comp == c) v[c] += u[k];
      w[c] = Real(0);
    }
    Real ell;
    const int C = P.n_comp;
    if (C == 1) {
      ell = v[0];
      w[0] = Real(1);
    } else if (NL >= 2 && C == 2) {
      Real dv = v[1] - v[0];
      Real e = F::exp(-fabs(dv));
      Real s = Real(1) + e;
      Real rs = F::rcp(s);
      ell = fmax(v[0], v[1]) + F::log(s);
      Real wb = rs, ws = e * rs;
      w[0] = dv > Real(0) ? ws : wb;
      w[1] = dv > Real(0) ? wb : ws;
    } else {
      Real m = v[0];
#pragma unroll
      for (int c = 1; c < NL; ++c)
        if (c < C) m = fmax(m, v[c]);
      Real s = Real(0);
#pragma unroll
      for (int c = 0; c < NL; ++c) {
        w[c] = (c < C) ? F::exp(v[c] - m) : Real(0);
        s += w[c];
      }
      ell = m + F::log(s);
      Real rs = F::rcp(s);
#pragma unroll
      for (int c = 0; c < NL; ++c) w[c] *= rs;
    }
    q[0] += ell;
    if (K.zero_mask == 0) {
#pragma unroll
      for (int c = 0; c < NL; ++c) q[1 + c] += w[c];
    } else {
#pragma unroll
      for (int c = 0; c < NL; ++c) {
        Real vc = K.delta_nc[c];
#pragma unroll
        for (int k = 0; k < NL; ++k)
          if (P.leaf[k].comp == c) vc += u[k];
        q[1 + c] += comp_weight<Real>(K.zero_mask, c, vc, ell, w[c]);
      }
    }
#pragma unroll
    for (int k = 0; k < NL; ++k) {
      const int comp = P.leaf[k].comp;
      Real wk = w[0];
#pragma unroll
      for (int c = 1; c < NL; ++c)
        if (comp == c) wk = w[c];
      const int gm = P.leaf[k].gmask;
#pragma unroll
      for (int j = 0; j < RF_LEAF_MAXP; ++j)
        if ((gm >> j) & 1) q[1 + NL + k * RF_LEAF_MAXP + j] += wk * g[k][j];
    }
  }
};

// ---------------------------------------------------------- event loading
template <typename Col>
struct Vec;
template <>
struct Vec<float> {
  static constexpr int W = 4;
  typedef float4 T;
};
template <>
struct Vec<double> {
  static constexpr int W = 2;
  typedef double2 T;
};

template <typename Real, typename Col, int NL, int NCOL, int EPT>
__device__ __forceinline__ void load_full(const RfProgram& P, const Col* __restrict__ ev,
                                          int64_t stride, int64_t i0, bool vec,
                                          Real (&x)[NL][EPT]) {
  constexpr int W = Vec<Col>::W;
  static_assert(EPT % W == 0, "EPT must be a multiple of the vector width");
#pragma unroll
  for (int c = 0; c < NL; ++c) {
    if (c < NCOL && c < P.n_cols) {
      const Col* col = ev + (int64_t)P.col_obs[c] * stride + i0;
      if (vec) {
        const typename Vec<Col>::T* vp = reinterpret_cast<const typename Vec<Col>::T*>(col);
#pragma unroll
        for (int v = 0; v < EPT / W; ++v) {
#ifdef RF_EVENTS_KEEP_L2
          typename Vec<Col>::T t = __ldg(vp + v);
#else
          // events are read once per call: streaming (evict-first) loads, so
          // they do not push the prologue's code and constants out of L2
          typename Vec<Col>::T t = __ldcs(vp + v);
#endif
          const Col* tc = reinterpret_cast<const Col*>(&t);
#pragma unroll
          for (int e = 0; e < W; ++e) x[c][v * W + e] = cvt<Real, Col>(tc[e]);
        }
      } else {
#pragma unroll
        for (int e = 0; e < EPT; ++e) x[c][e] = cvt<Real, Col>(__ldcs(col + e));
      }
    } else {
#pragma unroll
      for (int e = 0; e < EPT; ++e) x[c][e] = Real(0);
    }
  }
}

// Kahan-compensated running sums (value = s - c) over the accumulators in
// MASK; the others stay zero and generate no instructions.
template <typename Real, int N, unsigned long long MASK>
struct Acc {
  Real s[N], c[N];
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int i = 0; i < N; ++i) s[i] = c[i] = Real(0);
  }
  __device__ __forceinline__ void add(const Real (&q)[N]) {
#pragma unroll
    for (int i = 0; i < N; ++i) {
      if (!((MASK >> i) & 1ull)) continue;
      Real y = q[i] - c[i];
      Real t = s[i] + y;
      c[i] = (t - s[i]) - y;
      s[i] = t;
    }
  }
  __device__ __forceinline__ double value(int i) const {
    return ((MASK >> i) & 1ull) ? (double)s[i] - (double)c[i] : 0.0;
  }
};

// Block-wide FP64 totals of the per-thread accumulators, fixed order.
template <typename Real, int NA, unsigned long long MASK>
struct BlockReduce;
template <int NA, unsigned long long MASK>
struct BlockReduce<float, NA, MASK> {  // FP32 evaluation: FP32-pair arithmetic
  static __device__ __forceinline__ void run(const Acc<float, NA, MASK>& acc, void* red,
                                             double* tot) {
    float ls[NA];
#pragma unroll
    for (int i = 0; i < NA; ++i) ls[i] = -acc.c[i];  // Kahan keeps -(lost low part)
    block_sum_ds<NA, MASK>(acc.s, ls, static_cast<float2*>(red), tot);
  }
};
template <int NA, unsigned long long MASK>
struct BlockReduce<double, NA, MASK> {  // FP64 evaluation
  static __device__ __forceinline__ void run(const Acc<double, NA, MASK>& acc, void* red,
                                             double* tot) {
    double val[NA];
#pragma unroll
    for (int i = 0; i < NA; ++i) val[i] = acc.value(i);
    block_sum<NA>(val, static_cast<double*>(red), tot);
  }
};

// EPT events already in registers -> the iteration's partial sums -> acc.
template <class M, typename Real, int EPT>
__device__ __forceinline__ void compute_full(const RfProgram& P,
                                             const EvalConsts<Real, M::NL_>& K,
                                             const Real (&x)[M::NL_][EPT],
                                             Acc<Real, RF_NACC(M::NL_), M::AMASK>& acc) {
  constexpr int NL = M::NL_;
  Real q[RF_NACC(NL)];
#pragma unroll
  for (int i = 0; i < RF_NACC(NL); ++i) q[i] = Real(0);
#pragma unroll
  for (int e = 0; e < EPT; ++e) {
    Real xc[NL];
#pragma unroll
    for (int c = 0; c < NL; ++c) xc[c] = x[c][e];
    M::template event<Real>(P, K, xc, q);
  }
  acc.add(q);
}

// Chunks first, first+step, ... < nfull of EPT events each (chunk c starts at
// event base + c*EPT).  The next chunk's 128-bit loads are issued before the
// current chunk is computed (register double buffering), so the memory
// latency overlaps the arithmetic.
template <class M, typename Real, typename Col, int EPT>
__device__ __forceinline__ void stream_chunks(const RfProgram& P,
                                              const EvalConsts<Real, M::NL_>& K,
                                              const Col* __restrict__ ev, int64_t stride,
                                              int64_t base, int64_t first, int64_t step,
                                              int64_t nfull, bool vec,
                                              Acc<Real, RF_NACC(M::NL_), M::AMASK>& acc) {
  constexpr int NL = M::NL_;
  if (first >= nfull) return;
  Real xa[NL][EPT];
  load_full<Real, Col, NL, M::NCOL, EPT>(P, ev, stride, base + first * EPT, vec, xa);
  for (int64_t ch = first;;) {
    const int64_t nx = ch + step;
    const bool more = nx < nfull;
    Real xb[NL][EPT];
    if (more) load_full<Real, Col, NL, M::NCOL, EPT>(P, ev, stride, base + nx * EPT, vec, xb);
    compute_full<M, Real, EPT>(P, K, xa, acc);
    if (!more) break;
#pragma unroll
    for (int c = 0; c < NL; ++c)
#pragma unroll
      for (int e = 0; e < EPT; ++e) xa[c][e] = xb[c][e];
    ch = nx;
  }
}

template <class M, typename Real, typename Col>
__device__ inline void iterate_scalar(const RfProgram& P, const EvalConsts<Real, M::NL_>& K,
                                      const Col* __restrict__ ev, int64_t stride, int64_t i0,
                                      int64_t i1, Acc<Real, RF_NACC(M::NL_), M::AMASK>& acc) {
  constexpr int NL = M::NL_;
  for (int64_t i = i0; i < i1; ++i) {
    Real xc[NL];
#pragma unroll
    for (int c = 0; c < NL; ++c)
      xc[c] = (c < M::NCOL && c < P.n_cols) ? cvt<Real, Col>(ev[(int64_t)P.col_obs[c] * stride + i])
                                            : Real(0);
    Real q[RF_NACC(NL)];
#pragma unroll
    for (int j = 0; j < RF_NACC(NL); ++j) q[j] = Real(0);
    M::template event<Real>(P, K, xc, q);
    acc.add(q);
  }
}

// Prologue run by every block: leaf k by lane 0 of warp k (their FP64 work
// proceeds in parallel), then the combination by thread 0.
template <typename Real>
__device__ inline void block_prologue(const RfProgram& P, const double* params,
                                      RfConsts<Real>& K, double* lnI, int* ok) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
  for (int k = wid; k < P.n_leaves; k += nw)
    if (lane == 0) ok[k] = leaf_consts(P, params, K, k, &lnI[k]) ? 1 : 0;
  __syncthreads();
  if (threadIdx.x == 0) {
    bool all = true;
    for (int k = 0; k < P.n_leaves; ++k) all &= ok[k] != 0;
    comb_consts(P, params, K, lnI, all);
  }
  __syncthreads();
}

// ------------------------------------------------------ single dataset
template <class M, typename Real, typename Col, int EPT>
__device__ __forceinline__ void fused_body(const RfProgram& P, const Col* __restrict__ ev,
                                           int64_t n, int64_t head, int vec,
                                           const double* __restrict__ params, RfWork& W,
                                           double* nll, double* grad) {
  constexpr int NL = M::NL_;
  constexpr int NA = RF_NACC(NL);
  __shared__ RfConsts<Real> K;
  __shared__ double lnI[RF_MAXL];
  __shared__ int ok[RF_MAXL];
  __shared__ double red[32 * NA];
  __shared__ double tot[NA];
  __shared__ int s_last;

  if (W.consts) {
    // constants from the prologue kernel, which this launch may overlap:
    // wait for it (a no-op when this grid was not launched as its dependent)
    asm volatile("griddepcontrol.wait;" ::: "memory");
    constexpr int kWords = (int)(sizeof(RfConsts<Real>) / sizeof(double));
    const double* src = static_cast<const double*>(W.consts);
    double* dst = reinterpret_cast<double*>(&K);
    for (int w = threadIdx.x; w < kWords; w += blockDim.x) dst[w] = __ldcg(src + w);
    __syncthreads();
  } else {
    block_prologue(P, params, K, lnI, ok);
  }

  Acc<Real, NA, M::AMASK> acc;
  acc.zero();
  if (!K.bad) {
    EvalConsts<Real, NL> E;
    E.load(K);
    const int64_t h = head < n ? head : n;
    const int64_t nfull = (n - h) / EPT;
    const int64_t gsz = (int64_t)gridDim.x * blockDim.x;
    stream_chunks<M, Real, Col, EPT>(P, E, ev, n, h, (int64_t)blockIdx.x * blockDim.x + threadIdx.x,
                                     gsz, nfull, vec != 0, acc);
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == blockDim.x - 1) {
      iterate_scalar<M, Real, Col>(P, E, ev, n, 0, h, acc);
      iterate_scalar<M, Real, Col>(P, E, ev, n, h + nfull * EPT, n, acc);
    }
  }

  BlockReduce<Real, NA, M::AMASK>::run(acc, red, tot);
  if (threadIdx.x < NA) W.partials[(int64_t)blockIdx.x * RF_NACC_MAX + threadIdx.x] = tot[threadIdx.x];
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = (atomicAdd(W.counter, 1u) == gridDim.x - 1) ? 1 : 0;
  __syncthreads();
  if (s_last) {
    __threadfence();
    rows_sum<NA>(W.partials, 0, gridDim.x, red, tot);
    if (threadIdx.x == 0) {
      epilogue<Real, NL>(P, K, tot, n, nll, grad, W.status);
      *W.counter = 0u;
    }
  }
}

// Per-event log P(x_i) = beta_ref + ell_i (FP64 output), one event per thread.
template <class M, typename Real, typename Col>
__device__ __forceinline__ void logp_body(const RfProgram& P, const Col* __restrict__ ev,
                                          int64_t n, const double* __restrict__ params,
                                          double* logp) {
  constexpr int NL = M::NL_;
  constexpr int NA = RF_NACC(NL);
  __shared__ RfConsts<Real> K;
  __shared__ double lnI[RF_MAXL];
  __shared__ int ok[RF_MAXL];
  block_prologue(P, params, K, lnI, ok);
  EvalConsts<Real, NL> E;
  E.load(K);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    Real xc[NL];
#pragma unroll
    for (int c = 0; c < NL; ++c)
      xc[c] = (c < M::NCOL && c < P.n_cols) ? cvt<Real, Col>(ev[(int64_t)P.col_obs[c] * n + i])
                                            : Real(0);
    Real q[NA];
#pragma unroll
    for (int j = 0; j < NA; ++j) q[j] = Real(0);
    M::template event<Real>(P, E, xc, q);
    logp[i] = K.bad ? kNaN() : K.beta_ref + (double)q[0];
  }
}

// The single-dataset prologue as its own grid: block k computes leaf k (the
// FP64 work of different leaves runs on different SMs), the last block to
// finish combines.  It lets the dependent fused grid launch immediately.
template <typename Real>
__device__ __forceinline__ void prologue_body(const RfProgram& P, const double* __restrict__ params,
                                              RfWork& W) {
  asm volatile("griddepcontrol.launch_dependents;");
  RfConsts<Real>* K = static_cast<RfConsts<Real>*>(W.consts);
  const int k = blockIdx.x;
  if (threadIdx.x != 0 || k >= P.n_leaves) return;
  double lnI = 0.0;
  const bool ok = leaf_consts(P, params, *K, k, &lnI);
  W.pro_lnI[k] = lnI;
  W.pro_ok[k] = ok ? 1 : 0;
  __threadfence();
  if (atomicAdd(W.pro_ticket, 1u) == (unsigned)P.n_leaves - 1u) {
    __threadfence();
    double l[RF_MAXL];
    bool all = true;
    for (int j = 0; j < P.n_leaves; ++j) {
      l[j] = __ldcg(W.pro_lnI + j);
      all &= __ldcg(W.pro_ok + j) != 0;
    }
    comb_consts(P, params, *K, l, all);
    *W.pro_ticket = 0u;
  }
}

// ------------------------------------------------------ toy studies
// One thread per toy: the toy's FP64 normalisations and coefficients.
template <typename Real>
__device__ __forceinline__ void toy_prep_body(const RfProgram& P, const double* __restrict__ pm,
                                              int32_t toys, RfConsts<Real>* consts,
                                              unsigned int* next_tile, int32_t* adam_t) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t == 0) {
    *next_tile = 0u;
    if (adam_t) *adam_t += 1;
  }
  if (t < toys) {
    RfConsts<Real> K;
    build_consts_serial(P, pm + (int64_t)t * P.n_par, K);
    consts[t] = K;
  }
}

// Persistent blocks take tiles from an atomic counter; a tile holds events of
// one toy only; the last tile of a toy to finish (per-toy ticket) sums that
// toy's tile partials in tile order and writes (NLL, grad), optionally
// followed by one Adam step on the toy's parameter row.  Results do not
// depend on which block ran which tile.
template <class M, typename Real, typename Col, int EPT>
__device__ __forceinline__ void toy_tile_body(const RfProgram& P, const Col* __restrict__ ev,
                                              int64_t stride, int vec,
                                              const int64_t* __restrict__ offsets, int32_t toys,
                                              int64_t tile_ev, double* pm, double* out,
                                              RfWork& W, const double* __restrict__ adam_scale,
                                              double adam_lr, int64_t max_rows) {
  constexpr int NL = M::NL_;
  constexpr int NA = RF_NACC(NL);
  __shared__ RfConsts<Real> K;
  __shared__ double red[32 * NA];
  __shared__ double tot[NA];
  __shared__ int64_t s_tile, s_toy, s_b, s_e, s_total;
  __shared__ int s_last;
  const RfConsts<Real>* consts = static_cast<const RfConsts<Real>*>(W.toy_consts);
  constexpr int kWords = (int)(sizeof(RfConsts<Real>) / sizeof(double));
  static_assert(sizeof(RfConsts<Real>) % sizeof(double) == 0, "RfConsts size");

  if (threadIdx.x == 0) s_total = __ldcg(W.tile_start + toys);
  __syncthreads();
  const int64_t total = s_total < max_rows ? s_total : max_rows;
  // Thread 0 takes the next tile from the counter at the start of an
  // iteration and loads its (toy, event range) after the compute, so that
  // both round trips overlap the current tile's work.
  int64_t nx_tile = 0, nx_b = 0, nx_e = 0;
  int nx_toy = 0;
  auto load_meta = [&]() {
    if (nx_tile < total) {
      nx_toy = __ldcg(W.tile_toy + nx_tile);
      const longlong2 be = __ldcg(reinterpret_cast<const longlong2*>(W.tile_be) + nx_tile);
      nx_b = be.x;
      nx_e = be.y;
    }
  };
  if (threadIdx.x == 0) {
    nx_tile = (int64_t)atomicAdd(W.next_tile, 1u);
    load_meta();
  }
  for (;;) {
    if (threadIdx.x == 0) {
      s_tile = nx_tile;
      s_toy = nx_toy;
      s_b = nx_b;
      s_e = nx_e;
    }
    __syncthreads();
    const int64_t tl = s_tile;
    if (tl >= total) break;
    const int64_t toy = s_toy, b = s_b, e = s_e;
    if (threadIdx.x == 0) nx_tile = (int64_t)atomicAdd(W.next_tile, 1u);
    {
      const double* src = reinterpret_cast<const double*>(consts + toy);
      double* dst = reinterpret_cast<double*>(&K);
      for (int w = threadIdx.x; w < kWords; w += blockDim.x) dst[w] = __ldcg(src + w);
    }
    __syncthreads();

    Acc<Real, NA, M::AMASK> acc;
    acc.zero();
    if (!K.bad && e > b) {
      EvalConsts<Real, NL> E;
      E.load(K);
      int64_t h = 0;
      if (vec) {
        uintptr_t a = reinterpret_cast<uintptr_t>(ev + (int64_t)P.col_obs[0] * stride + b);
        h = (int64_t)(((16u - (a & 15u)) & 15u) / sizeof(Col));
        if (h > e - b) h = e - b;
      }
      const int64_t nfull = (e - b - h) / EPT;
      stream_chunks<M, Real, Col, EPT>(P, E, ev, stride, b + h, threadIdx.x, blockDim.x, nfull,
                                       vec != 0, acc);
      if (threadIdx.x == blockDim.x - 1) {
        iterate_scalar<M, Real, Col>(P, E, ev, stride, b, b + h, acc);
        iterate_scalar<M, Real, Col>(P, E, ev, stride, b + h + nfull * EPT, e, acc);
      }
    }
    if (threadIdx.x == 0) load_meta();
    BlockReduce<Real, NA, M::AMASK>::run(acc, red, tot);
    if (threadIdx.x < NA) W.partials[tl * RF_NACC_MAX + threadIdx.x] = tot[threadIdx.x];
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
      int64_t r0 = __ldcg(W.tile_start + toy), r1 = __ldcg(W.tile_start + toy + 1);
      unsigned need = (unsigned)(r1 - r0);
      s_last = (atomicAdd(W.toy_counter + toy, 1u) == need - 1u) ? 1 : 0;
    }
    __syncthreads();
    if (s_last) {
      __threadfence();
      int64_t r0 = __ldcg(W.tile_start + toy), r1 = __ldcg(W.tile_start + toy + 1);
      rows_sum_few<NA>(W.partials, r0, r1, tot);
      if (threadIdx.x == 0) {
        int64_t ob = offsets[toy], oe = offsets[toy + 1];
        ob = ob < 0 ? 0 : (ob > stride ? stride : ob);
        oe = oe < ob ? ob : (oe > stride ? stride : oe);
        int64_t nt = oe - ob;
        double* row = out + toy * (int64_t)(1 + P.n_par);
        epilogue<Real, NL>(P, K, tot, nt, row, row + 1, W.status);
        W.toy_counter[toy] = 0u;
        if (adam_scale && isfinite(row[0])) {
          // Adam (Kingma & Ba 2015) in units of the toy's scale row
          const int step = *W.adam_t;
          const double b1 = 0.9, b2 = 0.999, eps = 1e-8;
          const double c1 = 1.0 - pow(b1, (double)step), c2 = 1.0 - pow(b2, (double)step);
          double* th = pm + toy * (int64_t)P.n_par;
          double* m1 = W.adam_m1 + toy * (int64_t)P.n_par;
          double* m2 = W.adam_m2 + toy * (int64_t)P.n_par;
          for (int p = 0; p < P.n_par; ++p) {
            bool fx = p < 64 ? ((P.fixed_lo >> p) & 1) : ((P.fixed_hi >> (p - 64)) & 1);
            if (fx) continue;
            const double sc = adam_scale[toy * (int64_t)P.n_par + p];
            double gsc = row[1 + p] * sc;
            m1[p] = b1 * m1[p] + (1.0 - b1) * gsc;
            m2[p] = b2 * m2[p] + (1.0 - b2) * gsc * gsc;
            double mh = m1[p] / c1, vh = m2[p] / c2;
            th[p] -= sc * adam_lr * mh / (sqrt(vh) + eps);
          }
        }
      }
    }
    __syncthreads();
  }
}

}  // namespace rf
