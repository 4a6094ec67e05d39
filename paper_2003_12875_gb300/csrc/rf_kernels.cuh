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

template <typename T>
struct IsF32 {
  static constexpr bool v = false;
};
template <>
struct IsF32<float> {
  static constexpr bool v = true;
};

template <int NL>
struct GenericModel {
  static constexpr int NL_ = NL;
  static constexpr int NCOL = NL;
  static constexpr unsigned long long AMASK = ~0ull;

  // One event entirely in FP64 (FP32 evaluation of a call with a coefficient
  // exactly 0; x: the event's column values in their own precision): the same
  // formulas on the FP64 constants, the absent components' P_c/P from FP64
  // log-densities.  Adds the event's terms to q (FP32 sums) and returns
  // log2 P - beta_ref / ln 2.  Not inlined: it stays out of the event loops.
  static __device__ __noinline__ double event_exact(const RfExact* __restrict__ Kp,
                                                    const double* __restrict__ x,
                                                    float* __restrict__ q) {
    const RfExact& K = *Kp;
    double u[NL], g[NL][RF_LEAF_MAXP];
    int comp[NL], gms[NL];
#pragma unroll
    for (int k = 0; k < NL; ++k) {
      const int m = K.lmeta[k];
      gms[k] = (m >> 8) & 0xff;
      comp[k] = (m >> 16) & 0xff;
      eval_leaf<double>(m & 0xff, gms[k], x[(m >> 24) & 0xff], K.pcd[k], u[k], g[k]);
    }
    const int C = K.n_comp;
    double v[NL], w[NL], vm = -kInf();
#pragma unroll
    for (int c = 0; c < NL; ++c) {
      v[c] = c < C ? K.delta_d[c] : -kInf();
#pragma unroll
      for (int k = 0; k < NL; ++k)
        if (comp[k] == c) v[c] += u[k];
      vm = fmax(vm, v[c]);
    }
    double sw = 0.0;
#pragma unroll
    for (int c = 0; c < NL; ++c) {
      w[c] = c < C ? exp2(v[c] - vm) : 0.0;
      sw += w[c];
    }
    const double ell = vm + log2(sw);
    q[0] += (float)ell;
#pragma unroll
    for (int c = 0; c < NL; ++c) {
      if (c >= C) continue;
      w[c] /= sw;
      double vnc = K.delta_nc_d[c];
#pragma unroll
      for (int k = 0; k < NL; ++k)
        if (comp[k] == c) vnc += u[k];
      q[1 + c] += (float)(((K.zero_mask >> c) & 1) ? exp2(vnc - ell) : w[c]);
    }
#pragma unroll
    for (int k = 0; k < NL; ++k)
#pragma unroll
      for (int j = 0; j < RF_LEAF_MAXP; ++j)
        if ((gms[k] >> j) & 1) q[1 + NL + k * RF_LEAF_MAXP + j] += (float)(w[comp[k]] * g[k][j]);
    return ell;
  }

  // leaves -> components -> log-sum-exp -> adjoint weights, into q.
  // ANYZERO false: the caller knows no coefficient is zero (no per-event test)
  template <typename Real, bool ANYZERO = true>
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
      Real dv = v[1] - v[0];  // base-2 units, as everything per event
      Real e = F::ex2(-fabs(dv));
      Real s = Real(1) + e;
      Real rs = F::rcp(s);
      ell = fmax(v[0], v[1]) + F::lg2(s);
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
        w[c] = (c < C) ? F::ex2(v[c] - m) : Real(0);
        s += w[c];
      }
      ell = m + F::lg2(s);
      Real rs = F::rcp(s);
#pragma unroll
      for (int c = 0; c < NL; ++c) w[c] *= rs;
    }
    q[0] += ell;
    if (!ANYZERO || K.zero_mask == 0) {
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

// Chunk ch of EPT events per thread from event `base`: with 128-bit loads
// (vec) the EPT consecutive events base + ch*EPT ...; without (the columns do
// not share a 16-byte phase) the lanes of a warp interleave, so that each
// 32-bit load of the warp reads 32 consecutive events: lane l (= ch mod 32)
// of warp chunk ch/32 takes base + (ch/32)*32*EPT + l + 32 e.  Either way the
// chunks 0 .. nfull-1 cover [base, base + nfull*EPT) once (without vec, nfull
// is a multiple of 32).
template <int EPT>
__device__ __forceinline__ int64_t chunk_start(int64_t base, int64_t ch, bool vec) {
  return vec ? base + ch * EPT : base + (ch >> 5) * (32 * EPT) + (ch & 31);
}
template <int EPT>
__device__ __forceinline__ int64_t full_chunks(int64_t len, bool vec) {
  return vec ? len / EPT : (len / (32 * EPT)) * 32;
}

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
          // events are read once per call: streaming (evict-first) loads, so
          // they do not push the prologue's code and constants out of L2
          typename Vec<Col>::T t = __ldcs(vp + v);
          const Col* tc = reinterpret_cast<const Col*>(&t);
#pragma unroll
          for (int e = 0; e < W; ++e) x[c][v * W + e] = cvt<Real, Col>(tc[e]);
        }
      } else {
#pragma unroll
        for (int e = 0; e < EPT; ++e) x[c][e] = cvt<Real, Col>(__ldcs(col + 32 * e));
      }
    } else {
#pragma unroll
      for (int e = 0; e < EPT; ++e) x[c][e] = Real(0);
    }
  }
}

// A thread's running sums over the accumulators in MASK (the others stay
// zero and generate no instructions).  The log-likelihood sum (accumulator 0,
// held to the tighter NLL bound) is Kahan-compensated (value = s - c); the
// weight and gradient sums, whose bound is relative to the sum of the terms'
// magnitudes, are plain sums of the per-chunk partials (c stays 0).
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
      if (i == 0) {
        Real y = q[i] - c[i];
        Real t = s[i] + y;
        c[i] = (t - s[i]) - y;
        s[i] = t;
      } else {
        s[i] += q[i];
      }
    }
  }
  __device__ __forceinline__ double value(int i) const {
    return ((MASK >> i) & 1ull) ? (double)s[i] - (double)c[i] : 0.0;
  }
};

// A block's row of partial sums, in FP64.  FP32 evaluation: the per-thread
// Kahan sums are added over the block in FP32 pairs (TwoSum; about 48
// significant bits, the FP64 pipe of this GPU is narrow), and each of the
// block's pair totals is converted to FP64 once, when the row is written (a
// few FP64 instructions per block).  FP64 evaluation: FP64 throughout.  red:
// shared, 32 * NA doubles.
template <typename Real, int NA, unsigned long long MASK>
struct BlockRow;
template <int NA, unsigned long long MASK>
struct BlockRow<float, NA, MASK> {
  static __device__ __forceinline__ void write(const Acc<float, NA, MASK>& acc, double* red,
                                               double* row) {
    __shared__ float2 pr[NA];
    float ls[NA];
#pragma unroll
    for (int i = 0; i < NA; ++i) ls[i] = -acc.c[i];  // Kahan keeps -(lost low part)
    block_sum_ds2<NA, MASK>(acc.s, ls, reinterpret_cast<float2*>(red), pr);
    if (threadIdx.x < NA)
      row[threadIdx.x] = ((MASK >> threadIdx.x) & 1ull)
                             ? (double)pr[threadIdx.x].x + (double)pr[threadIdx.x].y
                             : 0.0;
  }
};
template <int NA, unsigned long long MASK>
struct BlockRow<double, NA, MASK> {
  static __device__ __forceinline__ void write(const Acc<double, NA, MASK>& acc, double* red,
                                               double* row) {
    __shared__ double bt[NA];
    double val[NA];
#pragma unroll
    for (int i = 0; i < NA; ++i) val[i] = acc.value(i);
    block_sum_m<NA, MASK>(val, red, bt);
    if (threadIdx.x < NA) row[threadIdx.x] = bt[threadIdx.x];
  }
};

// The grid's FP64 tree over the block rows (see RF_TREE_GROUPS): called by
// every block after its row is written; returns true in the one block that
// holds the grid totals in tot[0..NA) (shared) afterwards.  The groups are
// contiguous runs of gsz rows; each level sums its rows in a fixed order, so
// the totals depend only on the grid size.  A grid of at most RF_TREE_GROUPS
// blocks has one level: its last block sums the block rows (a first level of
// one-row groups would only add a ticket and its fences to a short call).
// Each ticket is reset by the block that takes its last number.
template <int NA, unsigned long long MASK>
__device__ __forceinline__ bool grid_tree(double* partials, unsigned int* counter, double* red,
                                          double* tot) {
  __shared__ int s_last;
  const int64_t G = gridDim.x;
  if (G <= RF_TREE_GROUPS) {
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
      const bool last = atomicAdd(counter, 1u) == (unsigned)(G - 1);
      if (last) *counter = 0u;
      s_last = last ? 1 : 0;
    }
    __syncthreads();
    if (!s_last) return false;
    __threadfence();
    rows_tree<NA, MASK>(partials, 0, G, red, tot);
    return true;
  }
  const int64_t gsz = (G + RF_TREE_GROUPS - 1) / RF_TREE_GROUPS;
  const int64_t ng = (G + gsz - 1) / gsz;
  const int64_t g = blockIdx.x / gsz;
  const int64_t r0 = g * gsz, r1 = (r0 + gsz < G) ? r0 + gsz : G;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned int* tk = counter + RF_TREE_GROUPS + g;
    const bool last = atomicAdd(tk, 1u) == (unsigned)(r1 - r0 - 1);
    if (last) *tk = 0u;
    s_last = last ? 1 : 0;
  }
  __syncthreads();
  if (!s_last) return false;
  __threadfence();
  rows_tree<NA, MASK>(partials, r0, r1, red, tot);
  if (threadIdx.x < NA) partials[(G + g) * RF_NACC_MAX + threadIdx.x] = tot[threadIdx.x];
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const bool last = atomicAdd(counter, 1u) == (unsigned)(ng - 1);
    if (last) *counter = 0u;
    s_last = last ? 1 : 0;
  }
  __syncthreads();
  if (!s_last) return false;
  __threadfence();
  rows_tree<NA, MASK>(partials, G, G + ng, red, tot);
  return true;
}

// EPT events already in registers -> the iteration's partial sums -> acc.
template <class M, typename Real, int EPT, bool ANYZERO>
__device__ __forceinline__ void compute_full(const RfProgram& P,
                                             const EvalConsts<Real, M::NL_>& K,
                                             const Real (&x)[M::NL_][EPT],
                                             Acc<Real, RF_NACC(M::NL_), M::AMASK>& acc) {
  constexpr int NL = M::NL_;
  // -0: the first event's additions fold into moves (x + -0 == x)
  Real q[RF_NACC(NL)];
#pragma unroll
  for (int i = 0; i < RF_NACC(NL); ++i) q[i] = Real(-0.0);
#pragma unroll
  for (int e = 0; e < EPT; ++e) {
    Real xc[NL];
#pragma unroll
    for (int c = 0; c < NL; ++c) xc[c] = x[c][e];
    M::template event<Real, ANYZERO>(P, K, xc, q);
  }
  acc.add(q);
}

// Chunks first, first+step, ... < nfull of EPT events each (chunk c starts at
// event base + c*EPT).  The next chunk's 128-bit loads are issued before the
// current chunk is computed (register double buffering), so the memory
// latency overlaps the arithmetic.  ANYZERO: some coefficient may be exactly
// zero (the per-event code then tests for it); the callers pick the variant
// once from the call's constants.
template <class M, typename Real, typename Col, int EPT, bool ANYZERO = true>
__device__ __forceinline__ void stream_chunks(const RfProgram& P,
                                              const EvalConsts<Real, M::NL_>& K,
                                              const Col* __restrict__ ev, int64_t stride,
                                              int64_t base, int64_t first, int64_t step,
                                              int64_t nfull, bool vec,
                                              Acc<Real, RF_NACC(M::NL_), M::AMASK>& acc) {
  constexpr int NL = M::NL_;
  if (first >= nfull) return;
  // two register buffers used in turn (unrolled by two, so no buffer is
  // copied into the other)
  Real xa[NL][EPT], xb[NL][EPT];
  load_full<Real, Col, NL, M::NCOL, EPT>(P, ev, stride, chunk_start<EPT>(base, first, vec), vec,
                                         xa);
  for (int64_t ch = first;;) {
    const int64_t nb = ch + step;
    if (nb >= nfull) {
      compute_full<M, Real, EPT, ANYZERO>(P, K, xa, acc);
      break;
    }
    load_full<Real, Col, NL, M::NCOL, EPT>(P, ev, stride, chunk_start<EPT>(base, nb, vec), vec,
                                           xb);
    compute_full<M, Real, EPT, ANYZERO>(P, K, xa, acc);
    const int64_t na = nb + step;
    if (na >= nfull) {
      compute_full<M, Real, EPT, ANYZERO>(P, K, xb, acc);
      break;
    }
    load_full<Real, Col, NL, M::NCOL, EPT>(P, ev, stride, chunk_start<EPT>(base, na, vec), vec,
                                           xa);
    compute_full<M, Real, EPT, ANYZERO>(P, K, xb, acc);
    ch = na;
  }
}

// Events i0, i0 + step, ... < i1 through the model's FP64 event (FP32
// evaluation of a call or toy with a coefficient exactly 0), the column
// values read in their own precision.
template <class M, typename Col>
__device__ inline void iterate_exact(const RfProgram& P, const EvalConsts<float, M::NL_>& K,
                                     const Col* __restrict__ ev, int64_t stride, int64_t i0,
                                     int64_t i1, int64_t step,
                                     Acc<float, RF_NACC(M::NL_), M::AMASK>& acc) {
  constexpr int NL = M::NL_;
  for (int64_t i = i0; i < i1; i += step) {
    double x[NL];
#pragma unroll
    for (int c = 0; c < NL; ++c)
      x[c] = (c < M::NCOL && c < P.n_cols) ? (double)ev[(int64_t)P.col_obs[c] * stride + i] : 0.0;
    float q[RF_NACC(NL)];
#pragma unroll
    for (int j = 0; j < RF_NACC(NL); ++j) q[j] = 0.f;
    M::event_exact(K.full, x, q);
    acc.add(q);
  }
}

template <class M, typename Real, typename Col>
__device__ inline void iterate_scalar(const RfProgram& P, const EvalConsts<Real, M::NL_>& K,
                                      const Col* __restrict__ ev, int64_t stride, int64_t i0,
                                      int64_t i1, Acc<Real, RF_NACC(M::NL_), M::AMASK>& acc,
                                      int step = 1) {
  constexpr int NL = M::NL_;
  if constexpr (IsF32<Real>::v) {
    if (K.zero_mask != 0) {
      iterate_exact<M, Col>(P, K, ev, stride, i0, i1, step, acc);
      return;
    }
  }
  for (int64_t i = i0; i < i1; i += step) {
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

// Prologue of one block.  The FP64 unit of an SM sub-partition takes one warp
// instruction about every 64 cycles, whatever the number of active lanes, so
// a chain's length is its instruction count: the work is cut into
// independent tasks on separate warps (sub-partitions), and like functions go
// on separate lanes of one instruction.  Task k < L: leaf k's integral on
// lanes 0-1 (leaf_norm_pair); task L + k: leaf k's per-event constants on
// lane 0; task 2L: the coefficients, their logs one per lane (CoefPre).  Warps take tasks
// round robin (warp w: tasks w, w + warps, ...), so any block of 32 threads
// or more works; 2L + 1 warps run them all at once.  Then lanes 0-7 of warp 0
// combine, one component per lane (no transcendental function left there).
template <typename Real>
__device__ inline void block_prologue(const RfProgram& P, const double* params,
                                      RfConsts<Real>& K, double* lnI, int* ok,
                                      RfExact* X = nullptr) {
  __shared__ CoefPre cpre;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
  const int NL = P.n_leaves, ntask = 2 * NL + 1;
  for (int task = wid; task < ntask; task += nw) {
    if (task < NL) {
      if (lane < 2) {
        double l = 0.0;
        const bool o = leaf_norm_pair(P, params, K, task, &l);
        if (lane == 0) {
          ok[task] = o ? 1 : 0;
          lnI[task] = l;
        }
      }
    } else if (task < 2 * NL) {
      if (lane == 0) leaf_eval_consts(P, params, K, task - NL);
    } else {
      coef_pre_lanes(P, params, lane, &cpre);
    }
  }
  __syncthreads();
  if (wid == 0) {
    bool all = true;
    for (int k = 0; k < NL; ++k) all &= ok[k] != 0;
    comb_consts_group<Real, 8>(P, params, K, lnI, 1, all, X, &cpre, lane < 8);
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
  __shared__ RfExact Xs;  // FP64 constants when the block builds its own

  const RfExact* X = W.consts_x;
  // A product root (one component, coefficient 1) whose leaves need nothing
  // from the normalisation kernel: the event pass uses only the leaves'
  // per-event constants (a few FP64 divisions), so every block builds those
  // itself and streams at once, beside the prologue.  The integrals and the
  // combination enter only the epilogue: each block waits for the prologue
  // before it writes its row (the prologue has itself waited for the
  // previous call's grid, which is then done with the rows and tickets), and
  // the block that finishes the tree loads the prologue's constants.
  const bool early = W.consts && P.kind == RF_KIND_PROD && !P.formula_norm;
  if (early) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nw = (blockDim.x + 31) >> 5;
    for (int k = wid; k < P.n_leaves; k += nw)
      if (lane == 0) leaf_eval_consts(P, params, K, k);
    if (threadIdx.x < RF_MAXC) {
      K.delta[threadIdx.x] = Real(0);
      K.delta_nc[threadIdx.x] = Real(0);
    }
    if (threadIdx.x == 0) {
      K.zero_mask = 0;
      K.bad = 0;
    }
    __syncthreads();
    // the next call's prologue may start (it publishes new constants only
    // after this grid has finished)
    asm volatile("griddepcontrol.launch_dependents;");
  } else if (W.consts) {
    // constants from the prologue kernel, which this launch may overlap:
    // wait for it (a no-op when this grid was not launched as its dependent)
    asm volatile("griddepcontrol.wait;" ::: "memory");
    constexpr int kWords = (int)(sizeof(RfConsts<Real>) / sizeof(double));
    const double* src = static_cast<const double*>(W.consts);
    double* dst = reinterpret_cast<double*>(&K);
    for (int w = threadIdx.x; w < kWords; w += blockDim.x) dst[w] = __ldcg(src + w);
    __syncthreads();
    // the constants are in shared memory: the next call's prologue may start
    // (it publishes new constants only after this grid has finished)
    asm volatile("griddepcontrol.launch_dependents;");
  } else {
    block_prologue(P, params, K, lnI, ok, &Xs);
    X = &Xs;
  }

  Acc<Real, NA, M::AMASK> acc;
  acc.zero();
  if (!K.bad) {
    EvalConsts<Real, NL> E;
    E.load(K, X);
    const int64_t h = head < n ? head : n;
    const int64_t nfull = full_chunks<EPT>(n - h, vec != 0);
    const int64_t gsz = (int64_t)gridDim.x * blockDim.x;
    const int64_t first = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    bool exact = false;
    if constexpr (IsF32<Real>::v) {
      // a coefficient exactly 0: every event in FP64 (rare; speed is no aim)
      if (E.zero_mask != 0) {
        iterate_exact<M, Col>(P, E, ev, n, first, n, gsz, acc);
        exact = true;
      }
    }
    if (!exact) {
      if (E.zero_mask == 0)
        stream_chunks<M, Real, Col, EPT, false>(P, E, ev, n, h, first, gsz, nfull, vec != 0, acc);
      else
        stream_chunks<M, Real, Col, EPT, true>(P, E, ev, n, h, first, gsz, nfull, vec != 0, acc);
      // the events before the first aligned one and after the last full
      // chunk: at most one each per thread, coalesced
      iterate_scalar<M, Real, Col>(P, E, ev, n, first, h, acc, (int)gsz);
      iterate_scalar<M, Real, Col>(P, E, ev, n, h + nfull * EPT + first, n, acc, (int)gsz);
    }
  }

  if (early) asm volatile("griddepcontrol.wait;" ::: "memory");
  BlockRow<Real, NA, M::AMASK>::write(acc, red, W.partials + (int64_t)blockIdx.x * RF_NACC_MAX);
  if (grid_tree<NA, M::AMASK>(W.partials, W.counter, red, tot)) {
    if (early) {  // the prologue's constants (integrals, combination)
      constexpr int kWords = (int)(sizeof(RfConsts<Real>) / sizeof(double));
      const double* src = static_cast<const double*>(W.consts);
      double* dst = reinterpret_cast<double*>(&K);
      for (int w = threadIdx.x; w < kWords; w += blockDim.x) dst[w] = __ldcg(src + w);
      __syncthreads();
    }
    if (threadIdx.x < 32) epilogue_warp<Real, NL>(P, K, tot, n, nll, grad, W.status);
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
  __shared__ RfExact Xs;
  block_prologue(P, params, K, lnI, ok, &Xs);
  EvalConsts<Real, NL> E;
  E.load(K, &Xs);
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
    if constexpr (IsF32<Real>::v) {
      if (E.zero_mask != 0) {  // FP64 event, as in the NLL kernels
        double xd[NL];
#pragma unroll
        for (int c = 0; c < NL; ++c)
          xd[c] = (c < M::NCOL && c < P.n_cols) ? (double)ev[(int64_t)P.col_obs[c] * n + i] : 0.0;
        const double ell = M::event_exact(E.full, xd, q);
        logp[i] = K.bad ? kNaN() : K.beta_ref + kLn2 * ell;
        continue;
      }
    }
    M::template event<Real>(P, E, xc, q);
    logp[i] = K.bad ? kNaN() : K.beta_ref + kLn2 * (double)q[0];
  }
}

}  // namespace rf
