// rf_fused.cuh -- the fused single-dataset kernel: FP64 prologue (leaf
// normalisations and coefficients, once per block), a grid-stride loop over
// the events with 128-bit coalesced loads of the SoA columns, the per-event
// log-density and adjoint in registers, compensated per-thread sums, and a
// deterministic FP64 reduction finished by the last block to arrive, which
// writes the NLL and its gradient.  One launch per call; no host sync.
#pragma once
#include "rf_device.cuh"

namespace rf {

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

template <typename Real, typename Col, int NL, int EPT>
__global__ void __launch_bounds__(256)
    fused_nll_kernel(const RfProgram P, const Col* __restrict__ ev, int64_t n,
                     int64_t head, int vec, const double* __restrict__ params,
                     RfWork W, double* nll, double* grad) {
  constexpr int NA = RF_NACC(NL);
  __shared__ RfConsts<Real> K;
  __shared__ double lnI[RF_MAXL];
  __shared__ int ok[RF_MAXL];
  __shared__ double red[32 * NA];
  __shared__ double tot[NA];
  __shared__ int s_last;

  block_prologue(P, params, K, lnI, ok);

  Acc<Real, NA> acc;
  acc.zero();
  if (!K.bad) {
    EvalConsts<Real, NL> E;
    E.load(K);
    const int64_t h = head < n ? head : n;
    const int64_t nfull = (n - h) / EPT;
    const int64_t gsz = (int64_t)gridDim.x * blockDim.x;
    for (int64_t ch = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; ch < nfull; ch += gsz)
      iterate_full<Real, Col, NL, EPT>(P, E, ev, n, h + ch * EPT, vec != 0, acc);
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == blockDim.x - 1) {
      iterate_scalar<Real, Col, NL>(P, E, ev, n, 0, h, acc);
      iterate_scalar<Real, Col, NL>(P, E, ev, n, h + nfull * EPT, n, acc);
    }
  }

  double val[NA];
#pragma unroll
  for (int i = 0; i < NA; ++i) val[i] = (double)acc.s[i] - (double)acc.c[i];
  block_sum<NA>(val, red, tot);
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
template <typename Real, typename Col, int NL>
__global__ void __launch_bounds__(256)
    logp_kernel(const RfProgram P, const Col* __restrict__ ev, int64_t n,
                const double* __restrict__ params, double* logp) {
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
      xc[c] = (c < P.n_cols) ? (Real)ev[(int64_t)P.col_obs[c] * n + i] : Real(0);
    Real q[NA];
#pragma unroll
    for (int j = 0; j < NA; ++j) q[j] = Real(0);
    event_accumulate<Real, NL>(P, E, xc, q);
    logp[i] = K.bad ? CUDART_NAN : K.beta_ref + (double)q[0];
  }
}

// Vector path if every column read shares one 16-byte phase; head = events
// before the first aligned one.
template <typename Col>
inline void vec_plan(const RfProgram& P, const void* events, int64_t stride,
                     int* vec, int64_t* head) {
  const uintptr_t base = reinterpret_cast<uintptr_t>(events);
  uintptr_t ph0 = 0;
  bool same = true;
  for (int c = 0; c < P.n_cols; ++c) {
    uintptr_t a = base + (uintptr_t)((int64_t)P.col_obs[c] * stride * (int64_t)sizeof(Col));
    uintptr_t ph = a & 15u;
    if (c == 0) ph0 = ph;
    else if (ph != ph0) same = false;
  }
  if (same && (ph0 % sizeof(Col)) == 0) {
    *vec = 1;
    *head = (int64_t)(((16u - ph0) & 15u) / sizeof(Col));
  } else {
    *vec = 0;
    *head = 0;
  }
}

inline int grid_for(int64_t work_items, int block, int num_sms, int bps) {
  int64_t want = (work_items + block - 1) / block;
  int64_t cap = (int64_t)num_sms * bps;
  if (want > cap) want = cap;
  if (want < 1) want = 1;
  return (int)want;
}

template <typename Real, typename Col, int NL, int EPT>
inline int launch_fused_nl(const RfProgram& P, const RfLaunchCfg& cfg, int num_sms,
                           const void* events, int64_t n, const double* params,
                           RfWork W, double* nll, double* grad, cudaStream_t st) {
  int vec;
  int64_t head;
  vec_plan<Col>(P, events, n, &vec, &head);
  int64_t chunks = n / EPT;
  int grid = grid_for(chunks, cfg.block, num_sms, cfg.blocks_per_sm);
  fused_nll_kernel<Real, Col, NL, EPT><<<grid, cfg.block, 0, st>>>(
      P, static_cast<const Col*>(events), n, head, vec, params, W, nll, grad);
  return (int)cudaGetLastError();
}

template <typename Real, typename Col, int EPT>
inline int launch_fused_ept(const RfProgram& P, const RfLaunchCfg& cfg, int num_sms,
                            const void* events, int64_t n, const double* params,
                            RfWork W, double* nll, double* grad, cudaStream_t st) {
  switch (P.n_leaves) {
    case 1: return launch_fused_nl<Real, Col, 1, EPT>(P, cfg, num_sms, events, n, params, W, nll, grad, st);
    case 2: return launch_fused_nl<Real, Col, 2, EPT>(P, cfg, num_sms, events, n, params, W, nll, grad, st);
    case 3: return launch_fused_nl<Real, Col, 3, EPT>(P, cfg, num_sms, events, n, params, W, nll, grad, st);
    case 4: return launch_fused_nl<Real, Col, 4, EPT>(P, cfg, num_sms, events, n, params, W, nll, grad, st);
  }
  return (int)cudaErrorInvalidValue;
}

template <typename Real, typename Col>
inline int launch_logp_T(const RfProgram& P, const void* events, int64_t n,
                         const double* params, double* logp, cudaStream_t st) {
  int grid = (int)((n + 255) / 256);
  if (grid < 1) grid = 1;
  if (grid > 65535 * 8) grid = 65535 * 8;
  const Col* e = static_cast<const Col*>(events);
  switch (P.n_leaves) {
    case 1: logp_kernel<Real, Col, 1><<<grid, 256, 0, st>>>(P, e, n, params, logp); break;
    case 2: logp_kernel<Real, Col, 2><<<grid, 256, 0, st>>>(P, e, n, params, logp); break;
    case 3: logp_kernel<Real, Col, 3><<<grid, 256, 0, st>>>(P, e, n, params, logp); break;
    case 4: logp_kernel<Real, Col, 4><<<grid, 256, 0, st>>>(P, e, n, params, logp); break;
    default: return (int)cudaErrorInvalidValue;
  }
  return (int)cudaGetLastError();
}

}  // namespace rf
