// rf_fused.cuh -- the precompiled (generic-model) single-dataset kernels and
// their host-side launch helpers.  The fused kernel: FP64 prologue (leaf
// normalisations and coefficients, once per block), a grid-stride loop over
// the events with 128-bit coalesced loads of the SoA columns, the per-event
// log-density and adjoint in registers, compensated per-thread sums, and a
// deterministic FP64 reduction finished by the last block to arrive, which
// writes the NLL and its gradient.  One launch per call; no host sync.
#pragma once
#include "rf_kernels.cuh"

namespace rf {

template <typename Real, typename Col, int NL, int EPT>
__global__ void __launch_bounds__(256)
    fused_nll_kernel(const RfProgram P, const Col* __restrict__ ev, int64_t n,
                     int64_t head, int vec, const double* __restrict__ params,
                     RfWork W, double* nll, double* grad) {
  fused_body<GenericModel<NL>, Real, Col, EPT>(P, ev, n, head, vec, params, W, nll, grad);
}

template <typename Real, typename Col, int NL>
__global__ void __launch_bounds__(256)
    logp_kernel(const RfProgram P, const Col* __restrict__ ev, int64_t n,
                const double* __restrict__ params, double* logp) {
  logp_body<GenericModel<NL>, Real, Col>(P, ev, n, params, logp);
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
  cudaLaunchConfig_t lc = {};
  lc.gridDim = dim3(grid);
  lc.blockDim = dim3(cfg.block);
  lc.stream = st;
  cudaLaunchAttribute at[1];
  if (W.consts) {  // dependent of the prologue kernel launched just before
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    lc.attrs = at;
    lc.numAttrs = 1;
  }
  const Col* ev = static_cast<const Col*>(events);
  return (int)cudaLaunchKernelEx(&lc, fused_nll_kernel<Real, Col, NL, EPT>, P, ev, n, head, vec,
                                 params, W, nll, grad);
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
