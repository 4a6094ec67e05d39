// rf_batched.cuh -- many datasets (toys) of uneven size sharing one graph.
//
//  plan kernel     (k_toys_common.cu) offsets -> tile_start (exclusive scan of ceil(n_t / T),
//                  at least one tile per toy so that empty toys still get
//                  their extended term); one block.
//  prep kernel     one thread per toy: the toy's FP64 normalisations and
//                  coefficients (RfConsts) from its parameter row.
//  tile kernel     persistent blocks take tiles from an atomic counter; a tile
//                  holds events of one toy only; its block partial goes to
//                  partials[tile]; the last tile of a toy to finish (per-toy
//                  ticket) sums that toy's tiles in tile order and writes
//                  (NLL, grad) -- optionally followed by one Adam step on the
//                  toy's parameter row.
// Results do not depend on which block ran which tile.
#pragma once
#include "rf_kernels.cuh"

namespace rf {

template <typename Real>
__global__ void toy_prep_kernel(const RfProgram P, const double* __restrict__ pm,
                                int32_t toys, RfConsts<Real>* consts,
                                unsigned int* next_tile, int32_t* adam_t) {
  toy_prep_body<Real>(P, pm, toys, consts, next_tile, adam_t);
}

template <typename Real, typename Col, int NL, int EPT>
__global__ void __launch_bounds__(256)
    toy_tile_kernel(const RfProgram P, const Col* __restrict__ ev, int64_t stride,
                    int vec, const int64_t* __restrict__ offsets, int32_t toys,
                    int64_t tile_ev, double* pm, double* out, RfWork W,
                    const double* __restrict__ adam_scale, double adam_lr,
                    int64_t max_rows) {
  toy_tile_body<GenericModel<NL>, Real, Col, EPT>(P, ev, stride, vec, offsets, toys, tile_ev,
                                                  pm, out, W, adam_scale, adam_lr, max_rows);
}

template <typename Real, typename Col, int NL, int EPT>
inline int launch_toys_nl(const RfProgram& P, const RfLaunchCfg& cfg, int num_sms,
                          const void* events, int64_t n_events, const int64_t* offsets,
                          int32_t toys, double* pm, double* out, RfWork W,
                          const double* adam_scale, double adam_lr, int64_t max_rows,
                          cudaStream_t st) {
  int vec;
  int64_t head;
  // tiles start anywhere: vector loads need every column at the same phase
  {
    const uintptr_t base = reinterpret_cast<uintptr_t>(events);
    uintptr_t ph0 = 0;
    bool same = true;
    for (int c = 0; c < P.n_cols; ++c) {
      uintptr_t a = base + (uintptr_t)((int64_t)P.col_obs[c] * n_events * (int64_t)sizeof(Col));
      if (c == 0) ph0 = a & 15u;
      else if ((a & 15u) != ph0) same = false;
    }
    vec = (same && ph0 % sizeof(Col) == 0) ? 1 : 0;
    head = 0;
    (void)head;
  }
  int grid = num_sms * cfg.blocks_per_sm;
  toy_tile_kernel<Real, Col, NL, EPT><<<grid, cfg.block, 0, st>>>(
      P, static_cast<const Col*>(events), n_events, vec, offsets, toys, cfg.tile, pm,
      out, W, adam_scale, adam_lr, max_rows);
  return (int)cudaGetLastError();
}

template <typename Real, typename Col, int EPT>
inline int launch_toys_ept(const RfProgram& P, const RfLaunchCfg& cfg, int num_sms,
                           const void* events, int64_t n_events, const int64_t* offsets,
                           int32_t toys, double* pm, double* out, RfWork W,
                           const double* adam_scale, double adam_lr, int64_t max_rows,
                           cudaStream_t st) {
  switch (P.n_leaves) {
    case 1: return launch_toys_nl<Real, Col, 1, EPT>(P, cfg, num_sms, events, n_events, offsets, toys, pm, out, W, adam_scale, adam_lr, max_rows, st);
    case 2: return launch_toys_nl<Real, Col, 2, EPT>(P, cfg, num_sms, events, n_events, offsets, toys, pm, out, W, adam_scale, adam_lr, max_rows, st);
    case 3: return launch_toys_nl<Real, Col, 3, EPT>(P, cfg, num_sms, events, n_events, offsets, toys, pm, out, W, adam_scale, adam_lr, max_rows, st);
    case 4: return launch_toys_nl<Real, Col, 4, EPT>(P, cfg, num_sms, events, n_events, offsets, toys, pm, out, W, adam_scale, adam_lr, max_rows, st);
  }
  return (int)cudaErrorInvalidValue;
}

}  // namespace rf
