// rf_batched.cuh -- many datasets (toys) of uneven size sharing one graph.
//
//  prep kernel      one thread per toy: the toy's FP64 normalisations and
//                   coefficients (RfConsts) from its parameter row; checks
//                   the toy's offsets.
//  segment kernel   the toys' events split evenly over the launch's warps;
//                   each warp writes one FP64 row per toy its range meets
//                   (launched as a programmatic dependent of the prep kernel);
//                   the warp that writes a toy's last row sums its rows in
//                   order and runs the FP64 epilogue (NLL, gradient),
//                   optionally one Adam step.
// Results depend only on the inputs and the launch shape, not on timing.
#pragma once
#include "rf_toys.cuh"

namespace rf {

// Prep kernel: blocks of n_leaves warps and 32 toys; warp k computes leaf k
// of every toy of the block (lane l: toy 32 b + l), so the leaves' FP64
// chains run side by side on different SM sub-partitions, then warp 0 checks
// the toys' offsets and combines.  Constants are written straight to the
// toy's global slot.  Lets the segment kernel launch at once.
template <typename Real>
__device__ __forceinline__ void toy_prep_body(const RfProgram& P, const double* __restrict__ pm,
                                              const int64_t* __restrict__ offsets,
                                              int32_t toys, int64_t n_events,
                                              RfConsts<Real>* consts, unsigned int* status,
                                              int32_t* adam_t, unsigned int* ticket) {
  asm volatile("griddepcontrol.launch_dependents;");
  __shared__ double lnI_s[RF_MAXL][32];
  __shared__ int ok_s[RF_MAXL][32];
  const int lane = threadIdx.x & 31, k = threadIdx.x >> 5;
  const int64_t t = (int64_t)blockIdx.x * 32 + lane;
  if (blockIdx.x == 0 && threadIdx.x == 0 && adam_t) *adam_t += 1;
  if (t < toys && k < P.n_leaves) {
    double l = 0.0;
    ok_s[k][lane] = leaf_consts(P, pm + t * P.n_par, consts[t], k, &l) ? 1 : 0;
    lnI_s[k][lane] = l;
  }
  __syncthreads();
  if (k == 0 && t < toys) {
    ticket[t] = 0u;  // rows of this call's segment kernel counted from zero
    const int64_t b = offsets[t], e = offsets[t + 1];
    if (b < 0 || e < b || e > n_events) atomicOr(status, RF_STATUS_NONFINITE_BIT);
    double l[RF_MAXL];
    bool all = true;
    for (int j = 0; j < P.n_leaves; ++j) {
      l[j] = lnI_s[j][lane];
      all &= ok_s[j][lane] != 0;
    }
    comb_consts(P, pm + t * P.n_par, consts[t], l, all);
  }
}

template <typename Real>
__global__ void toy_prep_kernel(const RfProgram P, const double* __restrict__ pm,
                                const int64_t* __restrict__ offsets, int32_t toys,
                                int64_t n_events, RfConsts<Real>* consts,
                                unsigned int* status, int32_t* adam_t, unsigned int* ticket) {
  toy_prep_body<Real>(P, pm, offsets, toys, n_events, consts, status, adam_t, ticket);
}

template <typename Real, typename Col, int NL, int EPT>
__global__ void __launch_bounds__(256)
    toy_segment_kernel(const RfProgram P, const Col* __restrict__ ev, int64_t stride, int vec,
                       const int64_t* __restrict__ offsets, int32_t toys, int stages, RfWork W) {
  toy_segment_body_reg<GenericModel<NL>, Real, Col, EPT>(P, ev, stride, vec, offsets, toys, stages,
                                                         W);
}

template <typename Real, typename Col, int NL, int EPT>
inline int launch_toys_nl(const RfProgram& P, int grid, int block, int vec, int stages,
                          size_t smem, const void* events, int64_t n_events,
                          const int64_t* offsets, int32_t toys, RfWork W, cudaStream_t st) {
  auto kern = toy_segment_kernel<Real, Col, NL, EPT>;  // register form: no shared memory
  (void)smem;
  cudaLaunchConfig_t lc = {};
  lc.gridDim = dim3(grid);
  lc.blockDim = dim3(block);
  lc.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  lc.attrs = at;
  lc.numAttrs = 1;
  return (int)cudaLaunchKernelEx(&lc, kern, P, static_cast<const Col*>(events), n_events, vec,
                                 offsets, toys, stages, W);
}

template <typename Real, typename Col, int EPT>
inline int launch_toys_ept(const RfProgram& P, int grid, int block, int vec, int stages,
                           size_t smem, const void* events, int64_t n_events,
                           const int64_t* offsets, int32_t toys, RfWork W, cudaStream_t st) {
  switch (P.n_leaves) {
    case 1: return launch_toys_nl<Real, Col, 1, EPT>(P, grid, block, vec, stages, smem, events, n_events, offsets, toys, W, st);
    case 2: return launch_toys_nl<Real, Col, 2, EPT>(P, grid, block, vec, stages, smem, events, n_events, offsets, toys, W, st);
    case 3: return launch_toys_nl<Real, Col, 3, EPT>(P, grid, block, vec, stages, smem, events, n_events, offsets, toys, W, st);
    case 4: return launch_toys_nl<Real, Col, 4, EPT>(P, grid, block, vec, stages, smem, events, n_events, offsets, toys, W, st);
  }
  return (int)cudaErrorInvalidValue;
}

}  // namespace rf
