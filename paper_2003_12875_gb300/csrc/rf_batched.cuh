// rf_batched.cuh -- many datasets (toys) of uneven size sharing one graph.
//
//  prep kernel      one thread per toy: the toy's FP64 normalisations and
//                   coefficients (RfConsts) from its parameter row; checks
//                   the toy's offsets.
//  segment kernel   the toys' events split evenly over the launch's warps;
//                   each warp writes one FP64 row per toy its range meets
//                   (launched as a programmatic dependent of the prep kernel).
//  finalize kernel  one warp per toy: its rows summed in order, the FP64
//                   epilogue (NLL, gradient), optionally one Adam step.
// Results depend only on the inputs and the launch shape, not on timing.
#pragma once
#include "rf_kernels.cuh"

namespace rf {

template <typename Real>
__global__ void toy_prep_kernel(const RfProgram P, const double* __restrict__ pm,
                                const int64_t* __restrict__ offsets, int32_t toys,
                                int64_t n_events, RfConsts<Real>* consts,
                                unsigned int* status, int32_t* adam_t) {
  toy_prep_body<Real>(P, pm, offsets, toys, n_events, consts, status, adam_t);
}

template <typename Real, typename Col, int NL, int EPT>
__global__ void __launch_bounds__(256)
    toy_segment_kernel(const RfProgram P, const Col* __restrict__ ev, int64_t stride, int vec,
                       const int64_t* __restrict__ offsets, int32_t toys, int stages, RfWork W) {
  toy_segment_body<GenericModel<NL>, Real, Col, EPT>(P, ev, stride, vec, offsets, toys, stages, W);
}

template <typename Real, int NL>
__global__ void __launch_bounds__(256)
    toy_finalize_kernel(const RfProgram P, const int64_t* __restrict__ offsets, int32_t toys,
                        int64_t stride, int64_t warps, double* pm, double* out, RfWork W,
                        const double* __restrict__ adam_scale, double adam_lr) {
  toy_finalize_body<Real, NL>(P, offsets, toys, stride, warps, pm, out, W, adam_scale, adam_lr);
}

template <typename Real, typename Col, int NL, int EPT>
inline int launch_toys_nl(const RfProgram& P, int grid, int block, int vec, int stages,
                          size_t smem, const void* events, int64_t n_events,
                          const int64_t* offsets, int32_t toys, RfWork W, cudaStream_t st) {
  auto kern = toy_segment_kernel<Real, Col, NL, EPT>;
  static bool sized = false;  // opt in to more than 48 KB of dynamic shared memory once
  if (!sized) {
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
    sized = true;
  }
  cudaLaunchConfig_t lc = {};
  lc.gridDim = dim3(grid);
  lc.blockDim = dim3(block);
  lc.dynamicSmemBytes = smem;
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
