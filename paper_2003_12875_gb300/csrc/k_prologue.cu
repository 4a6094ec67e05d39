// The single-dataset FP64 prologue kernel (normalisation integrals, their
// derivatives and the coefficients), shared by the generic and the
// per-graph fused kernels.  One block of one warp per leaf.
#include "rf_kernels.cuh"

namespace rf {
template <typename Real>
__global__ void __launch_bounds__(32 * RF_MAXL) prologue_kernel(const RfProgram P,
                                                                const double* __restrict__ params,
                                                                RfWork W) {
  prologue_body<Real>(P, params, W);
}
}  // namespace rf

int rf_launch_prologue(const RfProgram& P, int eval, const double* params, RfWork W,
                       cudaStream_t st) {
  cudaLaunchConfig_t lc = {};
  lc.gridDim = dim3(1);
  lc.blockDim = dim3(32 * (P.n_leaves > 0 ? P.n_leaves : 1));
  lc.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  lc.attrs = at;
  lc.numAttrs = 1;
  if (eval) return (int)cudaLaunchKernelEx(&lc, rf::prologue_kernel<double>, P, params, W);
  return (int)cudaLaunchKernelEx(&lc, rf::prologue_kernel<float>, P, params, W);
}
