// The single-dataset FP64 prologue kernel (normalisation integrals, their
// derivatives and the coefficients), shared by the generic and the
// per-graph fused kernels.
#include "rf_kernels.cuh"

namespace rf {
template <typename Real>
__global__ void __launch_bounds__(32) prologue_kernel(const RfProgram P,
                                                      const double* __restrict__ params, RfWork W) {
  prologue_body<Real>(P, params, W);
}
}  // namespace rf

int rf_launch_prologue(const RfProgram& P, int eval, const double* params, RfWork W,
                       cudaStream_t st) {
  if (eval) rf::prologue_kernel<double><<<P.n_leaves, 32, 0, st>>>(P, params, W);
  else rf::prologue_kernel<float><<<P.n_leaves, 32, 0, st>>>(P, params, W);
  return (int)cudaGetLastError();
}
