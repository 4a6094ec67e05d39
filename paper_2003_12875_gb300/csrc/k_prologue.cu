// The single-dataset FP64 prologue kernel (normalisation integrals, their
// derivatives and the coefficients), shared by the generic and the
// per-graph fused kernels.  One block of 2 n_leaves + 1 warps (block_prologue's
// tasks, all at once).
#include "rf_kernels.cuh"

namespace rf {
// Single-dataset prologue: one block; each leaf's integral, each leaf's
// per-event constants and the coefficients' logs on warps of their own (the
// FP64 chains run on different SM sub-partitions), thread 0 combines, all in
// shared memory.  It lets its dependent (the fused
// kernel) launch at once, and it is itself launched as a programmatic
// dependent of the previous kernel in the stream: when that is the previous
// call's fused kernel, this FP64 work overlaps it, and the wait before the
// constants are published keeps that kernel's readers safe.
template <typename Real>
__device__ __forceinline__ void prologue_body(const RfProgram& P, const double* __restrict__ params,
                                              RfWork& W) {
  asm volatile("griddepcontrol.launch_dependents;");
  __shared__ RfConsts<Real> K;
  __shared__ double lnI[RF_MAXL];
  __shared__ int ok[RF_MAXL];
  __shared__ RfExact Xs;
  // formula leaves: their integrals come from the normalisation kernel just
  // before, so wait for it first
  if (P.formula_norm) asm volatile("griddepcontrol.wait;" ::: "memory");
  block_prologue(P, params, K, lnI, ok, &Xs);
  asm volatile("griddepcontrol.wait;" ::: "memory");
  constexpr int kWords = (int)(sizeof(RfConsts<Real>) / sizeof(double));
  const double* src = reinterpret_cast<const double*>(&K);
  double* dst = static_cast<double*>(W.consts);
  for (int w = threadIdx.x; w < kWords; w += blockDim.x) dst[w] = src[w];
  if (sizeof(Real) == 4 && K.zero_mask != 0 && W.consts_x) {
    constexpr int kx = (int)(sizeof(RfExact) / sizeof(double));
    const double* xs = reinterpret_cast<const double*>(&Xs);
    double* xd = reinterpret_cast<double*>(W.consts_x);
    for (int w = threadIdx.x; w < kx; w += blockDim.x) xd[w] = xs[w];
  }
}

template <typename Real>
__global__ void __launch_bounds__(32 * (2 * RF_MAXL + 1)) prologue_kernel(const RfProgram P,
                                                                const double* __restrict__ params,
                                                                RfWork W) {
  prologue_body<Real>(P, params, W);
}
}  // namespace rf

int rf_launch_prologue(const RfProgram& P, int eval, const double* params, RfWork W,
                       bool chain, cudaStream_t st) {
  cudaLaunchConfig_t lc = {};
  lc.gridDim = dim3(1);
  lc.blockDim = dim3(32 * (2 * (P.n_leaves > 0 ? P.n_leaves : 1) + 1));
  lc.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  lc.attrs = chain ? at : nullptr;
  lc.numAttrs = chain ? 1 : 0;
  if (eval) return (int)cudaLaunchKernelEx(&lc, rf::prologue_kernel<double>, P, params, W);
  return (int)cudaLaunchKernelEx(&lc, rf::prologue_kernel<float>, P, params, W);
}
