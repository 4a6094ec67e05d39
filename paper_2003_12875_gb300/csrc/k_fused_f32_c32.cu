// Fused single-dataset kernels: float per-event arithmetic, float columns.
#include "rf_fused.cuh"

int rf_fused_f32_c32(const RfProgram& P, const RfLaunchCfg& cfg, int sms,
                      const void* ev, int64_t n, const double* params, RfWork W,
                      double* nll, double* grad, cudaStream_t st) {
  if (cfg.ept == 8)
    return rf::launch_fused_ept<float, float, 8>(P, cfg, sms, ev, n, params, W, nll, grad, st);
  return rf::launch_fused_ept<float, float, 4>(P, cfg, sms, ev, n, params, W, nll, grad, st);
}

int rf_logp_f32_c32(const RfProgram& P, const void* ev, int64_t n,
                     const double* params, double* logp, cudaStream_t st) {
  return rf::launch_logp_T<float, float>(P, ev, n, params, logp, st);
}
