// Fused single-dataset kernels: double per-event arithmetic, double columns.
#include "rf_fused.cuh"

int rf_fused_f64_c64(const RfProgram& P, const RfLaunchCfg& cfg, int sms,
                      const void* ev, int64_t n, const double* params, RfWork W,
                      double* nll, double* grad, cudaStream_t st) {
  if (cfg.ept == 4)
    return rf::launch_fused_ept<double, double, 4>(P, cfg, sms, ev, n, params, W, nll, grad, st);
  return rf::launch_fused_ept<double, double, 2>(P, cfg, sms, ev, n, params, W, nll, grad, st);
}

int rf_logp_f64_c64(const RfProgram& P, const void* ev, int64_t n,
                     const double* params, double* logp, cudaStream_t st) {
  return rf::launch_logp_T<double, double>(P, ev, n, params, logp, st);
}
