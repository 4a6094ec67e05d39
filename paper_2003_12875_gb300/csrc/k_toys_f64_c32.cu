// Batched-toy tile kernels: double per-event arithmetic, float columns.
#include "rf_batched.cuh"

int rf_toys_f64_c32(const RfProgram& P, const RfLaunchCfg& cfg, int sms,
                     const void* ev, int64_t n_events, const int64_t* offsets,
                     int32_t toys, double* pm, double* out, RfWork W,
                     const double* adam_scale, double adam_lr, int64_t max_rows,
                     cudaStream_t st) {
  if (cfg.ept == 4)
    return rf::launch_toys_ept<double, float, 4>(P, cfg, sms, ev, n_events, offsets, toys, pm,
                                                  out, W, adam_scale, adam_lr, max_rows, st);
  return rf::launch_toys_ept<double, float, 4>(P, cfg, sms, ev, n_events, offsets, toys, pm,
                                                out, W, adam_scale, adam_lr, max_rows, st);
}
