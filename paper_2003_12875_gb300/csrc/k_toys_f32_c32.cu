// Batched-toy segment kernels (precompiled, generic model): float per-event arithmetic, float columns.
#include "rf_batched.cuh"

int rf_toys_f32_c32(const RfProgram& P, int ept, int grid, int block, int vec, int stages,
                 size_t smem, const void* ev, int64_t n_events, const int64_t* offsets,
                 int32_t toys, RfWork W, cudaStream_t st) {
  if (ept == 16)
    return rf::launch_toys_ept<float, float, 16>(P, grid, block, vec, stages, smem, ev, n_events, offsets, toys, W, st);
  if (ept == 8)
    return rf::launch_toys_ept<float, float, 8>(P, grid, block, vec, stages, smem, ev, n_events, offsets, toys, W, st);
  return (int)cudaErrorInvalidValue;
}
