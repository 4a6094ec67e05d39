// Toy-study orchestration: tile plan, per-toy prologue, tile kernel.
#include "rf_batched.cuh"

#define RF_TOYS_DECL(R, C)                                                          \
  int rf_toys_##R##_##C(const RfProgram&, const RfLaunchCfg&, int, const void*,   \
                        int64_t, const int64_t*, int32_t, double*, double*, RfWork, \
                        const double*, double, int64_t, cudaStream_t);
RF_TOYS_DECL(f32, c32)
RF_TOYS_DECL(f32, c64)
RF_TOYS_DECL(f64, c32)
RF_TOYS_DECL(f64, c64)

namespace rf {
__global__ void __launch_bounds__(1024)
    toy_plan_kernel(const int64_t* __restrict__ offsets, int32_t toys,
                    int64_t tile, int64_t max_rows, int64_t n_events, int64_t* tile_start,
                    int32_t* tile_toy, int64_t* tile_be, unsigned int* status) {
  __shared__ int64_t wsum[32];
  __shared__ int64_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int64_t base = 0; base < toys; base += blockDim.x) {
    int64_t t = base + threadIdx.x;
    int64_t nt = 0;
    if (t < toys) {
      int64_t b = offsets[t], e = offsets[t + 1];
      if (e < b) {
        atomicOr(status, RF_STATUS_NONFINITE_BIT);
        e = b;
      }
      nt = (e - b + tile - 1) / tile;
      if (nt < 1) nt = 1;
    }
    // inclusive warp scan, then across warps
    int64_t v = nt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int64_t y = __shfl_up_sync(0xffffffffu, v, o);
      if (lane >= o) v += y;
    }
    if (lane == 31) wsum[wid] = v;
    __syncthreads();
    if (wid == 0) {
      int64_t w = (lane < (int)(blockDim.x >> 5)) ? wsum[lane] : 0;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        int64_t y = __shfl_up_sync(0xffffffffu, w, o);
        if (lane >= o) w += y;
      }
      wsum[lane] = w;
    }
    __syncthreads();
    int64_t incl = v + (wid > 0 ? wsum[wid - 1] : 0) + carry;
    if (t < toys) tile_start[t] = incl - nt;
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry = incl;
    __syncthreads();
  }
  if (threadIdx.x == 0) tile_start[toys] = carry;
  __syncthreads();
  // tile -> (toy, event range); offsets are clamped to the bound columns so
  // that a bad offset table reads nothing outside; tiles beyond the
  // workspace are never run
  for (int64_t t = threadIdx.x; t < toys; t += blockDim.x) {
    int64_t ob = offsets[t], oe = offsets[t + 1];
    ob = ob < 0 ? 0 : (ob > n_events ? n_events : ob);
    oe = oe < ob ? ob : (oe > n_events ? n_events : oe);
    const int64_t r0 = tile_start[t];
    const int64_t r1 = tile_start[t + 1] < max_rows ? tile_start[t + 1] : max_rows;
    for (int64_t r = r0; r < r1; ++r) {
      const int64_t b = ob + (r - r0) * tile;
      tile_toy[r] = (int32_t)t;
      tile_be[2 * r] = b < oe ? b : oe;
      tile_be[2 * r + 1] = b + tile < oe ? b + tile : oe;
    }
  }
}

}  // namespace rf

size_t rf_consts_size(int eval) {
  return eval ? sizeof(RfConsts<double>) : sizeof(RfConsts<float>);
}

int rf_toys_plan(const int64_t* offsets, int32_t toys, int64_t tile, int64_t max_rows,
                 int64_t n_events, RfWork W, void* stream) {
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  rf::toy_plan_kernel<<<1, 1024, 0, st>>>(offsets, toys, tile, max_rows, n_events, W.tile_start,
                                          W.tile_toy, W.tile_be, W.status);
  return (int)cudaGetLastError();
}

int rf_launch_batched(const RfProgram& P, int eval, int coldt, const RfLaunchCfg& cfg,
                      int num_sms, const void* events, int64_t n_events,
                      const int64_t* offsets, int32_t toys, double* pm, double* out,
                      RfWork W, const double* adam_scale, double adam_lr, bool plan,
                      int64_t max_rows, struct CUkern_st* jit_toys, void* stream,
                      int* launches) {
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int n = 0, rc;
  if (plan) {
    rc = rf_toys_plan(offsets, toys, cfg.tile, max_rows, n_events, W, stream);
    ++n;
    if (rc) return rc;
  }
  const int pb = 32;  // few threads per block: the FP64 prologue spreads over SMs
  const int pg = (toys + pb - 1) / pb > 0 ? (toys + pb - 1) / pb : 1;
  int32_t* at = adam_scale ? W.adam_t : nullptr;
  if (eval)
    rf::toy_prep_kernel<double><<<pg, pb, 0, st>>>(
        P, pm, toys, static_cast<RfConsts<double>*>(W.toy_consts), W.next_tile, at);
  else
    rf::toy_prep_kernel<float><<<pg, pb, 0, st>>>(
        P, pm, toys, static_cast<RfConsts<float>*>(W.toy_consts), W.next_tile, at);
  ++n;
  rc = (int)cudaGetLastError();
  if (rc) return rc;
  if (jit_toys)
    rc = rf_jit_launch_toys(jit_toys, P, coldt, cfg, num_sms, events, n_events, offsets, toys, pm,
                            out, W, adam_scale, adam_lr, max_rows, st);
  else if (eval == 0 && coldt == 0)
    rc = rf_toys_f32_c32(P, cfg, num_sms, events, n_events, offsets, toys, pm, out, W, adam_scale, adam_lr, max_rows, st);
  else if (eval == 0)
    rc = rf_toys_f32_c64(P, cfg, num_sms, events, n_events, offsets, toys, pm, out, W, adam_scale, adam_lr, max_rows, st);
  else if (coldt == 0)
    rc = rf_toys_f64_c32(P, cfg, num_sms, events, n_events, offsets, toys, pm, out, W, adam_scale, adam_lr, max_rows, st);
  else
    rc = rf_toys_f64_c64(P, cfg, num_sms, events, n_events, offsets, toys, pm, out, W, adam_scale, adam_lr, max_rows, st);
  ++n;
  if (launches) *launches = n;
  return rc;
}
