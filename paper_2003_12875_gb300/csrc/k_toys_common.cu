// Toy-study orchestration: prep kernel, segment kernel, finalize kernel.
#include <algorithm>
#include <cstdlib>

#include "rf_batched.cuh"

#define RF_TOYS_DECL(R, C)                                                              \
  int rf_toys_##R##_##C(const RfProgram&, int, int, int, int, int, size_t, const void*, \
                        int64_t, const int64_t*, int32_t, RfWork, cudaStream_t);
RF_TOYS_DECL(f32, c32)
RF_TOYS_DECL(f32, c64)
RF_TOYS_DECL(f64, c32)
RF_TOYS_DECL(f64, c64)

namespace {
__global__ void columns_to_f32_kernel(const double* __restrict__ in, float* __restrict__ out,
                                      int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = __double2float_rn(in[i]);
}
}  // namespace

int rf_columns_to_f32(const double* in, float* out, int64_t n, void* stream) {
  if (n <= 0) return 0;
  int64_t g = (n + 255) / 256;
  const int grid = (int)(g > 65536 ? 65536 : g);
  columns_to_f32_kernel<<<grid, 256, 0, static_cast<cudaStream_t>(stream)>>>(in, out, n);
  return (int)cudaGetLastError();
}

size_t rf_consts_size(int eval) {
  return eval ? sizeof(RfConsts<double>) : sizeof(RfConsts<float>);
}

namespace {

template <typename Real>
int launch_finalize(const RfProgram& P, const int64_t* offsets, int32_t toys, int64_t stride,
                    int64_t warps, double* pm, double* out, RfWork W,
                    const double* adam_scale, double adam_lr, cudaStream_t st) {
  // 32 toys per block, RF_FIN_GROUP lanes per toy
  const int fb = 32 * RF_FIN_GROUP, fg = (toys + 31) / 32;
  switch (P.n_leaves) {
    case 1: rf::toy_finalize_kernel<Real, 1><<<fg, fb, 0, st>>>(P, offsets, toys, stride, warps, pm, out, W, adam_scale, adam_lr); break;
    case 2: rf::toy_finalize_kernel<Real, 2><<<fg, fb, 0, st>>>(P, offsets, toys, stride, warps, pm, out, W, adam_scale, adam_lr); break;
    case 3: rf::toy_finalize_kernel<Real, 3><<<fg, fb, 0, st>>>(P, offsets, toys, stride, warps, pm, out, W, adam_scale, adam_lr); break;
    case 4: rf::toy_finalize_kernel<Real, 4><<<fg, fb, 0, st>>>(P, offsets, toys, stride, warps, pm, out, W, adam_scale, adam_lr); break;
    case 5: rf::toy_finalize_kernel<Real, 5><<<fg, fb, 0, st>>>(P, offsets, toys, stride, warps, pm, out, W, adam_scale, adam_lr); break;
    case 6: rf::toy_finalize_kernel<Real, 6><<<fg, fb, 0, st>>>(P, offsets, toys, stride, warps, pm, out, W, adam_scale, adam_lr); break;
    default: return (int)cudaErrorInvalidValue;
  }
  return (int)cudaGetLastError();
}

}  // namespace

int rf_launch_batched(const RfProgram& P, int eval, int coldt, const RfLaunchCfg& cfg,
                      int num_sms, const void* events, int64_t n_events,
                      const int64_t* offsets, int32_t toys, double* pm, double* out,
                      RfWork W, const double* adam_scale, double adam_lr, int64_t max_rows,
                      struct CUkern_st* jit_toys, bool bulk, void* stream, int* launches) {
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (launches) *launches = 0;
  // segment rows: one per (warp, toy) pair that shares events, at most
  // warps + toys of them
  const int wpb = cfg.block / 32;
  int vec = 0;
  int64_t head = 0;
  const size_t esz = coldt ? 8 : 4;
  rf_vec_plan(P, events, n_events, (int)esz, &vec, &head);
  // bulk-copy form: a stage ring per warp, as many stages of 32*EPT events
  // (all columns) as fit in about 64 KB per block, 2..8; the register form
  // uses no shared memory
  const size_t stage_bytes = (size_t)std::max(P.n_cols, 1) * 32 * cfg.ept * esz;
  const int stages =
      (int)std::min<size_t>(8, std::max<size_t>(2, (64u << 10) / (wpb * stage_bytes)));
  const size_t smem = bulk ? (size_t)wpb * (8 * 8 + stages * stage_bytes) : 0;
  // grid: the SMs times the blocks of this size that fit on one (registers,
  // shared memory), at least the configured blocks per SM
  int fit = 0;
  if (jit_toys &&
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fit, reinterpret_cast<const void*>(jit_toys),
                                                    cfg.block, smem) != cudaSuccess) {
    cudaGetLastError();
    fit = 0;
  }
  int64_t grid = (int64_t)num_sms * std::max(cfg.blocks_per_sm, std::min(fit, 8));
  const int64_t room = max_rows - toys;
  if (wpb < 1 || room < wpb) return (int)cudaErrorInvalidValue;
  if (grid * wpb > room) grid = room / wpb;
  const int64_t warps = grid * wpb;

  // prep: blocks of 32 toys and 3 warps per leaf + 1
  const int pb = 32 * (3 * std::max(P.n_leaves, 1) + 1);
  const int pg = (toys + 31) / 32 > 0 ? (toys + 31) / 32 : 1;
  int32_t* at = adam_scale ? W.adam_t : nullptr;
  // a programmatic dependent of the kernel before it (back to back: the
  // previous call's finalize kernel), publishing its constants after it
  cudaLaunchConfig_t plc = {};
  plc.gridDim = dim3(pg);
  plc.blockDim = dim3(pb);
  plc.stream = st;
  cudaLaunchAttribute pat[1];
  pat[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  pat[0].val.programmaticStreamSerializationAllowed = 1;
  plc.attrs = pat;
  plc.numAttrs = 1;
  const double* pmc = pm;
  int rc = eval ? (int)cudaLaunchKernelEx(&plc, rf::toy_prep_kernel<double>, P, pmc, offsets,
                                          toys, n_events,
                                          static_cast<RfConsts<double>*>(W.toy_consts), W.status,
                                          at, W.toy_consts_x)
                : (int)cudaLaunchKernelEx(&plc, rf::toy_prep_kernel<float>, P, pmc, offsets, toys,
                                          n_events, static_cast<RfConsts<float>*>(W.toy_consts),
                                          W.status, at, W.toy_consts_x);
  if (rc) return rc;
  const int g = (int)grid;
  if (jit_toys)
    rc = rf_jit_launch_toys(jit_toys, P, g, cfg.block, vec, stages, smem, events, n_events,
                            offsets, toys, W, st);
  else if (eval == 0 && coldt == 0)
    rc = rf_toys_f32_c32(P, cfg.ept, g, cfg.block, vec, stages, smem, events, n_events, offsets, toys, W, st);
  else if (eval == 0)
    rc = rf_toys_f32_c64(P, cfg.ept, g, cfg.block, vec, stages, smem, events, n_events, offsets, toys, W, st);
  else if (coldt == 0)
    rc = rf_toys_f64_c32(P, cfg.ept, g, cfg.block, vec, stages, smem, events, n_events, offsets, toys, W, st);
  else
    rc = rf_toys_f64_c64(P, cfg.ept, g, cfg.block, vec, stages, smem, events, n_events, offsets, toys, W, st);
  if (rc) return rc;
  rc = eval ? launch_finalize<double>(P, offsets, toys, n_events, warps, pm, out, W, adam_scale,
                                      adam_lr, st)
            : launch_finalize<float>(P, offsets, toys, n_events, warps, pm, out, W, adam_scale,
                                     adam_lr, st);
  if (launches) *launches = 3;
  return rc;
}
