// rf_batched.cuh -- many datasets (toys) of uneven size sharing one graph.
//
//  prep kernel      32 toys per block, their FP64 normalisations, per-event
//                   constants and coefficients (RfConsts) from their
//                   parameter rows on separate warps; checks the offsets.
//  segment kernel   the toys' events split evenly over the launch's warps;
//                   each warp writes one FP64 row per toy its range meets
//                   (launched as a programmatic dependent of the prep kernel).
//  finalize kernel  a group of lanes per toy: its rows summed in order, the
//                   FP64 epilogue (NLL, gradient), optionally one Adam step.
// Results depend only on the inputs and the launch shape, not on timing.
#pragma once
#include "rf_toys.cuh"

namespace rf {

// Prep kernel: blocks of 32 toys and 3 n_leaves + 1 warps, the tasks of the
// single-dataset prologue for 32 toys at once (the FP64 unit takes one warp
// instruction at a time, so the toys share each instruction and the tasks run
// on separate SM sub-partitions): warps 2k and 2k + 1 take leaf k's integral
// of the block's toys 0-15 and 16-31, one lane pair per toy
// (leaf_norm_pair); warp 2L + k leaf k's per-event constants, lane l for toy
// l; warp 3L the coefficients and their logs (CoefPre), lane l for toy l.
// Then warps 0-3 check the toys' offsets and combine, 4 lanes per toy
// (comb_consts_group).  Lets the segment kernel launch at once.  The constants are built in shared memory and published
// only after the wait for the kernel before (the previous call's finalize
// kernel, which reads them), so back to back the FP64 chains of this call's
// prep run beside the previous call's finalize.  A fit step (adam_t set)
// reads parameter rows that the previous finalize kernel has just updated, so
// it waits first.
template <typename Real>
__device__ __forceinline__ void toy_prep_body(const RfProgram& P, const double* __restrict__ pm,
                                              const int64_t* __restrict__ offsets,
                                              int32_t toys, int64_t n_events,
                                              RfConsts<Real>* consts, unsigned int* status,
                                              int32_t* adam_t, RfExact* consts_x) {
  asm volatile("griddepcontrol.launch_dependents;");
  __shared__ RfConsts<Real> Ks[32];
  __shared__ double lnI_s[RF_MAXL][32];
  __shared__ int ok_s[RF_MAXL][32];
  __shared__ CoefPre cp_s[32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, NL = P.n_leaves;
  const int64_t t0 = (int64_t)blockIdx.x * 32;
  if (adam_t) {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    if (blockIdx.x == 0 && threadIdx.x == 0) *adam_t += 1;
  }
  if (w < 2 * NL) {
    const int k = w >> 1, j = 16 * (w & 1) + (lane >> 1);
    const int64_t t = t0 + j;
    if (t < toys) {  // the same for both lanes of a pair
      double l = 0.0;
      const bool o = leaf_norm_pair(P, pm + t * P.n_par, Ks[j], k, &l);
      if ((lane & 1) == 0) {
        ok_s[k][j] = o ? 1 : 0;
        lnI_s[k][j] = l;
      }
    }
  } else if (w < 3 * NL) {
    const int64_t t = t0 + lane;
    if (t < toys) leaf_eval_consts(P, pm + t * P.n_par, Ks[lane], w - 2 * NL);
  } else if (w == 3 * NL) {
    const int64_t t = t0 + lane;
    if (t < toys) coef_pre_serial(P, pm + t * P.n_par, &cp_s[lane]);
  }
  __syncthreads();
  if (w < 4) {  // combine: 4 lanes per toy (comb_consts_group), 8 toys per warp
    const int j = 8 * w + (lane >> 2);
    const int64_t t = t0 + j;
    const bool valid = t < toys;
    bool all = true;
    if (valid) {
      if ((lane & 3) == 0) {
        const int64_t b = offsets[t], e = offsets[t + 1];
        if (b < 0 || e < b || e > n_events) atomicOr(status, RF_STATUS_NONFINITE_BIT);
      }
      for (int k = 0; k < NL; ++k) all &= ok_s[k][j] != 0;
    }
    comb_consts_group<Real, 4>(P, pm + (valid ? t : 0) * P.n_par, Ks[j], &lnI_s[0][j], 32, all,
                               (consts_x && valid) ? consts_x + t : nullptr, &cp_s[j], valid);
  }
  asm volatile("griddepcontrol.wait;" ::: "memory");
  __syncthreads();
  // publish: the block's toys' constants, a contiguous stretch of words
  const int64_t nt = toys - t0 < 32 ? toys - t0 : 32;
  constexpr int kWords = (int)(sizeof(RfConsts<Real>) / sizeof(double));
  const double* src = reinterpret_cast<const double*>(Ks);
  double* dst = reinterpret_cast<double*>(consts + t0);
  for (int64_t q = threadIdx.x; q < nt * kWords; q += blockDim.x) dst[q] = src[q];
}

// Finalize kernel: blocks of 32 toys and RF_FIN_GROUP lanes per toy (toy j
// of the block on lanes j G .. j G + G - 1).  The group sums the toy's
// segment rows in row order (value i on group lane i mod G) while the
// block's constants arrive by one bulk copy, then runs the FP64 epilogue
// spread over its lanes (epilogue_group) into out row t and, for a fit,
// applies one Adam step (Kingma & Ba 2015) to the toy's free parameters in
// units of its scale row (parameter p on group lane p mod G).  The FP64 unit
// takes one warp instruction at a time whatever the number of active lanes,
// so the group's chains are what the kernel waits for, about G times shorter
// than one thread's.
template <typename Real, int NL>
__device__ __forceinline__ void toy_finalize_body(const RfProgram& P,
                                                  const int64_t* __restrict__ offsets,
                                                  int32_t toys, int64_t stride, int64_t warps,
                                                  double* pm, double* out, RfWork& W,
                                                  const double* __restrict__ adam_scale,
                                                  double adam_lr) {
  constexpr int NA = RF_NACC(NL);
  constexpr int G = RF_FIN_GROUP;
  constexpr int NV = (NA + G - 1) / G;  // values per group lane
  // the block's (up to 32) toys' constants: one bulk copy into shared memory
  // (RfConsts is a multiple of 16 bytes, the array 256-byte aligned)
  __shared__ RfConsts<Real> Ks[32];
  __shared__ double tot_s[32][NA];
  __shared__ __align__(8) uint64_t bar;
  const int64_t t0 = (int64_t)blockIdx.x * 32;
  const int64_t nt = toys - t0 < 32 ? toys - t0 : 32;
  const int j = threadIdx.x / G, q = threadIdx.x & (G - 1);
  const int64_t t = t0 + j;
  const bool valid = t < toys;
  // the next call's prep kernel may start at once: it publishes new
  // constants only after this grid has finished, and writes no segment row
  asm volatile("griddepcontrol.launch_dependents;");
  if (threadIdx.x == 0) {
    const uint32_t bytes = (uint32_t)(nt * (int64_t)sizeof(RfConsts<Real>));
    bulk::bar_init(&bar, 1);
    bulk::fence_bar_init();
    bulk::arrive_expect_tx(&bar, bytes);
    bulk::copy(Ks, static_cast<const RfConsts<Real>*>(W.toy_consts) + t0, bytes, &bar);
  }
  // the segment rows: after the segment kernel (a no-op in stream order)
  asm volatile("griddepcontrol.wait;" ::: "memory");
  int64_t ob = 0, oe = 0;
  double acc[NV];
#pragma unroll
  for (int m = 0; m < NV; ++m) acc[m] = 0.0;
  if (valid) {
    const ToySplit S = toy_split(offsets, toys, stride, warps);
    ob = toy_off(offsets, t, stride);
    oe = toy_off(offsets, t + 1, stride);
    ob = ob < S.B ? S.B : ob;
    oe = oe > S.E ? S.E : oe;
    if (oe < ob) oe = ob;
    if (oe > ob) {  // a toy meets a few warp ranges: plain FP64 sums of a few rows
      const int64_t r1 = S.warp_of(oe - 1) + t;
      for (int64_t r = S.warp_of(ob) + t; r <= r1; ++r) {
        const double* row = W.partials + r * RF_NACC_MAX;
#pragma unroll
        for (int m = 0; m < NV; ++m)
          if (q + m * G < NA) acc[m] += WarpRow<Real, NA, 0>::value(__ldcg(row + q + m * G));
      }
    }
  }
#pragma unroll
  for (int m = 0; m < NV; ++m)
    if (q + m * G < NA) tot_s[j][q + m * G] = acc[m];
  __syncthreads();  // the totals; the barrier's initialisation
  const bool ok = bulk::wait(&bar, 0u);
  if (__syncthreads_or(!ok)) {
    if (threadIdx.x == 0) atomicOr(W.status, RF_STATUS_TIMEOUT_BIT);
    return;
  }
  double* row = out + t * (int64_t)(1 + P.n_par);
  const double v = epilogue_group<Real, NL, G>(P, Ks[j], tot_s[j], oe - ob, valid ? row : nullptr,
                                               valid ? row + 1 : nullptr, W.status, valid);
  if (adam_scale) {
    // bias corrections 1 - b^step: both powers in one FP64 pass (group lanes
    // 0 and 1), shared over the group
    const int step = *W.adam_t;
    const double b1 = 0.9, b2 = 0.999, eps = 1e-8;
    const double pw = pow(q == 1 ? b2 : b1, (double)step);
    const int g0 = (threadIdx.x & 31) & ~(G - 1);
    const double c1 = 1.0 - __shfl_sync(0xffffffffu, pw, g0);
    const double c2 = 1.0 - __shfl_sync(0xffffffffu, pw, g0 + 1);
    if (valid && isfinite(v)) {
      double* th = pm + t * (int64_t)P.n_par;
      double* m1 = W.adam_m1 + t * (int64_t)P.n_par;
      double* m2 = W.adam_m2 + t * (int64_t)P.n_par;
      for (int p = q; p < P.n_par; p += G) {
        const bool fx = p < 64 ? ((P.fixed_lo >> p) & 1) : ((P.fixed_hi >> (p - 64)) & 1);
        if (fx) continue;
        const double sc = adam_scale[t * (int64_t)P.n_par + p];
        const double gsc = row[1 + p] * sc;
        m1[p] = b1 * m1[p] + (1.0 - b1) * gsc;
        m2[p] = b2 * m2[p] + (1.0 - b2) * gsc * gsc;
        const double mh = m1[p] / c1, vh = m2[p] / c2;
        th[p] -= sc * adam_lr * mh / (sqrt(vh) + eps);
      }
    }
  }
}

template <typename Real>
__global__ void toy_prep_kernel(const RfProgram P, const double* __restrict__ pm,
                                const int64_t* __restrict__ offsets, int32_t toys,
                                int64_t n_events, RfConsts<Real>* consts,
                                unsigned int* status, int32_t* adam_t, RfExact* consts_x) {
  toy_prep_body<Real>(P, pm, offsets, toys, n_events, consts, status, adam_t, consts_x);
}

template <typename Real, typename Col, int NL, int EPT>
__global__ void __launch_bounds__(256)
    toy_segment_kernel(const RfProgram P, const Col* __restrict__ ev, int64_t stride, int vec,
                       const int64_t* __restrict__ offsets, int32_t toys, int stages, RfWork W) {
  toy_segment_body_reg<GenericModel<NL>, Real, Col, EPT>(P, ev, stride, vec, offsets, toys, stages,
                                                         W);
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
  auto kern = toy_segment_kernel<Real, Col, NL, EPT>;  // register form: no shared memory
  (void)smem;
  cudaLaunchConfig_t lc = {};
  lc.gridDim = dim3(grid);
  lc.blockDim = dim3(block);
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
