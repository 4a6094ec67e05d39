// rf_batched.cuh -- many datasets (toys) of uneven size sharing one graph.
//
//  plan kernel     (k_toys_common.cu) offsets -> tile_start (exclusive scan of ceil(n_t / T),
//                  at least one tile per toy so that empty toys still get
//                  their extended term); one block.
//  prep kernel     one thread per toy: the toy's FP64 normalisations and
//                  coefficients (RfConsts) from its parameter row.
//  tile kernel     persistent blocks take tiles from an atomic counter; a tile
//                  holds events of one toy only; its block partial goes to
//                  partials[tile]; the last tile of a toy to finish (per-toy
//                  ticket) sums that toy's tiles in tile order and writes
//                  (NLL, grad) -- optionally followed by one Adam step on the
//                  toy's parameter row.
// Results do not depend on which block ran which tile.
#pragma once
#include "rf_device.cuh"

namespace rf {

template <typename Real>
__global__ void toy_prep_kernel(const RfProgram P, const double* __restrict__ pm,
                                int32_t toys, RfConsts<Real>* consts,
                                unsigned int* next_tile, int32_t* adam_t) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t == 0) {
    *next_tile = 0u;
    if (adam_t) *adam_t += 1;
  }
  if (t < toys) {
    RfConsts<Real> K;
    build_consts_serial(P, pm + (int64_t)t * P.n_par, K);
    consts[t] = K;
  }
}

template <typename Real, typename Col, int NL, int EPT>
__global__ void __launch_bounds__(256)
    toy_tile_kernel(const RfProgram P, const Col* __restrict__ ev, int64_t stride,
                    int vec, const int64_t* __restrict__ offsets, int32_t toys,
                    int64_t tile_ev, double* pm, double* out, RfWork W,
                    const double* __restrict__ adam_scale, double adam_lr,
                    int64_t max_rows) {
  constexpr int NA = RF_NACC(NL);
  __shared__ RfConsts<Real> K;
  __shared__ double red[32 * NA];
  __shared__ double tot[NA];
  __shared__ int64_t s_tile, s_toy, s_b, s_e, s_total;
  __shared__ int s_last;
  const RfConsts<Real>* consts = static_cast<const RfConsts<Real>*>(W.toy_consts);
  constexpr int kWords = (int)(sizeof(RfConsts<Real>) / sizeof(double));
  static_assert(sizeof(RfConsts<Real>) % sizeof(double) == 0, "RfConsts size");

  if (threadIdx.x == 0) s_total = __ldcg(W.tile_start + toys);
  __syncthreads();
  const int64_t total = s_total < max_rows ? s_total : max_rows;
  for (;;) {
    if (threadIdx.x == 0) {
      int64_t tl = (int64_t)atomicAdd(W.next_tile, 1u);
      s_tile = tl;
      if (tl < total) {
        int lo = 0, hi = toys - 1;  // last toy with tile_start <= tl
        while (lo < hi) {
          int mid = (lo + hi + 1) >> 1;
          if (__ldcg(W.tile_start + mid) <= tl) lo = mid;
          else hi = mid - 1;
        }
        int64_t j = tl - __ldcg(W.tile_start + lo);
        // clamp to the bound columns: a bad offset table reads nothing outside
        int64_t ob = offsets[lo], oe = offsets[lo + 1];
        ob = ob < 0 ? 0 : (ob > stride ? stride : ob);
        oe = oe < ob ? ob : (oe > stride ? stride : oe);
        int64_t b = ob + j * tile_ev;
        int64_t e = b + tile_ev < oe ? b + tile_ev : oe;
        s_toy = lo;
        s_b = b < oe ? b : oe;
        s_e = e;
      }
    }
    __syncthreads();
    const int64_t tl = s_tile;
    if (tl >= total) break;
    const int64_t toy = s_toy, b = s_b, e = s_e;
    {
      const double* src = reinterpret_cast<const double*>(consts + toy);
      double* dst = reinterpret_cast<double*>(&K);
      for (int w = threadIdx.x; w < kWords; w += blockDim.x) dst[w] = __ldcg(src + w);
    }
    __syncthreads();

    Acc<Real, NA> acc;
    acc.zero();
    if (!K.bad && e > b) {
      EvalConsts<Real, NL> E;
      E.load(K);
      int64_t h = 0;
      if (vec) {
        uintptr_t a = reinterpret_cast<uintptr_t>(ev + (int64_t)P.col_obs[0] * stride + b);
        h = (int64_t)(((16u - (a & 15u)) & 15u) / sizeof(Col));
        if (h > e - b) h = e - b;
      }
      const int64_t nfull = (e - b - h) / EPT;
      for (int64_t ch = threadIdx.x; ch < nfull; ch += blockDim.x)
        iterate_full<Real, Col, NL, EPT>(P, E, ev, stride, b + h + ch * EPT, vec != 0, acc);
      if (threadIdx.x == blockDim.x - 1) {
        iterate_scalar<Real, Col, NL>(P, E, ev, stride, b, b + h, acc);
        iterate_scalar<Real, Col, NL>(P, E, ev, stride, b + h + nfull * EPT, e, acc);
      }
    }
    double val[NA];
#pragma unroll
    for (int i = 0; i < NA; ++i) val[i] = (double)acc.s[i] - (double)acc.c[i];
    block_sum<NA>(val, red, tot);
    if (threadIdx.x < NA) W.partials[tl * RF_NACC_MAX + threadIdx.x] = tot[threadIdx.x];
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
      int64_t r0 = __ldcg(W.tile_start + toy), r1 = __ldcg(W.tile_start + toy + 1);
      unsigned need = (unsigned)(r1 - r0);
      s_last = (atomicAdd(W.toy_counter + toy, 1u) == need - 1u) ? 1 : 0;
    }
    __syncthreads();
    if (s_last) {
      __threadfence();
      int64_t r0 = __ldcg(W.tile_start + toy), r1 = __ldcg(W.tile_start + toy + 1);
      rows_sum<NA>(W.partials, r0, r1, red, tot);
      if (threadIdx.x == 0) {
        int64_t ob = offsets[toy], oe = offsets[toy + 1];
        ob = ob < 0 ? 0 : (ob > stride ? stride : ob);
        oe = oe < ob ? ob : (oe > stride ? stride : oe);
        int64_t nt = oe - ob;
        double* row = out + toy * (int64_t)(1 + P.n_par);
        epilogue<Real, NL>(P, K, tot, nt, row, row + 1, W.status);
        W.toy_counter[toy] = 0u;
        if (adam_scale && isfinite(row[0])) {
          // Adam (Kingma & Ba 2015) in units of scale: u = theta / scale
          const int step = *W.adam_t;
          const double b1 = 0.9, b2 = 0.999, eps = 1e-8;
          const double c1 = 1.0 - pow(b1, (double)step), c2 = 1.0 - pow(b2, (double)step);
          double* th = pm + toy * (int64_t)P.n_par;
          double* m1 = W.adam_m1 + toy * (int64_t)P.n_par;
          double* m2 = W.adam_m2 + toy * (int64_t)P.n_par;
          for (int p = 0; p < P.n_par; ++p) {
            bool fx = p < 64 ? ((P.fixed_lo >> p) & 1) : ((P.fixed_hi >> (p - 64)) & 1);
            if (fx) continue;
            const double sc = adam_scale[toy * (int64_t)P.n_par + p];
            double gsc = row[1 + p] * sc;
            m1[p] = b1 * m1[p] + (1.0 - b1) * gsc;
            m2[p] = b2 * m2[p] + (1.0 - b2) * gsc * gsc;
            double mh = m1[p] / c1, vh = m2[p] / c2;
            th[p] -= sc * adam_lr * mh / (sqrt(vh) + eps);
          }
        }
      }
    }
    __syncthreads();
  }
}

template <typename Real, typename Col, int NL, int EPT>
inline int launch_toys_nl(const RfProgram& P, const RfLaunchCfg& cfg, int num_sms,
                          const void* events, int64_t n_events, const int64_t* offsets,
                          int32_t toys, double* pm, double* out, RfWork W,
                          const double* adam_scale, double adam_lr, int64_t max_rows,
                          cudaStream_t st) {
  int vec;
  int64_t head;
  // tiles start anywhere: vector loads need every column at the same phase
  {
    const uintptr_t base = reinterpret_cast<uintptr_t>(events);
    uintptr_t ph0 = 0;
    bool same = true;
    for (int c = 0; c < P.n_cols; ++c) {
      uintptr_t a = base + (uintptr_t)((int64_t)P.col_obs[c] * n_events * (int64_t)sizeof(Col));
      if (c == 0) ph0 = a & 15u;
      else if ((a & 15u) != ph0) same = false;
    }
    vec = (same && ph0 % sizeof(Col) == 0) ? 1 : 0;
    head = 0;
    (void)head;
  }
  int grid = num_sms * cfg.blocks_per_sm;
  toy_tile_kernel<Real, Col, NL, EPT><<<grid, cfg.block, 0, st>>>(
      P, static_cast<const Col*>(events), n_events, vec, offsets, toys, cfg.tile, pm,
      out, W, adam_scale, adam_lr, max_rows);
  return (int)cudaGetLastError();
}

template <typename Real, typename Col, int EPT>
inline int launch_toys_ept(const RfProgram& P, const RfLaunchCfg& cfg, int num_sms,
                           const void* events, int64_t n_events, const int64_t* offsets,
                           int32_t toys, double* pm, double* out, RfWork W,
                           const double* adam_scale, double adam_lr, int64_t max_rows,
                           cudaStream_t st) {
  switch (P.n_leaves) {
    case 1: return launch_toys_nl<Real, Col, 1, EPT>(P, cfg, num_sms, events, n_events, offsets, toys, pm, out, W, adam_scale, adam_lr, max_rows, st);
    case 2: return launch_toys_nl<Real, Col, 2, EPT>(P, cfg, num_sms, events, n_events, offsets, toys, pm, out, W, adam_scale, adam_lr, max_rows, st);
    case 3: return launch_toys_nl<Real, Col, 3, EPT>(P, cfg, num_sms, events, n_events, offsets, toys, pm, out, W, adam_scale, adam_lr, max_rows, st);
    case 4: return launch_toys_nl<Real, Col, 4, EPT>(P, cfg, num_sms, events, n_events, offsets, toys, pm, out, W, adam_scale, adam_lr, max_rows, st);
  }
  return (int)cudaErrorInvalidValue;
}

}  // namespace rf
