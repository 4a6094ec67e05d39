// rf_toys.cuh -- device code of the toy-study segment kernel: the even split
// of all toys' events over warps, the toy walk, per-segment rows, and the two
// streaming forms (registers; bulk-copy stage rings).  Compiled into the
// per-graph toy kernels only (its own NVRTC prelude text).
#pragma once
#include "rf_kernels.cuh"

namespace rf {

// ------------------------------------------------------ toy studies
// The toys' events [B, E) (B = offsets[0], E = offsets[toys], clamped to the
// bound columns) are split into N contiguous ranges of (almost) equal size,
// one per warp of the segment kernel: warp w takes [start(w), start(w+1)),
// N = min(warps, E - B) so that no range is empty.  The part of toy t inside
// warp w's range is segment (w, t); its partial sums go to row w + t of the
// partials, which no other segment uses (w + t counts the warp starts and toy
// starts before the segment).  Toy t's segments are therefore the rows w + t
// for w = warp_of(offsets[t]) .. warp_of(offsets[t+1] - 1), summed in that
// order by the finalize kernel.  Every warp reads one contiguous stretch of
// the columns, and no warp waits on another.
struct ToySplit {
  int64_t B, E, N;
  __device__ __forceinline__ int64_t start(int64_t w) const {
    return B + (int64_t)(((unsigned long long)w * (unsigned long long)(E - B)) /
                         (unsigned long long)N);
  }
  // the warp whose range holds event i (B <= i < E): the largest w with
  // start(w) <= i, i.e. floor(((i - B + 1) N - 1) / (E - B))
  __device__ __forceinline__ int64_t warp_of(int64_t i) const {
    const unsigned long long r =
        ((unsigned long long)(i - B + 1) * (unsigned long long)N - 1ull) /
        (unsigned long long)(E - B);
    return (int64_t)r < N ? (int64_t)r : N - 1;
  }
};

// offsets[t] clamped to the bound columns [0, n]
__device__ __forceinline__ int64_t toy_off(const int64_t* __restrict__ off, int64_t t, int64_t n) {
  const int64_t v = off[t];
  return v < 0 ? 0 : (v > n ? n : v);
}

__device__ __forceinline__ ToySplit toy_split(const int64_t* __restrict__ off, int32_t toys,
                                              int64_t n, int64_t warps) {
  ToySplit s;
  s.B = toy_off(off, 0, n);
  s.E = toy_off(off, toys, n);
  if (s.E < s.B) s.E = s.B;
  const int64_t len = s.E - s.B;
  s.N = warps < len ? warps : len;
  if (s.N < 1) s.N = 1;
  return s;
}

// The largest t in [0, toys) with offsets[t] <= i (clamped offsets), by a
// 32-way search: each round the 31 lanes probe 31 evenly spaced toys and a
// ballot keeps the bracket between the last probe at or below i and the next
// one.  Every lane returns the same t; the bracket shrinks every round, so at
// most ceil(log32(toys)) + 1 rounds run (a non-monotone offset table gives
// some t in [0, toys), never an index outside it).
__device__ inline int32_t find_toy(const int64_t* __restrict__ off, int32_t toys, int64_t n,
                                   int64_t i) {
  const int lane = threadIdx.x & 31;
  int64_t lo = 0, hi = toys;
  for (int round = 0; round < 16 && hi - lo > 1; ++round) {
    const int64_t span = hi - lo;
    const int64_t p = lo + (span * (lane + 1)) / 32;
    const bool le = lane < 31 && (p == lo || toy_off(off, p, n) <= i);
    const int k = __popc(__ballot_sync(0xffffffffu, le));
    const int64_t nlo = k > 0 ? lo + (span * k) / 32 : lo;
    int64_t nhi = k < 31 ? lo + (span * (k + 1)) / 32 : hi;
    if (nhi <= nlo) nhi = nlo + 1;
    lo = nlo;
    hi = nhi;
  }
  return (int32_t)lo;
}

// Warp-wide fixed-order totals of the per-lane accumulators (FP32 pairs for
// FP32 evaluation, FP64 otherwise); lane 0 writes the FP64 row.
template <typename Real, int NA, unsigned long long MASK>
struct WarpRow;
// FP32 rows hold each sum as its FP32 pair (h, l) packed into the 64-bit slot:
// the segment kernel then issues no FP64 instruction (one takes its
// sub-partition's FP64 unit for ~64 cycles, stalling the FP32 event loop of
// the warps beside it), and the finalize kernel widens h + l.
template <int NA, unsigned long long MASK>
struct WarpRow<float, NA, MASK> {
  static __device__ __forceinline__ void write(const Acc<float, NA, MASK>& acc, double* row) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int i = 0; i < NA; ++i) {
      float h = 0.0f, l = 0.0f;
      if ((MASK >> i) & 1ull) {
        h = acc.s[i];
        l = -acc.c[i];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          const float h2 = __shfl_xor_sync(0xffffffffu, h, o);
          const float l2 = __shfl_xor_sync(0xffffffffu, l, o);
          ds_add(h, l, h2, l2);
        }
      }
      if (lane == 0)
        reinterpret_cast<unsigned long long*>(row)[i] =
            ((unsigned long long)__float_as_uint(l) << 32) | __float_as_uint(h);
    }
  }
  static __device__ __forceinline__ double value(double stored) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(stored);
    return (double)__uint_as_float((unsigned)(b & 0xffffffffull)) +
           (double)__uint_as_float((unsigned)(b >> 32));
  }
};
template <int NA, unsigned long long MASK>
struct WarpRow<double, NA, MASK> {
  static __device__ __forceinline__ void write(const Acc<double, NA, MASK>& acc, double* row) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int i = 0; i < NA; ++i) {
      const double r = ((MASK >> i) & 1ull) ? warp_sum(acc.value(i)) : 0.0;
      if (lane == 0) row[i] = r;
    }
  }
  static __device__ __forceinline__ double value(double stored) { return stored; }
};

// ------------------------------------------------ bulk-copy event streaming
// Each warp streams its own contiguous event range through a ring of S
// shared-memory stages.  Lane 0 fills a stage with one cp.async.bulk (TMA
// bulk copy) per column, completing on the stage's mbarrier; the lanes wait
// on the barrier's phase, evaluate the stage from shared memory, and lane 0
// refills it with the chunk S ahead.  Up to S chunks are in flight per warp
// without holding registers.  Every wait is bounded: a wait that gives up
// raises RF_STATUS_TIMEOUT_BIT and the warp stops streaming.
namespace bulk {
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void bar_init(uint64_t* b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(b)), "r"(count) : "memory");
}
// make initialised barriers visible to the bulk-copy (async) proxy
__device__ __forceinline__ void fence_bar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void arrive_expect_tx(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(b)),
               "r"(bytes)
               : "memory");
}
// global -> shared, `bytes` a multiple of 16, both addresses 16-byte aligned
__device__ __forceinline__ void copy(void* dst, const void* src, uint32_t bytes, uint64_t* b) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(b))
      : "memory");
}
__device__ __forceinline__ bool try_wait(uint64_t* b, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}" : "=r"(done) : "r"(smem_addr(b)), "r"(parity) : "memory");
  return done != 0;
}
// bounded wait for the phase with the given parity (about a second at most)
__device__ __forceinline__ bool wait(uint64_t* b, uint32_t parity) {
  for (uint32_t it = 0; it < (1u << 22); ++it)
    if (try_wait(b, parity)) return true;
  return false;
}
constexpr int kMaxStages = 8;
}  // namespace bulk

// Evaluate events [p0, p1) of a chunk that starts at event c0 and holds
// CE = 32*EPT events, column c at buf[c * CE + j].  Lanes read 128-bit
// vectors (conflict-free: a warp's loads cover contiguous 512 bytes): lane l
// takes vectors l + 32 m, i.e. events V (l + 32 m) + r.  FULL: the chunk lies
// inside [p0, p1) (no per-event test).  ANYZERO: some coefficient of the
// toy may be exactly zero (the per-event test; see the register form).
template <class M, typename Real, typename Col, int EPT, bool FULL, bool ANYZERO>
__device__ __forceinline__ void eval_chunk(const RfProgram& P, const EvalConsts<Real, M::NL_>& E,
                                           Acc<Real, RF_NACC(M::NL_), M::AMASK>& acc,
                                           const Col* buf, int64_t c0, int64_t p0, int64_t p1) {
  constexpr int NL = M::NL_;
  constexpr int NA = RF_NACC(NL);
  constexpr int CE = 32 * EPT;
  constexpr int V = Vec<Col>::W;
  static_assert(EPT % V == 0, "EPT must be a multiple of the vector width");
  typedef typename Vec<Col>::T VT;
  const int lane = threadIdx.x & 31;
  Real q[NA];
#pragma unroll
  for (int i = 0; i < NA; ++i) q[i] = Real(0);
#pragma unroll
  for (int m = 0; m < EPT / V; ++m) {
    const int vi = lane + 32 * m;
    Col xv[NL][V];
#pragma unroll
    for (int c = 0; c < NL; ++c) {
      if (c < M::NCOL && c < P.n_cols) {
        const VT t = reinterpret_cast<const VT*>(buf + c * CE)[vi];
        const Col* tc = reinterpret_cast<const Col*>(&t);
#pragma unroll
        for (int r = 0; r < V; ++r) xv[c][r] = tc[r];
      } else {
#pragma unroll
        for (int r = 0; r < V; ++r) xv[c][r] = Col(0);
      }
    }
#pragma unroll
    for (int r = 0; r < V; ++r) {
      const int j = V * vi + r;
      if (FULL || (c0 + j >= p0 && c0 + j < p1)) {
        if constexpr (ANYZERO && IsF32<Real>::v) {
          if (E.zero_mask != 0) {  // a coefficient exactly 0: the FP64 event
            double xd[NL];
            float qe[NA];
#pragma unroll
            for (int c = 0; c < NL; ++c) xd[c] = (double)xv[c][r];
#pragma unroll
            for (int i = 0; i < NA; ++i) qe[i] = 0.f;
            M::event_exact(E.full, xd, qe);
#pragma unroll
            for (int i = 0; i < NA; ++i) q[i] += qe[i];
            continue;
          }
        }
        Real xc[NL];
#pragma unroll
        for (int c = 0; c < NL; ++c) xc[c] = cvt<Real, Col>(xv[c][r]);
        M::template event<Real, ANYZERO>(P, E, xc, q);
      }
    }
  }
  acc.add(q);
}

// The toy a warp is in: its event range [tb, te), constants, running sums.
// seek() moves to the toy holding event p, writing the finished toy's row
// (when it had events) and skipping empty toys; false only when p lies past
// the last toy (a non-monotone offset table).
template <class M, typename Real>
struct ToyState {
  static constexpr int NL = M::NL_;
  static constexpr int NA = RF_NACC(NL);
  int32_t t;
  int64_t tb, te;
  bool bad, any;
  EvalConsts<Real, NL> E;
  Acc<Real, NA, M::AMASK> acc;
  const RfExact* xs;  // the toys' FP64 constants (zero-coefficient toys)
  __device__ __forceinline__ void open(const RfConsts<Real>* consts, const int64_t* offsets,
                                       int64_t stride, int32_t tt) {
    t = tt;
    tb = toy_off(offsets, t, stride);
    te = toy_off(offsets, (int64_t)t + 1, stride);
    bad = consts[t].bad != 0;
    if (!bad) E.load(consts[t], xs ? xs + t : nullptr);
    acc.zero();
    any = false;
  }
  __device__ __forceinline__ void close(double* rows) {
    if (any) WarpRow<Real, NA, M::AMASK>::write(acc, rows + (int64_t)t * RF_NACC_MAX);
  }
  __device__ __forceinline__ bool seek(const RfConsts<Real>* consts, const int64_t* offsets,
                                       int64_t stride, int32_t toys, int64_t p, double* rows) {
    while (te <= p && t + 1 < toys) {
      close(rows);
      open(consts, offsets, stride, t + 1);
    }
    return te > p;
  }
};

// Segment kernel: warp w streams [start(w), start(w+1)) through its stage
// ring (chunks of 32*EPT events from the first 16-byte-aligned event; the
// ragged ends are read directly), switching toy constants at toy boundaries
// and writing one FP64 row per toy it meets.  The bulk copies of the first
// stages and the search for the first toy need only the offsets and the
// events, so they are issued before the wait for the prep kernel.
// Dynamic shared memory: warps * (kMaxStages barriers + S stages of
// n_cols * 32*EPT column values).
template <class M, typename Real, typename Col, int EPT>
__device__ __forceinline__ void toy_segment_body(const RfProgram& P, const Col* __restrict__ ev,
                                                 int64_t stride, int vec,
                                                 const int64_t* __restrict__ offsets,
                                                 int32_t toys, int stages, RfWork& W) {
  constexpr int NL = M::NL_;
  constexpr int NA = RF_NACC(NL);
  constexpr int CE = 32 * EPT;
  extern __shared__ __align__(128) unsigned char rf_dyn_smem[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int wpb = blockDim.x >> 5;
  uint64_t* bars = reinterpret_cast<uint64_t*>(rf_dyn_smem) + wib * bulk::kMaxStages;
  const int stage_elems = P.n_cols * CE;
  Col* ring = reinterpret_cast<Col*>(rf_dyn_smem + (size_t)wpb * bulk::kMaxStages * 8) +
              (size_t)wib * stages * stage_elems;
  const uint32_t stage_bytes = (uint32_t)(stage_elems * sizeof(Col));

  const int64_t w = (int64_t)blockIdx.x * wpb + wib;
  const ToySplit Sp = toy_split(offsets, toys, stride, (int64_t)gridDim.x * wpb);
  const bool active = w < Sp.N && Sp.E > Sp.B;
  int64_t wb = 0, we = 0, a0 = 0, nch = 0;
  int32_t t = 0;
  if (active) {
    wb = Sp.start(w);
    we = Sp.start(w + 1);
    t = find_toy(offsets, toys, stride, wb);
    a0 = we;
    if (vec) {
      const uintptr_t a = reinterpret_cast<uintptr_t>(ev + (int64_t)P.col_obs[0] * stride + wb);
      a0 = wb + (int64_t)(((16u - (a & 15u)) & 15u) / sizeof(Col));
      if (a0 > we) a0 = we;
      nch = (we - a0) / CE;
    }
  }
  if (lane == 0) {
    for (int s = 0; s < stages; ++s) bulk::bar_init(&bars[s], 1);
    bulk::fence_bar_init();
    for (int64_t c = 0; c < nch && c < stages; ++c) {
      Col* dst = ring + (size_t)c * stage_elems;
      bulk::arrive_expect_tx(&bars[c], stage_bytes);
      for (int col = 0; col < P.n_cols; ++col)
        bulk::copy(dst + col * CE, ev + (int64_t)P.col_obs[col] * stride + a0 + c * CE,
                   (uint32_t)(CE * sizeof(Col)), &bars[c]);
    }
  }
  __syncwarp();
  asm volatile("griddepcontrol.wait;" ::: "memory");
  if (!active) return;

  const RfConsts<Real>* consts = static_cast<const RfConsts<Real>*>(W.toy_consts);
  ToyState<M, Real> T;
  T.xs = W.toy_consts_x;
  T.open(consts, offsets, stride, t);
  double* rows = W.partials + w * RF_NACC_MAX;  // row of (w, t) = rows + t * RF_NACC_MAX
  // ragged head, straight from the columns
  for (int64_t p = wb; p < a0;) {
    if (!T.seek(consts, offsets, stride, toys, p, rows)) break;
    const int64_t q = a0 < T.te ? a0 : T.te;
    if (!T.bad) iterate_scalar<M, Real, Col>(P, T.E, ev, stride, p + lane, q, T.acc, 32);
    T.any = true;
    p = q;
  }
  // aligned chunks through the stage ring; s and ph: stage and phase of chunk c
  int s = 0;
  uint32_t ph = 0;
  int64_t c0 = a0;
  for (int64_t c = 0; c < nch; ++c, c0 += CE) {
    if (!bulk::wait(&bars[s], ph)) {
      if (lane == 0) atomicOr(W.status, RF_STATUS_TIMEOUT_BIT);
      // let the copies already issued land before the warp leaves: first one
      // more bounded wait on the stage whose copy did not arrive, then on the
      // stages after it (the status bit stays set whatever these waits give)
      bulk::wait(&bars[s], ph);
      int ds = s;
      uint32_t dph = ph;
      for (int64_t d = c + 1; d < nch && d < c + stages; ++d) {
        if (++ds == stages) { ds = 0; dph ^= 1u; }
        bulk::wait(&bars[ds], dph);
      }
      return;
    }
    const Col* buf = ring + s * stage_elems;
    if (c0 + CE <= T.te && c0 >= T.tb) {  // the whole chunk in the current toy
      if (!T.bad && T.E.zero_mask == 0)
        eval_chunk<M, Real, Col, EPT, true, false>(P, T.E, T.acc, buf, c0, c0, c0 + CE);
      else if (!T.bad)
        eval_chunk<M, Real, Col, EPT, true, true>(P, T.E, T.acc, buf, c0, c0, c0 + CE);
      T.any = true;
    } else {
      for (int64_t p = c0; p < c0 + CE;) {
        if (!T.seek(consts, offsets, stride, toys, p, rows)) break;
        const int64_t q = c0 + CE < T.te ? c0 + CE : T.te;
        if (!T.bad) eval_chunk<M, Real, Col, EPT, false, true>(P, T.E, T.acc, buf, c0, p, q);
        T.any = true;
        p = q;
      }
    }
    __syncwarp();
    if (lane == 0 && c + stages < nch) {  // refill the stage with the chunk `stages` ahead
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      bulk::arrive_expect_tx(&bars[s], stage_bytes);
      const int64_t src = a0 + (c + stages) * CE;
      for (int col = 0; col < P.n_cols; ++col)
        bulk::copy(const_cast<Col*>(buf) + col * CE, ev + (int64_t)P.col_obs[col] * stride + src,
                   (uint32_t)(CE * sizeof(Col)), &bars[s]);
    }
    if (++s == stages) {
      s = 0;
      ph ^= 1u;
    }
  }
  // ragged tail
  for (int64_t p = a0 + nch * CE; p < we;) {
    if (!T.seek(consts, offsets, stride, toys, p, rows)) break;
    const int64_t q = we < T.te ? we : T.te;
    if (!T.bad) iterate_scalar<M, Real, Col>(P, T.E, ev, stride, p + lane, q, T.acc, 32);
    T.any = true;
    p = q;
  }
  T.close(rows);
}

// Segment kernel, register-streaming form: the same warp ranges, toy walk
// and rows, but each segment's aligned middle is read with 128-bit loads into
// registers, the next chunk's loads issued before the current chunk is
// evaluated (as in the fused kernel); lanes take chunks of EPT events in turn.
// No shared memory.
template <class M, typename Real, typename Col, int EPT>
__device__ __forceinline__ void toy_segment_body_reg(const RfProgram& P,
                                                     const Col* __restrict__ ev, int64_t stride,
                                                     int vec, const int64_t* __restrict__ offsets,
                                                     int32_t toys, int stages, RfWork& W) {
  (void)stages;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int wpb = blockDim.x >> 5;
  const int64_t w = (int64_t)blockIdx.x * wpb + wib;
  const ToySplit Sp = toy_split(offsets, toys, stride, (int64_t)gridDim.x * wpb);
  const bool active = w < Sp.N && Sp.E > Sp.B;
  int64_t wb = 0, we = 0;
  int32_t t = 0;
  if (active) {
    wb = Sp.start(w);
    we = Sp.start(w + 1);
    t = find_toy(offsets, toys, stride, wb);
  }
  asm volatile("griddepcontrol.wait;" ::: "memory");
  if (!active) return;
  const RfConsts<Real>* consts = static_cast<const RfConsts<Real>*>(W.toy_consts);
  ToyState<M, Real> T;
  T.xs = W.toy_consts_x;
  T.open(consts, offsets, stride, t);
  double* rows = W.partials + w * RF_NACC_MAX;
  for (int64_t p = wb; p < we;) {
    if (!T.seek(consts, offsets, stride, toys, p, rows)) break;
    const int64_t q = we < T.te ? we : T.te;
    if (!T.bad && T.E.zero_mask == 0) {
      int64_t h = 0;
      if (vec) {
        const uintptr_t a = reinterpret_cast<uintptr_t>(ev + (int64_t)P.col_obs[0] * stride + p);
        h = (int64_t)(((16u - (a & 15u)) & 15u) / sizeof(Col));
        if (h > q - p) h = q - p;
      }
      const int64_t nfull = full_chunks<EPT>(q - p - h, vec != 0);
      // the chunk loop without the per-event zero-coefficient test (with it,
      // the 4096 Gauss + Exponential toys ran 43.8 instructions per event,
      // without it 37.7, at 8 events per lane)
      stream_chunks<M, Real, Col, EPT, false>(P, T.E, ev, stride, p + h, lane, 32, nfull,
                                              vec != 0, T.acc);
      iterate_scalar<M, Real, Col>(P, T.E, ev, stride, p + lane, p + h, T.acc, 32);
      iterate_scalar<M, Real, Col>(P, T.E, ev, stride, p + h + nfull * EPT + lane, q, T.acc, 32);
    } else if (!T.bad) {
      // a toy with a coefficient exactly zero (rare): the event loop with the
      // test, one event per lane at a time (a second copy of the chunk loop
      // measured 14% slower for all toys)
      iterate_scalar<M, Real, Col>(P, T.E, ev, stride, p + lane, q, T.acc, 32);
    }
    T.any = true;
    p = q;
  }
  T.close(rows);
}

}  // namespace rf
