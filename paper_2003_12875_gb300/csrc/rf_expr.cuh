// rf_expr.cuh -- device side of formula leaves (PDFs given as text, the
// formula PDFs of Sec. 4): forward-mode dual numbers that the translated
// formula is written in, and the FP64 normalisation kernel body.
//
// A formula's value carries its derivatives with respect to the leaf's
// parameters (Dual<Real, N>: value v and d[j] = dv/dp_j); the observable and
// the literals are plain Real, so parameter-free subexpressions cost what they
// cost without derivatives.  The per-event leaf is u = log2 f, g_j = f_j / f;
// its normalisation I = int f over the range and dI/dp_j are taken in FP64 by
// composite Gauss-Legendre quadrature, 16 nodes on each of 128 equal panels.
#pragma once

namespace rf {

template <typename R, int N>
struct Dual {
  R v;
  R d[N];
  static __device__ __forceinline__ Dual var(R value, int j) {
    Dual a;
    a.v = value;
#pragma unroll
    for (int i = 0; i < N; ++i) a.d[i] = i == j ? R(1) : R(0);
    return a;
  }
};

// a one-argument function of a dual: value fv and slope s = f'(a.v)
template <typename R, int N>
__device__ __forceinline__ Dual<R, N> chain(const Dual<R, N>& a, R fv, R s) {
  Dual<R, N> r;
  r.v = fv;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = s * a.d[i];
  return r;
}

template <typename R, int N>
__device__ __forceinline__ Dual<R, N> operator-(const Dual<R, N>& a) {
  return chain(a, -a.v, R(-1));
}
template <typename R, int N>
__device__ __forceinline__ Dual<R, N> operator+(const Dual<R, N>& a, const Dual<R, N>& b) {
  Dual<R, N> r;
  r.v = a.v + b.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] + b.d[i];
  return r;
}
template <typename R, int N>
__device__ __forceinline__ Dual<R, N> operator-(const Dual<R, N>& a, const Dual<R, N>& b) {
  Dual<R, N> r;
  r.v = a.v - b.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] - b.d[i];
  return r;
}
template <typename R, int N>
__device__ __forceinline__ Dual<R, N> operator*(const Dual<R, N>& a, const Dual<R, N>& b) {
  Dual<R, N> r;
  r.v = a.v * b.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * b.v + a.v * b.d[i];
  return r;
}
template <typename R, int N>
__device__ __forceinline__ Dual<R, N> operator/(const Dual<R, N>& a, const Dual<R, N>& b) {
  Dual<R, N> r;
  const R ib = R(1) / b.v;
  r.v = a.v * ib;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = (a.d[i] - r.v * b.d[i]) * ib;
  return r;
}
// with a plain value on one side
template <typename R, int N>
__device__ __forceinline__ Dual<R, N> operator+(const Dual<R, N>& a, R b) {
  Dual<R, N> r = a;
  r.v = a.v + b;
  return r;
}
template <typename R, int N>
__device__ __forceinline__ Dual<R, N> operator+(R a, const Dual<R, N>& b) {
  return b + a;
}
template <typename R, int N>
__device__ __forceinline__ Dual<R, N> operator-(const Dual<R, N>& a, R b) {
  Dual<R, N> r = a;
  r.v = a.v - b;
  return r;
}
template <typename R, int N>
__device__ __forceinline__ Dual<R, N> operator-(R a, const Dual<R, N>& b) {
  return chain(b, a - b.v, R(-1));
}
template <typename R, int N>
__device__ __forceinline__ Dual<R, N> operator*(const Dual<R, N>& a, R b) {
  return chain(a, a.v * b, b);
}
template <typename R, int N>
__device__ __forceinline__ Dual<R, N> operator*(R a, const Dual<R, N>& b) {
  return chain(b, a * b.v, a);
}
template <typename R, int N>
__device__ __forceinline__ Dual<R, N> operator/(const Dual<R, N>& a, R b) {
  const R ib = R(1) / b;
  return chain(a, a.v * ib, ib);
}
template <typename R, int N>
__device__ __forceinline__ Dual<R, N> operator/(R a, const Dual<R, N>& b) {
  const R ib = R(1) / b.v, v = a * ib;
  return chain(b, v, -v * ib);
}

// the functions a formula may call, for plain values and duals
namespace fx {
__device__ __forceinline__ float exp(float a) { return ::expf(a); }
__device__ __forceinline__ double exp(double a) { return ::exp(a); }
__device__ __forceinline__ float log(float a) { return ::logf(a); }
__device__ __forceinline__ double log(double a) { return ::log(a); }
__device__ __forceinline__ float sqrt(float a) { return ::sqrtf(a); }
__device__ __forceinline__ double sqrt(double a) { return ::sqrt(a); }
__device__ __forceinline__ float sin(float a) { return ::sinf(a); }
__device__ __forceinline__ double sin(double a) { return ::sin(a); }
__device__ __forceinline__ float cos(float a) { return ::cosf(a); }
__device__ __forceinline__ double cos(double a) { return ::cos(a); }
__device__ __forceinline__ float tanh(float a) { return ::tanhf(a); }
__device__ __forceinline__ double tanh(double a) { return ::tanh(a); }
__device__ __forceinline__ float sinh(float a) { return ::sinhf(a); }
__device__ __forceinline__ double sinh(double a) { return ::sinh(a); }
__device__ __forceinline__ float cosh(float a) { return ::coshf(a); }
__device__ __forceinline__ double cosh(double a) { return ::cosh(a); }
__device__ __forceinline__ float asinh(float a) { return ::asinhf(a); }
__device__ __forceinline__ double asinh(double a) { return ::asinh(a); }
__device__ __forceinline__ float atan(float a) { return ::atanf(a); }
__device__ __forceinline__ double atan(double a) { return ::atan(a); }
__device__ __forceinline__ float erf(float a) { return ::erff(a); }
__device__ __forceinline__ double erf(double a) { return ::erf(a); }
__device__ __forceinline__ float erfc(float a) { return ::erfcf(a); }
__device__ __forceinline__ double erfc(double a) { return ::erfc(a); }
__device__ __forceinline__ float abs(float a) { return ::fabsf(a); }
__device__ __forceinline__ double abs(double a) { return ::fabs(a); }

template <typename R>
__device__ __forceinline__ R two_over_sqrt_pi() {
  return R(1.1283791670955125739);
}

template <typename R, int N>
__device__ __forceinline__ Dual<R, N> exp(const Dual<R, N>& a) {
  const R v = exp(a.v);
  return chain(a, v, v);
}
template <typename R, int N>
__device__ __forceinline__ Dual<R, N> log(const Dual<R, N>& a) {
  return chain(a, log(a.v), R(1) / a.v);
}
template <typename R, int N>
__device__ __forceinline__ Dual<R, N> sqrt(const Dual<R, N>& a) {
  const R v = sqrt(a.v);
  return chain(a, v, R(0.5) / v);
}
template <typename R, int N>
__device__ __forceinline__ Dual<R, N> sin(const Dual<R, N>& a) {
  return chain(a, sin(a.v), cos(a.v));
}
template <typename R, int N>
__device__ __forceinline__ Dual<R, N> cos(const Dual<R, N>& a) {
  return chain(a, cos(a.v), -sin(a.v));
}
template <typename R, int N>
__device__ __forceinline__ Dual<R, N> tanh(const Dual<R, N>& a) {
  const R v = tanh(a.v);
  return chain(a, v, R(1) - v * v);
}
template <typename R, int N>
__device__ __forceinline__ Dual<R, N> sinh(const Dual<R, N>& a) {
  return chain(a, sinh(a.v), cosh(a.v));
}
template <typename R, int N>
__device__ __forceinline__ Dual<R, N> cosh(const Dual<R, N>& a) {
  return chain(a, cosh(a.v), sinh(a.v));
}
template <typename R, int N>
__device__ __forceinline__ Dual<R, N> asinh(const Dual<R, N>& a) {
  return chain(a, asinh(a.v), R(1) / sqrt(R(1) + a.v * a.v));
}
template <typename R, int N>
__device__ __forceinline__ Dual<R, N> atan(const Dual<R, N>& a) {
  return chain(a, atan(a.v), R(1) / (R(1) + a.v * a.v));
}
template <typename R, int N>
__device__ __forceinline__ Dual<R, N> erf(const Dual<R, N>& a) {
  return chain(a, erf(a.v), two_over_sqrt_pi<R>() * exp(-a.v * a.v));
}
template <typename R, int N>
__device__ __forceinline__ Dual<R, N> erfc(const Dual<R, N>& a) {
  return chain(a, erfc(a.v), -two_over_sqrt_pi<R>() * exp(-a.v * a.v));
}
template <typename R, int N>
__device__ __forceinline__ Dual<R, N> abs(const Dual<R, N>& a) {
  return chain(a, abs(a.v), a.v < R(0) ? R(-1) : R(1));
}

// a^K for an integer literal K: repeated squaring, any sign of a
template <int K, typename R>
__device__ __forceinline__ R powi_plain(R a) {
  if (K < 0) return R(1) / powi_plain<(K < 0 ? -K : 1), R>(a);
  R r = R(1), b = a;
#pragma unroll
  for (int e = K; e > 0; e >>= 1) {
    if (e & 1) r *= b;
    b *= b;
  }
  return r;
}
template <int K>
__device__ __forceinline__ float powi(float a) {
  return powi_plain<K, float>(a);
}
template <int K>
__device__ __forceinline__ double powi(double a) {
  return powi_plain<K, double>(a);
}
template <int K, typename R, int N>
__device__ __forceinline__ Dual<R, N> powi(const Dual<R, N>& a) {
  if (K == 0) return chain(a, R(1), R(0));
  return chain(a, powi_plain<K, R>(a.v), R(K) * powi_plain<(K == 0 ? 0 : K - 1), R>(a.v));
}

// a^b = exp(b log a) otherwise
__device__ __forceinline__ float pow(float a, float b) { return exp(b * log(a)); }
__device__ __forceinline__ double pow(double a, double b) { return exp(b * log(a)); }
template <typename R, int N>
__device__ __forceinline__ Dual<R, N> pow(const Dual<R, N>& a, R b) {
  return exp(b * log(a));
}
template <typename R, int N>
__device__ __forceinline__ Dual<R, N> pow(R a, const Dual<R, N>& b) {
  return exp(b * log(a));
}
template <typename R, int N>
__device__ __forceinline__ Dual<R, N> pow(const Dual<R, N>& a, const Dual<R, N>& b) {
  return exp(b * log(a));
}
}  // namespace fx

// a formula's result as a dual (a parameter-free formula is a plain value)
template <class D>
__device__ __forceinline__ D dual_const(D a) {
#pragma unroll
  for (int i = 0; i < (int)(sizeof(a.d) / sizeof(a.d[0])); ++i) a.d[i] = 0;
  return a;
}
template <class D>
__device__ __forceinline__ D as_dual(float v) {
  D a;
  a.v = v;
  return dual_const(a);
}
template <class D>
__device__ __forceinline__ D as_dual(double v) {
  D a;
  a.v = v;
  return dual_const(a);
}
template <class D>
__device__ __forceinline__ D as_dual(const D& a) {
  return a;
}

// Per-event formula leaf: u = add + log2 f, g_j = (df/dp_j) / f for wanted j.
template <class F, typename Real, int GM>
__device__ __forceinline__ void formula_leaf(Real x, const Real* __restrict__ pc, Real& u,
                                             Real (&g)[RF_LEAF_MAXP], Real add = Real(-0.0)) {
  const auto f = F::template eval<Real>(x, pc);
  // the log and reciprocal of the built-in leaves (hardware approximations
  // in FP32); the formula's own functions keep CUDA's accurate versions
  u = Fn<Real>::lg2(f.v) + add;  // base-2 units, as the built-in leaves
  const Real r = Fn<Real>::rcp(f.v);
#pragma unroll
  for (int j = 0; j < RF_LEAF_MAXP; ++j)
    g[j] = (j < F::NP && ((GM >> j) & 1)) ? f.d[j < F::NP ? j : 0] * r : Real(0);
}

// Normalisation of formula leaf k (FP64): composite 16-point Gauss-Legendre on
// RF_FORMULA_PANELS equal panels, one node per thread, blocks of 128 threads,
// gridDim.x = RF_FORMULA_BLOCKS.  Each block writes its partial sums (value
// and the NP derivatives) in a fixed-order tree; the last block to finish
// (ticket) adds the partials in block order and writes, for the prologue,
// out[0] = log I (NaN when I is not positive and finite) and out[1+j] =
// (dI/dp_j) / I.
template <class F>
__device__ __forceinline__ void formula_norm_body(const RfProgram& P, int k,
                                                  const double* __restrict__ params,
                                                  const double* gl_t, const double* gl_w,
                                                  double* part, unsigned int* ticket,
                                                  double* out) {
  constexpr int NP = F::NP, NV = 1 + NP;
  __shared__ double red[4][NV];
  __shared__ int s_last;
  asm volatile("griddepcontrol.launch_dependents;");
  const RfLeafProg& L = P.leaf[k];
  double th[RF_LEAF_MAXP] = {0.0, 0.0, 0.0, 0.0};
  for (int j = 0; j < NP; ++j) th[j] = params[L.par[j]];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;  // node
  const int panel = i >> 4, node = i & 15;
  const double h = (L.hi - L.lo) / RF_FORMULA_PANELS;
  const double x = L.lo + h * (panel + 0.5 + 0.5 * gl_t[node]);
  const double wt = 0.5 * h * gl_w[node];
  const auto f = F::template eval<double>(x, th);
  double v[NV];
  v[0] = wt * f.v;
#pragma unroll
  for (int j = 0; j < NP; ++j) v[1 + j] = wt * f.d[j];
#pragma unroll
  for (int c = 0; c < NV; ++c) {
    double s = v[c];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5][c] = s;
  }
  __syncthreads();
  if (threadIdx.x < NV) {
    const int c = threadIdx.x;
    part[(k * RF_FORMULA_BLOCKS + blockIdx.x) * RF_FORMULA_NV + c] =
        (red[0][c] + red[1][c]) + (red[2][c] + red[3][c]);
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(&ticket[k], 1u) == gridDim.x - 1 ? 1 : 0;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  __shared__ double tot[NV];
  if (threadIdx.x < NV) {
    const int c = threadIdx.x;
    double s = 0.0;
    for (int b = 0; b < (int)gridDim.x; ++b)
      s += *((volatile double*)&part[(k * RF_FORMULA_BLOCKS + b) * RF_FORMULA_NV + c]);
    tot[c] = s;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const double I = tot[0];
    const bool ok = I > 0.0 && isfinite(I);
    out[k * RF_FORMULA_NV] = ok ? ::log(I) : __longlong_as_double(0x7ff8000000000000ll);
    for (int j = 0; j < RF_LEAF_MAXP; ++j)
      out[k * RF_FORMULA_NV + 1 + j] = (ok && j < NP) ? tot[1 + j] / I : 0.0;
    ticket[k] = 0u;
  }
}

}  // namespace rf
