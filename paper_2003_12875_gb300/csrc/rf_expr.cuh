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

// ------------------------------------------------------------------ Hypatia2
// Modified Bessel function of the second kind of real order from its integral
// representation K_nu(z) = int_0^inf e^{-z cosh t} cosh(nu t) dt (z > 0), by
// the trapezoid rule (exponentially convergent for this analytic, rapidly
// decaying integrand; Trefethen & Weideman, SIAM Review 56 (2014) 385) on the
// scaled integrand phi(t) = e^{-z (cosh t - 1)} with step h = 0.2/sqrt(max(1, z))
// (the integrand's width shrinks as 1/sqrt(z)), summed until past the peak
// t* = asinh(|nu|/z) the largest moment's term is below eps of the sum (FP64
// 1e-17, FP32 1e-9).  cosh t - 1 = expm1(t)^2 / (2 e^t), without cancellation.
// s0 = e^z K, s1 = e^z dK/dz, s2 = e^z dK/dnu, s3 = e^z d2K/dz2,
// s4 = e^z d2K/dz dnu.
template <typename R>
struct BesselKSums {
  R s0, s1, s2, s3, s4;
};

template <typename R>
__device__ __noinline__ BesselKSums<R> besselk_sums(R nu, R z) {
  const R h = R(0.2) / fx::sqrt(z > R(1) ? z : R(1));
  const R an = fx::abs(nu), tp = fx::asinh(an / z);
  const R eps = sizeof(R) == 4 ? R(1e-9) : R(1e-17);
  // t = 0 carries half weight: phi = 1, cosh t = 1, cosh(nu t) = 1, sinh = 0
  R s[5] = {R(0.5), R(-0.5), R(0), R(0.5), R(0)};
  // FP32: Kahan compensation on every sum (some twenty terms of order one
  // each; their rounding repeats for events of similar z, so it would not
  // average out over a dataset)
  R c[5] = {R(0), R(0), R(0), R(0), R(0)};
  for (int j = 1; j < 4000; ++j) {
    const R t = R(j) * h;
    const R em = expm1(t), et = em + R(1);
    const R chm1 = em * em / (R(2) * et), ch = chm1 + R(1);
    const R ph = fx::exp(-z * chm1);
    const R en = fx::exp(an * t), ien = R(1) / en;
    const R cn = R(0.5) * (en + ien), sn = copysign(R(0.5) * (en - ien), nu);
    const R pcn = ph * cn, psn = ph * sn;
    const R v[5] = {pcn, -(ch * pcn), t * psn, ch * ch * pcn, -(t * ch * psn)};
#pragma unroll
    for (int i = 0; i < 5; ++i) {
      if constexpr (sizeof(R) == 4) {
        const R y = v[i] - c[i], tt = s[i] + y;
        c[i] = (tt - s[i]) - y;
        s[i] = tt;
      } else {
        s[i] += v[i];
      }
    }
    if (t > tp && v[3] <= eps * s[0]) break;
  }
  return BesselKSums<R>{h * (s[0] - c[0]), h * (s[1] - c[1]), h * (s[2] - c[2]),
                        h * (s[3] - c[3]), h * (s[4] - c[4])};
}

// log K_nu(z) and d log K_nu / dz as duals, their derivatives through nu, z
template <typename R, int N>
__device__ __forceinline__ Dual<R, N> log_besselk(const Dual<R, N>& nu, const Dual<R, N>& z) {
  const BesselKSums<R> S = besselk_sums(nu.v, z.v);
  const R q1 = S.s1 / S.s0, q2 = S.s2 / S.s0;
  Dual<R, N> r;
  r.v = fx::log(S.s0) - z.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = q2 * nu.d[i] + q1 * z.d[i];
  return r;
}
template <typename R, int N>
__device__ __forceinline__ Dual<R, N> dlog_besselk(const Dual<R, N>& nu, const Dual<R, N>& z) {
  const BesselKSums<R> S = besselk_sums(nu.v, z.v);
  const R q1 = S.s1 / S.s0, q2 = S.s2 / S.s0;
  Dual<R, N> r;
  r.v = q1;
#pragma unroll
  for (int i = 0; i < N; ++i)
    r.d[i] = (S.s4 / S.s0 - q1 * q2) * nu.d[i] + (S.s3 / S.s0 - q1 * q1) * z.d[i];
  return r;
}

// Hypatia2 (the paper names it among the improved PDFs; the form is a
// reading): parameters p = (lambda, zeta, beta, sigma, mu, a, n, a2, n2).
// With d = x - mu, phi = K_{lambda+1}(zeta)/K_lambda(zeta),
// delta = sigma sqrt(zeta/phi), alpha = sqrt(zeta phi)/sigma, nu = lambda - 1/2:
//   core  L(d) = (nu/2) log(d^2 + delta^2) + beta d + log K_nu(alpha r) + zeta,
//         r = sqrt(d^2 + delta^2) (a generalised hyperbolic density up to a
//         constant; + zeta keeps e^L of order one near the peak),
//   tails below d_L = -a sigma and above d_R = a2 sigma:
//         L(d_J) - m log(1 - (d - d_J) k(d_J)/m), (d_J, m) = (d_L, n) or (d_R, n2),
//         k(d) = dL/dd = nu d/(d^2 + delta^2) + beta + alpha (d/r) dlogK/dz(alpha r),
// so value and slope are continuous at both junctions.  log f = -inf where a
// tail's base is not positive; NaN for parameters outside their domain.
struct Hypatia2Leaf {
  static constexpr int NP = 9;
  // the normalisation kernel exports log phi and its derivatives in lambda
  // and zeta (FP64) into the row of the leaf's second slot
  static constexpr int kShapeRow = 1;
  template <typename R, int N>
  static __device__ __forceinline__ Dual<R, N> core(const Dual<R, N>& d, const Dual<R, N>& nu,
                                                    const Dual<R, N>& beta,
                                                    const Dual<R, N>& alpha,
                                                    const Dual<R, N>& delta2, Dual<R, N>* slope) {
    const Dual<R, N> q = d * d + delta2, r = fx::sqrt(q), z = alpha * r;
    const Dual<R, N> L = (R(0.5) * (nu * fx::log(q)) + beta * d) + log_besselk(nu, z);
    if (slope) *slope = (nu * d / q + beta) + (alpha * d / r) * dlog_besselk(nu, z);
    return L;
  }
  static __device__ __forceinline__ bool in_domain(const double* p) {
    return p[1] > 0.0 && p[3] > 0.0 && p[5] > 0.0 && p[6] > 0.0 && p[7] > 0.0 && p[8] > 0.0;
  }
  template <typename R>
  static __device__ __forceinline__ bool in_domain(const R* p) {
    return p[1] > R(0) && p[3] > R(0) && p[5] > R(0) && p[6] > R(0) && p[7] > R(0) && p[8] > R(0);
  }
  // log f - zeta and its derivatives d/dp_j from the nine parameters p[0..8]
  // and the per-call shape constants p[9..22] (computed once in FP64):
  // delta^2 and its derivatives in (lambda, zeta, sigma) p[9..12], alpha and
  // its derivatives in the same three p[13..16], then the low FP32 parts of
  // those six derivatives p[17..22] (zero in FP64).  zeta enters only through
  // delta^2 and alpha: the per-event sums then carry no constant term (the
  // prologue takes zeta off log I and 1 off d log I/d zeta instead).  The
  // duals carry d/d delta^2 (slot 1) and d/d alpha (slot 9) rather than the
  // chain through them, which is applied at the end with the derivatives as
  // hi + lo pairs: rounded once per call, those would otherwise shift every
  // event's derivative alike.
  template <typename R>
  static __device__ __noinline__ Dual<R, 9> logf_shaped(R x, const R* __restrict__ p) {
    using D = Dual<R, 10>;
    const D lam = D::var(p[0], 0), beta = D::var(p[2], 2);
    const D sigma = D::var(p[3], 3), mu = D::var(p[4], 4), a = D::var(p[5], 5);
    const D n = D::var(p[6], 6), a2 = D::var(p[7], 7), n2 = D::var(p[8], 8);
    const D delta2 = D::var(p[9], 1), alpha = D::var(p[13], 9);
    D L;
    if (!in_domain<R>(p)) {
      L.v = R(0) / R(0);
#pragma unroll
      for (int i = 0; i < 10; ++i) L.d[i] = R(0);
    } else {
      const D nu = lam - R(0.5);
      const D d = x - mu;
      const D dL = -(a * sigma), dR = a2 * sigma;
      if (d.v < dL.v || d.v > dR.v) {
        const bool left = d.v < dL.v;
        const D dJ = left ? dL : dR, m = left ? n : n2;
        D k;
        const D LJ = core<R, 10>(dJ, nu, beta, alpha, delta2, &k);
        const D base = R(1) - (d - dJ) * k / m;
        if (!(base.v > R(0))) {
          L.v = -R(1) / R(0);
#pragma unroll
          for (int i = 0; i < 10; ++i) L.d[i] = R(0);
        } else {
          L = LJ - m * fx::log(base);
        }
      } else {
        L = core<R, 10>(d, nu, beta, alpha, delta2, nullptr);
      }
    }
    // chain rule through delta^2 and alpha, the products of the high parts
    // first, then those of the low parts
    const R A = L.d[1], B = L.d[9];
    Dual<R, 9> out;
    out.v = L.v;
#pragma unroll
    for (int i = 0; i < 9; ++i) out.d[i] = L.d[i];
    out.d[0] = L.d[0] + fma(A, p[10], B * p[14]) + fma(A, p[17], B * p[20]);
    out.d[1] = fma(A, p[11], B * p[15]) + fma(A, p[18], B * p[21]);
    out.d[3] = L.d[3] + fma(A, p[12], B * p[16]) + fma(A, p[19], B * p[22]);
    return out;
  }
  // log f and d log f / dp_j from the nine parameters alone (FP64, for the
  // normalisation kernel): log phi = log K_{lambda+1}(zeta) - log K_lambda(zeta)
  // computed here, and written as (value, d/d lambda, d/d zeta) to lp_out when
  // it is given (NaN outside the domain); log f includes the + zeta of the
  // core
  template <typename R>
  static __device__ __forceinline__ Dual<R, 9> logf(R x, const R* __restrict__ p,
                                                    R* lp_out = nullptr) {
    using D = Dual<R, 9>;
    R q[23];
#pragma unroll
    for (int j = 0; j < 9; ++j) q[j] = p[j];
#pragma unroll
    for (int j = 17; j < 23; ++j) q[j] = R(0);
    if (!in_domain<R>(p)) {
      if (lp_out) lp_out[0] = lp_out[1] = lp_out[2] = R(0) / R(0);
      return logf_shaped<R>(x, q);
    }
    const D lam = D::var(p[0], 0), zeta = D::var(p[1], 1), sigma = D::var(p[3], 3);
    const D logphi = log_besselk(lam + R(1), zeta) - log_besselk(lam, zeta);
    if (lp_out) lp_out[0] = logphi.v, lp_out[1] = logphi.d[0], lp_out[2] = logphi.d[1];
    const D logz = fx::log(zeta), logs = fx::log(sigma);
    const D delta2 = fx::exp(R(2) * logs + (logz - logphi));
    const D alpha = fx::exp(R(0.5) * (logz + logphi) - logs);
    q[9] = delta2.v, q[10] = delta2.d[0], q[11] = delta2.d[1], q[12] = delta2.d[3];
    q[13] = alpha.v, q[14] = alpha.d[0], q[15] = alpha.d[1], q[16] = alpha.d[3];
    D L = logf_shaped<R>(x, q);
    if (L.v > -R(1) / R(0)) {  // + zeta keeps e^L of order one near the peak
      L.v += p[1];
      L.d[1] += R(1);
    }
    return L;
  }
  // f and df/dp_j (for the normalisation kernel)
  template <typename R>
  static __device__ __forceinline__ Dual<R, 9> eval(R x, const R* __restrict__ p,
                                                    R* lp_out = nullptr) {
    const Dual<R, 9> L = logf<R>(x, p, lp_out);
    if (!(L.v > -R(1) / R(0))) {  // f = 0 (or NaN)
      Dual<R, 9> z;
      z.v = L.v == L.v ? R(0) : L.v;
#pragma unroll
      for (int i = 0; i < 9; ++i) z.d[i] = R(0);
      return z;
    }
    return fx::exp(L);
  }
  // the normalisation's pieces: [lo, mu - a sigma], [mu - a sigma,
  // mu + a2 sigma], [mu + a2 sigma, hi], clipped to the range
  static __device__ __forceinline__ int cuts(const double* p, double lo, double hi, double* c) {
    c[0] = lo;
    c[1] = fmin(fmax(p[4] - p[5] * p[3], lo), hi);
    c[2] = fmin(fmax(p[4] + p[7] * p[3], lo), hi);
    c[3] = hi;
    return 3;
  }
};

// The per-event Hypatia2 leaf: u = add + log2 f, g_j = d log f/dp_j for the
// wanted j (GM9: bit j for parameter j).  Its nine parameters and fourteen
// shape constants sit in three consecutive leaf slots of the per-event
// constants: row k p0..p3 then delta^2 (value, d/d lambda, d/d zeta,
// d/d sigma), row k+1 p4..p7 then alpha (the same four), row k+2 p8 then the
// low parts of delta^2's three derivatives and of alpha's.
template <typename Real, int GM9>
__device__ __forceinline__ void hypatia2_leaf(Real x, const Real* __restrict__ pc, Real& u,
                                              Real (&g)[9], Real add = Real(-0.0)) {
  Real p[23];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    p[j] = pc[j];
    p[4 + j] = pc[RF_PC + j];
    p[9 + j] = pc[4 + j];
    p[13 + j] = pc[RF_PC + 4 + j];
  }
  p[8] = pc[2 * RF_PC];
#pragma unroll
  for (int j = 0; j < 6; ++j) p[17 + j] = pc[2 * RF_PC + 1 + j];
  const Dual<Real, 9> L = Hypatia2Leaf::logf_shaped<Real>(x, p);
  u = L.v * Real(1.44269504088896340736) + add;
#pragma unroll
  for (int j = 0; j < 9; ++j) g[j] = ((GM9 >> j) & 1) ? L.d[j] : Real(0);
}

// Normalisation of formula leaf k (FP64): composite 16-point Gauss-Legendre on
// RF_FORMULA_PANELS equal panels, one node per thread, blocks of 128 threads,
// gridDim.x = RF_FORMULA_BLOCKS.  Each block writes its partial sums (value
// and the NP derivatives) in a fixed-order tree; the last block to finish
// (ticket) adds the partials in block order and writes, for the prologue,
// out[0] = log I (NaN when I is not positive and finite) and out[1+j] =
// (dI/dp_j) / I.
// F::cuts (where a leaf's normalisation must be split into pieces), if F has it
template <class F, class = void>
struct HasCuts {
  static constexpr bool v = false;
};
template <class F>
struct HasCuts<F, decltype((void)&F::cuts)> {
  static constexpr bool v = true;
};

// F::kShapeRow (a leaf that exports per-call shape constants), if F has it
template <class F, class = void>
struct HasShape {
  static constexpr bool v = false;
};
template <class F>
struct HasShape<F, decltype((void)F::kShapeRow)> {
  static constexpr bool v = true;
};
template <class F>
__device__ __forceinline__ auto norm_eval(double x, const double* th, double* sh) {
  if constexpr (HasShape<F>::v)
    return F::template eval<double>(x, th, sh);
  else
    return F::template eval<double>(x, th);
}

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
  // parameters j >= 4 sit in the slots after the leaf's (four per slot)
  double th[NP > 0 ? NP : 1];
  for (int j = 0; j < NP; ++j) th[j] = params[P.leaf[k + (j >> 2)].par[j & 3]];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;  // node
  int panel = i >> 4;
  const int node = i & 15;
  double a = L.lo, h = (L.hi - L.lo) / RF_FORMULA_PANELS;
  if constexpr (HasCuts<F>::v) {
    // panels shared among the pieces in proportion to their lengths (at
    // least one each), so that no panel straddles a piece's end
    double c[4];
    const int np = F::cuts(th, L.lo, L.hi, c);
    int first = 0;
    for (int q = 0; q < np; ++q) {
      const double len = c[q + 1] - c[q];
      int cnt = (int)(RF_FORMULA_PANELS * len / (L.hi - L.lo));
      if (len > 0.0 && cnt < 1) cnt = 1;
      if (q == np - 1 || first + cnt > RF_FORMULA_PANELS) cnt = RF_FORMULA_PANELS - first;
      if (panel < first + cnt || q == np - 1) {
        a = c[q];
        h = cnt > 0 ? len / cnt : 0.0;
        panel -= first;
        break;
      }
      first += cnt;
    }
  }
  const double x = a + h * (panel + 0.5 + 0.5 * gl_t[node]);
  const double wt = 0.5 * h * gl_w[node];
  double* sh = nullptr;  // one node's thread writes the leaf's shape constants
  if constexpr (HasShape<F>::v)
    if (blockIdx.x == 0 && threadIdx.x == 0) sh = out + (k + F::kShapeRow) * RF_FORMULA_NV;
  const auto f = norm_eval<F>(x, th, sh);
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
    for (int j = 0; j < RF_FORMULA_NV - 1; ++j)
      out[k * RF_FORMULA_NV + 1 + j] = (ok && j < NP) ? tot[1 + j] / I : 0.0;
    ticket[k] = 0u;
  }
}

}  // namespace rf
