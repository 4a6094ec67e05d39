// rf_device.cuh -- device building blocks of the fused NLL + adjoint kernels.
//
//  * FP64 normalisation integrals I_k and d log I_k / d theta (the parameter-
//    only "constant branches" of Sec. 5.1, hoisted out of the event loop),
//  * per-event leaf log-densities and their parameter derivatives in the
//    evaluation precision (FP32 or FP64), branch-free where the paper's
//    Sec. 5.3 replaces branches by selects,
//  * compensated per-thread accumulation, a fixed-order FP64 block/grid
//    reduction (deterministic for a fixed launch configuration),
//  * the FP64 epilogue that turns the accumulated sums into the NLL and
//    its gradient, including the normalisation-integral derivatives.
//
// Leaf definitions (the paper prints none; standard forms):
//  Gaussian    f = exp(-(x-mu)^2/(2 sigma^2))
//  Exponential f = exp(lambda x)
//  Chebychev   f = 1 + sum_j c_j T_j(x'), x' = (2x - lo - hi)/(hi - lo)
//  CrystalBall t = s (x-m0)/sigma, s = sign(alpha), A = |alpha|:
//              f = exp(-t^2/2) (t > -A), else exp(-A^2/2) D^-n,
//              D = 1 - (A/n)(A + t)
//  ARGUS       f = x tau^(1/2) exp(c tau), tau = 1 - (x/m0)^2 (x < m0)
#pragma once
#ifndef __CUDACC_RTC__
#include <cuda_runtime.h>
#endif
#include "rf_internal.h"

namespace rf {

__device__ __forceinline__ double kInf() { return __longlong_as_double(0x7ff0000000000000LL); }
__device__ __forceinline__ double kNaN() { return __longlong_as_double(0x7ff8000000000000LL); }

constexpr double kSqrt2 = 1.41421356237309504880;
constexpr double kInvSqrt2 = 0.70710678118654752440;
constexpr double kSqrtHalfPi = 1.25331413731550025121;
constexpr double kSqrtPi = 1.77245385090551602730;
// The per-event code works in base-2 log units (u / ln 2): the hardware's
// lg2 and ex2 then need no conversion factor, and the FP64 epilogue turns the
// summed log-likelihood back into natural units once.
constexpr double kLn2 = 0.693147180559945309417;
constexpr double kLog2e = 1.44269504088896340736;
// sqrt(log2(e) / 2): the Gaussian's -d^2/2 in base-2 units is -(kG d)^2
constexpr double kG = 0.84932180028801904272;

// ------------------------------------------------------------------ FP64 math
// One out-of-line copy of each FP64 function the prologue calls: the prologue
// runs once per call on a few threads, so code size (instruction-cache misses
// on cold code) matters more than call overhead.
static __device__ __noinline__ double d_exp(double x) { return exp(x); }
static __device__ __noinline__ double d_log(double x) { return log(x); }
static __device__ __noinline__ double d_erf(double x) { return erf(x); }
static __device__ __noinline__ double d_erfc(double x) { return erfc(x); }
static __device__ __noinline__ double d_expm1(double x) { return expm1(x); }
static __device__ __noinline__ double d_pow(double x, double y) { return pow(x, y); }

__device__ inline double erf_diff(double z1, double z2) {  // d_erf(z2)-d_erf(z1)
  if (z1 >= 0.0) return d_erfc(z1) - d_erfc(z2);
  if (z2 <= 0.0) return d_erfc(-z2) - d_erfc(-z1);
  return d_erf(z2) - d_erf(z1);
}

// (e^y - 1)/y and its derivative d/dy = (e^y (y - 1) + 1) / y^2.  The
// derivative's closed form cancels near 0, where the Taylor series
// sum_{k>=1} k y^(k-1) / (k+1)! is summed by Horner's rule instead (22 terms:
// the first omitted one is below 2^-60 of the sum for |y| < 1).  ey = e^y is
// passed in by the caller, which needs it anyway.
__device__ inline double expm1_over(double y) {
  return y == 0.0 ? 1.0 : d_expm1(y) / y;
}
struct ExpmSeries {
  double c[23];
  __host__ __device__ constexpr ExpmSeries() : c() {
    double f = 1.0;
    for (int k = 1; k <= 22; ++k) {
      f *= (double)(k + 1);
      c[k] = (double)k / f;
    }
  }
};
__device__ inline double expm1_over_d(double y, double ey) {
  if (fabs(y) < 1.0) {
    constexpr ExpmSeries S;
    double acc = S.c[22];
#pragma unroll
    for (int k = 21; k >= 1; --k) acc = fma(acc, y, S.c[k]);
    return acc;
  }
  return (ey * (y - 1.0) + 1.0) / (y * y);
}

// J_q(tau) = int_0^tau s^q e^{c s} ds for q = 1/2 and q = 3/2, and e^{c tau}.
// For c < 0 and -c tau >= 1/2 the incomplete-gamma closed forms share one erf
// and one exp: with k = -c, u = k tau, gamma(3/2, u) = (sqrt(pi)/2) erf(sqrt u)
// - sqrt(u) e^-u, gamma(5/2, u) = (3/2) gamma(3/2, u) - u^(3/2) e^-u, and
// J_q = gamma(q + 1, u) / k^(q + 1).  Otherwise both power series
// J_q = tau^(q+1) sum_j (c tau)^j / (j! (j + q + 1)) run in one loop.
__device__ inline void argus_int2(double tau, double c, double* J12, double* J32,
                                  double* ect) {
  if (tau <= 0.0) {
    *J12 = *J32 = 0.0;
    *ect = 1.0;
    return;
  }
  const double y = c * tau;
  if (c < 0.0 && -y >= 0.5) {
    const double k = -c, u = -y, su = sqrt(u), eu = d_exp(-u), sk = sqrt(k);
    const double g32 = 0.5 * kSqrtPi * d_erf(su) - su * eu;
    const double g52 = 1.5 * g32 - u * su * eu;
    *J12 = g32 / (k * sk);
    *J32 = g52 / (k * k * sk);
    *ect = eu;
    return;
  }
  double s12 = 0.0, s32 = 0.0, term = 1.0;
  for (int j = 0; j < 2000; ++j) {
    const double a12 = term / (j + 1.5), a32 = term / (j + 2.5);
    s12 += a12;
    s32 += a32;
    if (j > fabs(y) && fabs(a12) < 1e-18 * fabs(s12) && fabs(a32) < 1e-18 * fabs(s32)) break;
    term *= y / (j + 1.0);
  }
  const double st = tau * sqrt(tau);
  *J12 = st * s12;
  *J32 = st * tau * s32;
  *ect = d_exp(y);
}

// d_log(I) - off and d(log I - off)/d theta_j for one leaf (FP64).  `off` is
// the constant the per-event code leaves out of u = log f - off (Exponential:
// lambda * lo, so that u = lambda (x - lo) stays small).  Returns false when
// the parameters are outside the leaf's definition range.
// ARGUS with a general power p, s = p + 1 > 1: J(t) = int_0^t tau^p e^{c tau}
// d tau and dJ/dp, for 0 <= t <= 1.  Both series have positive terms only:
//   c <= 0 (k = -c): J = t^s e^{ct} sum_n T_n, T_n = (kt)^n / (s (s+1) ... (s+n))
//     (the lower incomplete gamma's Kummer series, J = gamma(s, kt) / k^s);
//     dJ/ds = log(t) J - t^s e^{ct} sum_n T_n H_n, H_n = sum_{j<=n} 1/(s+j)
//   c > 0: J = t^s sum_n U_n, U_n = (ct)^n / (n! (s+n));
//     dJ/ds = log(t) J - t^s sum_n U_n / (s+n)
// The terms grow while n < |c| t, then fall; the sums stop once a term is
// below 1e-18 of its sum past that point.
__device__ inline void argus_jp(double t, double c, double s, double* J, double* dJ) {
  if (t <= 0.0) {
    *J = 0.0;
    *dJ = 0.0;
    return;
  }
  const double y = fabs(c) * t, lt = d_log(t), ts = d_exp(s * lt);
  double sum = 0.0, dsum = 0.0;
  if (c <= 0.0) {
    double T = 1.0 / s, H = 1.0 / s;
    for (int n = 0; n < 4000; ++n) {
      sum += T;
      dsum += T * H;
      if (n > y && T < 1e-18 * sum) break;
      T *= y / (s + n + 1.0);
      H += 1.0 / (s + n + 1.0);
    }
    const double e = d_exp(c * t);
    *J = ts * e * sum;
    *dJ = lt * *J - ts * e * dsum;
  } else {
    double a = 1.0;  // (ct)^n / n!
    for (int n = 0; n < 4000; ++n) {
      const double U = a / (s + n);
      sum += U;
      dsum += U / (s + n);
      if (n > y && U < 1e-18 * sum) break;
      a *= y / (n + 1.0);
    }
    *J = ts * sum;
    *dJ = lt * *J - ts * dsum;
  }
}

// gm: the leaf's gradient mask (ARGUS: bit 2 selects the general-p form)
static __device__ __noinline__ bool leaf_lognorm(int type, int gm, const double* th, double lo,
                                    double hi, double* lnI, double* dln) {
  for (int j = 0; j < RF_LEAF_MAXP; ++j) dln[j] = 0.0;
  switch (type) {
    case RFL_GAUSS: {
      double mu = th[0], sg = th[1];
      if (!(sg > 0.0)) return false;
      double za = (lo - mu) / sg, zb = (hi - mu) / sg;
      double I = sg * kSqrtHalfPi * erf_diff(za / kSqrt2, zb / kSqrt2);
      double pa = d_exp(-0.5 * za * za), pb = d_exp(-0.5 * zb * zb);
      *lnI = d_log(I);
      dln[0] = (pa - pb) / I;
      dln[1] = 1.0 / sg + (za * pa - zb * pb) / I;
      return I > 0.0 && isfinite(I);
    }
    case RFL_EXP: {
      // I = e^{lambda lo} L E1(lambda L); off = lambda lo.
      double lam = th[0], L = hi - lo, s = lam * L;
      *lnI = d_log(L * expm1_over(s));
      // d log I / d lambda - lo = <x> - lo = L (1/(1-e^-s) - 1/s)
      double m = (fabs(s) < 1e-3)
                     ? 0.5 + s / 12.0 - s * s * s / 720.0 + s * s * s * s * s / 30240.0
                     : 1.0 / (-d_expm1(-s)) - 1.0 / s;
      dln[0] = L * m;
      return isfinite(*lnI);
    }
    case RFL_CHEB: {
      // int_{-1}^1 T_j = (1 + (-1)^j)/(1 - j^2), 0 for j = 1
      double half = 0.5 * (hi - lo), J = 2.0, dJ[RF_LEAF_MAXP];
      for (int j = 1; j <= RF_LEAF_MAXP; ++j) {
        double tj = (j & 1) ? 0.0 : 2.0 / (1.0 - (double)(j * j));
        J += th[j - 1] * tj;
        dJ[j - 1] = tj;
      }
      if (!(J > 0.0)) return false;
      *lnI = d_log(half * J);
      for (int j = 0; j < RF_LEAF_MAXP; ++j) dln[j] = dJ[j] / J;
      return true;
    }
    case RFL_CB: {
      double m0 = th[0], sg = th[1], al = th[2], n = th[3];
      if (!(sg > 0.0) || !(n > 0.0) || al == 0.0) return false;
      double s = al > 0.0 ? 1.0 : -1.0, A = fabs(al);
      double tlo = (s > 0.0) ? (lo - m0) / sg : (m0 - hi) / sg;
      double thi = (s > 0.0) ? (hi - m0) / sg : (m0 - lo) / sg;
      double core = 0.0;
      if (thi > -A) core = kSqrtHalfPi * erf_diff(fmax(tlo, -A) / kSqrt2, thi / kSqrt2);
      double tail = 0.0, dA = 0.0, dn = 0.0;
      const double eA = d_exp(-0.5 * A * A);
      // integrand g(t) at the two range ends; in the tail g = e^{-A^2/2} D^-n
      // = e^{-A^2/2 - n log D}, which reuses the logs the tail integral needs
      double glo = 0.0, ghi = 0.0;
      if (tlo < -A) {
        // substitute D = 1 - (A/n)(A+t): tail = (n/A) e^{-A^2/2} int D^-n dD
        double D1 = 1.0 - (A / n) * (A + tlo);
        double t2 = fmin(thi, -A);
        double D2 = 1.0 - (A / n) * (A + t2);
        double L1 = d_log(D1), L2 = (t2 == -A) ? 0.0 : d_log(D2), dL = L1 - L2, eps = 1.0 - n;
        double ez = (L2 == 0.0) ? 1.0 : d_exp(eps * L2);                // D2^(1-n)
        // y = (1-n) log(D1/D2): e^y and e^y - 1 from one call (e^y - 1 is
        // only formed by subtraction where it cannot cancel, |y| >= 1)
        const double y = eps * dL;
        double ey, em1;
        if (fabs(y) >= 1.0) {
          ey = d_exp(y);
          em1 = ey - 1.0;
        } else {
          em1 = d_expm1(y);
          ey = 1.0 + em1;
        }
        double Phi = ez * dL * (y == 0.0 ? 1.0 : em1 / y);               // int D^-n
        double PhiL = L2 * Phi + ez * dL * dL * expm1_over_d(y, ey);     // int D^-n log D
        // D^-n = D^(1-n) / D at both ends
        double p1 = ez * ey / D1, p2 = (L2 == 0.0) ? 1.0 : ez / D2;
        double Psi = (p2 - p1) / n;                                      // int D^-n-1
        double pre = (n / A) * eA;
        tail = pre * Phi;
        dA = pre * (A + n / A) * (Psi - Phi);
        dn = pre * (Phi - PhiL - Psi);
        glo = eA * p1;
        if (thi <= -A) ghi = eA * p2;
      } else {
        glo = d_exp(-0.5 * tlo * tlo);
      }
      if (thi > -A) ghi = d_exp(-0.5 * thi * thi);
      double J = core + tail;
      double I = sg * J;
      *lnI = d_log(I);
      dln[0] = -s * (ghi - glo) / I;
      dln[1] = (J + tlo * glo - thi * ghi) / I;
      dln[2] = s * dA / J;
      dln[3] = dn / J;
      return I > 0.0 && isfinite(I);
    }
    case RFL_JOHNSON: {
      // u = -log(1 + z^2)/2 - w^2/2 per event (z = (x-mu)/lambda, w = gamma +
      // delta asinh z): I = lambda sqrt(2 pi)/delta (Phi(w(hi)) - Phi(w(lo)))
      double mu = th[0], lam = th[1], gam = th[2], del = th[3];
      if (!(lam > 0.0) || !(del > 0.0)) return false;
      double za = (lo - mu) / lam, zb = (hi - mu) / lam;
      double asa = asinh(za), asb = asinh(zb);
      double wa = gam + del * asa, wb = gam + del * asb;
      double dP = 0.5 * erf_diff(wa / kSqrt2, wb / kSqrt2);
      double pa = d_exp(-0.5 * wa * wa) * 0.3989422804014327;
      double pb = d_exp(-0.5 * wb * wb) * 0.3989422804014327;
      double ra = sqrt(1.0 + za * za), rb = sqrt(1.0 + zb * zb);
      *lnI = d_log(lam * 2.5066282746310002 / del * dP);
      dln[0] = (pb * (-del / (lam * rb)) - pa * (-del / (lam * ra))) / dP;
      dln[1] = 1.0 / lam + (pb * (-del * zb / (lam * rb)) - pa * (-del * za / (lam * ra))) / dP;
      dln[2] = (pb - pa) / dP;
      dln[3] = -1.0 / del + (pb * asb - pa * asa) / dP;
      return dP > 0.0 && isfinite(*lnI);
    }
    case RFL_ARGUS: {
      double m0 = th[0], c = th[1], p = th[2];
      if (!(m0 > lo) || lo < 0.0) return false;
      double b = fmin(hi, m0);
      double ta = 1.0 - (lo / m0) * (lo / m0), tb = 1.0 - (b / m0) * (b / m0);
      double h = 0.5 * m0 * m0;
      if (gm & (4 | RF_ARGUS_GENERAL)) {  // general p (free, or fixed away from 1/2)
        if (!(p > 0.0)) return false;
        // I = (m0^2/2) [J(tau_a) - J(tau_b)]; d/dc takes J at p + 1; d/dm0
        // adds the limits' motion: 2I/m0 + (lo^2/m0) tau_a^p e^{c tau_a}
        // - (b'^2/m0) tau_b^p e^{c tau_b}
        double Ja, Pa, Jb, Pb, Ka, Kb, dummy;
        argus_jp(ta, c, p + 1.0, &Ja, &Pa);
        argus_jp(tb, c, p + 1.0, &Jb, &Pb);
        argus_jp(ta, c, p + 2.0, &Ka, &dummy);
        argus_jp(tb, c, p + 2.0, &Kb, &dummy);
        const double I = h * (Ja - Jb);
        const double ea = ta > 0.0 ? d_exp(p * d_log(ta) + c * ta) : 0.0;
        const double eb = tb > 0.0 ? d_exp(p * d_log(tb) + c * tb) : 0.0;
        *lnI = d_log(I);
        dln[0] = (2.0 * I / m0 + (lo * lo / m0) * ea - (b * b / m0) * eb) / I;
        dln[1] = h * (Ka - Kb) / I;
        dln[2] = h * (Pa - Pb) / I;
        return I > 0.0 && isfinite(I);
      }
      if (p != 0.5) return false;  // the p = 1/2 form was compiled for this leaf
      double Ja, Ka, Ea, Jb, Kb, Eb;
      argus_int2(ta, c, &Ja, &Ka, &Ea);
      argus_int2(tb, c, &Jb, &Kb, &Eb);
      double I = h * (Ja - Jb);
      double dIc = h * (Ka - Kb);
      double ea = (1.0 - ta) * sqrt(ta) * Ea;
      double eb = tb > 0.0 ? (1.0 - tb) * sqrt(tb) * Eb : 0.0;
      double dIm = m0 * (ea - eb) + 2.0 * I / m0;
      // log I + log m0: the per-event p = 1/2 form carries log m0 (leaf_argus);
      // the derivatives stay those of log I, like the per-event ones, and
      // the two constants cancel in the gradient
      *lnI = d_log(I * m0);
      dln[0] = dIm / I;
      dln[1] = dIc / I;
      return I > 0.0 && isfinite(I);
    }
  }
  return false;
}

// The Gaussian's and the Exponential's log I and d log I/d theta on an
// aligned lane pair: both lanes call it, lane e (0 or 1) takes range end e of
// each pair of like transcendental functions (the two ends' erf and exp for
// the Gaussian, e^s - 1 and e^-s - 1 for the Exponential), so the FP64 unit
// evaluates both in one pass (it takes one warp instruction at a time however
// many lanes are active), then both lanes finish with the same values.
// Same formulas as leaf_lognorm; reciprocals are formed once and multiplied.
static __device__ __noinline__ bool lognorm_pair(int type, const double* th, double lo,
                                                 double hi, int e, double* lnI, double* dln) {
  const unsigned pm = 3u << ((threadIdx.x & 31) & 30);
  for (int j = 0; j < RF_LEAF_MAXP; ++j) dln[j] = 0.0;
  if (type == RFL_GAUSS) {
    const double mu = th[0], sg = th[1];
    if (!(sg > 0.0)) return false;
    const double rs = 1.0 / sg;
    const double za = (lo - mu) * rs, zb = (hi - mu) * rs;
    // erfc at both ends on one side of the mean (no cancellation), else erf
    const int mode = za >= 0.0 ? 0 : (zb <= 0.0 ? 1 : 2);
    const double z = e ? zb : za, w = z * kInvSqrt2;
    const double F = mode == 2 ? d_erf(w) : d_erfc(mode == 0 ? w : -w);
    const double g = d_exp(-0.5 * z * z);
    const double Fo = __shfl_xor_sync(pm, F, 1), go = __shfl_xor_sync(pm, g, 1);
    const double Fa = e ? Fo : F, Fb = e ? F : Fo, pa = e ? go : g, pb = e ? g : go;
    const double I = sg * kSqrtHalfPi * (mode == 0 ? Fa - Fb : Fb - Fa);
    *lnI = d_log(I);
    const double rI = 1.0 / I;
    dln[0] = (pa - pb) * rI;
    dln[1] = rs + (za * pa - zb * pb) * rI;
    return I > 0.0 && isfinite(I);
  }
  // Exponential: I = e^{lambda lo} L (e^s - 1)/s with s = lambda L (off =
  // lambda lo); d log I/d lambda - lo = L (1/(1 - e^-s) - 1/s)
  const double lam = th[0], L = hi - lo, s = lam * L;
  const double q = d_expm1(e ? -s : s);
  const double qo = __shfl_xor_sync(pm, q, 1);
  const double q0 = e ? qo : q, q1 = e ? q : qo;
  // one division pass: lane 0 (e^s - 1)/s, lane 1 1/(1 - e^-s) - 1/s
  const double r = e ? (s + q1) / (-s * q1) : q0 / s;
  const double ro = __shfl_xor_sync(pm, r, 1);
  const double E = s == 0.0 ? 1.0 : (e ? ro : r), M = e ? r : ro;
  *lnI = d_log(L * E);
  const double m = (fabs(s) < 1e-3)
                       ? 0.5 + s / 12.0 - s * s * s / 720.0 + s * s * s * s * s / 30240.0
                       : M;
  dln[0] = L * m;
  return isfinite(*lnI);
}

// --------------------------------------------------------- prologue (FP64)
template <typename Real>
__device__ inline void split_hi_lo(double v, Real& hi, Real& lo) {
  hi = (Real)v;
  lo = (Real)(v - (double)hi);
}

// Leaf L's per-event constants in type T from its parameters th (FP64):
// location-like values split into T pairs (hi, lo), the rest rounded to T.
template <typename T>
__device__ inline void leaf_pc(const RfLeafProg& L, const double* th, T* pc) {
  for (int j = 0; j < RF_PC; ++j) pc[j] = T(0);
  switch (L.type) {
    case RFL_GAUSS: {  // d = kG (x - mu) / sigma, so that u (base 2) = -d^2
      T lo;
      split_hi_lo(th[0], pc[0], lo);
      pc[2] = (T)(kG / th[1]);
      pc[1] = (T)(-(double)lo * (double)pc[2]);
      break;
    }
    case RFL_EXP:
      pc[0] = (T)(th[0] * kLog2e);  // lambda in base-2 units
      split_hi_lo(L.lo, pc[1], pc[2]);
      break;
    case RFL_CHEB:  // x' = (x - mid) * (2/(hi-lo))
      pc[0] = (T)(2.0 / (L.hi - L.lo));
      pc[1] = (T)(-(L.hi + L.lo) / (L.hi - L.lo));
      for (int j = 0; j < RF_LEAF_MAXP; ++j) pc[2 + j] = (T)th[j];
      break;
    case RFL_CB: {
      // s = kG t, t = s_alpha (x - m0)/sigma
      const double sg = th[2] > 0.0 ? 1.0 : -1.0, A = fabs(th[2]), n = th[3];
      T lo;
      split_hi_lo(th[0], pc[0], lo);
      pc[2] = (T)(kG * sg / th[1]);
      pc[1] = (T)(-(double)lo * (double)pc[2]);
      pc[3] = (T)(1.0 - A * A / n);        // D = pc[3] + pc[5] s
      pc[4] = (T)(-kG * A);                // the tail: s <= pc[4]
      pc[5] = (T)(-A / (n * kG));
      pc[6] = (T)(-n);
      pc[7] = (T)(-0.5 * A * A * kLog2e);
      break;
    }
    case RFL_JOHNSON: {
      T lo;
      split_hi_lo(th[0], pc[0], lo);
      pc[2] = (T)(1.0 / th[1]);
      pc[1] = (T)(-(double)lo * (double)pc[2]);
      pc[3] = (T)th[2];
      pc[4] = (T)th[3];
      break;
    }
    case RFL_FORMULA:  // the formula runs on the parameters rounded to T
    case RFL_HYPATIA2:
    case RFL_PARAMS:
      for (int j = 0; j < L.npar; ++j) pc[j] = (T)th[j];
      break;
    case RFL_ARGUS: {
      // m0^2 as the exact pair sq + e (e = the FMA's rounding error of the
      // product), then as T's hi + lo
      const double sq = th[0] * th[0], e = fma(th[0], th[0], -sq);
      pc[0] = (T)sq;
      pc[1] = (T)((sq - (double)pc[0]) + e);
      pc[2] = (T)(1.0 / sq);
      pc[3] = (T)(th[1] * kLog2e);  // c in base-2 units (for u)
      pc[4] = (T)(th[1] * kLog2e / sq);  // the same over m0^2 (the p = 1/2 form)
      split_hi_lo(th[2], pc[5], pc[7]);  // p (general-p form), hi + lo
      pc[6] = (T)th[1];  // c (for the m0 derivative)
      break;
    }
  }
}

// Hypatia2's shape constants (per call, FP64): with phi = K_{lambda+1}(zeta)/
// K_lambda(zeta) and log phi's derivatives in lambda and zeta (exported by
// the normalisation kernel), delta^2 = sigma^2 zeta/phi and alpha =
// sqrt(zeta phi)/sigma, each as (value, d/d lambda, d/d zeta, d/d sigma).
// Slot 0 of the leaf (k0) takes delta^2's four in columns 4..7, slot 1
// alpha's, slot 2 the low parts (v - (T)v) of the six derivatives in columns
// 1..6.  k is one of the leaf's three slots.
template <typename T>
__device__ __forceinline__ void hyp2_shape_pc(const RfProgram& P, int k, const double* params,
                                              T* pc) {
  const RfLeafProg& L = P.leaf[k];
  const int part = L.type == RFL_PARAMS ? L.part : 0;
  const int k0 = k - part;
  const RfLeafProg& M = P.leaf[k0];
  const double zeta = params[M.par[1]], sigma = params[M.par[3]];
  const double* sh = P.formula_norm + (k0 + 1) * RF_FORMULA_NV;
  const double lp = sh[0], dl = sh[1], dz = sh[2];
  const double d2 = sigma * sigma * zeta * exp(-lp);
  const double al = sqrt(zeta * exp(lp)) / sigma;
  const double v[8] = {d2, -d2 * dl, d2 * (1.0 / zeta - dz), 2.0 * d2 / sigma,
                       al, 0.5 * al * dl, 0.5 * al * (1.0 / zeta + dz), -al / sigma};
  if (part < 2) {
    for (int j = 0; j < 4; ++j) pc[4 + j] = (T)v[4 * part + j];
  } else {
    for (int j = 0; j < 3; ++j) {
      pc[1 + j] = (T)(v[1 + j] - (double)(T)v[1 + j]);
      pc[4 + j] = (T)(v[5 + j] - (double)(T)v[5 + j]);
    }
  }
}
__device__ __forceinline__ bool hyp2_shape_slot(const RfLeafProg& L) {
  return L.type == RFL_HYPATIA2 || L.type == RFL_PARAMS;
}

// Leaf k's per-event constants: K.pc[k], K.dtheta[k], K.gmul[k] (nothing
// here needs the integral, so it runs beside leaf_norm).
template <typename Real>
__device__ __noinline__ void leaf_eval_consts(const RfProgram& P, const double* params,
                                              RfConsts<Real>& K, int k) {
  const RfLeafProg& L = P.leaf[k];
  double th[RF_LEAF_MAXP] = {0.0, 0.0, 0.0, 0.0};
  for (int j = 0; j < L.npar; ++j) th[j] = params[L.par[j]];
  Real* pc = K.pc[k];
  leaf_pc<Real>(L, th, pc);
  if (hyp2_shape_slot(L)) hyp2_shape_pc<Real>(P, k, params, pc);
  for (int j = 0; j < RF_LEAF_MAXP; ++j) {
    K.dtheta[k][j] = 0.0;
    K.gmul[k][j] = 1.0;
  }
  // dtheta: the parameter value the per-event code uses (through its rounded
  // constants) minus the parameter; gmul: the constant factor of d u/d theta
  // that the per-event sums leave out
  switch (L.type) {
    case RFL_GAUSS:
      K.dtheta[k][1] = kG / (double)pc[2] - th[1];
      K.gmul[k][0] = 1.0 / (kG * th[1]);         // d u/d mu = (x - mu)/sigma^2 = d / (kG sigma)
      K.gmul[k][1] = 1.0 / (kG * kG * th[1]);    // d u/d sigma = d^2 / (kG^2 sigma)
      break;
    case RFL_EXP:
      K.dtheta[k][0] = kLn2 * (double)pc[0] - th[0];
      break;
    case RFL_CHEB:
      for (int j = 0; j < RF_LEAF_MAXP; ++j) K.dtheta[k][j] = (double)pc[2 + j] - th[j];
      break;
    case RFL_CB: {
      // per event h = -kG du/dt (t = s_alpha (x - m0)/sigma), h s = -kG^2 t du/dt
      const double sg = th[2] > 0.0 ? 1.0 : -1.0;
      K.dtheta[k][1] = kG / fabs((double)pc[2]) - th[1];
      K.gmul[k][0] = sg / (kG * th[1]);        // d u/d m0 = -(s_alpha/sigma) du/dt
      K.gmul[k][1] = 1.0 / (kG * kG * th[1]);  // d u/d sigma = -(t/sigma) du/dt
      K.gmul[k][2] = sg / kG;                  // d u/d alpha = s_alpha d u/d|alpha|
      break;
    }
    case RFL_JOHNSON:
      K.dtheta[k][1] = 1.0 / (double)pc[2] - th[1];
      K.dtheta[k][2] = (double)pc[3] - th[2];
      K.dtheta[k][3] = (double)pc[4] - th[3];
      K.gmul[k][0] = K.gmul[k][1] = -1.0 / th[1];  // d u/d mu = -du/dz / lambda, etc.
      K.gmul[k][2] = K.gmul[k][3] = -1.0;         // d u/d gamma = -w, d u/d delta = -w asinh z
      break;
    case RFL_FORMULA:  // first-order correction through dtheta, as for the built-ins
    case RFL_HYPATIA2:
    case RFL_PARAMS:
      for (int j = 0; j < L.npar; ++j) K.dtheta[k][j] = (double)pc[j] - th[j];
      // Hypatia2's zeta reaches the per-event code only through the FP64
      // shape constants
      if (L.type == RFL_HYPATIA2) K.dtheta[k][1] = 0.0;
      break;
    case RFL_ARGUS:
      if (L.gmask & (4 | RF_ARGUS_GENERAL)) {
        K.dtheta[k][1] = kLn2 * (double)pc[3] - th[1];
      } else {  // p = 1/2: c' = c log2(e)/m0^2 per event, d u/d c = tq/m0^2
        K.dtheta[k][1] = kLn2 * (double)pc[4] * (th[0] * th[0]) - th[1];
        K.gmul[k][1] = 1.0 / (th[0] * th[0]);
      }
      if (L.gmask & 4) K.dtheta[k][2] = ((double)pc[5] + (double)pc[7]) - th[2];
      K.gmul[k][0] = 2.0 / th[0];  // d u/d m0 = (2/m0) (p/tau + c)(1 - tau)
      break;
  }
}

// Leaf k's log I and d log I/d theta (K.lnI[k], K.dlogI[k] and lnI_out);
// false when its parameters are outside the leaf's definition range.
template <typename Real>
__device__ __noinline__ bool leaf_norm(const RfProgram& P, const double* params,
                                       RfConsts<Real>& K, int k, double* lnI_out) {
  const RfLeafProg& L = P.leaf[k];
  double th[RF_LEAF_MAXP] = {0.0, 0.0, 0.0, 0.0};
  for (int j = 0; j < L.npar; ++j) th[j] = params[L.par[j]];
  double dln[RF_LEAF_MAXP] = {0.0, 0.0, 0.0, 0.0};
  bool ok;
  if (L.type == RFL_FORMULA || L.type == RFL_HYPATIA2) {
    // log I and (dI/dp_j)/I from the normalisation kernel (NaN: I <= 0)
    const double* nrm = P.formula_norm + k * RF_FORMULA_NV;
    *lnI_out = nrm[0];
    for (int j = 0; j < RF_LEAF_MAXP; ++j) dln[j] = nrm[1 + j];
    ok = isfinite(*lnI_out);
    if (L.type == RFL_HYPATIA2) {
      // the per-event code evaluates f e^{-zeta} (its core's + zeta left out),
      // so its integral is I e^{-zeta}
      *lnI_out -= th[1];
      dln[1] -= 1.0;
    }
  } else if (L.type == RFL_PARAMS) {
    // parameters 4 part .. of the leaf `part` slots before: their share of
    // that leaf's (dI/dp_j)/I; the integral itself is counted there
    const double* nrm = P.formula_norm + (k - L.part) * RF_FORMULA_NV;
    *lnI_out = 0.0;
    for (int j = 0; j < RF_LEAF_MAXP; ++j) {
      const int q = RF_LEAF_MAXP * L.part + j;
      dln[j] = q < RF_FORMULA_MAXP ? nrm[1 + q] : 0.0;
    }
    ok = true;
  } else {
    ok = leaf_lognorm(L.type, L.gmask, th, L.lo, L.hi, lnI_out, dln);
  }
  K.lnI[k] = *lnI_out;
  for (int j = 0; j < RF_LEAF_MAXP; ++j) K.dlogI[k][j] = dln[j];
  return ok;
}

// leaf_norm on an aligned lane pair (both lanes call it; lane e = threadIdx.x
// & 1): the Gaussian and the Exponential split their range ends over the two
// lanes (lognorm_pair), the other leaves run on the pair's first lane.  Only
// the first lane writes K and lnI_out and its return value counts.
template <typename Real>
__device__ __noinline__ bool leaf_norm_pair(const RfProgram& P, const double* params,
                                            RfConsts<Real>& K, int k, double* lnI_out) {
  const RfLeafProg& L = P.leaf[k];
  const int e = threadIdx.x & 1;
  if (L.type == RFL_GAUSS || L.type == RFL_EXP) {
    double th[RF_LEAF_MAXP] = {0.0, 0.0, 0.0, 0.0};
    for (int j = 0; j < L.npar; ++j) th[j] = params[L.par[j]];
    double l = 0.0, dln[RF_LEAF_MAXP];
    const bool ok = lognorm_pair(L.type, th, L.lo, L.hi, e, &l, dln);
    if (e == 0) {
      *lnI_out = l;
      K.lnI[k] = l;
      for (int j = 0; j < RF_LEAF_MAXP; ++j) K.dlogI[k][j] = dln[j];
    }
    return ok;
  }
  if (e != 0) return true;
  return leaf_norm<Real>(P, params, K, k, lnI_out);
}

// Leaf k's constants, all of them in one thread.
template <typename Real>
__device__ __forceinline__ bool leaf_consts(const RfProgram& P, const double* params,
                                            RfConsts<Real>& K, int k, double* lnI_out) {
  leaf_eval_consts<Real>(P, params, K, k);
  return leaf_norm<Real>(P, params, K, k, lnI_out);
}

// The root's coefficients from the parameters (fractions, the last one 1 -
// their sum; yields; 1 for a product), the extended term sum(nu) (weighted)
// and whether a coefficient is outside its range.
__device__ __forceinline__ void root_coefs(const RfProgram& P, const double* params,
                                           double* coef, double* ext_sum, bool* bad) {
  const int C = P.n_comp;
  for (int c = 0; c < RF_MAXC; ++c) coef[c] = 0.0;
  *ext_sum = 0.0;
  if (P.kind == RF_KIND_PROD) {
    coef[0] = 1.0;
  } else if (P.kind == RF_KIND_FRAC) {
    double rest = 1.0;
    for (int c = 0; c < C - 1; ++c) {
      double f = params[P.coef_par[c]];
      if (!(f >= 0.0 && f <= 1.0)) *bad = true;
      coef[c] = f;
      rest -= f;
    }
    if (rest < 0.0) {
      if (rest < -1e-15) *bad = true;
      rest = 0.0;
    }
    coef[C - 1] = rest;
  } else {
    for (int c = 0; c < C; ++c) {
      double v = params[P.coef_par[c]];
      if (!(v >= 0.0) || !isfinite(v)) *bad = true;
      coef[c] = v;
      *ext_sum += v;
    }
    *ext_sum *= P.ext_weight;
  }
}

// The root's coefficients made ready for comb_consts (in shared memory, so
// that the combination reads no parameter from global memory): the values,
// their logs (-inf for a zero coefficient), sum(nu) and the range check.
struct CoefPre {
  double coef[RF_MAXC];
  double logc[RF_MAXC];
  double ext_sum;
  int32_t bad;
};

// CoefPre by one warp: lane c computes log coef_c (one FP64 pass for all
// components), lane 0 writes the rest.
__device__ __forceinline__ void coef_pre_lanes(const RfProgram& P, const double* params,
                                               int lane, CoefPre* cp) {
  double coef[RF_MAXC], es;
  bool bad = false;
  root_coefs(P, params, coef, &es, &bad);
  double c = 0.0;
  for (int j = 0; j < RF_MAXC; ++j)
    if (j == lane) c = coef[j];
  if (lane < P.n_comp) cp->logc[lane] = c > 0.0 ? d_log(c) : -kInf();
  if (lane == 0) {
    for (int j = 0; j < RF_MAXC; ++j) cp->coef[j] = coef[j];
    cp->ext_sum = es;
    cp->bad = bad ? 1 : 0;
  }
}

// CoefPre by one thread (the toy prep: one lane per toy).
__device__ __forceinline__ void coef_pre_serial(const RfProgram& P, const double* params,
                                                CoefPre* cp) {
  double coef[RF_MAXC], es;
  bool bad = false;
  root_coefs(P, params, coef, &es, &bad);
  for (int j = 0; j < RF_MAXC; ++j) {
    cp->coef[j] = coef[j];
    cp->logc[j] = (j < P.n_comp && coef[j] > 0.0) ? d_log(coef[j]) : -kInf();
  }
  cp->ext_sum = es;
  cp->bad = bad ? 1 : 0;
}

// Combination constants (one thread), after every leaf's lnI is known.  X
// (may be NULL): where FP32 evaluation with a zero coefficient gets its FP64
// constants.  cp (may be NULL): the coefficients made ready (CoefPre);
// without it they are computed here.
template <typename Real>
__device__ __noinline__ void comb_consts(const RfProgram& P, const double* params,
                                   RfConsts<Real>& K, const double* lnI,
                                   bool leaves_ok, RfExact* X = nullptr,
                                   const CoefPre* cp = nullptr) {
  bool bad = !leaves_ok;
  const int C = P.n_comp;
  double coef[RF_MAXC], base[RF_MAXC];
  for (int c = 0; c < RF_MAXC; ++c) base[c] = 0.0;
  if (cp) {
    for (int c = 0; c < RF_MAXC; ++c) coef[c] = cp->coef[c];
    K.ext_sum = cp->ext_sum;
    bad |= cp->bad != 0;
  } else {
    root_coefs(P, params, coef, &K.ext_sum, &bad);
  }
  for (int k = 0; k < P.n_leaves; ++k) base[P.leaf[k].comp] -= lnI[k];
  double beta[RF_MAXC];
  double ref = -kInf();
  int zero = 0;
  for (int c = 0; c < C; ++c) {
    if (coef[c] > 0.0) {
      beta[c] = (cp ? cp->logc[c] : d_log(coef[c])) + base[c];
      ref = fmax(ref, beta[c]);
    } else {
      beta[c] = -kInf();
      zero |= 1 << c;
    }
  }
  if (!(ref > -kInf()) || !isfinite(ref)) {
    bad = true;
    ref = 0.0;
  }
  K.beta_ref = ref;
  K.zero_mask = zero;
  for (int c = 0; c < RF_MAXC; ++c) {
    K.coef[c] = coef[c];
    if (c < C && !((zero >> c) & 1)) {
      // in base-2 units per event; the remainder in natural units
      double d = beta[c] - ref;
      K.delta[c] = (Real)(d * kLog2e);
      K.delta_lo[c] = d - kLn2 * (double)K.delta[c];
    } else {
      K.delta[c] = (Real)(-kInf());
      K.delta_lo[c] = 0.0;
    }
    K.delta_nc[c] = (Real)(c < C ? (base[c] - ref) * kLog2e : 0.0);
  }
  if (sizeof(Real) == 4 && zero != 0 && X) {
    // FP32 evaluation with a zero coefficient runs every event in FP64 on the
    // exact constants (built only here, the rare case): nothing to correct
    // for rounding
    X->zero_mask = zero;
    X->n_comp = C;
    for (int c = 0; c < RF_MAXC; ++c) {
      X->delta_d[c] = (c < C && !((zero >> c) & 1)) ? (beta[c] - ref) * kLog2e : -kInf();
      X->delta_nc_d[c] = c < C ? (base[c] - ref) * kLog2e : 0.0;
      K.delta_lo[c] = 0.0;
    }
    for (int k = 0; k < P.n_leaves; ++k) {
      const RfLeafProg& L = P.leaf[k];
      double th[RF_LEAF_MAXP] = {0.0, 0.0, 0.0, 0.0};
      for (int j = 0; j < L.npar; ++j) th[j] = params[L.par[j]];
      leaf_pc<double>(L, th, X->pcd[k]);
      if (hyp2_shape_slot(L)) hyp2_shape_pc<double>(P, k, params, X->pcd[k]);
      X->lmeta[k] = (L.type & 0xff) | ((L.gmask & 0xff) << 8) | ((L.comp & 0xff) << 16) |
                    ((L.col & 0xff) << 24);
    }
    for (int k = 0; k < RF_MAXL; ++k)
      for (int j = 0; j < RF_LEAF_MAXP; ++j) K.dtheta[k][j] = 0.0;
  }
  K.bad = bad ? 1 : 0;
}

// comb_consts on an aligned group of G lanes (all 32 lanes of the warp call
// it, each group for its own dataset): component c on group lane c mod G, so
// the per-component FP64 steps (the deltas and their FP32 roundings) run in
// one pass, the reference beta_ref and the zero mask by shuffles over the
// group.  lnI of leaf k at lnI[k * lnI_stride]; cp: the coefficients made
// ready (required).  valid: the group has a dataset (false: it only takes
// part in the shuffles, writes nothing).  A call with a zero coefficient and
// X set (FP32 evaluation's exact constants) goes to comb_consts on the
// group's first lane: same values, the rare path.
template <typename Real, int G>
__device__ __forceinline__ void comb_consts_group(const RfProgram& P, const double* params,
                                                  RfConsts<Real>& K, const double* lnI,
                                                  int lnI_stride, bool leaves_ok, RfExact* X,
                                                  const CoefPre* cp, bool valid) {
  constexpr int NCL = (RF_MAXC + G - 1) / G;  // components per lane
  const int q = threadIdx.x & (G - 1);
  const int C = P.n_comp;
  double base[NCL], beta[NCL];
  double ref = -kInf();
  int zero = 0;
#pragma unroll
  for (int m = 0; m < NCL; ++m) {
    const int c = q + m * G;
    base[m] = 0.0;
    beta[m] = -kInf();
    if (c < C) {
      for (int k = 0; k < P.n_leaves; ++k)
        if (P.leaf[k].comp == c) base[m] -= lnI[k * lnI_stride];
      if (cp->coef[c] > 0.0) {
        beta[m] = cp->logc[c] + base[m];
        ref = fmax(ref, beta[m]);
      } else {
        zero |= 1 << c;
      }
    }
  }
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) {
    ref = fmax(ref, __shfl_xor_sync(0xffffffffu, ref, o));
    zero |= __shfl_xor_sync(0xffffffffu, zero, o);
  }
  bool bad = !leaves_ok || cp->bad != 0;
  if (!(ref > -kInf()) || !isfinite(ref)) {
    bad = true;
    ref = 0.0;
  }
  if (!valid) return;
  if (sizeof(Real) == 4 && zero != 0 && X) {
    if (q == 0) {
      double l[RF_MAXL];
      for (int k = 0; k < P.n_leaves; ++k) l[k] = lnI[k * lnI_stride];
      comb_consts<Real>(P, params, K, l, leaves_ok, X, cp);
    }
    return;
  }
#pragma unroll
  for (int m = 0; m < NCL; ++m) {
    const int c = q + m * G;
    if (c >= RF_MAXC) continue;
    K.coef[c] = cp->coef[c];
    if (c < C && !((zero >> c) & 1)) {
      // in base-2 units per event; the remainder in natural units
      const double d = beta[m] - ref;
      K.delta[c] = (Real)(d * kLog2e);
      K.delta_lo[c] = d - kLn2 * (double)K.delta[c];
    } else {
      K.delta[c] = (Real)(-kInf());
      K.delta_lo[c] = 0.0;
    }
    K.delta_nc[c] = (Real)(c < C ? (base[m] - ref) * kLog2e : 0.0);
  }
  if (q == 0) {
    K.beta_ref = ref;
    K.zero_mask = zero;
    K.ext_sum = cp->ext_sum;
    K.bad = bad ? 1 : 0;
  }
}

// All constants by one thread (batched prologue: one thread per toy).
template <typename Real>
__device__ inline void build_consts_serial(const RfProgram& P,
                                           const double* params,
                                           RfConsts<Real>& K) {
  double lnI[RF_MAXL];
  bool ok = true;
  for (int k = 0; k < P.n_leaves; ++k) ok &= leaf_consts(P, params, K, k, &lnI[k]);
  comb_consts(P, params, K, lnI, ok);
}

// ------------------------------------------------------------ event math
// FP32 natural logarithm of the per-event code: the hardware base-2
// logarithm (lg2.approx; the PTX specification bounds its error by 2^-22.6
// absolute for arguments in [0.5, 2] and 2^-22 relative to log2 x elsewhere)
// times ln 2.  Per-event logs enter the log-likelihood additively, so their
// absolute error is what counts: at most ~1e-7 * max(1, |log2 x|), the same
// order as a correctly rounded FP32 log of the same argument.  Zero gives
// -inf, negative arguments and NaN give NaN, +inf gives +inf (ftz: subnormal
// arguments count as zero).  This is the trade the paper makes with VDT's
// approximate log/exp (Sec. 5.3), and it is tested against an FP64
// reference and CUDA logf in the GPU tests.
__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float log_fast(float x) {
  float r;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r * 0.693147182f;
}
// exp(x) for x <= 0 through the hardware base-2 exponential (max relative
// error 2^-22 by the PTX specification) of x * log2(e).
__device__ __forceinline__ float exp_neg_approx(float x) {
  float r;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x * 1.44269504f));
  return r;
}
// The same hardware functions in base 2, as the per-event code uses them:
// lg2.approx (error as above, in log2 units) and ex2.approx (2^-22 relative;
// the mixture weights 2^-|dv| in (0, 1] thus carry an absolute error below
// 4e-8).
__device__ __forceinline__ float lg2_fast(float x) {
  float r;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float ex2_fast(float x) {
  float r;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// double -> float, round to nearest even, with integer operations only: on
// this GPU the hardware conversion runs on the FP64 pipe, which is far
// slower than the integer pipe.  For a double with a float-normal exponent
// the result is sign | (e - 896) << 23 | top 23 mantissa bits, plus one ulp
// when the dropped 29 bits exceed half an ulp (or equal it and the kept
// mantissa is odd); a carry out of the mantissa correctly bumps the
// exponent.  Zero, float-subnormal, overflowing, infinite and NaN inputs go
// through the hardware conversion.  Tested bit for bit against it.
__device__ __forceinline__ float d2f_rn(double x) {
  const unsigned hi = (unsigned)__double2hiint(x);
  const unsigned lo = (unsigned)__double2loint(x);
  const unsigned e = (hi >> 20) & 0x7ffu;
  if (e - 897u >= 253u) return __double2float_rn(x);  // float exponent outside 1..253
  unsigned bits = (hi & 0x80000000u) | ((e - 896u) << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29);
  const unsigned rem = lo & 0x1fffffffu;
  bits += (rem > 0x10000000u || (rem == 0x10000000u && (bits & 1u))) ? 1u : 0u;
  return __uint_as_float(bits);
}

template <typename To, typename From>
__device__ __forceinline__ To cvt(From x) { return (To)x; }
template <>
__device__ __forceinline__ float cvt<float, double>(double x) { return d2f_rn(x); }

template <typename Real>
struct Fn;
template <>
struct Fn<float> {
  static __device__ __forceinline__ float log(float x) { return log_fast(x); }
  // x known positive and finite wherever its result is used
  static __device__ __forceinline__ float logp(float x) { return log_fast(x); }
  static __device__ __forceinline__ float exp_neg(float x) { return exp_neg_approx(x); }
  static __device__ __forceinline__ float lg2(float x) { return lg2_fast(x); }
  static __device__ __forceinline__ float ex2(float x) { return ex2_fast(x); }
  static __device__ __forceinline__ float ex2_exact(float x) { return exp2f(x); }
  static __device__ __forceinline__ float exp(float x) { return expf(x); }
  static __device__ __forceinline__ float rcp(float x) { return rcp_approx(x); }
  // 1/x from lg2x = lg2(x), already at hand: 2^(-lg2x), one ex2 (the special
  // function unit issues ex2 at twice the rate of rcp)
  static __device__ __forceinline__ float rcp_lg(float x, float lg2x) {
    (void)x;
    return ex2_fast(-lg2x);
  }
  static __device__ __forceinline__ float sqrt(float x) { return sqrtf(x); }
  static __device__ __forceinline__ float ninf() { return -__int_as_float(0x7f800000); }
};
template <>
struct Fn<double> {
  static __device__ __forceinline__ double log(double x) { return ::log(x); }
  static __device__ __forceinline__ double logp(double x) { return ::log(x); }
  static __device__ __forceinline__ double exp_neg(double x) { return ::exp(x); }
  static __device__ __forceinline__ double lg2(double x) { return ::log2(x); }
  static __device__ __forceinline__ double ex2(double x) { return ::exp2(x); }
  static __device__ __forceinline__ double ex2_exact(double x) { return ::exp2(x); }
  static __device__ __forceinline__ double exp(double x) { return ::exp(x); }
  static __device__ __forceinline__ double rcp(double x) { return 1.0 / x; }
  static __device__ __forceinline__ double rcp_lg(double x, double lg2x) {
    (void)lg2x;
    return 1.0 / x;
  }
  static __device__ __forceinline__ double sqrt(double x) { return ::sqrt(x); }
  static __device__ __forceinline__ double ninf() { return -kInf(); }
};

// Typed leaves: u = add + (log f(x) - off) / ln 2, in base-2 units, and
// g_j = d (log f)/d theta_j in natural units (up to the constant factor gmul
// applied in the epilogue).  GM is the compile-time mask of the derivatives
// that are needed; the others are 0.  `add` is a per-call constant the caller
// wants added to u (the graph compiler folds a component's log-coefficient
// into its first leaf this way); its default -0 adds nothing (x + -0 == x
// for every x, so the addition folds away).
// Location-like parameters enter as (x - hi) * scale + lo', lo' = -lo *
// scale: the difference is exact for x near hi, and one FMA applies the
// scale and the low part.

template <typename Real, int GM>
__device__ __forceinline__ void leaf_gauss(Real x, const Real* __restrict__ pc, Real& u,
                                           Real (&g)[RF_LEAF_MAXP], Real add = Real(-0.0)) {
  const Real d = fma(x - pc[0], pc[2], pc[1]);  // kG (x - mu) / sigma
  const Real dd = d * d;
  u = add - dd;                                  // -(x - mu)^2 / (2 sigma^2) in base 2
  g[0] = (GM & 1) ? d : Real(0);       // times 1/(kG sigma) (gmul)
  g[1] = (GM & 2) ? dd : Real(0);      // times 1/(kG^2 sigma) (gmul)
  g[2] = g[3] = Real(0);
}

template <typename Real, int GM>
__device__ __forceinline__ void leaf_exp(Real x, const Real* __restrict__ pc, Real& u,
                                         Real (&g)[RF_LEAF_MAXP], Real add = Real(-0.0)) {
  const Real d = (GM & RF_GM_AT0) ? x : (x - pc[1]) - pc[2];  // x - lo
  u = fma(pc[0], d, add);
  g[0] = (GM & 1) ? d : Real(0);
  g[1] = g[2] = g[3] = Real(0);
}

template <typename Real, int GM>
__device__ __forceinline__ void leaf_cheb(Real x, const Real* __restrict__ pc, Real& u,
                                          Real (&g)[RF_LEAF_MAXP], Real add = Real(-0.0)) {
  typedef Fn<Real> F;
  const Real xp = fma(x, pc[0], pc[1]);
  const Real x2 = xp + xp;
  const Real t1 = xp, t2 = fma(x2, t1, Real(-1));
  const Real t3 = fma(x2, t2, -t1), t4 = fma(x2, t3, -t2);
  const Real f = fma(pc[5], t4, fma(pc[4], t3, fma(pc[3], t2, fma(pc[2], t1, Real(1)))));
  u = F::lg2(f) + add;
  if (GM & 15) {
    const Real r = F::rcp(f);
    g[0] = (GM & 1) ? t1 * r : Real(0);
    g[1] = (GM & 2) ? t2 * r : Real(0);
    g[2] = (GM & 4) ? t3 * r : Real(0);
    g[3] = (GM & 8) ? t4 * r : Real(0);
  } else {
    g[0] = g[1] = g[2] = g[3] = Real(0);
  }
}

// Crystal Ball, in s = kG s_alpha (x - m0)/sigma (the core is then -s^2 in
// base 2): tail for s <= pc[4] = -kG A, D = 1 - (A/n)(A + t) = pc[3] + pc[5] s,
// u = add + pc[7] - n log2 D there; both pieces are evaluated and one is
// selected (no divergence).  Derivatives (times gmul): h = pc[4] / D in the
// tail, s in the core (-kG du/dt); h s; the tail's d/dA and d/dn.
template <typename Real, int GM>
__device__ __forceinline__ void leaf_cb(Real x, const Real* __restrict__ pc, Real& u,
                                        Real (&g)[RF_LEAF_MAXP], Real add = Real(-0.0)) {
  typedef Fn<Real> F;
  const Real s = fma(x - pc[0], pc[2], pc[1]);
  const bool tail = s <= pc[4];
  const Real D = fma(pc[5], s, pc[3]);
  const Real Lg = F::lg2(D);  // log2 D, used only in the tail, where D >= 1
  u = tail ? fma(pc[6], Lg, pc[7] + add) : fma(-s, s, add);
  if (GM & 15) {
    const Real rD = F::rcp_lg(D, Lg);  // used in the tail, where D >= 1
    const Real h = tail ? pc[4] * rD : s;
    g[0] = (GM & 1) ? h : Real(0);
    g[1] = (GM & 2) ? h * s : Real(0);
    g[2] = (GM & 4) ? (tail ? fma(s - Real(2) * pc[4], rD, pc[4]) : Real(0)) : Real(0);
    g[3] = (GM & 8) ? (tail ? fma(Real(-kLn2), Lg, Real(1) - rD) : Real(0)) : Real(0);
  } else {
    g[0] = g[1] = g[2] = g[3] = Real(0);
  }
}

// ARGUS: u = log x + p log tau + c tau, -inf at and above m0, with
// tau = (m0^2 - x^2) / m0^2 (m0^2 = pc[0] + pc[1]; one FMA forms m0^2 - x^2
// from the exact square, so tau keeps its relative precision near m0).  In the general form (GM bit 2: p free, or
// RF_ARGUS_GENERAL: p fixed away from 1/2) p = pc[5] + pc[7], and with bit 2
// d u/d p = log tau; otherwise p is 1/2 and u = (1/2) log2(x^2 tau) + c tau
// (one log; x^2 tau clamped at 0 gives -inf at and above m0, where the
// component's weight, and so every derivative term, is 0), evaluated on
// m0^2 - x^2 itself (see the p = 1/2 branch).
template <typename Real, int GM>
__device__ __forceinline__ void leaf_argus(Real x, const Real* __restrict__ pc, Real& u,
                                           Real (&g)[RF_LEAF_MAXP], Real add = Real(-0.0)) {
  typedef Fn<Real> F;
  const Real tq = fma(-x, x, pc[0]) + pc[1];  // m0^2 - x^2
  constexpr bool general = (GM & (4 | RF_ARGUS_GENERAL)) != 0;
  Real tau;
  if (general) {
    tau = tq * pc[2];
    // pc[3] = c log2(e) for u (base 2)
    const Real ct = fma(pc[3], tau, add);
    const bool ok = tau > Real(0);
    // p = pc[5] + pc[7] (hi + lo: a fixed p has no d/dp sum to correct its
    // rounding with)
    const Real lt = F::lg2(tau);
    u = ok ? fma(pc[7], lt, fma(pc[5], lt, ct) + F::lg2(x)) : F::ninf();
    g[2] = ((GM & 4) && ok) ? Real(kLn2) * lt : Real(0);
    g[1] = (GM & 2) ? tau : Real(0);
  } else {
    // p = 1/2 on the unnormalised tq = m0^2 tau: u = (1/2) log2(x^2 tq) +
    // c' tq with c' = c log2(e)/m0^2 (pc[4]), the form above plus log2 m0
    // (the prologue adds ln m0 to log I), one multiply fewer per event
    u = fma(Real(0.5), F::lg2(fmax(x * x * tq, Real(0))), fma(pc[4], tq, add));
    g[2] = Real(0);
    g[1] = (GM & 2) ? tq : Real(0);  // times 1/m0^2 (gmul)
    if (GM & 1) tau = tq * pc[2];
  }
  if (GM & 1) {
    // pc[6] = c
    const Real p = general ? pc[5] : Real(0.5);
    const Real r = F::rcp(tau);
    g[0] = tau > Real(0) ? (p * r + pc[6]) * (Real(1) - tau) : Real(0);  // times 2/m0 (gmul)
  } else {
    g[0] = Real(0);
  }
  g[3] = Real(0);
}

// Johnson's SU: t = 1 + z^2, u = -(log t + w^2)/2 with w = gamma + delta asinh z
// (asinh z = sign(z) log(|z| + sqrt t)); du/dz = -(z + w delta sqrt t)/t.
// Constant factors (-1/lambda, -1) are applied to the sums (gmul).
template <typename Real, int GM>
__device__ __forceinline__ void leaf_johnson(Real x, const Real* __restrict__ pc, Real& u,
                                             Real (&g)[RF_LEAF_MAXP], Real add = Real(-0.0)) {
  typedef Fn<Real> F;
  const Real z = fma(x - pc[0], pc[2], pc[1]);
  const Real t = fma(z, z, Real(1));
  const Real r = F::sqrt(t);
  const Real as = copysign(F::logp(fabs(z) + r), z);
  const Real w = fma(pc[4], as, pc[3]);
  u = fma(Real(-0.5), F::lg2(t), fma(Real(-0.5 * kLog2e) * w, w, add));
  if (GM & 3) {
    const Real dudz = -(z + w * pc[4] * r) * F::rcp(t);
    g[0] = (GM & 1) ? dudz : Real(0);
    g[1] = (GM & 2) ? dudz * z : Real(0);
  } else {
    g[0] = g[1] = Real(0);
  }
  g[2] = (GM & 4) ? w : Real(0);
  g[3] = (GM & 8) ? w * as : Real(0);
}

// Runtime dispatch (the generic, precompiled model): all derivatives are
// computed; the accumulation step keeps the ones in the leaf's gmask.
template <typename Real>
__device__ __forceinline__ void eval_leaf(int type, int gm, Real x,
                                          const Real* __restrict__ pc, Real& u,
                                          Real (&g)[RF_LEAF_MAXP]) {
  switch (type) {
    case RFL_GAUSS: leaf_gauss<Real, 3>(x, pc, u, g); break;
    case RFL_EXP: leaf_exp<Real, 1>(x, pc, u, g); break;
    case RFL_CHEB: leaf_cheb<Real, 15>(x, pc, u, g); break;
    case RFL_CB: leaf_cb<Real, 15>(x, pc, u, g); break;
    case RFL_ARGUS:
      if (gm & (4 | RF_ARGUS_GENERAL)) leaf_argus<Real, 7>(x, pc, u, g);
      else if (gm & 1) leaf_argus<Real, 3>(x, pc, u, g);
      else leaf_argus<Real, 2>(x, pc, u, g);
      break;
    case RFL_JOHNSON: leaf_johnson<Real, 15>(x, pc, u, g); break;
    default:
      u = Real(0);
      g[0] = g[1] = g[2] = g[3] = Real(0);
  }
}

// log sum_c exp(v_c) with a max shift, and the weights w_c = exp(v_c - ell).
template <typename Real, int NC>
__device__ __forceinline__ Real lse(const Real (&v)[NC], Real (&w)[NC]) {
  typedef Fn<Real> F;
  if constexpr (NC == 1) {
    w[0] = Real(1);
    return v[0];
  } else if constexpr (NC == 2) {
    Real dv = v[1] - v[0];
    Real e = F::ex2(-fabs(dv));
    Real s = Real(1) + e;
    const Real ls = F::lg2(s);  // s in [1, 2], or NaN from NaN inputs
    Real rs = F::rcp_lg(s, ls);
    Real wb = rs, ws = e * rs;
    w[0] = dv > Real(0) ? ws : wb;
    w[1] = dv > Real(0) ? wb : ws;
    return fmax(v[0], v[1]) + ls;
  } else {
    Real m = v[0];
#pragma unroll
    for (int c = 1; c < NC; ++c) m = fmax(m, v[c]);
    Real s = Real(0);
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      w[c] = F::ex2(v[c] - m);
      s += w[c];
    }
    Real rs = F::rcp(s);
#pragma unroll
    for (int c = 0; c < NC; ++c) w[c] *= rs;
    return m + F::lg2(s);
  }
}

// What component c contributes to its accumulator: w_c, or P_c/P when its
// coefficient is exactly 0 (vnc = delta_nc_c + sum of the component's u).
template <typename Real>
__device__ __forceinline__ Real comp_weight(int zero_mask, int c, Real vnc, Real ell, Real wc) {
  // CUDA's accurate exp2: this weight is not bounded by 1, so the
  // approximation's relative error would not stay small in absolute terms
  if ((zero_mask >> c) & 1) return Fn<Real>::ex2_exact(vnc - ell);
  return wc;
}

// Per-event constants copied from shared memory into registers.
template <typename Real, int NL>
struct EvalConsts {
  Real pc[NL][RF_PC];
  Real delta[NL];
  Real delta_nc[NL];
  int zero_mask;
  const RfExact* full;  // FP64 constants (FP32 evaluation, a zero coefficient)
  __device__ __forceinline__ void load(const RfConsts<Real>& K, const RfExact* X = nullptr) {
    full = X;
#pragma unroll
    for (int k = 0; k < NL; ++k)
#pragma unroll
      for (int j = 0; j < RF_PC; ++j) pc[k][j] = K.pc[k][j];
#pragma unroll
    for (int c = 0; c < NL; ++c) {
      delta[c] = K.delta[c];
      delta_nc[c] = K.delta_nc[c];
    }
    zero_mask = K.zero_mask;
  }
};

// --------------------------------------------------------------- reduction
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum N per-thread values over the block in a fixed order; result in
// out[0..N) (shared), valid after the trailing barrier.  red: [32*N] shared.
template <int N>
__device__ inline void block_sum(const double (&val)[N], double* red,
                                 double* out) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int i = 0; i < N; ++i) {
    double v = warp_sum(val[i]);
    if (lane == 0) red[wid * N + i] = v;
  }
  __syncthreads();
  if (threadIdx.x < N) {
    double s = 0.0;
    for (int w = 0; w < nw; ++w) s += red[w * N + threadIdx.x];
    out[threadIdx.x] = s;
  }
  __syncthreads();
}

// Double-single (FP32 pair) addition: (h, l) += (h2, l2) with Knuth's TwoSum
// for the high parts; the pair carries about 48 significant bits.
__device__ __forceinline__ void ds_add(float& h, float& l, float h2, float l2) {
  const float s = h + h2;
  const float v = s - h;
  float e = (h - (s - v)) + (h2 - v);
  e += l + l2;
  h = s + e;
  l = e - (h - s);
}

// Block sum of N per-thread FP32 pairs (h_i + l_i) in a fixed order, entirely
// in FP32 pair arithmetic (the FP64 pipe of this GPU is narrow: one warp
// instruction per ~64 cycles per sub-partition); the block totals stay FP32
// pairs, out[i] (shared).  Accumulators not in MASK give 0.  red: [32*N]
// float2 shared; valid after the trailing barrier.
template <int N, unsigned long long MASK>
__device__ inline void block_sum_ds2(const float (&hs)[N], const float (&ls)[N], float2* red,
                                     float2* out) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int i = 0; i < N; ++i) {
    if (!((MASK >> i) & 1ull)) continue;
    float h = hs[i], l = ls[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float h2 = __shfl_xor_sync(0xffffffffu, h, o);
      const float l2 = __shfl_xor_sync(0xffffffffu, l, o);
      ds_add(h, l, h2, l2);
    }
    if (lane == 0) red[wid * N + i] = make_float2(h, l);
  }
  __syncthreads();
  if (threadIdx.x < N) {
    float h = 0.f, l = 0.f;
    if ((MASK >> threadIdx.x) & 1ull)
      for (int w = 0; w < nw; ++w) ds_add(h, l, red[w * N + threadIdx.x].x, red[w * N + threadIdx.x].y);
    out[threadIdx.x] = make_float2(h, l);
  }
  __syncthreads();
}

// FP64 block sum of the accumulators in MASK (the others give 0), in a
// fixed order: a shuffle tree per warp, then warp totals in warp order.
// red: [32*N] shared; result in out[0..N) (shared), valid after the trailing
// barrier.
template <int N, unsigned long long MASK>
__device__ inline void block_sum_m(const double (&val)[N], double* red, double* out) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int i = 0; i < N; ++i) {
    if (!((MASK >> i) & 1ull)) continue;
    const double v = warp_sum(val[i]);
    if (lane == 0) red[wid * N + i] = v;
  }
  __syncthreads();
  if (threadIdx.x < N) {
    double s = 0.0;
    if ((MASK >> threadIdx.x) & 1ull)
      for (int w = 0; w < nw; ++w) s += red[w * N + threadIdx.x];
    out[threadIdx.x] = s;
  }
  __syncthreads();
}

// One level of the grid's FP64 tree: rows [r0, r1) of
// partials[row * RF_NACC_MAX + i] summed for the accumulators i in MASK, in a
// fixed order (warp w takes rows r0 + w, r0 + w + warps, ... with lane i on
// accumulator i; the warps' sums are then added in warp order).  One warp
// instruction covers every accumulator, so a level of up to ~40 rows costs
// a few FP64 instructions per warp.  red: [32*N] shared; result in out[0..N)
// (shared), valid after the trailing barrier.
template <int N, unsigned long long MASK>
__device__ inline void rows_tree(const double* partials, int64_t r0, int64_t r1, double* red,
                                 double* out) {
  static_assert(N <= 32, "one lane per accumulator");
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
  if (lane < N) {
    double s = 0.0;
    if ((MASK >> lane) & 1ull)
      for (int64_t r = r0 + wid; r < r1; r += nw) s += __ldcg(partials + r * RF_NACC_MAX + lane);
    red[wid * N + lane] = s;
  }
  __syncthreads();
  if (threadIdx.x < N) {
    double s = 0.0;
    for (int w = 0; w < nw; ++w) s += red[w * N + threadIdx.x];
    out[threadIdx.x] = s;
  }
  __syncthreads();
}

// Sum rows [r0, r1) of partials[row * RF_NACC_MAX + i] for i < N, in a fixed
// order for a given block size; result in out[0..N) (shared).
template <int N>
__device__ inline void rows_sum(const double* partials, int64_t r0, int64_t r1,
                                double* red, double* out) {
  double v[N];
#pragma unroll
  for (int i = 0; i < N; ++i) v[i] = 0.0;
  double cmp[N];
#pragma unroll
  for (int i = 0; i < N; ++i) cmp[i] = 0.0;
  for (int64_t r = r0 + threadIdx.x; r < r1; r += blockDim.x) {
#pragma unroll
    for (int i = 0; i < N; ++i) {  // Neumaier
      double x = __ldcg(partials + r * RF_NACC_MAX + i);
      double t = v[i] + x;
      cmp[i] += (fabs(v[i]) >= fabs(x)) ? (v[i] - t) + x : (x - t) + v[i];
      v[i] = t;
    }
  }
#pragma unroll
  for (int i = 0; i < N; ++i) v[i] += cmp[i];
  block_sum<N>(v, red, out);
}

// ---------------------------------------------------------------- epilogue
// T: FP64 totals of the accumulators, n: events.  Writes NLL and gradient.
// The gradient is summed in a thread-local array and stored once per
// component: updating it in place in global memory would put a round trip to
// L2 behind every term.
template <typename Real, int NL>
__device__ __noinline__ void epilogue(const RfProgram& P, const RfConsts<Real>& K,
                                const double* T, int64_t n, double* nll,
                                double* grad_out, unsigned int* status) {
  double g_local[RF_MAXPAR];
  double* grad = grad_out ? g_local : nullptr;
  const int C = P.n_comp;
  double L = kLn2 * T[0];  // the per-event sums are in base-2 units
  for (int c = 0; c < C; ++c)
    if (!((K.zero_mask >> c) & 1)) L += T[1 + c] * K.delta_lo[c];
  for (int k = 0; k < P.n_leaves; ++k)
    for (int j = 0; j < RF_LEAF_MAXP; ++j)
      if ((P.leaf[k].gmask >> j) & 1)
        L -= T[1 + NL + k * RF_LEAF_MAXP + j] * K.gmul[k][j] * K.dtheta[k][j];
  double v = -((double)n * K.beta_ref + L) + K.ext_sum;
  bool bad = K.bad || !isfinite(v);
  if (grad) {
    for (int p = 0; p < P.n_par; ++p) grad[p] = 0.0;
    for (int k = 0; k < P.n_leaves; ++k) {
      const RfLeafProg& lf = P.leaf[k];
      double S = ((K.zero_mask >> lf.comp) & 1) ? 0.0 : T[1 + lf.comp];
      for (int j = 0; j < RF_LEAF_MAXP; ++j)
        if ((lf.gmask >> j) & 1)
          grad[lf.par[j]] -= T[1 + NL + k * RF_LEAF_MAXP + j] * K.gmul[k][j] - S * K.dlogI[k][j];
    }
    double R[RF_MAXC];
    for (int c = 0; c < C; ++c)
      R[c] = ((K.zero_mask >> c) & 1) ? T[1 + c] : T[1 + c] / K.coef[c];
    if (P.kind == RF_KIND_FRAC) {
      for (int c = 0; c < C - 1; ++c)
        if ((P.coef_free >> c) & 1) grad[P.coef_par[c]] -= R[c] - R[C - 1];
    } else if (P.kind == RF_KIND_EXT) {
      for (int c = 0; c < C; ++c)
        if ((P.coef_free >> c) & 1) grad[P.coef_par[c]] += P.ext_weight - R[c];
    }
    for (int p = 0; p < P.n_par; ++p) {
      bool fx = p < 64 ? ((P.fixed_lo >> p) & 1) : ((P.fixed_hi >> (p - 64)) & 1);
      if (fx) grad[p] = 0.0;
      if (bad) grad[p] = kNaN();
      grad_out[p] = grad[p];
    }
  }
  if (bad) {
    v = kInf();
    if (status)
      atomicOr(status, K.bad ? (unsigned)RF_STATUS_PARAM_DOMAIN_BIT
                             : (unsigned)RF_STATUS_NONFINITE_BIT);
  }
  *nll = v;
}

// The epilogue on one warp (all 32 lanes): the NLL's terms on separate lanes
// summed by a shuffle tree, and gradient component p on lane p (the FP64 unit
// takes one warp instruction at a time however many lanes are active, so the
// parallel form is as cheap per instruction as the serial one and its chains
// are short).  Same formulas as epilogue().
template <typename Real, int NL>
__device__ __forceinline__ void epilogue_warp(const RfProgram& P, const RfConsts<Real>& K,
                                     const double* T, int64_t n, double* nll, double* grad,
                                     unsigned int* status) {
  const int lane = threadIdx.x & 31;
  const int C = P.n_comp;
  double term = 0.0;
  if (lane == 0) {
    term = kLn2 * T[0];  // the per-event sums are in base-2 units
  } else if (lane <= C) {
    const int c = lane - 1;
    if (!((K.zero_mask >> c) & 1)) term = T[1 + c] * K.delta_lo[c];
  } else {
    const int idx = lane - 1 - C, k = idx >> 2, j = idx & 3;
    if (k < P.n_leaves && ((P.leaf[k].gmask >> j) & 1))
      term = -(T[1 + NL + k * RF_LEAF_MAXP + j] * K.gmul[k][j] * K.dtheta[k][j]);
  }
  const double L = warp_sum(term);
  double v = -((double)n * K.beta_ref + L) + K.ext_sum;
  const bool bad = K.bad || !isfinite(v);
  if (grad) {
    for (int p = lane; p < P.n_par; p += 32) {
      double g = 0.0;
      for (int k = 0; k < P.n_leaves; ++k) {
        const RfLeafProg& lf = P.leaf[k];
        for (int j = 0; j < RF_LEAF_MAXP; ++j)
          if (((lf.gmask >> j) & 1) && lf.par[j] == p) {
            const double S = ((K.zero_mask >> lf.comp) & 1) ? 0.0 : T[1 + lf.comp];
            g -= T[1 + NL + k * RF_LEAF_MAXP + j] * K.gmul[k][j] - S * K.dlogI[k][j];
          }
      }
      for (int c = 0; c < C; ++c) {
        if (!((P.coef_free >> c) & 1)) continue;
        if (P.kind == RF_KIND_FRAC && c < C - 1 && P.coef_par[c] == p) {
          const double Rc = ((K.zero_mask >> c) & 1) ? T[1 + c] : T[1 + c] / K.coef[c];
          const int l = C - 1;
          const double Rl = ((K.zero_mask >> l) & 1) ? T[1 + l] : T[1 + l] / K.coef[l];
          g -= Rc - Rl;
        } else if (P.kind == RF_KIND_EXT && P.coef_par[c] == p) {
          const double Rc = ((K.zero_mask >> c) & 1) ? T[1 + c] : T[1 + c] / K.coef[c];
          g += P.ext_weight - Rc;
        }
      }
      const bool fx = p < 64 ? ((P.fixed_lo >> p) & 1) : ((P.fixed_hi >> (p - 64)) & 1);
      if (fx) g = 0.0;
      if (bad) g = kNaN();
      grad[p] = g;
    }
  }
  if (lane == 0) {
    if (bad) {
      v = kInf();
      if (status)
        atomicOr(status, K.bad ? (unsigned)RF_STATUS_PARAM_DOMAIN_BIT
                               : (unsigned)RF_STATUS_NONFINITE_BIT);
    }
    *nll = v;
  }
}

// The epilogue on an aligned group of G lanes (G divides 32; all 32 lanes of
// the warp call it, each group for its own totals T and constants K): the
// NLL's terms split over the group's lanes and summed by a shuffle tree,
// gradient component p on group lane p mod G.  Same formulas as epilogue();
// the group's chains are about G times shorter (the FP64 unit takes one warp
// instruction at a time however many lanes are active).  valid: the group
// has a dataset (false: it only takes part in the shuffles, writes nothing).
// Returns the NLL (+inf when bad) on every lane of the group.
template <typename Real, int NL, int G>
__device__ __forceinline__ double epilogue_group(const RfProgram& P, const RfConsts<Real>& K,
                                                 const double* T, int64_t n, double* nll,
                                                 double* grad, unsigned int* status, bool valid) {
  const int q = threadIdx.x & (G - 1);
  const int C = P.n_comp;
  const int nterm = 1 + C + RF_LEAF_MAXP * P.n_leaves;
  double L = 0.0;
  for (int tau = q; tau < nterm; tau += G) {
    double term = 0.0;
    if (tau == 0) {
      term = kLn2 * T[0];  // the per-event sums are in base-2 units
    } else if (tau <= C) {
      const int c = tau - 1;
      if (!((K.zero_mask >> c) & 1)) term = T[1 + c] * K.delta_lo[c];
    } else {
      const int idx = tau - 1 - C, k = idx >> 2, j = idx & 3;
      if ((P.leaf[k].gmask >> j) & 1)
        term = -(T[1 + NL + k * RF_LEAF_MAXP + j] * K.gmul[k][j] * K.dtheta[k][j]);
    }
    L += term;
  }
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) L += __shfl_xor_sync(0xffffffffu, L, o);
  double v = -((double)n * K.beta_ref + L) + K.ext_sum;
  const bool bad = K.bad || !isfinite(v);
  if (grad && valid) {
    for (int p = q; p < P.n_par; p += G) {
      double g = 0.0;
      for (int k = 0; k < P.n_leaves; ++k) {
        const RfLeafProg& lf = P.leaf[k];
        for (int j = 0; j < RF_LEAF_MAXP; ++j)
          if (((lf.gmask >> j) & 1) && lf.par[j] == p) {
            const double S = ((K.zero_mask >> lf.comp) & 1) ? 0.0 : T[1 + lf.comp];
            g -= T[1 + NL + k * RF_LEAF_MAXP + j] * K.gmul[k][j] - S * K.dlogI[k][j];
          }
      }
      for (int c = 0; c < C; ++c) {
        if (!((P.coef_free >> c) & 1)) continue;
        if (P.kind == RF_KIND_FRAC && c < C - 1 && P.coef_par[c] == p) {
          const double Rc = ((K.zero_mask >> c) & 1) ? T[1 + c] : T[1 + c] / K.coef[c];
          const int l = C - 1;
          const double Rl = ((K.zero_mask >> l) & 1) ? T[1 + l] : T[1 + l] / K.coef[l];
          g -= Rc - Rl;
        } else if (P.kind == RF_KIND_EXT && P.coef_par[c] == p) {
          const double Rc = ((K.zero_mask >> c) & 1) ? T[1 + c] : T[1 + c] / K.coef[c];
          g += P.ext_weight - Rc;
        }
      }
      const bool fx = p < 64 ? ((P.fixed_lo >> p) & 1) : ((P.fixed_hi >> (p - 64)) & 1);
      if (fx) g = 0.0;
      if (bad) g = kNaN();
      grad[p] = g;
    }
  }
  if (bad) v = kInf();
  if (valid && q == 0) {
    if (bad && status)
      atomicOr(status, K.bad ? (unsigned)RF_STATUS_PARAM_DOMAIN_BIT
                             : (unsigned)RF_STATUS_NONFINITE_BIT);
    *nll = v;
  }
  return v;
}

}  // namespace rf
