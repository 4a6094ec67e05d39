// k_generate.cu -- toy generation on the device: the events of many datasets
// drawn from the graph at per-toy parameters (RooStats-style toy studies,
// Sec. 1), written straight into the columns the toy kernels read.
//
// Event i of toy t belongs to component c by its position in the toy (the
// toy's events are its components' counts in order); each observable is
// drawn from the component's leaf on it, in FP64: inverse CDF for the
// Gaussian, the Exponential and the Crystal Ball, accept-reject for the
// Chebychev polynomial and ARGUS.  Uniforms come from Philox4x64-10 (Salmon,
// Moraes, Dror, Shaw, SC'11) with key {seed, kToyKey} and counter {event,
// observable, attempt, 0}: an event's values do not depend on the launch
// shape.  A value is rounded to the column type and accepted only inside the
// observable's range (ARGUS: below m0).
#include <cuda_runtime.h>

#include "rf_internal.h"

namespace {

constexpr unsigned long long kToyKey = 0x52462D544F595321ull;
constexpr int kMaxAttempts = 4096;

struct U4 {
  double u[4];
};

// Philox4x64-10 block: ten rounds of two 64 x 64 -> 128-bit products, the
// key bumped by the Weyl constants between rounds.
__device__ __forceinline__ U4 philox_uniforms(unsigned long long c0, unsigned long long c1,
                                              unsigned long long c2, unsigned long long seed) {
  const unsigned long long M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
  const unsigned long long W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
  unsigned long long c3 = 0ull, k0 = seed, k1 = kToyKey;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const unsigned long long hi0 = __umul64hi(M0, c0), lo0 = M0 * c0;
    const unsigned long long hi1 = __umul64hi(M1, c2), lo1 = M1 * c2;
    const unsigned long long n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
    if (r < 9) {
      k0 += W0;
      k1 += W1;
    }
  }
  // ((w >> 11) + 1/2) 2^-53: uniform on (0, 1), never 0 or 1
  U4 o;
  o.u[0] = ((double)(c0 >> 11) + 0.5) * 0x1p-53;
  o.u[1] = ((double)(c1 >> 11) + 0.5) * 0x1p-53;
  o.u[2] = ((double)(c2 >> 11) + 0.5) * 0x1p-53;
  o.u[3] = ((double)(c3 >> 11) + 0.5) * 0x1p-53;
  return o;
}

// z with Phi(z) = Phi(za) + u (Phi(zb) - Phi(za)) (standard normal CDF),
// through the lower- or the upper-tail probability, whichever is small.
__device__ double tn_inv(double u, double za, double zb) {
  const double r2 = 1.4142135623730951;
  const double Pa = 0.5 * erfc(-za / r2), Pb = 0.5 * erfc(-zb / r2);
  const double P = Pa + u * (Pb - Pa);
  if (P <= 0.5) return -r2 * erfcinv(2.0 * P);
  const double Qa = 0.5 * erfc(za / r2), Qb = 0.5 * erfc(zb / r2);
  const double Q = Qb + (1.0 - u) * (Qa - Qb);
  return r2 * erfcinv(2.0 * Q);
}

__device__ double erf_diff(double z1, double z2) {  // erf(z2) - erf(z1)
  if (z1 >= 0.0) return erfc(z1) - erfc(z2);
  if (z2 <= 0.0) return erfc(-z2) - erfc(-z1);
  return erf(z2) - erf(z1);
}

// One candidate value of leaf `type` (parameters th) on [a, b] from one
// attempt's four uniforms; *accept = false asks for another attempt.
__device__ double sample_leaf(int type, const double* th, int npar, double a, double b,
                              const U4& U, bool* accept) {
  const double* u = U.u;
  *accept = true;
  switch (type) {
    case RFL_GAUSS: {
      const double mu = th[0], sg = th[1];
      return mu + sg * tn_inv(u[0], (a - mu) / sg, (b - mu) / sg);
    }
    case RFL_EXP: {
      // CDF expm1(lam (x - a)) / expm1(lam L), inverted from the end whose
      // exponential cannot overflow
      const double lam = th[0], L = b - a;
      if (lam == 0.0) return a + u[0] * L;
      if (lam < 0.0) return a + log1p(u[0] * expm1(lam * L)) / lam;
      return b + log1p((1.0 - u[0]) * expm1(-lam * L)) / lam;
    }
    case RFL_CHEB: {
      // uniform proposal on [-1, 1], accepted under f = 1 + sum c_j T_j,
      // bounded by 1 + sum |c_j|
      const double xp = -1.0 + 2.0 * u[0];
      double fmax = 1.0, f = 1.0, tm = 1.0, t = xp;
      for (int j = 0; j < npar; ++j) {
        fmax += fabs(th[j]);
        f += th[j] * t;
        const double tn = 2.0 * xp * t - tm;
        tm = t;
        t = tn;
      }
      *accept = u[1] * fmax <= f;
      return a + 0.5 * (xp + 1.0) * (b - a);
    }
    case RFL_CB: {
      // t = s (x - m0)/sigma; core e^{-t^2/2} for t > -A, tail e^{-A^2/2}
      // D^-n with D = 1 - (A/n)(A + t); tail mass from tlo to t is
      // pre (G(D(tlo)) - G(D(t))), G(D) = D^(1-n)/(1-n) (log D at n = 1)
      const double m0 = th[0], sg = th[1], al = th[2], n = th[3];
      const double s = al > 0.0 ? 1.0 : -1.0, A = fabs(al);
      const double tlo = s > 0.0 ? (a - m0) / sg : (m0 - b) / sg;
      const double thi = s > 0.0 ? (b - m0) / sg : (m0 - a) / sg;
      const double tc = tlo > -A ? tlo : -A;
      const double r2 = 1.4142135623730951;
      const double core = thi > -A ? 1.2533141373155003 * erf_diff(tc / r2, thi / r2) : 0.0;
      const double pre = (n / A) * exp(-0.5 * A * A);
      double tail = 0.0, G1 = 0.0;
      if (tlo < -A) {
        const double t2 = thi < -A ? thi : -A;
        const double D1 = 1.0 - (A / n) * (A + tlo), D2 = 1.0 - (A / n) * (A + t2);
        G1 = n == 1.0 ? log(D1) : pow(D1, 1.0 - n) / (1.0 - n);
        const double G2 = n == 1.0 ? log(D2) : pow(D2, 1.0 - n) / (1.0 - n);
        tail = pre * (G1 - G2);
      }
      const double T = u[0] * (core + tail);
      double t;
      if (T < tail) {
        const double G = G1 - T / pre;
        const double Dt = n == 1.0 ? exp(G) : pow((1.0 - n) * G, 1.0 / (1.0 - n));
        t = (n / A) * (1.0 - Dt) - A;
      } else {
        t = tn_inv(core > 0.0 ? (T - tail) / core : 0.0, tc, thi);
      }
      return s > 0.0 ? m0 + sg * t : m0 - sg * t;
    }
    case RFL_JOHNSON: {
      // w = gamma + delta asinh z is standard normal on [w(a), w(b)]
      const double mu = th[0], lam = th[1], gam = th[2], del = th[3];
      const double wa = gam + del * asinh((a - mu) / lam), wb = gam + del * asinh((b - mu) / lam);
      const double w = tn_inv(u[0], wa, wb);
      return mu + lam * sinh((w - gam) / del);
    }
    case RFL_ARGUS: {
      // m dm ~ sqrt(tau) e^{c tau} d tau, tau = 1 - (m/m0)^2: for c < 0 a
      // Gamma(3/2, rate -c) variate (E + Z^2/2)/(-c), E exponential and Z
      // normal (Box-Muller), kept inside [tau(b), tau(a)]; for c >= 0 a uniform
      // tau accepted under the increasing bound sqrt(tau_a) e^{c tau_a}
      const double m0 = th[0], c = th[1];
      const double bb = b < m0 ? b : m0;
      const double ta = 1.0 - (a / m0) * (a / m0), tb = 1.0 - (bb / m0) * (bb / m0);
      double tau;
      if (c < 0.0) {
        const double E = -log(u[0]);
        const double Z = sqrt(-2.0 * log(u[1])) * cos(6.283185307179586 * u[2]);
        tau = (E + 0.5 * Z * Z) / (-c);
        *accept = tau >= tb && tau <= ta;
      } else {
        tau = tb + u[0] * (ta - tb);
        const double gmax = sqrt(ta) * exp(c * ta);
        *accept = u[1] * gmax <= sqrt(tau) * exp(c * tau);
      }
      return m0 * sqrt(1.0 - tau);
    }
  }
  *accept = true;
  return nan("");
}

template <typename Col>
__global__ void __launch_bounds__(256)
    generate_kernel(const RfProgram P, const double* __restrict__ pm,
                    const int64_t* __restrict__ counts, const int64_t* __restrict__ offsets,
                    int32_t toys, unsigned long long seed, Col* __restrict__ ev, int64_t n_events,
                    unsigned int* status) {
  int64_t E = offsets[toys];
  E = E < 0 ? 0 : (E > n_events ? n_events : E);
  const int K = P.n_comp;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < E;
       i += (int64_t)gridDim.x * blockDim.x) {
    // the toy holding event i: the last t with offsets[t] <= i
    int32_t lo = 0, hi = toys;  // offsets[lo] <= i < offsets[hi] for monotone offsets
    while (hi - lo > 1) {
      const int32_t mid = (lo + hi) >> 1;
      if (offsets[mid] <= i) lo = mid;
      else hi = mid;
    }
    const int32_t t = lo;
    // its component: the counts of the toy's components, in order
    int64_t pos = i - offsets[t];
    int c = -1;
    for (int k = 0; k < K; ++k) {
      const int64_t nk = counts[(int64_t)t * K + k];
      if (pos < nk) {
        c = k;
        break;
      }
      pos -= nk;
    }
    if (c < 0) {  // the toy's counts do not fill its event range
      atomicOr(status, RF_STATUS_NONFINITE_BIT);
      for (int col = 0; col < P.n_cols; ++col) ev[(int64_t)P.col_obs[col] * n_events + i] = Col(nan(""));
      continue;
    }
    const double* row = pm + (int64_t)t * P.n_par;
    for (int k = 0; k < P.n_leaves; ++k) {
      const RfLeafProg& L = P.leaf[k];
      if (L.comp != c) continue;
      const int obs = P.col_obs[L.col];
      double th[RF_LEAF_MAXP];
      for (int j = 0; j < L.npar; ++j) th[j] = row[L.par[j]];
      if (L.type == RFL_ARGUS && th[2] != 0.5) {  // the sampler draws p = 1/2 only
        atomicOr(status, RF_STATUS_PARAM_DOMAIN_BIT);
        ev[(int64_t)obs * n_events + i] = Col(nan(""));
        continue;
      }
      double x = nan("");
      bool ok = false;
      Col v = Col(0);
      for (int r = 0; r < kMaxAttempts && !ok; ++r) {
        const U4 U = philox_uniforms((unsigned long long)i, (unsigned long long)obs,
                                     (unsigned long long)r, seed);
        x = sample_leaf(L.type, th, L.npar, L.lo, L.hi, U, &ok);
        v = (Col)x;  // round to the column type
        const double xs = (double)v;
        if (ok && !(xs >= L.lo && xs <= L.hi)) ok = false;
        if (ok && L.type == RFL_ARGUS && !(xs < th[0])) ok = false;
      }
      if (!ok) atomicOr(status, RF_STATUS_GEN_EXHAUSTED_BIT);
      ev[(int64_t)obs * n_events + i] = v;
    }
  }
}

}  // namespace

int rf_launch_generate(const RfProgram& P, int coldt, const double* params_matrix,
                       const int64_t* comp_counts, const int64_t* offsets, int32_t toys,
                       unsigned long long seed, void* events, int64_t n_events,
                       unsigned int* status, int num_sms, cudaStream_t st) {
  const int block = 256, grid = num_sms * 8;
  if (coldt)
    generate_kernel<double><<<grid, block, 0, st>>>(P, params_matrix, comp_counts, offsets, toys,
                                                    seed, static_cast<double*>(events), n_events,
                                                    status);
  else
    generate_kernel<float><<<grid, block, 0, st>>>(P, params_matrix, comp_counts, offsets, toys,
                                                   seed, static_cast<float*>(events), n_events,
                                                   status);
  return (int)cudaGetLastError();
}
