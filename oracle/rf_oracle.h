/*
 * rf_oracle.h -- the FP64 CPU oracle for the unbinned negative log-likelihood
 * of a PDF computation graph (Hageboeck, "A Faster, More Intuitive RooFit",
 * Sec. 5.1: per-entry probability of the top node of a graph of observables,
 * parameters and PDFs; normalisation by analytic integrals, Sec. 3).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * bench's CPU-baseline / reference arm may load this library.  It shares no
 * code, header, table or constant with the CUDA library and includes nothing
 * from it.
 *
 * The oracle is deliberately plain: every event walks the graph node by node
 * (the classic evaluation the paper describes in Sec. 5.1), every PDF and every
 * integral is written out from its textbook definition in FP64, the gradient
 * is forward-mode (each node returns its value and its derivative vector with
 * respect to all parameters), and sums are Neumaier-compensated in event order.
 * Parameter-only quantities (the normalisation integrals) are computed once per
 * call, as the paper's constant branches are (Sec. 5.1).
 *
 * Functions whose values have no independent pin are listed as "parity
 * unpinned" in the header comment of rf_oracle.c.
 */
#ifndef RF_ORACLE_H
#define RF_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* node types (the oracle's own numbering) */
enum {
  ORC_GAUSS = 1,    /* params (mu, sigma)                      */
  ORC_EXP = 2,      /* params (lambda)                         */
  ORC_CHEB = 3,     /* params (c_1 .. c_m), m <= ORC_MAXNP     */
  ORC_CB = 4,       /* params (m0, sigma, alpha, n)            */
  ORC_ARGUS = 5,    /* params (m0, c, p), p > 0                */
  ORC_ADD_FRAC = 6, /* K children, K-1 fraction params         */
  ORC_ADD_EXT = 7,  /* K children, K yield params; root only   */
  ORC_PROD = 8,     /* K children on disjoint observables      */
  ORC_JOHNSON = 9,  /* params (mu, lambda, gamma, delta): Johnson's SU */
  ORC_EXPR = 10,    /* params p0 .. p(m-1) of a formula f(x; p) given as text */
  ORC_HYPATIA2 = 11 /* params (lambda, zeta, beta, sigma, mu, a, n, a2, n2):
                       a generalised hyperbolic core with power-law tails */
};

#define ORC_MAXCH 8   /* children per node   */
#define ORC_MAXNP 12  /* params per node     */
#define ORC_MAXPAR 64 /* params per model    */
#define ORC_MAXNODE 32

/* return codes */
enum { ORC_OK = 0, ORC_EINVAL = 1, ORC_EUNSUPPORTED = 2, ORC_EDOMAIN = 3 };

/* A model is given as flat arrays, one entry per node:
 *   type[i], obs[i] (leaves), nchild[i], child[i*ORC_MAXCH + k],
 *   npar[i], par[i*ORC_MAXNP + j] (indices into the parameter vector).
 * obs_lo/obs_hi give each observable's range [lo, hi]. */
typedef struct {
  int32_t n_nodes;
  int32_t root;
  int32_t n_obs;
  int32_t n_par;
  const int32_t* type;
  const int32_t* obs;
  const int32_t* nchild;
  const int32_t* child;
  const int32_t* npar;
  const int32_t* par;
  const double* obs_lo;
  const double* obs_hi;
  const char* const* expr; /* [n_nodes]: formula of each ORC_EXPR node (others
                              ignored); may be NULL without ORC_EXPR nodes */
} orc_model;

/* Unnormalised log-density of one leaf and its derivatives with respect to the
 * leaf's own parameters (dlogf[j] for theta[j]).  For a point outside the
 * support (ARGUS m >= m0) *logf = -inf and dlogf = 0. */
int orc_leaf_logf(int type, const double* theta, int ntheta, double lo,
                  double hi, double x, double* logf, double* dlogf);

/* Normalisation integral I = int_lo^hi f(x) dx of one leaf and dI/dtheta_j. */
int orc_leaf_norm(int type, const double* theta, int ntheta, double lo,
                  double hi, double* I, double* dI);

/* Formula leaves (ORC_EXPR).  Grammar: sums, products, quotients, unary
 * minus, '^' (right-associative), numbers, the observable x, parameters
 * p0 .. p(ntheta-1), and exp log sqrt sin cos tanh sinh cosh asinh atan erf
 * erfc abs pow(a, b).  An integer literal exponent is a repeated product; any
 * other a^b is exp(b log a).  check: ORC_OK or ORC_EINVAL.  logf: log f(x) and
 * d log f/dp_j.  norm: I = int_lo^hi f and dI/dp_j by adaptive Gauss-Legendre
 * quadrature (20 points, bisection until both halves reproduce their parent to
 * 1e-14 of the integral of |.|); ORC_EDOMAIN when f is not finite or I <= 0. */
int orc_expr_check(const char* text, int npar);
int orc_expr_logf(const char* text, const double* theta, int ntheta, double x,
                  double* logf, double* dlogf);
int orc_expr_norm(const char* text, const double* theta, int ntheta, double lo,
                  double hi, double* I, double* dI);

/* Modified Bessel function of the second kind of real order nu, z > 0, from
 * its integral representation K_nu(z) = int_0^inf e^{-z cosh t} cosh(nu t) dt
 * (adaptive Gauss-Legendre quadrature): out[0] = K_nu(z), out[1] = dK/dz,
 * out[2] = dK/dnu. */
int orc_besselk(double nu, double z, double* out);

/* NLL = -sum_i log P(x_i)  (+ sum_k nu_k for an extended root) and, if grad is
 * not NULL, dNLL/dtheta for every parameter.  cols: observable j of event i at
 * cols[j*col_stride + i].  nthreads <= 0: all available cores.  The result does
 * not depend on nthreads (fixed chunks merged in chunk order).  A non-positive
 * or non-finite P_i gives *nll = +inf and returns ORC_EDOMAIN. */
int orc_nll(const orc_model* m, const double* params, const double* cols,
            int64_t col_stride, int64_t n, int nthreads, double* nll,
            double* grad);

/* As orc_nll, and gscale[k] = sum_i |d(-log P_i)/dtheta_k| (+1 for a yield's
 * extended term): the L1 scale that gradient errors are measured against,
 * because the gradient itself vanishes at the minimum. */
int orc_nll_scaled(const orc_model* m, const double* params, const double* cols,
                   int64_t col_stride, int64_t n, int nthreads, double* nll,
                   double* grad, double* gscale);

/* Per-event log P(x_i) (extended root: log of sum_k nu_k f_k/I_k). */
int orc_logp(const orc_model* m, const double* params, const double* cols,
             int64_t col_stride, int64_t n, double* logp);

/* Toys: toy t owns events [offsets[t], offsets[t+1]) and parameter row
 * params_matrix[t*n_par ..].  out[t*(1+n_par)] = NLL, then the gradient. */
int orc_nll_batched(const orc_model* m, const double* cols, int64_t col_stride,
                    const int64_t* offsets, int32_t toys,
                    const double* params_matrix, int nthreads, double* out);

/* One Adam step (Kingma & Ba 2015, Algorithm 1) on parameters expressed in
 * units of scale[j]: u = theta/scale, g_u = grad*scale.  Only entries with
 * free[j] != 0 move.  t is the 1-based step number. */
void orc_adam_step(int n_par, double* theta, const double* grad,
                   const double* scale, const uint8_t* free_mask, double* m1,
                   double* m2, int t, double lr, double beta1, double beta2,
                   double eps);

/* Toy generation.
 * Philox4x64-10 block for counter ctr and key (Salmon et al., SC'11). */
void orc_philox4x64(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4]);
/* inverse complementary error function on (0, 2) */
double orc_erfcinv(double q);
/* Events of `toys` datasets: toy t's events [offsets[t], ...) are, in order,
 * comp_counts[t*K + c] events of component c (K = root's children for an Add,
 * else 1), each observable drawn from the component's leaf on it with the
 * toy's parameter row: inverse CDF (Gaussian, Exponential, Crystal Ball) or
 * accept-reject (Chebychev, ARGUS), uniforms ((w >> 11) + 0.5) 2^-53 from the
 * 64-bit words w of Philox4x64-10 with key {seed, 0x52462D544F595321} and
 * counter {event, observable, attempt, 0}; a value is stored rounded to the
 * column type (col_f32) and accepted only inside the observable's range
 * (ARGUS: below m0).  *exhausted counts values that took 4096 attempts. */
int orc_generate(const orc_model* m, const double* params_matrix, int32_t toys,
                 const int64_t* comp_counts, const int64_t* offsets, uint64_t seed,
                 int col_f32, double* cols, int64_t col_stride, int64_t* exhausted);

#ifdef __cplusplus
}
#endif
#endif
