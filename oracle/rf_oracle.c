/*
 * rf_oracle.c -- FP64 CPU oracle for the unbinned NLL of a PDF graph.
 *
 * TEST INFRASTRUCTURE ONLY: loaded by tests/, __graft_entry__.smoke() and the
 * bench's CPU-baseline leg, never by the product path.  Shares no code with the
 * CUDA library.
 *
 * What it computes (Hageboeck, "A Faster, More Intuitive RooFit"):
 *  - Sec. 5.1: the likelihood of each dataset entry is the probability of the
 *    top node of a computation graph whose leaves hold the entry's observables;
 *    the NLL is minus the sum of their logs.  The walk below evaluates every
 *    node for every entry, as the classic single-value evaluation does.
 *  - Sec. 5.1 (constant branches): parameter-only values -- here the leaf
 *    normalisation integrals and their derivatives -- are computed once.
 *  - Sec. 3 ("Analytic Integrals"): each PDF is divided by its integral over
 *    the observable range, taken analytically.
 *  - Sec. 3 ("Checking parameters"): parameters outside a PDF's definition
 *    range, or an entry with non-positive / non-finite probability, give
 *    NLL = +inf instead of a silent NaN.
 * The paper prints no PDF formula; the leaf definitions are the standard ones:
 *  Gaussian   f = exp(-(x-mu)^2 / (2 sigma^2))
 *  Exponential f = exp(lambda x)
 *  Chebychev  f = 1 + sum_{j>=1} c_j T_j(x'),  x' = (2x-lo-hi)/(hi-lo)
 *             (implicit T_0 coefficient 1; order = number of coefficients)
 *  CrystalBall t = s (x-m0)/sigma with s = sign(alpha), A = |alpha|:
 *             f = exp(-t^2/2) for t > -A, else
 *             f = exp(-A^2/2) * D^-n, D = 1 - (A/n)(A+t)   (== A'(B-t)^-n)
 *  ARGUS      f = x tau^p exp(c tau), tau = 1-(x/m0)^2 for x < m0, else 0
 *  Johnson SU f = delta/(lambda sqrt(2 pi (1+z^2))) exp(-(gamma+delta asinh z)^2/2)
 *  Formula    f = the node's text in x and p0..p(m-1) (Sec. 4, formula PDFs),
 *             normalised by adaptive Gauss-Legendre quadrature
 *  Add (fractions)  P = sum_{k<K-1} f_k P_k + (1 - sum f_k) P_{K-1}
 *  Add (extended)   P = sum_k nu_k P_k,  NLL += sum_k nu_k  (no log n! term)
 *  Prod             P = prod_k P_k   (children on disjoint observables)
 * Gradient: forward mode; each node returns P and dP/dtheta for all theta.
 * Sums: Neumaier compensated, in event order, per fixed chunk of events;
 * chunk results are merged in chunk order, so nthreads does not change them.
 *
 * Pins (tests/test_oracle_*.py): every normalised leaf integrates to one by
 * high-precision quadrature; normalisation derivatives against finite
 * differences of the quadrature-pinned integrals; the Gaussian NLL against its
 * closed form from sufficient statistics; ML mu and sigma against the sample
 * mean and 1/n standard deviation; Add/Prod against hand-expanded formulas;
 * Crystal Ball value and slope continuity at t=-A; the gradient against
 * Richardson-extrapolated central differences; the extended-ML invariant
 * sum nu = n; Adam against its published update written out by hand.
 * Formula leaves: texts that spell out a built-in leaf reproduce it (value,
 * derivatives, integral, whole-model NLL); values against Python's own
 * evaluation of the text; integrals against mpmath quadrature and a
 * Breit-Wigner's arctangent closed form.
 */
#include "rf_oracle.h"

#include <float.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define SQRT2 1.41421356237309504880
#define SQRT_PI_2 1.25331413731550025121 /* sqrt(pi/2) */
#define SQRT_PI 1.77245385090551602730
#define PI_VAL 3.14159265358979323846

/* ------------------------------------------------------------------ */
/* small helpers                                                       */
/* ------------------------------------------------------------------ */

/* erf(z2) - erf(z1) for z1 <= z2, taken from erfc when both arguments are on
 * the same side of zero so that tails do not cancel. */
static double erf_diff(double z1, double z2) {
  if (z1 >= 0.0) return erfc(z1) - erfc(z2);
  if (z2 <= 0.0) return erfc(-z2) - erfc(-z1);
  return erf(z2) - erf(z1);
}

/* E1(y) = (e^y - 1)/y, 1 at y = 0 */
static double e1(double y) { return y == 0.0 ? 1.0 : expm1(y) / y; }

/* dE1/dy = (e^y (y-1) + 1)/y^2; Taylor series sum_{k>=1} k y^(k-1)/(k+1)!
 * near 0, where the closed form cancels. */
static double e1_prime(double y) {
  if (fabs(y) < 1.0) {
    double s = 0.0, ypow = 1.0, fact = 2.0; /* (k+1)! for k = 1 */
    for (int k = 1; k <= 30; ++k) {
      s += k * ypow / fact;
      ypow *= y;
      fact *= (double)(k + 2);
    }
    return s;
  }
  return (exp(y) * (y - 1.0) + 1.0) / (y * y);
}

/* Neumaier compensated accumulator */
typedef struct {
  double s, c;
} nsum;
static void nsum_add(nsum* a, double x) {
  double t = a->s + x;
  if (fabs(a->s) >= fabs(x))
    a->c += (a->s - t) + x;
  else
    a->c += (x - t) + a->s;
  a->s = t;
}
static double nsum_val(const nsum* a) { return a->s + a->c; }

/* ------------------------------------------------------------------ */
/* expression leaves (ORC_EXPR)                                        */
/* ------------------------------------------------------------------ */
/* Formula PDFs (Sec. 4: RooGenericPdf, a PDF written as a formula string and
 * compiled just in time).  Here the text is parsed into a tree once per call
 * and the tree is walked for every value, with forward-mode derivatives with
 * respect to the leaf's parameters p0 .. p(m-1); the normalisation integral
 * and its derivatives come from adaptive Gauss-Legendre quadrature.
 * Grammar:
 *   sum   := prod (('+' | '-') prod)*
 *   prod  := unary (('*' | '/') unary)*
 *   unary := ('-' | '+') unary | power
 *   power := atom ('^' unary)?          (right-associative; -a^2 = -(a^2))
 *   atom  := number | 'x' | 'p'digits | name '(' sum ')' | 'pow' '(' sum ',' sum ')'
 *            | '(' sum ')'
 *   number: digits ['.' digits] [('e'|'E') ['+'|'-'] digits], or '.' digits ...
 *   name: exp log sqrt sin cos tanh sinh cosh asinh atan erf erfc abs
 * a^b (and pow(a, b)) with b an integer literal is a repeated product, valid
 * for any sign of a; any other b gives exp(b log a). */
enum {
  X_NUM, X_VAR, X_PAR, X_NEG, X_ADD, X_SUB, X_MUL, X_DIV, X_POWI, X_POW,
  X_EXP, X_LOG, X_SQRT, X_SIN, X_COS, X_TANH, X_SINH, X_COSH, X_ASINH, X_ATAN,
  X_ERF, X_ERFC, X_ABS
};
#define ORC_XMAX 256
#define ORC_XLEN 4096
typedef struct {
  int op, a, b;
  double c;
} xnode;
typedef struct {
  xnode n[ORC_XMAX];
  int len, root;
} xprog;
typedef struct {
  const char* s;
  int pos, npar, err, depth;
  xprog* p;
} xparser;

static const struct {
  const char* name;
  int op;
} xfuncs[] = {{"exp", X_EXP},     {"log", X_LOG},   {"sqrt", X_SQRT}, {"sin", X_SIN},
              {"cos", X_COS},     {"tanh", X_TANH}, {"sinh", X_SINH}, {"cosh", X_COSH},
              {"asinh", X_ASINH}, {"atan", X_ATAN}, {"erf", X_ERF},   {"erfc", X_ERFC},
              {"abs", X_ABS}};

static int xnew(xparser* q, int op, int a, int b, double c) {
  if (q->p->len >= ORC_XMAX) {
    q->err = 1;
    return 0;
  }
  xnode* n = &q->p->n[q->p->len];
  n->op = op;
  n->a = a;
  n->b = b;
  n->c = c;
  return q->p->len++;
}
static void xskip(xparser* q) {
  while (q->s[q->pos] == ' ' || q->s[q->pos] == '\t' || q->s[q->pos] == '\n') q->pos++;
}
static int xisdigit(char c) { return c >= '0' && c <= '9'; }
static int xisalpha(char c) { return (c >= 'a' && c <= 'z') || (c >= 'A' && c <= 'Z') || c == '_'; }
static int xsum(xparser* q);
static int xunary(xparser* q);

/* a^b: an integer literal exponent becomes X_POWI (exponent in c) */
static int xpow_node(xparser* q, int base, int ex) {
  const xnode* e = &q->p->n[ex];
  if (e->op == X_NUM && e->c == floor(e->c) && fabs(e->c) <= 64.0)
    return xnew(q, X_POWI, base, -1, e->c);
  if (e->op == X_NEG && q->p->n[e->a].op == X_NUM) {
    double v = -q->p->n[e->a].c;
    if (v == floor(v) && fabs(v) <= 64.0) return xnew(q, X_POWI, base, -1, v);
  }
  return xnew(q, X_POW, base, ex, 0.0);
}

static int xatom(xparser* q) {
  xskip(q);
  const char* s = q->s;
  char c = s[q->pos];
  if (xisdigit(c) || (c == '.' && xisdigit(s[q->pos + 1]))) {
    int b = q->pos;
    while (xisdigit(s[q->pos])) q->pos++;
    if (s[q->pos] == '.') {
      q->pos++;
      while (xisdigit(s[q->pos])) q->pos++;
    }
    if (s[q->pos] == 'e' || s[q->pos] == 'E') {
      int save = q->pos++;
      if (s[q->pos] == '+' || s[q->pos] == '-') q->pos++;
      if (!xisdigit(s[q->pos])) {
        q->pos = save;
        q->err = 1;
        return 0;
      }
      while (xisdigit(s[q->pos])) q->pos++;
    }
    char buf[64];
    int len = q->pos - b;
    if (len >= (int)sizeof(buf)) {
      q->err = 1;
      return 0;
    }
    memcpy(buf, s + b, (size_t)len);
    buf[len] = 0;
    return xnew(q, X_NUM, -1, -1, strtod(buf, NULL));
  }
  if (xisalpha(c)) {
    int b = q->pos;
    while (xisalpha(s[q->pos]) || xisdigit(s[q->pos])) q->pos++;
    int len = q->pos - b;
    if (len == 1 && c == 'x') return xnew(q, X_VAR, -1, -1, 0.0);
    if (c == 'p' && len >= 2) {
      int k = 0, allnum = 1;
      for (int i = 1; i < len; ++i) {
        if (!xisdigit(s[b + i])) allnum = 0;
        else k = k * 10 + (s[b + i] - '0');
        if (k > 1000) allnum = 0;
      }
      if (allnum) {
        if (k >= q->npar) {
          q->err = 1;
          return 0;
        }
        return xnew(q, X_PAR, k, -1, 0.0);
      }
    }
    int op = -1, is_pow = (len == 3 && strncmp(s + b, "pow", 3) == 0);
    for (size_t i = 0; i < sizeof(xfuncs) / sizeof(xfuncs[0]); ++i)
      if ((int)strlen(xfuncs[i].name) == len && strncmp(s + b, xfuncs[i].name, (size_t)len) == 0)
        op = xfuncs[i].op;
    if (op < 0 && !is_pow) {
      q->err = 1;
      return 0;
    }
    xskip(q);
    if (s[q->pos] != '(') {
      q->err = 1;
      return 0;
    }
    q->pos++;
    int a = xsum(q);
    if (q->err) return 0;
    xskip(q);
    int r;
    if (is_pow) {
      if (s[q->pos] != ',') {
        q->err = 1;
        return 0;
      }
      q->pos++;
      int e = xsum(q);
      if (q->err) return 0;
      xskip(q);
      r = xpow_node(q, a, e);
    } else {
      r = xnew(q, op, a, -1, 0.0);
    }
    if (s[q->pos] != ')') {
      q->err = 1;
      return 0;
    }
    q->pos++;
    return r;
  }
  if (c == '(') {
    q->pos++;
    int a = xsum(q);
    if (q->err) return 0;
    xskip(q);
    if (s[q->pos] != ')') {
      q->err = 1;
      return 0;
    }
    q->pos++;
    return a;
  }
  q->err = 1;
  return 0;
}

static int xpower(xparser* q) {
  int a = xatom(q);
  if (q->err) return 0;
  xskip(q);
  if (q->s[q->pos] == '^') {
    q->pos++;
    int e = xunary(q);
    if (q->err) return 0;
    return xpow_node(q, a, e);
  }
  return a;
}

static int xunary(xparser* q) {
  if (++q->depth > 200) {
    q->err = 1;
    return 0;
  }
  xskip(q);
  int r;
  if (q->s[q->pos] == '-') {
    q->pos++;
    int a = xunary(q);
    r = q->err ? 0 : xnew(q, X_NEG, a, -1, 0.0);
  } else if (q->s[q->pos] == '+') {
    q->pos++;
    r = xunary(q);
  } else {
    r = xpower(q);
  }
  q->depth--;
  return r;
}

static int xprod(xparser* q) {
  int a = xunary(q);
  while (!q->err) {
    xskip(q);
    char c = q->s[q->pos];
    if (c != '*' && c != '/') break;
    q->pos++;
    int b = xunary(q);
    if (q->err) return 0;
    a = xnew(q, c == '*' ? X_MUL : X_DIV, a, b, 0.0);
  }
  return a;
}

static int xsum(xparser* q) {
  if (++q->depth > 200) {
    q->err = 1;
    return 0;
  }
  int a = xprod(q);
  while (!q->err) {
    xskip(q);
    char c = q->s[q->pos];
    if (c != '+' && c != '-') break;
    q->pos++;
    int b = xprod(q);
    if (q->err) return 0;
    a = xnew(q, c == '+' ? X_ADD : X_SUB, a, b, 0.0);
  }
  q->depth--;
  return a;
}

/* Parses text with parameters p0 .. p(npar-1).  ORC_EINVAL on any error. */
static int xparse(const char* text, int npar, xprog* p) {
  if (!text || npar < 0 || npar > ORC_MAXNP || strlen(text) > ORC_XLEN) return ORC_EINVAL;
  xparser q = {text, 0, npar, 0, 0, p};
  p->len = 0;
  p->root = xsum(&q);
  xskip(&q);
  if (q.err || text[q.pos] != 0) return ORC_EINVAL;
  return ORC_OK;
}

/* value v and dv[j] = dv/dp_j (j < m) of node i */
static void xeval(const xprog* p, int i, double x, const double* th, int m, double* v,
                  double* dv) {
  const xnode* n = &p->n[i];
  double a, da[ORC_MAXNP], b, db[ORC_MAXNP];
  for (int j = 0; j < m; ++j) dv[j] = 0.0;
  switch (n->op) {
    case X_NUM:
      *v = n->c;
      return;
    case X_VAR:
      *v = x;
      return;
    case X_PAR:
      *v = th[n->a];
      dv[n->a] = 1.0;
      return;
    default:
      break;
  }
  xeval(p, n->a, x, th, m, &a, da);
  if (n->op >= X_ADD && n->op <= X_DIV) xeval(p, n->b, x, th, m, &b, db);
  if (n->op == X_POW) xeval(p, n->b, x, th, m, &b, db);
  double s = 0.0; /* dv = s * da (one-argument functions) */
  switch (n->op) {
    case X_NEG: *v = -a; s = -1.0; break;
    case X_ADD:
      *v = a + b;
      for (int j = 0; j < m; ++j) dv[j] = da[j] + db[j];
      return;
    case X_SUB:
      *v = a - b;
      for (int j = 0; j < m; ++j) dv[j] = da[j] - db[j];
      return;
    case X_MUL:
      *v = a * b;
      for (int j = 0; j < m; ++j) dv[j] = da[j] * b + a * db[j];
      return;
    case X_DIV:
      *v = a / b;
      for (int j = 0; j < m; ++j) dv[j] = (da[j] - *v * db[j]) / b;
      return;
    case X_POWI: {
      double k = n->c;
      *v = pow(a, k);
      s = k == 0.0 ? 0.0 : k * pow(a, k - 1.0);
      break;
    }
    case X_POW: {
      double la = log(a);
      *v = exp(b * la);
      for (int j = 0; j < m; ++j) dv[j] = *v * (db[j] * la + b * da[j] / a);
      return;
    }
    case X_EXP: *v = exp(a); s = *v; break;
    case X_LOG: *v = log(a); s = 1.0 / a; break;
    case X_SQRT: *v = sqrt(a); s = 0.5 / *v; break;
    case X_SIN: *v = sin(a); s = cos(a); break;
    case X_COS: *v = cos(a); s = -sin(a); break;
    case X_TANH: *v = tanh(a); s = 1.0 - *v * *v; break;
    case X_SINH: *v = sinh(a); s = cosh(a); break;
    case X_COSH: *v = cosh(a); s = sinh(a); break;
    case X_ASINH: *v = asinh(a); s = 1.0 / sqrt(1.0 + a * a); break;
    case X_ATAN: *v = atan(a); s = 1.0 / (1.0 + a * a); break;
    case X_ERF: *v = erf(a); s = (2.0 / SQRT_PI) * exp(-a * a); break;
    case X_ERFC: *v = erfc(a); s = -(2.0 / SQRT_PI) * exp(-a * a); break;
    case X_ABS: *v = fabs(a); s = a < 0.0 ? -1.0 : 1.0; break;
    default: *v = NAN; return;
  }
  for (int j = 0; j < m; ++j) dv[j] = s * da[j];
}

/* n-point Gauss-Legendre nodes and weights on [-1, 1]: Newton's method on
 * P_n(t) from the usual cosine first guesses, P_n and P_n' by the three-term
 * recurrence (Golub & Welsch's alternative is not needed at n = 20). */
#define ORC_GLN 20
static void gl_rule(double* t, double* w) {
  const int n = ORC_GLN;
  for (int i = 0; i < n; ++i) {
    double z = cos(PI_VAL * (i + 0.75) / (n + 0.5)), dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      double dz = p1 / dp;
      z -= dz;
      if (fabs(dz) < 1e-17) break;
    }
    t[i] = z;
    w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

/* integrand: v[0] = f(x), v[1..m] = its parameter derivatives */
typedef void (*qfn)(double x, const void* ctx, int m, double* v);
typedef struct {
  qfn fn;
  const void* ctx;
  int m;
  double t[ORC_GLN], w[ORC_GLN];
  double floor[1 + ORC_MAXNP]; /* absolute error allowed per unit length */
  long budget;
  int bad;
} xquad;

/* rule on [a, b]: out[c] = int v[c]; mag[] = int |v[c]| */
static void xrule(xquad* Q, double a, double b, double* out, double* mag) {
  double mid = 0.5 * (a + b), half = 0.5 * (b - a);
  for (int c = 0; c <= Q->m; ++c) out[c] = mag[c] = 0.0;
  for (int i = 0; i < ORC_GLN; ++i) {
    double v[1 + ORC_MAXNP];
    Q->fn(mid + half * Q->t[i], Q->ctx, Q->m, v);
    double wh = Q->w[i] * half;
    for (int c = 0; c <= Q->m; ++c) {
      if (!isfinite(v[c])) Q->bad = 1;
      out[c] += wh * v[c];
      mag[c] += wh * fabs(v[c]);
    }
  }
  Q->budget--;
}

/* adaptive bisection: accept the halves once they reproduce the whole to
 * 1e-14 of the absolute integrand in every component, or to the panel's share
 * of 1e-15 of the whole range's absolute integral (rounding noise of the
 * integrand near a singular end point must not force endless refinement) */
static void xadapt(xquad* Q, double a, double b, const double* whole, int depth, double* acc) {
  double l[1 + ORC_MAXNP], lm[1 + ORC_MAXNP], r[1 + ORC_MAXNP], rm[1 + ORC_MAXNP];
  double mid = 0.5 * (a + b);
  xrule(Q, a, mid, l, lm);
  xrule(Q, mid, b, r, rm);
  int done = depth >= 50 || Q->budget <= 0 || Q->bad;
  for (int c = 0; c <= Q->m && !done; ++c)
    if (fabs(l[c] + r[c] - whole[c]) > 1e-14 * (lm[c] + rm[c]) + Q->floor[c] * (b - a) + 1e-300)
      done = -1;
  if (done != -1) {
    for (int c = 0; c <= Q->m; ++c) acc[c] += l[c] + r[c];
    return;
  }
  xadapt(Q, a, mid, l, depth + 1, acc);
  xadapt(Q, mid, b, r, depth + 1, acc);
}

/* out[c] = int_lo^hi v[c] over 16 starting panels, adaptively refined;
 * returns 1 when the integrand was not finite somewhere */
static int quad(qfn fn, const void* ctx, int m, double lo, double hi, double* out) {
  xquad Q;
  Q.fn = fn;
  Q.ctx = ctx;
  Q.m = m;
  Q.budget = 200000;
  Q.bad = 0;
  gl_rule(Q.t, Q.w);
  double whole[16][1 + ORC_MAXNP], mag[1 + ORC_MAXNP], tot[1 + ORC_MAXNP] = {0};
  for (int k = 0; k < 16; ++k) {
    double a = lo + (hi - lo) * k / 16.0, b = k == 15 ? hi : lo + (hi - lo) * (k + 1) / 16.0;
    xrule(&Q, a, b, whole[k], mag);
    for (int c = 0; c <= m; ++c) tot[c] += mag[c];
  }
  for (int c = 0; c <= m; ++c) {
    Q.floor[c] = 1e-15 * tot[c] / (hi - lo);
    out[c] = 0.0;
  }
  for (int k = 0; k < 16; ++k) {
    double a = lo + (hi - lo) * k / 16.0, b = k == 15 ? hi : lo + (hi - lo) * (k + 1) / 16.0;
    xadapt(&Q, a, b, whole[k], 0, out);
  }
  return Q.bad;
}

typedef struct {
  const xprog* p;
  const double* th;
} xctx;

static void formula_fn(double x, const void* ctx, int m, double* v) {
  const xctx* c = (const xctx*)ctx;
  xeval(c->p, c->p->root, x, c->th, m, &v[0], &v[1]);
}

/* I = int_lo^hi f, dI[j] = int df/dp_j */
static int xnorm(const xprog* p, const double* th, int m, double lo, double hi, double* I,
                 double* dI) {
  xctx c = {p, th};
  double acc[1 + ORC_MAXNP];
  int bad = quad(formula_fn, &c, m, lo, hi, acc);
  *I = acc[0];
  for (int j = 0; j < m; ++j) dI[j] = acc[1 + j];
  if (bad || !isfinite(*I) || !(*I > 0.0)) return ORC_EDOMAIN;
  return ORC_OK;
}

/* ARGUS density x tau^p e^{c tau} and its c and p derivatives (tau and
 * log tau times it), zero from m0 up */
typedef struct {
  double m0, c, p;
} argus_ctx;

static void argus_fn(double x, const void* ctx, int m, double* v) {
  const argus_ctx* a = (const argus_ctx*)ctx;
  (void)m;
  if (x >= a->m0) {
    v[0] = v[1] = v[2] = 0.0;
    return;
  }
  double tau = (a->m0 - x) * (a->m0 + x) / (a->m0 * a->m0); /* no cancellation near m0 */
  double f = x * pow(tau, a->p) * exp(a->c * tau);
  v[0] = f;
  v[1] = f * tau;
  v[2] = f * log(tau);
}

/* ------------------------------------------------------------------ */
/* Bessel K of real order and the Hypatia2 leaf (ORC_HYPATIA2)         */
/* ------------------------------------------------------------------ */
/* K_nu(z) = int_0^inf e^{-z cosh t} cosh(nu t) dt (z > 0), in the scaled form
 * e^z K_nu(z) = int_0^inf phi(t) cosh(nu t) dt, phi = e^{-z (cosh t - 1)}.
 * bk_sums integrates, over [0, T], with the adaptive Gauss-Legendre rule:
 *   S0 = int phi cosh(nu t)            = e^z K
 *   S1 = -int cosh t phi cosh(nu t)    = e^z dK/dz
 *   S2 = int t phi sinh(nu t)          = e^z dK/dnu
 *   S3 = int cosh^2 t phi cosh(nu t)   = e^z d2K/dz2
 *   S4 = -int t cosh t phi sinh(nu t)  = e^z d2K/dz dnu
 * T lies past the integrand's peak t* = asinh(|nu|/z) where the largest
 * moment has fallen by e^-46 from its value at t*. */
typedef struct {
  double nu, z;
} bk_ctx;

static void bk_fn(double t, const void* ctx, int m, double* v) {
  const bk_ctx* b = (const bk_ctx*)ctx;
  (void)m;
  double ch = cosh(t), ph = exp(-b->z * (ch - 1.0));
  double cn = cosh(b->nu * t), sn = sinh(b->nu * t);
  v[0] = ph * cn;
  v[1] = -ch * ph * cn;
  v[2] = t * ph * sn;
  v[3] = ch * ch * ph * cn;
  v[4] = -t * ch * ph * sn;
}

static int bk_sums(double nu, double z, double* S) {
  if (!(z > 0.0) || !isfinite(z) || !isfinite(nu)) return ORC_EDOMAIN;
  double an = fabs(nu), tp = asinh(an / z);
  /* log of the largest moment's integrand, up to constants */
  double gpk = -z * (cosh(tp) - 1.0) + an * tp + 2.0 * tp + log(tp + 1.0);
  double T = tp + 0.5, step = 0.5;
  for (int it = 0; it < 400; ++it) {
    double g = -z * (cosh(T) - 1.0) + an * T + 2.0 * T + log(T + 1.0);
    if (g < gpk - 46.0) break;
    T += step;
  }
  bk_ctx c = {nu, z};
  int bad = quad(bk_fn, &c, 4, 0.0, T, S);
  return bad || !(S[0] > 0.0) ? ORC_EDOMAIN : ORC_OK;
}

int orc_besselk(double nu, double z, double* out) {
  double S[5];
  int rc = bk_sums(nu, z, S);
  if (rc) return rc;
  double ez = exp(-z);
  out[0] = S[0] * ez;
  out[1] = S[1] * ez;
  out[2] = S[2] * ez;
  return ORC_OK;
}

/* forward-mode dual numbers over the nine Hypatia2 parameters */
#define ORC_HNP 9
typedef struct {
  double v, d[ORC_HNP];
} hd;

static hd hd_c(double v) {
  hd r;
  r.v = v;
  for (int j = 0; j < ORC_HNP; ++j) r.d[j] = 0.0;
  return r;
}
static hd hd_var(double v, int k) {
  hd r = hd_c(v);
  r.d[k] = 1.0;
  return r;
}
static hd hd_add(hd a, hd b) {
  for (int j = 0; j < ORC_HNP; ++j) a.d[j] += b.d[j];
  a.v += b.v;
  return a;
}
static hd hd_sub(hd a, hd b) {
  for (int j = 0; j < ORC_HNP; ++j) a.d[j] -= b.d[j];
  a.v -= b.v;
  return a;
}
static hd hd_mul(hd a, hd b) {
  hd r;
  r.v = a.v * b.v;
  for (int j = 0; j < ORC_HNP; ++j) r.d[j] = a.d[j] * b.v + a.v * b.d[j];
  return r;
}
static hd hd_div(hd a, hd b) {
  hd r;
  r.v = a.v / b.v;
  for (int j = 0; j < ORC_HNP; ++j) r.d[j] = (a.d[j] - r.v * b.d[j]) / b.v;
  return r;
}
static hd hd_scale(hd a, double s) {
  a.v *= s;
  for (int j = 0; j < ORC_HNP; ++j) a.d[j] *= s;
  return a;
}
static hd hd_shift(hd a, double s) {
  a.v += s;
  return a;
}
/* f(a) from its value fv and slope fs at a.v */
static hd hd_chain(hd a, double fv, double fs) {
  hd r;
  r.v = fv;
  for (int j = 0; j < ORC_HNP; ++j) r.d[j] = fs * a.d[j];
  return r;
}
static hd hd_log(hd a) { return hd_chain(a, log(a.v), 1.0 / a.v); }
static hd hd_exp(hd a) {
  double e = exp(a.v);
  return hd_chain(a, e, e);
}
static hd hd_sqrt(hd a) {
  double s = sqrt(a.v);
  return hd_chain(a, s, 0.5 / s);
}
/* log K_nu(z) and d log K_nu(z)/dz, each with its derivatives through nu, z */
static hd hd_logK(hd nu, hd z, int* rc) {
  double S[5];
  if (bk_sums(nu.v, z.v, S)) {
    *rc = ORC_EDOMAIN;
    return hd_c(NAN);
  }
  hd r;
  r.v = log(S[0]) - z.v;
  for (int j = 0; j < ORC_HNP; ++j) r.d[j] = S[2] / S[0] * nu.d[j] + S[1] / S[0] * z.d[j];
  return r;
}
static hd hd_dlogK(hd nu, hd z, int* rc) {
  double S[5];
  if (bk_sums(nu.v, z.v, S)) {
    *rc = ORC_EDOMAIN;
    return hd_c(NAN);
  }
  const double q1 = S[1] / S[0], q2 = S[2] / S[0];
  hd r;
  r.v = q1;
  for (int j = 0; j < ORC_HNP; ++j)
    r.d[j] = (S[4] / S[0] - q1 * q2) * nu.d[j] + (S[3] / S[0] - q1 * q1) * z.d[j];
  return r;
}

/* Hypatia2 (a reading: the paper names the PDF only).  With d = x - mu,
 * phi = K_{lambda+1}(zeta) / K_lambda(zeta), delta = sigma sqrt(zeta / phi),
 * alpha = sqrt(zeta phi) / sigma (alpha delta = zeta; beta enters through
 * e^{beta d} only) and nu = lambda - 1/2, the core is the generalised
 * hyperbolic density up to a constant factor:
 *   L(d) = (nu/2) log(d^2 + delta^2) + beta d + log K_nu(alpha sqrt(d^2 + delta^2)) + zeta
 * (the constant zeta keeps e^L of order one near the peak).  Below
 * d_L = -a sigma and above d_R = a2 sigma, power-law tails continue it with
 * the same value and slope k = dL/dd at the junction:
 *   L = L(d_J) - m log(1 - (d - d_J) k(d_J) / m),  (d_J, m) = (d_L, n) or (d_R, n2).
 * k(d) = nu d / (d^2 + delta^2) + beta + alpha (d / r) (d log K_nu / dz)(alpha r).
 * Returns log f and its derivatives with respect to the nine parameters;
 * log f = -inf where a tail's base is not positive. */
static hd hyp2_core(hd d, hd nu, hd beta, hd alpha, hd delta2, hd zeta, hd* slope, int* rc) {
  hd q = hd_add(hd_mul(d, d), delta2), r = hd_sqrt(q), z = hd_mul(alpha, r);
  hd L = hd_add(hd_add(hd_scale(hd_mul(nu, hd_log(q)), 0.5), hd_mul(beta, d)),
                hd_add(hd_logK(nu, z, rc), zeta));
  if (slope)
    *slope = hd_add(hd_add(hd_div(hd_mul(nu, d), q), beta),
                    hd_mul(hd_div(hd_mul(alpha, d), r), hd_dlogK(nu, z, rc)));
  return L;
}

static int hyp2_logf(const double* th, double x, double* logf, double* dlogf) {
  hd lam = hd_var(th[0], 0), zeta = hd_var(th[1], 1), beta = hd_var(th[2], 2);
  hd sigma = hd_var(th[3], 3), mu = hd_var(th[4], 4), a = hd_var(th[5], 5);
  hd n = hd_var(th[6], 6), a2 = hd_var(th[7], 7), n2 = hd_var(th[8], 8);
  if (!(th[1] > 0.0) || !(th[3] > 0.0) || !(th[5] > 0.0) || !(th[6] > 0.0) ||
      !(th[7] > 0.0) || !(th[8] > 0.0))
    return ORC_EDOMAIN;
  int rc = ORC_OK;
  hd logphi = hd_sub(hd_logK(hd_shift(lam, 1.0), zeta, &rc), hd_logK(lam, zeta, &rc));
  hd logz = hd_log(zeta), logs = hd_log(sigma);
  hd delta2 = hd_exp(hd_add(hd_scale(logs, 2.0), hd_sub(logz, logphi)));
  hd alpha = hd_exp(hd_sub(hd_scale(hd_add(logz, logphi), 0.5), logs));
  hd nu = hd_shift(lam, -0.5);
  hd d = hd_sub(hd_c(x), mu);
  hd dL = hd_scale(hd_mul(a, sigma), -1.0), dR = hd_mul(a2, sigma);
  hd L;
  if (d.v < dL.v || d.v > dR.v) {
    const int left = d.v < dL.v;
    hd dJ = left ? dL : dR, m = left ? n : n2, k;
    hd LJ = hyp2_core(dJ, nu, beta, alpha, delta2, zeta, &k, &rc);
    hd base = hd_sub(hd_c(1.0), hd_div(hd_mul(hd_sub(d, dJ), k), m));
    if (!(base.v > 0.0)) {
      *logf = -INFINITY;
      for (int j = 0; j < ORC_HNP; ++j) dlogf[j] = 0.0;
      return rc;
    }
    L = hd_sub(LJ, hd_mul(m, hd_log(base)));
  } else {
    L = hyp2_core(d, nu, beta, alpha, delta2, zeta, NULL, &rc);
  }
  *logf = L.v;
  for (int j = 0; j < ORC_HNP; ++j) dlogf[j] = L.d[j];
  return rc;
}

/* integrand of the normalisation: v[0] = f, v[1 + j] = df/dtheta_j */
typedef struct {
  const double* th;
  int bad;
} hyp2_ctx;

static void hyp2_fn(double x, const void* ctx, int m, double* v) {
  hyp2_ctx* c = (hyp2_ctx*)ctx;
  double lf, dl[ORC_HNP];
  if (hyp2_logf(c->th, x, &lf, dl)) c->bad = 1;
  double f = exp(lf);
  v[0] = f;
  for (int j = 0; j < m; ++j) v[1 + j] = f == 0.0 ? 0.0 : f * dl[j];
}

int orc_expr_check(const char* text, int npar) {
  xprog* p = (xprog*)malloc(sizeof(xprog));
  if (!p) return ORC_EINVAL;
  int rc = xparse(text, npar, p);
  free(p);
  return rc;
}

int orc_expr_logf(const char* text, const double* theta, int ntheta, double x, double* logf,
                  double* dlogf) {
  xprog* p = (xprog*)malloc(sizeof(xprog));
  if (!p) return ORC_EINVAL;
  int rc = xparse(text, ntheta, p);
  if (rc == ORC_OK) {
    double v, dv[ORC_MAXNP];
    xeval(p, p->root, x, theta, ntheta, &v, dv);
    *logf = v > 0.0 ? log(v) : (v == 0.0 ? -INFINITY : NAN);
    for (int j = 0; j < ntheta; ++j) dlogf[j] = v > 0.0 ? dv[j] / v : 0.0;
  }
  free(p);
  return rc;
}

int orc_expr_norm(const char* text, const double* theta, int ntheta, double lo, double hi,
                  double* I, double* dI) {
  if (!(hi > lo)) return ORC_EINVAL;
  xprog* p = (xprog*)malloc(sizeof(xprog));
  if (!p) return ORC_EINVAL;
  int rc = xparse(text, ntheta, p);
  if (rc == ORC_OK) rc = xnorm(p, theta, ntheta, lo, hi, I, dI);
  free(p);
  return rc;
}

/* ------------------------------------------------------------------ */
/* leaves: unnormalised value f and d log f / d theta_j                */
/* ------------------------------------------------------------------ */

/* Returns f(x) (may be 0, or negative for a Chebychev polynomial) and fills
 * dlogf[j] = d log f / d theta_j where f > 0. */
static int leaf_value(int type, const double* th, int nth, double lo, double hi,
                      double x, const xprog* xp, double* f_out, double* dlogf) {
  for (int j = 0; j < nth; ++j) dlogf[j] = 0.0;
  switch (type) {
    case ORC_HYPATIA2: {
      if (nth != 9) return ORC_EINVAL;
      double lf;
      int rc = hyp2_logf(th, x, &lf, dlogf);
      if (rc) return rc;
      *f_out = exp(lf);
      return ORC_OK;
    }
    case ORC_EXPR: {
      if (!xp) return ORC_EINVAL;
      double dv[ORC_MAXNP];
      xeval(xp, xp->root, x, th, nth, f_out, dv);
      if (*f_out > 0.0)
        for (int j = 0; j < nth; ++j) dlogf[j] = dv[j] / *f_out;
      return ORC_OK;
    }
    case ORC_GAUSS: {
      if (nth != 2) return ORC_EINVAL;
      double mu = th[0], sigma = th[1];
      double d = (x - mu) / sigma;
      *f_out = exp(-0.5 * d * d);
      dlogf[0] = (x - mu) / (sigma * sigma);
      dlogf[1] = (x - mu) * (x - mu) / (sigma * sigma * sigma);
      return ORC_OK;
    }
    case ORC_EXP: {
      if (nth != 1) return ORC_EINVAL;
      *f_out = exp(th[0] * x);
      dlogf[0] = x;
      return ORC_OK;
    }
    case ORC_CHEB: {
      if (nth < 1 || nth > ORC_MAXNP) return ORC_EINVAL;
      double xp = (2.0 * x - lo - hi) / (hi - lo);
      double T[ORC_MAXNP + 1];
      T[0] = 1.0;
      T[1] = xp;
      for (int j = 2; j <= nth; ++j) T[j] = 2.0 * xp * T[j - 1] - T[j - 2];
      double f = 1.0;
      for (int j = 1; j <= nth; ++j) f += th[j - 1] * T[j];
      *f_out = f;
      for (int j = 1; j <= nth; ++j) dlogf[j - 1] = T[j] / f;
      return ORC_OK;
    }
    case ORC_CB: {
      if (nth != 4) return ORC_EINVAL;
      double m0 = th[0], sigma = th[1], alpha = th[2], n = th[3];
      double s = alpha >= 0.0 ? 1.0 : -1.0;
      double A = fabs(alpha);
      double t = s * (x - m0) / sigma;
      double du_dt, du_dA = 0.0, du_dn = 0.0, u;
      if (t > -A) {
        u = -0.5 * t * t;
        du_dt = -t;
      } else {
        double D = 1.0 - (A / n) * (A + t);
        u = -0.5 * A * A - n * log(D);
        du_dt = A / D;
        du_dA = -A + (2.0 * A + t) / D;
        du_dn = -log(D) + 1.0 - 1.0 / D;
      }
      *f_out = exp(u);
      dlogf[0] = du_dt * (-s / sigma);
      dlogf[1] = du_dt * (-t / sigma);
      dlogf[2] = s * du_dA;
      dlogf[3] = du_dn;
      return ORC_OK;
    }
    case ORC_ARGUS: {
      if (nth != 3) return ORC_EINVAL;
      double m0 = th[0], c = th[1], p = th[2];
      if (x >= m0) {
        *f_out = 0.0;
        return ORC_OK;
      }
      /* tau = 1 - (x/m0)^2 as (m0 - x)(m0 + x) / m0^2: the same value
       * without the cancellation of 1 - r^2 as x approaches m0 */
      double tau = (m0 - x) * (m0 + x) / (m0 * m0);
      *f_out = x * pow(tau, p) * exp(c * tau);
      dlogf[0] = (p / tau + c) * 2.0 * x * x / (m0 * m0 * m0);
      dlogf[1] = tau;
      dlogf[2] = log(tau);
      return ORC_OK;
    }
    case ORC_JOHNSON: {
      /* Johnson's SU (N. L. Johnson, Biometrika 36 (1949) 149): z = (x-mu)/lambda,
       * w = gamma + delta asinh z standard normal;
       * f = delta / (lambda sqrt(2 pi) sqrt(1 + z^2)) exp(-w^2 / 2) */
      if (nth != 4) return ORC_EINVAL;
      double mu = th[0], lam = th[1], gam = th[2], del = th[3];
      double z = (x - mu) / lam, r = sqrt(1.0 + z * z), as = asinh(z);
      double w = gam + del * as;
      *f_out = del / (lam * 2.5066282746310002 * r) * exp(-0.5 * w * w);
      double dz = -z / (r * r) - w * del / r; /* d log f / dz */
      dlogf[0] = dz * (-1.0 / lam);
      dlogf[1] = -1.0 / lam + dz * (-z / lam);
      dlogf[2] = -w;
      dlogf[3] = 1.0 / del - w * as;
      return ORC_OK;
    }
    default:
      return ORC_EINVAL;
  }
}

/* ------------------------------------------------------------------ */
/* leaves: normalisation integrals and their derivatives               */
/* ------------------------------------------------------------------ */

/* G(q, tau, c) = int_0^tau s^q e^{c s} ds for q = 1/2 or 3/2.
 * Closed form through the lower incomplete gamma function when c < 0 and
 * k tau >= 1/2 (k = -c):
 *   gamma(3/2, y) = (sqrt(pi)/2) erf(sqrt y) - sqrt(y) e^-y
 *   gamma(5/2, y) = (3/2) gamma(3/2, y) - y^(3/2) e^-y
 *   G = k^-(q+1) gamma(q+1, k tau);
 * otherwise the power series tau^(q+1) sum_j (c tau)^j / (j! (j+q+1)). */
static double argus_G(double q, double tau, double c) {
  if (tau <= 0.0) return 0.0;
  double y = c * tau;
  if (c < 0.0 && -y >= 0.5) {
    double k = -c, ky = -y;
    double g32 = 0.5 * SQRT_PI * erf(sqrt(ky)) - sqrt(ky) * exp(-ky);
    if (q == 0.5) return pow(k, -1.5) * g32;
    double g52 = 1.5 * g32 - pow(ky, 1.5) * exp(-ky);
    return pow(k, -2.5) * g52;
  }
  double sum = 0.0, term = 1.0; /* y^j / j! */
  for (int j = 0; j < 2000; ++j) {
    double add = term / (j + q + 1.0);
    sum += add;
    if (j > fabs(y) && fabs(add) < 1e-18 * fabs(sum)) break;
    term *= y / (j + 1.0);
  }
  return pow(tau, q + 1.0) * sum;
}

static int leaf_norm(int type, const double* th, int nth, double lo, double hi,
                     const xprog* xp, double* I_out, double* dI) {
  for (int j = 0; j < nth; ++j) dI[j] = 0.0;
  if (!(hi > lo)) return ORC_EINVAL;
  switch (type) {
    case ORC_EXPR:
      if (!xp) return ORC_EINVAL;
      return xnorm(xp, th, nth, lo, hi, I_out, dI);
    case ORC_HYPATIA2: {
      /* no closed form: adaptive quadrature of f and its derivatives, on
       * the pieces between the tail junctions mu - a sigma, mu + a2 sigma
       * (the second derivative jumps there) */
      if (nth != 9) return ORC_EINVAL;
      hyp2_ctx c = {th, 0};
      double cut[4] = {lo, th[4] - th[5] * th[3], th[4] + th[7] * th[3], hi};
      int bad = 0;
      *I_out = 0.0;
      for (int k = 0; k < 3; ++k) {
        double a = cut[k] < lo ? lo : (cut[k] > hi ? hi : cut[k]);
        double b = cut[k + 1] < lo ? lo : (cut[k + 1] > hi ? hi : cut[k + 1]);
        if (!(b > a)) continue;
        double acc[1 + ORC_MAXNP];
        bad |= quad(hyp2_fn, &c, 9, a, b, acc);
        *I_out += acc[0];
        for (int j = 0; j < 9; ++j) dI[j] += acc[1 + j];
      }
      if (bad || c.bad || !isfinite(*I_out) || !(*I_out > 0.0)) return ORC_EDOMAIN;
      return ORC_OK;
    }
    case ORC_GAUSS: {
      if (nth != 2) return ORC_EINVAL;
      double mu = th[0], sigma = th[1];
      if (!(sigma > 0.0)) return ORC_EDOMAIN;
      double ua = (lo - mu) / sigma, ub = (hi - mu) / sigma;
      double I = sigma * SQRT_PI_2 * erf_diff(ua / SQRT2, ub / SQRT2);
      double fa = exp(-0.5 * ua * ua), fb = exp(-0.5 * ub * ub);
      *I_out = I;
      dI[0] = fa - fb;                       /* int (x-mu)/sigma^2 f dx  */
      dI[1] = ua * fa - ub * fb + I / sigma; /* int (x-mu)^2/sigma^3 f dx */
      return ORC_OK;
    }
    case ORC_EXP: {
      if (nth != 1) return ORC_EINVAL;
      double lam = th[0], L = hi - lo, s = lam * L;
      double I = exp(lam * lo) * L * e1(s);
      /* d I / d lambda = int x e^{lambda x} dx = I * <x>,
       * <x> = lo + L * (1/(1 - e^-s) - 1/s), series near s = 0 */
      double mfrac;
      if (fabs(s) < 1e-3)
        mfrac = 0.5 + s / 12.0 - s * s * s / 720.0 + s * s * s * s * s / 30240.0;
      else
        mfrac = 1.0 / (-expm1(-s)) - 1.0 / s;
      *I_out = I;
      dI[0] = I * (lo + L * mfrac);
      return ORC_OK;
    }
    case ORC_CHEB: {
      if (nth < 1 || nth > ORC_MAXNP) return ORC_EINVAL;
      /* int_{-1}^{1} T_j = (1 + (-1)^j)/(1 - j^2) for j != 1, 0 for j = 1 */
      double half = 0.5 * (hi - lo);
      double J = 2.0;
      for (int j = 1; j <= nth; ++j) {
        double tj = (j == 1) ? 0.0 : (1.0 + ((j % 2) ? -1.0 : 1.0)) / (1.0 - (double)j * j);
        J += th[j - 1] * tj;
        dI[j - 1] = half * tj;
      }
      *I_out = half * J;
      if (!(*I_out > 0.0)) return ORC_EDOMAIN;
      return ORC_OK;
    }
    case ORC_CB: {
      if (nth != 4) return ORC_EINVAL;
      double m0 = th[0], sigma = th[1], alpha = th[2], n = th[3];
      if (!(sigma > 0.0) || !(n > 0.0) || alpha == 0.0) return ORC_EDOMAIN;
      double s = alpha >= 0.0 ? 1.0 : -1.0, A = fabs(alpha);
      double tlo, thi;
      if (s > 0) {
        tlo = (lo - m0) / sigma;
        thi = (hi - m0) / sigma;
      } else {
        tlo = -(hi - m0) / sigma;
        thi = -(lo - m0) / sigma;
      }
      /* Gaussian core over [max(tlo,-A), thi] */
      double core = 0.0;
      if (thi > -A) {
        double c1 = tlo > -A ? tlo : -A;
        core = SQRT_PI_2 * erf_diff(c1 / SQRT2, thi / SQRT2);
      }
      /* power-law tail over [tlo, min(thi,-A)], in the variable D:
       * dt = -(n/A) dD, so tail = (n/A) e^{-A^2/2} int_{D2}^{D1} D^-n dD.
       * With eps = 1-n, L = log D, Delta = L1 - L2:
       *   Phi  = int D^{eps-1} dD       = e^{eps L2} Delta E1(eps Delta)
       *   Phi' = int D^{eps-1} log D dD = L2 Phi + e^{eps L2} Delta^2 E1'(eps Delta)
       *   Psi  = int D^{-n-1} dD        = (D2^-n - D1^-n)/n
       * and, at fixed t-limits (the integrand is continuous at t=-A, so the
       * moving split point contributes nothing),
       *   d tail/dA = (n/A) e^{-A^2/2} (A + n/A) (Psi - Phi)
       *   d tail/dn = (n/A) e^{-A^2/2} (Phi - Phi' - Psi). */
      double tail = 0.0, dT_dA = 0.0, dT_dn = 0.0;
      if (tlo < -A) {
        double t1 = tlo, t2 = thi < -A ? thi : -A;
        double D1 = 1.0 - (A / n) * (A + t1), D2 = 1.0 - (A / n) * (A + t2);
        double L1 = log(D1), L2 = log(D2), Dl = L1 - L2, eps = 1.0 - n;
        double ez = exp(eps * L2);
        double Phi = ez * Dl * e1(eps * Dl);
        double dPhi = L2 * Phi + ez * Dl * Dl * e1_prime(eps * Dl);
        double Psi = (pow(D2, -n) - pow(D1, -n)) / n;
        double pref = (n / A) * exp(-0.5 * A * A);
        tail = pref * Phi;
        dT_dA = pref * (A + n / A) * (Psi - Phi);
        dT_dn = pref * (Phi - dPhi - Psi);
      }
      double J = core + tail;
      /* integrand g(t) at the two ends of the range */
      double g_lo, g_hi;
      {
        double t = tlo;
        g_lo = (t > -A) ? exp(-0.5 * t * t)
                        : exp(-0.5 * A * A) * pow(1.0 - (A / n) * (A + t), -n);
        t = thi;
        g_hi = (t > -A) ? exp(-0.5 * t * t)
                        : exp(-0.5 * A * A) * pow(1.0 - (A / n) * (A + t), -n);
      }
      *I_out = sigma * J;
      dI[0] = -s * (g_hi - g_lo);
      dI[1] = J + (tlo * g_lo - thi * g_hi);
      dI[2] = s * sigma * dT_dA;
      dI[3] = sigma * dT_dn;
      return ORC_OK;
    }
    case ORC_ARGUS: {
      if (nth != 3) return ORC_EINVAL;
      double m0 = th[0], c = th[1], p = th[2];
      if (!(m0 > lo) || lo < 0.0 || !(p > 0.0)) return ORC_EDOMAIN;
      double bp = hi < m0 ? hi : m0;
      /* the integral and its c and p derivatives by quadrature of the
       * density (the p derivative always: it has no closed form) */
      argus_ctx ac = {m0, c, p};
      double q[3];
      if (quad(argus_fn, &ac, 2, lo, bp, q)) return ORC_EDOMAIN;
      dI[2] = q[2];
      if (p != 0.5) {
        /* d/dm0 by differentiating under the integral sign with the limit
         * b' = min(hi, m0): in tau = 1 - (x/m0)^2 the integral is
         * (m0^2/2) int_{tau(b')}^{tau(lo)} tau^p e^{c tau}, whose m0
         * derivative is 2I/m0 + (lo^2/m0) f_tau(tau(lo)) - (b'^2/m0) f_tau(tau(b')) */
        double ta = 1.0 - (lo / m0) * (lo / m0), tb = 1.0 - (bp / m0) * (bp / m0);
        double ea = pow(ta, p) * exp(c * ta), eb = tb > 0.0 ? pow(tb, p) * exp(c * tb) : 0.0;
        *I_out = q[0];
        dI[1] = q[1];
        dI[0] = 2.0 * q[0] / m0 + (lo * lo / m0) * ea - (bp * bp / m0) * eb;
        return ORC_OK;
      }
      double ra = lo / m0, rb = bp / m0;
      double ta = 1.0 - ra * ra, tb = 1.0 - rb * rb;
      /* m dm = -(m0^2/2) d tau */
      double h = 0.5 * m0 * m0;
      double I = h * (argus_G(0.5, ta, c) - argus_G(0.5, tb, c));
      *I_out = I;
      dI[1] = h * (argus_G(1.5, ta, c) - argus_G(1.5, tb, c));
      double ea = (1.0 - ta) * pow(ta, p) * exp(c * ta);
      double eb = tb > 0.0 ? (1.0 - tb) * pow(tb, p) * exp(c * tb) : 0.0;
      dI[0] = m0 * (ea - eb) + 2.0 * I / m0;
      return ORC_OK;
    }
    case ORC_JOHNSON: {
      /* the density integrates to 1 on the real line: on [lo, hi] it is
       * Phi(w(hi)) - Phi(w(lo)), w = gamma + delta asinh((x - mu)/lambda) */
      if (nth != 4) return ORC_EINVAL;
      double mu = th[0], lam = th[1], gam = th[2], del = th[3];
      if (!(lam > 0.0) || !(del > 0.0)) return ORC_EDOMAIN;
      double za = (lo - mu) / lam, zb = (hi - mu) / lam;
      double asa = asinh(za), asb = asinh(zb);
      double wa = gam + del * asa, wb = gam + del * asb;
      *I_out = 0.5 * erf_diff(wa / SQRT2, wb / SQRT2);
      double pa = exp(-0.5 * wa * wa) / 2.5066282746310002;
      double pb = exp(-0.5 * wb * wb) / 2.5066282746310002;
      double ra = sqrt(1.0 + za * za), rb = sqrt(1.0 + zb * zb);
      /* dI/dtheta = phi(wb) dwb/dtheta - phi(wa) dwa/dtheta */
      dI[0] = pb * (-del / (lam * rb)) - pa * (-del / (lam * ra));
      dI[1] = pb * (-del * zb / (lam * rb)) - pa * (-del * za / (lam * ra));
      dI[2] = pb - pa;
      dI[3] = pb * asb - pa * asa;
      return ORC_OK;
    }
    default:
      return ORC_EINVAL;
  }
}

int orc_leaf_logf(int type, const double* theta, int ntheta, double lo,
                  double hi, double x, double* logf, double* dlogf) {
  double f;
  int rc = leaf_value(type, theta, ntheta, lo, hi, x, NULL, &f, dlogf);
  if (rc) return rc;
  *logf = f > 0.0 ? log(f) : (f == 0.0 ? -INFINITY : NAN);
  return ORC_OK;
}

int orc_leaf_norm(int type, const double* theta, int ntheta, double lo,
                  double hi, double* I, double* dI) {
  return leaf_norm(type, theta, ntheta, lo, hi, NULL, I, dI);
}

/* ------------------------------------------------------------------ */
/* graph walk                                                          */
/* ------------------------------------------------------------------ */

static int is_leaf(int t) {
  return (t >= ORC_GAUSS && t <= ORC_ARGUS) || t == ORC_JOHNSON || t == ORC_EXPR ||
         t == ORC_HYPATIA2;
}

#define ORC_MAXXL 4 /* expression leaves per model */
typedef struct {
  double I[ORC_MAXNODE];
  double dlogI[ORC_MAXNODE][ORC_MAXNP];
  int xslot[ORC_MAXNODE]; /* parsed expression of node i, or -1 */
  xprog xp[ORC_MAXXL];
} leaf_cache;

/* bit mask of the observables a subtree depends on; -1 on a malformed graph */
static int64_t obs_mask(const orc_model* m, int i, int depth) {
  if (i < 0 || i >= m->n_nodes || depth > m->n_nodes) return -1;
  int t = m->type[i];
  if (is_leaf(t)) {
    int o = m->obs[i];
    if (o < 0 || o >= m->n_obs || o >= 62) return -1;
    return (int64_t)1 << o;
  }
  int64_t acc = 0;
  for (int k = 0; k < m->nchild[i]; ++k) {
    int64_t c = obs_mask(m, m->child[i * ORC_MAXCH + k], depth + 1);
    if (c < 0) return -1;
    if (t == ORC_PROD && (acc & c)) return -2; /* shared observable */
    acc |= c;
  }
  return acc;
}

static int validate(const orc_model* m) {
  if (!m || m->n_nodes <= 0 || m->n_nodes > ORC_MAXNODE) return ORC_EINVAL;
  if (m->root < 0 || m->root >= m->n_nodes) return ORC_EINVAL;
  if (m->n_par < 0 || m->n_par > ORC_MAXPAR) return ORC_EINVAL;
  for (int i = 0; i < m->n_nodes; ++i) {
    int t = m->type[i];
    if (t < ORC_GAUSS || t > ORC_HYPATIA2) return ORC_EINVAL;
    if (t == ORC_EXPR && !(m->expr && m->expr[i])) return ORC_EINVAL;
    if (m->npar[i] < 0 || m->npar[i] > ORC_MAXNP) return ORC_EINVAL;
    for (int j = 0; j < m->npar[i]; ++j) {
      int p = m->par[i * ORC_MAXNP + j];
      if (p < 0 || p >= m->n_par) return ORC_EINVAL;
    }
    if (!is_leaf(t)) {
      int K = m->nchild[i];
      if (K < 1 || K > ORC_MAXCH) return ORC_EINVAL;
      if (t == ORC_ADD_FRAC && (K < 2 || m->npar[i] != K - 1)) return ORC_EINVAL;
      if (t == ORC_ADD_EXT && m->npar[i] != K) return ORC_EINVAL;
      if (t == ORC_ADD_EXT && i != m->root) return ORC_EUNSUPPORTED;
      if (t == ORC_PROD && m->npar[i] != 0) return ORC_EINVAL;
    }
  }
  int64_t mask = obs_mask(m, m->root, 0);
  if (mask == -2) return ORC_EUNSUPPORTED;
  if (mask < 0) return ORC_EINVAL;
  for (int o = 0; o < m->n_obs; ++o)
    if (!(m->obs_hi[o] > m->obs_lo[o])) return ORC_EINVAL;
  return ORC_OK;
}

static int fill_cache(const orc_model* m, const double* params, leaf_cache* lc) {
  int rc_any = ORC_OK, nx = 0;
  for (int i = 0; i < m->n_nodes; ++i) {
    lc->xslot[i] = -1;
    if (m->type[i] != ORC_EXPR) continue;
    if (nx == ORC_MAXXL) return ORC_EUNSUPPORTED;
    if (xparse(m->expr[i], m->npar[i], &lc->xp[nx])) return ORC_EINVAL;
    lc->xslot[i] = nx++;
  }
  for (int i = 0; i < m->n_nodes; ++i) {
    if (!is_leaf(m->type[i])) continue;
    double th[ORC_MAXNP], dI[ORC_MAXNP];
    int np = m->npar[i];
    for (int j = 0; j < np; ++j) th[j] = params[m->par[i * ORC_MAXNP + j]];
    int o = m->obs[i];
    double I;
    const xprog* xp = lc->xslot[i] >= 0 ? &lc->xp[lc->xslot[i]] : NULL;
    int rc = leaf_norm(m->type[i], th, np, m->obs_lo[o], m->obs_hi[o], xp, &I, dI);
    if (rc == ORC_EINVAL || rc == ORC_EUNSUPPORTED) return rc;
    if (rc == ORC_EDOMAIN || !(I > 0.0) || !isfinite(I)) rc_any = ORC_EDOMAIN;
    lc->I[i] = I;
    for (int j = 0; j < np; ++j) lc->dlogI[i][j] = dI[j] / I;
  }
  return rc_any;
}

/* value v and derivative dv[n_par] (may be NULL) of node i at one event */
static void eval_node(const orc_model* m, int i, const double* params,
                      const double* xrow, const leaf_cache* lc, double* v,
                      double* dv) {
  int P = m->n_par;
  int t = m->type[i];
  if (dv)
    for (int p = 0; p < P; ++p) dv[p] = 0.0;
  if (is_leaf(t)) {
    double th[ORC_MAXNP] = {0}, dlogf[ORC_MAXNP], f;
    int np = m->npar[i], o = m->obs[i];
    for (int j = 0; j < np; ++j) th[j] = params[m->par[i * ORC_MAXNP + j]];
    leaf_value(t, th, np, m->obs_lo[o], m->obs_hi[o], xrow[o],
               lc->xslot[i] >= 0 ? &lc->xp[lc->xslot[i]] : NULL, &f, dlogf);
    double val = f / lc->I[i];
    *v = val;
    if (dv && f != 0.0)
      for (int j = 0; j < np; ++j)
        dv[m->par[i * ORC_MAXNP + j]] += val * (dlogf[j] - lc->dlogI[i][j]);
    return;
  }
  int K = m->nchild[i];
  double cv[ORC_MAXCH];
  double cdv[ORC_MAXCH][ORC_MAXPAR];
  for (int k = 0; k < K; ++k)
    eval_node(m, m->child[i * ORC_MAXCH + k], params, xrow, lc, &cv[k],
              dv ? cdv[k] : NULL);
  if (t == ORC_PROD) {
    double prod = 1.0;
    for (int k = 0; k < K; ++k) prod *= cv[k];
    *v = prod;
    if (dv)
      for (int k = 0; k < K; ++k) {
        double others = 1.0;
        for (int j = 0; j < K; ++j)
          if (j != k) others *= cv[j];
        for (int p = 0; p < P; ++p) dv[p] += others * cdv[k][p];
      }
    return;
  }
  /* Add: coefficients */
  double coef[ORC_MAXCH];
  if (t == ORC_ADD_FRAC) {
    double rest = 1.0;
    for (int k = 0; k < K - 1; ++k) {
      coef[k] = params[m->par[i * ORC_MAXNP + k]];
      rest -= coef[k];
    }
    coef[K - 1] = rest;
  } else {
    for (int k = 0; k < K; ++k) coef[k] = params[m->par[i * ORC_MAXNP + k]];
  }
  double sum = 0.0;
  for (int k = 0; k < K; ++k) sum += coef[k] * cv[k];
  *v = sum;
  if (dv) {
    for (int k = 0; k < K; ++k)
      for (int p = 0; p < P; ++p) dv[p] += coef[k] * cdv[k][p];
    if (t == ORC_ADD_FRAC) {
      for (int k = 0; k < K - 1; ++k)
        dv[m->par[i * ORC_MAXNP + k]] += cv[k] - cv[K - 1];
    } else {
      for (int k = 0; k < K; ++k) dv[m->par[i * ORC_MAXNP + k]] += cv[k];
    }
  }
}

/* parameter checks of the composite nodes (fractions in [0,1], yields >= 0) */
static int check_coefs(const orc_model* m, const double* params) {
  for (int i = 0; i < m->n_nodes; ++i) {
    int t = m->type[i];
    if (t == ORC_ADD_FRAC) {
      double rest = 1.0;
      for (int k = 0; k < m->nchild[i] - 1; ++k) {
        double f = params[m->par[i * ORC_MAXNP + k]];
        if (!(f >= 0.0 && f <= 1.0)) return ORC_EDOMAIN;
        rest -= f;
      }
      if (rest < -1e-15) return ORC_EDOMAIN;
    } else if (t == ORC_ADD_EXT) {
      for (int k = 0; k < m->nchild[i]; ++k)
        if (!(params[m->par[i * ORC_MAXNP + k]] >= 0.0)) return ORC_EDOMAIN;
    }
  }
  return ORC_OK;
}

#define ORC_CHUNK 4096

int orc_nll(const orc_model* m, const double* params, const double* cols,
            int64_t col_stride, int64_t n, int nthreads, double* nll,
            double* grad) {
  return orc_nll_scaled(m, params, cols, col_stride, n, nthreads, nll, grad,
                        NULL);
}

int orc_nll_scaled(const orc_model* m, const double* params, const double* cols,
                   int64_t col_stride, int64_t n, int nthreads, double* nll,
                   double* grad, double* gscale) {
  int rc = validate(m);
  if (rc) return rc;
  if (n < 0 || !params || !nll || (n > 0 && !cols)) return ORC_EINVAL;
  int P = m->n_par;
  leaf_cache lc;
  int drc = fill_cache(m, params, &lc);
  if (drc == ORC_EINVAL || drc == ORC_EUNSUPPORTED) return drc;
  if (drc == ORC_OK) drc = check_coefs(m, params);
  if (drc != ORC_OK) {
    *nll = INFINITY;
    if (grad)
      for (int p = 0; p < P; ++p) grad[p] = NAN;
    return ORC_EDOMAIN;
  }
  int64_t nchunks = (n + ORC_CHUNK - 1) / ORC_CHUNK;
  int want_scale = gscale != NULL && grad != NULL;
  int W = 1 + P + (want_scale ? P : 0);
  double* part = (double*)calloc((size_t)(nchunks > 0 ? nchunks : 1) * W, sizeof(double));
  int* bad = (int*)calloc((size_t)(nchunks > 0 ? nchunks : 1), sizeof(int));
  if (!part || !bad) {
    free(part);
    free(bad);
    return ORC_EINVAL;
  }
  int want_grad = grad != NULL;
#ifdef _OPENMP
  int nt = nthreads > 0 ? nthreads : omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(nt)
#endif
  for (int64_t ch = 0; ch < nchunks; ++ch) {
    nsum acc[1 + 2 * ORC_MAXPAR];
    memset(acc, 0, sizeof(acc));
    double xrow[64];
    double dv[ORC_MAXPAR];
    int64_t i0 = ch * ORC_CHUNK, i1 = i0 + ORC_CHUNK < n ? i0 + ORC_CHUNK : n;
    for (int64_t i = i0; i < i1; ++i) {
      for (int o = 0; o < m->n_obs; ++o) xrow[o] = cols[o * col_stride + i];
      double v;
      eval_node(m, m->root, params, xrow, &lc, &v, want_grad ? dv : NULL);
      if (!(v > 0.0) || !isfinite(v)) {
        bad[ch] = 1;
        continue;
      }
      nsum_add(&acc[0], -log(v));
      if (want_grad)
        for (int p = 0; p < P; ++p) nsum_add(&acc[1 + p], -dv[p] / v);
      if (want_scale)
        for (int p = 0; p < P; ++p) nsum_add(&acc[1 + P + p], fabs(dv[p] / v));
    }
    for (int w = 0; w < W; ++w) part[ch * W + w] = nsum_val(&acc[w]);
  }
  nsum tot[1 + 2 * ORC_MAXPAR];
  memset(tot, 0, sizeof(tot));
  int any_bad = 0;
  for (int64_t ch = 0; ch < nchunks; ++ch) {
    any_bad |= bad[ch];
    for (int w = 0; w < W; ++w) nsum_add(&tot[w], part[ch * W + w]);
  }
  free(part);
  free(bad);
  /* extended term: + sum_k nu_k, d/dnu_k = 1 */
  if (m->type[m->root] == ORC_ADD_EXT) {
    int r = m->root;
    for (int k = 0; k < m->nchild[r]; ++k) {
      int p = m->par[r * ORC_MAXNP + k];
      nsum_add(&tot[0], params[p]);
      nsum_add(&tot[1 + p], 1.0);
      if (want_scale) nsum_add(&tot[1 + P + p], 1.0);
    }
  }
  if (any_bad) {
    *nll = INFINITY;
    if (grad)
      for (int p = 0; p < P; ++p) grad[p] = NAN;
    return ORC_EDOMAIN;
  }
  *nll = nsum_val(&tot[0]);
  if (grad)
    for (int p = 0; p < P; ++p) grad[p] = nsum_val(&tot[1 + p]);
  if (want_scale)
    for (int p = 0; p < P; ++p) gscale[p] = nsum_val(&tot[1 + P + p]);
  return ORC_OK;
}

int orc_logp(const orc_model* m, const double* params, const double* cols,
             int64_t col_stride, int64_t n, double* logp) {
  int rc = validate(m);
  if (rc) return rc;
  leaf_cache lc;
  int drc = fill_cache(m, params, &lc);
  if (drc == ORC_EINVAL || drc == ORC_EUNSUPPORTED) return drc;
  double xrow[64];
  for (int64_t i = 0; i < n; ++i) {
    for (int o = 0; o < m->n_obs; ++o) xrow[o] = cols[o * col_stride + i];
    double v;
    eval_node(m, m->root, params, xrow, &lc, &v, NULL);
    logp[i] = v > 0.0 ? log(v) : (v == 0.0 ? -INFINITY : NAN);
  }
  return drc;
}

int orc_nll_batched(const orc_model* m, const double* cols, int64_t col_stride,
                    const int64_t* offsets, int32_t toys,
                    const double* params_matrix, int nthreads, double* out) {
  int rc = validate(m);
  if (rc) return rc;
  if (toys < 0 || (toys > 0 && (!offsets || !params_matrix || !out)))
    return ORC_EINVAL;
  for (int32_t t = 0; t < toys; ++t)
    if (offsets[t + 1] < offsets[t]) return ORC_EINVAL;
  int P = m->n_par;
  int worst = ORC_OK;
  /* toys are independent: one toy per thread, each summed in event order */
#ifdef _OPENMP
  int nt = nthreads > 0 ? nthreads : omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(nt)
#endif
  for (int32_t t = 0; t < toys; ++t) {
    int64_t b = offsets[t], e = offsets[t + 1];
    int r = orc_nll(m, params_matrix + (int64_t)t * P, cols + b, col_stride,
                    e - b, 1, out + (int64_t)t * (1 + P),
                    out + (int64_t)t * (1 + P) + 1);
    if (r) {
#ifdef _OPENMP
#pragma omp critical
#endif
      if (r > worst) worst = r;
    }
  }
  return worst;
}

void orc_adam_step(int n_par, double* theta, const double* grad,
                   const double* scale, const uint8_t* free_mask, double* m1,
                   double* m2, int t, double lr, double beta1, double beta2,
                   double eps) {
  for (int j = 0; j < n_par; ++j) {
    if (!free_mask[j]) continue;
    double g = grad[j] * scale[j]; /* gradient in units of scale */
    m1[j] = beta1 * m1[j] + (1.0 - beta1) * g;
    m2[j] = beta2 * m2[j] + (1.0 - beta2) * g * g;
    double mh = m1[j] / (1.0 - pow(beta1, t));
    double vh = m2[j] / (1.0 - pow(beta2, t));
    theta[j] -= scale[j] * lr * mh / (sqrt(vh) + eps);
  }
}

/* ------------------------------------------------------------------ */
/* toy generation                                                      */
/* ------------------------------------------------------------------ */

/* Philox4x64-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as
 * easy as 1, 2, 3", SC'11): ten rounds of two 64x64->128 multiplications,
 * the key bumped by the Weyl constants between rounds. */
static void mulhilo64(uint64_t a, uint64_t b, uint64_t* hi, uint64_t* lo) {
  unsigned __int128 p = (unsigned __int128)a * (unsigned __int128)b;
  *hi = (uint64_t)(p >> 64);
  *lo = (uint64_t)p;
}

void orc_philox4x64(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4]) {
  const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
  const uint64_t W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
  uint64_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3], k0 = key[0], k1 = key[1];
  for (int r = 0; r < 10; ++r) {
    uint64_t hi0, lo0, hi1, lo1;
    mulhilo64(M0, c0, &hi0, &lo0);
    mulhilo64(M1, c2, &hi1, &lo1);
    uint64_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
    if (r < 9) {
      k0 += W0;
      k1 += W1;
    }
  }
  out[0] = c0;
  out[1] = c1;
  out[2] = c2;
  out[3] = c3;
}

/* inverse of erfc on (0, 2): Newton's method on erfc from a rough start,
 * to convergence in FP64 */
double orc_erfcinv(double q) {
  if (!(q > 0.0 && q < 2.0)) return q == 0.0 ? INFINITY : (q == 2.0 ? -INFINITY : NAN);
  if (q >= 0.5 && q <= 1.5) {
    /* erf(z) = 1 - q, exact here (Sterbenz): Newton on erf keeps the small
     * root's relative accuracy */
    double e = 1.0 - q, z = 0.8862269254527580 * e;
    for (int it = 0; it < 100; ++it) {
      double f = erf(z) - e;
      double dz = f / (1.1283791670955126 * exp(-z * z));
      dz = dz / (1.0 - z * dz);
      z -= dz;
      if (fabs(dz) <= 1e-17 * fabs(z) + 1e-300) break;
    }
    return z;
  }
  if (q > 1.0) return -orc_erfcinv(2.0 - q);
  /* start: erfc(z) ~ exp(-z^2) / (z sqrt(pi)) for large z; z = 0.5 * (1-q) near 1 */
  double z = q > 0.3 ? 0.8862269254527580 * (1.0 - q)
                     : sqrt(-log(q)) - 0.25 * log(-log(q) * 3.141592653589793) / sqrt(-log(q));
  for (int it = 0; it < 100; ++it) {
    double f = erfc(z) - q;
    double fp = -1.1283791670955126 * exp(-z * z); /* d erfc/dz = -2/sqrt(pi) e^{-z^2} */
    double dz = f / fp;
    /* Halley's correction: f'' / f' = -2 z */
    dz = dz / (1.0 + z * dz);
    z -= dz;
    if (fabs(dz) <= 1e-17 * fabs(z) + 1e-300) break;
  }
  return z;
}

/* z with Phi(z) = Phi(za) + u (Phi(zb) - Phi(za)), Phi the standard normal
 * CDF; the lower- or upper-tail form is used whichever is small */
static double tn_inv(double u, double za, double zb) {
  const double r2 = 1.4142135623730951;
  double Pa = 0.5 * erfc(-za / r2), Pb = 0.5 * erfc(-zb / r2);
  double P = Pa + u * (Pb - Pa);
  if (P <= 0.5) return -r2 * orc_erfcinv(2.0 * P);
  double Qa = 0.5 * erfc(za / r2), Qb = 0.5 * erfc(zb / r2);
  double Q = Qb + (1.0 - u) * (Qa - Qb);
  return r2 * orc_erfcinv(2.0 * Q);
}

/* One candidate value of a leaf from the four uniforms of one attempt;
 * *accept = 0 asks for another attempt (accept-reject). */
static double sample_leaf(int type, const double* th, int nth, double a, double b,
                          const double* u, int* accept) {
  *accept = 1;
  switch (type) {
    case ORC_GAUSS: {
      double mu = th[0], sg = th[1];
      return mu + sg * tn_inv(u[0], (a - mu) / sg, (b - mu) / sg);
    }
    case ORC_EXP: {
      double lam = th[0], L = b - a;
      if (lam == 0.0) return a + u[0] * L;
      /* CDF expm1(lam (x - a)) / expm1(lam L), inverted from the end whose
       * exponential does not overflow */
      if (lam < 0.0) return a + log1p(u[0] * expm1(lam * L)) / lam;
      /* 1 - F(x) = expm1(lam (x - b)) / expm1(-lam L) */
      return b + log1p((1.0 - u[0]) * expm1(-lam * L)) / lam;
    }
    case ORC_CHEB: {
      /* uniform proposal on [-1, 1]; f = 1 + sum c_j T_j <= 1 + sum |c_j| */
      double xp = -1.0 + 2.0 * u[0], fmax = 1.0, f = 1.0, tm = 1.0, t = xp;
      for (int j = 0; j < nth; ++j) {
        fmax += fabs(th[j]);
        f += th[j] * t;
        double tn = 2.0 * xp * t - tm;
        tm = t;
        t = tn;
      }
      *accept = u[1] * fmax <= f;
      return a + 0.5 * (xp + 1.0) * (b - a);
    }
    case ORC_CB: {
      double m0 = th[0], sg = th[1], al = th[2], n = th[3];
      double s = al > 0.0 ? 1.0 : -1.0, A = fabs(al);
      double tlo = s > 0.0 ? (a - m0) / sg : (m0 - b) / sg;
      double thi = s > 0.0 ? (b - m0) / sg : (m0 - a) / sg;
      double tc = tlo > -A ? tlo : -A;
      double core = thi > -A ? 1.2533141373155003 * erf_diff(tc / 1.4142135623730951,
                                                              thi / 1.4142135623730951)
                             : 0.0;
      double tail = 0.0, pre = (n / A) * exp(-0.5 * A * A), D1 = 1.0, G1 = 0.0;
      double t2 = thi < -A ? thi : -A;
      if (tlo < -A) {
        /* D = 1 - (A/n)(A + t); tail mass from tlo to t = pre (G(D(tlo)) - G(D(t))),
         * G(D) = D^(1-n)/(1-n), log D at n = 1 */
        D1 = 1.0 - (A / n) * (A + tlo);
        double D2 = 1.0 - (A / n) * (A + t2);
        G1 = n == 1.0 ? log(D1) : pow(D1, 1.0 - n) / (1.0 - n);
        double G2 = n == 1.0 ? log(D2) : pow(D2, 1.0 - n) / (1.0 - n);
        tail = pre * (G1 - G2);
      }
      double T = u[0] * (core + tail), t;
      if (T < tail) {
        double G = G1 - T / pre;
        double Dt = n == 1.0 ? exp(G) : pow((1.0 - n) * G, 1.0 / (1.0 - n));
        t = (n / A) * (1.0 - Dt) - A;
      } else {
        double v = core > 0.0 ? (T - tail) / core : 0.0;
        t = tn_inv(v, tc, thi);
      }
      return s > 0.0 ? m0 + sg * t : m0 - sg * t;
    }
    case ORC_JOHNSON: {
      /* w = gamma + delta asinh z is standard normal on [w(a), w(b)] */
      double mu = th[0], lam = th[1], gam = th[2], del = th[3];
      double wa = gam + del * asinh((a - mu) / lam), wb = gam + del * asinh((b - mu) / lam);
      double w = tn_inv(u[0], wa, wb);
      return mu + lam * sinh((w - gam) / del);
    }
    case ORC_ARGUS: {
      /* m dm ~ sqrt(tau) e^{c tau} d tau with tau = 1 - (m/m0)^2 */
      double m0 = th[0], c = th[1];
      double bb = b < m0 ? b : m0;
      double ta = 1.0 - (a / m0) * (a / m0), tb = 1.0 - (bb / m0) * (bb / m0), tau;
      if (c < 0.0) {
        /* Gamma(3/2, rate -c) = (E + Z^2/2) / (-c): E exponential, Z normal
         * (Box-Muller), truncated to [tb, ta] by rejection */
        double E = -log(u[0]);
        double Z = sqrt(-2.0 * log(u[1])) * cos(6.283185307179586 * u[2]);
        tau = (E + 0.5 * Z * Z) / (-c);
        *accept = tau >= tb && tau <= ta;
      } else {
        tau = tb + u[0] * (ta - tb);
        double gmax = sqrt(ta) * exp(c * ta);
        *accept = u[1] * gmax <= sqrt(tau) * exp(c * tau);
      }
      return m0 * sqrt(1.0 - tau);
    }
  }
  *accept = 1;
  return NAN;
}

/* leaves (node indices) of component node i: the leaf itself or a Prod's */
static int comp_leaves(const orc_model* m, int i, int* out) {
  if (is_leaf(m->type[i])) {
    out[0] = i;
    return 1;
  }
  if (m->type[i] != ORC_PROD) return -1;
  int k = 0;
  for (int j = 0; j < m->nchild[i]; ++j) {
    int ch = m->child[i * ORC_MAXCH + j];
    if (!is_leaf(m->type[ch])) return -1;
    out[k++] = ch;
  }
  return k;
}

int orc_generate(const orc_model* m, const double* params_matrix, int32_t toys,
                 const int64_t* comp_counts, const int64_t* offsets, uint64_t seed,
                 int col_f32, double* cols, int64_t col_stride, int64_t* exhausted) {
  int rc = validate(m);
  if (rc) return rc;
  int comps[ORC_MAXCH], nc = 0;
  int rt = m->type[m->root];
  if (rt == ORC_ADD_FRAC || rt == ORC_ADD_EXT) {
    nc = m->nchild[m->root];
    for (int c = 0; c < nc; ++c) comps[c] = m->child[m->root * ORC_MAXCH + c];
  } else {
    nc = 1;
    comps[0] = m->root;
  }
  int lv[ORC_MAXCH][ORC_MAXCH], nlv[ORC_MAXCH];
  for (int c = 0; c < nc; ++c) {
    nlv[c] = comp_leaves(m, comps[c], lv[c]);
    if (nlv[c] < 0) return ORC_EUNSUPPORTED;
    for (int k = 0; k < nlv[c]; ++k)
      if (m->type[lv[c][k]] == ORC_EXPR || m->type[lv[c][k]] == ORC_HYPATIA2)
        return ORC_EUNSUPPORTED; /* no sampler */
    int64_t cover = 0;
    for (int k = 0; k < nlv[c]; ++k) cover |= (int64_t)1 << m->obs[lv[c][k]];
    if (cover != ((int64_t)1 << m->n_obs) - 1) return ORC_EUNSUPPORTED;
  }
  const uint64_t key[2] = {seed, 0x52462D544F595321ULL};
  *exhausted = 0;
  for (int32_t t = 0; t < toys; ++t) {
    const double* p = params_matrix + (int64_t)t * m->n_par;
    int64_t i = offsets[t];
    for (int c = 0; c < nc; ++c) {
      for (int64_t e = 0; e < comp_counts[(int64_t)t * nc + c]; ++e, ++i) {
        for (int k = 0; k < nlv[c]; ++k) {
          int node = lv[c][k], o = m->obs[node];
          double th[ORC_MAXNP];
          for (int j = 0; j < m->npar[node]; ++j) th[j] = p[m->par[node * ORC_MAXNP + j]];
          if (m->type[node] == ORC_ARGUS && th[2] != 0.5) return ORC_EUNSUPPORTED;
          double lo = m->obs_lo[o], hi = m->obs_hi[o], x = NAN;
          int ok = 0;
          for (uint64_t r = 0; r < 4096 && !ok; ++r) {
            uint64_t ctr[4] = {(uint64_t)i, (uint64_t)o, r, 0}, w[4];
            double u[4];
            orc_philox4x64(ctr, key, w);
            for (int q = 0; q < 4; ++q) u[q] = ((double)(w[q] >> 11) + 0.5) * 0x1p-53;
            x = sample_leaf(m->type[node], th, m->npar[node], lo, hi, u, &ok);
            if (col_f32) x = (double)(float)x;
            /* the stored value must lie in the range (ARGUS: below m0) */
            if (ok && !(x >= lo && x <= hi)) ok = 0;
            if (ok && m->type[node] == ORC_ARGUS && !(x < th[0])) ok = 0;
          }
          if (!ok) ++*exhausted;
          cols[(int64_t)o * col_stride + i] = x;
        }
      }
    }
  }
  return ORC_OK;
}
