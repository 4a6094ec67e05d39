// expr.cpp -- formula leaves: a PDF given as text (the formula PDFs of Sec. 4,
// RooGenericPdf, which the paper compiles just in time with cling).
//
// rf_expr_translate parses the text and writes it back as a CUDA expression
// over the library's dual numbers (rf_expr.cuh), which the graph's NVRTC
// compile then inlines into the fused, log P and normalisation kernels: the
// per-event code of a formula is as specialised as a built-in leaf's.
//
// Grammar (the whole language):
//   sum   := prod (('+' | '-') prod)*
//   prod  := unary (('*' | '/') unary)*
//   unary := ('-' | '+') unary | power
//   power := atom ('^' unary)?        right-associative; -a^2 = -(a^2)
//   atom  := number | 'x' | 'p'<digits> | func '(' sum ')' | 'pow' '(' sum ',' sum ')'
//            | '(' sum ')'
//   number: digits ['.' digits] [('e' | 'E') ['+' | '-'] digits]  (or starting with '.')
//   func:   exp log sqrt sin cos tanh sinh cosh asinh atan erf erfc abs
// x is the leaf's observable, p<j> its j-th parameter (j < the leaf's count).
// An exponent that is an integer literal (|n| <= 64, optionally negated) is a
// repeated product, defined for negative bases; any other a^b is exp(b log a).
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>

#include "rf_internal.h"

namespace {

struct Node {
  std::string code;  // CUDA text
  int lit = 0;       // 1: a number literal, 2: a negated number literal
  bool is_int = false;
  long ival = 0;     // value when is_int (an integral literal, possibly negated once)
};

struct Parser {
  const char* s;
  size_t pos = 0;
  int npar;
  int depth = 0;
  std::string err;

  bool fail(const std::string& what) {
    if (err.empty()) err = what + " at offset " + std::to_string(pos);
    return false;
  }
  void skip() {
    while (s[pos] == ' ' || s[pos] == '\t' || s[pos] == '\n' || s[pos] == '\r') ++pos;
  }
  static bool digit(char c) { return c >= '0' && c <= '9'; }
  static bool alpha(char c) { return (c >= 'a' && c <= 'z') || (c >= 'A' && c <= 'Z') || c == '_'; }

  static std::string literal(double v) {
    char buf[64];
    snprintf(buf, sizeof(buf), "%a", v);  // exact
    return std::string("Real(") + buf + ")";
  }

  static std::string power(const Node& a, const Node& e) {
    if (e.is_int && e.ival >= -64 && e.ival <= 64)
      return "rf::fx::powi<" + std::to_string(e.ival) + ">(" + a.code + ")";
    return "rf::fx::pow(" + a.code + ", " + e.code + ")";
  }

  bool number(Node* out) {
    const size_t b = pos;
    while (digit(s[pos])) ++pos;
    if (s[pos] == '.') {
      ++pos;
      while (digit(s[pos])) ++pos;
    }
    if (s[pos] == 'e' || s[pos] == 'E') {
      ++pos;
      if (s[pos] == '+' || s[pos] == '-') ++pos;
      if (!digit(s[pos])) return fail("exponent without digits");
      while (digit(s[pos])) ++pos;
    }
    const std::string text(s + b, pos - b);
    const double v = std::strtod(text.c_str(), nullptr);
    out->code = literal(v);
    // an integral exponent is judged by the literal's value (2, 2.0, 1e1)
    out->lit = 1;
    out->is_int = v == std::floor(v) && std::fabs(v) <= 64.0;
    out->ival = out->is_int ? (long)v : 0;
    return true;
  }

  bool atom(Node* out) {
    skip();
    const char c = s[pos];
    if (digit(c) || (c == '.' && digit(s[pos + 1]))) return number(out);
    if (alpha(c)) {
      const size_t b = pos;
      while (alpha(s[pos]) || digit(s[pos])) ++pos;
      const std::string name(s + b, pos - b);
      if (name == "x") {
        out->code = "x";
        return true;
      }
      if (name.size() >= 2 && name[0] == 'p' &&
          name.find_first_not_of("0123456789", 1) == std::string::npos && name.size() <= 12) {
        const long j = std::strtol(name.c_str() + 1, nullptr, 10);
        if (j >= npar) return fail("parameter " + name + " beyond the leaf's " + std::to_string(npar));
        out->code = "p" + std::to_string(j);  // p01 is p1
        return true;
      }
      static const char* const kFuncs[] = {"exp",   "log",  "sqrt", "sin", "cos",  "tanh", "sinh",
                                           "cosh",  "asinh", "atan", "erf", "erfc", "abs"};
      bool known = name == "pow";
      for (const char* f : kFuncs) known = known || name == f;
      if (!known) return fail("unknown name '" + name + "'");
      skip();
      if (s[pos] != '(') return fail("'(' expected after " + name);
      ++pos;
      Node a;
      if (!sum(&a)) return false;
      skip();
      if (name == "pow") {
        if (s[pos] != ',') return fail("pow needs two arguments");
        ++pos;
        Node e;
        if (!sum(&e)) return false;
        skip();
        out->code = power(a, e);
      } else {
        out->code = "rf::fx::" + name + "(" + a.code + ")";
      }
      if (s[pos] != ')') return fail("')' expected");
      ++pos;
      return true;
    }
    if (c == '(') {
      ++pos;
      Node a;
      if (!sum(&a)) return false;
      skip();
      if (s[pos] != ')') return fail("')' expected");
      ++pos;
      out->code = "(" + a.code + ")";
      out->lit = a.lit;
      out->is_int = a.is_int;
      out->ival = a.ival;
      return true;
    }
    return fail(c ? "unexpected character" : "unexpected end");
  }

  bool pow_level(Node* out) {
    Node a;
    if (!atom(&a)) return false;
    skip();
    if (s[pos] != '^') {
      *out = a;
      return true;
    }
    ++pos;
    Node e;
    if (!unary(&e)) return false;
    out->code = "(" + power(a, e) + ")";
    out->lit = 0;
    out->is_int = false;
    return true;
  }

  bool unary(Node* out) {
    if (++depth > 200) return fail("nesting too deep");
    skip();
    bool ok;
    if (s[pos] == '-') {
      ++pos;
      Node a;
      ok = unary(&a);
      if (ok) {
        out->code = "(-" + a.code + ")";
        out->lit = a.lit == 1 ? 2 : 0;  // only a literal negated once stays one
        out->is_int = a.lit == 1 && a.is_int;
        out->ival = -a.ival;
      }
    } else if (s[pos] == '+') {
      ++pos;
      ok = unary(out);
    } else {
      ok = pow_level(out);
    }
    --depth;
    return ok;
  }

  bool prod(Node* out) {
    Node a;
    if (!unary(&a)) return false;
    for (;;) {
      skip();
      const char c = s[pos];
      if (c != '*' && c != '/') break;
      ++pos;
      Node b;
      if (!unary(&b)) return false;
      a.code = "(" + a.code + (c == '*' ? " * " : " / ") + b.code + ")";
      a.lit = 0;
      a.is_int = false;
    }
    *out = a;
    return true;
  }

  bool sum(Node* out) {
    if (++depth > 200) return fail("nesting too deep");
    Node a;
    if (!prod(&a)) return false;
    for (;;) {
      skip();
      const char c = s[pos];
      if (c != '+' && c != '-') break;
      ++pos;
      Node b;
      if (!prod(&b)) return false;
      a.code = "(" + a.code + (c == '+' ? " + " : " - ") + b.code + ")";
      a.lit = 0;
      a.is_int = false;
    }
    --depth;
    *out = a;
    return true;
  }
};

}  // namespace

bool rf_expr_translate(const char* text, int npar, std::string* code, std::string* err) {
  if (!text) {
    *err = "formula text is NULL";
    return false;
  }
  if (npar < 0 || npar > RF_LEAF_MAXP) {
    *err = "a formula leaf takes at most 4 parameters";
    return false;
  }
  if (std::strlen(text) > 4096) {
    *err = "formula longer than 4096 characters";
    return false;
  }
  Parser p{text, 0, npar};
  Node n;
  bool ok = p.sum(&n);
  if (ok) {
    p.skip();
    if (text[p.pos] != 0) ok = p.fail("unexpected text");
  }
  if (!ok) {
    *err = "formula '" + std::string(text) + "': " + p.err;
    return false;
  }
  *code = n.code;
  return true;
}

// 16-point Gauss-Legendre nodes and weights on [-1, 1]: Newton's method on
// P_16 from cosine first guesses, P_16 and its derivative by the three-term
// recurrence.
void rf_gauss_legendre16(double* t, double* w) {
  const int n = 16;
  for (int i = 0; i < n; ++i) {
    double z = std::cos(3.14159265358979323846 * (i + 0.75) / (n + 0.5)), dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double a = 1.0, b = z;
      for (int k = 2; k <= n; ++k) {
        const double c = ((2.0 * k - 1.0) * z * b - (k - 1.0) * a) / k;
        a = b;
        b = c;
      }
      dp = n * (z * b - a) / (z * z - 1.0);
      const double dz = b / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-17) break;
    }
    t[i] = z;
    w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}
