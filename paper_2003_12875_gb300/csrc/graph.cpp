// graph.cpp -- host side of librfgpu: descriptor validation, the graph
// compiler (canonical sum-of-products program, accumulator slots, hoisted
// parameter-only work), workspace ownership, autotuning and every C-ABI entry
// point of include/rf.h.
//
// Paper correspondence: the compiled program is the computation graph of
// Sec. 5.1 with its parameter-only branches (normalisations, coefficients)
// evaluated once per call instead of once per entry; rf_nll is the fused
// replacement of the per-entry walk; rf_nll_plain keeps the node-per-call
// batch interface of Sec. 5.2 as the baseline; the range checks follow
// Sec. 3 ("Checking parameters").
#include <cuda_runtime.h>
#include <sys/stat.h>
#include <unistd.h>

#include <algorithm>
#include <atomic>
#include <cstdlib>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/rf.h"
#include "rf_internal.h"

namespace {

thread_local std::string g_err;

rf_status fail(rf_status s, const std::string& msg) {
  g_err = msg;
  return s;
}

rf_status cuda_fail(cudaError_t e, const char* where) {
  g_err = std::string(where) + ": " + cudaGetErrorString(e);
  return RF_ECUDA;
}

bool is_leaf(int t) {
  return (t >= RF_GAUSS && t <= RF_ARGUS) || t == RF_JOHNSON || t == RF_FORMULA ||
         t == RF_HYPATIA2;
}

// leaf slots a leaf takes in the compiled program (four parameters a slot)
int leaf_slots(int t) { return t == RF_HYPATIA2 ? 3 : 1; }

int leaf_nparams_ok(int t, int np) {
  switch (t) {
    case RF_GAUSS: return np == 2;
    case RF_EXP: return np == 1;
    case RF_CHEB: return np >= 1 && np <= RF_LEAF_MAXP;
    case RF_CB: return np == 4;
    case RF_ARGUS: return np == 3;
    case RF_JOHNSON: return np == 4;
    case RF_FORMULA: return np >= 0 && np <= RF_LEAF_MAXP;
    case RF_HYPATIA2: return np == 9;
  }
  return 0;
}

// Structural validation shared by rf_graph_validate and rf_graph_compile.
rf_status validate_desc(const rf_graph_desc* d) {
  if (!d) return fail(RF_EINVAL, "descriptor is NULL");
  if (d->n_nodes <= 0 || d->n_nodes > RF_MAX_NODES || !d->nodes)
    return fail(RF_EINVAL, "n_nodes must be in 1..32 and nodes non-NULL");
  if (d->root < 0 || d->root >= d->n_nodes) return fail(RF_EINVAL, "root out of range");
  if (d->n_obs <= 0 || d->n_obs > 62 || !d->obs_lo || !d->obs_hi)
    return fail(RF_EINVAL, "n_obs must be in 1..62 with ranges given");
  if (d->n_params < 0 || d->n_params > RF_MAX_PARAMS)
    return fail(RF_EINVAL, "n_params must be in 0..64");
  if (d->column_dtype != RF_F32 && d->column_dtype != RF_F64)
    return fail(RF_EINVAL, "column_dtype must be RF_F32 or RF_F64");
  if (d->eval_precision != RF_EVAL_FP32 && d->eval_precision != RF_EVAL_FP64)
    return fail(RF_EINVAL, "eval_precision must be RF_EVAL_FP32 or RF_EVAL_FP64");
  for (int o = 0; o < d->n_obs; ++o)
    if (!(d->obs_hi[o] > d->obs_lo[o]) || !std::isfinite(d->obs_lo[o]) ||
        !std::isfinite(d->obs_hi[o]))
      return fail(RF_EINVAL, "observable " + std::to_string(o) + " has an empty or non-finite range");
  for (int i = 0; i < d->n_nodes; ++i) {
    const rf_node_desc& n = d->nodes[i];
    if (n.type < RF_GAUSS || n.type > RF_HYPATIA2)
      return fail(RF_EINVAL, "node " + std::to_string(i) + ": unknown type");
    if (n.n_params < 0 || n.n_params > RF_MAX_NODE_PARAMS)
      return fail(RF_EINVAL, "node " + std::to_string(i) + ": bad n_params");
    for (int j = 0; j < n.n_params; ++j)
      if (n.params[j] < 0 || n.params[j] >= d->n_params)
        return fail(RF_EINVAL, "node " + std::to_string(i) + ": parameter index out of range");
    if (is_leaf(n.type)) {
      if (n.obs < 0 || n.obs >= d->n_obs)
        return fail(RF_EINVAL, "node " + std::to_string(i) + ": observable index out of range");
      if (n.type == RF_CHEB && n.n_params > RF_LEAF_MAXP)
        return fail(RF_EUNSUPPORTED, "Chebychev order above 4 is not supported on the GPU");
      if (!leaf_nparams_ok(n.type, n.n_params))
        return fail(RF_EINVAL, "node " + std::to_string(i) + ": wrong parameter count for its type");
      if (n.type == RF_FORMULA) {
        std::string code, err;
        if (!rf_expr_translate(n.formula, n.n_params, &code, &err))
          return fail(RF_EINVAL, "node " + std::to_string(i) + ": " + err);
      }
    } else {
      if (n.n_children < 1 || n.n_children > RF_MAX_CHILDREN)
        return fail(RF_EINVAL, "node " + std::to_string(i) + ": bad n_children");
      for (int k = 0; k < n.n_children; ++k)
        if (n.children[k] < 0 || n.children[k] >= d->n_nodes || n.children[k] == i)
          return fail(RF_EINVAL, "node " + std::to_string(i) + ": child index out of range");
      if (n.type == RF_ADD_FRAC && (n.n_children < 2 || n.n_params != n.n_children - 1))
        return fail(RF_EINVAL, "node " + std::to_string(i) + ": ADD_FRAC needs K>=2 children and K-1 fractions");
      if (n.type == RF_ADD_EXT && n.n_params != n.n_children)
        return fail(RF_EINVAL, "node " + std::to_string(i) + ": ADD_EXT needs one yield per child");
      if (n.type == RF_ADD_EXT && i != d->root)
        return fail(RF_EUNSUPPORTED, "ADD_EXT is only supported at the root");
      if (n.type == RF_PROD && n.n_params != 0)
        return fail(RF_EINVAL, "node " + std::to_string(i) + ": PROD takes no parameters");
    }
  }
  return RF_OK;
}

struct Canon {
  RfProgram prog;
};

// Map the descriptor onto the sum-of-products program (fixed-size arrays
// only: no heap allocation on the success path).
rf_status canonicalise(const rf_graph_desc* d, RfProgram* P, int* leaf_node = nullptr) {
  std::memset(P, 0, sizeof(*P));
  P->ext_weight = 1.0;
  const rf_node_desc& root = d->nodes[d->root];
  int comp_leaf[RF_MAX_CHILDREN][RF_MAX_CHILDREN];  // leaf node ids per component
  int comp_n[RF_MAX_CHILDREN] = {0};
  int n_comps = 0;
  auto leaves_of = [&](int id, int c) -> rf_status {
    const rf_node_desc& n = d->nodes[id];
    if (is_leaf(n.type)) {
      comp_leaf[c][comp_n[c]++] = id;
      return RF_OK;
    }
    if (n.type == RF_PROD) {
      for (int k = 0; k < n.n_children; ++k) {
        const rf_node_desc& ch = d->nodes[n.children[k]];
        if (!is_leaf(ch.type))
          return fail(RF_EUNSUPPORTED, "a PROD child must be a leaf on the GPU path");
        comp_leaf[c][comp_n[c]++] = n.children[k];
      }
      return RF_OK;
    }
    return fail(RF_EUNSUPPORTED, "an ADD child must be a leaf or a PROD of leaves");
  };
  int kind = RF_KIND_PROD;
  if (is_leaf(root.type) || root.type == RF_PROD) {
    rf_status s = leaves_of(d->root, n_comps++);
    if (s) return s;
  } else {
    kind = root.type == RF_ADD_FRAC ? RF_KIND_FRAC : RF_KIND_EXT;
    for (int k = 0; k < root.n_children; ++k) {
      rf_status s = leaves_of(root.children[k], n_comps++);
      if (s) return s;
    }
    if (n_comps <= RF_MAXC)
      for (int j = 0; j < root.n_params; ++j) P->coef_par[j] = root.params[j];
  }
  int nl = 0;
  for (int c = 0; c < n_comps; ++c)
    for (int li = 0; li < comp_n[c]; ++li) nl += leaf_slots(d->nodes[comp_leaf[c][li]].type);
  if (n_comps > RF_MAXC) return fail(RF_EUNSUPPORTED, "more than 6 components");
  if (nl > RF_MAXL) return fail(RF_EUNSUPPORTED, "more than 6 leaves");
  P->n_leaves = nl;
  P->n_comp = n_comps;
  P->kind = kind;
  P->n_par = d->n_params;
  auto fixed = [&](int p) { return d->param_fixed && d->param_fixed[p]; };
  for (int p = 0; p < d->n_params; ++p)
    if (fixed(p)) {
      if (p < 64) P->fixed_lo |= 1ull << p;
      else P->fixed_hi |= 1ull << (p - 64);
    }
  if (kind != RF_KIND_PROD) {
    int ncoef = kind == RF_KIND_FRAC ? P->n_comp - 1 : P->n_comp;
    for (int c = 0; c < ncoef; ++c)
      if (!fixed(P->coef_par[c])) P->coef_free |= 1 << c;
  }
  int n_cols = 0;
  int k = 0;
  for (int c = 0; c < P->n_comp; ++c) {
    uint64_t comp_obs = 0;
    for (int li = 0; li < comp_n[c]; ++li) {
      const rf_node_desc& n = d->nodes[comp_leaf[c][li]];
      if (comp_n[c] > 1) {
        if (comp_obs & (1ull << n.obs))
          return fail(RF_EUNSUPPORTED, "PROD children must use disjoint observables");
        comp_obs |= 1ull << n.obs;
      }
      if (leaf_node) leaf_node[k] = comp_leaf[c][li];
      RfLeafProg& L = P->leaf[k++];
      L.type = n.type;  // RF_<leaf> == RFL_<leaf>
      L.comp = c;
      L.npar = n.n_params;
      for (int j = 0; j < RF_LEAF_MAXP; ++j) L.par[j] = j < n.n_params ? n.params[j] : 0;
      L.lo = d->obs_lo[n.obs];
      L.hi = d->obs_hi[n.obs];
      int slot = -1;
      for (int s = 0; s < n_cols; ++s)
        if (P->col_obs[s] == n.obs) slot = s;
      if (slot < 0) {
        slot = n_cols;
        P->col_obs[n_cols++] = n.obs;
      }
      L.col = slot;
      int gm = 0;
      for (int j = 0; j < n.n_params && j < RF_LEAF_MAXP; ++j)
        if (!fixed(n.params[j])) gm |= 1 << j;
      // ARGUS: a free p selects the general-p form (d/dp included); so does
      // a fixed p whose compile-time value is not 1/2 (without d/dp);
      // otherwise a fixed p must be 1/2 at run time (checked in the prologue)
      if (n.type == RF_ARGUS && !(gm & 4) && d->param_values &&
          d->param_values[n.params[2]] != 0.5)
        gm |= RF_ARGUS_GENERAL;
      L.gmask = gm;
      if (n.type == RF_HYPATIA2) {
        L.npar = RF_LEAF_MAXP;
        // its parameters 4.. in the next slots: same component and column,
        // no per-event work of their own
        for (int part = 1; part < leaf_slots(n.type); ++part) {
          if (leaf_node) leaf_node[k] = comp_leaf[c][li];
          RfLeafProg& X = P->leaf[k++];
          X = L;
          X.type = RFL_PARAMS;
          X.part = part;
          X.npar = 0;
          X.gmask = 0;
          for (int j = 0; j < RF_LEAF_MAXP; ++j) {
            const int q = RF_LEAF_MAXP * part + j;
            X.par[j] = q < n.n_params ? n.params[q] : 0;
            if (q < n.n_params) {
              X.npar = j + 1;
              if (!fixed(n.params[q])) X.gmask |= 1 << j;
            }
          }
        }
      }
    }
  }
  P->n_cols = n_cols;
  return RF_OK;
}

// events per thread: FP32 evaluation 4 or 8, and 16 in the specialised
// kernels (the generic ones are not instantiated for it); FP64 2 or 4
bool ept_ok(int eval, int coldt, int ept, bool jit) {
  if (eval == RF_EVAL_FP32) return ept == 4 || ept == 8 || (jit && ept == 16);
  if (coldt == RF_F64) return ept == 2 || ept == 4;
  return ept == 4;
}

}  // namespace

struct rf_graph {
  RfProgram prog;
  int eval = 0, coldt = 0, n_obs = 0;
  int device = 0, num_sms = 0;
  RfLaunchCfg cfg{256, 4, 2, 3};
  RfWork work{};
  int64_t max_rows_single = 0;
  // batched
  const void* bound_events = nullptr;
  bool bound = false;
  // FP32 evaluation of FP64 columns: the toy columns rounded to FP32 once at
  // bind time (what every per-event conversion would give)
  float* bound32 = nullptr;
  size_t bound32_elems = 0;
  // toy segment kernel form, fixed at compile: register streaming, or
  // bulk-copy stage rings when RF_TOY_STREAM=bulk
  bool toy_bulk = false;
  int64_t bound_n = 0;
  int32_t max_toys = 0;
  int64_t max_toy_rows = 0;  // segment rows: launch warps + toys
  // host staging
  void* stage = nullptr;
  size_t stage_bytes = 0;
  // plain workspace
  double* plain_buf = nullptr;
  size_t plain_bytes = 0;
  double* plain_partials = nullptr;
  unsigned int* plain_counter = nullptr;
  cudaStream_t fit_stream = nullptr;
  void* pro_buf = nullptr;
  int last_launches = 0;
  // per-graph specialised kernels (NVRTC), by events per thread (index 0 or
  // 1 of the precision's two options) and, for the fused kernel, register
  // budget (min_blocks 2..4); compiled on first need
  bool jit = false;
  cudaKernel_t jk_fused[3][3] = {};
  cudaKernel_t jk_toys[3] = {nullptr, nullptr, nullptr};
  cudaKernel_t jk_logp = nullptr;
  // formula leaves: translated code, the normalisation kernel and its
  // workspace (log I and derivatives, block partials, tickets)
  int n_formula = 0;
  RfFormulaCode fcode;
  cudaKernel_t jk_norm = nullptr;
  double* formula_buf = nullptr;
  unsigned int* formula_ticket = nullptr;
  int jk_regs[3][3] = {};
};

// index of an events-per-thread option within its precision's set
static int ept_index(int eval, int coldt, int ept) {
  if (eval == RF_EVAL_FP32) return ept == 16 ? 2 : (ept == 8 ? 1 : 0);
  if (coldt == RF_F64) return ept == 4 ? 1 : 0;
  return 0;
}

static bool min_blocks_ok(int mb) { return mb >= 2 && mb <= 4; }

static const RfFormulaCode* fcode(const rf_graph* g) {
  return g->n_formula ? &g->fcode : nullptr;
}

static cudaKernel_t jit_fused(rf_graph* g, int ept, int min_blocks, std::string* err) {
  const int i = ept_index(g->eval, g->coldt, ept), m = min_blocks - 2;
  if (!g->jk_fused[i][m])
    g->jk_fused[i][m] = rf_jit_kernel(g->prog, fcode(g), g->eval, g->coldt, RF_JIT_FUSED, ept,
                                      min_blocks, &g->jk_regs[i][m], err);
  return g->jk_fused[i][m];
}

// column type the toy kernels read: FP32-evaluated graphs read FP32 columns
// (FP64 ones are converted at bind time)
static int toy_coldt(const rf_graph* g) { return g->eval == RF_EVAL_FP32 ? RF_F32 : g->coldt; }
// events per lane per chunk of the segment kernel (its per-chunk bookkeeping
// and compensated sums are spread over that many events)
static int toy_ept(const rf_graph* g) {
  if (const char* v = getenv("RF_TOY_EPT")) {  // tuning: 8 or 16 (FP32), 4 or 8 (FP64)
    const int e = atoi(v);
    if (g->eval == RF_EVAL_FP32 ? (e == 8 || e == 16) : (e == 4 || e == 8)) return e;
  }
  // measured on the 4096 Gauss + Exponential toys (1.3e8 events): FP32, 8
  // (0.174 ms a step) beats 16 (0.194 ms) since the per-event code shrank;
  // FP64, 8 beats 4
  return 8;
}
// register budget of the segment kernel: 0 = the compiler's choice, else
// launch bounds for 3 or 4 resident blocks of 256 threads (tuning)
static int toy_min_blocks() {
  if (const char* v = getenv("RF_TOY_MINBLOCKS")) {
    const int m = atoi(v);
    if (m == 3 || m == 4) return m;
  }
  return 0;
}
static RfLaunchCfg toy_cfg(const rf_graph* g) {
  RfLaunchCfg c = g->cfg;
  c.ept = toy_ept(g);
  return c;
}

static cudaKernel_t jit_toys(rf_graph* g, int ept, std::string* err) {
  int i = ept_index(g->eval, toy_coldt(g), ept);
  if (!g->jk_toys[i]) {
    cudaKernel_t k = rf_jit_kernel(g->prog, fcode(g), g->eval, toy_coldt(g),
                                   g->toy_bulk ? RF_JIT_TOYS_BULK : RF_JIT_TOYS, ept,
                                   toy_min_blocks(), nullptr, err);
    if (k && g->toy_bulk) {  // its stage ring may use more than 48 KB of shared memory
      int optin = 0;
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, g->device);
      cudaFuncAttributes fa;  // the kernel's static shared memory comes off the opt-in total
      cudaError_t e = cudaFuncGetAttributes(&fa, reinterpret_cast<const void*>(k));
      if (e == cudaSuccess)
        e = cudaFuncSetAttribute(reinterpret_cast<const void*>(k),
                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 optin - (int)fa.sharedSizeBytes);
      if (e != cudaSuccess) {
        *err = std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(e);
        return nullptr;
      }
    }
    g->jk_toys[i] = k;
  }
  return g->jk_toys[i];
}

static void free_work(rf_graph* g) {
  cudaFree(g->work.partials);
  cudaFree(g->work.counter);
  cudaFree(g->work.toy_consts);
  cudaFree(g->work.adam_m1);
  cudaFree(g->work.adam_m2);
  cudaFree(g->bound32);
  cudaFree(g->stage);
  cudaFree(g->plain_buf);
  cudaFree(g->plain_partials);
  if (g->fit_stream) cudaStreamDestroy(g->fit_stream);
  cudaFree(g->pro_buf);
  cudaFree(g->work.consts_x);
  cudaFree(g->work.toy_consts_x);
  cudaFree(g->formula_buf);
  cudaFree(g->formula_ticket);
}

// For other translation units of the library (noalloc.cu): validation plus
// canonicalisation of a descriptor, and setting the thread's error message.
rf_status rf_canonical_program(const rf_graph_desc* desc, RfProgram* P) {
  rf_status s = validate_desc(desc);
  if (s) return s;
  s = canonicalise(desc, P);
  if (s) return s;
  for (int k = 0; k < P->n_leaves; ++k)
    if (P->leaf[k].type == RFL_FORMULA || P->leaf[k].type == RFL_HYPATIA2)
      return fail(RF_EUNSUPPORTED,
                  "formula and Hypatia2 leaves need rf_graph_compile (specialised kernels)");
  if (P->n_leaves > RF_GENERIC_MAXL)
    return fail(RF_EUNSUPPORTED, "more than 4 leaves need rf_graph_compile (specialised kernels)");
  return RF_OK;
}

void rf_set_last_error(const char* msg) { g_err = msg; }

extern "C" {

const char* rf_last_error(void) { return g_err.c_str(); }

rf_status rf_graph_validate(const rf_graph_desc* desc) {
  g_err.clear();
  rf_status s = validate_desc(desc);
  if (s) return s;
  RfProgram P;
  return canonicalise(desc, &P);
}

rf_status rf_graph_compile(const rf_graph_desc* desc, rf_graph** out) {
  g_err.clear();
  if (!out) return fail(RF_EINVAL, "out is NULL");
  *out = nullptr;
  rf_status s = validate_desc(desc);
  if (s) return s;
  rf_graph* g = new rf_graph();
  int leaf_node[RF_MAXL] = {0};
  s = canonicalise(desc, &g->prog, leaf_node);
  if (s) {
    delete g;
    return s;
  }
  for (int k = 0; k < g->prog.n_leaves; ++k) {
    const int t = g->prog.leaf[k].type;
    if (t != RFL_FORMULA && t != RFL_HYPATIA2) continue;  // numerically normalised
    if (t == RFL_FORMULA) {
      const rf_node_desc& n = desc->nodes[leaf_node[k]];
      std::string err;
      rf_expr_translate(n.formula, n.n_params, &g->fcode.leaf[k], &err);  // validated above
    }
    ++g->n_formula;
  }
  g->eval = desc->eval_precision;
  g->coldt = desc->column_dtype;
  g->n_obs = desc->n_obs;
  if (const char* v = getenv("RF_TOY_STREAM")) g->toy_bulk = v[0] == 'b';
  if (g->eval == RF_EVAL_FP64) {
    g->cfg.ept = (g->coldt == RF_F64) ? 2 : 4;
    g->cfg.min_blocks = 2;  // FP64 evaluation runs out of registers at 80
  }
  cudaError_t e = cudaGetDevice(&g->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&g->num_sms, cudaDevAttrMultiProcessorCount, g->device);
  if (e != cudaSuccess) {
    delete g;
    return cuda_fail(e, "rf_graph_compile: device query");
  }
  // block rows of the largest grid (8 blocks per SM) and the group rows of the
  // grid's FP64 tree
  g->max_rows_single = (int64_t)g->num_sms * 8 + RF_TREE_GROUPS;
  e = cudaMalloc(&g->work.partials, sizeof(double) * RF_NACC_MAX * g->max_rows_single);
  if (e == cudaSuccess) e = cudaMalloc(&g->work.counter, RF_COUNTER_WORDS * sizeof(unsigned int));
  if (e == cudaSuccess) e = cudaMemset(g->work.counter, 0, RF_COUNTER_WORDS * sizeof(unsigned int));
  if (e != cudaSuccess) {
    free_work(g);
    delete g;
    return fail(RF_ENOMEM, std::string("rf_graph_compile: ") + cudaGetErrorString(e));
  }
  g->work.status = g->work.counter + 1;
  g->work.adam_t = reinterpret_cast<int32_t*>(g->work.counter + 2);
  // constants of the separate prologue kernel, and its FP64 constants for a
  // zero-coefficient call with FP32 evaluation
  e = cudaMalloc(&g->pro_buf, rf_consts_size(g->eval));
  if (e == cudaSuccess) e = cudaMalloc(&g->work.consts_x, sizeof(RfExact));
  if (e != cudaSuccess) {
    free_work(g);
    delete g;
    return fail(RF_ENOMEM, std::string("rf_graph_compile: ") + cudaGetErrorString(e));
  }
  g->work.consts = g->pro_buf;
  if (g->n_formula) {
    // [RF_MAXL * NV] log I and derivatives, then [RF_MAXL * blocks * NV]
    // partials; tickets
    const size_t nv = RF_FORMULA_NV;
    e = cudaMalloc(&g->formula_buf, sizeof(double) * nv * RF_MAXL * (1 + RF_FORMULA_BLOCKS));
    if (e == cudaSuccess) e = cudaMalloc(&g->formula_ticket, sizeof(unsigned int) * RF_MAXL);
    if (e == cudaSuccess) e = cudaMemset(g->formula_ticket, 0, sizeof(unsigned int) * RF_MAXL);
    if (e != cudaSuccess) {
      free_work(g);
      delete g;
      return fail(RF_ENOMEM, std::string("rf_graph_compile: ") + cudaGetErrorString(e));
    }
    g->prog.formula_norm = g->formula_buf;
  }
  // Specialise the fused kernel for this graph unless RF_JIT=0.  If that is
  // not possible the graph keeps the precompiled generic kernels (same device
  // code, run-time dispatch); rf_graph_uses_jit reports which one runs.
  // Formula leaves and graphs of more than 4 leaves exist only in
  // specialised kernels: without them the compile fails.
  const bool jit_only = g->n_formula || g->prog.n_leaves > RF_GENERIC_MAXL;
  const char* env = getenv("RF_JIT");
  if (!(env && env[0] == '0') || jit_only) {
    g->jit = true;
    std::string err;
    bool ok = jit_fused(g, g->cfg.ept, g->cfg.min_blocks, &err) != nullptr;
    if (ok && g->n_formula) {
      g->jk_norm = rf_jit_kernel(g->prog, fcode(g), g->eval, g->coldt, RF_JIT_NORM, 0, 0, nullptr,
                                 &err);
      ok = g->jk_norm != nullptr;
    }
    if (!ok && jit_only) {
      const std::string what = g->n_formula ? "formula leaves" : "more than 4 leaves";
      free_work(g);
      delete g;
      return fail(RF_ECUDA, what + " need the specialised kernels: " + err);
    }
    if (!ok) {
      g->jit = false;
      g_err = "JIT unavailable, generic kernels in use: " + err;
    }
  }
  *out = g;
  return RF_OK;
}

rf_status rf_graph_set_jit(rf_graph* g, int32_t enable) {
  if (!g) return fail(RF_EINVAL, "graph is NULL");
  if (!enable) {
    if (g->n_formula)
      return fail(RF_EUNSUPPORTED, "formula leaves run only in the specialised kernels");
    if (g->prog.n_leaves > RF_GENERIC_MAXL)
      return fail(RF_EUNSUPPORTED, "more than 4 leaves run only in the specialised kernels");
    g->jit = false;
    if (g->cfg.ept == 16) g->cfg.ept = 8;  // not instantiated in the generic kernels
    return RF_OK;
  }
  bool was = g->jit;
  g->jit = true;
  std::string err;
  if (!jit_fused(g, g->cfg.ept, g->cfg.min_blocks, &err)) {
    g->jit = was;
    return fail(RF_ECUDA, "JIT compile/load failed: " + err);
  }
  return RF_OK;
}

int32_t rf_graph_uses_jit(const rf_graph* g) { return g && g->jit ? 1 : 0; }

uint64_t rf_graph_kernel_hash(const rf_graph* g) {
  if (!g || !g->jit) return 0;
  return rf_jit_hash(g->prog, fcode(g), g->eval, g->coldt, RF_JIT_FUSED, g->cfg.ept,
                     g->cfg.min_blocks);
}

uint64_t rf_graph_toy_kernel_hash(const rf_graph* g) {
  if (!g || !g->jit || !g->bound) return 0;
  return rf_jit_hash(g->prog, fcode(g), g->eval, toy_coldt(g),
                     g->toy_bulk ? RF_JIT_TOYS_BULK : RF_JIT_TOYS, toy_ept(g), toy_min_blocks());
}

rf_status rf_graph_get_toy_launch(const rf_graph* g, int32_t* block, int32_t* events_per_lane,
                                  int32_t* regs) {
  g_err.clear();
  if (!g || !block || !events_per_lane || !regs) return fail(RF_EINVAL, "NULL argument");
  *block = g->cfg.block;
  *events_per_lane = toy_ept(g);
  *regs = 0;
  if (g->jit && g->bound) {
    const cudaKernel_t k = g->jk_toys[ept_index(g->eval, toy_coldt(g), toy_ept(g))];
    cudaFuncAttributes fa;
    if (k && cudaFuncGetAttributes(&fa, reinterpret_cast<const void*>(k)) == cudaSuccess)
      *regs = fa.numRegs;
    else
      cudaGetLastError();
  }
  return RF_OK;
}

int32_t rf_graph_kernel_regs(const rf_graph* g) {
  if (!g || !g->jit) return 0;
  return g->jk_regs[ept_index(g->eval, g->coldt, g->cfg.ept)][g->cfg.min_blocks - 2];
}

rf_status rf_jit_check(const rf_graph_desc* desc) {
  g_err.clear();
  rf_status s = validate_desc(desc);
  if (s) return s;
  RfProgram P;
  int leaf_node[RF_MAXL] = {0};
  s = canonicalise(desc, &P, leaf_node);
  if (s) return s;
  RfFormulaCode fc;
  int nf = 0;
  std::string err;
  for (int k = 0; k < P.n_leaves; ++k)
    if (P.leaf[k].type == RFL_FORMULA) {
      const rf_node_desc& n = desc->nodes[leaf_node[k]];
      rf_expr_translate(n.formula, n.n_params, &fc.leaf[k], &err);
      ++nf;
    } else if (P.leaf[k].type == RFL_HYPATIA2) {
      ++nf;
    }
  const RfFormulaCode* fcp = nf ? &fc : nullptr;
  const int ept = desc->eval_precision == RF_EVAL_FP32 ? 4 : (desc->column_dtype == RF_F64 ? 2 : 4);
  for (int kind : {RF_JIT_FUSED, RF_JIT_TOYS, RF_JIT_TOYS_BULK, RF_JIT_LOGP, RF_JIT_NORM}) {
    if (nf ? (kind == RF_JIT_TOYS || kind == RF_JIT_TOYS_BULK) : kind == RF_JIT_NORM) continue;
    // FP32-evaluated toy kernels read FP32 columns (converted at bind time)
    const bool fp32 = desc->eval_precision == RF_EVAL_FP32;
    const bool toy = kind == RF_JIT_TOYS || kind == RF_JIT_TOYS_BULK;
    const int cd = (toy && fp32) ? (int)RF_F32 : (int)desc->column_dtype;
    const int ke = toy ? 8 : ept;  // the segment kernel's events per lane
    if (!rf_jit_compile_only(P, fcp, desc->eval_precision, cd, kind, ke, toy ? 0 : 3, &err))
      return fail(RF_ECUDA, err);
  }
  return RF_OK;
}

rf_status rf_graph_destroy(rf_graph* g) {
  if (!g) return RF_OK;
  free_work(g);
  delete g;
  return RF_OK;
}

static rf_status check_events(const rf_graph* g, const void* events, int64_t n) {
  if (n < 0) return fail(RF_EINVAL, "n_events < 0");
  if (n > 0 && !events) return fail(RF_EINVAL, "events is NULL");
  size_t sz = g->coldt == RF_F64 ? 8 : 4;
  if (reinterpret_cast<uintptr_t>(events) % sz)
    return fail(RF_EALIGN, "event columns are not aligned to their element size");
  return RF_OK;
}

// One call = the FP64 prologue kernel, then the fused kernel as its
// programmatic dependent (it launches at once and waits for the constants).
static int fused_dispatch(rf_graph* g, const RfLaunchCfg& cfg, const void* ev, int64_t n,
                          const double* params, double* nll, double* grad, cudaStream_t st) {
  const RfProgram& P = g->prog;
  if (g->n_formula) {  // their integrals first; the prologue then runs after them
    int ne = rf_jit_launch_norm(g->jk_norm, P, g->n_formula, params,
                                g->formula_buf + RF_FORMULA_NV * RF_MAXL, g->formula_ticket, st);
    if (ne) return ne;
  }
  int pe = rf_launch_prologue(P, g->eval, params, g->work, true, st);
  if (pe) return pe;
  if (g->jit) {
    cudaKernel_t k = g->jk_fused[ept_index(g->eval, g->coldt, cfg.ept)][cfg.min_blocks - 2];
    if (!k) return (int)cudaErrorInvalidValue;  // compiled by compile/set_launch/tune
    return rf_jit_launch_fused(k, P, g->coldt, cfg, g->num_sms, ev, n, params, g->work, nll,
                               grad, st);
  }
  if (g->eval == RF_EVAL_FP32)
    return g->coldt == RF_F32
               ? rf_fused_f32_c32(P, cfg, g->num_sms, ev, n, params, g->work, nll, grad, st)
               : rf_fused_f32_c64(P, cfg, g->num_sms, ev, n, params, g->work, nll, grad, st);
  return g->coldt == RF_F32
             ? rf_fused_f64_c32(P, cfg, g->num_sms, ev, n, params, g->work, nll, grad, st)
             : rf_fused_f64_c64(P, cfg, g->num_sms, ev, n, params, g->work, nll, grad, st);
}

rf_status rf_nll(rf_graph* g, const void* events, int64_t n_events, const double* params,
                 double* nll, double* grad, rf_stream stream) {
  if (!g) return fail(RF_EINVAL, "graph is NULL");
  rf_status s = check_events(g, events, n_events);
  if (s) return s;
  if (!params && g->prog.n_par > 0) return fail(RF_EINVAL, "params is NULL");
  if (!nll) return fail(RF_EINVAL, "nll is NULL");
  int e = fused_dispatch(g, g->cfg, events, n_events, params, nll, grad,
                         reinterpret_cast<cudaStream_t>(stream));
  g->last_launches = g->n_formula ? 3 : 2;
  if (e) return cuda_fail((cudaError_t)e, "rf_nll launch");
  return RF_OK;
}

rf_status rf_nll_host(rf_graph* g, const void* host_events, int64_t n_events,
                      const double* host_params, double* host_nll, double* host_grad,
                      rf_stream stream) {
  if (!g) return fail(RF_EINVAL, "graph is NULL");
  if (n_events < 0 || (n_events > 0 && !host_events) || !host_nll ||
      (!host_params && g->prog.n_par > 0))
    return fail(RF_EINVAL, "NULL or negative argument");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const size_t sz = g->coldt == RF_F64 ? 8 : 4;
  const size_t ev_bytes = (size_t)g->n_obs * (size_t)n_events * sz;
  const size_t ev_pad = (ev_bytes + 255) & ~(size_t)255;
  const size_t need = ev_pad + sizeof(double) * (2 * RF_MAXPAR + 2);
  if (need > g->stage_bytes) {
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "rf_nll_host sync");
    cudaFree(g->stage);
    g->stage = nullptr;
    g->stage_bytes = 0;
    e = cudaMalloc(&g->stage, need);
    if (e != cudaSuccess) return fail(RF_ENOMEM, "rf_nll_host: staging allocation failed");
    g->stage_bytes = need;
  }
  char* base = static_cast<char*>(g->stage);
  double* dp = reinterpret_cast<double*>(base + ev_pad);
  double* dout = dp + RF_MAXPAR;
  const int np = g->prog.n_par;
  // Page-locked host memory the device can address is read by the fused
  // kernel in place (on a Grace-Blackwell node over NVLink-C2C: the link
  // carries each byte once and no staging copy is made); other host memory
  // is staged with one copy.  RF_HOST_DIRECT=0 always stages.
  const void* ev_dev = base;
  if (ev_bytes && !(getenv("RF_HOST_DIRECT") && getenv("RF_HOST_DIRECT")[0] == '0')) {
    cudaPointerAttributes pa;
    if (cudaPointerGetAttributes(&pa, host_events) == cudaSuccess &&
        pa.type == cudaMemoryTypeHost && pa.devicePointer)
      ev_dev = pa.devicePointer;
    else
      cudaGetLastError();  // not registered with CUDA: stage it
  }
  cudaError_t e = cudaSuccess;
  if (ev_bytes && ev_dev == base)
    e = cudaMemcpyAsync(base, host_events, ev_bytes, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && np)
    e = cudaMemcpyAsync(dp, host_params, sizeof(double) * np, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return cuda_fail(e, "rf_nll_host H2D");
  int le = fused_dispatch(g, g->cfg, ev_dev, n_events, dp, dout, host_grad ? dout + 1 : nullptr, st);
  g->last_launches = g->n_formula ? 3 : 2;
  if (le) return cuda_fail((cudaError_t)le, "rf_nll_host launch");
  e = cudaMemcpyAsync(host_nll, dout, sizeof(double), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && host_grad && np)
    e = cudaMemcpyAsync(host_grad, dout + 1, sizeof(double) * np, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "rf_nll_host D2H");
  return RF_OK;
}

rf_status rf_logp(rf_graph* g, const void* events, int64_t n_events, const double* params,
                  double* logp, rf_stream stream) {
  if (!g) return fail(RF_EINVAL, "graph is NULL");
  rf_status s = check_events(g, events, n_events);
  if (s) return s;
  if ((!params && g->prog.n_par > 0) || (!logp && n_events > 0))
    return fail(RF_EINVAL, "params or logp is NULL");
  if (n_events == 0) return RF_OK;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const RfProgram& P = g->prog;
  int e;
  if (g->jit && !g->jk_logp) {
    std::string err;  // first call compiles the kernel (host-synchronous)
    g->jk_logp = rf_jit_kernel(P, fcode(g), g->eval, g->coldt, RF_JIT_LOGP, 0, 0, nullptr, &err);
    if (!g->jk_logp) return fail(RF_ECUDA, "JIT log P kernel: " + err);
  }
  int launches = 1;
  if (g->n_formula) {
    e = rf_jit_launch_norm(g->jk_norm, P, g->n_formula, params,
                           g->formula_buf + RF_FORMULA_NV * RF_MAXL, g->formula_ticket, st);
    if (e) return cuda_fail((cudaError_t)e, "rf_logp normalisation launch");
    ++launches;
  }
  if (g->jit)
    e = rf_jit_launch_logp(g->jk_logp, P, events, n_events, params, logp, st);
  else if (g->eval == RF_EVAL_FP32)
    e = g->coldt == RF_F32 ? rf_logp_f32_c32(P, events, n_events, params, logp, st)
                           : rf_logp_f32_c64(P, events, n_events, params, logp, st);
  else
    e = g->coldt == RF_F32 ? rf_logp_f64_c32(P, events, n_events, params, logp, st)
                           : rf_logp_f64_c64(P, events, n_events, params, logp, st);
  g->last_launches = launches;
  if (e) return cuda_fail((cudaError_t)e, "rf_logp launch");
  return RF_OK;
}

rf_status rf_graph_bind_events(rf_graph* g, const void* events, int64_t n_events,
                               int32_t max_toys) {
  if (!g) return fail(RF_EINVAL, "graph is NULL");
  rf_status s = check_events(g, events, n_events);
  if (s) return s;
  if (max_toys < 1) return fail(RF_EINVAL, "max_toys must be >= 1");
  if (g->n_formula)
    return fail(RF_EUNSUPPORTED, "toy studies do not take formula leaves (per-toy quadrature)");
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(e, "rf_graph_bind_events sync");
  cudaFree(g->work.toy_consts);
  cudaFree(g->work.toy_consts_x);
  cudaFree(g->work.adam_m1);
  cudaFree(g->work.adam_m2);
  g->work.toy_consts = nullptr;
  g->work.toy_consts_x = nullptr;
  g->work.adam_m1 = g->work.adam_m2 = nullptr;
  g->bound = false;
  g->max_toys = 0;
  // one row per (warp, toy) segment: at most (launch warps) + toys, and a
  // launch has at most 8 blocks of 8 warps per SM
  const int64_t rows = (int64_t)max_toys + (int64_t)g->num_sms * 64 + RF_TREE_GROUPS;
  if (rows > g->max_rows_single) {
    cudaFree(g->work.partials);
    g->work.partials = nullptr;
    e = cudaMalloc(&g->work.partials, sizeof(double) * RF_NACC_MAX * rows);
    if (e != cudaSuccess) {
      g->max_rows_single = 0;
      return fail(RF_ENOMEM, "bind: partials allocation failed");
    }
    g->max_rows_single = rows;
  }
  const size_t np = (size_t)std::max(g->prog.n_par, 1);
  e = cudaMalloc(&g->work.toy_consts, rf_consts_size(g->eval) * (size_t)max_toys);
  if (e == cudaSuccess) e = cudaMalloc(&g->work.toy_consts_x, sizeof(RfExact) * (size_t)max_toys);
  if (e == cudaSuccess) e = cudaMalloc(&g->work.adam_m1, sizeof(double) * np * (size_t)max_toys);
  if (e == cudaSuccess) e = cudaMalloc(&g->work.adam_m2, sizeof(double) * np * (size_t)max_toys);
  if (e != cudaSuccess) return fail(RF_ENOMEM, "bind: toy workspace allocation failed");
  const void* toy_events = events;
  if (g->eval == RF_EVAL_FP32 && g->coldt == RF_F64) {
    const size_t elems = (size_t)g->n_obs * (size_t)n_events;
    if (elems > g->bound32_elems) {
      cudaFree(g->bound32);
      g->bound32 = nullptr;
      g->bound32_elems = 0;
      e = cudaMalloc(&g->bound32, sizeof(float) * std::max<size_t>(elems, 1));
      if (e != cudaSuccess) return fail(RF_ENOMEM, "bind: FP32 column allocation failed");
      g->bound32_elems = elems;
    }
    int ce = rf_columns_to_f32(static_cast<const double*>(events), g->bound32, (int64_t)elems,
                               nullptr);
    if (ce == 0) ce = (int)cudaDeviceSynchronize();
    if (ce) return cuda_fail((cudaError_t)ce, "bind: FP32 column conversion");
    toy_events = g->bound32;
  }
  if (g->jit) {
    std::string err;
    if (!jit_toys(g, toy_ept(g), &err)) return fail(RF_ECUDA, "JIT toy kernel: " + err);
  }
  g->bound_events = toy_events;
  g->bound = true;
  g->bound_n = n_events;
  g->max_toys = max_toys;
  g->max_toy_rows = rows;
  return RF_OK;
}

static rf_status batched_checks(rf_graph* g, const int64_t* offsets, int32_t toys,
                                const double* pm, const double* out) {
  if (!g) return fail(RF_EINVAL, "graph is NULL");
  if (!g->bound) return fail(RF_EINVAL, "rf_graph_bind_events was not called");
  if (toys < 1 || toys > g->max_toys) return fail(RF_EINVAL, "toys must be in 1..max_toys");
  if (!offsets || !pm || !out) return fail(RF_EINVAL, "NULL argument");
  if (g->jit && !g->jk_toys[ept_index(g->eval, toy_coldt(g), toy_ept(g))]) {
    std::string err;
    if (!jit_toys(g, toy_ept(g), &err)) return fail(RF_ECUDA, "JIT toy kernel: " + err);
  }
  return RF_OK;
}

rf_status rf_nll_batched(rf_graph* g, const int64_t* offsets, int32_t toys,
                         const double* params_matrix, double* out, rf_stream stream) {
  rf_status s = batched_checks(g, offsets, toys, params_matrix, out);
  if (s) return s;
  int n = 0;
  int e = rf_launch_batched(g->prog, g->eval, toy_coldt(g), toy_cfg(g), g->num_sms, g->bound_events,
                            g->bound_n, offsets, toys, const_cast<double*>(params_matrix), out,
                            g->work, nullptr, 0.0, g->max_toy_rows,
                            g->jit ? g->jk_toys[ept_index(g->eval, toy_coldt(g), toy_ept(g))] : nullptr,
                            g->jit && g->toy_bulk,
                            stream, &n);
  g->last_launches = n;
  if (e) return cuda_fail((cudaError_t)e, "rf_nll_batched launch");
  return RF_OK;
}

rf_status rf_fit_toys(rf_graph* g, const int64_t* offsets, int32_t toys,
                      double* params_matrix, const double* scale, int32_t iters, double lr,
                      double* out, rf_stream stream) {
  rf_status s = batched_checks(g, offsets, toys, params_matrix, out);
  if (s) return s;
  if (!scale || iters < 0) return fail(RF_EINVAL, "scale is NULL or iters < 0");
  cudaStream_t user = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e = cudaSuccess;
  if (!g->fit_stream) e = cudaStreamCreateWithFlags(&g->fit_stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) return cuda_fail(e, "rf_fit_toys stream");
  cudaStream_t fs = g->fit_stream;
  cudaEvent_t ev;
  e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventRecord(ev, user);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(fs, ev, 0);
  if (e != cudaSuccess) return cuda_fail(e, "rf_fit_toys order");
  const size_t np = (size_t)std::max(g->prog.n_par, 1);
  e = cudaMemsetAsync(g->work.adam_m1, 0, sizeof(double) * np * toys, fs);
  if (e == cudaSuccess) e = cudaMemsetAsync(g->work.adam_m2, 0, sizeof(double) * np * toys, fs);
  if (e == cudaSuccess) e = cudaMemsetAsync(g->work.adam_t, 0, sizeof(int32_t), fs);
  if (e != cudaSuccess) return cuda_fail(e, "rf_fit_toys reset");
  int le = 0;
  int launches = 0;
  if (iters > 0) {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    e = cudaStreamBeginCapture(fs, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(e, "rf_fit_toys capture");
    int n = 0;
    le = rf_launch_batched(g->prog, g->eval, toy_coldt(g), toy_cfg(g), g->num_sms, g->bound_events,
                           g->bound_n, offsets, toys, params_matrix, out, g->work, scale, lr,
                           g->max_toy_rows,
                           g->jit ? g->jk_toys[ept_index(g->eval, toy_coldt(g), toy_ept(g))] : nullptr,
                            g->jit && g->toy_bulk,
                           fs, &n);
    e = cudaStreamEndCapture(fs, &graph);
    if (le) {
      if (graph) cudaGraphDestroy(graph);
      return cuda_fail((cudaError_t)le, "rf_fit_toys captured launch");
    }
    if (e != cudaSuccess) return cuda_fail(e, "rf_fit_toys end capture");
    e = cudaGraphInstantiate(&exec, graph, 0);
    if (e != cudaSuccess) {
      cudaGraphDestroy(graph);
      return cuda_fail(e, "rf_fit_toys instantiate");
    }
    for (int it = 0; it < iters && e == cudaSuccess; ++it) e = cudaGraphLaunch(exec, fs);
    launches += n * iters;
    cudaError_t e2 = cudaStreamSynchronize(fs);
    cudaGraphExecDestroy(exec);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(e, "rf_fit_toys replay");
    if (e2 != cudaSuccess) return cuda_fail(e2, "rf_fit_toys sync");
  }
  e = cudaEventRecord(ev, fs);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(user, ev, 0);
  if (e == cudaSuccess) e = cudaStreamSynchronize(fs);
  cudaEventDestroy(ev);
  g->last_launches = launches;
  if (e != cudaSuccess) return cuda_fail(e, "rf_fit_toys finish");
  return RF_OK;
}

rf_status rf_graph_set_shard_weight(rf_graph* g, double w) {
  if (!g) return fail(RF_EINVAL, "graph is NULL");
  if (!std::isfinite(w)) return fail(RF_EINVAL, "weight must be finite");
  g->prog.ext_weight = w;
  return RF_OK;
}

rf_status rf_generate_toys(rf_graph* g, const double* params_matrix, const int64_t* comp_counts,
                           const int64_t* offsets, int32_t toys, uint64_t seed, void* events,
                           int64_t n_events, rf_stream stream) {
  if (!g) return fail(RF_EINVAL, "graph is NULL");
  if (toys < 1 || !params_matrix || !comp_counts || !offsets || n_events < 0 ||
      (n_events > 0 && !events))
    return fail(RF_EINVAL, "NULL or negative argument");
  if (g->n_formula) return fail(RF_EUNSUPPORTED, "formula leaves have no sampler");
  const RfProgram& P = g->prog;
  // every component must draw every observable
  if (P.n_cols != g->n_obs) return fail(RF_EUNSUPPORTED, "an observable no leaf reads");
  for (int c = 0; c < P.n_comp; ++c) {
    int mask = 0;
    for (int k = 0; k < P.n_leaves; ++k)
      if (P.leaf[k].comp == c) mask |= 1 << P.leaf[k].col;
    if (mask != (1 << P.n_cols) - 1)
      return fail(RF_EUNSUPPORTED, "a component does not cover every observable");
  }
  if (n_events == 0) return RF_OK;
  int e = rf_launch_generate(P, g->coldt, params_matrix, comp_counts, offsets, toys,
                             (unsigned long long)seed, events, n_events, g->work.status,
                             g->num_sms, reinterpret_cast<cudaStream_t>(stream));
  g->last_launches = 1;
  if (e) return cuda_fail((cudaError_t)e, "rf_generate_toys launch");
  return RF_OK;
}

rf_status rf_nll_plain(rf_graph* g, const void* events, int64_t n_events, const double* params,
                       double* nll, double* grad, rf_stream stream) {
  if (!g) return fail(RF_EINVAL, "graph is NULL");
  if (g->n_formula) return fail(RF_EUNSUPPORTED, "the node-by-node baseline has no formula leaves");
  rf_status s = check_events(g, events, n_events);
  if (s) return s;
  if ((!params && g->prog.n_par > 0) || !nll) return fail(RF_EINVAL, "NULL argument");
  size_t need = rf_plain_bytes(g->prog, n_events);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (need > g->plain_bytes) {
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "rf_nll_plain sync");
    cudaFree(g->plain_buf);
    g->plain_buf = nullptr;
    g->plain_bytes = 0;
    e = cudaMalloc(&g->plain_buf, need);
    if (e != cudaSuccess) return fail(RF_ENOMEM, "rf_nll_plain: node buffers allocation failed");
    g->plain_bytes = need;
  }
  if (!g->plain_partials) {
    cudaError_t e = cudaMalloc(&g->plain_partials, sizeof(double) * RF_NACC_MAX * 4096 + 64);
    if (e != cudaSuccess) return fail(RF_ENOMEM, "rf_nll_plain: partials allocation failed");
    g->plain_counter = reinterpret_cast<unsigned int*>(g->plain_partials + RF_NACC_MAX * 4096);
    e = cudaMemset(g->plain_counter, 0, 64);
    if (e != cudaSuccess) return cuda_fail(e, "rf_nll_plain memset");
  }
  int n = 0;
  int e = rf_launch_plain(g->prog, g->coldt, events, n_events, params, g->plain_buf, nll, grad,
                          g->plain_partials, g->plain_counter, st, &n);
  g->last_launches = n;
  if (e) return cuda_fail((cudaError_t)e, "rf_nll_plain launch");
  return RF_OK;
}

rf_status rf_graph_get_launch(const rf_graph* g, rf_launch* cfg) {
  if (!g || !cfg) return fail(RF_EINVAL, "NULL argument");
  cfg->block = g->cfg.block;
  cfg->ept = g->cfg.ept;
  cfg->blocks_per_sm = g->cfg.blocks_per_sm;
  cfg->min_blocks = g->cfg.min_blocks;
  return RF_OK;
}

rf_status rf_graph_set_launch(rf_graph* g, const rf_launch* cfg) {
  if (!g || !cfg) return fail(RF_EINVAL, "NULL argument");
  if (cfg->block != 64 && cfg->block != 128 && cfg->block != 256)
    return fail(RF_EINVAL, "block must be 64, 128 or 256");
  if (!ept_ok(g->eval, g->coldt, cfg->ept, g->jit))
    return fail(RF_EINVAL, "events per thread not available for this precision / dtype");
  if (cfg->blocks_per_sm < 1 || cfg->blocks_per_sm > 8)
    return fail(RF_EINVAL, "blocks_per_sm must be in 1..8");
  if (!min_blocks_ok(cfg->min_blocks)) return fail(RF_EINVAL, "min_blocks must be 2, 3 or 4");
  if (g->jit) {
    std::string err;
    if (!jit_fused(g, cfg->ept, cfg->min_blocks, &err))
      return fail(RF_ECUDA, "JIT fused kernel: " + err);
    if (g->bound && !jit_toys(g, toy_ept(g), &err))
      return fail(RF_ECUDA, "JIT toy kernel: " + err);
  }
  g->cfg.block = cfg->block;
  g->cfg.ept = cfg->ept;
  g->cfg.blocks_per_sm = cfg->blocks_per_sm;
  g->cfg.min_blocks = cfg->min_blocks;
  return RF_OK;
}

}  // extern "C"

namespace {

// Key of a tuning result in the on-disk cache: the kernel it was timed with
// (the graph-specialised source, else the structure the generic kernels
// branch on and the library build), the precisions, the size bucket
// floor(log2 n) and the device (compute capability and SM count).
uint64_t tune_key(const rf_graph* g, int64_t n_events) {
  std::string k;
  char buf[96];
  if (g->jit) {
    snprintf(buf, sizeof(buf), "jit %016llx",
             (unsigned long long)rf_jit_hash(g->prog, fcode(g), g->eval, g->coldt,
                                             RF_JIT_FUSED, 4, 2));
    k = buf;
  } else {
    k = std::string("generic ") + __DATE__ + " " + __TIME__;
    const RfProgram& P = g->prog;
    snprintf(buf, sizeof(buf), " %d %d %d %d %d", P.kind, P.n_leaves, P.n_comp, P.n_cols,
             P.coef_free);
    k += buf;
    for (int i = 0; i < P.n_leaves; ++i) {
      snprintf(buf, sizeof(buf), " %d/%d", P.leaf[i].type, P.leaf[i].gmask);
      k += buf;
    }
  }
  int dev = 0, sms = 0, maj = 0, mnr = 0, bucket = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&maj, cudaDevAttrComputeCapabilityMajor, dev);
  cudaDeviceGetAttribute(&mnr, cudaDevAttrComputeCapabilityMinor, dev);
  for (int64_t n = n_events; n > 1; n >>= 1) ++bucket;
  snprintf(buf, sizeof(buf), "|%d|%d|%d|sm%d%d|%d", g->eval, g->coldt, bucket, maj, mnr, sms);
  return rf_text_hash(k + buf);
}

std::string tune_path(uint64_t key) {
  char name[64];
  snprintf(name, sizeof(name), "/tune-%016llx.txt", (unsigned long long)key);
  return rf_cache_dir() + name;
}

bool tune_load(uint64_t key, rf_launch* c) {
  FILE* f = fopen(tune_path(key).c_str(), "r");
  if (!f) return false;
  const bool ok = fscanf(f, "rf-tune 1 %d %d %d %d", &c->block, &c->ept, &c->blocks_per_sm,
                         &c->min_blocks) == 4;
  fclose(f);
  return ok;
}

// written under a temporary name and renamed, so readers never see a partial file
void tune_store(uint64_t key, const RfLaunchCfg& c) {
  const std::string dir = rf_cache_dir(), path = tune_path(key);
  mkdir(dir.c_str(), 0700);
  static std::atomic<unsigned> seq{0};  // graphs tuned from several threads
  const std::string tmp = path + "." + std::to_string(getpid()) + "." + std::to_string(seq++);
  if (FILE* f = fopen(tmp.c_str(), "w")) {
    const bool ok = fprintf(f, "rf-tune 1 %d %d %d %d\n", c.block, c.ept, c.blocks_per_sm,
                            c.min_blocks) > 0;
    fclose(f);
    if (ok) rename(tmp.c_str(), path.c_str());
    else remove(tmp.c_str());
  }
}

// Time of five fused calls with configuration c, issued back to back after
// two warm-up calls (a queue of evaluations: each call's FP64 prologue
// overlaps the previous call's event pass, so the time is the event pass's).
cudaError_t time_config(rf_graph* g, const RfLaunchCfg& c, const void* events, int64_t n_events,
                        const double* params, double* dout, cudaEvent_t a, cudaEvent_t b,
                        cudaStream_t st, float* tsum) {
  cudaError_t e = cudaSuccess;
  *tsum = 0.f;
  for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep)
    e = (cudaError_t)fused_dispatch(g, c, events, n_events, params, dout, dout + 1, st);
  if (e == cudaSuccess) e = cudaEventRecord(a, st);
  for (int rep = 0; rep < 5 && e == cudaSuccess; ++rep)
    e = (cudaError_t)fused_dispatch(g, c, events, n_events, params, dout, dout + 1, st);
  if (e == cudaSuccess) e = cudaEventRecord(b, st);
  if (e == cudaSuccess) e = cudaEventSynchronize(b);
  if (e == cudaSuccess) e = cudaEventElapsedTime(tsum, a, b);
  return e;
}

}  // namespace

extern "C" {

rf_status rf_graph_tune(rf_graph* g, const void* events, int64_t n_events, const double* params,
                        rf_stream stream, double* best_ms) {
  return rf_graph_tune_ex(g, events, n_events, params, stream, 0, best_ms, nullptr);
}

rf_status rf_graph_tune_ex(rf_graph* g, const void* events, int64_t n_events,
                           const double* params, rf_stream stream, int32_t flags,
                           double* best_ms, int32_t* from_cache) {
  if (!g) return fail(RF_EINVAL, "graph is NULL");
  if (flags & ~(RF_TUNE_NO_CACHE | RF_TUNE_REFRESH)) return fail(RF_EINVAL, "unknown tune flags");
  rf_status s = check_events(g, events, n_events);
  if (s) return s;
  if (from_cache) *from_cache = 0;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const bool use_cache = !(flags & RF_TUNE_NO_CACHE);
  const uint64_t key = use_cache ? tune_key(g, n_events) : 0;
  double* dout = nullptr;
  cudaError_t e = cudaMalloc(&dout, sizeof(double) * (1 + RF_MAXPAR));
  if (e != cudaSuccess) return fail(RF_ENOMEM, "tune scratch");
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  const RfLaunchCfg old = g->cfg;
  RfLaunchCfg best = g->cfg;
  float best_t = 1e30f;
  rf_launch hit;
  // a cached entry that no longer validates (another library version, a
  // damaged file) is ignored and overwritten
  if (use_cache && !(flags & RF_TUNE_REFRESH) && tune_load(key, &hit) &&
      rf_graph_set_launch(g, &hit) == RF_OK) {
    e = time_config(g, g->cfg, events, n_events, params, dout, a, b, st, &best_t);
    best = g->cfg;
    if (from_cache) *from_cache = 1;
  } else {
    const int blocks[3] = {64, 128, 256};
    const int bpss[6] = {1, 2, 3, 4, 6, 8};
    int epts[3], n_ept;
    if (g->eval == RF_EVAL_FP32) {
      epts[0] = 4;
      epts[1] = 8;
      epts[2] = 16;
      n_ept = g->jit ? 3 : 2;
    } else if (g->coldt == RF_F64) {
      epts[0] = 2;
      epts[1] = 4;
      n_ept = 2;
    } else {
      epts[0] = 4;
      n_ept = 1;
    }
    // register budgets: three for the specialised kernel (compiled in
    // parallel first), the generic kernels have one
    const int n_mb = g->jit ? 3 : 1;
    const int mbs[3] = {g->jit ? 2 : g->cfg.min_blocks, 3, 4};
    if (g->jit) {
      std::vector<std::string> srcs;
      for (int ei = 0; ei < n_ept; ++ei)
        for (int mi = 0; mi < n_mb; ++mi)
          srcs.push_back(rf_jit_source(g->prog, fcode(g), g->eval, g->coldt, RF_JIT_FUSED,
                                       epts[ei], mbs[mi]));
      rf_jit_precompile(srcs);
      std::string err;
      for (int ei = 0; ei < n_ept; ++ei)
        for (int mi = 0; mi < n_mb; ++mi)
          if (!jit_fused(g, epts[ei], mbs[mi], &err)) {
            cudaEventDestroy(a);
            cudaEventDestroy(b);
            cudaFree(dout);
            return fail(RF_ECUDA, "JIT fused kernel: " + err);
          }
    }
    for (int bi = 0; bi < 3 && e == cudaSuccess; ++bi)
      for (int ei = 0; ei < n_ept && e == cudaSuccess; ++ei)
        for (int pi = 0; pi < 6 * n_mb && e == cudaSuccess; ++pi) {
          RfLaunchCfg c = g->cfg;
          c.block = blocks[bi];
          c.ept = epts[ei];
          c.blocks_per_sm = bpss[pi % 6];
          c.min_blocks = mbs[pi / 6];
          float tsum = 0.f;
          e = time_config(g, c, events, n_events, params, dout, a, b, st, &tsum);
          if (e == cudaSuccess && tsum < best_t) {
            best_t = tsum;
            best = c;
          }
        }
    if (e == cudaSuccess && use_cache) tune_store(key, best);
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  cudaFree(dout);
  if (e != cudaSuccess) {
    g->cfg = old;
    return cuda_fail(e, "rf_graph_tune");
  }
  g->cfg.block = best.block;
  g->cfg.ept = best.ept;
  g->cfg.blocks_per_sm = best.blocks_per_sm;
  g->cfg.min_blocks = best.min_blocks;
  if (best_ms) *best_ms = best_t / 5.0;
  return RF_OK;
}

rf_status rf_graph_status(rf_graph* g, uint32_t* flags) {
  if (!g || !flags) return fail(RF_EINVAL, "NULL argument");
  cudaError_t e = cudaDeviceSynchronize();
  unsigned int v = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&v, g->work.status, sizeof(v), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemset(g->work.status, 0, sizeof(v));
  if (e != cudaSuccess) return cuda_fail(e, "rf_graph_status");
  *flags = v;
  return RF_OK;
}

int32_t rf_graph_last_launches(const rf_graph* g) { return g ? g->last_launches : 0; }

rf_status rf_check_d2f(const double* x, float* y_fast, float* y_ref, int64_t n,
                       rf_stream stream) {
  if (n < 0 || (n > 0 && (!x || !y_fast || !y_ref))) return fail(RF_EINVAL, "bad argument");
  int e = rf_run_check_d2f(x, y_fast, y_ref, n, reinterpret_cast<cudaStream_t>(stream));
  if (e) return cuda_fail((cudaError_t)e, "rf_check_d2f");
  return RF_OK;
}

rf_status rf_check_log(const float* x, float* y_fast, float* y_ref, int64_t n,
                       rf_stream stream) {
  if (n < 0 || (n > 0 && (!x || !y_fast || !y_ref))) return fail(RF_EINVAL, "bad argument");
  int e = rf_run_check_log(x, y_fast, y_ref, n, reinterpret_cast<cudaStream_t>(stream));
  if (e) return cuda_fail((cudaError_t)e, "rf_check_log");
  return RF_OK;
}

rf_status rf_microbench(double* out) {
  if (!out) return fail(RF_EINVAL, "out is NULL");
  int e = rf_run_microbench(out);
  if (e) return cuda_fail((cudaError_t)e, "rf_microbench");
  return RF_OK;
}

}  // extern "C"
