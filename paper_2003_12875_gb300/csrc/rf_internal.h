// rf_internal.h -- compiled-graph layout shared by the host graph compiler and
// the CUDA kernels of librfgpu.  Not part of the public C-ABI (include/rf.h).
//
// A graph is compiled into a "sum of products" program: P(x) = sum_c coef_c *
// prod_{k in c} f_k(x_obs(k)) / I_k, with at most RF_MAXL leaves and RF_MAXC
// components (the root is a leaf, a Prod of leaves, or an Add whose children
// are leaves or Prods of leaves).  Per event the kernels work in log space:
//   u_k   = log f_k(x) - off_k                (unnormalised leaf log-density)
//   v_c   = delta_c + sum_{k in c} u_k,  delta_c = beta_c - beta_ref
//   beta_c = log coef_c + sum_{k in c} (off_k - log I_k)     (FP64, hoisted)
//   ell   = log sum_c exp(v_c),  log P = beta_ref + ell
// so the NLL is -(n beta_ref + sum_i ell_i) (+ sum of yields if extended).
#pragma once
#ifdef __CUDACC_RTC__
typedef int int32_t;
typedef unsigned int uint32_t;
typedef long long int64_t;
typedef unsigned long long uint64_t;
typedef unsigned long long uintptr_t;
#else
#include <stddef.h>
#include <stdint.h>
#endif

#define RF_MAXL 6        // leaves per compiled graph (specialised kernels)
#define RF_MAXC 6        // components (Add children)
// the precompiled generic kernels (run-time dispatch) take up to 4 leaves;
// graphs with more run only in the kernels specialised for them
#define RF_GENERIC_MAXL 4
#define RF_LEAF_MAXP 4   // parameters per leaf
#define RF_PC 8          // per-leaf evaluation constants
#define RF_MAXPAR 64
// per-thread accumulators: ell, one per component, one per (leaf, leaf param)
#define RF_NACC(NL) (1 + (NL) + (NL) * RF_LEAF_MAXP)
#define RF_NACC_MAX RF_NACC(RF_MAXL)
// blocks whose partial sums fit the static scratch of rf_nll_noalloc
#define RF_NOALLOC_MAX_BLOCKS 1024
// Grid reduction of the single-dataset kernels: a two-level fixed-order FP64
// tree.  The block rows are split into at most RF_TREE_GROUPS contiguous
// groups; the last block of a group to finish sums the group's rows into a
// group row (rows gridDim.x + g of the partials), and the last group sums the
// group rows (a grid of at most RF_TREE_GROUPS blocks: one level, the last
// block sums the block rows).  Ticket words (RfWork::counter,
// RF_COUNTER_WORDS of them): [0] the group ticket (the grid ticket of a
// one-level tree), [1] status, [2] Adam step, [RF_TREE_GROUPS ..
// 2*RF_TREE_GROUPS) one ticket per group.
#define RF_TREE_GROUPS 32
#define RF_COUNTER_WORDS (2 * RF_TREE_GROUPS)
// lanes per toy of the toy finalize kernel (blocks of 32 toys)
#define RF_FIN_GROUP 4
// formula-leaf normalisation: 16-point Gauss-Legendre on RF_FORMULA_PANELS
// panels, one node per thread, RF_FORMULA_BLOCKS blocks of 128 threads; per
// leaf 1 + RF_LEAF_MAXP values (log I, then (dI/dp_j)/I)
#define RF_FORMULA_PANELS 128
#define RF_FORMULA_BLOCKS 16
#define RF_FORMULA_MAXP 9  // parameters of a numerically normalised leaf (Hypatia2: 9)
#define RF_FORMULA_NV (1 + RF_FORMULA_MAXP)

enum { RF_KIND_PROD = 0, RF_KIND_FRAC = 1, RF_KIND_EXT = 2 };
// gmask bit of an ARGUS leaf whose fixed p is not 1/2 (general-p form, no
// d/dp accumulator; bits 0..3 are the per-parameter gradient bits)
#define RF_ARGUS_GENERAL 16
// compile-time leaf form bit (never in a gmask): an Exponential whose range
// starts at 0 needs no shift of x
#define RF_GM_AT0 32
// device status bits (same values as RF_STATUS_* in include/rf.h)
#define RF_STATUS_PARAM_DOMAIN_BIT 1u
#define RF_STATUS_NONFINITE_BIT 2u
#define RF_STATUS_TIMEOUT_BIT 4u
#define RF_STATUS_GEN_EXHAUSTED_BIT 8u
enum {
  RFL_GAUSS = 1,
  RFL_EXP = 2,
  RFL_CHEB = 3,
  RFL_CB = 4,
  RFL_ARGUS = 5,
  RFL_JOHNSON = 9,
  RFL_FORMULA = 10,  // a formula given as text; specialised kernels only
  RFL_HYPATIA2 = 11, // Hypatia2 (9 parameters, numeric normalisation);
                     // specialised kernels only
  RFL_PARAMS = 12    // parameters 4.. of the Hypatia2 leaf in the slot before
                     // (no per-event work of its own)
};

struct RfLeafProg {
  int32_t type;      // RFL_*
  int32_t col;       // index among the loaded columns (0..n_cols-1)
  int32_t comp;      // component index
  int32_t npar;      // parameters of this leaf
  int32_t par[RF_LEAF_MAXP];  // global parameter slots
  int32_t gmask;     // bit j: gradient of leaf param j is wanted; ARGUS:
                     // RF_ARGUS_GENERAL selects the general-p form for a
                     // fixed p (a free p, bit 2, always takes it)
  int32_t part;      // RFL_PARAMS: which four parameters of the leaf `part`
                     // slots before (parameters 4 part .. 4 part + 3)
  double lo, hi;     // observable range
};

struct RfProgram {
  int32_t n_leaves;  // 1..RF_MAXL
  int32_t n_comp;    // 1..RF_MAXC
  int32_t kind;      // RF_KIND_*
  int32_t n_par;     // parameters in the vector
  int32_t n_cols;    // distinct observables read
  int32_t col_obs[RF_MAXL];  // column slot -> observable index in the SoA
  int32_t coef_par[RF_MAXC]; // FRAC: K-1 fraction slots; EXT: K yield slots
  int32_t coef_free;         // bit c: gradient of coefficient c wanted
  uint64_t fixed_lo, fixed_hi;  // bit p: parameter p is fixed (grad = 0)
  double ext_weight;         // weight of the extended term sum(nu) and its
                             // gradient (1; 0 on all shards but one)
  double* formula_norm;      // device [RF_MAXL * RF_FORMULA_NV]: row k holds log I
                             // and (dI/dp_j)/I of the formula or Hypatia2 leaf in
                             // slot k; a Hypatia2 leaf's second row holds log phi
                             // and its derivatives in lambda and zeta.  Written
                             // by the normalisation kernel before the prologue
                             // reads them
  RfLeafProg leaf[RF_MAXL];
};

// Per-call constants, computed in FP64 from the parameter vector (prologue).
template <typename Real>
struct alignas(16) RfConsts {  // 16-byte multiple: arrays of it are bulk-copied
  Real pc[RF_MAXL][RF_PC];     // per-leaf evaluation constants
  Real delta[RF_MAXC];         // delta_c rounded to Real (-inf: coef_c == 0)
  Real delta_nc[RF_MAXC];      // delta_c - log coef_c (used when coef_c == 0)
  double beta_ref;
  double lnI[RF_MAXL];         // log I_k - off_k
  double delta_lo[RF_MAXC];    // delta_c - (double)delta[c]
  double dlogI[RF_MAXL][RF_LEAF_MAXP];   // d(log I_k - off_k)/d theta_kj
  double dtheta[RF_MAXL][RF_LEAF_MAXP];  // theta used per event - theta
  double gmul[RF_MAXL][RF_LEAF_MAXP];    // d u/d theta = gmul * (per-event factor)
  double coef[RF_MAXC];
  double ext_sum;              // sum of yields (extended) else 0
  int32_t zero_mask;           // bit c: coef_c == 0
  int32_t bad;                 // parameter outside its definition range
};

// FP32 evaluation of a call (or toy) with a coefficient exactly 0 evaluates
// every event in FP64 (the absent component's P_c/P grows without bound in
// the tails of the others, beyond what FP32 log-densities resolve): the
// per-event constants and the deltas in FP64, and each leaf's form.  Written
// by the prologues only for such calls.
struct alignas(16) RfExact {
  double pcd[RF_MAXL][RF_PC];  // pc in FP64 (hi + lo pairs as (value, 0))
  double delta_d[RF_MAXC];     // delta_c in base-2 units (-inf: coef_c == 0)
  double delta_nc_d[RF_MAXC];  // (delta_c - log coef_c) in base-2 units
  int32_t lmeta[RF_MAXL];      // type | gmask << 8 | comp << 16 | col << 24
  int32_t n_comp;
  int32_t zero_mask;
};

// Device workspace owned by an rf_graph.
struct RfWork {
  double* partials;        // [rows * RF_NACC_MAX]: block rows and group rows
                           // (single dataset) or segment partials (toys)
  unsigned int* counter;   // [RF_COUNTER_WORDS] tickets (single dataset)
  unsigned int* status;    // [1] RF_STATUS_* bits
  // batched mode
  void* toy_consts;        // [max_toys] RfConsts<Real>
  double* adam_m1;         // [max_toys * n_par]
  double* adam_m2;
  int32_t* adam_t;         // [1] step counter
  // single dataset: constants from the separate prologue kernel (NULL: each
  // block computes them itself)
  void* consts;            // [1] RfConsts<Real>
  RfExact* consts_x;       // [1] (single dataset) FP64 constants of a
                           // zero-coefficient call with FP32 evaluation
  RfExact* toy_consts_x;   // [max_toys] the same per toy
};

struct RfLaunchCfg {
  int block;
  int ept;
  int blocks_per_sm;
  int min_blocks;  // register budget of the specialised fused kernel (2..4)
};

#ifndef __CUDACC_RTC__
// ---- launchers (defined in the .cu files) -------------------------------
// All return a cudaError_t value (0 = success).  `stream` is a cudaStream_t.
typedef struct CUstream_st* rf_cuda_stream;
#define RF_DECL_FUSED(R, C)                                                      \
  int rf_fused_##R##_##C(const RfProgram&, const RfLaunchCfg&, int, const void*, \
                         int64_t, const double*, RfWork, double*, double*,       \
                         rf_cuda_stream);                                         \
  int rf_logp_##R##_##C(const RfProgram&, const void*, int64_t, const double*,   \
                        double*, rf_cuda_stream);
RF_DECL_FUSED(f32, c32)
RF_DECL_FUSED(f32, c64)
RF_DECL_FUSED(f64, c32)
RF_DECL_FUSED(f64, c64)

// FP64 prologue kernel for the single-dataset path: one block, one warp per
// leaf; writes W.consts.  With chain, launched as a programmatic dependent of
// the previous kernel in the stream (its FP64 work overlaps that kernel's
// end; without chain it starts after it, as it must after the normalisation
// kernel of formula leaves whose results it reads); either way it lets its
// own dependent (the fused kernel) launch at once.
int rf_launch_prologue(const RfProgram& P, int eval, const double* params, RfWork W,
                       bool chain, rf_cuda_stream st);

// Toy studies: prep kernel (per-toy FP64 constants), segment kernel (events
// split evenly over the launch's warps), finalize kernel (one warp per toy:
// fixed-order sum of its segments, epilogue, optional Adam step).
int rf_launch_batched(const RfProgram& P, int eval, int coldt,
                      const RfLaunchCfg& cfg, int num_sms, const void* events,
                      int64_t n_events, const int64_t* offsets, int32_t toys,
                      double* pm, double* out, RfWork W,
                      const double* adam_scale, double adam_lr,
                      int64_t max_rows, struct CUkern_st* jit_toys, bool bulk, void* stream,
                      int* launches);
// toy generation (k_generate.cu)
int rf_launch_generate(const RfProgram& P, int coldt, const double* params_matrix,
                       const int64_t* comp_counts, const int64_t* offsets, int32_t toys,
                       unsigned long long seed, void* events, int64_t n_events,
                       unsigned int* status, int num_sms, rf_cuda_stream st);
// FP64 -> FP32 (round to nearest) of n values, for the toy columns of an
// FP32-evaluated graph (converted once at bind time)
int rf_columns_to_f32(const double* in, float* out, int64_t n, void* stream);
int rf_launch_plain(const RfProgram& prog, int coldt, const void* events,
                    int64_t n, const double* params, double* node_buf,
                    double* nll, double* grad, double* partials,
                    unsigned int* counter, void* stream, int* launches);
size_t rf_plain_bytes(const RfProgram& prog, int64_t n);
int rf_run_microbench(double* out);
int rf_run_check_d2f(const double* x, float* y_fast, float* y_ref, int64_t n, rf_cuda_stream st);
int rf_run_check_log(const float* x, float* y_fast, float* y_ref, int64_t n, rf_cuda_stream st);
size_t rf_consts_size(int eval);

// vector-load plan shared by the generic and specialised launchers
// (rf_launch.cpp): vec = every column read starts at the same 16-byte phase;
// head = events before the first aligned one.
void rf_vec_plan(const RfProgram& P, const void* events, int64_t stride, int elem_bytes,
                 int* vec, int64_t* head);

// per-graph specialised kernels (jit.cpp)
#include <string>
#include <vector>
// toy segment kernel: register streaming (RF_JIT_TOYS) or bulk-copy stage
// rings (RF_JIT_TOYS_BULK)
// RF_JIT_NORM: the FP64 normalisation kernel of a graph's formula leaves
enum { RF_JIT_FUSED = 0, RF_JIT_TOYS = 1, RF_JIT_LOGP = 2, RF_JIT_TOYS_BULK = 3, RF_JIT_NORM = 4 };
// CUDA text of each formula leaf (rf_expr_translate), empty for the others
struct RfFormulaCode {
  std::string leaf[RF_MAXL];
};
bool rf_expr_translate(const char* text, int npar, std::string* code, std::string* err);
void rf_gauss_legendre16(double* t, double* w);
typedef struct CUkern_st* rf_cuda_kernel;  // == cudaKernel_t
// min_blocks: launch bounds of the fused and toy kernels (resident blocks of 256
// threads per SM; 0 for the toy kernel: none); the log P kernel ignores it
// fc: the graph's formula-leaf code (NULL without formula leaves)
std::string rf_jit_source(const RfProgram& P, const RfFormulaCode* fc, int eval, int coldt,
                          int kind, int ept, int min_blocks);
uint64_t rf_jit_hash(const RfProgram& P, const RfFormulaCode* fc, int eval, int coldt, int kind,
                     int ept, int min_blocks);
bool rf_jit_compile_only(const RfProgram& P, const RfFormulaCode* fc, int eval, int coldt,
                         int kind, int ept, int min_blocks, std::string* err);
rf_cuda_kernel rf_jit_kernel(const RfProgram& P, const RfFormulaCode* fc, int eval, int coldt,
                             int kind, int ept, int min_blocks, int* regs, std::string* err);
// on-disk cache folder (RF_JIT_CACHE_DIR, else $TMPDIR/rfgpu-jit) and the
// FNV-1a hash its file names use
std::string rf_cache_dir();
uint64_t rf_text_hash(const std::string& s);
// compiles the sources not yet in the on-disk cache, in parallel threads
void rf_jit_precompile(const std::vector<std::string>& sources);
// normalisation kernel of the formula leaves (grid RF_FORMULA_BLOCKS x leaves)
int rf_jit_launch_norm(rf_cuda_kernel k, const RfProgram& P, int n_formula,
                       const double* params, double* part, unsigned int* ticket,
                       rf_cuda_stream st);
int rf_jit_launch_fused(rf_cuda_kernel k, const RfProgram& P, int coldt, const RfLaunchCfg& cfg,
                        int num_sms, const void* events, int64_t n, const double* params,
                        RfWork W, double* nll, double* grad, rf_cuda_stream st);
// segment kernel of a toy study, as a programmatic dependent of the prep
// kernel launched just before it
int rf_jit_launch_toys(rf_cuda_kernel k, const RfProgram& P, int grid, int block, int vec,
                       int stages, size_t smem, const void* events, int64_t n_events,
                       const int64_t* offsets, int32_t toys, RfWork W, rf_cuda_stream st);
int rf_jit_launch_logp(rf_cuda_kernel k, const RfProgram& P, const void* events, int64_t n,
                       const double* params, double* logp, rf_cuda_stream st);
#endif  // __CUDACC_RTC__
