// jit.cpp -- per-graph specialisation of the fused kernels.
//
// rf_graph_compile turns the graph into a small Model struct in which the leaf
// types, the column each leaf reads, the component sums and the gradient
// masks are compile-time constants, appends it to the library's own device
// headers (rf_internal.h, rf_device.cuh, rf_kernels.cuh, embedded at build
// time), and compiles the fused, toy-tile and log P kernels for sm_103a with
// NVRTC.  The per-event code then has no run-time dispatch and computes only
// the derivatives that are needed.  Compiled modules are cached for the
// process by their source text and device.  The paper's own just-in-time path
// (Sec. 4: formula PDFs compiled by cling) motivates the form; here the
// compiler specialises the built-in PDFs of one graph.
#include <cuda_runtime.h>
#include <nvrtc.h>

#include <sys/stat.h>
#include <unistd.h>

#include <cstdio>
#include <cstdlib>
#include <map>
#include <memory>
#include <mutex>
#include <sstream>
#include <atomic>
#include <string>
#include <thread>
#include <vector>

#include "rf_internal.h"
#include "rf_jit_prelude.inc"  // kRfJitPrelude, kRfJitToysPrelude, kRfJitFormulaPrelude:
                               // device headers as text

namespace {

std::mutex g_mu;
std::map<std::string, cudaKernel_t> g_cache;      // (device | source) -> kernel
std::vector<cudaLibrary_t> g_libs;                // kept loaded for the process

const char* leaf_fn(int type) {
  switch (type) {
    case RFL_GAUSS: return "leaf_gauss";
    case RFL_EXP: return "leaf_exp";
    case RFL_CHEB: return "leaf_cheb";
    case RFL_CB: return "leaf_cb";
    case RFL_ARGUS: return "leaf_argus";
    case RFL_JOHNSON: return "leaf_johnson";
  }
  return nullptr;
}

// The leaf function's compile-time mask: the gradient bits, and for an
// Exponential whose range starts at 0 the form without the shift
int leaf_gm(const RfLeafProg& L) {
  return L.gmask | ((L.type == RFL_EXP && L.lo == 0.0) ? RF_GM_AT0 : 0);
}

// FNV-1a, for the on-disk cache file name
uint64_t fnv1a(const std::string& s) {
  uint64_t h = 1469598103934665603ull;
  for (unsigned char c : s) {
    h ^= c;
    h *= 1099511628211ull;
  }
  return h;
}

std::string cache_dir() {
  if (const char* d = getenv("RF_JIT_CACHE_DIR")) return d;
  const char* tmp = getenv("TMPDIR");
  return std::string(tmp ? tmp : "/tmp") + "/rfgpu-jit";
}

}  // namespace

namespace {

// leaves normalised numerically (formula and Hypatia2 leaves): they need the
// device header of formula leaves and the normalisation kernel
bool has_formula(const RfProgram& P) {
  for (int k = 0; k < P.n_leaves; ++k)
    if (P.leaf[k].type == RFL_FORMULA || P.leaf[k].type == RFL_HYPATIA2) return true;
  return false;
}

// derivatives a leaf returns per event (Hypatia2: nine, over its slots)
int leaf_nder(const RfLeafProg& L) { return L.type == RFL_HYPATIA2 ? 9 : RF_LEAF_MAXP; }

// whether the derivative j of leaf k is wanted (j >= 4: the next slots')
bool wants(const RfProgram& P, int k, int j) {
  return (P.leaf[k + j / RF_LEAF_MAXP].gmask >> (j % RF_LEAF_MAXP)) & 1;
}

// the per-event call of leaf k in type R on constants `pc` (empty for a slot
// that only holds parameters of the leaf before)
std::string leaf_call(const RfProgram& P, int k, const char* R, const std::string& pc,
                      const std::string& add) {
  const RfLeafProg& L = P.leaf[k];
  if (L.type == RFL_PARAMS) return std::string();
  std::ostringstream o;
  const std::string ks = std::to_string(k);
  o << "    " << R << " u" << ks << ", g" << ks << "[" << leaf_nder(L) << "];\n    ";
  if (L.type == RFL_FORMULA) {
    o << "rf::formula_leaf<RfFormula" << ks << ", " << R << ", " << L.gmask << ">";
  } else if (L.type == RFL_HYPATIA2) {
    int gm9 = 0;
    for (int j = 0; j < 9; ++j)
      if (wants(P, k, j)) gm9 |= 1 << j;
    o << "rf::hypatia2_leaf<" << R << ", " << gm9 << ">";
  } else {
    o << "rf::" << leaf_fn(L.type) << "<" << R << ", " << leaf_gm(L) << ">";
  }
  o << "(x[" << L.col << "], " << pc << ", u" << ks << ", g" << ks;
  if (!add.empty()) o << ", " << add;
  o << ");\n";
  return o.str();
}

// One struct per formula leaf k: NP and eval<Real>(x, p) -> Dual<Real, NP'>
// (the translated text over the leaf's parameters as duals).
void emit_formulas(std::ostringstream& o, const RfProgram& P, const RfFormulaCode* fc) {
  o << kRfJitFormulaPrelude << "\n";
  for (int k = 0; k < P.n_leaves; ++k) {
    const RfLeafProg& L = P.leaf[k];
    if (L.type != RFL_FORMULA) continue;
    const int np = L.npar, nd = np > 0 ? np : 1;
    o << "struct RfFormula" << k << " {\n  static constexpr int NP = " << np << ";\n"
      << "  template <typename Real>\n  static __device__ __forceinline__ rf::Dual<Real, " << nd
      << "> eval(Real x, const Real* __restrict__ pc) {\n"
      << "    using D = rf::Dual<Real, " << nd << ">;\n";
    for (int j = 0; j < np; ++j)
      o << "    const D p" << j << " = D::var(pc[" << j << "], " << j << ");\n";
    o << "    (void)x;\n    (void)pc;\n"
      << "    return rf::as_dual<D>(" << (fc ? fc->leaf[k] : std::string("Real(1)")) << ");\n  }\n};\n";
  }
}

}  // namespace

std::string rf_jit_source(const RfProgram& P, const RfFormulaCode* fc, int eval, int coldt,
                          int kind, int ept, int min_blocks) {
  const int NL = P.n_leaves, NC = P.n_comp;
  unsigned long long amask = 1ull;  // ell
  for (int c = 0; c < NC; ++c) amask |= 1ull << (1 + c);
  for (int k = 0; k < NL; ++k)
    for (int j = 0; j < RF_LEAF_MAXP; ++j)
      if ((P.leaf[k].gmask >> j) & 1) amask |= 1ull << (1 + NL + k * RF_LEAF_MAXP + j);
  std::ostringstream o;
  o << kRfJitPrelude << "\n";
  if (has_formula(P)) emit_formulas(o, P, fc);
  if (kind == RF_JIT_NORM) {
    // FP64 normalisation of the formula leaves: blockIdx.y = formula number
    double t[16], w[16];
    rf_gauss_legendre16(t, w);
    char buf[64];
    o << "__device__ const double kRfGlT[16] = {";
    for (int i = 0; i < 16; ++i) {
      snprintf(buf, sizeof(buf), "%a%s", t[i], i < 15 ? ", " : "};\n");
      o << buf;
    }
    o << "__device__ const double kRfGlW[16] = {";
    for (int i = 0; i < 16; ++i) {
      snprintf(buf, sizeof(buf), "%a%s", w[i], i < 15 ? ", " : "};\n");
      o << buf;
    }
    o << "extern \"C\" __global__ void __launch_bounds__(128) rf_norm_jit(const RfProgram P, "
         "const double* __restrict__ params, double* part, unsigned int* ticket) {\n"
         "  switch (blockIdx.y) {\n";
    int f = 0;
    for (int k = 0; k < NL; ++k)
      if (P.leaf[k].type == RFL_FORMULA || P.leaf[k].type == RFL_HYPATIA2)
        o << "    case " << f++ << ": rf::formula_norm_body<"
          << (P.leaf[k].type == RFL_HYPATIA2 ? std::string("rf::Hypatia2Leaf")
                                              : "RfFormula" + std::to_string(k))
          << ">(P, " << k << ", params, kRfGlT, kRfGlW, part, ticket, P.formula_norm); break;\n";
    o << "  }\n}\n";
    return o.str();
  }
  o << "// ---- model emitted for this graph\n";
  o << "struct RfModel {\n  static constexpr int NL_ = " << NL << ";\n"
    << "  static constexpr int NCOL = " << P.n_cols << ";\n"
    << "  static constexpr unsigned long long AMASK = " << amask << "ull;\n"
    << "  template <typename Real, bool ANYZERO = true>\n  static __device__ __forceinline__ void "
       "event(const RfProgram& P, "
       "const rf::EvalConsts<Real, NL_>& K, const Real (&x)[NL_], Real (&q)[RF_NACC(NL_)]) {\n";
  // Without a zero coefficient (ANYZERO false) each component's delta is
  // added inside its first leaf (folded into a constant or an FMA there);
  // otherwise the leaves return the bare log-densities and delta / delta_nc
  // are added here.
  std::vector<int> first(NC, -1);
  for (int k = 0; k < NL; ++k)
    if (first[P.leaf[k].comp] < 0) first[P.leaf[k].comp] = k;
  for (int k = 0; k < NL; ++k)
    o << leaf_call(P, k, "Real", "K.pc[" + std::to_string(k) + "]",
                   first[P.leaf[k].comp] == k
                       ? "ANYZERO ? Real(-0.0) : K.delta[" + std::to_string(P.leaf[k].comp) + "]"
                       : std::string());
  o << "    Real v[" << NC << "], w[" << NC << "];\n";
  std::vector<std::string> usum(NC);
  for (int c = 0; c < NC; ++c) {
    std::string s;
    for (int k = 0; k < NL; ++k)
      if (P.leaf[k].comp == c && P.leaf[k].type != RFL_PARAMS)
        s += (s.empty() ? "u" : " + u") + std::to_string(k);
    usum[c] = " + " + s;
    o << "    if constexpr (ANYZERO) v[" << c << "] = K.delta[" << c << "] + " << s << ";\n"
      << "    else v[" << c << "] = " << s << ";\n";
  }
  o << "    const Real ell = rf::lse<Real, " << NC << ">(v, w);\n    q[0] += ell;\n";
  if (NC == 1) {
    o << "    q[1] += Real(1);\n";
  } else {
    // common case first: no coefficient is exactly zero (one uniform branch)
    o << "    if (!ANYZERO || K.zero_mask == 0) {\n";
    for (int c = 0; c < NC; ++c) o << "      q[" << 1 + c << "] += w[" << c << "];\n";
    o << "    } else {\n";
    for (int c = 0; c < NC; ++c)
      o << "      q[" << 1 + c << "] += rf::comp_weight<Real>(K.zero_mask, " << c
        << ", K.delta_nc[" << c << "]" << usum[c] << ", ell, w[" << c << "]);\n";
    o << "    }\n";
  }
  for (int k = 0; k < NL; ++k) {
    if (P.leaf[k].type == RFL_PARAMS) continue;
    for (int j = 0; j < leaf_nder(P.leaf[k]); ++j)
      if (wants(P, k, j))
        o << "    q[" << 1 + NL + k * RF_LEAF_MAXP + j << "] += w[" << P.leaf[k].comp << "] * g" << k
          << "[" << j << "];\n";
  }
  o << "  }\n";
  // The same event in FP64 on the FP64 constants, for FP32 evaluation of a
  // call or toy with a coefficient exactly 0 (x: the column values in their
  // own precision); returns log2 P - beta_ref / ln 2.
  o << "  static __device__ __noinline__ double event_exact(const RfExact* __restrict__ Kp, "
       "const double* __restrict__ x, float* __restrict__ q) {\n"
       "    const RfExact& K = *Kp;\n";
  for (int k = 0; k < NL; ++k)
    o << leaf_call(P, k, "double", "K.pcd[" + std::to_string(k) + "]", std::string());
  o << "    double v[" << NC << "], w[" << NC << "];\n";
  for (int c = 0; c < NC; ++c) o << "    v[" << c << "] = K.delta_d[" << c << "]" << usum[c] << ";\n";
  o << "    const double ell = rf::lse<double, " << NC << ">(v, w);\n    q[0] += (float)ell;\n";
  if (NC == 1) {
    o << "    q[1] += 1.0f;\n";
  } else {
    for (int c = 0; c < NC; ++c)
      o << "    q[" << 1 + c << "] += (float)(((K.zero_mask >> " << c << ") & 1) ? exp2(K.delta_nc_d["
        << c << "]" << usum[c] << " - ell) : w[" << c << "]);\n";
  }
  for (int k = 0; k < NL; ++k) {
    if (P.leaf[k].type == RFL_PARAMS) continue;
    for (int j = 0; j < leaf_nder(P.leaf[k]); ++j)
      if (wants(P, k, j))
        o << "    q[" << 1 + NL + k * RF_LEAF_MAXP + j << "] += (float)(w[" << P.leaf[k].comp
          << "] * g" << k << "[" << j << "]);\n";
  }
  o << "    return ell;\n  }\n};\n";
  const char* R = eval ? "double" : "float";
  const char* C = coldt ? "double" : "float";
  // The fused kernel is declared for min_blocks resident blocks of 256
  // threads per SM: a register budget of 80 (3 blocks) or 128 (2 blocks).
  // The best budget depends on the graph (the FP32 Crystal Ball + ARGUS
  // model runs 1.5% faster at 80 registers than at 93; the FP64 and the
  // three-observable models lose at 80), so it is a tuned launch parameter.
  // A fixed minimum also keeps ptxas's budget from depending on the rest of
  // the kernel (an FP64 tail once pulled the event loop to 80 registers
  // with spills).
  const std::string lb = "__launch_bounds__(256, " + std::to_string(min_blocks) + ")";
  if (kind == RF_JIT_FUSED) {
    o << "extern \"C\" __global__ void " << lb << " rf_fused_jit(const RfProgram P, const "
      << C << "* __restrict__ ev, int64_t n, int64_t head, int vec, const double* __restrict__ "
              "params, RfWork W, double* nll, double* grad) {\n  rf::fused_body<RfModel, "
      << R << ", " << C << ", " << ept << ">(P, ev, n, head, vec, params, W, nll, grad);\n}\n";
  } else if (kind == RF_JIT_TOYS || kind == RF_JIT_TOYS_BULK) {
    o << kRfJitToysPrelude << "\n";
    // min_blocks > 0: launch bounds for that many resident blocks of 256
    const std::string tlb = min_blocks > 0 ? "__launch_bounds__(256, " + std::to_string(min_blocks) + ")"
                                           : std::string("__launch_bounds__(256)");
    o << "extern \"C\" __global__ void " << tlb << " rf_toys_jit(const RfProgram P, const "
      << C << "* __restrict__ ev, int64_t stride, int vec, const int64_t* __restrict__ offsets, "
              "int32_t toys, int stages, RfWork W) {\n  rf::"
      << (kind == RF_JIT_TOYS ? "toy_segment_body_reg" : "toy_segment_body") << "<RfModel, "
      << R << ", " << C << ", " << ept << ">(P, ev, stride, vec, offsets, toys, stages, W);\n}\n";
  } else {
    o << "extern \"C\" __global__ void __launch_bounds__(256) rf_logp_jit(const RfProgram P, const "
      << C << "* __restrict__ ev, int64_t n, const double* __restrict__ params, double* logp) {\n"
              "  rf::logp_body<RfModel, "
      << R << ", " << C << ">(P, ev, n, params, logp);\n}\n";
  }
  return o.str();
}

// NVRTC: source -> cubin for sm_103a (no device needed).
static bool compile_cubin(const std::string& src, std::vector<char>* cubin, std::string* err) {
  if (const char* dump = getenv("RF_JIT_DUMP")) {  // write the emitted source for inspection
    std::string path = std::string(dump) + "." + std::to_string(fnv1a(src) & 0xffff) + ".cu";
    if (FILE* f = fopen(path.c_str(), "w")) {
      fputs(src.c_str(), f);
      fclose(f);
    }
  }
  nvrtcProgram prog;
  if (nvrtcCreateProgram(&prog, src.c_str(), "rf_graph.cu", 0, nullptr, nullptr) != NVRTC_SUCCESS) {
    *err = "nvrtcCreateProgram failed";
    return false;
  }
  const char* opts[] = {"--gpu-architecture=sm_103a", "--std=c++17", "-lineinfo", "-DRF_JIT=1"};
  nvrtcResult r = nvrtcCompileProgram(prog, 4, opts);
  size_t log_size = 0;
  nvrtcGetProgramLogSize(prog, &log_size);
  std::string log(log_size, '\0');
  if (log_size) nvrtcGetProgramLog(prog, &log[0]);
  if (getenv("RF_JIT_VERBOSE")) fprintf(stderr, "[rf jit] %s\n", log.c_str());
  if (r != NVRTC_SUCCESS) {
    *err = std::string("NVRTC: ") + nvrtcGetErrorString(r) + "\n" + log;
    nvrtcDestroyProgram(&prog);
    return false;
  }
  size_t cubin_size = 0;
  nvrtcGetCUBINSize(prog, &cubin_size);
  cubin->resize(cubin_size);
  nvrtcGetCUBIN(prog, cubin->data());
  nvrtcDestroyProgram(&prog);
  return true;
}

namespace {

std::string cubin_path(const std::string& src) {
  char name[64];
  snprintf(name, sizeof(name), "/%016llx.cubin", (unsigned long long)fnv1a(src + "|sm_103a|v11"));
  return cache_dir() + name;
}

// written under a temporary name and renamed, so readers never see a partial file
void store_cubin(const std::string& path, const std::vector<char>& cubin) {
  mkdir(cache_dir().c_str(), 0700);
  static std::atomic<unsigned> seq{0};
  const std::string tmp = path + "." + std::to_string(getpid()) + "." + std::to_string(seq++);
  if (FILE* f = fopen(tmp.c_str(), "wb")) {
    const bool ok = fwrite(cubin.data(), 1, cubin.size(), f) == cubin.size();
    fclose(f);
    if (ok) rename(tmp.c_str(), path.c_str());
    else remove(tmp.c_str());
  }
}

}  // namespace

void rf_jit_precompile(const std::vector<std::string>& sources) {
  std::vector<std::thread> th;
  for (const std::string& src : sources) {
    const std::string path = cubin_path(src);
    if (access(path.c_str(), R_OK) == 0) continue;
    th.emplace_back([src, path] {
      std::vector<char> cubin;
      std::string err;  // a failure here is reported by the compile that follows
      if (compile_cubin(src, &cubin, &err)) store_cubin(path, cubin);
    });
  }
  for (std::thread& t : th) t.join();
}

std::string rf_cache_dir() { return cache_dir(); }

uint64_t rf_text_hash(const std::string& s) { return fnv1a(s); }

uint64_t rf_jit_hash(const RfProgram& P, const RfFormulaCode* fc, int eval, int coldt, int kind,
                     int ept, int min_blocks) {
  return fnv1a(rf_jit_source(P, fc, eval, coldt, kind, ept, min_blocks));
}

bool rf_jit_compile_only(const RfProgram& P, const RfFormulaCode* fc, int eval, int coldt,
                         int kind, int ept, int min_blocks, std::string* err) {
  std::vector<char> cubin;
  return compile_cubin(rf_jit_source(P, fc, eval, coldt, kind, ept, min_blocks), &cubin, err);
}

// The kernel of the given kind specialised for P: from the process cache, else
// from the on-disk cache, else compiled with NVRTC (and written to disk).
// Host-synchronous; returns nullptr and fills *err on failure.
cudaKernel_t rf_jit_kernel(const RfProgram& P, const RfFormulaCode* fc, int eval, int coldt,
                           int kind, int ept, int min_blocks, int* regs, std::string* err) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    *err = "no current device";
    return nullptr;
  }
  std::string src = rf_jit_source(P, fc, eval, coldt, kind, ept, min_blocks);
  std::string key = std::to_string(dev) + "|" + src;
  std::lock_guard<std::mutex> lk(g_mu);
  auto it = g_cache.find(key);
  cudaKernel_t k = nullptr;
  if (it != g_cache.end()) {
    k = it->second;
  } else {
    const std::string path = cubin_path(src);
    std::vector<char> cubin;
    if (FILE* f = fopen(path.c_str(), "rb")) {
      fseek(f, 0, SEEK_END);
      long sz = ftell(f);
      fseek(f, 0, SEEK_SET);
      if (sz > 0) {
        cubin.resize((size_t)sz);
        if (fread(cubin.data(), 1, (size_t)sz, f) != (size_t)sz) cubin.clear();
      }
      fclose(f);
    }
    if (cubin.empty()) {
      if (!compile_cubin(src, &cubin, err)) return nullptr;
      store_cubin(path, cubin);
    }
    cudaLibrary_t lib = nullptr;
    cudaError_t e = cudaLibraryLoadData(&lib, cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0);
    if (e != cudaSuccess) {
      *err = std::string("cudaLibraryLoadData: ") + cudaGetErrorString(e);
      return nullptr;
    }
    const char* kname = kind == RF_JIT_FUSED ? "rf_fused_jit"
                        : (kind == RF_JIT_TOYS || kind == RF_JIT_TOYS_BULK) ? "rf_toys_jit"
                        : kind == RF_JIT_NORM ? "rf_norm_jit" : "rf_logp_jit";
    e = cudaLibraryGetKernel(&k, lib, kname);
    if (e != cudaSuccess) {
      *err = std::string("cudaLibraryGetKernel: ") + cudaGetErrorString(e);
      cudaLibraryUnload(lib);
      return nullptr;
    }
    g_libs.push_back(lib);
    g_cache[key] = k;
  }
  if (regs) {
    cudaFuncAttributes a;
    *regs = cudaFuncGetAttributes(&a, reinterpret_cast<const void*>(k)) == cudaSuccess ? a.numRegs : 0;
  }
  return k;
}

int rf_jit_launch_fused(cudaKernel_t k, const RfProgram& P, int coldt, const RfLaunchCfg& cfg,
                        int num_sms, const void* events, int64_t n, const double* params,
                        RfWork W, double* nll, double* grad, cudaStream_t st) {
  int vec = 0;
  int64_t head = 0;
  rf_vec_plan(P, events, n, coldt ? 8 : 4, &vec, &head);
  int64_t chunks = n / cfg.ept;
  int64_t want = (chunks + cfg.block - 1) / cfg.block;
  int64_t cap = (int64_t)num_sms * cfg.blocks_per_sm;
  int grid = (int)(want < 1 ? 1 : (want > cap ? cap : want));
  RfProgram Pc = P;
  const void* ev = events;
  void* args[] = {&Pc, &ev, &n, &head, &vec, &params, &W, &nll, &grad};
  cudaLaunchConfig_t lc = {};
  lc.gridDim = dim3(grid);
  lc.blockDim = dim3(cfg.block);
  lc.stream = st;
  cudaLaunchAttribute at[1];
  if (W.consts) {  // dependent of the prologue kernel launched just before
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    lc.attrs = at;
    lc.numAttrs = 1;
  }
  return (int)cudaLaunchKernelExC(&lc, reinterpret_cast<const void*>(k), args);
}

int rf_jit_launch_toys(cudaKernel_t k, const RfProgram& P, int grid, int block, int vec,
                       int stages, size_t smem, const void* events, int64_t n_events,
                       const int64_t* offsets, int32_t toys, RfWork W, cudaStream_t st) {
  RfProgram Pc = P;
  const void* ev = events;
  int64_t stride = n_events;
  void* args[] = {&Pc, &ev, &stride, &vec, &offsets, &toys, &stages, &W};
  cudaLaunchConfig_t lc = {};
  lc.gridDim = dim3(grid);
  lc.blockDim = dim3(block);
  lc.dynamicSmemBytes = smem;
  lc.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  lc.attrs = at;
  lc.numAttrs = 1;
  return (int)cudaLaunchKernelExC(&lc, reinterpret_cast<const void*>(k), args);
}

int rf_jit_launch_norm(cudaKernel_t k, const RfProgram& P, int n_formula, const double* params,
                       double* part, unsigned int* ticket, cudaStream_t st) {
  RfProgram Pc = P;
  void* args[] = {&Pc, &params, &part, &ticket};
  // a programmatic dependent of the kernel before it (as the prologue is);
  // the prologue after it waits for it before reading the integrals
  cudaLaunchConfig_t lc = {};
  lc.gridDim = dim3(RF_FORMULA_BLOCKS, n_formula);
  lc.blockDim = dim3(128);
  lc.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  lc.attrs = at;
  lc.numAttrs = 1;
  return (int)cudaLaunchKernelExC(&lc, reinterpret_cast<const void*>(k), args);
}

int rf_jit_launch_logp(cudaKernel_t k, const RfProgram& P, const void* events, int64_t n,
                       const double* params, double* logp, cudaStream_t st) {
  int64_t g = (n + 255) / 256;
  int grid = (int)(g < 1 ? 1 : (g > 65535 * 8 ? 65535 * 8 : g));
  RfProgram Pc = P;
  const void* ev = events;
  void* args[] = {&Pc, &ev, &n, &params, &logp};
  return (int)cudaLaunchKernel(reinterpret_cast<const void*>(k), dim3(grid), dim3(256), args, 0,
                               st);
}
