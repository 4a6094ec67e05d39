// noalloc.cu -- rf_nll_noalloc: the NLL and gradient of one dataset for
// callers that cannot allocate device memory at all.
//
// Some callers cannot call cudaMalloc: code running inside a host callback or
// a driver-level hook, real-time loops whose allocator is locked after start-
// up, or hosts whose memory pool is owned by another framework.  They cannot
// build an rf_graph either, because rf_graph_compile allocates the graph's
// workspace.  This entry point takes the descriptor directly, evaluates it with
// the precompiled generic fused kernel, and gives that kernel its scratch --
// the per-block and per-group partial sums, the tickets and the status word -- from a
// file-scope static device array instead of an allocation.
//
// The array (kBytes, 256 KiB) is part of this library's device
// image: every GPU that loads the library holds it until the process exits.
// Every call shares it and it keeps the last call's contents, so calls that
// overlap on the GPU (two streams, or two threads on one stream without
// ordering) race on it; the ticket and status words are cleared on the
// caller's stream at the start of each call.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/rf.h"
#include "rf_internal.h"

rf_status rf_canonical_program(const rf_graph_desc* desc, RfProgram* P);
void rf_set_last_error(const char* msg);

namespace {

constexpr int kMaxBlocks = RF_NOALLOC_MAX_BLOCKS;
// ticket and status words (RF_COUNTER_WORDS), then the rows of the grid's
// FP64 tree: one per block and one per group
constexpr size_t kHeader = 256;
static_assert(kHeader >= RF_COUNTER_WORDS * sizeof(unsigned int), "ticket words");
constexpr size_t kBytes =
    kHeader + sizeof(double) * RF_NACC_MAX * (size_t)(kMaxBlocks + RF_TREE_GROUPS);

// The scratch.  In host code this name is only a stand-in for the device
// symbol; its device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_scratch[kBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {nullptr};
int g_sms[kMaxDevices] = {0};

// Once per device, with that device current: the scratch's device address
// and the SM count.  Returns 0 or a cudaError_t value.
int setup(int dev, void** addr, int* sms) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess) return (int)e;
    int n = 0;
    e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return (int)e;
    g_sms[dev] = n;
    g_addr[dev] = p;
  }
  *addr = g_addr[dev];
  *sms = g_sms[dev];
  return 0;
}

}  // namespace

extern "C" rf_status rf_nll_noalloc(const rf_graph_desc* desc, const void* events,
                                    int64_t n_events, const double* params, double* nll,
                                    double* grad, int32_t blocks, rf_stream stream) {
  RfProgram P;
  rf_status s = rf_canonical_program(desc, &P);
  if (s) return s;
  if (n_events < 0 || (n_events > 0 && !events) || !nll || (!params && P.n_par > 0)) {
    rf_set_last_error("rf_nll_noalloc: NULL or negative argument");
    return RF_EINVAL;
  }
  const int elem = desc->column_dtype == RF_F64 ? 8 : 4;
  if (reinterpret_cast<uintptr_t>(events) % (uintptr_t)elem) {
    rf_set_last_error("rf_nll_noalloc: event columns are not aligned to their element size");
    return RF_EALIGN;
  }
  if (blocks < 0 || blocks > kMaxBlocks) {
    rf_set_last_error("rf_nll_noalloc: blocks must be in 0..1024 (the static scratch holds the "
                      "partial sums of at most 1024 blocks)");
    return RF_EINVAL;
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    rf_set_last_error("rf_nll_noalloc: no usable current device");
    return RF_ECUDA;
  }
  void* base = nullptr;
  int sms = 0;
  int se = setup(dev, &base, &sms);
  if (se) {
    rf_set_last_error("rf_nll_noalloc: cudaGetSymbolAddress of the static scratch failed");
    return RF_ECUDA;
  }
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  unsigned int* words = static_cast<unsigned int*>(base);
  // tickets and status start at 0
  e = cudaMemsetAsync(words, 0, RF_COUNTER_WORDS * sizeof(unsigned int), st);
  if (e != cudaSuccess) {
    rf_set_last_error("rf_nll_noalloc: clearing the ticket failed");
    return RF_ECUDA;
  }
  RfWork W{};
  W.counter = words;
  W.status = words + 1;
  W.partials = reinterpret_cast<double*>(static_cast<unsigned char*>(base) + kHeader);
  if (blocks == 0) blocks = sms * 2 < kMaxBlocks ? sms * 2 : kMaxBlocks;
  // grid = min(ceil(chunks / block), blocks): launch with "SM count" = blocks, 1 per SM
  RfLaunchCfg cfg;
  cfg.block = 256;
  cfg.blocks_per_sm = 1;
  cfg.min_blocks = 2;  // not used by the generic kernels
  int le;
  if (desc->eval_precision == RF_EVAL_FP32) {
    cfg.ept = 4;
    le = desc->column_dtype == RF_F32
             ? rf_fused_f32_c32(P, cfg, blocks, events, n_events, params, W, nll, grad, st)
             : rf_fused_f32_c64(P, cfg, blocks, events, n_events, params, W, nll, grad, st);
  } else {
    cfg.ept = desc->column_dtype == RF_F64 ? 2 : 4;
    le = desc->column_dtype == RF_F32
             ? rf_fused_f64_c32(P, cfg, blocks, events, n_events, params, W, nll, grad, st)
             : rf_fused_f64_c64(P, cfg, blocks, events, n_events, params, W, nll, grad, st);
  }
  if (le) {
    rf_set_last_error("rf_nll_noalloc: kernel launch failed");
    return RF_ECUDA;
  }
  return RF_OK;
}
