/*
 * rf.h -- C-ABI of librfgpu: the unbinned negative log-likelihood (NLL) of a
 * PDF computation graph and its gradient, evaluated on one GB300 GPU.
 *
 * What is computed (Hageboeck, "A Faster, More Intuitive RooFit", Sec. 5.1):
 * for every dataset entry the probability of the top node of a graph whose
 * leaves are PDFs of the entry's observables, normalised by their analytic
 * integrals over the observable ranges (Sec. 3, "Analytic Integrals");
 * NLL = -sum_i log P(x_i).  The graph is compiled once (parameter-only
 * branches -- normalisations, coefficients -- are hoisted out of the event
 * loop, as the paper's constant branches are computed once, Sec. 5.1), and one
 * fused kernel streams the event columns and produces the NLL and its
 * gradient in the same pass.  The batch interface of Sec. 5.2 (contiguous
 * arrays in, node-owned contiguous arrays out) is kept as the plain FP64
 * node-by-node baseline, rf_nll_plain.
 *
 * Leaves (parameter order in rf_node_desc.params):
 *   RF_GAUSS  (mu, sigma)            exp(-(x-mu)^2/(2 sigma^2))
 *   RF_EXP    (lambda)               exp(lambda x)
 *   RF_CHEB   (c_1..c_m), m <= 4     1 + sum_j c_j T_j(x'), x' = (2x-lo-hi)/(hi-lo)
 *   RF_CB     (m0, sigma, alpha, n)  Crystal Ball; alpha > 0: tail below m0
 *   RF_ARGUS  (m0, c, p)             x tau^p exp(c tau), tau = 1-(x/m0)^2, x < m0;
 *             p = 1/2 has a one-log form and a closed-form integral; any other
 *             p > 0 takes the general form (two logs per event; the integral
 *             and d/dp from positive-term series of the incomplete gamma
 *             function).  A free p always takes the general form; a fixed p
 *             takes it when rf_graph_desc.param_values gives it a value other
 *             than 1/2 (without values, a fixed p must be 1/2).  Toy
 *             generation draws p = 1/2 only
 *   RF_JOHNSON (mu, lambda, gamma, delta)  Johnson's SU (Sec. 3): with
 *             z = (x-mu)/lambda, w = gamma + delta asinh z standard normal:
 *             delta / (lambda sqrt(2 pi (1+z^2))) exp(-w^2/2)
 *   RF_HYPATIA2 (lambda, zeta, beta, sigma, mu, a, n, a2, n2)  Hypatia2
 *             (Sec. 3): with d = x - mu, phi = K_{lambda+1}(zeta)/K_lambda(zeta),
 *             delta = sigma sqrt(zeta/phi), alpha = sqrt(zeta phi)/sigma, a
 *             generalised hyperbolic core
 *               (d^2 + delta^2)^((lambda - 1/2)/2) e^{beta d}
 *               K_{lambda-1/2}(alpha sqrt(d^2 + delta^2))
 *             for -a sigma <= d <= a2 sigma and power-law tails beyond,
 *             f(d_J) (1 - (d - d_J) k_J / m)^-m with the core's value and
 *             logarithmic slope k_J at the junction d_J (m = n below, n2
 *             above).  K_nu of real order by the trapezoid rule on its
 *             integral representation; the integral over the range and its
 *             derivatives numerically in FP64 (as for formula leaves, the
 *             panels split at the junctions); zeta, sigma, a, n, a2, n2 must
 *             be positive.  Takes three of the graph's six leaf slots;
 *             specialised kernels only, no toy studies, generation, plain
 *             baseline or rf_nll_noalloc (RF_EUNSUPPORTED)
 *   RF_FORMULA (p0 .. p(m-1)), m <= 4   a density written as text in the
 *             observable x and the node's parameters p0..p3 -- the formula
 *             PDFs of Sec. 4 (RooGenericPdf, compiled just in time).  Grammar:
 *             + - * / and unary minus, '^' (right-associative, binds tighter
 *             than unary minus), decimal literals, parentheses, and exp log
 *             sqrt sin cos tanh sinh cosh asinh atan erf erfc abs pow(a, b).
 *             An integer literal exponent is a repeated product (any base);
 *             any other a^b is exp(b log a).  The text is compiled (NVRTC)
 *             into the graph's kernels with forward-mode derivatives; its
 *             integral over the range and the integral's derivatives are
 *             computed numerically in FP64 on every call (16-point
 *             Gauss-Legendre on 128 equal panels: exact to rounding for
 *             formulas whose features are wider than about 1/100 of the
 *             range).  Under RF_EVAL_FP32 the formula runs in FP32 on the
 *             parameters rounded to FP32 (first-order corrected, as the
 *             built-ins) and on its literals rounded to FP32 (not corrected:
 *             give location-like constants as fixed parameters).  The
 *             density must be positive on the range (else NLL = +inf and
 *             RF_STATUS_NONFINITE; a non-positive integral gives
 *             RF_STATUS_PARAM_DOMAIN).  Graphs with formula leaves need the
 *             specialised kernels (rf_graph_set_jit(g, 0) returns
 *             RF_EUNSUPPORTED, as does rf_graph_compile without NVRTC) and do
 *             not take toy studies, toy generation, the plain baseline or
 *             rf_nll_noalloc (RF_EUNSUPPORTED).
 * Composites:
 *   RF_ADD_FRAC (K children, K-1 fractions)  P = sum_{k<K-1} f_k P_k + (1-sum f) P_{K-1}
 *   RF_ADD_EXT  (K children, K yields; root) P = sum nu_k P_k, NLL += sum nu_k
 *   RF_PROD     (children on disjoint observables) P = prod P_k
 * The GPU compiler accepts graphs whose root is a leaf, a PROD of leaves, or
 * an ADD (fractions or extended) whose children are leaves or PRODs of leaves;
 * at most 6 leaves and 6 components (the precompiled generic kernels, and so
 * rf_graph_set_jit(g, 0) and rf_nll_noalloc, take at most 4 leaves).  Other
 * shapes return RF_EUNSUPPORTED.
 *
 * Memory: every pointer argument marked "dev" is caller-owned device memory
 * (e.g. a torch tensor).  Event columns are structure-of-arrays: observable j
 * of event i is at events[j*n_events + i], FP32 or FP64 as the descriptor says.
 * The graph owns its workspace (block and segment partials, tickets), sized
 * at compile / bind time; rf_nll and rf_nll_batched allocate nothing and never
 * synchronise the host, so they may be captured in a CUDA graph.
 *
 * Concurrency: calls are asynchronous and ordered on the given stream.  One
 * rf_graph must not be used on two streams at the same time.
 *
 * Errors: structural problems (bad descriptor, NULL, negative sizes, a
 * misaligned column base) return an error code before any launch, and
 * rf_last_error() describes them (thread-local).  Parameter-domain problems
 * (sigma <= 0, a fraction outside [0,1], a negative yield, ARGUS m0 below the
 * range) and events with a non-positive or non-finite probability do not
 * trap: they set the NLL to +inf, the gradient to NaN, and a status bit read
 * by rf_graph_status (Sec. 3, "Checking parameters").
 */
#ifndef RF_H
#define RF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* rf_stream; /* == cudaStream_t; NULL = legacy default */

typedef enum {
  RF_OK = 0,
  RF_EINVAL = 1,       /* malformed descriptor or argument */
  RF_EUNSUPPORTED = 2, /* valid graph the GPU compiler does not handle */
  RF_EALIGN = 3,       /* column base not aligned to its element size */
  RF_ECUDA = 4,        /* a CUDA call failed (message in rf_last_error) */
  RF_ENOMEM = 5        /* device allocation failed at compile/bind time */
} rf_status;

enum {
  RF_GAUSS = 1,
  RF_EXP = 2,
  RF_CHEB = 3,
  RF_CB = 4,
  RF_ARGUS = 5,
  RF_ADD_FRAC = 6,
  RF_ADD_EXT = 7,
  RF_PROD = 8,
  RF_JOHNSON = 9,
  RF_FORMULA = 10,
  RF_HYPATIA2 = 11
};

enum { RF_F32 = 0, RF_F64 = 1 };           /* column dtype              */
enum { RF_EVAL_FP32 = 0, RF_EVAL_FP64 = 1 }; /* per-event arithmetic      */

/* status bits (rf_graph_status) */
enum {
  RF_STATUS_PARAM_DOMAIN = 1u, /* a parameter outside its definition range */
  RF_STATUS_NONFINITE = 2u,    /* an event with P <= 0 or a non-finite log P */
  RF_STATUS_TIMEOUT = 4u,      /* a bounded wait inside a kernel gave up (an event
                                  copy did not arrive); that call's results are
                                  not valid */
  RF_STATUS_GEN_EXHAUSTED = 8u /* rf_generate_toys: a value took the maximum of
                                  4096 accept-reject attempts (the last one is
                                  stored) */
};

#define RF_MAX_CHILDREN 8
#define RF_MAX_NODE_PARAMS 12
#define RF_MAX_NODES 32
#define RF_MAX_PARAMS 64

typedef struct {
  int32_t type;     /* RF_GAUSS .. RF_HYPATIA2                               */
  int32_t obs;      /* leaves: observable (column) index; composites: -1     */
  int32_t n_children;
  int32_t children[RF_MAX_CHILDREN]; /* node indices                        */
  int32_t n_params;
  int32_t params[RF_MAX_NODE_PARAMS]; /* indices into the parameter vector  */
  const char* formula; /* RF_FORMULA: the density's text (NUL-terminated, at
                          most 4096 characters; read during validate/compile
                          only); ignored for other types                     */
} rf_node_desc;

typedef struct {
  int32_t n_nodes;
  const rf_node_desc* nodes;
  int32_t root;
  int32_t n_obs;
  const double* obs_lo; /* [n_obs] observable ranges, host */
  const double* obs_hi;
  int32_t n_params;
  const uint8_t* param_fixed; /* [n_params] or NULL: 1 = no gradient wanted   */
  int32_t column_dtype;       /* RF_F32 / RF_F64                              */
  int32_t eval_precision;     /* RF_EVAL_FP32: per-event math in FP32; the
                                 normalisations in FP64; each thread's sums
                                 Kahan-compensated in FP32, a block's (or a
                                 toy segment's) sums added in FP32 pairs and
                                 converted once to FP64, every sum above that
                                 (blocks, groups, a toy's segments) and the
                                 gradient epilogue in FP64.
                                 RF_EVAL_FP64: all FP64                       */
  const double* param_values; /* [n_params] or NULL, host, read at validate /
                                 compile only: values known when the graph is
                                 compiled.  They select forms, not results:
                                 an ARGUS p that is fixed at a value other
                                 than 1/2 here gets the general-p form (calls
                                 still take their parameters from `params`) */
} rf_graph_desc;

typedef struct rf_graph rf_graph;

/* Check a descriptor on the host only (no GPU needed).  Returns RF_OK,
 * RF_EINVAL or RF_EUNSUPPORTED; the reason is in rf_last_error(). */
rf_status rf_graph_validate(const rf_graph_desc* desc);

/* Validate, canonicalise (sum of products of leaves), assign accumulator
 * slots, and allocate the graph's device workspace on the current device.
 * Host-synchronous.  *out is owned by the caller: rf_graph_destroy it. */
rf_status rf_graph_compile(const rf_graph_desc* desc, rf_graph** out);
rf_status rf_graph_destroy(rf_graph* g);

/* NLL and gradient of one dataset (Sec. 5.1 problem statement).
 *   events  dev, SoA columns, n_events >= 0 (0 gives the extended term only)
 *   params  dev [n_params] FP64
 *   nll     dev [1] FP64
 *   grad    dev [n_params] FP64 or NULL; entries of fixed params are 0
 * Two launches on `stream`, no allocation, no host sync: an FP64 prologue
 * (normalisations, coefficients) and the fused event kernel (with formula
 * leaves a third before them: their normalisation).  The first kernel of a
 * call is a programmatic dependent of the kernel before it in the stream, so that
 * back-to-back calls overlap a call's FP64 prologue with the previous call's
 * event pass; it reads `params` while that kernel may still run, so params
 * must not be written by the kernels of the call immediately before on the
 * same stream (e.g. passing one call's gradient output as the next call's
 * params).  When the root is a leaf or a product of leaves, the event kernel
 * too starts beside the prologue (it builds the leaves' per-event constants
 * itself and waits for the integrals only before its reduction), under the
 * same condition.  Work of any other kind between the two calls orders as
 * usual. */
rf_status rf_nll(rf_graph* g, const void* events, int64_t n_events,
                 const double* params, double* nll, double* grad,
                 rf_stream stream);

/* As rf_nll with HOST buffers: evaluates, copies nll / grad back, and
 * synchronises the stream.  Page-locked host memory that the device can
 * address (cudaHostAlloc / cudaHostRegister, e.g. a pinned torch tensor) is
 * read by the fused kernel in place -- on a Grace-Blackwell node over
 * NVLink-C2C, each byte crossing the link once; other host memory is first
 * copied into the graph's device staging area (RF_HOST_DIRECT=0 in the
 * environment forces the copy).  The staging area grows (cudaMalloc) when
 * n_events exceeds its size, so this entry point is not capturable.
 * host_grad may be NULL. */
rf_status rf_nll_host(rf_graph* g, const void* host_events, int64_t n_events,
                      const double* host_params, double* host_nll,
                      double* host_grad, rf_stream stream);

/* Per-event log P(x_i) in FP64 (dev [n_events]); same arithmetic as rf_nll. */
rf_status rf_logp(rf_graph* g, const void* events, int64_t n_events,
                  const double* params, double* logp, rf_stream stream);

/* Toy studies (RooStats-style, Sec. 1): many datasets of uneven size that
 * share one graph.  rf_graph_bind_events records the concatenated event
 * columns (dev; column j at events + j*n_events); toy t owns events
 * [offsets[t], offsets[t+1]).  Sizes the toy workspace for up to max_toys.
 * A graph evaluated in FP32 over FP64 columns converts the columns to FP32
 * here, once (round to nearest: the value every per-event conversion would
 * give), and its toy calls read that copy (n_obs * n_events * 4 bytes, owned
 * by the graph); bind again after changing the events.  Host-synchronous. */
rf_status rf_graph_bind_events(rf_graph* g, const void* events,
                               int64_t n_events, int32_t max_toys);

/*   offsets        dev int64 [toys+1], non-decreasing, offsets[toys] <= n_events
 *   params_matrix  dev FP64 [toys * n_params], row t = toy t's parameters
 *   out            dev FP64 [toys * (1 + n_params)], row t = (NLL_t, grad_t)
 * Three kernels: a per-toy FP64 prologue (blocks of 32 toys, the leaves'
 * integrals, per-event constants and coefficients on separate warps, then a
 * 4-lane combine per toy); a segment kernel that splits all toys' events
 * [offsets[0], offsets[toys]) evenly over its warps (one grid of SMs x
 * blocks_per_sm blocks) and writes one row of partial sums per (warp, toy)
 * pair that share events (FP32 evaluation: each sum as an FP32 pair, FP64
 * evaluation: FP64); and a finalize kernel, 4 lanes per toy, that widens the
 * toy's rows to FP64, sums them in a fixed order and writes (NLL, grad).
 * Results depend on the inputs and the launch shape only.  Offsets outside [0, n_events] are clamped and a decreasing pair
 * raises RF_STATUS_NONFINITE (the affected toys' results are then
 * meaningless, but nothing outside the bound columns is read).  No
 * allocation, no host sync: capturable. */
rf_status rf_nll_batched(rf_graph* g, const int64_t* offsets, int32_t toys,
                         const double* params_matrix, double* out,
                         rf_stream stream);

/* A gradient fit of every toy: `iters` Adam steps (Kingma & Ba 2015) on the
 * parameters of toy t in units of scale[t*n_params + j] (dev FP64
 * [toys * n_params]; e.g. each toy's starting |theta|), learning rate lr,
 * beta = (0.9, 0.999), eps = 1e-8; fixed parameters do not move, and a toy
 * whose NLL is not finite keeps its parameters for that step.  The
 * per-iteration work (the three kernels of rf_nll_batched, the Adam step
 * fused into the finalize kernel) is captured once into a CUDA graph and
 * replayed `iters` times.  params_matrix (dev) is updated in place; out
 * (dev [toys*(1+n_params)]) holds the NLL and gradient of the last
 * evaluation (at the parameters before the last step).  Host-synchronous. */
rf_status rf_fit_toys(rf_graph* g, const int64_t* offsets, int32_t toys,
                      double* params_matrix, const double* scale, int32_t iters,
                      double lr, double* out, rf_stream stream);

/* Sharded evaluation (the multi-process mode of Sec. 5.2, footnote: a
 * dataset's contiguous batches divided among processes).  Each process
 * evaluates its shard with rf_nll; the NLLs and gradients of the shards add
 * up to the whole dataset's once the extended term sum(nu) (and its +1 in
 * d/d nu) is counted on exactly one shard.  w is that term's weight in this
 * graph (default 1): 1 on one shard, 0 on the others.  Host only. */
rf_status rf_graph_set_shard_weight(rf_graph* g, double w);

/* Toy generation: the events of `toys` datasets drawn from the graph, on the
 * device, in the layout rf_graph_bind_events / rf_nll_batched read.
 *   params_matrix dev FP64 [toys * n_params]: each toy's generating parameters
 *   comp_counts   dev int64 [toys * n_comp]: events of each component per toy
 *                 (Poisson draws around the yields for an extended model, a
 *                 multinomial split for fractions; drawn by the caller)
 *   offsets       dev int64 [toys + 1]: toy t owns [offsets[t], offsets[t+1]),
 *                 offsets[t+1] - offsets[t] = the sum of its counts
 *   events        dev, column j (observable j) at events + j * n_events, of the
 *                 graph's column type; n_events >= offsets[toys]
 * Toy t's events are, in order, comp_counts[t*n_comp + c] events of component
 * c; each observable comes from the component's leaf on it, drawn in FP64 by
 * inverse CDF (Gaussian, Exponential, Crystal Ball) or accept-reject
 * (Chebychev, ARGUS), from uniforms ((w >> 11) + 1/2) 2^-53 of the words w of
 * Philox4x64-10 (Salmon et al. 2011) with key {seed, 0x52462D544F595321} and
 * counter {event, observable, attempt, 0} -- the values do not depend on the
 * launch.  A value is rounded to the column type and accepted only inside
 * the observable's range (ARGUS: below m0).  Every component must cover every
 * observable (RF_EUNSUPPORTED otherwise).  A toy whose counts do not fill its
 * range gets NaN events there and RF_STATUS_NONFINITE.  Asynchronous. */
rf_status rf_generate_toys(rf_graph* g, const double* params_matrix,
                           const int64_t* comp_counts, const int64_t* offsets,
                           int32_t toys, uint64_t seed, void* events,
                           int64_t n_events, rf_stream stream);

/* Baseline: the batch interface of Sec. 5.2 on the GPU, in FP64 -- one kernel
 * per graph node, each writing an n-length node-owned FP64 array, then a log
 * kernel and a reduction kernel.  The gradient (if grad != NULL) is taken by
 * central finite differences (2 evaluations per free parameter, step
 * 1e-6 * max(|theta|, 1e-3)).  Needs n_events * (n_nodes + 1) * 8 bytes of
 * workspace, allocated on first use (not capturable). */
rf_status rf_nll_plain(rf_graph* g, const void* events, int64_t n_events,
                       const double* params, double* nll, double* grad,
                       rf_stream stream);

/* Launch configuration: threads per block (64, 128 or 256) and resident
 * blocks per SM used to size the grid (1..8) of the fused and segment
 * kernels, and events per thread per iteration of the fused kernel (FP32
 * eval: 4, 8, or 16 with the graph-specialised kernels; FP64 eval: 2 or 4;
 * the toy segment kernel takes its own: 8 events per lane).  min_blocks
 * (2, 3 or 4) is the register budget the graph-specialised fused kernel is
 * compiled for: room for that many blocks
 * of 256 threads on one SM (at most 128, 80 or 64 registers per thread); the
 * generic kernels ignore it.  Defaults: 3 for FP32 evaluation, 2 for FP64;
 * rf_graph_tune tries 2, 3 and 4. */
typedef struct {
  int32_t block;
  int32_t ept;
  int32_t blocks_per_sm;
  int32_t min_blocks;
} rf_launch;

rf_status rf_graph_get_launch(const rf_graph* g, rf_launch* cfg);
rf_status rf_graph_set_launch(rf_graph* g, const rf_launch* cfg);

/* Autotune: times every launch configuration (block x events per thread x
 * blocks per SM x, for the graph-specialised kernel, register budget) on the
 * given data with CUDA events -- five calls issued back to back, after two
 * warm-up calls -- and keeps the fastest (host-synchronous).
 * The choice is cached on disk, in the folder RF_JIT_CACHE_DIR (default
 * $TMPDIR/rfgpu-jit, else /tmp/rfgpu-jit), keyed by the kernel (the
 * specialised source, else the graph structure and library build), the
 * column and evaluation precisions, floor(log2 n_events) and the device's
 * compute capability and SM count; a later rf_graph_tune with the same key
 * applies the cached configuration and times only that one.  best_ms (may be
 * NULL) receives the mean time of one call (back to back) with the chosen
 * configuration.
 * Same errors as rf_nll; the configuration is unchanged on error. */
rf_status rf_graph_tune(rf_graph* g, const void* events, int64_t n_events,
                        const double* params, rf_stream stream,
                        double* best_ms);

#define RF_TUNE_NO_CACHE 1 /* neither read nor write the on-disk cache */
#define RF_TUNE_REFRESH 2  /* time every configuration and overwrite the entry */

/* rf_graph_tune with flags (RF_TUNE_*; other bits: RF_EINVAL).  *from_cache
 * (may be NULL) is set to 1 when the configuration came from the cache, else
 * 0.  An entry that no longer validates is ignored and overwritten. */
rf_status rf_graph_tune_ex(rf_graph* g, const void* events, int64_t n_events,
                           const double* params, rf_stream stream, int32_t flags,
                           double* best_ms, int32_t* from_cache);

/* NLL and gradient for callers that cannot allocate device memory (no
 * counterpart in the paper).  Some callers cannot call cudaMalloc at all --
 * code in a host callback or driver hook, a real-time loop whose allocator
 * is frozen after start-up, a host whose device memory pool belongs to
 * another framework -- so they cannot build an rf_graph, whose compile step
 * allocates its workspace.  This entry point takes the descriptor directly
 * and runs the precompiled generic fused kernel with its scratch (per-block
 * partial sums, block ticket, status word) in a file-scope static device
 * array of the library: 256 KiB, enough for the partial sums of
 * blocks <= 1024 and of the grid tree's 32 groups (0 = twice the SM count,
 * capped at 1024; larger values return RF_EINVAL).  Every GPU that loads the library holds that array until
 * the process exits.  It allocates nothing: no cudaMalloc/cudaFree and no
 * allocating library routine.  Its first call on a device looks up the
 * array's device address (cudaGetSymbolAddress) with that device current;
 * make that first call before any stream capture.  The address is kept for
 * the process: a cudaDeviceReset unloads the library's device image and
 * makes it stale, so do not call this entry point on a device after
 * resetting it.  Every call shares the
 * array and it keeps the last call's contents: the ticket and status words
 * are cleared on `stream` at the start of each call, and calls that overlap
 * on the GPU race on the array.  Arguments, layout and results as rf_nll
 * (events, params, nll, grad are caller-owned device memory); domain errors
 * give NLL = +inf and a NaN gradient (the status word is not reported). */
rf_status rf_nll_noalloc(const rf_graph_desc* desc, const void* events,
                         int64_t n_events, const double* params, double* nll,
                         double* grad, int32_t blocks, rf_stream stream);

/* Kernel specialisation.  rf_graph_compile also emits, for its graph, a
 * model in which the leaf types, columns, component sums and gradient masks
 * are compile-time constants, and compiles the fused, toy and log P kernels
 * for it with NVRTC (sm_103a), caching the module for the process; without
 * it (RF_JIT=0 in the environment, or NVRTC unavailable) the precompiled
 * generic kernels run the same device code with run-time dispatch.
 * rf_graph_set_jit(g, 0/1) switches between them (1 compiles if needed and
 * returns RF_ECUDA with the compiler log in rf_last_error on failure);
 * rf_graph_uses_jit tells which is in use; rf_graph_kernel_regs gives the
 * registers per thread of the specialised fused kernel (0 if generic). */
rf_status rf_graph_set_jit(rf_graph* g, int32_t enable);
/* Compile the specialised kernels of a descriptor with NVRTC without loading
 * them (no GPU needed): RF_OK, or RF_ECUDA with the compiler log. */
rf_status rf_jit_check(const rf_graph_desc* desc);
int32_t rf_graph_uses_jit(const rf_graph* g);
/* FNV-1a hash of the specialised fused kernel's source for the current
 * launch configuration (0 for the generic kernels): identifies the exact
 * kernel a profile was taken on. */
uint64_t rf_graph_kernel_hash(const rf_graph* g);
/* The same for the toy segment kernel of the bound toy sample (0 before
 * rf_graph_bind_events or with the generic kernels). */
uint64_t rf_graph_toy_kernel_hash(const rf_graph* g);
/* The toy segment kernel's launch (Sec. 5.1's batches, one per toy, run as
 * one grid): threads per block, events per lane per chunk, and registers per
 * thread of the specialised kernel of the bound toy sample (0 before
 * rf_graph_bind_events or with the generic kernels).  The grid is the SM
 * count times the resident blocks of that size.  RF_EINVAL for a NULL
 * argument; writes only the three outputs. */
rf_status rf_graph_get_toy_launch(const rf_graph* g, int32_t* block, int32_t* events_per_lane,
                                  int32_t* regs);
int32_t rf_graph_kernel_regs(const rf_graph* g);

/* Synchronises the device, returns the OR of RF_STATUS_* bits raised since
 * the last call, and clears them. */
rf_status rf_graph_status(rf_graph* g, uint32_t* flags);

/* Kernels the last rf_nll / rf_nll_batched call launched (for accounting). */
int32_t rf_graph_last_launches(const rf_graph* g);

/* Thread-local description of the last error ("" if none). */
const char* rf_last_error(void);

/* Diagnostics: y_fast[i] = the library's FP32 natural log of x[i] (used for
 * per-event log-densities), y_ref[i] = CUDA logf(x[i]); dev arrays [n]. */
rf_status rf_check_log(const float* x, float* y_fast, float* y_ref, int64_t n,
                       rf_stream stream);
/* Diagnostics: y_fast[i] = the library's integer-pipe FP64 -> FP32 rounding
 * of x[i] (used when FP64 columns are evaluated in FP32), y_ref[i] = the
 * hardware conversion (__double2float_rn); dev arrays [n]. */
rf_status rf_check_d2f(const double* x, float* y_fast, float* y_ref, int64_t n,
                       rf_stream stream);

/* Throughput of single operations on this GPU, in operations per second,
 * measured by dedicated kernels (used for the compute roofline):
 * out[0] FP32 FMA, out[1] expf, out[2] logf, out[3] FP32 reciprocal (IEEE),
 * out[4] FP64 FMA, out[5] exp (FP64), out[6] log (FP64), out[7] erf (FP64),
 * out[8] the library's FP32 log, out[9] its FP32 exp(-x) (x >= 0),
 * out[10] the approximate FP32 reciprocal, out[11] FP32 FMAs/s issued as
 * packed FP32x2 FMA instructions; then latencies in ns per dependent
 * operation within one warp: out[12] FP64 FMA with 1 active lane, out[13]
 * FP64 FMA with 32 active lanes, out[14] exp (FP64) with 1 lane, out[15]
 * exp (FP64) with 32 lanes; then throughputs again: out[16] sqrtf (IEEE),
 * out[17] the hardware FP32 square root (sqrt.approx), out[18] log2 (FP64),
 * out[19] exp2 (FP64), out[20] FP64 division, out[21] the hardware base-2
 * log (lg2.approx), out[22] the hardware base-2 exp (ex2.approx), out[23]
 * sqrt (FP64).  out has 24 entries.
 * Host-synchronous; allocates a small scratch buffer. */
rf_status rf_microbench(double* out);

#ifdef __cplusplus
}
#endif
#endif /* RF_H */
