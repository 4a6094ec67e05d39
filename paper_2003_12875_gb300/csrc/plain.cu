// plain.cu -- the baseline: the batch interface of Sec. 5.2 moved to the GPU
// in FP64.  Every node of the compiled graph is one kernel that reads its
// inputs from contiguous arrays and writes its n values into its own
// node-owned array (leaves: normalised densities; products; the Add), then a
// log kernel writes -log P_i and a reduction kernel sums them (Neumaier per
// thread, FP64 tree, last-block finish).  The gradient is taken by central
// finite differences, two evaluations per free parameter, each evaluation
// on a perturbed copy of the parameter vector made on the device.
#include <cuda_runtime.h>

#include "rf_device.cuh"

namespace rf {
// device pointer table of one evaluation: the component arrays, then the
// leaf arrays of every component
constexpr int kPtrSlots = RF_MAXC + RF_MAXC * RF_MAXL;


__global__ void plain_consts_kernel(const RfProgram P, const double* params,
                                    RfConsts<double>* K) {
  if (blockIdx.x == 0 && threadIdx.x == 0) build_consts_serial(P, params, *K);
}

template <typename Col>
__global__ void plain_leaf_kernel(const RfProgram P, int k,
                                  const Col* __restrict__ ev, int64_t n,
                                  const RfConsts<double>* __restrict__ K,
                                  double* __restrict__ out) {
  const RfLeafProg& L = P.leaf[k];
  const Col* col = ev + (int64_t)P.col_obs[L.col] * n;
  double pc[RF_PC];
  for (int j = 0; j < RF_PC; ++j) pc[j] = K->pc[k][j];
  const double lnI = K->lnI[k];
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double u, g[RF_LEAF_MAXP];
    eval_leaf<double>(L.type, L.gmask & (4 | RF_ARGUS_GENERAL), (double)col[i], pc, u, g);  // ARGUS form
    out[i] = exp(kLn2 * u - lnI);  // u is in base-2 units
  }
}

// out = prod of the leaf arrays of component c
__global__ void plain_prod_kernel(const double* const* __restrict__ in, int m,
                                  int64_t n, double* __restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double v = in[0][i];
    for (int j = 1; j < m; ++j) v *= in[j][i];
    out[i] = v;
  }
}

// out = sum_c coef_c * comp_c
__global__ void plain_add_kernel(const double* const* __restrict__ in, int C,
                                 const RfConsts<double>* __restrict__ K,
                                 int64_t n, double* __restrict__ out) {
  double coef[RF_MAXC];
  for (int c = 0; c < C; ++c) coef[c] = K->coef[c];
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double v = 0.0;
    for (int c = 0; c < C; ++c) v += coef[c] * in[c][i];
    out[i] = v;
  }
}

__global__ void plain_log_kernel(const double* __restrict__ p, int64_t n,
                                 double* __restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = -log(p[i]);
}

// sum of x[0..n) plus the extended term -> *res (+inf on a domain error)
__global__ void __launch_bounds__(256)
    plain_reduce_kernel(const double* __restrict__ x, int64_t n,
                        const RfConsts<double>* __restrict__ K, double* partials,
                        unsigned int* counter, double* res) {
  __shared__ double red[32];
  __shared__ double tot[1];
  __shared__ int s_last;
  double s = 0.0, c = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double v = x[i], t = s + v;
    c += (fabs(s) >= fabs(v)) ? (s - t) + v : (v - t) + s;
    s = t;
  }
  double val[1] = {s + c};
  block_sum<1>(val, red, tot);
  if (threadIdx.x == 0) partials[blockIdx.x * RF_NACC_MAX] = tot[0];
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = (atomicAdd(counter, 1u) == gridDim.x - 1) ? 1 : 0;
  __syncthreads();
  if (s_last) {
    __threadfence();
    rows_sum<1>(partials, 0, gridDim.x, red, tot);
    if (threadIdx.x == 0) {
      double v = tot[0] + K->ext_sum;
      *res = (K->bad || !isfinite(v)) ? kInf() : v;
      *counter = 0u;
    }
  }
}

// params_out = params with parameter p moved by sgn * h_p
__global__ void plain_perturb_kernel(const double* __restrict__ params, int np,
                                     int p, double sgn, double* params_out,
                                     double* h_out) {
  int j = threadIdx.x;
  if (j < np) {
    double v = params[j];
    if (j == p) {
      double h = 1e-6 * fmax(fabs(v), 1e-3);
      v += sgn * h;
      if (h_out) h_out[p] = h;
    }
    params_out[j] = v;
  }
}

__global__ void plain_fd_kernel(const double* __restrict__ fvals, const double* __restrict__ h,
                                const RfProgram P, double* grad) {
  int p = threadIdx.x;
  if (p < P.n_par) {
    bool fx = p < 64 ? ((P.fixed_lo >> p) & 1) : ((P.fixed_hi >> (p - 64)) & 1);
    grad[p] = fx ? 0.0 : (fvals[2 * p] - fvals[2 * p + 1]) / (2.0 * h[p]);
  }
}

// Workspace layout in node_buf (doubles): [NL leaf arrays][C component
// arrays][1 sum array][1 log array] each n long, then pointer tables, the
// FD scratch and one RfConsts<double>.
template <typename Col>
static int plain_eval(const RfProgram& P, const Col* ev, int64_t n,
                      const double* params, double* nb, double* partials,
                      unsigned int* counter, double* res, RfConsts<double>* K,
                      const double** ptrs, cudaStream_t st, int* launches) {
  const int NL = P.n_leaves, C = P.n_comp;
  int grid = (int)((n + 255) / 256);
  if (grid > 152 * 16) grid = 152 * 16;
  if (grid < 1) grid = 1;
  plain_consts_kernel<<<1, 32, 0, st>>>(P, params, K);
  ++*launches;
  double* leafb = nb;
  double* compb = nb + (int64_t)NL * n;
  double* sumb = compb + (int64_t)C * n;
  double* logb = sumb + n;
  for (int k = 0; k < NL; ++k) {
    plain_leaf_kernel<Col><<<grid, 256, 0, st>>>(P, k, ev, n, K, leafb + (int64_t)k * n);
    ++*launches;
  }
  // components: a single leaf is its own array, otherwise a product kernel
  const double** comp_in = ptrs;           // [C] component arrays
  const double** prod_in = ptrs + RF_MAXC; // [RF_MAXC * RF_MAXL] leaf arrays per component
  const double* comp_ptr[RF_MAXC];
  const double* prod_ptr[RF_MAXC * RF_MAXL];
  for (int c = 0; c < C; ++c) {
    int m = 0, last = -1;
    for (int k = 0; k < NL; ++k)
      if (P.leaf[k].comp == c) {
        prod_ptr[c * RF_MAXL + m++] = leafb + (int64_t)k * n;
        last = k;
      }
    comp_ptr[c] = (m == 1) ? leafb + (int64_t)last * n : compb + (int64_t)c * n;
  }
  // pointer tables live in device memory (written with one async copy each)
  cudaMemcpyAsync(comp_in, comp_ptr, sizeof(comp_ptr), cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(prod_in, prod_ptr, sizeof(prod_ptr), cudaMemcpyHostToDevice, st);
  for (int c = 0; c < C; ++c) {
    int m = 0;
    for (int k = 0; k < NL; ++k)
      if (P.leaf[k].comp == c) ++m;
    if (m > 1) {
      plain_prod_kernel<<<grid, 256, 0, st>>>(prod_in + c * RF_MAXL, m, n, compb + (int64_t)c * n);
      ++*launches;
    }
  }
  plain_add_kernel<<<grid, 256, 0, st>>>(comp_in, C, K, n, sumb);
  plain_log_kernel<<<grid, 256, 0, st>>>(sumb, n, logb);
  plain_reduce_kernel<<<grid, 256, 0, st>>>(logb, n, K, partials, counter, res);
  *launches += 3;
  return (int)cudaGetLastError();
}

template <typename Col>
static int plain_all(const RfProgram& P, const void* events, int64_t n,
                     const double* params, double* nb, double* nll, double* grad,
                     double* partials, unsigned int* counter, cudaStream_t st,
                     int* launches) {
  const Col* ev = static_cast<const Col*>(events);
  // scratch after the node arrays
  const int NL = P.n_leaves, C = P.n_comp;
  double* tail = nb + (int64_t)(NL + C + 2) * n;
  const double** ptrs = reinterpret_cast<const double**>(tail);   // kPtrSlots slots
  double* pp = tail + kPtrSlots;                                   // [RF_MAXPAR]
  double* fvals = pp + RF_MAXPAR;                                  // [2*RF_MAXPAR]
  double* hs = fvals + 2 * RF_MAXPAR;                              // [RF_MAXPAR]
  RfConsts<double>* K = reinterpret_cast<RfConsts<double>*>(hs + RF_MAXPAR);
  int rc = plain_eval<Col>(P, ev, n, params, nb, partials, counter, nll, K, ptrs, st, launches);
  if (rc || !grad) return rc;
  for (int p = 0; p < P.n_par; ++p) {
    bool fx = p < 64 ? ((P.fixed_lo >> p) & 1) : ((P.fixed_hi >> (p - 64)) & 1);
    if (fx) continue;
    for (int s = 0; s < 2; ++s) {
      plain_perturb_kernel<<<1, RF_MAXPAR, 0, st>>>(params, P.n_par, p, s ? -1.0 : 1.0, pp, hs);
      ++*launches;
      rc = plain_eval<Col>(P, ev, n, pp, nb, partials, counter, fvals + 2 * p + s, K, ptrs, st,
                           launches);
      if (rc) return rc;
    }
  }
  plain_fd_kernel<<<1, RF_MAXPAR, 0, st>>>(fvals, hs, P, grad);
  ++*launches;
  return (int)cudaGetLastError();
}

}  // namespace rf

size_t rf_plain_bytes(const RfProgram& P, int64_t n) {
  return sizeof(double) * ((size_t)(P.n_leaves + P.n_comp + 2) * (size_t)n + rf::kPtrSlots +
                           4 * RF_MAXPAR) +
         sizeof(RfConsts<double>) + 256;
}

int rf_launch_plain(const RfProgram& prog, int coldt, const void* events, int64_t n,
                    const double* params, double* node_buf, double* nll, double* grad,
                    double* partials, unsigned int* counter, void* stream, int* launches) {
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  *launches = 0;
  if (coldt == 0)
    return rf::plain_all<float>(prog, events, n, params, node_buf, nll, grad, partials, counter,
                                st, launches);
  return rf::plain_all<double>(prog, events, n, params, node_buf, nll, grad, partials, counter,
                               st, launches);
}
