// microbench.cu -- throughput of single operations on this GPU, for the
// compute side of the roofline.  Each thread runs 8 independent dependency
// chains of one operation; the result feeds a store that never fires, so the
// work cannot be removed.  Ops/s = threads * 8 * iterations / kernel time.
#include <cuda_runtime.h>

#include "rf_device.cuh"

namespace {

template <int OP>
struct Op;
template <> struct Op<0> { typedef float T; static __device__ __forceinline__ float f(float a) { return fmaf(a, 0.9999f, 0.0001f); } };
template <> struct Op<1> { typedef float T; static __device__ __forceinline__ float f(float a) { return expf(-a); } };
template <> struct Op<2> { typedef float T; static __device__ __forceinline__ float f(float a) { return logf(a + 2.0f); } };
template <> struct Op<3> { typedef float T; static __device__ __forceinline__ float f(float a) { return __frcp_rn(a + 1.0f); } };
template <> struct Op<4> { typedef double T; static __device__ __forceinline__ double f(double a) { return fma(a, 0.9999, 0.0001); } };
template <> struct Op<5> { typedef double T; static __device__ __forceinline__ double f(double a) { return exp(-a); } };
template <> struct Op<6> { typedef double T; static __device__ __forceinline__ double f(double a) { return log(a + 2.0); } };
template <> struct Op<7> { typedef double T; static __device__ __forceinline__ double f(double a) { return erf(a) + 0.25; } };
// the library's own FP32 per-event functions
template <> struct Op<8> { typedef float T; static __device__ __forceinline__ float f(float a) { return rf::log_fast(a + 2.0f); } };
template <> struct Op<9> { typedef float T; static __device__ __forceinline__ float f(float a) { return rf::exp_neg_approx(-a); } };
template <> struct Op<10> { typedef float T; static __device__ __forceinline__ float f(float a) { return rf::rcp_approx(a + 1.0f); } };
// packed FP32x2 FMA (two FMAs per instruction)
template <> struct Op<11> {
  typedef float2 T;
  static __device__ __forceinline__ float2 f(float2 a) {
    return __ffma2_rn(a, make_float2(0.9999f, 0.9998f), make_float2(0.0001f, 0.0002f));
  }
};

// more single operations for the roofline's op list: IEEE sqrtf, the
// hardware square root, FP64 log2 / exp2 / division / square root (the FP64
// kernels' per-event functions), and the hardware base-2 log / exp as the
// per-event code issues them (one instruction each)
template <> struct Op<12> { typedef float T; static __device__ __forceinline__ float f(float a) { return sqrtf(a + 1.0f); } };
template <> struct Op<13> {
  typedef float T;
  static __device__ __forceinline__ float f(float a) {
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a + 1.0f));
    return r;
  }
};
template <> struct Op<14> { typedef double T; static __device__ __forceinline__ double f(double a) { return log2(a + 2.0); } };
template <> struct Op<15> { typedef double T; static __device__ __forceinline__ double f(double a) { return exp2(-a); } };
template <> struct Op<16> { typedef double T; static __device__ __forceinline__ double f(double a) { return 1.0 / (a + 1.0); } };
template <> struct Op<17> { typedef float T; static __device__ __forceinline__ float f(float a) { return rf::lg2_fast(a + 2.0f); } };
template <> struct Op<18> { typedef float T; static __device__ __forceinline__ float f(float a) { return rf::ex2_fast(-a); } };
template <> struct Op<19> { typedef double T; static __device__ __forceinline__ double f(double a) { return sqrt(a + 1.0); } };

template <int OP>
__global__ void __launch_bounds__(256) mb_kernel(typename Op<OP>::T* sink, int iters) {
  typedef typename Op<OP>::T T;
  T a[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) a[j] = (T)(0.1 + 0.01 * j + 1e-6 * threadIdx.x);
  for (int it = 0; it < iters; ++it)
#pragma unroll
    for (int j = 0; j < 8; ++j) a[j] = Op<OP>::f(a[j]);
  T s = 0;
#pragma unroll
  for (int j = 0; j < 8; ++j) s += a[j];
  if (s == (T)-12345.0) sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <>
__global__ void __launch_bounds__(256) mb_kernel<11>(float2* sink, int iters) {
  float2 a[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) a[j] = make_float2(0.1f + 0.01f * j, 0.2f + 1e-6f * threadIdx.x);
  for (int it = 0; it < iters; ++it)
#pragma unroll
    for (int j = 0; j < 8; ++j) a[j] = Op<11>::f(a[j]);
  float s = 0.f;
#pragma unroll
  for (int j = 0; j < 8; ++j) s += a[j].x + a[j].y;
  if (s == -12345.0f) sink[blockIdx.x * blockDim.x + threadIdx.x] = make_float2(s, s);
}

// Latency of one dependent chain per active lane in a single warp: the time
// per operation with 1 and with 32 active lanes shows whether the FP64 pipe
// serialises lanes (then 32 lanes cost more per step) or not.
template <int OP>
__global__ void lat_kernel(typename Op<OP>::T* sink, int iters, int lanes) {
  typedef typename Op<OP>::T T;
  if ((int)threadIdx.x >= lanes) return;
  T a = (T)(0.1 + 1e-6 * threadIdx.x);
  for (int it = 0; it < iters; ++it) a = Op<OP>::f(a);
  if (a == (T)-12345.0) sink[threadIdx.x] = a;
}

template <int OP>
double lat_ns(void* sink, int iters, int lanes) {
  typedef typename Op<OP>::T T;
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  lat_kernel<OP><<<1, 32>>>(static_cast<T*>(sink), iters / 10, lanes);  // warm-up
  cudaEventRecord(a);
  lat_kernel<OP><<<1, 32>>>(static_cast<T*>(sink), iters, lanes);
  cudaEventRecord(b);
  cudaEventSynchronize(b);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, a, b);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return (double)ms * 1e6 / iters;
}

template <int OP>
double run(int sms, void* sink, int iters) {
  const int block = 256, grid = sms * 8;
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  typedef typename Op<OP>::T T;
  mb_kernel<OP><<<grid, block>>>(static_cast<T*>(sink), iters / 10);  // warm-up
  cudaEventRecord(a);
  mb_kernel<OP><<<grid, block>>>(static_cast<T*>(sink), iters);
  cudaEventRecord(b);
  cudaEventSynchronize(b);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, a, b);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return (double)grid * block * 8.0 * iters / (ms * 1e-3);
}

}  // namespace

int rf_run_microbench(double* out) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  void* sink = nullptr;
  cudaError_t e = cudaMalloc(&sink, (size_t)sms * 8 * 256 * sizeof(double));
  if (e != cudaSuccess) return (int)e;
  out[0] = run<0>(sms, sink, 4096);
  out[1] = run<1>(sms, sink, 1024);
  out[2] = run<2>(sms, sink, 1024);
  out[3] = run<3>(sms, sink, 1024);
  out[4] = run<4>(sms, sink, 256);
  out[5] = run<5>(sms, sink, 32);
  out[6] = run<6>(sms, sink, 32);
  out[7] = run<7>(sms, sink, 32);
  out[8] = run<8>(sms, sink, 1024);
  out[9] = run<9>(sms, sink, 1024);
  out[10] = run<10>(sms, sink, 1024);
  out[11] = 2.0 * run<11>(sms, sink, 4096);  // FMAs per second
  out[12] = lat_ns<4>(sink, 200000, 1);
  out[13] = lat_ns<4>(sink, 200000, 32);
  out[14] = lat_ns<5>(sink, 20000, 1);
  out[15] = lat_ns<5>(sink, 20000, 32);
  out[16] = run<12>(sms, sink, 1024);
  out[17] = run<13>(sms, sink, 1024);
  out[18] = run<14>(sms, sink, 32);
  out[19] = run<15>(sms, sink, 32);
  out[20] = run<16>(sms, sink, 64);
  out[21] = run<17>(sms, sink, 1024);
  out[22] = run<18>(sms, sink, 1024);
  out[23] = run<19>(sms, sink, 64);
  e = cudaGetLastError();
  cudaFree(sink);
  return (int)e;
}

// The library's FP32 logarithm next to CUDA's logf on the same inputs (for the
// accuracy test of the former).
__global__ void check_log_kernel(const float* x, float* yf, float* yr, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    yf[i] = rf::log_fast(x[i]);
    yr[i] = logf(x[i]);
  }
}

int rf_run_check_log(const float* x, float* y_fast, float* y_ref, int64_t n, cudaStream_t st) {
  if (n == 0) return 0;
  int64_t g = (n + 255) / 256;
  int grid = (int)(g > 4096 ? 4096 : g);
  check_log_kernel<<<grid, 256, 0, st>>>(x, y_fast, y_ref, n);
  return (int)cudaGetLastError();
}

// The library's integer-pipe double -> float conversion next to the hardware
// conversion (for the bit-exactness test of the former).
__global__ void check_d2f_kernel(const double* x, float* yf, float* yr, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    yf[i] = rf::d2f_rn(x[i]);
    yr[i] = __double2float_rn(x[i]);
  }
}

int rf_run_check_d2f(const double* x, float* y_fast, float* y_ref, int64_t n, cudaStream_t st) {
  if (n == 0) return 0;
  int64_t g = (n + 255) / 256;
  int grid = (int)(g > 4096 ? 4096 : g);
  check_d2f_kernel<<<grid, 256, 0, st>>>(x, y_fast, y_ref, n);
  return (int)cudaGetLastError();
}
