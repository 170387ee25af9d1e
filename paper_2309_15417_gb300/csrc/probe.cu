// probe.cu -- measurement support for the roofline: the FP32 / FP64 peak of
// this GPU from FMA chains, and the exact FP32 operation count of the
// triangle-pair distance as the pair kernel evaluates it.  Neither is part of
// the contact-detection method; the benchmark uses them to state its
// roofline fractions against measured denominators.
#include <nvtx3/nvToolsExt.h>

#include "dem_probe.h"
#include "internal.cuh"

namespace dem {
namespace {

// Each thread runs CH independent FMA chains for `iters` steps.  The chains'
// multiplier is just below 1 and the addend tiny, so values stay finite and
// normal; the result is stored only if it matches an impossible value, which
// the compiler cannot prove, so no chain is eliminated.
constexpr int CH = 8;

template <class T>
__global__ void __launch_bounds__(256) k_fma_chains(int iters, T mul, T add, T *sink) {
  T a[CH];
#pragma unroll
  for (int c = 0; c < CH; ++c) a[c] = T(threadIdx.x + c) * T(1e-3);
  for (int it = 0; it < iters; ++it)
#pragma unroll
    for (int c = 0; c < CH; ++c) a[c] = fma(a[c], mul, add);
  T r = T(0);
#pragma unroll
  for (int c = 0; c < CH; ++c) r += a[c];
  if (r == T(-12345.678)) sink[0] = r;
}

__device__ float g_sink32[1];
__device__ double g_sink64[1];

// Counting arithmetic: FP32 values, every add, sub, mul, div and sqrt counted
// once in a per-thread slot (a fused multiply-add therefore counts 2).
constexpr int CNT_THREADS = 1 << 15;
__device__ unsigned long long g_ops[CNT_THREADS];

__device__ __forceinline__ void count_op() {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  g_ops[t] += 1;
}

struct OpsCnt {
  using T = float;
  static __device__ __forceinline__ float add(float a, float b) { count_op(); return a + b; }
  static __device__ __forceinline__ float sub(float a, float b) { count_op(); return a - b; }
  static __device__ __forceinline__ float mul(float a, float b) { count_op(); return a * b; }
  static __device__ __forceinline__ float div(float a, float b) { count_op(); return __fdividef(a, b); }
  static __device__ __forceinline__ float sqrt(float a) { count_op(); return OpsF::sqrt(a); }
  static __device__ __forceinline__ float inf() { return OpsF::inf(); }
};

// tri: [n][18] floats: triangle a (3 vertices xyz), then triangle b
__global__ void k_count_dist(const float *tri, int64_t n, int64_t *ops) {
  using G = Geo<OpsCnt>;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  for (int64_t k = t; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    V3<float> A[3], B[3], pa, pb;
    const float *f = tri + 18 * k;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      A[q] = V3<float>{f[3 * q], f[3 * q + 1], f[3 * q + 2]};
      B[q] = V3<float>{f[9 + 3 * q], f[9 + 3 * q + 1], f[9 + 3 * q + 2]};
    }
    g_ops[t] = 0;
    const float d2 = G::tri_dist2(A, B, pa, pb);
    OpsCnt::sqrt(d2);  // the distance itself
    ops[k] = (int64_t)g_ops[t];
  }
}

}  // namespace
}  // namespace dem

extern "C" dem_status dem_probe_fma_peak(int32_t precision, int32_t iters, void *stream, double *flops_per_s) {
  using namespace dem;
  nvtxRangePushA("dem_probe_fma_peak");
  struct Pop {
    ~Pop() { nvtxRangePop(); }
  } pop;
  if (!flops_per_s || iters <= 0 || (precision != 0 && precision != 1)) return DEM_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return DEM_ERR_CUDA;
  const int blocks = sms * 8, threads = 256;  // 64 warps per SM
  float *s32 = nullptr;
  double *s64 = nullptr;
  if (cudaGetSymbolAddress((void **)&s32, g_sink32) != cudaSuccess ||
      cudaGetSymbolAddress((void **)&s64, g_sink64) != cudaSuccess)
    return DEM_ERR_CUDA;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return DEM_ERR_CUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return DEM_ERR_CUDA;
  }
  float best = 1e30f;
  cudaError_t e = cudaSuccess;
  for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {  // the first run warms up
    cudaEventRecord(e0, s);
    if (precision == 0)
      k_fma_chains<float><<<blocks, threads, 0, s>>>(iters, 0.999999f, 1e-7f, s32);
    else
      k_fma_chains<double><<<blocks, threads, 0, s>>>(iters, 0.999999999, 1e-12, s64);
    cudaEventRecord(e1, s);
    e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0 && ms < best) best = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return DEM_ERR_CUDA;
  const double flops = 2.0 * CH * (double)iters * (double)blocks * threads;
  *flops_per_s = flops / (best * 1e-3);
  return DEM_OK;
}

extern "C" dem_status dem_count_dist_flops(const float *tri, int64_t n, int64_t *ops, void *stream) {
  using namespace dem;
  if (n < 0 || (n > 0 && (!tri || !ops))) return DEM_ERR_ARG;
  if (n == 0) return DEM_OK;
  const int threads = 256, blocks = CNT_THREADS / threads;
  k_count_dist<<<blocks, threads, 0, static_cast<cudaStream_t>(stream)>>>(tri, n, ops);
  return cudaGetLastError() == cudaSuccess ? DEM_OK : DEM_ERR_CUDA;
}
