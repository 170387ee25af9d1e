// scan.cu -- grid-wide exclusive prefix sums (three launches, no inter-block
// waits): per-block sums, one-block scan of the sums, per-block scan with the
// block's offset.  Up to SCAN_BLOCK * SCAN_PART_CAP elements.
#include "internal.cuh"

namespace dem {

namespace {

constexpr int ST = 256;                       // threads per scan block
constexpr int PER = (int)(SCAN_BLOCK / ST);   // elements per thread

template <class TI>
__global__ void __launch_bounds__(ST) k_block_sums(const TI *in, int64_t n, int64_t *part) {
  __shared__ int64_t red[ST / 32];
  const int64_t base = (int64_t)blockIdx.x * SCAN_BLOCK + (int64_t)threadIdx.x * PER;
  int64_t s = 0;
#pragma unroll
  for (int q = 0; q < PER; ++q)
    if (base + q < n) s += (int64_t)in[base + q];
#pragma unroll
  for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    int64_t t = 0;
    for (int q = 0; q < ST / 32; ++q) t += red[q];
    part[blockIdx.x] = t;
  }
}

// exclusive scan of up to SCAN_PART_CAP partial sums in one block of 1024
__global__ void __launch_bounds__(1024) k_scan_parts(int64_t *part, int64_t np, int64_t *total) {
  __shared__ int64_t wsum[32];
  constexpr int P = (int)(SCAN_PART_CAP / 1024);
  int64_t v[P];
  int64_t s = 0;
  const int64_t base = (int64_t)threadIdx.x * P;
#pragma unroll
  for (int q = 0; q < P; ++q) {
    v[q] = base + q < np ? part[base + q] : 0;
    s += v[q];
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int64_t inc = s;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int64_t y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) wsum[w] = inc;
  __syncthreads();
  if (w == 0) {
    int64_t x = wsum[lane];
    int64_t xi = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t y = __shfl_up_sync(0xffffffffu, xi, o);
      if (lane >= o) xi += y;
    }
    wsum[lane] = xi - x;  // exclusive warp offsets
    if (lane == 31 && total) *total = xi;
  }
  __syncthreads();
  int64_t run = wsum[w] + inc - s;
#pragma unroll
  for (int q = 0; q < P; ++q) {
    if (base + q < np) part[base + q] = run;
    run += v[q];
  }
}

template <class TI>
__global__ void __launch_bounds__(ST) k_apply(const TI *in, int64_t *out, int64_t n, const int64_t *part) {
  __shared__ int64_t wsum[ST / 32];
  const int64_t base = (int64_t)blockIdx.x * SCAN_BLOCK + (int64_t)threadIdx.x * PER;
  int64_t v[PER];
  int64_t s = 0;
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    v[q] = base + q < n ? (int64_t)in[base + q] : 0;
    s += v[q];
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int64_t inc = s;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int64_t y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) wsum[w] = inc;
  __syncthreads();
  if (threadIdx.x == 0) {
    int64_t r = 0;
    for (int q = 0; q < ST / 32; ++q) {
      const int64_t t = wsum[q];
      wsum[q] = r;
      r += t;
    }
  }
  __syncthreads();
  int64_t run = part[blockIdx.x] + wsum[w] + inc - s;
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    if (base + q < n) out[base + q] = run;
    run += v[q];
  }
}

template <class TI>
int scan_impl(const TI *in, int64_t *out, int64_t n, int64_t *total, int64_t *part, cudaStream_t s) {
  if (n <= 0) {
    if (total) cudaMemsetAsync(total, 0, sizeof(int64_t), s);
    return 0;
  }
  const int64_t nb = (n + SCAN_BLOCK - 1) / SCAN_BLOCK;  // callers keep nb <= SCAN_PART_CAP
  k_block_sums<TI><<<(unsigned)nb, ST, 0, s>>>(in, n, part);
  k_scan_parts<<<1, 1024, 0, s>>>(part, nb, total);
  k_apply<TI><<<(unsigned)nb, ST, 0, s>>>(in, out, n, part);
  return 3;
}

}  // namespace

int scan_exclusive_i64(const int64_t *in, int64_t *out, int64_t n, int64_t *total, int64_t *part,
                       cudaStream_t s) {
  return scan_impl<int64_t>(in, out, n, total, part, s);
}

int scan_exclusive_i32_to_i64(const int32_t *in, int64_t *out, int64_t n, int64_t *part, cudaStream_t s) {
  return scan_impl<int32_t>(in, out, n, nullptr, part, s);
}

}  // namespace dem
