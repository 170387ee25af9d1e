// noalloc.cu -- candidate pairs without any device allocation.
//
// dem_build_candidates needs a context, and creating a context allocates its
// scratch with cudaMalloc.  Some callers cannot allocate device memory at the
// point where they need candidates: for example a host application that hands
// the whole device memory pool to another framework, or a real-time loop in
// which an allocation could block, fail or be forbidden.  For them this file
// offers dem_build_candidates_noalloc: the same broad-phase kernels, with
// their scratch in a fixed, file-scope device array that exists from the
// moment the library is loaded until the process exits (on every GPU that
// loads the library).
//
// The array is sized for DEM_NOALLOC_MAX_PARTICLES particles (about 5.3 MB).
// Larger inputs are rejected with DEM_ERR_CAPACITY before anything is
// launched.  The first call on each device looks the array's device address
// up with cudaGetSymbolAddress (with that device current); make that first
// call before capturing a stream into a graph.  All calls share the one
// array and it keeps the previous call's contents, so every call clears what
// must start at zero; two calls whose work overlaps on the GPU (other streams,
// other host threads) race on the array and must be serialised by the caller.
// The array's error word is the exception: it collects what the kernels met
// (bad index, non-finite state, capacity) until dem_noalloc_check reads and
// clears it, the context-free counterpart of dem_check.
#include <mutex>

#include "internal.cuh"

namespace dem {
namespace {

constexpr int64_t NA_MAX = DEM_NOALLOC_MAX_PARTICLES;
constexpr int64_t NA_TABLE = 2 * NA_MAX;  // hash buckets (power of two)

// byte layout of the fixed scratch
constexpr size_t align256(size_t v) { return (v + 255) & ~size_t(255); }
constexpr size_t OFF_ERR = 0;
constexpr size_t OFF_STATS = align256(OFF_ERR + sizeof(uint32_t));
constexpr size_t OFF_WORK = align256(OFF_STATS + sizeof(unsigned long long) * ST_N);
constexpr size_t OFF_PART = align256(OFF_WORK + sizeof(unsigned int) * 4);
constexpr size_t OFF_TMP = align256(OFF_PART + sizeof(int64_t) * SCAN_PART_CAP);
constexpr size_t OFF_SPH = align256(OFF_TMP + sizeof(int64_t) * 8);
constexpr size_t OFF_CELL = align256(OFF_SPH + sizeof(Sphere4) * NA_MAX);
constexpr size_t OFF_BCNT = align256(OFF_CELL + sizeof(int4) * NA_MAX);
constexpr size_t OFF_BSTART = align256(OFF_BCNT + sizeof(int32_t) * NA_TABLE);
constexpr size_t OFF_BCUR = align256(OFF_BSTART + sizeof(int64_t) * NA_TABLE);
constexpr size_t OFF_IDS = align256(OFF_BCUR + sizeof(int32_t) * NA_TABLE);
constexpr size_t OFF_BSPH = align256(OFF_IDS + sizeof(int32_t) * NA_MAX);
constexpr size_t OFF_BSPH32 = align256(OFF_BSPH + sizeof(Sphere4) * NA_MAX);
constexpr size_t OFF_BCELL = align256(OFF_BSPH32 + sizeof(float4) * NA_MAX);
constexpr size_t OFF_PCNT = align256(OFF_BCELL + sizeof(int4) * NA_MAX);
constexpr size_t OFF_POFF = align256(OFF_PCNT + sizeof(int64_t) * NA_MAX);
constexpr size_t OFF_RHO = align256(OFF_POFF + sizeof(int64_t) * NA_MAX);
constexpr size_t OFF_SIDS = align256(OFF_RHO + sizeof(unsigned long long));
constexpr size_t OFF_NST = align256(OFF_SIDS + sizeof(int32_t) * NA_MAX);
constexpr size_t OFF_SPOSE = align256(OFF_NST + sizeof(int32_t));
constexpr size_t OFF_SBOX = align256(OFF_SPOSE + sizeof(double) * 12 * NA_MAX);
constexpr size_t OFF_SBOX32 = align256(OFF_SBOX + sizeof(unsigned long long) * 6 * NA_MAX);
constexpr size_t NA_BYTES = align256(OFF_SBOX32 + sizeof(float) * 6 * NA_MAX);

static __device__ __align__(256) unsigned char g_noalloc_scratch[NA_BYTES];

constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
unsigned char *g_base[MAX_DEVICES] = {nullptr};

// device address of the fixed scratch on the current device (looked up once)
cudaError_t scratch_base(unsigned char **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= MAX_DEVICES) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_base[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_base[dev] = static_cast<unsigned char *>(p);
  }
  *out = g_base[dev];
  return cudaSuccess;
}

}  // namespace
}  // namespace dem

extern "C" dem_status dem_build_candidates_noalloc(const dem_particles *P, int32_t *pairs, int64_t cap,
                                                   int64_t *n_pairs, void *stream) {
  using namespace dem;
  // a launch error left on this thread by an earlier, unrelated call would
  // otherwise be reported as this call's: drain it first
  (void)cudaGetLastError();
  if (!P || P->n < 0 || !n_pairs || cap < 0 || (cap > 0 && !pairs)) return DEM_ERR_ARG;
  if (P->n > 0 && (!P->state || !P->tri_off)) return DEM_ERR_ARG;
  if (P->n > NA_MAX) return DEM_ERR_CAPACITY;
  unsigned char *b = nullptr;
  if (scratch_base(&b) != cudaSuccess) return DEM_ERR_CUDA;
  Scratch S;
  S.err = reinterpret_cast<uint32_t *>(b + OFF_ERR);
  S.stats = reinterpret_cast<unsigned long long *>(b + OFF_STATS);
  S.work = reinterpret_cast<unsigned int *>(b + OFF_WORK);
  S.scan_part = reinterpret_cast<int64_t *>(b + OFF_PART);
  S.tmp = reinterpret_cast<int64_t *>(b + OFF_TMP);
  S.cap_particles = NA_MAX;
  S.table_size = NA_TABLE;
  S.sph = reinterpret_cast<Sphere4 *>(b + OFF_SPH);
  S.cell = reinterpret_cast<int4 *>(b + OFF_CELL);
  S.bucket_cnt = reinterpret_cast<int32_t *>(b + OFF_BCNT);
  S.bucket_start = reinterpret_cast<int64_t *>(b + OFF_BSTART);
  S.bucket_cur = reinterpret_cast<int32_t *>(b + OFF_BCUR);
  S.bucket_ids = reinterpret_cast<int32_t *>(b + OFF_IDS);
  S.bucket_sph = reinterpret_cast<Sphere4 *>(b + OFF_BSPH);
  S.bucket_sph32 = reinterpret_cast<float4 *>(b + OFF_BSPH32);
  S.bucket_cell = reinterpret_cast<int4 *>(b + OFF_BCELL);
  S.pcnt = reinterpret_cast<int64_t *>(b + OFF_PCNT);
  S.poff = reinterpret_cast<int64_t *>(b + OFF_POFF);
  S.rho_max = reinterpret_cast<unsigned long long *>(b + OFF_RHO);
  S.static_ids = reinterpret_cast<int32_t *>(b + OFF_SIDS);
  S.n_static = reinterpret_cast<int32_t *>(b + OFF_NST);
  S.spose = reinterpret_cast<double *>(b + OFF_SPOSE);
  S.sbox = reinterpret_cast<unsigned long long *>(b + OFF_SBOX);
  S.sbox32 = reinterpret_cast<float *>(b + OFF_SBOX32);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // the error word collects the conditions met since the last
  // dem_noalloc_check, which reads and clears it
  if (launch_broad(*P, pairs, cap, n_pairs, S, s) != cudaSuccess) return DEM_ERR_CUDA;
  return DEM_OK;
}

extern "C" dem_status dem_noalloc_check(void *stream) {
  using namespace dem;
  (void)cudaGetLastError();
  unsigned char *b = nullptr;
  if (scratch_base(&b) != cudaSuccess) return DEM_ERR_CUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (cudaStreamSynchronize(s) != cudaSuccess) return DEM_ERR_CUDA;
  uint32_t bits = 0;
  // a pageable host target: the copy completes before cudaMemcpy returns,
  // and nothing is allocated
  if (cudaMemcpy(&bits, b + OFF_ERR, sizeof(bits), cudaMemcpyDeviceToHost) != cudaSuccess) return DEM_ERR_CUDA;
  if (!bits) return DEM_OK;
  if (cudaMemset(b + OFF_ERR, 0, sizeof(uint32_t)) != cudaSuccess) return DEM_ERR_CUDA;
  if (bits & ERR_INDEX) return DEM_ERR_INDEX;
  if (bits & ERR_NONFINITE) return DEM_ERR_NONFINITE;
  if (bits & ERR_CAPACITY) return DEM_ERR_CAPACITY;
  return DEM_ERR_TIMEOUT;
}
