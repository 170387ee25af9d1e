// internal.cuh -- declarations shared by the library's translation units.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "dem.h"
#include "geom.cuh"

namespace dem {

// sticky device error bits (context error word)
constexpr uint32_t ERR_CAPACITY = 1u;   // an output capacity was exceeded
constexpr uint32_t ERR_TIMEOUT = 2u;    // a bounded wait ran out
constexpr uint32_t ERR_INDEX = 4u;      // an index out of range was met
constexpr uint32_t ERR_NONFINITE = 8u;  // a state field or a vertex is NaN or infinite
constexpr uint32_t ERR_DRAIN = 16u;     // after a timeout, the wait for the copy in flight also ran out

// polls of the first bounded wait on a tile copy (the wait that follows a
// timeout, for the copy in flight to land, always uses this default)
constexpr uint32_t WAIT_POLLS_DEFAULT = 1u << 22;

// counters, same order as dem_stats
enum {
  ST_SPHERE = 0,
  ST_GROUP,
  ST_FP32,
  ST_FP64,
  ST_EVALS,
  ST_CHECKS,
  ST_BISECT,
  ST_CONTACTS,
  ST_PAIRS,
  ST_HOST_LAUNCHES,  // slot of dem_stats.kernel_launches (host-side count)
  ST_TILES,
  ST_ROLLBACK,
  ST_ROLLBACK_BAD,
  ST_ADVANCE,
  ST_BUSY,      // pair kernel: CTA busy time (ns), summed
  ST_BUSYMAX,   // ... its maximum (atomicMax)
  ST_CTAS,      // ... CTAs counted
  ST_N = 18
};

// swept sphere of a particle (centre, radius), binary64
struct __align__(32) Sphere4 {
  double x, y, z, w;
};

// Launch groups timed by the trace (dem_trace): CUDA events recorded on the
// launching stream before and after each group, also inside a stream capture
// (as event-record nodes of the graph).
enum {
  TR_BROAD = DEM_TR_BROAD,
  TR_TILES = DEM_TR_TILES,
  TR_PAIRS = DEM_TR_PAIRS,
  TR_CONTACTS = DEM_TR_CONTACTS,
  TR_CLUSTERS = DEM_TR_CLUSTERS,
  TR_LTS = DEM_TR_LTS
};

struct Trace {
  int cap = 0;                    // records available
  int n = 0;                      // records taken since the trace was (re)started
  cudaEvent_t *ev = nullptr;      // [2 * cap] begin / end of each record
  int32_t *site = nullptr;        // [cap] launch group of each record
};

// launch configuration of the pair kernel, per precision and mode
// (autotuned by dem_autotune): CTAs per SM of the persistent grid (0 = as
// many as fit), warp candidate-list flush size, pairs handed out costliest
// first (by triangle counts) or in index order
struct Tune {
  int ctas_per_sm = 0;
  int wflush = 64;
  int order = 1;
};
constexpr int N_MODES = 4;  // narrow phase, collision times, both, narrowing

struct Scratch {
  Trace *trace = nullptr;         // launch-group timing (null: off)
  Tune tune[2][N_MODES];          // [precision][mode]
  int32_t *order = nullptr;       // [cap_pairs] hand-out order of the pair kernel
  unsigned long long *ilg = nullptr;  // [MAX_PAIR_CTAS][ilg_cap] spill of the pair-interval lists
  int64_t ilg_cap = 0;
  uint8_t *cost_bucket = nullptr; // [cap_pairs] cost class of each pair
  unsigned int *cost_hist = nullptr;  // [128] counts (64) and cursors (64) of the cost classes
  int64_t launches = 0;           // host-side count of kernel launches issued
  uint32_t wait_polls = WAIT_POLLS_DEFAULT;  // first bounded wait of the pair kernel's tile copies
  // common
  uint32_t *err;                  // [1]
  unsigned long long *stats;      // [ST_N]
  unsigned int *work;             // [4] work counters of persistent kernels
  // scan temporaries
  int64_t *scan_part;             // [SCAN_PART_CAP]
  int64_t *tmp;                   // [8] device scalars (totals)
  // broad phase
  int64_t cap_particles;
  int64_t table_size;             // hash buckets (power of two)
  Sphere4 *sph;                   // [n] swept spheres (mx, my, mz, rho)
  int4 *cell;                     // [n] (cx, cy, cz, bucket)
  int32_t *bucket_cnt;            // [table]
  int64_t *bucket_start;          // [table]
  int32_t *bucket_cur;            // [table]
  int32_t *bucket_ids;            // [n] moving particles in bucket order
  Sphere4 *bucket_sph;            // [n] their swept spheres, same order
  float4 *bucket_sph32;           // [n] the same spheres rounded to FP32
  int4 *bucket_cell;              // [n] their cells, same order
  int64_t *pcnt;                  // [n] candidates per particle
  int64_t *poff;                  // [n]
  int32_t *pcache = nullptr;      // [n][PCACHE] partners found by the count pass (optional)
  uint8_t *pcache_ok = nullptr;   // [n] 1: the particle's partners are all in pcache
  unsigned long long *rho_max;    // [1] (bits of a non-negative double)
  int32_t *static_ids;            // [n] static particles, in order of discovery
  int32_t *n_static;              // [1]
  double *spose;                  // [n][12] rotation (row-major) and centre of each static at t_cur
  unsigned long long *sbox;       // [n][6] order keys of its world-vertex extremes (min xyz, max xyz),
                                  // then the bits of the widened box (lo xyz, hi xyz, binary64)
  float *sbox32;                  // [n][6] the widened box rounded outwards to FP32
  // narrow phase
  int64_t cap_pairs;
  int64_t cap_contacts;
  int32_t *st_keys;               // [cap_contacts][3] staging
  double *st_geom;                // [cap_contacts][7]
  unsigned long long *st_count;   // [1]
  int64_t *pc;                    // [cap_pairs] contacts per pair
  int64_t *po;                    // [cap_pairs] exclusive offsets
  int32_t *pcur;                  // [cap_pairs] scatter cursors
  int32_t *sidx;                  // [cap_contacts] staging index per output slot
  // bounding spheres of the TILE_TRIS-triangle tiles of particles with more
  // than one tile (body frame: centre, radius); tile k of particle p is slot
  // tri_off[p] / TILE_TRIS + p + k, distinct for every (p, k)
  int64_t cap_triangles;
  int64_t cap_tiles;
  float4 *tile_sph;               // [cap_tiles]
  float4 *tile_box;               // [cap_tiles][2] body-frame box (lo xyz, hi xyz) of the tile's vertices
  int2 *tile_list;                // [cap_tiles] (particle, tile) entries to compute
  // local time stepping: per-cluster order keys (indexed by cluster id)
  unsigned long long *lts_tmin;   // [n] earliest t_cur of the cluster
  unsigned long long *lts_step;   // [n] smallest member step
  unsigned long long *lts_tnew;   // [n] new time stamp
  unsigned long long *lts_tglob;  // [1] minimum of the new time stamps
  uint8_t *lts_touch;             // [n] particle in contact at the end of its step
};

constexpr int TILE_TRIS = 320;                 // triangles per shared-memory tile of the pair kernel
constexpr int MAX_PAIR_CTAS_PER_SM = 4;        // persistent CTAs of the pair kernel per SM, at most
constexpr int PCACHE = 8;                      // partners per particle the broad phase's count pass keeps
constexpr int64_t SCAN_BLOCK = 2048;           // elements per scan block
constexpr int64_t SCAN_PART_CAP = 4096;        // partial sums (=> up to 8M elements)

// exclusive scan of n int64 values (in may alias out); total written to
// *total if non-null.  Grid-wide, no inter-block waits.
// return the number of kernels launched
int scan_exclusive_i64(const int64_t *in, int64_t *out, int64_t n, int64_t *total,
                       int64_t *part, cudaStream_t s);
int scan_exclusive_i32_to_i64(const int32_t *in, int64_t *out, int64_t n, int64_t *part,
                              cudaStream_t s);

// trace records around a launch group (no-ops when the trace is off or
// full); trace_begin returns the record index or -1
int trace_begin(Scratch &S, int site, cudaStream_t s);
void trace_end(Scratch &S, int rec, cudaStream_t s);

// launchers
// hose_old: the old snapshots for the space-time hose test of moving pairs
// (nullptr: the swept-sphere and box tests alone)
cudaError_t launch_broad(const dem_particles &P, int32_t *pairs, int64_t cap, int64_t *n_pairs,
                         Scratch &S, cudaStream_t s, const double *hose_old = nullptr);
cudaError_t launch_narrow(int prec, const dem_particles &P, const int32_t *pairs, int64_t max_pairs,
                          const int64_t *n_pairs, const double *t_eval, const dem_narrow_out &out,
                          Scratch &S, int num_sms, cudaStream_t s);
cudaError_t launch_detect(int prec, const dem_particles &P, const int32_t *pairs, int64_t max_pairs,
                          const int64_t *n_pairs, const dem_narrow_out &out, int K, double tol, double *t_coll,
                          uint8_t *status, int32_t *tri_ab, Scratch &S, int num_sms, cudaStream_t s);
cudaError_t launch_ctime(int prec, int method, const dem_particles &P, const int32_t *pairs, int64_t max_pairs,
                         const int64_t *n_pairs, int K, double tol, double *t_coll,
                         uint8_t *status, int32_t *tri_ab, Scratch &S, int num_sms,
                         cudaStream_t s);
cudaError_t launch_clusters(int64_t n, const int32_t *edges, int64_t max_edges,
                            const int64_t *n_edges, const uint8_t *is_static, int32_t *id,
                            int64_t *n_clusters, Scratch &S, cudaStream_t s);
cudaError_t launch_lts(int prec, int method, int K, double tol, const dem_particles &P, double *cur, double *old,
                       const dem_lts_params &prm, const dem_lts_out &out, Scratch &S, int num_sms,
                       cudaStream_t s);

__device__ __forceinline__ void set_err(uint32_t *err, uint32_t bit) { atomicOr(err, bit); }

// order-preserving unsigned key of a double (atomic min / max of doubles)
__device__ __forceinline__ unsigned long long okey(double x) {
  const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(x));
  return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
__device__ __forceinline__ double okey_value(unsigned long long k) {
  return __longlong_as_double(static_cast<long long>((k >> 63) ? (k & 0x7fffffffffffffffull) : ~k));
}

}  // namespace dem
