// lts.cu -- one sweep of the local-time-stepping cycle (paper Section 2.2
// substeps; Section 3, damped particle steps; Section 4, consolidation;
// Section 5, time step size; cluster masking; snapshot roll-over).
//
// Per-cluster reductions (earliest time stamp, smallest step, new time
// stamp) are atomic minima on order-preserving 64-bit keys of the binary64
// values: a minimum is exact, so the result does not depend on the order in
// which particles or pairs arrive.  Every arithmetic step is the oracle's,
// one rounding at a time, so the sweep equals the oracle's bit for bit.
#include "internal.cuh"

namespace dem {
namespace {

using D = OpsD;
constexpr int SNAP_FIELDS = 14;  // x y z | v | q | w | t_cur: the fields a snapshot rolls over

__device__ __forceinline__ bool is_st(const uint8_t *st, int64_t p) { return st && st[p]; }

// 1. particle steps
__global__ void k_lts_step(int64_t n, double *cur, const double *old, const uint8_t *st, double dt_max,
                           double alpha) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
    if (is_st(st, p)) continue;
    const double tc = cur[13 * n + p], to = old[13 * n + p];
    const double d = tc > to ? D::mul(alpha, D::sub(tc, to)) : dt_max;
    cur[14 * n + p] = d < dt_max ? d : dt_max;
  }
}

// 4a. earliest time stamp and smallest step per cluster
__global__ void k_lts_reduce(int64_t n, const double *cur, const uint8_t *st, const int32_t *ids,
                             unsigned long long *tmin, unsigned long long *step, uint32_t *err) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
    if (is_st(st, p)) continue;
    const int64_t c = ids[p];
    if (c < 0 || c >= n) {
      set_err(err, ERR_INDEX);
      continue;
    }
    atomicMin(&tmin[c], okey(cur[13 * n + p]));
    atomicMin(&step[c], okey(cur[14 * n + p]));
  }
}

// 4b. roll back to the cluster's time stamp, take the cluster step; the
// cluster root seeds the new time stamp with the end of the interval
__global__ void k_lts_consolidate(int64_t n, double *cur, const double *old, const uint8_t *st, const int32_t *ids,
                                  const unsigned long long *tmin, const unsigned long long *step,
                                  unsigned long long *tnew, unsigned long long *stats) {
  __shared__ double rc[POSE_TERMS + 1], rs[POSE_TERMS + 1];
  if (threadIdx.x == 0) pose_reciprocals(rc, rs);
  __syncthreads();
  unsigned long long rb = 0, bad = 0;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
    if (is_st(st, p)) continue;
    const int64_t c = ids[p];
    if (c < 0 || c >= n) continue;  // reported by k_lts_reduce
    const double tm = okey_value(tmin[c]), dc = okey_value(step[c]);
    if (cur[13 * n + p] > tm) {
      double Q[4], X[3];
      pose_quat_exact(old, n, p, tm, rc, rs, Q, X);
      ++rb;
      if (tm < old[13 * n + p]) ++bad;
      for (int k = 0; k < 3; ++k) cur[k * n + p] = X[k];
      for (int k = 0; k < 4; ++k) cur[(6 + k) * n + p] = Q[k];
      cur[13 * n + p] = tm;
    }
    cur[14 * n + p] = dc;
    if (c == p) tnew[c] = okey(D::add(tm, dc));
  }
  if (rb) atomicAdd(&stats[ST_ROLLBACK], rb);
  if (bad) atomicAdd(&stats[ST_ROLLBACK_BAD], bad);
}

__device__ __forceinline__ int64_t pair_total(const int64_t *n_pairs, int64_t max_pairs) {
  const int64_t m = *n_pairs;
  return m < max_pairs ? m : max_pairs;
}

// 6. earliest proper collision per cluster (the first member is never static)
__global__ void k_lts_tnew(int64_t n, const int32_t *pairs, const int64_t *n_pairs, int64_t max_pairs,
                           const uint8_t *status, const double *tcol, const int32_t *ids, unsigned long long *tnew) {
  const int64_t m = pair_total(n_pairs, max_pairs);
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < m; k += (int64_t)gridDim.x * blockDim.x) {
    if (status[k] != 2) continue;
    const int64_t i = pairs[2 * k];
    if (i < 0 || i >= n) continue;
    const int64_t c = ids[i];
    if (c >= 0 && c < n) atomicMin(&tnew[c], okey(tcol[k]));
  }
}

// 7. the masking bound: minimum new time stamp over the cluster roots
__global__ void k_lts_global(int64_t n, const uint8_t *st, const int32_t *ids, const unsigned long long *tnew,
                             unsigned long long *tglob) {
  unsigned long long v = ~0ull;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x)
    if (!is_st(st, p) && ids[p] == p) v = min(v, tnew[p]);
#pragma unroll
  for (int o = 16; o; o >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, o));
  if ((threadIdx.x & 31) == 0 && v != ~0ull) atomicMin(tglob, v);
}

// 8a. particles in contact at the end of their step
__global__ void k_lts_touch(int64_t n, const int32_t *pairs, const int64_t *n_pairs, int64_t max_pairs,
                            const uint8_t *status, const double *tcol, const int32_t *ids, const uint8_t *st,
                            const unsigned long long *tnew, uint8_t *touch) {
  const int64_t m = pair_total(n_pairs, max_pairs);
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < m; k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = pairs[2 * k], j = pairs[2 * k + 1];
    if (i < 0 || i >= n || j < 0 || j >= n) continue;
    const int64_t c = ids[i];
    if (c < 0 || c >= n) continue;
    if (status[k] == 1 || (status[k] == 2 && tcol[k] == okey_value(tnew[c]))) {
      touch[i] = 1;
      if (!is_st(st, j)) touch[j] = 1;
    }
  }
}

// 8b. advance the active clusters, roll the snapshots over, stand-in update
__global__ void k_lts_advance(int64_t n, double *cur, double *old, const uint8_t *st, const int32_t *ids,
                              const unsigned long long *tmin, const unsigned long long *tnew,
                              const unsigned long long *tglob, const uint8_t *touch, double gx, double gy, double gz,
                              int zero_on_contact, uint8_t *active, double *t_global, unsigned long long *stats) {
  __shared__ double rc[POSE_TERMS + 1], rs[POSE_TERMS + 1];
  if (threadIdx.x == 0) pose_reciprocals(rc, rs);
  __syncthreads();
  const double tg = okey_value(*tglob);
  if (blockIdx.x == 0 && threadIdx.x == 0) *t_global = *tglob == ~0ull ? OpsD::inf() : tg;
  unsigned long long adv = 0;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
    active[p] = 0;
    if (is_st(st, p)) continue;
    const int64_t c = ids[p];
    if (c < 0 || c >= n) continue;
    if (!(okey_value(tmin[c]) <= tg)) continue;
    active[p] = 1;
    ++adv;
    const double tn = okey_value(tnew[c]);
    const double h = D::sub(tn, cur[13 * n + p]);
#pragma unroll
    for (int q = 0; q < SNAP_FIELDS; ++q) old[q * n + p] = cur[q * n + p];
    double Q[4], X[3];
    pose_quat_exact(old, n, p, tn, rc, rs, Q, X);
    for (int k = 0; k < 3; ++k) cur[k * n + p] = X[k];
    for (int k = 0; k < 4; ++k) cur[(6 + k) * n + p] = Q[k];
    cur[13 * n + p] = tn;
    if (zero_on_contact && touch[p]) {
      for (int k = 3; k < 6; ++k) cur[k * n + p] = 0.0;
      for (int k = 10; k < 13; ++k) cur[k * n + p] = 0.0;
    } else {
      cur[3 * n + p] = D::add(cur[3 * n + p], D::mul(gx, h));
      cur[4 * n + p] = D::add(cur[4 * n + p], D::mul(gy, h));
      cur[5 * n + p] = D::add(cur[5 * n + p], D::mul(gz, h));
    }
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) adv += __shfl_xor_sync(0xffffffffu, adv, o);
  if ((threadIdx.x & 31) == 0 && adv) atomicAdd(&stats[ST_ADVANCE], adv);
}

}  // namespace

cudaError_t launch_lts(int prec, int method, int K, double tol, const dem_particles &P, double *cur, double *old,
                       const dem_lts_params &prm, const dem_lts_out &out, Scratch &S, int num_sms, cudaStream_t s) {
  const int64_t n = P.n;
  cudaError_t e;
  const size_t kb = sizeof(unsigned long long) * (size_t)(n > 0 ? n : 1);
  if ((e = cudaMemsetAsync(S.lts_tmin, 0xff, kb, s)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(S.lts_step, 0xff, kb, s)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(S.lts_tnew, 0xff, kb, s)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(S.lts_tglob, 0xff, sizeof(unsigned long long), s)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(S.lts_touch, 0, (size_t)(n > 0 ? n : 1), s)) != cudaSuccess) return e;
  const int tb = 256;
  const unsigned grid = (unsigned)(n > 0 ? (n + tb - 1) / tb : 1);
  const unsigned pgrid = (unsigned)(out.max_pairs > 0 ? (out.max_pairs + tb - 1) / tb : 1);
  int rec = trace_begin(S, TR_LTS, s);
  k_lts_step<<<grid, tb, 0, s>>>(n, cur, old, P.is_static, prm.dt_max, prm.alpha);
  S.launches += 1;
  trace_end(S, rec, s);
  if ((e = launch_broad(P, out.pairs, out.max_pairs, out.n_pairs, S, s, prm.hose ? old : nullptr)) != cudaSuccess)
    return e;
  if ((e = launch_clusters(n, out.pairs, out.max_pairs, out.n_pairs, P.is_static, out.cluster_id, out.n_clusters, S,
                           s)) != cudaSuccess)
    return e;
  rec = trace_begin(S, TR_LTS, s);
  k_lts_reduce<<<grid, tb, 0, s>>>(n, cur, P.is_static, out.cluster_id, S.lts_tmin, S.lts_step, S.err);
  k_lts_consolidate<<<grid, tb, 0, s>>>(n, cur, old, P.is_static, out.cluster_id, S.lts_tmin, S.lts_step, S.lts_tnew,
                                        S.stats);
  S.launches += 2;
  trace_end(S, rec, s);
  if (out.max_pairs > 0 && out.narrow && method == DEM_CTIME_SAMPLES) {
    // narrow phase at the pair start and collision times in one launch
    if ((e = launch_detect(prec, P, out.pairs, out.max_pairs, out.n_pairs, *out.narrow, K, tol, out.t_coll,
                           out.status, out.tri_ab, S, num_sms, s)) != cudaSuccess)
      return e;
  } else if (out.max_pairs > 0) {
    if (out.narrow &&
        (e = launch_narrow(prec, P, out.pairs, out.max_pairs, out.n_pairs, nullptr, *out.narrow, S, num_sms, s)) !=
            cudaSuccess)
      return e;
    if ((e = launch_ctime(prec, method, P, out.pairs, out.max_pairs, out.n_pairs, K, tol, out.t_coll, out.status, out.tri_ab,
                          S, num_sms, s)) != cudaSuccess)
      return e;
  }
  rec = trace_begin(S, TR_LTS, s);
  if (out.max_pairs > 0) {
    k_lts_tnew<<<pgrid, tb, 0, s>>>(n, out.pairs, out.n_pairs, out.max_pairs, out.status, out.t_coll,
                                    out.cluster_id, S.lts_tnew);
    S.launches += 1;
  }
  k_lts_global<<<grid, tb, 0, s>>>(n, P.is_static, out.cluster_id, S.lts_tnew, S.lts_tglob);
  S.launches += 1;
  if (out.max_pairs > 0) {
    k_lts_touch<<<pgrid, tb, 0, s>>>(n, out.pairs, out.n_pairs, out.max_pairs, out.status, out.t_coll,
                                     out.cluster_id, P.is_static, S.lts_tnew, S.lts_touch);
    S.launches += 1;
  }
  k_lts_advance<<<grid, tb, 0, s>>>(n, cur, old, P.is_static, out.cluster_id, S.lts_tmin, S.lts_tnew, S.lts_tglob,
                                    S.lts_touch, prm.gravity[0], prm.gravity[1], prm.gravity[2],
                                    prm.zero_on_contact, out.active, out.t_global, S.stats);
  S.launches += 1;
  trace_end(S, rec, s);
  return cudaGetLastError();
}

}  // namespace dem
