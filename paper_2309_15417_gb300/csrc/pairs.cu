// pairs.cu -- host side of the pair kernel (launchers for the narrow phase,
// collision times and the fused form), the contact sort and the tile
// bounding spheres.  The kernel itself is in pair_kernel.cuh; its
// instantiations are compiled in pairs_fp32_*.cu and pairs_fp64_*.cu.
#include "pair_kernel.cuh"

namespace dem {
namespace pk {

extern template cudaError_t launch_pairs<0, MODE_NARROW>(const PairArgs &, int, cudaStream_t);
extern template cudaError_t launch_pairs<0, MODE_CTIME>(const PairArgs &, int, cudaStream_t);
extern template cudaError_t launch_pairs<0, MODE_BOTH>(const PairArgs &, int, cudaStream_t);
extern template cudaError_t launch_pairs<0, MODE_NTIME>(const PairArgs &, int, cudaStream_t);
extern template cudaError_t launch_pairs<1, MODE_NARROW>(const PairArgs &, int, cudaStream_t);
extern template cudaError_t launch_pairs<1, MODE_CTIME>(const PairArgs &, int, cudaStream_t);
extern template cudaError_t launch_pairs<1, MODE_BOTH>(const PairArgs &, int, cudaStream_t);
extern template cudaError_t launch_pairs<1, MODE_NTIME>(const PairArgs &, int, cudaStream_t);

constexpr int SORT_CAP = 4096;

// Contact candidates of the FP32 mode, decided in binary64: the feature the
// FP32 pass found closest (its binary64 value within eps_pair makes the
// pair's binary64 distance within it), else the full binary64 triangle
// distance.  The pose of both particles at the pair's evaluation time is
// recomputed here exactly as the pair kernel computes it.  Accepted
// candidates get their binary64 distance and points and are counted per
// pair; rejected ones are marked (pair index -1).
__global__ void __launch_bounds__(256) contact_verify(const PairArgs A) {
  __shared__ double rc[POSE_TERMS + 1], rs[POSE_TERMS + 1];
  if (threadIdx.x == 0) pose_reciprocals(rc, rs);
  __syncthreads();
  using GD = Geo<OpsD>;
  using D = OpsD;
  const int64_t nst = min((int64_t)*A.st_count, A.st_cap);
  const int64_t n = A.n;
  const double *st = A.st;
  unsigned long long n64 = 0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nst; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t pk = A.st_keys[3 * e];
    const int a = A.st_keys[3 * e + 1], b = A.st_keys[3 * e + 2];
    const int feat = int(A.st_geom[7 * e]);
    const int64_t i = A.pairs[2 * pk], j = A.pairs[2 * pk + 1];
    const double eps = D::add(st[15 * n + i], st[15 * n + j]);
    double t;
    if (A.t_eval) {
      t = A.t_eval[pk];
    } else {  // the pair start, as the pair kernel sets it
      const double ti = st[13 * n + i], tj = st[13 * n + j];
      const bool si = A.is_static && A.is_static[i], sj = A.is_static && A.is_static[j];
      t = (sj && !si) ? ti : ((si && !sj) ? tj : (ti < tj ? ti : tj));
    }
    double RA[9], XA[3], RB[9], XB[3];
    pose_exact(st, n, i, t, rc, rs, RA, XA);
    pose_exact(st, n, j, t, rc, rs, RB, XB);
    const int64_t oa = A.tri_off[i], ob = A.tri_off[j];
    V3<double> X[3], Y[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      const float4 f = A.tris[q * A.n_tris + oa + a], g = A.tris[q * A.n_tris + ob + b];
      X[q] = to_world_exact(RA, XA, f.x, f.y, f.z);
      Y[q] = to_world_exact(RB, XB, g.x, g.y, g.z);
    }
    V3<double> pa, pb;
    double e2 = GD::feature_dist2(feat, X, Y, pa, pb);
    ++n64;
    double dd = D::sqrt(e2);
    if (!(dd <= eps)) {
      e2 = GD::tri_dist2(X, Y, pa, pb);
      dd = D::sqrt(e2);
    }
    if (dd <= eps) {
      atomicAdd(reinterpret_cast<unsigned long long *>(&A.pc[pk]), 1ull);
      double *gg = A.st_geom + 7 * e;
      gg[0] = dd;
      gg[1] = pa.x; gg[2] = pa.y; gg[3] = pa.z;
      gg[4] = pb.x; gg[5] = pb.y; gg[6] = pb.z;
    } else {
      A.st_keys[3 * e] = -1;
    }
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) n64 += __shfl_xor_sync(0xffffffffu, n64, o);
  if ((threadIdx.x & 31) == 0 && n64) atomicAdd(&A.stats[ST_FP64], n64);
}

__global__ void contact_scatter(const int32_t *st_keys, const unsigned long long *st_count, int64_t st_cap,
                                const int64_t *po, int32_t *pcur, int32_t *sidx, int64_t cap,
                                uint32_t *err) {
  const int64_t nst = min((int64_t)*st_count, st_cap);
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nst;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int32_t pk = st_keys[3 * e];
    if (pk < 0) continue;  // a candidate the binary64 decision rejected
    const int64_t slot = po[pk] + atomicAdd(&pcur[pk], 1);
    if (slot < cap) sidx[slot] = int32_t(e);
  }
}

__global__ void __launch_bounds__(256) contact_sort(const int32_t *st_keys, const double *st_geom,
                                                   int64_t st_cap, const int64_t *pc, const int64_t *po,
                                                   const int64_t *n_pairs, int64_t max_pairs,
                                                   const int32_t *sidx, int32_t *out_keys,
                                                   double *out_geom, int64_t cap, uint32_t *err) {
  __shared__ unsigned long long key[SORT_CAP];
  __shared__ int32_t val[SORT_CAP];
  int64_t m = max_pairs;
  if (n_pairs) m = min(m, *n_pairs);
  for (int64_t pk = blockIdx.x; pk < m; pk += gridDim.x) {
    const int64_t cnt = pc[pk], base = po[pk];
    if (cnt == 0) continue;
    if (base + cnt > cap) {
      if (threadIdx.x == 0) set_err(err, ERR_CAPACITY);
      continue;
    }
    if (cnt > SORT_CAP) {  // too many for the shared-memory sort: copy unsorted, flag
      if (threadIdx.x == 0) set_err(err, ERR_CAPACITY);
      for (int64_t q = threadIdx.x; q < cnt; q += blockDim.x) {
        const int e = sidx[base + q];
        if (e < 0 || e >= st_cap) continue;
        const int64_t o = base + q;
        out_keys[3 * o] = int32_t(pk);
        out_keys[3 * o + 1] = st_keys[3 * (int64_t)e + 1];
        out_keys[3 * o + 2] = st_keys[3 * (int64_t)e + 2];
        for (int c = 0; c < 7; ++c) out_geom[7 * o + c] = st_geom[7 * (int64_t)e + c];
      }
      __syncthreads();
      continue;
    }
    int n2 = 1;
    while (n2 < cnt) n2 <<= 1;
    for (int q = threadIdx.x; q < n2; q += blockDim.x) {
      const int e = q < cnt ? sidx[base + q] : -1;
      if (e >= 0 && e < st_cap) {
        key[q] = (static_cast<unsigned long long>(static_cast<uint32_t>(st_keys[3 * (int64_t)e + 1])) << 32) |
                 static_cast<uint32_t>(st_keys[3 * (int64_t)e + 2]);
        val[q] = e;
      } else {
        key[q] = ~0ull;
        val[q] = -1;
      }
    }
    __syncthreads();
    for (int k = 2; k <= n2; k <<= 1)
      for (int j = k >> 1; j > 0; j >>= 1) {
        for (int q = threadIdx.x; q < n2; q += blockDim.x) {
          const int l = q ^ j;
          if (l > q) {
            const bool up = (q & k) == 0;
            const unsigned long long kq = key[q], kl = key[l];
            if ((kq > kl) == up) {
              key[q] = kl;
              key[l] = kq;
              const int32_t t = val[q];
              val[q] = val[l];
              val[l] = t;
            }
          }
        }
        __syncthreads();
      }
    for (int q = threadIdx.x; q < cnt; q += blockDim.x) {
      const int e = val[q];
      if (e < 0) continue;
      const int64_t o = base + q;
      out_keys[3 * o] = int32_t(pk);
      out_keys[3 * o + 1] = st_keys[3 * e + 1];
      out_keys[3 * o + 2] = st_keys[3 * e + 2];
      for (int c = 0; c < 7; ++c) out_geom[7 * o + c] = st_geom[7 * (int64_t)e + c];
    }
    __syncthreads();
  }
}

// The number of contacts; if the staging area overflowed, the number staged
// instead (FP32 mode: candidates, at least the contacts), a capacity that
// suffices for calling again
__global__ void contact_total(const int64_t *total, const unsigned long long *st_count, int64_t st_cap,
                              int64_t *n_contacts, uint32_t *err) {
  const int64_t t = *total;
  const int64_t staged = (int64_t)*st_count;
  *n_contacts = staged > st_cap ? (staged > t ? staged : t) : t;
  if (staged > st_cap) set_err(err, ERR_CAPACITY);
}

// Tiles of the particles with more than one tile, listed as (particle, tile)
// entries (the order of the list does not matter: each entry writes its own
// slot), then their bounding spheres with one warp per tile.
__global__ void k_tile_list(int64_t n, const int64_t *tri_off, int64_t n_tris, int2 *list, int64_t cap_tiles,
                            unsigned long long *count, uint32_t *err) {
  constexpr int TT = TILE_TRIS;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
    const int64_t o = tri_off[p], cnt = tri_off[p + 1] - o;
    if (cnt <= TT) continue;
    if (o < 0 || o + cnt > n_tris) {
      set_err(err, ERR_INDEX);
      continue;
    }
    const int64_t nt = (cnt + TT - 1) / TT;
    const unsigned long long base = atomicAdd(count, (unsigned long long)nt);
    for (int64_t k = 0; k < nt; ++k) {
      if ((int64_t)(base + k) >= cap_tiles || o / TT + p + k >= cap_tiles) {
        set_err(err, ERR_CAPACITY);
        break;
      }
      list[base + k] = make_int2(int(p), int(k));
    }
  }
}

// Bounding sphere of one listed tile per warp: centre = the middle of the
// vertices' bounding box, radius = the largest centre-vertex distance,
// enlarged by 2^-20 relative (and 1e-18 absolute) so that it covers every
// float32 vertex despite the rounding of its own computation.
__global__ void k_tile_spheres(const int64_t *tri_off, const float4 *tris, int64_t n_tris, const int2 *list,
                               const unsigned long long *count, float4 *tile_sph, float4 *tile_box,
                               int64_t cap_tiles) {
  constexpr int TT = TILE_TRIS;
  const int lane = threadIdx.x & 31;
  const int64_t nwarp = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t m = (int64_t)(*count < (unsigned long long)cap_tiles ? *count : (unsigned long long)cap_tiles);
  for (int64_t e = (((int64_t)blockIdx.x * blockDim.x) + threadIdx.x) >> 5; e < m; e += nwarp) {
    const int2 pk = list[e];
    const int64_t p = pk.x, k = pk.y;
    const int64_t o = tri_off[p], cnt = tri_off[p + 1] - o;
    const int64_t slot = o / TT + p + k;
    if (slot >= cap_tiles) continue;
    const int64_t t0 = o + k * TT, mt = cnt - k * TT < TT ? cnt - k * TT : TT;
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t t = lane; t < mt; t += 32)
#pragma unroll
      for (int v = 0; v < 3; ++v) {
        const float4 f = tris[v * n_tris + t0 + t];
        lo[0] = fminf(lo[0], f.x);
        lo[1] = fminf(lo[1], f.y);
        lo[2] = fminf(lo[2], f.z);
        hi[0] = fmaxf(hi[0], f.x);
        hi[1] = fmaxf(hi[1], f.y);
        hi[2] = fmaxf(hi[2], f.z);
      }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      lo[c] = seg_min(lo[c], 32);
      hi[c] = seg_max(hi[c], 32);
    }
    const float cx = 0.5f * (lo[0] + hi[0]), cy = 0.5f * (lo[1] + hi[1]), cz = 0.5f * (lo[2] + hi[2]);
    float r2 = 0.f;
    for (int64_t t = lane; t < mt; t += 32)
#pragma unroll
      for (int v = 0; v < 3; ++v) {
        const float4 f = tris[v * n_tris + t0 + t];
        const float dx = f.x - cx, dy = f.y - cy, dz = f.z - cz;
        r2 = fmaxf(r2, dx * dx + dy * dy + dz * dz);
      }
    r2 = seg_max(r2, 32);
    if (lane == 0) {
      tile_sph[slot] = make_float4(cx, cy, cz, sqrtf(r2) * (1.0f + 0x1p-20f) + 1e-18f);
      tile_box[2 * slot] = make_float4(lo[0], lo[1], lo[2], 0.f);  // exact: extremes of float32 values
      tile_box[2 * slot + 1] = make_float4(hi[0], hi[1], hi[2], 0.f);
    }
  }
}

// returns the error of the first call that failed
cudaError_t prepare_tiles(const dem_particles &P, Scratch &S, cudaStream_t s) {
  if (P.n <= 0) return cudaSuccess;
  const int rec = trace_begin(S, TR_TILES, s);
  unsigned long long *count = reinterpret_cast<unsigned long long *>(S.tmp + 4);
  cudaError_t e = cudaMemsetAsync(count, 0, sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  const unsigned grid = (unsigned)((P.n + 255) / 256);
  k_tile_list<<<grid, 256, 0, s>>>(P.n, P.tri_off, P.n_tris, S.tile_list, S.cap_tiles, count, S.err);
  k_tile_spheres<<<1216, 256, 0, s>>>(P.tri_off, reinterpret_cast<const float4 *>(P.tris), P.n_tris, S.tile_list,
                                      count, S.tile_sph, S.tile_box, S.cap_tiles);
  S.launches += 2;
  trace_end(S, rec, s);
  return cudaGetLastError();
}


// Hand-out order of the persistent pair kernel: pairs by decreasing cost
// class (leading zeros of T_i * T_j, so each class spans a factor of two),
// a counting sort over 64 classes; the order inside a class is that of the
// atomic cursors (it does not affect any result, only the schedule).
__global__ void k_cost_class(const int32_t *pairs, const int64_t *n_pairs, int64_t max_pairs,
                             const int64_t *tri_off, int64_t n, uint8_t *bucket, unsigned int *hist) {
  int64_t m = max_pairs;
  if (n_pairs) m = min(m, *n_pairs);
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < m; k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = pairs[2 * k], j = pairs[2 * k + 1];
    unsigned long long cost = 0;
    if (i >= 0 && j >= 0 && i < n && j < n) {
      const int64_t a = tri_off[i + 1] - tri_off[i], b = tri_off[j + 1] - tri_off[j];
      if (a > 0 && b > 0) cost = (unsigned long long)a * (unsigned long long)b;
    }
    const int c = cost ? __clzll(cost) : 63;  // 0 .. 63, costliest first
    bucket[k] = uint8_t(c);
    atomicAdd(&hist[c], 1u);
  }
}

__global__ void k_cost_offsets(unsigned int *hist) {
  if (threadIdx.x == 0) {
    unsigned int acc = 0;
    for (int c = 0; c < 64; ++c) {
      const unsigned int v = hist[c];
      hist[c] = acc;       // start of class c
      hist[64 + c] = 0u;   // its cursor
      acc += v;
    }
  }
}

__global__ void k_cost_scatter(const int64_t *n_pairs, int64_t max_pairs, const uint8_t *bucket, unsigned int *hist,
                               int32_t *order) {
  int64_t m = max_pairs;
  if (n_pairs) m = min(m, *n_pairs);
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < m; k += (int64_t)gridDim.x * blockDim.x) {
    const int c = bucket[k];
    order[hist[c] + atomicAdd(&hist[64 + c], 1u)] = int32_t(k);
  }
}

cudaError_t prepare_order(const dem_particles &P, const int32_t *pairs, int64_t max_pairs, const int64_t *n_pairs,
                          Scratch &S, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(S.cost_hist, 0, sizeof(unsigned int) * 128, s);
  if (e != cudaSuccess) return e;
  const unsigned grid = (unsigned)((max_pairs + 255) / 256);
  k_cost_class<<<grid, 256, 0, s>>>(pairs, n_pairs, max_pairs, P.tri_off, P.n, S.cost_bucket, S.cost_hist);
  k_cost_offsets<<<1, 32, 0, s>>>(S.cost_hist);
  k_cost_scatter<<<grid, 256, 0, s>>>(n_pairs, max_pairs, S.cost_bucket, S.cost_hist, S.order);
  S.launches += 3;
  return cudaGetLastError();
}

PairArgs make_args(const dem_particles &P, const int32_t *pairs, int64_t max_pairs, const int64_t *n_pairs,
                   Scratch &S, int prec, int mode) {
  PairArgs a{};
  const Tune &t = S.tune[prec][mode];
  a.order = t.order ? S.order : nullptr;
  a.wflush = t.wflush == 32 ? 32 : 64;
  a.ctas_per_sm = t.ctas_per_sm;
  a.n = P.n;
  a.st = P.state;
  a.is_static = P.is_static;
  a.tri_off = P.tri_off;
  a.tris = reinterpret_cast<const float4 *>(P.tris);
  a.n_tris = P.n_tris;
  a.pairs = pairs;
  a.max_pairs = max_pairs;
  a.n_pairs = n_pairs;
  a.tile_sph = S.tile_sph;
  a.tile_box = S.tile_box;
  a.cap_tiles = S.cap_tiles;
  a.work = S.work;
  a.err = S.err;
  a.stats = S.stats;
  a.wait_polls = S.wait_polls;
  a.ilg = S.ilg;
  a.ilg_cap = S.ilg_cap;
  return a;
}

}  // namespace pk

using namespace pk;

// memsets, the pair kernel (narrow or fused mode), contact offsets, scatter
// and per-pair sort
cudaError_t finish_narrow(int prec, PairArgs &a, const dem_particles &P, const int32_t *pairs, int64_t max_pairs,
                          const int64_t *n_pairs, const dem_narrow_out &out, Scratch &S, int num_sms,
                          cudaStream_t s, bool fused) {
  cudaError_t e;
  if ((e = cudaMemsetAsync(S.work, 0, sizeof(unsigned int), s)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(S.st_count, 0, sizeof(unsigned long long), s)) != cudaSuccess) return e;
  if (max_pairs > 0) {
    if ((e = cudaMemsetAsync(S.pc, 0, sizeof(int64_t) * max_pairs, s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(S.pcur, 0, sizeof(int32_t) * max_pairs, s)) != cudaSuccess) return e;
    if ((e = prepare_tiles(P, S, s)) != cudaSuccess) return e;
    if (a.order && (e = prepare_order(P, pairs, max_pairs, n_pairs, S, s)) != cudaSuccess) return e;
    const int rec = trace_begin(S, TR_PAIRS, s);
    if (fused)
      e = prec == 0 ? launch_pairs<0, MODE_BOTH>(a, num_sms, s) : launch_pairs<1, MODE_BOTH>(a, num_sms, s);
    else
      e = prec == 0 ? launch_pairs<0, MODE_NARROW>(a, num_sms, s) : launch_pairs<1, MODE_NARROW>(a, num_sms, s);
    if (e != cudaSuccess) return e;
    trace_end(S, rec, s);
    S.launches += 1;
  }
  // per-pair offsets, scatter, sort (FP32 mode: the candidates decided in
  // binary64 first)
  const int rec_c = trace_begin(S, TR_CONTACTS, s);
  if (prec == 0 && max_pairs > 0) {
    contact_verify<<<num_sms * 8, 256, 0, s>>>(a);
    S.launches += 1;
  }
  int64_t *total = S.tmp;
  if (max_pairs > 0) {
    S.launches += scan_exclusive_i64(S.pc, S.po, max_pairs, total, S.scan_part, s);
  } else {
    if ((e = cudaMemsetAsync(total, 0, sizeof(int64_t), s)) != cudaSuccess) return e;
  }
  if (max_pairs > 0) {
    const int64_t ocap = out.contact_cap < S.cap_contacts ? out.contact_cap : S.cap_contacts;
    contact_scatter<<<num_sms * 4, 256, 0, s>>>(S.st_keys, S.st_count, S.cap_contacts, S.po, S.pcur, S.sidx, ocap,
                                                S.err);
    contact_sort<<<num_sms * 4, 256, 0, s>>>(S.st_keys, S.st_geom, S.cap_contacts, S.pc, S.po, n_pairs,
                                             max_pairs, S.sidx, out.contacts, out.contact_geom, ocap, S.err);
    S.launches += 2;
  }
  contact_total<<<1, 1, 0, s>>>(total, S.st_count, S.cap_contacts, out.n_contacts, S.err);
  S.launches += 1;
  trace_end(S, rec_c, s);
  return cudaGetLastError();
}

cudaError_t launch_narrow(int prec, const dem_particles &P, const int32_t *pairs, int64_t max_pairs,
                          const int64_t *n_pairs, const double *t_eval, const dem_narrow_out &out,
                          Scratch &S, int num_sms, cudaStream_t s) {
  PairArgs a = make_args(P, pairs, max_pairs, n_pairs, S, prec, MODE_NARROW);
  a.t_eval = t_eval;
  a.dmin = out.dmin;
  a.pa = out.pa;
  a.pb = out.pb;
  a.tri_ab = out.tri_ab;
  a.flag = out.flag;
  a.dmin32 = out.dmin32;
  a.st_keys = S.st_keys;
  a.st_geom = S.st_geom;
  a.st_count = S.st_count;
  a.st_cap = S.cap_contacts;
  a.pc = S.pc;
  return finish_narrow(prec, a, P, pairs, max_pairs, n_pairs, out, S, num_sms, s, false);
}

cudaError_t launch_detect(int prec, const dem_particles &P, const int32_t *pairs, int64_t max_pairs,
                          const int64_t *n_pairs, const dem_narrow_out &out, int K, double tol, double *t_coll,
                          uint8_t *status, int32_t *tri_ab, Scratch &S, int num_sms, cudaStream_t s) {
  PairArgs a = make_args(P, pairs, max_pairs, n_pairs, S, prec, MODE_BOTH);
  a.dmin = out.dmin;
  a.pa = out.pa;
  a.pb = out.pb;
  a.tri_ab = out.tri_ab;
  a.flag = out.flag;
  a.dmin32 = out.dmin32;
  a.st_keys = S.st_keys;
  a.st_geom = S.st_geom;
  a.st_count = S.st_count;
  a.st_cap = S.cap_contacts;
  a.pc = S.pc;
  a.t_coll = t_coll;
  a.status = status;
  a.ct_ab = tri_ab;
  a.K = K;
  a.tol = tol;
  return finish_narrow(prec, a, P, pairs, max_pairs, n_pairs, out, S, num_sms, s, true);
}

cudaError_t launch_ctime(int prec, int method, const dem_particles &P, const int32_t *pairs, int64_t max_pairs,
                         const int64_t *n_pairs, int K, double tol, double *t_coll, uint8_t *status,
                         int32_t *tri_ab, Scratch &S, int num_sms, cudaStream_t s) {
  PairArgs a = make_args(P, pairs, max_pairs, n_pairs, S, prec,
                         method == DEM_CTIME_NARROWING ? MODE_NTIME : MODE_CTIME);
  a.t_coll = t_coll;
  a.status = status;
  a.ct_ab = tri_ab;
  a.K = K;
  a.tol = tol;
  cudaError_t e;
  if ((e = cudaMemsetAsync(S.work, 0, sizeof(unsigned int), s)) != cudaSuccess) return e;
  if (max_pairs <= 0) return cudaSuccess;
  if ((e = prepare_tiles(P, S, s)) != cudaSuccess) return e;
  if (a.order && (e = prepare_order(P, pairs, max_pairs, n_pairs, S, s)) != cudaSuccess) return e;
  S.launches += 1;
  const int rec = trace_begin(S, TR_PAIRS, s);
  if (method == DEM_CTIME_NARROWING)
    e = prec == 0 ? launch_pairs<0, MODE_NTIME>(a, num_sms, s) : launch_pairs<1, MODE_NTIME>(a, num_sms, s);
  else
    e = prec == 0 ? launch_pairs<0, MODE_CTIME>(a, num_sms, s) : launch_pairs<1, MODE_CTIME>(a, num_sms, s);
  trace_end(S, rec, s);
  return e;
}

}  // namespace dem
