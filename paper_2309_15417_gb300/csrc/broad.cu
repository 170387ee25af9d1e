// broad.cu -- candidate pairs (paper Section 3: free-flight extrapolation of
// each particle over its own step, bounding spheres that cover the particle and
// its halo, a symmetric pairwise overlap test).
//
// Swept sphere of p over [t_cur, t_cur + dt]: centre m = x + v (dt/2), radius
// rho = (radius + eps) + |v| (dt/2).  (i, j), i < j, is a candidate iff
// |m_i - m_j|^2 <= (rho_i + rho_j)^2, evaluated in binary64 with each
// operation rounded on its own; two static particles never pair.
//
// A uniform grid with cell size h >= 2 max rho is hashed into a power-of-two
// table (counting sort of particles into buckets).  Overlapping spheres lie in
// the same or adjacent cells, so scanning the 27 neighbour cells finds every
// candidate; the binary64 predicate then decides, so the set equals the
// brute-force set.  Per particle (one warp, lanes over the 27 cells) the
// candidates are counted, offsets are scanned, and each particle writes its
// partners sorted by j: the output is in (i, j) order without a global sort.
#include "internal.cuh"

namespace dem {

namespace {

using D = OpsD;

__global__ void k_prep(int64_t n, const double *st, Sphere4 *sph, unsigned long long *rho_max) {
  __shared__ double red[8];
  double mx = 0.0;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
    const double hdt = D::mul(st[14 * n + p], 0.5);
    const double vx = st[3 * n + p], vy = st[4 * n + p], vz = st[5 * n + p];
    Sphere4 s;
    s.x = D::add(st[0 * n + p], D::mul(vx, hdt));
    s.y = D::add(st[1 * n + p], D::mul(vy, hdt));
    s.z = D::add(st[2 * n + p], D::mul(vz, hdt));
    const double vv = D::add(D::add(D::mul(vx, vx), D::mul(vy, vy)), D::mul(vz, vz));
    s.w = D::add(D::add(st[16 * n + p], st[15 * n + p]), D::mul(D::sqrt(vv), hdt));
    sph[p] = s;
    mx = fmax(mx, s.w);
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int q = 1; q < (int)(blockDim.x >> 5); ++q) mx = fmax(mx, red[q]);
    atomicMax(rho_max, static_cast<unsigned long long>(__double_as_longlong(mx)));
  }
}

__device__ __forceinline__ double inv_cell(const unsigned long long *rho_max) {
  const double rm = __longlong_as_double(static_cast<long long>(*rho_max));
  const double h = fmax(2.0 * rm * (1.0 + 9.5367431640625e-07), 1e-300);
  return 1.0 / h;
}

__device__ __forceinline__ uint32_t bucket_of(int cx, int cy, int cz, uint32_t mask) {
  const uint32_t h = (uint32_t(cx) * 73856093u) ^ (uint32_t(cy) * 19349663u) ^ (uint32_t(cz) * 83492791u);
  return (h ^ (h >> 16)) & mask;
}

__device__ __forceinline__ int cell_coord(double v, double ih) {
  const double c = floor(v * ih);
  return c > 1e9 ? 1000000000 : (c < -1e9 ? -1000000000 : int(c));
}

__global__ void k_count(int64_t n, const Sphere4 *sph, const unsigned long long *rho_max, uint32_t mask,
                        int4 *cell, int32_t *bcnt) {
  const double ih = inv_cell(rho_max);
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
    const Sphere4 s = sph[p];
    const int cx = cell_coord(s.x, ih), cy = cell_coord(s.y, ih), cz = cell_coord(s.z, ih);
    const uint32_t b = bucket_of(cx, cy, cz, mask);
    cell[p] = make_int4(cx, cy, cz, int(b));
    atomicAdd(&bcnt[b], 1);
  }
}

__global__ void k_scatter(int64_t n, const int4 *cell, const int64_t *bstart, int32_t *bcur, int32_t *ids) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
    const int b = cell[p].w;
    ids[bstart[b] + atomicAdd(&bcur[b], 1)] = int32_t(p);
  }
}

// One warp per particle i: lane c < 27 scans neighbour cell c; counts are
// combined with a warp prefix sum.  WRITE: the partners are written at the
// particle's offset and sorted by j (bitonic in registers for up to 32).
template <bool WRITE>
__global__ void k_pairs(int64_t n, const Sphere4 *sph, const int4 *cell, const uint8_t *is_static,
                        const int32_t *bcnt, const int64_t *bstart, const int32_t *ids, uint32_t mask,
                        int64_t *pcnt, const int64_t *poff, int32_t *pairs, int64_t cap,
                        const int64_t *n_pairs, uint32_t *err) {
  if (WRITE && blockIdx.x == 0 && threadIdx.x == 0 && *n_pairs > cap) set_err(err, ERR_CAPACITY);
  const int lane = threadIdx.x & 31;
  const int64_t nwarp = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = (((int64_t)blockIdx.x * blockDim.x) + threadIdx.x) >> 5; i < n; i += nwarp) {
    const Sphere4 si = sph[i];
    const int4 ci = cell[i];
    const bool sti = is_static && is_static[i];
    const int cx = ci.x + (lane % 3) - 1, cy = ci.y + ((lane / 3) % 3) - 1, cz = ci.z + (lane / 9) - 1;
    int64_t b0 = 0, b1 = 0;
    if (lane < 27) {
      const uint32_t b = bucket_of(cx, cy, cz, mask);
      b0 = bstart[b];
      b1 = b0 + bcnt[b];
    }
    // the binary64 candidate predicate (same operation order as the oracle)
    auto is_pair = [&](int32_t j) {
      if (j <= i) return false;
      const int4 cj = cell[j];
      if (cj.x != cx || cj.y != cy || cj.z != cz) return false;  // other cell, same bucket
      if (sti && is_static[j]) return false;
      const Sphere4 sj = sph[j];
      const double ddx = D::sub(si.x, sj.x), ddy = D::sub(si.y, sj.y), ddz = D::sub(si.z, sj.z);
      const double dd = D::add(D::add(D::mul(ddx, ddx), D::mul(ddy, ddy)), D::mul(ddz, ddz));
      const double rr = D::add(si.w, sj.w);
      return dd <= D::mul(rr, rr);
    };
    int c = 0;
    for (int64_t q = b0; q < b1; ++q) c += is_pair(ids[q]) ? 1 : 0;
    int inc = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += y;
    }
    const int total = __shfl_sync(0xffffffffu, inc, 31);
    if (!WRITE) {
      if (lane == 0) pcnt[i] = total;
      continue;
    }
    const int64_t o = poff[i];
    int64_t pos = o + inc - c;
    for (int64_t q = b0; q < b1; ++q) {
      const int32_t j = ids[q];
      if (is_pair(j)) {
        if (pos < cap) {
          pairs[2 * pos] = int32_t(i);
          pairs[2 * pos + 1] = j;
        }
        ++pos;
      }
    }
    __syncwarp();
    const int64_t e = o + total < cap ? o + total : cap;
    const int m = int(e > o ? e - o : 0);
    if (m <= 32) {
      int32_t key = lane < m ? pairs[2 * (o + lane) + 1] : 0x7fffffff;
      for (int k = 2; k <= 32; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
          const int32_t other = __shfl_xor_sync(0xffffffffu, key, j);
          const bool lower = (lane & j) == 0, up = (lane & k) == 0;
          key = (lower == up) ? min(key, other) : max(key, other);
        }
      if (lane < m) pairs[2 * (o + lane) + 1] = key;
    } else if (lane == 0) {
      for (int64_t a = o + 1; a < e; ++a) {  // long lists (a large particle): insertion sort
        const int32_t v = pairs[2 * a + 1];
        int64_t b = a - 1;
        while (b >= o && pairs[2 * b + 1] > v) {
          pairs[2 * (b + 1) + 1] = pairs[2 * b + 1];
          --b;
        }
        pairs[2 * (b + 1) + 1] = v;
      }
    }
    __syncwarp();
  }
}

}  // namespace

cudaError_t launch_broad(const dem_particles &P, int32_t *pairs, int64_t cap, int64_t *n_pairs, Scratch &S,
                         cudaStream_t s) {
  const int64_t n = P.n;
  cudaError_t e;
  if ((e = cudaMemsetAsync(S.rho_max, 0, sizeof(unsigned long long), s)) != cudaSuccess) return e;
  if (n <= 0) return cudaMemsetAsync(n_pairs, 0, sizeof(int64_t), s);
  const uint32_t mask = uint32_t(S.table_size - 1);
  const int tb = 256;
  const unsigned grid = (unsigned)((n + tb - 1) / tb);
  if ((e = cudaMemsetAsync(S.bucket_cnt, 0, sizeof(int32_t) * S.table_size, s)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(S.bucket_cur, 0, sizeof(int32_t) * S.table_size, s)) != cudaSuccess) return e;
  k_prep<<<grid, tb, 0, s>>>(n, P.state, S.sph, S.rho_max);
  k_count<<<grid, tb, 0, s>>>(n, S.sph, S.rho_max, mask, S.cell, S.bucket_cnt);
  S.launches += 2 + scan_exclusive_i32_to_i64(S.bucket_cnt, S.bucket_start, S.table_size, S.scan_part, s);
  k_scatter<<<grid, tb, 0, s>>>(n, S.cell, S.bucket_start, S.bucket_cur, S.bucket_ids);
  const unsigned wgrid = (unsigned)((n + 7) / 8);  // one warp per particle
  k_pairs<false><<<wgrid, tb, 0, s>>>(n, S.sph, S.cell, P.is_static, S.bucket_cnt, S.bucket_start, S.bucket_ids,
                                      mask, S.pcnt, nullptr, nullptr, 0, nullptr, S.err);
  S.launches += 2 + scan_exclusive_i64(S.pcnt, S.poff, n, n_pairs, S.scan_part, s);
  k_pairs<true><<<wgrid, tb, 0, s>>>(n, S.sph, S.cell, P.is_static, S.bucket_cnt, S.bucket_start, S.bucket_ids,
                                     mask, nullptr, S.poff, pairs, cap, n_pairs, S.err);
  S.launches += 1;
  return cudaGetLastError();
}

}  // namespace dem
