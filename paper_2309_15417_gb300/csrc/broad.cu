// broad.cu -- candidate pairs (paper Section 3: free-flight extrapolation of
// each particle over its own step, bounding volumes that cover the particle
// and its halo, a symmetric pairwise overlap test; static geometry apart).
//
// Swept sphere of a moving p over [t_cur, t_cur + dt]: centre m = x + v (dt/2),
// radius rho = (radius + eps) + |v| (dt/2).  Two moving particles (i, j),
// i < j, are a candidate iff |m_i - m_j|^2 <= (rho_i + rho_j)^2.  A static
// particle s is the axis-aligned box of its world vertices at t_cur widened
// by eps_s; (p, s) is a candidate iff p's swept sphere meets the box, and the
// static member is written second.  Every predicate is evaluated in binary64
// with each operation rounded on its own; two static particles never pair.
//
// Moving particles go into a uniform grid with cell size h >= 2 max rho,
// hashed into a power-of-two table (counting sort of particles into buckets).
// Overlapping spheres lie in the same or adjacent cells, so scanning the 27
// neighbour cells finds every moving partner; every static box is tested
// directly (static objects are few: floors, walls).  Per particle (one warp,
// lanes over the 27 cells and then over the static boxes) the candidates are
// counted, offsets are scanned, and each particle writes its partners sorted:
// the output is in (first, second) order without a global sort.
#include "internal.cuh"

namespace dem {

namespace {

using D = OpsD;

// swept spheres of all particles; max rho over moving particles; static
// particles listed with their pose at t_cur and an empty box.  A particle
// with a non-finite state field sets ERR_NONFINITE and gets a NaN sphere and
// no static entry: it takes part in no pair.
__global__ void k_prep(int64_t n, const double *st, const uint8_t *is_static, Sphere4 *sph,
                       unsigned long long *rho_max, int32_t *static_ids, int32_t *n_static, double *spose,
                       unsigned long long *sbox, uint32_t *err) {
  __shared__ double red[8];
  __shared__ double rc[POSE_TERMS + 1], rs[POSE_TERMS + 1];
  if (threadIdx.x == 0) pose_reciprocals(rc, rs);
  __syncthreads();
  double mx = 0.0;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
    bool fin = true;
#pragma unroll
    for (int f = 0; f < DEM_NFIELDS; ++f) fin = fin && isfinite(st[f * n + p]);
    if (!fin) {
      set_err(err, ERR_NONFINITE);
      const double nan = __longlong_as_double(0x7ff8000000000000LL);
      sph[p] = Sphere4{nan, nan, nan, nan};
      continue;
    }
    const double hdt = D::mul(st[14 * n + p], 0.5);
    const double vx = st[3 * n + p], vy = st[4 * n + p], vz = st[5 * n + p];
    Sphere4 s;
    s.x = D::add(st[0 * n + p], D::mul(vx, hdt));
    s.y = D::add(st[1 * n + p], D::mul(vy, hdt));
    s.z = D::add(st[2 * n + p], D::mul(vz, hdt));
    const double vv = D::add(D::add(D::mul(vx, vx), D::mul(vy, vy)), D::mul(vz, vz));
    s.w = D::add(D::add(st[16 * n + p], st[15 * n + p]), D::mul(D::sqrt(vv), hdt));
    sph[p] = s;
    if (is_static && is_static[p]) {
      const int32_t q = atomicAdd(n_static, 1);
      static_ids[q] = int32_t(p);
      double R[9], X[3];
      pose_exact(st, n, p, st[13 * n + p], rc, rs, R, X);
      for (int k = 0; k < 9; ++k) spose[12 * (int64_t)q + k] = R[k];
      for (int k = 0; k < 3; ++k) spose[12 * (int64_t)q + 9 + k] = X[k];
      for (int k = 0; k < 3; ++k) {  // empty box: min = +inf, max = -inf
        sbox[6 * (int64_t)q + k] = okey(OpsD::inf());
        sbox[6 * (int64_t)q + 3 + k] = okey(-OpsD::inf());
      }
    } else {
      mx = fmax(mx, s.w);
    }
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

// world-vertex extremes of every static particle at t_cur (binary64, the
// same vertex transform as the exact narrow phase); min and max are exact,
// so the order of the reduction does not matter
__global__ void k_static_box(int64_t n, const int64_t *tri_off, const float4 *tris, int64_t n_tris,
                             const int32_t *static_ids, const int32_t *n_static, const double *spose,
                             unsigned long long *sbox, uint32_t *err) {
  const int ns = *n_static;
  const int64_t gid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x, gstride = (int64_t)gridDim.x * blockDim.x;
  for (int q = 0; q < ns; ++q) {
    const int64_t p = static_ids[q];
    const int64_t o = tri_off[p], cnt = tri_off[p + 1] - o;
    if (cnt < 0 || o < 0 || o + cnt > n_tris) {
      if (gid == 0) set_err(err, ERR_INDEX);
      continue;
    }
    const double *R = spose + 12 * (int64_t)q, *X = R + 9;
    double lo[3] = {OpsD::inf(), OpsD::inf(), OpsD::inf()}, hi[3] = {-OpsD::inf(), -OpsD::inf(), -OpsD::inf()};
    for (int64_t k = gid; k < cnt; k += gstride)
#pragma unroll
      for (int v = 0; v < 3; ++v) {
        const float4 f = tris[v * n_tris + o + k];
        const V3<double> w = to_world_exact(R, X, f.x, f.y, f.z);
        lo[0] = fmin(lo[0], w.x);
        lo[1] = fmin(lo[1], w.y);
        lo[2] = fmin(lo[2], w.z);
        hi[0] = fmax(hi[0], w.x);
        hi[1] = fmax(hi[1], w.y);
        hi[2] = fmax(hi[2], w.z);
      }
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
      for (int sh = 16; sh; sh >>= 1) {
        lo[k] = fmin(lo[k], __shfl_xor_sync(0xffffffffu, lo[k], sh));
        hi[k] = fmax(hi[k], __shfl_xor_sync(0xffffffffu, hi[k], sh));
      }
    if ((threadIdx.x & 31) == 0 && lo[0] <= hi[0]) {
      for (int k = 0; k < 3; ++k) {
        atomicMin(&sbox[6 * (int64_t)q + k], okey(lo[k]));
        atomicMax(&sbox[6 * (int64_t)q + 3 + k], okey(hi[k]));
      }
    }
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

__global__ void k_count(int64_t n, const Sphere4 *sph, const uint8_t *is_static,
                        const unsigned long long *rho_max, uint32_t mask, int4 *cell, int32_t *bcnt) {
  const double ih = inv_cell(rho_max);
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
    const Sphere4 s = sph[p];
    if ((is_static && is_static[p]) || !(s.w >= 0.0)) {  // static and non-finite particles are not binned
      cell[p] = make_int4(0, 0, 0, -1);
      continue;
    }
    const int cx = cell_coord(s.x, ih), cy = cell_coord(s.y, ih), cz = cell_coord(s.z, ih);
    const uint32_t b = bucket_of(cx, cy, cz, mask);
    cell[p] = make_int4(cx, cy, cz, int(b));
    atomicAdd(&bcnt[b], 1);
  }
}

// moving particles into bucket order, with copies of their sphere and cell
// (the pair test then reads a partner's data without first reading its index)
__global__ void k_scatter(int64_t n, const int4 *cell, const Sphere4 *sph, const int64_t *bstart, int32_t *bcur,
                          int32_t *ids, Sphere4 *bsph, float4 *bsph32, int4 *bcell) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
    const int4 c = cell[p];
    if (c.w < 0) continue;
    const int64_t q = bstart[c.w] + atomicAdd(&bcur[c.w], 1);
    const Sphere4 s = sph[p];
    ids[q] = int32_t(p);
    bsph[q] = s;
    bsph32[q] = make_float4(float(s.x), float(s.y), float(s.z), float(s.w));
    bcell[q] = c;
  }
}

// The widened box of every static particle, once: lo = min - eps_s and
// hi = max + eps_s in binary64 (the oracle's operations), stored as bits in
// place of the order keys, and rounded outwards to FP32 for the screening.
__global__ void k_static_fin(int64_t n, const double *st, const int32_t *static_ids, const int32_t *n_static,
                             unsigned long long *sbox, float *sbox32) {
  const int ns = *n_static;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < ns; q += gridDim.x * blockDim.x) {
    const double e = st[15 * n + static_ids[q]];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const double lo = D::sub(okey_value(sbox[6 * (int64_t)q + k]), e);
      const double hi = D::add(okey_value(sbox[6 * (int64_t)q + 3 + k]), e);
      sbox[6 * (int64_t)q + k] = static_cast<unsigned long long>(__double_as_longlong(lo));
      sbox[6 * (int64_t)q + 3 + k] = static_cast<unsigned long long>(__double_as_longlong(hi));
      sbox32[6 * (int64_t)q + k] = __double2float_rd(lo);
      sbox32[6 * (int64_t)q + 3 + k] = __double2float_ru(hi);
    }
  }
}

// The sphere predicate dd <= rr^2 (binary64, oracle order) decided in FP32
// where that is certain.  From FP32 copies (each coordinate and radius
// rounded once, u = 2^-24) the computed dd^ and rr^2^ satisfy, with M the
// largest coordinate magnitude of the two centres,
//   |dd^ - dd|     <= 11 M u (sqrt(dd^) + 3 M u) + 27 M^2 u^2 + 4 u dd^,
//   |rr^2^ - rr^2| <= 8 u rr^2^,
// and the binary64 values differ from the exact ones by far less (1e-14
// relative covers them); B is twice the sum.  Returns 1 (pair), 0 (no pair)
// or -1 (within B: the binary64 predicate decides).
__device__ __forceinline__ int sphere_test32(float4 a, float4 b) {
  const float dx = a.x - b.x, dy = a.y - b.y, dz = a.z - b.z;
  const float dd = dx * dx + dy * dy + dz * dz;
  const float rr = a.w + b.w, r2 = rr * rr;
  const float M = fmaxf(fmaxf(fmaxf(fabsf(a.x), fabsf(b.x)), fmaxf(fabsf(a.y), fabsf(b.y))),
                        fmaxf(fabsf(a.z), fabsf(b.z)));
  const float u = 5.9604644775390625e-08f;  // 2^-24
  const float Mu = M * u;
  const float B = 2.0f * (11.0f * Mu * (sqrtf(dd) + 3.0f * Mu) + 27.0f * Mu * Mu + 4.0f * u * dd + 8.0f * u * r2 +
                          1e-14f * (dd + r2));
  if (dd + B < r2) return 1;
  if (dd - B > r2) return 0;
  return -1;
}

// Space-time hose test (Check 2 of the paper's broad phase) of moving
// particles i, j over their pair interval: bounding spheres (R + eps) on the
// straight segment from the old snapshot to the current one, then with the
// current velocity; true iff they overlap at some common time.  On each
// piece between the knots the squared distance of the relative linear motion
// d0 + u s is smallest at s = -(d0 . u) / (u . u), clamped to the piece.
__device__ __forceinline__ V3<double> hose_at(const double *cur, const double *old, int64_t n, int64_t p, double t,
                                              bool on_old, V3<double> &v) {
  const double *s = on_old ? old : cur;
  v = V3<double>{s[3 * n + p], s[4 * n + p], s[5 * n + p]};
  const double h = D::sub(t, s[13 * n + p]);
  return V3<double>{D::add(s[0 * n + p], D::mul(v.x, h)), D::add(s[1 * n + p], D::mul(v.y, h)),
                    D::add(s[2 * n + p], D::mul(v.z, h))};
}

__device__ __noinline__ bool hose_meet(const double *cur, const double *old, int64_t n, int64_t i, int64_t j) {
  using G = Geo<OpsD>;
  const double ti = cur[13 * n + i], tj = cur[13 * n + j];
  const double ts = ti < tj ? ti : tj, t2 = ti < tj ? tj : ti;
  const double di = cur[14 * n + i], dj = cur[14 * n + j];
  const double te = D::add(ts, di < dj ? di : dj);
  const double r = D::add(D::add(cur[16 * n + i], cur[15 * n + i]), D::add(cur[16 * n + j], cur[15 * n + j]));
  double kk[3];
  int nk = 0;
  kk[nk++] = ts;
  if (t2 > ts && t2 < te) kk[nk++] = t2;
  kk[nk++] = te;
  for (int q = 0; q + 1 < nk; ++q) {
    const double a = kk[q], b = kk[q + 1];
    V3<double> vi, vj;
    const V3<double> xi = hose_at(cur, old, n, i, a, b <= ti, vi);
    const V3<double> xj = hose_at(cur, old, n, j, a, b <= tj, vj);
    const V3<double> d0 = G::sub(xi, xj), u = G::sub(vi, vj);
    const double uu = G::dot(u, u), du = G::dot(d0, u);
    double s = 0.0;
    if (uu > 0.0) {
      s = D::div(-du, uu);
      if (s < 0.0) s = 0.0;
      const double ba = D::sub(b, a);
      if (s > ba) s = ba;
    }
    const V3<double> dm = G::axpy(d0, u, s);
    if (G::dot(dm, dm) <= D::mul(r, r)) return true;
  }
  return false;
}

// One warp per moving particle i, taken in bucket order (spatially coherent:
// consecutive warps share neighbour buckets in cache): lane c < 27 scans
// neighbour cell c, then the lanes share the static boxes; counts are
// combined with warp prefix sums.  WRITE: the partners are written at the
// particle's offset and sorted by partner index (bitonic in registers for up
// to 32).  With a partner cache (pc, pc_ok), the count pass also keeps a
// particle's partners when at most PCACHE of them, at most two grid partners
// per lane and one static partner per lane, were found; the write pass then
// copies them instead of scanning the cells again.
__device__ __forceinline__ int warp_incl_sum(int v, int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += y;
  }
  return v;
}

template <bool WRITE>
__global__ void __launch_bounds__(256, 6) k_pairs(int64_t n, const double *st, const Sphere4 *bsph,
                                                  const float4 *bsph32, const int4 *bcell, const float *sbox32,
                        const int32_t *bcnt, const int64_t *bstart, const int32_t *ids,
                        uint32_t mask, const int32_t *static_ids, const int32_t *n_static,
                        const unsigned long long *sbox, const double *hose_old, int64_t *pcnt,
                        const int64_t *poff, int32_t *pairs, int64_t cap, const int64_t *n_pairs,
                        int32_t *pc, uint8_t *pc_ok, uint32_t *err) {
  if (WRITE && blockIdx.x == 0 && threadIdx.x == 0 && *n_pairs > cap) set_err(err, ERR_CAPACITY);
  const int lane = threadIdx.x & 31;
  const int64_t nwarp = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int ns = *n_static;
  const int64_t nm = n - ns;  // moving particles, all in bucket order
  for (int64_t r = (((int64_t)blockIdx.x * blockDim.x) + threadIdx.x) >> 5; r < nm; r += nwarp) {
    const int64_t i = ids[r];
    if (WRITE && pc_ok && pc_ok[i]) {
      // the count pass kept every partner: copy and sort them
      const int64_t o = poff[i];
      const int tot = int(pcnt[i]);
      int32_t key = lane < tot ? pc[(int64_t)PCACHE * i + lane] : 0x7fffffff;
      for (int k = 2; k <= 32; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
          const int32_t other = __shfl_xor_sync(0xffffffffu, key, j);
          const bool lower = (lane & j) == 0, up = (lane & k) == 0;
          key = (lower == up) ? min(key, other) : max(key, other);
        }
      if (lane < tot && o + lane < cap) {
        pairs[2 * (o + lane)] = int32_t(i);
        pairs[2 * (o + lane) + 1] = key;
      }
      continue;
    }
    const Sphere4 si = bsph[r];
    const float4 si32 = bsph32[r];
    const int4 ci = bcell[r];
    const int cx = ci.x + (lane % 3) - 1, cy = ci.y + ((lane / 3) % 3) - 1, cz = ci.z + (lane / 9) - 1;
    int64_t b0 = 0, b1 = 0;
    if (lane < 27) {
      const uint32_t b = bucket_of(cx, cy, cz, mask);
      b0 = bstart[b];
      b1 = b0 + bcnt[b];
    }
    // moving partner j > i at bucket position q (the binary64 sphere
    // predicate, oracle order)
    auto is_pair = [&](int64_t q, int32_t j) {
      if (j <= i) return false;
      // both loads issued together (q is in bounds either way)
      const int4 cj = bcell[q];
      const float4 sj32 = bsph32[q];
      if (cj.x != cx || cj.y != cy || cj.z != cz) return false;  // other cell, same bucket
      const int t32 = sphere_test32(si32, sj32);
      if (t32 == 0) return false;
      if (t32 < 0) {
        const Sphere4 sj = bsph[q];
        const double ddx = D::sub(si.x, sj.x), ddy = D::sub(si.y, sj.y), ddz = D::sub(si.z, sj.z);
        const double dd = D::add(D::add(D::mul(ddx, ddx), D::mul(ddy, ddy)), D::mul(ddz, ddz));
        const double rr = D::add(si.w, sj.w);
        if (!(dd <= D::mul(rr, rr))) return false;
      }
      return hose_old == nullptr || hose_meet(st, hose_old, n, i, j);
    };
    // static partner number q: the swept sphere meets the widened box.
    // FP32 screen first: the box rounded outwards contains the binary64 box,
    // and the FP32 rounding of the centre and of the few operations stays
    // below 1e-6 (M + rho) (M the largest magnitude involved), far inside
    // the margin 1e-4 (M + rho); a sphere that clears the FP32 box by more
    // than the margin clears the binary64 box.
    auto meets_box = [&](int q) {
      {
        const float *b32 = sbox32 + 6 * (int64_t)q;
        const float c[3] = {si32.x, si32.y, si32.z};
        float gg = 0.f, M = 0.f;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          const float lo = b32[k], hi = b32[3 + k];
          const float gk = c[k] < lo ? lo - c[k] : (c[k] > hi ? c[k] - hi : 0.f);
          gg += gk * gk;
          M = fmaxf(M, fmaxf(fabsf(c[k]), fmaxf(fabsf(lo), fabsf(hi))));
        }
        if (sqrtf(gg) > si32.w + 1e-4f * (M + si32.w)) return false;
      }
      const double m[3] = {si.x, si.y, si.z};
      double g[3];
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const double lo = __longlong_as_double(static_cast<long long>(sbox[6 * (int64_t)q + k]));
        const double hi = __longlong_as_double(static_cast<long long>(sbox[6 * (int64_t)q + 3 + k]));
        g[k] = m[k] < lo ? D::sub(lo, m[k]) : (m[k] > hi ? D::sub(m[k], hi) : 0.0);
      }
      const double gg = D::add(D::add(D::mul(g[0], g[0]), D::mul(g[1], g[1])), D::mul(g[2], g[2]));
      return gg <= D::mul(si.w, si.w);
    };
    int c = 0, cs = 0;
    int32_t g0 = -1, g1 = -1, s0 = -1;  // the count pass's first partners of this lane
    for (int64_t q = b0; q < b1; ++q) {
      const int32_t j = ids[q];
      if (is_pair(q, j)) {
        if (c == 0) g0 = j;
        if (c == 1) g1 = j;
        ++c;
      }
    }
    for (int q = lane; q < ns; q += 32)
      if (meets_box(q)) {
        if (cs == 0) s0 = static_ids[q];
        ++cs;
      }
    const int inc = warp_incl_sum(c, lane), incs = warp_incl_sum(cs, lane);
    const int tgrid = __shfl_sync(0xffffffffu, inc, 31);
    const int total = tgrid + __shfl_sync(0xffffffffu, incs, 31);
    if (!WRITE) {
      if (lane == 0) pcnt[i] = total;
      if (pc) {
        // every lane votes; the cache holds the list only if it is complete
        const bool fits = __all_sync(0xffffffffu, c <= 2 && cs <= 1) && total <= PCACHE;
        if (fits) {
          int32_t *row = pc + (int64_t)PCACHE * i;
          if (c > 0) row[inc - c] = g0;
          if (c > 1) row[inc - c + 1] = g1;
          if (cs > 0) row[tgrid + incs - cs] = s0;
        }
        if (lane == 0) pc_ok[i] = fits ? 1 : 0;
      }
      continue;
    }
    const int64_t o = poff[i];
    auto put = [&](int64_t pos, int32_t j) {
      if (pos < cap) {
        pairs[2 * pos] = int32_t(i);
        pairs[2 * pos + 1] = j;
      }
    };
    int64_t pos = o + inc - c;
    for (int64_t q = b0; q < b1; ++q) {
      const int32_t j = ids[q];
      if (is_pair(q, j)) put(pos++, j);
    }
    pos = o + tgrid + incs - cs;
    for (int q = lane; q < ns; q += 32)
      if (meets_box(q)) put(pos++, static_ids[q]);
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
                         cudaStream_t s, const double *hose_old) {
  const int64_t n = P.n;
  cudaError_t e;
  if ((e = cudaMemsetAsync(S.rho_max, 0, sizeof(unsigned long long), s)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(S.n_static, 0, sizeof(int32_t), s)) != cudaSuccess) return e;
  if (n <= 0) return cudaMemsetAsync(n_pairs, 0, sizeof(int64_t), s);
  const uint32_t mask = uint32_t(S.table_size - 1);
  const int tb = 256;
  const unsigned grid = (unsigned)((n + tb - 1) / tb);
  const int rec = trace_begin(S, TR_BROAD, s);
  if ((e = cudaMemsetAsync(S.bucket_cnt, 0, sizeof(int32_t) * S.table_size, s)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(S.bucket_cur, 0, sizeof(int32_t) * S.table_size, s)) != cudaSuccess) return e;
  k_prep<<<grid, tb, 0, s>>>(n, P.state, P.is_static, S.sph, S.rho_max, S.static_ids, S.n_static, S.spose, S.sbox,
                             S.err);
  S.launches += 1;
  if (P.is_static) {
    k_static_box<<<304, tb, 0, s>>>(n, P.tri_off, reinterpret_cast<const float4 *>(P.tris), P.n_tris,
                                     S.static_ids, S.n_static, S.spose, S.sbox, S.err);
    k_static_fin<<<grid, tb, 0, s>>>(n, P.state, S.static_ids, S.n_static, S.sbox, S.sbox32);
    S.launches += 2;
  }
  k_count<<<grid, tb, 0, s>>>(n, S.sph, P.is_static, S.rho_max, mask, S.cell, S.bucket_cnt);
  S.launches += 1 + scan_exclusive_i32_to_i64(S.bucket_cnt, S.bucket_start, S.table_size, S.scan_part, s);
  k_scatter<<<grid, tb, 0, s>>>(n, S.cell, S.sph, S.bucket_start, S.bucket_cur, S.bucket_ids, S.bucket_sph,
                                S.bucket_sph32, S.bucket_cell);
  // static particles never start a pair: their counts stay 0
  if ((e = cudaMemsetAsync(S.pcnt, 0, sizeof(int64_t) * n, s)) != cudaSuccess) return e;
  const unsigned wgrid = (unsigned)((n + 7) / 8);  // one warp per particle
  k_pairs<false><<<wgrid, tb, 0, s>>>(n, P.state, S.bucket_sph, S.bucket_sph32, S.bucket_cell, S.sbox32,
                                      S.bucket_cnt, S.bucket_start,
                                      S.bucket_ids, mask, S.static_ids, S.n_static, S.sbox, hose_old, S.pcnt,
                                      nullptr, nullptr, 0, nullptr, S.pcache, S.pcache_ok, S.err);
  S.launches += 2 + scan_exclusive_i64(S.pcnt, S.poff, n, n_pairs, S.scan_part, s);
  k_pairs<true><<<wgrid, tb, 0, s>>>(n, P.state, S.bucket_sph, S.bucket_sph32, S.bucket_cell, S.sbox32,
                                     S.bucket_cnt, S.bucket_start,
                                     S.bucket_ids, mask, S.static_ids, S.n_static, S.sbox, hose_old, S.pcnt,
                                     S.poff, pairs, cap, n_pairs, S.pcache, S.pcache_ok, S.err);
  S.launches += 1;
  trace_end(S, rec, s);
  return cudaGetLastError();
}

}  // namespace dem
