#pragma once
// pair_kernel.cuh -- the pair kernel: narrow phase and collision-time search
// over candidate pairs (one persistent CTA per pair at a time).
//
// Paper Section 5 ("Time step size calculation"): for a candidate pair the
// minimum triangle-pair distance is evaluated at given times; a contact is a
// triangle pair within eps_i + eps_j (Definition of a contact point); the
// collision time stamp is the first time the halos meet in the pair's
// interval (case distinction; narrowing by K samples and bisection; the upper
// bracket end as "widening").
//
// GPU design (one persistent CTA works on one pair at a time, pairs taken from
// an atomic counter):
//  * Triangle tiles of both particles are staged in shared memory by bulk
//    copies (cp.async.bulk + mbarrier).  In FP32 mode particle A stays in its
//    body frame (its float32 vertices are exact) and B is moved into A's frame
//    with the relative pose, computed in FP64 and rounded once per time.
//  * Culling: bounding spheres of groups of 32 consecutive triangles, then of
//    triangles; only triangle pairs whose spheres come within the threshold
//    reach the full distance.  The culling is conservative by construction
//    (margins below), so it never changes a result.
//  * Each warp owns a candidate list and evaluates it itself (no block-wide
//    barrier in the inner loop).
//  * FP32 mode decides nothing from an FP32 distance.  For each triangle pair
//    the FP32 pass yields closest points pa, pb and a certificate: the
//    separation of the two triangles along n = pb - pa, less E = ERR_REL32 * S
//    (S = R_A + R_B + |t|, the coordinate scale of the frame; a tile-local
//    frame uses its own, smaller S).  Whatever pa and pb are, the certificate
//    is below the binary64 distance by more than m64 = ERR_REL64_LB *
//    (S + |X_A| + |X_B|) (the derivation is beside the constants).  "Apart"
//    is certified (L > eps + m64); "in contact" comes only from binary64
//    feature values computed exactly as the binary64 distance computes them;
//    the closest pair is the binary64 minimum over every triangle pair whose
//    certificate does not exceed a binary64 reference distance.  Decisions,
//    closest pairs and collision times are therefore the binary64 ones.
//  * FP64 mode computes every distance in binary64 in the world frame.
#include <cstdio>

#include "internal.cuh"

namespace dem {
namespace pk {


constexpr int G = 32;        // triangles per group
constexpr int H = 8;         // triangles per subgroup
constexpr int WCAP = 96;     // per-warp candidate list capacity
constexpr int XQCAP = 64;    // per-warp binary64 queue capacity
constexpr int ACAP = 512;    // closest-pair candidates per evaluation
constexpr int WFLUSH = 64;   // default: a warp evaluates its candidate list at this size (<= WCAP - 32)
constexpr int QWARP = 12;    // binary64 queues up to this size run one triangle pair per warp
constexpr int GRID_MAX = 16; // sample times whose poses are computed up front
constexpr int ILCAP = 512;   // triangle pairs of the pair-interval candidate list in shared memory
                             // (more spill to the CTA's region of the global list, PairArgs::ilg)
// Margin E of an FP32 certificate, relative to the frame's coordinate scale M
// (|every coordinate| <= M; M <= S).  Forward error, u = 2^-24, fmaf rounding
// once, rsqrtf within 2 ulp:
//  * B's vertex in A's frame, Rr b + t with Rr, t formed in FP32 from the
//    rounded binary64 poses (entries within 5u, t within 5u |t|) and the fmaf
//    chain (3 roundings): moved by at most 24u M from its exact image;
//    A's vertices are its exact float32 body coordinates;
//  * each dot product n.x (two fmaf, one product): within 3u |n| M, so the
//    gap min n.y - max n.x within 6u |n| M, its rounding 2u |n| M;
//  * the scale gap * rsqrtf(n.n): relative 1.5u (n.n) + 4u (rsqrtf) + u, on a
//    value of at most 2M: 13u M.
// Total 45u M < 128u M = 2^-17 M, a factor 2.8 to spare.
constexpr double ERR_REL32 = 7.62939453125e-06;  // 2^-17
// Binary64 margin relative to S + |X_A| + |X_B|: the oracle's world vertices
// round relative to the particles' positions, its distance relative to S, and
// the rotation matrices deviate from orthogonal by a few units of 2^-53;
// 2^-40 leaves 2^13 such units.  Also the FP64 mode's culling margin.
constexpr double ERR_REL64_LB = 9.094947017729282e-13;  // 2^-40

constexpr int MODE_NARROW = 0;
constexpr int MODE_CTIME = 1;
constexpr int MODE_BOTH = 2;  // narrow phase at the pair start + collision times
constexpr int MODE_NTIME = 3; // collision times by the paper's narrowing
constexpr int NARROW_MAX_ITER = 64;

constexpr int pow2_at_least(int v) { return v <= 1 ? 1 : 2 * pow2_at_least((v + 1) / 2); }

template <int PREC>
struct Cfg;
// FP32: 4 warps per CTA, 4 CTAs per SM (about 52 KB of shared memory each);
// FP64: 8 warps per CTA, 2 CTAs per SM.  A tile holds 320 triangles.
template <>
struct Cfg<0> {
  static constexpr int TT = 320;
  static constexpr int NT = 128;
  static constexpr int MINB = 4;
  using T = float;
  using O = OpsF;
};
template <>
struct Cfg<1> {
  static constexpr int TT = 320;
  static constexpr int NT = 256;
  static constexpr int MINB = 2;
  using T = double;
  using O = OpsD;
};
static_assert(Cfg<0>::TT == TILE_TRIS && Cfg<1>::TT == TILE_TRIS, "tile spheres assume one tile size");

struct PairArgs {
  int64_t n;
  const double *st;
  const uint8_t *is_static;
  const int64_t *tri_off;
  const float4 *tris;
  int64_t n_tris;
  const int32_t *pairs;
  int64_t max_pairs;
  const int64_t *n_pairs;
  // narrow phase
  const double *t_eval;
  double *dmin, *pa, *pb;
  int32_t *tri_ab;
  uint8_t *flag;
  float *dmin32;
  int32_t *st_keys;
  double *st_geom;
  unsigned long long *st_count;
  int64_t st_cap;
  int64_t *pc;
  // collision times
  double *t_coll;
  uint8_t *status;
  int32_t *ct_ab;
  int K;
  double tol;
  // bounding spheres of the tiles of particles with more than one tile
  const float4 *tile_sph;
  const float4 *tile_box;
  int64_t cap_tiles;
  // bookkeeping
  unsigned int *work;
  uint32_t *err;
  unsigned long long *stats;
  uint32_t wait_polls;  // polls of the first wait on a tile copy
  // spill of the pair-interval list beyond ILCAP entries: ilg_cap entries per
  // CTA at ilg + blockIdx.x * ilg_cap (NULL / 0: none)
  unsigned long long *ilg;
  int64_t ilg_cap;
  // launch configuration (autotuned per context): hand-out order of the pairs
  // (NULL: index order), warp candidate-list flush size, CTAs per SM
  const int32_t *order;
  int wflush;
  int ctas_per_sm;
};

template <int PREC>
struct __align__(128) Smem {
  using T = typename Cfg<PREC>::T;
  static constexpr int TT = Cfg<PREC>::TT;
  static constexpr int NT = Cfg<PREC>::NT;
  static constexpr int NW = NT / 32;
  static constexpr int NG = TT / G;   // groups of 32 triangles
  static constexpr int NH = TT / H;   // subgroups of 8 triangles
  static constexpr int GPCAP = pow2_at_least(NG * NG);  // the sort pads to a power of two
  float4 Ab[3][TT];                   // A tile, body frame (bulk copy target)
  T Ae[PREC ? 9 : 1][PREC ? TT : 1];  // A tile, evaluation frame (FP64 only)
  T Be[9][TT];                        // B tile, evaluation frame [slot*3+coord][tri]
  T SA[4][TT];                        // triangle spheres of A (cx, cy, cz, r)
  T SB[4][TT];
  T GA[4][NG];                        // group spheres
  T GB[4][NG];
  T HA[4][NH];                        // subgroup spheres
  T HB[4][NH];
  uint32_t gp[GPCAP];                 // group pairs passing the group test
  float gplb[GPCAP];                  // their lower bounds (rounded down)
  uint32_t wl[NW][WCAP];              // per-warp candidate lists (a << 16 | b)
  uint32_t xq[NW][XQCAP];             // per-warp binary64 queue (why << 28 | a << 14 | b)
  unsigned long long ac_key[ACAP];    // closest-pair candidates (global a << 32 | b)
  float ac_d[ACAP];                   // their FP32 distances
  double rc[POSE_TERMS + 1], rs[POSE_TERMS + 1];
  double RA[9], XA[3], RB[9], XB[3];
  float Rr[9], tr[3];
  double eps, ts, T_, Ed, Elb;
  double m64;                         // binary64 underestimate margin (FP32 mode: 2^-40 S)
  double Et;                          // FP32 margin E of the B tile in frames (its local scale)
  float oo[3], to[3];                 // that tile's local origin (B body frame) and its position in A's frame
  double Eam;                         // closest-pair collection slack (2 E; widened by a re-run)
  double cull;                        // threshold the last closest-pair search culled with
  unsigned long long ref_key;         // closest-pair reference candidate
  int redo;                           // the closest-pair search must re-run with a wider slack
  int64_t i, j, offA, offB;
  int nA, nB, ngp, gpnext, found, resA, resB, frmA, frmB, bad, abort, nac, ngrid;
  int wcnt[NW];
  // pair-interval candidates: (dq << 48) | (a << 24) | b, a and b within the
  // particles (< 2^24), dq the top 16 bits of a float not above the pair's
  // binary64 distance at the pair start (a lower bound, for the narrowing)
  unsigned long long il[ILCAP];
  int nil, ilover, ilcol;
  uint32_t tmask[NW];                 // near tile pairs of a chunk, one ballot per warp
  double ilthr;                       // threshold of the list: FP32, on certificates, eps + delta + m64; FP64 th0
  double delta;                       // bound on the change of any distance over the interval
  double gR[GRID_MAX][2][9], gX[GRID_MAX][2][3];  // poses at the sample times
  unsigned long long bound;           // bits of a non-negative double
  unsigned long long mbar;
  double red_d[NW];
  unsigned long long red_k[NW];
  double mhat;
  double best_d2;
  unsigned long long best_key;
  double best_pa[3], best_pb[3];
  unsigned int work_item;
  int tfirst;                         // nearest tile pair (argmin pass)
  unsigned long long cnt[ST_N];
};

// ---------------------------------------------------------------- PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}
__device__ __forceinline__ void mbar_init(unsigned long long *bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)));
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes,
                                         unsigned long long *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long *bar, uint32_t phase) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(phase)
      : "memory");
  return ok != 0;
}
// bounded wait on the barrier phase (at most `polls` polls); false if it ran out
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, uint32_t phase,
                                          uint32_t polls = WAIT_POLLS_DEFAULT) {
  for (uint32_t it = 0; it < polls; ++it)
    if (mbar_try_wait(bar, phase)) return true;
  return false;
}

__device__ __forceinline__ float warp_min(float v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ double warp_min(double v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
// min / max over aligned segments of `width` lanes
template <class T>
__device__ __forceinline__ T seg_min(T v, int width) {
  for (int o = width >> 1; o; o >>= 1) {
    const T u = __shfl_xor_sync(0xffffffffu, v, o);
    v = u < v ? u : v;
  }
  return v;
}
template <class T>
__device__ __forceinline__ T seg_max(T v, int width) {
  for (int o = width >> 1; o; o >>= 1) {
    const T u = __shfl_xor_sync(0xffffffffu, v, o);
    v = u > v ? u : v;
  }
  return v;
}

__device__ __forceinline__ unsigned long long dbits(double x) {
  return static_cast<unsigned long long>(__double_as_longlong(x));
}
__device__ __forceinline__ double bitsd(unsigned long long b) {
  return __longlong_as_double(static_cast<long long>(b));
}
// float not above x
__device__ __forceinline__ float down_f(float x) { return x; }
__device__ __forceinline__ float down_f(double x) { return __double2float_rd(x); }

constexpr uint32_t WHY_DEC = 1u, WHY_CON = 2u, WHY_ARG = 4u;

// ---------------------------------------------------------------- the CTA
template <int PREC>
struct Cta {
  using T = typename Cfg<PREC>::T;
  using O = typename Cfg<PREC>::O;
  using GT = Geo<O>;
  using GD = Geo<OpsD>;
  using V = V3<T>;
  static constexpr int TT = Cfg<PREC>::TT;
  static constexpr int NT = Cfg<PREC>::NT;
  static constexpr int NW = NT / 32;
  static constexpr int NG = TT / G;
  static constexpr int NH = TT / H;

  Smem<PREC> &s;
  const PairArgs &A;
  int tid, w, lane;
  uint32_t phase;
  // per-evaluation warp state
  T mw;                        // warp minimum of the evaluated distances
  double bd2;                  // lane best exact (d^2, key) and its points
  unsigned long long bkey;
  double bpa[3], bpb[3];
  double wbd2;                 // warp best (uniform), for pruning candidates
  unsigned long long wbkey;
  int qn;                      // entries in this warp's binary64 queue

  __device__ Cta(Smem<PREC> &s_, const PairArgs &A_) : s(s_), A(A_) {
    tid = threadIdx.x;
    w = tid >> 5;
    lane = tid & 31;
    phase = 0;
    qn = 0;
  }

  __device__ void stat(int k, unsigned long long v) {
    if (v) atomicAdd(&s.cnt[k], v);
  }

  __device__ int ntiles(int n) const { return (n + TT - 1) / TT; }

  // entry k of the pair-interval list: shared memory, then the CTA's spill region
  __device__ __forceinline__ unsigned long long il_entry(int k) const {
    return k < ILCAP ? s.il[k] : A.ilg[(int64_t)blockIdx.x * A.ilg_cap + (k - ILCAP)];
  }
  __device__ __forceinline__ int il_count() const {
    const int64_t cap = (int64_t)ILCAP + (A.ilg ? A.ilg_cap : 0);
    return s.nil < cap ? s.nil : int(cap);
  }

  // --- tile culling (particles with more than one tile) ---------------------
  // Bounding sphere of tile k of A or B in the evaluation frame: the stored
  // body-frame tile sphere of a multi-tile particle, else the body origin with
  // the particle radius; moved like the vertices (FP32: B into A's frame;
  // FP64: both into the world frame).
  __device__ void tile_sphere(bool isA, int k, T c[3], T &r) const {
    const int64_t p = isA ? s.i : s.j, off = isA ? s.offA : s.offB;
    const int n = isA ? s.nA : s.nB;
    float4 f = make_float4(0.f, 0.f, 0.f, __double2float_ru(A.st[16 * A.n + p]));
    const int64_t slot = off / TT + p + k;
    if (n > TT && slot < A.cap_tiles) f = A.tile_sph[slot];
    r = T(f.w);
    if constexpr (PREC == 0) {
      if (isA) {
        c[0] = f.x;
        c[1] = f.y;
        c[2] = f.z;
      } else {
        const float *R = s.Rr;
        c[0] = fmaf(R[0], f.x, fmaf(R[1], f.y, fmaf(R[2], f.z, s.tr[0])));
        c[1] = fmaf(R[3], f.x, fmaf(R[4], f.y, fmaf(R[5], f.z, s.tr[1])));
        c[2] = fmaf(R[6], f.x, fmaf(R[7], f.y, fmaf(R[8], f.z, s.tr[2])));
      }
    } else {
      const V3<double> q = to_world_exact(isA ? s.RA : s.RB, isA ? s.XA : s.XB, f.x, f.y, f.z);
      c[0] = q.x;
      c[1] = q.y;
      c[2] = q.z;
    }
  }
  // distance between the centres of the tile spheres of (ta, tb)
  __device__ T tile_gap(int ta, int tb, T &ra, T &rb) const {
    T ca[3], cb[3];
    tile_sphere(true, ta, ca, ra);
    tile_sphere(false, tb, cb, rb);
    const T dx = ca[0] - cb[0], dy = ca[1] - cb[1], dz = ca[2] - cb[2];
    return O::sqrt(dx * dx + dy * dy + dz * dz);
  }
  // distance from point c (body frame of the particle) to its tile k's box
  __device__ double box_gap(bool isA, int k, const double c[3]) const {
    const int64_t p = isA ? s.i : s.j, off = isA ? s.offA : s.offB;
    const int64_t slot = off / TT + p + k;
    const float4 lo = A.tile_box[2 * slot], hi = A.tile_box[2 * slot + 1];
    const double l[3] = {lo.x, lo.y, lo.z}, h[3] = {hi.x, hi.y, hi.z};
    double gg = 0.0;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      const double g = c[q] < l[q] ? l[q] - c[q] : (c[q] > h[q] ? c[q] - h[q] : 0.0);
      gg += g * g;
    }
    return sqrt(gg);
  }
  // the evaluation-frame point c in the body frame of A (isA) or B
  __device__ void to_body(bool isA, const T c[3], double out[3]) const {
    if constexpr (PREC == 0) {
      if (isA) {  // A's body frame is the evaluation frame
        out[0] = c[0];
        out[1] = c[1];
        out[2] = c[2];
      } else {  // B's vertices are Rr v + tr: v = Rr^T (c - tr)
        const float *R = s.Rr;
        const float p0 = c[0] - s.tr[0], p1 = c[1] - s.tr[1], p2 = c[2] - s.tr[2];
        out[0] = R[0] * p0 + R[3] * p1 + R[6] * p2;
        out[1] = R[1] * p0 + R[4] * p1 + R[7] * p2;
        out[2] = R[2] * p0 + R[5] * p1 + R[8] * p2;
      }
    } else {  // world frame: R^T (c - X)
      const double *R = isA ? s.RA : s.RB, *X = isA ? s.XA : s.XB;
      const double p0 = c[0] - X[0], p1 = c[1] - X[1], p2 = c[2] - X[2];
      out[0] = R[0] * p0 + R[3] * p1 + R[6] * p2;
      out[1] = R[1] * p0 + R[4] * p1 + R[7] * p2;
      out[2] = R[2] * p0 + R[5] * p1 + R[8] * p2;
    }
  }
  // false only if no triangle pair of tiles (ta, tb) can come within thr.
  // Lower bounds: the distance of the two tile spheres, and for a tile of a
  // multi-tile particle the distance from the other tile's sphere to its
  // body-frame box (a floor's flat tiles are far tighter as boxes).  The
  // margin 2 Elb covers the rounding of the sphere test (as for groups) and
  // of moving a centre between frames.
  __device__ bool tile_near(int ta, int tb, double thr) const {
    T ca[3], cb[3], ra, rb;
    tile_sphere(true, ta, ca, ra);
    tile_sphere(false, tb, cb, rb);
    const T dx = ca[0] - cb[0], dy = ca[1] - cb[1], dz = ca[2] - cb[2];
    double lb = double(O::sqrt(dx * dx + dy * dy + dz * dz) - ra - rb);
    const int64_t slotA = s.offA / TT + s.i + ta, slotB = s.offB / TT + s.j + tb;
    if (s.nB > TT && slotB < A.cap_tiles) {
      double q[3];
      to_body(false, ca, q);
      lb = fmax(lb, box_gap(false, tb, q) - double(ra));
    }
    if (s.nA > TT && slotA < A.cap_tiles) {
      double q[3];
      to_body(true, cb, q);
      lb = fmax(lb, box_gap(true, ta, q) - double(rb));
    }
    return lb <= thr + 2.0 * s.Elb;
  }
  // Lower the shared bound with the upper bound every tile pair gives on the
  // smallest triangle-pair distance (any point of one tile sphere is within
  // gap + ra + rb of any point of the other), and return the tile pair
  // q = ta * ntb + tb with the smallest lower bound (ties: smallest q).
  __device__ int bound_by_tiles(int nta, int ntb) {
    double best = OpsD::inf(), ub = OpsD::inf();
    int bq = 0;
    for (int q = tid; q < nta * ntb; q += NT) {
      T ra, rb;
      const T g = tile_gap(q / ntb, q % ntb, ra, rb);
      const double lb = double(g - ra - rb);
      ub = fmin(ub, double(g + ra + rb) + 2.0 * s.Elb + 2.0 * s.Ed + s.Eam);
      if (lb < best) {
        best = lb;
        bq = q;
      }
    }
    if (ub < OpsD::inf()) atomicMin(&s.bound, dbits(ub));
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      const double ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int oq = __shfl_xor_sync(0xffffffffu, bq, o);
      if (ob < best || (ob == best && oq < bq)) {
        best = ob;
        bq = oq;
      }
    }
    if (lane == 0) {
      s.red_d[w] = best;
      s.red_k[w] = (unsigned long long)bq;
    }
    __syncthreads();
    if (tid == 0) {
      double b = s.red_d[0];
      int q = int(s.red_k[0]);
      for (int k = 1; k < NW; ++k)
        if (s.red_d[k] < b || (s.red_d[k] == b && int(s.red_k[k]) < q)) {
          b = s.red_d[k];
          q = int(s.red_k[k]);
        }
      s.tfirst = q;
    }
    __syncthreads();
    return s.tfirst;
  }

  // --- tiles -------------------------------------------------------------
  // Make body tile ta of A resident (B is read from global memory when its
  // frame is built); false if the copy timed out.
  __device__ bool load_tiles(int ta, int tb) {
    const bool needA = s.resA != ta;
    __syncthreads();  // all reads of the previous tile are done
    if (tid == 0 && s.resB != tb) {
      s.resB = tb;
      s.frmB = -1;
    }
    if (!needA) {
      __syncthreads();
      return true;
    }
    const int na = min(TT, s.nA - ta * TT);
    if (tid == 0) {
      s.resA = ta;
      s.frmA = -1;
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mbar_expect_tx(&s.mbar, 3u * 16u * na);
      for (int sl = 0; sl < 3; ++sl)
        bulk_g2s(&s.Ab[sl][0], A.tris + sl * A.n_tris + s.offA + (int64_t)ta * TT, 16u * na, &s.mbar);
    }
    bool ok = mbar_wait(&s.mbar, phase, A.wait_polls);
    ok = __syncthreads_and(ok) != 0;
    phase ^= 1u;
    if (!ok) {
      if (tid == 0) {
        set_err(A.err, ERR_TIMEOUT);
        s.abort = 1;
      }
      // let the copy in flight land (full-length wait); if this runs out too,
      // the copy may still write this CTA's shared memory after it exits
      if (!mbar_wait(&s.mbar, phase ^ 1u) && tid == 0) set_err(A.err, ERR_DRAIN);
    }
    __syncthreads();
    return ok;
  }

  // triangle spheres (centroid, max vertex distance) of n triangles
  __device__ void spheres(T (*S)[TT], int n, bool isA) {
    for (int k = tid; k < n; k += NT) {
      V v[3];
      load_vtx(isA, k, v);
      T third = T(1) / T(3);
      T cx = (v[0].x + v[1].x + v[2].x) * third;
      T cy = (v[0].y + v[1].y + v[2].y) * third;
      T cz = (v[0].z + v[1].z + v[2].z) * third;
      T r2 = T(0);
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        T dx = v[q].x - cx, dy = v[q].y - cy, dz = v[q].z - cz;
        T d = dx * dx + dy * dy + dz * dz;
        r2 = d > r2 ? d : r2;
      }
      // a non-finite vertex makes the centre or the radius non-finite; its
      // sphere then fails every culling test, so the pair's result would be
      // silently incomplete: report it
      if (!(r2 <= T(3.0e38)) || !(fabs(double(cx) + double(cy) + double(cz)) <= 1.0e300)) set_err(A.err, ERR_NONFINITE);
      S[0][k] = cx;
      S[1][k] = cy;
      S[2][k] = cz;
      S[3][k] = O::sqrt(r2);
    }
  }
  // group (32 triangles) and subgroup (8 triangles) spheres: box centre of
  // the triangle spheres, radius covering every triangle sphere
  __device__ void groups(T (*S)[TT], T (*GS)[NG], T (*HS)[NH], int n) {
    const int ng = (n + G - 1) / G;
    const T big = O::inf();
    for (int g = w; g < ng; g += NW) {
      const int k = g * G + lane;
      const bool v = k < n;
      const T cx = v ? S[0][k] : T(0), cy = v ? S[1][k] : T(0), cz = v ? S[2][k] : T(0), r = v ? S[3][k] : T(0);
#pragma unroll
      for (int lvl = 0; lvl < 2; ++lvl) {
        const int wd = lvl == 0 ? G : H;
        const T lox = seg_min(v ? cx - r : big, wd), hix = seg_max(v ? cx + r : -big, wd);
        const T loy = seg_min(v ? cy - r : big, wd), hiy = seg_max(v ? cy + r : -big, wd);
        const T loz = seg_min(v ? cz - r : big, wd), hiz = seg_max(v ? cz + r : -big, wd);
        const T gx = (lox + hix) * T(0.5), gy = (loy + hiy) * T(0.5), gz = (loz + hiz) * T(0.5);
        const T dx = cx - gx, dy = cy - gy, dz = cz - gz;
        const T gr = seg_max(v ? O::sqrt(dx * dx + dy * dy + dz * dz) + r : T(0), wd);
        if (lvl == 0 && lane == 0) {
          GS[0][g] = gx;
          GS[1][g] = gy;
          GS[2][g] = gz;
          GS[3][g] = gr;
        }
        if (lvl == 1 && (lane & (H - 1)) == 0) {
          const int h = g * (G / H) + (lane / H);
          HS[0][h] = gx;
          HS[1][h] = gy;
          HS[2][h] = gz;
          HS[3][h] = gr;
        }
      }
    }
  }

  // vertices of triangle k of the A or B tile in the evaluation frame
  __device__ __forceinline__ void load_vtx(bool isA, int k, V v[3]) const {
    if constexpr (PREC == 0) {
      if (isA) {
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          float4 f = s.Ab[q][k];
          v[q] = V{T(f.x), T(f.y), T(f.z)};
        }
      } else {
#pragma unroll
        for (int q = 0; q < 3; ++q) v[q] = V{s.Be[3 * q][k], s.Be[3 * q + 1][k], s.Be[3 * q + 2][k]};
      }
    } else {
      if (isA) {
#pragma unroll
        for (int q = 0; q < 3; ++q) v[q] = V{s.Ae[3 * q][k], s.Ae[3 * q + 1][k], s.Ae[3 * q + 2][k]};
      } else {
#pragma unroll
        for (int q = 0; q < 3; ++q) v[q] = V{s.Be[3 * q][k], s.Be[3 * q + 1][k], s.Be[3 * q + 2][k]};
      }
    }
  }

  // evaluation-frame data for tiles (ta, tb) at the current time
  __device__ void frames(int ta, int tb) {
    const int na = min(TT, s.nA - ta * TT), nb = min(TT, s.nB - tb * TT);
    const bool doA = s.frmA != ta, doB = s.frmB != tb;
    if (!doA && !doB) return;
    if constexpr (PREC == 1) {
      if (doA)
        for (int k = tid; k < na; k += NT)
#pragma unroll
          for (int q = 0; q < 3; ++q) {
            float4 f = s.Ab[q][k];
            V3<double> p = to_world_exact(s.RA, s.XA, f.x, f.y, f.z);
            s.Ae[3 * q][k] = T(p.x);
            s.Ae[3 * q + 1][k] = T(p.y);
            s.Ae[3 * q + 2][k] = T(p.z);
          }
    }
    if constexpr (PREC == 0) {
      if (doB) {
        if (tid == 0) tile_frame(tb);
        __syncthreads();
      }
    }
    if (doB) {
      for (int k = tid; k < nb; k += NT)
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          const float4 f = A.tris[q * A.n_tris + s.offB + tb * TT + k];
          if constexpr (PREC == 0) {
            // relative to the tile's local origin: every term of the FP32
            // transform is at the tile's scale, not the whole mesh's
            const float *R = s.Rr;
            const float bx = f.x - s.oo[0], by = f.y - s.oo[1], bz = f.z - s.oo[2];
            s.Be[3 * q][k] = T(fmaf(R[0], bx, fmaf(R[1], by, fmaf(R[2], bz, s.to[0]))));
            s.Be[3 * q + 1][k] = T(fmaf(R[3], bx, fmaf(R[4], by, fmaf(R[5], bz, s.to[1]))));
            s.Be[3 * q + 2][k] = T(fmaf(R[6], bx, fmaf(R[7], by, fmaf(R[8], bz, s.to[2]))));
          } else {
            V3<double> p = to_world_exact(s.RB, s.XB, f.x, f.y, f.z);
            s.Be[3 * q][k] = T(p.x);
            s.Be[3 * q + 1][k] = T(p.y);
            s.Be[3 * q + 2][k] = T(p.z);
          }
        }
    }
    __syncthreads();
    if (doA) spheres(s.SA, na, true);
    if (doB) spheres(s.SB, nb, false);
    __syncthreads();
    if (doA) groups(s.SA, s.GA, s.HA, na);
    if (doB) groups(s.SB, s.GB, s.HB, nb);
    __syncthreads();
    if (tid == 0) {
      s.frmA = ta;
      s.frmB = tb;
    }
  }

  // --- exact binary64 triangle pair (world frame, fixed operation order) --
  // triangles a, b (indices within particles i, j), read from global memory
  __device__ __noinline__ double exact_global(int a, int b, V3<double> &pa, V3<double> &pb) const {
    V3<double> X[3], Y[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      const float4 f = A.tris[q * A.n_tris + s.offA + a];
      X[q] = to_world_exact(s.RA, s.XA, f.x, f.y, f.z);
      const float4 g = A.tris[q * A.n_tris + s.offB + b];
      Y[q] = to_world_exact(s.RB, s.XB, g.x, g.y, g.z);
    }
    return GD::tri_dist2(X, Y, pa, pb);
  }

  // FP32 frame of B's tile tb (thread 0): local origin o = the tile sphere's
  // centre for a particle of several tiles, else B's body origin; its
  // position t_o = R_A^T (R_B o + X_B - X_A) in A's frame (binary64, rounded
  // once); margin E of the tile = 2^-17 (R_A + r + |t_o|), r bounding the
  // tile's vertices about o -- the scale of every FP32 coordinate and term of
  // the tile's transform Rr (b - o) + t_o.
  __device__ void tile_frame(int tb) {
    const int64_t slot = s.offB / TT + s.j + tb;
    float o[3] = {0.f, 0.f, 0.f};
    double r = A.st[16 * A.n + s.j];
    if (s.nB > TT && slot < A.cap_tiles) {
      const float4 f = A.tile_sph[slot];
      o[0] = f.x;
      o[1] = f.y;
      o[2] = f.z;
      r = f.w;
    }
    double t[3];
    local_origin(o, t);
    for (int c = 0; c < 3; ++c) {
      s.oo[c] = o[c];
      s.to[c] = float(t[c]);
    }
    s.Et = ERR_REL32 * (A.st[16 * A.n + s.i] + r + sqrt(t[0] * t[0] + t[1] * t[1] + t[2] * t[2]));
  }
  // position in A's frame of B's body-frame point o: R_A^T (R_B o + X_B - X_A)
  __device__ void local_origin(const float o[3], double t[3]) const {
    double w[3];
    for (int r = 0; r < 3; ++r)
      w[r] = s.RB[3 * r] * double(o[0]) + s.RB[3 * r + 1] * double(o[1]) + s.RB[3 * r + 2] * double(o[2]) +
             (s.XB[r] - s.XA[r]);
    for (int c = 0; c < 3; ++c) t[c] = s.RA[c] * w[0] + s.RA[3 + c] * w[1] + s.RA[6 + c] * w[2];
  }

  // Certified lower bound (FP32 mode) of the binary64 distance of the A-frame
  // FP32 triangles X, Y whose computed closest points are pa, pb: their
  // separation along pb - pa less E (the rounding of the separation, of the
  // FP32 relative pose and the binary64 underestimate; E = 2^-17 S of the
  // frame the coordinates come from); -inf when the points coincide.
  __device__ __forceinline__ double certificate(const V3<float> X[3], const V3<float> Y[3], V3<float> pa,
                                                V3<float> pb, double E) const {
    const V3<float> n{pb.x - pa.x, pb.y - pa.y, pb.z - pa.z};
    return double(cert_sep(X, 3, Y, 3, n)) - E;
  }

  // One feature of triangles a (particle i) and b (particle j) in binary64,
  // world frame, exactly as the binary64 triangle distance computes it.
  __device__ __noinline__ double feature64(int f, int a, int b, V3<double> &pa, V3<double> &pb) const {
    V3<double> X[3], Y[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      const float4 fa = A.tris[q * A.n_tris + s.offA + a];
      X[q] = to_world_exact(s.RA, s.XA, fa.x, fa.y, fa.z);
      const float4 fb = A.tris[q * A.n_tris + s.offB + b];
      Y[q] = to_world_exact(s.RB, s.XB, fb.x, fb.y, fb.z);
    }
    return GD::feature_dist2(f, X, Y, pa, pb);
  }

  // The same binary64 triangle distance with one warp per triangle pair.
  // Lanes 0..5 run the six edge-triangle crossing tests in binary64.  Lanes
  // 8..13 (vertex-triangle) and 16..24 (edge-edge) first compute their
  // feature in FP32 (A's frame) with its certificate; the feature closest in
  // FP32 is recomputed in binary64 as the reference, then every feature whose
  // certificate does not exceed the reference (plus m64): every feature that
  // can attain the binary64 minimum is among them, so the minimum and its
  // first attaining feature (sequential order, strict "<") are those of
  // Geo<OpsD>::tri_dist2.  cross = false skips the crossing tests: the caller
  // has certified the pair's binary64 distance positive, so no crossing
  // exists.  a, b index triangles within particles i, j.  Every lane returns
  // the result.
  __device__ __noinline__ double exact_warp(int a, int b, V3<double> &pa, V3<double> &pb, bool cross = true) const {
    using GF = Geo<OpsF>;
    V3<double> v{0.0, 0.0, 0.0};
    V3<float> vf{0.f, 0.f, 0.f};
    if (lane < 6) {
      const int q = lane < 3 ? lane : lane - 3;
      const float4 f = lane < 3 ? A.tris[q * A.n_tris + s.offA + a] : A.tris[q * A.n_tris + s.offB + b];
      if (lane < 3) {
        v = to_world_exact(s.RA, s.XA, f.x, f.y, f.z);
        vf = V3<float>{f.x, f.y, f.z};
      } else {
        v = to_world_exact(s.RB, s.XB, f.x, f.y, f.z);
        const float *R = s.Rr;
        vf = V3<float>{fmaf(R[0], f.x, fmaf(R[1], f.y, fmaf(R[2], f.z, s.tr[0]))),
                       fmaf(R[3], f.x, fmaf(R[4], f.y, fmaf(R[5], f.z, s.tr[1]))),
                       fmaf(R[6], f.x, fmaf(R[7], f.y, fmaf(R[8], f.z, s.tr[2])))};
      }
    }
    V3<double> X[3], Y[3];
    V3<float> Xf[3], Yf[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      X[q] = V3<double>{__shfl_sync(0xffffffffu, v.x, q), __shfl_sync(0xffffffffu, v.y, q),
                        __shfl_sync(0xffffffffu, v.z, q)};
      Y[q] = V3<double>{__shfl_sync(0xffffffffu, v.x, q + 3), __shfl_sync(0xffffffffu, v.y, q + 3),
                        __shfl_sync(0xffffffffu, v.z, q + 3)};
      Xf[q] = V3<float>{__shfl_sync(0xffffffffu, vf.x, q), __shfl_sync(0xffffffffu, vf.y, q),
                        __shfl_sync(0xffffffffu, vf.z, q)};
      Yf[q] = V3<float>{__shfl_sync(0xffffffffu, vf.x, q + 3), __shfl_sync(0xffffffffu, vf.y, q + 3),
                        __shfl_sync(0xffffffffu, vf.z, q + 3)};
    }
    const bool fvt = lane >= 8 && lane < 14, fee = lane >= 16 && lane < 25;
    const int ord = lane < 11 ? lane - 8 : (lane < 14 ? lane - 8 : lane - 10);
    const int vi = lane < 11 ? lane - 8 : lane - 11;       // vertex index of a VT lane
    const int ei = (lane - 16) / 3, ej = (lane - 16) % 3;  // edge indices of an EE lane
    // binary64 crossing tests
    bool hit = false;
    V3<double> p1{0.0, 0.0, 0.0}, p2{0.0, 0.0, 0.0};
    if (!cross) {
    } else if (lane < 3) {
      hit = GD::seg_tri_cross(X[lane], X[lane == 2 ? 0 : lane + 1], Y[0], Y[1], Y[2], p1);
    } else if (lane < 6) {
      const int j = lane - 3;
      hit = GD::seg_tri_cross(Y[j], Y[j == 2 ? 0 : j + 1], X[0], X[1], X[2], p1);
    }
    // FP32 feature distances and their certified lower bounds
    float df = OpsF::inf();
    double Lf = -OpsD::inf();
    {
      V3<float> q1, q2;
      if (fvt) {
        if (lane < 11) {
          df = GF::closest_pt_tri(Xf[vi], Yf[0], Yf[1], Yf[2], q1);
          Lf = double(cert_sep(&Xf[vi], 1, Yf, 3, V3<float>{q1.x - Xf[vi].x, q1.y - Xf[vi].y, q1.z - Xf[vi].z}));
        } else {
          df = GF::closest_pt_tri(Yf[vi], Xf[0], Xf[1], Xf[2], q1);
          Lf = double(cert_sep(Xf, 3, &Yf[vi], 1, V3<float>{Yf[vi].x - q1.x, Yf[vi].y - q1.y, Yf[vi].z - q1.z}));
        }
      } else if (fee) {
        const V3<float> sa[2] = {Xf[ei], Xf[ei == 2 ? 0 : ei + 1]}, sb[2] = {Yf[ej], Yf[ej == 2 ? 0 : ej + 1]};
        df = GF::seg_seg(sa[0], sa[1], sb[0], sb[1], q1, q2);
        Lf = double(cert_sep(sa, 2, sb, 2, V3<float>{q2.x - q1.x, q2.y - q1.y, q2.z - q1.z}));
      }
      df = OpsF::sqrt(df);
      Lf -= s.Ed;
    }
    const uint32_t hm = __ballot_sync(0xffffffffu, hit) & 0x3fu;
    if (hm) {
      const int src = __ffs(hm) - 1;
      pa = V3<double>{__shfl_sync(0xffffffffu, p1.x, src), __shfl_sync(0xffffffffu, p1.y, src),
                      __shfl_sync(0xffffffffu, p1.z, src)};
      pb = pa;
      return 0.0;
    }
    // the feature closest in FP32 (ties: the definition's order) gives the
    // binary64 reference; every feature whose certificate does not exceed it
    // can attain the binary64 minimum and is recomputed in binary64
    float rm = (fvt || fee) ? df : OpsF::inf();
    int ro = (fvt || fee) ? ord : 99;
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      const float om = __shfl_xor_sync(0xffffffffu, rm, o);
      const int oo = __shfl_xor_sync(0xffffffffu, ro, o);
      if (om < rm || (om == rm && oo < ro)) {
        rm = om;
        ro = oo;
      }
    }
    auto feature_b64 = [&](double &d2) {
      if (fvt) {
        if (lane < 11) {
          d2 = GD::closest_pt_tri(X[vi], Y[0], Y[1], Y[2], p2);
          p1 = X[vi];
        } else {
          d2 = GD::closest_pt_tri(Y[vi], X[0], X[1], X[2], p1);
          p2 = Y[vi];
        }
      } else {
        d2 = GD::seg_seg(X[ei], X[ei == 2 ? 0 : ei + 1], Y[ej], Y[ej == 2 ? 0 : ej + 1], p1, p2);
      }
    };
    const bool isref = (fvt || fee) && ord == ro;
    double d2 = OpsD::inf();
    if (isref) feature_b64(d2);
    const int rsrc = ro < 3 ? 8 + ro : (ro < 6 ? 11 + (ro - 3) : 16 + (ro - 6));
    const double dref = OpsD::sqrt(__shfl_sync(0xffffffffu, d2, rsrc));
    const bool need = (fvt || fee) && !isref && Lf <= dref + s.m64;
    if (need) feature_b64(d2);
    double bd = d2;
    int bo = (need || isref) ? ord : 99;
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      const double od = __shfl_xor_sync(0xffffffffu, bd, o);
      const int oo = __shfl_xor_sync(0xffffffffu, bo, o);
      if (od < bd || (od == bd && oo < bo)) {
        bd = od;
        bo = oo;
      }
    }
    const int src = bo < 3 ? 8 + bo : (bo < 6 ? 11 + (bo - 3) : 16 + (bo - 6));
    pa = V3<double>{__shfl_sync(0xffffffffu, p1.x, src), __shfl_sync(0xffffffffu, p1.y, src),
                    __shfl_sync(0xffffffffu, p1.z, src)};
    pb = V3<double>{__shfl_sync(0xffffffffu, p2.x, src), __shfl_sync(0xffffffffu, p2.y, src),
                    __shfl_sync(0xffffffffu, p2.z, src)};
    return bd;
  }

  __device__ void world_of_A_frame(const V &p, double out[3]) const {
    // FP32 points live in A's body frame: x_world = R_A p + X_A (explicit
    // FMA chain: the same result in every kernel that uses it)
    const double x = p.x, y = p.y, z = p.z;
    out[0] = __fma_rn(s.RA[0], x, __fma_rn(s.RA[1], y, __fma_rn(s.RA[2], z, s.XA[0])));
    out[1] = __fma_rn(s.RA[3], x, __fma_rn(s.RA[4], y, __fma_rn(s.RA[5], z, s.XA[1])));
    out[2] = __fma_rn(s.RA[6], x, __fma_rn(s.RA[7], y, __fma_rn(s.RA[8], z, s.XA[2])));
  }

  __device__ __forceinline__ unsigned long long key_of(int a, int b, int ta, int tb) const {
    return (static_cast<unsigned long long>(ta * TT + a) << 32) | static_cast<unsigned>(tb * TT + b);
  }

  // write a warp's contacts (lanes with con) to the staging area
  __device__ void put_contacts(bool con, int64_t pk, int ag, int bg, double gd, const double *ga3,
                               const double *gb3) {
    const uint32_t m = __ballot_sync(0xffffffffu, con);
    if (!m) return;
    unsigned long long base = 0;
    if (lane == 0) {
      base = atomicAdd(A.st_count, (unsigned long long)__popc(m));
      atomicAdd(reinterpret_cast<unsigned long long *>(&A.pc[pk]), (unsigned long long)__popc(m));
      atomicAdd(&s.cnt[ST_CONTACTS], (unsigned long long)__popc(m));
    }
    base = __shfl_sync(0xffffffffu, base, 0);
    if (con) {
      const unsigned long long slot = base + __popc(m & lanemask_lt());
      if (slot < (unsigned long long)A.st_cap) {
        A.st_keys[3 * slot] = int32_t(pk);
        A.st_keys[3 * slot + 1] = ag;
        A.st_keys[3 * slot + 2] = bg;
        double *gg = A.st_geom + 7 * slot;
        gg[0] = gd;
        gg[1] = ga3[0]; gg[2] = ga3[1]; gg[3] = ga3[2];
        gg[4] = gb3[0]; gg[5] = gb3[1]; gg[6] = gb3[2];
      } else {
        set_err(A.err, ERR_CAPACITY);
      }
    }
  }

  // FP32 mode: stage a warp's contact candidates (pairs not certified apart)
  // with the feature the FP32 pass found closest; contact_verify decides each
  // in binary64 after the launch and counts the accepted ones per pair
  __device__ void put_candidates(bool cand, int64_t pk, int ag, int bg, int feat) {
    const uint32_t m = __ballot_sync(0xffffffffu, cand);
    if (!m) return;
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(A.st_count, (unsigned long long)__popc(m));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (cand) {
      const unsigned long long slot = base + __popc(m & lanemask_lt());
      if (slot < (unsigned long long)A.st_cap) {
        A.st_keys[3 * slot] = int32_t(pk);
        A.st_keys[3 * slot + 1] = ag;
        A.st_keys[3 * slot + 2] = bg;
        A.st_geom[7 * slot] = double(feat);
      } else {
        set_err(A.err, ERR_CAPACITY);
      }
    }
  }

  __device__ void update_best(double d2, unsigned long long key, const V3<double> &pa, const V3<double> &pb) {
    if (d2 < bd2 || (d2 == bd2 && key < bkey)) {
      bd2 = d2;
      bkey = key;
      bpa[0] = pa.x; bpa[1] = pa.y; bpa[2] = pa.z;
      bpb[0] = pb.x; bpb[1] = pb.y; bpb[2] = pb.z;
    }
  }

  // warp-wide best (d^2, key) into the uniform wbd2 / wbkey
  __device__ void warp_best() {
    double d = bd2;
    unsigned long long k = bkey;
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      const double od = __shfl_xor_sync(0xffffffffu, d, o);
      const unsigned long long ok = __shfl_xor_sync(0xffffffffu, k, o);
      if (od < d || (od == d && ok < k)) {
        d = od;
        k = ok;
      }
    }
    wbd2 = d;
    wbkey = k;
  }

  // --- the warp's binary64 queue: full-lane passes ---------------------------
  template <bool DECIDE, bool ARGMIN, bool CONTACTS>
  __device__ void flush_queue(int ta, int tb, int64_t pk) {
    unsigned long long n64 = 0;
    if (qn <= QWARP) {
      // few entries: one triangle pair at a time, lanes over its features
      for (int q = 0; q < qn; ++q) {
        const uint32_t ent = s.xq[w][q];
        const uint32_t why = ent >> 28;
        const int a = int((ent >> 14) & 0x3fffu), b = int(ent & 0x3fffu);
        const unsigned long long key = key_of(a, b, ta, tb);
        if (why == WHY_ARG && wbd2 == 0.0 && key > wbkey) continue;
        if (DECIDE && !ARGMIN && !CONTACTS) {
          // one read per warp, broadcast: the exit is warp-uniform
          const int f = lane == 0 ? *(volatile int *)&s.found : 0;
          if (__shfl_sync(0xffffffffu, f, 0)) break;
        }
        V3<double> qa, qb;
        // a queued pair is not certified apart: it may cross
        const double e2 = exact_warp(ta * TT + a, tb * TT + b, qa, qb, true);
        ++n64;
        const double de = OpsD::sqrt(e2);
        if (DECIDE && (why & WHY_DEC) && de <= s.eps && lane == 0) s.found = 1;
        if (CONTACTS) {
          const bool con = lane == 0 && (why & WHY_CON) && de <= s.eps;
          const double ga3[3] = {qa.x, qa.y, qa.z}, gb3[3] = {qb.x, qb.y, qb.z};
          put_contacts(con, pk, ta * TT + a, tb * TT + b, de, ga3, gb3);
        }
        if (ARGMIN && (why & WHY_ARG)) {
          update_best(e2, key, qa, qb);
          warp_best();
        }
      }
      qn = 0;
      if (lane == 0) stat(ST_FP64, n64);
      return;
    }
    for (int q0 = 0; q0 < qn; q0 += 32) {
      const int k = q0 + lane;
      const bool have = k < qn;
      const uint32_t ent = have ? s.xq[w][k] : 0u;
      const uint32_t why = ent >> 28;
      const int a = int((ent >> 14) & 0x3fffu), b = int(ent & 0x3fffu);
      const unsigned long long key = key_of(a, b, ta, tb);
      // an argmin-only candidate that cannot beat a zero-distance best is skipped
      const bool skip = why == WHY_ARG && wbd2 == 0.0 && key > wbkey;
      double e2 = OpsD::inf();
      V3<double> qa{}, qb{};
      if (have && !skip) {
        e2 = exact_global(ta * TT + a, tb * TT + b, qa, qb);
        ++n64;
      }
      const double de = OpsD::sqrt(e2);
      if (DECIDE) {
        const bool yes = have && (why & WHY_DEC) && de <= s.eps;
        if (__any_sync(0xffffffffu, yes) && lane == 0) s.found = 1;
      }
      if (CONTACTS) {
        const bool con = have && (why & WHY_CON) && de <= s.eps;
        const double ga3[3] = {qa.x, qa.y, qa.z}, gb3[3] = {qb.x, qb.y, qb.z};
        put_contacts(con, pk, ta * TT + a, tb * TT + b, de, ga3, gb3);
      }
      if (ARGMIN) {
        if (have && !skip && (why & WHY_ARG)) update_best(e2, key, qa, qb);
        warp_best();
      }
    }
    qn = 0;
#pragma unroll
    for (int o = 16; o; o >>= 1) n64 += __shfl_xor_sync(0xffffffffu, n64, o);
    if (lane == 0) stat(ST_FP64, n64);
  }

  // --- evaluate a warp's candidate list ------------------------------------
  template <bool DECIDE, bool ARGMIN, bool CONTACTS>
  __device__ void warp_eval(const uint32_t *list, int cnt, int ta, int tb, int64_t pk, bool pass1) {
    const T eps = T(s.eps);
    const T Ed = T(s.Ed);
    unsigned long long n32 = 0, nv64 = 0;
    for (int e = 0; e < cnt; e += 32) {
      const int k = e + lane;
      const bool have = k < cnt;
      const uint32_t ent = have ? list[k] : 0u;
      const int a = int(ent >> 16), b = int(ent & 0xffffu);
      T d2 = O::inf();
      V pa{}, pb{};
      int feat = 0;
      double L = -OpsD::inf();  // FP32: certified lower bound of the binary64 distance
      if (have) {
        V X[3], Y[3];
        load_vtx(true, a, X);
        load_vtx(false, b, Y);
        if constexpr (PREC == 0) {
          // a decision alone needs no FP32 crossing test: crossing triangles
          // have no separating direction, so their certificate never clears them
          if (DECIDE && !ARGMIN && !CONTACTS)
            d2 = GT::tri_dist2_features(X, Y, pa, pb, feat);
          else
            d2 = GT::tri_dist2(X, Y, pa, pb, feat);
          L = certificate(X, Y, pa, pb, s.Et);
        } else if (DECIDE && !ARGMIN && !CONTACTS) {
          // features first; the crossing test only when they do not settle it
          d2 = GT::tri_dist2_features(X, Y, pa, pb);
          if (!(O::sqrt(d2) < eps - Ed)) {
            V x;
            bool hit = false;
            for (int q = 0; q < 3 && !hit; ++q)
              hit = GT::seg_tri_cross(X[q], X[q == 2 ? 0 : q + 1], Y[0], Y[1], Y[2], x);
            for (int q = 0; q < 3 && !hit; ++q)
              hit = GT::seg_tri_cross(Y[q], Y[q == 2 ? 0 : q + 1], X[0], X[1], X[2], x);
            if (hit) d2 = T(0);
          }
        } else {
          d2 = GT::tri_dist2(X, Y, pa, pb);
        }
        ++n32;
      }
      const T d = O::sqrt(d2);
      if (s.ilcol) {
        // remember the triangle pair for the rest of the pair interval when
        // it can come within eps in the interval: its distance at ts is at
        // most eps + delta (FP32: its certified lower bound; FP64: its value),
        // no other pair can
        const bool col = have && (PREC == 0 ? L : double(d)) <= s.ilthr;
        const uint32_t m = __ballot_sync(0xffffffffu, col);
        if (m) {
          int base = 0;
          if (lane == 0) base = atomicAdd(&s.nil, __popc(m));
          base = __shfl_sync(0xffffffffu, base, 0);
          if (col) {
            const int pos = base + __popc(m & lanemask_lt());
            const int ag = ta * TT + a, bg = tb * TT + b;
            // lower bound of the binary64 distance (FP32: the certificate,
            // rounded down), truncated to 16 bits of its float pattern
            float dlb;
            if constexpr (PREC == 0)
              dlb = __double2float_rd(L);
            else
              dlb = __double2float_rd(double(d));
            const unsigned long long dq = __float_as_uint(dlb > 0.0f ? dlb : 0.0f) >> 16;
            const unsigned long long ent =
                (dq << 48) | (static_cast<unsigned long long>(ag) << 24) | static_cast<uint32_t>(bg);
            if (pos < ILCAP)
              s.il[pos] = ent;
            else if (A.ilg && pos - ILCAP < A.ilg_cap)
              A.ilg[(int64_t)blockIdx.x * A.ilg_cap + (pos - ILCAP)] = ent;
            else
              s.ilover = 1;
          }
        }
      }
      const unsigned long long key = key_of(a, b, ta, tb);
      if constexpr (PREC == 0) {
        uint32_t why = 0;
        bool yes = false;
        double gd = 0.0;
        const bool apart = !have || L > s.eps + s.m64;
        if (DECIDE && ARGMIN) {
          // the decision is the binary64 closest pair's (eval); a pair not
          // certified apart only calls for that search
          if (__any_sync(0xffffffffu, !apart) && lane == 0) s.found = 1;
        } else if (DECIDE) {
          // apart: certified; in contact: the binary64 value of the feature
          // the FP32 pass found closest is within eps (the pair's binary64
          // distance can only be smaller) -- checked for the lane with the
          // smallest FP32 distance; otherwise binary64 in full
          const bool cand = have && !apart && d < eps;
          const T dm = warp_min(cand ? d : O::inf());
          const uint32_t pm = __ballot_sync(0xffffffffu, cand && d == dm);
          const bool pick = pm && lane == __ffs(pm) - 1;
          bool ok = false;
          if (pm) {
            V3<double> qa{0.0, 0.0, 0.0}, qb{0.0, 0.0, 0.0};
            double e2 = OpsD::inf();
            if (pick) {
              e2 = feature64(feat, ta * TT + a, tb * TT + b, qa, qb);
              ++nv64;
            }
            gd = OpsD::sqrt(e2);
            ok = pick && gd <= s.eps;
          }
          yes = ok;
          // every lane votes (a vote behind a lane-dependent && would leave
          // the lanes that skip it out of a full-mask collective)
          const bool any_ok = __any_sync(0xffffffffu, ok);
          if (!apart && !any_ok) why |= WHY_DEC;
        }
        if (CONTACTS) put_candidates(have && !apart, pk, ta * TT + a, tb * TT + b, feat);
        if (ARGMIN) {
          mw = fmin(mw, warp_min(have ? d : O::inf()));
          // candidates for the closest pair: certificate within the current
          // FP32 minimum plus the slack (checked against the binary64
          // reference distance in argmin_list)
          const bool am = have && L <= double(mw) + s.Eam;
          const uint32_t mm = __ballot_sync(0xffffffffu, am);
          if (mm) {
            int base = 0;
            if (lane == 0) base = atomicAdd(&s.nac, __popc(mm));
            base = __shfl_sync(0xffffffffu, base, 0);
            const int pos = base + __popc(mm & lanemask_lt());
            if (base + __popc(mm) <= ACAP) {
              if (am) {
                s.ac_key[pos] = key;
                s.ac_d[pos] = __double2float_rd(L);
              }
            } else {
              // list full: mark the reserved slots empty, recompute through the queue
              if (am && pos < ACAP) s.ac_key[pos] = ~0ull;
              if (am) why |= WHY_ARG;
            }
          }
        }
        if (DECIDE && __any_sync(0xffffffffu, yes) && lane == 0) s.found = 1;
        // queue the binary64 recomputations
        const uint32_t m = __ballot_sync(0xffffffffu, why != 0);
        if (m) {
          if (why) s.xq[w][qn + __popc(m & lanemask_lt())] = (why << 28) | (uint32_t(a) << 14) | uint32_t(b);
          qn += __popc(m);
          __syncwarp();
          if (qn > XQCAP - 32) flush_queue<DECIDE, ARGMIN, CONTACTS>(ta, tb, pk);
        }
      } else {
        if (DECIDE) {
          const bool yes = have && d <= eps;
          if (__any_sync(0xffffffffu, yes) && lane == 0) s.found = 1;
        }
        if (ARGMIN) {
          mw = fmin(mw, warp_min(have ? d : O::inf()));
          if (have) update_best(double(d2), key, V3<double>{pa.x, pa.y, pa.z}, V3<double>{pb.x, pb.y, pb.z});
        }
        if (CONTACTS) {
          const bool con = have && d <= eps;
          const double ga3[3] = {pa.x, pa.y, pa.z}, gb3[3] = {pb.x, pb.y, pb.z};
          put_contacts(con, pk, ta * TT + a, tb * TT + b, double(d), ga3, gb3);
        }
      }
      if (ARGMIN && pass1 && lane == 0) {
        // tighten the shared bound with this warp's minimum
        const double nb = double(mw) + s.Eam + s.Ed + s.Elb;
        atomicMin(&s.bound, dbits(nb));
      }
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      n32 += __shfl_xor_sync(0xffffffffu, n32, o);
      nv64 += __shfl_xor_sync(0xffffffffu, nv64, o);
    }
    if (lane == 0) {
      stat(ST_FP32, n32);
      stat(ST_FP64, nv64);
    }
  }

  // block-wide sort of the group-pair list by lower bound (bitonic)
  __device__ void sort_groups() {
    const int n = s.ngp;
    int n2 = 1;
    while (n2 < n) n2 <<= 1;
    for (int q = n + tid; q < n2; q += NT) {
      s.gplb[q] = __int_as_float(0x7f800000);
      s.gp[q] = 0u;
    }
    __syncthreads();
    for (int k = 2; k <= n2; k <<= 1)
      for (int j = k >> 1; j > 0; j >>= 1) {
        for (int q = tid; q < n2; q += NT) {
          const int l = q ^ j;
          if (l > q) {
            const bool up = (q & k) == 0;
            const float kq = s.gplb[q], kl = s.gplb[l];
            if ((kq > kl) == up) {
              s.gplb[q] = kl;
              s.gplb[l] = kq;
              const uint32_t t = s.gp[q];
              s.gp[q] = s.gp[l];
              s.gp[l] = t;
            }
          }
        }
        __syncthreads();
      }
  }

  // --- one pass over tile pair (ta, tb) -------------------------------------
  // pass 0: triangle pairs with sphere bound LB <= th0;
  // pass 1: LB <= bound (shared, shrinking), group pairs in order of their
  // lower bounds; the pairs with LB <= th0 are left out only when pass 0
  // scanned this tile pair (seen0) -- a tile pair that pass 0's tile test
  // culled has never had any of its pairs evaluated.
  template <bool DECIDE, bool ARGMIN, bool CONTACTS>
  __device__ void scan_tiles(int ta, int tb, bool pass1, T th0, int64_t pk, bool seen0 = true, bool merged = false) {
    const int na = min(TT, s.nA - ta * TT), nb = min(TT, s.nB - tb * TT);
    const int nga = (na + G - 1) / G, ngb = (nb + G - 1) / G;
    // culling margin: FP32 spheres of the tiles' FP32 vertices, the tile's scale
    const T Elb = T(PREC == 0 ? s.Et : s.Elb);
    // a merged pass (closest pair, contacts and interval list in one scan)
    // never culls below the first pass's threshold th0
    const T lift = merged ? th0 : -O::inf();
    if (tid == 0) {
      s.ngp = 0;
      s.gpnext = 0;
    }
    __syncthreads();
    // level 1: group pairs (32 x 32 triangles)
    {
      const T gth = pass1 ? fmax(T(bitsd(s.bound)), lift) + Elb : th0 + Elb;
      for (int q = tid; q < nga * ngb; q += NT) {
        const int ga = q / ngb, gb = q - ga * ngb;
        const T dx = s.GA[0][ga] - s.GB[0][gb], dy = s.GA[1][ga] - s.GB[1][gb], dz = s.GA[2][ga] - s.GB[2][gb];
        const T lb = O::sqrt(dx * dx + dy * dy + dz * dz) - s.GA[3][ga] - s.GB[3][gb];
        if (lb <= gth) {
          const int pos = atomicAdd(&s.ngp, 1);
          s.gp[pos] = (uint32_t(ga) << 16) | uint32_t(gb);
          s.gplb[pos] = down_f(lb);
        }
      }
      if (tid == 0) stat(ST_GROUP, (unsigned long long)(nga * ngb));
    }
    __syncthreads();
    if (pass1) sort_groups();
    // levels 2 and 3: warp w takes group pairs w, w + NW, ...; inside a group
    // pair the 16 subgroup pairs (8 x 8 triangles) are tested by lanes 0..15,
    // then each passing subgroup pair is two rows of 4 x 8 triangle pairs
    const int ngp = s.ngp;
    int cnt = 0;
    unsigned long long ntests = 0, nsub = 0;
    for (;;) {
      // group pairs are handed out one at a time (balanced across warps)
      int p = 0, f = 0;
      if (lane == 0) {
        p = atomicAdd(&s.gpnext, 1);
        if (DECIDE && !ARGMIN) f = *(volatile int *)&s.found;
      }
      p = __shfl_sync(0xffffffffu, p, 0);
      f = __shfl_sync(0xffffffffu, f, 0);
      if (p >= ngp || f) break;
      T bnd = T(0);
      if (pass1) {
        unsigned long long bb = lane == 0 ? *(volatile unsigned long long *)&s.bound : 0ull;
        bb = __shfl_sync(0xffffffffu, bb, 0);
        bnd = fmax(T(bitsd(bb)), lift);
        if (double(s.gplb[p]) > double(bnd) + double(Elb)) break;  // sorted: later ones fail too
      }
      const uint32_t gpe = s.gp[p];
      const int ga = int(gpe >> 16), gb = int(gpe & 0xffffu);
      // level 2
      const int ha = ga * (G / H) + ((lane >> 2) & 3), hb = gb * (G / H) + (lane & 3);
      bool subok = lane < 16 && ha * H < na && hb * H < nb;
      nsub += __popc(__ballot_sync(0xffffffffu, subok));
      if (subok) {
        const T dx = s.HA[0][ha] - s.HB[0][hb], dy = s.HA[1][ha] - s.HB[1][hb], dz = s.HA[2][ha] - s.HB[2][hb];
        const T lb = O::sqrt(dx * dx + dy * dy + dz * dz) - s.HA[3][ha] - s.HB[3][hb];
        subok = lb <= (pass1 ? bnd : th0) + Elb;
      }
      uint32_t m2 = __ballot_sync(0xffffffffu, subok);
      while (m2) {
        const int sidx = __ffs(m2) - 1;
        m2 &= m2 - 1;
        const int sa = ga * (G / H) + (sidx >> 2), sb = gb * (G / H) + (sidx & 3);
#pragma unroll 1
        for (int h = 0; h < 2; ++h) {
          const int a = sa * H + h * 4 + (lane >> 3);
          const int b = sb * H + (lane & 7);
          const bool valid = a < na && b < nb;
          T dx = T(0), dy = T(0), dz = T(0), ar = T(0), br = T(0);
          if (valid) {
            dx = s.SA[0][a] - s.SB[0][b];
            dy = s.SA[1][a] - s.SB[1][b];
            dz = s.SA[2][a] - s.SB[2][b];
            ar = s.SA[3][a];
            br = s.SB[3][b];
          }
          const T d2c = dx * dx + dy * dy + dz * dz;
          const T t0 = th0 + ar + br;
          bool cand;
          if (!pass1) {
            cand = valid && d2c <= t0 * t0;
          } else {
            // every centroid pair bounds the minimum distance from above
            const T rowmin = warp_min(valid ? d2c : O::inf());
            if (lane == 0) {
              const double ub = double(O::sqrt(rowmin)) + 2.0 * s.Elb + 2.0 * s.Ed + s.Eam;
              atomicMin(&s.bound, dbits(ub));
            }
            __syncwarp();
            const T bn = fmax(T(bitsd(*(volatile unsigned long long *)&s.bound)) + Elb, lift);
            const T t1 = bn + ar + br;
            cand = valid && d2c <= t1 * t1 && !(seen0 && d2c <= t0 * t0);
          }
          ntests += __popc(__ballot_sync(0xffffffffu, valid));
          const uint32_t m = __ballot_sync(0xffffffffu, cand);
          if (cand) s.wl[w][cnt + __popc(m & lanemask_lt())] = (uint32_t(a) << 16) | uint32_t(b);
          cnt += __popc(m);
          __syncwarp();
          if (cnt >= A.wflush) {
            warp_eval<DECIDE, ARGMIN, CONTACTS>(s.wl[w], cnt, ta, tb, pk, pass1);
            cnt = 0;
            __syncwarp();
          }
        }
      }
    }
    // the leftover lists of all warps, evaluated together in rounds of 32
    {
      uint32_t e0 = lane < cnt ? s.wl[w][lane] : 0u;
      uint32_t e1 = lane + 32 < cnt ? s.wl[w][lane + 32] : 0u;
      uint32_t e2 = lane + 64 < cnt ? s.wl[w][lane + 64] : 0u;
      if (lane == 0) s.wcnt[w] = cnt;
      __syncthreads();
      int start = 0, tot = 0;
#pragma unroll
      for (int q = 0; q < NW; ++q) {
        start = q == w ? tot : start;
        tot += s.wcnt[q];
      }
      uint32_t *flat = &s.wl[0][0];
      __syncthreads();
      if (lane < cnt) flat[start + lane] = e0;
      if (lane + 32 < cnt) flat[start + lane + 32] = e1;
      if (lane + 64 < cnt) flat[start + lane + 64] = e2;
      __syncthreads();
      for (int r = w; r * 32 < tot; r += NW) {
        if (DECIDE && !ARGMIN) {
          const int f = lane == 0 ? *(volatile int *)&s.found : 0;
          if (__shfl_sync(0xffffffffu, f, 0)) break;
        }
        warp_eval<DECIDE, ARGMIN, CONTACTS>(flat + r * 32, min(32, tot - r * 32), ta, tb, pk, pass1);
      }
    }
    if (PREC == 0 && qn) flush_queue<DECIDE, ARGMIN, CONTACTS>(ta, tb, pk);
    if (lane == 0) {
      stat(ST_SPHERE, ntests);
      stat(ST_GROUP, nsub);
    }
    __syncthreads();
  }

  // --- pose at t ------------------------------------------------------------
  // Poses at the pair's sample times t_q = ts + (T q) / K, q = 0..K, all
  // computed in one parallel pass (lane 2q: particle i, lane 2q+1: j).
  __device__ void pose_grid(int K) {
    const int ng = K + 1 <= GRID_MAX ? K + 1 : 0;
    if (w == 0 && lane < 2 * ng) {
      using D = OpsD;
      const int q = lane >> 1, side = lane & 1;
      const double tq = q == 0 ? s.ts : D::add(s.ts, D::div(D::mul(s.T_, double(q)), double(K)));
      pose_exact(A.st, A.n, side == 0 ? s.i : s.j, tq, s.rc, s.rs, s.gR[q][side], s.gX[q][side]);
    }
    if (tid == 0) s.ngrid = ng;
    __syncthreads();
  }

  // pose at t; kidx >= 0: t is sample time kidx of the pose grid
  __device__ void set_time(double t, int kidx = -1) {
    if (kidx >= 0 && kidx < s.ngrid) {
      if (tid < 24) {
        const int side = tid / 12, e = tid % 12;
        double *R = side == 0 ? s.RA : s.RB, *X = side == 0 ? s.XA : s.XB;
        if (e < 9)
          R[e] = s.gR[kidx][side][e];
        else
          X[e - 9] = s.gX[kidx][side][e - 9];
      }
    } else if (tid < 2) {
      // the two binary64 poses by lanes 0 and 1 of one warp (one FP64 pass)
      const int64_t p = tid == 0 ? s.i : s.j;
      pose_exact(A.st, A.n, p, t, s.rc, s.rs, tid == 0 ? s.RA : s.RB, tid == 0 ? s.XA : s.XB);
    }
    __syncthreads();
    if (w == 0) {
      // relative pose of B in A's frame in FP32 (its error is part of the
      // margin E): lane 3r+c computes Rr[r][c], lane 9+r computes tr[r]
      const int r = lane < 9 ? lane / 3 : (lane < 12 ? lane - 9 : 0), c = lane < 9 ? lane % 3 : 0;
      const float ra0 = float(s.RA[r]), ra1 = float(s.RA[3 + r]), ra2 = float(s.RA[6 + r]);
      float v;
      if (lane < 9)
        v = ra0 * float(s.RB[c]) + ra1 * float(s.RB[3 + c]) + ra2 * float(s.RB[6 + c]);
      else
        v = ra0 * float(s.XB[0] - s.XA[0]) + ra1 * float(s.XB[1] - s.XA[1]) + ra2 * float(s.XB[2] - s.XA[2]);
      if (lane < 9)
        s.Rr[lane] = v;
      else if (lane < 12)
        s.tr[lane - 9] = v;
      const float tr0 = __shfl_sync(0xffffffffu, v, 9), tr1 = __shfl_sync(0xffffffffu, v, 10),
                  tr2 = __shfl_sync(0xffffffffu, v, 11);
      if (lane == 0) {
        const float tr[3] = {tr0, tr1, tr2};
        const double ri = A.st[16 * A.n + s.i], rj = A.st[16 * A.n + s.j];
        if (PREC == 0) {
          const double S = ri + rj + sqrtf(tr[0] * tr[0] + tr[1] * tr[1] + tr[2] * tr[2]);
          s.Ed = S * ERR_REL32;
          s.Elb = s.Ed;
          s.Et = s.Ed;
          // the oracle's world vertices round relative to |X|, not S
          s.m64 = (S + sqrt(s.XA[0] * s.XA[0] + s.XA[1] * s.XA[1] + s.XA[2] * s.XA[2]) +
                   sqrt(s.XB[0] * s.XB[0] + s.XB[1] * s.XB[1] + s.XB[2] * s.XB[2])) *
                  ERR_REL64_LB;
          s.Eam = 2.0 * s.Ed;
          // FP32 A-frame data stay valid; B moves
          s.frmB = -1;
        } else {
          const double S = ri + rj + sqrt(s.XA[0] * s.XA[0] + s.XA[1] * s.XA[1] + s.XA[2] * s.XA[2]) +
                           sqrt(s.XB[0] * s.XB[0] + s.XB[1] * s.XB[1] + s.XB[2] * s.XB[2]);
          s.Ed = 0.0;
          s.Elb = S * ERR_REL64_LB;
          s.Et = s.Elb;
          s.m64 = 0.0;
          s.Eam = 0.0;
          s.frmA = -1;
          s.frmB = -1;
        }
        s.found = 0;
        s.nac = 0;
        s.bound = dbits(OpsD::inf());
      }
    }
    __syncthreads();
  }

  // --- one evaluation of the pair at time t ---------------------------------
  // DECIDE: returns whether some triangle pair is within eps (binary64).
  // ARGMIN: leaves the exact closest pair in s.best_*, FP32 minimum in s.mhat.
  // DECIDE and ARGMIN together: the decision, and the closest pair only when
  // the decision is true.
  // extra > 0: candidates up to eps + extra, all remembered in the interval
  // list (see decide_list).
  template <bool DECIDE, bool ARGMIN, bool CONTACTS>
  __device__ bool eval(double t, int64_t pk, int kidx = -1, double extra = 0.0) {
    set_time(t, kidx);
    mw = O::inf();
    bd2 = OpsD::inf();
    bkey = ~0ull;
    wbd2 = OpsD::inf();
    wbkey = ~0ull;
    qn = 0;
    bpa[0] = bpa[1] = bpa[2] = 0.0;
    bpb[0] = bpb[1] = bpb[2] = 0.0;
    const int nta = ntiles(s.nA), ntb = ntiles(s.nB);
    const T th0 = T(s.eps) + T(s.Elb) + T(extra);
    if (tid == 0) {
      // only a collecting evaluation starts a new list; the others (samples
      // after an overflow, the final argmin) leave the list and its overflow
      // flag as they are
      if (extra > 0.0) {
        s.nil = 0;
        s.ilover = 0;
        s.ilthr = PREC == 0 ? s.eps + extra + s.m64 : double(th0);
      }
      s.ilcol = extra > 0.0 ? 1 : 0;
    }
    __syncthreads();
    // Closest pair (with contacts and the interval list on the way) of two
    // single-tile meshes in the FP32 mode: one scan whose culling threshold is
    // the larger of th0 and the shrinking closest-pair bound, so every
    // triangle pair within th0 is evaluated once and the closest pair is
    // searched in the same traversal.  Large meshes (a floor) keep the two
    // passes, and so does the FP64 mode: the closest-pair bound starts loose
    // (tile and triangle-centroid distances), and a first pass at th0 often
    // settles the pair alone, which pays where every evaluation is binary64.
    if (PREC == 0 && !DECIDE && ARGMIN && nta == 1 && ntb == 1) {
      for (int attempt = 0;; ++attempt) {
        const bool ok = attempt == 0 ? argmin_pass<CONTACTS>(th0, nta, ntb, pk, true)
                                     : argmin_pass<false>(th0, nta, ntb, pk, true);
        if (!ok) return false;
        if (tid == 0) s.ilcol = 0;
        const double mh2 = block_min(double(mw));
        if (tid == 0) s.cull = fmax(bitsd(s.bound), double(th0));
        __syncthreads();
        if constexpr (PREC == 0) {
          argmin_list(mh2);
          if (s.redo && attempt < 2) {
            // the binary64 reference lies beyond the slack the candidates or
            // the culling used: search again, argmin alone, with a wider one
            __syncthreads();
            if (tid == 0) {
              s.Eam = attempt == 0 ? s.Eam * 1024.0 : OpsD::inf();
              s.nac = 0;
              s.redo = 0;
            }
            mw = O::inf();
            bd2 = OpsD::inf();
            bkey = ~0ull;
            wbd2 = OpsD::inf();
            wbkey = ~0ull;
            qn = 0;
            __syncthreads();
            continue;
          }
        }
        reduce_best();
        if (tid == 0) s.mhat = mh2;
        __syncthreads();
        return false;
      }
    }
    if (!pass0<DECIDE, ARGMIN, CONTACTS>(th0, nta, ntb, pk)) return false;
    if (tid == 0) s.ilcol = 0;
    if (DECIDE && ARGMIN) {
      const bool f = *(volatile int *)&s.found != 0;
      __syncthreads();
      if (!f) return false;
    }
    if (ARGMIN) {
      for (int attempt = 0;; ++attempt) {
        // FP32 (FP64) minimum over the evaluated pairs
        const double mh = block_min(double(mw));
        const double slack = s.Eam + s.Ed + s.Elb;
        const bool complete = mh + slack <= double(th0);
        if (!complete && nta > 0 && ntb > 0) {
          if (tid == 0) s.bound = dbits(mh + slack);  // inf if nothing seen
          __syncthreads();
          if (!argmin_pass<false>(th0, nta, ntb, pk, false)) return false;
        }
        const double mh2 = block_min(double(mw));
        if (tid == 0) s.cull = complete ? double(th0) : bitsd(s.bound);
        __syncthreads();
        if constexpr (PREC == 0) {
          argmin_list(mh2);
          if (s.redo && attempt < 2) {
            // the binary64 reference lies beyond the slack the candidates or
            // the culling used: search again, argmin alone, with a wider one
            __syncthreads();
            if (tid == 0) {
              s.Eam = attempt == 0 ? s.Eam * 1024.0 : OpsD::inf();
              s.nac = 0;
              s.redo = 0;
            }
            mw = O::inf();
            bd2 = OpsD::inf();
            bkey = ~0ull;
            wbd2 = OpsD::inf();
            wbkey = ~0ull;
            qn = 0;
            __syncthreads();
            if (!pass0<false, true, false>(th0, nta, ntb, pk)) return false;
            continue;
          }
        }
        reduce_best();
        if (tid == 0) {
          s.mhat = mh2;
          // FP32 mode: a decision with the closest pair is that pair's
          // binary64 distance within eps (the definition of f(t) <= eps)
          if (PREC == 0 && DECIDE) s.found = s.best_key != ~0ull && OpsD::sqrt(s.best_d2) <= s.eps;
        }
        __syncthreads();
        break;
      }
    }
    const bool f = DECIDE ? (*(volatile int *)&s.found != 0) : false;
    __syncthreads();
    return f;
  }

  // The closest-pair search over the tile pairs: the nearest tile pair first
  // (it tightens the bound), then the others in chunks tested in parallel
  // against the bound at the chunk's start; a selected tile pair is tested
  // again against the bound as it is when its turn comes.  After a first
  // pass (merged = false) s.bound holds its minimum plus the slack and tile
  // pairs that pass scanned skip the triangle pairs it evaluated; a merged
  // pass starts from an unbounded search and never culls below th0.  False
  // if a tile copy timed out.
  template <bool CONTACTS>
  __device__ bool argmin_pass(T th0, int nta, int ntb, int64_t pk, bool merged) {
    if (nta <= 0 || ntb <= 0) return true;
    const bool multi = nta > 1 || ntb > 1;
    const int nq = nta * ntb;
    if (merged) {
      if (tid == 0) s.bound = dbits(OpsD::inf());
      __syncthreads();
    }
    const double lift = merged ? double(th0) : -OpsD::inf();
    const int q0 = multi ? bound_by_tiles(nta, ntb) : 0;
    {
      const int ta = q0 / ntb, tb = q0 - (q0 / ntb) * ntb;
      // whether a first pass scanned this tile pair (the same test, same pose)
      const bool seen0 = !merged && (!multi || __syncthreads_or(tid == 0 && tile_near(ta, tb, double(th0))));
      if (!load_tiles(ta, tb)) return false;
      frames(ta, tb);
      if (tid == 0) stat(ST_TILES, 1);
      scan_tiles<false, true, CONTACTS>(ta, tb, true, th0, pk, seen0, merged);
    }
    for (int c0 = 0; multi && c0 < nq; c0 += NT) {
      const int q = c0 + tid;
      const bool near = q < nq && q != q0 &&
                        tile_near(q / ntb, q - (q / ntb) * ntb,
                                  fmax(bitsd(*(volatile unsigned long long *)&s.bound), lift));
      const uint32_t m = __ballot_sync(0xffffffffu, near);
      if (lane == 0) s.tmask[w] = m;
      __syncthreads();
      for (int wq = 0; wq < NW; ++wq) {
        uint32_t mm = s.tmask[wq];
        while (mm) {
          const int qq = c0 + wq * 32 + __ffs(mm) - 1;
          mm &= mm - 1;
          const int ta = qq / ntb, tb = qq - ta * ntb;
          if (!__syncthreads_or(tid == 0 && tile_near(ta, tb, fmax(bitsd(*(volatile unsigned long long *)&s.bound),
                                                                   lift))))
            continue;
          const bool seen0 = !merged && __syncthreads_or(tid == 0 && tile_near(ta, tb, double(th0)));
          if (!load_tiles(ta, tb)) return false;
          frames(ta, tb);
          if (tid == 0) stat(ST_TILES, 1);
          scan_tiles<false, true, CONTACTS>(ta, tb, true, th0, pk, seen0, merged);
        }
      }
      __syncthreads();
    }
    return true;
  }

  // The first pass of an evaluation: every tile pair whose tile bound is
  // within th0 (in chunks of NT tile pairs: every thread tests one, the warps
  // publish ballots, the CTA scans the near ones in order); a decision alone
  // stops at the first triangle pair within eps.  False if a tile copy timed
  // out.
  template <bool DECIDE, bool ARGMIN, bool CONTACTS>
  __device__ bool pass0(T th0, int nta, int ntb, int64_t pk) {
    bool stop = false;
    const bool multi = nta > 1 || ntb > 1;
    const int nq = nta * ntb;
    for (int c0 = 0; c0 < nq && !stop; c0 += NT) {
      const int q = c0 + tid;
      const bool near = q < nq && (!multi || tile_near(q / ntb, q - (q / ntb) * ntb, double(th0)));
      const uint32_t m = __ballot_sync(0xffffffffu, near);
      if (lane == 0) s.tmask[w] = m;
      __syncthreads();
      for (int wq = 0; wq < NW && !stop; ++wq) {
        uint32_t mm = s.tmask[wq];
        while (mm && !stop) {
          const int qq = c0 + wq * 32 + __ffs(mm) - 1;
          mm &= mm - 1;
          const int ta = qq / ntb, tb = qq - ta * ntb;
          if (!load_tiles(ta, tb)) return false;
          frames(ta, tb);
          if (tid == 0) stat(ST_TILES, 1);
          scan_tiles<DECIDE, ARGMIN, CONTACTS>(ta, tb, false, th0, pk);
          if (DECIDE && !ARGMIN && s.found) stop = true;
        }
      }
      __syncthreads();  // the next chunk rewrites s.tmask
    }
    return true;
  }

  // Closest pair (FP32 mode) among the collected candidates, each with its
  // certified lower bound L of the binary64 distance.  The candidate with the
  // smallest L is the reference: its binary64 distance dref bounds the
  // binary64 minimum from above, so only candidates with L <= dref + m64 can
  // attain it; they are sorted by (a, b) and recomputed in binary64, one per
  // warp per round, stopping after a round that found a zero (no later key
  // can win then).  A reference beyond the slack the candidates were
  // collected with, or beyond the culling threshold, sets s.redo: a pair that
  // was not collected or not evaluated could then attain the minimum.
  __device__ void argmin_list(double mh) {
    const int n0 = min(s.nac, ACAP);
    if (w == 0) {
      float bl = OpsF::inf();
      unsigned long long bk = ~0ull;
      for (int q = lane; q < n0; q += 32) {
        const unsigned long long key = s.ac_key[q];
        const float L = s.ac_d[q];
        if (key != ~0ull && (L < bl || (L == bl && key < bk))) {
          bl = L;
          bk = key;
        }
      }
#pragma unroll
      for (int o = 16; o; o >>= 1) {
        const float ol = __shfl_xor_sync(0xffffffffu, bl, o);
        const unsigned long long ok = __shfl_xor_sync(0xffffffffu, bk, o);
        if (ol < bl || (ol == bl && ok < bk)) {
          bl = ol;
          bk = ok;
        }
      }
      if (lane == 0) {
        s.ref_key = bk;
        s.red_d[0] = double(bl);
      }
    }
    __syncthreads();
    const unsigned long long rk = s.ref_key;
    unsigned long long n64 = 0;
    double dref = OpsD::inf();
    if (rk != ~0ull) {
      if (w == 0) {
        V3<double> qa, qb;
        const double e2 = exact_warp(int(rk >> 32), int(rk & 0xffffffffu), qa, qb, !(s.red_d[0] > s.m64));
        update_best(e2, rk, qa, qb);
        ++n64;
        if (lane == 0) s.red_d[1] = OpsD::sqrt(e2);
      }
      __syncthreads();
      dref = s.red_d[1];
      if (tid == 0) s.redo = (dref + s.m64 > mh + s.Eam) || (dref + s.m64 > s.cull);
    } else if (tid == 0) {
      s.redo = 0;
    }
    __syncthreads();
    if (s.redo) return;
    // candidates that can attain the binary64 minimum (a zero reference: only
    // smaller keys), compacted by warp 0; their smallest certificate decides
    // whether the crossing tests can be skipped
    if (w == 0) {
      int m = 0;
      float lmin = OpsF::inf();
      for (int q0 = 0; q0 < n0; q0 += 32) {
        const int q = q0 + lane;
        const unsigned long long key = q < n0 ? s.ac_key[q] : ~0ull;
        const bool keep = key != ~0ull && key != rk && double(s.ac_d[q]) <= dref + s.m64 && (dref > 0.0 || key < rk);
        const uint32_t mk = __ballot_sync(0xffffffffu, keep);
        if (keep) lmin = fminf(lmin, s.ac_d[q]);
        __syncwarp();
        if (keep) s.ac_key[m + __popc(mk & lanemask_lt())] = key;
        m += __popc(mk);
        __syncwarp();
      }
      lmin = warp_min(lmin);
      if (lane == 0) {
        s.nac = m;
        s.red_d[2] = double(lmin);
      }
    }
    __syncthreads();
    const int n = s.nac;
    const bool cross = !(s.red_d[2] > s.m64);
    int n2 = 1;
    while (n2 < n) n2 <<= 1;
    if (n2 <= 32) {
      if (w == 0) {
        // one candidate per lane, bitonic sort in registers
        unsigned long long key = lane < n ? s.ac_key[lane] : ~0ull;
        for (int k = 2; k <= 32; k <<= 1)
          for (int j = k >> 1; j > 0; j >>= 1) {
            const unsigned long long o = __shfl_xor_sync(0xffffffffu, key, j);
            const bool lower = (lane & j) == 0, up = (lane & k) == 0;
            key = (lower == up) ? (key < o ? key : o) : (key > o ? key : o);
          }
        if (lane < n) s.ac_key[lane] = key;
      }
      __syncthreads();
    } else {
      for (int q = n + tid; q < n2; q += NT) s.ac_key[q] = ~0ull;
      __syncthreads();
      for (int k = 2; k <= n2; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
          for (int q = tid; q < n2; q += NT) {
            const int l = q ^ j;
            if (l > q) {
              const bool up = (q & k) == 0;
              const unsigned long long kq = s.ac_key[q], kl = s.ac_key[l];
              if ((kq > kl) == up) {
                s.ac_key[q] = kl;
                s.ac_key[l] = kq;
              }
            }
          }
          __syncthreads();
        }
    }
    for (int r0 = 0; r0 < n; r0 += NW) {
      const int q = r0 + w;
      const unsigned long long key = q < n ? s.ac_key[q] : ~0ull;
      double e2 = OpsD::inf();
      if (key != ~0ull) {
        V3<double> qa, qb;
        e2 = exact_warp(int(key >> 32), int(key & 0xffffffffu), qa, qb, cross);
        update_best(e2, key, qa, qb);
        ++n64;
      }
      // stop after a round that found a zero distance
      if (__syncthreads_or(key != ~0ull && e2 == 0.0)) break;
    }
    if (lane == 0) stat(ST_FP64, n64);
    __syncthreads();
  }

  // Decision f(t) <= eps on the pair-interval list: every triangle pair that
  // can come within eps anywhere in [ts, ts + T] is on it (its sphere bound
  // at ts was within eps + delta, delta bounding how much any distance can
  // change over the interval), so the list decides exactly like the full scan.
  __device__ bool decide_list(double t, int kidx) {
    set_time(t, kidx);
    const int n = il_count();
    const T eps = T(s.eps), Ed = T(s.Ed);
    bool yes_any = false;
    unsigned long long n32 = 0, n64 = 0;
    for (int r0 = w * 32; r0 < n; r0 += NT) {
      const int k = r0 + lane;
      const bool have = k < n;
      const unsigned long long ent = have ? il_entry(k) : 0ull;
      const int ag = int((ent >> 24) & 0xffffffu), bg = int(ent & 0xffffffu);
      T d = O::inf();
      double L = -OpsD::inf();
      int feat = 0;
      if (have) {
        V X[3], Y[3];
        // FP32: B's triangle in its tile's local frame (a particle of several
        // tiles), with that tile's margin; else B's body frame and the pair's
        float o[3] = {0.f, 0.f, 0.f}, to[3] = {s.tr[0], s.tr[1], s.tr[2]};
        double Eloc = s.Ed;
        if constexpr (PREC == 0) {
          const int64_t slot = s.offB / TT + s.j + bg / TT;
          if (s.nB > TT && slot < A.cap_tiles) {
            const float4 f = A.tile_sph[slot];
            o[0] = f.x;
            o[1] = f.y;
            o[2] = f.z;
            double t[3];
            local_origin(o, t);
            to[0] = float(t[0]);
            to[1] = float(t[1]);
            to[2] = float(t[2]);
            Eloc = ERR_REL32 * (A.st[16 * A.n + s.i] + double(f.w) + sqrt(t[0] * t[0] + t[1] * t[1] + t[2] * t[2]));
          }
        }
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          const float4 f = A.tris[q * A.n_tris + s.offA + ag];
          const float4 g = A.tris[q * A.n_tris + s.offB + bg];
          if constexpr (PREC == 0) {
            X[q] = V{f.x, f.y, f.z};
            const float *R = s.Rr;
            const float bx = g.x - o[0], by = g.y - o[1], bz = g.z - o[2];
            Y[q] = V{fmaf(R[0], bx, fmaf(R[1], by, fmaf(R[2], bz, to[0]))),
                     fmaf(R[3], bx, fmaf(R[4], by, fmaf(R[5], bz, to[1]))),
                     fmaf(R[6], bx, fmaf(R[7], by, fmaf(R[8], bz, to[2])))};
          } else {
            const V3<double> x = to_world_exact(s.RA, s.XA, f.x, f.y, f.z);
            const V3<double> y = to_world_exact(s.RB, s.XB, g.x, g.y, g.z);
            X[q] = V{T(x.x), T(x.y), T(x.z)};
            Y[q] = V{T(y.x), T(y.y), T(y.z)};
          }
        }
        V pa, pb;
        T d2;
        if constexpr (PREC == 0) {
          // features only: crossing triangles have no separating direction,
          // so their certificate never clears them
          d2 = GT::tri_dist2_features(X, Y, pa, pb, feat);
          L = certificate(X, Y, pa, pb, Eloc);
        } else {
          d2 = GT::tri_dist2_features(X, Y, pa, pb);
          if (!(O::sqrt(d2) <= eps)) {
            V x;
            bool hit = false;
            for (int q = 0; q < 3 && !hit; ++q)
              hit = GT::seg_tri_cross(X[q], X[q == 2 ? 0 : q + 1], Y[0], Y[1], Y[2], x);
            for (int q = 0; q < 3 && !hit; ++q)
              hit = GT::seg_tri_cross(Y[q], Y[q == 2 ? 0 : q + 1], X[0], X[1], X[2], x);
            if (hit) d2 = T(0);
          }
        }
        d = O::sqrt(d2);
        ++n32;
      }
      bool yes = have && PREC == 1 && d <= eps;
      bool apart = !have;
      if constexpr (PREC == 0) {
        // certified apart, or in contact by the binary64 value of the
        // closest FP32 feature; the rest in binary64 in full below
        apart = !have || L > s.eps + s.m64;
        // the lane with the smallest FP32 distance among those within eps
        const bool cand = have && !apart && d < eps;
        const T dm = warp_min(cand ? d : O::inf());
        const uint32_t pm = __ballot_sync(0xffffffffu, cand && d == dm);
        if (pm) {
          const bool pick = lane == __ffs(pm) - 1;
          V3<double> qa, qb;
          double e2 = OpsD::inf();
          if (pick) {
            e2 = feature64(feat, ag, bg, qa, qb);
            ++n64;
          }
          yes = pick && OpsD::sqrt(e2) <= s.eps;
        }
      }
      if (__any_sync(0xffffffffu, yes)) {
        yes_any = true;
        break;
      }
      if constexpr (PREC == 0) {
        // not settled: binary64, one triangle pair per warp
        uint32_t bm = __ballot_sync(0xffffffffu, have && !apart);
        while (bm && !yes_any) {
          const int src = __ffs(bm) - 1;
          bm &= bm - 1;
          V3<double> qa, qb;
          const double e2 = exact_warp(__shfl_sync(0xffffffffu, ag, src), __shfl_sync(0xffffffffu, bg, src), qa, qb,
                                       true);
          ++n64;
          // lane 0's value: the loop condition stays warp-uniform whatever e2 is
          if (__shfl_sync(0xffffffffu, OpsD::sqrt(e2) <= s.eps ? 1 : 0, 0)) yes_any = true;
        }
        if (yes_any) break;
      }
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) n32 += __shfl_xor_sync(0xffffffffu, n32, o);
    if (lane == 0) {
      stat(ST_FP32, n32);
      stat(ST_FP64, n64);
    }
    return __syncthreads_or(yes_any) != 0;
  }

  __device__ double block_min(double v) {
    v = warp_min(v);
    __syncthreads();
    if (lane == 0) s.red_d[w] = v;
    __syncthreads();
    double r = s.red_d[0];
#pragma unroll
    for (int q = 1; q < NW; ++q) r = fmin(r, s.red_d[q]);
    __syncthreads();
    return r;
  }

  // block-wide smallest (d^2, key) and its points into s.best_*
  __device__ void reduce_best() {
    double d = bd2;
    unsigned long long k = bkey;
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      const double od = __shfl_xor_sync(0xffffffffu, d, o);
      const unsigned long long ok = __shfl_xor_sync(0xffffffffu, k, o);
      if (od < d || (od == d && ok < k)) {
        d = od;
        k = ok;
      }
    }
    __syncthreads();
    if (lane == 0) {
      s.red_d[w] = d;
      s.red_k[w] = k;
    }
    __syncthreads();
    if (tid == 0) {
      double bd = s.red_d[0];
      unsigned long long bk = s.red_k[0];
      for (int q = 1; q < NW; ++q)
        if (s.red_d[q] < bd || (s.red_d[q] == bd && s.red_k[q] < bk)) {
          bd = s.red_d[q];
          bk = s.red_k[q];
        }
      s.best_d2 = bd;
      s.best_key = bk;
      for (int q = 0; q < 3; ++q) s.best_pa[q] = s.best_pb[q] = 0.0;
    }
    __syncthreads();
    if (bkey != ~0ull && bkey == s.best_key && bd2 == s.best_d2) {
      for (int q = 0; q < 3; ++q) {
        s.best_pa[q] = bpa[q];
        s.best_pb[q] = bpb[q];
      }
    }
    __syncthreads();
  }

  // --- the paper's narrowing (second collision-time procedure) ------------
  // Poses of the narrowing: gR/gX slot 0 = ts, 1 = span end te, 2 = middle.
  using VD = V3<double>;
  // body-frame position R^T (W - X), rows summed left to right
  static __device__ __forceinline__ VD rel_pos(const double *R, const double *X, VD W) {
    using O = OpsD;
    const VD d = GD::sub(W, VD{X[0], X[1], X[2]});
    return VD{O::add(O::add(O::mul(R[0], d.x), O::mul(R[3], d.y)), O::mul(R[6], d.z)),
              O::add(O::add(O::mul(R[1], d.x), O::mul(R[4], d.y)), O::mul(R[7], d.z)),
              O::add(O::add(O::mul(R[2], d.x), O::mul(R[5], d.y)), O::mul(R[8], d.z))};
  }
  // earliest vertex-triangle candidate: the vertex (world W0 at ts, W1 at te)
  // on its straight path in the triangle particle's frame; the end point and
  // the plane crossing (heights h = n . (P - a), n = (b - a) x (c - a))
  static __device__ double vt_candidate(VD W0, VD W1, const double *R0, const double *X0, const double *R1,
                                        const double *X1, const VD *Tr, double eps, double ts, double te) {
    using O = OpsD;
    const VD P0 = rel_pos(R0, X0, W0), P1 = rel_pos(R1, X1, W1);
    VD q;
    double best = O::inf();
    if (O::sqrt(GD::closest_pt_tri(P1, Tr[0], Tr[1], Tr[2], q)) <= eps) best = te;
    const VD nrm = GD::cross(GD::sub(Tr[1], Tr[0]), GD::sub(Tr[2], Tr[0]));
    const double h0 = GD::dot(nrm, GD::sub(P0, Tr[0])), h1 = GD::dot(nrm, GD::sub(P1, Tr[0]));
    if ((h0 > 0.0 && h1 < 0.0) || (h0 < 0.0 && h1 > 0.0)) {
      const double sx = O::div(h0, O::sub(h0, h1));
      const VD Ps = GD::axpy(P0, GD::sub(P1, P0), sx);
      const double t = O::add(ts, O::mul(sx, O::sub(te, ts)));
      if (O::sqrt(GD::closest_pt_tri(Ps, Tr[0], Tr[1], Tr[2], q)) <= eps && t < best) best = t;
    }
    return best;
  }
  // earliest candidate of triangle pair (a, b) over [ts, te] (binary64)
  __device__ __noinline__ double narrow_pair(int a, int b, double ts, double te, double tm) const {
    using O = OpsD;
    VD BA[3], BB[3], WA0[3], WA1[3], WAm[3], WB0[3], WB1[3], WBm[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      const float4 f = A.tris[q * A.n_tris + s.offA + a], g = A.tris[q * A.n_tris + s.offB + b];
      BA[q] = VD{f.x, f.y, f.z};
      BB[q] = VD{g.x, g.y, g.z};
      WA0[q] = to_world_exact(s.gR[0][0], s.gX[0][0], f.x, f.y, f.z);
      WA1[q] = to_world_exact(s.gR[1][0], s.gX[1][0], f.x, f.y, f.z);
      WAm[q] = to_world_exact(s.gR[2][0], s.gX[2][0], f.x, f.y, f.z);
      WB0[q] = to_world_exact(s.gR[0][1], s.gX[0][1], g.x, g.y, g.z);
      WB1[q] = to_world_exact(s.gR[1][1], s.gX[1][1], g.x, g.y, g.z);
      WBm[q] = to_world_exact(s.gR[2][1], s.gX[2][1], g.x, g.y, g.z);
    }
    const double eps = s.eps;
    double tab = O::inf();
    for (int q = 0; q < 3; ++q)
      tab = fmin(tab, vt_candidate(WA0[q], WA1[q], s.gR[0][1], s.gX[0][1], s.gR[1][1], s.gX[1][1], BB, eps, ts, te));
    for (int q = 0; q < 3; ++q)
      tab = fmin(tab, vt_candidate(WB0[q], WB1[q], s.gR[0][0], s.gX[0][0], s.gR[1][0], s.gX[1][0], BA, eps, ts, te));
    for (int p = 0; p < 3; ++p)
      for (int q = 0; q < 3; ++q) {
        const int p1 = p == 2 ? 0 : p + 1, q1 = q == 2 ? 0 : q + 1;
        VD c1, c2;
        if (tm < tab && O::sqrt(GD::seg_seg(WAm[p], WAm[p1], WBm[q], WBm[q1], c1, c2)) <= eps) tab = tm;
        if (te < tab && O::sqrt(GD::seg_seg(WA1[p], WA1[p1], WB1[q], WB1[q1], c1, c2)) <= eps) tab = te;
      }
    return tab;
  }
  // Lower bound on the distance at ts of triangles a (particle i) and b
  // (particle j) from their bounding spheres (centroid, largest vertex
  // distance) in A's frame, B's centre moved by the FP32 relative pose at ts
  // (Rr, tr).  The FP32 errors of the pose, the centres and the radii are
  // below 2^-20 S; the margin mg = 2^-14 S covers them many times over.
  __device__ double tri_sphere_gap(int a, int b, float mg) const {
    float c[2][3], r[2];
#pragma unroll
    for (int side = 0; side < 2; ++side) {
      const int64_t o = side == 0 ? s.offA + a : s.offB + b;
      const float4 v0 = A.tris[o], v1 = A.tris[A.n_tris + o], v2 = A.tris[2 * A.n_tris + o];
      const float cx = (v0.x + v1.x + v2.x) * (1.0f / 3.0f), cy = (v0.y + v1.y + v2.y) * (1.0f / 3.0f),
                  cz = (v0.z + v1.z + v2.z) * (1.0f / 3.0f);
      const float e0 = (v0.x - cx) * (v0.x - cx) + (v0.y - cy) * (v0.y - cy) + (v0.z - cz) * (v0.z - cz);
      const float e1 = (v1.x - cx) * (v1.x - cx) + (v1.y - cy) * (v1.y - cy) + (v1.z - cz) * (v1.z - cz);
      const float e2 = (v2.x - cx) * (v2.x - cx) + (v2.y - cy) * (v2.y - cy) + (v2.z - cz) * (v2.z - cz);
      r[side] = sqrtf(fmaxf(e0, fmaxf(e1, e2)));
      if (side == 0) {
        c[0][0] = cx;
        c[0][1] = cy;
        c[0][2] = cz;
      } else {
        const float *R = s.Rr;
        c[1][0] = fmaf(R[0], cx, fmaf(R[1], cy, fmaf(R[2], cz, s.tr[0])));
        c[1][1] = fmaf(R[3], cx, fmaf(R[4], cy, fmaf(R[5], cz, s.tr[1])));
        c[1][2] = fmaf(R[6], cx, fmaf(R[7], cy, fmaf(R[8], cz, s.tr[2])));
      }
    }
    const float dx = c[0][0] - c[1][0], dy = c[0][1] - c[1][1], dz = c[0][2] - c[1][2];
    return double(sqrtf(dx * dx + dy * dy + dz * dz)) - double(r[0]) - double(r[1]) - double(mg);
  }
  // Certified lower bound of the binary64 distance of triangles a, b at ts
  // (A's frame, B moved by the FP32 relative pose, as in the tile scan): the
  // same lower bound the pair-interval list keeps.
  __device__ double tri_dist32_lb(int a, int b) const {
    using GF = Geo<OpsF>;
    V3<float> X[3], Y[3];
    const float *R = s.Rr;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      const float4 f = A.tris[q * A.n_tris + s.offA + a], g = A.tris[q * A.n_tris + s.offB + b];
      X[q] = V3<float>{f.x, f.y, f.z};
      Y[q] = V3<float>{fmaf(R[0], g.x, fmaf(R[1], g.y, fmaf(R[2], g.z, s.tr[0]))),
                       fmaf(R[3], g.x, fmaf(R[4], g.y, fmaf(R[5], g.z, s.tr[1]))),
                       fmaf(R[6], g.x, fmaf(R[7], g.y, fmaf(R[8], g.z, s.tr[2])))};
    }
    V3<float> pa, pb;
    GF::tri_dist2_features(X, Y, pa, pb);
    return certificate(X, Y, pa, pb, s.Ed);
  }
  // The narrowing loop after a false decision at ts.  The triangle pairs are
  // those of the pair-interval list collected at ts with the narrowing's
  // motion bound (all pairs if the list overflowed).  Returns the status and
  // sets tc, ta, tb and the number of iterations.
  __device__ uint8_t narrowing(int &iters, double &tc, int32_t &ta, int32_t &tb) {
    using O = OpsD;
    if (tid < 24) {  // keep the poses at ts (slot 0)
      const int side = tid / 12, e = tid % 12;
      if (e < 9)
        s.gR[0][side][e] = side == 0 ? s.RA[e] : s.RB[e];
      else
        s.gX[0][side][e - 9] = side == 0 ? s.XA[e - 9] : s.XB[e - 9];
    }
    const double ts = s.ts, T = s.T_, wid = O::mul(A.tol, T);  // widening
    double te = O::add(ts, T);
    bool found = false;
    iters = 0;
    // Visit the listed triangle pairs nearest first: a pair whose distance
    // at ts is d cannot meet (distance <= eps) before ts + (d - eps) / rate,
    // rate = the motion bound per unit time; once that exceeds the earliest
    // candidate time found so far (shared, atomic), the pair is skipped --
    // the paper's unfolding constrained by a global contact time.
    const bool useL0 = s.ilover == 0;
    if (useL0) {
      // the shared-memory part is sorted; a spilled part is visited unsorted
      const int n = s.nil < ILCAP ? s.nil : ILCAP;
      int n2 = 1;
      while (n2 < n) n2 <<= 1;
      for (int q = n + tid; q < n2; q += NT) s.il[q] = ~0ull;
      __syncthreads();
      for (int k = 2; k <= n2; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
          for (int q = tid; q < n2; q += NT) {
            const int l = q ^ j;
            if (l > q) {
              const bool up = (q & k) == 0;
              const unsigned long long kq = s.il[q], kl = s.il[l];
              if ((kq > kl) == up) {
                s.il[q] = kl;
                s.il[l] = kq;
              }
            }
          }
          __syncthreads();
        }
    }
    const double rate = s.delta / T;
    // after an overflow every triangle pair is visited, each first bounded by
    // its bounding spheres at ts (the same rate argument as for the list)
    const float mg = float(8.0 * ERR_REL32 *
                           (A.st[16 * A.n + s.i] + A.st[16 * A.n + s.j] +
                            double(sqrtf(s.tr[0] * s.tr[0] + s.tr[1] * s.tr[1] + s.tr[2] * s.tr[2]))));
    for (;;) {
      const double tm = O::add(ts, O::mul(0.5, O::sub(te, ts)));
      __syncthreads();
      if (tid < 4) {
        const int side = tid & 1, which = tid >> 1;
        pose_exact(A.st, A.n, side ? s.j : s.i, which ? tm : te, s.rc, s.rs, s.gR[1 + which][side],
                   s.gX[1 + which][side]);
      }
      __syncthreads();
      const bool useL = useL0;
      const int64_t cnt = useL ? (int64_t)il_count() : (int64_t)s.nA * s.nB;
      if (tid == 0) s.bound = okey(O::inf());  // earliest candidate time so far
      __syncthreads();
      double best = O::inf();
      unsigned long long bk = ~0ull, evaluated = 0;
      for (int64_t q = tid; q < cnt; q += NT) {
        int a, b;
        if (useL) {
          const unsigned long long ent = il_entry(int(q));
          a = int((ent >> 24) & 0xffffffu);
          b = int(ent & 0xffffffu);
          const double dlb = double(__uint_as_float(uint32_t(ent >> 48) << 16));
          const double tlb = dlb > s.eps ? ts + (dlb - s.eps) / rate * (1.0 - 1e-9) : -O::inf();
          if (tlb > okey_value(*(volatile unsigned long long *)&s.bound)) {
            // sorted by distance in shared memory: this thread's later shared
            // entries cannot be earlier; go on with its spilled ones
            if (q < ILCAP) q = tid + (int64_t)((ILCAP - tid + NT - 1) / NT) * NT - NT;
            continue;
          }
        } else {
          a = int(q / s.nB);
          b = int(q - (int64_t)a * s.nB);
          // every candidate of the pair lies in [ts, te]; none can precede the
          // earliest time its spheres allow, nor (FP32 mode) the earliest
          // time its FP32 distance allows
          const double thr = fmin(te, okey_value(*(volatile unsigned long long *)&s.bound));
          const double dlb = tri_sphere_gap(a, b, mg);
          if (dlb > s.eps && ts + (dlb - s.eps) / rate * (1.0 - 1e-9) > thr) continue;
          if constexpr (PREC == 0) {
            const double d32 = tri_dist32_lb(a, b);
            if (d32 > s.eps && ts + (d32 - s.eps) / rate * (1.0 - 1e-9) > thr) continue;
          }
        }
        const double t = narrow_pair(a, b, ts, te, tm);
        ++evaluated;
        if (t < O::inf()) atomicMin(&s.bound, okey(t));
        const unsigned long long key = (static_cast<unsigned long long>(a) << 32) | static_cast<uint32_t>(b);
        if (t < best || (t == best && key < bk)) {
          best = t;
          bk = key;
        }
      }
      stat(ST_FP64, evaluated);
      // block minimum of (time, key)
#pragma unroll
      for (int o = 16; o; o >>= 1) {
        const double ob = __shfl_xor_sync(0xffffffffu, best, o);
        const unsigned long long ok = __shfl_xor_sync(0xffffffffu, bk, o);
        if (ob < best || (ob == best && ok < bk)) {
          best = ob;
          bk = ok;
        }
      }
      __syncthreads();
      if (lane == 0) {
        s.red_d[w] = best;
        s.red_k[w] = bk;
      }
      __syncthreads();
      best = s.red_d[0];
      bk = s.red_k[0];
      for (int q = 1; q < NW; ++q)
        if (s.red_d[q] < best || (s.red_d[q] == best && s.red_k[q] < bk)) {
          best = s.red_d[q];
          bk = s.red_k[q];
        }
      ++iters;
      if (!(best < O::inf())) break;
      found = true;
      ta = int32_t(bk >> 32);
      tb = int32_t(bk & 0xffffffffu);
      if (!(best < O::sub(te, wid)) || iters >= NARROW_MAX_ITER) break;
      te = O::add(best, wid);
    }
    __syncthreads();
    if (!found) {
      ta = tb = -1;
      tc = O::add(ts, T);
      return 0;
    }
    tc = te;
    return 2;
  }

  // --- per pair setup --------------------------------------------------------
  __device__ bool setup_pair(int64_t k) {
    if (tid == 0) {
      const int64_t i = A.pairs[2 * k], j = A.pairs[2 * k + 1];
      s.bad = 0;
      if (i < 0 || j < 0 || i >= A.n || j >= A.n) {
        set_err(A.err, ERR_INDEX);
        s.bad = 1;
        s.i = s.j = 0;
        s.nA = s.nB = 0;
      } else {
        s.i = i;
        s.j = j;
        s.offA = A.tri_off[i];
        s.offB = A.tri_off[j];
        const int64_t nA = A.tri_off[i + 1] - s.offA, nB = A.tri_off[j + 1] - s.offB;
        if (nA < 0 || nB < 0 || s.offA < 0 || s.offB < 0 || s.offA + nA > A.n_tris ||
            s.offB + nB > A.n_tris || nA >= (1 << 24) || nB >= (1 << 24)) {
          set_err(A.err, ERR_INDEX);
          s.bad = 1;
          s.nA = s.nB = 0;
        } else {
          s.nA = int(nA);
          s.nB = int(nB);
        }
      }
      const double *st = A.st;
      const int64_t n = A.n;
      if (!s.bad) {
        bool fin = true;
        for (int f = 0; f < DEM_NFIELDS; ++f) fin = fin && isfinite(st[f * n + s.i]) && isfinite(st[f * n + s.j]);
        if (!fin) {  // skip the pair: its outputs are those of a pair without triangles
          set_err(A.err, ERR_NONFINITE);
          s.bad = 1;
          s.nA = s.nB = 0;
        }
      }
      s.eps = OpsD::add(st[15 * n + s.i], st[15 * n + s.j]);
      const double ti = st[13 * n + s.i], tj = st[13 * n + s.j];
      const double di = st[14 * n + s.i], dj = st[14 * n + s.j];
      // a static member has no step of its own: the moving member's interval
      const bool si = A.is_static && A.is_static[s.i], sj = A.is_static && A.is_static[s.j];
      if (sj && !si) {
        s.ts = ti;
        s.T_ = di;
      } else if (si && !sj) {
        s.ts = tj;
        s.T_ = dj;
      } else {
        s.ts = ti < tj ? ti : tj;
        s.T_ = di < dj ? di : dj;
      }
      s.resA = s.resB = -1;
      s.frmA = s.frmB = -1;
    }
    __syncthreads();
    return !s.bad;
  }
};

__device__ __forceinline__ int64_t pair_count(const PairArgs &A) {
  int64_t m = A.max_pairs;
  if (A.n_pairs) {
    const int64_t c = *A.n_pairs;
    m = c < m ? c : m;
  }
  return m < 0 ? 0 : m;
}

template <int PREC, int MODE>
__global__ void __launch_bounds__(Cfg<PREC>::NT, Cfg<PREC>::MINB) pair_kernel(PairArgs A) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  Smem<PREC> &s = *reinterpret_cast<Smem<PREC> *>(smem_raw);
  Cta<PREC> c(s, A);
  unsigned long long t_begin = 0;
  if (c.tid == 0) asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t_begin));
  if (c.tid < ST_N) s.cnt[c.tid] = 0;
  if (c.tid == 0) {
    mbar_init(&s.mbar);
    s.abort = 0;
    pose_reciprocals(s.rc, s.rs);
  }
  __syncthreads();
  const int64_t m = pair_count(A);
  for (;;) {
    if (c.tid == 0) {
      const unsigned int q = atomicAdd(A.work, 1u);
      // the q-th pair handed out: in the given order (costliest first), else q
      int64_t k = q;
      if (A.order && (int64_t)q < m) {
        k = A.order[q];
        if (k < 0 || k >= m) {  // not a permutation of the pairs: report and stop
          set_err(A.err, ERR_INDEX);
          k = m;
        }
      }
      s.work_item = (unsigned int)((int64_t)q >= m ? m : k);
    }
    __syncthreads();
    const int64_t k = s.work_item;
    const bool quit = s.abort != 0;
    __syncthreads();
    if (k >= m || quit) break;
    const bool ok = c.setup_pair(k);
    const double chk = double(s.nA) * double(s.nB);
    using D = OpsD;
    // narrow-phase outputs of pair k from the closest pair in s.best_*
    auto write_narrow = [&]() {
      if (c.tid == 0) {
        const bool have = ok && s.best_key != ~0ull && s.nA > 0 && s.nB > 0;
        const double d = have ? OpsD::sqrt(s.best_d2) : OpsD::inf();
        A.dmin[k] = d;
        for (int q = 0; q < 3; ++q) {
          A.pa[3 * k + q] = have ? s.best_pa[q] : 0.0;
          A.pb[3 * k + q] = have ? s.best_pb[q] : 0.0;
        }
        A.tri_ab[2 * k] = have ? int32_t(s.best_key >> 32) : -1;
        A.tri_ab[2 * k + 1] = have ? int32_t(s.best_key & 0xffffffffu) : -1;
        A.flag[k] = uint8_t(have && d <= s.eps);
        if (A.dmin32) A.dmin32[k] = have ? float(s.mhat) : __int_as_float(0x7f800000);
      }
    };
    // bound on the change of any triangle-pair distance over [ts, ts+T]:
    // each vertex moves at most (|v| + |w| R) per unit time
    auto motion_bound = [&]() {
      if (c.tid == 0) {
        const double *st = A.st;
        const int64_t n = A.n;
        double m = 0.0;
        for (int side = 0; side < 2; ++side) {
          const int64_t p = side == 0 ? s.i : s.j;
          const double v = sqrt(st[3 * n + p] * st[3 * n + p] + st[4 * n + p] * st[4 * n + p] +
                                st[5 * n + p] * st[5 * n + p]);
          const double om = sqrt(st[10 * n + p] * st[10 * n + p] + st[11 * n + p] * st[11 * n + p] +
                                 st[12 * n + p] * st[12 * n + p]);
          m += v + om * st[16 * n + p];
        }
        s.delta = m * s.T_ * (1.0 + 1e-9) + 1e-300;
      }
      __syncthreads();
    };
    // Motion bound of the narrowing: how far a vertex can move in the other
    // particle's frame, or any feature distance change, over the interval:
    // (|v_i| + |v_j| + |w_i| R_i + |w_j| R_j
    //  + (|w_i| + |w_j|) (R_i + R_j + D0 + (|v_i| + |v_j|) T)) T,
    // D0 bounding the centre distance at ts (the frame's rotation moves a
    // point at distance r from its centre by |w| r per time).
    auto motion_bound_narrowing = [&]() {
      if (c.tid == 0) {
        const double *st = A.st;
        const int64_t n = A.n;
        double vs = 0.0, wr = 0.0, ws = 0.0, rs = 0.0, back = 0.0;
        for (int side = 0; side < 2; ++side) {
          const int64_t p = side == 0 ? s.i : s.j;
          const double v = sqrt(st[3 * n + p] * st[3 * n + p] + st[4 * n + p] * st[4 * n + p] +
                                st[5 * n + p] * st[5 * n + p]);
          const double om = sqrt(st[10 * n + p] * st[10 * n + p] + st[11 * n + p] * st[11 * n + p] +
                                 st[12 * n + p] * st[12 * n + p]);
          vs += v;
          ws += om;
          wr += om * st[16 * n + p];
          rs += st[16 * n + p];
          back += v * fabs(s.ts - st[13 * n + p]);
        }
        const double dx = st[0 * n + s.i] - st[0 * n + s.j], dy = st[1 * n + s.i] - st[1 * n + s.j],
                     dz = st[2 * n + s.i] - st[2 * n + s.j];
        const double D0 = sqrt(dx * dx + dy * dy + dz * dz) + back;
        s.delta = (vs + wr + ws * (rs + D0 + vs * s.T_)) * s.T_ * (1.0 + 1e-9) + 1e-300;
      }
      __syncthreads();
    };
    // the K samples and the bisection after a false decision at ts
    // (binary64, operations in the order of the definition, each rounded on
    // its own); returns the status and sets tc / ta / tb
    auto search = [&](int &evals, int &bis, double &tc, int32_t &ta, int32_t &tb) -> uint8_t {
      const double ts = s.ts, T = s.T_;
      bool fnd = false;
      double lo = ts, hi = ts;
      for (int q = 1; q <= A.K; ++q) {
        const double tq = D::add(ts, D::div(D::mul(T, double(q)), double(A.K)));
        ++evals;
        const bool useL = s.ilover == 0;
        if (useL ? c.decide_list(tq, q) : c.template eval<true, false, false>(tq, k, q)) {
          lo = D::add(ts, D::div(D::mul(T, double(q - 1)), double(A.K)));
          hi = tq;
          fnd = true;
          break;
        }
      }
      if (!fnd) return 0;
      const double lim = D::mul(A.tol, T);
      while (D::sub(hi, lo) > lim) {
        const double mid = D::add(lo, D::mul(0.5, D::sub(hi, lo)));
        ++evals;
        ++bis;
        const bool useL = s.ilover == 0;
        if (useL ? c.decide_list(mid, -1) : c.template eval<true, false, false>(mid, k))
          hi = mid;
        else
          lo = mid;
      }
      tc = hi;
      c.template eval<false, true, false>(hi, k);
      ta = int32_t(s.best_key >> 32);
      tb = int32_t(s.best_key & 0xffffffffu);
      return 2;
    };
    // performed: pair evaluations done; method: evaluations the method defines
    auto write_times = [&](uint8_t status, double tc, int32_t ta, int32_t tb, int performed, int method, int bis) {
      if (c.tid == 0) {
        A.t_coll[k] = tc;
        A.status[k] = status;
        A.ct_ab[2 * k] = ta;
        A.ct_ab[2 * k + 1] = tb;
        atomicAdd(&s.cnt[ST_EVALS], (unsigned long long)performed);
        atomicAdd(&s.cnt[ST_CHECKS], (unsigned long long)(chk * method));
        atomicAdd(&s.cnt[ST_BISECT], (unsigned long long)bis);
        atomicAdd(&s.cnt[ST_PAIRS], 1ull);
      }
    };
    if (MODE == MODE_NARROW) {
      const double t = A.t_eval ? A.t_eval[k] : s.ts;
      if (ok) c.template eval<false, true, true>(t, k);
      write_narrow();
      if (c.tid == 0) {
        atomicAdd(&s.cnt[ST_EVALS], 1ull);
        atomicAdd(&s.cnt[ST_CHECKS], (unsigned long long)chk);
        atomicAdd(&s.cnt[ST_PAIRS], 1ull);
      }
    } else if (MODE == MODE_NTIME) {
      int iters = 0;
      uint8_t status = 0;
      double tc = D::add(s.ts, s.T_);
      int32_t ta = -1, tb = -1;
      if (ok && s.nA > 0 && s.nB > 0) {
        motion_bound_narrowing();
        if (c.template eval<true, true, false>(s.ts, k, -1, s.delta)) {
          status = 1;
          ta = int32_t(s.best_key >> 32);
          tb = int32_t(s.best_key & 0xffffffffu);
        } else {
          status = c.narrowing(iters, tc, ta, tb);
        }
      }
      // performed evaluations: the decision at ts and one per narrowing
      // iteration, each over every triangle pair by the method's count
      write_times(status, tc, ta, tb, 1 + iters, 1 + iters, 0);
    } else if (MODE == MODE_CTIME) {
      int evals = 0, bis = 0;
      uint8_t status = 0;
      double tc = D::add(s.ts, s.T_);
      int32_t ta = -1, tb = -1;
      if (ok && s.nA > 0 && s.nB > 0) {
        ++evals;
        motion_bound();
        if (c.template eval<true, true, false>(s.ts, k, -1, s.delta)) {
          status = 1;
          ta = int32_t(s.best_key >> 32);
          tb = int32_t(s.best_key & 0xffffffffu);
        } else {
          c.pose_grid(A.K);  // the sample times' poses, only when the search runs
          status = search(evals, bis, tc, ta, tb);
        }
      }
      write_times(status, tc, ta, tb, evals, evals, bis);
    } else {
      // one evaluation at ts gives the narrow phase, the decision at ts
      // (closest distance <= eps), the closest pair for status 1 and the
      // interval list for the search
      int evals = 0, bis = 0;
      uint8_t status = 0;
      double tc = D::add(s.ts, s.T_);
      int32_t ta = -1, tb = -1;
      if (ok && s.nA > 0 && s.nB > 0) {
        ++evals;
        motion_bound();
        c.template eval<false, true, true>(s.ts, k, -1, s.delta);
        write_narrow();
        if (s.best_key != ~0ull && OpsD::sqrt(s.best_d2) <= s.eps) {
          status = 1;
          ta = int32_t(s.best_key >> 32);
          tb = int32_t(s.best_key & 0xffffffffu);
        } else {
          c.pose_grid(A.K);  // the sample times' poses, only when the search runs
          status = search(evals, bis, tc, ta, tb);
        }
      } else {
        if (ok) c.template eval<false, true, true>(s.ts, k);
        write_narrow();
      }
      // the method's count: one narrow-phase evaluation plus the search's
      // (the evaluation at ts serves both)
      write_times(status, tc, ta, tb, evals > 0 ? evals : 1, evals + 1, bis);
    }
    __syncthreads();
  }
  __syncthreads();
  if (c.tid == 0) {  // this CTA's busy time: from its start to the end of its last pair
    unsigned long long t_end;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t_end));
    s.cnt[ST_BUSY] = t_end - t_begin;
    s.cnt[ST_CTAS] = 1;
    atomicMax(&A.stats[ST_BUSYMAX], t_end - t_begin);
  }
  __syncthreads();
  if (c.tid < ST_N && c.tid != ST_BUSYMAX && s.cnt[c.tid]) atomicAdd(&A.stats[c.tid], s.cnt[c.tid]);
}

// ------------------------------------------------------------- contact sort
// Contacts of each pair are gathered from the staging area and sorted by
// (a, b) in shared memory (bitonic), then written in order.
template <int PREC, int MODE>
cudaError_t launch_pairs(const PairArgs &a, int num_sms, cudaStream_t s) {
  const size_t smem = sizeof(Smem<PREC>);
  // attribute and occupancy once per process (kept out of graph captures)
  static int per_sm = 0;
  if (per_sm == 0) {
    cudaError_t e = cudaFuncSetAttribute(pair_kernel<PREC, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    int q = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&q, pair_kernel<PREC, MODE>, Cfg<PREC>::NT, smem);
    if (e != cudaSuccess) return e;
    per_sm = q < 1 ? 1 : q;
  }
  const int want = a.ctas_per_sm > 0 && a.ctas_per_sm < per_sm ? a.ctas_per_sm : per_sm;
  int64_t grid = (int64_t)num_sms * (want < MAX_PAIR_CTAS_PER_SM ? want : MAX_PAIR_CTAS_PER_SM);
  if (a.max_pairs < grid) grid = a.max_pairs > 0 ? a.max_pairs : 1;
  pair_kernel<PREC, MODE><<<(unsigned)grid, Cfg<PREC>::NT, smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace pk
}  // namespace dem
