// geom.cuh -- device geometry for the contact-detection kernels.
//
// Triangle-triangle distance (paper Section 5, "Collision time detection": the
// closest points of two triangles are a vertex and the other triangle's
// surface, or two edges; intersecting triangles are at distance 0) and the
// free-flight pose (Section 2.1: constant linear and angular velocity between
// snapshots, spherical interpolation of the rotation).
//
// Every routine is a template over an arithmetic policy:
//   OpsD -- binary64 with every operation rounded on its own (__dadd_rn etc.
//           are never fused into FMA).  With OpsD the routines evaluate each
//           formula in one fixed order, the order documented beside it, so
//           that an FP64 result (and every decision taken on it) is a
//           well-defined function of the inputs.
//   OpsF -- binary32, FMA contraction allowed; used for the bulk filter,
//           whose error is bounded by the caller (see pairs.cu).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace dem {

struct OpsD {
  using T = double;
  static __device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
  static __device__ __forceinline__ double sub(double a, double b) { return __dsub_rn(a, b); }
  static __device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
  static __device__ __forceinline__ double div(double a, double b) { return __ddiv_rn(a, b); }
  static __device__ __forceinline__ double sqrt(double a) { return __dsqrt_rn(a); }
  static __device__ __forceinline__ double inf() { return __longlong_as_double(0x7ff0000000000000LL); }
};

struct OpsF {
  using T = float;
  static __device__ __forceinline__ float add(float a, float b) { return a + b; }
  static __device__ __forceinline__ float sub(float a, float b) { return a - b; }
  static __device__ __forceinline__ float mul(float a, float b) { return a * b; }
  // hardware-approximate quotient and square root (a few ulp): FP32 closest
  // points only choose the direction of a separation certificate (a lower
  // bound whatever the direction) and rank candidates, so their accuracy
  // decides how much binary64 work follows, never a result
  static __device__ __forceinline__ float div(float a, float b) { return __fdividef(a, b); }
  static __device__ __forceinline__ float sqrt(float a) {
    return a > 1e-30f ? a * rsqrtf(a) : __fsqrt_rn(a);  // tiny and denormal inputs: exact path
  }
  static __device__ __forceinline__ float inf() { return __int_as_float(0x7f800000); }
};

template <class T>
struct V3 {
  T x, y, z;
};

template <class O>
struct Geo {
  using T = typename O::T;
  using V = V3<T>;

  static __device__ __forceinline__ V mk(T x, T y, T z) { return V{x, y, z}; }
  static __device__ __forceinline__ V sub(V a, V b) {
    return mk(O::sub(a.x, b.x), O::sub(a.y, b.y), O::sub(a.z, b.z));
  }
  // (ax bx + ay by) + az bz
  static __device__ __forceinline__ T dot(V a, V b) {
    return O::add(O::add(O::mul(a.x, b.x), O::mul(a.y, b.y)), O::mul(a.z, b.z));
  }
  static __device__ __forceinline__ V cross(V a, V b) {
    return mk(O::sub(O::mul(a.y, b.z), O::mul(a.z, b.y)), O::sub(O::mul(a.z, b.x), O::mul(a.x, b.z)),
              O::sub(O::mul(a.x, b.y), O::mul(a.y, b.x)));
  }
  // a + d s, componentwise
  static __device__ __forceinline__ V axpy(V a, V d, T s) {
    return mk(O::add(a.x, O::mul(d.x, s)), O::add(a.y, O::mul(d.y, s)), O::add(a.z, O::mul(d.z, s)));
  }
  static __device__ __forceinline__ T clamp01(T s) {
    return s < T(0) ? T(0) : (s > T(1) ? T(1) : s);
  }
  // clamp to [0, 1] in the FP32 filter only (binary64: unchanged, the
  // operation order of the definition)
  static __device__ __forceinline__ T fp32_clamp01(T s) {
    if constexpr (sizeof(T) == 4) return clamp01(s);
    return s;
  }

  // Closest point q of triangle (a,b,c) to p, by Voronoi regions of the
  // triangle (Ericson, Real-Time Collision Detection, Sec. 5.1.5).  e1 = b-a,
  // e2 = c-a; s1..s6 project p-a, p-b, p-c on e1, e2; va, vb, vc are the
  // (scaled) barycentric areas.  Returns |p-q|^2.
  static __device__ __forceinline__ T closest_pt_tri(V p, V a, V b, V c, V &q) {
    V e1 = sub(b, a), e2 = sub(c, a);
    V pa = sub(p, a);
    T s1 = dot(e1, pa), s2 = dot(e2, pa);
    if (s1 <= T(0) && s2 <= T(0)) {
      q = a;
    } else {
      V pb = sub(p, b);
      T s3 = dot(e1, pb), s4 = dot(e2, pb);
      if (s3 >= T(0) && s4 <= s3) {
        q = b;
      } else {
        T vc = O::sub(O::mul(s1, s4), O::mul(s3, s2));
        if (vc <= T(0) && s1 >= T(0) && s3 <= T(0)) {
          q = axpy(a, e1, fp32_clamp01(O::div(s1, O::sub(s1, s3))));
        } else {
          V pc = sub(p, c);
          T s5 = dot(e1, pc), s6 = dot(e2, pc);
          if (s6 >= T(0) && s5 <= s6) {
            q = c;
          } else {
            T vb = O::sub(O::mul(s5, s2), O::mul(s1, s6));
            if (vb <= T(0) && s2 >= T(0) && s6 <= T(0)) {
              q = axpy(a, e2, fp32_clamp01(O::div(s2, O::sub(s2, s6))));
            } else {
              T va = O::sub(O::mul(s3, s6), O::mul(s5, s4));
              T u43 = O::sub(s4, s3), u56 = O::sub(s5, s6);
              if (va <= T(0) && u43 >= T(0) && u56 >= T(0)) {
                q = axpy(b, sub(c, b), fp32_clamp01(O::div(u43, O::add(u43, u56))));
              } else {
                T sum = O::add(O::add(va, vb), vc);
                T v = O::div(vb, sum), w = O::div(vc, sum);
                if constexpr (sizeof(T) == 4) {
                  // FP32 filter only: barycentric weights in the triangle, so
                  // q is a point of the triangle up to the rounding of q itself
                  v = fminf(fmaxf(v, 0.f), 1.f);
                  w = fminf(fmaxf(w, 0.f), 1.f - v);
                }
                q = mk(O::add(O::add(a.x, O::mul(e1.x, v)), O::mul(e2.x, w)),
                       O::add(O::add(a.y, O::mul(e1.y, v)), O::mul(e2.y, w)),
                       O::add(O::add(a.z, O::mul(e1.z, v)), O::mul(e2.z, w)));
              }
            }
          }
        }
      }
    }
    V d = sub(p, q);
    return dot(d, d);
  }

  // Closest points of segments p1 + s d1, p2 + t d2 (s, t in [0,1]): the
  // stationary point of the quadratic, s clamped, t re-solved for s; if t is
  // clamped, s re-solved for t (Ericson 2005, Sec. 5.1.9).  Returns |c1-c2|^2.
  static __device__ __forceinline__ T seg_seg(V p1, V q1, V p2, V q2, V &c1, V &c2) {
    V d1 = sub(q1, p1), d2 = sub(q2, p2), r = sub(p1, p2);
    T a = dot(d1, d1), e = dot(d2, d2), f = dot(d2, r);
    T s, t;
    if (a <= T(0) && e <= T(0)) {
      s = T(0);
      t = T(0);
    } else if (a <= T(0)) {
      s = T(0);
      t = clamp01(O::div(f, e));
    } else {
      T c = dot(d1, r);
      if (e <= T(0)) {
        t = T(0);
        s = clamp01(O::div(-c, a));
      } else {
        T b = dot(d1, d2);
        T denom = O::sub(O::mul(a, e), O::mul(b, b));
        s = denom > T(0) ? clamp01(O::div(O::sub(O::mul(b, f), O::mul(c, e)), denom)) : T(0);
        t = O::div(O::add(O::mul(b, s), f), e);
        if (t < T(0)) {
          t = T(0);
          s = clamp01(O::div(-c, a));
        } else if (t > T(1)) {
          t = T(1);
          s = clamp01(O::div(O::sub(b, c), a));
        }
      }
    }
    c1 = axpy(p1, d1, s);
    c2 = axpy(p2, d2, t);
    V d = sub(c1, c2);
    return dot(d, d);
  }

  // Segment pq crosses triangle (a,b,c): the signed heights of p and q over
  // the plane do not share a strict sign (both zero = coplanar, left to the
  // vertex/edge distances) and the crossing point x is on the inner side of
  // all three edges.
  static __device__ __forceinline__ bool seg_tri_cross(V p, V q, V a, V b, V c, V &x) {
    V nrm = cross(sub(b, a), sub(c, a));
    T sp = dot(nrm, sub(p, a)), sq = dot(nrm, sub(q, a));
    if ((sp > T(0) && sq > T(0)) || (sp < T(0) && sq < T(0)) || (sp == T(0) && sq == T(0)))
      return false;
    T t = fp32_clamp01(O::div(sp, O::sub(sp, sq)));
    x = axpy(p, sub(q, p), t);
    T g0 = dot(cross(sub(b, a), sub(x, a)), nrm);
    T g1 = dot(cross(sub(c, b), sub(x, b)), nrm);
    T g2 = dot(cross(sub(a, c), sub(x, c)), nrm);
    return g0 >= T(0) && g1 >= T(0) && g2 >= T(0);
  }

  // Triangle-triangle squared distance and closest points.  Intersecting
  // triangles: 0 and the first edge-triangle crossing (edges of A against B,
  // then of B against A) as both points.  Otherwise the first minimum, under
  // strict "<", in the order: vertices of A against B, vertices of B against
  // A, edge i of A against edge j of B (i major).
  // Feature ids (the order of the definition): 0..2 vertex i of A against
  // B, 3..5 vertex j of B against A, 6 + 3 i + j edge i of A against edge j
  // of B, 15 + i edge i of A crossing B, 18 + j edge j of B crossing A.
  static __device__ __forceinline__ T tri_dist2(const V A[3], const V B[3], V &pa, V &pb) {
    int f;
    return tri_dist2(A, B, pa, pb, f);
  }
  static __device__ __forceinline__ T tri_dist2(const V A[3], const V B[3], V &pa, V &pb, int &feat) {
    V x;
#pragma unroll 1
    for (int i = 0; i < 3; ++i)
      if (seg_tri_cross(A[i], A[i == 2 ? 0 : i + 1], B[0], B[1], B[2], x)) {
        pa = x;
        pb = x;
        feat = 15 + i;
        return T(0);
      }
#pragma unroll 1
    for (int j = 0; j < 3; ++j)
      if (seg_tri_cross(B[j], B[j == 2 ? 0 : j + 1], A[0], A[1], A[2], x)) {
        pa = x;
        pb = x;
        feat = 18 + j;
        return T(0);
      }
    return tri_dist2_features(A, B, pa, pb, feat);
  }

  // Minimum over the 15 vertex-triangle and edge-edge feature pairs only.
  static __device__ __forceinline__ T tri_dist2_features(const V A[3], const V B[3], V &pa, V &pb) {
    int f;
    return tri_dist2_features(A, B, pa, pb, f);
  }
  static __device__ __forceinline__ T tri_dist2_features(const V A[3], const V B[3], V &pa, V &pb, int &feat) {
    T best = O::inf();
    V q, c1, c2;
    feat = 0;
#pragma unroll 1
    for (int i = 0; i < 3; ++i) {
      T d2 = closest_pt_tri(A[i], B[0], B[1], B[2], q);
      if (d2 < best) {
        best = d2;
        pa = A[i];
        pb = q;
        feat = i;
      }
    }
#pragma unroll 1
    for (int j = 0; j < 3; ++j) {
      T d2 = closest_pt_tri(B[j], A[0], A[1], A[2], q);
      if (d2 < best) {
        best = d2;
        pa = q;
        pb = B[j];
        feat = 3 + j;
      }
    }
#pragma unroll 1
    for (int i = 0; i < 3; ++i)
#pragma unroll 1
      for (int j = 0; j < 3; ++j) {
        T d2 = seg_seg(A[i], A[i == 2 ? 0 : i + 1], B[j], B[j == 2 ? 0 : j + 1], c1, c2);
        if (d2 < best) {
          best = d2;
          pa = c1;
          pb = c2;
          feat = 6 + 3 * i + j;
        }
      }
    return best;
  }

  // One feature's squared distance and points, computed exactly as the full
  // routine computes that feature (so in binary64 it is the definition's
  // value for that feature); a crossing feature gives 0 and the crossing
  // point if the edge crosses, else infinity.
  static __device__ __forceinline__ T feature_dist2(int f, const V A[3], const V B[3], V &pa, V &pb) {
    if (f < 3) {
      pa = A[f];
      return closest_pt_tri(A[f], B[0], B[1], B[2], pb);
    }
    if (f < 6) {
      pb = B[f - 3];
      return closest_pt_tri(B[f - 3], A[0], A[1], A[2], pa);
    }
    if (f < 15) {
      const int i = (f - 6) / 3, j = (f - 6) % 3;
      return seg_seg(A[i], A[i == 2 ? 0 : i + 1], B[j], B[j == 2 ? 0 : j + 1], pa, pb);
    }
    V x{T(0), T(0), T(0)};
    bool hit;
    if (f < 18) {
      const int i = f - 15;
      hit = seg_tri_cross(A[i], A[i == 2 ? 0 : i + 1], B[0], B[1], B[2], x);
    } else {
      const int j = f - 18;
      hit = seg_tri_cross(B[j], B[j == 2 ? 0 : j + 1], A[0], A[1], A[2], x);
    }
    pa = x;
    pb = x;
    return hit ? T(0) : O::inf();
  }
};

// ---------------------------------------------------------------------------
// Separation certificates (FP32 filter).  For any direction n and convex
// sets P, Q: d(P, Q) >= (min over Q of n.y - max over P of n.x) / |n|, and
// for a triangle or a segment the extremes are at its vertices.  With n the
// difference of two computed closest points the bound is close to the
// distance; it is a lower bound whatever n is, so the FP32 decisions built on
// it need no assumption on how accurately the closest points were found.
// Returned raw: the caller subtracts the rounding margin of these dot
// products, the norm and the FP32 relative pose (E of the pair kernel).
__device__ __forceinline__ float cert_dot(V3<float> n, V3<float> v) {
  return fmaf(n.z, v.z, fmaf(n.y, v.y, n.x * v.x));
}
__device__ __forceinline__ float cert_scale(float gap, V3<float> n) {
  const float nn = cert_dot(n, n);
  if (!(nn > 1e-30f)) return -OpsF::inf();
  return gap * rsqrtf(nn);
}
// P = {p1..pk} (k = np points), Q = {q1..qm}: separation along n
__device__ __forceinline__ float cert_sep(const V3<float> *P, int np, const V3<float> *Q, int nq, V3<float> n) {
  float mx = -OpsF::inf(), mn = OpsF::inf();
  for (int k = 0; k < np; ++k) mx = fmaxf(mx, cert_dot(n, P[k]));
  for (int k = 0; k < nq; ++k) mn = fminf(mn, cert_dot(n, Q[k]));
  return cert_scale(mn - mx, n);
}

// ---------------------------------------------------------------------------
// Free-flight pose at time t in binary64, every operation rounded on its own
// (paper Section 2.1).  h = t - t_cur, X = x + v h, q(t) = dq (x) q0 with
// dq = (cos phi, (sin phi / phi) (h/2) w), phi = |w| h / 2.  cos phi and
// sin phi / phi come from their Taylor series in z = phi^2 = (|w|^2 h^2) / 4,
// Horner form with 10 terms, k = 10..1, factors rc[k] = 1/((2k-1)2k) and
// rs[k] = 1/(2k(2k+1)), each the correctly rounded binary64 quotient (see
// pose_reciprocals); no square root, no library trigonometry; truncation
// error below 1e-17 for phi <= 1.5.  R is the rotation matrix of q(t),
// row-major.
constexpr int POSE_TERMS = 10;

// rc[k], rs[k] for k = 1..POSE_TERMS (index 0 unused)
__device__ __forceinline__ void pose_reciprocals(double *rc, double *rs) {
  for (int k = 1; k <= POSE_TERMS; ++k) {
    rc[k] = OpsD::div(1.0, (double)((2 * k - 1) * (2 * k)));
    rs[k] = OpsD::div(1.0, (double)((2 * k) * (2 * k + 1)));
  }
}

// quaternion (w, x, y, z) and centre of the free-flight pose at t
__device__ __forceinline__ void pose_quat_exact(const double *st, int64_t n, int64_t p, double t,
                                                const double *rc, const double *rs, double Q[4], double X[3]) {
  using O = OpsD;
  const double h = O::sub(t, st[13 * n + p]);
  const double wx = st[10 * n + p], wy = st[11 * n + p], wz = st[12 * n + p];
  const double w2 = O::add(O::add(O::mul(wx, wx), O::mul(wy, wy)), O::mul(wz, wz));
  const double z = O::mul(O::mul(w2, O::mul(h, h)), 0.25);
  double c = 1.0, sn = 1.0;
#pragma unroll
  for (int k = POSE_TERMS; k >= 1; --k) {
    c = O::sub(1.0, O::mul(O::mul(z, rc[k]), c));
    sn = O::sub(1.0, O::mul(O::mul(z, rs[k]), sn));
  }
  const double g = O::mul(O::mul(h, 0.5), sn);
  const double pw = c, px = O::mul(g, wx), py = O::mul(g, wy), pz = O::mul(g, wz);
  const double qw = st[6 * n + p], qx = st[7 * n + p], qy = st[8 * n + p], qz = st[9 * n + p];
  // Hamilton product dq (x) q0, each component summed left to right
  Q[0] = O::sub(O::sub(O::sub(O::mul(pw, qw), O::mul(px, qx)), O::mul(py, qy)), O::mul(pz, qz));
  Q[1] = O::sub(O::add(O::add(O::mul(pw, qx), O::mul(px, qw)), O::mul(py, qz)), O::mul(pz, qy));
  Q[2] = O::add(O::add(O::sub(O::mul(pw, qy), O::mul(px, qz)), O::mul(py, qw)), O::mul(pz, qx));
  Q[3] = O::add(O::sub(O::add(O::mul(pw, qz), O::mul(px, qy)), O::mul(py, qx)), O::mul(pz, qw));
  X[0] = O::add(st[0 * n + p], O::mul(st[3 * n + p], h));
  X[1] = O::add(st[1 * n + p], O::mul(st[4 * n + p], h));
  X[2] = O::add(st[2 * n + p], O::mul(st[5 * n + p], h));
}

__device__ __forceinline__ void pose_exact(const double *st, int64_t n, int64_t p, double t,
                                           const double *rc, const double *rs, double R[9], double X[3]) {
  using O = OpsD;
  double Q[4];
  pose_quat_exact(st, n, p, t, rc, rs, Q, X);
  const double rw = Q[0], rx = Q[1], ry = Q[2], rz = Q[3];
  R[0] = O::sub(1.0, O::mul(2.0, O::add(O::mul(ry, ry), O::mul(rz, rz))));
  R[1] = O::mul(2.0, O::sub(O::mul(rx, ry), O::mul(rw, rz)));
  R[2] = O::mul(2.0, O::add(O::mul(rx, rz), O::mul(rw, ry)));
  R[3] = O::mul(2.0, O::add(O::mul(rx, ry), O::mul(rw, rz)));
  R[4] = O::sub(1.0, O::mul(2.0, O::add(O::mul(rx, rx), O::mul(rz, rz))));
  R[5] = O::mul(2.0, O::sub(O::mul(ry, rz), O::mul(rw, rx)));
  R[6] = O::mul(2.0, O::sub(O::mul(rx, rz), O::mul(rw, ry)));
  R[7] = O::mul(2.0, O::add(O::mul(ry, rz), O::mul(rw, rx)));
  R[8] = O::sub(1.0, O::mul(2.0, O::add(O::mul(rx, rx), O::mul(ry, ry))));
}

// World position R b + X of a body-frame vertex: ((R0 bx + R1 by) + R2 bz) + X0.
__device__ __forceinline__ V3<double> to_world_exact(const double *R, const double *X, float bx,
                                                     float by, float bz) {
  using O = OpsD;
  const double x = bx, y = by, z = bz;
  return V3<double>{
      O::add(O::add(O::add(O::mul(R[0], x), O::mul(R[1], y)), O::mul(R[2], z)), X[0]),
      O::add(O::add(O::add(O::mul(R[3], x), O::mul(R[4], y)), O::mul(R[5], z)), X[1]),
      O::add(O::add(O::add(O::mul(R[6], x), O::mul(R[7], y)), O::mul(R[8], z)), X[2])};
}

}  // namespace dem
