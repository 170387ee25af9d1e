/*
 * dem_oracle.c -- plain FP64 CPU oracle for the space-time contact-detection
 * path of Noble & Weinzierl, "Parallel local time stepping for rigid bodies
 * represented by triangulated meshes".
 *
 * TEST INFRASTRUCTURE ONLY: the slow, obviously correct definition that the
 * CUDA library is checked against.  Only tests, the smoke check and the
 * benchmark's CPU-baseline leg load it.  It shares no code with the CUDA
 * library.
 *
 * Arithmetic: IEEE binary64, compiled with -ffp-contract=off (no fused
 * multiply-add), every expression evaluated left to right as written.  The
 * order of operations of every formula is part of the definition: the CUDA
 * library's FP64 decisions follow the same order so that decisions near a
 * threshold come out the same.
 *
 * Pins (tests/test_oracle_*.py): closed forms for poses and triangle
 * distances, symmetry, rigid-motion invariance, convex QP via scipy,
 * brute-force barycentric sampling, icosphere distance bounds, closed-form
 * collision times, k-d tree broad phase, scipy connected components.
 */
#include "dem_oracle.h"

#include <math.h>
#include <pthread.h>
#include <stdatomic.h>
#include <stdlib.h>
#include <string.h>

enum { FX = 0, FY, FZ, FVX, FVY, FVZ, FQW, FQX, FQY, FQZ, FWX, FWY, FWZ, FTCUR, FDT, FEPS,
       FRADIUS };

typedef struct { double x, y, z; } vec3;

static vec3 mk(double x, double y, double z) { vec3 r; r.x = x; r.y = y; r.z = z; return r; }
static vec3 sub(vec3 a, vec3 b) { return mk(a.x - b.x, a.y - b.y, a.z - b.z); }
static double dot(vec3 a, vec3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
static vec3 cross(vec3 a, vec3 b) {
  return mk(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
/* a + d * s, componentwise */
static vec3 axpy(vec3 a, vec3 d, double s) { return mk(a.x + d.x * s, a.y + d.y * s, a.z + d.z * s); }
static double clamp01(double s) { return s < 0.0 ? 0.0 : (s > 1.0 ? 1.0 : s); }
static vec3 ld(const double *p) { return mk(p[0], p[1], p[2]); }
static void st(double *p, vec3 v) { p[0] = v.x; p[1] = v.y; p[2] = v.z; }

/* ------------------------------------------------------------------------ */
/* Pose at time t (paper Section 2.1: snapshots of position, velocity,
 * rotation and angular velocity; between snapshots the position moves
 * linearly and the rotation along the great circle, i.e. free flight with
 * constant linear velocity v and constant world-frame angular velocity w).
 *
 *   h = t - t_cur,  X(t) = x + v h,  q(t) = dq (x) q0,
 *   dq = (cos(phi), sin(phi)/phi * (h/2) * w),  phi = |w| h / 2.
 *
 * cos(phi) and sin(phi)/phi are evaluated from their Taylor series in
 * z = phi^2 = |w|^2 h^2 / 4 (Horner form, 10 terms; the factors are the
 * binary64 reciprocals 1/((2k-1)2k) and 1/(2k(2k+1)), each the correctly
 * rounded quotient of 1 by an exact integer); no square root, no library
 * trigonometry.  Truncation error < 1e-17 for phi <= 1.5. */
#define POSE_TERMS 10

/* unit quaternion (w, x, y, z) and centre of particle p at time t */
static void pose_q(const double *state, int64_t n, int64_t p, double t, double Q[4], double X[3]) {
  const double *s = state;
  double h = t - s[FTCUR * n + p];
  vec3 w = mk(s[FWX * n + p], s[FWY * n + p], s[FWZ * n + p]);
  double w2 = dot(w, w);
  double z = (w2 * (h * h)) * 0.25;
  double c = 1.0, sn = 1.0;
  for (int k = POSE_TERMS; k >= 1; --k) {
    const double rc = 1.0 / (double)((2 * k - 1) * (2 * k));
    const double rs = 1.0 / (double)((2 * k) * (2 * k + 1));
    c = 1.0 - (z * rc) * c;
    sn = 1.0 - (z * rs) * sn;
  }
  double g = (h * 0.5) * sn;
  /* dq = (c, g w) */
  double pw = c, px = g * w.x, py = g * w.y, pz = g * w.z;
  double qw = s[FQW * n + p], qx = s[FQX * n + p], qy = s[FQY * n + p], qz = s[FQZ * n + p];
  /* Hamilton product dq (x) q0 */
  double rw = pw * qw - px * qx - py * qy - pz * qz;
  double rx = pw * qx + px * qw + py * qz - pz * qy;
  double ry = pw * qy - px * qz + py * qw + pz * qx;
  double rz = pw * qz + px * qy - py * qx + pz * qw;
  Q[0] = rw;
  Q[1] = rx;
  Q[2] = ry;
  Q[3] = rz;
  X[0] = s[FX * n + p] + s[FVX * n + p] * h;
  X[1] = s[FY * n + p] + s[FVY * n + p] * h;
  X[2] = s[FZ * n + p] + s[FVZ * n + p] * h;
}

void demo_pose(const double *state, int64_t n, int64_t p, double t, double R[9], double X[3]) {
  double Q[4];
  pose_q(state, n, p, t, Q, X);
  double rw = Q[0], rx = Q[1], ry = Q[2], rz = Q[3];
  /* rotation matrix of the unit quaternion (row-major) */
  R[0] = 1.0 - 2.0 * (ry * ry + rz * rz);
  R[1] = 2.0 * (rx * ry - rw * rz);
  R[2] = 2.0 * (rx * rz + rw * ry);
  R[3] = 2.0 * (rx * ry + rw * rz);
  R[4] = 1.0 - 2.0 * (rx * rx + rz * rz);
  R[5] = 2.0 * (ry * rz - rw * rx);
  R[6] = 2.0 * (rx * rz - rw * ry);
  R[7] = 2.0 * (ry * rz + rw * rx);
  R[8] = 1.0 - 2.0 * (rx * rx + ry * ry);
}

/* world position of body-frame vertex b: R b + X, rows left to right */
static vec3 to_world(const double R[9], const double X[3], vec3 b) {
  return mk(R[0] * b.x + R[1] * b.y + R[2] * b.z + X[0],
            R[3] * b.x + R[4] * b.y + R[5] * b.z + X[1],
            R[6] * b.x + R[7] * b.y + R[8] * b.z + X[2]);
}

/* ------------------------------------------------------------------------ */
/* Closest point of triangle (a,b,c) to p by Voronoi-region classification
 * (Ericson, Real-Time Collision Detection, 2005, Sec. 5.1.5).  With
 * e1 = b-a, e2 = c-a and the six projections s1..s6 of p-a, p-b, p-c on
 * e1, e2, the signs of s_i and of the three barycentric areas va, vb, vc
 * select a vertex, an edge or the face.  Returns |p-q|^2. */
static double closest_pt_tri(vec3 p, vec3 a, vec3 b, vec3 c, vec3 *q) {
  vec3 e1 = sub(b, a), e2 = sub(c, a);
  vec3 pa = sub(p, a);
  double s1 = dot(e1, pa), s2 = dot(e2, pa);
  if (s1 <= 0.0 && s2 <= 0.0) { *q = a; goto done; }
  {
    vec3 pb = sub(p, b);
    double s3 = dot(e1, pb), s4 = dot(e2, pb);
    if (s3 >= 0.0 && s4 <= s3) { *q = b; goto done; }
    double vc = s1 * s4 - s3 * s2;
    if (vc <= 0.0 && s1 >= 0.0 && s3 <= 0.0) {
      *q = axpy(a, e1, s1 / (s1 - s3));
      goto done;
    }
    vec3 pc = sub(p, c);
    double s5 = dot(e1, pc), s6 = dot(e2, pc);
    if (s6 >= 0.0 && s5 <= s6) { *q = c; goto done; }
    double vb = s5 * s2 - s1 * s6;
    if (vb <= 0.0 && s2 >= 0.0 && s6 <= 0.0) {
      *q = axpy(a, e2, s2 / (s2 - s6));
      goto done;
    }
    double va = s3 * s6 - s5 * s4;
    double u43 = s4 - s3, u56 = s5 - s6;
    if (va <= 0.0 && u43 >= 0.0 && u56 >= 0.0) {
      *q = axpy(b, sub(c, b), u43 / (u43 + u56));
      goto done;
    }
    double sum = va + vb + vc;
    double v = vb / sum, w = vc / sum;
    *q = mk(a.x + e1.x * v + e2.x * w, a.y + e1.y * v + e2.y * w, a.z + e1.z * v + e2.z * w);
  }
done:;
  vec3 d = sub(p, *q);
  return dot(d, d);
}

/* Closest points of segments p1 + s d1 and p2 + t d2, s,t in [0,1]
 * (Ericson 2005, Sec. 5.1.9): stationary point of the quadratic in (s,t),
 * clamped, with t re-solved for the clamped s and s re-solved when t is
 * clamped.  Returns |c1-c2|^2. */
static double seg_seg(vec3 p1, vec3 q1, vec3 p2, vec3 q2, vec3 *c1, vec3 *c2) {
  vec3 d1 = sub(q1, p1), d2 = sub(q2, p2), r = sub(p1, p2);
  double a = dot(d1, d1), e = dot(d2, d2), f = dot(d2, r);
  double s, t;
  if (a <= 0.0 && e <= 0.0) {
    s = 0.0;
    t = 0.0;
  } else if (a <= 0.0) {
    s = 0.0;
    t = clamp01(f / e);
  } else {
    double c = dot(d1, r);
    if (e <= 0.0) {
      t = 0.0;
      s = clamp01(-c / a);
    } else {
      double b = dot(d1, d2);
      double denom = a * e - b * b;
      s = denom > 0.0 ? clamp01((b * f - c * e) / denom) : 0.0;
      t = (b * s + f) / e;
      if (t < 0.0) {
        t = 0.0;
        s = clamp01(-c / a);
      } else if (t > 1.0) {
        t = 1.0;
        s = clamp01((b - c) / a);
      }
    }
  }
  *c1 = axpy(p1, d1, s);
  *c2 = axpy(p2, d2, t);
  vec3 d = sub(*c1, *c2);
  return dot(d, d);
}

/* Does segment pq cross triangle (a,b,c)?  Signed heights of p and q over the
 * triangle's plane must not have the same strict sign (both zero = coplanar,
 * left to the vertex/edge distances); the crossing point x must lie on the
 * inner side of all three edges. */
static int seg_tri_cross(vec3 p, vec3 q, vec3 a, vec3 b, vec3 c, vec3 *x) {
  vec3 nrm = cross(sub(b, a), sub(c, a));
  double sp = dot(nrm, sub(p, a)), sq = dot(nrm, sub(q, a));
  if ((sp > 0.0 && sq > 0.0) || (sp < 0.0 && sq < 0.0) || (sp == 0.0 && sq == 0.0)) return 0;
  double t = sp / (sp - sq);
  *x = axpy(p, sub(q, p), t);
  double g0 = dot(cross(sub(b, a), sub(*x, a)), nrm);
  double g1 = dot(cross(sub(c, b), sub(*x, b)), nrm);
  double g2 = dot(cross(sub(a, c), sub(*x, c)), nrm);
  return g0 >= 0.0 && g1 >= 0.0 && g2 >= 0.0;
}

/* Triangle-triangle distance (paper Section 5, "Collision time detection":
 * the closest points of two triangles are a vertex and the other triangle's
 * surface, or lie on two edges).  Intersecting triangles have distance 0 and
 * the first edge-triangle crossing point (edges of A against B, then edges of
 * B against A) as both closest points.  Otherwise the minimum over the 6
 * vertex-triangle and 9 edge-edge distances, first attaining feature pair in
 * the order VT(A->B), VT(B->A), EE(i of A major, j of B minor), strict "<".
 * Returns the squared distance. */
static double tri_dist2(const vec3 A[3], const vec3 B[3], vec3 *pa, vec3 *pb) {
  vec3 x;
  for (int i = 0; i < 3; ++i)
    if (seg_tri_cross(A[i], A[(i + 1) % 3], B[0], B[1], B[2], &x)) { *pa = x; *pb = x; return 0.0; }
  for (int j = 0; j < 3; ++j)
    if (seg_tri_cross(B[j], B[(j + 1) % 3], A[0], A[1], A[2], &x)) { *pa = x; *pb = x; return 0.0; }
  double best = INFINITY;
  vec3 q, c1, c2;
  for (int i = 0; i < 3; ++i) {
    double d2 = closest_pt_tri(A[i], B[0], B[1], B[2], &q);
    if (d2 < best) { best = d2; *pa = A[i]; *pb = q; }
  }
  for (int j = 0; j < 3; ++j) {
    double d2 = closest_pt_tri(B[j], A[0], A[1], A[2], &q);
    if (d2 < best) { best = d2; *pa = q; *pb = B[j]; }
  }
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double d2 = seg_seg(A[i], A[(i + 1) % 3], B[j], B[(j + 1) % 3], &c1, &c2);
      if (d2 < best) { best = d2; *pa = c1; *pb = c2; }
    }
  return best;
}

double demo_tri_dist(const double A[9], const double B[9], double pa[3], double pb[3]) {
  vec3 a[3] = {ld(A), ld(A + 3), ld(A + 6)}, b[3] = {ld(B), ld(B + 3), ld(B + 6)};
  vec3 x, y;
  double d2 = tri_dist2(a, b, &x, &y);
  st(pa, x);
  st(pb, y);
  return sqrt(d2);
}

double demo_closest_pt_tri(const double p[3], const double T[9], double q[3]) {
  vec3 r;
  double d2 = closest_pt_tri(ld(p), ld(T), ld(T + 3), ld(T + 6), &r);
  st(q, r);
  return d2;
}

double demo_seg_seg(const double p1[3], const double q1[3], const double p2[3], const double q2[3],
                    double c1[3], double c2[3]) {
  vec3 x, y;
  double d2 = seg_seg(ld(p1), ld(q1), ld(p2), ld(q2), &x, &y);
  st(c1, x);
  st(c2, y);
  return d2;
}

/* ------------------------------------------------------------------------ */
/* Pair evaluation at one time: world vertices of both particles, then every
 * triangle pair in (a, b) lexicographic order. */

typedef struct {
  double d2min;
  int32_t a, b;
  vec3 pa, pb;
  /* contact list (optional) */
  int64_t nc, capc;
  int32_t *cab;   /* (a,b) per contact */
  double *cgeom;  /* (d, pa, pb) per contact */
} pair_eval;

static vec3 *world_verts(const double *state, int64_t n, const int64_t *tri_off, const float *tris,
                         int64_t n_tris, int64_t p, double t) {
  double R[9], X[3];
  demo_pose(state, n, p, t, R, X);
  int64_t t0 = tri_off[p], cnt = tri_off[p + 1] - tri_off[p];
  vec3 *w = (vec3 *)malloc(sizeof(vec3) * 3 * (size_t)(cnt > 0 ? cnt : 1));
  for (int64_t k = 0; k < cnt; ++k)
    for (int s = 0; s < 3; ++s) {
      const float *v = tris + ((size_t)s * (size_t)n_tris + (size_t)(t0 + k)) * 4;
      w[3 * k + s] = to_world(R, X, mk((double)v[0], (double)v[1], (double)v[2]));
    }
  return w;
}

/* ------------------------------------------------------------------------ */
/* Broad phase (paper Section 3: free-flight extrapolation of each particle
 * over its own step, bounding volumes that cover the particle and its halo,
 * a symmetric pairwise overlap test; static geometry treated apart).
 *
 * Swept sphere of a moving particle p over [t_cur, t_cur+dt]: centre
 * m = x + v (dt/2), radius rho = (radius + eps) + |v| (dt/2).  Two moving
 * particles i < j are a candidate iff |m_i - m_j|^2 <= (rho_i + rho_j)^2.
 *
 * A static particle s (paper Section 3, "Static geometric objects"; the
 * axis-aligned boxes of Check 1) is represented by the box of its world
 * vertices at t_cur, widened by eps_s on every side: a floor made of a few
 * huge triangles would otherwise have a bounding sphere that reaches far
 * above it.  A moving p and a static s are a candidate iff p's swept sphere
 * meets that box, and the pair is written (p, s): the static particle is
 * always second.  Two static particles never pair.  Output order: by first
 * member, then by second.  Brute force over all pairs. */
static void swept_sphere(const double *s, int64_t n, int64_t p, vec3 *m, double *rho) {
  double hdt = s[FDT * n + p] * 0.5;
  vec3 v = mk(s[FVX * n + p], s[FVY * n + p], s[FVZ * n + p]);
  *m = mk(s[FX * n + p] + v.x * hdt, s[FY * n + p] + v.y * hdt, s[FZ * n + p] + v.z * hdt);
  *rho = (s[FRADIUS * n + p] + s[FEPS * n + p]) + sqrt(dot(v, v)) * hdt;
}

static int spheres_meet(vec3 ma, double ra, vec3 mb, double rb) {
  vec3 d = sub(ma, mb);
  double rr = ra + rb;
  return dot(d, d) <= rr * rr;
}

/* box [lo, hi] of static particle s: componentwise extremes of its world
 * vertices at t_cur, then lo - eps_s and hi + eps_s (empty mesh: +inf/-inf,
 * which meets no sphere) */
static void static_box(const double *state, int64_t n, const int64_t *tri_off, const float *tris,
                       int64_t n_tris, int64_t s, vec3 *lo, vec3 *hi) {
  vec3 *w = world_verts(state, n, tri_off, tris, n_tris, s, state[FTCUR * n + s]);
  int64_t nv = 3 * (tri_off[s + 1] - tri_off[s]);
  vec3 l = mk(INFINITY, INFINITY, INFINITY), h = mk(-INFINITY, -INFINITY, -INFINITY);
  for (int64_t k = 0; k < nv; ++k) {
    l = mk(fmin(l.x, w[k].x), fmin(l.y, w[k].y), fmin(l.z, w[k].z));
    h = mk(fmax(h.x, w[k].x), fmax(h.y, w[k].y), fmax(h.z, w[k].z));
  }
  free(w);
  double e = state[FEPS * n + s];
  *lo = mk(l.x - e, l.y - e, l.z - e);
  *hi = mk(h.x + e, h.y + e, h.z + e);
}

/* distance of coordinate m outside [lo, hi] (0 inside) */
static double gap(double m, double lo, double hi) { return m < lo ? lo - m : (m > hi ? m - hi : 0.0); }

static int sphere_meets_box(vec3 m, double rho, vec3 lo, vec3 hi) {
  vec3 g = mk(gap(m.x, lo.x, hi.x), gap(m.y, lo.y, hi.y), gap(m.z, lo.z, hi.z));
  return dot(g, g) <= rho * rho;
}

static int is_st(const uint8_t *is_static, int64_t p) { return is_static && is_static[p]; }

static void emit(int32_t *pairs, int64_t cap, int64_t *cnt, int64_t a, int64_t b) {
  if (*cnt < cap) {
    pairs[2 * *cnt] = (int32_t)a;
    pairs[2 * *cnt + 1] = (int32_t)b;
  }
  ++*cnt;
}

int64_t demo_broad_phase(const double *state, const uint8_t *is_static, int64_t n, const int64_t *tri_off,
                         const float *tris, int64_t n_tris, int32_t *pairs, int64_t cap) {
  vec3 *m = (vec3 *)malloc(sizeof(vec3) * (size_t)(n > 0 ? n : 1));
  vec3 *lo = (vec3 *)malloc(sizeof(vec3) * (size_t)(n > 0 ? n : 1));
  vec3 *hi = (vec3 *)malloc(sizeof(vec3) * (size_t)(n > 0 ? n : 1));
  double *rho = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  for (int64_t p = 0; p < n; ++p) {
    swept_sphere(state, n, p, &m[p], &rho[p]);
    if (is_st(is_static, p)) static_box(state, n, tri_off, tris, n_tris, p, &lo[p], &hi[p]);
  }
  int64_t cnt = 0;
  for (int64_t a = 0; a < n; ++a) {
    if (is_st(is_static, a)) continue; /* a static particle is never first */
    for (int64_t b = 0; b < n; ++b) {
      if (b == a) continue;
      if (is_st(is_static, b)) {
        if (sphere_meets_box(m[a], rho[a], lo[b], hi[b])) emit(pairs, cap, &cnt, a, b);
      } else if (b > a && spheres_meet(m[a], rho[a], m[b], rho[b])) {
        emit(pairs, cap, &cnt, a, b);
      }
    }
  }
  free(m);
  free(lo);
  free(hi);
  free(rho);
  return cnt;
}

/* Space-time hose test (Section 3, Check 2) of two moving particles over
 * their pair interval [ts, ts + T] (ts = min t_cur, T = min dt): each
 * bounding sphere (radius R + eps) moves on the straight segment from its old
 * snapshot to its current one (x_old + v_old (t - t_old)) and then with its
 * current velocity (x + v (t - t_cur)); the hoses meet iff the centres come
 * within r_i + r_j at some time of the interval.  The interval is cut at the
 * later t_cur if it lies inside; on each piece the relative position is
 * d0 + u s (s = time into the piece), whose squared length is smallest at
 * s = -(d0 . u) / (u . u) clamped to the piece (s = 0 when u = 0). */
static vec3 hose_at(const double *cur, const double *old, int64_t n, int64_t p, double t, int on_old, vec3 *v) {
  const double *s = on_old ? old : cur;
  *v = mk(s[FVX * n + p], s[FVY * n + p], s[FVZ * n + p]);
  double h = t - s[FTCUR * n + p];
  return mk(s[FX * n + p] + v->x * h, s[FY * n + p] + v->y * h, s[FZ * n + p] + v->z * h);
}

static int hose_meet(const double *cur, const double *old, int64_t n, int64_t i, int64_t j) {
  double ti = cur[FTCUR * n + i], tj = cur[FTCUR * n + j];
  double ts = ti < tj ? ti : tj, t2 = ti < tj ? tj : ti;
  double di = cur[FDT * n + i], dj = cur[FDT * n + j];
  double te = ts + (di < dj ? di : dj);
  double r = (cur[FRADIUS * n + i] + cur[FEPS * n + i]) + (cur[FRADIUS * n + j] + cur[FEPS * n + j]);
  int nk = 0;
  double kk[3];
  kk[nk++] = ts;
  if (t2 > ts && t2 < te) kk[nk++] = t2;
  kk[nk++] = te;
  for (int q = 0; q + 1 < nk; ++q) {
    double a = kk[q], b = kk[q + 1];
    vec3 vi, vj;
    vec3 xi = hose_at(cur, old, n, i, a, b <= ti, &vi);
    vec3 xj = hose_at(cur, old, n, j, a, b <= tj, &vj);
    vec3 d0 = sub(xi, xj), u = sub(vi, vj);
    double uu = dot(u, u), du = dot(d0, u), s = 0.0;
    if (uu > 0.0) {
      s = -du / uu;
      if (s < 0.0) s = 0.0;
      if (s > b - a) s = b - a;
    }
    vec3 dm = axpy(d0, u, s);
    if (dot(dm, dm) <= r * r) return 1;
  }
  return 0;
}

int demo_hose_meet(const double *cur, const double *old, int64_t n, int64_t i, int64_t j) {
  return hose_meet(cur, old, n, i, j);
}

static int cmp_pair(const void *x, const void *y) {
  const int32_t *a = (const int32_t *)x, *b = (const int32_t *)y;
  if (a[0] != b[0]) return a[0] < b[0] ? -1 : 1;
  return a[1] < b[1] ? -1 : (a[1] > b[1] ? 1 : 0);
}

/* Candidate pairs that contain particle p (same predicates and pair order as
 * demo_broad_phase), brute force over the other particles, then sorted by
 * (first, second).  Returns the number of pairs; writes at most cap. */
int64_t demo_broad_partners(const double *state, const uint8_t *is_static, int64_t n, const int64_t *tri_off,
                            const float *tris, int64_t n_tris, int64_t p, int32_t *pairs, int64_t cap) {
  int64_t cnt = 0, room = 64;
  int32_t *all = (int32_t *)malloc(sizeof(int32_t) * 2 * (size_t)room);
  vec3 mp, lp, hp;
  double rp;
  swept_sphere(state, n, p, &mp, &rp);
  if (is_st(is_static, p)) static_box(state, n, tri_off, tris, n_tris, p, &lp, &hp);
  for (int64_t q = 0; q < n; ++q) {
    if (q == p || (is_st(is_static, p) && is_st(is_static, q))) continue;
    vec3 mq, lq, hq;
    double rq;
    swept_sphere(state, n, q, &mq, &rq);
    int64_t a, b;
    int hit;
    if (is_st(is_static, p)) {
      hit = sphere_meets_box(mq, rq, lp, hp);
      a = q;
      b = p;
    } else if (is_st(is_static, q)) {
      static_box(state, n, tri_off, tris, n_tris, q, &lq, &hq);
      hit = sphere_meets_box(mp, rp, lq, hq);
      a = p;
      b = q;
    } else {
      hit = p < q ? spheres_meet(mp, rp, mq, rq) : spheres_meet(mq, rq, mp, rp);
      a = p < q ? p : q;
      b = p < q ? q : p;
    }
    if (!hit) continue;
    if (cnt == room) {
      room *= 2;
      all = (int32_t *)realloc(all, sizeof(int32_t) * 2 * (size_t)room);
    }
    all[2 * cnt] = (int32_t)a;
    all[2 * cnt + 1] = (int32_t)b;
    ++cnt;
  }
  qsort(all, (size_t)cnt, 2 * sizeof(int32_t), cmp_pair);
  memcpy(pairs, all, sizeof(int32_t) * 2 * (size_t)(cnt < cap ? cnt : cap));
  free(all);
  return cnt;
}

static void push_contact(pair_eval *e, int32_t a, int32_t b, double d, vec3 pa, vec3 pb) {
  if (e->nc == e->capc) {
    e->capc = e->capc ? 2 * e->capc : 64;
    e->cab = (int32_t *)realloc(e->cab, sizeof(int32_t) * 2 * (size_t)e->capc);
    e->cgeom = (double *)realloc(e->cgeom, sizeof(double) * 7 * (size_t)e->capc);
  }
  e->cab[2 * e->nc] = a;
  e->cab[2 * e->nc + 1] = b;
  double *g = e->cgeom + 7 * e->nc;
  g[0] = d;
  st(g + 1, pa);
  st(g + 4, pb);
  e->nc++;
}

/* eps_pair = eps_i + eps_j (paper Section 2.1: particles touch when their
 * halos overlap; the contact-point definition of Section 5 bounds the
 * distance by the halo). */
static double eps_pair(const double *s, int64_t n, int64_t i, int64_t j) {
  return s[FEPS * n + i] + s[FEPS * n + j];
}

static void eval_pair(const double *state, int64_t n, const int64_t *tri_off, const float *tris,
                      int64_t n_tris, int64_t i, int64_t j, double t, int want_contacts,
                      pair_eval *e) {
  vec3 *WA = world_verts(state, n, tri_off, tris, n_tris, i, t);
  vec3 *WB = world_verts(state, n, tri_off, tris, n_tris, j, t);
  int64_t na = tri_off[i + 1] - tri_off[i], nb = tri_off[j + 1] - tri_off[j];
  double eps = eps_pair(state, n, i, j);
  e->d2min = INFINITY;
  e->a = e->b = -1;
  e->pa = e->pb = mk(0, 0, 0);
  for (int64_t a = 0; a < na; ++a)
    for (int64_t b = 0; b < nb; ++b) {
      vec3 pa, pb;
      double d2 = tri_dist2(WA + 3 * a, WB + 3 * b, &pa, &pb);
      if (d2 < e->d2min) {
        e->d2min = d2;
        e->a = (int32_t)a;
        e->b = (int32_t)b;
        e->pa = pa;
        e->pb = pb;
      }
      if (want_contacts) {
        double d = sqrt(d2);
        if (d <= eps) push_contact(e, (int32_t)a, (int32_t)b, d, pa, pb);
      }
    }
  free(WA);
  free(WB);
}

/* Pair interval (Section 3, Eq. "max time span between two particles"):
 * ts = min of the members' t_cur, T = min of their steps.  A static member
 * has no time step of its own (static objects take no part in the
 * extrapolation, Section 3): then the interval is the moving member's. */
static double pair_start(const double *s, const uint8_t *sta, int64_t n, int64_t i, int64_t j) {
  if (sta && sta[j] && !sta[i]) return s[FTCUR * n + i];
  if (sta && sta[i] && !sta[j]) return s[FTCUR * n + j];
  double a = s[FTCUR * n + i], b = s[FTCUR * n + j];
  return a < b ? a : b;
}
static double pair_span(const double *s, const uint8_t *sta, int64_t n, int64_t i, int64_t j) {
  if (sta && sta[j] && !sta[i]) return s[FDT * n + i];
  if (sta && sta[i] && !sta[j]) return s[FDT * n + j];
  double a = s[FDT * n + i], b = s[FDT * n + j];
  return a < b ? a : b;
}

/* ------------------------------------------------------------------------ */
/* threading over independent pairs */
typedef struct {
  const double *state;
  const uint8_t *is_static;
  int64_t n;
  const int64_t *tri_off;
  const float *tris;
  int64_t n_tris;
  const int32_t *pairs;
  int64_t m;
  const double *t_eval;
  int K;
  double tol;
  pair_eval *ev;         /* narrow */
  double *t_coll;        /* collision times */
  uint8_t *status;
  int32_t *tri_ab;
  int32_t *n_evals;
  atomic_llong next;
  int mode;              /* 0 narrow, 1 collision times (samples), 2 collision times (narrowing) */
} job;

/* Collision time of one pair (paper Section 5, case distinction and the
 * definition of narrowing; interval of Eq. "max time span between two
 * particles").  Interval [ts, ts+T], ts = min(t_cur_i, t_cur_j),
 * T = min(dt_i, dt_j).  f(t) <= eps  <=>  some triangle pair is within
 * eps_pair at t.
 *   f(ts) <= eps           -> status 1, t = ts + T (already touching)
 *   first k in 1..K with f(ts + T k / K) <= eps -> bisection on
 *     [t_{k-1}, t_k] while hi - lo > tol T with mid = lo + (hi-lo)/2;
 *     the returned time is hi (the upper bracket: the halos overlap there,
 *     the "widening" of Section 5) -> status 2
 *   no sample touches     -> status 0, t = ts + T. */
static void collision_time_one(job *J, int64_t k) {
  int64_t i = J->pairs[2 * k], j = J->pairs[2 * k + 1];
  const double *s = J->state;
  int64_t n = J->n;
  double eps = eps_pair(s, n, i, j);
  double ts = pair_start(s, J->is_static, n, i, j), T = pair_span(s, J->is_static, n, i, j);
  pair_eval e;
  memset(&e, 0, sizeof e);
  int evals = 0;
#define FLE(tt) (eval_pair(s, n, J->tri_off, J->tris, J->n_tris, i, j, (tt), 0, &e), ++evals, \
                 sqrt(e.d2min) <= eps)
  uint8_t status;
  double tc;
  int32_t ta = -1, tb = -1;
  if (FLE(ts)) {
    status = 1;
    tc = ts + T;
    ta = e.a;
    tb = e.b;
  } else {
    int found = 0;
    double lo = ts, hi = ts;
    for (int q = 1; q <= J->K; ++q) {
      double tq = ts + (T * (double)q) / (double)J->K;
      if (FLE(tq)) {
        lo = ts + (T * (double)(q - 1)) / (double)J->K;
        hi = tq;
        found = 1;
        break;
      }
    }
    if (!found) {
      status = 0;
      tc = ts + T;
    } else {
      double lim = J->tol * T;
      while (hi - lo > lim) {
        double mid = lo + 0.5 * (hi - lo);
        if (FLE(mid))
          hi = mid;
        else
          lo = mid;
      }
      status = 2;
      tc = hi;
      /* closest triangle pair at the returned time */
      eval_pair(s, n, J->tri_off, J->tris, J->n_tris, i, j, hi, 0, &e);
      ta = e.a;
      tb = e.b;
    }
  }
#undef FLE
  J->t_coll[k] = tc;
  J->status[k] = status;
  J->tri_ab[2 * k] = ta;
  J->tri_ab[2 * k + 1] = tb;
  if (J->n_evals) J->n_evals[k] = evals;
}

/* ------------------------------------------------------------------------ */
/* The paper's narrowing (Section 5, "Collision time detection", definitions
 * of narrowing and widening), as a second collision-time procedure.  It
 * approximates the contact time per triangle pair over the current search
 * span [ts, te] and narrows te to the earliest contact found:
 *   vertex-triangle (each vertex of one triangle against the other triangle):
 *     the vertex is taken into the body frame of the triangle's particle at
 *     ts and at te (P0, P1: R^T (W - X) with the actual poses) and moves on
 *     the straight segment P0 -> P1 in between (rotation neglected); its
 *     distance to the triangle is checked at the end P1 (time te) and where
 *     the segment crosses the triangle's plane, if it does (time
 *     ts + s (te - ts), s = h0 / (h0 - h1) from the signed plane heights
 *     h = n . (P - a), n = (b - a) x (c - a));
 *   edge-edge (each edge pair): the distance with the actual poses at the
 *     middle ts + 0.5 (te - ts) and at te;
 *   a candidate is a time whose distance is <= eps_pair; the span's start
 *   needs no check (the pair is apart there, or status 1 was returned).
 * Iteration: tc = the earliest candidate over all triangle pairs; none ->
 * stop; otherwise a contact is found, and if tc < te - w (w = tol T, the
 * widening) the span narrows to te = tc + w and the tests rerun, else stop
 * (at most 64 iterations).  Status 1 as in the sampling procedure (distance at
 * ts <= eps_pair, t = ts + T); a found contact gives status 2 with t = te and
 * the closest (smallest (a, b)) triangle pair of the earliest candidate of the
 * last iteration; none gives status 0, t = ts + T. */
#define NARROW_MAX_ITER 64

/* body-frame position of world point W in the frame (R, X): R^T (W - X) */
static vec3 rel_pos(const double R[9], const double X[3], vec3 W) {
  vec3 d = sub(W, ld(X));
  return mk(R[0] * d.x + R[3] * d.y + R[6] * d.z, R[1] * d.x + R[4] * d.y + R[7] * d.z,
            R[2] * d.x + R[5] * d.y + R[8] * d.z);
}

/* earliest vertex-triangle candidate of world vertex (W0 at ts, W1 at te)
 * against body triangle A of the particle with frames (R0, X0) at ts and
 * (R1, X1) at te; INFINITY if none */
static double vt_candidate(vec3 W0, vec3 W1, const double R0[9], const double X0[3], const double R1[9],
                           const double X1[3], const vec3 A[3], double eps, double ts, double te) {
  vec3 P0 = rel_pos(R0, X0, W0), P1 = rel_pos(R1, X1, W1), q;
  double best = INFINITY;
  if (sqrt(closest_pt_tri(P1, A[0], A[1], A[2], &q)) <= eps) best = te;
  vec3 nrm = cross(sub(A[1], A[0]), sub(A[2], A[0]));
  double h0 = dot(nrm, sub(P0, A[0])), h1 = dot(nrm, sub(P1, A[0]));
  if ((h0 > 0.0 && h1 < 0.0) || (h0 < 0.0 && h1 > 0.0)) {
    double s = h0 / (h0 - h1);
    vec3 Ps = axpy(P0, sub(P1, P0), s);
    double t = ts + s * (te - ts);
    if (sqrt(closest_pt_tri(Ps, A[0], A[1], A[2], &q)) <= eps && t < best) best = t;
  }
  return best;
}

static void narrowing_one(job *J, int64_t k) {
  int64_t i = J->pairs[2 * k], j = J->pairs[2 * k + 1];
  const double *s = J->state;
  int64_t n = J->n;
  double eps = eps_pair(s, n, i, j);
  double ts = pair_start(s, J->is_static, n, i, j), T = pair_span(s, J->is_static, n, i, j);
  pair_eval e;
  memset(&e, 0, sizeof e);
  eval_pair(s, n, J->tri_off, J->tris, J->n_tris, i, j, ts, 0, &e);
  int iters = 0;
  if (sqrt(e.d2min) <= eps) {
    J->t_coll[k] = ts + T;
    J->status[k] = 1;
    J->tri_ab[2 * k] = e.a;
    J->tri_ab[2 * k + 1] = e.b;
    if (J->n_evals) J->n_evals[k] = 0;
    return;
  }
  int64_t na = J->tri_off[i + 1] - J->tri_off[i], nb = J->tri_off[j + 1] - J->tri_off[j];
  /* body-frame triangles (float32 values promoted exactly) */
  vec3 *BA = (vec3 *)malloc(sizeof(vec3) * 3 * (size_t)(na > 0 ? na : 1));
  vec3 *BB = (vec3 *)malloc(sizeof(vec3) * 3 * (size_t)(nb > 0 ? nb : 1));
  for (int64_t a = 0; a < na; ++a)
    for (int q = 0; q < 3; ++q) {
      const float *v = J->tris + ((size_t)q * (size_t)J->n_tris + (size_t)(J->tri_off[i] + a)) * 4;
      BA[3 * a + q] = mk((double)v[0], (double)v[1], (double)v[2]);
    }
  for (int64_t b = 0; b < nb; ++b)
    for (int q = 0; q < 3; ++q) {
      const float *v = J->tris + ((size_t)q * (size_t)J->n_tris + (size_t)(J->tri_off[j] + b)) * 4;
      BB[3 * b + q] = mk((double)v[0], (double)v[1], (double)v[2]);
    }
  double RA0[9], XA0[3], RB0[9], XB0[3];
  demo_pose(s, n, i, ts, RA0, XA0);
  demo_pose(s, n, j, ts, RB0, XB0);
  vec3 *WA0 = world_verts(s, n, J->tri_off, J->tris, J->n_tris, i, ts);
  vec3 *WB0 = world_verts(s, n, J->tri_off, J->tris, J->n_tris, j, ts);
  double w = J->tol * T, te = ts + T;
  int found = 0;
  int32_t ta = -1, tb = -1;
  for (;;) {
    double tm = ts + 0.5 * (te - ts);
    double RA1[9], XA1[3], RB1[9], XB1[3];
    demo_pose(s, n, i, te, RA1, XA1);
    demo_pose(s, n, j, te, RB1, XB1);
    vec3 *WA1 = world_verts(s, n, J->tri_off, J->tris, J->n_tris, i, te);
    vec3 *WB1 = world_verts(s, n, J->tri_off, J->tris, J->n_tris, j, te);
    vec3 *WAm = world_verts(s, n, J->tri_off, J->tris, J->n_tris, i, tm);
    vec3 *WBm = world_verts(s, n, J->tri_off, J->tris, J->n_tris, j, tm);
    double best = INFINITY;
    int32_t ba = -1, bb = -1;
    for (int64_t a = 0; a < na; ++a)
      for (int64_t b = 0; b < nb; ++b) {
        double tab = INFINITY, t;
        /* vertices of a against triangle b (frame of j), then of b against a */
        for (int q = 0; q < 3; ++q) {
          t = vt_candidate(WA0[3 * a + q], WA1[3 * a + q], RB0, XB0, RB1, XB1, BB + 3 * b, eps, ts, te);
          if (t < tab) tab = t;
        }
        for (int q = 0; q < 3; ++q) {
          t = vt_candidate(WB0[3 * b + q], WB1[3 * b + q], RA0, XA0, RA1, XA1, BA + 3 * a, eps, ts, te);
          if (t < tab) tab = t;
        }
        /* edge pairs at the middle and the end of the span */
        for (int p = 0; p < 3; ++p)
          for (int q = 0; q < 3; ++q) {
            vec3 c1, c2;
            int p1 = p == 2 ? 0 : p + 1, q1 = q == 2 ? 0 : q + 1;
            if (tm < tab && sqrt(seg_seg(WAm[3 * a + p], WAm[3 * a + p1], WBm[3 * b + q], WBm[3 * b + q1], &c1,
                                         &c2)) <= eps)
              tab = tm;
            if (te < tab && sqrt(seg_seg(WA1[3 * a + p], WA1[3 * a + p1], WB1[3 * b + q], WB1[3 * b + q1], &c1,
                                         &c2)) <= eps)
              tab = te;
          }
        if (tab < best) {
          best = tab;
          ba = (int32_t)a;
          bb = (int32_t)b;
        }
      }
    free(WA1);
    free(WB1);
    free(WAm);
    free(WBm);
    ++iters;
    if (best == INFINITY) break;
    found = 1;
    ta = ba;
    tb = bb;
    if (!(best < te - w) || iters >= NARROW_MAX_ITER) break;
    te = best + w;
  }
  free(WA0);
  free(WB0);
  free(BA);
  free(BB);
  J->t_coll[k] = found ? te : ts + T;
  J->status[k] = found ? 2 : 0;
  J->tri_ab[2 * k] = found ? ta : -1;
  J->tri_ab[2 * k + 1] = found ? tb : -1;
  if (J->n_evals) J->n_evals[k] = iters;
}

static void *worker(void *arg) {
  job *J = (job *)arg;
  for (;;) {
    int64_t k = (int64_t)atomic_fetch_add(&J->next, 1);
    if (k >= J->m) break;
    if (J->mode == 0) {
      int64_t i = J->pairs[2 * k], j = J->pairs[2 * k + 1];
      double t = J->t_eval ? J->t_eval[k] : pair_start(J->state, J->is_static, J->n, i, j);
      eval_pair(J->state, J->n, J->tri_off, J->tris, J->n_tris, i, j, t, 1, &J->ev[k]);
    } else if (J->mode == 1) {
      collision_time_one(J, k);
    } else {
      narrowing_one(J, k);
    }
  }
  return NULL;
}

static void run_job(job *J, int n_threads) {
  atomic_init(&J->next, 0);
  if (n_threads <= 1 || J->m <= 1) {
    worker(J);
    return;
  }
  if (n_threads > 256) n_threads = 256;
  pthread_t th[256];
  int started = 0;
  for (int k = 0; k < n_threads; ++k)
    if (pthread_create(&th[k], NULL, worker, J) == 0) ++started;
  if (started == 0) worker(J);
  for (int k = 0; k < started; ++k) pthread_join(th[k], NULL);
}

int64_t demo_narrow_phase(const double *state, const uint8_t *is_static, int64_t n, const int64_t *tri_off,
                          const float *tris, int64_t n_tris, const int32_t *pairs, int64_t m,
                          const double *t_eval, double *dmin, double *pa, double *pb, int32_t *tri_ab,
                          uint8_t *flag, int32_t *contacts, double *geom, int64_t cap, int n_threads) {
  job J;
  memset(&J, 0, sizeof J);
  J.state = state;
  J.is_static = is_static;
  J.n = n;
  J.tri_off = tri_off;
  J.tris = tris;
  J.n_tris = n_tris;
  J.pairs = pairs;
  J.m = m;
  J.t_eval = t_eval;
  J.mode = 0;
  J.ev = (pair_eval *)calloc((size_t)(m > 0 ? m : 1), sizeof(pair_eval));
  run_job(&J, n_threads);
  int64_t nc = 0;
  for (int64_t k = 0; k < m; ++k) {
    pair_eval *e = &J.ev[k];
    int64_t i = pairs[2 * k], j = pairs[2 * k + 1];
    double d = sqrt(e->d2min);
    dmin[k] = d;
    st(pa + 3 * k, e->pa);
    st(pb + 3 * k, e->pb);
    tri_ab[2 * k] = e->a;
    tri_ab[2 * k + 1] = e->b;
    flag[k] = (uint8_t)(d <= eps_pair(state, n, i, j));
    for (int64_t c = 0; c < e->nc; ++c, ++nc) {
      if (nc < cap) {
        contacts[3 * nc] = (int32_t)k;
        contacts[3 * nc + 1] = e->cab[2 * c];
        contacts[3 * nc + 2] = e->cab[2 * c + 1];
        memcpy(geom + 7 * nc, e->cgeom + 7 * c, 7 * sizeof(double));
      }
    }
    free(e->cab);
    free(e->cgeom);
  }
  free(J.ev);
  return nc;
}

void demo_collision_times(const double *state, const uint8_t *is_static, int64_t n, const int64_t *tri_off,
                          const float *tris, int64_t n_tris, const int32_t *pairs, int64_t m, int K,
                          double tol, double *t_coll, uint8_t *status, int32_t *tri_ab, int32_t *n_evals,
                          int n_threads) {
  job J;
  memset(&J, 0, sizeof J);
  J.state = state;
  J.is_static = is_static;
  J.n = n;
  J.tri_off = tri_off;
  J.tris = tris;
  J.n_tris = n_tris;
  J.pairs = pairs;
  J.m = m;
  J.K = K;
  J.tol = tol;
  J.t_coll = t_coll;
  J.status = status;
  J.tri_ab = tri_ab;
  J.n_evals = n_evals;
  J.mode = 1;
  run_job(&J, n_threads);
}

void demo_collision_times_narrowing(const double *state, const uint8_t *is_static, int64_t n,
                                    const int64_t *tri_off,
                                    const float *tris, int64_t n_tris, const int32_t *pairs, int64_t m,
                                    double tol, double *t_coll, uint8_t *status, int32_t *tri_ab,
                                    int32_t *n_iter, int n_threads) {
  job J;
  memset(&J, 0, sizeof J);
  J.state = state;
  J.is_static = is_static;
  J.n = n;
  J.tri_off = tri_off;
  J.tris = tris;
  J.n_tris = n_tris;
  J.pairs = pairs;
  J.m = m;
  J.tol = tol;
  J.t_coll = t_coll;
  J.status = status;
  J.tri_ab = tri_ab;
  J.n_evals = n_iter;
  J.mode = 2;
  run_job(&J, n_threads);
}

/* ------------------------------------------------------------------------ */
/* Clusters (paper Section 3: the pruned graph splits into disconnected
 * subgraphs; each is a cluster; static objects take no part).  The paper
 * relabels nodes iteratively from their neighbours until nothing changes;
 * read as minimum-label propagation: every non-static node starts with its
 * own index and repeatedly takes the minimum label over itself and its
 * neighbours, until a sweep changes nothing.  The fixpoint labels every
 * connected component with its smallest index. */
int64_t demo_clusters(int64_t n, const int32_t *edges, int64_t e, const uint8_t *is_static,
                      int32_t *id) {
  for (int64_t i = 0; i < n; ++i) id[i] = (is_static && is_static[i]) ? -1 : (int32_t)i;
  int changed = 1;
  while (changed) {
    changed = 0;
    for (int64_t k = 0; k < e; ++k) {
      int32_t u = edges[2 * k], v = edges[2 * k + 1];
      if (id[u] < 0 || id[v] < 0) continue;
      int32_t lo = id[u] < id[v] ? id[u] : id[v];
      if (id[u] != lo) { id[u] = lo; changed = 1; }
      if (id[v] != lo) { id[v] = lo; changed = 1; }
    }
  }
  int64_t c = 0;
  for (int64_t i = 0; i < n; ++i)
    if (id[i] == (int32_t)i) ++c;
  return c;
}

/* ------------------------------------------------------------------------ */
/* One sweep of the local-time-stepping cycle (paper Section 2.2, the
 * substeps of a time step; Section 3, particle step sizes; Section 4, cluster
 * consolidation; Section 5, time step size; cluster masking and snapshot
 * roll-over).  Each substep below is written out as the paper orders them;
 * the collision itself (the impulse solver) is outside the method's contact
 * detection and replaced by a stand-in update (velocities zeroed on contact,
 * gravity otherwise).
 *
 * cur[DEMO_NFIELDS][n]: current snapshot (x, v, q, w, t_cur; dt is written);
 * old[DEMO_NFIELDS][n]: old snapshot (x, q, t_cur fields) with the v and w
 * that carried the particle from it to the current snapshot (other fields
 * unused).  Static particles are never changed. */
int64_t demo_lts_sweep(double *cur, double *old, const uint8_t *is_static, int64_t n, const int64_t *tri_off,
                       const float *tris, int64_t n_tris, int K, double tol, double dt_max, double alpha,
                       const double gravity[3], int zero_on_contact, int hose, int32_t *pairs_out, int64_t cap,
                       uint8_t *status_out, double *t_coll_out, int32_t *cluster_id, uint8_t *active,
                       double *t_global, int64_t *rollbacks, int64_t *rollbacks_before_old, int n_threads,
                       double *consolidated) {
  /* 1. particle step sizes (Eq. "damped particle time step size"): a creeping
   *    average of the previous step, capped by the global span; no history
   *    (t_old = t_cur) gives the global span */
  for (int64_t p = 0; p < n; ++p) {
    if (is_st(is_static, p)) continue;
    double tc = cur[FTCUR * n + p], to = old[FTCUR * n + p];
    double d = tc > to ? alpha * (tc - to) : dt_max;
    cur[FDT * n + p] = d < dt_max ? d : dt_max;
  }
  /* 2. candidates over each particle's own step; with the hose check, pairs
   *    of two moving particles whose space-time hoses do not meet are
   *    dropped (Section 3, Check 2) */
  int64_t m = demo_broad_phase(cur, is_static, n, tri_off, tris, n_tris, pairs_out, 0);
  int32_t *pairs = (int32_t *)malloc(sizeof(int32_t) * 2 * (size_t)(m > 0 ? m : 1));
  demo_broad_phase(cur, is_static, n, tri_off, tris, n_tris, pairs, m);
  if (hose) {
    int64_t kept = 0;
    for (int64_t k = 0; k < m; ++k) {
      int64_t i = pairs[2 * k], j = pairs[2 * k + 1];
      if (!is_st(is_static, j) && !hose_meet(cur, old, n, i, j)) continue;
      pairs[2 * kept] = pairs[2 * k];
      pairs[2 * kept + 1] = pairs[2 * k + 1];
      ++kept;
    }
    m = kept;
  }
  /* 3. clusters of the candidate graph */
  demo_clusters(n, pairs, m, is_static, cluster_id);
  /* 4. consolidation: every member of a cluster rolls back to the cluster's
   *    earliest time stamp by interpolating between its old and current
   *    snapshots (free flight from the old snapshot with the velocities that
   *    produced the current one: linear in x, the slerp geodesic in q), and
   *    takes the cluster's step (the smallest member step, Eq. "cluster time
   *    step") */
  double *tmin = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  double *dtc = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  double *tnew = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  for (int64_t c = 0; c < n; ++c) tmin[c] = dtc[c] = INFINITY;
  for (int64_t p = 0; p < n; ++p) {
    if (is_st(is_static, p)) continue;
    int64_t c = cluster_id[p];
    if (cur[FTCUR * n + p] < tmin[c]) tmin[c] = cur[FTCUR * n + p];
    if (cur[FDT * n + p] < dtc[c]) dtc[c] = cur[FDT * n + p];
  }
  int64_t rb = 0, rb_bad = 0;
  for (int64_t p = 0; p < n; ++p) {
    if (is_st(is_static, p)) continue;
    int64_t c = cluster_id[p];
    if (cur[FTCUR * n + p] > tmin[c]) {
      double Q[4], X[3];
      pose_q(old, n, p, tmin[c], Q, X);
      ++rb;
      if (tmin[c] < old[FTCUR * n + p]) ++rb_bad; /* would contradict Theorem "valid snapshots" */
      cur[FX * n + p] = X[0];
      cur[FY * n + p] = X[1];
      cur[FZ * n + p] = X[2];
      cur[FQW * n + p] = Q[0];
      cur[FQX * n + p] = Q[1];
      cur[FQY * n + p] = Q[2];
      cur[FQZ * n + p] = Q[3];
      cur[FTCUR * n + p] = tmin[c];
    }
    cur[FDT * n + p] = dtc[c];
  }
  /* the snapshot the collision times (and a narrow phase at the pair start)
   * are evaluated on */
  if (consolidated) memcpy(consolidated, cur, sizeof(double) * DEMO_NFIELDS * (size_t)n);
  /* 5. collision time stamps of every candidate pair over the (now common)
   *    cluster interval */
  uint8_t *status = (uint8_t *)malloc((size_t)(m > 0 ? m : 1));
  double *tcol = (double *)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
  int32_t *tab = (int32_t *)malloc(sizeof(int32_t) * 2 * (size_t)(m > 0 ? m : 1));
  demo_collision_times(cur, is_static, n, tri_off, tris, n_tris, pairs, m, K, tol, tcol, status, tab, NULL,
                       n_threads);
  /* 6. effective step of a cluster: its new time stamp is the earliest proper
   *    collision of its pairs, else the end of its interval (statuses 0 and 1
   *    do not constrain it) */
  for (int64_t c = 0; c < n; ++c) tnew[c] = INFINITY;
  for (int64_t p = 0; p < n; ++p) {
    if (is_st(is_static, p)) continue;
    int64_t c = cluster_id[p];
    if (c == p) tnew[c] = tmin[c] + dtc[c];
  }
  for (int64_t k = 0; k < m; ++k) {
    int64_t c = cluster_id[pairs[2 * k]];
    if (status[k] == 2 && tcol[k] < tnew[c]) tnew[c] = tcol[k];
  }
  /* 7. masking (Eq. "cluster masking: min collision time"): the earliest new
   *    time stamp over all clusters; clusters whose time stamp lies beyond it
   *    do not advance */
  double tg = INFINITY;
  for (int64_t c = 0; c < n; ++c)
    if (tnew[c] < tg) tg = tnew[c];
  *t_global = tg;
  /* 8. stand-in for the collision update: particles in contact at the end of
   *    the step (touching at its start, or attaining the cluster's collision
   *    time) stop; the others accelerate under gravity */
  uint8_t *touch = (uint8_t *)calloc((size_t)(n > 0 ? n : 1), 1);
  for (int64_t k = 0; k < m; ++k) {
    int64_t i = pairs[2 * k], j = pairs[2 * k + 1];
    int64_t c = cluster_id[i];
    if (status[k] == 1 || (status[k] == 2 && tcol[k] == tnew[c])) {
      touch[i] = 1;
      if (!is_st(is_static, j)) touch[j] = 1;
    }
  }
  /* 9. advance the active clusters to their new time stamp and roll the
   *    snapshots over: old <- current, current <- new */
  for (int64_t p = 0; p < n; ++p) {
    active[p] = 0;
    if (is_st(is_static, p)) continue;
    int64_t c = cluster_id[p];
    if (!(tmin[c] <= tg)) continue;
    active[p] = 1;
    double h = tnew[c] - cur[FTCUR * n + p];
    const int f[] = {FX, FY, FZ, FVX, FVY, FVZ, FQW, FQX, FQY, FQZ, FWX, FWY, FWZ, FTCUR};
    for (int q = 0; q < 14; ++q) old[f[q] * n + p] = cur[f[q] * n + p];
    double Q[4], X[3];
    pose_q(old, n, p, tnew[c], Q, X);
    cur[FX * n + p] = X[0];
    cur[FY * n + p] = X[1];
    cur[FZ * n + p] = X[2];
    cur[FQW * n + p] = Q[0];
    cur[FQX * n + p] = Q[1];
    cur[FQY * n + p] = Q[2];
    cur[FQZ * n + p] = Q[3];
    cur[FTCUR * n + p] = tnew[c];
    if (zero_on_contact && touch[p]) {
      for (int q = 3; q < 6; ++q) cur[q * n + p] = 0.0;
      for (int q = 10; q < 13; ++q) cur[q * n + p] = 0.0;
    } else {
      cur[FVX * n + p] = cur[FVX * n + p] + gravity[0] * h;
      cur[FVY * n + p] = cur[FVY * n + p] + gravity[1] * h;
      cur[FVZ * n + p] = cur[FVZ * n + p] + gravity[2] * h;
    }
  }
  for (int64_t k = 0; k < m && k < cap; ++k) {
    pairs_out[2 * k] = pairs[2 * k];
    pairs_out[2 * k + 1] = pairs[2 * k + 1];
    status_out[k] = status[k];
    t_coll_out[k] = tcol[k];
  }
  *rollbacks = rb;
  *rollbacks_before_old = rb_bad;
  free(pairs);
  free(tmin);
  free(dtc);
  free(tnew);
  free(status);
  free(tcol);
  free(tab);
  free(touch);
  return m;
}
