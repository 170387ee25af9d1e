/*
 * dem_oracle.h -- plain FP64 CPU oracle for space-time contact detection
 * between rigid triangulated particles (Noble & Weinzierl, "Parallel local
 * time stepping for rigid bodies represented by triangulated meshes").
 *
 * TEST INFRASTRUCTURE ONLY.  This library is the slow, obviously correct
 * definition the CUDA library is checked against.  Only the tests, the smoke
 * check and the benchmark's CPU-baseline leg may load it; the product path
 * never calls it and shares no code with it.
 *
 * All arrays are host arrays.  Particle data use the same layout as the CUDA
 * library (field-major double state[DEMO_NFIELDS][n], float4 triangle soup
 * tris[3][n_tris][4], int64 tri_off[n+1]) because both are fed by the same
 * seeded generators.
 */
#ifndef DEM_ORACLE_H
#define DEM_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define DEMO_NFIELDS 17

/* Pose of particle p at time t: rotation matrix R (row-major) and centre X. */
void demo_pose(const double *state, int64_t n, int64_t p, double t, double R[9], double X[3]);

/* Triangle-triangle minimum distance and closest points (world frame).
 * A, B: 3 vertices x 3 coordinates each.  Returns d (not squared). */
double demo_tri_dist(const double A[9], const double B[9], double pa[3], double pb[3]);

/* Closest point on triangle T to point p; returns squared distance. */
double demo_closest_pt_tri(const double p[3], const double T[9], double q[3]);

/* Closest points of segments (p1,q1) and (p2,q2); returns squared distance. */
double demo_seg_seg(const double p1[3], const double q1[3], const double p2[3],
                    const double q2[3], double c1[3], double c2[3]);

/* Broad phase: every candidate pair.  Two moving particles i < j pair when
 * their swept halo spheres overlap; a moving particle p and a static
 * particle s pair, written (p, s), when p's swept sphere meets the box of
 * s's world vertices at t_cur widened by eps_s; two static particles never
 * pair.  Pairs sorted by (first, second); writes up to cap pairs (first,
 * second interleaved); returns the number of pairs. */
int64_t demo_broad_phase(const double *state, const uint8_t *is_static, int64_t n,
                         const int64_t *tri_off, const float *tris, int64_t n_tris,
                         int32_t *pairs, int64_t cap);

/* The candidate pairs that contain particle p alone (same predicates and
 * order, brute force over the other particles); returns the count. */
int64_t demo_broad_partners(const double *state, const uint8_t *is_static, int64_t n,
                            const int64_t *tri_off, const float *tris, int64_t n_tris, int64_t p,
                            int32_t *pairs, int64_t cap);

/* Pair interval of (i, j): ts = min(t_cur_i, t_cur_j), T = min(dt_i, dt_j);
 * when one member is static (is_static may be NULL) the interval is the
 * moving member's.
 *
 * Narrow phase over m pairs at times t_eval[k] (NULL: the pair's start time).
 * Per pair: dmin, pa[3], pb[3], tri_ab[2] (indices local to each particle),
 * flag (dmin <= eps_pair).  Contacts (all triangle pairs with d <= eps_pair)
 * in (pair, a, b) order: contacts[3*c] = (pair, a, b), geom[7*c] =
 * (d, pa, pb).  Returns the number of contacts (may exceed cap; then only
 * cap are written).  n_threads >= 1 splits the pairs over threads. */
int64_t demo_narrow_phase(const double *state, const uint8_t *is_static, int64_t n,
                          const int64_t *tri_off, const float *tris, int64_t n_tris,
                          const int32_t *pairs, int64_t m, const double *t_eval, double *dmin,
                          double *pa, double *pb, int32_t *tri_ab, uint8_t *flag,
                          int32_t *contacts, double *geom, int64_t cap, int n_threads);

/* Collision-time search over m pairs: K uniform samples, then bisection to
 * tol * T.  Outputs t_coll, status (0 none, 1 in contact at start, 2 proper),
 * tri_ab[2] of the closest triangles at the returned time (-1 for status 0),
 * n_evals (number of pair-distance evaluations the search made; may be NULL). */
void demo_collision_times(const double *state, const uint8_t *is_static, int64_t n,
                          const int64_t *tri_off, const float *tris, int64_t n_tris,
                          const int32_t *pairs, int64_t m, int K, double tol, double *t_coll,
                          uint8_t *status, int32_t *tri_ab, int32_t *n_evals, int n_threads);

/* The same interface with the paper's narrowing procedure (Section 5):
 * per triangle pair, vertex-triangle candidates on the straight relative
 * path of the vertex in the triangle particle's frame (its end and its
 * plane crossing) and edge-edge distances at the middle and end of the
 * search span; the span narrows to the earliest candidate plus the widening
 * tol * T while that shortens it (at most 64 iterations).  Status 1 as above;
 * status 2 with t = the final span end when a contact was found; else 0.
 * n_iter (may be NULL) = narrowing iterations per pair. */
void demo_collision_times_narrowing(const double *state, const uint8_t *is_static, int64_t n,
                                    const int64_t *tri_off, const float *tris, int64_t n_tris,
                                    const int32_t *pairs, int64_t m, double tol, double *t_coll,
                                    uint8_t *status, int32_t *tri_ab, int32_t *n_iter, int n_threads);

/* Connected components of the graph over n particles with e edges (pairs of
 * indices, interleaved); edges with a static endpoint are ignored.  id[i] =
 * smallest particle index in i's component, -1 for static particles.
 * Returns the number of components among non-static particles. */
int64_t demo_clusters(int64_t n, const int32_t *edges, int64_t e, const uint8_t *is_static,
                      int32_t *id);

/* Space-time hose test (Check 2 of the broad phase) of moving particles i
 * and j over their pair interval: bounding spheres (R + eps) on the old ->
 * current segment, then with the current velocity; 1 iff they overlap at some
 * common time.  cur/old as in demo_lts_sweep. */
int demo_hose_meet(const double *cur, const double *old, int64_t n, int64_t i, int64_t j);

/* One sweep of the local-time-stepping cycle (hose != 0: candidates of two
 * moving particles must also pass the hose test): particle steps
 * dt_p = min(alpha (t_cur - t_old), dt_max) (dt_max without history), broad
 * phase, clusters, consolidation (members roll back to the cluster's earliest
 * t_cur by free flight from the old snapshot, and take the smallest member
 * step), collision times, each cluster's new time stamp (earliest status-2
 * time, else t_min + dt), masking (clusters with t_min > the global minimum
 * of the new time stamps stay), advance and roll-over of the others, with the
 * stand-in update: v, w zeroed for particles in contact, else
 * v += gravity * step.  cur and old are [DEMO_NFIELDS][n] and are updated in
 * place (old holds x, q, t_cur of the old snapshot and the v, w that carried
 * the particle to cur).  Outputs: candidate pairs, their status and t_coll
 * (up to cap), cluster ids, active[n], the global minimum, the number of
 * roll-backs and of roll-backs to before a particle's old snapshot, and
 * (consolidated, [DEMO_NFIELDS][n], NULL to skip) the current snapshot after
 * the consolidation, on which the collision times are evaluated.  Returns
 * the number of candidate pairs. */
int64_t demo_lts_sweep(double *cur, double *old, const uint8_t *is_static, int64_t n,
                       const int64_t *tri_off, const float *tris, int64_t n_tris, int K, double tol,
                       double dt_max, double alpha, const double gravity[3], int zero_on_contact, int hose,
                       int32_t *pairs, int64_t cap, uint8_t *status, double *t_coll,
                       int32_t *cluster_id, uint8_t *active, double *t_global, int64_t *rollbacks,
                       int64_t *rollbacks_before_old, int n_threads, double *consolidated);

#ifdef __cplusplus
}
#endif
#endif
