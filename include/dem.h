/*
 * dem.h -- C-ABI of the GB300 (sm_103a) space-time contact-detection library
 * for rigid particles represented by triangulated meshes, after Noble &
 * Weinzierl, "Parallel local time stepping for rigid bodies represented by
 * triangulated meshes" (arXiv:2309.15417).
 *
 * Four calls make up one detection step: candidate pairs (broad phase),
 * triangle-pair distances and contacts (narrow phase), collision time stamps,
 * and clusters (connected components).
 *
 * Conventions shared by every call:
 *  - Every array argument is a DEVICE pointer owned by the caller, unless the
 *    comment says "host".  The library never frees caller memory; it owns only
 *    the scratch it allocates in dem_create().
 *  - Calls are asynchronous on `stream` (a cudaStream_t passed as void*; NULL
 *    = legacy default stream).  No call synchronises except dem_check() and
 *    dem_get_stats().  No call allocates device memory, so a sequence of calls
 *    can be captured into a CUDA graph.
 *  - Argument errors (null pointers, sizes beyond the capacities given to
 *    dem_create, misaligned triangle buffers) are detected on the host and
 *    returned immediately as DEM_ERR_ARG / DEM_ERR_CAPACITY; nothing is
 *    launched then.
 *  - Conditions found on the device (an output capacity exceeded, an index
 *    out of range, a non-finite input, a bounded wait that ran out) set a
 *    sticky error word in the context.  dem_check() synchronises the stream,
 *    returns the most severe such condition as a status (index, non-finite,
 *    capacity, timeout, in that order) and clears the word.  Kernels never
 *    trap and never read out of bounds: a bad index skips its pair.
 *  - Every call is wrapped in an NVTX range named after it (visible in
 *    profilers; a no-op otherwise).
 *  - Counts that kernels produce are written to device int64 scalars, and the
 *    consuming calls read them on the device (`n_pairs` below), so a whole
 *    step runs without host round trips.
 *  - Pairs (and edges) are int32 [M][2] (i, j interleaved), with i < j.
 *
 * Particle data (paper Section 2.1, "Physical model"; Section 5, "Geometric
 * model"): see dem_particles.
 */
#ifndef DEM_H
#define DEM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dem_ctx dem_ctx;

typedef enum {
  DEM_OK = 0,
  DEM_ERR_ARG = -1,       /* invalid argument (detected on the host) */
  DEM_ERR_CAPACITY = -2,  /* a size exceeds a capacity (host or device) */
  DEM_ERR_CUDA = -3,      /* a CUDA runtime call failed; see dem_last_error */
  DEM_ERR_NONFINITE = -4, /* a particle's state or a triangle vertex is NaN or infinite; the
                             pairs and particles concerned are skipped, other outputs stay valid */
  DEM_ERR_TIMEOUT = -5,   /* a bounded device wait ran out.  Every output of the launch that
                             reported it, and of every later launch on the same stream up to the
                             dem_check that returns it, is invalid and must be discarded (a CTA
                             that gave up may have left a tile copy unfinished).  dem_last_error
                             says whether the wait for that copy to land also ran out. */
  DEM_ERR_INDEX = -6      /* a device kernel met an index out of range (pairs, tri_off) and
                             skipped the access */
} dem_status;

/* Collision-time procedure of dem_collision_times, dem_detect and
 * dem_lts_sweep. */
enum {
  DEM_CTIME_SAMPLES = 0,  /* K uniform samples, then bisection to bisect_tol * T */
  DEM_CTIME_NARROWING = 1 /* the paper's narrowing (Section 5): vertex-triangle on the straight
                             relative path (end point, plane crossing), edge-edge at the middle and
                             end of the span; the span narrows to the earliest contact plus the
                             widening bisect_tol * T while that shortens it (at most 64 times);
                             binary64 throughout on the GPU */
};

/* Arithmetic of the triangle-pair distances. */
enum {
  DEM_PREC_FP32_FIXUP = 0, /* FP32 bulk, FP64 recomputation within the FP32 error bound */
  DEM_PREC_FP64 = 1        /* every distance in FP64 */
};

/* Fields of the particle state, field-major: state[f * n + p]. */
#define DEM_NFIELDS 17
enum {
  DEM_F_X = 0, DEM_F_Y, DEM_F_Z,        /* centre of mass at t_cur (world) */
  DEM_F_VX, DEM_F_VY, DEM_F_VZ,         /* linear velocity (world) */
  DEM_F_QW, DEM_F_QX, DEM_F_QY, DEM_F_QZ, /* unit quaternion body -> world at t_cur */
  DEM_F_WX, DEM_F_WY, DEM_F_WZ,         /* angular velocity (world frame) */
  DEM_F_TCUR,                           /* the particle's current time stamp */
  DEM_F_DT,                             /* the particle's own step size */
  DEM_F_EPS,                            /* halo width eps(p) */
  DEM_F_RADIUS                          /* bound on |body-frame vertex| */
};

/* Particles (paper Section 2.1): rigid triangle meshes with a halo, moving in
 * free flight with constant linear velocity v and constant world-frame angular
 * velocity w between snapshots.  The pose at time t is
 *   X(t) = x + v (t - t_cur),  q(t) = dq(w, t - t_cur) (x) q,
 * dq the rotation by angle |w| (t - t_cur) about w.
 * Triangles (Section 5, "Geometric model") are given in the body frame as a
 * float4 soup: tris[(s * n_tris + k) * 4 + c], vertex slot s = 0..2, triangle
 * k, coordinate c = x,y,z (the 4th float is ignored).  Particle p owns
 * triangles tri_off[p] .. tri_off[p+1]-1. */
typedef struct {
  int64_t n;                /* number of particles */
  const double *state;      /* device [DEM_NFIELDS][n] */
  const uint8_t *is_static; /* device [n], nonzero = static object; NULL = none */
  const int64_t *tri_off;   /* device [n+1], non-decreasing, tri_off[0] = 0 */
  const float *tris;        /* device float4 [3][n_tris], 16-byte aligned */
  int64_t n_tris;           /* total triangles = tri_off[n] */
} dem_particles;

typedef struct {
  int32_t K;            /* collision-time samples per pair interval (>= 1; 0 -> 8) */
  double bisect_tol;    /* bisection stops at bracket <= bisect_tol * T (0 -> 1e-3) */
  int32_t precision;    /* DEM_PREC_* */
  int32_t ctime_method; /* DEM_CTIME_* */
  int64_t max_particles; /* capacity: particles per call (0 -> 65536) */
  int64_t max_pairs;     /* capacity: pairs / edges per call (0 -> 1<<20) */
  int64_t max_contacts;  /* capacity: contact staging per narrow-phase call (0 -> 1<<20) */
  int64_t max_triangles; /* capacity: n_tris per call (0 -> 1280 * max_particles); sizes the
                            bounding spheres of the 320-triangle tiles of large meshes */
  int64_t list_spill;    /* collision times: triangle pairs per persistent CTA that the pair-interval
                            list (the triangle pairs that can meet within a pair's interval) keeps in
                            global memory beyond the 512 held in shared memory (0 -> 8192; a longer
                            list makes that pair's evaluations visit every triangle pair, culled) */
} dem_config;

/* Outputs of dem_narrow_phase.  Per pair k (M = pair count):
 *   dmin[k]        minimum triangle-pair distance (FP64)
 *   pa[3k..], pb[3k..]  its closest points on particle i and j (world, FP64)
 *   tri_ab[2k..]   (a, b): the closest triangle pair, indices local to each
 *                  particle, smallest (a, b) among equal distances; -1 if a
 *                  particle has no triangles
 *   flag[k]        1 iff dmin <= eps_i + eps_j
 *   dmin32[k]      optional (NULL to skip): the pair minimum as computed in
 *                  FP32 before any FP64 recomputation (FP32 mode); dmin in
 *                  FP64 mode
 * Contacts: every triangle pair with distance <= eps_i + eps_j, sorted by
 * (pair, a, b): contacts[3c..] = (pair index k, a, b) int32,
 * contact_geom[7c..] = (d, pa.xyz, pb.xyz) FP64 world.  *n_contacts (device)
 * receives the total; only min(total, contact_cap) are written.  When the
 * context's contact staging (max_contacts) overflows, dem_check reports
 * DEM_ERR_CAPACITY and *n_contacts is a capacity that suffices for a re-call
 * (the FP32 mode stages candidates before deciding them in binary64, so this
 * can exceed the final count). */
typedef struct {
  double *dmin;
  double *pa;
  double *pb;
  int32_t *tri_ab;
  uint8_t *flag;
  float *dmin32;
  int32_t *contacts;
  double *contact_geom;
  int64_t contact_cap;
  int64_t *n_contacts;
} dem_narrow_out;

/* Device counters, summed since the last reset. */
typedef struct {
  int64_t sphere_tests;     /* triangle-pair bounding-sphere tests */
  int64_t group_tests;      /* triangle-group bounding-sphere tests */
  int64_t dist_fp32;        /* triangle-pair distances in FP32 */
  int64_t dist_fp64;        /* triangle-pair distances in FP64 */
  int64_t pair_evals;       /* pair-distance evaluations (decisions + minima) */
  int64_t method_checks;    /* sum over the method's evaluations of T_i * T_j */
  int64_t bisect_steps;     /* bisection steps */
  int64_t contacts;         /* contacts found */
  int64_t pairs_done;       /* pairs processed */
  int64_t kernel_launches;  /* kernels launched by this context (host-side count) */
  int64_t tile_pairs;       /* 320 x 320-triangle tile pairs scanned (not culled by tile spheres) */
  int64_t rollbacks;        /* local time stepping: particles rolled back by consolidation */
  int64_t rollbacks_before_old; /* ... of which to before their old snapshot (0 if the theorem holds) */
  int64_t advances;         /* local time stepping: particle advances (particle-steps) */
  int64_t cta_busy_ns;      /* pair kernel: sum over its CTAs of the time from start to the last pair */
  int64_t cta_busy_ns_max;  /* ... the largest such time (mean / max = the launch's load balance) */
  int64_t ctas;             /* ... CTAs counted */
  int64_t reserved[1];
} dem_stats;

/* Create a context: validates and copies *cfg, allocates scratch for the
 * capacities it names.  Returns DEM_ERR_CUDA if allocation fails. */
dem_status dem_create(const dem_config *cfg, dem_ctx **out);

/* Destroy a context and free its scratch (NULL is a no-op). */
void dem_destroy(dem_ctx *ctx);

/* Message of the last host-side error of ctx (never NULL). */
const char *dem_last_error(const dem_ctx *ctx);

/* Broad phase (paper Section 3, "Broad phase collision detection to identify
 * clusters", and the pair interval of Eq. "max time span between two
 * particles"): the candidate pairs c(i, j) = true.  Each moving particle is
 * extruded over its own step in free flight: swept sphere centre
 * m = x + v dt/2, radius rho = (radius + eps) + |v| dt/2; two moving
 * particles i < j are a candidate iff |m_i - m_j|^2 <= (rho_i + rho_j)^2
 * (binary64).  A static particle s (Section 3, "Static geometric objects")
 * is represented by the axis-aligned box of its world vertices at its t_cur,
 * widened by eps_s; a moving p and s are a candidate iff p's swept sphere
 * meets that box (binary64), written (p, s): the static member is always
 * second.  Two static particles never pair.  Moving particles are binned in a
 * uniform hashed cell grid of cell size >= 2 max rho (over moving particles)
 * and every moving particle tests every static box; the result equals the
 * brute-force set.
 * Output: pairs [cap][2] sorted by (first, second), *n_pairs (device) =
 * number of candidates; if it exceeds cap only cap are written and
 * dem_check() returns DEM_ERR_CAPACITY. */
dem_status dem_build_candidates(dem_ctx *ctx, const dem_particles *P, int32_t *pairs, int64_t cap,
                                int64_t *n_pairs, void *stream);

/* Narrow phase (paper Section 5, "Geometric model", Definition of a contact
 * point, and "Collision time detection": triangle distance = minimum over
 * vertex-triangle and edge-edge distances, 0 for intersecting triangles).
 * Evaluates every triangle pair of every pair at time t_eval[k] (NULL: the
 * pair's start time min(t_cur_i, t_cur_j)).
 * pairs: [max_pairs][2]; n_pairs: device count (NULL: max_pairs pairs); the
 * call processes min(*n_pairs, max_pairs) pairs. */
dem_status dem_narrow_phase(dem_ctx *ctx, const dem_particles *P, const int32_t *pairs,
                            int64_t max_pairs, const int64_t *n_pairs, const double *t_eval,
                            const dem_narrow_out *out, void *stream);

/* Collision time stamps (paper Section 5, "Time step size calculation": case
 * distinction, narrowing and widening; interval of Eq. "max time span between
 * two particles").  Pair interval [ts, ts + T], ts = min(t_cur_i, t_cur_j),
 * T = min(dt_i, dt_j); with a static member (no step of its own, Section 3)
 * the moving member's t_cur and dt.  f(t) = minimum triangle-pair distance
 * at t.  (The narrow phase with t_eval = NULL evaluates at this ts.)
 *   f(ts) <= eps_pair                  -> status 1, t_coll = ts + T
 *   first k in 1..K: f(ts + T k/K) <= eps_pair -> bisection on
 *     [ts + T (k-1)/K, ts + T k/K] until the bracket is <= tol T,
 *     t_coll = the upper end                                -> status 2
 *   otherwise                          -> status 0, t_coll = ts + T
 * tri_ab[2k..]: the closest triangle pair at t_coll for status 1 (at ts) and
 * 2; -1 for status 0.  Every decision f(t) <= eps_pair equals the binary64
 * decision of the definition. */
dem_status dem_collision_times(dem_ctx *ctx, const dem_particles *P, const int32_t *pairs,
                               int64_t max_pairs, const int64_t *n_pairs, double *t_coll,
                               uint8_t *status, int32_t *tri_ab, void *stream);

/* Narrow phase at the pair start and collision times in one launch: the
 * outputs of dem_narrow_phase(..., t_eval = NULL, out) and of
 * dem_collision_times(..., t_coll, status, tri_ab), identical to the two
 * separate calls.  The evaluation at the pair start serves both (the paper's
 * narrow collision and time-step-size phases, Section 5, evaluated at the
 * same snapshot). */
dem_status dem_detect(dem_ctx *ctx, const dem_particles *P, const int32_t *pairs, int64_t max_pairs,
                      const int64_t *n_pairs, const dem_narrow_out *out, double *t_coll, uint8_t *status,
                      int32_t *tri_ab, void *stream);

/* Clusters (paper Section 3: the pruned graph's disconnected subgraphs are
 * the clusters; static objects take no part in the clustering).  Connected
 * components of the undirected graph over n particles given by edges
 * [max_edges][2] (count: device *n_edges, NULL = max_edges); edges with a
 * static endpoint are ignored.  cluster_id[i] = smallest particle index in
 * i's component, -1 for static particles; *n_clusters (device) = number of
 * components among non-static particles.  is_static may be NULL. */
dem_status dem_clusters(dem_ctx *ctx, int64_t n, const int32_t *edges, int64_t max_edges,
                        const int64_t *n_edges, const uint8_t *is_static, int32_t *cluster_id,
                        int64_t *n_clusters, void *stream);

/* Parameters of one local-time-stepping sweep. */
typedef struct {
  double dt_max;           /* the global admissible time span (> 0) */
  double alpha;            /* damping of the particle step (Section 3; the paper uses 2) */
  double gravity[3];       /* stand-in update: acceleration of particles not in contact */
  int32_t zero_on_contact; /* stand-in update: particles in contact stop (v = w = 0) */
  int32_t hose;            /* 1: candidates of two moving particles must also pass the space-time
                              hose test (Section 3, Check 2): bounding spheres (R + eps) on the
                              old -> current segment, then with the current velocity, overlapping
                              at some common time of the pair interval (binary64) */
} dem_lts_params;

/* Outputs of one sweep (caller-owned device arrays). */
typedef struct {
  int32_t *pairs;        /* [max_pairs][2] the sweep's candidate pairs */
  int64_t max_pairs;
  int64_t *n_pairs;      /* [1] */
  double *t_coll;        /* [max_pairs] collision time stamps of the pairs */
  uint8_t *status;       /* [max_pairs] their status (0, 1, 2) */
  int32_t *tri_ab;       /* [max_pairs][2] */
  int32_t *cluster_id;   /* [n] clusters of the candidate graph (-1: static) */
  int64_t *n_clusters;   /* [1] */
  uint8_t *active;       /* [n] 1 if the particle advanced in this sweep */
  double *t_global;      /* [1] earliest new time stamp over all clusters (the masking bound) */
  const dem_narrow_out *narrow; /* optional (NULL: none): the narrow phase of the sweep's pairs at
                                   their start time after consolidation (dem_narrow_phase's outputs,
                                   computed in the same launch as the collision times) */
} dem_lts_out;

/* One sweep of the local-time-stepping cycle (paper Section 2.2 substeps,
 * Sections 3-5).  In order, all on the stream, without host round trips:
 *  1. particle steps dt_p = min(alpha (t_cur - t_old), dt_max), dt_max when
 *     t_old = t_cur (Eq. "damped particle time step size"), written to cur;
 *  2. candidate pairs (dem_build_candidates; with prm->hose, moving pairs
 *     whose space-time hoses do not meet are dropped) and 3. their clusters;
 *  4. consolidation (Section 4): every member of a cluster goes back to the
 *     cluster's earliest t_cur by free flight from its old snapshot (the
 *     interpolation between the snapshots) and takes the cluster step (the
 *     smallest member step, Eq. "cluster time step");
 *  5. collision times of every pair (dem_collision_times; with out->narrow,
 *     dem_detect: also the narrow phase of every pair at its start time);
 *  6. each cluster's new time stamp: its earliest status-2 time, else
 *     t_min + step; 7. masking: t_global = the minimum over clusters;
 *     clusters with t_min > t_global do not advance;
 *  8. the others advance to their new time stamp in free flight and roll
 *     their snapshots over (old <- current, current <- new), with the
 *     stand-in for the collision update: particles in contact at the end of
 *     the step (status 1, or status 2 at the cluster's time) stop when
 *     zero_on_contact, the others gain gravity * (advanced time).
 * cur, old: device [DEM_NFIELDS][n] binary64, read and written; cur is the
 * current snapshot, old the previous one (x, q, t_cur fields) with the v, w
 * that carried the particle to cur; start a run with old = cur.  P gives the
 * geometry (n, is_static, tri_off, tris, n_tris); P->state must be NULL or
 * cur.  Static particles are never changed.  The results equal the oracle's
 * sweep bit for bit (every comparison and rounding is the binary64 one).
 * Errors: DEM_ERR_ARG for bad arguments, DEM_ERR_CAPACITY when
 * out->max_pairs exceeds the context's max_pairs; a device capacity overflow
 * is reported by dem_check. */
dem_status dem_lts_sweep(dem_ctx *ctx, const dem_particles *P, double *cur, double *old,
                         const dem_lts_params *prm, const dem_lts_out *out, void *stream);

/* Candidate pairs without any device allocation (no context needed).  The
 * paper has no counterpart: this is for callers that cannot allocate device
 * memory when they need candidates -- e.g. an application whose device memory
 * pool belongs to another framework, or a real-time loop in which an
 * allocation could block or fail.  Same predicate, output and order as
 * dem_build_candidates.  Scratch lives in a fixed device array inside the
 * library, sized for at most DEM_NOALLOC_MAX_PARTICLES particles (about
 * 5.3 MB, held on every GPU that loads the library until the process exits);
 * larger inputs return DEM_ERR_CAPACITY without launching anything.  No
 * cudaMalloc / cudaFree is called.  The first call on each device looks up
 * the array's device address (cudaGetSymbolAddress, with that device
 * current): make that first call before any stream capture.  All calls share
 * the array and it keeps the last call's contents; each call clears what must
 * start at zero, and calls that overlap on the GPU race, so serialise them.
 * Capacity overflow shows as *n_pairs > cap (only cap pairs are written).
 * Conditions met on the device (a bad static tri_off range, a non-finite
 * state, the capacity overflow) accumulate in an error word of the array
 * until dem_noalloc_check reads and clears it. */
#define DEM_NOALLOC_MAX_PARTICLES 16384
dem_status dem_build_candidates_noalloc(const dem_particles *P, int32_t *pairs, int64_t cap,
                                        int64_t *n_pairs, void *stream);

/* Error word of dem_build_candidates_noalloc (no context): synchronise
 * `stream`, return (and clear) the conditions its kernels met since the
 * previous dem_noalloc_check, as dem_check does for a context (DEM_ERR_INDEX
 * for a static particle whose tri_off range leaves the triangles,
 * DEM_ERR_NONFINITE for a non-finite state, DEM_ERR_CAPACITY when *n_pairs
 * exceeded cap).  Allocates nothing. */
dem_status dem_noalloc_check(void *stream);

/* Synchronise `stream`, return (and clear) the sticky device error as a
 * status (DEM_OK if none). */
dem_status dem_check(dem_ctx *ctx, void *stream);

/* Polls of the first bounded wait on a pair-kernel tile copy (default
 * DEM_WAIT_POLLS_DEFAULT).  polls = 0 makes every such wait run out at once
 * (the launch then reports DEM_ERR_TIMEOUT; the wait for the copy in flight
 * keeps its full length, so no copy is abandoned): a way to exercise the
 * timeout path without a fault.  DEM_ERR_ARG if polls is outside
 * [0, 2^32 - 1]. */
#define DEM_WAIT_POLLS_DEFAULT 4194304
dem_status dem_set_wait_polls(dem_ctx *ctx, int64_t polls);

/* Launch-group timing.  dem_trace(ctx, cap) with cap > 0 starts (or
 * restarts) recording: every later launch group of a call made with ctx takes
 * one record -- a CUDA event on the call's stream before and after the group,
 * recorded as event-record nodes when the stream is being captured into a
 * graph, so replays of the graph re-time them -- until cap records are taken.
 * cap = 0 stops and frees the events (do not do that while a graph captured
 * with the trace on may still be replayed).  Start the trace outside a
 * capture.  dem_trace_read synchronises the recorded events and copies
 * min(n, cap) records to the host arrays site[] (DEM_TR_*) and ms[]
 * (milliseconds between the two events, as of the latest launch or replay);
 * *n = records taken. */
enum {
  DEM_TR_BROAD = 0,   /* dem_build_candidates' kernels (and the sweep's broad phase) */
  DEM_TR_TILES = 1,   /* tile list and tile bounding spheres before a pair-kernel launch */
  DEM_TR_PAIRS = 2,   /* the pair kernel (narrow phase / collision times / both) */
  DEM_TR_CONTACTS = 3,/* contact offsets, scatter and sort after a narrow phase */
  DEM_TR_CLUSTERS = 4,/* connected components */
  DEM_TR_LTS = 5      /* the bookkeeping kernels of a local-time-stepping sweep */
};
dem_status dem_trace(dem_ctx *ctx, int32_t cap);
dem_status dem_trace_read(dem_ctx *ctx, int32_t *site /* host */, float *ms /* host */, int32_t cap,
                          int32_t *n /* host */);

/* Launch configuration of the pair kernel (one per precision and call kind,
 * held by the context).  Not part of the paper's method: it decides only the
 * schedule, never a result. */
typedef struct {
  int32_t ctas_per_sm; /* persistent CTAs per SM (0 = as many as fit, at most 4 in FP32, 2 in FP64) */
  int32_t wflush;      /* triangle pairs a warp collects before it evaluates them (32 or 64) */
  int32_t cost_order;  /* 1: pairs handed out costliest first (classes of T_i * T_j, a factor of two
                          each); 0: in index order */
  float ms;            /* dem_autotune: the chosen configuration's time (milliseconds) */
} dem_tuning;

enum { DEM_TUNE_NARROW = 0, DEM_TUNE_CTIME = 1, DEM_TUNE_DETECT = 2, DEM_TUNE_NARROWING = 3 };

/* Autotuner: times the call selected by `kind` (DEM_TUNE_NARROW:
 * dem_narrow_phase at the pair start; DEM_TUNE_CTIME / DEM_TUNE_NARROWING:
 * dem_collision_times by samples / by the narrowing; DEM_TUNE_DETECT:
 * dem_detect) in the context's precision on the given pairs for every
 * configuration of CTAs per SM {1, 2, 3, 4} x wflush {32, 64} x cost_order
 * {0, 1} (reps timed runs each after one warm-up run, CUDA events on
 * `stream`), keeps the fastest in the context for that kind and writes it to
 * *best (host, optional).  The outputs (out, t_coll, status, tri_ab, as the
 * tuned call takes them) hold the last run's results, which every
 * configuration computes identically.  Synchronises `stream`; do not call it
 * during a stream capture.  DEM_ERR_ARG for bad arguments. */
dem_status dem_autotune(dem_ctx *ctx, int32_t kind, const dem_particles *P, const int32_t *pairs, int64_t max_pairs,
                        const int64_t *n_pairs, const dem_narrow_out *out, double *t_coll, uint8_t *status,
                        int32_t *tri_ab, int32_t reps, dem_tuning *best, void *stream);

/* Read or set the configuration used for call kind `kind` (host struct). */
dem_status dem_get_tuning(dem_ctx *ctx, int32_t kind, dem_tuning *out);
dem_status dem_set_tuning(dem_ctx *ctx, int32_t kind, const dem_tuning *in);

/* Synchronise the device, copy the counters to host *out; reset them if
 * `reset` is nonzero. */
dem_status dem_get_stats(dem_ctx *ctx, dem_stats *out, int reset);

#ifdef __cplusplus
}
#endif
#endif /* DEM_H */
