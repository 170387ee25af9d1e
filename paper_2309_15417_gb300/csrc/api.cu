// api.cu -- the C-ABI entry points (include/dem.h): argument checks on the
// host, scratch ownership, launches on the caller's stream, sticky device
// error word and counters.
#include <cstdio>
#include <cstring>
#include <string>

#include <nvtx3/nvToolsExt.h>

#include "internal.cuh"

struct dem_ctx {
  dem_config cfg;
  dem::Scratch S;
  dem::Trace trace;
  int device;
  int num_sms;
  std::string last_error;
  void *allocs[48];
  int n_allocs;
};

static_assert(DEM_WAIT_POLLS_DEFAULT == dem::WAIT_POLLS_DEFAULT, "default wait polls");
static_assert(sizeof(dem_stats) == sizeof(int64_t) * dem::ST_N, "dem_stats mirrors the device counters");

namespace dem {

int trace_begin(Scratch &S, int site, cudaStream_t s) {
  Trace *t = S.trace;
  if (!t || t->n >= t->cap) return -1;
  const int r = t->n++;
  t->site[r] = site;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(s, &cs);
  // inside a capture the record becomes an event-record node of the graph
  if (cs == cudaStreamCaptureStatusActive)
    cudaEventRecordWithFlags(t->ev[2 * r], s, cudaEventRecordExternal);
  else
    cudaEventRecord(t->ev[2 * r], s);
  return r;
}

void trace_end(Scratch &S, int rec, cudaStream_t s) {
  Trace *t = S.trace;
  if (!t || rec < 0) return;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(s, &cs);
  if (cs == cudaStreamCaptureStatusActive)
    cudaEventRecordWithFlags(t->ev[2 * rec + 1], s, cudaEventRecordExternal);
  else
    cudaEventRecord(t->ev[2 * rec + 1], s);
}

}  // namespace dem

namespace {

// NVTX range around one C-ABI call
struct Range {
  explicit Range(const char *name) { nvtxRangePushA(name); }
  ~Range() { nvtxRangePop(); }
};

void trace_free(dem_ctx *c) {
  dem::Trace &t = c->trace;
  for (int q = 0; q < 2 * t.cap; ++q)
    if (t.ev[q]) cudaEventDestroy(t.ev[q]);
  delete[] t.ev;
  delete[] t.site;
  t = dem::Trace{};
  c->S.trace = nullptr;
}

dem_status fail(dem_ctx *c, dem_status st, const std::string &msg) {
  if (c) c->last_error = msg;
  return st;
}

dem_status cuda_fail(dem_ctx *c, cudaError_t e, const char *where) {
  return fail(c, DEM_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

template <class T>
bool alloc(dem_ctx *c, T **p, size_t count) {
  constexpr int max_allocs = int(sizeof(c->allocs) / sizeof(c->allocs[0]));
  if (c->n_allocs >= max_allocs) return false;
  const size_t bytes = count * sizeof(T) > 0 ? count * sizeof(T) : 16;
  void *q = nullptr;
  if (cudaMalloc(&q, bytes) != cudaSuccess) return false;
  if (cudaMemset(q, 0, bytes) != cudaSuccess) {
    cudaFree(q);
    return false;
  }
  c->allocs[c->n_allocs++] = q;
  *p = static_cast<T *>(q);
  return true;
}

int64_t pow2_at_least(int64_t v) {
  int64_t p = 1;
  while (p < v) p <<= 1;
  return p;
}

dem_status check_particles(dem_ctx *c, const dem_particles *P) {
  if (!P) return fail(c, DEM_ERR_ARG, "particles: null");
  if (P->n < 0) return fail(c, DEM_ERR_ARG, "particles: n < 0");
  if (P->n > c->S.cap_particles) return fail(c, DEM_ERR_CAPACITY, "particles: n exceeds max_particles");
  if (P->n > 0 && (!P->state || !P->tri_off)) return fail(c, DEM_ERR_ARG, "particles: null state or tri_off");
  if (P->n_tris < 0) return fail(c, DEM_ERR_ARG, "particles: n_tris < 0");
  if (P->n_tris > c->S.cap_triangles) return fail(c, DEM_ERR_CAPACITY, "particles: n_tris exceeds max_triangles");
  if (P->n_tris > 0 && !P->tris) return fail(c, DEM_ERR_ARG, "particles: null tris");
  if (reinterpret_cast<uintptr_t>(P->tris) % 16 != 0)
    return fail(c, DEM_ERR_ARG, "particles: tris must be 16-byte aligned (float4)");
  return DEM_OK;
}

}  // namespace

extern "C" {

dem_status dem_create(const dem_config *cfg, dem_ctx **out) {
  if (!out) return DEM_ERR_ARG;
  *out = nullptr;
  dem_ctx *c = new dem_ctx();
  c->n_allocs = 0;
  dem_config k{};
  if (cfg) k = *cfg;
  if (k.K == 0) k.K = 8;
  if (k.bisect_tol == 0.0) k.bisect_tol = 1e-3;
  if (k.max_particles == 0) k.max_particles = 65536;
  if (k.max_pairs == 0) k.max_pairs = 1 << 20;
  if (k.max_contacts == 0) k.max_contacts = 1 << 20;
  if (k.max_triangles == 0) k.max_triangles = 1280 * k.max_particles;
  if (k.list_spill == 0) k.list_spill = 8192;
  if (k.K < 1 || !(k.bisect_tol > 0.0) || (k.precision != DEM_PREC_FP32_FIXUP && k.precision != DEM_PREC_FP64) ||
      (k.ctime_method != DEM_CTIME_SAMPLES && k.ctime_method != DEM_CTIME_NARROWING) ||
      k.max_particles < 0 || k.max_pairs < 0 || k.max_contacts < 0 || k.max_triangles < 0 || k.list_spill < 0 ||
      k.list_spill > ((int64_t)1 << 24) ||
      k.max_triangles > ((int64_t)1 << 40) ||
      k.max_particles > (int64_t)(dem::SCAN_BLOCK * dem::SCAN_PART_CAP / 2) ||
      k.max_pairs > (int64_t)(dem::SCAN_BLOCK * dem::SCAN_PART_CAP) || k.max_contacts > ((int64_t)1 << 31) - 1) {
    delete c;
    return DEM_ERR_ARG;
  }
  c->cfg = k;
  cudaError_t e = cudaGetDevice(&c->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device);
  if (e != cudaSuccess) {
    delete c;
    return DEM_ERR_CUDA;
  }
  dem::Scratch &S = c->S;
  S.cap_particles = k.max_particles;
  S.table_size = pow2_at_least(2 * (k.max_particles > 512 ? k.max_particles : 512));
  S.cap_pairs = k.max_pairs;
  S.cap_contacts = k.max_contacts;
  S.cap_triangles = k.max_triangles;
  S.cap_tiles = k.max_triangles / dem::TILE_TRIS + k.max_particles + 1;
  const int64_t np = k.max_particles, nq = k.max_pairs, nc = k.max_contacts;
  bool ok = alloc(c, &S.err, 1) && alloc(c, &S.stats, dem::ST_N) && alloc(c, &S.work, 4) &&
            alloc(c, &S.scan_part, dem::SCAN_PART_CAP) && alloc(c, &S.tmp, 8) && alloc(c, &S.sph, np) &&
            alloc(c, &S.cell, np) && alloc(c, &S.bucket_cnt, S.table_size) &&
            alloc(c, &S.bucket_start, S.table_size) && alloc(c, &S.bucket_cur, S.table_size) &&
            alloc(c, &S.bucket_ids, np) && alloc(c, &S.bucket_sph, np) && alloc(c, &S.bucket_sph32, np) &&
            alloc(c, &S.bucket_cell, np) && alloc(c, &S.pcnt, np) && alloc(c, &S.poff, np) &&
            alloc(c, &S.pcache, (size_t)dem::PCACHE * (size_t)np) && alloc(c, &S.pcache_ok, np) &&
            alloc(c, &S.rho_max, 1) && alloc(c, &S.static_ids, np) && alloc(c, &S.n_static, 1) &&
            alloc(c, &S.spose, 12 * np) && alloc(c, &S.sbox, 6 * np) && alloc(c, &S.sbox32, 6 * np) && alloc(c, &S.st_keys, 3 * nc) && alloc(c, &S.st_geom, 7 * nc) &&
            alloc(c, &S.st_count, 1) && alloc(c, &S.pc, nq) && alloc(c, &S.po, nq) && alloc(c, &S.pcur, nq) &&
            alloc(c, &S.sidx, nc) && alloc(c, &S.tile_sph, S.cap_tiles) && alloc(c, &S.tile_box, 2 * S.cap_tiles) && alloc(c, &S.tile_list, S.cap_tiles) && alloc(c, &S.lts_tmin, np) &&
            alloc(c, &S.lts_step, np) && alloc(c, &S.lts_tnew, np) && alloc(c, &S.lts_tglob, 1) &&
            alloc(c, &S.lts_touch, np) && alloc(c, &S.order, nq) && alloc(c, &S.cost_bucket, nq) &&
            alloc(c, &S.cost_hist, 128) &&
            alloc(c, &S.ilg, (size_t)c->num_sms * dem::MAX_PAIR_CTAS_PER_SM * (size_t)k.list_spill);
  S.ilg_cap = k.list_spill;
  if (!ok) {
    dem_destroy(c);
    return DEM_ERR_CUDA;
  }
  *out = c;
  return DEM_OK;
}

void dem_destroy(dem_ctx *c) {
  if (!c) return;
  trace_free(c);
  for (int q = 0; q < c->n_allocs; ++q) cudaFree(c->allocs[q]);
  delete c;
}

const char *dem_last_error(const dem_ctx *c) {
  if (!c) return "null context";
  return c->last_error.c_str();
}

dem_status dem_build_candidates(dem_ctx *c, const dem_particles *P, int32_t *pairs, int64_t cap,
                                int64_t *n_pairs, void *stream) {
  Range range("dem_build_candidates");
  if (!c) return DEM_ERR_ARG;
  dem_status st = check_particles(c, P);
  if (st != DEM_OK) return st;
  if (!n_pairs || (cap > 0 && !pairs) || cap < 0) return fail(c, DEM_ERR_ARG, "build_candidates: bad output");
  cudaError_t e = dem::launch_broad(*P, pairs, cap, n_pairs, c->S, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(c, e, "build_candidates");
  return DEM_OK;
}

dem_status dem_narrow_phase(dem_ctx *c, const dem_particles *P, const int32_t *pairs, int64_t max_pairs,
                            const int64_t *n_pairs, const double *t_eval, const dem_narrow_out *out,
                            void *stream) {
  Range range("dem_narrow_phase");
  if (!c) return DEM_ERR_ARG;
  dem_status st = check_particles(c, P);
  if (st != DEM_OK) return st;
  if (max_pairs < 0 || (max_pairs > 0 && !pairs)) return fail(c, DEM_ERR_ARG, "narrow_phase: bad pairs");
  if (max_pairs > c->S.cap_pairs) return fail(c, DEM_ERR_CAPACITY, "narrow_phase: max_pairs exceeds capacity");
  if (!out || !out->n_contacts || out->contact_cap < 0 ||
      (max_pairs > 0 && (!out->dmin || !out->pa || !out->pb || !out->tri_ab || !out->flag)) ||
      (out->contact_cap > 0 && (!out->contacts || !out->contact_geom)))
    return fail(c, DEM_ERR_ARG, "narrow_phase: bad outputs");
  cudaError_t e = dem::launch_narrow(c->cfg.precision, *P, pairs, max_pairs, n_pairs, t_eval, *out, c->S,
                                     c->num_sms, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(c, e, "narrow_phase");
  return DEM_OK;
}

dem_status dem_collision_times(dem_ctx *c, const dem_particles *P, const int32_t *pairs, int64_t max_pairs,
                               const int64_t *n_pairs, double *t_coll, uint8_t *status, int32_t *tri_ab,
                               void *stream) {
  Range range("dem_collision_times");
  if (!c) return DEM_ERR_ARG;
  dem_status st = check_particles(c, P);
  if (st != DEM_OK) return st;
  if (max_pairs < 0 || (max_pairs > 0 && (!pairs || !t_coll || !status || !tri_ab)))
    return fail(c, DEM_ERR_ARG, "collision_times: bad arguments");
  if (max_pairs > c->S.cap_pairs) return fail(c, DEM_ERR_CAPACITY, "collision_times: max_pairs exceeds capacity");
  cudaError_t e = dem::launch_ctime(c->cfg.precision, c->cfg.ctime_method, *P, pairs, max_pairs, n_pairs, c->cfg.K,
                                    c->cfg.bisect_tol,
                                    t_coll, status, tri_ab, c->S, c->num_sms, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(c, e, "collision_times");
  return DEM_OK;
}

dem_status dem_detect(dem_ctx *c, const dem_particles *P, const int32_t *pairs, int64_t max_pairs,
                      const int64_t *n_pairs, const dem_narrow_out *out, double *t_coll, uint8_t *status,
                      int32_t *tri_ab, void *stream) {
  Range range("dem_detect");
  if (!c) return DEM_ERR_ARG;
  dem_status st = check_particles(c, P);
  if (st != DEM_OK) return st;
  if (max_pairs < 0 || (max_pairs > 0 && (!pairs || !t_coll || !status || !tri_ab)))
    return fail(c, DEM_ERR_ARG, "detect: bad pairs or collision-time outputs");
  if (max_pairs > c->S.cap_pairs) return fail(c, DEM_ERR_CAPACITY, "detect: max_pairs exceeds capacity");
  if (!out || !out->n_contacts || out->contact_cap < 0 ||
      (max_pairs > 0 && (!out->dmin || !out->pa || !out->pb || !out->tri_ab || !out->flag)) ||
      (out->contact_cap > 0 && (!out->contacts || !out->contact_geom)))
    return fail(c, DEM_ERR_ARG, "detect: bad narrow-phase outputs");
  cudaError_t e;
  if (c->cfg.ctime_method == DEM_CTIME_NARROWING) {
    // the narrowing has no fused form: the two calls, same outputs
    e = dem::launch_narrow(c->cfg.precision, *P, pairs, max_pairs, n_pairs, nullptr, *out, c->S, c->num_sms,
                           static_cast<cudaStream_t>(stream));
    if (e == cudaSuccess)
      e = dem::launch_ctime(c->cfg.precision, c->cfg.ctime_method, *P, pairs, max_pairs, n_pairs, c->cfg.K,
                            c->cfg.bisect_tol, t_coll, status, tri_ab, c->S, c->num_sms,
                            static_cast<cudaStream_t>(stream));
  } else {
    e = dem::launch_detect(c->cfg.precision, *P, pairs, max_pairs, n_pairs, *out, c->cfg.K, c->cfg.bisect_tol,
                           t_coll, status, tri_ab, c->S, c->num_sms, static_cast<cudaStream_t>(stream));
  }
  if (e != cudaSuccess) return cuda_fail(c, e, "detect");
  return DEM_OK;
}

dem_status dem_clusters(dem_ctx *c, int64_t n, const int32_t *edges, int64_t max_edges, const int64_t *n_edges,
                        const uint8_t *is_static, int32_t *cluster_id, int64_t *n_clusters, void *stream) {
  Range range("dem_clusters");
  if (!c) return DEM_ERR_ARG;
  if (n < 0 || max_edges < 0 || (max_edges > 0 && !edges) || (n > 0 && !cluster_id) || !n_clusters)
    return fail(c, DEM_ERR_ARG, "clusters: bad arguments");
  if (n > (int64_t)INT32_MAX) return fail(c, DEM_ERR_CAPACITY, "clusters: n exceeds int32 ids");
  cudaError_t e = dem::launch_clusters(n, edges, max_edges, n_edges, is_static, cluster_id, n_clusters, c->S,
                                       static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(c, e, "clusters");
  return DEM_OK;
}

dem_status dem_lts_sweep(dem_ctx *c, const dem_particles *P, double *cur, double *old, const dem_lts_params *prm,
                         const dem_lts_out *out, void *stream) {
  Range range("dem_lts_sweep");
  if (!c) return DEM_ERR_ARG;
  if (!P || !prm || !out) return fail(c, DEM_ERR_ARG, "lts_sweep: null argument");
  if (P->state && P->state != cur) return fail(c, DEM_ERR_ARG, "lts_sweep: P->state must be NULL or cur");
  dem_particles G = *P;
  G.state = cur;
  dem_status st = check_particles(c, &G);
  if (st != DEM_OK) return st;
  if (P->n > 0 && (!cur || !old || !out->cluster_id || !out->active))
    return fail(c, DEM_ERR_ARG, "lts_sweep: null state or per-particle output");
  if (!out->n_pairs || !out->n_clusters || !out->t_global || out->max_pairs < 0 ||
      (out->max_pairs > 0 && (!out->pairs || !out->t_coll || !out->status || !out->tri_ab)))
    return fail(c, DEM_ERR_ARG, "lts_sweep: bad outputs");
  if (out->max_pairs > c->S.cap_pairs) return fail(c, DEM_ERR_CAPACITY, "lts_sweep: max_pairs exceeds capacity");
  const dem_narrow_out *nw = out->narrow;
  if (nw && (!nw->n_contacts || nw->contact_cap < 0 ||
             (out->max_pairs > 0 && (!nw->dmin || !nw->pa || !nw->pb || !nw->tri_ab || !nw->flag)) ||
             (nw->contact_cap > 0 && (!nw->contacts || !nw->contact_geom))))
    return fail(c, DEM_ERR_ARG, "lts_sweep: bad narrow-phase outputs");
  if (!(prm->dt_max > 0.0) || !(prm->alpha > 0.0)) return fail(c, DEM_ERR_ARG, "lts_sweep: dt_max, alpha > 0");
  cudaError_t e = dem::launch_lts(c->cfg.precision, c->cfg.ctime_method, c->cfg.K, c->cfg.bisect_tol, G, cur, old, *prm, *out, c->S,
                                  c->num_sms, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(c, e, "lts_sweep");
  return DEM_OK;
}

dem_status dem_check(dem_ctx *c, void *stream) {
  Range range("dem_check");
  if (!c) return DEM_ERR_ARG;
  cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(c, e, "check: stream");
  uint32_t bits = 0;
  e = cudaMemcpy(&bits, c->S.err, sizeof(bits), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(c, e, "check: read error word");
  if (!bits) return DEM_OK;
  e = cudaMemset(c->S.err, 0, sizeof(uint32_t));
  if (e != cudaSuccess) return cuda_fail(c, e, "check: clear error word");
  if (bits & dem::ERR_INDEX) return fail(c, DEM_ERR_INDEX, "device: index out of range");
  if (bits & dem::ERR_NONFINITE) return fail(c, DEM_ERR_NONFINITE, "device: non-finite state or vertex");
  if (bits & dem::ERR_CAPACITY) return fail(c, DEM_ERR_CAPACITY, "device: output capacity exceeded");
  if (bits & dem::ERR_DRAIN)
    return fail(c, DEM_ERR_TIMEOUT, "device: bounded wait ran out, and so did the wait for the copy in flight");
  return fail(c, DEM_ERR_TIMEOUT, "device: bounded wait ran out (the copy in flight landed)");
}

dem_status dem_get_tuning(dem_ctx *c, int32_t kind, dem_tuning *out) {
  if (!c || !out || kind < 0 || kind >= dem::N_MODES) return DEM_ERR_ARG;
  const dem::Tune &t = c->S.tune[c->cfg.precision][kind];
  out->ctas_per_sm = t.ctas_per_sm;
  out->wflush = t.wflush;
  out->cost_order = t.order;
  out->ms = 0.f;
  return DEM_OK;
}

dem_status dem_set_tuning(dem_ctx *c, int32_t kind, const dem_tuning *in) {
  if (!c || !in || kind < 0 || kind >= dem::N_MODES) return DEM_ERR_ARG;
  if (in->ctas_per_sm < 0 || in->ctas_per_sm > 16 || (in->wflush != 32 && in->wflush != 64) ||
      (in->cost_order != 0 && in->cost_order != 1))
    return fail(c, DEM_ERR_ARG, "set_tuning: out of range");
  dem::Tune &t = c->S.tune[c->cfg.precision][kind];
  t.ctas_per_sm = in->ctas_per_sm;
  t.wflush = in->wflush;
  t.order = in->cost_order;
  return DEM_OK;
}

dem_status dem_autotune(dem_ctx *c, int32_t kind, const dem_particles *P, const int32_t *pairs, int64_t max_pairs,
                        const int64_t *n_pairs, const dem_narrow_out *out, double *t_coll, uint8_t *status,
                        int32_t *tri_ab, int32_t reps, dem_tuning *best, void *stream) {
  if (!c) return DEM_ERR_ARG;
  Range range("dem_autotune");
  if (kind < 0 || kind >= dem::N_MODES || reps < 1) return fail(c, DEM_ERR_ARG, "autotune: bad kind or reps");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone)
    return fail(c, DEM_ERR_ARG, "autotune: stream is being captured");
  const int method = kind == DEM_TUNE_NARROWING ? DEM_CTIME_NARROWING : DEM_CTIME_SAMPLES;
  auto run = [&]() -> dem_status {
    if (kind == DEM_TUNE_NARROW) return dem_narrow_phase(c, P, pairs, max_pairs, n_pairs, nullptr, out, stream);
    if (kind == DEM_TUNE_DETECT) return dem_detect(c, P, pairs, max_pairs, n_pairs, out, t_coll, status, tri_ab, stream);
    const int keep = c->cfg.ctime_method;
    c->cfg.ctime_method = method;
    const dem_status st = dem_collision_times(c, P, pairs, max_pairs, n_pairs, t_coll, status, tri_ab, stream);
    c->cfg.ctime_method = keep;
    return st;
  };
  dem::Trace *tr = c->S.trace;
  c->S.trace = nullptr;  // the tuning runs take no trace records
  dem::Tune &t = c->S.tune[c->cfg.precision][kind];
  const dem::Tune saved = t;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    c->S.trace = tr;
    return fail(c, DEM_ERR_CUDA, "autotune: events");
  }
  dem::Tune best_t = saved;
  float best_ms = 3.0e38f;
  dem_status st = DEM_OK;
  for (int order = 0; order < 2 && st == DEM_OK; ++order)
    for (int wf = 32; wf <= 64 && st == DEM_OK; wf += 32)
      for (int cps = 1; cps <= 4 && st == DEM_OK; ++cps) {
        t.ctas_per_sm = cps;
        t.wflush = wf;
        t.order = order;
        float tot = 0.f;
        for (int r = 0; r <= reps && st == DEM_OK; ++r) {  // run 0 warms up
          cudaEventRecord(e0, s);
          st = run();
          cudaEventRecord(e1, s);
          if (st == DEM_OK && cudaEventSynchronize(e1) != cudaSuccess) st = DEM_ERR_CUDA;
          float ms = 0.f;
          if (st == DEM_OK) cudaEventElapsedTime(&ms, e0, e1);
          if (r > 0) tot += ms;
        }
        if (st == DEM_OK && tot / reps < best_ms) {
          best_ms = tot / reps;
          best_t = t;
        }
      }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  c->S.trace = tr;
  t = st == DEM_OK ? best_t : saved;
  if (st != DEM_OK) return st;
  if (best) {
    best->ctas_per_sm = t.ctas_per_sm;
    best->wflush = t.wflush;
    best->cost_order = t.order;
    best->ms = best_ms;
  }
  return DEM_OK;
}

dem_status dem_set_wait_polls(dem_ctx *c, int64_t polls) {
  if (!c) return DEM_ERR_ARG;
  if (polls < 0 || polls > (int64_t)UINT32_MAX) return fail(c, DEM_ERR_ARG, "set_wait_polls: out of range");
  c->S.wait_polls = polls == 0 ? 0u : (uint32_t)polls;
  return DEM_OK;
}

dem_status dem_trace(dem_ctx *c, int32_t capacity) {
  if (!c || capacity < 0) return DEM_ERR_ARG;
  if (capacity == 0) {
    trace_free(c);
    return DEM_OK;
  }
  dem::Trace &t = c->trace;
  if (t.cap != capacity) {
    trace_free(c);
    t.ev = new cudaEvent_t[2 * (size_t)capacity]();
    t.site = new int32_t[capacity]();
    t.cap = capacity;
    for (int q = 0; q < 2 * capacity; ++q) {
      cudaError_t e = cudaEventCreate(&t.ev[q]);
      if (e != cudaSuccess) {
        t.ev[q] = nullptr;
        trace_free(c);
        return cuda_fail(c, e, "trace: event");
      }
    }
  }
  t.n = 0;
  c->S.trace = &t;
  return DEM_OK;
}

dem_status dem_trace_read(dem_ctx *c, int32_t *site, float *ms, int32_t cap, int32_t *n) {
  if (!c || !n || cap < 0 || (cap > 0 && (!site || !ms))) return DEM_ERR_ARG;
  const dem::Trace &t = c->trace;
  *n = t.n;
  const int m = t.n < cap ? t.n : cap;
  for (int r = 0; r < m; ++r) {
    site[r] = t.site[r];
    cudaError_t e = cudaEventSynchronize(t.ev[2 * r + 1]);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms[r], t.ev[2 * r], t.ev[2 * r + 1]);
    if (e != cudaSuccess) return cuda_fail(c, e, "trace_read");
  }
  return DEM_OK;
}

dem_status dem_get_stats(dem_ctx *c, dem_stats *out, int reset) {
  Range range("dem_get_stats");
  if (!c || !out) return DEM_ERR_ARG;
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(c, e, "get_stats");
  unsigned long long v[dem::ST_N];
  e = cudaMemcpy(v, c->S.stats, sizeof(v), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(c, e, "get_stats: copy");
  std::memset(out, 0, sizeof(*out));
  int64_t *o = reinterpret_cast<int64_t *>(out);
  for (int q = 0; q < dem::ST_N && q < (int)(sizeof(dem_stats) / sizeof(int64_t)); ++q) o[q] = (int64_t)v[q];
  out->kernel_launches = c->S.launches;
  if (reset) {
    e = cudaMemset(c->S.stats, 0, sizeof(v));
    if (e != cudaSuccess) return cuda_fail(c, e, "get_stats: reset");
    c->S.launches = 0;
  }
  return DEM_OK;
}

}  // extern "C"
