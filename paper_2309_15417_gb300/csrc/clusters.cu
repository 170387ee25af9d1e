// clusters.cu -- connected components of the candidate (or contact) graph
// (paper Section 3: the pruned graph's disconnected subgraphs are the
// clusters; static objects are left out of the clustering).
//
// Lock-free union-find: every non-static particle starts as its own root; an
// edge (u, v) links the larger of the two roots under the smaller one with
// compare-and-swap, retrying when another thread relinked a root in between.
// A root is only ever linked under a smaller index, so parent[x] <= x and the
// final root of each component is its smallest particle index -- the same
// label as the paper's iterative relabelling reaches at its fixpoint.
// Integer work only; results are deterministic.
#include "internal.cuh"

namespace dem {

namespace {

__global__ void k_cc_init(int64_t n, const uint8_t *is_static, int32_t *parent) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    parent[i] = (is_static && is_static[i]) ? -1 : int32_t(i);
}

__device__ __forceinline__ int32_t find_root(const int32_t *parent, int32_t x) {
  // parent pointers only decrease; a bounded walk (depth < n)
  for (int it = 0; it < (1 << 30); ++it) {
    const int32_t p = *(volatile const int32_t *)&parent[x];
    if (p == x) return x;
    x = p;
  }
  return x;
}

__global__ void k_cc_hook(int64_t n, const int32_t *edges, int64_t max_edges, const int64_t *n_edges,
                          int32_t *parent, uint32_t *err) {
  int64_t m = max_edges;
  if (n_edges) m = min(m, *n_edges);
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < m; k += (int64_t)gridDim.x * blockDim.x) {
    const int32_t u = edges[2 * k], v = edges[2 * k + 1];
    if (u < 0 || v < 0 || u >= n || v >= n) {
      set_err(err, ERR_INDEX);
      continue;
    }
    if (parent[u] < 0 || parent[v] < 0) continue;  // static endpoint
    bool done = false;
    for (int it = 0; it < (1 << 20) && !done; ++it) {
      int32_t ru = find_root(parent, u), rv = find_root(parent, v);
      if (ru == rv) {
        done = true;
        break;
      }
      if (ru > rv) {
        const int32_t t = ru;
        ru = rv;
        rv = t;
      }
      // link the larger root rv under the smaller root ru
      if (atomicCAS(&parent[rv], rv, ru) == rv) done = true;
    }
    if (!done) set_err(err, ERR_TIMEOUT);
  }
}

__global__ void k_cc_final(int64_t n, int32_t *parent, unsigned long long *count) {
  unsigned long long c = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t p = parent[i];
    if (p < 0) continue;
    const int32_t r = find_root(parent, int32_t(i));
    if (r == i) ++c;
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(count, c);
}

// flatten after counting (roots do not move any more)
__global__ void k_cc_flatten(int64_t n, int32_t *parent) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t p = parent[i];
    if (p < 0) continue;
    parent[i] = find_root(parent, int32_t(i));
  }
}

}  // namespace

cudaError_t launch_clusters(int64_t n, const int32_t *edges, int64_t max_edges, const int64_t *n_edges,
                            const uint8_t *is_static, int32_t *id, int64_t *n_clusters, Scratch &S,
                            cudaStream_t s) {
  cudaError_t e;
  if ((e = cudaMemsetAsync(n_clusters, 0, sizeof(int64_t), s)) != cudaSuccess) return e;
  if (n <= 0) return cudaSuccess;
  const int tb = 256;
  const unsigned g = (unsigned)((n + tb - 1) / tb);
  const int rec = trace_begin(S, TR_CLUSTERS, s);
  k_cc_init<<<g, tb, 0, s>>>(n, is_static, id);
  if (max_edges > 0) {
    const unsigned ge = (unsigned)((max_edges + tb - 1) / tb);
    k_cc_hook<<<ge, tb, 0, s>>>(n, edges, max_edges, n_edges, id, S.err);
    S.launches += 1;
  }
  S.launches += 3;
  k_cc_final<<<g, tb, 0, s>>>(n, id, reinterpret_cast<unsigned long long *>(n_clusters));
  k_cc_flatten<<<g, tb, 0, s>>>(n, id);
  trace_end(S, rec, s);
  return cudaGetLastError();
}

}  // namespace dem
