/*
 * dem_probe.h -- measurement support of the contact-detection library (not
 * part of the paper's method; the paper has no counterpart).  The benchmark
 * states its roofline fractions against these measured figures.
 */
#ifndef DEM_PROBE_H
#define DEM_PROBE_H

#include "dem.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Arithmetic peak of the current GPU from fused multiply-add chains: 8 blocks
 * of 256 threads per SM, each thread running 8 independent chains of `iters`
 * FMAs in FP32 (precision 0) or FP64 (precision 1), timed with CUDA events on
 * `stream` (best of 3 runs after one warm-up run).  *flops_per_s (host) =
 * 2 x FMAs / seconds.  Allocates no device memory; synchronises the stream.
 * DEM_ERR_ARG for a null output, iters <= 0 or another precision. */
dem_status dem_probe_fma_peak(int32_t precision, int32_t iters, void *stream, double *flops_per_s);

/* FP32 operations of the triangle-pair distance exactly as the pair kernel's
 * FP32 filter evaluates it (the crossing tests, then the six vertex-triangle
 * and nine edge-edge closest-point computations of the Voronoi-region and
 * clamped segment algorithms, then the square root), counted per input pair:
 * every add, subtract, multiply, divide and square root counts 1, so a fused
 * multiply-add counts 2.  tri: device float [n][18] (triangle a's three
 * vertices x y z, then triangle b's); ops: device int64 [n] (caller-owned).
 * Asynchronous on `stream`; serialise concurrent calls (they share a
 * per-thread counter array inside the library). */
dem_status dem_count_dist_flops(const float *tri, int64_t n, int64_t *ops, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* DEM_PROBE_H */
