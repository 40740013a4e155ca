// Declarations of the data-parallel primitives (prims.cu, cluster.cu).
#pragma once

#include "otgb_internal.cuh"

namespace otgb {

// Bounding box of the first D coordinates of n points (stride floats apart).
// d_part: scratch of 64 * 2 * D floats.
void bbox(const float *x, int n, int D, int stride, float *d_lo, float *d_hi, float *d_part, cudaStream_t st);

// S of Eq. (6) in double from the four duals (internal order) and the weights;
// rho = +inf selects the balanced form.  d_part: scratch of 128 doubles.
void divergence_sum(const float *wa, const float *f, const float *aa, int N, const float *wb, const float *g,
                    const float *bb, int M, double eps, double rho, double *d_out, double *d_part,
                    cudaStream_t st);

// Translation step of the cross duals (unbalanced): c = (rho/2) log(<a, e^{-f/rho}> / <b, e^{-g/rho}>),
// f += c, g -= c, in place.  d_part: 64 double2; *d_c receives c (may be null).
void translate_duals(const float *wa, float *f, int N, const float *wb, float *g, int M, double rho, double2 *d_part,
                     double *d_c, cudaStream_t st);

size_t scan_scratch_ints(int n);
size_t scan_scratch_ints_level(int nb);
// Exclusive prefix sum of n ints; scratch of scan_scratch_ints(n) ints.
void exclusive_scan(const int *in, int *out, int n, int *scratch, cudaStream_t st);

size_t radix_sort_scratch_bytes(int n);
// Stable sort of keys (only the low nbits matter); vals receives the original
// position of each sorted key.  keys are sorted in place.
void radix_sort_pairs(uint32_t *keys, int *vals, int n, int nbits, void *scratch, cudaStream_t st);

void iota(int *v, int n, cudaStream_t st);

// Internal layout: D <= 3 -> float4 (x - c, log w); D > 3 -> D4 floats (x - c, 0-padded)
// and a separate log w.  perm (optional) gives the source index of each output row.
void pack_points(const float *x, const float *w, const int *perm, int n, int D, const float *d_center, float *out,
                 float *logw, float *w_sorted, cudaStream_t st);
void unpermute(const float *in, const int *perm, int n, float *out, cudaStream_t st);
void permute(const float *in, const int *perm, int n, float *out, cudaStream_t st);

// Validation helpers: flag bits in *d_bad (1: bad weight, 2: non-finite point, 4: non-finite value).
void check_weights(const float *w, int n, int *d_bad, double *d_mass_part, cudaStream_t st);
void check_points(const float *x, size_t n, int *d_bad, cudaStream_t st);
void check_finite(const float *v, int n, int *d_bad, cudaStream_t st);
// *d_out = max(*d_out, max_i |v_i|) as the bits of a non-negative float (zero it first).
void absmax(const float *v, int n, unsigned *d_out, cudaStream_t st);

// Per-cluster mass, weighted centroid (cstride floats per centroid; for D <= 3 and
// cstride = 4 the 4th float is log mass), radius (max distance to the centroid)
// and, when ssq is non-null, sum_i w_i |x_i - c|^2, from packed sorted points.
void cluster_stats(const float *pts, int stride, int D, const float *w_sorted, const int *off, int ncl, float *cent,
                   int cstride, float *mass, float *radius, float *ssq, cudaStream_t st);

// ---- clustering (cluster.cu) ----
// Grid keys: Morton code of floor((x - lo) / cell), single precision.  Sets bit 8 of
// *d_bad when a cell coordinate exceeds 1023.  Returns nothing; keys on device.
void grid_keys(const float *x, int n, int D, int stride, const float *d_lo, float cell, uint32_t *keys, int *d_bad,
               cudaStream_t st);
// From sorted keys: offsets of the runs of equal keys and the run index of each
// sorted position.  Writes *d_ncl.  scratch: scan_scratch_ints(n) + 2n ints.
void segment_keys(const uint32_t *sorted_keys, int n, int *offsets, int *run_of_pos, int *d_ncl, int *scratch,
                  cudaStream_t st);
// labels[perm[k]] = run_of_pos[k]
void scatter_labels(const int *perm, const int *run_of_pos, int n, int *labels, cudaStream_t st);

struct GridClusters {
    int *perm = nullptr;     // sorted position -> original index
    int *offsets = nullptr;  // n_clusters + 1
    int *run = nullptr;      // cluster of each sorted position
    int n_clusters = 0;
};
// Grid clustering of n points (stride D, caller layout): Morton keys of the
// cells of width `cell` anchored at the per-axis minimum (d_lo_hint when given),
// stable sort, runs of equal keys.  Synchronises the stream.
GridClusters grid_cluster(otgb_ctx *ctx, const std::string &tag, const float *x, int n, int D, float cell,
                          const float *d_lo_hint);

}  // namespace otgb
