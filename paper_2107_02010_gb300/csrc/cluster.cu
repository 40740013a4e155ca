// Clustering for the coarse-to-fine strategy of Section 2: grid cells (D <= 3)
// and weighted Lloyd K-means, followed by a stable sort of the points by
// cluster (see prims.cu for the sort).
#include <cfloat>
#include <cmath>

#include "prims.cuh"

namespace otgb {
namespace {

__device__ __forceinline__ uint32_t spread3(uint32_t v) {
    // bit b of v (b < 10) moves to bit 3b
    v &= 0x3ffu;
    v = (v | (v << 16)) & 0x030000ffu;
    v = (v | (v << 8)) & 0x0300f00fu;
    v = (v | (v << 4)) & 0x030c30c3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}

__global__ void grid_keys_kernel(const float *x, int n, int D, int stride, const float *lo, float cell,
                                 uint32_t *keys, int *bad) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint32_t k = 0;
    for (int d = 0; d < D; ++d) {
        const float q = __fdiv_rn(__fsub_rn(x[(size_t)i * stride + d], lo[d]), cell);
        const float c = floorf(q);
        if (!(c <= 1023.0f)) {
            atomicOr(bad, 8);
            keys[i] = 0;
            return;
        }
        k |= spread3((uint32_t)c) << d;
    }
    keys[i] = k;
}

__global__ void seg_flags_kernel(const uint32_t *keys, int n, int *flags) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) flags[k] = (k == 0 || keys[k] != keys[k - 1]) ? 1 : 0;
}

__global__ void seg_finish_kernel(const int *flags, const int *excl, int n, int *offsets, int *run_of_pos,
                                  int *ncl) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int run = excl[k] + flags[k] - 1;
    run_of_pos[k] = run;
    if (flags[k]) offsets[run] = k;
    if (k == n - 1) {
        *ncl = run + 1;
        offsets[run + 1] = n;
    }
}

__global__ void scatter_labels_kernel(const int *perm, const int *run_of_pos, int n, int *labels) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) labels[perm[k]] = run_of_pos[k];
}

}  // namespace

void grid_keys(const float *x, int n, int D, int stride, const float *d_lo, float cell, uint32_t *keys, int *d_bad,
               cudaStream_t st) {
    grid_keys_kernel<<<(n + 255) / 256, 256, 0, st>>>(x, n, D, stride, d_lo, cell, keys, d_bad);
    OTGB_CHECK_LAUNCH();
}

void segment_keys(const uint32_t *sorted_keys, int n, int *offsets, int *run_of_pos, int *d_ncl, int *scratch,
                  cudaStream_t st) {
    int *flags = scratch, *excl = scratch + n, *scr = scratch + 2 * (size_t)n;
    seg_flags_kernel<<<(n + 255) / 256, 256, 0, st>>>(sorted_keys, n, flags);
    OTGB_CHECK_LAUNCH();
    exclusive_scan(flags, excl, n, scr, st);
    seg_finish_kernel<<<(n + 255) / 256, 256, 0, st>>>(flags, excl, n, offsets, run_of_pos, d_ncl);
    OTGB_CHECK_LAUNCH();
}

void scatter_labels(const int *perm, const int *run_of_pos, int n, int *labels, cudaStream_t st) {
    scatter_labels_kernel<<<(n + 255) / 256, 256, 0, st>>>(perm, run_of_pos, n, labels);
    OTGB_CHECK_LAUNCH();
}

}  // namespace otgb
