// Weighted Lloyd K-means (kmeans.cu).
#pragma once

#include <string>
#include <vector>

#include "otgb_internal.cuh"

namespace otgb {

struct KmeansResult {
    float *centroids = nullptr;  // K x cstride
    int cstride = 0;
    int K = 0;
    int *labels = nullptr;       // caller order
    int *perm = nullptr;         // sorted position -> original index
    int *offsets = nullptr;      // K + 1 (empty clusters included)
    uint32_t *sorted_keys = nullptr;  // cluster of each sorted position
};

std::vector<int> sample_distinct(int n, int K, unsigned long long seed);
void kmeans_assign(const float *x, int n, int D, const float *cent, int K, int *labels, cudaStream_t st);
// x: n x D (caller layout), w optional.  init (optional): K x D device centroids.
// sample_max > 0 and n > sample_max: the Lloyd iterations run on every s-th
// point (s = ceil(n / sample_max)), then every point is assigned once to the
// resulting centroids; the labels, order and offsets cover all n points.
KmeansResult kmeans(otgb_ctx *ctx, const std::string &tag, const float *x, const float *w, int n, int D, int K,
                    int iters, unsigned long long seed, const float *init, int sample_max = 0);

}  // namespace otgb
