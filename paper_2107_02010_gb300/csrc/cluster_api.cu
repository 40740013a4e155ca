// C-ABI entry points of the clustering step of the coarse-to-fine strategy
// (Section 2): cluster_grid and cluster_kmeans, and otgb_plan_free.
#include <cmath>
#include <cstring>
#include <vector>

#include "kmeans.cuh"
#include "multiscale.cuh"
#include "prims.cuh"
#include "solver.cuh"

using namespace otgb;

namespace otgb {

GridClusters grid_cluster(otgb_ctx *ctx, const std::string &tag, const float *x, int n, int D, float cell,
                          const float *d_lo_hint) {
    cudaStream_t st = ctx_stream(ctx);
    Workspace &ws = ctx_ws(ctx);
    GridClusters gc;
    float *lo = ws.get<float>(tag + ":lo", 128);
    if (d_lo_hint) {
        OTGB_CUDA_TRY(cudaMemcpyAsync(lo, d_lo_hint, 64 * sizeof(float), cudaMemcpyDeviceToDevice, st));
    } else {
        float *bpart = ws.get<float>("bpart", 64 * 2 * 64);
        bbox(x, n, D, D, lo, lo + 64, bpart, st);
    }
    uint32_t *keys = ws.get<uint32_t>(tag + ":keys", n);
    gc.perm = ws.get<int>(tag + ":perm", n);
    gc.offsets = ws.get<int>(tag + ":off", n + 1);
    gc.run = ws.get<int>(tag + ":run", n);
    int *bad = ws.get<int>("gbad", 1);
    int *ncl = ws.get<int>("gncl", 1);
    OTGB_CUDA_TRY(cudaMemsetAsync(bad, 0, sizeof(int), st));
    grid_keys(x, n, D, D, lo, cell, keys, bad, st);
    void *scr = ws.get("sort:scratch", radix_sort_scratch_bytes(n));
    radix_sort_pairs(keys, gc.perm, n, 30, scr, st);
    int *sscr = ws.get<int>("seg:scratch", scan_scratch_ints(n) + 2 * (size_t)n + 64);
    segment_keys(keys, n, gc.offsets, gc.run, ncl, sscr, st);
    int h[2] = {0, 0};
    OTGB_CUDA_TRY(cudaMemcpyAsync(&h[0], bad, sizeof(int), cudaMemcpyDeviceToHost, st));
    OTGB_CUDA_TRY(cudaMemcpyAsync(&h[1], ncl, sizeof(int), cudaMemcpyDeviceToHost, st));
    OTGB_CUDA_TRY(cudaStreamSynchronize(st));
    require(!(h[0] & 8), "cluster_grid: more than 1024 cells along an axis");
    gc.n_clusters = h[1];
    return gc;
}

}  // namespace otgb

extern "C" int cluster_grid(otgb_ctx *ctx, const float *x, const float *w, int N, int D, float cell,
                            int32_t *labels, int32_t *perm, int32_t *offsets, int *n_clusters, float *centroids) {
    if (!ctx) return fail(nullptr, Error{OTGB_EINVAL, "cluster_grid: null context"});
    try {
        ctx_set_device(ctx);
        require(x && labels && perm && offsets && n_clusters, "cluster_grid: null pointer argument");
        require(N >= 1, "cluster_grid: N must be >= 1");
        require(D >= 1 && D <= 3, "cluster_grid: D must be in [1, 3]");
        require(cell > 0.f && std::isfinite(cell), "cluster_grid: cell must be > 0");
        cudaStream_t st = ctx_stream(ctx);
        Workspace &ws = ctx_ws(ctx);
        int *bad = ws.get<int>("bad", 4);
        OTGB_CUDA_TRY(cudaMemsetAsync(bad, 0, sizeof(int), st));
        check_points(x, (size_t)N * D, bad, st);
        int hb = 0;
        OTGB_CUDA_TRY(cudaMemcpyAsync(&hb, bad, sizeof(int), cudaMemcpyDeviceToHost, st));
        OTGB_CUDA_TRY(cudaStreamSynchronize(st));
        require(!hb, "cluster_grid: points must be finite");
        GridClusters gc = grid_cluster(ctx, "cg", x, N, D, cell, nullptr);
        OTGB_CUDA_TRY(cudaMemcpyAsync(perm, gc.perm, sizeof(int) * N, cudaMemcpyDeviceToDevice, st));
        OTGB_CUDA_TRY(
            cudaMemcpyAsync(offsets, gc.offsets, sizeof(int) * (gc.n_clusters + 1), cudaMemcpyDeviceToDevice, st));
        scatter_labels(gc.perm, gc.run, N, labels, st);
        if (centroids) {
            float *pts = ws.get<float>("cg:pts", (size_t)N * 4);
            float *wsort = ws.get<float>("cg:w", N);
            float *zero = ws.get<float>("cg:zero", 64);
            float *mass = ws.get<float>("cg:mass", gc.n_clusters);
            float *rad = ws.get<float>("cg:rad", gc.n_clusters);
            OTGB_CUDA_TRY(cudaMemsetAsync(zero, 0, 64 * sizeof(float), st));
            pack_points(x, w, gc.perm, N, D, zero, pts, nullptr, wsort, st);
            cluster_stats(pts, 4, D, wsort, gc.offsets, gc.n_clusters, centroids, D, mass, rad, nullptr, st);
        }
        OTGB_CUDA_TRY(cudaStreamSynchronize(st));
        *n_clusters = gc.n_clusters;
        return OTGB_OK;
    } catch (const Error &e) {
        return fail(ctx, e);
    }
}

extern "C" int cluster_kmeans(otgb_ctx *ctx, const float *x, const float *w, int N, int D, int K, int iters,
                              unsigned long long seed, const float *init, int32_t *labels, float *centroids,
                              int32_t *perm, int32_t *offsets) {
    if (!ctx) return fail(nullptr, Error{OTGB_EINVAL, "cluster_kmeans: null context"});
    try {
        ctx_set_device(ctx);
        require(x && labels && centroids && perm && offsets, "cluster_kmeans: null pointer argument");
        require(N >= 1, "cluster_kmeans: N must be >= 1");
        require(D >= 1 && D <= 64, "cluster_kmeans: D must be in [1, 64]");
        require(K >= 1 && K <= N, "cluster_kmeans: K must be in [1, N]");
        require(iters >= 0, "cluster_kmeans: iters must be >= 0");
        KmeansResult r = kmeans(ctx, "km", x, w, N, D, K, iters, seed, init);
        cudaStream_t st = ctx_stream(ctx);
        OTGB_CUDA_TRY(cudaMemcpyAsync(labels, r.labels, sizeof(int) * N, cudaMemcpyDeviceToDevice, st));
        OTGB_CUDA_TRY(cudaMemcpyAsync(perm, r.perm, sizeof(int) * N, cudaMemcpyDeviceToDevice, st));
        OTGB_CUDA_TRY(cudaMemcpyAsync(offsets, r.offsets, sizeof(int) * (K + 1), cudaMemcpyDeviceToDevice, st));
        OTGB_CUDA_TRY(cudaMemcpy2DAsync(centroids, sizeof(float) * D, r.centroids, sizeof(float) * r.cstride,
                                        sizeof(float) * D, K, cudaMemcpyDeviceToDevice, st));
        OTGB_CUDA_TRY(cudaStreamSynchronize(st));
        return OTGB_OK;
    } catch (const Error &e) {
        return fail(ctx, e);
    }
}

extern "C" void otgb_plan_free(otgb_plan *plan) { delete plan; }
