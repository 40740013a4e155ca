// Weighted Lloyd K-means, the "simple K-means" coarse subsampling of
// Section 2: seeded sample of K distinct points as initial centroids, then
// rounds of nearest-centroid assignment (lowest index on ties) and
// weighted-mean update (an empty cluster keeps its centroid), a final
// assignment, and a stable sort of the points by cluster.
#include <cfloat>
#include <cmath>
#include <unordered_set>
#include <vector>

#include "kmeans.cuh"
#include "prims.cuh"
#include "solver.cuh"

namespace otgb {
namespace {

constexpr int kAT = 256;   // threads
constexpr int kAR = 128;   // points per CTA
constexpr int kAC = 64;    // centroids per tile

// Nearest centroid by argmin_k (|c_k|^2 - 2 x.c_k): each thread keeps 8 points
// x 4 centroids of dot products, register-tiled like a GEMM.
struct AssignSmem {
    float xs[64][kAR];
    float cs[64][kAC];
    float cn[kAC];
    float bd[16][kAR];
    int bk[16][kAR];
};

__global__ void __launch_bounds__(kAT) kmeans_assign_kernel(const float *x, int n, int D, int D4, const float *cent,
                                                            int K, int *labels) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    AssignSmem &S = *reinterpret_cast<AssignSmem *>(smem_raw);
    const int t = threadIdx.x, r0 = blockIdx.x * kAR;
    for (int e = t; e < kAR * D4; e += kAT) {
        const int r = e / D4, k = e - r * D4;
        S.xs[k][r] = (r0 + r < n && k < D) ? x[(size_t)(r0 + r) * D + k] : 0.f;
    }
    const int tr = t >> 4, tc = t & 15;
    float best[8];
    int bidx[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) { best[i] = INFINITY; bidx[i] = 0x7fffffff; }
    for (int c0 = 0; c0 < K; c0 += kAC) {
        __syncthreads();
        for (int e = t; e < kAC * D4; e += kAT) {
            const int c = e / D4, k = e - c * D4;
            S.cs[k][c] = (c0 + c < K && k < D) ? cent[(size_t)(c0 + c) * D4 + k] : 0.f;
        }
        __syncthreads();
        if (t < kAC) {
            float acc = 0.f;
            for (int k = 0; k < D4; ++k) acc = fmaf(S.cs[k][t], S.cs[k][t], acc);
            S.cn[t] = (c0 + t < K) ? acc : INFINITY;
        }
        __syncthreads();
        float acc[8][4];
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
        for (int k = 0; k < D4; ++k) {
            const float4 xa = *reinterpret_cast<const float4 *>(&S.xs[k][tr * 8]);
            const float4 xb = *reinterpret_cast<const float4 *>(&S.xs[k][tr * 8 + 4]);
            const float4 cv = *reinterpret_cast<const float4 *>(&S.cs[k][tc * 4]);
            const float xv[8] = {xa.x, xa.y, xa.z, xa.w, xb.x, xb.y, xb.z, xb.w};
            const float cc[4] = {cv.x, cv.y, cv.z, cv.w};
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(xv[i], cc[j], acc[i][j]);
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int c = c0 + tc * 4 + j;
            const float cn = S.cn[tc * 4 + j];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const float d = fmaf(-2.f, acc[i][j], cn);
                if (d < best[i] || (d == best[i] && c < bidx[i])) { best[i] = d; bidx[i] = c; }
            }
        }
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) { S.bd[tc][tr * 8 + i] = best[i]; S.bk[tc][tr * 8 + i] = bidx[i]; }
    __syncthreads();
    if (t < kAR && r0 + t < n) {
        float b = S.bd[0][t];
        int k = S.bk[0][t];
        for (int q = 1; q < 16; ++q) {
            const float d = S.bd[q][t];
            const int kk = S.bk[q][t];
            if (d < b || (d == b && kk < k)) { b = d; k = kk; }
        }
        labels[r0 + t] = k;
    }
}

// every s-th row (and weight) of x: out row i = x row i s
__global__ void strided_rows_kernel(const float *x, const float *w, int D, int s, int ni, float *out, float *wout) {
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (size_t)ni * D) return;
    const size_t i = e / D, d = e - i * D;
    out[e] = x[i * (size_t)s * D + d];
    if (w && d == 0) wout[i] = w[i * (size_t)s];
}

// Weighted mean of each cluster from the points sorted by cluster: CTA k sums
// its cluster's rows in a fixed order (4 interleaved row groups, combined in a
// fixed tree), so the centroids do not depend on scheduling.  An empty cluster
// keeps its centroid.
__global__ void kmeans_segment_mean_kernel(const float *x, const float *w, int D, int D4, const int *perm,
                                           const int *off, float *cent) {
    __shared__ float ps[4][64];
    __shared__ float pm[4];
    const int k = blockIdx.x, t = threadIdx.x, d = t & 63, g = t >> 6;
    const int a = off[k], b = off[k + 1];
    float s = 0.f, m = 0.f;
    for (int i = a + g; i < b; i += 4) {
        const int src = perm[i];
        const float wi = w ? w[src] : 1.f;
        if (d < D) s = fmaf(wi, x[(size_t)src * D + d], s);
        m += wi;
    }
    ps[g][d] = s;
    if (d == 0) pm[g] = m;
    __syncthreads();
    if (g == 0 && d < D) {
        const float S = (ps[0][d] + ps[1][d]) + (ps[2][d] + ps[3][d]);
        const float M = (pm[0] + pm[1]) + (pm[2] + pm[3]);
        if (M > 0.f) cent[(size_t)k * D4 + d] = S / M;
    }
}

__global__ void gather_rows_kernel(const float *x, int D, const int *idx, int K, float *out, int D4) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= K * D4) return;
    const int k = e / D4, d = e - k * D4;
    out[e] = d < D ? x[(size_t)idx[k] * D + d] : 0.f;
}

__global__ void copy_rows_kernel(const float *src, int D, int K, float *out, int D4) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= K * D4) return;
    const int k = e / D4, d = e - k * D4;
    out[e] = d < D ? src[(size_t)k * D + d] : 0.f;
}

__global__ void label_keys_kernel(const int *labels, int n, uint32_t *keys, int *counts) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        keys[i] = (uint32_t)labels[i];
        atomicAdd(&counts[labels[i]], 1);
    }
}

__global__ void offsets_finish_kernel(const int *excl, const int *counts, int K, int *offsets) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < K) offsets[k] = excl[k];
    if (k == K - 1) offsets[K] = excl[k] + counts[k];
}

uint64_t splitmix64(uint64_t &s) {
    uint64_t z = (s += 0x9e3779b97f4a7c15ull);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

}  // namespace

// K distinct indices in [0, n) by Floyd's sampling with a splitmix64 stream.
std::vector<int> sample_distinct(int n, int K, unsigned long long seed) {
    std::vector<int> out;
    std::unordered_set<int> used;
    uint64_t s = seed;
    for (int j = n - K; j < n; ++j) {
        const int t = (int)(splitmix64(s) % (uint64_t)(j + 1));
        if (used.count(t)) { used.insert(j); out.push_back(j); }
        else { used.insert(t); out.push_back(t); }
    }
    return out;
}

void kmeans_assign(const float *x, int n, int D, const float *cent, int K, int *labels, cudaStream_t st) {
    const int D4 = (D + 3) & ~3;
    static PerDevice<int> attr;
    attr.get([] {
        OTGB_CUDA_TRY(cudaFuncSetAttribute(kmeans_assign_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)sizeof(AssignSmem)));
        return 1;
    });
    kmeans_assign_kernel<<<(n + kAR - 1) / kAR, kAT, sizeof(AssignSmem), st>>>(x, n, D, D4, cent, K, labels);
    OTGB_CHECK_LAUNCH();
}

KmeansResult kmeans(otgb_ctx *ctx, const std::string &tag, const float *x, const float *w, int n, int D, int K,
                    int iters, unsigned long long seed, const float *init, int sample_max) {
    cudaStream_t st = ctx_stream(ctx);
    Workspace &ws = ctx_ws(ctx);
    const int D4 = (D + 3) & ~3;
    KmeansResult r;
    r.cstride = D4;
    r.K = K;
    r.centroids = ws.get<float>(tag + ":cent", (size_t)K * D4);
    r.labels = ws.get<int>(tag + ":lab", n);
    r.perm = ws.get<int>(tag + ":perm", n);
    r.offsets = ws.get<int>(tag + ":off", K + 1);
    // the points the Lloyd iterations run on: all of them, or every s-th
    const float *xi = x, *wi = w;
    int ni = n;
    if (sample_max > 0 && n > sample_max) {
        const int sstep = (n + sample_max - 1) / sample_max;
        ni = (n + sstep - 1) / sstep;
        float *xs = ws.get<float>(tag + ":xs", (size_t)ni * D);
        float *wsub = w ? ws.get<float>(tag + ":ws", ni) : nullptr;
        strided_rows_kernel<<<(unsigned)(((size_t)ni * D + 255) / 256), 256, 0, st>>>(x, w, D, sstep, ni, xs, wsub);
        OTGB_CHECK_LAUNCH();
        xi = xs;
        wi = wsub;
    }
    if (init) {
        copy_rows_kernel<<<(K * D4 + 255) / 256, 256, 0, st>>>(init, D, K, r.centroids, D4);
        OTGB_CHECK_LAUNCH();
    } else {
        std::vector<int> idx = sample_distinct(ni, K, seed);
        int *d_idx = ws.get<int>(tag + ":idx", K);
        OTGB_CUDA_TRY(cudaMemcpyAsync(d_idx, idx.data(), sizeof(int) * K, cudaMemcpyHostToDevice, st));
        gather_rows_kernel<<<(K * D4 + 255) / 256, 256, 0, st>>>(xi, D, d_idx, K, r.centroids, D4);
        OTGB_CHECK_LAUNCH();
        OTGB_CUDA_TRY(cudaStreamSynchronize(st));  // idx is host memory about to go out of scope
    }
    // stable sort by cluster and offsets of all K clusters (empty ones included)
    uint32_t *keys = ws.get<uint32_t>(tag + ":keys", n);
    int *counts = ws.get<int>(tag + ":cnt", K + 1);
    int *excl = ws.get<int>(tag + ":excl", K + 1);
    int bits = 0;
    while ((1 << bits) < K) ++bits;
    void *scr = ws.get("sort:scratch", radix_sort_scratch_bytes(n));
    int *sscr = ws.get<int>("scan:scratch", scan_scratch_ints(K + 1) + 64);
    // labels, order and offsets of the first m points of the buffers (m = ni during the iterations, n at the end)
    auto sort_by_label = [&](int m) {
        OTGB_CUDA_TRY(cudaMemsetAsync(counts, 0, sizeof(int) * (K + 1), st));
        label_keys_kernel<<<(m + 255) / 256, 256, 0, st>>>(r.labels, m, keys, counts);
        OTGB_CHECK_LAUNCH();
        radix_sort_pairs(keys, r.perm, m, bits, scr, st);
        exclusive_scan(counts, excl, K, sscr, st);
        offsets_finish_kernel<<<(K + 255) / 256, 256, 0, st>>>(excl, counts, K, r.offsets);
        OTGB_CHECK_LAUNCH();
    };
    for (int it = 0; it < iters; ++it) {
        kmeans_assign(xi, ni, D, r.centroids, K, r.labels, st);
        sort_by_label(ni);
        kmeans_segment_mean_kernel<<<K, 256, 0, st>>>(xi, wi, D, D4, r.perm, r.offsets, r.centroids);
        OTGB_CHECK_LAUNCH();
    }
    kmeans_assign(x, n, D, r.centroids, K, r.labels, st);
    sort_by_label(n);
    r.sorted_keys = keys;
    return r;
}

}  // namespace otgb
