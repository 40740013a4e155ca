// transport_apply: label transfer through the smooth plan, Eq. (7):
//   Lab_il = sum_{j : l_j = l} b_j exp((f_i + g_j - |x_i - y_j|^2/2) / eps).
// The atlas points are stably sorted by label, so that each thread walks the
// columns of one class after another and keeps a single running sum; the sum
// of a class is finished when the class ends.  Per pair the arithmetic is the
// one of the softmin kernels (centred dot-product form, per-row shift, ex2).
#include <cfloat>
#include <cmath>
#include <cstring>

#include "kmeans.cuh"
#include "multiscale.cuh"
#include "prims.cuh"
#include "solver.cuh"

namespace otgb {
namespace {

constexpr int kTT = 128;  // threads = rows per CTA
constexpr int kTC = 128;  // columns per tile

struct TransportArgs {
    const float *rows;     // n x stride (internal order of rows)
    const float *f;        // f on rows (internal order)
    const float *cols;     // m x stride, sorted by label
    const float *col_logw; // D > 3
    const float *g;        // g on columns (sorted order)
    const int *col_lab;    // label of each sorted column (L for ignored ones, which sort last)
    int n, m, D, stride, L;
    float eps, s;
    double eps_ln2;
    float *scores;         // n x L in internal row order (may be null)
    int *argmax;
    float *mass;
    int4 *fallback;
    int *n_fallback;
};

__device__ __forceinline__ float ex2f_(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__global__ void __launch_bounds__(kTT) transport_kernel(const __grid_constant__ TransportArgs A) {
    __shared__ float Ys[kTC][4];
    __shared__ int Ls[kTC];
    __shared__ float red[kTT / 32];
    __shared__ float cen[3];
    const int t = threadIdx.x;
    const int r = blockIdx.x * kTT + t;
    const bool valid = r < A.n;
    float x0 = 0.f, x1 = 0.f, x2 = 0.f;
    if (valid) {
        x0 = A.rows[(size_t)r * 4];
        if (A.D > 1) x1 = A.rows[(size_t)r * 4 + 1];
        if (A.D > 2) x2 = A.rows[(size_t)r * 4 + 2];
    }
    // centre = middle of the rows' bounding box
    float lo[3] = {valid ? x0 : FLT_MAX, valid ? x1 : FLT_MAX, valid ? x2 : FLT_MAX};
    float hi[3] = {valid ? x0 : -FLT_MAX, valid ? x1 : -FLT_MAX, valid ? x2 : -FLT_MAX};
    for (int d = 0; d < 3; ++d) {
        float l = lo[d], h = hi[d];
        for (int o = 16; o > 0; o >>= 1) {
            l = fminf(l, __shfl_xor_sync(0xffffffffu, l, o));
            h = fmaxf(h, __shfl_xor_sync(0xffffffffu, h, o));
        }
        __syncthreads();
        if ((t & 31) == 0) red[t >> 5] = l;
        __syncthreads();
        if (t == 0) { float v = red[0]; for (int k = 1; k < kTT / 32; ++k) v = fminf(v, red[k]); cen[d] = v; }
        __syncthreads();
        if ((t & 31) == 0) red[t >> 5] = h;
        __syncthreads();
        if (t == 0) { float v = red[0]; for (int k = 1; k < kTT / 32; ++k) v = fmaxf(v, red[k]); cen[d] = 0.5f * (cen[d] + v); }
        __syncthreads();
    }
    const float xt0 = valid ? x0 - cen[0] : 0.f, xt1 = valid ? x1 - cen[1] : 0.f, xt2 = valid ? x2 - cen[2] : 0.f;
    const float s = A.s;
    const double hx = 0.5 * ((double)xt0 * xt0 + (double)xt1 * xt1 + (double)xt2 * xt2);
    // each term is 2^(H_j - m + xt.Y_j) with m = s (|xt|^2/2 - f_i): the exact
    // base-2 exponent of b_j exp((f_i + g_j - C_ij)/eps); near the fixed point a
    // row sums to e^{-f_i/rho} = O(1), so no further shift is needed
    const float m = valid ? (float)((double)s * (hx - (double)A.f[r])) : 0.f;

    float acc = 0.f, tot = 0.f, best = -1.f;
    int cur = -1, bestl = -1;
    double mass = 0.0;
    auto flush = [&](int lab) {
        if (lab < 0 || lab >= A.L) return;
        tot += acc;
        const float v = acc;
        if (valid && A.scores) A.scores[(size_t)r * A.L + lab] = v;
        mass += v;
        if (v > best) { best = v; bestl = lab; }
    };
    // classes with no column get a zero score
    if (valid && A.scores)
        for (int l = 0; l < A.L; ++l) A.scores[(size_t)r * A.L + l] = 0.f;
    for (int p0 = 0; p0 < A.m; p0 += kTC) {
        __syncthreads();
        {
            const int j = p0 + t;
            if (j < A.m) {
                const float4 q = reinterpret_cast<const float4 *>(A.cols)[j];
                const float y0 = q.x - cen[0], y1 = q.y - cen[1], y2 = q.z - cen[2];
                const float H = s * (fmaf(A.eps, q.w, A.g[j]) - 0.5f * (y0 * y0 + y1 * y1 + y2 * y2));
                Ys[t][0] = s * y0; Ys[t][1] = s * y1; Ys[t][2] = s * y2; Ys[t][3] = H;
                Ls[t] = A.col_lab[j];
            } else {
                Ls[t] = 0x7fffffff;
            }
        }
        __syncthreads();
        const int n = min(kTC, A.m - p0);
        for (int c = 0; c < n; ++c) {
            const int lab = Ls[c];
            if (lab != cur) {  // uniform: columns are shared by the CTA
                flush(cur);
                cur = lab;
                acc = 0.f;
                if (cur >= A.L) break;
            }
            float v = fmaf(xt2, Ys[c][2], Ys[c][3] - m);
            v = fmaf(xt1, Ys[c][1], v);
            v = fmaf(xt0, Ys[c][0], v);
            acc += ex2f_(v);
        }
        if (cur >= A.L) break;
    }
    flush(cur);
    if (!valid) return;
    if (!(tot >= 0x1p-60f && tot <= 0x1p60f) && A.m > 0) {
        const int k = atomicAdd(A.n_fallback, 1);
        A.fallback[k] = make_int4(r, 0, 0, 0);
        return;
    }
    A.argmax[r] = bestl;
    if (A.mass) A.mass[r] = (float)mass;
}


// 3 < D <= 64: 256 threads, a block of at most 128 rows (one k-means cluster
// piece); the columns of each class form one contiguous range of the
// label-sorted atlas and are swept in tiles of 64, register-tiled 8 rows x 4
// columns per thread like the softmin kernel; the class sum of a row is final
// when its range ends.
constexpr int kTG = 256, kTBM = 128, kTBN = 64;
struct TransportGenSmem {
    float xs[64][kTBM];
    float ys[64][kTBN];
    float hs[kTBN];
    float cen[64];
    float mrow[kTBM];
    float best[kTBM];
    int bestl[kTBM];
    float mass[kTBM];
    float tot[kTBM];
};

__global__ void __launch_bounds__(kTG) transport_gen_kernel(const __grid_constant__ TransportArgs A, const int *blk_row0,
                                                            const int *lab_off, int D4) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TransportGenSmem &S = *reinterpret_cast<TransportGenSmem *>(smem_raw);
    const int t = threadIdx.x, b = blockIdx.x;
    const int r0 = blk_row0[b], nr = min(blk_row0[b + 1] - r0, kTBM);
    const float s = A.s;
    for (int e = t; e < kTBM * D4; e += kTG) {
        const int r = e / D4, k = e - r * D4;
        S.xs[k][r] = (r < nr) ? A.rows[(size_t)(r0 + r) * D4 + k] : 0.f;
    }
    __syncthreads();
    for (int k = t; k < D4; k += kTG) {
        float acc = 0.f;
        for (int r = 0; r < nr; ++r) acc += S.xs[k][r];
        S.cen[k] = nr > 0 ? acc / (float)nr : 0.f;
    }
    __syncthreads();
    for (int e = t; e < kTBM * D4; e += kTG) {
        const int k = e / kTBM, r = e - k * kTBM;
        S.xs[k][r] = (r < nr) ? S.xs[k][r] - S.cen[k] : 0.f;
    }
    __syncthreads();
    if (t < kTBM) {
        float acc = 0.f;
        for (int k = 0; k < D4; ++k) acc = fmaf(S.xs[k][t], S.xs[k][t], acc);
        // 2^(H_j - m + X.yt) = b_j exp((f_i + g_j - C_ij)/eps) with m = s (|xt|^2/2 - f_i)
        S.mrow[t] = t < nr ? (float)((double)s * (0.5 * (double)acc - (double)A.f[r0 + t])) : 0.f;
        S.best[t] = -1.f;
        S.bestl[t] = -1;
        S.mass[t] = 0.f;
        S.tot[t] = 0.f;
    }
    __syncthreads();
    for (int e = t; e < kTBM * D4; e += kTG) {
        const int k = e / kTBM, r = e - k * kTBM;
        S.xs[k][r] *= s;
    }
    const int tr = t >> 4, tc = t & 15;
    float mreg[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) mreg[i] = S.mrow[tr * 8 + i];
    const int D44 = D4 >> 2;
    for (int l = 0; l < A.L; ++l) {
        const int lb = lab_off[l], le = lab_off[l + 1];
        float rs[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) rs[i] = 0.f;
        for (int p0 = lb; p0 < le; p0 += kTBN) {
            __syncthreads();
            for (int e = t; e < kTBN * D44; e += kTG) {
                const int col = e % kTBN, qq = e / kTBN;
                const int j = p0 + col;
                float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                if (j < le) {
                    v = *reinterpret_cast<const float4 *>(A.cols + (size_t)j * D4 + 4 * qq);
                    v.x -= S.cen[4 * qq]; v.y -= S.cen[4 * qq + 1]; v.z -= S.cen[4 * qq + 2]; v.w -= S.cen[4 * qq + 3];
                }
                S.ys[4 * qq][col] = v.x; S.ys[4 * qq + 1][col] = v.y; S.ys[4 * qq + 2][col] = v.z;
                S.ys[4 * qq + 3][col] = v.w;
            }
            __syncthreads();
            if (t < kTBN) {
                const int j = p0 + t;
                float acc = 0.f;
                for (int k = 0; k < D4; ++k) acc = fmaf(S.ys[k][t], S.ys[k][t], acc);
                S.hs[t] = j < le ? s * (fmaf(A.eps, A.col_logw[j], A.g[j]) - 0.5f * acc) : -INFINITY;
            }
            __syncthreads();
            float acc[8][4];
            const float4 h4 = *reinterpret_cast<const float4 *>(&S.hs[tc * 4]);
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                acc[i][0] = h4.x - mreg[i]; acc[i][1] = h4.y - mreg[i];
                acc[i][2] = h4.z - mreg[i]; acc[i][3] = h4.w - mreg[i];
            }
#pragma unroll 4
            for (int k = 0; k < D4; ++k) {
                const float4 xa = *reinterpret_cast<const float4 *>(&S.xs[k][tr * 8]);
                const float4 xb = *reinterpret_cast<const float4 *>(&S.xs[k][tr * 8 + 4]);
                const float4 yv = *reinterpret_cast<const float4 *>(&S.ys[k][tc * 4]);
                const float xv[8] = {xa.x, xa.y, xa.z, xa.w, xb.x, xb.y, xb.z, xb.w};
                const float yy[4] = {yv.x, yv.y, yv.z, yv.w};
#pragma unroll
                for (int i = 0; i < 8; ++i)
#pragma unroll
                    for (int jj = 0; jj < 4; ++jj) acc[i][jj] = fmaf(xv[i], yy[jj], acc[i][jj]);
            }
#pragma unroll
            for (int i = 0; i < 8; ++i)
                rs[i] += (ex2f_(acc[i][0]) + ex2f_(acc[i][1])) + (ex2f_(acc[i][2]) + ex2f_(acc[i][3]));
        }
#pragma unroll
        for (int i = 0; i < 8; ++i)
            for (int o = 8; o > 0; o >>= 1) rs[i] += __shfl_xor_sync(0xffffffffu, rs[i], o);
        if (tc == 0) {
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int rr = tr * 8 + i;
                if (rr >= nr) continue;
                const float v = rs[i];
                if (A.scores) A.scores[(size_t)(r0 + rr) * A.L + l] = v;
                S.tot[rr] += v;
                if (v > S.best[rr]) { S.best[rr] = v; S.bestl[rr] = l; }
            }
        }
    }
    __syncthreads();
    if (t < nr) {
        const int r = r0 + t;
        const float tot = S.tot[t];
        if (!(tot >= 0x1p-60f && tot <= 0x1p60f) && A.m > 0) {
            const int k = atomicAdd(A.n_fallback, 1);
            A.fallback[k] = make_int4(r, 0, 0, 0);
        } else {
            A.argmax[r] = S.bestl[t];
            if (A.mass) A.mass[r] = tot;
        }
    }
}

// Rows whose sums fell outside the safe range: one warp per row, two passes
// per class in the direct form.
__global__ void transport_fallback_kernel(const __grid_constant__ TransportArgs A) {
    const int count = *A.n_fallback;
    const int lane = threadIdx.x & 31;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < count; w += nw) {
        const int r = A.fallback[w].x;
        const float *xi = A.rows + (size_t)r * A.stride;
        double mass = 0.0, best = -1.0;
        int bestl = -1;
        for (int l = 0; l < A.L; ++l) {
            float m = -INFINITY;
            for (int j = lane; j < A.m; j += 32) {
                if (A.col_lab[j] != l) continue;
                const float *yj = A.cols + (size_t)j * A.stride;
                float d2 = 0.f;
                for (int k = 0; k < A.D; ++k) { const float u = xi[k] - yj[k]; d2 = fmaf(u, u, d2); }
                const float lw = A.col_logw ? A.col_logw[j] : yj[3];
                m = fmaxf(m, A.s * (fmaf(A.eps, lw, A.g[j]) - 0.5f * d2));
            }
            for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
            double acc = 0.0;
            if (m > -INFINITY)
                for (int j = lane; j < A.m; j += 32) {
                    if (A.col_lab[j] != l) continue;
                    const float *yj = A.cols + (size_t)j * A.stride;
                    float d2 = 0.f;
                    for (int k = 0; k < A.D; ++k) { const float u = xi[k] - yj[k]; d2 = fmaf(u, u, d2); }
                    const float lw = A.col_logw ? A.col_logw[j] : yj[3];
                    acc += (double)exp2f(A.s * (fmaf(A.eps, lw, A.g[j]) - 0.5f * d2) - m);
                }
            for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            const double v = (m > -INFINITY) ? exp2((double)A.s * A.f[r] + m + log2(acc)) : 0.0;
            if (lane == 0 && A.scores) A.scores[(size_t)r * A.L + l] = (float)v;
            mass += v;
            if (v > best) { best = v; bestl = l; }
        }
        if (lane == 0) {
            A.argmax[r] = bestl;
            if (A.mass) A.mass[r] = (float)mass;
        }
    }
}

__global__ void label_hist_kernel(const uint32_t *sorted_keys, int m, int L, int *off) {
    // off[l] = first sorted position with label >= l (labels sorted ascending)
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= m) return;
    const int cur = (int)sorted_keys[j];
    const int prev = j > 0 ? (int)sorted_keys[j - 1] : -1;
    for (int l = prev + 1; l <= cur && l <= L; ++l) off[l] = j;
    if (j == m - 1)
        for (int l = cur + 1; l <= L; ++l) off[l] = m;
}

__global__ void label_sort_keys_kernel(const int *labels, int m, int L, uint32_t *keys) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < m) {
        const int l = labels[j];
        keys[j] = (l >= 0 && l < L) ? (uint32_t)l : (uint32_t)L;
    }
}

__global__ void unpermute_rows_kernel(const float *sc, const int *am, const float *ms, const int *perm, int n, int L,
                                      float *sc_out, int *am_out, float *ms_out) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int i = perm ? perm[k] : k;
    am_out[i] = am[k];
    if (ms_out) ms_out[i] = ms[k];
    if (sc_out)
        for (int l = 0; l < L; ++l) sc_out[(size_t)i * L + l] = sc[(size_t)k * L + l];
}

}  // namespace
}  // namespace otgb

using namespace otgb;

extern "C" int transport_apply(otgb_ctx *ctx, const otgb_plan *plan, const float *f, const float *g,
                               const int32_t *labels, int L, float *scores, int32_t *argmax, float *row_mass) {
    if (!ctx) return fail(nullptr, Error{OTGB_EINVAL, "transport_apply: null context"});
    try {
        ctx_set_device(ctx);
        require(plan != nullptr, "transport_apply: null plan");
        require(plan->p == 2, "transport_apply: label transfer is built for plans of the cost |x - y|^2 / 2 (p = 2)");
        require(f && g && labels && argmax, "transport_apply: null pointer argument");
        require(L >= 1 && L <= 1024, "transport_apply: L must be in [1, 1024]");
        const int N = plan->N, M = plan->M, D = plan->D;
        const int stride = D <= 3 ? 4 : ((D + 3) & ~3);
        cudaStream_t st = ctx_stream(ctx);
        Workspace &ws = ctx_ws(ctx);
        // centre of the columns
        float *box = ws.get<float>("box", 4 * 64);
        float *bpart = ws.get<float>("bpart", 64 * 2 * 64);
        bbox(plan->y, M, D, D, box, box + 64, bpart, st);
        std::vector<float> h(128);
        OTGB_CUDA_TRY(cudaMemcpyAsync(h.data(), box, 128 * sizeof(float), cudaMemcpyDeviceToHost, st));
        OTGB_CUDA_TRY(cudaStreamSynchronize(st));
        std::vector<float> cen(64, 0.f);
        for (int d = 0; d < D; ++d) cen[d] = 0.5f * (h[d] + h[64 + d]);
        float *d_cen = ws.get<float>("cen", 64);
        OTGB_CUDA_TRY(cudaMemcpyAsync(d_cen, cen.data(), 64 * sizeof(float), cudaMemcpyHostToDevice, st));
        // columns sorted by label
        uint32_t *keys = ws.get<uint32_t>("ta:keys", M);
        int *cperm = ws.get<int>("ta:cperm", M);
        label_sort_keys_kernel<<<(M + 255) / 256, 256, 0, st>>>(labels, M, L, keys);
        OTGB_CHECK_LAUNCH();
        int bits = 0;
        while ((1 << bits) < L + 1) ++bits;
        void *scr = ws.get("sort:scratch", radix_sort_scratch_bytes(std::max(N, M)));
        radix_sort_pairs(keys, cperm, M, bits, scr, st);
        float *C = ws.get<float>("ta:C", (size_t)M * stride);
        float *Clw = D > 3 ? ws.get<float>("ta:Clw", M) : nullptr;
        float *gs = ws.get<float>("ta:g", M);
        pack_points(plan->y, plan->b, cperm, M, D, d_cen, C, Clw, nullptr, st);
        permute(g, cperm, M, gs, st);
        float *Rw = ws.get<float>("ta:R", (size_t)N * stride);
        float *fs = ws.get<float>("ta:f", N);
        float *sc = scores ? ws.get<float>("ta:sc", (size_t)N * L) : nullptr;
        int *am = ws.get<int>("ta:am", N);
        float *ms = ws.get<float>("ta:ms", N);
        int *nfb = ws.get<int>("ta:nfb", 1);
        int4 *fb = ws.get<int4>("ta:fb", N);
        OTGB_CUDA_TRY(cudaMemsetAsync(nfb, 0, sizeof(int), st));
        TransportArgs A;
        std::memset(&A, 0, sizeof(A));
        A.cols = C; A.col_logw = Clw; A.g = gs; A.col_lab = reinterpret_cast<const int *>(keys);
        A.n = N; A.m = M; A.D = D; A.stride = stride; A.L = L;
        A.eps = (float)plan->eps;
        A.s = (float)(1.4426950408889634 / plan->eps);
        A.eps_ln2 = plan->eps * 0.69314718055994530942;
        A.scores = sc; A.argmax = am; A.mass = ms; A.fallback = fb; A.n_fallback = nfb;
        const int *row_perm = nullptr;
        if (D <= 3) {
            // rows in Morton order of a fine grid (compact CTAs)
            float *rlo = ws.get<float>("ta:rlo", 128);
            bbox(plan->x, N, D, D, rlo, rlo + 64, bpart, st);
            std::vector<float> hb(128);
            OTGB_CUDA_TRY(cudaMemcpyAsync(hb.data(), rlo, 128 * sizeof(float), cudaMemcpyDeviceToHost, st));
            OTGB_CUDA_TRY(cudaStreamSynchronize(st));
            float ext = 0.f;
            for (int d = 0; d < D; ++d) ext = std::max(ext, hb[64 + d] - hb[d]);
            int per_axis = std::max(1, std::min(512, (int)std::ceil(std::cbrt((double)N / 4.0))));
            const float cell = ext > 0.f ? ext / (float)per_axis * 1.0001f : 1.0f;
            GridClusters gc = grid_cluster(ctx, "ta:rows", plan->x, N, D, cell, rlo);
            row_perm = gc.perm;
            pack_points(plan->x, nullptr, gc.perm, N, D, d_cen, Rw, nullptr, nullptr, st);
            permute(f, gc.perm, N, fs, st);
            A.rows = Rw; A.f = fs;
            transport_kernel<<<(N + kTT - 1) / kTT, kTT, 0, st>>>(A);
            OTGB_CHECK_LAUNCH();
        } else {
            // rows ordered by a short K-means; blocks of <= 128 rows inside clusters
            const int K = std::max(1, std::min(N / 64, 4096));
            KmeansResult kr = kmeans(ctx, "ta:km", plan->x, nullptr, N, D, K, 4, 12345, nullptr);
            std::vector<int> off(K + 1);
            OTGB_CUDA_TRY(cudaMemcpyAsync(off.data(), kr.offsets, sizeof(int) * (K + 1), cudaMemcpyDeviceToHost, st));
            OTGB_CUDA_TRY(cudaStreamSynchronize(st));
            std::vector<int> hb = make_row_blocks(N, 128, &off);
            int *d_blk = ws.get<int>("ta:blk", hb.size());
            OTGB_CUDA_TRY(cudaMemcpyAsync(d_blk, hb.data(), sizeof(int) * hb.size(), cudaMemcpyHostToDevice, st));
            int *lab_off = ws.get<int>("ta:laboff", L + 1);
            label_hist_kernel<<<(M + 255) / 256, 256, 0, st>>>(keys, M, L, lab_off);
            OTGB_CHECK_LAUNCH();
            row_perm = kr.perm;
            pack_points(plan->x, nullptr, kr.perm, N, D, d_cen, Rw, nullptr, nullptr, st);
            permute(f, kr.perm, N, fs, st);
            A.rows = Rw; A.f = fs;
            static PerDevice<int> attr;
            attr.get([] {
                OTGB_CUDA_TRY(cudaFuncSetAttribute(transport_gen_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   (int)sizeof(TransportGenSmem)));
                return 1;
            });
            transport_gen_kernel<<<(int)hb.size() - 1, kTG, sizeof(TransportGenSmem), st>>>(A, d_blk, lab_off, stride);
            OTGB_CHECK_LAUNCH();
            OTGB_CUDA_TRY(cudaStreamSynchronize(st));  // hb, off released
        }
        transport_fallback_kernel<<<64, 256, 0, st>>>(A);
        OTGB_CHECK_LAUNCH();
        unpermute_rows_kernel<<<(N + 255) / 256, 256, 0, st>>>(sc, am, ms, row_perm, N, L, scores, argmax, row_mass);
        OTGB_CHECK_LAUNCH();
        OTGB_CUDA_TRY(cudaStreamSynchronize(st));
        return OTGB_OK;
    } catch (const Error &e) {
        return fail(ctx, e);
    }
}
