// Gradient of the debiased Sinkhorn divergence in the points, and the
// free-support Wasserstein barycenter built on it.
//
// Section 2 ("Unbiased Sinkhorn divergences"): at the fixed point, S is a
// function of the points whose gradient is an expression of the converged
// duals (envelope theorem).  For the cost C(x, y) = |x - y|^2 / 2,
//   dS/dx_i = alpha_i [ sum_j beta_j  e^{(f_i + g_j - C(x_i, y_j)) / eps} (x_i - y_j)
//                     - sum_k alpha_k e^{(a_i + a_k - C(x_i, x_k)) / eps} (x_i - x_k) ],
// the first sum from OT(alpha, beta), the second from -OT(alpha, alpha)/2 (x_i
// enters that term twice).  The barycenter ("Track density atlas" of Section 2)
// moves the support of alpha down the mean gradient of S(alpha, beta_k).
//
// Each CTA owns 128 rows (one per thread, the row's point and its gradient in
// registers); column tiles are staged in shared memory and read as broadcasts.
// Two forms: every pair (sinkhorn_grad_x, from the caller's points and duals),
// and the kept cluster pairs of a solve's last truncation (the barycenter's
// steps, from inside the solve).
// Per pair: the direct difference form of the cost (no cancellation), one
// ex2, and the weighted difference accumulated with an online maximum (a term
// larger than every earlier one rescales the running sums), so no shift has
// to be known in advance.
#include <cmath>
#include <cstring>
#include <vector>

#include "multiscale.cuh"
#include "solver.cuh"

namespace otgb {
namespace {

constexpr int kGR = 128;  // rows per CTA, one per thread
constexpr int kGC = 64;   // columns per shared tile

struct GradPart {
    const float *cols;  // m x D (caller layout)
    const float *w;     // m weights
    const float *pot;   // m potential values
    int m;
    float sign;
};

struct GradArgs {
    const float *rows;     // n x D (caller layout)
    const float *row_w;    // n weights
    const float *rpot[2];  // the row's potential in each part
    GradPart part[2];
    int n, D;
    int p1;                // 1: cost |x - y|, gradient (x - y) / |x - y|; 0: cost |x - y|^2 / 2
    float s;               // log2(e) / eps
    float scale;           // multiplies the result
    int accumulate;        // 1: grad += result, 0: grad = result
    float *grad;           // n x D
};

__device__ __forceinline__ float ex2g(float v) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(v));
    return y;
}

template <int D4>
__global__ void __launch_bounds__(kGR) grad_kernel(const __grid_constant__ GradArgs A) {
    __shared__ float ys[kGC][D4];
    __shared__ float yt[kGC];
    const int t = threadIdx.x;
    const int i = blockIdx.x * kGR + t;
    const bool valid = i < A.n;
    const int D = A.D;
    float x[D4], out[D4];
#pragma unroll
    for (int d = 0; d < D4; ++d) {
        x[d] = (valid && d < D) ? A.rows[(size_t)i * D + d] : 0.f;
        out[d] = 0.f;
    }
    for (int q = 0; q < 2; ++q) {
        const GradPart &P = A.part[q];
        // base-2 exponent of each term: s f_i + (log2 w_j + s pot_j) - s C_ij
        const float rt = valid ? A.s * A.rpot[q][i] : 0.f;
        float m = -INFINITY;
        float v[D4];
#pragma unroll
        for (int d = 0; d < D4; ++d) v[d] = 0.f;
        for (int c0 = 0; c0 < P.m; c0 += kGC) {
            const int nc = min(kGC, P.m - c0);
            __syncthreads();
            for (int e = t; e < kGC * D4; e += kGR) {
                const int c = e / D4, d = e - c * D4;
                ys[c][d] = (c < nc && d < D) ? P.cols[(size_t)(c0 + c) * D + d] : 0.f;
            }
            if (t < kGC) {
                const float w = t < nc ? P.w[c0 + t] : 0.f;
                yt[t] = w > 0.f ? log2f(w) + A.s * P.pot[c0 + t] : -INFINITY;
            }
            __syncthreads();
            for (int c = 0; c < nc; ++c) {
                const float ct = yt[c];
                if (ct == -INFINITY) continue;  // the same column for every thread
                float sq = 0.f;
#pragma unroll
                for (int d = 0; d < D4; ++d) {
                    const float df = x[d] - ys[c][d];
                    sq = fmaf(df, df, sq);
                }
                const float dist = A.p1 ? sqrtf(sq) : 0.f;
                const float e = A.p1 ? fmaf(-A.s, dist, rt + ct) : fmaf(-0.5f * A.s, sq, rt + ct);
                if (e > m) {  // rescale the running sums to the new maximum
                    const float sc = ex2g(m - e);
#pragma unroll
                    for (int d = 0; d < D4; ++d) v[d] *= sc;
                    m = e;
                }
                float w = ex2g(e - m);
                if (A.p1) w = dist > 0.f ? w / dist : 0.f;  // grad_1 |x - y| = (x - y) / |x - y|
#pragma unroll
                for (int d = 0; d < D4; ++d) v[d] = fmaf(w, x[d] - ys[c][d], v[d]);
            }
        }
        // the part's sum is 2^m v (m = -inf: no term, nothing to add)
        if (m > -INFINITY) {
            const float em = P.sign * exp2f(m);
#pragma unroll
            for (int d = 0; d < D4; ++d) out[d] = fmaf(em, v[d], out[d]);
        }
    }
    if (!valid) return;
    const float aw = A.row_w[i] * A.scale;
    for (int d = 0; d < D; ++d) {
        float r = aw * out[d];
        if (A.accumulate) r += A.grad[(size_t)i * D + d];
        A.grad[(size_t)i * D + d] = r;
    }
}

void grad_launch(const GradArgs &A, cudaStream_t st) {
    const int grid = (A.n + kGR - 1) / kGR;
    const int D4 = (A.D + 3) & ~3;
    switch (D4) {
#define OTGB_GRAD_CASE(K) \
    case K: grad_kernel<K><<<grid, kGR, 0, st>>>(A); break;
        OTGB_GRAD_CASE(4) OTGB_GRAD_CASE(8) OTGB_GRAD_CASE(12) OTGB_GRAD_CASE(16)
        OTGB_GRAD_CASE(20) OTGB_GRAD_CASE(24) OTGB_GRAD_CASE(28) OTGB_GRAD_CASE(32)
        OTGB_GRAD_CASE(36) OTGB_GRAD_CASE(40) OTGB_GRAD_CASE(44) OTGB_GRAD_CASE(48)
        OTGB_GRAD_CASE(52) OTGB_GRAD_CASE(56) OTGB_GRAD_CASE(60) OTGB_GRAD_CASE(64)
#undef OTGB_GRAD_CASE
        default: throw Error{OTGB_EINTERNAL, "grad_launch: D out of range"};
    }
    OTGB_CHECK_LAUNCH();
}

GradArgs grad_args(const float *x, const float *alpha, int N, const float *y, const float *beta, int M, int D,
                   int p, double eps, const float *a_self, const float *f, const float *g, float *grad,
                   float scale, int accumulate) {
    GradArgs A;
    std::memset(&A, 0, sizeof(A));
    A.rows = x;
    A.row_w = alpha;
    A.rpot[0] = f;       // OT(alpha, beta): f on x against (y, beta, g)
    A.rpot[1] = a_self;  // OT(alpha, alpha): a on x against (x, alpha, a)
    A.part[0] = GradPart{y, beta, g, M, 1.f};
    A.part[1] = GradPart{x, alpha, a_self, N, -1.f};
    A.n = N;
    A.D = D;
    A.p1 = p == 1 ? 1 : 0;
    A.s = (float)(1.4426950408889634 / eps);
    A.scale = scale;
    A.accumulate = accumulate;
    A.grad = grad;
    return A;
}

// ---- the same gradient over the kept cluster pairs of a solve (internal order)
// One CTA per row block of the first measure (the solve's own blocks, at most
// 128 rows, one per thread); part 0 walks the block's kept columns of the
// second measure (instance 3: rows x against (y, beta, g)), part 1 those of the
// first (instance 0: rows x against (x, alpha, a)).  The terms left out are
// those the truncation dropped, each below e^-tau of its row's total.
struct SpGradArgs {
    SoftminInst inst[2];
    const float *rpot[2];  // f, a (internal order)
    const float *cpot[2];  // g, a
    float sign[2];
    const float *row_w;    // alpha (internal order)
    const int *perm;       // internal position -> caller index (null: identity)
    int n, D, stride, small, p1;
    float s;               // log2(e) / eps
    float scale;
    int accumulate;
    float *grad;           // caller's order, n x D
};

template <int D4>
__global__ void __launch_bounds__(kGR) grad_sparse_kernel(const __grid_constant__ SpGradArgs A) {
    __shared__ float ys[kGC][D4];
    __shared__ float yt[kGC];
    __shared__ int jidx[kGC];
    const int t = threadIdx.x, blk = blockIdx.x;
    const int D = A.D;
    int r0 = A.inst[0].blk_row0[blk], r1 = A.inst[0].blk_row0[blk + 1];
    OTGB_DCLAMP(r0, 0, A.n + 1);
    OTGB_DCLAMP(r1, r0, min(A.n, r0 + kGR) + 1);
    const int i = r0 + t;
    const bool valid = i < r1;
    const int rs = A.small ? 4 : A.stride;  // floats per point
    float x[D4], out[D4];
#pragma unroll
    for (int d = 0; d < D4; ++d) {
        x[d] = (valid && d < D) ? A.inst[0].rows[(size_t)i * rs + d] : 0.f;
        out[d] = 0.f;
    }
    for (int q = 0; q < 2; ++q) {
        const SoftminInst &I = A.inst[q];
        const int nk = kept_cols(I, blk);
        ColWalk walk;
        if (t < kGC) walk.start(I, blk, t);
        const float rt = valid ? A.s * A.rpot[q][i] : 0.f;
        float m = -INFINITY;
        float v[D4];
#pragma unroll
        for (int d = 0; d < D4; ++d) v[d] = 0.f;
        for (int p0 = 0; p0 < nk; p0 += kGC) {
            const int nc = min(kGC, nk - p0);
            __syncthreads();  // the previous tile is consumed
            if (t < kGC) {
                int j = -1;
                float ct = -INFINITY;
                if (t < nc) {
                    j = walk.at(p0 + t);
                    OTGB_DCLAMP(j, 0, I.n_cols);
                    const float lw = A.small ? I.cols[(size_t)j * 4 + 3] : I.col_logw[j];
                    if (lw > -INFINITY) ct = lw * 1.4426950408889634f + A.s * A.cpot[q][j];
                }
                jidx[t] = j;
                yt[t] = ct;
            }
            __syncthreads();
            for (int e = t; e < kGC * D4; e += kGR) {
                const int c = e / D4, d = e - c * D4;
                const int j = jidx[c];
                ys[c][d] = (j >= 0 && d < D) ? I.cols[(size_t)j * rs + d] : 0.f;
            }
            __syncthreads();
            for (int c = 0; c < nc; ++c) {
                const float ct = yt[c];
                if (ct == -INFINITY) continue;  // the same column for every thread
                float sq = 0.f;
#pragma unroll
                for (int d = 0; d < D4; ++d) {
                    const float df = x[d] - ys[c][d];
                    sq = fmaf(df, df, sq);
                }
                const float dist = A.p1 ? sqrtf(sq) : 0.f;
                const float e = A.p1 ? fmaf(-A.s, dist, rt + ct) : fmaf(-0.5f * A.s, sq, rt + ct);
                if (e > m) {
                    const float sc = ex2g(m - e);
#pragma unroll
                    for (int d = 0; d < D4; ++d) v[d] *= sc;
                    m = e;
                }
                float w = ex2g(e - m);
                if (A.p1) w = dist > 0.f ? w / dist : 0.f;
#pragma unroll
                for (int d = 0; d < D4; ++d) v[d] = fmaf(w, x[d] - ys[c][d], v[d]);
            }
        }
        if (m > -INFINITY) {
            const float em = A.sign[q] * exp2f(m);
#pragma unroll
            for (int d = 0; d < D4; ++d) out[d] = fmaf(em, v[d], out[d]);
        }
    }
    if (!valid) return;
    int gi = A.perm ? A.perm[i] : i;
    OTGB_DCLAMP(gi, 0, A.n);
    const float aw = A.row_w[i] * A.scale;
    for (int d = 0; d < D; ++d) {
        float r = aw * out[d];
        if (A.accumulate) r += A.grad[(size_t)gi * D + d];
        A.grad[(size_t)gi * D + d] = r;
    }
}

void grad_sparse_run(const Solver &s, double eps, const GradRequest &gr, cudaStream_t st) {
    SpGradArgs A;
    std::memset(&A, 0, sizeof(A));
    A.inst[0] = s.launch.inst[3];  // rows x against (y, beta, g)
    A.inst[1] = s.launch.inst[0];  // rows x against (x, alpha, a)
    A.rpot[0] = s.pf[s.cur];
    A.cpot[0] = s.pg[s.cur];
    A.rpot[1] = s.pa[s.cur];
    A.cpot[1] = s.pa[s.cur];
    A.sign[0] = 1.f;
    A.sign[1] = -1.f;
    A.row_w = s.X.w;
    A.perm = s.X.perm;
    A.n = s.X.n;
    A.D = s.D;
    A.stride = s.X.stride;
    A.small = s.D <= 3 ? 1 : 0;
    A.p1 = s.p == 1 ? 1 : 0;
    A.s = (float)(1.4426950408889634 / eps);
    A.scale = gr.scale;
    A.accumulate = gr.accumulate;
    A.grad = gr.grad;
    require(s.nblk_x >= 1 && A.inst[0].blk_row0 && A.inst[1].blk_row0, "gradient: the solve has no row blocks",
            OTGB_EINTERNAL);
    const int D4 = (s.D + 3) & ~3;
    switch (D4) {
#define OTGB_SGRAD_CASE(K) \
    case K: grad_sparse_kernel<K><<<s.nblk_x, kGR, 0, st>>>(A); break;
        OTGB_SGRAD_CASE(4) OTGB_SGRAD_CASE(8) OTGB_SGRAD_CASE(12) OTGB_SGRAD_CASE(16)
        OTGB_SGRAD_CASE(20) OTGB_SGRAD_CASE(24) OTGB_SGRAD_CASE(28) OTGB_SGRAD_CASE(32)
        OTGB_SGRAD_CASE(36) OTGB_SGRAD_CASE(40) OTGB_SGRAD_CASE(44) OTGB_SGRAD_CASE(48)
        OTGB_SGRAD_CASE(52) OTGB_SGRAD_CASE(56) OTGB_SGRAD_CASE(60) OTGB_SGRAD_CASE(64)
#undef OTGB_SGRAD_CASE
        default: throw Error{OTGB_EINVAL, "gradient: D must be in [1, 64]"};
    }
    OTGB_CHECK_LAUNCH();
}

// x_i <- x_i - lr G_i / alpha_i (rows with alpha_i = 0 stay)
__global__ void descent_kernel(float *x, const float *alpha, const float *G, int n, int D, float lr) {
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (size_t)n * D) return;
    const float w = alpha[e / D];
    if (w > 0.f) x[e] -= lr * G[e] / w;
}

}  // namespace

void grad_sparse_launch(const Solver &s, double eps, const GradRequest &gr, cudaStream_t st) {
    grad_sparse_run(s, eps, gr, st);
}

}  // namespace otgb

using namespace otgb;

extern "C" int sinkhorn_grad_x(otgb_ctx *ctx, const float *x, const float *alpha, int N, const float *y,
                               const float *beta, int M, int D, int p, double eps, const float *f, const float *g,
                               const float *a_self, float *grad) {
    if (!ctx) return fail(nullptr, Error{OTGB_EINVAL, "sinkhorn_grad_x: null context"});
    try {
        ctx_set_device(ctx);
        require(x && alpha && y && beta && f && g && a_self && grad, "sinkhorn_grad_x: null pointer argument");
        require(N >= 1 && M >= 1, "sinkhorn_grad_x: N and M must be >= 1");
        require(D >= 1 && D <= 64, "sinkhorn_grad_x: D must be in [1, 64]");
        require(p == 1 || p == 2, "sinkhorn_grad_x: p must be 1 or 2");
        require(eps > 0.0 && std::isfinite(eps), "sinkhorn_grad_x: eps must be > 0");
        cudaStream_t st = ctx_stream(ctx);
        grad_launch(grad_args(x, alpha, N, y, beta, M, D, p, eps, a_self, f, g, grad, 1.f, 0), st);
        OTGB_CUDA_TRY(cudaStreamSynchronize(st));
        return OTGB_OK;
    } catch (const Error &e) {
        return fail(ctx, e);
    }
}

extern "C" int sinkhorn_barycenter(otgb_ctx *ctx, float *x, const float *alpha, int N, int K,
                                   const float *const *ys, const float *const *betas, const int *Ms, int D,
                                   const otgb_params *params, int iters, double lr, double *S_hist) {
    if (!ctx) return fail(nullptr, Error{OTGB_EINVAL, "sinkhorn_barycenter: null context"});
    try {
        ctx_set_device(ctx);
        require(x && alpha && ys && betas && Ms, "sinkhorn_barycenter: null pointer argument");
        require(N >= 1 && K >= 1 && iters >= 0, "sinkhorn_barycenter: N, K >= 1 and iters >= 0 required");
        require(D >= 1 && D <= 64, "sinkhorn_barycenter: D must be in [1, 64]");
        require(lr > 0.0 && std::isfinite(lr), "sinkhorn_barycenter: lr must be > 0");
        otgb_params P;
        if (params) P = *params;
        else otgb_default_params(&P);
        require(P.p == 1 || P.p == 2, "sinkhorn_barycenter: p must be 1 or 2");
        for (int k = 0; k < K; ++k) require(ys[k] && betas[k] && Ms[k] >= 1, "sinkhorn_barycenter: bad measure");
        cudaStream_t st = ctx_stream(ctx);
        Workspace &ws = ctx_ws(ctx);
        int Mmax = 0;
        for (int k = 0; k < K; ++k) Mmax = std::max(Mmax, Ms[k]);
        // buffers that survive the solves' own workspace use: named apart.  The four duals of each
        // measure are kept from one step to the next: the points move little per step, so after the
        // first step every solve starts at blur from the duals of the previous one (the fixed point
        // decides the result, the start only its cost).
        float *G = ws.get<float>("bary:G", (size_t)N * D);
        std::vector<float *> fk(K), gk(K), ak(K), bk(K);
        for (int k = 0; k < K; ++k) {
            const std::string s = std::to_string(k);
            fk[k] = ws.get<float>("bary:f" + s, N);
            ak[k] = ws.get<float>("bary:a" + s, N);
            gk[k] = ws.get<float>("bary:g" + s, Ms[k]);
            bk[k] = ws.get<float>("bary:b" + s, Ms[k]);
        }
        for (int it = 0; it <= iters; ++it) {
            double Ssum = 0.0;
            const bool last = it == iters;
            if (last && !S_hist) break;
            for (int k = 0; k < K; ++k) {
                double S = 0.0;
                otgb_params Pk = P;
                if (it > 0) {
                    Pk.f_init = fk[k];
                    Pk.g_init = gk[k];
                    Pk.a_init = ak[k];
                    Pk.b_init = bk[k];
                    Pk.sigma_start = P.blur;
                }
                float *f = fk[k], *g = gk[k], *a = ak[k];
                // the gradient comes from inside the solve, over the kept cluster pairs of its last
                // truncation (the dense form, sinkhorn_grad_x, pays for every pair of the self term)
                const GradRequest gr{G, (float)(1.0 / K), k > 0 ? 1 : 0};
                const int rc = solve_divergence(ctx, x, alpha, N, ys[k], betas[k], Ms[k], D, &Pk, &S, f, g, a,
                                                bk[k], nullptr, nullptr, last ? nullptr : &gr);
                if (rc != OTGB_OK && rc != OTGB_ENOCONV) return rc;  // the message is already set
                Ssum += S;
            }
            if (S_hist) S_hist[it] = Ssum / K;
            if (last) break;
            const size_t tot = (size_t)N * D;
            descent_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(x, alpha, G, N, D, (float)lr);
            OTGB_CHECK_LAUNCH();
        }
        OTGB_CUDA_TRY(cudaStreamSynchronize(st));
        return OTGB_OK;
    } catch (const Error &e) {
        return fail(ctx, e);
    }
}
