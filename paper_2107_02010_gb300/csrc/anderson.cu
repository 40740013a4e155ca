// Anderson acceleration (type II, Walker & Ni, SIAM J. Numer. Anal. 2011) of
// the fixed-point map G = one averaged Sinkhorn step (followed by the
// translation step when enabled), on the concatenated duals z = (a, f, b, g).
//
// With residuals r_k = G(z_k) - z_k, differences dR_j = r_{j+1} - r_j and
// dG_j = G(z_{j+1}) - G(z_j) over the last m steps:
//   theta = argmin |r_k - dR theta|^2 + reg |theta|^2,
//   z_{k+1} = G(z_k) - dG theta.
// A fixed point of G is a fixed point of the accelerated iteration (r = 0
// gives theta = 0), so the result is the same; only the number of steps
// changes.  Everything stays on the device (no host synchronisation): the
// Gram matrix of the stored residuals is kept in double precision and updated
// by one row per step; a single CTA solves the small system by Cholesky.
// Safeguard: when the residual norm grows by more than a factor 4 over the
// best one in the current history, the history restarts from the plain step.
#include <cmath>

#include "anderson.cuh"

namespace otgb {
namespace {

constexpr int kAT = 256;
constexpr int kAB = 456;  // CTAs of the dot-product pass (3 per SM on 152 SMs)

// Store G_k and r_k = G_k - z_k in ring slot `slot`; partial dot products
// <r_k, r_s> for every slot s (the slots not yet filled give garbage that the
// solver ignores).
__global__ void aa_dots_kernel(const float *z, const float *G, int n, float *Rring, float *Gring, int slots,
                               const int *state, double *part) {
    __shared__ double red[kAT / 32][kAAMax + 1];
    const int slot = state[0];
    float *rs = Rring + (size_t)slot * n;
    float *gs = Gring + (size_t)slot * n;
    // a thread sums its few elements in float; double from the warp sums on
    float acc[kAAMax + 1];
#pragma unroll
    for (int s = 0; s <= kAAMax; ++s) acc[s] = 0.f;
    for (int i = blockIdx.x * kAT + threadIdx.x; i < n; i += gridDim.x * kAT) {
        const float g = G[i];
        const float r = g - z[i];
        rs[i] = r;
        gs[i] = g;
#pragma unroll
        for (int s = 0; s <= kAAMax; ++s)
            if (s < slots) acc[s] = fmaf(r, s == slot ? r : Rring[(size_t)s * n + i], acc[s]);
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
#pragma unroll
    for (int s = 0; s <= kAAMax; ++s) {
        double v = (double)acc[s];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (l == 0) red[w][s] = v;
    }
    __syncthreads();
    if (threadIdx.x <= kAAMax) {
        double v = 0.0;
        for (int q = 0; q < kAT / 32; ++q) v += red[q][threadIdx.x];
        part[(size_t)blockIdx.x * (kAAMax + 1) + threadIdx.x] = v;
    }
}

// One thread: finish the dots, update the Gram ring, pick the history, solve.
// state: [0] slot of the newest entry, [1] number of valid entries, [2] restarts
// theta_out[0..m-1]: coefficients over the differences, ordered oldest first;
// coef[0..slots-1]: the resulting combination c_s of the stored G vectors,
// z_{k+1} = sum_s coef[s] G_s.
__global__ void aa_solve_kernel(const double *part, int nblk, int slots, int m, double reg, int *state, double *Q,
                                double *best, double *coef) {
    if (blockIdx.x != 0 || threadIdx.x >= 32) return;
    // the block partials: lane l sums blocks l, l + 32, ... (fixed order), then the warp
    const int lane = threadIdx.x;
    double d[kAAMax + 1];
#pragma unroll
    for (int s = 0; s <= kAAMax; ++s) {
        double v = 0.0;
        if (s < slots)
            for (int b = lane; b < nblk; b += 32) v += part[(size_t)b * (kAAMax + 1) + s];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        d[s] = v;
    }
    // the Gram ring in shared memory for the serial part below
    __shared__ double Qs[(kAAMax + 1) * (kAAMax + 1)];
    for (int e = lane; e < slots * slots; e += 32) Qs[e] = Q[e];
    __syncwarp();
    if (lane != 0) return;
    const int slot = state[0];
    int cnt = state[1] + 1;
    if (cnt > slots) cnt = slots;
    for (int s = 0; s < slots; ++s) {
        Q[slot * slots + s] = d[s];
        Q[s * slots + slot] = d[s];
        Qs[slot * slots + s] = d[s];
        Qs[s * slots + slot] = d[s];
    }
    const double rr = d[slot];
    // safeguard: restart when the residual grew well above the best of this history
    if (cnt > 1 && rr > 16.0 * best[0]) {
        cnt = 1;
        state[2] += 1;
    }
    if (cnt == 1 || rr < best[0]) best[0] = rr;
    // history, oldest first: slots slot-cnt+1 .. slot (mod slots)
    int idx[kAAMax + 1];
    for (int q = 0; q < cnt; ++q) idx[q] = ((slot - (cnt - 1) + q) % slots + slots) % slots;
    for (int s = 0; s < slots; ++s) coef[s] = 0.0;
    const int k = cnt - 1 < m ? cnt - 1 : m;  // number of differences used
    if (k <= 0) {
        coef[slot] = 1.0;
    } else {
        // differences j = 0..k-1 between idx[cnt-1-k+j] and idx[cnt-k+j]
        double A[kAAMax][kAAMax], bvec[kAAMax];
        for (int i = 0; i < k; ++i) {
            const int i0 = idx[cnt - 1 - k + i], i1 = idx[cnt - k + i];
            for (int j = 0; j < k; ++j) {
                const int j0 = idx[cnt - 1 - k + j], j1 = idx[cnt - k + j];
                A[i][j] = Qs[i1 * slots + j1] - Qs[i1 * slots + j0] - Qs[i0 * slots + j1] + Qs[i0 * slots + j0];
            }
            bvec[i] = Qs[i1 * slots + slot] - Qs[i0 * slots + slot];
        }
        double tr = 0.0;
        for (int i = 0; i < k; ++i) tr += A[i][i];
        const double lam = reg * (tr > 0.0 ? tr / k : 1.0) + 1e-300;
        for (int i = 0; i < k; ++i) A[i][i] += lam;
        // Cholesky A = L L^T in place (lower triangle); one division per column
        // (double division and square root are slow on this part)
        bool ok = true;
        double inv[kAAMax];
        for (int j = 0; j < k && ok; ++j) {
            double s = A[j][j];
            for (int q = 0; q < j; ++q) s -= A[j][q] * A[j][q];
            if (!(s > 0.0)) { ok = false; break; }
            A[j][j] = sqrt(s);
            inv[j] = 1.0 / A[j][j];
            for (int i = j + 1; i < k; ++i) {
                double t = A[i][j];
                for (int q = 0; q < j; ++q) t -= A[i][q] * A[j][q];
                A[i][j] = t * inv[j];
            }
        }
        double th[kAAMax];
        if (ok) {
            for (int i = 0; i < k; ++i) {
                double t = bvec[i];
                for (int q = 0; q < i; ++q) t -= A[i][q] * th[q];
                th[i] = t * inv[i];
            }
            for (int i = k - 1; i >= 0; --i) {
                double t = th[i];
                for (int q = i + 1; q < k; ++q) t -= A[q][i] * th[q];
                th[i] = t * inv[i];
            }
            for (int i = 0; i < k; ++i) ok = ok && isfinite(th[i]);
        }
        if (!ok) {
            coef[slot] = 1.0;
            cnt = 1;
            state[2] += 1;
        } else {
            // z_{k+1} = G_k - sum_j th_j (G_{j1} - G_{j0})
            coef[slot] += 1.0;
            for (int j = 0; j < k; ++j) {
                coef[idx[cnt - k + j]] -= th[j];
                coef[idx[cnt - 1 - k + j]] += th[j];
            }
        }
    }
    state[1] = cnt;
    state[0] = (slot + 1) % slots;  // the next entry's slot
}

// out[i] = sum_s coef[s] G_s[i]
__global__ void aa_mix_kernel(const float *Gring, int n, int slots, const double *coef, float *out) {
    __shared__ float c[kAAMax + 1];
    if (threadIdx.x <= kAAMax) c[threadIdx.x] = threadIdx.x < slots ? (float)coef[threadIdx.x] : 0.f;
    __syncthreads();
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        float v = 0.f;
        for (int s = 0; s < slots; ++s)
            if (c[s] != 0.f) v = fmaf(c[s], Gring[(size_t)s * n + i], v);
        out[i] = v;
    }
}

}  // namespace

void Anderson::init(Workspace &ws, const std::string &tag, int n_, int m_, cudaStream_t st) {
    n = n_;
    m = m_ < 1 ? 1 : (m_ > kAAMax ? kAAMax : m_);
    slots = m + 1;
    Rring = ws.get<float>(tag + "aaR", (size_t)slots * n);
    Gring = ws.get<float>(tag + "aaG", (size_t)slots * n);
    part = ws.get<double>(tag + "aapart", (size_t)kAB * (kAAMax + 1));
    Q = ws.get<double>(tag + "aaQ", (size_t)slots * slots);
    coef = ws.get<double>(tag + "aacoef", kAAMax + 1);
    state = ws.get<int>(tag + "aastate", 4);
    best = ws.get<double>(tag + "aabest", 1);
    reset(st);
}

void Anderson::reset(cudaStream_t st) {
    OTGB_CUDA_TRY(cudaMemsetAsync(state, 0, 4 * sizeof(int), st));
}

void Anderson::step(const float *z, float *G, cudaStream_t st) {
    aa_dots_kernel<<<kAB, kAT, 0, st>>>(z, G, n, Rring, Gring, slots, state, part);
    OTGB_CHECK_LAUNCH();
    aa_solve_kernel<<<1, 32, 0, st>>>(part, kAB, slots, m, reg, state, Q, best, coef);
    OTGB_CHECK_LAUNCH();
    aa_mix_kernel<<<256, 256, 0, st>>>(Gring, n, slots, coef, G);
    OTGB_CHECK_LAUNCH();
}

}  // namespace otgb
