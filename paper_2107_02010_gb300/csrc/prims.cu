// Data-parallel primitives of the solver: reductions (bounding box, FP64
// divergence sums), exclusive scan, stable LSD radix sort, packing of the
// point clouds into the internal layout, cluster statistics.
#include <cfloat>
#include <cmath>

#include "prims.cuh"

namespace otgb {
namespace {

constexpr int kRB = 256;  // threads per block for the reductions

// ------------------------------------------------------------------ bbox --
__global__ void bbox_partial_kernel(const float *x, int n, int D, int stride, float *part, int nblk) {
    // part: [nblk][2*D]: lo then hi of this block
    __shared__ float s_lo[kRB], s_hi[kRB];
    for (int d = 0; d < D; ++d) {
        float lo = FLT_MAX, hi = -FLT_MAX;
        for (int i = blockIdx.x * kRB + threadIdx.x; i < n; i += gridDim.x * kRB) {
            const float v = x[(size_t)i * stride + d];
            lo = fminf(lo, v);
            hi = fmaxf(hi, v);
        }
        s_lo[threadIdx.x] = lo;
        s_hi[threadIdx.x] = hi;
        __syncthreads();
        for (int o = kRB / 2; o > 0; o >>= 1) {
            if (threadIdx.x < o) {
                s_lo[threadIdx.x] = fminf(s_lo[threadIdx.x], s_lo[threadIdx.x + o]);
                s_hi[threadIdx.x] = fmaxf(s_hi[threadIdx.x], s_hi[threadIdx.x + o]);
            }
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            part[(size_t)blockIdx.x * 2 * D + d] = s_lo[0];
            part[(size_t)blockIdx.x * 2 * D + D + d] = s_hi[0];
        }
        __syncthreads();
    }
}

__global__ void bbox_final_kernel(const float *part, int nblk, int D, float *lo, float *hi) {
    const int d = threadIdx.x;
    if (d >= D) return;
    float l = FLT_MAX, h = -FLT_MAX;
    for (int b = 0; b < nblk; ++b) {
        l = fminf(l, part[(size_t)b * 2 * D + d]);
        h = fmaxf(h, part[(size_t)b * 2 * D + D + d]);
    }
    lo[d] = l;
    hi[d] = h;
}

// ------------------------------------------------------- FP64 sums (Eq. 6) --
// Balanced: sum_i a_i (f_i - aa_i) + sum_j b_j (g_j - bb_j).
// Unbalanced: -(rho + eps/2) [ sum_i a_i e^{-aa_i/rho} expm1(-(f_i - aa_i)/rho) + (same for b) ].
__global__ void divsum_partial_kernel(const float *wa, const float *f, const float *aa, int N, const float *wb,
                                      const float *g, const float *bb, int M, double rho, int balanced,
                                      double *part) {
    __shared__ double s[kRB];
    double acc = 0.0;
    const int total = N + M;
    for (int k = blockIdx.x * kRB + threadIdx.x; k < total; k += gridDim.x * kRB) {
        double w, p, q;
        if (k < N) { w = wa[k]; p = f[k]; q = aa[k]; }
        else { const int j = k - N; w = wb[j]; p = g[j]; q = bb[j]; }
        if (w == 0.0) continue;
        acc += balanced ? w * (p - q) : w * exp(-q / rho) * expm1(-(p - q) / rho);
    }
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int o = kRB / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = s[0];
}

__global__ void divsum_final_kernel(const double *part, int nblk, double rho, double eps, int balanced,
                                    double *out) {
    if (threadIdx.x != 0) return;
    double acc = 0.0;
    for (int b = 0; b < nblk; ++b) acc += part[b];  // fixed order: deterministic
    *out = balanced ? acc : -(rho + 0.5 * eps) * acc;
}

// ----------------------------------------------- translation of (f, g) ----
// part[b] = (sum_i a_i e^{-f_i/rho}, sum_j b_j e^{-g_j/rho}) over a grid-stride share.
__global__ void transl_partial_kernel(const float *wa, const float *f, int N, const float *wb, const float *g, int M,
                                      double rho, double2 *part) {
    __shared__ double sa[kRB], sb[kRB];
    // exp in single precision where it cannot overflow or flush (|t| < 80),
    // in double elsewhere; the sums in double
    const float inv_rho = (float)(1.0 / rho);
    auto term = [&](float w, float v) -> double {
        const float t = -v * inv_rho;
        return fabsf(t) < 80.f ? (double)(w * expf(t)) : (double)w * exp(-(double)v / rho);
    };
    double A = 0.0, B = 0.0;
    for (int i = blockIdx.x * kRB + threadIdx.x; i < N; i += gridDim.x * kRB) A += term(wa[i], f[i]);
    for (int j = blockIdx.x * kRB + threadIdx.x; j < M; j += gridDim.x * kRB) B += term(wb[j], g[j]);
    sa[threadIdx.x] = A;
    sb[threadIdx.x] = B;
    __syncthreads();
    for (int o = kRB / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) { sa[threadIdx.x] += sa[threadIdx.x + o]; sb[threadIdx.x] += sb[threadIdx.x + o]; }
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = make_double2(sa[0], sb[0]);
}

// c = (rho/2) log(A/B) from the partial sums (fixed order), then f += c, g -= c.
__global__ void transl_apply_kernel(const double2 *part, int nblk, double rho, float *f, int N, float *g, int M,
                                    double *c_out) {
    __shared__ float cs;
    if (threadIdx.x < 32) {
        double A = 0.0, B = 0.0;
        for (int b = threadIdx.x; b < nblk; b += 32) { A += part[b].x; B += part[b].y; }
        for (int o = 16; o > 0; o >>= 1) {
            A += __shfl_xor_sync(0xffffffffu, A, o);
            B += __shfl_xor_sync(0xffffffffu, B, o);
        }
        double c = (A > 0.0 && B > 0.0) ? 0.5 * rho * log(A / B) : 0.0;
        if (!isfinite(c)) c = 0.0;
        if (threadIdx.x == 0) {
            cs = (float)c;
            if (blockIdx.x == 0 && c_out) *c_out = c;
        }
    }
    __syncthreads();
    const float c = cs;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N + M; i += gridDim.x * blockDim.x) {
        if (i < N) f[i] += c;
        else g[i - N] -= c;
    }
}

// ------------------------------------------------------------------- scan --
constexpr int kScanB = 1024;

__global__ void scan_block_kernel(const int *in, int *out, int n, int *block_sums) {
    __shared__ int s[kScanB];
    const int i = blockIdx.x * kScanB + threadIdx.x;
    const int v = i < n ? in[i] : 0;
    s[threadIdx.x] = v;
    __syncthreads();
    for (int o = 1; o < kScanB; o <<= 1) {
        const int a = threadIdx.x >= o ? s[threadIdx.x - o] : 0;
        __syncthreads();
        s[threadIdx.x] += a;
        __syncthreads();
    }
    if (i < n) out[i] = s[threadIdx.x] - v;  // exclusive
    if (threadIdx.x == kScanB - 1) block_sums[blockIdx.x] = s[kScanB - 1];
}

__global__ void scan_add_kernel(int *out, int n, const int *block_off) {
    const int i = blockIdx.x * kScanB + threadIdx.x;
    if (i < n) out[i] += block_off[blockIdx.x];
}

// ------------------------------------------------------------- radix sort --
// Stable LSD radix sort of (key, value) pairs, 8-bit digits.  Each CTA owns a
// chunk of kChunk consecutive elements; per pass: digit histograms per chunk,
// an exclusive scan in digit-major order, then a stable scatter where each
// element's rank among equal digits of its chunk follows input order.
constexpr int kSortT = 256;
constexpr int kPerT = 8;
constexpr int kChunk = kSortT * kPerT;

__global__ void radix_hist_kernel(const uint32_t *keys, int n, int shift, int *counts, int nchunks) {
    __shared__ int h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const int base = blockIdx.x * kChunk;
    for (int k = 0; k < kPerT; ++k) {
        const int i = base + k * kSortT + threadIdx.x;
        if (i < n) atomicAdd(&h[(keys[i] >> shift) & 255u], 1);
    }
    __syncthreads();
    counts[(size_t)threadIdx.x * nchunks + blockIdx.x] = h[threadIdx.x];
}

__global__ void radix_scatter_kernel(const uint32_t *keys, const int *vals, int n, int shift,
                                     const int *offsets, int nchunks, uint32_t *keys_out, int *vals_out) {
    __shared__ int run[256];         // running output position per digit
    __shared__ int wc[kSortT / 32][256];  // per-warp digit counts of the current round
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    run[t] = offsets[(size_t)t * nchunks + blockIdx.x];
    const int base = blockIdx.x * kChunk;
    for (int k = 0; k < kPerT; ++k) {
        for (int q = 0; q < kSortT / 32; ++q) wc[q][t] = 0;
        __syncthreads();
        const int i = base + k * kSortT + t;
        const bool valid = i < n;
        const uint32_t key = valid ? keys[i] : 0u;
        const int dig = valid ? (int)((key >> shift) & 255u) : 256 + lane;  // unique for invalid
        const unsigned peers = __match_any_sync(0xffffffffu, dig);
        const int rank = __popc(peers & ((1u << lane) - 1u));
        if (valid && rank == 0) wc[w][dig] = __popc(peers);
        __syncthreads();
        if (valid) {
            int pos = run[dig] + rank;
            for (int q = 0; q < w; ++q) pos += wc[q][dig];
            OTGB_DCLAMP(pos, 0, n);
            keys_out[pos] = key;
            vals_out[pos] = vals ? vals[i] : i;
        }
        __syncthreads();
        int add = 0;
        for (int q = 0; q < kSortT / 32; ++q) add += wc[q][t];
        run[t] += add;
        __syncthreads();
    }
}

// ------------------------------------------------------------- packing ---
// D <= 3: out[k] = (x - c, log w) as float4 (zero-padded coordinates).
// D >  3: out row k = x - c padded with zeros to D4 floats; logw[k] = log w.
__global__ void pack_kernel(const float *x, const float *w, const int *perm, int n, int D, int D4,
                            const float *center, float *out, float *logw, float *w_sorted) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    int i = perm ? perm[k] : k;
    OTGB_DCLAMP(i, 0, n);
    const float wi = w ? w[i] : 1.0f;
    const float lw = wi > 0.f ? logf(wi) : -INFINITY;
    if (D <= 3) {
        float v[3] = {0.f, 0.f, 0.f};
        for (int d = 0; d < D; ++d) v[d] = x[(size_t)i * D + d] - center[d];
        reinterpret_cast<float4 *>(out)[k] = make_float4(v[0], v[1], v[2], lw);
    } else {
        for (int d = 0; d < D4; ++d) out[(size_t)k * D4 + d] = d < D ? x[(size_t)i * D + d] - center[d] : 0.f;
    }
    if (logw) logw[k] = lw;
    if (w_sorted) w_sorted[k] = wi;
}

__global__ void iota_kernel(int *v, int n) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) v[k] = k;
}

__global__ void unpermute_kernel(const float *in, const int *perm, int n, float *out) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    int i = perm ? perm[k] : k;
    OTGB_DCLAMP(i, 0, n);
    out[i] = in[k];
}

__global__ void permute_kernel(const float *in, const int *perm, int n, float *out) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    int i = perm ? perm[k] : k;
    OTGB_DCLAMP(i, 0, n);
    out[k] = in[i];
}

__global__ void check_weights_kernel(const float *w, int n, int *bad, double *mass_part) {
    __shared__ double s[kRB];
    double acc = 0.0;
    for (int i = blockIdx.x * kRB + threadIdx.x; i < n; i += gridDim.x * kRB) {
        const float v = w[i];
        if (!(v >= 0.f) || !(v < INFINITY)) atomicOr(bad, 1);
        else acc += v;
    }
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int o = kRB / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) mass_part[blockIdx.x] = s[0];
}

__global__ void check_points_kernel(const float *x, size_t n, int *bad) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        if (!isfinite(x[i])) atomicOr(bad, 2);
}

__global__ void absmax_kernel(const float *v, int n, unsigned *out) {
    float m = 0.f;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) m = fmaxf(m, fabsf(v[i]));
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(m));
}

__global__ void finite_kernel(const float *v, int n, int *bad) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        if (!isfinite(v[i])) atomicOr(bad, 4);
}

// ------------------------------------------------------ cluster statistics --
// One CTA per cluster k over sorted positions [off[k], off[k+1]) of the packed
// points (stride floats per point): mass = sum w, centroid = weighted mean
// (plain mean when the mass is 0), radius = max distance to the centroid.
__global__ void cluster_stats_kernel(const float *pts, int stride, int D, const float *w_sorted, const int *off,
                                     int ncl, float *cent, int cstride, float *mass, float *radius, float *ssq) {
    __shared__ double red[128];
    __shared__ float c_s[64];
    const int k = blockIdx.x;
    if (k >= ncl) return;
    const int a = off[k], b = off[k + 1];
    const int t = threadIdx.x;
    double m = 0.0;
    for (int i = a + t; i < b; i += 128) m += w_sorted[i];
    red[t] = m;
    __syncthreads();
    for (int o = 64; o > 0; o >>= 1) {
        if (t < o) red[t] += red[t + o];
        __syncthreads();
    }
    const double mass_k = red[0];
    __syncthreads();
    for (int d = 0; d < D; ++d) {
        double acc = 0.0;
        for (int i = a + t; i < b; i += 128)
            acc += (mass_k > 0.0 ? (double)w_sorted[i] : 1.0) * pts[(size_t)i * stride + d];
        red[t] = acc;
        __syncthreads();
        for (int o = 64; o > 0; o >>= 1) {
            if (t < o) red[t] += red[t + o];
            __syncthreads();
        }
        if (t == 0) c_s[d] = (float)(red[0] / (mass_k > 0.0 ? mass_k : (double)(b - a)));
        __syncthreads();
    }
    float r2 = 0.f;
    double wss = 0.0;
    for (int i = a + t; i < b; i += 128) {
        float s2 = 0.f;
        for (int d = 0; d < D; ++d) { const float u = pts[(size_t)i * stride + d] - c_s[d]; s2 = fmaf(u, u, s2); }
        r2 = fmaxf(r2, s2);
        wss += (double)w_sorted[i] * s2;
    }
    red[t] = r2;
    __syncthreads();
    for (int o = 64; o > 0; o >>= 1) {
        if (t < o) red[t] = fmax(red[t], red[t + o]);
        __syncthreads();
    }
    if (t == 0) {
        mass[k] = (float)mass_k;
        radius[k] = sqrtf((float)red[0]) * (1.0f + 1e-6f) + 1e-30f;
    }
    __syncthreads();
    red[t] = wss;
    __syncthreads();
    for (int o = 64; o > 0; o >>= 1) {
        if (t < o) red[t] += red[t + o];
        __syncthreads();
    }
    if (t == 0 && ssq) ssq[k] = (float)red[0];
    // D <= 3 packs the coarse measure like the points: (centroid, log mass)
    if (t < cstride) {
        float v = t < D ? c_s[t] : 0.f;
        if (D <= 3 && cstride == 4 && t == 3) v = mass_k > 0.0 ? (float)log(mass_k) : -INFINITY;
        cent[(size_t)k * cstride + t] = v;
    }
}

}  // namespace

// =================================================================== host ==
void bbox(const float *x, int n, int D, int stride, float *d_lo, float *d_hi, float *d_part, cudaStream_t st) {
    const int nblk = 64;
    bbox_partial_kernel<<<nblk, kRB, 0, st>>>(x, n, D, stride, d_part, nblk);
    OTGB_CHECK_LAUNCH();
    bbox_final_kernel<<<1, 64, 0, st>>>(d_part, nblk, D, d_lo, d_hi);
    OTGB_CHECK_LAUNCH();
}

void divergence_sum(const float *wa, const float *f, const float *aa, int N, const float *wb, const float *g,
                    const float *bb, int M, double eps, double rho, double *d_out, double *d_part,
                    cudaStream_t st) {
    const int nblk = 128;
    const int balanced = std::isinf(rho) ? 1 : 0;
    divsum_partial_kernel<<<nblk, kRB, 0, st>>>(wa, f, aa, N, wb, g, bb, M, rho, balanced, d_part);
    OTGB_CHECK_LAUNCH();
    divsum_final_kernel<<<1, 32, 0, st>>>(d_part, nblk, rho, eps, balanced, d_out);
    OTGB_CHECK_LAUNCH();
}

void translate_duals(const float *wa, float *f, int N, const float *wb, float *g, int M, double rho, double2 *d_part,
                     double *d_c, cudaStream_t st) {
    const int nblk = 64;  // d_part holds 64 partials
    transl_partial_kernel<<<nblk, kRB, 0, st>>>(wa, f, N, wb, g, M, rho, d_part);
    OTGB_CHECK_LAUNCH();
    transl_apply_kernel<<<128, 256, 0, st>>>(d_part, nblk, rho, f, N, g, M, d_c);
    OTGB_CHECK_LAUNCH();
}

size_t scan_scratch_ints(int n) {
    const int nb = (n + kScanB - 1) / kScanB;
    return (size_t)nb + scan_scratch_ints_level(nb);
}
size_t scan_scratch_ints_level(int nb) {
    if (nb <= 1) return 2;
    return scan_scratch_ints(nb) + (size_t)nb;
}

void exclusive_scan(const int *in, int *out, int n, int *scratch, cudaStream_t st) {
    if (n <= 0) return;
    const int nb = (n + kScanB - 1) / kScanB;
    int *bsum = scratch;
    scan_block_kernel<<<nb, kScanB, 0, st>>>(in, out, n, bsum);
    OTGB_CHECK_LAUNCH();
    if (nb > 1) {
        int *boff = scratch + nb;
        exclusive_scan(bsum, boff, nb, boff + nb, st);
        scan_add_kernel<<<nb, kScanB, 0, st>>>(out, n, boff);
        OTGB_CHECK_LAUNCH();
    }
}

size_t radix_sort_scratch_bytes(int n) {
    const int nchunks = (n + kChunk - 1) / kChunk;
    const size_t cnt = (size_t)256 * nchunks;
    return sizeof(int) * (2 * cnt + scan_scratch_ints((int)cnt) + 64) + (sizeof(uint32_t) + sizeof(int)) * (size_t)n +
           256;
}

void radix_sort_pairs(uint32_t *keys, int *vals, int n, int nbits, void *scratch, cudaStream_t st) {
    if (n <= 1 || nbits <= 0) {
        if (n == 1) OTGB_CUDA_TRY(cudaMemsetAsync(vals, 0, sizeof(int), st));
        if (n > 1 && nbits <= 0) {
            // keys all equal: identity permutation
            iota(vals, n, st);
        }
        return;
    }
    const int nchunks = (n + kChunk - 1) / kChunk;
    const size_t cnt = (size_t)256 * nchunks;
    int *counts = static_cast<int *>(scratch);
    int *offs = counts + cnt;
    int *scan_scr = offs + cnt;
    uint8_t *p = reinterpret_cast<uint8_t *>(scan_scr + scan_scratch_ints((int)cnt) + 64);
    uint32_t *k2 = reinterpret_cast<uint32_t *>(p);
    int *v2 = reinterpret_cast<int *>(k2 + n);
    uint32_t *kin = keys, *kout = k2;
    int *vin = nullptr, *vout = v2;  // first pass: values are the input positions
    const int passes = (nbits + 7) / 8;
    for (int ps = 0; ps < passes; ++ps) {
        radix_hist_kernel<<<nchunks, kSortT, 0, st>>>(kin, n, 8 * ps, counts, nchunks);
        OTGB_CHECK_LAUNCH();
        exclusive_scan(counts, offs, (int)cnt, scan_scr, st);
        radix_scatter_kernel<<<nchunks, kSortT, 0, st>>>(kin, vin, n, 8 * ps, offs, nchunks, kout, vout);
        OTGB_CHECK_LAUNCH();
        // the next pass reads what this one wrote and overwrites the other buffer
        uint32_t *tk = kin;
        kin = kout;
        kout = tk;
        int *tv = vin ? vin : vals;
        vin = vout;
        vout = tv;
    }
    if (kin != keys) {
        OTGB_CUDA_TRY(cudaMemcpyAsync(keys, kin, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, st));
        OTGB_CUDA_TRY(cudaMemcpyAsync(vals, vin, sizeof(int) * n, cudaMemcpyDeviceToDevice, st));
    }
}

void iota(int *v, int n, cudaStream_t st) {
    iota_kernel<<<(n + 255) / 256, 256, 0, st>>>(v, n);
    OTGB_CHECK_LAUNCH();
}

void pack_points(const float *x, const float *w, const int *perm, int n, int D, const float *d_center, float *out,
                 float *logw, float *w_sorted, cudaStream_t st) {
    const int D4 = D <= 3 ? 4 : ((D + 3) & ~3);
    pack_kernel<<<(n + 255) / 256, 256, 0, st>>>(x, w, perm, n, D, D4, d_center, out, logw, w_sorted);
    OTGB_CHECK_LAUNCH();
}

void unpermute(const float *in, const int *perm, int n, float *out, cudaStream_t st) {
    unpermute_kernel<<<(n + 255) / 256, 256, 0, st>>>(in, perm, n, out);
    OTGB_CHECK_LAUNCH();
}

void permute(const float *in, const int *perm, int n, float *out, cudaStream_t st) {
    permute_kernel<<<(n + 255) / 256, 256, 0, st>>>(in, perm, n, out);
    OTGB_CHECK_LAUNCH();
}

void check_weights(const float *w, int n, int *d_bad, double *d_mass_part, cudaStream_t st) {
    check_weights_kernel<<<64, kRB, 0, st>>>(w, n, d_bad, d_mass_part);
    OTGB_CHECK_LAUNCH();
}

void check_points(const float *x, size_t n, int *d_bad, cudaStream_t st) {
    check_points_kernel<<<256, 256, 0, st>>>(x, n, d_bad);
    OTGB_CHECK_LAUNCH();
}

void absmax(const float *v, int n, unsigned *d_out, cudaStream_t st) {
    absmax_kernel<<<64, 256, 0, st>>>(v, n, d_out);
    OTGB_CHECK_LAUNCH();
}

void check_finite(const float *v, int n, int *d_bad, cudaStream_t st) {
    finite_kernel<<<128, 256, 0, st>>>(v, n, d_bad);
    OTGB_CHECK_LAUNCH();
}

void cluster_stats(const float *pts, int stride, int D, const float *w_sorted, const int *off, int ncl, float *cent,
                   int cstride, float *mass, float *radius, float *ssq, cudaStream_t st) {
    if (ncl <= 0) return;
    cluster_stats_kernel<<<ncl, 128, 0, st>>>(pts, stride, D, w_sorted, off, ncl, cent, cstride, mass, radius, ssq);
    OTGB_CHECK_LAUNCH();
}

}  // namespace otgb
