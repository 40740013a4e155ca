// Softmin in the direct difference form, for the costs C(x, y) = |x - y|
// (p = 1 in the cost |x - y|^p / p of Section 2) and |x - y|^2 / 2 (p = 2):
//
//   tilde_i = -lam * eps * log sum_j w_j exp((pot_j - C(q_i, p_j)) / eps)
//
// For p = 1 the distance is not a polynomial in the coordinates, so the
// dot-product shortcut of the other kernels does not apply.  For p = 2 this
// kernel is the accurate one: the dot-product form adds terms as large as
// s |x - c| |y - c| (c the block's centre) whose rounding does not shrink with
// the pair's cost, while |x - y|^2 summed from differences is exact to a few
// units in the last place of the cost itself -- small for every pair that
// matters.  Per pair: D subtractions and FMAs (and a square root for p = 1),
// then one ex2.
// One CTA of 128 threads owns a row block (one row per thread, its point in
// registers); the block's columns are staged in shared memory, 32 per tile,
// and read as broadcasts.  Each row keeps a running maximum of its base-2
// exponents and rescales its sum when the maximum grows, so no shift has to
// be known in advance and no row needs a second pass.
#include <cmath>

#include "otgb_internal.cuh"

namespace otgb {
namespace {

constexpr int kP1R = 128;  // rows per CTA (row blocks have at most 128 rows)
constexpr int kP1C = 32;   // columns per shared tile

__device__ __forceinline__ float ex2p(float v) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(v));
    return y;
}

// D4 = padded width of a point: 4 for D <= 3 (float4 (x, y, z, log w) columns), else round_up(D, 4).
template <int D4, bool P1>
__global__ void __launch_bounds__(kP1R) softmin_direct_kernel(const __grid_constant__ SoftminLaunch L, int D) {
    __shared__ float ys[kP1C][D4];
    __shared__ float yh[kP1C];  // log2 w_j + s pot_j (-inf: no column)
    __shared__ int yj[kP1C];    // column index of each tile column
    __shared__ float red[kP1R / 32];
    int4 item = L.items[blockIdx.x];
    OTGB_DCLAMP(item.x, 0, L.n_inst);
    const SoftminInst &I = L.inst[item.x];
    const int blk = item.y;
    int r0 = I.blk_row0[blk], r1 = I.blk_row0[blk + 1];
    OTGB_DCLAMP(r0, 0, I.n_rows + 1);
    OTGB_DCLAMP(r1, r0, min(I.n_rows, r0 + kP1R) + 1);
    const int nr = r1 - r0;
    const int t = threadIdx.x;
    const bool valid = t < nr;
    const int r = r0 + t;
    const int ncoord = D <= 3 ? D : D4;  // coordinates past D are zero on both sides when D > 3
    float x[D4];
#pragma unroll
    for (int d = 0; d < D4; ++d) x[d] = (valid && d < ncoord) ? I.rows[(size_t)r * D4 + d] : 0.f;

    const int nkept = kept_cols(I, blk);
    int cb = item.z, ce = item.w;
    OTGB_DCLAMP(cb, 0, nkept + 1);
    OTGB_DCLAMP(ce, cb, nkept + 1);
    const int ncol = ce - cb;
    const float s = L.s;
    float m = -INFINITY, acc = 0.f;
    // thread t < kP1C finds column p0 + t of each tile
    ColWalk walk;
    walk.start(I, blk, cb);
    for (int p0 = 0; p0 < ncol; p0 += kP1C) {
        const int nc = min(kP1C, ncol - p0);
        __syncthreads();
        if (t < kP1C) {
            float h = -INFINITY;
            int j = -1;
            if (t < nc) {
                j = walk.at(cb + p0 + t);
                OTGB_DCLAMP(j, 0, I.n_cols);
                const float lw = D <= 3 ? I.cols[(size_t)j * 4 + 3] : I.col_logw[j];
                h = lw == -INFINITY ? -INFINITY : fmaf(kLog2e, lw, s * I.col_pot[j]);
            }
            yj[t] = j;
            yh[t] = h;
        }
        __syncthreads();
        for (int e = t; e < kP1C * D4; e += kP1R) {
            const int c = e / D4, d = e - c * D4;
            float v = 0.f;
            if (c < nc && d < ncoord) {
                int j = yj[c];
                OTGB_DCLAMP(j, 0, I.n_cols);
                v = I.cols[(size_t)j * D4 + d];
            }
            ys[c][d] = v;
        }
        __syncthreads();
        for (int c = 0; c < nc; ++c) {
            const float h = yh[c];
            if (h == -INFINITY) continue;  // the same column for every thread
            float sq = 0.f;
#pragma unroll
            for (int d = 0; d < D4; ++d) {
                const float df = x[d] - ys[c][d];
                sq = fmaf(df, df, sq);
            }
            const float e = P1 ? fmaf(-s, sqrtf(sq), h) : fmaf(-0.5f * s, sq, h);
            if (e > m) {
                acc *= ex2p(m - e);
                m = e;
            }
            acc += ex2p(e - m);
        }
    }
    float dmax = 0.f;
    if (valid) {
        // L2 = m + log2(acc): the base-2 log of sum_j w_j exp((pot_j - C(q_i, p_j)) / eps)
        const double L2 = (m > -INFINITY) ? (double)m + log2((double)acc) : -INFINITY;
        const double tilde = -(double)I.lam * (L.eps_ln2 * L2);
        double nw = tilde;
        if (I.row_old) {
            const double old = (double)I.row_old[r];
            nw = old + (double)I.omega * (tilde - old);
            dmax = fmaxf(dmax, (float)(fabs(nw - old) / (double)L.eps));
        }
        I.row_out[r] = (float)nw;
    }
    for (int o = 16; o > 0; o >>= 1) dmax = fmaxf(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
    if ((t & 31) == 0) red[t >> 5] = dmax;
    __syncthreads();
    if (t == 0) {
        for (int k = 1; k < kP1R / 32; ++k) dmax = fmaxf(dmax, red[k]);
        if (L.delta_max) atomicMax(L.delta_max, __float_as_uint(dmax));
        if (L.pairs) atomicAdd(L.pairs, (unsigned long long)nr * (unsigned long long)ncol);
    }
}

}  // namespace

void softmin_direct_launch(const SoftminLaunch &L, int D, cudaStream_t st) {
    require(!L.part, "softmin_direct_launch: split blocks are not supported", OTGB_EINTERNAL);
    const int D4 = D <= 3 ? 4 : ((D + 3) & ~3);
    switch (D4 + (L.cost_p1 ? 1000 : 0)) {
#define OTGB_P1_CASE(K)                                                                   \
    case K: softmin_direct_kernel<K, false><<<L.n_items, kP1R, 0, st>>>(L, D); break;     \
    case 1000 + K: softmin_direct_kernel<K, true><<<L.n_items, kP1R, 0, st>>>(L, D); break;
        OTGB_P1_CASE(4) OTGB_P1_CASE(8) OTGB_P1_CASE(12) OTGB_P1_CASE(16)
        OTGB_P1_CASE(20) OTGB_P1_CASE(24) OTGB_P1_CASE(28) OTGB_P1_CASE(32)
        OTGB_P1_CASE(36) OTGB_P1_CASE(40) OTGB_P1_CASE(44) OTGB_P1_CASE(48)
        OTGB_P1_CASE(52) OTGB_P1_CASE(56) OTGB_P1_CASE(60) OTGB_P1_CASE(64)
#undef OTGB_P1_CASE
        default: throw Error{OTGB_EINTERNAL, "softmin_direct_launch: D out of range"};
    }
    OTGB_CHECK_LAUNCH();
}

}  // namespace otgb
