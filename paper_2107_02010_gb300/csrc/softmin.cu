// Fused softmin kernels: the log-domain update of the Algorithm in Section 2,
//
//   tilde_i = -lam * eps * log sum_j w_j exp((pot_j - |q_i - p_j|^2 / 2) / eps)
//   out_i   = old_i + omega (tilde_i - old_i)          (omega = 1/2: the paper's average)
//
// for up to four instances per launch (alpha<->alpha, beta<->beta, alpha->beta,
// beta->alpha), dense or over the kept columns of each row block (the
// block-sparse kernel truncation of Section 2).
//
// Arithmetic per pair.  Each CTA owns a block of rows; it picks a centre c (the
// centre of the rows' bounding box, or their mean in high dimension) and works
// in the shifted frame xt = x - c, yt = y - c, where
//   -|xt - yt|^2/2 = -|xt|^2/2 - |yt|^2/2 + xt.yt.
// The row term leaves the sum; per column the CTA stages, in shared memory,
//   Y_j = s yt_j  and  H_j = s (eps log w_j + pot_j - |yt_j|^2 / 2),   s = log2(e)/eps,
// and each row i carries a shift m_i, an estimate of its base-2 log-sum, so that
// each (i, j) term is 2^((H_j - m_i) + xt_i . Y_j): one add, D FMAs, one MUFU
// ex2, one add.  The shift comes from the old value of the row
// (m_i = s (|xt_i|^2/2 - old_i/lam), exact at the fixed point), or, when there is
// no old value, from a first pass that takes the exact maximum over the
// columns.  A row whose sum ends outside [2^-60, 2^60] (the estimate was off by
// more than 60 binades, so terms may have been flushed or may overflow) is
// recomputed by the safe two-pass kernel in the direct form -|x - y|^2/2.
// The per-row finish (log of the sum, the row term, the blend) is done in
// double precision.
#include <cfloat>
#include <cmath>

#include "otgb_internal.cuh"

namespace otgb {
namespace {

typedef unsigned long long u64;

__device__ __forceinline__ float ex2(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ u64 fma2(u64 a, u64 b, u64 c) {
    u64 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ u64 add2(u64 a, u64 b) {
    u64 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ u64 pack2(float lo, float hi) {
    u64 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void unpack2(u64 v, float &lo, float &hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}

template <int NT>
__device__ __forceinline__ float block_max(float v, float *red) {
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) red[w] = v;
    __syncthreads();
    float r = red[0];
#pragma unroll
    for (int k = 1; k < NT / 32; ++k) r = fmaxf(r, red[k]);
    return r;
}
template <int NT>
__device__ __forceinline__ float block_min(float v, float *red) {
    return -block_max<NT>(-v, red);
}

// The row finish shared by all kernels.  L2 = log2 sum_j 2^(...) including K;
// half_x2 = |xt_i|^2/2 (0 for the direct-difference fallback).
__device__ __forceinline__ void finish_row(const SoftminLaunch &L, const SoftminInst &I, int r, double L2,
                                           double half_x2, float &dmax) {
    const double tilde = -(double)I.lam * (L.eps_ln2 * L2 - half_x2);
    double nw = tilde;
    if (I.row_old) {
        const double old = (double)I.row_old[r];
        nw = old + (double)I.omega * (tilde - old);
        dmax = fmaxf(dmax, (float)(fabs(nw - old) / (double)L.eps));
    }
    I.row_out[r] = (float)nw;
}

__device__ __forceinline__ void push_fallback(const SoftminLaunch &L, int inst, int r, int blk) {
    const int k = atomicAdd(L.n_fallback, 1);
    if (k < L.fallback_cap) L.fallback[k] = make_int4(inst, r, blk, 0);
}

// ------------------------------------------------------------ D <= 3 ------
// Warp-granular: a block is the 32 x R rows of ONE warp (lane l owns rows
// r0 + l + 32 k, k < R), with its own column list; a CTA runs four independent
// warps.  Blocks therefore stay small (tight truncation unions) while each
// staged column still feeds R rows per lane, and no CTA barrier is needed.
// With R >= 2 the rows go in pairs through packed f32x2 FMAs.  Each warp
// stages 32 columns per tile as (Y0,Y0,Y1,Y1 | Y2,Y2,H,H), double buffered, so
// that one 16-byte shared load feeds a packed operand pair.  TWO = true: an
// exact-maximum first pass gives each row's shift (no old value).
// Tile width and resident CTAs per SM: 128 columns and 6 CTAs (80 registers)
// measured fastest on the track-density workload among 32/64/128 columns and
// 5-8 CTAs (the occupancy changes the step time by under 5 %).
#ifndef OTGB_SM3_TILE
#define OTGB_SM3_TILE 128
#endif
#ifndef OTGB_SM3_MINB
#define OTGB_SM3_MINB 6
#endif
constexpr int kW3 = 4;               // warps per CTA
constexpr int kT3 = OTGB_SM3_TILE;   // columns per warp tile (kT3 / 32 staged per lane)
constexpr int kCPL = kT3 / 32;

__device__ __forceinline__ bool row_sum_ok(float a) { return a >= 0x1p-60f && a <= 0x1p60f; }

__device__ __forceinline__ float warp_max(float v) {
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ float warp_min(float v) {
    for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Rows of a warp block in registers, translated by the centre of their
// bounding box; m = per-row shift from the old values (or 0 with TWO).
template <int R, bool TWO>
__device__ __forceinline__ void setup_rows3(const SoftminLaunch &L, const SoftminInst &I, int r0, int r1,
                                            float (&xr)[R][3], float (&m)[R], float (&c)[3]) {
    const int lane = threadIdx.x & 31;
    const float4 *rows4 = reinterpret_cast<const float4 *>(I.rows);
    float lo[3] = {FLT_MAX, FLT_MAX, FLT_MAX}, hi[3] = {-FLT_MAX, -FLT_MAX, -FLT_MAX};
#pragma unroll
    for (int k = 0; k < R; ++k) {
        const int r = r0 + lane + 32 * k;
        float4 p = make_float4(0.f, 0.f, 0.f, 0.f);
        if (r < r1) {
            p = rows4[r];
            lo[0] = fminf(lo[0], p.x); hi[0] = fmaxf(hi[0], p.x);
            lo[1] = fminf(lo[1], p.y); hi[1] = fmaxf(hi[1], p.y);
            lo[2] = fminf(lo[2], p.z); hi[2] = fmaxf(hi[2], p.z);
        }
        xr[k][0] = p.x; xr[k][1] = p.y; xr[k][2] = p.z;
    }
#pragma unroll
    for (int d = 0; d < 3; ++d) c[d] = 0.5f * (warp_min(lo[d]) + warp_max(hi[d]));
    const float s = L.s;
#pragma unroll
    for (int k = 0; k < R; ++k) {
        const int r = r0 + lane + 32 * k;
#pragma unroll
        for (int d = 0; d < 3; ++d) xr[k][d] = (r < r1) ? xr[k][d] - c[d] : 0.f;
        m[k] = 0.f;
        if (!TWO && r < r1) {
            const double hx = 0.5 * ((double)xr[k][0] * xr[k][0] + (double)xr[k][1] * xr[k][1] +
                                     (double)xr[k][2] * xr[k][2]);
            m[k] = (float)((double)s * (hx - (double)I.row_old[r] / (double)I.lam));
        }
    }
}

// Finish the R rows of this lane from their sums: flag, log, blend, write.
// The translated row point is recomputed from the packed rows (the same float
// subtraction as in setup_rows3, hence the same value), so that the row
// coordinates need not stay in registers through the column loop.
template <int R>
__device__ __forceinline__ void finish_rows3(const SoftminLaunch &L, const SoftminInst &I, int inst, int blk, int r0,
                                             int r1, const float (&c)[3], const float (&m)[R],
                                             const float (&tot)[R]) {
    const int lane = threadIdx.x & 31;
    const float4 *rows4 = reinterpret_cast<const float4 *>(I.rows);
    float dmax = 0.f;
#pragma unroll
    for (int k = 0; k < R; ++k) {
        const int r = r0 + lane + 32 * k;
        if (r >= r1) continue;
        const float a = tot[k];
        if (!row_sum_ok(a)) {
            push_fallback(L, inst, r, blk);
            continue;
        }
        const float4 p = rows4[r];
        const float x0 = p.x - c[0], x1 = p.y - c[1], x2 = p.z - c[2];
        const double hx = 0.5 * ((double)x0 * x0 + (double)x1 * x1 + (double)x2 * x2);
        finish_row(L, I, r, (double)m[k] + log2((double)a), hx, dmax);
    }
    dmax = warp_max(dmax);
    if (lane == 0 && L.delta_max) atomicMax(L.delta_max, __float_as_uint(dmax));
}

// One work item of the D <= 3 sweep, computed by one warp in its shared-memory
// slice `tile`.
template <int R, bool TWO>
__device__ __forceinline__ void softmin3_item(const SoftminLaunch &L, int it, float4 (*tile)[kT3][2]) {
    const int lane = threadIdx.x & 31;
    int4 item = L.items[it];
    OTGB_DCLAMP(item.x, 0, L.n_inst);
    const SoftminInst &I = L.inst[item.x];
    const int blk = item.y;
    int r0 = I.blk_row0[blk], r1 = I.blk_row0[blk + 1];
    OTGB_DCLAMP(r0, 0, I.n_rows + 1);
    OTGB_DCLAMP(r1, r0, min(I.n_rows, r0 + 32 * R) + 1);
    const float4 *cols4 = reinterpret_cast<const float4 *>(I.cols);
    const float eps = L.eps, s = L.s;

    float xr[R][3], m[R], c[3];
    setup_rows3<R, TWO>(L, I, r0, r1, xr, m, c);

    // this item's columns: positions [cb, ce) of the block's column sequence
    const int nkept = kept_cols(I, blk);
    int cb = item.z, ce = item.w;
    OTGB_DCLAMP(cb, 0, nkept + 1);
    OTGB_DCLAMP(ce, cb, nkept + 1);
    const int ncol = ce - cb;
    const int ntiles = (ncol + kT3 - 1) / kT3;
    ColWalk walk;

    // staging of one tile: lane l handles columns p0 + l + 32 u, u < kCPL.  The
    // column indices are fetched one tile ahead of the column data, so that the
    // list -> point dependency of a tile is resolved while the tile before it
    // is computed.
    auto load_idx = [&](int p0, int (&j)[kCPL]) {
#pragma unroll
        for (int u = 0; u < kCPL; ++u) {
            const int p = p0 + lane + 32 * u;
            int jj = -1;
            if (p < ncol) {
                jj = walk.at(cb + p);
                OTGB_DCLAMP(jj, 0, I.n_cols);
            }
            j[u] = jj;
        }
    };
    auto load_col = [&](const int (&j)[kCPL], float4 (&q)[kCPL], float (&pot)[kCPL]) {
#pragma unroll
        for (int u = 0; u < kCPL; ++u) {
            if (j[u] >= 0) {
                q[u] = cols4[j[u]];
                pot[u] = I.col_pot[j[u]];
            } else {
                q[u] = make_float4(0.f, 0.f, 0.f, -INFINITY);
                pot[u] = 0.f;
            }
        }
    };
    auto store_col = [&](int buf, const float4 (&q)[kCPL], const float (&pot)[kCPL]) {
#pragma unroll
        for (int u = 0; u < kCPL; ++u) {
            const float y0 = q[u].x - c[0], y1 = q[u].y - c[1], y2 = q[u].z - c[2];
            const float stuff = fmaf(eps, q[u].w, pot[u]);
            const float H = s * (stuff - 0.5f * (y0 * y0 + y1 * y1 + y2 * y2));
            const float Y0 = s * y0, Y1 = s * y1, Y2 = s * y2;
            tile[buf][lane + 32 * u][0] = make_float4(Y0, Y0, Y1, Y1);
            tile[buf][lane + 32 * u][1] = make_float4(Y2, Y2, H, H);
        }
    };

    constexpr int P = R / 2;  // packed row pairs
    u64 X0[P > 0 ? P : 1], X1[P > 0 ? P : 1], X2[P > 0 ? P : 1];
#pragma unroll
    for (int p = 0; p < P; ++p) {
        X0[p] = pack2(xr[2 * p][0], xr[2 * p + 1][0]);
        X1[p] = pack2(xr[2 * p][1], xr[2 * p + 1][1]);
        X2[p] = pack2(xr[2 * p][2], xr[2 * p + 1][2]);
    }

    float4 q[kCPL];
    float pot[kCPL];
    if constexpr (TWO) {
        // first pass: exact maximum of the exponents of each row
        float mx[R];
#pragma unroll
        for (int k = 0; k < R; ++k) mx[k] = -INFINITY;
        int jn[kCPL];
        walk.start(I, blk, cb);
        if (ntiles > 0) { load_idx(0, jn); load_col(jn, q, pot); store_col(0, q, pot); }
        if (ntiles > 1) load_idx(kT3, jn);
        __syncwarp();
        for (int tt = 0; tt < ntiles; ++tt) {
            const int buf = tt & 1;
            const bool more = tt + 1 < ntiles;
            if (more) {
                load_col(jn, q, pot);
                if (tt + 2 < ntiles) load_idx((tt + 2) * kT3, jn);
            }
            const int n = min(kT3, ncol - tt * kT3);
            for (int cc = 0; cc < n; ++cc) {
                const float4 a = tile[buf][cc][0], b = tile[buf][cc][1];
#pragma unroll
                for (int k = 0; k < R; ++k) {
                    float v = fmaf(xr[k][2], b.x, b.z);
                    v = fmaf(xr[k][1], a.z, v);
                    v = fmaf(xr[k][0], a.x, v);
                    mx[k] = fmaxf(mx[k], v);
                }
            }
            if (more) store_col(buf ^ 1, q, pot);
            __syncwarp();
        }
#pragma unroll
        for (int k = 0; k < R; ++k) m[k] = mx[k] > -INFINITY ? mx[k] : 0.f;
    }

    float tot[R];
#pragma unroll
    for (int k = 0; k < R; ++k) tot[k] = 0.f;
    u64 Mn[P > 0 ? P : 1];
#pragma unroll
    for (int p = 0; p < P; ++p) Mn[p] = pack2(-m[2 * p], -m[2 * p + 1]);

    int jn[kCPL];
    walk.start(I, blk, cb);
    if (ntiles > 0) { load_idx(0, jn); load_col(jn, q, pot); store_col(0, q, pot); }
    if (ntiles > 1) load_idx(kT3, jn);
    __syncwarp();
    for (int tt = 0; tt < ntiles; ++tt) {
        const int buf = tt & 1;
        const bool more = tt + 1 < ntiles;
        if (more) {
            load_col(jn, q, pot);
            if (tt + 2 < ntiles) load_idx((tt + 2) * kT3, jn);
        }
        int n = min(kT3, ncol - tt * kT3);
        n = (n + 3) & ~3;  // padded columns carry H = -inf
        if constexpr (R >= 2) {
            // two accumulators per row pair (even / odd columns) shorten the add chain
            u64 acc[P][2];
#pragma unroll
            for (int p = 0; p < P; ++p) acc[p][0] = acc[p][1] = 0ull;
            const ulonglong2 *tp = reinterpret_cast<const ulonglong2 *>(&tile[buf][0][0]);
#pragma unroll 4
            for (int cc = 0; cc < n; ++cc) {
                const ulonglong2 a = tp[2 * cc], b = tp[2 * cc + 1];
#pragma unroll
                for (int p = 0; p < P; ++p) {
                    u64 v = add2(b.y, Mn[p]);
                    v = fma2(X2[p], b.x, v);
                    v = fma2(X1[p], a.y, v);
                    v = fma2(X0[p], a.x, v);
                    float vl, vh;
                    unpack2(v, vl, vh);
                    acc[p][cc & 1] = add2(acc[p][cc & 1], pack2(ex2(vl), ex2(vh)));
                }
            }
#pragma unroll
            for (int p = 0; p < P; ++p) {
                float al, ah, bl, bh;
                unpack2(acc[p][0], al, ah);
                unpack2(acc[p][1], bl, bh);
                tot[2 * p] += al + bl;
                tot[2 * p + 1] += ah + bh;
            }
        } else {
            float acc0 = 0.f, acc1 = 0.f;
#pragma unroll 4
            for (int cc = 0; cc < n; cc += 2) {
                const float4 a = tile[buf][cc][0], b = tile[buf][cc][1];
                float v = fmaf(xr[0][2], b.x, b.z - m[0]);
                v = fmaf(xr[0][1], a.z, v);
                v = fmaf(xr[0][0], a.x, v);
                acc0 += ex2(v);
                const float4 a2 = tile[buf][cc + 1][0], b2 = tile[buf][cc + 1][1];
                float w = fmaf(xr[0][2], b2.x, b2.z - m[0]);
                w = fmaf(xr[0][1], a2.z, w);
                w = fmaf(xr[0][0], a2.x, w);
                acc1 += ex2(w);
            }
            tot[0] += acc0 + acc1;
        }
        __syncwarp();  // every lane is done reading buf before it is refilled
        if (more) store_col(buf ^ 1, q, pot);
        __syncwarp();
    }

    if (lane == 0 && L.pairs) atomicAdd(L.pairs, (unsigned long long)(r1 - r0) * (unsigned long long)ncol);
    if (L.part) {
        // split block: partial sums, finished by the warp that completes the
        // block's last item (or by softmin3_finalize_kernel)
#pragma unroll
        for (int k = 0; k < R; ++k) L.part[(size_t)it * kPartRows + lane + 32 * k] = tot[k];
        if (L.fin_count) {
            __threadfence();
            int fi = 0, done = 0;
            if (lane == 0) {
                fi = L.item_fin[it];
                OTGB_DCLAMP(fi, 0, L.n_fin);
                done = atomicAdd(L.fin_count + fi, 1) + 1;
            }
            fi = __shfl_sync(0xffffffffu, fi, 0);
            done = __shfl_sync(0xffffffffu, done, 0);
            const int4 fe = L.fin[fi];
            if (done == fe.w) {
                __threadfence();
#pragma unroll
                for (int k = 0; k < R; ++k) tot[k] = 0.f;
                for (int q = 0; q < fe.w; ++q) {
                    int item_q = fe.z + q;
                    OTGB_DCLAMP(item_q, 0, L.n_items);
#pragma unroll
                    for (int k = 0; k < R; ++k) tot[k] += __ldcg(L.part + (size_t)item_q * kPartRows + lane + 32 * k);
                }
                if constexpr (R >= 2) {
#pragma unroll
                    for (int p = 0; p < P; ++p) {
                        float lo, hi;
                        unpack2(Mn[p], lo, hi);
                        m[2 * p] = -lo;
                        m[2 * p + 1] = -hi;
                    }
                }
                finish_rows3<R>(L, I, item.x, blk, r0, r1, c, m, tot);
            }
        }
    } else {
        if constexpr (R >= 2) {
#pragma unroll
            for (int p = 0; p < P; ++p) {
                float lo, hi;
                unpack2(Mn[p], lo, hi);
                m[2 * p] = -lo;
                m[2 * p + 1] = -hi;
            }
        }
        finish_rows3<R>(L, I, item.x, blk, r0, r1, c, m, tot);
    }
}

// Warps take work items in order: statically (item = global warp index) or,
// when L.work_counter is set, from the counter until none is left, so that no
// warp idles while a slow item of its CTA finishes and the grid can be sized
// to the resident capacity.  Every item writes only its own rows or partial
// sums, so the result does not depend on which warp computed it.
template <int R, bool TWO>
__global__ void __launch_bounds__(32 * kW3, OTGB_SM3_MINB) softmin3_kernel(const __grid_constant__ SoftminLaunch L) {
    __shared__ __align__(16) float4 tiles[kW3][2][kT3][2];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float4 (*tile)[kT3][2] = tiles[warp];
    if (!L.work_counter) {
        const int it = blockIdx.x * kW3 + warp;
        if (it < L.n_items) softmin3_item<R, TWO>(L, it, tile);
        return;
    }
    for (;;) {
        int it = 0;
        if (lane == 0) it = atomicAdd(L.work_counter, 1);
        it = __shfl_sync(0xffffffffu, it, 0);
        if (it >= L.n_items) return;  // whole warp: no CTA-wide barrier in this kernel
        softmin3_item<R, TWO>(L, it, tile);
        __syncwarp();
    }
}

// Split blocks: one warp per block sums the partial sums of its items in item
// order (deterministic) and finishes the rows.  Only the EST shift is used
// with splitting.
template <int R>
__global__ void __launch_bounds__(32 * kW3) softmin3_finalize_kernel(const __grid_constant__ SoftminLaunch L) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int fi = blockIdx.x * kW3 + warp;
    if (fi >= L.n_fin) return;
    int4 fe = L.fin[fi];
    OTGB_DCLAMP(fe.x, 0, L.n_inst);
    const SoftminInst &I = L.inst[fe.x];
    const int blk = fe.y;
    int r0 = I.blk_row0[blk], r1 = I.blk_row0[blk + 1];
    OTGB_DCLAMP(r0, 0, I.n_rows + 1);
    OTGB_DCLAMP(r1, r0, min(I.n_rows, r0 + 32 * R) + 1);
    float xr[R][3], m[R], c[3];
    setup_rows3<R, false>(L, I, r0, r1, xr, m, c);
    float tot[R];
#pragma unroll
    for (int k = 0; k < R; ++k) tot[k] = 0.f;
    for (int q = 0; q < fe.w; ++q) {
        int item = fe.z + q;
        OTGB_DCLAMP(item, 0, L.n_items);
#pragma unroll
        for (int k = 0; k < R; ++k) tot[k] += L.part[(size_t)item * kPartRows + lane + 32 * k];
    }
    finish_rows3<R>(L, I, fe.x, blk, r0, r1, c, m, tot);
}

// ------------------------------------------------------------ 3 < D <= 64 --
// Register-tiled, packed along the coordinates: 256 threads, a block of 128
// rows times tiles of 64 columns; each thread computes 8 rows x 4 columns.
// Rows are staged once as X = s (x - c) and columns per tile as yt = y - c,
// both as PAIRS of consecutive coordinates (k-pair major), so that one packed
// f32x2 FMA advances one (row, column) term by two coordinates: the two
// halves of the accumulator hold the even and the odd partial dot products
// and are added once at the end.  The k-pair after the last coordinate pair
// carries the rest of the exponent: (1, -m_i) in the row operand against
// (H_j, 1) in the column operand, so the accumulator ends at
// H_j - m_i + X_i . yt_j and the epilogue is one add, ex2 and the sum.
// Per pair that is D/2 + 1 packed FMAs (D + 2 FP32 operations) for half the
// instructions of the scalar form.
//
// Column tiles flow through a two-stage pipeline without register staging:
// cp.async copies the raw coordinates (and log w_j, pot_j) of tile t+1 into
// shared memory while the CTA multiplies tile t; after the products each
// thread centres and repacks the part of tile t+1 that it copied itself (so
// the copy needs no barrier), issues the copies of tile t+2 into the slots it
// just read, and meets the others at one barrier per tile.  Each k-pair row of
// the column operand is padded by 16 bytes (kYS), so that every operand load
// address is a register plus an immediate and the loads are free of bank
// conflicts; the repacking stores, once per tile, take a 4-way conflict.
// TWO = true: an exact-maximum first pass gives each row's shift.
constexpr int kNTg = 256;
constexpr int kBM = 128;
constexpr int kBN = 64;
constexpr int kKP = 33;       // 32 coordinate pairs + the folded pair
constexpr int kXS = kBM + 2;  // float2 stride of a k-pair of X (spreads the staging stores over banks)
constexpr int kYS = kBN + 2;  // float2 stride of a k-pair of the column operand (16-byte aligned rows)

struct GenSmem {
    float2 xs[kKP][kXS];     // X pairs; pair KPD = (1, -m_i)
    float2 ys[3][kKP][kYS];  // yt pairs (columns 0 .. kBN-1 of each row); pair KPD = (H_j, 1); three tiles in flight
    float raw[kBN][64];      // raw column coordinates of the next tile, as copied
    float rlw[kBN];
    float rpot[kBN];
    float cen[64];
    float hx[kBM];           // |xt|^2 / 2
    float red[kNTg / 32];
    unsigned long long tbar;  // tile barrier (mbarrier, kNTg arrivals per phase)
};

__device__ __forceinline__ void mbar_arrive(unsigned long long *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"((uint32_t)__cvta_generic_to_shared(bar))
                 : "memory");
}
// true when the phase with the given parity completed within the iteration limit
__device__ __forceinline__ bool mbar_wait_parity(unsigned long long *bar, uint32_t parity) {
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(bar);
    uint32_t done = 0;
    for (int it = 0; it < (1 << 24) && !done; ++it)
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
    return done != 0;
}

__device__ __forceinline__ void cp_async16(void *dst, const void *src, int bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
                 "l"(src), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async4(void *dst, const void *src, int bytes) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
                 "l"(src), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait0() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ u64 mul2(u64 a, u64 b) {
    u64 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}


template <bool TWO, int KPT>
__global__ void __launch_bounds__(kNTg, 2) softmin_gen_kernel(const __grid_constant__ SoftminLaunch L, int D, int D4) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    GenSmem &S = *reinterpret_cast<GenSmem *>(smem_raw);
    int4 item = L.items[blockIdx.x];
    OTGB_DCLAMP(item.x, 0, L.n_inst);
    const SoftminInst &I = L.inst[item.x];
    const int blk = item.y;
    int r0 = I.blk_row0[blk], r1 = I.blk_row0[blk + 1];
    OTGB_DCLAMP(r0, 0, I.n_rows + 1);
    OTGB_DCLAMP(r1, r0, min(I.n_rows, r0 + kBM) + 1);
    const int nr = r1 - r0;
    const int t = threadIdx.x;
    const float eps = L.eps, s = L.s;
    OTGB_DCLAMP(D4, 4, 65);
    const int KPD = KPT > 0 ? KPT : (D4 >> 1);  // coordinate pairs; pair KPD is the folded one

    if (t == 0)
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"((uint32_t)__cvta_generic_to_shared(&S.tbar)),
                     "r"(kNTg));
    int nphase = 0;  // tile-barrier phases this thread has arrived at so far (all sweeps)
    bool timed_out = false;

    // ---- rows: raw pairs, centre (mean), X = s (x - c), |xt|^2 / 2, fold pair
    float *xsf = reinterpret_cast<float *>(&S.xs[0][0]);
    for (int e = t; e < kBM * D4; e += kNTg) {
        const int r = e / D4, k = e - r * D4;
        xsf[(k >> 1) * (2 * kXS) + 2 * r + (k & 1)] = (r < nr) ? I.rows[(size_t)(r0 + r) * D4 + k] : 0.f;
    }
    __syncthreads();
    if (t < 64) {
        float acc = 0.f;
        if (t < D4)
            for (int r = 0; r < nr; ++r) acc += xsf[(t >> 1) * (2 * kXS) + 2 * r + (t & 1)];
        S.cen[t] = (t < D4 && nr > 0) ? acc / (float)nr : 0.f;
    }
    __syncthreads();
    if (t < kBM) {
        float sq = 0.f;
        for (int kp = 0; kp < KPD; ++kp) {
            float2 v = S.xs[kp][t];
            v.x = (t < nr) ? v.x - S.cen[2 * kp] : 0.f;
            v.y = (t < nr) ? v.y - S.cen[2 * kp + 1] : 0.f;
            sq = fmaf(v.x, v.x, fmaf(v.y, v.y, sq));
            S.xs[kp][t] = make_float2(s * v.x, s * v.y);
        }
        const float h = 0.5f * sq;
        S.hx[t] = h;
        float m = 0.f;
        if (!TWO && t < nr) m = (float)((double)s * ((double)h - (double)I.row_old[r0 + t] / (double)I.lam));
        S.xs[KPD][t] = make_float2(1.f, -m);
    }

    // ---- columns of this item: positions [cb, ce) of the block's columns (never split for D > 3)
    const int nkept = kept_cols(I, blk);
    int cb = item.z, ce = item.w;
    OTGB_DCLAMP(cb, 0, nkept + 1);
    OTGB_DCLAMP(ce, cb, nkept + 1);
    const int ncol = ce - cb;
    const int ntiles = (ncol + kBN - 1) / kBN;
    ColWalk walk;

    // copy/repack roles: chunk ch (coordinates 8 ch .. 8 ch + 7) of columns colb and colb + 32
    const int ch = t & 7, colb = t >> 3;
    // product roles: rows 8 tr .. 8 tr + 7, 16-byte chunks tc and tc + 16 of a row (columns 2 tc, 2 tc + 1, +32)
    const int tr = t >> 4, tc = t & 15;

    auto load_idx = [&](int tile, int (&j)[2]) {
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int p = tile * kBN + colb + 32 * q;
            int jj = -1;
            if (tile < ntiles && p < ncol) {
                jj = walk.at(cb + p);
                OTGB_DCLAMP(jj, 0, I.n_cols);
            }
            j[q] = jj;
        }
    };
    auto issue = [&](const int (&j)[2]) {
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int col = colb + 32 * q;
            const bool ok = j[q] >= 0;
            // a copy of size 0 fills zeros and reads nothing; its source is then the valid base
            const bool k0 = ok && 8 * ch + 4 <= D4, k1 = ok && 8 * ch + 8 <= D4;
            const float *src = I.cols + (ok ? (size_t)j[q] * D4 + 8 * ch : 0);
            cp_async16(&S.raw[col][8 * ch], k0 ? src : I.cols, k0 ? 16 : 0);
            cp_async16(&S.raw[col][8 * ch + 4], k1 ? src + 4 : I.cols, k1 ? 16 : 0);
            if (ch == 0) {
                cp_async4(&S.rlw[col], ok ? I.col_logw + j[q] : I.col_logw, ok ? 4 : 0);
                cp_async4(&S.rpot[col], ok ? I.col_pot + j[q] : I.col_pot, ok ? 4 : 0);
            }
        }
    };
    // centre and repack into ys[buf] the part of tile `tile` this thread copied into raw
    // (a column past the end has H = -inf, which zeroes its terms whatever its coordinates)
    auto repack = [&](int buf, int tile) {
        const float4 ca = *reinterpret_cast<const float4 *>(&S.cen[8 * ch]);
        const float4 cc = *reinterpret_cast<const float4 *>(&S.cen[8 * ch + 4]);
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int col = colb + 32 * q;
            const bool ok = tile * kBN + col < ncol;
            const float4 a = *reinterpret_cast<const float4 *>(&S.raw[col][8 * ch]);
            const float4 b = *reinterpret_cast<const float4 *>(&S.raw[col][8 * ch + 4]);
            float v[8] = {a.x - ca.x, a.y - ca.y, a.z - ca.z, a.w - ca.w, b.x - cc.x, b.y - cc.y, b.z - cc.z, b.w - cc.w};
            float sq = 0.f;
#pragma unroll
            for (int e = 0; e < 8; ++e) sq = fmaf(v[e], v[e], sq);
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int kp = 4 * ch + e;
                if (kp < KPD) S.ys[buf][kp][col] = make_float2(v[2 * e], v[2 * e + 1]);
            }
            sq += __shfl_xor_sync(0xffffffffu, sq, 1);
            sq += __shfl_xor_sync(0xffffffffu, sq, 2);
            sq += __shfl_xor_sync(0xffffffffu, sq, 4);
            if (ch == 0) {
                const float H = ok ? s * (fmaf(eps, S.rlw[col], S.rpot[col]) - 0.5f * sq) : -INFINITY;
                S.ys[buf][KPD][col] = make_float2(H, 1.f);
            }
        }
    };

    // acc[i][jj] = X_i . yt_j over the folded pair (first) and every coordinate pair of the
    // tile in ys[buf]; KPT > 0 unrolls the k-pairs completely, so that every shared
    // address is a register plus an immediate
    const int kpd = KPD;
    auto products = [&](int buf, u64 (&acc)[8][4]) {
        const char *xs0 = reinterpret_cast<const char *>(&S.xs[0][tr * 8]);
        const char *ys0 = reinterpret_cast<const char *>(&S.ys[buf][0][0]);
        auto step = [&](int kp, bool first) {
            const char *yp = ys0 + kp * (kYS * 8) + (tc << 4);
            const ulonglong2 y0 = *reinterpret_cast<const ulonglong2 *>(yp);
            const ulonglong2 y1 = *reinterpret_cast<const ulonglong2 *>(yp + 256);
            const u64 yv[4] = {y0.x, y0.y, y1.x, y1.y};
            const char *xp = xs0 + kp * (kXS * 8);
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                const ulonglong2 x2 = *reinterpret_cast<const ulonglong2 *>(xp + 16 * h);
#pragma unroll
                for (int jj = 0; jj < 4; ++jj) {
                    acc[2 * h][jj] = first ? mul2(x2.x, yv[jj]) : fma2(x2.x, yv[jj], acc[2 * h][jj]);
                    acc[2 * h + 1][jj] = first ? mul2(x2.y, yv[jj]) : fma2(x2.y, yv[jj], acc[2 * h + 1][jj]);
                }
            }
        };
        step(kpd, true);  // acc = (H_j, -m_i)
        if constexpr (KPT > 0) {
#pragma unroll
            for (int kp = 0; kp < KPT; ++kp) step(kp, false);
        } else {
#pragma unroll 1
            for (int kp = 0; kp < KPD; kp += 2) {  // KPD is even (D4 is a multiple of 4)
                step(kp, false);
                step(kp + 1, false);
            }
        }
    };

    // one sweep over the column tiles; MAXP: per-row maximum of the exponent, else the sum
    float res[8];
    auto sweep = [&](bool MAXP) {
#pragma unroll
        for (int i = 0; i < 8; ++i) res[i] = MAXP ? -INFINITY : 0.f;
        if (ntiles == 0) return;
        // Three column tiles in flight: tiles t and t+1 are repacked while the CTA multiplies
        // tile t, and the repack of tile t+2 (into the buffer of tile t-1) needs only that every
        // thread has finished iteration t-1 -- one tile of slack, so a warp that is ahead does not
        // wait for the slowest warp's products of the same tile.  Iteration t: products(t); wait
        // for phase t-1 (all threads past repack(t+1), hence past products(t-1)); repack(t+2);
        // arrive at phase t; fold tile t into the row sums.  (Checked on a CPU model of the
        // mbarrier over random interleavings before it ran on a GPU.)
        int jn[2];
        walk.start(I, blk, cb);
        load_idx(0, jn);
        issue(jn);
        cp_async_commit();
        load_idx(1, jn);
        cp_async_wait0();
        repack(0, 0);
        issue(jn);  // tile 1 (nothing past the end)
        cp_async_commit();
        load_idx(2, jn);
        cp_async_wait0();
        repack(1, 1);
        issue(jn);  // tile 2
        cp_async_commit();
        load_idx(3, jn);
        __syncthreads();
        const int ph0 = nphase;
        for (int tt = 0; tt < ntiles; ++tt) {
            const int buf = tt % 3;
            u64 acc[8][4];
            products(buf, acc);
            if (tt >= 1 && tt + 1 < ntiles) {  // phase tt - 1 was arrived at (tt + 1 < ntiles)
                if (!mbar_wait_parity(&S.tbar, (uint32_t)((ph0 + tt - 1) & 1))) timed_out = true;
            }
            if (tt + 2 < ntiles) {
                cp_async_wait0();  // this thread's copies of tile tt+2
                repack((tt + 2) % 3, tt + 2);
                if (tt + 3 < ntiles) issue(jn);  // into the raw slots just consumed
                cp_async_commit();
                load_idx(tt + 4, jn);
                mbar_arrive(&S.tbar);  // phase ph0 + tt
                ++nphase;
            }
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                float e[4];
#pragma unroll
                for (int jj = 0; jj < 4; ++jj) {
                    float lo, hi;
                    unpack2(acc[i][jj], lo, hi);
                    e[jj] = lo + hi;
                }
                if (MAXP) res[i] = fmaxf(res[i], fmaxf(fmaxf(e[0], e[1]), fmaxf(e[2], e[3])));
                else res[i] += (ex2(e[0]) + ex2(e[1])) + (ex2(e[2]) + ex2(e[3]));
            }
        }
        cp_async_wait0();
    };

    if constexpr (TWO) {
        sweep(true);
#pragma unroll
        for (int i = 0; i < 8; ++i)
            for (int o = 8; o > 0; o >>= 1) res[i] = fmaxf(res[i], __shfl_xor_sync(0xffffffffu, res[i], o));
        __syncthreads();
        if (tc == 0)
#pragma unroll
            for (int i = 0; i < 8; ++i) S.xs[kpd][tr * 8 + i].y = res[i] > -INFINITY ? -res[i] : 0.f;
    }
    __syncthreads();
    sweep(false);
    // reduce the 16 column-threads of each row group (lanes of one half-warp); lane tc < 8
    // then finishes row 8 tr + tc
#pragma unroll
    for (int i = 0; i < 8; ++i)
        for (int o = 8; o > 0; o >>= 1) res[i] += __shfl_xor_sync(0xffffffffu, res[i], o);
    float a = res[0];
#pragma unroll
    for (int i = 1; i < 8; ++i) a = (tc == i) ? res[i] : a;
    float dmax = 0.f;
    const int rr = tr * 8 + tc;
    if (tc < 8 && rr < nr) {
        const int r = r0 + rr;
        const float mi = -S.xs[kpd][rr].y;
        if (!row_sum_ok(a)) push_fallback(L, item.x, r, blk);
        else finish_row(L, I, r, (double)mi + log2((double)a), (double)S.hx[rr], dmax);
    }
    dmax = block_max<kNTg>(dmax, S.red);
    if (t == 0) {
        if (L.delta_max) atomicMax(L.delta_max, __float_as_uint(dmax));
        if (L.pairs) atomicAdd(L.pairs, (unsigned long long)nr * (unsigned long long)ncol);
    }
    if (timed_out && L.tc_err) atomicOr(L.tc_err, 2u);
}

// ------------------------------------------------------------- fallback ---
// Rows flagged by the fast kernels, one CTA per row (grid-stride over the
// device-side count, so the launch needs no host synchronisation): two passes
// over the row's columns in the direct form -|x - y|^2/2 (no cancellation),
// max first, then the shifted sum in double.
constexpr int kFbThreads = 256;

__global__ void __launch_bounds__(kFbThreads) softmin_fallback_kernel(const __grid_constant__ SoftminLaunch L, int D,
                                                                      int stride) {
    __shared__ __align__(16) float xs[64];
    __shared__ float redf[kFbThreads / 32];
    __shared__ double redd[kFbThreads / 32];
    const int count = min(*L.n_fallback, L.fallback_cap);
    if (blockIdx.x == 0 && threadIdx.x == 0 && L.fallback_total && count > 0)
        atomicAdd(L.fallback_total, (unsigned long long)count);
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    for (int q = blockIdx.x; q < count; q += gridDim.x) {
        int4 fb = L.fallback[q];
        OTGB_DCLAMP(fb.x, 0, L.n_inst);
        const SoftminInst &I = L.inst[fb.x];
        OTGB_DCLAMP(fb.y, 0, I.n_rows);
        const int r = fb.y, blk = fb.z;
        const int n = kept_cols(I, blk);
        ColWalk walk;
        __syncthreads();  // the previous row is done with xs and the reductions
        if (t < stride) xs[t] = I.rows[(size_t)r * stride + t];
        __syncthreads();
        const float eps = L.eps, s = L.s;
        const int n4 = stride >> 2;
        auto term = [&](int p) -> float {
            int j = walk.at(p);
            OTGB_DCLAMP(j, 0, I.n_cols);
            const float4 *yj = reinterpret_cast<const float4 *>(I.cols + (size_t)j * stride);
            float d2 = 0.f, lw;
            if (D <= 3) {
                const float4 v = yj[0];
                const float t0 = xs[0] - v.x, t1 = D > 1 ? xs[1] - v.y : 0.f, t2 = D > 2 ? xs[2] - v.z : 0.f;
                d2 = fmaf(t0, t0, fmaf(t1, t1, t2 * t2));
                lw = v.w;
            } else {
                // coordinates past D are zero on both sides
                for (int k4 = 0; k4 < n4; ++k4) {
                    const float4 v = yj[k4];
                    const float4 u = *reinterpret_cast<const float4 *>(&xs[4 * k4]);
                    const float t0 = u.x - v.x, t1 = u.y - v.y, t2 = u.z - v.z, t3 = u.w - v.w;
                    d2 = fmaf(t0, t0, fmaf(t1, t1, fmaf(t2, t2, fmaf(t3, t3, d2))));
                }
                lw = I.col_logw[j];
            }
            return s * (fmaf(eps, lw, I.col_pot[j]) - 0.5f * d2);
        };
        float m = -INFINITY;
        walk.start(I, blk, t);
        for (int p = t; p < n; p += kFbThreads) m = fmaxf(m, term(p));
        for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (lane == 0) redf[wid] = m;
        __syncthreads();
        m = redf[0];
#pragma unroll
        for (int k = 1; k < kFbThreads / 32; ++k) m = fmaxf(m, redf[k]);
        double acc = 0.0;
        walk.start(I, blk, t);
        if (m > -INFINITY)
            for (int p = t; p < n; p += kFbThreads) acc += (double)exp2f(term(p) - m);
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) redd[wid] = acc;
        __syncthreads();
        if (t == 0) {
            acc = 0.0;
            for (int k = 0; k < kFbThreads / 32; ++k) acc += redd[k];
            float dmax = 0.f;
            const double L2 = (m > -INFINITY) ? (double)m + log2(acc) : -INFINITY;
            finish_row(L, I, r, L2, 0.0, dmax);
            if (L.delta_max) atomicMax(L.delta_max, __float_as_uint(dmax));
        }
    }
}

__global__ void uniform_blocks_kernel(int *blk_row0, int n, int block_rows, int nb) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k <= nb) blk_row0[k] = min(k * block_rows, n);
}

}  // namespace

int uniform_blocks(int *d_blk_row0, int n, int block_rows, cudaStream_t st) {
    const int nb = (n + block_rows - 1) / block_rows;
    uniform_blocks_kernel<<<(nb + 1 + 255) / 256, 256, 0, st>>>(d_blk_row0, n, block_rows, nb);
    OTGB_CHECK_LAUNCH();
    return nb;
}

namespace {

// Grid of the D <= 3 kernel: one warp per item, or, with a work counter, at most
// the CTAs that fit on the GPU at once (each warp then takes items until none
// is left).
template <int R, bool TWO>
void launch_softmin3(const SoftminLaunch &L, cudaStream_t st) {
    int grid = (L.n_items + kW3 - 1) / kW3;
    if (L.work_counter) {
        static PerDevice<int> cap_of;
        const int cap = cap_of.get([] {
            int dev = 0, sms = 0, occ = 0;
            OTGB_CUDA_TRY(cudaGetDevice(&dev));
            OTGB_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
            OTGB_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, softmin3_kernel<R, TWO>, 32 * kW3, 0));
            return sms * (occ > 0 ? occ : 1);
        });
        grid = grid < cap ? grid : cap;
    }
    softmin3_kernel<R, TWO><<<grid, 32 * kW3, 0, st>>>(L);
}

}  // namespace

namespace {
int fallback_grid_sms() {
    static PerDevice<int> sms_of;
    return sms_of.get([] {
        int dev = 0, sms = 0;
        OTGB_CUDA_TRY(cudaGetDevice(&dev));
        OTGB_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        return sms > 0 ? sms : 1;
    });
}
}  // namespace

void softmin_run(const SoftminLaunch &L, int D, int rows_per_thread, cudaStream_t st) {
    if (L.n_items <= 0) return;
    OTGB_CUDA_TRY(cudaMemsetAsync(L.n_fallback, 0, sizeof(int), st));
    if (L.cost_p1 || L.direct) {  // the direct form with a running maximum: no shift estimate, no fallback rows
        softmin_direct_launch(L, D, st);
        return;
    }
    // the first-pass maximum is needed when some instance has no old value
    bool two = L.exact_max != 0;
    for (int k = 0; k < L.n_inst; ++k) two = two || (L.inst[k].row_old == nullptr);
    require(!(two && L.part), "softmin_run: split blocks need old values", OTGB_EINTERNAL);
    require(!(D > 3 && L.part), "softmin_run: split blocks are D <= 3 only", OTGB_EINTERNAL);
    if (D <= 3 && L.use_tc3 && !two && rows_per_thread <= 4 && (!L.part || L.fin_count)) {
        if (L.part) OTGB_CUDA_TRY(cudaMemsetAsync(L.fin_count, 0, sizeof(int) * L.n_fin, st));
        softmin3_tc_launch(L, st);
    } else if (D <= 3) {
        if (L.work_counter) OTGB_CUDA_TRY(cudaMemsetAsync(L.work_counter, 0, sizeof(int), st));
        if (L.part && L.fin_count) OTGB_CUDA_TRY(cudaMemsetAsync(L.fin_count, 0, sizeof(int) * L.n_fin, st));
        switch (rows_per_thread + (two ? 8 : 0)) {
            case 1: launch_softmin3<1, false>(L, st); break;
            case 2: launch_softmin3<2, false>(L, st); break;
            case 4: launch_softmin3<4, false>(L, st); break;
            case 9: launch_softmin3<1, true>(L, st); break;
            case 10: launch_softmin3<2, true>(L, st); break;
            default: launch_softmin3<4, true>(L, st); break;
        }
        OTGB_CHECK_LAUNCH();
        if (L.part && L.n_fin > 0 && !L.fin_count) {
            const int fgrid = (L.n_fin + kW3 - 1) / kW3;
            switch (rows_per_thread) {
                case 1: softmin3_finalize_kernel<1><<<fgrid, 32 * kW3, 0, st>>>(L); break;
                case 2: softmin3_finalize_kernel<2><<<fgrid, 32 * kW3, 0, st>>>(L); break;
                default: softmin3_finalize_kernel<4><<<fgrid, 32 * kW3, 0, st>>>(L); break;
            }
            OTGB_CHECK_LAUNCH();
        }
    } else {
        const int D4 = (D + 3) & ~3;
        static PerDevice<int> attr;
        attr.get([] {
            const int bytes = (int)sizeof(GenSmem);
            OTGB_CUDA_TRY(cudaFuncSetAttribute(softmin_gen_kernel<false, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
            OTGB_CUDA_TRY(cudaFuncSetAttribute(softmin_gen_kernel<false, 30>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
            OTGB_CUDA_TRY(cudaFuncSetAttribute(softmin_gen_kernel<false, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
            OTGB_CUDA_TRY(cudaFuncSetAttribute(softmin_gen_kernel<true, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
            return 1;
        });
        if (two) {
            softmin_gen_kernel<true, 0><<<L.n_items, kNTg, sizeof(GenSmem), st>>>(L, D, D4);
            OTGB_CHECK_LAUNCH();
        } else if (L.use_tc && D >= 16) {
            if (L.use_tcc) softmin_tcc_launch(L, D, st);
            else softmin_tc_launch(L, D, st);
        } else {
            // the k-pair loop unrolled at compile time for 60- and 64-wide points
            if (D4 == 60) softmin_gen_kernel<false, 30><<<L.n_items, kNTg, sizeof(GenSmem), st>>>(L, D, D4);
            else if (D4 == 64) softmin_gen_kernel<false, 32><<<L.n_items, kNTg, sizeof(GenSmem), st>>>(L, D, D4);
            else softmin_gen_kernel<false, 0><<<L.n_items, kNTg, sizeof(GenSmem), st>>>(L, D, D4);
            OTGB_CHECK_LAUNCH();
        }
    }
    const int stride = D <= 3 ? 4 : ((D + 3) & ~3);
    softmin_fallback_kernel<<<2 * fallback_grid_sms(), kFbThreads, 0, st>>>(L, D, stride);
    OTGB_CHECK_LAUNCH();
}

}  // namespace otgb
