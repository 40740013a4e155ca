// Cluster-tiled tensor-core form of the softmin sweep (16 <= D, D4 <= 60, coarse-to-fine solves): the
// reduced-precision cross term of the tensor-core form, with the column operand prepared once per solve.
//
// In the kernel truncation of Section 2 every row block walks the columns of its kept column clusters J.
// Centring the pair at the column cluster's centre c_J instead of at the row block's centre,
//   -|x_i - y_j|^2 / 2 = (x_i - c_J) . yh_j - |x_i - c_J|^2 / 2 - |yh_j|^2 / 2,   yh_j = y_j - c_J,
// makes the column operand yh_j independent of the row block: it is split into BF16 hi + lo once per solve
// and stored in global memory as ready tiles of 128 columns in the canonical K-major layout of the tensor
// core (tcc_build), so the kernel copies each tile with one bulk TMA copy and the CUDA cores do no column
// work at all.  The rest of the exponent rides in the free K slots 60..63 (D4 <= 60):
//   column slots: 60 = (H1 | H2 in the lo piece), 61 = H3, 62 = 1, 63 = 1,
//                 H_j = s (eps log w_j + pot_j - |yh_j|^2 / 2) in three BF16 pieces (rewritten every step
//                 by tcc_update);
//   row slots:    60 = 1, 61 = 1, 62 = (R1 | R2 in the lo piece), 63 = R3,
//                 R_iJ = -s |x_i - c_J|^2 / 2 - M_i in three pieces, M_i = -s old_i / lam,
// so that the three products hi.hi + hi.lo + lo.hi of every K step leave in the accumulator
//   e_ij = s (x_i - c_J) . yh_j + H_j + R_iJ = (exponent of the pair in base 2) - M_i,
// and the finish takes M_i + log2 sum_j 2^e_ij in double.  The row operand s (x_i - c_J) (hi + lo, with
// the R slots) is restaged once per kept cluster of the block.
//
// One CTA (4 warps, one tensor-memory lane per row) owns a block of at most 128 rows.  Thread 0 issues the
// bulk copies (two shared-memory stages of a 32 KiB tile: hi then lo) and the MMAs (two 128-column
// accumulators), so that the MMA of tile k+1 runs while the CTA sums tile k; the threads hand an
// accumulator back through an mbarrier, so the only CTA barriers are the restagings of the row operand.
// Every wait is bounded; a timeout sets an error word and the kernel still releases its tensor memory.
#include <cfloat>
#include <cmath>

#include <cuda_bf16.h>

#include "otgb_internal.cuh"
#include "tcgen05.cuh"

namespace otgb {
namespace {

constexpr int kM = 128, kN = 128, kK = 64;
constexpr int kPiece = kN * kK * 2;    // 16 KiB: one BF16 piece of a tile
constexpr int kTile = 2 * kPiece;      // hi, then lo
constexpr uint32_t kTmemCols = 256;    // two 128-column FP32 accumulators
constexpr int kMaxWords = kTccMaxWords;

struct TccSmem {
    unsigned char a[2][kPiece];        // row operand: hi, lo
    unsigned char b[2][kTile];         // two stages of column tiles
    unsigned words[kMaxWords];         // kept column clusters of this block
    unsigned long long mb_tma[2], mb_mma[2], mb_free[2];
    uint32_t tslot;
    int ncols;
};

__device__ __forceinline__ uint16_t bfbits(float v) { return __bfloat16_as_ushort(__float2bfloat16_rn(v)); }
__device__ __forceinline__ float bfval(uint16_t b) { return __uint_as_float((uint32_t)b << 16); }
__device__ __forceinline__ uint32_t pk(uint16_t lo, uint16_t hi) { return (uint32_t)lo | ((uint32_t)hi << 16); }
constexpr uint16_t kOne = 0x3F80;  // 1.0 in BF16

// v ~ h + m + l in BF16 (about 24 significant bits)
__device__ __forceinline__ void split3(float v, uint16_t &h, uint16_t &m, uint16_t &l) {
    h = bfbits(v);
    const float r = v - bfval(h);
    m = bfbits(r);
    l = bfbits(r - bfval(m));
}

// Two values rounded to BF16 by one packed conversion (its own pipe, not the MUFU unit's): `hi` in the high
// half, `lo` in the low half, each to nearest even as the scalar conversion rounds.
__device__ __forceinline__ uint32_t bf2(float hi, float lo) {
    uint32_t d;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
    return d;
}

// 8 consecutive values -> BF16 hi and lo parts as two 16-byte vectors (value 2q in the low half of word q)
__device__ __forceinline__ void split8(const float (&v)[8], uint4 &hi, uint4 &lo) {
    uint32_t h[4], l[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        h[q] = bf2(v[2 * q + 1], v[2 * q]);
        l[q] = bf2(v[2 * q + 1] - __uint_as_float(h[q] & 0xFFFF0000u), v[2 * q] - __uint_as_float(h[q] << 16));
    }
    hi = make_uint4(h[0], h[1], h[2], h[3]);
    lo = make_uint4(l[0], l[1], l[2], l[3]);
}

__device__ __forceinline__ float ex2f(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ void tma_tile(void *dst, const void *src, unsigned long long *bar) {
    const uint32_t b = tc::smem_u32(bar);
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b), "r"(kTile) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     tc::smem_u32(dst)),
                 "l"(src), "r"(kTile), "r"(b)
                 : "memory");
}

// Walks the tiles of the kept column clusters of a block in cluster order.
struct TileIt {
    int w = -1;
    unsigned u = 0u;
    int J = -1, g = 0, gend = 0;
};
__device__ __forceinline__ bool tile_next(TileIt &it, const unsigned *words, int nwords, const int *tile0) {
    if (it.g + 1 < it.gend) {
        ++it.g;
        return true;
    }
    for (;;) {
        while (it.u == 0u) {
            if (++it.w >= nwords) return false;
            it.u = words[it.w];
        }
        const int bit = __ffs(it.u) - 1;
        it.u &= it.u - 1u;
        it.J = it.w * 32 + bit;
        it.g = tile0[it.J];
        it.gend = tile0[it.J + 1];
        if (it.g < it.gend) return true;
    }
}

__global__ void __launch_bounds__(128, 2) softmin_tcc_kernel(const __grid_constant__ SoftminLaunch L, int D4) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    TccSmem &S = *reinterpret_cast<TccSmem *>(smem_raw);
    const int t = threadIdx.x, warp = t >> 5;
    int4 item = L.items[blockIdx.x];
    OTGB_DCLAMP(item.x, 0, L.n_inst);
    const SoftminInst &I = L.inst[item.x];
    const int blk = item.y;
    int r0 = I.blk_row0[blk], r1 = I.blk_row0[blk + 1];
    OTGB_DCLAMP(r0, 0, I.n_rows + 1);
    OTGB_DCLAMP(r1, r0, min(I.n_rows, r0 + kM) + 1);
    const int nr = r1 - r0;
    const float s = L.s;
    const int nwords = L.tcc_nwords;

    // ---- kept column clusters of this block: union of its row clusters' keep bits
    const int cl0 = I.tcc_blk_cl[2 * blk], cl1 = I.tcc_blk_cl[2 * blk + 1];
    if (t == 0) {
        S.ncols = 0;
        tc::mbar_init(&S.mb_tma[0], 1);
        tc::mbar_init(&S.mb_tma[1], 1);
        tc::mbar_init(&S.mb_mma[0], 1);
        tc::mbar_init(&S.mb_mma[1], 1);
        tc::mbar_init(&S.mb_free[0], kM);
        tc::mbar_init(&S.mb_free[1], kM);
        tc::mbar_init_fence();
    }
    __syncthreads();
    int ncols = 0;
    for (int w = t; w < nwords; w += kM) {
        unsigned u = 0u;
        for (int c = cl0; c < cl1; ++c) u |= I.tcc_bits[(size_t)c * nwords + w];
        S.words[w] = u;
        while (u) {
            const int J = w * 32 + __ffs(u) - 1;
            u &= u - 1u;
            ncols += I.tcc_coff[J + 1] - I.tcc_coff[J];
        }
    }
    if (ncols) atomicAdd(&S.ncols, ncols);

    // ---- this thread's row: M_i = -s old_i / lam
    const bool valid = t < nr;
    const float *xr = I.rows + (size_t)(r0 + (valid ? t : 0)) * D4;
    float Mi = 0.f;
    if (valid) Mi = (float)(-(double)s * (double)I.row_old[r0 + t] / (double)I.lam);

    // row operand for column cluster J: s (x - c_J) split hi / lo, R_iJ in slots 62, 63
    const float4 *xr4 = reinterpret_cast<const float4 *>(xr);
    auto stage_rows = [&](int J) {
        const float4 *cj4 = reinterpret_cast<const float4 *>(I.tcc_ccen + (size_t)J * D4);
        float sq = 0.f;
#pragma unroll
        for (int ch = 0; ch < 8; ++ch) {
            float v[8];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int k4 = 2 * ch + h;
                float4 d = make_float4(0.f, 0.f, 0.f, 0.f);
                if (valid && 4 * k4 < D4) {
                    const float4 a = xr4[k4], c = cj4[k4];
                    d = make_float4(a.x - c.x, a.y - c.y, a.z - c.z, a.w - c.w);
                }
                sq = fmaf(d.x, d.x, fmaf(d.y, d.y, fmaf(d.z, d.z, fmaf(d.w, d.w, sq))));
                v[4 * h] = s * d.x;
                v[4 * h + 1] = s * d.y;
                v[4 * h + 2] = s * d.z;
                v[4 * h + 3] = s * d.w;
            }
            uint4 hi, lo;
            split8(v, hi, lo);
            if (ch == 7) {
                const float R = valid ? -0.5f * s * sq - Mi : 0.f;
                uint16_t R1, R2, R3;
                split3(R, R1, R2, R3);
                hi.z = pk(kOne, kOne);
                hi.w = pk(R1, R3);
                lo.z = 0u;
                lo.w = pk(R2, 0);
            }
            *reinterpret_cast<uint4 *>(S.a[0] + tc::core_off(t, 8 * ch)) = hi;
            *reinterpret_cast<uint4 *>(S.a[1] + tc::core_off(t, 8 * ch)) = lo;
        }
    };

    if (warp == 0) tc::tmem_alloc(&S.tslot, kTmemCols);
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = S.tslot;
    const uint32_t idesc = tc::idesc_bf16(kM, kN);
    auto issue = [&](int buf) {  // tile in stage buf -> accumulator buf
        const uint32_t d = tmem + (uint32_t)(buf * kN);
        const uint32_t ah = tc::smem_u32(S.a[0]), al = tc::smem_u32(S.a[1]);
        const uint32_t bh = tc::smem_u32(S.b[buf]), bl = bh + kPiece;
#pragma unroll
        for (int kk = 0; kk < kK / 16; ++kk) {
            const uint32_t off = kk * 256;
            tc::mma_bf16(d, tc::sdesc(ah + off), tc::sdesc(bh + off), idesc, kk > 0 ? 1u : 0u);
            tc::mma_bf16(d, tc::sdesc(ah + off), tc::sdesc(bl + off), idesc, 1u);
            tc::mma_bf16(d, tc::sdesc(al + off), tc::sdesc(bh + off), idesc, 1u);
        }
        tc::commit(&S.mb_mma[buf]);
    };

    const int *tile0 = I.tcc_tile0;
    const unsigned char *tiles = I.tcc_tiles;
    bool ok = true;
    float tot = 0.f;
    // bit b: parity of the next completion of stage b's copy / accumulator b's MMA / accumulator b's release
    uint32_t ph_tma = 0u, ph_mma = 0u, ph_free = 0u;
    TileIt itL, itM;
    bool have = tile_next(itM, S.words, nwords, tile0);
    if (t == 0) {
        for (int q = 0; q < 2; ++q)
            if (tile_next(itL, S.words, nwords, tile0)) tma_tile(S.b[q], tiles + (size_t)itL.g * kTile, &S.mb_tma[q]);
    }
    int aJ = -1;
    if (have) {
        stage_rows(itM.J);
        aJ = itM.J;
        tc::fence_proxy_async();
        tc::fence_before();
        __syncthreads();
        tc::fence_after();
        if (t == 0) {
            if (!tc::mbar_wait(&S.mb_tma[0], ph_tma & 1u)) ok = false;
            ph_tma ^= 1u;
            tc::fence_after();
            issue(0);
        }
    }
    int k = 0;
    while (have) {
        const int buf = k & 1, nb = buf ^ 1;
        TileIt itN = itM;
        const bool haveN = tile_next(itN, S.words, nwords, tile0);
        if (haveN) {
            if (itN.J != aJ) {
                // the row operand changes: the MMA of tile k (the last one issued) must be done with it
                if (!tc::mbar_wait(&S.mb_mma[buf], (ph_mma >> buf) & 1u)) ok = false;
                tc::fence_after();
                stage_rows(itN.J);
                aJ = itN.J;
                tc::fence_proxy_async();
                tc::fence_before();
                __syncthreads();
                tc::fence_after();
            }
            if (t == 0) {
                if (k >= 1) {  // every thread has read accumulator nb (tile k-1)
                    if (!tc::mbar_wait(&S.mb_free[nb], (ph_free >> nb) & 1u)) ok = false;
                    ph_free ^= 1u << nb;
                }
                if (!tc::mbar_wait(&S.mb_tma[nb], (ph_tma >> nb) & 1u)) ok = false;
                ph_tma ^= 1u << nb;
                tc::fence_after();
                issue(nb);
            }
        }
        // sums of tile k
        if (!tc::mbar_wait(&S.mb_mma[buf], (ph_mma >> buf) & 1u)) ok = false;
        ph_mma ^= 1u << buf;
        // stage buf is free (MMA k completed): the copy of tile k+2 starts before the sums
        if (t == 0 && tile_next(itL, S.words, nwords, tile0))
            tma_tile(S.b[buf], tiles + (size_t)itL.g * kTile, &S.mb_tma[buf]);
        ok = __all_sync(0xffffffffu, ok);  // tcgen05.ld below is warp-collective
        tc::fence_after();
        if (ok) {
            const uint32_t base = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(buf * kN);
            uint32_t va[32], vb[32];
            auto sum32 = [&](const uint32_t (&v)[32]) {
                float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
#pragma unroll
                for (int q = 0; q < 32; q += 4) {
                    a0 += ex2f(__uint_as_float(v[q]));
                    a1 += ex2f(__uint_as_float(v[q + 1]));
                    a2 += ex2f(__uint_as_float(v[q + 2]));
                    a3 += ex2f(__uint_as_float(v[q + 3]));
                }
                tot += (a0 + a1) + (a2 + a3);
            };
            tc::ld32_async(base, va);
            tc::ld_wait(va);
            tc::ld32_async(base + 32, vb);
            sum32(va);
            tc::ld_wait(vb);
            tc::ld32_async(base + 64, va);
            sum32(vb);
            tc::ld_wait(va);
            tc::ld32_async(base + 96, vb);
            sum32(va);
            tc::ld_wait(vb);
            sum32(vb);
        }
        // accumulator buf is read: released to the MMA issuer without a CTA barrier
        tc::fence_before();
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::smem_u32(&S.mb_free[buf])) : "memory");
        itM = itN;
        have = haveN;
        ++k;
    }
    // copies issued past the last tile: none (the loads walk the same sequence, two ahead, and stop at its end)
    ok = __syncthreads_and(ok) != 0;
    if (!ok && t == 0 && L.tc_err) atomicOr(L.tc_err, 1u);
    tc::fence_after();
    if (warp == 0) tc::tmem_dealloc(tmem, kTmemCols);

    if (t == 0 && L.pairs) atomicAdd(L.pairs, (unsigned long long)nr * (unsigned long long)S.ncols);
    float dmax = 0.f;
    if (valid && ok) {
        const int r = r0 + t;
        if (!(tot >= 0x1p-60f && tot <= 0x1p60f)) {
            const int q = atomicAdd(L.n_fallback, 1);
            if (q < L.fallback_cap) L.fallback[q] = make_int4(item.x, r, blk, 0);
        } else {
            const double tilde = -(double)I.lam * L.eps_ln2 * ((double)Mi + log2((double)tot));
            double nw = tilde;
            if (I.row_old) {
                const double old = (double)I.row_old[r];
                nw = old + (double)I.omega * (tilde - old);
                dmax = (float)(fabs(nw - old) / (double)L.eps);
            }
            I.row_out[r] = (float)nw;
        }
    }
    for (int o = 16; o > 0; o >>= 1) dmax = fmaxf(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
    if ((t & 31) == 0 && L.delta_max) atomicMax(L.delta_max, __float_as_uint(dmax));
}

// Column tiles of one side: tile g of cluster J = tile_cl[g] holds columns off[J] + 128 (g - tile0[J]) + c,
// c < 128 (past the cluster's end: zero), centred at c_J and split hi / lo; half_norm = |yh|^2 / 2.
// Written into `copies` buffers at once.
__global__ void tcc_build_kernel(const float *pts, int D4, const int *off, const int *tile0, const int *tile_cl,
                                 const float *cen, unsigned char *dst0, unsigned char *dst1, float *half_norm) {
    const int g = blockIdx.x, c = threadIdx.x;
    const int J = tile_cl[g];
    const int j = off[J] + (g - tile0[J]) * kN + c;
    const bool ok = j < off[J + 1];
    const float *y = pts + (size_t)(ok ? j : 0) * D4;
    const float *cj = cen + (size_t)J * D4;
    float sq = 0.f;
    for (int ch = 0; ch < 8; ++ch) {
        float v[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const int k = 8 * ch + e;
            v[e] = (ok && k < D4) ? y[k] - cj[k] : 0.f;
            sq = fmaf(v[e], v[e], sq);
        }
        uint4 hi, lo;
        split8(v, hi, lo);
        unsigned char *t0 = dst0 + (size_t)g * kTile, *t1 = dst1 + (size_t)g * kTile;
        *reinterpret_cast<uint4 *>(t0 + tc::core_off(c, 8 * ch)) = hi;
        *reinterpret_cast<uint4 *>(t0 + kPiece + tc::core_off(c, 8 * ch)) = lo;
        *reinterpret_cast<uint4 *>(t1 + tc::core_off(c, 8 * ch)) = hi;
        *reinterpret_cast<uint4 *>(t1 + kPiece + tc::core_off(c, 8 * ch)) = lo;
    }
    half_norm[(size_t)g * kN + c] = 0.5f * sq;
}

// Per step: H_j = s (eps log w_j + pot_j - |yh_j|^2 / 2) in three BF16 pieces into slots 60..63 of the
// column tiles of every instance (past a cluster's end, or for w_j = 0: a large negative H).
struct TccUpdate {
    unsigned char *tiles[kMaxInst];
    const float *half_norm[kMaxInst];
    const float *logw[kMaxInst];
    const float *pot[kMaxInst];
    const int *off[kMaxInst], *tile0[kMaxInst], *tile_cl[kMaxInst];
    int ntiles[kMaxInst];
    float s, eps;
};

__global__ void tcc_update_kernel(const __grid_constant__ TccUpdate U) {
    const int q = blockIdx.y, c = threadIdx.x;
    for (int g = blockIdx.x; g < U.ntiles[q]; g += gridDim.x) {
        const int J = U.tile_cl[q][g];
        const int j = U.off[q][J] + (g - U.tile0[q][J]) * kN + c;
        float H = -1e30f;
        if (j < U.off[q][J + 1])
            H = U.s * (fmaf(U.eps, U.logw[q][j], U.pot[q][j]) - U.half_norm[q][(size_t)g * kN + c]);
        if (!(H > -1e30f)) H = -1e30f;  // zero weight (log w = -inf) or past the end
        uint16_t h1, h2, h3;
        split3(H, h1, h2, h3);
        unsigned char *t0 = U.tiles[q] + (size_t)g * kTile;
        *reinterpret_cast<uint2 *>(t0 + tc::core_off(c, 60)) = make_uint2(pk(h1, h3), pk(kOne, kOne));
        *reinterpret_cast<uint2 *>(t0 + kPiece + tc::core_off(c, 60)) = make_uint2(pk(h2, 0), 0u);
    }
}

}  // namespace

size_t tcc_tile_bytes() { return (size_t)kTile; }

void tcc_build_side(const float *pts, int D4, const int *d_off, const int *d_tile0, const int *d_tile_cl,
                    int ntiles, const float *cen, unsigned char *dst0, unsigned char *dst1, float *half_norm,
                    cudaStream_t st) {
    require(D4 <= 60, "tcc_build_side: D4 must be <= 60", OTGB_EINTERNAL);
    if (ntiles <= 0) return;
    tcc_build_kernel<<<ntiles, kN, 0, st>>>(pts, D4, d_off, d_tile0, d_tile_cl, cen, dst0, dst1, half_norm);
    OTGB_CHECK_LAUNCH();
}

void tcc_update(const SoftminLaunch &L, cudaStream_t st) {
    TccUpdate U;
    int mx = 0;
    for (int q = 0; q < kMaxInst; ++q) {
        const SoftminInst &I = L.inst[q];
        U.tiles[q] = const_cast<unsigned char *>(I.tcc_tiles);
        U.half_norm[q] = I.tcc_half_norm;
        U.logw[q] = I.col_logw;
        U.pot[q] = I.col_pot;
        U.off[q] = I.tcc_coff;
        U.tile0[q] = I.tcc_tile0;
        U.tile_cl[q] = I.tcc_tile_cl;
        U.ntiles[q] = q < L.n_inst ? I.tcc_ntiles : 0;
        mx = std::max(mx, U.ntiles[q]);
    }
    U.s = L.s;
    U.eps = L.eps;
    if (mx <= 0) return;
    tcc_update_kernel<<<dim3(std::min(mx, 65535), L.n_inst), kN, 0, st>>>(U);
    OTGB_CHECK_LAUNCH();
}

void softmin_tcc_launch(const SoftminLaunch &L, int D, cudaStream_t st) {
    const int D4 = (D + 3) & ~3;
    require(D4 <= 60 && L.tcc_nwords <= kMaxWords, "softmin_tcc_launch: unsupported shape", OTGB_EINTERNAL);
    static PerDevice<int> attr;
    attr.get([] {
        OTGB_CUDA_TRY(cudaFuncSetAttribute(softmin_tcc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)sizeof(TccSmem)));
        return 1;
    });
    softmin_tcc_kernel<<<L.n_items, kM, sizeof(TccSmem), st>>>(L, D4);
    OTGB_CHECK_LAUNCH();
}

}  // namespace otgb
