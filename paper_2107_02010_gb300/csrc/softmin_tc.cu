// Tensor-core form of the softmin sweep for 16 <= D <= 64 (the reduced-precision
// cross term): in the centred frame of each row block the cross term
// s xt_i . yt_j of the exponent is a dense contraction over the D coordinates,
// computed by tcgen05.mma in BF16 with the operands split hi + lo
// (x = x_hi + x_lo, y = y_hi + y_lo, products hi.hi + hi.lo + lo.hi, about 16
// significant bits) and FP32 accumulation in tensor memory.  The rest of each
// term -- H_j = s (eps log w_j + pot_j - |yt_j|^2 / 2), the row shift m_i, ex2,
// the sum -- stays FP32 on the CUDA cores, as does the per-row finish in double.
//
// One CTA (4 warps) owns a block of at most 128 rows (M = 128, one TMEM lane
// per row); columns come in tiles of 128 (N = 128), K = 64 (D zero-padded).
// Pipeline per tile: the CTA stages the next tile's operands (centre, split)
// into the other shared-memory buffer while the tensor core multiplies the
// current one into one of two TMEM accumulators; then each thread reads its
// row of the finished accumulator (tcgen05.ld) and folds it into its sum.
// Operands use the canonical K-major layout without swizzle: 8-row x 16-byte
// core matrices, contiguous along K (LBO = 128 B), 8-row groups 1024 B apart.
// Every wait is bounded; a timeout sets an error word and the kernel still
// releases its tensor memory.
#include <cfloat>
#include <cmath>

#include <cuda_bf16.h>

#include "otgb_internal.cuh"

namespace otgb {
namespace {

constexpr int kTcM = 128, kTcN = 128, kTcK = 64;
constexpr int kTileBytes = kTcM * kTcK * 2;  // 16 KiB per bf16 operand tile
constexpr uint32_t kTmemCols = 256;          // two 128-column FP32 accumulators
constexpr int kWaitLimit = 1 << 24;

struct TcSmem {
    unsigned char a_hi[kTileBytes];
    unsigned char a_lo[kTileBytes];
    unsigned char b_hi[2][kTileBytes];
    unsigned char b_lo[2][kTileBytes];
    float h[2][kTcN];
    float cen[64];
    float red[4];
    unsigned long long mbar[2];
    uint32_t tslot;
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ int core_off(int r, int k) {
    return (r >> 3) * 1024 + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2;
}

__device__ __forceinline__ uint64_t sdesc(uint32_t addr) {
    uint64_t d = (uint64_t)((addr & 0x3FFFF) >> 4);
    d |= (uint64_t)(128 >> 4) << 16;   // K-direction core-matrix stride
    d |= (uint64_t)(1024 >> 4) << 32;  // 8-row group stride
    d |= (uint64_t)1 << 46;            // descriptor version for this architecture
    return d;
}

__device__ __forceinline__ float ex2(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// 8 consecutive values -> bf16 hi and lo parts as two 16-byte vectors
__device__ __forceinline__ void split8(const float (&v)[8], uint4 &hi, uint4 &lo) {
    uint32_t h[4], l[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const __nv_bfloat16 h0 = __float2bfloat16_rn(v[2 * q]), h1 = __float2bfloat16_rn(v[2 * q + 1]);
        const __nv_bfloat16 l0 = __float2bfloat16_rn(v[2 * q] - __bfloat162float(h0));
        const __nv_bfloat16 l1 = __float2bfloat16_rn(v[2 * q + 1] - __bfloat162float(h1));
        h[q] = (uint32_t)__bfloat16_as_ushort(h0) | ((uint32_t)__bfloat16_as_ushort(h1) << 16);
        l[q] = (uint32_t)__bfloat16_as_ushort(l0) | ((uint32_t)__bfloat16_as_ushort(l1) << 16);
    }
    hi = make_uint4(h[0], h[1], h[2], h[3]);
    lo = make_uint4(l[0], l[1], l[2], l[3]);
}

__device__ __forceinline__ bool mbar_wait(uint32_t addr, uint32_t parity) {
    uint32_t done = 0;
    for (int it = 0; it < kWaitLimit && !done; ++it)
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
            : "=r"(done)
            : "r"(addr), "r"(parity));
    return done != 0;
}

__device__ __forceinline__ void finish_row_tc(const SoftminLaunch &L, const SoftminInst &I, int r, double L2,
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

// FOLD (D4 <= 60): the free K slots 60..63 carry the rest of the exponent, so
// that the accumulator holds H_j - m_i + s xt_i . yt_j and the epilogue is
// just ex2 and a sum: column slots 60-62 hold H_j as three BF16 pieces (about
// 24 significant bits) against 1.0 in the row operand, row slot 63 holds the
// row shift rounded to BF16 against 1.0 in the column operand.  Any shift is
// valid as long as the finish adds back the same value, so the rounded shift
// costs nothing in accuracy.
template <bool FOLD>
__global__ void __launch_bounds__(128, 2) softmin_tc_kernel(const __grid_constant__ SoftminLaunch L, int D4) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    TcSmem &S = *reinterpret_cast<TcSmem *>(smem_raw);
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    int4 item = L.items[blockIdx.x];
    OTGB_DCLAMP(item.x, 0, L.n_inst);
    const SoftminInst &I = L.inst[item.x];
    const int blk = item.y;
    int r0 = I.blk_row0[blk], r1 = I.blk_row0[blk + 1];
    OTGB_DCLAMP(r0, 0, I.n_rows + 1);
    OTGB_DCLAMP(r1, r0, min(I.n_rows, r0 + kTcM) + 1);
    const int nr = r1 - r0;
    const float eps = L.eps, s = L.s;

    // ---- rows: centre (mean), X = s (x - c) split hi/lo, |xt|^2 / 2
    for (int k = t; k < 64; k += 128) {
        float acc = 0.f;
        if (k < D4)
            for (int r = 0; r < nr; ++r) acc += I.rows[(size_t)(r0 + r) * D4 + k];
        S.cen[k] = (k < D4 && nr > 0) ? acc / (float)nr : 0.f;
    }
    if (t == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&S.mbar[0])), "r"(1));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&S.mbar[1])), "r"(1));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    __syncthreads();
    for (int u = t; u < kTcM * 8; u += 128) {  // lanes 8q..8q+7 share a row
        const int r = u >> 3, ch = u & 7;
        float v[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const int k = ch * 8 + e;
            v[e] = (r < nr && k < D4) ? I.rows[(size_t)(r0 + r) * D4 + k] - S.cen[k] : 0.f;
        }
        float sq = 0.f;
#pragma unroll
        for (int e = 0; e < 8; ++e) { sq = fmaf(v[e], v[e], sq); v[e] *= s; }
        uint4 hi, lo;
        split8(v, hi, lo);
        if (FOLD && ch == 7) {  // slots 60, 61, 62 = 1.0 (the H pieces); 63 = the shift, written below
            hi.z = 0x3F803F80u;
            hi.w = 0x00003F80u;
        }
        *reinterpret_cast<uint4 *>(S.a_hi + core_off(r, ch * 8)) = hi;
        *reinterpret_cast<uint4 *>(S.a_lo + core_off(r, ch * 8)) = lo;
        // |xt|^2 of row r: sum over its 8 chunks (8 consecutive lanes)
        for (int o = 4; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
        if (ch == 0) S.h[0][r] = sq;  // held here until every row is done
    }
    __syncthreads();
    // this thread's row: t (TMEM lane t)
    const int myr = t;
    const bool valid = myr < nr;
    const float x2 = S.h[0][myr];
    const double hx = 0.5 * (double)x2;
    float m = 0.f;
    if (valid) m = (float)((double)s * (hx - (double)I.row_old[r0 + myr] / (double)I.lam));
    // FOLD: a block constant C (the largest row shift) is taken out of both
    // folded terms, so that the accumulator adds H_j - C and -(m_i - C), small
    // for every pair that matters, instead of two large values that cancel.
    float Cb = 0.f;
    double m_eff = (double)m;  // the row shift the finish adds back
    if (FOLD) {
        float mx = valid ? m : -INFINITY;
        for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if (lane == 0) S.red[warp] = mx;
        __syncthreads();
        Cb = fmaxf(fmaxf(S.red[0], S.red[1]), fmaxf(S.red[2], S.red[3]));
        if (!(Cb > -INFINITY)) Cb = 0.f;
        const __nv_bfloat16 mb = __float2bfloat16_rn(-(m - Cb));
        m_eff = (double)Cb - (double)__bfloat162float(mb);  // the shift the accumulator applies
        *reinterpret_cast<__nv_bfloat16 *>(S.a_hi + core_off(myr, 63)) = mb;
    }
    __syncthreads();  // S.h[0] is reused for the columns

    // ---- columns of this item
    const int nkept = kept_cols(I, blk);
    int cb = item.z, ce = item.w;
    OTGB_DCLAMP(cb, 0, nkept + 1);
    OTGB_DCLAMP(ce, cb, nkept + 1);
    const int ncol = ce - cb;
    ColWalk walk;
    walk.start(I, blk, cb);
    const int ntiles = (ncol + kTcN - 1) / kTcN;

    // Staging of a column tile, software-pipelined over three tiles: the
    // column indices of tile t+3 and the raw coordinates of tile t+2 are
    // loaded into registers while the tensor core multiplies tile t+1 and the
    // CTA finishes tile t, so no load latency sits between two tiles.  Thread
    // t handles chunk ch = t % 8 (coordinates 8 ch .. 8 ch + 7) of the columns
    // t / 8 + 16 k, k < 8; the 8 threads of a column sum its |yt|^2.
    constexpr int kU = kTcN * 8 / 128;
    const int ch = t & 7, colb = t >> 3;
    int jc[kU], jn[kU];
    float4 ra[kU], rb[kU];
    float rlw[kU], rpot[kU];
    auto load_idx = [&](int tile, int (&j)[kU]) {
        const int p0 = tile * kTcN;
#pragma unroll
        for (int k = 0; k < kU; ++k) {
            const int p = p0 + colb + 16 * k;
            int jj = -1;
            if (tile < ntiles && p < ncol) {
                jj = walk.at(cb + p);
                OTGB_DCLAMP(jj, 0, I.n_cols);
            }
            j[k] = jj;
        }
    };
    auto load_raw = [&]() {
#pragma unroll
        for (int k = 0; k < kU; ++k) {
            const int jj = jc[k];
            float4 a = make_float4(0.f, 0.f, 0.f, 0.f), b = a;
            float lw = 0.f, pt = 0.f;
            if (jj >= 0) {
                const float *src = I.cols + (size_t)jj * D4 + ch * 8;
                if (ch * 8 + 4 <= D4) a = *reinterpret_cast<const float4 *>(src);
                if (ch * 8 + 8 <= D4) b = *reinterpret_cast<const float4 *>(src + 4);
                if (ch == (FOLD ? 7 : 0)) {
                    lw = I.col_logw[jj];
                    pt = I.col_pot[jj];
                }
            }
            ra[k] = a;
            rb[k] = b;
            rlw[k] = lw;
            rpot[k] = pt;
        }
    };
    auto convert = [&](int buf) {
#pragma unroll
        for (int k = 0; k < kU; ++k) {
            const int col = colb + 16 * k;
            const bool ok_col = jc[k] >= 0;
            const float *cn = S.cen + ch * 8;
            float v[8] = {ra[k].x - cn[0], ra[k].y - cn[1], ra[k].z - cn[2], ra[k].w - cn[3],
                          rb[k].x - cn[4], rb[k].y - cn[5], rb[k].z - cn[6], rb[k].w - cn[7]};
            float sq = 0.f;
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                v[e] = ok_col ? v[e] : 0.f;
                sq = fmaf(v[e], v[e], sq);
            }
            uint4 hi, lo;
            split8(v, hi, lo);
            for (int o = 4; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
            if (FOLD) {
                if (ch == 7) {  // slots 60-62: H in three BF16 pieces; 63: 1.0 against the row shift
                    const float H = ok_col ? s * (fmaf(eps, rlw[k], rpot[k]) - 0.5f * sq) - Cb : -1e30f;
                    const __nv_bfloat16 h1 = __float2bfloat16_rn(H);
                    const float r1 = H - __bfloat162float(h1);
                    const __nv_bfloat16 h2 = __float2bfloat16_rn(r1);
                    const __nv_bfloat16 h3 = __float2bfloat16_rn(r1 - __bfloat162float(h2));
                    hi.z = (uint32_t)__bfloat16_as_ushort(h1) | ((uint32_t)__bfloat16_as_ushort(h2) << 16);
                    hi.w = (uint32_t)__bfloat16_as_ushort(h3) | (0x3F80u << 16);
                    lo.z = 0u;
                    lo.w = 0u;
                }
            } else if (ch == 0) {
                S.h[buf][col] = ok_col ? s * (fmaf(eps, rlw[k], rpot[k]) - 0.5f * sq) : -INFINITY;
            }
            *reinterpret_cast<uint4 *>(S.b_hi[buf] + core_off(col, ch * 8)) = hi;
            *reinterpret_cast<uint4 *>(S.b_lo[buf] + core_off(col, ch * 8)) = lo;
        }
    };

    // tensor memory: two 128-column accumulators
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&S.tslot)),
                     "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = S.tslot;
    // D f32, A and B bf16, both K-major, N = 128, M = 128
    const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kTcN >> 3) << 17) |
                           ((uint32_t)(kTcM >> 4) << 24);
    auto issue = [&](int buf) {
        const uint32_t d = tmem + (uint32_t)(buf * kTcN);
        const uint32_t ah = smem_u32(S.a_hi), al = smem_u32(S.a_lo);
        const uint32_t bh = smem_u32(S.b_hi[buf]), bl = smem_u32(S.b_lo[buf]);
        uint32_t acc = 0;
#pragma unroll
        for (int kk = 0; kk < kTcK / 16; ++kk) {
            const uint32_t off = kk * 256;
            const uint64_t pa[3] = {sdesc(ah + off), sdesc(ah + off), sdesc(al + off)};
            const uint64_t pb[3] = {sdesc(bh + off), sdesc(bl + off), sdesc(bh + off)};
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                             " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d),
                             "l"(pa[q]), "l"(pb[q]), "r"(idesc), "r"(acc));
                acc = 1;
            }
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(&S.mbar[buf])));
    };

    float tot = 0.f;
    uint32_t phase[2] = {0u, 0u};
    bool ok = true;
    if (ntiles > 0) {
        load_idx(0, jc);
        load_raw();
        convert(0);
        load_idx(1, jc);
        load_raw();
        load_idx(2, jn);
    }
    asm volatile("fence.proxy.async.shared::cta;");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (t == 0 && ntiles > 0) issue(0);
    for (int tt = 0; tt < ntiles; ++tt) {
        const int buf = tt & 1;
        if (tt + 1 < ntiles) {
            convert(buf ^ 1);  // tile tt+1 from registers
#pragma unroll
            for (int k = 0; k < kU; ++k) jc[k] = jn[k];
            load_raw();             // tile tt+2 (nothing past the end)
            load_idx(tt + 3, jn);   // indices of tile tt+3
        }
        asm volatile("fence.proxy.async.shared::cta;");
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;");
        if (t == 0 && tt + 1 < ntiles) issue(buf ^ 1);
        if (!mbar_wait(smem_u32(&S.mbar[buf]), phase[buf])) ok = false;
        ok = __all_sync(0xffffffffu, ok);  // tcgen05.ld below is warp-collective
        phase[buf] ^= 1u;
        asm volatile("tcgen05.fence::after_thread_sync;");
        if (ok) {
#pragma unroll
            for (int c = 0; c < kTcN; c += 32) {
                uint32_t v[32];
                const uint32_t a = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(buf * kTcN + c);
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                    "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                    : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                      "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
                      "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]),
                      "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]),
                      "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
                    : "r"(a));
                asm volatile("tcgen05.wait::ld.sync.aligned;");
                float a0 = 0.f, a1 = 0.f;
                if (FOLD) {
                    float a2 = 0.f, a3 = 0.f;
#pragma unroll
                    for (int q = 0; q < 32; q += 4) {
                        a0 += ex2(__uint_as_float(v[q]));
                        a1 += ex2(__uint_as_float(v[q + 1]));
                        a2 += ex2(__uint_as_float(v[q + 2]));
                        a3 += ex2(__uint_as_float(v[q + 3]));
                    }
                    tot += (a0 + a1) + (a2 + a3);
                } else {
#pragma unroll
                    for (int q = 0; q < 32; q += 2) {
                        a0 += ex2(__uint_as_float(v[q]) + (S.h[buf][c + q] - m));
                        a1 += ex2(__uint_as_float(v[q + 1]) + (S.h[buf][c + q + 1] - m));
                    }
                    tot += a0 + a1;
                }
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();  // buffers of this tile are free again
    }
    if (!ok && L.tc_err) atomicOr(L.tc_err, 1u);
    // release tensor memory (every MMA was waited for)
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));

    if (lane == 0 && warp == 0 && L.pairs)
        atomicAdd(L.pairs, (unsigned long long)nr * (unsigned long long)ncol);
    float dmax = 0.f;
    if (valid && ok) {
        const int r = r0 + myr;
        if (!(tot >= 0x1p-60f && tot <= 0x1p60f)) {
            const int k = atomicAdd(L.n_fallback, 1);
            if (k < L.fallback_cap) L.fallback[k] = make_int4(item.x, r, blk, 0);
        } else {
            finish_row_tc(L, I, r, m_eff + log2((double)tot), hx, dmax);
        }
    }
    for (int o = 16; o > 0; o >>= 1) dmax = fmaxf(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
    if (lane == 0 && L.delta_max) atomicMax(L.delta_max, __float_as_uint(dmax));
}

}  // namespace

size_t softmin_tc_smem_bytes() { return sizeof(TcSmem); }

void softmin_tc_launch(const SoftminLaunch &L, int D, cudaStream_t st) {
    const int D4 = (D + 3) & ~3;
    static PerDevice<int> attr;
    attr.get([] {
        OTGB_CUDA_TRY(cudaFuncSetAttribute(softmin_tc_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)softmin_tc_smem_bytes()));
        OTGB_CUDA_TRY(cudaFuncSetAttribute(softmin_tc_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)softmin_tc_smem_bytes()));
        return 1;
    });
    if (D4 <= 60) softmin_tc_kernel<true><<<L.n_items, 128, softmin_tc_smem_bytes(), st>>>(L, D4);
    else softmin_tc_kernel<false><<<L.n_items, 128, softmin_tc_smem_bytes(), st>>>(L, D4);
    OTGB_CHECK_LAUNCH();
}

}  // namespace otgb
