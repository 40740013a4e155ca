// Tensor-core form of the D <= 3 softmin sweep at float32 accuracy.
//
// The whole exponent of a pair,
//   v_ij = s xt_i . yt_j + H_j - m_i,   H_j = s (eps log w_j + pot_j - |yt_j|^2 / 2),
// is one dot product of length K = 32 between a row vector and a column
// vector of BF16 values, computed by tcgen05.mma with FP32 accumulation in
// tensor memory, so that the CUDA cores only evaluate ex2 and the sum.  Every
// float operand is split into three BF16 pieces (h + m + l, about 24
// significant bits, i.e. float32 accuracy); per coordinate the six products
// that matter at that accuracy (h.h, h.m, m.h, h.l, l.h, m.m) take six K
// slots, so the three coordinates use 18 slots.  H_j - C goes in three slots
// against 1.0, and the row shift -(m_i - C), rounded to BF16, in one slot
// against 1.0; C is the largest row shift of the block, so that the folded
// terms are small for every pair that matters.  The finish adds back exactly
// the shift the accumulator applied, in double precision.
//
// One CTA (8 warps) owns a row block of at most 128 rows (one tensor-memory
// lane per row); columns come in tiles of kN.  Column staging is software
// pipelined: the indices of tile t+2 and the point of tile t+1 are loaded
// while the tensor core multiplies tile t+1 and the CTA sums tile t.  The
// indices come from the block's kept ranges (copied into shared memory once
// per CTA): every kChunkTiles tiles the CTA writes the column index of each
// position of the next chunk into one of two shared buffers, each thread
// kPerThr consecutive positions after one binary search.  Every wait is
// bounded.  Split blocks write partial sums; the CTA that completes a
// block's last item sums them in item order and finishes the rows.
#include <cfloat>
#include <cmath>

#include <cuda_bf16.h>

#include "otgb_internal.cuh"
#include "tcgen05.cuh"

namespace otgb {
namespace {

// Measured on the track-density workload (softmin rate): 256-column tiles with
// one accumulator and two warpgroups 5.0e12 pairs/s; 128 columns with two
// accumulators 4.4-4.6e12; deeper pipelines (4-8 accumulators) were slower;
// a warp-specialised variant (staging, MMA and sum warps handing tiles over
// through mbarriers, no CTA barrier per tile) reached 4.6e12; overlapping the
// tensor-memory loads with the sums changed nothing.  The MUFU ex2 unit (32 per
// clock per SM) is half busy at 5.0e12.
#ifndef OTGB_TC3_N
#define OTGB_TC3_N 256
#endif
#ifndef OTGB_TC3_STAGES
#define OTGB_TC3_STAGES 1
#endif
#ifndef OTGB_TC3_MINB
#define OTGB_TC3_MINB 2
#endif
#ifndef OTGB_TC3_THREADS
#define OTGB_TC3_THREADS 256
#endif
// Column tiles of kN columns; kStages accumulators in tensor memory and as
// many staged column tiles, so that the MMA of a tile is issued kStages - 1
// tiles before its sums are taken.
// kThreads = 256: two warpgroups read the same tensor-memory lanes (rows) and
// each takes half of a tile's columns in the epilogue.
constexpr int kM = 128, kN = OTGB_TC3_N, kK = 32, kStages = OTGB_TC3_STAGES, kThreads = OTGB_TC3_THREADS;
constexpr int kHalves = kThreads / 128;
constexpr int kATile = kM * kK * 2;  // 8 KiB
constexpr int kBTile = kN * kK * 2;
constexpr uint32_t kTmemCols = kStages * kN <= 32 ? 32u : (kStages * kN <= 64 ? 64u : (kStages * kN <= 128 ? 128u
                                   : (kStages * kN <= 256 ? 256u : 512u)));
// range entries of a block staged in shared memory; a block with more reads them from global memory
constexpr int kRngSmem = 1024;
// positions per expansion chunk (two buffers in flight) and per thread of an expansion
constexpr int kChunkTiles = 16, kChunk = kChunkTiles * kN, kPerThr = kChunk / kThreads;
static_assert(kPerThr * kThreads == kChunk && kPerThr % 4 == 0, "an expansion writes whole int4 groups");
static_assert(kChunkTiles >= kStages + 2, "a chunk is expanded at least one barrier before its first read");

// Word of position q (of a chunk) in the index buffer: 16-byte groups of four positions, group g stored at
// g ^ ((g >> 2) & 7) (a permutation of each aligned run of eight groups), so that both the expansion's
// 16-byte stores (a thread writes 16 consecutive positions) and the staging reads (a warp reads 32
// consecutive positions) are free of bank conflicts.
__device__ __forceinline__ int idx_word(int q) {
    const int g = q >> 2;
    return ((g ^ ((g >> 2) & 7)) << 2) | (q & 3);
}

// Column index of positions p0 .. p0 + kPerThr - 1 (those below `end`) from one block's range entries
// r[0 .. n) (the sentinel last, its position above every position asked for): a binary search for the
// first, then a forward walk.
template <typename Entries>
__device__ __forceinline__ void expand_positions(const Entries &r, int n, int p0, int end, int (&v)[kPerThr]) {
    int lo = 0, hi = n - 2;  // the last real entry
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (r(mid).y <= p0) lo = mid;
        else hi = mid - 1;
    }
    int k = lo;
    int2 cur = r(k), nxt = r(k + 1);
#pragma unroll
    for (int i = 0; i < kPerThr; ++i) {
        const int pq = p0 + i;
        v[i] = 0;
        if (pq < end) {
            while (nxt.y <= pq && k + 2 < n) {
                ++k;
                cur = nxt;
                nxt = r(k + 1);
            }
            v[i] = cur.x + (pq - cur.y);
        }
    }
}

struct Tc3Smem {
    unsigned char a[kATile];
    unsigned char b[kStages][kBTile];
    float red[4][8];
    float tot1[128];
    int bc[2];
    unsigned long long mbar[kStages];
    uint32_t tslot;
    int2 rng[kRngSmem];
    alignas(16) int idx[2][kChunk];
};

// K-major canonical layout of a tile with 32 K-columns: 8-row x 16-byte core
// matrices, 4 along K (leading byte offset 128), 8-row groups 512 bytes apart
__device__ __forceinline__ int off32(int r, int k) {
    return (r >> 3) * 512 + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2;
}

__device__ __forceinline__ uint64_t sdesc32(uint32_t addr) {
    uint64_t d = (uint64_t)((addr & 0x3FFFF) >> 4);
    d |= (uint64_t)(128 >> 4) << 16;
    d |= (uint64_t)(512 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

__device__ __forceinline__ float ex2f(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Scalar split for the row operand (once per CTA).  The per-tile column operand
// uses the packed form below.  (Rounding with integer operations instead, which
// also frees the MUFU unit, measured 2 % slower: it costs issue slots.)
__device__ __forceinline__ uint16_t bfbits(float v) { return __bfloat16_as_ushort(__float2bfloat16_rn(v)); }
__device__ __forceinline__ float bfval(uint16_t b) { return __uint_as_float((uint32_t)b << 16); }

// v ~ h + m + l in BF16 (about 24 significant bits)
__device__ __forceinline__ void split3(float v, uint16_t &h, uint16_t &m, uint16_t &l) {
    h = bfbits(v);
    const float r = v - bfval(h);
    m = bfbits(r);
    l = bfbits(r - bfval(m));
}

__device__ __forceinline__ uint32_t pk(uint16_t lo, uint16_t hi) { return (uint32_t)lo | ((uint32_t)hi << 16); }

// Two values split at once: H, M, L hold the h, m, l pieces of a in their high halves and of b in their low
// halves.  The packed conversion rounds each half to nearest even, as the scalar one does, so the pieces are
// those of split3; it runs on its own pipe, leaving the MUFU unit to ex2.
__device__ __forceinline__ uint32_t bf2(float hi, float lo) {
    uint32_t d;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
    return d;
}
__device__ __forceinline__ float hi_val(uint32_t w) { return __uint_as_float(w & 0xFFFF0000u); }
__device__ __forceinline__ float lo_val(uint32_t w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ void split3x2(float a, float b, uint32_t &H, uint32_t &M, uint32_t &L) {
    H = bf2(a, b);
    const float ra = a - hi_val(H), rb = b - lo_val(H);
    M = bf2(ra, rb);
    L = bf2(ra - hi_val(M), rb - lo_val(M));
}

constexpr uint16_t kOne = 0x3F80;  // 1.0 in BF16

__global__ void __launch_bounds__(kThreads, OTGB_TC3_MINB) softmin3_tc_kernel(const __grid_constant__ SoftminLaunch L) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    Tc3Smem &S = *reinterpret_cast<Tc3Smem *>(smem_raw);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int t = tid & 127, half = tid >> 7;  // row (tensor-memory lane) and warpgroup
    const int it = blockIdx.x;
    int4 item = L.items[it];
    OTGB_DCLAMP(item.x, 0, L.n_inst);
    const SoftminInst &I = L.inst[item.x];
    const int blk = item.y;
    int r0 = I.blk_row0[blk], r1 = I.blk_row0[blk + 1];
    OTGB_DCLAMP(r0, 0, I.n_rows + 1);
    OTGB_DCLAMP(r1, r0, min(I.n_rows, r0 + kM) + 1);
    const int nr = r1 - r0;
    const float eps = L.eps, s = L.s;
    const float4 *rows4 = reinterpret_cast<const float4 *>(I.rows);
    const float4 *cols4 = reinterpret_cast<const float4 *>(I.cols);

    // ---- the columns of this item: positions [cb, ce) of the block's kept columns; the block's
    // range entries (the sentinel last) into shared memory, visible after the first barrier below
    const int nkept = kept_cols(I, blk);
    int cb = item.z, ce = item.w;
    OTGB_DCLAMP(cb, 0, nkept + 1);
    OTGB_DCLAMP(ce, cb, nkept + 1);
    const int ncol = ce - cb;
    const int ntiles = (ncol + kN - 1) / kN;
    const bool ranged = I.col_rng != nullptr;
    const int nE = ranged ? I.rng_ptr[blk + 1] - I.rng_ptr[blk] : 0;
    const int2 *rb = ranged ? I.col_rng + I.rng_ptr[blk] : nullptr;
    const bool rng_local = ranged && nE <= kRngSmem;
    if (rng_local)
        for (int q = tid; q < nE; q += kThreads) S.rng[q] = rb[q];

    // ---- rows: centre of the block's bounding box, shifts, the row operand
    const bool valid = half == 0 && t < nr;
    float4 p = make_float4(0.f, 0.f, 0.f, 0.f);
    if (valid) p = rows4[r0 + t];
    if (half == 0) {
        float v[6] = {valid ? p.x : FLT_MAX, valid ? p.y : FLT_MAX, valid ? p.z : FLT_MAX,
                      valid ? -p.x : FLT_MAX, valid ? -p.y : FLT_MAX, valid ? -p.z : FLT_MAX};
#pragma unroll
        for (int q = 0; q < 6; ++q) {
            for (int o = 16; o > 0; o >>= 1) v[q] = fminf(v[q], __shfl_xor_sync(0xffffffffu, v[q], o));
            if (lane == 0) S.red[warp][q] = v[q];
        }
    }
    if (tid == 0) {
        for (int q = 0; q < kStages; ++q) tc::mbar_init(&S.mbar[q], 1);
        tc::mbar_init_fence();
    }
    __syncthreads();
    // column index of every position of chunk ch (tiles ch * kChunkTiles ..) into S.idx[ch & 1]; the
    // sentinel's position (the block's number of kept columns) exceeds every position of the item
    auto expand = [&](int ch) {
        const int q0 = ch * kChunk + tid * kPerThr;  // item-relative position of this thread's first
        if (!ranged || q0 >= ncol) return;
        int v[kPerThr];
        if (rng_local) expand_positions([&](int k) { return S.rng[k]; }, nE, cb + q0, ce, v);
        else expand_positions([&](int k) { return rb[k]; }, nE, cb + q0, ce, v);
#pragma unroll
        for (int i = 0; i < kPerThr / 4; ++i)
            *reinterpret_cast<int4 *>(&S.idx[ch & 1][idx_word(tid * kPerThr + 4 * i)]) =
                make_int4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
    };
    expand(0);  // read after the barriers of the row setup
    float c[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const float lo = fminf(fminf(S.red[0][d], S.red[1][d]), fminf(S.red[2][d], S.red[3][d]));
        const float nhi = fminf(fminf(S.red[0][d + 3], S.red[1][d + 3]), fminf(S.red[2][d + 3], S.red[3][d + 3]));
        c[d] = 0.5f * (lo - nhi);
    }
    const float x0 = valid ? p.x - c[0] : 0.f, x1 = valid ? p.y - c[1] : 0.f, x2 = valid ? p.z - c[2] : 0.f;
    const double hx = 0.5 * ((double)x0 * x0 + (double)x1 * x1 + (double)x2 * x2);
    float m = -INFINITY;
    if (valid) m = (float)((double)s * (hx - (double)I.row_old[r0 + t] / (double)I.lam));
    __syncthreads();  // S.red is reused
    if (half == 0) {
        float mx = m;
        for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if (lane == 0) S.red[warp][6] = mx;
    }
    __syncthreads();
    float Cb = fmaxf(fmaxf(S.red[0][6], S.red[1][6]), fmaxf(S.red[2][6], S.red[3][6]));
    if (!(Cb > -INFINITY)) Cb = 0.f;
    const uint16_t mb = valid ? bfbits(-(m - Cb)) : (uint16_t)0;
    const double m_eff = (double)Cb - (double)bfval(mb);  // the shift the accumulator applies
    if (half == 0) {
        uint16_t h[3], md[3], l[3];
        split3(s * x0, h[0], md[0], l[0]);
        split3(s * x1, h[1], md[1], l[1]);
        split3(s * x2, h[2], md[2], l[2]);
        uint32_t w[16];
        // slots 6d .. 6d+5: h h m h l m (against the column's h m h l h m)
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const int b0 = 3 * d;  // three words per coordinate
            w[b0] = pk(h[d], h[d]);
            w[b0 + 1] = pk(md[d], h[d]);
            w[b0 + 2] = pk(l[d], md[d]);
        }
        w[9] = pk(kOne, kOne);  // slots 18, 19: against H pieces 1, 2
        w[10] = pk(kOne, mb);   // slot 20: H piece 3; slot 21: the shift
#pragma unroll
        for (int q = 11; q < 16; ++q) w[q] = 0u;
#pragma unroll
        for (int q = 0; q < 4; ++q)
            *reinterpret_cast<uint4 *>(S.a + off32(t, 8 * q)) =
                make_uint4(w[4 * q], w[4 * q + 1], w[4 * q + 2], w[4 * q + 3]);
    }

    // ---- column staging: thread tid < kN stages column tid of each tile
    const bool stager = tid < kN;
    auto load_idx = [&](int tile) -> int {
        const int pp = tile * kN + tid;
        int jj = -1;
        if (stager && tile < ntiles && pp < ncol) {
            jj = ranged ? S.idx[(tile / kChunkTiles) & 1][idx_word((tile % kChunkTiles) * kN + tid)] : cb + pp;
            OTGB_DCLAMP(jj, 0, I.n_cols);
        }
        return jj;
    };
    int jc = -1, jn = -1;
    float4 rq = make_float4(0.f, 0.f, 0.f, 0.f);
    float rpot = 0.f;
    auto load_raw = [&]() {
        if (jc >= 0) {
            rq = cols4[jc];
            rpot = I.col_pot[jc];
        }
    };
    auto convert = [&](int buf) {
        if (!stager) return;
        const bool okc = jc >= 0;
        const float y0 = okc ? rq.x - c[0] : 0.f, y1 = okc ? rq.y - c[1] : 0.f, y2 = okc ? rq.z - c[2] : 0.f;
        const float sq = y0 * y0 + y1 * y1 + y2 * y2;
        const float H = okc ? s * (fmaf(eps, rq.w, rpot) - 0.5f * sq) - Cb : -1e30f;
        uint32_t H01, M01, L01, H2h, M2h, L2h;
        split3x2(y0, y1, H01, M01, L01);
        split3x2(y2, H, H2h, M2h, L2h);
        const uint16_t h[3] = {(uint16_t)(H01 >> 16), (uint16_t)H01, (uint16_t)(H2h >> 16)};
        const uint16_t md[3] = {(uint16_t)(M01 >> 16), (uint16_t)M01, (uint16_t)(M2h >> 16)};
        const uint16_t l[3] = {(uint16_t)(L01 >> 16), (uint16_t)L01, (uint16_t)(L2h >> 16)};
        const uint16_t hh[3] = {(uint16_t)H2h, (uint16_t)M2h, (uint16_t)L2h};
        uint32_t w[16];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const int b0 = 3 * d;
            w[b0] = pk(h[d], md[d]);
            w[b0 + 1] = pk(h[d], l[d]);
            w[b0 + 2] = pk(h[d], md[d]);
        }
        w[9] = pk(hh[0], hh[1]);
        w[10] = pk(hh[2], kOne);
#pragma unroll
        for (int q = 11; q < 16; ++q) w[q] = 0u;
#pragma unroll
        for (int q = 0; q < 4; ++q)
            *reinterpret_cast<uint4 *>(S.b[buf] + off32(tid, 8 * q)) =
                make_uint4(w[4 * q], w[4 * q + 1], w[4 * q + 2], w[4 * q + 3]);
    };

    if (warp == 0) tc::tmem_alloc(&S.tslot, kTmemCols);
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = S.tslot;
    const uint32_t idesc = tc::idesc_bf16(kM, kN);
    auto issue = [&](int buf) {
        const uint32_t d = tmem + (uint32_t)(buf * kN);
        const uint32_t a = tc::smem_u32(S.a), b = tc::smem_u32(S.b[buf]);
#pragma unroll
        for (int kk = 0; kk < kK / 16; ++kk)
            tc::mma_bf16(d, sdesc32(a + kk * 256), sdesc32(b + kk * 256), idesc, kk > 0 ? 1u : 0u);
        tc::commit(&S.mbar[buf]);
    };

    float tot = 0.f;
    uint32_t phase_bits = 0u;  // bit q: parity of the next completion of accumulator q
    bool ok = true;
    // rows of this warp that exist: the epilogue of an empty warp is skipped
    const bool warp_rows = (warp & 3) * 32 < nr;
    // prologue: tiles 0 .. kStages-2 staged, tile kStages-1 in registers
    for (int q = 0; q < kStages - 1; ++q) {
        if (q < ntiles) {
            jc = load_idx(q);
            load_raw();
            convert(q);
        }
    }
    jc = load_idx(kStages - 1);
    load_raw();
    jn = load_idx(kStages);
    tc::fence_proxy_async();
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    if (tid == 0)
        for (int q = 0; q < kStages - 1 && q < ntiles; ++q) issue(q);
    for (int tt = 0; tt < ntiles; ++tt) {
        const int buf = tt % kStages;
        const int ahead = tt + kStages - 1;  // the tile whose MMA is issued now
        if (ahead < ntiles) {
            convert(ahead % kStages);  // from registers
            jc = jn;
            load_raw();                // tile ahead + 1
            jn = load_idx(ahead + 2);
        }
        tc::fence_proxy_async();
        tc::fence_before();
        __syncthreads();
        tc::fence_after();
        if (tid == 0 && ahead < ntiles) issue(ahead % kStages);
        // chunk c + 1 in the first iteration of chunk c, while the tensor core works: the index of
        // tile T is read at the top of iteration T - kStages - 1, so the last read of chunk c - 1 (same
        // buffer) came kStages + 2 iterations before, and the first read of chunk c + 1 comes
        // kChunkTiles - kStages - 1 >= 1 iterations later, past this iteration's closing barrier
        if (tt % kChunkTiles == 0 && tt + kChunkTiles < ntiles) expand(tt / kChunkTiles + 1);
        if (!tc::mbar_wait(&S.mbar[buf], (phase_bits >> buf) & 1u)) ok = false;
        ok = __all_sync(0xffffffffu, ok);  // tcgen05.ld below is warp-collective
        phase_bits ^= 1u << buf;
        tc::fence_after();
        if (ok && warp_rows) {
            // the load of chunk k+1 flies while chunk k is summed
            constexpr int kChunks = kN / kHalves / 32;
            const uint32_t base = tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)(buf * kN + half * (kN / kHalves));
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
#pragma unroll
            for (int k = 0; k < kChunks; k += 2) {
                if (k + 1 < kChunks) tc::ld32_async(base + 32 * (k + 1), vb);
                sum32(va);
                if (k + 1 < kChunks) {
                    tc::ld_wait(vb);
                    if (k + 2 < kChunks) tc::ld32_async(base + 32 * (k + 2), va);
                    sum32(vb);
                    if (k + 2 < kChunks) tc::ld_wait(va);
                }
            }
        }
        tc::fence_before();
        __syncthreads();  // the buffers of this tile are free again
    }
    ok = __syncthreads_and(ok) != 0;
    if (!ok && tid == 0 && L.tc_err) atomicOr(L.tc_err, 1u);
    tc::fence_after();
    if (warp == 0) tc::tmem_dealloc(tmem, kTmemCols);
    if (!ok) return;  // uniform
    // the two warpgroups' sums of a row
    if (kHalves > 1) {
        if (half == 1) S.tot1[t] = tot;
        __syncthreads();
        if (half == 0) tot += S.tot1[t];
    }

    if (tid == 0 && L.pairs) atomicAdd(L.pairs, (unsigned long long)nr * (unsigned long long)ncol);

    if (L.part) {
        // split block: partial sums; the CTA that completes the block's last item finishes it
        if (half == 0) L.part[(size_t)it * kPartRows + t] = tot;
        __threadfence();
        __syncthreads();
        if (tid == 0) {
            int fi = L.item_fin[it];
            OTGB_DCLAMP(fi, 0, L.n_fin);
            S.bc[0] = fi;
            S.bc[1] = atomicAdd(L.fin_count + fi, 1) + 1;
        }
        __syncthreads();
        const int4 fe = L.fin[S.bc[0]];
        if (S.bc[1] != fe.w) return;  // uniform
        __threadfence();
        tot = 0.f;
        if (half == 0)
            for (int q = 0; q < fe.w; ++q) {
                int iq = fe.z + q;
                OTGB_DCLAMP(iq, 0, L.n_items);
                tot += __ldcg(L.part + (size_t)iq * kPartRows + t);
            }
    }
    float dmax = 0.f;
    if (valid) {
        const int r = r0 + t;
        if (!(tot >= 0x1p-60f && tot <= 0x1p60f)) {
            const int k = atomicAdd(L.n_fallback, 1);
            if (k < L.fallback_cap) L.fallback[k] = make_int4(item.x, r, blk, 0);
        } else {
            const double L2 = m_eff + log2((double)tot);
            const double tilde = -(double)I.lam * (L.eps_ln2 * L2 - hx);
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
    if (lane == 0 && L.delta_max) atomicMax(L.delta_max, __float_as_uint(dmax));
}


}  // namespace

void softmin3_tc_launch(const SoftminLaunch &L, cudaStream_t st) {
    static PerDevice<int> attr;
    attr.get([] {
        OTGB_CUDA_TRY(cudaFuncSetAttribute(softmin3_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)sizeof(Tc3Smem)));
        return 1;
    });
    softmin3_tc_kernel<<<L.n_items, kThreads, sizeof(Tc3Smem), st>>>(L);
    OTGB_CHECK_LAUNCH();
}

}  // namespace otgb
