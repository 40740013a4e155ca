// Per-clock throughput of the units that bound the softmin kernels, measured
// on the device: MUFU ex2 (ex2.approx.ftz.f32), scalar FP32 FMA and packed
// FP32x2 FMA.  These are the per-SM, per-clock rates the rooflines use.
//
// Each CTA runs 256 threads, each with 8 independent dependency chains of the
// instruction under test, and records its SM and its first and last cycle
// (the SM's own counter); the grid holds about 4 CTAs per SM.  The rate of an
// SM is the work of the CTAs it ran over the span from its first start to its
// last end; the result is the mean over the SMs.
#include <algorithm>
#include <map>
#include <vector>

#include "solver.cuh"

namespace otgb {
namespace {

constexpr int kRT = 256, kRCtasPerSm = 4, kRIters = 4096, kRChains = 8;

__device__ __forceinline__ float ex2r(float v) {
    float y;
    asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(v));
    return y;
}
__device__ __forceinline__ unsigned long long fma2r(unsigned long long a, unsigned long long b,
                                                   unsigned long long c) {
    unsigned long long d;
    asm volatile("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

// kind 0: ex2, 1: scalar FMA, 2: packed FMA.  rec[3 blockIdx.x ..] = (SM id, start, end); sink keeps
// the results alive (written only when a chain ends at an impossible value).
__global__ void __launch_bounds__(kRT) rates_kernel(int kind, long long *rec, float *sink) {
    float v[kRChains];
    unsigned long long p[kRChains];
#pragma unroll
    for (int c = 0; c < kRChains; ++c) {
        v[c] = -1.0f - 1e-3f * (float)(threadIdx.x + c);
        p[c] = ((unsigned long long)__float_as_uint(v[c]) << 32) | __float_as_uint(v[c]);
    }
    const float a = 0.999f, b = 1e-4f;
    const unsigned long long a2 = ((unsigned long long)__float_as_uint(a) << 32) | __float_as_uint(a);
    const unsigned long long b2 = ((unsigned long long)__float_as_uint(b) << 32) | __float_as_uint(b);
    __syncthreads();
    const long long t0 = clock64();
    if (kind == 0) {
        for (int it = 0; it < kRIters; ++it)
#pragma unroll
            for (int c = 0; c < kRChains; ++c) v[c] = ex2r(v[c]) - 1.5f;  // stays in (-1.5, -0.5)
    } else if (kind == 1) {
        for (int it = 0; it < kRIters; ++it)
#pragma unroll
            for (int c = 0; c < kRChains; ++c) v[c] = fmaf(v[c], a, b);
    } else {
        for (int it = 0; it < kRIters; ++it)
#pragma unroll
            for (int c = 0; c < kRChains; ++c) p[c] = fma2r(p[c], a2, b2);
    }
    __syncthreads();
    const long long t1 = clock64();
    float acc = 0.f;
#pragma unroll
    for (int c = 0; c < kRChains; ++c) acc += v[c] + __uint_as_float((unsigned)p[c]);
    if (acc == 12345.f) sink[threadIdx.x] = acc;
    if (threadIdx.x == 0) {
        unsigned smid;
        asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
        rec[3 * blockIdx.x] = smid;
        rec[3 * blockIdx.x + 1] = t0;
        rec[3 * blockIdx.x + 2] = t1;
    }
}

}  // namespace
}  // namespace otgb

using namespace otgb;

extern "C" int otgb_unit_rates(otgb_ctx *ctx, double *ex2_per_clk_sm, double *fma_per_clk_sm,
                               double *fma2_per_clk_sm) {
    if (!ctx) return fail(nullptr, Error{OTGB_EINVAL, "otgb_unit_rates: null context"});
    try {
        ctx_set_device(ctx);
        require(ex2_per_clk_sm && fma_per_clk_sm && fma2_per_clk_sm, "otgb_unit_rates: null pointer argument");
        cudaStream_t st = ctx_stream(ctx);
        const int sms = ctx_sm_count(ctx), grid = sms * kRCtasPerSm;
        long long *rec = ctx_ws(ctx).get<long long>("rates:rec", 3 * (size_t)grid);
        float *sink = ctx_ws(ctx).get<float>("rates:sink", kRT);
        std::vector<long long> h(3 * (size_t)grid);
        double *out[3] = {ex2_per_clk_sm, fma_per_clk_sm, fma2_per_clk_sm};
        for (int kind = 0; kind < 3; ++kind) {
            for (int rep = 0; rep < 2; ++rep) {  // the first launch warms up; the second is kept
                rates_kernel<<<grid, kRT, 0, st>>>(kind, rec, sink);
                OTGB_CHECK_LAUNCH();
            }
            OTGB_CUDA_TRY(cudaMemcpyAsync(h.data(), rec, sizeof(long long) * h.size(), cudaMemcpyDeviceToHost, st));
            OTGB_CUDA_TRY(cudaStreamSynchronize(st));
            // lane operations per CTA: ex2 and scalar FMA one per instruction and lane, packed FMA two
            const double ops = (double)kRT * kRIters * kRChains * (kind == 2 ? 2.0 : 1.0);
            std::map<long long, std::pair<long long, long long>> span;
            std::map<long long, int> n;
            for (int b = 0; b < grid; ++b) {
                const long long sm = h[3 * b], a = h[3 * b + 1], e = h[3 * b + 2];
                auto it = span.find(sm);
                if (it == span.end()) span[sm] = {a, e};
                else it->second = {std::min(it->second.first, a), std::max(it->second.second, e)};
                ++n[sm];
            }
            double rate = 0.0;
            for (auto &kv : span) rate += n[kv.first] * ops / (double)std::max(1LL, kv.second.second - kv.second.first);
            *out[kind] = rate / (double)span.size();
        }
        return OTGB_OK;
    } catch (const Error &e) {
        return fail(ctx, e);
    }
}
