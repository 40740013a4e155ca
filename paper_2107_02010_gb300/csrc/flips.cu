// Flip augmentation of fiber tractograms and the choice of the matched
// version after label transfer (Section 2: the feature space of fibers
// resampled to P points is R^{3P}; the orientation of a fiber is arbitrary, so
// the tractogram is augmented with the mirror flip of every fiber, the plan is
// computed on the augmented data, and only the version that the plan matches
// is kept for the transfer of labels).
#include "solver.cuh"

namespace otgb {
namespace {

// out rows 0..N-1: the fibers; rows N..2N-1: point k of the flip is point P-1-k
__global__ void flip_fibers_kernel(const float *x, int N, int P, float *out) {
    const int D = 3 * P;
    const size_t total = (size_t)N * D;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        const size_t i = e / D;
        const int d = (int)(e - i * D);
        const int k = d / 3, c = d - 3 * k;
        const float v = x[e];
        out[e] = v;
        out[(size_t)(N + i) * D + 3 * (P - 1 - k) + c] = v;
    }
}

// version 1 (the flip) when its row mass is larger, else the original
__global__ void select_flips_kernel(const float *row_mass, const int *argmax, int N, int *label, int *version,
                                    float *mass) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int v = row_mass[N + i] > row_mass[i] ? 1 : 0;
    if (label) label[i] = argmax[v * N + i];
    if (version) version[i] = v;
    if (mass) mass[i] = row_mass[v * N + i];
}

}  // namespace
}  // namespace otgb

using namespace otgb;

extern "C" int otgb_flip_fibers(otgb_ctx *ctx, const float *x, int N, int P, float *out) {
    if (!ctx) return fail(nullptr, Error{OTGB_EINVAL, "otgb_flip_fibers: null context"});
    try {
        ctx_set_device(ctx);
        require(x && out, "otgb_flip_fibers: null pointer argument");
        require(N >= 1 && P >= 1 && 3 * P <= 64, "otgb_flip_fibers: N >= 1 and 1 <= P <= 21 required");
        cudaStream_t st = ctx_stream(ctx);
        const size_t total = (size_t)N * 3 * P;
        const int grid = (int)std::min<size_t>((total + 255) / 256, (size_t)ctx_sm_count(ctx) * 16);
        flip_fibers_kernel<<<grid, 256, 0, st>>>(x, N, P, out);
        OTGB_CHECK_LAUNCH();
        OTGB_CUDA_TRY(cudaStreamSynchronize(st));
        return OTGB_OK;
    } catch (const Error &e) {
        return fail(ctx, e);
    }
}

extern "C" int otgb_select_flips(otgb_ctx *ctx, const float *row_mass, const int32_t *argmax, int N, int32_t *label,
                                 int32_t *version, float *mass) {
    if (!ctx) return fail(nullptr, Error{OTGB_EINVAL, "otgb_select_flips: null context"});
    try {
        ctx_set_device(ctx);
        require(row_mass && argmax && label, "otgb_select_flips: null pointer argument");
        require(N >= 1, "otgb_select_flips: N >= 1 required");
        cudaStream_t st = ctx_stream(ctx);
        select_flips_kernel<<<(N + 255) / 256, 256, 0, st>>>(row_mass, argmax, N, label, version, mass);
        OTGB_CHECK_LAUNCH();
        OTGB_CUDA_TRY(cudaStreamSynchronize(st));
        return OTGB_OK;
    } catch (const Error &e) {
        return fail(ctx, e);
    }
}
