// Host driver of the symmetric, debiased, eps-scaled Sinkhorn loop
// (the Algorithm of Section 2) and the C ABI declared in include/otgb.h.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <cstdlib>
#include <memory>

#include "prims.cuh"
#include "solver.cuh"

using namespace otgb;

struct otgb_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    Workspace ws;
    std::string err;
    cudaEvent_t ev[8] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    // pinned host mailbox for small device->host reads
    void *pinned = nullptr;
};

static thread_local std::string g_err;

namespace otgb {
static unsigned long long g_launches = 0;
bool debug_sync_enabled() {
    static int v = -1;
    if (v < 0) {
        const char *e = std::getenv("OTGB_DEBUG_SYNC");
        v = (e && e[0] == '1') ? 1 : 0;
    }
    return v == 1;
}
void count_launch() { __atomic_add_fetch(&g_launches, 1ull, __ATOMIC_RELAXED); }
unsigned long long launch_count() { return __atomic_load_n(&g_launches, __ATOMIC_RELAXED); }
int current_device() {
    int d = 0;
    OTGB_CUDA_TRY(cudaGetDevice(&d));
    return d;
}
}  // namespace otgb

namespace otgb {

void *Workspace::get(const std::string &name, size_t bytes) {
    for (auto &b : bufs)
        if (b.name == name) {
            if (b.bytes >= bytes) return b.ptr;
            OTGB_CUDA_TRY(cudaFreeAsync(b.ptr, stream));
            b.ptr = nullptr;
            b.bytes = 0;
            const cudaError_t e = cudaMallocAsync(&b.ptr, bytes, stream);
            if (e != cudaSuccess) throw Error{OTGB_ENOMEM, "device allocation of " + std::to_string(bytes) + " bytes failed"};
            b.bytes = bytes;
            return b.ptr;
        }
    Buf b;
    b.name = name;
    const cudaError_t e = cudaMallocAsync(&b.ptr, bytes, stream);
    if (e != cudaSuccess) throw Error{OTGB_ENOMEM, "device allocation of " + std::to_string(bytes) + " bytes failed"};
    b.bytes = bytes;
    bufs.push_back(b);
    return b.ptr;
}

void Workspace::release() {
    for (auto &b : bufs)
        if (b.ptr) cudaFreeAsync(b.ptr, stream);
    bufs.clear();
}

// ------------------------------------------------------------ schedule ----
// sigma_k = d q^k for k = 0 .. K-1, K = ceil(log(d/blur)/log(1/q)), then blur.
std::vector<double> make_schedule(double d, double blur, double q) {
    std::vector<double> s;
    if (d > blur) {
        const int K = (int)std::ceil(std::log(d / blur) / std::log(1.0 / q));
        for (int k = 0; k < K; ++k) s.push_back(d * std::pow(q, (double)k));
    }
    s.push_back(blur);
    return s;
}

double lambda_of(double sigma, double reach, int p) {
    if (!(reach > 0.0) || std::isinf(reach)) return 1.0;
    return 1.0 / (1.0 + std::pow(sigma / reach, (double)p));
}

}  // namespace otgb

// ------------------------------------------------------------------ ABI ----
extern "C" {

void otgb_default_params(otgb_params *p) {
    std::memset(p, 0, sizeof(*p));
    p->p = 2;
    p->blur = 0.05;
    p->reach = 0.0;
    p->scaling = 0.5;
    p->diameter = 0.0;
    p->multiscale = 0;
    p->cluster = OTGB_CLUSTER_GRID;
    p->cell = 0.0;
    p->k_clusters = 0;
    p->kmeans_iters = 10;
    p->seed = 0;
    p->sigma_switch = 0.0;
    p->trunc_tau = 27.6;
    p->tol = 1e-6;
    p->min_iters = 3;
    p->max_iters = 100000;
    p->check_every = 10;
    p->fixed_iters = 0;
    p->precision = OTGB_FP32;
    p->sigma_start = 0.0;
    p->translation = 1;
    p->anderson = 5;
}

int otgb_create(otgb_ctx **out, int device, void *cuda_stream) {
    if (!out) {
        g_err = "otgb_create: null output";
        return OTGB_EINVAL;
    }
    *out = nullptr;
    try {
        int n = 0;
        OTGB_CUDA_TRY(cudaGetDeviceCount(&n));
        require(device >= 0 && device < n, "otgb_create: no such device");
        OTGB_CUDA_TRY(cudaSetDevice(device));
        std::unique_ptr<otgb_ctx> c(new otgb_ctx);
        c->device = device;
        c->stream = static_cast<cudaStream_t>(cuda_stream);
        c->ws.stream = c->stream;
        for (auto &e : c->ev) OTGB_CUDA_TRY(cudaEventCreate(&e));
        OTGB_CUDA_TRY(cudaMallocHost(&c->pinned, 4096));
        *out = c.release();
        return OTGB_OK;
    } catch (const Error &e) {
        g_err = e.msg;
        return e.code;
    }
}

int otgb_destroy(otgb_ctx *ctx) {
    if (!ctx) return OTGB_OK;
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    ctx->ws.release();
    cudaStreamSynchronize(ctx->stream);
    for (auto &e : ctx->ev)
        if (e) cudaEventDestroy(e);
    if (ctx->pinned) cudaFreeHost(ctx->pinned);
    delete ctx;
    return OTGB_OK;
}

const char *otgb_last_error(const otgb_ctx *ctx) { return ctx ? ctx->err.c_str() : g_err.c_str(); }

unsigned long long otgb_kernel_launches(void) { return otgb::launch_count(); }

}  // extern "C"

namespace otgb {

int fail(otgb_ctx *ctx, const Error &e) {
    if (ctx) ctx->err = e.msg;
    g_err = e.msg;
    return e.code;
}

cudaStream_t ctx_stream(otgb_ctx *ctx) { return ctx->stream; }
Workspace &ctx_ws(otgb_ctx *ctx) { return ctx->ws; }
void *ctx_pinned(otgb_ctx *ctx) { return ctx->pinned; }
cudaEvent_t ctx_event(otgb_ctx *ctx, int k) { return ctx->ev[k]; }
void ctx_set_device(otgb_ctx *ctx) { OTGB_CUDA_TRY(cudaSetDevice(ctx->device)); }
int ctx_sm_count(otgb_ctx *ctx) {
    int n = 0;
    OTGB_CUDA_TRY(cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, ctx->device));
    return n;
}

}  // namespace otgb
