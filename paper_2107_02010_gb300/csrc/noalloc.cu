// otgb_softmin_noalloc: the softmin sweep of otgb_softmin for callers that may
// not allocate device memory.  All scratch lives in one file-scope device
// array of fixed size (kNoAllocBytes); no cudaMalloc, cudaFree or allocating
// library routine is called, and no context object is needed.
#include <cmath>
#include <cstring>
#include <mutex>

#include "prims.cuh"
#include "solver.cuh"

namespace otgb {
namespace {

constexpr size_t kNoAllocBytes = 16u << 20;  // 16 MiB, held by every device that loads the library
__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

std::mutex g_noalloc_mu;
void *g_noalloc_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device (looked up once
// per device; the array's host-side name is not a device address).
void *scratch_address() {
    int dev = 0;
    OTGB_CUDA_TRY(cudaGetDevice(&dev));
    require(dev >= 0 && dev < kMaxDevices, "otgb_softmin_noalloc: device ordinal out of range");
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        OTGB_CUDA_TRY(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        g_noalloc_ptr[dev] = p;
    }
    return g_noalloc_ptr[dev];
}

__global__ void centre_kernel(const float *lo, const float *hi, int D, float *c) {
    const int d = threadIdx.x;
    if (d < 64) c[d] = d < D ? 0.5f * (lo[d] + hi[d]) : 0.f;
}

__global__ void dense_items_kernel(int4 *items, int nb, int n_in) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < nb) items[k] = make_int4(0, k, 0, n_in);
}

// Bump allocator over the scratch array (256-byte aligned pieces).  With a
// null base it only adds up the sizes (no pointer is formed), which decides
// whether a problem fits before anything is launched.
struct Carve {
    unsigned char *base;
    size_t used = 0;
    template <class T> T *take(size_t count) {
        const size_t off = used;
        used += (count * sizeof(T) + 255) & ~size_t(255);
        return base ? reinterpret_cast<T *>(base + off) : nullptr;
    }
};

}  // namespace
}  // namespace otgb

using namespace otgb;

extern "C" int otgb_softmin_noalloc(const float *q, int n_out, const float *p, const float *w, const float *pot,
                                    int n_in, int D, double eps, double lam, const float *old, double omega,
                                    float *out, void *cuda_stream) {
    try {
        require(q && p && w && pot && out, "otgb_softmin_noalloc: null pointer argument");
        require(n_out >= 1 && n_in >= 1, "otgb_softmin_noalloc: sizes must be >= 1");
        require(D >= 1 && D <= 64, "otgb_softmin_noalloc: D must be in [1, 64]");
        require(eps > 0.0 && std::isfinite(eps), "otgb_softmin_noalloc: eps must be > 0");
        cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
        const int stride = D <= 3 ? 4 : ((D + 3) & ~3);
        int sms = 0, dev = 0;
        OTGB_CUDA_TRY(cudaGetDevice(&dev));
        OTGB_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        int rpt = 1;
        if (D <= 3)
            for (int r : {4, 2})
                if ((n_out + 32 * r - 1) / (32 * r) >= 8 * sms) { rpt = r; break; }
        const int block_rows = D <= 3 ? 32 * rpt : 128;
        const int nb = (n_out + block_rows - 1) / block_rows;
        // scratch layout; the sizes decide admissibility
        Carve dry{nullptr};
        dry.take<float>(128);                         // lo, hi
        dry.take<float>(64);                          // centre
        dry.take<float>(64 * 2 * 64);                 // bbox partials
        dry.take<float>((size_t)n_out * stride);      // packed rows
        dry.take<float>((size_t)n_in * stride);       // packed columns
        if (D > 3) dry.take<float>(n_in);             // column log-weights
        dry.take<int>(nb + 1);                        // row blocks
        dry.take<int4>(nb);                           // work items
        dry.take<int4>((size_t)n_out + 64);           // fallback rows
        dry.take<int>(1);                             // fallback count
        if (dry.used > kNoAllocBytes)
            throw Error{OTGB_EINVAL, "otgb_softmin_noalloc: problem needs " + std::to_string(dry.used) +
                                         " bytes of scratch, more than the fixed " +
                                         std::to_string(kNoAllocBytes) + " (reduce n_out, n_in or D)"};
        Carve c{static_cast<unsigned char *>(scratch_address())};
        float *lohi = c.take<float>(128);
        float *cen = c.take<float>(64);
        float *bpart = c.take<float>(64 * 2 * 64);
        float *R = c.take<float>((size_t)n_out * stride);
        float *Cc = c.take<float>((size_t)n_in * stride);
        float *Clw = D > 3 ? c.take<float>(n_in) : nullptr;
        int *blk = c.take<int>(nb + 1);
        int4 *items = c.take<int4>(nb);
        int4 *fb = c.take<int4>((size_t)n_out + 64);
        int *nfb = c.take<int>(1);

        bbox(p, n_in, D, D, lohi, lohi + 64, bpart, st);
        centre_kernel<<<1, 64, 0, st>>>(lohi, lohi + 64, D, cen);
        OTGB_CHECK_LAUNCH();
        pack_points(q, nullptr, nullptr, n_out, D, cen, R, nullptr, nullptr, st);
        pack_points(p, w, nullptr, n_in, D, cen, Cc, Clw, nullptr, st);
        uniform_blocks(blk, n_out, block_rows, st);
        dense_items_kernel<<<(nb + 255) / 256, 256, 0, st>>>(items, nb, n_in);
        OTGB_CHECK_LAUNCH();
        SoftminLaunch L;
        std::memset(&L, 0, sizeof(L));
        L.n_inst = 1;
        SoftminInst &I = L.inst[0];
        I.rows = R; I.cols = Cc; I.col_logw = Clw; I.col_pot = pot; I.row_old = old; I.row_out = out;
        I.n_rows = n_out; I.n_cols = n_in; I.lam = (float)lam; I.omega = (float)omega;
        I.blk_row0 = blk;
        L.items = items;
        L.n_items = nb;
        L.exact_max = 1;
        L.eps = (float)eps;
        L.s = (float)(1.4426950408889634 / eps);
        L.eps_ln2 = eps * 0.69314718055994530942;
        L.fallback = fb;
        L.n_fallback = nfb;  // zeroed by softmin_run before the kernels
        L.fallback_cap = n_out + 64;
        softmin_run(L, D, rpt, st);
        OTGB_CUDA_TRY(cudaStreamSynchronize(st));
        return OTGB_OK;
    } catch (const Error &e) {
        return fail(nullptr, e);
    }
}
