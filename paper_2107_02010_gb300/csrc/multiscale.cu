// Coarse-to-fine strategy of Section 2: cluster both clouds (grid cells or
// K-means), run the eps-scaled symmetric loop on the cluster measures while
// sigma is above the cluster scale, extrapolate the four duals to the points
// with one softmin each, then iterate at full resolution over the cluster
// pairs that the current duals do not prove negligible (kernel truncation),
// re-deciding the kept pairs at every new sigma and periodically at blur.
//
// Truncation bound.  For row cluster I and column cluster J (centroids c,
// radii r) every point pair satisfies |x_i - y_j| >= (|c_I - c_J| - r_I - r_J)_+,
// so the log-plan term of a pair relative to its row total,
//   eps log w_j + pot_j - C_ij + old_i / lam   (old_i / lam ~ -eps LSE_i),
// is at most  B(I,J) = max_J (eps log w + pot) - (|c_I - c_J| - r_I - r_J)_+^2 / 2
//                      + max_I old / lam.
// A pair (I, J) is kept when B(I,J) >= min(-tau eps, max_J' B(I,J') - tau eps):
// every dropped term is below e^-tau times its row total at the fixed point,
// and every row cluster keeps at least the pairs within tau of its best bound.
#include <algorithm>
#include <cfloat>
#include <cmath>
#include <cstring>

#include "kmeans.cuh"
#include "multiscale.cuh"
#include "prims.cuh"
#include "solver.cuh"

namespace otgb {
namespace {

// Per cluster c of one side (sorted positions [off[c], off[c+1])): maxima of
// two potentials u, v and of eps log w + u, eps log w + v.
__global__ void cluster_max_kernel(const int *off, int ncl, const float *u, const float *v, const float *lw,
                                   int lw_stride, float eps, float4 *out) {
    __shared__ float red[4][4];
    const int c = blockIdx.x;
    if (c >= ncl) return;
    const int a = off[c], b = off[c + 1];
    float m0 = -INFINITY, m1 = -INFINITY, m2 = -INFINITY, m3 = -INFINITY;
    for (int i = a + threadIdx.x; i < b; i += blockDim.x) {
        const float l = lw[(size_t)i * lw_stride];
        const float ui = u[i], vi = v[i];
        m0 = fmaxf(m0, ui);
        m1 = fmaxf(m1, vi);
        m2 = fmaxf(m2, fmaf(eps, l, ui));
        m3 = fmaxf(m3, fmaf(eps, l, vi));
    }
    for (int o = 16; o > 0; o >>= 1) {
        m0 = fmaxf(m0, __shfl_xor_sync(0xffffffffu, m0, o));
        m1 = fmaxf(m1, __shfl_xor_sync(0xffffffffu, m1, o));
        m2 = fmaxf(m2, __shfl_xor_sync(0xffffffffu, m2, o));
        m3 = fmaxf(m3, __shfl_xor_sync(0xffffffffu, m3, o));
    }
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) { red[w][0] = m0; red[w][1] = m1; red[w][2] = m2; red[w][3] = m3; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 1; k < (int)(blockDim.x >> 5); ++k) {
            m0 = fmaxf(m0, red[k][0]); m1 = fmaxf(m1, red[k][1]);
            m2 = fmaxf(m2, red[k][2]); m3 = fmaxf(m3, red[k][3]);
        }
        out[c] = make_float4(m0, m1, m2, m3);
    }
}

struct MaskInst {
    const float *cen_r, *cen_c;   // centroids (stride floats)
    const float *rad_r, *rad_c;
    const float4 *max_r;          // row side maxima, component row_sel = max old
    const float4 *max_c;          // column side maxima, component col_sel = max (eps log w + pot)
    int row_sel, col_sel;
    int ncl_r, ncl_c;
    float inv_lam;
    unsigned *bits;               // ncl_r x nwords
};

struct MaskLaunch {
    MaskInst inst[4];
    int D, stride, nwords;
    int p1;  // 1: cost |x - y| (lower bound gap), else |x - y|^2 / 2 (gap^2 / 2)
    float eps, tau;
};

__device__ __forceinline__ float comp(const float4 &v, int k) {
    return k == 0 ? v.x : (k == 1 ? v.y : (k == 2 ? v.z : v.w));
}

// Grid (ncl_r, 4): the keep bits of row cluster I for every column cluster J.
__global__ void mask_kernel(const __grid_constant__ MaskLaunch M) {
    __shared__ float red[8];
    __shared__ float cI[64];
    const MaskInst &P = M.inst[blockIdx.y];
    const int I = blockIdx.x;
    if (I >= P.ncl_r) return;
    for (int d = threadIdx.x; d < M.D; d += blockDim.x) cI[d] = P.cen_r[(size_t)I * M.stride + d];
    __syncthreads();
    const float rI = P.rad_r[I];
    const float rowterm = comp(P.max_r[I], P.row_sel) * P.inv_lam;
    auto bound = [&](int J) -> float {
        const float *cJ = P.cen_c + (size_t)J * M.stride;
        float d2 = 0.f;
        for (int d = 0; d < M.D; ++d) { const float t = cI[d] - cJ[d]; d2 = fmaf(t, t, d2); }
        const float gap = fmaxf(sqrtf(d2) - rI - P.rad_c[J], 0.f);
        return comp(P.max_c[J], P.col_sel) - (M.p1 ? gap : 0.5f * gap * gap) + rowterm;
    };
    float bm = -INFINITY;
    for (int J = threadIdx.x; J < P.ncl_c; J += blockDim.x) bm = fmaxf(bm, bound(J));
    for (int o = 16; o > 0; o >>= 1) bm = fmaxf(bm, __shfl_xor_sync(0xffffffffu, bm, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = bm;
    __syncthreads();
    bm = red[0];
    for (int k = 1; k < (int)(blockDim.x >> 5); ++k) bm = fmaxf(bm, red[k]);
    const float thr = fminf(-M.tau * M.eps, bm - M.tau * M.eps);
    // 256 threads: 8 warps cover 256 consecutive J per round, one word per warp
    for (int base = 0; base < M.nwords * 32; base += blockDim.x) {
        const int J = base + threadIdx.x;
        const bool keep = J < P.ncl_c && bound(J) >= thr;
        const unsigned word = __ballot_sync(0xffffffffu, keep);
        const int wi = J >> 5;
        if ((threadIdx.x & 31) == 0 && wi < M.nwords) P.bits[(size_t)I * M.nwords + wi] = word;
    }
}

struct ListInst {
    const unsigned *bits;   // ncl_r x nwords
    const int *blk_cl;      // 2 ints per block: first and end row cluster
    const int *off_c;       // column cluster offsets (ncl_c + 1)
    int nblk;
};

struct ListLaunch {
    ListInst inst[4];
    int base[5];            // flat index of (inst, 0)
    int nwords;
    int *counts;            // count pass, per flat block: kept columns, kept clusters (2 ints)
    const int *rng_ptr;     // write pass, per flat block: first range entry
    int2 *rng;              // write pass: (first column, position) per kept cluster, then the sentinel
};

__device__ __forceinline__ void flat_to_inst(const ListLaunch &L, int f, int &k, int &b) {
    k = 0;
    while (k < 3 && f >= L.base[k + 1]) ++k;
    b = f - L.base[k];
}

// Kept columns of a block: the union of the keep bits of its row clusters.
// The columns are sorted by cluster, so every kept cluster J is one range of
// consecutive columns [off_c[J], off_c[J+1]), and a run of kept clusters
// J, J+1, .., J+k is one range [off_c[J], off_c[J+k+1]).  Each thread owns a
// contiguous range of bit words and writes one entry per run within them (a
// run that crosses into the next thread's words continues as a second entry),
// so the ranges come out in increasing order.
// WRITE = false: count the kept columns and the entries; true: write the
// entries with their positions (exclusive scans over the threads), then the
// sentinel.
template <bool WRITE>
__global__ void list_kernel(const __grid_constant__ ListLaunch L) {
    __shared__ int scan[256], sscan2[256];
    int k, b;
    flat_to_inst(L, blockIdx.x, k, b);
    const ListInst &P = L.inst[k];
    const int cl0 = P.blk_cl[2 * b], cl1 = P.blk_cl[2 * b + 1];
    const int wpt = (L.nwords + blockDim.x - 1) / blockDim.x;
    const int w0 = threadIdx.x * wpt, w1 = min(L.nwords, w0 + wpt);
    int cnt = 0, nq = 0, last = -2;  // last: the previous kept cluster of this thread
    for (int w = w0; w < w1; ++w) {
        unsigned u = 0;
        for (int I = cl0; I < cl1; ++I) u |= P.bits[(size_t)I * L.nwords + w];
        while (u) {
            const int J = w * 32 + __ffs(u) - 1;
            u &= u - 1;
            nq += J != last + 1;
            last = J;
            cnt += P.off_c[J + 1] - P.off_c[J];
        }
    }
    // inclusive scans of the per-thread column and cluster counts
    scan[threadIdx.x] = cnt;
    sscan2[threadIdx.x] = nq;
    __syncthreads();
    for (int o = 1; o < (int)blockDim.x; o <<= 1) {
        const int v = threadIdx.x >= o ? scan[threadIdx.x - o] : 0;
        const int v2 = threadIdx.x >= o ? sscan2[threadIdx.x - o] : 0;
        __syncthreads();
        scan[threadIdx.x] += v;
        sscan2[threadIdx.x] += v2;
        __syncthreads();
    }
    const int T = scan[blockDim.x - 1], Q = sscan2[blockDim.x - 1];
    if (!WRITE) {
        if (threadIdx.x == 0) {
            L.counts[2 * blockIdx.x] = T;
            L.counts[2 * blockIdx.x + 1] = Q;
        }
        return;
    }
    int2 *out = L.rng + L.rng_ptr[blockIdx.x];
    int pos = scan[threadIdx.x] - cnt, q = sscan2[threadIdx.x] - nq;
    last = -2;
    for (int w = w0; w < w1; ++w) {
        unsigned u = 0;
        for (int I = cl0; I < cl1; ++I) u |= P.bits[(size_t)I * L.nwords + w];
        while (u) {
            const int J = w * 32 + __ffs(u) - 1;
            u &= u - 1;
            if (J != last + 1) out[q++] = make_int2(P.off_c[J], pos);
            last = J;
            pos += P.off_c[J + 1] - P.off_c[J];
        }
    }
    if (threadIdx.x == blockDim.x - 1) out[Q] = make_int2(0, T);
}

__global__ void log_kernel(const float *m, int n, float *out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = m[i] > 0.f ? logf(m[i]) : -INFINITY;
}

// Row blocks of at most `br` rows made of consecutive clusters; a cluster
// larger than br is cut into pieces.  Writes starts (nblk + 1) and the
// cluster range of each block.  merge = false keeps one cluster per block:
// consecutive k-means clusters need not be neighbours, and a block that spans
// two distant clusters (two fiber bundles) has a large spread around its
// centre, which the dot-product form of the cost turns into rounding error
// (the terms s |x - c|^2 / 2 grow with the spread while the exponent of a
// relevant pair stays small).  Grid cells in Morton order are neighbours, so
// the grid blocks merge.
void group_blocks(const std::vector<int> &off, int br, bool merge, std::vector<int> &starts, std::vector<int> &cl) {
    starts.clear();
    cl.clear();
    const int ncl = (int)off.size() - 1;
    int c = 0;
    while (c < ncl) {
        const int sz = off[c + 1] - off[c];
        if (sz > br) {
            for (int r = off[c]; r < off[c + 1]; r += br) {
                starts.push_back(r);
                cl.push_back(c);
                cl.push_back(c + 1);
            }
            ++c;
            continue;
        }
        const int first = c;
        int rows = 0;
        while (c < ncl && off[c + 1] - off[c] <= br && rows + (off[c + 1] - off[c]) <= br &&
               (merge || c == first)) {
            rows += off[c + 1] - off[c];
            ++c;
        }
        starts.push_back(off[first]);
        cl.push_back(first);
        cl.push_back(c);
    }
    starts.push_back(off[ncl]);
}

}  // namespace

void Multiscale::cluster(Solver &s, const otgb_params &P, const float *x, const float *a, const float *y,
                         const float *b, const std::vector<float> &lox, const std::vector<float> &hix,
                         const std::vector<float> &loy, const std::vector<float> &hiy, float *d_box) {
    cudaStream_t st = s.st;
    const int D = s.D;
    reach = P.reach;
    tau = P.trunc_tau > 0.0 ? P.trunc_tau : 27.6;
    rebuild_every = std::max(1, P.check_every);
    auto fetch_offsets = [&](const int *d_off, int n_plus_1, std::vector<int> &h, bool drop_empty) {
        std::vector<int> t(n_plus_1);
        OTGB_CUDA_TRY(cudaMemcpyAsync(t.data(), d_off, sizeof(int) * n_plus_1, cudaMemcpyDeviceToHost, st));
        OTGB_CUDA_TRY(cudaStreamSynchronize(st));
        h.clear();
        for (int k = 0; k < n_plus_1; ++k)
            if (!drop_empty || k == 0 || t[k] != h.back()) h.push_back(t[k]);
    };
    if (P.cluster == OTGB_CLUSTER_GRID) {
        require(D <= 3, "sinkhorn_divergence: grid clustering needs D <= 3");
        require(P.cell > 0.0, "sinkhorn_divergence: grid clustering needs cell > 0");
        GridClusters gx = grid_cluster(s.ctx, "msx", x, s.X.n, D, (float)P.cell, d_box);
        GridClusters gy = grid_cluster(s.ctx, "msy", y, s.Y.n, D, (float)P.cell, d_box + 128);
        s.X.perm = gx.perm;
        s.Y.perm = gy.perm;
        fetch_offsets(gx.offsets, gx.n_clusters + 1, s.X_off, false);
        fetch_offsets(gy.offsets, gy.n_clusters + 1, s.Y_off, false);
        sigma_switch = P.sigma_switch > 0.0 ? P.sigma_switch : P.cell;
    } else {
        const int Kx = std::max(1, std::min(P.k_clusters > 0 ? P.k_clusters : s.X.n / 1000, s.X.n));
        const int Ky = std::max(1, std::min(P.k_clusters > 0 ? P.k_clusters : s.Y.n / 1000, s.Y.n));
        // the Lloyd iterations on at most 131,072 points per side (every s-th point), then one assignment of
        // all points: at 1M points and 1000 clusters the iterations would otherwise dominate the preparation,
        // and clusters only decide the truncation's granularity, not the result
        constexpr int kKmeansSample = 131072;
        KmeansResult rx = kmeans(s.ctx, "msx", x, a, s.X.n, D, Kx, std::max(0, P.kmeans_iters), P.seed, nullptr,
                                 kKmeansSample);
        fetch_offsets(rx.offsets, Kx + 1, s.X_off, true);
        KmeansResult ry = kmeans(s.ctx, "msy", y, b, s.Y.n, D, Ky, std::max(0, P.kmeans_iters), P.seed + 1, nullptr,
                                 kKmeansSample);
        fetch_offsets(ry.offsets, Ky + 1, s.Y_off, true);
        s.X.perm = rx.perm;
        s.Y.perm = ry.perm;
        sigma_switch = P.sigma_switch;  // <= 0: set from the cluster spread in run_schedule
    }
    ncl_x = (int)s.X_off.size() - 1;
    ncl_y = (int)s.Y_off.size() - 1;
    (void)lox; (void)hix; (void)loy; (void)hiy;
}

int Multiscale::run_schedule(Solver &s, const otgb_params &P, const std::vector<double> &sched, int block_rows) {
    cudaStream_t st = s.st;
    Workspace &ws = *s.ws;
    const int D = s.D, stride = s.X.stride;
    // cluster offsets on the device and the coarse measures
    d_off_x = ws.get<int>("ms:offx", ncl_x + 1);
    d_off_y = ws.get<int>("ms:offy", ncl_y + 1);
    OTGB_CUDA_TRY(cudaMemcpyAsync(d_off_x, s.X_off.data(), sizeof(int) * (ncl_x + 1), cudaMemcpyHostToDevice, st));
    OTGB_CUDA_TRY(cudaMemcpyAsync(d_off_y, s.Y_off.data(), sizeof(int) * (ncl_y + 1), cudaMemcpyHostToDevice, st));
    cen_x = ws.get<float>("ms:cenx", (size_t)ncl_x * stride);
    cen_y = ws.get<float>("ms:ceny", (size_t)ncl_y * stride);
    mass_x = ws.get<float>("ms:massx", ncl_x);
    mass_y = ws.get<float>("ms:massy", ncl_y);
    rad_x = ws.get<float>("ms:radx", ncl_x);
    rad_y = ws.get<float>("ms:rady", ncl_y);
    float *ssq_x = ws.get<float>("ms:ssqx", ncl_x), *ssq_y = ws.get<float>("ms:ssqy", ncl_y);
    cluster_stats(s.X.pts, stride, D, s.X.w, d_off_x, ncl_x, cen_x, stride, mass_x, rad_x, ssq_x, st);
    cluster_stats(s.Y.pts, stride, D, s.Y.w, d_off_y, ncl_y, cen_y, stride, mass_y, rad_y, ssq_y, st);
    if (D > 3) {
        lm_x = ws.get<float>("ms:lmx", ncl_x);
        lm_y = ws.get<float>("ms:lmy", ncl_y);
        log_kernel<<<(ncl_x + 255) / 256, 256, 0, st>>>(mass_x, ncl_x, lm_x);
        OTGB_CHECK_LAUNCH();
        log_kernel<<<(ncl_y + 255) / 256, 256, 0, st>>>(mass_y, ncl_y, lm_y);
        OTGB_CHECK_LAUNCH();
    }
    if (!(sigma_switch > 0.0)) {
        // K-means: twice the mass-weighted RMS distance of the points to their centroid
        std::vector<float> hs(ncl_x + ncl_y);
        OTGB_CUDA_TRY(cudaMemcpyAsync(hs.data(), ssq_x, sizeof(float) * ncl_x, cudaMemcpyDeviceToHost, st));
        OTGB_CUDA_TRY(cudaMemcpyAsync(hs.data() + ncl_x, ssq_y, sizeof(float) * ncl_y, cudaMemcpyDeviceToHost, st));
        OTGB_CUDA_TRY(cudaStreamSynchronize(st));
        double t = 0.0;
        for (float v : hs) t += v;
        sigma_switch = 2.0 * std::sqrt(t / (s.X.mass + s.Y.mass));
    }

    // fine row blocks made of consecutive clusters
    const bool merge = P.cluster == OTGB_CLUSTER_GRID;
    group_blocks(s.X_off, block_rows, merge, hbx, hclx);
    group_blocks(s.Y_off, block_rows, merge, hby, hcly);
    d_clx = ws.get<int>("ms:clx", hclx.size());
    d_cly = ws.get<int>("ms:cly", hcly.size());
    OTGB_CUDA_TRY(cudaMemcpyAsync(d_clx, hclx.data(), sizeof(int) * hclx.size(), cudaMemcpyHostToDevice, st));
    OTGB_CUDA_TRY(cudaMemcpyAsync(d_cly, hcly.data(), sizeof(int) * hcly.size(), cudaMemcpyHostToDevice, st));
    s.setup_instances(hbx, hby);
    setup_tcc(s);

    // coarse phase on the cluster measures while sigma > sigma_switch
    size_t k = 0;
    const bool warm = P.f_init || P.g_init || P.a_init || P.b_init;
    if (!warm && !sched.empty() && sched[0] > sigma_switch) {
        Solver cs;
        cs.tag = "c:";
        cs.ctx = s.ctx;
        cs.st = st;
        cs.ws = s.ws;
        cs.D = D;
        cs.p = s.p;
        cs.reach = s.reach;
        cs.rho = s.rho;
        cs.timing = false;
        cs.X.n = ncl_x; cs.X.D = D; cs.X.stride = stride; cs.X.pts = cen_x; cs.X.logw = lm_x; cs.X.w = mass_x;
        cs.X.mass = s.X.mass;
        cs.Y.n = ncl_y; cs.Y.D = D; cs.Y.stride = stride; cs.Y.pts = cen_y; cs.Y.logw = lm_y; cs.Y.w = mass_y;
        cs.Y.mass = s.Y.mass;
        cs.alloc_common();
        otgb_params Pc = P;
        Pc.f_init = Pc.g_init = Pc.a_init = Pc.b_init = nullptr;
        cs.alloc_pots(Pc);
        cs.rows_per_thread = D <= 3 ? 4 : 1;
        cs.setup_dense_instances(D <= 3 ? 32 * cs.rows_per_thread : 128);
        for (; k < sched.size() && sched[k] > sigma_switch && s.steps < P.max_iters; ++k) {
            cs.step(sched[k], false);
            ++s.steps;
            ++s.coarse_steps;
        }
        // extrapolation: one softmin per dual, points against the cluster measures,
        // at the first fine scale (or blur when the schedule ended coarse)
        const double sig = k < sched.size() ? sched[k] : P.blur;
        const double eps = s.eps_of(sig);
        SoftminLaunch E = s.launch;  // fallback buffers, counters
        E.use_tcc = 0;
        E.eps = (float)eps;
        E.s = (float)(1.4426950408889634 / eps);
        E.eps_ln2 = eps * 0.69314718055994530942;
        E.delta_max = nullptr;
        E.pairs = nullptr;
        E.part = nullptr;
        E.fin = nullptr;
        E.n_fin = 0;
        const float lam = (float)s.lam_of(sig);
        const Cloud *ccols[4] = {&cs.X, &cs.Y, &cs.X, &cs.Y};
        const float *cpot[4] = {cs.pa[cs.cur], cs.pb[cs.cur], cs.pf[cs.cur], cs.pg[cs.cur]};
        float *outp[4] = {s.pa[s.cur], s.pb[s.cur], s.pg[s.cur], s.pf[s.cur]};
        for (int q = 0; q < 4; ++q) {
            SoftminInst &I = E.inst[q];
            I.cols = ccols[q]->pts;
            I.col_logw = ccols[q]->logw;
            I.n_cols = ccols[q]->n;
            I.col_pot = cpot[q];
            I.row_old = nullptr;
            I.row_out = outp[q];
            I.lam = lam;
            I.omega = 1.0f;
            I.col_rng = nullptr;
            I.rng_ptr = nullptr;
        }
        std::vector<int4> items;
        for (int q = 0; q < 4; ++q) {
            const int nb = (q == 0 || q == 3) ? s.nblk_x : s.nblk_y;
            for (int bl = 0; bl < nb; ++bl) items.push_back(make_int4(q, bl, 0, E.inst[q].n_cols));
        }
        int4 *d_items = ws.get<int4>("ms:xitems", items.size());
        OTGB_CUDA_TRY(cudaMemcpyAsync(d_items, items.data(), items.size() * sizeof(int4), cudaMemcpyHostToDevice, st));
        E.items = d_items;
        E.n_items = (int)items.size();
        softmin_run(E, D, s.rows_per_thread, st);
        OTGB_CUDA_TRY(cudaStreamSynchronize(st));
    }
    OTGB_CUDA_TRY(cudaEventRecord(ctx_event(s.ctx, 3), st));  // end of the coarse phase
    // fine phase over the rest of the schedule
    for (; k < sched.size() && s.steps < P.max_iters; ++k) s.fine_step(sched[k]);
    return OTGB_OK;
}

// Rebuild the kept cluster pairs when sigma changed or every `rebuild_every`
// steps at a fixed sigma; then the four instances walk their blocks' column lists.
void Multiscale::before_fine_step(Solver &s, double sigma) {
    if (sigma == mask_sigma && steps_since_mask < rebuild_every) {
        ++steps_since_mask;
        return;
    }
    mask_sigma = sigma;
    steps_since_mask = 1;
    cudaStream_t st = s.st;
    Workspace &ws = *s.ws;
    const int D = s.D, stride = s.X.stride;
    const float eps = (float)s.eps_of(sigma);
    const int c = s.cur;
    // cluster maxima of the current duals
    float4 *mx = ws.get<float4>("ms:maxx", ncl_x);
    float4 *my = ws.get<float4>("ms:maxy", ncl_y);
    const float *lwx = D <= 3 ? s.X.pts + 3 : s.X.logw, *lwy = D <= 3 ? s.Y.pts + 3 : s.Y.logw;
    const int lws = D <= 3 ? 4 : 1;
    cluster_max_kernel<<<ncl_x, 128, 0, st>>>(d_off_x, ncl_x, s.pa[c], s.pf[c], lwx, lws, eps, mx);
    OTGB_CHECK_LAUNCH();
    cluster_max_kernel<<<ncl_y, 128, 0, st>>>(d_off_y, ncl_y, s.pb[c], s.pg[c], lwy, lws, eps, my);
    OTGB_CHECK_LAUNCH();
    // keep bits per instance; x-side maxima: (a, f, eps log a + a, eps log a + f),
    // y-side: (b, g, eps log b + b, eps log b + g)
    const int ncmax = std::max(ncl_x, ncl_y);
    const int nwords = (ncmax + 31) / 32;
    MaskLaunch M;
    std::memset(&M, 0, sizeof(M));
    M.D = D;
    M.stride = stride;
    M.nwords = nwords;
    M.eps = eps;
    M.tau = (float)tau;
    M.p1 = s.p == 1 ? 1 : 0;
    const float inv_lam = (float)(1.0 / s.lam_of(sigma));
    unsigned *bits = ws.get<unsigned>("ms:bits", (size_t)4 * ncmax * nwords);
    // inst 0: rows x, cols x (a); 1: rows y, cols y (b); 2: rows y, cols x (g from f); 3: rows x, cols y (f from g)
    const float *cr[4] = {cen_x, cen_y, cen_y, cen_x}, *cc[4] = {cen_x, cen_y, cen_x, cen_y};
    const float *rr[4] = {rad_x, rad_y, rad_y, rad_x}, *rc[4] = {rad_x, rad_y, rad_x, rad_y};
    const float4 *mr[4] = {mx, my, my, mx}, *mc[4] = {mx, my, mx, my};
    const int rsel[4] = {0, 0, 1, 1}, csel[4] = {2, 2, 3, 3};
    const int nr[4] = {ncl_x, ncl_y, ncl_y, ncl_x}, nc[4] = {ncl_x, ncl_y, ncl_x, ncl_y};
    for (int q = 0; q < 4; ++q) {
        MaskInst &I = M.inst[q];
        I.cen_r = cr[q]; I.cen_c = cc[q]; I.rad_r = rr[q]; I.rad_c = rc[q];
        I.max_r = mr[q]; I.max_c = mc[q]; I.row_sel = rsel[q]; I.col_sel = csel[q];
        I.ncl_r = nr[q]; I.ncl_c = nc[q]; I.inv_lam = inv_lam;
        I.bits = bits + (size_t)q * ncmax * nwords;
    }
    mask_kernel<<<dim3(ncmax, 4), 256, 0, st>>>(M);
    OTGB_CHECK_LAUNCH();
    if (s.launch.use_tcc) {
        require(nwords == s.launch.tcc_nwords, "before_fine_step: keep-bit words changed", OTGB_EINTERNAL);
        for (int q = 0; q < 4; ++q) s.launch.inst[q].tcc_bits = M.inst[q].bits;
    }
    // column lists per (instance, block): count, host prefix, write
    ListLaunch LL;
    std::memset(&LL, 0, sizeof(LL));
    const int nb[4] = {s.nblk_x, s.nblk_y, s.nblk_y, s.nblk_x};
    const int *bcl[4] = {d_clx, d_cly, d_cly, d_clx};
    const int *offc[4] = {d_off_x, d_off_y, d_off_x, d_off_y};
    LL.base[0] = 0;
    for (int q = 0; q < 4; ++q) {
        LL.inst[q].bits = M.inst[q].bits;
        LL.inst[q].blk_cl = bcl[q];
        LL.inst[q].off_c = offc[q];
        LL.inst[q].nblk = nb[q];
        LL.base[q + 1] = LL.base[q] + nb[q];
    }
    LL.nwords = nwords;
    const int nflat = LL.base[4];
    LL.counts = ws.get<int>("ms:cnt", 2 * (size_t)nflat);
    list_kernel<false><<<nflat, 256, 0, st>>>(LL);
    OTGB_CHECK_LAUNCH();
    std::vector<int> cq(2 * (size_t)nflat), cnt(nflat), ptr(nflat + 1);
    OTGB_CUDA_TRY(cudaMemcpyAsync(cq.data(), LL.counts, sizeof(int) * 2 * nflat, cudaMemcpyDeviceToHost, st));
    OTGB_CUDA_TRY(cudaStreamSynchronize(st));
    // range entries per block: one per run of kept clusters, then a sentinel; kRngPad padding entries after the
    // last block keep every entry the walk reads past a sentinel readable
    ptr[0] = 0;
    for (int f = 0; f < nflat; ++f) {
        cnt[f] = cq[2 * f];
        ptr[f + 1] = ptr[f] + cq[2 * f + 1] + 1;
    }
    int *d_ptr = ws.get<int>("ms:rngptr", nflat + 1);
    OTGB_CUDA_TRY(cudaMemcpyAsync(d_ptr, ptr.data(), sizeof(int) * (nflat + 1), cudaMemcpyHostToDevice, st));
    int2 *d_rng = ws.get<int2>("ms:rng", (size_t)ptr[nflat] + kRngPad);
    OTGB_CUDA_TRY(cudaMemsetAsync(d_rng + ptr[nflat], 0, sizeof(int2) * kRngPad, st));
    LL.rng_ptr = d_ptr;
    LL.rng = d_rng;
    list_kernel<true><<<nflat, 256, 0, st>>>(LL);
    OTGB_CHECK_LAUNCH();
    // instances walk the ranges; work items split long sequences of kept columns
    std::vector<std::vector<int>> ncols(4);
    double kept = 0.0, dense = 0.0;
    for (int q = 0; q < 4; ++q) {
        SoftminInst &I = s.launch.inst[q];
        I.rng_ptr = d_ptr + LL.base[q];
        I.col_rng = d_rng;
        ncols[q].assign(cnt.begin() + LL.base[q], cnt.begin() + LL.base[q + 1]);
        const std::vector<int> &hb = (q == 0 || q == 3) ? hbx : hby;
        for (int bl = 0; bl < nb[q]; ++bl) kept += (double)cnt[LL.base[q] + bl] * (hb[bl + 1] - hb[bl]);
        dense += (double)I.n_rows * I.n_cols;
    }
    last_kept_fraction = dense > 0 ? kept / dense : 1.0;
    s.set_work(ncols, D <= 3 && s.p == 2);
}

void Multiscale::setup_tcc(Solver &s) {
    const int D4 = s.X.stride;
    const int nwords = (std::max(ncl_x, ncl_y) + 31) / 32;
    s.launch.use_tcc = 0;
    if (!s.use_tc || s.D <= 3 || D4 > 60 || nwords > kTccMaxWords) return;
    cudaStream_t st = s.st;
    Workspace &ws = *s.ws;
    struct Side {
        int *tile0, *tile_cl;
        int ntiles;
        unsigned char *copy[2];
        float *half_norm;
    } side[2];
    const std::vector<int> *offs[2] = {&s.X_off, &s.Y_off};
    const char *tag[2] = {"x", "y"};
    for (int k = 0; k < 2; ++k) {
        const std::vector<int> &off = *offs[k];
        const int ncl = (int)off.size() - 1;
        std::vector<int> t0(ncl + 1), tcl;
        t0[0] = 0;
        for (int J = 0; J < ncl; ++J) {
            const int nt = (off[J + 1] - off[J] + 127) / 128;
            for (int q = 0; q < nt; ++q) tcl.push_back(J);
            t0[J + 1] = t0[J] + nt;
        }
        Side &S = side[k];
        S.ntiles = t0[ncl];
        S.tile0 = ws.get<int>(std::string("tcc:t0") + tag[k], ncl + 1);
        S.tile_cl = ws.get<int>(std::string("tcc:tcl") + tag[k], std::max(S.ntiles, 1));
        OTGB_CUDA_TRY(cudaMemcpyAsync(S.tile0, t0.data(), sizeof(int) * (ncl + 1), cudaMemcpyHostToDevice, st));
        if (S.ntiles)
            OTGB_CUDA_TRY(cudaMemcpyAsync(S.tile_cl, tcl.data(), sizeof(int) * S.ntiles, cudaMemcpyHostToDevice, st));
        const size_t bytes = (size_t)std::max(S.ntiles, 1) * tcc_tile_bytes();
        S.copy[0] = static_cast<unsigned char *>(ws.get(std::string("tcc:tiles0") + tag[k], bytes));
        S.copy[1] = static_cast<unsigned char *>(ws.get(std::string("tcc:tiles1") + tag[k], bytes));
        S.half_norm = ws.get<float>(std::string("tcc:hn") + tag[k], (size_t)std::max(S.ntiles, 1) * 128);
        tcc_build_side(k == 0 ? s.X.pts : s.Y.pts, D4, k == 0 ? d_off_x : d_off_y, S.tile0, S.tile_cl, S.ntiles,
                       k == 0 ? cen_x : cen_y, S.copy[0], S.copy[1], S.half_norm, st);
        OTGB_CUDA_TRY(cudaStreamSynchronize(st));  // host vectors go out of scope
    }
    // instance 0: rows x, cols x; 1: rows y, cols y; 2: rows y, cols x; 3: rows x, cols y
    const int colside[4] = {0, 1, 0, 1}, copy[4] = {0, 0, 1, 1};
    const int *blk_cl[4] = {d_clx, d_cly, d_cly, d_clx};
    for (int q = 0; q < 4; ++q) {
        SoftminInst &I = s.launch.inst[q];
        const Side &S = side[colside[q]];
        I.tcc_tiles = S.copy[copy[q]];
        I.tcc_half_norm = S.half_norm;
        I.tcc_tile0 = S.tile0;
        I.tcc_tile_cl = S.tile_cl;
        I.tcc_ntiles = S.ntiles;
        I.tcc_coff = colside[q] == 0 ? d_off_x : d_off_y;
        I.tcc_ccen = colside[q] == 0 ? cen_x : cen_y;
        I.tcc_bits = nullptr;  // set with every new mask
        I.tcc_blk_cl = blk_cl[q];
    }
    s.launch.tcc_nwords = nwords;
    s.launch.use_tcc = 1;
}

}  // namespace otgb
