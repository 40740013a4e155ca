// sinkhorn_divergence and otgb_softmin: the eps-scaled, symmetric, averaged
// Sinkhorn loop of the Algorithm in Section 2, with the debiased divergence of
// Eq. (5) returned through its dual form Eq. (6).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <memory>

#include "kmeans.cuh"
#include "multiscale.cuh"
#include "prims.cuh"
#include "solver.cuh"

namespace otgb {

bool trace_enabled() {
    static int v = -1;
    if (v < 0) {
        const char *e = std::getenv("OTGB_TRACE");
        v = (e && e[0] == '1') ? 1 : 0;
    }
    return v == 1;
}

namespace {

// Pinned mailbox layout (bytes).
constexpr size_t kMbBad = 0, kMbMass = 64, kMbBox = 64 + 128 * 8, kMbS = kMbBox + 4 * 64 * 4, kMbDelta = kMbS + 16;

struct DeviceChecks {
    int bad = 0;
    double mass_a = 0.0, mass_b = 0.0;
    std::vector<float> lox, hix, loy, hiy;
};

DeviceChecks validate_and_bound(otgb_ctx *ctx, const float *x, const float *a, int N, const float *y,
                                const float *b, int M, int D) {
    cudaStream_t st = ctx_stream(ctx);
    Workspace &ws = ctx_ws(ctx);
    int *bad = ws.get<int>("bad", 4);
    double *mpart = ws.get<double>("mpart", 128);
    float *box = ws.get<float>("box", 4 * 64);
    float *bpart = ws.get<float>("bpart", 64 * 2 * 64);
    OTGB_CUDA_TRY(cudaMemsetAsync(bad, 0, sizeof(int), st));
    check_weights(a, N, bad, mpart, st);
    check_weights(b, M, bad, mpart + 64, st);
    check_points(x, (size_t)N * D, bad, st);
    check_points(y, (size_t)M * D, bad, st);
    bbox(x, N, D, D, box, box + 64, bpart, st);
    bbox(y, M, D, D, box + 128, box + 192, bpart, st);
    char *mb = static_cast<char *>(ctx_pinned(ctx));
    OTGB_CUDA_TRY(cudaMemcpyAsync(mb + kMbBad, bad, sizeof(int), cudaMemcpyDeviceToHost, st));
    OTGB_CUDA_TRY(cudaMemcpyAsync(mb + kMbMass, mpart, 128 * sizeof(double), cudaMemcpyDeviceToHost, st));
    OTGB_CUDA_TRY(cudaMemcpyAsync(mb + kMbBox, box, 4 * 64 * sizeof(float), cudaMemcpyDeviceToHost, st));
    OTGB_CUDA_TRY(cudaStreamSynchronize(st));
    DeviceChecks c;
    c.bad = *reinterpret_cast<int *>(mb + kMbBad);
    const double *mp = reinterpret_cast<const double *>(mb + kMbMass);
    for (int k = 0; k < 64; ++k) { c.mass_a += mp[k]; c.mass_b += mp[64 + k]; }
    const float *bx = reinterpret_cast<const float *>(mb + kMbBox);
    c.lox.assign(bx, bx + D);
    c.hix.assign(bx + 64, bx + 64 + D);
    c.loy.assign(bx + 128, bx + 128 + D);
    c.hiy.assign(bx + 192, bx + 192 + D);
    return c;
}

// Morton-sort positions of a D <= 3 cloud on a grid of about n/4 cells, for
// spatially compact row blocks.  Returns perm (device) of n ints.
int *spatial_sort(otgb_ctx *ctx, const std::string &tag, const float *x, int n, int D, const std::vector<float> &lo,
                  const std::vector<float> &hi, float *d_lo) {
    cudaStream_t st = ctx_stream(ctx);
    Workspace &ws = ctx_ws(ctx);
    float ext = 0.f;
    for (int d = 0; d < D; ++d) ext = std::max(ext, hi[d] - lo[d]);
    int per_axis = (int)std::ceil(std::cbrt((double)n / 4.0));
    per_axis = std::max(1, std::min(per_axis, 512));
    float cell = ext > 0.f ? ext / (float)per_axis * 1.0001f : 1.0f;
    uint32_t *keys = ws.get<uint32_t>(tag + ":keys", n);
    int *perm = ws.get<int>(tag + ":perm", n);
    int *bad = ws.get<int>("bad", 4);
    grid_keys(x, n, D, D, d_lo, cell, keys, bad, st);
    int bits = 0;
    while ((1 << bits) < per_axis + 1) ++bits;
    void *scr = ws.get("sort:scratch", radix_sort_scratch_bytes(n));
    radix_sort_pairs(keys, perm, n, 3 * bits, scr, st);
    return perm;
}

// The bounded-wait error path, exercised on purpose (params.debug_wait_probe):
// one thread polls a device word that nothing writes, pausing between polls,
// and gives up after `polls` polls by flagging the error word that the
// tensor-core and tile waits flag when they give up.
__global__ void wait_probe_kernel(const volatile unsigned *flag, unsigned *err, int polls) {
    if (threadIdx.x != 0) return;
    for (int k = 0; k < polls; ++k) {
        if (*flag) return;
        __nanosleep(1000);
    }
    atomicOr(err, 4u);
}

}  // namespace

// One averaged step of the four instances at temperature eps.
void Solver::step(double sigma, bool count_pairs) {
    const double eps = eps_of(sigma);
    SoftminLaunch &L = launch;
    L.eps = (float)eps;
    L.s = (float)(1.4426950408889634 / eps);
    L.eps_ln2 = eps * 0.69314718055994530942;
    const float lam = (float)lam_of(sigma);
    const int c = cur, n = cur ^ 1;
    // alpha <-> alpha: a~ on x from (x, alpha, a)
    L.inst[0].col_pot = pa[c]; L.inst[0].row_old = pa[c]; L.inst[0].row_out = pa[n];
    // beta <-> beta: b~ on y from (y, beta, b)
    L.inst[1].col_pot = pb[c]; L.inst[1].row_old = pb[c]; L.inst[1].row_out = pb[n];
    // alpha -> beta: g~ on y from (x, alpha, f)
    L.inst[2].col_pot = pf[c]; L.inst[2].row_old = pg[c]; L.inst[2].row_out = pg[n];
    // beta -> alpha: f~ on x from (y, beta, g)
    L.inst[3].col_pot = pg[c]; L.inst[3].row_old = pf[c]; L.inst[3].row_out = pf[n];
    for (int k = 0; k < 4; ++k) { L.inst[k].lam = lam; L.inst[k].omega = 0.5f; }
    L.pairs = count_pairs ? d_pairs : nullptr;
    OTGB_CUDA_TRY(cudaMemsetAsync(L.delta_max, 0, sizeof(unsigned), st));
    if (timing && ev_used == kEvPool) {  // pool full: wait for the oldest window, then reuse it
        OTGB_CUDA_TRY(cudaEventSynchronize(ev_pool[2 * kEvPool - 1]));
        harvest_timing();
    }
    if (timing) OTGB_CUDA_TRY(cudaEventRecord(ev_pool[2 * ev_used], st));
    if (L.use_tcc) tcc_update(L, st);
    softmin_run(L, D, rows_per_thread, st);
    if (timing) {
        OTGB_CUDA_TRY(cudaEventRecord(ev_pool[2 * ev_used + 1], st));
        ++ev_used;
    }
    cur = n;
    ++steps;
}

void Solver::harvest_timing() {
    if (!timing) return;
    for (int k = 0; k < ev_used; ++k) {
        float ms = 0.f;
        OTGB_CUDA_TRY(cudaEventElapsedTime(&ms, ev_pool[2 * k], ev_pool[2 * k + 1]));
        softmin_ms += ms;
        ++softmin_launches;
    }
    ev_used = 0;
}

double Solver::divergence(double eps) {
    double *dS = ws->get<double>(nm("S"), 1);
    double *dpart = ws->get<double>(nm("Spart"), 128);
    unsigned *dmax = ws->get<unsigned>(nm("potmax"), 1);
    divergence_sum(X.w, pf[cur], pa[cur], X.n, Y.w, pg[cur], pb[cur], Y.n, eps, rho, dS, dpart, st);
    OTGB_CUDA_TRY(cudaMemsetAsync(dmax, 0, sizeof(unsigned), st));
    absmax(pf[cur], X.n, dmax, st);
    absmax(pa[cur], X.n, dmax, st);
    absmax(pg[cur], Y.n, dmax, st);
    absmax(pb[cur], Y.n, dmax, st);
    char *mb = static_cast<char *>(ctx_pinned(ctx));
    OTGB_CUDA_TRY(cudaMemcpyAsync(mb + kMbS, dS, sizeof(double), cudaMemcpyDeviceToHost, st));
    OTGB_CUDA_TRY(cudaMemcpyAsync(mb + kMbDelta, launch.delta_max, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
    OTGB_CUDA_TRY(cudaMemcpyAsync(mb + kMbDelta + 4, dmax, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
    OTGB_CUDA_TRY(cudaStreamSynchronize(st));
    harvest_timing();
    float df, pm;
    std::memcpy(&df, mb + kMbDelta, sizeof(float));
    std::memcpy(&pm, mb + kMbDelta + 4, sizeof(float));
    last_delta = df;
    last_potmax = pm;
    return *reinterpret_cast<double *>(mb + kMbS);
}

// Row blocks: rows [start[k], start[k+1]).  Uniform blocks of block_rows rows,
// or, when cluster offsets are given, blocks that never straddle two clusters
// (a cluster larger than block_rows is split), so that every block is
// spatially compact.
std::vector<int> make_row_blocks(int n, int block_rows, const std::vector<int> *offsets) {
    std::vector<int> b;
    if (!offsets) {
        for (int r = 0; r < n; r += block_rows) b.push_back(r);
    } else {
        for (size_t k = 0; k + 1 < offsets->size(); ++k)
            for (int r = (*offsets)[k]; r < (*offsets)[k + 1]; r += block_rows) b.push_back(r);
    }
    b.push_back(n);
    return b;
}

void Solver::setup_instances(const std::vector<int> &hx, const std::vector<int> &hy) {
    int *bx = ws->get<int>(nm("blk:x"), hx.size());
    int *by = ws->get<int>(nm("blk:y"), hy.size());
    OTGB_CUDA_TRY(cudaMemcpyAsync(bx, hx.data(), hx.size() * sizeof(int), cudaMemcpyHostToDevice, st));
    OTGB_CUDA_TRY(cudaMemcpyAsync(by, hy.data(), hy.size() * sizeof(int), cudaMemcpyHostToDevice, st));
    SoftminLaunch &L = launch;
    L.n_inst = 4;
    const Cloud *rows[4] = {&X, &Y, &Y, &X}, *cols[4] = {&X, &Y, &X, &Y};
    const int rows_x[4] = {1, 0, 0, 1};  // instances 0 and 3 have x rows
    for (int k = 0; k < 4; ++k) {
        SoftminInst &I = L.inst[k];
        I.rows = rows[k]->pts;
        I.cols = cols[k]->pts;
        I.col_logw = cols[k]->logw;
        I.n_rows = rows[k]->n;
        I.n_cols = cols[k]->n;
        I.blk_row0 = rows_x[k] ? bx : by;
        I.rng_ptr = nullptr;
        I.col_rng = nullptr;
    }
    nblk_x = (int)hx.size() - 1;
    nblk_y = (int)hy.size() - 1;
}

void Solver::setup_dense_instances(int block_rows) {
    std::vector<int> hx = make_row_blocks(X.n, block_rows, X_off.empty() ? nullptr : &X_off);
    std::vector<int> hy = make_row_blocks(Y.n, block_rows, Y_off.empty() ? nullptr : &Y_off);
    setup_instances(hx, hy);
    std::vector<std::vector<int>> ncols(4);
    const int rows_x[4] = {1, 0, 0, 1};
    for (int k = 0; k < 4; ++k) ncols[k].assign(rows_x[k] ? nblk_x : nblk_y, launch.inst[k].n_cols);
    set_work(ncols, D <= 3 && p == 2);
}

// Items (inst, blk, cb, ce): a block's columns are cut into chunks of CH
// positions, CH chosen so that the launch has about three waves of items
// (D <= 3: one item per warp, 6 CTAs of 4 warps resident per SM); every block
// of a split launch goes through the finalize pass, which sums its items'
// partial sums in item order.
void Solver::set_work(const std::vector<std::vector<int>> &ncols, bool allow_split) {
    const int sms = ctx_sm_count(ctx);
    double W = 0.0;
    for (auto &v : ncols)
        for (int c : v) W += c;
#ifndef OTGB_TC3_ITEMS_PER_SM
#define OTGB_TC3_ITEMS_PER_SM 10.0
#endif
    // D <= 3 warp kernel: about three waves of warps (6 CTAs of 4 warps per SM);
    // tensor-core form: one CTA per item, fewer and longer items
    const double target = use_tc3 ? OTGB_TC3_ITEMS_PER_SM * sms : 3.0 * 5.0 * 4.0 * sms;
    int CH = 1 << 30;
    if (allow_split) {
        CH = (int)std::ceil(W / target);
        CH = std::max(512, (CH + 127) / 128 * 128);
    }
    std::vector<int4> items, fin;
    std::vector<int> item_fin;
    for (int k = 0; k < (int)ncols.size(); ++k)
        for (int b = 0; b < (int)ncols[k].size(); ++b) {
            const int n = ncols[k][b];
            const int first = (int)items.size();
            if (n <= CH) items.push_back(make_int4(k, b, 0, n));
            else
                for (int c = 0; c < n; c += CH) items.push_back(make_int4(k, b, c, std::min(n, c + CH)));
            item_fin.resize(items.size(), (int)fin.size());
            fin.push_back(make_int4(k, b, first, (int)items.size() - first));
        }
    const bool split = items.size() > fin.size();
    // Without split blocks the items go longest first (the hardware hands out
    // CTAs in index order), so that the last wave holds the short items.
    if (!split)
        std::stable_sort(items.begin(), items.end(),
                         [](const int4 &p, const int4 &q) { return p.w - p.z > q.w - q.z; });
    work_ncols = ncols;
    int4 *d_items = ws->get<int4>(nm("items"), items.size() + 1);
    OTGB_CUDA_TRY(cudaMemcpyAsync(d_items, items.data(), items.size() * sizeof(int4), cudaMemcpyHostToDevice, st));
    launch.items = d_items;
    launch.n_items = (int)items.size();
    launch.part = nullptr;
    launch.fin = nullptr;
    launch.n_fin = 0;
    launch.item_fin = nullptr;
    launch.fin_count = nullptr;
    if (split) {
        int4 *d_fin = ws->get<int4>(nm("fin"), fin.size() + 1);
        OTGB_CUDA_TRY(cudaMemcpyAsync(d_fin, fin.data(), fin.size() * sizeof(int4), cudaMemcpyHostToDevice, st));
        launch.part = ws->get<float>(nm("part"), items.size() * (size_t)kPartRows);
        launch.fin = d_fin;
        launch.n_fin = (int)fin.size();
        int *d_ifin = ws->get<int>(nm("itemfin"), items.size() + 1);
        OTGB_CUDA_TRY(cudaMemcpyAsync(d_ifin, item_fin.data(), item_fin.size() * sizeof(int), cudaMemcpyHostToDevice, st));
        launch.item_fin = d_ifin;
        launch.fin_count = ws->get<int>(nm("fincnt"), fin.size() + 1);
    }
    OTGB_CUDA_TRY(cudaStreamSynchronize(st));  // host vectors go out of scope
}

void Solver::alloc_common() {
    launch = SoftminLaunch();
    launch.delta_max = ws->get<unsigned>(nm("delta"), 1);
    const int cap = 2 * (X.n + Y.n) + 64;
    launch.fallback = ws->get<int4>(nm("fb"), cap);
    launch.n_fallback = ws->get<int>(nm("nfb"), 1);
    launch.work_counter = ws->get<int>(nm("wctr"), 1);
    launch.fallback_cap = cap;
    d_fb_total = ws->get<unsigned long long>(nm("fbtot"), 1);
    launch.fallback_total = d_fb_total;
    d_pairs = ws->get<unsigned long long>(nm("pairs"), 1);
    launch.tc_err = ws->get<unsigned>(nm("tcerr"), 1);
    OTGB_CUDA_TRY(cudaMemsetAsync(launch.tc_err, 0, sizeof(unsigned), st));
    launch.use_tc = use_tc ? 1 : 0;
    launch.use_tc3 = use_tc3 ? 1 : 0;
    launch.cost_p1 = p == 1 ? 1 : 0;
    OTGB_CUDA_TRY(cudaMemsetAsync(d_fb_total, 0, sizeof(unsigned long long), st));
    OTGB_CUDA_TRY(cudaMemsetAsync(d_pairs, 0, sizeof(unsigned long long), st));
    if (timing && ev_pool.empty()) {
        ev_pool.resize(2 * kEvPool);
        for (auto &e : ev_pool) OTGB_CUDA_TRY(cudaEventCreate(&e));
    }
}

Solver::~Solver() {
    for (auto &e : ev_pool)
        if (e) cudaEventDestroy(e);
}

void Solver::alloc_pots(const otgb_params &P) {
    for (int k = 0; k < 2; ++k) {
        Z[k] = ws->get<float>(nm("Z" + std::to_string(k)), 2 * (size_t)X.n + 2 * (size_t)Y.n);
        pa[k] = Z[k];
        pf[k] = Z[k] + X.n;
        pb[k] = Z[k] + 2 * (size_t)X.n;
        pg[k] = Z[k] + 2 * (size_t)X.n + Y.n;
    }
    cur = 0;
    auto init = [&](float *dst, const float *src, const int *perm, int n) {
        if (src) permute(src, perm, n, dst, st);
        else OTGB_CUDA_TRY(cudaMemsetAsync(dst, 0, sizeof(float) * n, st));
    };
    init(pa[0], P.a_init, X.perm, X.n);
    init(pf[0], P.f_init, X.perm, X.n);
    init(pb[0], P.b_init, Y.perm, Y.n);
    init(pg[0], P.g_init, Y.perm, Y.n);
}

// Stopping rule at sigma = blur, evaluated every `check_every` steps.  Both S
// and the potentials converge geometrically; the remaining change of each is
// estimated as the tail of a geometric sequence, d r / (1 - r), from its last
// increment d and the contraction r seen between checks:
//  - S: d = S_k - S_{k-1}, r = d / (S_{k-1} - S_{k-2});
//  - potentials: d = max |new - old| of the last step, r = (d_k / d_{k-1})^(1/m)
//    per step (m steps between checks).
// S can settle long before the potentials (it is insensitive to the slow
// translation mode (f + c, g - c)), so both tails must be small:
//   S tail <= tol |S| + floor,   potential tail <= max(tol, 1e-6) (max|pot| + eps).
// At the float32 floor the step no longer contracts: two checks in a row
// whose step is at most two units in the last place of the largest dual, or
// three checks without a new smallest step while the step is below
// 1e-5 (max|pot| + eps), count as converged.
bool Solver::converged(const std::vector<double> &hist, double tol, double floor_abs, double *rem_out) {
    const size_t k = hist.size();
    if (k < 3) return false;
    const double d1 = hist[k - 1] - hist[k - 2], d0 = hist[k - 2] - hist[k - 3];
    const double Sa = std::fabs(hist[k - 1]);
    double rem = std::fabs(d1);
    if (d0 != 0.0) {
        const double r = d1 / d0;
        if (r > 0.0 && r < 1.0) rem = std::fabs(d1) * r / (1.0 - r);
    }
    if (rem_out) *rem_out = rem / std::max(Sa, 1e-300);
    // two successive increments at the float32 rounding level of S also satisfy the S rule
    if (std::fabs(d1) <= 1e-7 * Sa && std::fabs(d0) <= 1e-7 * Sa) return true;
    return rem <= tol * Sa + floor_abs;
}

bool Solver::potentials_converged(double delta_prev, double delta, int m, double eps, double potmax,
                                  double tol) {
    // delta is in units of eps
    const double scale = potmax + eps;
    const double tol_pot = std::max(tol, 1e-6) * scale;
    if (!(delta_prev > 0.0) || m <= 0) return false;
    // progress = a new smallest step (by at least 1 %) since the last check
    if (delta < 0.99 * delta_best) {
        delta_best = delta;
        no_progress = 0;
    } else {
        ++no_progress;
    }
    const double r = std::pow(delta / delta_prev, 1.0 / m);
    if (r < 0.999 && delta * eps * r / (1.0 - r) <= tol_pot) return true;  // geometric tail
    // the float32 floor: a step of at most two units in the last place of the
    // largest dual can only move the duals by rounding, so two such windows in a
    // row end the loop
    const float pm = (float)potmax;
    const double ulp = (double)(std::nextafter(pm, INFINITY) - pm);
    floor_hits = (delta * eps <= 2.0 * ulp) ? floor_hits + 1 : 0;
    if (floor_hits >= 2) return true;
    // three windows without a new smallest step: the float32 rounding floor of
    // the duals; accept when the step itself is small
    return no_progress >= 3 && delta * eps <= 1e-5 * scale;
}

int Solver::iterate_at_blur(const otgb_params &P, int it_budget) {
    const double eps = eps_of(P.blur);
    if (P.fixed_iters > 0) {
        for (int k = 0; k < P.fixed_iters && steps < P.max_iters; ++k) fine_step(P.blur);
        S = divergence(eps);
        return OTGB_OK;
    }
    std::vector<double> hist;
    const int every = std::max(1, std::min(P.check_every, kEvPool));
    int at_blur = 0;
    double delta_prev = -1.0;
    if (P.anderson > 0) {
        aa.init(*ws, tag, 2 * X.n + 2 * Y.n, P.anderson, st);
        aa_active = true;
    }
    for (;;) {
        int m = 0;
        for (int k = 0; k < every && steps < P.max_iters; ++k, ++at_blur, ++m) fine_step(P.blur);
        S = divergence(eps);
        if (!std::isfinite(S) || !std::isfinite(last_delta)) return OTGB_ENONFINITE;
        hist.push_back(S);
        double rem = 0.0;
        const bool ok_s = converged(hist, P.tol, 1e-12 * eps * (X.mass + Y.mass), &rem);
        const bool ok_p = potentials_converged(delta_prev, last_delta, m, eps, last_potmax, P.tol);
        if (trace_enabled())
            std::fprintf(stderr, "otgb: step %d S %.12g rem %.3g delta %.3g potmax %.4g ok_s %d ok_p %d\n", steps, S,
                         rem, last_delta, last_potmax, (int)ok_s, (int)ok_p);
        delta_prev = last_delta;
        last_rel = rem;
        if (ok_s && ok_p && at_blur >= P.min_iters) return OTGB_OK;
        if (steps >= P.max_iters) return OTGB_ENOCONV;
        (void)it_budget;
    }
}

// One sweep of the alpha -> beta instance with no old value: g_j = -lam eps
// LSE_i(log alpha_i + (f_i - C(x_i, y_j)) / eps), over the kept columns of the
// current work (all columns when dense).
void Solver::sweep_g(double sigma) {
    const double eps = eps_of(sigma);
    SoftminLaunch E = launch;
    E.eps = (float)eps;
    E.s = (float)(1.4426950408889634 / eps);
    E.eps_ln2 = eps * 0.69314718055994530942;
    SoftminInst &I = E.inst[2];
    I.col_pot = pf[cur];
    I.row_old = nullptr;
    I.row_out = pg[cur];
    I.lam = (float)lam_of(sigma);
    I.omega = 1.0f;
    require(work_ncols.size() == 4, "sweep_g: no work decomposition", OTGB_EINTERNAL);
    std::vector<int4> items;
    for (int bl = 0; bl < (int)work_ncols[2].size(); ++bl) items.push_back(make_int4(2, bl, 0, work_ncols[2][bl]));
    int4 *d_items = ws->get<int4>(nm("gitems"), items.size() + 1);
    OTGB_CUDA_TRY(cudaMemcpyAsync(d_items, items.data(), items.size() * sizeof(int4), cudaMemcpyHostToDevice, st));
    E.items = d_items;
    E.n_items = (int)items.size();
    E.part = nullptr;
    E.fin = nullptr;
    E.n_fin = 0;
    E.delta_max = nullptr;
    E.pairs = d_pairs;
    softmin_run(E, D, rows_per_thread, st);
    OTGB_CUDA_TRY(cudaStreamSynchronize(st));  // the host item list goes out of scope
    ++steps;
}

void Solver::fine_step(double sigma) {
    if (g_from_f) {
        g_from_f = false;
        if (ms) ms->before_fine_step(*this, sigma);
        sweep_g(sigma);
        if (ms) ms->mask_sigma = -1.0;  // decide the kept pairs again with this g
    }
    if (ms) ms->before_fine_step(*this, sigma);
    step(sigma, true);
    ++fine_steps;
    if (translation && !std::isinf(rho)) {
        double2 *part = ws->get<double2>(nm("tpart"), 64);
        translate_duals(X.w, pf[cur], X.n, Y.w, pg[cur], Y.n, rho, part, nullptr, st);
    }
    if (aa_active) aa.step(Z[cur ^ 1], Z[cur], st);
}

}  // namespace otgb

using namespace otgb;

int otgb::solve_divergence(otgb_ctx *ctx, const float *x, const float *a, int N, const float *y, const float *b,
                           int M, int D, const otgb_params *params, double *cost_host, float *f, float *g,
                           float *a_self, float *b_self, otgb_plan **plan_out, otgb_stats *stats,
                           const GradRequest *gr) {
    if (!ctx) return fail(nullptr, Error{OTGB_EINVAL, "sinkhorn_divergence: null context"});
    try {
        ctx_set_device(ctx);
        otgb_params P;
        if (params) P = *params;
        else otgb_default_params(&P);
        require(x && a && y && b && cost_host && f && g, "sinkhorn_divergence: null pointer argument");
        require(N >= 1 && M >= 1, "sinkhorn_divergence: N and M must be >= 1");
        require(D >= 1 && D <= 64, "sinkhorn_divergence: D must be in [1, 64]");
        require(P.p == 1 || P.p == 2, "sinkhorn_divergence: p must be 1 or 2");
        require(P.blur > 0.0 && std::isfinite(P.blur), "sinkhorn_divergence: blur must be > 0");
        require(P.scaling > 0.0 && P.scaling < 1.0, "sinkhorn_divergence: scaling must be in (0, 1)");
        require(P.max_iters >= 1, "sinkhorn_divergence: max_iters must be >= 1");
        require(P.precision == OTGB_FP32 || P.precision == OTGB_FP32_SIMT ||
                    (P.precision == OTGB_TC_BF16X3 && D >= 16 && P.p == 2),
                "sinkhorn_divergence: precision must be FP32, FP32_SIMT, or TC_BF16X3 with D >= 16 and p = 2");
        if (plan_out) *plan_out = nullptr;

        Solver s;
        s.ctx = ctx;
        s.st = ctx_stream(ctx);
        s.ws = &ctx_ws(ctx);
        s.D = D;
        s.p = P.p;
        s.reach = P.reach;
        s.rho = (!(P.reach > 0.0) || std::isinf(P.reach)) ? INFINITY : std::pow(P.reach, (double)P.p);
        s.timing = stats != nullptr;
        s.translation = P.translation != 0;
        s.use_tc = P.precision == OTGB_TC_BF16X3 && D >= 16 && P.p == 2;
        s.use_tc3 = P.precision == OTGB_FP32 && D <= 3 && P.p == 2;
        cudaStream_t st = s.st;
        OTGB_CUDA_TRY(cudaEventRecord(ctx_event(ctx, 0), st));

        DeviceChecks chk = validate_and_bound(ctx, x, a, N, y, b, M, D);
        require(!(chk.bad & 1), "sinkhorn_divergence: weights must be finite and >= 0");
        require(!(chk.bad & 2), "sinkhorn_divergence: points must be finite");
        require(chk.mass_a > 0.0 && chk.mass_b > 0.0, "sinkhorn_divergence: total masses must be > 0");

        // common centre and diameter (bounding-box diagonal of x and y)
        std::vector<float> cen(64, 0.f);
        double diag2 = 0.0;
        for (int d = 0; d < D; ++d) {
            const float lo = std::min(chk.lox[d], chk.loy[d]), hi = std::max(chk.hix[d], chk.hiy[d]);
            cen[d] = 0.5f * (lo + hi);
            diag2 += ((double)hi - lo) * ((double)hi - lo);
        }
        const double diameter = P.diameter > 0.0 ? P.diameter : std::sqrt(diag2);
        float *d_cen = s.ws->get<float>("cen", 64);
        float *d_box = s.ws->get<float>("box", 4 * 64);
        OTGB_CUDA_TRY(cudaMemcpyAsync(d_cen, cen.data(), 64 * sizeof(float), cudaMemcpyHostToDevice, st));

        const int stride = D <= 3 ? 4 : ((D + 3) & ~3);
        s.X.n = N; s.X.D = D; s.X.stride = stride; s.X.mass = chk.mass_a;
        s.Y.n = M; s.Y.D = D; s.Y.stride = stride; s.Y.mass = chk.mass_b;

        std::unique_ptr<Multiscale> msp;
        if (P.multiscale) {
            msp.reset(new Multiscale());
            s.ms = msp.get();
            msp->cluster(s, P, x, a, y, b, chk.lox, chk.hix, chk.loy, chk.hiy, d_box);
        } else if (D <= 3) {
            s.X.perm = spatial_sort(ctx, "sx", x, N, D, chk.lox, chk.hix, d_box);
            s.Y.perm = spatial_sort(ctx, "sy", y, M, D, chk.loy, chk.hiy, d_box + 128);
        } else {
            // compact row blocks in high dimension: order the points by a short
            // K-means and keep blocks inside clusters (about 16 points per cluster
            // for the float32 kernel; about 128, one full tensor-core tile, for the
            // tensor-core form)
            const int per = s.use_tc ? 128 : 16;
            auto order = [&](const char *tag, const float *pts, const float *w, int n, std::vector<int> &off) {
                const int K = std::max(1, std::min(n / per, 8192));
                KmeansResult r = kmeans(ctx, tag, pts, w, n, D, K, 4, P.seed, nullptr);
                off.resize(K + 1);
                OTGB_CUDA_TRY(cudaMemcpyAsync(off.data(), r.offsets, sizeof(int) * (K + 1), cudaMemcpyDeviceToHost, st));
                OTGB_CUDA_TRY(cudaStreamSynchronize(st));
                return r.perm;
            };
            s.X.perm = order("kx", x, a, N, s.X_off);
            s.Y.perm = order("ky", y, b, M, s.Y_off);
        }
        s.X.pts = s.ws->get<float>("X", (size_t)N * stride);
        s.Y.pts = s.ws->get<float>("Y", (size_t)M * stride);
        s.X.w = s.ws->get<float>("Xw", N);
        s.Y.w = s.ws->get<float>("Yw", M);
        if (D > 3) {
            s.X.logw = s.ws->get<float>("Xlw", N);
            s.Y.logw = s.ws->get<float>("Ylw", M);
        }
        pack_points(x, a, s.X.perm, N, D, d_cen, s.X.pts, s.X.logw, s.X.w, st);
        pack_points(y, b, s.Y.perm, M, D, d_cen, s.Y.pts, s.Y.logw, s.Y.w, st);

        s.alloc_common();
        if (P.debug_wait_probe) {
            unsigned *flag = s.ws->get<unsigned>("probe", 1);
            OTGB_CUDA_TRY(cudaMemsetAsync(flag, 0, sizeof(unsigned), st));
            wait_probe_kernel<<<1, 32, 0, st>>>(flag, s.launch.tc_err, 1000);
            OTGB_CHECK_LAUNCH();
        }
        s.alloc_pots(P);
        s.g_from_f = P.init_g_from_f != 0 && P.f_init != nullptr && P.g_init == nullptr;

        // rows per CTA: enough CTAs to fill the GPU twice, else the smallest blocks
        // rows per thread (D <= 3): 4, so that one warp's block holds 128 rows
        // (each staged column feeds 4 rows per lane, and the block's kept set --
        // the union over its clusters -- stays small)
        s.rows_per_thread = 1;
        if (D <= 3) s.rows_per_thread = 4;
        if (D <= 3 && (P.rows_per_thread == 1 || P.rows_per_thread == 2 || P.rows_per_thread == 4))
            s.rows_per_thread = P.rows_per_thread;
        const int block_rows = D <= 3 ? 32 * s.rows_per_thread : 128;
        s.block_rows = block_rows;

        std::vector<double> sched = make_schedule(diameter, P.blur, P.scaling);
        if (P.sigma_start > 0.0) {
            std::vector<double> t;
            for (double v : sched)
                if (v <= P.sigma_start) t.push_back(v);
            if (t.empty()) t.push_back(P.blur);
            sched.swap(t);
        }
        int rc = OTGB_OK;
        // phase boundaries: 2 = points prepared (validated, clustered, packed),
        // 3 = coarse phase and extrapolation done, 4 = iterations done
        OTGB_CUDA_TRY(cudaEventRecord(ctx_event(ctx, 2), st));
        if (msp) {
            rc = msp->run_schedule(s, P, sched, block_rows);
        } else {
            OTGB_CUDA_TRY(cudaEventRecord(ctx_event(ctx, 3), st));
            s.setup_dense_instances(block_rows);
            for (size_t k = 0; k < sched.size() && s.steps < P.max_iters; ++k) s.fine_step(sched[k]);
        }
        if (rc == OTGB_OK) rc = s.iterate_at_blur(P, P.max_iters);
        if (rc == OTGB_OK && P.polish && D > 3) {
            // polish: the same loop on the direct difference form of the cost (see otgb_params.polish)
            s.launch.direct = 1;
            s.launch.use_tcc = 0;
            s.no_progress = 0;
            s.floor_hits = 0;
            s.delta_best = 1e300;
            // at least 30 steps: the Anderson history needs a few windows to resolve the slowly
            // contracting modes once the exponents are exact
            otgb_params Pp = P;
            Pp.min_iters = std::max(P.min_iters, 30);
            rc = s.iterate_at_blur(Pp, P.max_iters);
        }
        OTGB_CUDA_TRY(cudaEventRecord(ctx_event(ctx, 4), st));
        if (rc == OTGB_OK || rc == OTGB_ENOCONV) s.S = s.divergence(s.eps_of(P.blur));
        if (gr && (rc == OTGB_OK || rc == OTGB_ENOCONV)) grad_sparse_launch(s, s.eps_of(P.blur), *gr, st);

        // outputs in the caller's order
        unpermute(s.pf[s.cur], s.X.perm, N, f, st);
        unpermute(s.pg[s.cur], s.Y.perm, M, g, st);
        if (a_self) unpermute(s.pa[s.cur], s.X.perm, N, a_self, st);
        if (b_self) unpermute(s.pb[s.cur], s.Y.perm, M, b_self, st);
        int *bad = s.ws->get<int>("bad", 4);
        OTGB_CUDA_TRY(cudaMemsetAsync(bad, 0, sizeof(int), st));
        check_finite(f, N, bad, st);
        check_finite(g, M, bad, st);
        char *mb = static_cast<char *>(ctx_pinned(ctx));
        OTGB_CUDA_TRY(cudaMemcpyAsync(mb + kMbBad, bad, sizeof(int), cudaMemcpyDeviceToHost, st));
        OTGB_CUDA_TRY(cudaMemcpyAsync(mb + kMbMass, s.d_pairs, 8, cudaMemcpyDeviceToHost, st));
        OTGB_CUDA_TRY(cudaMemcpyAsync(mb + kMbMass + 8, s.d_fb_total, 8, cudaMemcpyDeviceToHost, st));
        OTGB_CUDA_TRY(cudaMemcpyAsync(mb + kMbMass + 16, s.launch.tc_err, 4, cudaMemcpyDeviceToHost, st));
        OTGB_CUDA_TRY(cudaEventRecord(ctx_event(ctx, 1), st));
        OTGB_CUDA_TRY(cudaStreamSynchronize(st));
        s.harvest_timing();
        *cost_host = s.S;
        if (*reinterpret_cast<int *>(mb + kMbBad) || !std::isfinite(s.S)) rc = OTGB_ENONFINITE;
        if (*reinterpret_cast<unsigned *>(mb + kMbMass + 16)) rc = OTGB_ETIMEOUT;

        if (plan_out && (rc == OTGB_OK || rc == OTGB_ENOCONV)) {
            otgb_plan *pl = new otgb_plan();
            pl->N = N; pl->M = M; pl->D = D;
            pl->x = x; pl->y = y; pl->b = b;
            pl->eps = s.eps_of(P.blur);
            pl->p = P.p;
            *plan_out = pl;
        }
        if (stats) {
            std::memset(stats, 0, sizeof(*stats));
            stats->iters_total = s.steps;
            stats->iters_coarse = s.coarse_steps;
            stats->iters_fine = s.fine_steps;
            stats->schedule_len = (int)sched.size();
            stats->diameter = diameter;
            stats->sigma_switch = msp ? msp->sigma_switch : 0.0;
            stats->n_clusters_x = msp ? msp->ncl_x : 0;
            stats->n_clusters_y = msp ? msp->ncl_y : 0;
            unsigned long long pairs, fbt;
            std::memcpy(&pairs, mb + kMbMass, 8);
            std::memcpy(&fbt, mb + kMbMass + 8, 8);
            stats->pairs_evaluated = (double)pairs;
            const double dense = (double)N * N + (double)M * M + 2.0 * N * M;
            stats->pairs_dense = dense * s.fine_steps;
            stats->kept_fraction = msp ? msp->last_kept_fraction : 1.0;
            stats->softmin_ms = s.softmin_ms;
            float tot = 0.f;
            OTGB_CUDA_TRY(cudaEventElapsedTime(&tot, ctx_event(ctx, 0), ctx_event(ctx, 1)));
            stats->total_ms = tot;
            auto span = [&](int a, int b) {
                float ms = 0.f;
                OTGB_CUDA_TRY(cudaEventElapsedTime(&ms, ctx_event(ctx, a), ctx_event(ctx, b)));
                return (double)ms;
            };
            stats->prep_ms = span(0, 2);
            stats->coarse_ms = span(2, 3);
            stats->fine_ms = span(3, 4);
            stats->final_ms = span(4, 1);
            stats->last_delta = s.last_delta;
            stats->last_rel_change = s.last_rel;
            stats->fallback_rows = (long long)fbt;
        }
        if (rc != OTGB_OK) {
            const char *m = rc == OTGB_ENOCONV   ? "sinkhorn_divergence: max_iters reached before the stopping rule held"
                            : rc == OTGB_ETIMEOUT ? "sinkhorn_divergence: a bounded device wait gave up"
                                                  : "sinkhorn_divergence: a potential or the divergence is not finite";
            return fail(ctx, Error{rc, m});
        }
        return OTGB_OK;
    } catch (const Error &e) {
        return fail(ctx, e);
    }
}

extern "C" int sinkhorn_divergence(otgb_ctx *ctx, const float *x, const float *a, int N, const float *y,
                                   const float *b, int M, int D, const otgb_params *params, double *cost_host,
                                   float *f, float *g, float *a_self, float *b_self, otgb_plan **plan_out,
                                   otgb_stats *stats) {
    return solve_divergence(ctx, x, a, N, y, b, M, D, params, cost_host, f, g, a_self, b_self, plan_out, stats,
                            nullptr);
}

extern "C" int otgb_softmin(otgb_ctx *ctx, const float *q, int n_out, const float *p, const float *w,
                            const float *pot, int n_in, int D, double eps, double lam, const float *old,
                            double omega, float *out) {
    if (!ctx) return fail(nullptr, Error{OTGB_EINVAL, "otgb_softmin: null context"});
    try {
        ctx_set_device(ctx);
        require(q && p && w && pot && out, "otgb_softmin: null pointer argument");
        require(n_out >= 1 && n_in >= 1, "otgb_softmin: sizes must be >= 1");
        require(D >= 1 && D <= 64, "otgb_softmin: D must be in [1, 64]");
        require(eps > 0.0 && std::isfinite(eps), "otgb_softmin: eps must be > 0");
        cudaStream_t st = ctx_stream(ctx);
        Workspace &ws = ctx_ws(ctx);
        const int stride = D <= 3 ? 4 : ((D + 3) & ~3);
        // common centre: middle of the bounding box of the columns
        float *box = ws.get<float>("box", 4 * 64);
        float *bpart = ws.get<float>("bpart", 64 * 2 * 64);
        bbox(p, n_in, D, D, box, box + 64, bpart, st);
        std::vector<float> h(128);
        OTGB_CUDA_TRY(cudaMemcpyAsync(h.data(), box, 128 * sizeof(float), cudaMemcpyDeviceToHost, st));
        OTGB_CUDA_TRY(cudaStreamSynchronize(st));
        std::vector<float> cen(64, 0.f);
        for (int d = 0; d < D; ++d) cen[d] = 0.5f * (h[d] + h[64 + d]);
        float *d_cen = ws.get<float>("cen", 64);
        OTGB_CUDA_TRY(cudaMemcpyAsync(d_cen, cen.data(), 64 * sizeof(float), cudaMemcpyHostToDevice, st));
        float *R = ws.get<float>("sm:R", (size_t)n_out * stride);
        float *C = ws.get<float>("sm:C", (size_t)n_in * stride);
        float *Clw = D > 3 ? ws.get<float>("sm:Clw", n_in) : nullptr;
        pack_points(q, nullptr, nullptr, n_out, D, d_cen, R, nullptr, nullptr, st);
        pack_points(p, w, nullptr, n_in, D, d_cen, C, Clw, nullptr, st);
        // rows per thread as in the solver: the largest R in {4, 2} that still
        // gives two CTAs per SM, else 1
        int rpt = 1;
        if (D <= 3) {
            const int sms = ctx_sm_count(ctx);
            for (int r : {4, 2})
                if ((n_out + 32 * r - 1) / (32 * r) >= 8 * sms) { rpt = r; break; }
        }
        const int block_rows = D <= 3 ? 32 * rpt : 128;
        int *blk = ws.get<int>("sm:blk", n_out / block_rows + 2);
        const int nb = uniform_blocks(blk, n_out, block_rows, st);
        std::vector<int4> items(nb);
        for (int k = 0; k < nb; ++k) items[k] = make_int4(0, k, 0, n_in);
        int4 *d_items = ws.get<int4>("sm:items", nb);
        OTGB_CUDA_TRY(cudaMemcpyAsync(d_items, items.data(), nb * sizeof(int4), cudaMemcpyHostToDevice, st));
        SoftminLaunch L;
        std::memset(&L, 0, sizeof(L));
        L.n_inst = 1;
        SoftminInst &I = L.inst[0];
        I.rows = R; I.cols = C; I.col_logw = Clw; I.col_pot = pot; I.row_old = old; I.row_out = out;
        I.n_rows = n_out; I.n_cols = n_in; I.lam = (float)lam; I.omega = (float)omega;
        I.blk_row0 = blk;
        L.items = d_items;
        L.n_items = nb;
        L.exact_max = 1;  // `old` is a blend target here, not an estimate of the result
        L.eps = (float)eps;
        L.s = (float)(1.4426950408889634 / eps);
        L.eps_ln2 = eps * 0.69314718055994530942;
        const int cap = n_out + 64;
        L.fallback = ws.get<int4>("sm:fb", cap);
        L.n_fallback = ws.get<int>("sm:nfb", 1);
        L.fallback_cap = cap;
        softmin_run(L, D, rpt, st);
        OTGB_CUDA_TRY(cudaStreamSynchronize(st));  // the host item vector is released here
        return OTGB_OK;
    } catch (const Error &e) {
        return fail(ctx, e);
    }
}
