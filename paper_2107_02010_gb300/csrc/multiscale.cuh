// The solver state shared by the dense loop (sinkhorn.cu) and the
// coarse-to-fine strategy (multiscale.cu).
#pragma once

#include <string>
#include <vector>

#include "anderson.cuh"
#include "otgb_internal.cuh"
#include "solver.cuh"

struct otgb_plan {
    int N = 0, M = 0, D = 0, p = 2;
    const float *x = nullptr, *y = nullptr, *b = nullptr;  // non-owning views
    double eps = 0.0;
};

namespace otgb {

struct Cloud;
struct Multiscale;

struct Cloud {
    int n = 0, D = 0, stride = 0;
    float *pts = nullptr;   // n x stride, translated by the common centre
    float *logw = nullptr;  // D > 3: log w (internal order)
    float *w = nullptr;     // weights (internal order)
    int *perm = nullptr;    // internal position -> caller index; null: identity
    double mass = 0.0;
};

struct Solver {
    static constexpr int kEvPool = 64;
    std::string tag;  // prefix of this solver's workspace buffers
    otgb_ctx *ctx = nullptr;
    cudaStream_t st = nullptr;
    Workspace *ws = nullptr;
    int D = 0;
    int p = 2;  // exponent of the cost |x - y|^p / p (1 or 2)
    double reach = 0.0, rho = 0.0;
    double eps_of(double sigma) const { return p == 1 ? sigma : sigma * sigma; }
    double lam_of(double sigma) const { return lambda_of(sigma, reach, p); }
    Cloud X, Y;
    std::vector<int> X_off, Y_off;  // cluster offsets (host) of the internal order, when clustered
    // the four duals of parity k live in one buffer Z[k] = (a | f | b | g)
    float *Z[2] = {nullptr, nullptr};
    float *pa[2] = {nullptr, nullptr}, *pf[2] = {nullptr, nullptr}, *pb[2] = {nullptr, nullptr},
          *pg[2] = {nullptr, nullptr};
    Anderson aa;
    bool aa_active = false;
    int cur = 0;
    SoftminLaunch launch;
    int rows_per_thread = 1, block_rows = 128;
    int nblk_x = 0, nblk_y = 0;
    unsigned long long *d_pairs = nullptr, *d_fb_total = nullptr;
    int steps = 0, fine_steps = 0, coarse_steps = 0;
    double S = 0.0, last_delta = 0.0, last_rel = 0.0, last_potmax = 0.0;
    bool timing = false;
    bool translation = false;
    bool use_tc = false;
    bool use_tc3 = false;
    std::vector<cudaEvent_t> ev_pool;
    int ev_used = 0;
    double softmin_ms = 0.0;
    long softmin_launches = 0;
    Multiscale *ms = nullptr;
    bool g_from_f = false;                    // before the first step: g = one plain softmin of f
    std::vector<std::vector<int>> work_ncols; // columns per (instance, block) of the current work

    ~Solver();
    void alloc_common();
    void alloc_pots(const otgb_params &P);
    void setup_dense_instances(int block_rows);
    // Instances 0..3 (a~, b~, g~, f~) over row blocks hx / hy (host starts).
    void setup_instances(const std::vector<int> &hx, const std::vector<int> &hy);
    // Work items: per instance and block the number of columns; blocks are
    // split into column chunks when allowed (D <= 3 and old values present).
    void set_work(const std::vector<std::vector<int>> &ncols, bool allow_split);
    std::string nm(const std::string &n) const { return tag + n; }
    void step(double sigma, bool count_pairs);
    void fine_step(double sigma);
    // g~ of f alone (instance 2, no blend) at sigma, written into the current g
    void sweep_g(double sigma);
    void harvest_timing();
    double divergence(double eps);
    int iterate_at_blur(const otgb_params &P, int it_budget);
    static bool converged(const std::vector<double> &hist, double tol, double floor_abs, double *rem_out);
    int no_progress = 0;
    int floor_hits = 0;
    double delta_best = 1e300;
    bool potentials_converged(double delta_prev, double delta, int m, double eps, double potmax, double tol);
};

std::vector<int> make_row_blocks(int n, int block_rows, const std::vector<int> *offsets);
bool trace_enabled();

// The gradient of S in the points of the first measure, computed inside a
// solve from its sorted points, final duals and the kept cluster pairs of its
// last truncation (grad.cu); the barycenter's steps use it.
struct GradRequest {
    float *grad;     // N x D, the caller's order
    float scale;     // multiplies the result
    int accumulate;  // 1: grad += result, 0: grad = result
};
void grad_sparse_launch(const Solver &s, double eps, const GradRequest &gr, cudaStream_t st);
// sinkhorn_divergence, with an optional gradient request (null: none)
int solve_divergence(otgb_ctx *ctx, const float *x, const float *a, int N, const float *y, const float *b, int M,
                     int D, const otgb_params *params, double *cost_host, float *f, float *g, float *a_self,
                     float *b_self, otgb_plan **plan_out, otgb_stats *stats, const GradRequest *gr);

struct Multiscale {
    double sigma_switch = 0.0;
    int ncl_x = 0, ncl_y = 0;
    double last_kept_fraction = 1.0;
    // device cluster data of the fine clouds (internal order)
    int *d_off_x = nullptr, *d_off_y = nullptr;  // ncl + 1
    float *cen_x = nullptr, *cen_y = nullptr;    // ncl x stride (coarse points; D <= 3: (c, log mass))
    float *lm_x = nullptr, *lm_y = nullptr;      // D > 3: log mass
    float *mass_x = nullptr, *mass_y = nullptr, *rad_x = nullptr, *rad_y = nullptr;
    // fine row blocks: host starts and cluster ranges
    std::vector<int> hbx, hby, hclx, hcly;       // hcl: 2 ints per block (cl0, cl1)
    int *d_clx = nullptr, *d_cly = nullptr;
    double mask_sigma = -1.0;
    int steps_since_mask = 0;
    int rebuild_every = 10;
    double tau = 27.6;
    double reach = 0.0;
    void cluster(Solver &s, const otgb_params &P, const float *x, const float *a, const float *y, const float *b,
                 const std::vector<float> &lox, const std::vector<float> &hix, const std::vector<float> &loy,
                 const std::vector<float> &hiy, float *d_box);
    int run_schedule(Solver &s, const otgb_params &P, const std::vector<double> &sched, int block_rows);
    void before_fine_step(Solver &s, double sigma);
    // the column tiles of the cluster-tiled tensor-core form, when it applies (tensor-core precision,
    // D4 <= 60, at most 32 x kTccMaxWords clusters per side)
    void setup_tcc(Solver &s);
};

}  // namespace otgb
