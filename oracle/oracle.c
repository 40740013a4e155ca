/*
 * FP64 CPU oracle for the symmetric, debiased Sinkhorn solver of
 * Feydy, Roussillon, Trouve, Gori, "Fast and Scalable Optimal Transport for
 * Brain Tractograms" (MICCAI 2019).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the CUDA library and
 * its Python binding) may include, link or call this file.  Only the test
 * suite, the smoke check and the benchmark's CPU-baseline leg use it.  It
 * shares no code, header, table or constant with the GPU path.
 *
 * Everything is plain, slow and written to be checked against the paper by
 * eye: double precision, dense loops, two-pass log-sum-exp (max first, then
 * the sum of shifted exponentials), OpenMP only across independent output
 * rows.  Inputs arrive as float (the same seeded arrays the GPU path reads)
 * and are promoted to double on entry.
 *
 * Notation follows Section 2 of the paper: alpha = sum_i alpha_i delta_{x_i},
 * beta = sum_j beta_j delta_{y_j}, cost C(x,y) = (1/p)|x-y|^p, temperature
 * eps = sigma^p, marginal strength rho = reach^p, damping
 * lambda = 1/(1 + eps/rho).  reach <= 0 or +inf means balanced OT (rho = inf,
 * lambda = 1).  The four dual vectors are a = a^{alpha<->alpha} (N),
 * b = b^{beta<->beta} (M), g = a^{alpha->beta} (M), f = b^{beta->alpha} (N).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Threads the OpenMP row loops run on (reported with the oracle's timings). */
int oracle_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Threads of the row loops from now on (n >= 1), for timings on one core. */
void oracle_set_threads(int n)
{
#ifdef _OPENMP
    if (n >= 1) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* ------------------------------------------------------------------------ */
/* Ground cost, Section 2: C(x, y) = (1/p) |x - y|^p.                          */
/* ------------------------------------------------------------------------ */
static double cost(const float *u, const float *v, int D, int p)
{
    double s = 0.0;
    for (int d = 0; d < D; ++d) {
        double t = (double)u[d] - (double)v[d];
        s += t * t;
    }
    if (p == 2) return 0.5 * s;
    return pow(sqrt(s), (double)p) / (double)p;
}

double oracle_cost(const float *u, const float *v, int D, int p) { return cost(u, v, D, p); }

static int balanced(double reach) { return !(reach > 0.0) || isinf(reach); }

/* rho = reach^p, or +inf when balanced. */
double oracle_rho(double reach, int p) { return balanced(reach) ? INFINITY : pow(reach, (double)p); }

/* lambda = 1 / (1 + (sigma/reach)^p), the unbalanced damping of the Algorithm
 * in Section 2; 1 when balanced. */
double oracle_lambda(double sigma, double reach, int p)
{
    if (balanced(reach)) return 1.0;
    return 1.0 / (1.0 + pow(sigma / reach, (double)p));
}

/* ------------------------------------------------------------------------ */
/* One softmin update of the Algorithm in Section 2:                            */
/*   out_i = -lam * eps * log sum_k w_k exp((pot_k - C(p_k, q_i)) / eps)      */
/* for rows q_i (n_out points) and columns p_k (n_in points).  Columns with     */
/* w_k = 0 contribute nothing (log 0 = -inf).  Two passes per row: the max of */
/* the exponents, then the sum of exp(exponent - max).                         */
/* ------------------------------------------------------------------------ */
void oracle_softmin(int n_out, const float *q, int n_in, const float *pts, const float *w,
                    const double *pot, int D, int p, double eps, double lam, double *out)
{
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n_out; ++i) {
        double m = -INFINITY;
        for (int k = 0; k < n_in; ++k) {
            if (!(w[k] > 0.0f)) continue;
            double e = log((double)w[k]) + (pot[k] - cost(pts + (size_t)k * D, q + (size_t)i * D, D, p)) / eps;
            if (e > m) m = e;
        }
        double s = 0.0;
        for (int k = 0; k < n_in; ++k) {
            if (!(w[k] > 0.0f)) continue;
            double e = log((double)w[k]) + (pot[k] - cost(pts + (size_t)k * D, q + (size_t)i * D, D, p)) / eps;
            s += exp(e - m);
        }
        out[i] = -lam * eps * (m + log(s));
    }
}

/* ------------------------------------------------------------------------ */
/* Diameter heuristic.  The Algorithm in Section 2 takes d = max_ij |x_i-y_j|;  */
/* this oracle, like the GPU path, uses the diagonal of the bounding box of    */
/* x and y together, an upper bound of that maximum (documented reading).      */
/* ------------------------------------------------------------------------ */
double oracle_diameter(const float *x, int N, const float *y, int M, int D)
{
    double s = 0.0;
    for (int d = 0; d < D; ++d) {
        double lo = INFINITY, hi = -INFINITY;
        for (int i = 0; i < N; ++i) { double v = x[(size_t)i * D + d]; if (v < lo) lo = v; if (v > hi) hi = v; }
        for (int j = 0; j < M; ++j) { double v = y[(size_t)j * D + d]; if (v < lo) lo = v; if (v > hi) hi = v; }
        if (hi > lo) s += (hi - lo) * (hi - lo);
    }
    return sqrt(s);
}

/* ------------------------------------------------------------------------ */
/* epsilon-scaling schedule of the Algorithm in Section 2:                     */
/*   sigma in [d, d q, d q^2, ..., blur].                                       */
/* Reading: sigma_k = d q^k for k = 0..K-1 with K = ceil(log(d/blur)/log(1/q)),  */
/* then blur.  When d <= blur the list is [blur].  Returns the length, writes   */
/* at most cap entries.                                                         */
/* ------------------------------------------------------------------------ */
int oracle_schedule(double d, double blur, double q, double *sigma, int cap)
{
    int n = 0;
    if (d > blur) {
        int K = (int)ceil(log(d / blur) / log(1.0 / q));
        for (int k = 0; k < K; ++k) { if (n < cap) sigma[n] = d * pow(q, (double)k); ++n; }
    }
    if (n < cap) sigma[n] = blur;
    return n + 1;
}

/* ------------------------------------------------------------------------ */
/* One symmetrised, averaged Sinkhorn step (the loop body of the Algorithm in */
/* Section 2): the four "tilde" softmins all read the OLD vectors, then each   */
/* vector becomes the average of its old value and its tilde.                  */
/* Returns max over the four vectors of |new - old| / eps.                      */
/* ------------------------------------------------------------------------ */
double oracle_sinkhorn_step(const float *x, const float *alpha, int N, const float *y, const float *beta,
                            int M, int D, int p, double eps, double lam, double *a, double *b, double *f,
                            double *g)
{
    double *ta = (double *)malloc(sizeof(double) * (size_t)N);
    double *tb = (double *)malloc(sizeof(double) * (size_t)M);
    double *tg = (double *)malloc(sizeof(double) * (size_t)M);
    double *tf = (double *)malloc(sizeof(double) * (size_t)N);
    oracle_softmin(N, x, N, x, alpha, a, D, p, eps, lam, ta); /* a~ on x from (x, alpha, a) */
    oracle_softmin(M, y, M, y, beta, b, D, p, eps, lam, tb);  /* b~ on y from (y, beta, b)  */
    oracle_softmin(M, y, N, x, alpha, f, D, p, eps, lam, tg); /* g~ on y from (x, alpha, f) */
    oracle_softmin(N, x, M, y, beta, g, D, p, eps, lam, tf);  /* f~ on x from (y, beta, g)  */
    double delta = 0.0;
    for (int i = 0; i < N; ++i) {
        double na = 0.5 * (a[i] + ta[i]), nf = 0.5 * (f[i] + tf[i]);
        delta = fmax(delta, fmax(fabs(na - a[i]), fabs(nf - f[i])));
        a[i] = na; f[i] = nf;
    }
    for (int j = 0; j < M; ++j) {
        double nb = 0.5 * (b[j] + tb[j]), ng = 0.5 * (g[j] + tg[j]);
        delta = fmax(delta, fmax(fabs(nb - b[j]), fabs(ng - g[j])));
        b[j] = nb; g[j] = ng;
    }
    free(ta); free(tb); free(tg); free(tf);
    return delta / eps;
}

/* ------------------------------------------------------------------------ */
/* Debiased Sinkhorn divergence from the four dual vectors, Eq. (6).          */
/*  unbalanced: S = -(rho + eps/2) [ <alpha, e^{-f/rho} - e^{-a/rho}>          */
/*                                 + <beta,  e^{-g/rho} - e^{-b/rho}> ]        */
/*  written as e^{-a/rho} expm1(-(f-a)/rho) to avoid cancellation;             */
/*  balanced (rho -> inf): S = <alpha, f - a> + <beta, g - b>.                 */
/* ------------------------------------------------------------------------ */
double oracle_divergence(const float *alpha, int N, const float *beta, int M, double eps, double rho,
                         const double *a, const double *b, const double *f, const double *g)
{
    double s = 0.0;
    if (isinf(rho)) {
        for (int i = 0; i < N; ++i) s += (double)alpha[i] * (f[i] - a[i]);
        for (int j = 0; j < M; ++j) s += (double)beta[j] * (g[j] - b[j]);
        return s;
    }
    for (int i = 0; i < N; ++i) s += (double)alpha[i] * exp(-a[i] / rho) * expm1(-(f[i] - a[i]) / rho);
    for (int j = 0; j < M; ++j) s += (double)beta[j] * exp(-b[j] / rho) * expm1(-(g[j] - b[j]) / rho);
    return -(rho + 0.5 * eps) * s;
}

/* ------------------------------------------------------------------------ */
/* Full solve.  Zero initialisation as the Algorithm of Section 2 starts, one */
/* averaged step per sigma of the schedule, then further averaged steps at   */
/* sigma = blur until max|new-old|/eps < tol or max_iters steps in total.     */
/* diameter <= 0 selects the bounding-box diagonal.  Outputs the four vectors,*/
/* S by Eq. (6), and info[0] = steps taken, info[1] = schedule length,        */
/* info[2] = last max|delta|/eps.  Returns 0 when converged, 1 otherwise.     */
/* ------------------------------------------------------------------------ */
int oracle_sinkhorn(const float *x, const float *alpha, int N, const float *y, const float *beta, int M,
                    int D, int p, double blur, double reach, double q, double diameter, double tol,
                    int max_iters, double *a, double *b, double *f, double *g, double *S, double *info)
{
    double d = diameter > 0.0 ? diameter : oracle_diameter(x, N, y, M, D);
    int K = oracle_schedule(d, blur, q, NULL, 0);
    double *sig = (double *)malloc(sizeof(double) * (size_t)K);
    oracle_schedule(d, blur, q, sig, K);
    for (int i = 0; i < N; ++i) a[i] = f[i] = 0.0;
    for (int j = 0; j < M; ++j) b[j] = g[j] = 0.0;
    double rho = oracle_rho(reach, p), eps = pow(blur, (double)p), delta = INFINITY;
    int it = 0;
    for (int k = 0; k < K && it < max_iters; ++k, ++it) {
        double e = pow(sig[k], (double)p);
        delta = oracle_sinkhorn_step(x, alpha, N, y, beta, M, D, p, e, oracle_lambda(sig[k], reach, p), a, b, f, g);
    }
    double lam = oracle_lambda(blur, reach, p);
    while (it < max_iters && !(delta < tol)) {
        delta = oracle_sinkhorn_step(x, alpha, N, y, beta, M, D, p, eps, lam, a, b, f, g);
        ++it;
    }
    *S = oracle_divergence(alpha, N, beta, M, eps, rho, a, b, f, g);
    if (info) { info[0] = it; info[1] = K; info[2] = delta; }
    free(sig);
    return delta < tol ? 0 : 1;
}

/* ------------------------------------------------------------------------ */
/* Regularised OT in dual form, Eq. (3), at given (f, g):                      */
/*  rho <alpha, 1 - e^{-f/rho}> + rho <beta, 1 - e^{-g/rho}>                   */
/*  + eps <alpha x beta, 1 - exp((f_i + g_j - C_ij)/eps)>.                     */
/* Balanced (rho = inf): the first two terms become <alpha,f> + <beta,g>.      */
/* ------------------------------------------------------------------------ */
double oracle_ot_dual(const float *x, const float *alpha, int N, const float *y, const float *beta, int M,
                      int D, int p, double eps, double rho, const double *f, const double *g)
{
    double s = 0.0;
    for (int i = 0; i < N; ++i)
        s += isinf(rho) ? (double)alpha[i] * f[i] : rho * (double)alpha[i] * -expm1(-f[i] / rho);
    for (int j = 0; j < M; ++j)
        s += isinf(rho) ? (double)beta[j] * g[j] : rho * (double)beta[j] * -expm1(-g[j] / rho);
    double t = 0.0;
    for (int i = 0; i < N; ++i)
        for (int j = 0; j < M; ++j)
            t += (double)alpha[i] * (double)beta[j] *
                 -expm1((f[i] + g[j] - cost(x + (size_t)i * D, y + (size_t)j * D, D, p)) / eps);
    return s + eps * t;
}

/* Generalised KL divergence, Section 2: KL(u, v) = sum u log(u/v) - u + v,
 * with 0 log 0 = 0. */
static double kl(const double *u, const double *v, int n)
{
    double s = 0.0;
    for (int k = 0; k < n; ++k) s += (u[k] > 0.0 ? u[k] * log(u[k] / v[k]) : 0.0) - u[k] + v[k];
    return s;
}

/* ------------------------------------------------------------------------ */
/* Regularised OT in primal form, Eq. (2), evaluated at the plan of Eq. (4):   */
/*  pi_ij = alpha_i beta_j exp((f_i + g_j - C_ij)/eps),                         */
/*  <pi, C> + eps KL(pi, alpha x beta) + rho KL(pi 1, alpha) + rho KL(pi^T 1,   */
/*  beta).  Balanced (rho = inf): the two marginal terms are dropped (they are  */
/*  constraints); marg_err receives max |pi 1 - alpha|, |pi^T 1 - beta|.        */
/* ------------------------------------------------------------------------ */
double oracle_ot_primal(const float *x, const float *alpha, int N, const float *y, const float *beta, int M,
                        int D, int p, double eps, double rho, const double *f, const double *g,
                        double *marg_err)
{
    double *r = (double *)calloc((size_t)N, sizeof(double)), *c = (double *)calloc((size_t)M, sizeof(double));
    double *al = (double *)malloc(sizeof(double) * (size_t)N), *be = (double *)malloc(sizeof(double) * (size_t)M);
    double lin = 0.0, ent = 0.0;
    for (int i = 0; i < N; ++i) al[i] = alpha[i];
    for (int j = 0; j < M; ++j) be[j] = beta[j];
    for (int i = 0; i < N; ++i)
        for (int j = 0; j < M; ++j) {
            double C = cost(x + (size_t)i * D, y + (size_t)j * D, D, p);
            double ab = al[i] * be[j];
            double pij = ab * exp((f[i] + g[j] - C) / eps);
            lin += pij * C;
            ent += (pij > 0.0 ? pij * log(pij / ab) : 0.0) - pij + ab;
            r[i] += pij; c[j] += pij;
        }
    double v = lin + eps * ent;
    if (!isinf(rho)) v += rho * kl(r, al, N) + rho * kl(c, be, M);
    if (marg_err) {
        double e = 0.0;
        for (int i = 0; i < N; ++i) e = fmax(e, fabs(r[i] - al[i]));
        for (int j = 0; j < M; ++j) e = fmax(e, fabs(c[j] - be[j]));
        *marg_err = e;
    }
    free(r); free(c); free(al); free(be);
    return v;
}

/* ------------------------------------------------------------------------ */
/* Label transfer, Eq. (7):                                                     */
/*  Lab_il = sum_{j : label_j = l} beta_j exp((f_i + g_j - C(x_i, y_j))/eps).   */
/* Computed per (row, class) as exp of a two-pass log-sum-exp.  argmax takes   */
/* the lowest class index on ties; row_mass = sum_l Lab_il.                     */
/* ------------------------------------------------------------------------ */
void oracle_transport_apply(const float *x, int N, const float *y, const float *beta, int M, int D, int p,
                            double eps, const double *f, const double *g, const int32_t *labels, int L,
                            double *scores, int32_t *argmax, double *row_mass)
{
#pragma omp parallel for schedule(static)
    for (int i = 0; i < N; ++i) {
        double *sc = scores + (size_t)i * L;
        for (int l = 0; l < L; ++l) {
            double m = -INFINITY;
            for (int j = 0; j < M; ++j) {
                if (labels[j] != l || !(beta[j] > 0.0f)) continue;
                double e = log((double)beta[j]) + (f[i] + g[j] - cost(x + (size_t)i * D, y + (size_t)j * D, D, p)) / eps;
                if (e > m) m = e;
            }
            if (m == -INFINITY) { sc[l] = 0.0; continue; }
            double s = 0.0;
            for (int j = 0; j < M; ++j) {
                if (labels[j] != l || !(beta[j] > 0.0f)) continue;
                double e = log((double)beta[j]) + (f[i] + g[j] - cost(x + (size_t)i * D, y + (size_t)j * D, D, p)) / eps;
                s += exp(e - m);
            }
            sc[l] = exp(m + log(s));
        }
        int best = 0;
        double tot = 0.0;
        for (int l = 0; l < L; ++l) { tot += sc[l]; if (sc[l] > sc[best]) best = l; }
        argmax[i] = best;
        row_mass[i] = tot;
    }
}

/* ------------------------------------------------------------------------ */
/* Grid clustering (the coarse subsampling of Section 2, grid variant).       */
/* Cell coordinate c_d = floor((x_d - origin_d) / cell), evaluated in float    */
/* (IEEE single, round to nearest) so that the integer decision matches a     */
/* single-precision implementation; origin is the per-axis float minimum of x. */
/* D <= 3.  The cell key is the Morton (bit-interleaved) code of (c_0, c_1,   */
/* c_2), 10 bits per axis.  Points are ordered by a stable sort on the key;   */
/* clusters are the occupied cells in key order.  Outputs: labels[N] (cluster */
/* of each point in original order), perm[N] (sorted position -> original     */
/* index), offsets[n+1], and the cluster count.  Returns -1 when a cell       */
/* coordinate needs more than 10 bits.                                          */
/* ------------------------------------------------------------------------ */
static uint32_t spread3(uint32_t v)
{
    /* bit b of v goes to bit 3b */
    uint32_t r = 0;
    for (int bit = 0; bit < 10; ++bit) r |= ((v >> bit) & 1u) << (3 * bit);
    return r;
}

static const uint32_t *g_sort_keys;
static int cmp_key_then_index(const void *pa, const void *pb)
{
    int a = *(const int *)pa, b = *(const int *)pb;
    uint32_t ka = g_sort_keys[a], kb = g_sort_keys[b];
    if (ka != kb) return ka < kb ? -1 : 1;
    return a < b ? -1 : (a > b); /* stable: ties keep input order */
}

int oracle_cluster_grid(const float *x, int N, int D, float cell, int32_t *labels, int32_t *perm,
                        int32_t *offsets, uint32_t *keys_out)
{
    float origin[3] = {0.f, 0.f, 0.f};
    for (int d = 0; d < D; ++d) {
        float lo = INFINITY;
        for (int i = 0; i < N; ++i) if (x[(size_t)i * D + d] < lo) lo = x[(size_t)i * D + d];
        origin[d] = lo;
    }
    uint32_t *key = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(N > 0 ? N : 1));
    for (int i = 0; i < N; ++i) {
        uint32_t k = 0;
        for (int d = 0; d < D; ++d) {
            volatile float diff = x[(size_t)i * D + d] - origin[d];
            volatile float qt = diff / cell;
            float c = floorf(qt);
            if (c > 1023.0f) { free(key); return -1; }
            k |= spread3((uint32_t)c) << d;
        }
        key[i] = k;
        if (keys_out) keys_out[i] = k;
    }
    for (int i = 0; i < N; ++i) perm[i] = i;
    g_sort_keys = key;
    qsort(perm, (size_t)N, sizeof(int32_t), cmp_key_then_index);
    int n = 0;
    for (int s = 0; s < N; ++s) {
        if (s == 0 || key[perm[s]] != key[perm[s - 1]]) offsets[n++] = s;
        labels[perm[s]] = n - 1;
    }
    offsets[n] = N;
    free(key);
    return n;
}

/* ------------------------------------------------------------------------ */
/* Lloyd's K-means (the "simple K-means" coarse subsampling of Section 2),     */
/* weighted: starting from the given centroids, repeat `iters` times: assign  */
/* each point to its nearest centroid (lowest index on ties), then move each  */
/* centroid to the weighted mean of its points (an empty cluster keeps its    */
/* centroid).  Writes labels[N] and centroids[K*D] (double).                   */
/* ------------------------------------------------------------------------ */
void oracle_kmeans(const float *x, const float *w, int N, int D, int K, int iters, const float *init,
                   int32_t *labels, double *cent)
{
    for (int k = 0; k < K * D; ++k) cent[k] = init[k];
    double *acc = (double *)malloc(sizeof(double) * (size_t)K * (size_t)D);
    double *mass = (double *)malloc(sizeof(double) * (size_t)K);
    for (int it = 0; it <= iters; ++it) {
#pragma omp parallel for schedule(static)
        for (int i = 0; i < N; ++i) {
            int best = 0;
            double bd = INFINITY;
            for (int k = 0; k < K; ++k) {
                double s = 0.0;
                for (int d = 0; d < D; ++d) { double t = (double)x[(size_t)i * D + d] - cent[(size_t)k * D + d]; s += t * t; }
                if (s < bd) { bd = s; best = k; }
            }
            labels[i] = best;
        }
        if (it == iters) break;
        memset(acc, 0, sizeof(double) * (size_t)K * (size_t)D);
        memset(mass, 0, sizeof(double) * (size_t)K);
        for (int i = 0; i < N; ++i) {
            double wi = w ? (double)w[i] : 1.0;
            mass[labels[i]] += wi;
            for (int d = 0; d < D; ++d) acc[(size_t)labels[i] * D + d] += wi * (double)x[(size_t)i * D + d];
        }
        for (int k = 0; k < K; ++k)
            if (mass[k] > 0.0)
                for (int d = 0; d < D; ++d) cent[(size_t)k * D + d] = acc[(size_t)k * D + d] / mass[k];
    }
    free(acc); free(mass);
}

/* ------------------------------------------------------------------------ */
/* Gradient of the debiased divergence with respect to the points x_i.      */
/* Section 2 (unbiased Sinkhorn divergences) states that the gradients of S  */
/* in the weights and the points are expressions of the four dual vectors.  */
/* Each OT term is a maximum over dual pairs of a function that sees the     */
/* points only through the cost, so at the optimal duals (envelope theorem)  */
/*   d OT(alpha, beta) / d x_i   = sum_j pi_ij grad_1 C(x_i, y_j),           */
/*   d OT(alpha, alpha) / d x_i  = 2 sum_k pi^aa_ik grad_1 C(x_i, x_k)       */
/* (x_i is in both arguments; C is symmetric), with the plans of Eq. (4):    */
/* pi_ij = alpha_i beta_j exp((f_i + g_j - C(x_i, y_j)) / eps) and           */
/* pi^aa_ik = alpha_i alpha_k exp((a_i + a_k - C(x_i, x_k)) / eps).  With    */
/* S = OT(alpha, beta) - OT(alpha, alpha)/2 - OT(beta, beta)/2 + (mass term, */
/* free of x):                                                               */
/*   dS/dx_i = sum_j pi_ij grad_1 C(x_i, y_j) - sum_k pi^aa_ik grad_1 C(x_i, x_k), */
/* grad_1 C(u, v) = |u - v|^(p-2) (u - v) for C = |u - v|^p / p.  The        */
/* gradient in y is the same expression with the roles of the two measures   */
/* exchanged (y, beta, g, b against x, alpha, f).                             */
/* ------------------------------------------------------------------------ */
static void add_grad_cost(const float *u, const float *v, int D, int p, double w, double *out)
{
    double s = 0.0;
    for (int d = 0; d < D; ++d) {
        double t = (double)u[d] - (double)v[d];
        s += t * t;
    }
    double scale = w;
    if (p != 2) {
        if (s == 0.0) return;
        scale *= pow(sqrt(s), (double)p - 2.0);
    }
    for (int d = 0; d < D; ++d) out[d] += scale * ((double)u[d] - (double)v[d]);
}

void oracle_grad_x(const float *x, const float *alpha, int N, const float *y, const float *beta, int M, int D,
                   int p, double eps, const double *a, const double *f, const double *g, double *grad)
{
#pragma omp parallel for schedule(static)
    for (int i = 0; i < N; ++i) {
        double *gi = grad + (size_t)i * D;
        for (int d = 0; d < D; ++d) gi[d] = 0.0;
        const float *xi = x + (size_t)i * D;
        for (int j = 0; j < M; ++j) {
            const float *yj = y + (size_t)j * D;
            double pij = (double)alpha[i] * (double)beta[j] * exp((f[i] + g[j] - cost(xi, yj, D, p)) / eps);
            add_grad_cost(xi, yj, D, p, pij, gi);
        }
        for (int k = 0; k < N; ++k) {
            const float *xk = x + (size_t)k * D;
            double pik = (double)alpha[i] * (double)alpha[k] * exp((a[i] + a[k] - cost(xi, xk, D, p)) / eps);
            add_grad_cost(xi, xk, D, p, -pik, gi);
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Flip augmentation (Section 2, fiber encoding): a fiber of P points in 3-D  */
/* is one point of R^{3P}; rows 0..N-1 of out are the fibers, rows N..2N-1    */
/* their mirror flips (the P points in reverse order, each point unchanged). */
/* ------------------------------------------------------------------------ */
void oracle_flip_fibers(const float *x, int N, int P, float *out)
{
    const int D = 3 * P;
    for (int i = 0; i < N; ++i) {
        for (int d = 0; d < D; ++d) out[(size_t)i * D + d] = x[(size_t)i * D + d];
        for (int k = 0; k < P; ++k)
            for (int c = 0; c < 3; ++c)
                out[(size_t)(N + i) * D + 3 * k + c] = x[(size_t)i * D + 3 * (P - 1 - k) + c];
    }
}

/* ------------------------------------------------------------------------ */
/* Label transfer on flip-augmented data (Section 2, label transfer): the plan */
/* matches one version of each fiber; of rows i and N+i the one with the       */
/* larger row mass (ties: the original) gives fiber i its label and mass.      */
/* ------------------------------------------------------------------------ */
void oracle_select_flips(const double *row_mass, const int32_t *argmax, int N, int32_t *label, int32_t *version,
                         double *mass)
{
    for (int i = 0; i < N; ++i) {
        const int v = row_mass[N + i] > row_mass[i] ? 1 : 0;
        version[i] = v;
        label[i] = argmax[v * N + i];
        mass[i] = row_mass[v * N + i];
    }
}
