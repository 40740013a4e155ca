/*
 * otgb -- multiscale, symmetric, debiased Sinkhorn on one GB300 (sm_103a).
 *
 * C ABI of libotgb.so.  Method: Feydy, Roussillon, Trouve, Gori, "Fast and
 * Scalable Optimal Transport for Brain Tractograms" (MICCAI 2019), Section 2.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Arrays are DEVICE pointers (cudaMalloc'd, or torch CUDA tensors), owned by
 *    the caller, row-major and contiguous: points are N x D float32, weights N
 *    float32, labels int32.  The library never frees or retains them beyond
 *    the call, except the non-owning views held by an otgb_plan (see below).
 *  - Host pointers are marked "host".  Scalars are passed by value.
 *  - All GPU work is enqueued on the context's CUDA stream.  A call returns
 *    after its results are complete on that stream unless stated otherwise.
 *  - Every function returns an otgb_status; on failure otgb_last_error() gives
 *    a message.  No exception crosses the ABI and no kernel traps.
 *  - Scratch memory comes from the context (stream-ordered allocations that
 *    grow on demand) and is released by otgb_destroy().
 *  - Ground cost: C(x, y) = |x - y|^p / p (Section 2) with p = 2 (the default,
 *    every engine) or p = 1 (C = |x - y|: sinkhorn_divergence on the CUDA cores,
 *    float32, direct form with a square root per pair; sinkhorn_grad_x;
 *    sinkhorn_barycenter).  eps = blur^p, rho = reach^p.  Other p are rejected
 *    with OTGB_EINVAL.  1 <= D <= 64.
 */
#ifndef OTGB_H
#define OTGB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    OTGB_OK = 0,
    OTGB_EINVAL = -1,     /* bad argument: shape, null pointer, blur <= 0, q not in (0,1), ... */
    OTGB_ECUDA = -2,      /* a CUDA runtime call failed */
    OTGB_ENOMEM = -3,     /* device scratch allocation failed */
    OTGB_ENOCONV = -4,    /* max_iters reached before the stopping rule held (results still written) */
    OTGB_ENONFINITE = -5, /* a potential or the divergence became NaN/Inf */
    OTGB_ETIMEOUT = -6,   /* a bounded device-side wait gave up */
    OTGB_EINTERNAL = -7   /* internal consistency check failed */
} otgb_status;

/* OTGB_FP32: float32 accuracy; for D <= 3 the exponent of every pair is one tensor-core dot
   product of three-piece BF16 operands (about 24 significant bits) with FP32 accumulation,
   elsewhere CUDA-core float32.  OTGB_TC_BF16X3: the reduced-precision tensor-core cross term
   for D >= 16 (about 16 bits); in coarse-to-fine solves with k-means clusters and
   round_up(D, 4) <= 60 the column operand is centred at its cluster's centroid and split once
   per solve, which holds 256 bytes per point and copy, two copies per side, in the context's
   scratch (about 0.5 KB per point of x and of y; at most 8192 clusters per side).
   OTGB_FP32_SIMT: float32 on the CUDA cores for every D. */
typedef enum { OTGB_FP32 = 0, OTGB_TC_BF16X3 = 1, OTGB_FP32_SIMT = 2 } otgb_precision;
typedef enum { OTGB_CLUSTER_GRID = 0, OTGB_CLUSTER_KMEANS = 1 } otgb_cluster_kind;

/* Opaque handles. */
typedef struct otgb_ctx otgb_ctx;   /* one device + one stream + scratch */
typedef struct otgb_plan otgb_plan; /* result of a solve, reused by transport_apply */

/* Solver parameters (Section 2: blur, reach, scaling; p = 2). */
typedef struct {
    int p;                 /* exponent of the cost |x - y|^p / p: 2 (default) or 1 (precision FP32 or
                              FP32_SIMT only; label transfer needs p = 2) */
    double blur;           /* finest scale sigma; eps = blur^p.  > 0 */
    double reach;          /* rho = reach^p; <= 0 or +inf: balanced OT (lambda = 1) */
    double scaling;        /* q in (0,1): sigma_{k+1} = q sigma_k (the paper's default is 0.9) */
    double diameter;       /* first sigma; <= 0: diagonal of the bounding box of x and y */
    int multiscale;        /* 1: cluster, coarse solve, extrapolate, truncate; 0: dense single scale */
    int cluster;           /* otgb_cluster_kind, used when multiscale = 1 */
    double cell;           /* grid cell width (same units as x), cluster = GRID; D <= 3 */
    int k_clusters;        /* k-means clusters per side, cluster = KMEANS */
    int kmeans_iters;      /* Lloyd iterations (default 10) */
    unsigned long long seed; /* seed of the k-means initial sample */
    double sigma_switch;   /* last coarse scale; <= 0: the cluster scale (cell, or 2 x RMS cluster radius) */
    double trunc_tau;      /* keep a cluster pair when its log plan bound >= -tau (default 27.6 = -log 1e-12) */
    double tol;            /* stopping rule at sigma = blur: estimated remaining relative change of S < tol */
    int min_iters;         /* at least this many steps at sigma = blur (default 3) */
    int max_iters;         /* cap on the total number of steps, schedule included */
    int check_every;       /* evaluate S and the stopping rule every k steps (default 10) */
    int fixed_iters;       /* > 0: run exactly this many steps at sigma = blur after the schedule, no stopping rule */
    int precision;         /* otgb_precision; OTGB_TC_BF16X3 only for D >= 16 */
    /* Optional warm start (device, caller order), used as the initial values of the
       four vectors when non-null; the schedule then starts at eps_start. */
    const float *f_init, *g_init, *a_init, *b_init;
    double sigma_start;    /* <= 0: the full schedule from the diameter */
    int translation;       /* unbalanced only: 1 = after every full-resolution step, move (f, g) to
                              (f + c, -c + g) with c = (rho/2) log(<alpha, e^{-f/rho}> / <beta, e^{-g/rho}>),
                              the exact dual ascent along the one direction the averaged loop contracts
                              slowly (rate (1 + lambda)/2); the fixed point is unchanged (c = 0 there).
                              0 = the paper's loop unchanged.  Default 1. */
    int anderson;          /* > 0: Anderson acceleration with this history length (<= 8) of the steps at
                              sigma = blur (Walker & Ni 2011); the fixed point is unchanged.  0: off.
                              Default 5. */
    int rows_per_thread;   /* D <= 3 kernel tuning: rows per thread (1, 2 or 4; a block holds 128 x this many
                              rows); 0 = automatic (4 dense, 2 multiscale). */
    int init_g_from_f;     /* 1 with f_init and no g_init: g starts as one plain softmin of f at the first
                              scale, g_j = -lam eps log sum_i alpha_i exp((f_i - C(x_i, y_j)) / eps), instead
                              of 0.  Default 0. */
    int warm_max_iters;    /* sinkhorn_divergence_warm: step budget of the warm attempt before it falls
                              back to the plain solve; <= 0: max_iters.  Default 0. */
    int debug_wait_probe;  /* test hook of the bounded-wait error path: 1 = the solve also runs one device
                              wait on a word that nothing writes; it gives up after about a millisecond,
                              flags the error word that the tensor-core and tile waits use, and the solve
                              (whose outputs are still written) returns OTGB_ETIMEOUT.  Nothing faults or
                              hangs and the context stays usable.  0 = off (default). */
    int polish;            /* D > 3 only: 1 = once the stopping rule holds, run the loop at blur again, to the
                              same rule, with every softmin in the direct difference form of the cost
                              (sum of squared coordinate differences, FP32 CUDA cores, about twice the work
                              per pair).  The fast forms add terms as large as the spread of a row block
                              times the distance of a column, whose rounding, amplified along the slowly
                              contracting bundle modes of unbalanced problems, leaves the duals a few 1e-5
                              from the fixed point on multi-bundle fiber problems while S is exact to ~1e-8;
                              the polish brings the duals to the float32 level.  0 = off (default). */
} otgb_params;

/* Statistics of one solve (host struct, filled when non-null). */
typedef struct {
    int iters_total;         /* averaged steps, all phases */
    int iters_coarse;        /* steps on the cluster measures */
    int iters_fine;          /* steps at full resolution */
    int n_clusters_x, n_clusters_y;
    int schedule_len;
    double diameter;
    double sigma_switch;
    double pairs_evaluated;  /* (i,j) terms computed by softmin kernels, all instances */
    double pairs_dense;      /* (N^2 + M^2 + 2NM) per fine step, summed over fine steps */
    double kept_fraction;    /* last fine step: evaluated / dense pairs */
    double softmin_ms;       /* device time of the softmin kernels (CUDA events) */
    double total_ms;         /* device time of the whole solve */
    double last_delta;       /* last max |new - old| / eps over the four vectors */
    double last_rel_change;  /* last estimated remaining relative change of S */
    long long fallback_rows; /* rows recomputed by the safe two-pass kernel */
    int warm_start;          /* sinkhorn_divergence_warm: 1 = the warm attempt converged, 2 = it fell back to
                                the plain solve (the other fields then describe the plain solve); 0 otherwise */
    int warm_iters;          /* steps spent in the warm attempt */
    double warm_ms;          /* device time of the warm attempt and the network's inference */
    /* device time of the phases of the solve (CUDA events; they add up to total_ms): */
    double prep_ms;          /* validation, bounding box, clustering (grid or k-means), reordering and packing */
    double coarse_ms;        /* coarse solve on the cluster measures and the extrapolation softmin */
    double fine_ms;          /* full-resolution steps: truncation masks, softmin sweeps, translation,
                                Anderson mixing and the convergence checks */
    double final_ms;         /* final FP64 sums of Eq. (6), outputs in the caller's order, finiteness checks */
} otgb_stats;

/* Fill *p with defaults: p = 2, blur = 0.05, reach = 0 (balanced), scaling = 0.5,
   multiscale = 0, cluster = GRID, kmeans_iters = 10, trunc_tau = 27.6, tol = 1e-6,
   min_iters = 3, max_iters = 100000, check_every = 10, precision = FP32, translation = 1,
   anderson = 5. */
void otgb_default_params(otgb_params *p);

/* Create a context on `device` that enqueues work on `cuda_stream`
   (a cudaStream_t; NULL: the legacy default stream).  *out receives the handle. */
int otgb_create(otgb_ctx **out, int device, void *cuda_stream);
/* Release the context and all its scratch memory. */
int otgb_destroy(otgb_ctx *ctx);
/* Last error message of the context (static storage when ctx is NULL). */
const char *otgb_last_error(const otgb_ctx *ctx);

/*
 * Debiased Sinkhorn divergence S_{eps,rho}(alpha, beta), Eq. (5) evaluated in
 * its dual form Eq. (6), with the symmetric, averaged, eps-scaled loop of the
 * Algorithm in Section 2 and, when params->multiscale = 1, the coarse-to-fine
 * strategy of Section 2 (clustering, coarse solve, extrapolation of the duals
 * by one softmin, kernel truncation of negligible cluster pairs).
 *
 *   x: N x D points, a: N weights (>= 0, positive total); y: M x D, b: M.
 *   cost_host (host, required): receives S in double precision.
 *   f (N), g (M): device outputs, the dual pair (f, g) = (b^{beta->alpha},
 *     a^{alpha->beta}) of OT(alpha, beta), in the caller's point order.
 *   a_self (N), b_self (M): optional device outputs, the symmetric duals of
 *     OT(alpha, alpha) and OT(beta, beta).
 *   plan_out: optional; receives a plan for transport_apply (free it with
 *     otgb_plan_free).  The plan keeps NON-OWNING views of x, y and b: they must
 *     stay valid until the plan is freed.
 *   stats: optional host struct.
 * Errors: EINVAL for N or M < 1, D outside [1, 64], p not in {1, 2}, blur <= 0, q outside
 * (0,1), negative or non-finite weights or a zero total mass; ENOCONV when
 * max_iters ends the loop first (outputs are written); ENONFINITE when a
 * potential turns NaN/Inf; ECUDA/ENOMEM from the runtime.
 */
int sinkhorn_divergence(otgb_ctx *ctx, const float *x, const float *a, int N, const float *y, const float *b,
                        int M, int D, const otgb_params *params, double *cost_host, float *f, float *g,
                        float *a_self, float *b_self, otgb_plan **plan_out, otgb_stats *stats);

/*
 * Label transfer through the smooth plan, Eq. (7):
 *   Lab_il = sum_{j : labels_j = l} b_j exp((f_i + g_j - C(x_i, y_j)) / eps),
 * eps = blur^p of the plan, i.e. (1/alpha_i)(pi l)_i with pi of Eq. (4).
 *   f (N), g (M): device duals in the caller's order (normally the ones
 *     sinkhorn_divergence wrote); labels: M int32 in [0, L) (others ignored).
 *   scores: N x L float32 (optional), argmax: N int32 (lowest class on ties;
 *     -1 when the row is empty), row_mass: N float32 = sum_l Lab_il (optional).
 * A row whose mass is near 0 is an outlier (Section 2, label transfer).
 * The sum runs over all atlas points (dense), for any 1 <= D <= 64.
 * Errors: EINVAL for a null plan, a plan of a p = 1 solve, L < 1 or L > 1024, null f/g/labels/argmax.
 */
int transport_apply(otgb_ctx *ctx, const otgb_plan *plan, const float *f, const float *g, const int32_t *labels,
                    int L, float *scores, int32_t *argmax, float *row_mass);
void otgb_plan_free(otgb_plan *plan);

/*
 * Flip augmentation of a fiber tractogram (Section 2, fiber encoding: fibers
 * resampled to P points are points of R^{3P}; their orientation is arbitrary,
 * so the tractogram is augmented with the mirror flip of every fiber).
 *   x: N x 3P device (fiber i = its P points (x, y, z) in order).
 *   out: 2N x 3P device output: rows 0..N-1 are the fibers, row N + i is fiber
 *   i with its points in reverse order (each point unchanged).
 * Solve and transfer labels on the augmented rows (weights: one per row),
 * then pick one version per fiber with otgb_select_flips.
 * Errors: EINVAL for null pointers, N < 1, P < 1 or 3P > 64.
 */
int otgb_flip_fibers(otgb_ctx *ctx, const float *x, int N, int P, float *out);

/*
 * The matched version of each fiber after transport_apply on flip-augmented
 * rows (Section 2, label transfer: the plan on the augmented data matches one
 * version of each fiber, and only that one is kept): of rows i and N + i, the
 * one with the larger row mass (ties: the original).
 *   row_mass (2N), argmax (2N): transport_apply's outputs on the 2N rows (device).
 *   label (N, required), version (N, optional; 0 = original, 1 = flip),
 *   mass (N, optional; the kept row mass, for outlier detection): device outputs.
 * Errors: EINVAL for null required pointers or N < 1.
 */
int otgb_select_flips(otgb_ctx *ctx, const float *row_mass, const int32_t *argmax, int N, int32_t *label,
                      int32_t *version, float *mass);

/*
 * Grid clustering (coarse subsampling, Section 2): cell coordinate
 * floor((x_d - min_d x) / cell) per axis, evaluated in IEEE single precision;
 * cells ordered by their Morton (bit-interleaved) key; points stably sorted by
 * key.  D <= 3; at most 1024 cells per axis.
 *   labels (N): cluster of each point (caller order).  perm (N): sorted position
 *   -> original index.  offsets (capacity N+1): cluster k holds sorted positions
 *   [offsets[k], offsets[k+1]).  n_clusters (host): number of clusters.
 *   centroids (optional, capacity N x D): weighted mean of each cluster, with
 *   weights w (optional, device, N; NULL = uniform).
 * Errors: EINVAL for D > 3, cell <= 0, or more than 1024 cells along an axis.
 */
int cluster_grid(otgb_ctx *ctx, const float *x, const float *w, int N, int D, float cell, int32_t *labels,
                 int32_t *perm, int32_t *offsets, int *n_clusters, float *centroids);

/*
 * Weighted K-means (Lloyd), the "simple K-means" of Section 2: K initial
 * centroids sampled without replacement from x with a seeded generator, then
 * `iters` rounds of nearest-centroid assignment and weighted-mean update (an
 * empty cluster keeps its centroid), then a final assignment.  Points are then
 * stably sorted by cluster.
 *   labels (N), centroids (K x D), perm (N), offsets (K+1).  w optional (NULL =
 *   uniform).  init (optional, device K x D) replaces the seeded sample.
 * Errors: EINVAL for K < 1, K > N, D outside [1, 64].
 */
int cluster_kmeans(otgb_ctx *ctx, const float *x, const float *w, int N, int D, int K, int iters,
                   unsigned long long seed, const float *init, int32_t *labels, float *centroids, int32_t *perm,
                   int32_t *offsets);

/*
 * Gradient of the debiased divergence in the points of the first measure
 * (Section 2, "Unbiased Sinkhorn divergences": at the fixed point the
 * gradients of S are expressions of the dual vectors).  With
 * G(u, v) = grad_u C(u, v) = u - v for p = 2 and (u - v) / |u - v| for p = 1
 * (0 at u = v):
 *   grad_i = alpha_i [ sum_j beta_j  exp((f_i + g_j - C(x_i, y_j)) / eps) G(x_i, y_j)
 *                    - sum_k alpha_k exp((a_i + a_k - C(x_i, x_k)) / eps) G(x_i, x_k) ]
 * = dS_{eps,rho}(alpha, beta) / dx_i, with (f, g) the dual pair of
 * OT(alpha, beta) and a the symmetric dual of OT(alpha, alpha) that
 * sinkhorn_divergence wrote (f, g, a_self; caller order) at eps = blur^p.
 * The gradient in y is the same call with the measures exchanged:
 * (y, beta, M, x, alpha, N, ..., f := g, g := f, a_self := b_self).
 *   x: N x D, alpha: N, y: M x D, beta: M, f: N, g: M, a_self: N (device);
 *   grad: N x D device output (float32).
 * Dense: every pair is summed (the direct difference form of the cost, FP32,
 * with a running maximum per row), for any 1 <= D <= 64.
 * Errors: EINVAL for null pointers, sizes < 1, D outside [1, 64], p not in {1, 2}, eps <= 0.
 */
int sinkhorn_grad_x(otgb_ctx *ctx, const float *x, const float *alpha, int N, const float *y, const float *beta,
                    int M, int D, int p, double eps, const float *f, const float *g, const float *a_self,
                    float *grad);

/*
 * Free-support Wasserstein barycenter (Section 2, "Track density atlas"):
 * minimises (1/K) sum_k S_{eps,rho}(alpha, beta_k) over the points x of alpha
 * (weights fixed) by `iters` steps of
 *   x_i <- x_i - lr (1/alpha_i) (1/K) sum_k dS(alpha, beta_k)/dx_i,
 * each gradient computed at the end of a solve of sinkhorn_divergence with
 * *params (after the first step every solve starts at blur from the previous
 * step's four duals).  The gradient is the expression of sinkhorn_grad_x.  In
 * a coarse-to-fine solve it is summed over the kept cluster pairs of the
 * solve's last truncation; each dropped term is below e^-tau of its row's
 * total.  With p = 2, lr = 1 and without the debiasing term, this is the
 * classical fixed-point update x_i <- mean_k of the barycentric projections.
 *   x: N x D device, updated in place; alpha: N device.
 *   ys, betas: HOST arrays of K device pointers (M_k x D points, M_k weights);
 *   Ms: host array of the K sizes.
 *   S_hist: optional host output of iters + 1 values, the objective
 *   (1/K) sum_k S(alpha, beta_k) before each step and after the last one.
 * Errors: those of sinkhorn_divergence, EINVAL for K < 1, iters < 0, lr <= 0.
 */
int sinkhorn_barycenter(otgb_ctx *ctx, float *x, const float *alpha, int N, int K, const float *const *ys,
                        const float *const *betas, const int *Ms, int D, const otgb_params *params, int iters,
                        double lr, double *S_hist);

/*
 * One softmin sweep of the Algorithm in Section 2, exposed for testing and for
 * custom loops:
 *   out_i = -lam * eps * log sum_k w_k exp((pot_k - C(p_k, q_i)) / eps)
 * for rows q (n_out x D) and columns p (n_in x D) with weights w (n_in) and
 * potential pot (n_in), dense.  When old is non-null the result is blended:
 *   out_i <- old_i + omega (out_i - old_i)   (omega = 1/2 is the paper's average).
 * Errors: EINVAL for sizes < 1, D outside [1, 64], eps <= 0.
 */
int otgb_softmin(otgb_ctx *ctx, const float *q, int n_out, const float *p, const float *w, const float *pot,
                 int n_in, int D, double eps, double lam, const float *old, double omega, float *out);

/*
 * otgb_softmin_noalloc: the same sweep as otgb_softmin, for callers that may
 * not allocate device memory.  The paper has no counterpart: this entry point
 * exists for integration only.
 *
 * Who needs it: code that runs where a device allocation is not allowed or
 * not wanted -- a host that gives a component a fixed memory budget and owns
 * every allocation itself (a serving process with a preallocated arena, an
 * embedded pipeline), code inside a latency-critical loop where an allocation
 * could stall on the driver, or a caller that has no otgb_ctx (which owns
 * allocated scratch).  This call needs no context and calls no cudaMalloc,
 * cudaFree or allocating library routine: its scratch is one fixed, file-scope
 * device array of 16 MiB that every GPU which loads the library holds until
 * the process exits.
 *
 *   q: n_out x D rows, p: n_in x D columns, w: n_in weights, pot: n_in
 *   potential, old (optional), out: n_out -- device pointers owned by the
 *   caller, as in otgb_softmin (same arguments, same result).
 *   cuda_stream: the cudaStream_t to run on (NULL: the legacy default stream).
 *   The call returns when the result is complete on that stream.
 * Limits and errors: EINVAL when the scratch of the problem exceeds 16 MiB --
 * about 32 n_out + 16 n_in bytes for D <= 3 (at most about 349,000 rows and
 * 349,000 columns when n_out = n_in), and
 * 4 round_up(D, 4) (n_out + n_in) + 4 n_in + 16 n_out bytes for D > 3, plus
 * about 34 KB in both cases -- and for the argument errors of otgb_softmin;
 * the message is available from otgb_last_error(NULL).
 * The first call on a device looks up the device address of the scratch
 * array (cudaGetSymbolAddress, with that device current); make that first
 * call before any stream capture.  Every call on a device shares the one
 * array, so calls that overlap on the GPU (from several host threads or
 * streams at once) race and must be serialised by the caller; the array keeps
 * the last call's contents, and every piece that must start at zero is
 * cleared by the call itself.
 */
int otgb_softmin_noalloc(const float *q, int n_out, const float *p, const float *w, const float *pot, int n_in,
                         int D, double eps, double lam, const float *old, double omega, float *out,
                         void *cuda_stream);

/*
 * Warm-start network (an addition; the paper has no learned component).  A
 * multilayer perceptron f(x) = out_mean + out_scale * MLP((x - in_mean) / in_scale),
 * D -> H -> H -> H -> 1 with SiLU activations, learns the subject-side dual f of
 * the transport problem against one fixed atlas from potentials the solver
 * produced; sinkhorn_divergence_warm uses it only as the initial f at the final
 * temperature, and the Sinkhorn iterations decide the result.
 *
 * Arithmetic: every layer is a tensor-core GEMM with BF16 operands (weights,
 * activations, gradients of the pre-activations) and FP32 accumulation; biases,
 * the head, the loss and the Adam state are FP32; the master weights are FP32.
 * Flat parameter vector (n_params floats, FP32): W1 (H x D, row-major, rows =
 * outputs), b1 (H), W2 (H x H), b2, W3 (H x H), b3, W4 (1 x H), b4 (1).
 * Loss: L = (1/2n) sum_i ((MLP_i - (f_i - out_mean)) / out_scale)^2, i.e. half the
 * mean squared error in normalised units.  Adam: beta1 = 0.9, beta2 = 0.999,
 * eps = 1e-8, with bias correction (Kingma & Ba 2015).
 * The network belongs to one context and runs on its stream; it owns its
 * device memory until otgb_mlp_destroy.
 */
typedef struct otgb_mlp otgb_mlp;

/* D in [1, 64], hidden in {128, 256}; weights uniform in +-sqrt(6/fan_in)
   (head +-sqrt(3/H)) from `seed`, biases 0, identity normalisation. */
int otgb_mlp_create(otgb_ctx *ctx, int D, int hidden, unsigned long long seed, otgb_mlp **out);
int otgb_mlp_destroy(otgb_mlp *mlp);
/* Number of FP32 parameters (or -1 for a null handle). */
int otgb_mlp_n_params(const otgb_mlp *mlp);
/* Normalisation from data: per-feature mean and standard deviation of x (n x D,
   device) and of f (n, device; NULL keeps the output normalisation).  A feature
   with zero spread gets scale 1. */
int otgb_mlp_fit_normalization(otgb_mlp *mlp, const float *x, const float *f, int n);
/* host arrays of D floats; scales > 0 */
int otgb_mlp_set_normalization(otgb_mlp *mlp, const float *in_mean, const float *in_scale, double out_mean,
                               double out_scale);
int otgb_mlp_get_normalization(const otgb_mlp *mlp, float *in_mean, float *in_scale, double *out_mean,
                               double *out_scale);
/* Host copy of the FP32 master parameters (n must equal n_params).  set also
   clears the Adam state. */
int otgb_mlp_set_params(otgb_mlp *mlp, const float *theta_host, int n);
int otgb_mlp_get_params(const otgb_mlp *mlp, float *theta_host, int n);
/* Loss (host, optional) and its gradient (device, n_params floats) over the n
   rows (x: n x D, f: n, device), 1 <= n <= 65536.  No update. */
int otgb_mlp_grad(otgb_mlp *mlp, const float *x, const float *f, int n, double *loss, float *grad);
/* One Adam update with a caller-supplied gradient (device, n_params floats). */
int otgb_mlp_adam_step(otgb_mlp *mlp, const float *grad, float lr);
/* otgb_mlp_grad on the n rows followed by one Adam update; loss optional (host). */
int otgb_mlp_train_step(otgb_mlp *mlp, const float *x, const float *f, int n, float lr, double *loss);
/* One pass over n rows in a seeded random order, batches of `batch` rows
   (128 <= batch <= 65536; the last batch may be smaller), one Adam update per
   batch.  mean_loss (host, optional): the row-weighted mean of the batch losses. */
int otgb_mlp_train_epoch(otgb_mlp *mlp, const float *x, const float *f, int n, int batch, float lr,
                         unsigned long long seed, double *mean_loss);
/* out (device, n) = f(x) in data units; x: n x D device. */
int otgb_mlp_infer(otgb_mlp *mlp, const float *x, int n, float *out);
/* Binary file: header (magic "OTGBMLP1", D, H, n_params, Adam step, normalisation)
   then FP32 parameters and Adam moments.  load requires matching D and H. */
int otgb_mlp_save(const otgb_mlp *mlp, const char *path);
int otgb_mlp_load(otgb_mlp *mlp, const char *path);

/*
 * Warm-started solve: f0 = network(x); the solve then starts at sigma = blur with
 * f = f0, g = one plain softmin of f0 (init_g_from_f), b = b_atlas when given (the
 * atlas' own symmetric dual from an earlier solve against the same y and b; it
 * depends on y and b only) and a = 0, and iterates the averaged loop at blur
 * with the stopping rule of sinkhorn_divergence.  When that attempt ends with
 * ENOCONV (params->warm_max_iters steps), ENONFINITE or ETIMEOUT, the plain
 * solve with *params runs instead.  Arguments and outputs as in
 * sinkhorn_divergence; mlp must belong to ctx and have D inputs.  stats->warm_start
 * tells which path produced the outputs.
 */
int sinkhorn_divergence_warm(otgb_ctx *ctx, otgb_mlp *mlp, const float *x, const float *a, int N, const float *y,
                             const float *b, int M, int D, const otgb_params *params, const float *b_atlas,
                             double *cost_host, float *f, float *g, float *a_self, float *b_self,
                             otgb_plan **plan_out, otgb_stats *stats);

/*
 * Measured per-SM, per-clock throughput of the units that bound the softmin
 * kernels (the denominators of their rooflines; the paper has no counterpart):
 * lane operations per clock per SM of MUFU ex2 (ex2.approx.ftz.f32), scalar
 * FP32 FMA and packed FP32x2 FMA (two lane operations each), from short
 * dependency-chain kernels timed with the SM cycle counter on the context's
 * device.  All three outputs are host doubles.
 */
int otgb_unit_rates(otgb_ctx *ctx, double *ex2_per_clk_sm, double *fma_per_clk_sm, double *fma2_per_clk_sm);

/* Number of CUDA kernels this library has launched in this process (all
   contexts), for accounting by benchmarks. */
unsigned long long otgb_kernel_launches(void);

#ifdef __cplusplus
}
#endif
#endif /* OTGB_H */
