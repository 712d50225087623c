/*
 * wos.h -- C ABI of the GB300 Walk-on-Spheres library (libwos.so).
 *
 * Walk on Spheres (WoS) estimates, at batches of query points x in a d-dimensional
 * configuration space, the solution u of the screened Poisson problem
 *
 *     Laplace(u) = sigma u   in Omega,        u = g   on the boundary of Omega
 *
 * (Sec. III, Eq. screened_poisson_wos, with the paper's c written sigma and f = 0) and its
 * spatial gradient grad u, which the gradient-following planner consumes at every step
 * (Sec. III, screened-harmonic paths; Sec. VII adaptive step).
 *
 * Estimators (Sec. IV-A):
 *   one walk:   u^(x_k) = g(xbar_k) once x_k is closer than eps to the boundary (xbar_k is the
 *               closest boundary point, Fig. 2), else C(R_k) u^(x_{k+1}) with x_{k+1} uniform on
 *               the largest empty sphere of radius R_k around x_k;
 *   normaliser: C(R) = (z/2)^nu / (Gamma(nu+1) I_nu(z)),  z = R sqrt(sigma),  nu = d/2 - 1;
 *   gradient:   grad^ = alpha(R_0) u^(x_1) v_0 with v_0 the first direction. The paper prints
 *               the Laplace factor d/R_0; for sigma > 0 the unbiased factor is
 *               alpha(R_0) = (d/R_0) C_{nu+1}(z_0), which this library uses unless
 *               WOS_FLAG_LAPLACE_FACTOR is set.
 * The walk geometry does not depend on sigma, so d u^/d sigma = u^ sum_k d log C(R_k)/d sigma
 * per walk is exact; for g = sum_k w_k exp(a_k . x), d u^/d w_k = prod C * exp(a_k . xbar).
 *
 * Conventions for every call:
 *   - Pointers named "device" are device pointers owned by the caller; "host" pointers are read
 *     during the call only. The library owns only what wos_domain_create / wos_batch_create
 *     allocate, and frees it in the matching destroy call.
 *   - Every call that takes a stream is asynchronous on that stream (a cudaStream_t passed as
 *     void*; NULL is the legacy default stream). Outputs are valid when the stream reaches the
 *     point of the call.
 *   - Every call returns a wos_status; the library never aborts or exits. wos_last_error()
 *     gives a thread-local one-line detail of the last failure.
 *   - A query point with no positive distance to the boundary (not in the open domain) gets
 *     NaN outputs and is counted in wos_stats.outside; the other queries still complete, and
 *     the call returns WOS_OK.
 *   - In WOS_MIXED the per-query sums are FP64 and formed in a fixed order, so repeated calls
 *     with the same inputs give the same outputs bit for bit. Every walk leaves a record of
 *     rec = 4 + K (+ d for gradient walks) floats, rounded up to a multiple of four (16 to 96
 *     bytes), in device scratch that the call allocates (Q * n_walks records), and one CTA per
 *     query and segment of 4096 walks sums them.
 *   - Random directions: Philox4x32-10 (Salmon et al., SC'11) with key = seed and counter =
 *     (walk_lo, walk_hi, step, block). Walk w of query q has the global index
 *     walk_offset + q * n_walks + w, so results are a pure function of (seed, index, step).
 */
#ifndef WOS_H
#define WOS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    WOS_OK = 0,
    WOS_ERR_INVALID_ARG = 1,   /* a size, pointer or value is out of range; nothing was launched */
    WOS_ERR_UNSUPPORTED = 2,   /* valid request this build does not implement (e.g. d > 12) */
    WOS_ERR_OOM = 3,           /* a device or host allocation failed */
    WOS_ERR_CUDA = 4,          /* a CUDA runtime call failed; see wos_last_error() */
    WOS_ERR_TIMEOUT = 5,       /* a device-side iteration budget ran out (status word set) */
    WOS_ERR_OUTSIDE_DOMAIN = 6 /* reserved for callers that treat outside queries as errors */
} wos_status;

typedef enum {
    WOS_FP64 = 0,       /* FP64 walkers, direct FP64 log-Bessel series per step (parity mode) */
    WOS_FP32_PLAIN = 1, /* one thread per walk, FP32 direct Bessel series, FP32 per-query sums */
    WOS_MIXED = 2       /* FP32 persistent walkers, FP64-built weight tables, FP64 per-query sums */
} wos_precision;

#define WOS_FLAG_LAPLACE_FACTOR 1 /* use the paper's printed gradient factor d/R0 */

/*
 * Control variate for the first-sphere gradient (gradient calls only: wos_grad, the planner,
 * gradient batches). The paper's estimator averages y_w = G t_w v_w over the N walks of a
 * query, with t_w the walk's value estimate, v_w its first direction and G = alpha(R0)/C(R0)
 * (R0 = distance at the query, so G is one number per query). Because E[v_w] = 0, subtracting
 * the sample mean tbar of the t_w changes nothing in expectation but removes the part of the
 * noise that the level of u contributes:
 *
 *     grad^ = G / (N - 1) * sum_w (t_w - tbar) v_w     (unbiased for N >= 2: it is G times the
 *                                                       sample covariance of t and v)
 *     grad_se = N/(N-1) * sqrt(var_w(G (t_w - tbar) v_w) / N)
 *
 * Walks capped at max_steps (t_w = 0) take part with their first direction. This is a
 * variance reduction in the spirit of the paper's closing discussion (Sec. IX), not an
 * estimator the paper prints. Cost: 3d more FP64 sums per query, and in mixed precision the
 * first direction of every walk is kept in its record (d floats). With N = 1 the plain estimate
 * is returned. Value-only calls ignore the flag.
 */
#define WOS_FLAG_GRAD_CONTROL_VARIATE 2

/*
 * Ball sets of at least 96 (d <= 4), 160 (d = 5..9) or 128 (d = 10..12) balls run, in WOS_MIXED,
 * on the tensor-core sphere-set walker (the same walker as point sets: |c|^2 - 2 x.c by
 * tcgen05.mma, exact FP32 refinement of the best 16-ball chunk -- 32-ball for sets of 8192 or
 * more in d <= 8 --, a proven lower bound for the rest). This flag keeps them on the CUDA-core
 * ball screen instead (for comparisons; both are exact up to their error bounds).
 */
#define WOS_FLAG_CUDA_CORE_BALLS 4

/*
 * Antithetic first directions (variance reduction of the paper's closing discussion, Sec. IX;
 * not an estimator the paper prints): the walks pair up by global walk index (2m, 2m + 1), and
 * walk 2m + 1 starts along the negated first direction of walk 2m (its own directions after).
 * Every direction is still uniform, so every estimate stays unbiased; standard errors come from
 * the spread of the N/2 pair means. Requires n_walks and walk_offset even (batches: every
 * problem's n_walks even); not combined with WOS_FLAG_GRAD_CONTROL_VARIATE (INVALID_ARG).
 */
#define WOS_FLAG_ANTITHETIC 8

#define WOS_MAX_D 12    /* dimensions 2..12 are supported */
#define WOS_MAX_EXP 8   /* at most 8 exponential boundary-data terms */

typedef struct wos_domain_s *wos_domain_t;
typedef struct wos_batch_s *wos_batch_t;

/*
 * Domain description (all host pointers, FP64, read during wos_domain_create only).
 * Omega = {inside the box, if any} and {inside the outer ball, if any}, minus the closed ball
 * obstacles, minus the goal ball, minus the point set. At least one of box / outer ball is
 * required so that every walk can terminate.
 * Distance to the boundary (Sec. VI, Eq. for d(x, dOmega); Sec. VII-A point-set distance):
 *   balls |x - c| - r, goal |x - c_g| - r_g, outer r_o - |x - c_o|, points |x - p|,
 *   box faces x_j - lo_j and hi_j - x_j; the minimum over all components.
 * Boundary data g: if n_exp > 0, g(x) = sum_k exp_w[k] exp(exp_a[k] . x) on the whole boundary;
 * otherwise g = 1 on the goal sphere and 0 on every other component (the planning field).
 */
typedef struct {
    int32_t d;                  /* dimension, 2..WOS_MAX_D */
    const double *box_lo;       /* d values, or NULL for no box */
    const double *box_hi;       /* d values, or NULL */
    const double *outer_c;      /* d values, or NULL for no outer ball */
    double outer_r;             /* > 0 when outer_c is given */
    const double *goal_c;       /* d values, or NULL for no goal */
    double goal_r;              /* > 0 when goal_c is given */
    int32_t n_balls;            /* >= 0 ball obstacles */
    const double *ball_c;       /* n_balls x d, row major */
    const double *ball_r;       /* n_balls radii, > 0 */
    int64_t n_points;           /* >= 0 obstacle points (point-cloud C-space, Sec. VII-A) */
    const double *points;       /* n_points x d, row major */
    int32_t n_exp;              /* 0..WOS_MAX_EXP exponential data terms */
    const double *exp_w;        /* n_exp weights */
    const double *exp_a;        /* n_exp x d exponents */
    const double *source_z;     /* d values: an impulse source at this point, or NULL for none */
    double source_q;            /* its strength q (the paper's unit impulse at the goal: 1) */
    int32_t proj_dims;          /* 0 or d: plain domain; 1..d-1: extruded (see below) */
    int32_t n_links;            /* 0, or 1..d: a planar arm in configuration space (see below) */
    const double *link_l;       /* n_links link lengths, > 0 */
    int64_t n_arm_obs;          /* >= 1 with an arm: task-space obstacle points */
    const double *arm_obs;      /* n_arm_obs x 2, row major */
    double sigma_max;           /* >= 0: build the WOS_MIXED weight tables for every sigma up to
                                   this one at creation (0: each on first use; see below) */
} wos_domain_desc;

/*
 * Weight tables (WOS_MIXED): log C_nu(z) and S_{nu+1}/S_nu(z), built in FP64 on the fixed grid
 * z_i = i / 1024 (linear interpolation), so a walk's weights depend on z = R sqrt(sigma) alone.
 * A domain needs the grid up to the smallest power of two 2^level >= sqrt(sigma) times its
 * largest distance (level <= 12; UNSUPPORTED beyond); a table of a higher level serves every
 * lower one. With sigma_max > 0, wos_domain_create builds the table for sigma_max, and no call
 * with sigma <= sigma_max allocates or waits for one. Otherwise the first WOS_MIXED call that
 * needs a larger table allocates it with cudaMalloc (8 KB times 2^level) and builds it on its
 * own stream (no host wait); calls on other streams wait for that build on the device. The
 * synchronous calls (wos_plan_path, wos_plan_paths, wos_batch_create) wait for it on the host.
 */

/*
 * Planar arm in configuration space (Sec. V, V-A; the RR validation of Sec. VII): the first
 * n_links coordinates are the joint angles of a planar chain with its base at the origin (link i
 * along the sum of the angles 0..i, length link_l[i]). The arm's collisions with the task-space
 * obstacle points are a boundary component known only implicitly; its distance is the safe-ball
 * radius d_tau(q) / K (Eq. safe_ball), d_tau the task-space distance between the links and the
 * points and K = sqrt(sum_n (sum_{i<=n} l_i)^2) the Lipschitz constant of the forward
 * kinematics -- a lower bound of the configuration-space distance, so every sphere stays
 * collision-free. A walk ending in its eps-shell reads g at its own position (the nearest
 * boundary point is not known). Component order: goal, balls, points, arm, outer ball, faces.
 * Mixed precision runs such domains on the CUDA-core walker for d <= 8 with at most 32
 * obstacle points (UNSUPPORTED beyond, and with a point set); FP64 and plain FP32 take any.
 */

/*
 * Impulse source (Sec. IV-A estimator with a source term; the paper's planning problems put a
 * unit impulse at the goal, Sec. VI, VII): with source_z given, u solves
 * Laplace(u) - sigma u = -q delta(x - source_z) in Omega, u = g on the boundary (g = 0 when the
 * domain has neither a goal ball nor exponential data, the paper's zero Dirichlet condition).
 * Each step whose largest empty ball B(x_k, R_k) contains the source adds q G_B(x_k, source_z)
 * times the walk's weight so far, G_B the Green's function of that ball with zero boundary
 * values (Yukawa potential minus its image part; logarithm / power laws at sigma = 0); the
 * first-sphere gradient adds q grad_x G_B(x_0, source_z). du_dsigma differentiates each walk's
 * value (the walk geometry does not depend on sigma): each source contribution adds q times the
 * weight so far times dG_B/dsigma plus G_B times the d log C / d sigma of the steps before
 * (dG_B/dsigma from the Bessel derivative identities, DLMF 10.29.2; at sigma = 0 from the
 * first-order term of G_B in sigma); du_dw is unaffected. Every walker has the source term
 * (the tensor-core sphere-set walker too: point sets and large ball sets).
 */

/*
 * Extruded domains (Sec. VI, dimensionality study: the obstacles and the outer boundary are
 * extruded along the added dimensions, which are free and unbounded): with 1 <= proj_dims = m < d,
 * every component is measured in the first m coordinates only (balls |P(x - c)| - r, goal,
 * outer |P(x - c_o)|, box faces in coordinates 0..m-1; the box's other coordinates are ignored).
 * Walks, directions, the impulse source and the boundary data stay d-dimensional; the closest
 * boundary point keeps the free coordinates of x. A box or an outer ball in the first m
 * coordinates still bounds every walk. Mixed precision runs such domains on the CUDA-core walker
 * (ball sets) and rejects extruded point sets (UNSUPPORTED).
 */

/*
 * Per-call options. A NULL options pointer means {WOS_MIXED, 0, seed 0, offset 0, 10000, 0, 0}.
 *
 * Russian roulette on the weight (roulette_w > 0; the closing discussion's roulette on C,
 * Sec. IX; no rule is printed): before jump k >= 1 of a walk whose weight W = prod C(R_i) is
 * below roulette_w, the walk survives with probability W / roulette_w and then carries the
 * weight roulette_w, or ends with its impulse-source contributions so far and no boundary value
 * (counted in wos_stats.killed). E[kept weight] = W keeps every estimate unbiased, and du/dsigma
 * stays pathwise unbiased. The uniform is the top 24 bits of Philox block 15 of (walk, k) times
 * 2^-24. Walks get shorter where the screening makes weights small (large sigma).
 */
typedef struct {
    int32_t precision;   /* wos_precision */
    int32_t flags;       /* WOS_FLAG_* */
    uint64_t seed;       /* Philox key */
    int64_t walk_offset; /* first global walk index of this call */
    int64_t max_steps;   /* jumps per walk before it is capped (contributes 0); <= 0: 10000;
                            below 2^28 in WOS_MIXED */
    double roulette_w;   /* > 0: Russian roulette below this weight; 0: off */
    int64_t wait_cycles; /* tensor-core sphere-set walker: SM clock cycles one wait of its main
                            loop may take before the launch gives up (see below); <= 0: 4e9
                            (~2 s) */
} wos_options;

/*
 * Failure detection. The tensor-core sphere-set walker's threads wait on each other through
 * shared-memory barriers (copies landed, products ready, accumulators read). Every wait is
 * bounded: one that takes more than wait_cycles SM clock cycles sets the launch's status word,
 * and every thread leaves through the same teardown, which first waits (up to 4e9 cycles each,
 * whatever wait_cycles is) for the products and copies already issued and then frees the
 * tensor memory. Such a call's outputs are NaN and wos_stats.timeouts is nonzero; the
 * asynchronous calls report it only there, wos_plan_path and wos_plan_paths return
 * WOS_ERR_TIMEOUT (the planner step flag is 16). The device stays usable: the next call runs
 * normally. A small wait_cycles makes a healthy launch give up (how failures are tested).
 */

/* Counters of one call, written to DEVICE memory when the stream completes (int64, exact). */
typedef struct {
    int64_t walks;           /* walks run (= Q * n_walks) */
    int64_t walk_steps;      /* distance evaluations (a walk with k jumps counts k + 1) */
    int64_t capped;          /* walks that hit max_steps */
    int64_t outside;         /* walks whose query was not in the open domain */
    int64_t shrinks;         /* tensor-core walker steps whose radius was set by a chunk bound */
    int64_t killed;          /* walks ended by the Russian roulette (wos_options.roulette_w) */
    int64_t timeouts;        /* nonzero: a tensor-core walker wait ran out (outputs NaN) */
} wos_stats;

/* ---- domain ------------------------------------------------------------------------- */

/* Copies the description to the device (FP64 and FP32 copies; BF16 split copies of the point
 * set). Synchronous. Errors: INVALID_ARG (bad sizes, radii <= 0, no box or outer ball),
 * UNSUPPORTED (d outside 2..12, n_exp > 8), OOM, CUDA. *out is NULL on failure. */
wos_status wos_domain_create(const wos_domain_desc *desc, wos_domain_t *out);

/* Frees everything the domain owns. Synchronises the device first. NULL is accepted. */
wos_status wos_domain_destroy(wos_domain_t dom);

/* Replaces the boundary-data weights exp_w (n_exp device doubles) on the stream, for the
 * autograd path where w is a learnable tensor. Errors: INVALID_ARG if n differs from n_exp. */
wos_status wos_domain_set_exp_w(wos_domain_t dom, const double *w_device, int32_t n, void *stream);

/*
 * Which walker the domain's obstacles run on in WOS_MIXED: *tensor_sphere_set = 1 if they form a
 * tensor-core sphere set (a point set, or a ball set of at least 96, 160 or 128 balls for
 * d <= 4, d = 5..9, d = 10..12), with *sphere_tiles
 * 64-sphere tiles; 0 (and 0 tiles) for the CUDA-core walker. Host outputs; either may be NULL.
 * No counterpart in the paper (introspection for schedulers and benchmarks).
 * Errors: INVALID_ARG (NULL domain).
 */
wos_status wos_domain_info(wos_domain_t dom, int32_t *tensor_sphere_set, int32_t *sphere_tiles);

/* ---- estimators (Sec. IV-A) --------------------------------------------------------- */

/*
 * u at Q query points: x is Q x d device doubles (row major); u and u_se (standard error of the
 * mean, may be NULL) are Q device doubles. stats: one device wos_stats or NULL.
 * Errors: INVALID_ARG (NULL x/u with Q > 0, n_walks < 1, eps <= 0, sigma < 0), CUDA, OOM.
 */
wos_status wos_solve(wos_domain_t dom, const wos_options *opt, const double *x, int64_t Q,
                     int64_t n_walks, double eps, double sigma, double *u, double *u_se,
                     wos_stats *stats, void *stream);

/*
 * u and grad u at Q query points with gradient walks (the first sphere is always taken).
 * Device outputs, any of which may be NULL except grad: u, u_se (Q); grad, grad_se (Q x d);
 * du_dsigma (Q); du_dw (Q x n_exp). Errors as wos_solve.
 */
wos_status wos_grad(wos_domain_t dom, const wos_options *opt, const double *x, int64_t Q,
                    int64_t n_walks, double eps, double sigma, double *u, double *u_se,
                    double *grad, double *grad_se, double *du_dsigma, double *du_dw,
                    wos_stats *stats, void *stream);

/*
 * Per-walk instrumentation for parity checks: runs Q x n_walks walks (value walks if
 * grad_mode == 0, gradient walks otherwise) and writes, per walk j = q * n_walks + w, the
 * terminal estimate term[j], the number of jumps jumps[j] (int64), grad[j*d + i] and
 * dsigma[j] (device; any pointer may be NULL). Errors as wos_solve.
 */
wos_status wos_walks(wos_domain_t dom, const wos_options *opt, const double *x, int64_t Q,
                     int64_t n_walks, double eps, double sigma, int32_t grad_mode, double *term,
                     int64_t *jumps, double *grad, double *dsigma, void *stream);

/* ---- planner (Sec. III screened-harmonic path; Sec. VII s = min(s_ub, d_bound / 2)) ---- */

/*
 * One planner step on the device point x (d device doubles, updated in place): if x is within
 * eps of the goal, flag = 1 and x is kept; otherwise grad u is estimated with n_walks gradient
 * walks (walk offset opt->walk_offset + step_idx * n_walks) and x <- x + s grad/|grad| with
 * s = min(s_ub, d_bound(x) / 2); flag = 2 if |grad| = 0 (x kept), 4 if x is outside, 16 if a
 * tensor-core walker wait ran out (x kept; the path stops).
 * flag: one device int32; grad_out: d device doubles or NULL. Errors as wos_solve.
 */
wos_status wos_plan_step(wos_domain_t dom, const wos_options *opt, double *x, int64_t n_walks,
                         double eps, double sigma, double s_ub, int64_t step_idx, int32_t *flag,
                         double *grad_out, void *stream);

/*
 * n_steps planner steps from x0 (d device doubles), recorded and replayed as one CUDA graph.
 * Synchronous (it records and replays the graph, then waits for the stream).
 * path: (n_steps + 1) x d device doubles (row 0 = x0; rows after the goal repeat the last
 * point); flags: n_steps device int32 (as wos_plan_step; 8 marks steps after the goal);
 * grads: n_steps x d device doubles or NULL. Errors as wos_solve.
 */
wos_status wos_plan_path(wos_domain_t dom, const wos_options *opt, const double *x0,
                         int64_t n_steps, int64_t n_walks, double eps, double sigma, double s_ub,
                         double *path, int32_t *flags, double *grads, void *stream);

/*
 * Many planner paths in one CUDA graph (the paper's multistart paths, Sec. VI Fig. 5; paths of
 * uneven d and domains): step i of every path is one batched launch -- each path's gradient
 * walks are one problem of the persistent walkers' work queues, as in wos_batch_create -- then
 * every path's step update on the device. A path that reaches its goal runs no more walks.
 * Path p is the path wos_plan_path gives for the same domain, options and arguments: the same
 * walks (walk offset opt->walk_offset + i n_walks at step i), the same per-query sums (formed in
 * the same fixed order) and so the same points, flags and gradients. WOS_MIXED only. Synchronous (it
 * records and replays the graph, then waits for the stream).
 */
typedef struct {
    wos_domain_t domain;
    const double *x0;   /* d device doubles: the start */
    int64_t n_walks;    /* gradient walks per step */
    double eps;
    double sigma;
    double s_ub;        /* the step bound of Sec. VII, s = min(s_ub, d_bound / 2) */
    double *path;       /* (n_steps + 1) x d device doubles (row 0 = x0) */
    int32_t *flags;     /* n_steps device int32 (as wos_plan_step; 8 after the goal) */
    double *grads;      /* n_steps x d device doubles or NULL */
} wos_path_problem;

wos_status wos_plan_paths(const wos_path_problem *paths, int32_t n_paths, int64_t n_steps,
                          const wos_options *opt, void *stream);

/* ---- backward of u(x; sigma, w) (autograd) --------------------------------------------- */

/*
 * Given the upstream gradient gout (Q device doubles) and the saved forward estimates grad
 * (Q x d), du_dsigma (Q, or NULL) and du_dw (Q x K, or NULL): gx[q*d+i] = gout[q] grad[q*d+i];
 * gsigma[0] = sum_q gout[q] du_dsigma[q]; gw[k] = sum_q gout[q] du_dw[q*K+k]. FP64 sums in a
 * fixed order (deterministic). All device pointers; gx/gsigma/gw may be NULL.
 */
wos_status wos_backward(const double *gout, const double *grad, const double *du_dsigma,
                        const double *du_dw, int64_t Q, int32_t d, int32_t K, double *gx,
                        double *gsigma, double *gw, void *stream);

/* ---- batched uneven problems in one persistent launch --------------------------------- */

typedef struct {
    wos_domain_t domain;
    const double *x;  /* n_queries x d device doubles */
    int64_t n_queries;
    int64_t n_walks;  /* walks per query */
    double eps;
    double sigma;
    double *u;        /* n_queries device doubles */
    double *u_se;     /* n_queries device doubles or NULL */
    double *grad;     /* n_queries x d device doubles or NULL (NULL: value walks) */
    double *grad_se;  /* n_queries x d device doubles or NULL */
    int64_t *walk_steps; /* n_queries device int64 or NULL: distance evaluations per query */
} wos_problem;

/* Launch shapes of the persistent kernels. A NULL config means "autotuned": the cached best for
 * this device and problem mix if any, else the built-in default. */
typedef struct {
    int32_t threads;            /* CUDA-core walker: threads per CTA, 32..768, multiple of 32 */
    int32_t ctas_per_sm;        /* CUDA-core walker: resident CTAs per SM requested (1..8) */
    int64_t item_work;          /* CUDA-core walker: target work per queue item (ball-dimension units) */
    int32_t sphere_ctas_per_sm; /* tensor-core walker: CTAs per SM in its persistent grids (1..4) */
    int32_t reserved;           /* 0 */
    int64_t sphere_item_walks;  /* tensor-core walker: walks per queue item (128..2^20, multiple of 128) */
} wos_batch_config;

/*
 * Builds a batch: uploads the problem table and the longest-first work queues, sizes the
 * persistent grids to a multiple of the SM count, and records one CUDA graph: [reset, the
 * CUDA-core persistent walker for the problems with small ball sets, in parallel one
 * tensor-core sphere-set walker launch per dimension and set size class (below 24 tiles of 64
 * spheres, 24 or more, 32-column sets) for the problems with tensor-core sphere sets (large ball sets or a point set; WOS_FLAG_CUDA_CORE_BALLS keeps ball sets off it), the
 * per-query reduction of the walks' records, finalize]. Problems may differ in d, obstacle
 * count, walk budget, sigma and eps. Precision is WOS_MIXED. The problems' domains and buffers
 * must outlive the batch; the batch holds a record of 16 to 96 bytes per walk (see below).
 * Errors: INVALID_ARG, UNSUPPORTED (a domain with both balls and points), OOM, CUDA.
 */
wos_status wos_batch_create(const wos_problem *probs, int32_t n_problems, const wos_options *opt,
                            const wos_batch_config *cfg, wos_batch_t *out);

/* Replays the batch graph on the stream; stats (device) may be NULL. */
wos_status wos_batch_run(wos_batch_t batch, wos_stats *stats, void *stream);

/* Reads back the launch shape in use (host struct). */
wos_status wos_batch_get_config(wos_batch_t batch, wos_batch_config *cfg);

/* Frees the batch (synchronises the device). NULL is accepted. */
wos_status wos_batch_destroy(wos_batch_t batch);

/* One-shot convenience: create, run, destroy. */
wos_status wos_solve_batch(const wos_problem *probs, int32_t n_problems, const wos_options *opt,
                           wos_stats *stats, void *stream);

/*
 * Autotuner: times candidate launch shapes on this batch (CUDA events, one run each after a
 * warm-up run) in two rounds -- the CUDA-core walker's shapes (threads, CTAs per SM, item work),
 * then, with the best of those, the tensor-core walker's (CTAs per SM in {4, 3, 2}, walks per
 * item in {2048, 4096, 8192}) -- keeps the fastest in the batch, and appends it to the text cache
 * file cache_path (may be NULL) keyed by device name and problem-mix signature, so later
 * wos_batch_create calls with a NULL config reuse it. best (host) may be NULL. Synchronous.
 */
wos_status wos_batch_autotune(wos_batch_t batch, const char *cache_path, wos_batch_config *best);

/* Sets the cache file consulted by wos_batch_create when cfg is NULL (NULL: no cache). */
wos_status wos_set_autotune_cache(const char *cache_path);

/* ---- allocation-free estimate ------------------------------------------------------------- */

#define WOS_NOALLOC_SCRATCH_BYTES (1u << 20) /* static device scratch of wos_solve_noalloc */

/*
 * wos_solve_noalloc: the estimate of wos_solve (u and its standard error per query) for
 * callers that cannot allocate device memory inside a call -- a control loop with a hard
 * deadline, where cudaMalloc/cudaFree can block on the driver's device-wide allocator and
 * synchronise the GPU, or a host application that has handed the device memory to its own
 * pool and forbids allocations from libraries. The paper has no counterpart: this is a
 * property of the library interface, not of the method.
 * It allocates nothing: the caller passes x, u, u_se and stats as for wos_solve, and the
 * per-query FP64 sums and counters live in one static device array of
 * WOS_NOALLOC_SCRATCH_BYTES (1 MiB) that every GPU which loads the library holds until the
 * process exits. Each query needs e (3 + 2d + n_exp) + 32 bytes of it, e = 8 for WOS_FP64 and
 * 4 for WOS_FP32_PLAIN: about 10900 queries for d = 2 with one exponential term in FP64, 3360
 * for d = 12 with eight.
 * Precision: WOS_FP64 or WOS_FP32_PLAIN (the one-thread-per-walk walker); WOS_MIXED needs its
 * weight table, which is allocated, and is rejected.
 * Each call looks up the device address of the array (cudaGetSymbolAddress, which allocates
 * nothing) with the caller's device current, so the address is never stale after a device reset.
 * Each call clears the array on its stream and then reuses it, and the array keeps the last call's contents:
 * calls whose work overlaps on the GPU (other streams, other host threads) race on it and
 * must be serialised by the caller.
 * Errors: as wos_solve; INVALID_ARG if Q exceeds the limit; UNSUPPORTED for WOS_MIXED.
 */
wos_status wos_solve_noalloc(wos_domain_t dom, const wos_options *opt, const double *x, int64_t Q,
                             int64_t n_walks, double eps, double sigma, double *u, double *u_se,
                             wos_stats *stats, void *stream);

/* ---- diagnostics ------------------------------------------------------------------------ */

const char *wos_status_string(wos_status s);
const char *wos_last_error(void);

/* Writes the library's log C_nu(z) and S_{nu+1}/S_nu tables as seen by the FP32 walkers for
 * dimension d over z in [0, z_max] (n nodes each, host doubles), for table-accuracy tests. */
wos_status wos_debug_weight_table(int32_t d, double z_max, int32_t n, double *log_c,
                                  double *ratio);

/* Writes the Philox4x32-10 blocks the walkers draw for walks walk0 .. walk0 + n - 1 at the given
 * step and block: out[4 i + c] (device uint32, n x 4), key = seed, counter =
 * (walk_lo, walk_hi, step, block). For bitwise checks of the random-stream contract. */
wos_status wos_debug_philox(uint64_t seed, uint64_t walk0, int64_t n, uint32_t step,
                            uint32_t block, uint32_t *out, void *stream);

/* Writes, for each point x[q] (Q x d device doubles), the distance bound the tensor-core
 * point-cloud walker uses there -- min over the FP32 refinement of its best candidate chunk (16
 * or 32 points), the second-best chunk minus the BF16 error bound, and the other components -- to
 * radius[q] (device doubles). Sec. VII-A point-set distance (and Sec. VI ball distance for a
 * tensor-core ball set); for checks that the bound never exceeds the exact distance.
 * Errors: UNSUPPORTED without a tensor-core sphere set. */
wos_status wos_debug_pointcloud_radius(wos_domain_t dom, const double *x, int64_t Q, double *radius,
                                       void *stream);

#ifdef __cplusplus
}
#endif

#endif /* WOS_H */
