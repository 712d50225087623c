/*
 * Walk on Spheres for the screened Poisson equation -- plain FP64 CPU oracle.
 *
 * TEST INFRASTRUCTURE ONLY. Only the test suite, the package's smoke check and
 * the benchmark's CPU-baseline / reference legs may load this library. It shares
 * no code, header, table or constant generator with the CUDA path, and it never
 * calls it. It is deliberately slow and written for reading against the paper:
 *
 *   PDE (Sec. III, Eq. screened_poisson_wos with c = sigma):  Laplace(u) = sigma u in Omega,
 *       u = g on the boundary.  f = 0 (no source term).
 *   One-point estimator (Sec. IV-A, recursive estimator):     u^(x_k) = g(xbar_k)  if x_k is within
 *       eps of the boundary, else C(x_k) u^(x_{k+1}), x_{k+1} uniform on the largest empty sphere.
 *   Normaliser C (Sec. IV-A, "depends on dimension and radius"):
 *       C_nu(z) = (z/2)^nu / (Gamma(nu+1) I_nu(z)),  z = R sqrt(sigma),  nu = d/2 - 1.
 *   First-sphere gradient (Sec. IV-A, gradient estimator):   grad^ = alpha(R0) u^(x_1) v(x_1).
 *       The paper prints the Laplace factor n/R; for sigma > 0 the unbiased factor is
 *       alpha = (d/R0) C_{nu+1}(z0) (it reduces to d/R0 at sigma = 0). The literal factor is
 *       available through or_options.laplace_factor.
 *   Control variate for the gradient (optional; a variance reduction in the spirit of Sec. IX,
 *       not an estimator the paper prints): with t_w the value estimate of walk w, v_w its first
 *       direction and G = alpha(R0)/C(R0), grad^ = G/(N-1) sum_w (t_w - tbar) v_w, tbar the
 *       sample mean of the t_w. E[v] = 0 makes it unbiased for every N >= 2 (G times the sample
 *       covariance of t and v). Computed here by its definition, in two passes over stored
 *       per-walk values.
 *   Impulse source (Sec. IV-A estimator with a source term; Sec. VI and VII: a unit impulse at
 *       the goal): for Laplace(u) - sigma u = -q delta_z, each step whose ball B(x_k, R_k)
 *       contains z adds q G_B(x_k, z) times the product of the C(R_i), i < k, where G_B is the
 *       Green's function of the ball with zero boundary values, evaluated between its centre and
 *       z; the first-sphere gradient adds q grad_x G_B(x_0, z). With r = |z - x|, k = sqrt(sigma),
 *       nu = d/2 - 1 and c0 = k^nu / (2 pi)^(d/2):
 *         G_B = c0 r^-nu [K_nu(k r) - K_nu(k R) I_nu(k r) / I_nu(k R)],
 *         grad_x G_B = (z - x)/r c0 k r^-nu [K_nu+1(k r) - K_nu+1(k R) I_nu+1(k r) / I_nu+1(k R)],
 *       and at sigma = 0: G_B = (r^(2-d) - R^(2-d)) / ((d-2) |S^(d-1)|) (ln(R/r)/(2 pi) for d = 2),
 *       grad_x G_B = (z - x)/|S^(d-1)| (r^-d - R^-d). K_nu from its integral
 *       int_0^inf exp(-x cosh t) cosh(nu t) dt (DLMF 10.32.9) by the trapezoidal rule.
 *       du/dsigma per walk (the walk geometry does not depend on sigma): the boundary part times
 *       the summed d log C / d sigma, plus, for each source contribution, q times the weight so
 *       far times (dG_B/dsigma + G_B times the d log C / d sigma of the steps before); dG_B/dsigma
 *       from the Bessel derivative identities (sigma > 0) and from the first-order term of G_B in
 *       sigma (sigma = 0), see or_ball_green_dsigma.
 *   Closest boundary point xbar (Fig. 2): g is read at the projection of x_k on the nearest
 *       boundary component.
 *   Planner (Sec. III screened-harmonic paths; Sec. VII adaptive step):
 *       x <- x + s grad/|grad|,  s = min(s_ub, 0.5 d_bound).
 *   Distance functions (Sec. VI, Eq. for d(x, dOmega); Sec. VII-A point-set distance):
 *       balls: |x - c| - r;  outer ball: r_o - |x - c_o|;  points: |x - p|;  box faces;
 *       a planar arm in configuration space (Sec. V, V-A): the safe-ball radius d_tau(q) / K,
 *       d_tau the task-space distance between the links and obstacle points, K the Lipschitz
 *       constant of the forward kinematics; a walk ending there reads g at its own position.
 *   Boundary data g (Sec. III, u = g on the boundary): the goal indicator of the planning
 *       field, sum_k w_k exp(a_k . x), and two forms used only by the closed-form pins: a
 *       polynomial sum_m c_m prod_j x_j^p_mj (harmonic ones solve sigma = 0 exactly) and one
 *       constant per box face (the unit square with g = 1 on one edge).
 *   Russian roulette on the weight (optional; the closing discussion's "Russian roulette on C"
 *       variance/cost trade-off, not an estimator the paper prints): before each jump k >= 1
 *       whose weight W = prod C is below w_min, the walk survives with probability W / w_min
 *       and then carries the weight w_min, or ends with its source contributions so far and no
 *       boundary value. E[kept weight] = W keeps u unbiased; the pathwise du/dsigma
 *       (term times the summed d log C / dsigma) stays unbiased because the survival
 *       probability's sigma-derivative is the summed d log C / dsigma up to that step. The
 *       uniform is the top 24 bits of Philox block 15 of (walk, step k), times 2^-24.
 *   Antithetic first directions (optional; the closing discussion's variance reduction): the
 *       walks of a query pair up (2m, 2m+1 of the global index, so walk_offset and N must be
 *       even); walk 2m+1 takes the negated first direction of walk 2m, later steps their own.
 *       Each direction stays uniform, so every estimate is unbiased; standard errors come from
 *       the spread of the N/2 pair means. Not combined with the control variate.
 *   Extruded domains (Sec. VI, dimensionality study): with proj_dims = m < d every boundary
 *       component is measured in the first m coordinates only (the obstacles and the outer
 *       boundary extruded along the others, which are free and unbounded); walks, sources and
 *       boundary data stay d-dimensional, and the closest boundary point keeps the free
 *       coordinates of x.
 *
 * Readings where the paper is silent (random stream, ties, caps) follow the build's
 * documented contract:
 *   - sphere directions: Philox4x32-10 (Salmon et al., SC'11), key = seed, counter =
 *     (walk_lo, walk_hi, step, block); Box-Muller on consecutive output pairs;
 *   - strict eps test (R < eps); ties between components go to the first in the order
 *     [goal, balls, points, arm, outer ball, box faces lo_0, hi_0, lo_1, ...];
 *   - a walk that reaches max_steps jumps without entering the eps shell contributes 0.
 *
 * Log-Bessel: S_mu(z) = Gamma(mu+1) (z/2)^-mu I_mu(z) = sum_k (z^2/4)^k / (k! (mu+1)_k)
 * (DLMF 10.25.2), summed directly; log C_nu(z) = -log S_nu(z).
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_MAXD 16
#define OR_PI 3.14159265358979323846
#define OR_MAXEXP 16
#define OR_CHUNK 256 /* walks per partial sum; fixed so results do not depend on threads */

#define OR_KIND_GOAL 0
#define OR_KIND_BALL 1
#define OR_KIND_POINT 2
#define OR_KIND_OUTER 3
#define OR_KIND_FACE 4
#define OR_KIND_ARM 5

typedef struct {
    int32_t d;
    int32_t has_box;
    double box_lo[OR_MAXD];
    double box_hi[OR_MAXD];
    int32_t has_outer;
    double outer_c[OR_MAXD];
    double outer_r;
    int32_t has_goal;
    double goal_c[OR_MAXD];
    double goal_r;
    int32_t n_balls;
    const double *ball_c; /* n_balls x d, row major */
    const double *ball_r; /* n_balls */
    int64_t n_points;
    const double *points; /* n_points x d */
    int32_t n_exp;        /* >0: g(x) = sum_k w_k exp(a_k . x) on the whole boundary */
    const double *exp_w;  /* n_exp */
    const double *exp_a;  /* n_exp x d */
    int32_t has_source;   /* 1: impulse source of strength source_q at source_z */
    double source_z[OR_MAXD];
    double source_q;
    int32_t proj_dims;    /* 0 or d: distances in all coordinates; m < d: in the first m only */
    int32_t n_poly;       /* >0 (and n_exp = 0): g(x) = sum_m poly_c[m] prod_j x_j^poly_p[m d + j] */
    const double *poly_c; /* n_poly coefficients */
    const int32_t *poly_p; /* n_poly x d exponents */
    int32_t has_face_g;   /* 1 (no exp or poly data): g = face_g[2j] on face lo_j, face_g[2j+1] on hi_j */
    double face_g[2 * OR_MAXD];
    int32_t n_links;      /* > 0: planar arm of n_links revolute joints, angles q_0..q_{n_links-1} */
    double link_l[OR_MAXD]; /* link lengths */
    int64_t n_arm_obs;    /* task-space obstacle points of the arm (planar) */
    const double *arm_obs; /* n_arm_obs x 2 */
} or_domain;

typedef struct {
    uint64_t seed;
    int64_t max_steps;
    int32_t grad;           /* 1: gradient walks (the first sphere is always taken) */
    int32_t laplace_factor; /* 1: the paper's printed factor d/R0 instead of alpha(R0) */
    int32_t control_variate; /* 1 (with grad): the control-variate gradient of or_solve */
    int32_t plant_free_space_source_grad; /* test only: drop the ball's image term in grad G_B */
    double roulette_w;      /* > 0: Russian roulette when the weight falls below it */
    int32_t plant_roulette_no_reweight; /* test only: survivors keep their weight */
    int32_t antithetic;     /* 1: walk 2m+1 takes the negated first direction of walk 2m */
} or_options;

typedef struct {
    double term;   /* u^ for this walk */
    int64_t jumps; /* sphere jumps k; distance evaluations = k + 1 */
    int32_t capped;
    int32_t outside;
    int32_t killed; /* ended by the roulette */
    int32_t comp_kind;
    int64_t comp_index;
    double grad[OR_MAXD];
    double dsigma;
    double dw[OR_MAXEXP];
    double gv0[OR_MAXD]; /* G v0 = alpha(R0)/C(R0) times the first direction, if k > 0; else 0 */
    double gsrc[OR_MAXD]; /* source part of the gradient, q grad_x G_B(x0, z) (0 without a source) */
} or_walk_out;

/* ------------------------------------------------------------------------- */
/* Philox4x32-10, from the definition in Salmon, Moraes, Dror, Shaw (SC'11):  */
/* 10 rounds of two 32x32->64 multiplies, Weyl key schedule.                  */
/* ------------------------------------------------------------------------- */
void or_philox4x32_10(const uint32_t key[2], const uint32_t ctr[4], uint32_t out[4])
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u; /* round multipliers */
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u; /* key increments    */
    uint32_t k0 = key[0], k1 = key[1];
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += W0;
            k1 += W1;
        }
        uint64_t p0 = (uint64_t)M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)M1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
    }
    out[0] = c0;
    out[1] = c1;
    out[2] = c2;
    out[3] = c3;
}

/* d standard normals for (walk, step): block b uses counter (walk_lo, walk_hi, step, b);
 * outputs (r0, r1) and (r2, r3) feed Box-Muller with u1 = (r + 1) 2^-32 in (0, 1] and
 * u2 = r 2^-32 in [0, 1). */
void or_normals(uint64_t seed, uint64_t walk, uint32_t step, int d, double *n)
{
    const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    const double two_m32 = 1.0 / 4294967296.0;
    const double two_pi = 6.283185307179586476925286766559;
    int nblocks = (d + 3) / 4;
    for (int b = 0; b < nblocks; ++b) {
        uint32_t ctr[4] = {(uint32_t)walk, (uint32_t)(walk >> 32), step, (uint32_t)b};
        uint32_t r[4];
        or_philox4x32_10(key, ctr, r);
        for (int pair = 0; pair < 2; ++pair) {
            double u1 = ((double)r[2 * pair] + 1.0) * two_m32;
            double u2 = (double)r[2 * pair + 1] * two_m32;
            double rad = sqrt(-2.0 * log(u1));
            int i0 = 4 * b + 2 * pair;
            if (i0 < d) n[i0] = rad * cos(two_pi * u2);
            if (i0 + 1 < d) n[i0 + 1] = rad * sin(two_pi * u2);
        }
    }
}

/* Uniform direction on the unit sphere: v = n / |n| (e_0 if |n| = 0). */
void or_direction(uint64_t seed, uint64_t walk, uint32_t step, int d, double *v)
{
    double n[OR_MAXD + 4];
    or_normals(seed, walk, step, d, n);
    double ss = 0.0;
    for (int j = 0; j < d; ++j) ss += n[j] * n[j];
    if (ss > 0.0) {
        double norm = sqrt(ss);
        for (int j = 0; j < d; ++j) v[j] = n[j] / norm;
    } else {
        for (int j = 0; j < d; ++j) v[j] = 0.0;
        v[0] = 1.0;
    }
}

/* ------------------------------------------------------------------------- */
/* Normaliser: S_mu(z) = sum_k (z^2/4)^k / (k! (mu+1)_k)   (DLMF 10.25.2)     */
/* ------------------------------------------------------------------------- */
double or_series_S(double mu, double z)
{
    double q = 0.25 * z * z;
    double term = 1.0, sum = 1.0;
    for (int k = 1; k < 5000; ++k) {
        term *= q / ((double)k * (mu + (double)k));
        sum += term;
        if (term <= 1e-17 * sum) break;
    }
    return sum;
}

/* log C_nu(z), C_nu(z) = (z/2)^nu / (Gamma(nu+1) I_nu(z)) = 1 / S_nu(z). Valid for z < ~700. */
double or_log_C(double nu, double z) { return -log(or_series_S(nu, z)); }

/* K_nu(x), x > 0: the integral int_0^inf exp(-x cosh t) cosh(nu t) dt (DLMF 10.32.9) by the
 * trapezoidal rule. The integrand is even and analytic in the strip |Im t| < pi/2; relative to
 * its size on the real line it grows like exp(x y^2 / 2) at height y, so the rule's relative
 * error is about exp(-2 pi^2 / (h^2 x)): a step min(1/8, 0.6/sqrt(x)) keeps it below 1e-23.
 * The sum stops once the terms are negligible. */
double or_bessel_K(double nu, double x)
{
    const double h = x > 23.04 ? 0.6 / sqrt(x) : 0.125;
    double sum = 0.5 * exp(-x);
    for (int i = 1; i < 1000000; ++i) {
        const double t = h * (double)i;
        const double c = x * cosh(t);
        const double term = 0.5 * (exp(nu * t - c) + exp(-nu * t - c));
        sum += term;
        if (c - nu * t > 50.0 && term < 1e-20 * sum) break;
    }
    return h * sum;
}

/* Ball Green's function (zero boundary values on the sphere of radius R) between the centre
 * and a point at distance r, 0 < r < R, for Laplace(u) - sigma u = -delta; *F is the factor
 * with grad_x G_B(x, y) = F (y - x) / r at the centre x. free_space: drop the image part of F
 * (a planted mistake for the tests). */
void or_ball_green(int d, double sigma, double r, double R, int free_space, double *G, double *F)
{
    const double nu = 0.5 * d - 1.0;
    const double omega = 2.0 * pow(OR_PI, 0.5 * d) / tgamma(0.5 * d); /* |S^(d-1)| */
    if (sigma == 0.0) {
        *G = d == 2 ? log(R / r) / (2.0 * OR_PI) : (pow(r, 2.0 - d) - pow(R, 2.0 - d)) / ((d - 2.0) * omega);
        *F = (pow(r, 1.0 - d) - (free_space ? 0.0 : r * pow(R, -(double)d))) / omega;
        return;
    }
    const double k = sqrt(sigma);
    const double c0 = pow(k, nu) / pow(2.0 * OR_PI, 0.5 * d);
    /* I_mu(k r) / I_mu(k R) = (r/R)^mu S_mu(k r) / S_mu(k R) (DLMF 10.25.2) */
    const double ratio0 = pow(r / R, nu) * or_series_S(nu, k * r) / or_series_S(nu, k * R);
    const double ratio1 = pow(r / R, nu + 1.0) * or_series_S(nu + 1.0, k * r) / or_series_S(nu + 1.0, k * R);
    *G = c0 * pow(r, -nu) * (or_bessel_K(nu, k * r) - or_bessel_K(nu, k * R) * ratio0);
    *F = c0 * k * pow(r, -nu) *
         (or_bessel_K(nu + 1.0, k * r) - (free_space ? 0.0 : or_bessel_K(nu + 1.0, k * R) * ratio1));
}

/* d/dsigma of G_B (or_ball_green) between the centre and a point at distance r, 0 < r < R.
 * sigma > 0: with k = sqrt(sigma), c0 = k^nu / (2 pi)^(d/2) and A(k) = K_nu(kr) - K_nu(kR) Q(k),
 * Q = I_nu(kr) / I_nu(kR), G = c0 r^-nu A, so dG/dk = (nu/k) G + c0 r^-nu A'(k), using
 * K_nu'(x) = -K_{nu+1}(x) + (nu/x) K_nu(x) (DLMF 10.29.2) and I_nu'(x) / I_nu(x) =
 * I_{nu+1}(x) / I_nu(x) + nu/x with I_{nu+1}(x) / I_nu(x) = x S_{nu+1}(x) / (2 (nu+1) S_nu(x))
 * (DLMF 10.29.2, 10.25.2); dG/dsigma = (dG/dk) / (2k).
 * sigma = 0: G = G_0 - sigma w + O(sigma^2), where w solves -Laplace(w) = G_0 in the ball with
 * w = 0 on the sphere (differentiate Laplace(G) - sigma G = -delta in sigma); G_0 is radial,
 * so w is the radial solution of (rho^(d-1) w')' = -rho^(d-1) G_0(rho), integrated twice. */
double or_ball_green_dsigma(int d, double sigma, double r, double R)
{
    const double nu = 0.5 * d - 1.0;
    const double omega = 2.0 * pow(OR_PI, 0.5 * d) / tgamma(0.5 * d);
    if (sigma == 0.0) {
        if (d == 2) return (0.25 * r * r * log(R / r) + 0.25 * (r * r - R * R)) / (2.0 * OR_PI);
        if (d == 4) return (-0.5 * log(R / r) - r * r / (8.0 * R * R) + 0.125) / (2.0 * omega);
        const double a = 1.0 / (2.0 * (4.0 - d)), b = 1.0 / (2.0 * d);
        return (a * pow(r, 4.0 - d) - b * r * r * pow(R, 2.0 - d) - (a - b) * pow(R, 4.0 - d)) / ((d - 2.0) * omega);
    }
    const double k = sqrt(sigma);
    const double c0 = pow(k, nu) / pow(2.0 * OR_PI, 0.5 * d);
    const double Ka0 = or_bessel_K(nu, k * r), Ka1 = or_bessel_K(nu + 1.0, k * r);
    const double Kb0 = or_bessel_K(nu, k * R), Kb1 = or_bessel_K(nu + 1.0, k * R);
    const double Sa0 = or_series_S(nu, k * r), Sa1 = or_series_S(nu + 1.0, k * r);
    const double Sb0 = or_series_S(nu, k * R), Sb1 = or_series_S(nu + 1.0, k * R);
    const double Q = pow(r / R, nu) * Sa0 / Sb0;
    const double A = Ka0 - Kb0 * Q;
    const double dQ = Q * k / (2.0 * (nu + 1.0)) * (r * r * Sa1 / Sa0 - R * R * Sb1 / Sb0);
    const double dA = -r * Ka1 + (nu / k) * Ka0 - Q * (-R * Kb1 + (nu / k) * Kb0) - Kb0 * dQ;
    const double dGdk = c0 * pow(r, -nu) * ((nu / k) * A + dA);
    return dGdk / (2.0 * k);
}

/* d/dsigma log C_nu(R sqrt(sigma)) = -(R^2 / (2d)) S_{nu+1}(z) / S_nu(z), d = 2 nu + 2. */
double or_dsigma_log_C(double nu, double R, double sigma)
{
    double z = R * sqrt(sigma);
    double d = 2.0 * nu + 2.0;
    return -(R * R / (2.0 * d)) * or_series_S(nu + 1.0, z) / or_series_S(nu, z);
}

/* ------------------------------------------------------------------------- */
/* Distance to the boundary and closest boundary point (Sec. VI, VII-A).      */
/* ------------------------------------------------------------------------- */
static double norm_diff(int d, const double *a, const double *b)
{
    double s = 0.0;
    for (int j = 0; j < d; ++j) {
        double t = a[j] - b[j];
        s += t * t;
    }
    return sqrt(s);
}

/* Planar arm (Sec. V-A): base at the origin, joint angles q_0..q_{n-1} accumulated along the
 * chain, link i from the end of link i-1 along the summed angle with length l_i. d_tau(q) is the
 * task-space distance between the links (segments) and the obstacle points. */
double or_arm_task_distance(const or_domain *D, const double *q)
{
    double px = 0.0, py = 0.0, ang = 0.0, best = INFINITY;
    for (int n = 0; n < D->n_links; ++n) {
        ang += q[n];
        const double ex = px + D->link_l[n] * cos(ang), ey = py + D->link_l[n] * sin(ang);
        const double sx = ex - px, sy = ey - py, ss = sx * sx + sy * sy;
        for (int64_t o = 0; o < D->n_arm_obs; ++o) {
            const double ox = D->arm_obs[2 * o] - px, oy = D->arm_obs[2 * o + 1] - py;
            double t = ss > 0.0 ? (ox * sx + oy * sy) / ss : 0.0;
            if (t < 0.0) t = 0.0;
            if (t > 1.0) t = 1.0;
            const double dx = ox - t * sx, dy = oy - t * sy;
            const double r = sqrt(dx * dx + dy * dy);
            if (r < best) best = r;
        }
        px = ex;
        py = ey;
    }
    return best;
}

/* Lipschitz constant of the planar chain's forward kinematics (Sec. V-A):
 * K = sqrt(sum_n (sum_{i<=n} l_i)^2). */
double or_arm_lipschitz(const or_domain *D)
{
    double reach = 0.0, k2 = 0.0;
    for (int n = 0; n < D->n_links; ++n) {
        reach += D->link_l[n];
        k2 += reach * reach;
    }
    return sqrt(k2);
}

/* Coordinates the boundary components are measured in: the first m of d. */
static int obstacle_dims(const or_domain *D)
{
    return D->proj_dims > 0 && D->proj_dims < D->d ? D->proj_dims : D->d;
}

double or_distance(const or_domain *D, const double *x, int32_t *kind, int64_t *index,
                   double *xbar)
{
    const int d = D->d, m = obstacle_dims(D);
    double best = INFINITY;
    int32_t bk = -1;
    int64_t bi = -1;
    if (D->has_goal) {
        double r = norm_diff(m, x, D->goal_c) - D->goal_r;
        if (r < best) { best = r; bk = OR_KIND_GOAL; bi = 0; }
    }
    for (int32_t i = 0; i < D->n_balls; ++i) {
        double r = norm_diff(m, x, D->ball_c + (int64_t)i * d) - D->ball_r[i];
        if (r < best) { best = r; bk = OR_KIND_BALL; bi = i; }
    }
    for (int64_t i = 0; i < D->n_points; ++i) {
        double r = norm_diff(m, x, D->points + i * d);
        if (r < best) { best = r; bk = OR_KIND_POINT; bi = i; }
    }
    if (D->n_links > 0) {
        /* the safe-ball radius d_tau / K underestimates the C-space distance (Sec. V, Eq. safe_ball) */
        double r = or_arm_task_distance(D, x) / or_arm_lipschitz(D);
        if (r < best) { best = r; bk = OR_KIND_ARM; bi = 0; }
    }
    if (D->has_outer) {
        double r = D->outer_r - norm_diff(m, x, D->outer_c);
        if (r < best) { best = r; bk = OR_KIND_OUTER; bi = 0; }
    }
    if (D->has_box) {
        for (int j = 0; j < m; ++j) {
            double rlo = x[j] - D->box_lo[j];
            if (rlo < best) { best = rlo; bk = OR_KIND_FACE; bi = 2 * j; }
            double rhi = D->box_hi[j] - x[j];
            if (rhi < best) { best = rhi; bk = OR_KIND_FACE; bi = 2 * j + 1; }
        }
    }
    if (kind) *kind = bk;
    if (index) *index = bi;
    if (xbar) {
        /* projection of x on the nearest component (in the first m coordinates; the others are
           those of x) */
        const double *c = NULL;
        double rad = 0.0;
        if (bk == OR_KIND_GOAL) { c = D->goal_c; rad = D->goal_r; }
        if (bk == OR_KIND_BALL) { c = D->ball_c + bi * d; rad = D->ball_r[bi]; }
        if (bk == OR_KIND_OUTER) { c = D->outer_c; rad = D->outer_r; }
        for (int j = m; j < d; ++j) xbar[j] = x[j];
        if (c) {
            double len = norm_diff(m, x, c);
            for (int j = 0; j < m; ++j)
                xbar[j] = len > 0.0 ? c[j] + rad * (x[j] - c[j]) / len : c[j] + (j == 0 ? rad : 0.0);
        } else if (bk == OR_KIND_POINT) {
            for (int j = 0; j < m; ++j) xbar[j] = D->points[bi * d + j];
        } else if (bk == OR_KIND_ARM) {
            /* the arm's boundary point is not known (the distance is only bounded below): the walk
               ends where it is and reads g there */
            for (int j = 0; j < d; ++j) xbar[j] = x[j];
        } else if (bk == OR_KIND_FACE) {
            for (int j = 0; j < d; ++j) xbar[j] = x[j];
            int j = (int)(bi / 2);
            xbar[j] = (bi % 2 == 0) ? D->box_lo[j] : D->box_hi[j];
        } else {
            for (int j = 0; j < d; ++j) xbar[j] = x[j];
        }
    }
    return best;
}

/* Boundary data g at the closest boundary point (Sec. III: u = g on the boundary):
 *   exp data:        sum_k w_k exp(a_k . xbar) on the whole boundary;
 *   polynomial data: sum_m c_m prod_j xbar_j^p_mj on the whole boundary (harmonic polynomials
 *                    are exact solutions at sigma = 0);
 *   face data:       a constant per box face (the unit square with g = 1 on one edge), 1 on the
 *                    goal, 0 on other components;
 *   otherwise:       1 on the goal, 0 elsewhere (the planning field). */
static double boundary_g(const or_domain *D, int32_t kind, int64_t index, const double *xbar, double *dw)
{
    if (D->n_exp > 0) {
        double g = 0.0;
        for (int k = 0; k < D->n_exp; ++k) {
            double dot = 0.0;
            for (int j = 0; j < D->d; ++j) dot += D->exp_a[k * D->d + j] * xbar[j];
            double e = exp(dot);
            if (dw) dw[k] = e;
            g += D->exp_w[k] * e;
        }
        return g;
    }
    if (D->n_poly > 0) {
        double g = 0.0;
        for (int m = 0; m < D->n_poly; ++m) {
            double t = D->poly_c[m];
            for (int j = 0; j < D->d; ++j)
                for (int e = 0; e < D->poly_p[m * D->d + j]; ++e) t *= xbar[j];
            g += t;
        }
        return g;
    }
    if (D->has_face_g && kind == OR_KIND_FACE) return D->face_g[index];
    return kind == OR_KIND_GOAL ? 1.0 : 0.0;
}

/* ------------------------------------------------------------------------- */
/* One walk (Sec. IV-A).                                                      */
/* ------------------------------------------------------------------------- */
void or_walk(const or_domain *D, const double *x0, uint64_t walk, double eps, double sigma,
             const or_options *opt, or_walk_out *out)
{
    const int d = D->d;
    const double nu = 0.5 * d - 1.0;
    const double sq = sqrt(sigma);
    double x[OR_MAXD], xbar[OR_MAXD], v[OR_MAXD], v0[OR_MAXD];
    double logw = 0.0, dsig = 0.0, R0 = 0.0, z0 = 0.0, logC0 = 0.0;
    double src = 0.0, src0 = 0.0; /* source contributions: all steps, and step 0 alone */
    double dsrc = 0.0;            /* d/dsigma of the source contributions */
    int64_t k = 0;
    int32_t kind = -1;
    int64_t index = -1;
    memset(out, 0, sizeof(*out));
    for (int j = 0; j < d; ++j) x[j] = x0[j];
    for (;;) {
        double R = or_distance(D, x, &kind, &index, xbar);
        if (k == 0 && !(R > 0.0)) { /* query not in the open domain */
            out->outside = 1;
            out->term = NAN;
            out->dsigma = NAN;
            for (int j = 0; j < d; ++j) out->grad[j] = NAN;
            for (int q = 0; q < D->n_exp; ++q) out->dw[q] = NAN;
            return;
        }
        int in_shell = R < eps;
        if (in_shell && !(opt->grad && k == 0)) {
            double dw[OR_MAXEXP];
            double g = boundary_g(D, kind, index, xbar, dw);
            double w = exp(logw);
            out->term = g * w + src;
            for (int q = 0; q < D->n_exp; ++q) out->dw[q] = w * dw[q];
            break;
        }
        if (k == opt->max_steps) {
            out->capped = 1;
            out->term = 0.0;
            break;
        }
        if (opt->roulette_w > 0.0 && k > 0 && exp(logw) < opt->roulette_w) {
            const uint32_t key[2] = {(uint32_t)opt->seed, (uint32_t)(opt->seed >> 32)};
            const uint32_t ctr[4] = {(uint32_t)walk, (uint32_t)(walk >> 32), (uint32_t)k, 15u};
            uint32_t r[4];
            or_philox4x32_10(key, ctr, r);
            const double u = (double)(r[0] >> 8) * (1.0 / 16777216.0);
            if (u < exp(logw) / opt->roulette_w) {
                if (!opt->plant_roulette_no_reweight) logw = log(opt->roulette_w);
            } else {
                out->killed = 1;
                out->term = src; /* source contributions so far, no boundary value */
                break;
            }
        }
        if (D->has_source) {
            /* the ball B(x_k, R) contains the source: q G_B(x_k, z) times the weight so far */
            const double r = norm_diff(d, x, D->source_z);
            if (r > 0.0 && r < R) {
                double G, F;
                or_ball_green(d, sigma, r, R, opt->plant_free_space_source_grad, &G, &F);
                const double c = D->source_q * exp(logw) * G;
                src += c;
                /* its sigma derivative along the walk: the weight's (the sum of d log C / d sigma
                 * of the steps before) and the Green's function's */
                dsrc += D->source_q * exp(logw) * (dsig * G + or_ball_green_dsigma(d, sigma, r, R));
                if (k == 0) {
                    src0 = c;
                    for (int j = 0; j < d; ++j) out->gsrc[j] = D->source_q * F * (D->source_z[j] - x[j]) / r;
                }
            }
        }
        if (k == 0 && opt->antithetic) {
            or_direction(opt->seed, walk & ~(uint64_t)1, 0u, d, v);
            if (walk & 1)
                for (int j = 0; j < d; ++j) v[j] = -v[j];
        } else {
            or_direction(opt->seed, walk, (uint32_t)k, d, v);
        }
        double z = R * sq;
        double Snu = or_series_S(nu, z);
        double Snu1 = or_series_S(nu + 1.0, z);
        double logC = -log(Snu);
        if (k == 0) {
            R0 = R;
            z0 = z;
            logC0 = logC;
            for (int j = 0; j < d; ++j) v0[j] = v[j];
        }
        logw += logC;
        dsig += -(R * R / (2.0 * d)) * Snu1 / Snu;
        for (int j = 0; j < d; ++j) x[j] = x[j] + R * v[j];
        ++k;
    }
    out->jumps = k;
    out->comp_kind = kind;
    out->comp_index = index;
    /* d/dsigma of the walk's value: its boundary part times the summed d log C / d sigma, plus
     * the source contributions' derivatives (the walk geometry does not depend on sigma); a
     * capped walk contributes 0 */
    out->dsigma = out->capped ? 0.0 : (out->term - src) * dsig + dsrc;
    if (k > 0) {
        /* u^(x_1) = term / C(R0);  alpha(R0) = (d/R0) C_{nu+1}(z0);  G = alpha(R0) / C(R0) */
        double factor = opt->laplace_factor ? (double)d / R0
                                            : ((double)d / R0) / or_series_S(nu + 1.0, z0);
        double G = factor * exp(-logC0);
        for (int j = 0; j < d; ++j) out->gv0[j] = G * v0[j];
        /* u^(x_1) C(R0) = the walk's value without its step-0 source part */
        double u1 = out->capped ? 0.0 : (out->term - src0) * exp(-logC0);
        for (int j = 0; j < d; ++j) out->grad[j] = factor * u1 * v0[j] + out->gsrc[j];
    }
}

/* ------------------------------------------------------------------------- */
/* Per-query estimates over N walks, threaded over fixed chunks of walks.     */
/* ------------------------------------------------------------------------- */
typedef struct {
    const or_domain *D;
    const double *X;
    int64_t Q, N, walk_offset;
    double eps, sigma;
    const or_options *opt;
    int64_t nchunks;   /* per query */
    int nfields;       /* doubles per chunk partial */
    double *partial;   /* Q x nchunks x nfields */
    int64_t *ipartial; /* Q x nchunks x 4: steps, capped, outside, killed */
    double *walk_term;
    int64_t *walk_jumps;
    double *walk_grad;
    double *walk_dsigma;
    double *cv_t;   /* control variate: Q x N walk values and Q x N x d values of G v0 */
    double *cv_gv0;
    double *cv_gsrc; /* Q x d: the source part of the gradient (the same for every walk of a query) */
    int64_t next; /* work cursor */
    pthread_mutex_t lock;
} solve_job;

static void run_unit(solve_job *J, int64_t unit)
{
    const int d = J->D->d;
    const int K = J->D->n_exp;
    int64_t q = unit / J->nchunks, c = unit % J->nchunks;
    int64_t w0 = c * OR_CHUNK, w1 = w0 + OR_CHUNK < J->N ? w0 + OR_CHUNK : J->N;
    double *P = J->partial + unit * J->nfields;
    int64_t *I = J->ipartial + unit * 4;
    memset(P, 0, sizeof(double) * J->nfields);
    I[0] = I[1] = I[2] = I[3] = 0;
    or_walk_out o;
    double pt = 0.0, pg[OR_MAXD]; /* antithetic: the even walk of the current pair */
    for (int64_t w = w0; w < w1; ++w) {
        uint64_t walk = (uint64_t)(J->walk_offset + q * J->N + w);
        or_walk(J->D, J->X + q * d, walk, J->eps, J->sigma, J->opt, &o);
        int64_t flat = q * J->N + w;
        if (J->walk_term) J->walk_term[flat] = o.term;
        if (J->walk_jumps) J->walk_jumps[flat] = o.jumps;
        if (J->walk_dsigma) J->walk_dsigma[flat] = o.dsigma;
        if (J->walk_grad)
            for (int j = 0; j < d; ++j) J->walk_grad[flat * d + j] = o.grad[j];
        if (J->cv_t) {
            J->cv_t[flat] = o.term;
            for (int j = 0; j < d; ++j) J->cv_gv0[flat * d + j] = o.gv0[j];
            for (int j = 0; j < d; ++j) J->cv_gsrc[q * d + j] = o.gsrc[j];
        }
        /* fields: [sum u, sum u^2, sum dsigma, grad[d], grad^2[d], dw[K]] */
        P[0] += o.term;
        P[1] += o.term * o.term;
        P[2] += o.dsigma;
        for (int j = 0; j < d; ++j) {
            P[3 + j] += o.grad[j];
            P[3 + d + j] += o.grad[j] * o.grad[j];
        }
        for (int k = 0; k < K; ++k) P[3 + 2 * d + k] += o.dw[k];
        if (J->opt->antithetic) {
            /* squares of the pair means, after the fields above: [u, grad[d]] */
            double *A = P + 3 + 2 * d + K;
            if ((w & 1) == 0) {
                pt = o.term;
                for (int j = 0; j < d; ++j) pg[j] = o.grad[j];
            } else {
                const double y = 0.5 * (pt + o.term);
                A[0] += y * y;
                for (int j = 0; j < d; ++j) {
                    const double g = 0.5 * (pg[j] + o.grad[j]);
                    A[1 + j] += g * g;
                }
            }
        }
        I[0] += o.jumps + 1;
        I[1] += o.capped;
        I[2] += o.outside;
        I[3] += o.killed;
    }
}

static void *solve_worker(void *arg)
{
    solve_job *J = (solve_job *)arg;
    const int64_t total = J->Q * J->nchunks;
    for (;;) {
        pthread_mutex_lock(&J->lock);
        int64_t unit = J->next++;
        pthread_mutex_unlock(&J->lock);
        if (unit >= total) break;
        run_unit(J, unit);
    }
    return NULL;
}

static double se_of(double s, double s2, int64_t n)
{
    if (n < 2) return 0.0;
    double var = (s2 - s * s / (double)n) / (double)(n - 1);
    return var > 0.0 ? sqrt(var / (double)n) : 0.0;
}

/*
 * Estimates at Q query points (X: Q x d), N walks each. Walk w of query q uses the global
 * walk index walk_offset + q N + w. Every output pointer may be NULL.
 *   u, u_se, du_dsigma, walk_steps, capped, outside, killed: Q;  grad, grad_se: Q x d;
 *   du_dw: Q x n_exp;
 *   walk_term, walk_jumps, walk_dsigma: Q x N;  walk_grad: Q x N x d.
 * Returns 0, or -1 on bad arguments / allocation failure.
 */
int or_solve(const or_domain *D, const double *X, int64_t Q, int64_t N, int64_t walk_offset,
             double eps, double sigma, const or_options *opt, int nthreads, double *u,
             double *u_se, double *grad, double *grad_se, double *du_dsigma, double *du_dw,
             int64_t *walk_steps, int64_t *capped, int64_t *outside, int64_t *killed, double *walk_term,
             int64_t *walk_jumps, double *walk_grad, double *walk_dsigma)
{
    if (!D || !X || !opt || D->d < 1 || D->d > OR_MAXD || D->n_exp < 0 || D->n_exp > OR_MAXEXP ||
        D->proj_dims < 0 || D->proj_dims > D->d || D->n_poly < 0 ||
        Q < 0 || N < 1 || sigma < 0.0 ||
        (opt->antithetic && (N % 2 != 0 || walk_offset % 2 != 0 || opt->control_variate)))
        return -1;
    const int d = D->d, K = D->n_exp;
    solve_job J;
    memset(&J, 0, sizeof(J));
    J.D = D;
    J.X = X;
    J.Q = Q;
    J.N = N;
    J.walk_offset = walk_offset;
    J.eps = eps;
    J.sigma = sigma;
    J.opt = opt;
    J.nchunks = (N + OR_CHUNK - 1) / OR_CHUNK;
    J.nfields = 3 + 2 * d + K + (opt->antithetic ? 1 + d : 0);
    J.walk_term = walk_term;
    J.walk_jumps = walk_jumps;
    J.walk_grad = walk_grad;
    J.walk_dsigma = walk_dsigma;
    int64_t units = Q * J.nchunks;
    const int cv = opt->grad && opt->control_variate && N >= 2;
    J.partial = (double *)malloc(sizeof(double) * (size_t)(units * J.nfields + 1));
    J.ipartial = (int64_t *)malloc(sizeof(int64_t) * (size_t)(units * 4 + 1));
    if (cv) {
        J.cv_t = (double *)malloc(sizeof(double) * (size_t)(Q * N + 1));
        J.cv_gv0 = (double *)malloc(sizeof(double) * (size_t)(Q * N * d + 1));
        J.cv_gsrc = (double *)calloc((size_t)(Q * d + 1), sizeof(double));
    }
    if (!J.partial || !J.ipartial || (cv && (!J.cv_t || !J.cv_gv0 || !J.cv_gsrc))) {
        free(J.partial);
        free(J.ipartial);
        free(J.cv_t);
        free(J.cv_gv0);
        free(J.cv_gsrc);
        return -1;
    }
    pthread_mutex_init(&J.lock, NULL);
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    pthread_t th[256];
    int started = 0;
    for (int t = 1; t < nthreads; ++t)
        if (pthread_create(&th[started], NULL, solve_worker, &J) == 0) ++started;
    solve_worker(&J);
    for (int t = 0; t < started; ++t) pthread_join(th[t], NULL);
    pthread_mutex_destroy(&J.lock);

    for (int64_t q = 0; q < Q; ++q) {
        double S[3 + 2 * OR_MAXD + OR_MAXEXP + 1 + OR_MAXD];
        int64_t I[4] = {0, 0, 0, 0};
        memset(S, 0, sizeof(S));
        for (int64_t c = 0; c < J.nchunks; ++c) {
            const double *P = J.partial + (q * J.nchunks + c) * J.nfields;
            const int64_t *IP = J.ipartial + (q * J.nchunks + c) * 4;
            for (int f = 0; f < J.nfields; ++f) S[f] += P[f];
            for (int f = 0; f < 4; ++f) I[f] += IP[f];
        }
        double inv = 1.0 / (double)N;
        if (u) u[q] = S[0] * inv;
        if (u_se) u_se[q] = I[2] ? NAN : se_of(S[0], S[1], N);
        if (du_dsigma) du_dsigma[q] = S[2] * inv;
        for (int j = 0; j < d; ++j) {
            if (grad) grad[q * d + j] = S[3 + j] * inv;
            if (grad_se) grad_se[q * d + j] = I[2] ? NAN : se_of(S[3 + j], S[3 + d + j], N);
        }
        if (opt->antithetic) {
            /* standard errors from the N/2 pair means (their sum is half the walks' sum) */
            const double *A = S + 3 + 2 * d + K;
            if (u_se) u_se[q] = I[2] ? NAN : se_of(0.5 * S[0], A[0], N / 2);
            for (int j = 0; j < d; ++j)
                if (grad_se) grad_se[q * d + j] = I[2] ? NAN : se_of(0.5 * S[3 + j], A[1 + j], N / 2);
        }
        if (cv) {
            /* first pass: tbar; second pass: y_w = G (t_w - tbar) v_w, its sum and spread */
            const double *t = J.cv_t + q * N;
            const double *gv = J.cv_gv0 + q * N * d;
            double tbar = 0.0;
            for (int64_t w = 0; w < N; ++w) tbar += t[w];
            tbar /= (double)N;
            for (int j = 0; j < d; ++j) {
                double sy = 0.0;
                for (int64_t w = 0; w < N; ++w) sy += (t[w] - tbar) * gv[w * d + j];
                const double ybar = sy / (double)N;
                double ss = 0.0;
                for (int64_t w = 0; w < N; ++w) {
                    const double e = (t[w] - tbar) * gv[w * d + j] - ybar;
                    ss += e * e;
                }
                const double var = ss / (double)(N - 1);
                if (grad) grad[q * d + j] = I[2] ? NAN : sy / (double)(N - 1) + J.cv_gsrc[q * d + j];
                if (grad_se)
                    grad_se[q * d + j] = I[2] ? NAN : ((double)N / (double)(N - 1)) * sqrt(var / (double)N);
            }
        }
        for (int k = 0; k < K; ++k)
            if (du_dw) du_dw[q * K + k] = S[3 + 2 * d + k] * inv;
        if (walk_steps) walk_steps[q] = I[0];
        if (capped) capped[q] = I[1];
        if (outside) outside[q] = I[2];
        if (killed) killed[q] = I[3];
    }
    free(J.partial);
    free(J.ipartial);
    free(J.cv_t);
    free(J.cv_gv0);
    free(J.cv_gsrc);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Screened-harmonic path (Sec. III; Sec. VII adaptive step s = min(s_ub, d/2)). */
/* Step i estimates grad u at x_i with N gradient walks, walk offset i N.      */
/* flags[i]: 1 goal reached before step i (no move; with an impulse source and no */
/* goal ball: the source is closer than s_ub), 2 no signal (|grad| = 0,           */
/* no move), 4 outside the domain (no move).                                  */
/* Returns the number of points written (the path stops at the goal).         */
/* ------------------------------------------------------------------------- */
int64_t or_plan_path(const or_domain *D, const double *x0, int64_t n_steps, int64_t N, double eps,
                     double sigma, double s_ub, const or_options *opt_in, int nthreads,
                     double *path, int32_t *flags, double *grads)
{
    const int d = D->d;
    or_options opt = *opt_in;
    opt.grad = 1;
    double x[OR_MAXD], g[OR_MAXD], xbar[OR_MAXD];
    for (int64_t i = 0; i < n_steps; ++i) flags[i] = 0;
    for (int j = 0; j < d; ++j) x[j] = path[j] = x0[j];
    int64_t written = 1;
    for (int64_t i = 0; i < n_steps; ++i) {
        flags[i] = 0;
        if (D->has_goal) {
            double rg = norm_diff(obstacle_dims(D), x, D->goal_c) - D->goal_r;
            if (rg < eps) {
                flags[i] = 1;
                break;
            }
        } else if (D->has_source && norm_diff(d, x, D->source_z) < s_ub) {
            /* the goal is the impulse source: reached once it is within one nominal step */
            flags[i] = 1;
            break;
        }
        int32_t kind;
        int64_t index;
        double R = or_distance(D, x, &kind, &index, xbar);
        int64_t out = 0;
        if (or_solve(D, x, 1, N, i * N, eps, sigma, &opt, nthreads, NULL, NULL, g, NULL, NULL, NULL,
                     NULL, NULL, &out, NULL, NULL, NULL, NULL, NULL) != 0 ||
            out > 0 || !(R > 0.0)) {
            flags[i] = 4;
            break;
        }
        if (grads)
            for (int j = 0; j < d; ++j) grads[i * d + j] = g[j];
        double gg = 0.0;
        for (int j = 0; j < d; ++j) gg += g[j] * g[j];
        if (gg > 0.0) {
            double gn = sqrt(gg);
            double s = 0.5 * R < s_ub ? 0.5 * R : s_ub;
            for (int j = 0; j < d; ++j) x[j] = x[j] + s * (g[j] / gn);
        } else {
            flags[i] = 2;
        }
        for (int j = 0; j < d; ++j) path[written * d + j] = x[j];
        ++written;
    }
    return written;
}
