// Direct-form geometry of a domain for the FP64 and plain FP32 walkers and the planner:
// distance to the boundary (Sec. VI, Eq. for d(x, dOmega); Sec. VII-A point-set distance)
// and the boundary value at the closest boundary point (Fig. 2).
#pragma once

#include <math_constants.h>

#include "wos_device.cuh"

namespace wos {

template <typename T>
__device__ __forceinline__ T inf_of() {
    return sizeof(T) == 8 ? (T)CUDART_INF : (T)CUDART_INF_F;
}

// |x - c| over the first m coordinates (m = D, or fewer for an extruded domain)
template <typename T, int D>
__device__ __forceinline__ T norm_diff(const T (&x)[D], const T *c, int m) {
    T s = T(0);
#pragma unroll
    for (int j = 0; j < D; ++j) {
        if (j < m) {
            const T t = x[j] - c[j];
            s += t * t;
        }
    }
    return sqrt(s);
}

// sine and cosine of a summed joint angle: FP64 sincos; FP32 sincospi of a / pi (exact range
// reduction, no large-argument path)
template <typename T>
__device__ __forceinline__ void sincos_t(T a, T *s, T *c) {
    if constexpr (sizeof(T) == 8) sincos(a, s, c);
    else sincospif(a * 0.318309886183790672f, s, c);
}

// Planar arm (Sec. V-A): joint angles x_0..x_{n-1} summed along the chain, base at the origin;
// d_tau = the smallest task-space distance between a link (segment) and an obstacle point. The
// returned safe-ball radius d_tau / K underestimates the configuration-space distance.
template <typename T, int D>
__device__ __forceinline__ T arm_distance(const DomainView<T> &dm, const T (&x)[D]) {
    T px = T(0), py = T(0), ang = T(0), best = inf_of<T>();
#pragma unroll
    for (int n = 0; n < D; ++n) {
        if (n >= dm.n_links) break;
        ang += x[n];
        T sn, cs;
        sincos_t<T>(ang, &sn, &cs);
        const T sx = dm.link_l[n] * cs, sy = dm.link_l[n] * sn, ss = sx * sx + sy * sy;
        for (int64_t o = 0; o < dm.n_arm_obs; ++o) {
            const T ox = dm.arm_obs[2 * o] - px, oy = dm.arm_obs[2 * o + 1] - py;
            T t = ss > T(0) ? (ox * sx + oy * sy) / ss : T(0);
            t = t < T(0) ? T(0) : (t > T(1) ? T(1) : t);
            const T dx = ox - t * sx, dy = oy - t * sy;
            const T r = sqrt(dx * dx + dy * dy);
            if (r < best) best = r;
        }
        px += sx;
        py += sy;
    }
    return best * dm.arm_inv_K;
}

// Distance to the boundary (minimum over components, strict '<' keeps the first in the order
// goal, balls, points, arm, outer ball, faces); an extruded domain measures every component in
// its first dm.proj coordinates.
template <typename T, int D>
__device__ __forceinline__ T distance(const DomainView<T> &dm, const T (&x)[D], int &kind, int64_t &idx) {
    const int m = dm.proj;
    T best = inf_of<T>();
    kind = -1;
    idx = -1;
    if (dm.has_goal) {
        const T r = norm_diff<T, D>(x, dm.goal_c, m) - dm.goal_r;
        if (r < best) { best = r; kind = kGoal; idx = 0; }
    }
    for (int i = 0; i < dm.n_balls; ++i) {
        const T r = norm_diff<T, D>(x, dm.ball_c + (int64_t)i * D, m) - dm.ball_r[i];
        if (r < best) { best = r; kind = kBall; idx = i; }
    }
    for (int64_t i = 0; i < dm.n_points; ++i) {
        const T r = norm_diff<T, D>(x, dm.points + i * D, m);
        if (r < best) { best = r; kind = kPoint; idx = i; }
    }
    if (dm.n_links > 0) {
        const T r = arm_distance<T, D>(dm, x);
        if (r < best) { best = r; kind = kArm; idx = 0; }
    }
    if (dm.has_outer) {
        const T r = dm.outer_r - norm_diff<T, D>(x, dm.outer_c, m);
        if (r < best) { best = r; kind = kOuter; idx = 0; }
    }
    if (dm.has_box) {
#pragma unroll
        for (int j = 0; j < D; ++j) {
            if (j >= m) continue;
            const T rlo = x[j] - dm.box_lo[j];
            if (rlo < best) { best = rlo; kind = kFace; idx = 2 * j; }
            const T rhi = dm.box_hi[j] - x[j];
            if (rhi < best) { best = rhi; kind = kFace; idx = 2 * j + 1; }
        }
    }
    return best;
}

// g at the closest boundary point xbar (Fig. 2; an arm's walk reads g at its own position);
// e[k] = exp(a_k . xbar) for exp data.
template <typename T, int D>
__device__ __forceinline__ T boundary_value(const DomainView<T> &dm, const T (&x)[D], int kind, int64_t idx,
                            T (&e)[kMaxExp]) {
    T xb[D];
    const T *c = nullptr;
    T rad = T(0);
    const int m = dm.proj;  // an extruded domain projects in these and keeps the free coordinates
    if (kind == kGoal) { c = dm.goal_c; rad = dm.goal_r; }
    if (kind == kBall) { c = dm.ball_c + idx * D; rad = dm.ball_r[idx]; }
    if (kind == kOuter) { c = dm.outer_c; rad = dm.outer_r; }
    if (c != nullptr) {
        const T len = norm_diff<T, D>(x, c, m);
#pragma unroll
        for (int j = 0; j < D; ++j)
            xb[j] = j >= m ? x[j] : (len > T(0) ? c[j] + rad * (x[j] - c[j]) / len : c[j] + (j == 0 ? rad : T(0)));
    } else if (kind == kPoint) {
#pragma unroll
        for (int j = 0; j < D; ++j) xb[j] = j >= m ? x[j] : dm.points[idx * D + j];
    } else {
#pragma unroll
        for (int j = 0; j < D; ++j) xb[j] = x[j];
        if (kind == kFace) {
            const int jf = (int)(idx >> 1);
            const T face = (idx & 1) ? dm.box_hi[jf] : dm.box_lo[jf];
#pragma unroll
            for (int j = 0; j < D; ++j)
                if (j == jf) xb[j] = face;
        }
    }
    if (dm.n_exp > 0) {
        T g = T(0);
#pragma unroll
        for (int k = 0; k < kMaxExp; ++k) {
            if (k < dm.n_exp) {
                T dot = T(0);
#pragma unroll
                for (int j = 0; j < D; ++j) dot += dm.exp_a[k * D + j] * xb[j];
                e[k] = exp(dot);
                g += dm.exp_w[k] * e[k];
            }
        }
        return g;
    }
    return kind == kGoal ? T(1) : T(0);
}

// ---- impulse source: Green's function of the largest empty ball ------------------------
// log K_nu(x) and log K_{nu+1}(x), x > 0, from int_0^inf exp(-x cosh t) cosh(mu t) dt
// (DLMF 10.32.9): trapezoidal rule (even integrand, analytic in |Im t| < pi/2; step
// min(1/8, 0.6/sqrt(x)) keeps the relative error below 1e-23) with the sum scaled by the peak
// of exp(-x cosh t + (nu+1) t), so that no term overflows.
__device__ inline void log_bessel_K_pair_f64(double nu, double x, double &l0, double &l1) {
    const double mu = nu + 1.0;
    const double ts = asinh(mu / x);
    const double m = mu * ts - x * cosh(ts);
    const double h = x > 23.04 ? 0.6 * rsqrt(x) : 0.125;
    double s0 = 0.0, s1 = 0.0;
    for (int i = 0; i < 8000; ++i) {
        const double t = h * (double)i, c = x * cosh(t), w = i == 0 ? 0.5 : 1.0;
        const double e1 = mu * t - c - m;
        s1 += w * (exp(e1) + exp(-mu * t - c - m));
        s0 += w * (exp(nu * t - c - m) + exp(-nu * t - c - m));
        if (t > ts && e1 < -45.0) break;
    }
    l0 = m + log(0.5 * h * s0);
    l1 = m + log(0.5 * h * s1);
}

// dG_B/dsigma at sigma = 0 between the centre of a ball of radius R and distance r: minus the
// radial solution w of -Laplace(w) = G_0 with w = 0 on the sphere (the first-order term of G_B
// in sigma); omega = |S^(d-1)|. FP64.
__device__ inline double source_green_dsigma0_f64(int d, double omega, double r, double R) {
    if (d == 2) return (0.25 * r * r * log(R / r) + 0.25 * (r * r - R * R)) / (2.0 * CUDART_PI);
    if (d == 4) return (-0.5 * log(R / r) - r * r / (8.0 * R * R) + 0.125) / (2.0 * omega);
    const double a = 1.0 / (2.0 * (4.0 - d)), b = 1.0 / (2.0 * d);
    return (a * pow(r, 4.0 - d) - b * r * r * pow(R, 2.0 - d) - (a - b) * pow(R, 4.0 - d)) / ((d - 2.0) * omega);
}

// Between the centre of a ball of radius R and a point at distance r (0 < r < R), for
// Laplace(u) - sigma u = -delta with zero values on the sphere: G = G_B and F with
// grad_x G_B = F (y - x)/r at the centre; k = sqrt(sigma), nu = d/2 - 1, c0 = k^nu/(2 pi)^(d/2):
//   G = c0 r^-nu [K_nu(kr) - K_nu(kR) I_nu(kr)/I_nu(kR)],
//   F = c0 k r^-nu [K_nu+1(kr) - K_nu+1(kR) I_nu+1(kr)/I_nu+1(kR)],
// I ratios from the series S (I_mu(z) is proportional to z^mu S_mu(z)); at sigma = 0 the
// Laplace forms (r^(2-d) - R^(2-d))/((d-2) omega), ln(R/r)/(2 pi) for d = 2, and
// F = (r^(1-d) - r R^-d)/omega, omega = |S^(d-1)|; *dG (when given): dG_B/dsigma. FP64.
__device__ inline void source_green_f64(int d, double k, double r, double R, double &G, double &F,
                                        double *dG = nullptr) {
    const double nu = 0.5 * d - 1.0;
    if (k == 0.0) {
        const double omega = 2.0 * pow(CUDART_PI, 0.5 * d) / tgamma(0.5 * d);
        G = d == 2 ? log(R / r) / (2.0 * CUDART_PI) : (pow(r, 2.0 - d) - pow(R, 2.0 - d)) / ((d - 2.0) * omega);
        F = (pow(r, 1.0 - d) - r * pow(R, -(double)d)) / omega;
        if (dG != nullptr) *dG = source_green_dsigma0_f64(d, omega, r, R);
        return;
    }
    double ka0, ka1, kb0, kb1;
    log_bessel_K_pair_f64(nu, k * r, ka0, ka1);
    log_bessel_K_pair_f64(nu, k * R, kb0, kb1);
    const double lc0 = nu * log(k) - 0.5 * d * log(2.0 * CUDART_PI);
    const double lrR = log(r / R), lr = log(r);
    const double Sa0 = bessel_S<double>(nu, k * r), Sb0 = bessel_S<double>(nu, k * R);
    const double Sa1 = bessel_S<double>(nu + 1.0, k * r), Sb1 = bessel_S<double>(nu + 1.0, k * R);
    const double i0 = nu * lrR + log(Sa0) - log(Sb0);
    const double i1 = (nu + 1.0) * lrR + log(Sa1) - log(Sb1);
    const double X = exp(kb0 - ka0 + i0);  // K_nu(kR) Q / K_nu(kr), Q = I_nu(kr) / I_nu(kR)
    const double P0 = exp(lc0 - nu * lr + ka0);
    G = P0 * (1.0 - X);
    F = exp(lc0 + log(k) - nu * lr + ka1) * (1.0 - exp(kb1 - ka1 + i1));
    if (dG != nullptr) {
        // dG/dk = (nu/k) G + c0 r^-nu A'(k), A = K_nu(kr) - K_nu(kR) Q, with
        // K_nu'(x) = -K_{nu+1}(x) + (nu/x) K_nu(x) and Q'/Q = k (r^2 s(kr) - R^2 s(kR)) / (2 (nu+1)),
        // s = S_{nu+1}/S_nu (DLMF 10.29.2, 10.25.2); dG/dsigma = (dG/dk) / (2k)
        const double br = (2.0 * nu / k) * (1.0 - X) - r * exp(ka1 - ka0) + R * X * exp(kb1 - kb0) -
                          X * k * (r * r * Sa1 / Sa0 - R * R * Sb1 / Sb0) / (2.0 * (nu + 1.0));
        *dG = P0 * br / (2.0 * k);
    }
}

}  // namespace wos
