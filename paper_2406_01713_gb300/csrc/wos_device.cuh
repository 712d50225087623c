// Device-side building blocks of the Walk-on-Spheres CUDA path (sm_103a).
//
// Counter-based sphere sampling, the screened normaliser, weight-table lookup and the
// device views of a domain. Everything here is the GPU path's own code.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/wos.h"

namespace wos {

constexpr int kMaxD = WOS_MAX_D;
constexpr int kMaxExp = WOS_MAX_EXP;

// Component kinds. Tie-break order of the distance query: goal, balls, points, arm, outer ball,
// box faces (lo_0, hi_0, lo_1, ...).
enum Kind : int { kGoal = 0, kBall = 1, kPoint = 2, kOuter = 3, kFace = 4, kArm = 5 };
constexpr int kMaxArmObs = 32;        // task-space obstacle points of an arm in the mixed walker
constexpr int kMaxArmLinksMixed = 8;  // the mixed walker runs arms in d <= 8

// ------------------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two 32x32 -> 64-bit
// multiplies mixed with a Weyl-sequence key schedule.
// ------------------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint32_t k0, uint32_t k1, uint4 c) {
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        const uint32_t a = c.x, b = c.z;
        const uint32_t hi_a = __umulhi(0xD2511F53u, a), lo_a = 0xD2511F53u * a;
        const uint32_t hi_b = __umulhi(0xCD9E8D57u, b), lo_b = 0xCD9E8D57u * b;
        c = make_uint4(hi_b ^ c.y ^ k0, lo_b, hi_a ^ c.w ^ k1, lo_a);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

__device__ __forceinline__ uint4 philox_block(uint64_t seed, uint64_t walk, uint32_t step,
                                              uint32_t block) {
    return philox4x32_10((uint32_t)seed, (uint32_t)(seed >> 32),
                         make_uint4((uint32_t)walk, (uint32_t)(walk >> 32), step, block));
}

// Uniform direction in R^D, FP64: Box-Muller on output pairs with u1 = (r + 1) 2^-32 in (0, 1],
// u2 = r 2^-32 in [0, 1), then v = n / |n| (e_0 if |n| = 0).
template <int D>
__device__ __forceinline__ void direction_f64(uint64_t seed, uint64_t walk, uint32_t step,
                                              double (&v)[D]) {
    constexpr double kTwoPi = 6.283185307179586476925286766559;
    constexpr double kInv32 = 2.3283064365386962890625e-10;  // 2^-32
#pragma unroll
    for (int b = 0; b < (D + 3) / 4; ++b) {
        const uint4 r = philox_block(seed, walk, step, (uint32_t)b);
        const uint32_t rr[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
        for (int p = 0; p < 2; ++p) {
            const int i = 4 * b + 2 * p;
            if (i < D) {
                const double u1 = ((double)rr[2 * p] + 1.0) * kInv32;
                const double u2 = (double)rr[2 * p + 1] * kInv32;
                const double rad = sqrt(-2.0 * log(u1));
                double s, c;
                sincos(kTwoPi * u2, &s, &c);
                v[i] = rad * c;
                if (i + 1 < D) v[i + 1] = rad * s;
            }
        }
    }
    double ss = 0.0;
#pragma unroll
    for (int j = 0; j < D; ++j) ss += v[j] * v[j];
    if (ss > 0.0) {
        const double nrm = sqrt(ss);
#pragma unroll
        for (int j = 0; j < D; ++j) v[j] = v[j] / nrm;
    } else {
#pragma unroll
        for (int j = 0; j < D; ++j) v[j] = (j == 0) ? 1.0 : 0.0;
    }
}

// FP32 direction from the same counters: u1 = (top 24 bits + 1) 2^-24, u2 = top 24 bits 2^-24.
// FAST (mixed walkers) takes the SFU approximations of log, square root, sine and cosine; the
// angle 2 pi u2 is evaluated as -(cos, sin)(2 pi u2 - pi), inside the range where the SFU sine
// and cosine are accurate, so the direction is the one of the exact sampler up to errors of
// order 1e-7 (it is normalised after) and the walks keep the same random stream as the FP64
// ones. Without FAST (plain baseline): logf, sqrtf and sincospif of 2 u2.
template <int D, bool FAST>
__device__ __forceinline__ void direction_f32(uint64_t seed, uint64_t walk, uint32_t step,
                                              float (&v)[D]) {
    constexpr float kInv24 = 5.9604644775390625e-08f;  // 2^-24
#pragma unroll
    for (int b = 0; b < (D + 3) / 4; ++b) {
        const uint4 r = philox_block(seed, walk, step, (uint32_t)b);
        const uint32_t rr[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
        for (int p = 0; p < 2; ++p) {
            const int i = 4 * b + 2 * p;
            if (i < D) {
                const float u1 = (float)((rr[2 * p] >> 8) + 1u) * kInv24;
                const float u2 = (float)(rr[2 * p + 1] >> 8) * kInv24;
                float rad, s, c;
                if (FAST) {
                    asm("sqrt.approx.f32 %0, %1;" : "=f"(rad) : "f"(-2.0f * __logf(u1)));
                    __sincosf(fmaf(6.283185307179586f, u2, -3.141592653589793f), &s, &c);
                    rad = -rad;
                } else {
                    rad = sqrtf(-2.0f * logf(u1));
                    sincospif(2.0f * u2, &s, &c);
                }
                v[i] = rad * c;
                if (i + 1 < D) v[i + 1] = rad * s;
            }
        }
    }
    float ss = 0.0f;
#pragma unroll
    for (int j = 0; j < D; ++j) ss = fmaf(v[j], v[j], ss);
    if (ss > 0.0f) {
        const float inv = rsqrtf(ss);
#pragma unroll
        for (int j = 0; j < D; ++j) v[j] *= inv;
    } else {
#pragma unroll
        for (int j = 0; j < D; ++j) v[j] = (j == 0) ? 1.0f : 0.0f;
    }
}

// Uniform of the Russian roulette before jump `step` of a walk: the top 24 bits of Philox block
// 15 of (walk, step) times 2^-24 (exact in FP32 and FP64; the direction blocks are 0..2).
__device__ __forceinline__ float roulette_uniform(uint64_t seed, uint64_t walk, uint32_t step) {
    const uint4 r = philox_block(seed, walk, step, 15u);
    return (float)(r.x >> 8) * 5.9604644775390625e-08f;
}

// Walk index whose step-0 stream gives a walk's first direction, and its sign: with antithetic
// pairs, walk 2m + 1 takes the negated first direction of walk 2m.
__device__ __forceinline__ uint64_t first_direction_walk(uint64_t walk, int antithetic) {
    return antithetic ? (walk & ~1ull) : walk;
}
__device__ __forceinline__ bool first_direction_negated(uint64_t walk, int antithetic) {
    return antithetic && (walk & 1ull);
}

// ------------------------------------------------------------------------------------
// Screened normaliser. With S_mu(z) = Gamma(mu+1) (z/2)^-mu I_mu(z) = sum_k q^k / (k! (mu+1)_k),
// q = z^2/4 (DLMF 10.25.2):  C_nu(z) = 1 / S_nu(z);  d/dz log C_nu = -(z/d) S_{nu+1}/S_nu;
// d/dsigma log C_nu(R sqrt(sigma)) = -(R^2 / (2d)) S_{nu+1}(z) / S_nu(z);
// first-sphere gradient factor alpha(R) = (d/R) C_{nu+1}(z) = (d/R) / S_{nu+1}(z).
// ------------------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T bessel_S(T mu, T z) {
    const T q = T(0.25) * z * z;
    T term = T(1), sum = T(1);
    const T tol = sizeof(T) == 8 ? T(1e-17) : T(3e-8);
    for (int k = 1; k < 4000; ++k) {
        term = term * q / (T(k) * (mu + T(k)));
        sum += term;
        if (term <= tol * sum) break;
    }
    return sum;
}

// Weight table entry: x = log C_nu(z), y = S_{nu+1}(z) / S_nu(z). Linear interpolation on a
// uniform grid z_i = i h, i = 0..n-1.
struct WeightTable {
    const float2 *nodes;
    float inv_h;
    int n;
};

__device__ __forceinline__ float2 table_lookup(const WeightTable &t, float z) {
    float s = z * t.inv_h;
    s = fminf(s, (float)(t.n - 1) - 1e-3f);
    const int i = (int)s;
    const float f = s - (float)i;
    const float2 a = __ldg(t.nodes + i);
    const float2 b = __ldg(t.nodes + i + 1);
    return make_float2(fmaf(f, b.x - a.x, a.x), fmaf(f, b.y - a.y, a.y));
}

// ------------------------------------------------------------------------------------
// Device views of a domain.
// ------------------------------------------------------------------------------------
template <typename T>
struct DomainView {
    int d, n_balls, n_exp, has_box, has_outer, has_goal, has_source;
    int proj;  // components are measured in coordinates 0..proj-1 (proj = d, or fewer: extruded)
    int64_t n_points;
    T outer_r, goal_r, source_q;
    const T *box_lo, *box_hi, *outer_c, *goal_c;  // d each
    const T *ball_c, *ball_r;                      // B x d, B
    const T *points;                               // M x d
    const T *exp_w, *exp_a;                        // K, K x d
    const T *source_z;                             // d (impulse source; has_source)
    int n_links;                                   // planar arm: joints 0..n_links-1 (0: none)
    int64_t n_arm_obs;
    T arm_inv_K;                                   // 1 / Lipschitz constant of the kinematics
    const T *link_l;                               // n_links
    const T *arm_obs;                              // n_arm_obs x 2 (task space)
};

// Per-query accumulator fields: [sum u, sum u^2, sum du/dsigma, sum grad (d), sum grad^2 (d),
// sum du/dw (K)]; with the gradient control variate, [sum v0 (d), sum t v0^2 (d),
// sum v0^2 (d), G] (v0 the first direction, t the walk's value, G = alpha(R0)/C(R0), one number
// per query because R0 is the distance at the query); with an impulse source in gradient walks,
// [s0, g_src (d)]: the step-0 source value and the source part of the gradient, also one per
// query (they depend only on the query). The gradient sums then hold G (t - s0) v0. int64
// counters [walks, walk_steps, capped, outside, killed] live apart. With antithetic pairs the
// squared fields hold the sums of the squared pair means instead ([u^2] and [grad^2]).
__host__ __device__ __forceinline__ int acc_fields(int d, int K, int cv = 0, int src = 0) {
    return 3 + 2 * d + K + (cv ? 3 * d + 1 : 0) + (src ? d + 1 : 0);
}
__host__ __device__ __forceinline__ int src_field(int d, int K, int cv) { return acc_fields(d, K, cv, 0); }
__host__ __device__ __forceinline__ int cv_field(int d, int K) { return 3 + 2 * d + K; }
constexpr int kCounters = 5;

// Control-variate gradient of one component from the one-pass sums of a query:
//   A = sum G t v, A2 = sum (G t v)^2, Sv = sum v, Stv2 = sum t v^2, Sv2 = sum v^2, St = sum t,
//   n walks. With y_w = G (t_w - tbar) v_w:
//   sum y = A - tbar G Sv,  sum y^2 = A2 - 2 tbar G^2 Stv2 + tbar^2 G^2 Sv2,
//   grad = sum y / (n - 1),  se = n/(n-1) sqrt(var(y) / n).
__host__ __device__ __forceinline__ void cv_estimate(double A, double A2, double Sv, double Stv2, double Sv2,
                                                     double G, double St, double n, double &g, double &se) {
    const double tbar = St / n;
    const double sy = A - tbar * G * Sv;
    const double sy2 = A2 + G * G * (tbar * tbar * Sv2 - 2.0 * tbar * Stv2);
    g = sy / (n - 1.0);
    const double var = (sy2 - sy * sy / n) / (n - 1.0);
    se = var > 0.0 ? (n / (n - 1.0)) * sqrt(var / n) : 0.0;
}

}  // namespace wos
