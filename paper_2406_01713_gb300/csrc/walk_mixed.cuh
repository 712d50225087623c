// Persistent mixed-precision Walk-on-Spheres walker (Sec. IV-A estimators, FP32 walkers).
//
// One launch serves many problems of uneven dimension, obstacle count and walk budget:
//   * a global work queue of items (problem, walk range) in longest-first order, pulled by
//     CTAs through an atomic cursor;
//   * the current problem's balls are staged in shared memory as 8-ball blocks
//     [m_0 x8][m_1 x8]...[m_{d-1} x8][e0 x8][e1 x8] with m = -2c, e0 = |c|^2 - r^2, e1 = -2r,
//     so two 128-bit shared loads fetch one field of eight balls, and the screen runs as
//     packed FP32x2 FMAs (two balls per instruction);
//   * every lane runs walks back to back, refilling from the item's walk counter the moment
//     its walk ends (walk lengths vary, so lanes never wait for the slowest walk of a batch);
//   * each finished walk writes a small FP32 record (value, d/dsigma, gradient factor, jumps,
//     outcome, first direction, du/dw terms) that reduce_kernel sums per query in FP64 in a
//     fixed order, so no per-lane accumulator occupies registers between walks and no atomic
//     orders the sums.
//
// Distance to the balls (Sec. VI, |x - c| - r): a ball can only beat the current best
// distance b if |x-c|^2 < (r+b)^2, i.e. if
//     L = e0 + e1 b + x.m  <  b^2 - |x|^2.
// L is evaluated in FP32 for every ball (d+1 FMAs) and compared against the threshold plus a
// slack E that bounds the FP32 rounding of both sides, so no true candidate is ever missed.
// Passing balls get distance bounds rebuilt from L; after the scan the best candidate is
// evaluated exactly with the direct form sqrt(sum (x_j - c_j)^2) - r.
//
// Walker positions are held as packed pairs (x_j, x_j), the operand the packed FMAs need. Each
// walker's coordinate sum is split into two halves, so one 8-ball block gives eight
// independent FMA chains.
// The radius used for the jump is the computed distance minus `shrink`, a bound on the FP32
// error of the distance evaluation and of the position update, so every sphere lies inside
// the FP64 domain.
#pragma once

#include <cuda_runtime.h>
#include <math_constants.h>

#include "wos_launch.h"

namespace wos {

struct MixedSmem {
    float geom[geom_count(kMaxD)];
    int problem;
    int item_problem;
    unsigned next_walk;
    unsigned end_walk;
    unsigned begin_walk;
    long long item;
};

// ---- packed FP32x2 helpers (sm_100+: fma.rn.f32x2, three-input min.f32) -----------------
typedef unsigned long long f32x2;

__device__ __forceinline__ f32x2 pack2(float lo, float hi) {
    f32x2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ float2 unpack2(f32x2 v) {
    float2 r;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(v));
    return r;
}
__device__ __forceinline__ f32x2 ffma2(f32x2 a, f32x2 b, f32x2 c) {
    f32x2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ float fmin3(float a, float b, float c) {
    float r;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}


constexpr int kBallBlock = 8;  // balls per shared-memory block

template <int D>
struct MixedWalker {
    f32x2 x2[D];              // position as packed pairs (x_j, x_j)
    float logw, dsig, gfac0;  // gfac0 = alpha(R0) / C(R0); v0 is regenerated from its counter
    float src, src0;          // impulse source: contributions so far, and the step-0 one
    float dsrc;               // d/dsigma of the source contributions
    int k;
    unsigned j;      // walk index within the problem
    long long q;     // query
    bool active;
};

template <int D>
__device__ __forceinline__ float xj(const f32x2 (&x2)[D], int j) { return unpack2(x2[j]).x; }

// sum of term(j, s) over the coordinates the components are measured in: all D, or the first m
// of an extruded domain (Sec. VI dimensionality study); the common case m = D takes no predicates
template <int D, typename F>
__device__ __forceinline__ float sum_coords(int m, F term) {
    float s = 0.f;
    if (m >= D) {
#pragma unroll
        for (int j = 0; j < D; ++j) s = term(j, s);
    } else {
#pragma unroll
        for (int j = 0; j < D; ++j)
            if (j < m) s = term(j, s);
    }
    return s;
}

// Planar arm (Sec. V-A): the safe-ball radius d_tau / K for the joint angles x_0..x_{n-1},
// d_tau the task-space distance between the links and the obstacle points. Sine and cosine of
// the summed angle as sincospi of angle / pi (exact range reduction, no large-argument path);
// the host adds the FP32 error of this evaluation to the jump's shrink. Only the walker
// instantiations for domains with an arm contain it.
template <int D>
__device__ __forceinline__ float arm_distance_f32(const MixedProblem &P, const float *geom, const f32x2 (&x2)[D]) {
    const float *ll = geom + geom_link(D), *ob = geom + geom_arm_obs(D);
    float px = 0.f, py = 0.f, ang = 0.f, dt = CUDART_INF_F;
#pragma unroll
    for (int n = 0; n < D; ++n) {
        if (n >= P.n_links) break;
        ang += xj(x2, n);
        float sn, cs;
        sincospif(ang * 0.318309886183790672f, &sn, &cs);
        const float sx = ll[n] * cs, sy = ll[n] * sn, ss = fmaf(sx, sx, sy * sy);
        for (int o = 0; o < P.n_arm_obs; ++o) {
            const float ox = ob[2 * o] - px, oy = ob[2 * o + 1] - py;
            const float t = fminf(fmaxf(fmaf(ox, sx, oy * sy) / ss, 0.f), 1.f);
            const float dx = fmaf(-t, sx, ox), dy = fmaf(-t, sy, oy);
            dt = fminf(dt, sqrtf(fmaf(dx, dx, dy * dy)));
        }
        px += sx;
        py += sy;
    }
    return dt * P.arm_inv_K;
}

// Distance to the components other than the balls. geom layout in shared memory: [0,d) box lo,
// [d,2d) box hi, [2d,3d) goal c, [3d,4d) outer c, [4d, 4d+K) exp w, then K x d exp a. An extruded
// domain's box has its free-coordinate faces far away (set on the host).
template <int D, bool ARM>
__device__ __forceinline__ void other_components(const MixedProblem &P, const float *geom,
                                                 const f32x2 (&x2)[D], float &goal, float &other,
                                                 int &okind, int &oidx) {
    goal = CUDART_INF_F;
    other = CUDART_INF_F;
    okind = -1;
    oidx = -1;
    if (P.has_goal) {
        const float s = sum_coords<D>(P.proj, [&](int j, float a) {
            const float t = xj(x2, j) - geom[2 * D + j];
            return fmaf(t, t, a);
        });
        goal = sqrtf(s) - P.goal_r;
    }
    if constexpr (ARM) {
        const float r = arm_distance_f32<D>(P, geom, x2);
        if (r < other) { other = r; okind = kArm; oidx = 0; }
    }
    if (P.has_outer) {
        const float s = sum_coords<D>(P.proj, [&](int j, float a) {
            const float t = xj(x2, j) - geom[3 * D + j];
            return fmaf(t, t, a);
        });
        const float r = P.outer_r - sqrtf(s);
        if (r < other) { other = r; okind = kOuter; oidx = 0; }
    }
    if (P.has_box) {
#pragma unroll
        for (int j = 0; j < D; ++j) {
            const float rlo = xj(x2, j) - geom[j];
            if (rlo < other) { other = rlo; okind = kFace; oidx = 2 * j; }
            const float rhi = geom[D + j] - xj(x2, j);
            if (rhi < other) { other = rhi; okind = kFace; oidx = 2 * j + 1; }
        }
    }
}

// Per-walker state of the ball screen. b: running upper bound of the distance (starts at the
// nearest other component); thr = b^2 - |x|^2 + E; lb1/lb2/bidx: the smallest and second
// smallest lower bound among the balls that passed, and the ball of the smallest.
struct ScreenState {
    float b, thr, xx, lb1, lb2;
    f32x2 b2;
    int bidx;
};

template <int D>
__device__ __forceinline__ void screen_init(ScreenState &S, const f32x2 (&x2)[D], float b0, float slack,
                                            int m) {
    // |x|^2 over the measured coordinates (an extruded domain's ball records are zero in the others)
    const float xx = sum_coords<D>(m, [&](int j, float a) { return fmaf(xj(x2, j), xj(x2, j), a); });
    S.xx = xx;
    S.b = b0;
    S.thr = fmaf(b0, b0, slack - xx);
    S.b2 = pack2(b0, b0);
    S.lb1 = CUDART_INF_F;
    S.lb2 = CUDART_INF_F;
    S.bidx = -1;
}

// Balls of one block that passed the screen: with L = |x-c|^2 - |x|^2 - r^2 - 2 r b_used,
// s = L + |x|^2 + r (r + 2 b_used) is |x-c|^2 up to the slack E, so
// lb = sqrt(s - E) - r <= d_i <= sqrt(s + E) - r = ub.
__device__ __forceinline__ void screen_passing(ScreenState &S, const float (&Lt)[kBallBlock],
                                               const float (&Rt)[kBallBlock], float slack, int blk) {
    const float bu = S.b;  // the bound these L values were computed with
#pragma unroll
    for (int t = 0; t < kBallBlock; ++t) {
        if (Lt[t] < S.thr) {
            const float st = fmaf(Rt[t], fmaf(2.f, bu, Rt[t]), Lt[t] + S.xx);
            const float lb = sqrtf(fmaxf(st - slack, 0.f)) - Rt[t];
            const float ub = sqrtf(st + slack) - Rt[t];
            if (lb < S.lb1) {
                S.lb2 = S.lb1;
                S.lb1 = lb;
                S.bidx = kBallBlock * blk + t;
            } else {
                S.lb2 = fminf(S.lb2, lb);
            }
            if (ub < S.b) {
                S.b = ub;
                S.thr = fmaf(ub, ub, slack - S.xx);
                S.b2 = pack2(ub, ub);
            }
        }
    }
}

__device__ __forceinline__ void block_radii(const ulonglong2 &e1a, const ulonglong2 &e1b,
                                            float (&Rt)[kBallBlock]) {
    const float2 ea = unpack2(e1a.x), eb = unpack2(e1a.y), ec = unpack2(e1b.x), ed = unpack2(e1b.y);
    Rt[0] = -0.5f * ea.x; Rt[1] = -0.5f * ea.y; Rt[2] = -0.5f * eb.x; Rt[3] = -0.5f * eb.y;
    Rt[4] = -0.5f * ec.x; Rt[5] = -0.5f * ec.y; Rt[6] = -0.5f * ed.x; Rt[7] = -0.5f * ed.y;
}

__device__ __forceinline__ float block_min(const f32x2 &L0, const f32x2 &L1, const f32x2 &L2, const f32x2 &L3,
                                           float (&Lt)[kBallBlock]) {
    const float2 l0 = unpack2(L0), l1 = unpack2(L1), l2 = unpack2(L2), l3 = unpack2(L3);
    Lt[0] = l0.x; Lt[1] = l0.y; Lt[2] = l1.x; Lt[3] = l1.y;
    Lt[4] = l2.x; Lt[5] = l2.y; Lt[6] = l3.x; Lt[7] = l3.y;
    return fminf(fmin3(l0.x, l0.y, l1.x), fmin3(fmin3(l1.y, l2.x, l2.y), l3.x, l3.y));
}

// After the scan: exact FP32 direct form for the best candidate (others bounded by lb2), then
// the component order goal, balls, outer, faces (strict '<').
template <int D>
__device__ __forceinline__ float screen_finish(const ScreenState &S, const ulonglong2 *B2,
                                               const f32x2 (&x2)[D], float goal, float other,
                                               int okind, int oidx, int m, int &kind, int &idx) {
    float best = CUDART_INF_F;
    kind = -1;
    idx = -1;
    if (goal < best) { best = goal; kind = kGoal; idx = 0; }
    float bball = CUDART_INF_F;
    if (S.bidx >= 0) {
        const float *Bf = reinterpret_cast<const float *>(B2 + (S.bidx / kBallBlock) * 2 * (D + 2));
        const int t = S.bidx % kBallBlock;
        const float s2 = sum_coords<D>(m, [&](int j, float a) {
            const float dj = fmaf(0.5f, Bf[kBallBlock * j + t], xj(x2, j));  // x_j - c_j
            return fmaf(dj, dj, a);
        });
        bball = fminf(sqrtf(s2) + 0.5f * Bf[kBallBlock * (D + 1) + t], S.lb2);
    }
    if (bball < best) { best = bball; kind = kBall; idx = S.bidx; }
    if (other < best) { best = other; kind = okind; idx = oidx; }
    return best;
}

template <int D, bool ARM>
__device__ __forceinline__ float distance_mixed(const MixedProblem &P, const float *geom,
                                                const float4 *balls, int nblk,
                                                const f32x2 (&x2)[D], float slack, int &kind,
                                                int &idx) {
    float goal, other;
    int okind, oidx;
    other_components<D, ARM>(P, geom, x2, goal, other, okind, oidx);
    ScreenState S;
    screen_init<D>(S, x2, fminf(goal, other), slack, P.proj);
    const ulonglong2 *B2 = reinterpret_cast<const ulonglong2 *>(balls);
    constexpr int H = D / 2;
#pragma unroll 1
    for (int blk = 0; blk < nblk; ++blk) {
        const ulonglong2 *F = B2 + blk * 2 * (D + 2);
        const ulonglong2 e0a = F[2 * D], e0b = F[2 * D + 1];
        const ulonglong2 e1a = F[2 * D + 2], e1b = F[2 * D + 3];
        f32x2 L0 = ffma2(e1a.x, S.b2, e0a.x);
        f32x2 L1 = ffma2(e1a.y, S.b2, e0a.y);
        f32x2 L2 = ffma2(e1b.x, S.b2, e0b.x);
        f32x2 L3 = ffma2(e1b.y, S.b2, e0b.y);
        f32x2 M0 = 0ull, M1 = 0ull, M2 = 0ull, M3 = 0ull;
#pragma unroll
        for (int j = 0; j < H; ++j) {
            const ulonglong2 ma = F[2 * j], mb = F[2 * j + 1];
            const ulonglong2 na = F[2 * (j + H)], nb = F[2 * (j + H) + 1];
            L0 = ffma2(x2[j], ma.x, L0);
            L1 = ffma2(x2[j], ma.y, L1);
            L2 = ffma2(x2[j], mb.x, L2);
            L3 = ffma2(x2[j], mb.y, L3);
            M0 = ffma2(x2[j + H], na.x, M0);
            M1 = ffma2(x2[j + H], na.y, M1);
            M2 = ffma2(x2[j + H], nb.x, M2);
            M3 = ffma2(x2[j + H], nb.y, M3);
        }
        if constexpr (D % 2 == 1) {
            const ulonglong2 ma = F[2 * (D - 1)], mb = F[2 * (D - 1) + 1];
            L0 = ffma2(x2[D - 1], ma.x, L0);
            L1 = ffma2(x2[D - 1], ma.y, L1);
            L2 = ffma2(x2[D - 1], mb.x, L2);
            L3 = ffma2(x2[D - 1], mb.y, L3);
        }
        const f32x2 one2 = pack2(1.f, 1.f);
        L0 = ffma2(one2, M0, L0);
        L1 = ffma2(one2, M1, L1);
        L2 = ffma2(one2, M2, L2);
        L3 = ffma2(one2, M3, L3);
        float Lt[kBallBlock];
        if (block_min(L0, L1, L2, L3, Lt) < S.thr) {
            float Rt[kBallBlock];
            block_radii(e1a, e1b, Rt);
            screen_passing(S, Lt, Rt, slack, blk);
        }
    }
    return screen_finish<D>(S, B2, x2, goal, other, okind, oidx, P.proj, kind, idx);
}

// Closest boundary point and g there, in log space: returns g(xbar) exp(logw) and
// e[k] = exp(a_k . xbar + logw).
template <int D>
__device__ __forceinline__ float terminal_value(const MixedProblem &P, const float *geom,
                                                const float4 *balls, const f32x2 (&x2)[D],
                                                int kind, int idx, float logw,
                                                float (&e)[kMaxExp]) {
    float xb[D];
    float cc[D];
    float rad = 0.f;
    bool sphere = false;
    if (kind == kGoal || kind == kOuter) {
        const float *c = geom + (kind == kGoal ? 2 * D : 3 * D);
#pragma unroll
        for (int j = 0; j < D; ++j) cc[j] = c[j];
        rad = kind == kGoal ? P.goal_r : P.outer_r;
        sphere = true;
    } else if (kind == kBall) {
        const float *Bf = reinterpret_cast<const float *>(balls + (idx / kBallBlock) * 2 * (D + 2));
        const int t = idx % kBallBlock;
#pragma unroll
        for (int j = 0; j < D; ++j) cc[j] = -0.5f * Bf[kBallBlock * j + t];
        rad = -0.5f * Bf[kBallBlock * (D + 1) + t];
        sphere = true;
    }
    if (sphere) {
        // an extruded domain projects in the measured coordinates and keeps the free ones
        const int m = P.proj;
        const float s = sum_coords<D>(m, [&](int j, float a) {
            const float t = xj(x2, j) - cc[j];
            return fmaf(t, t, a);
        });
        const float len = sqrtf(s);
        const float f = len > 0.f ? rad / len : 0.f;
#pragma unroll
        for (int j = 0; j < D; ++j)
            xb[j] = j >= m ? xj(x2, j)
                           : (len > 0.f ? fmaf(f, xj(x2, j) - cc[j], cc[j]) : cc[j] + (j == 0 ? rad : 0.f));
    } else {
#pragma unroll
        for (int j = 0; j < D; ++j) xb[j] = xj(x2, j);
        if (kind == kFace) {
            const int jf = idx >> 1;
#pragma unroll
            for (int j = 0; j < D; ++j)
                if (j == jf) xb[j] = (idx & 1) ? geom[D + j] : geom[j];
        }
    }
    if (P.n_exp > 0) {
        float g = 0.f;
        const float *w = geom + 4 * D;
        const float *a = geom + 4 * D + kMaxExp;
#pragma unroll
        for (int k = 0; k < kMaxExp; ++k) {
            if (k < P.n_exp) {
                float dot = logw;
#pragma unroll
                for (int j = 0; j < D; ++j) dot = fmaf(a[k * D + j], xb[j], dot);
                e[k] = expf(dot);
                g = fmaf(w[k], e[k], g);
            }
        }
        return g;
    }
    return kind == kGoal ? expf(logw) : 0.f;
}

// Writes the record of one finished walk (layout at rec_words): one 16-byte store of
// [term, dv, gt, info] (dv: d term / d sigma), the first direction when the reduction needs it,
// and the du/dw terms when the walk has a value.
template <int D>
__device__ __forceinline__ void write_record(const MixedProblem &P, long long j, int outcome, int k, float term,
                                             float dv, float gt, bool has_v0, const float (&v0)[D],
                                             const float (&e)[kMaxExp]) {
    if (P.rec == nullptr) return;
    float *r = P.rec + j * P.rec_words;
    const unsigned info = ((unsigned)k & kRecKMask) | ((unsigned)outcome << kRecOutcomeShift) | (has_v0 ? kRecHasV0 : 0u);
    *reinterpret_cast<float4 *>(r) = make_float4(term, dv, gt, __uint_as_float(info));
    if (has_v0) {  // only gradient walks (grad_mode) have the v0 words
#pragma unroll
        for (int i = 0; i + 3 < D; i += 4) *reinterpret_cast<float4 *>(r + 4 + i) = make_float4(v0[i], v0[i + 1], v0[i + 2], v0[i + 3]);
#pragma unroll
        for (int i = D & ~3; i < D; ++i) r[4 + i] = v0[i];
    }
    if (term != 0.f) {
        float *re = r + 4 + (P.grad_mode ? D : 0);  // the layout of rec_words(d, K, grad_mode)
#pragma unroll
        for (int kk = 0; kk < kMaxExp; ++kk)
            if (kk < P.n_exp) re[kk] = e[kk];
    }
}

// Warp-aggregated grab of one walk index per calling lane from the item's shared counter.
__device__ __forceinline__ unsigned grab_walk(MixedSmem &S) {
    const unsigned mask = __activemask();
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(mask) - 1;
    const unsigned rank = __popc(mask & ((1u << lane) - 1u));
    unsigned base = 0;
    if (lane == leader) base = atomicAdd(&S.next_walk, (unsigned)__popc(mask));
    base = __shfl_sync(mask, base, leader);
    return base + rank;
}

template <int D, bool GRAD>
__device__ __forceinline__ void start_walk(const MixedProblem &P, MixedWalker<D> &W, unsigned j) {
    W.j = j;
    W.q = (long long)(j / (unsigned long long)P.N);
    const double *xq = P.x + W.q * D;
#pragma unroll
    for (int i = 0; i < D; ++i) {
        const float v = (float)__ldg(xq + i);
        W.x2[i] = pack2(v, v);
    }
    W.logw = 0.f;
    W.dsig = 0.f;
    W.gfac0 = 0.f;
    W.src = 0.f;
    W.src0 = 0.f;
    W.dsrc = 0.f;
    W.k = 0;
}

// ---- impulse source: Green's function of the largest empty ball, FP32 -------------------
// log K_nu(x) and log K_{nu+1}(x), x > 0, from int_0^inf exp(-x cosh t) cosh(mu t) dt
// (DLMF 10.32.9) by the trapezoidal rule; step min(1/2, 1.1/sqrt(x)) keeps the relative error
// near 1e-7, and the sum is scaled by the peak of exp(-x cosh t + (nu+1) t).
__device__ __forceinline__ void log_bessel_K_pair_f32(float nu, float x, float &l0, float &l1) {
    const float mu = nu + 1.f;
    const float ts = asinhf(mu / x);
    const float m = mu * ts - x * coshf(ts);
    const float h = fminf(0.5f, 1.1f * rsqrtf(x));
    float s0 = 0.f, s1 = 0.f;
    for (int i = 0; i < 512; ++i) {
        const float t = h * (float)i, c = x * coshf(t), w = i == 0 ? 0.5f : 1.f;
        const float e1 = mu * t - c - m;
        s1 += w * (expf(e1) + expf(-mu * t - c - m));
        s0 += w * (expf(nu * t - c - m) + expf(-nu * t - c - m));
        if (t > ts && e1 < -18.f) break;
    }
    l0 = m + logf(0.5f * h * s0);
    l1 = m + logf(0.5f * h * s1);
}

// log K_{|nu-1|}(x), log K_nu(x) and log K_{nu+1}(x) by the same rule (for dG_B/dsigma).
__device__ __forceinline__ void log_bessel_K_triple_f32(float nu, float x, float &lm, float &l0, float &l1) {
    const float mu = nu + 1.f, mm = fabsf(nu - 1.f);
    const float ts = asinhf(mu / x);
    const float m = mu * ts - x * coshf(ts);
    const float h = fminf(0.5f, 1.1f * rsqrtf(x));
    float sm = 0.f, s0 = 0.f, s1 = 0.f;
    for (int i = 0; i < 512; ++i) {
        const float t = h * (float)i, c = x * coshf(t), w = i == 0 ? 0.5f : 1.f;
        const float e1 = mu * t - c - m;
        s1 += w * (expf(e1) + expf(-mu * t - c - m));
        s0 += w * (expf(nu * t - c - m) + expf(-nu * t - c - m));
        sm += w * (expf(mm * t - c - m) + expf(-mm * t - c - m));
        if (t > ts && e1 < -18.f) break;
    }
    lm = m + logf(0.5f * h * sm);
    l0 = m + logf(0.5f * h * s0);
    l1 = m + logf(0.5f * h * s1);
}

// dG_B/dsigma between the centre and distance r, FP32 forms without cancellation.
//   sigma = 0: minus the radial solution w1 of -Laplace(w1) = G_0 with w1 = 0 on the sphere.
//   d = 2, kR < 0.15: -w1 + 2 sigma w2 with -Laplace(w2) = w1 (G_B = G_0 - sigma w1 + sigma^2 w2
//     - ...), truncation below 1e-4 of the derivative's size.
//   otherwise: dG/dsigma = c0 r^-nu K_nu(kr) / (2k) times
//     [-r K_{nu-1}(kr)/K_nu(kr) + R X K_{nu-1}(kR)/K_nu(kR) - X k (r^2 s(kr) - R^2 s(kR))/(2(nu+1))],
//     X = K_nu(kR) Q / K_nu(kr), Q = I_nu(kr)/I_nu(kR), s = S_{nu+1}/S_nu: the derivative of
//     c0 r^-nu [K_nu(kr) - K_nu(kR) Q] in k with K_nu' = -K_{nu-1} - (nu/x) K_nu (DLMF 10.29.2),
//     which is K_nu' = -K_{nu+1} + (nu/x) K_nu rewritten by the recurrence so that the 1/k terms
//     cancel analytically; K_{nu-1} = K_{|nu-1|}.
template <int D>
__device__ __forceinline__ float source_green_dsigma0_f32(float inv_omega, float r, float R) {
    if constexpr (D == 2) {
        return (0.25f * r * r * logf(R / r) + 0.25f * (r * r - R * R)) * (0.5f / CUDART_PI_F);
    } else if constexpr (D == 4) {
        return (-0.5f * logf(R / r) - r * r / (8.f * R * R) + 0.125f) * (0.5f * inv_omega);
    } else {
        constexpr float a = 1.f / (2.f * (4.f - (float)D)), b = 1.f / (2.f * (float)D);
        return (a * powf(r, 4.f - D) - b * r * r * powf(R, 2.f - D) - (a - b) * powf(R, 4.f - D)) *
               (inv_omega / (float)(D - 2));
    }
}

// G = G_B between the centre of a ball of radius R and a point at distance r < R, and F with
// grad_x G_B = F (y - x)/r at the centre (Laplace(u) - sigma u = -delta, zero values on the
// sphere): c0 r^-nu [K_mu(kr) - K_mu(kR) I_mu(kr)/I_mu(kR)] for mu = nu (G) and nu + 1 (F,
// times k), the I ratios from the weight table (log S_nu = -log C_nu; S_nu+1 / S_nu); tR is the
// table entry at kR. Laplace forms at sigma = 0. Evaluated in log space.
template <int D>
__device__ __forceinline__ void source_green_f32(const MixedProblem &P, float r, float R, float2 tR, float &G,
                                                 float &F, float &dG) {
    const float nu = 0.5f * (float)D - 1.f;
    const float k = P.sqrt_sigma;
    const float lr = logf(r), lR = logf(R);
    if (k == 0.f) {
        G = D == 2 ? (lR - lr) * (0.5f / CUDART_PI_F)
                   : (expf((2.f - D) * lr) - expf((2.f - D) * lR)) * (P.src_inv_omega / (float)(D - 2));
        F = (expf((1.f - D) * lr) - r * expf(-(float)D * lR)) * P.src_inv_omega;
        dG = source_green_dsigma0_f32<D>(P.src_inv_omega, r, R);
        return;
    }
    float kam, ka0, ka1, kbm, kb0, kb1;
    log_bessel_K_triple_f32(nu, k * r, kam, ka0, ka1);
    log_bessel_K_triple_f32(nu, k * R, kbm, kb0, kb1);
    const float2 ta = table_lookup(P.table, k * r);
    const float lSa0 = -ta.x, lSb0 = -tR.x;
    const float lSa1 = lSa0 + logf(ta.y), lSb1 = lSb0 + logf(tR.y);
    const float P0 = expf(P.src_lc0 - nu * lr + ka0);
    const float X = expf(kb0 - ka0 + nu * (lr - lR) + lSa0 - lSb0);
    G = P0 * (1.f - X);
    F = expf(P.src_lc0 + logf(k) - nu * lr + ka1) *
        (1.f - expf(kb1 - ka1 + (nu + 1.f) * (lr - lR) + lSa1 - lSb1));
    if (D == 2 && k * R < 0.15f) {
        const float L = logf(R / r), r2 = r * r, R2 = R * R;
        const float w1 = (0.25f * R2 - 0.25f * r2 - 0.25f * r2 * L) * (0.5f / CUDART_PI_F);
        const float w2 = (-(R2 * r2 * (1.f / 16.f) - r2 * r2 * (6.f / 256.f) - r2 * r2 * (1.f / 64.f) * L) +
                          R2 * R2 * (10.f / 256.f)) *
                         (0.5f / CUDART_PI_F);
        dG = -w1 + 2.f * (k * k) * w2;
    } else {
        const float br = -r * expf(kam - ka0) + R * X * expf(kbm - kb0) -
                         X * k * (r * r * ta.y - R * R * tR.y) / (2.f * (nu + 1.f));
        dG = P0 * br / (2.f * k);
    }
}

// The source term of one step (not inlined: walkers without a source keep their registers):
// if the ball B(x_k, R) contains the source, add q G_B(x_k, z) times the weight so far; at
// step 0 of a gradient walk also record that value and store the query's step-0 value and
// source part of the gradient, q grad_x G_B(x_0, z) (every walk of the query writes the same).
template <int D, bool GRAD>
__device__ __noinline__ void source_step(const MixedProblem &P, MixedWalker<D> &W, float R, float2 t) {
    float rr = 0.f;
#pragma unroll
    for (int i = 0; i < D; ++i) {
        const float dz = P.source_z[i] - xj(W.x2, i);
        rr = fmaf(dz, dz, rr);
    }
    const float r = sqrtf(rr);
    if (!(r > 0.f && r < R)) return;
    float G, F, dG;
    source_green_f32<D>(P, r, R, t, G, F, dG);
    const float qw = P.source_q * expf(W.logw);
    const float c = qw * G;
    W.src += c;
    // d/dsigma: the weight's (the d log C / d sigma of the steps before) and G_B's
    W.dsrc += qw * fmaf(W.dsig, G, dG);
    if (GRAD && W.k == 0) {
        W.src0 = c;
        if (P.src) {
            double *sp = P.acc + W.q * acc_fields(D, P.n_exp, P.cv, 1) + src_field(D, P.n_exp, P.cv);
            sp[0] = (double)c;
#pragma unroll
            for (int i = 0; i < D; ++i) sp[1 + i] = (double)(P.source_q * F * (P.source_z[i] - xj(W.x2, i)) / r);
        }
    }
}

template <int D, bool GRAD>
__device__ __forceinline__ void first_walk(const MixedProblem &P, MixedSmem &S, MixedWalker<D> &W,
                                           unsigned end) {
#pragma unroll
    for (int i = 0; i < D; ++i) W.x2[i] = 0ull;
    const unsigned j = grab_walk(S);
    W.active = j < end;
    if (W.active) start_walk<D, GRAD>(P, W, j);
}

// Everything after the distance of one step: the eps test, the cap, the jump (sphere sample,
// screened weight, first-sphere gradient factor) or the end of the walk (boundary value,
// contribution, per-walk record) and the refill.
template <int D, bool GRAD>
__device__ __forceinline__ void step_walker(const MixedLaunch &L, const MixedProblem &P, MixedSmem &S,
                                            const float4 *balls, const float *geom, MixedWalker<D> &W,
                                            float R, int kind, int idx, unsigned end) {
    int outcome = 0;  // 0 jump, 1 boundary reached, 2 capped, 3 query outside, 4 roulette
    if (W.k == 0 && !(R > 0.f))
        outcome = 3;
    else if (R < P.eps && !(GRAD && P.grad_mode && W.k == 0))
        outcome = 1;
    else if (W.k >= L.max_steps)
        outcome = 2;
    else if (P.roulette_w > 0.f && W.k > 0 && W.logw < P.log_roulette_w) {
        // Russian roulette: survive with probability W / w_min carrying w_min
        if (roulette_uniform(L.seed, (uint64_t)(P.walk_base + (long long)W.j), (uint32_t)W.k) <
            expf(W.logw - P.log_roulette_w))
            W.logw = P.log_roulette_w;
        else
            outcome = 4;
    }
    if (outcome == 0) {
        float v[D];
        // antithetic pairs: the first direction of walk 2m + 1 is the negated one of walk 2m
        const uint64_t walk = (uint64_t)(P.walk_base + (long long)W.j);
        const bool first = W.k == 0;
        direction_f32<D, true>(L.seed, first ? first_direction_walk(walk, P.antithetic) : walk, (uint32_t)W.k, v);
        const float sgn = first && first_direction_negated(walk, P.antithetic) ? -1.f : 1.f;
        const float2 t = table_lookup(P.table, R * P.sqrt_sigma);
        if (P.has_source) source_step<D, GRAD>(P, W, R, t);
        if (GRAD && W.k == 0) {
            // alpha(R0) u^(x_1) = (d/R0) C_{nu+1}(z0) term / C_nu(z0) = (d/R0) term / ratio(z0)
            W.gfac0 = P.laplace ? ((float)D / R) * __expf(-t.x) : ((float)D / R) / t.y;
        }
        W.logw += t.x;
        W.dsig = fmaf(-(R * R) * (1.0f / (2.0f * (float)D)), t.y, W.dsig);
        const float Rs = sgn * R;
#pragma unroll
        for (int i = 0; i < D; ++i) {
            const float xn = fmaf(Rs, v[i], xj(W.x2, i));
            W.x2[i] = pack2(xn, xn);
        }
        ++W.k;
        return;
    }
    // ---- the walk ended: contribution, per-walk record, refill
    float term = 0.f;
    float e[kMaxExp];
#pragma unroll
    for (int k = 0; k < kMaxExp; ++k) e[k] = 0.f;
    if (outcome == 1) term = terminal_value<D>(P, geom, balls, W.x2, kind, idx, W.logw, e) + W.src;
    if (outcome == 4) term = W.src;  // ended by the roulette: the source contributions so far
    // (a value-only problem in a gradient launch has no gradient terms: its records carry none)
    const bool has_grad = GRAD && P.grad_mode && (outcome == 1 || outcome == 4) && W.k > 0;
    const bool cv_walk = GRAD && P.cv && W.k > 0 && outcome != 3;  // capped walks count too
    float v0[D];
#pragma unroll
    for (int i = 0; i < D; ++i) v0[i] = 0.f;
    // the first direction, regenerated from its counter: for the gradient terms, and for every
    // walk that took its first sphere when the control variate sums sum v0 and sum v0^2
    const bool need_v0 = (has_grad && (term != 0.f || W.src0 != 0.f)) || cv_walk;
    if constexpr (GRAD) {
        if (need_v0) {
            const uint64_t walk = (uint64_t)(P.walk_base + (long long)W.j);
            direction_f32<D, true>(L.seed, first_direction_walk(walk, P.antithetic), 0u, v0);
            const float sgn = first_direction_negated(walk, P.antithetic) ? -1.f : 1.f;
#pragma unroll
            for (int i = 0; i < D; ++i) v0[i] *= sgn;
        }
    }
    // u^(x_1) C(R0): the walk's value without its step-0 source part
    const float gt = has_grad ? W.gfac0 * (term - W.src0) : 0.f;
    // control variate: G = alpha(R0)/C(R0) is one number per query (every walk writes the same)
    if (cv_walk && W.gfac0 != 0.f)
        P.acc[W.q * acc_fields(D, P.n_exp, P.cv, P.src) + cv_field(D, P.n_exp) + 3 * D] = (double)W.gfac0;
    // d/dsigma of the walk's value: its boundary part times the summed d log C / d sigma, plus the
    // source contributions' derivatives (a capped walk, value 0, has none)
    const float dv = outcome == 2 ? 0.f : fmaf(term - W.src, W.dsig, W.dsrc);
    write_record<D>(P, (long long)W.j, outcome, W.k, term, dv, gt, GRAD && need_v0, v0, e);
    if (P.w_term != nullptr) P.w_term[W.j] = outcome == 3 ? (double)CUDART_NAN : (double)term;
    if (P.w_jumps != nullptr) P.w_jumps[W.j] = W.k;
    if (P.w_dsigma != nullptr) P.w_dsigma[W.j] = outcome == 3 ? (double)CUDART_NAN : (double)dv;
    if (P.w_grad != nullptr) {
        // with a source, the per-query source part of the gradient (stored at step 0)
        const double *sp = P.src ? P.acc + W.q * acc_fields(D, P.n_exp, P.cv, 1) + src_field(D, P.n_exp, P.cv) : nullptr;
#pragma unroll
        for (int i = 0; i < D; ++i)
            P.w_grad[(long long)W.j * D + i] = (double)(gt * v0[i]) + (sp != nullptr ? sp[1 + i] : 0.0);
    }
    const unsigned nj = grab_walk(S);
    W.active = nj < end;
    if (W.active) start_walk<D, GRAD>(P, W, nj);
}

// Not inlined: each dimension gets its own register allocation instead of the maximum over
// all eleven specialisations of the kernel. One walker per thread.
template <int D, bool GRAD, bool ARM>
__device__ __noinline__ void run_item(const MixedLaunch &L, const MixedProblem &P, MixedSmem &S,
                                      const float4 *balls) {
    const int nblk = (P.n_balls + kBallBlock - 1) / kBallBlock;
    const float *geom = S.geom;
    const unsigned end = S.end_walk;
    MixedWalker<D> W;
    first_walk<D, GRAD>(P, S, W, end);
    while (__any_sync(0xffffffffu, W.active)) {
        if (!W.active) continue;
        int kind, idx;
        const float R = distance_mixed<D, ARM>(P, geom, balls, nblk, W.x2, P.slack, kind, idx) - P.shrink;
        step_walker<D, GRAD>(L, P, S, balls, geom, W, R, kind, idx, end);
    }
}

// MAXT: the largest CTA this instantiation is launched with (one CTA per SM); it sets the
// register budget (65536 / MAXT per thread).
template <bool GRAD, int MAXT>
__global__ void __launch_bounds__(MAXT, 1) walk_mixed_kernel(const __grid_constant__ MixedLaunch L) {
    extern __shared__ float4 smem_balls[];
    __shared__ MixedSmem S;
    __shared__ MixedProblem SP;
    if (L.skip != nullptr && *L.skip != 0) return;
    if (threadIdx.x == 0) S.problem = -1;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) {
            const long long it = (long long)atomicAdd(L.cursor, 1ull);
            S.item = it;
            if (it < L.n_items) {
                if (L.items != nullptr) {
                    const MixedItem I = L.items[it];
                    S.item_problem = I.problem;
                    S.next_walk = (unsigned)I.j0;
                    S.end_walk = (unsigned)I.j1;
                    // a planner path that has reached its goal runs no walks
                    const int *dn = L.problems != nullptr ? L.problems[I.problem].done : nullptr;
                    if (dn != nullptr && *(volatile const int *)dn != 0) S.end_walk = S.next_walk;
                } else {
                    const long long j0 = it * L.walks_per_item;
                    const long long j1 = j0 + L.walks_per_item;
                    S.item_problem = 0;
                    S.next_walk = (unsigned)j0;
                    S.end_walk = (unsigned)(j1 < L.total_walks ? j1 : L.total_walks);
                }
            }
        }
        __syncthreads();
        if (S.item >= L.n_items) break;
        const int pi = S.item_problem;
        if (pi != S.problem) {
            const MixedProblem *src = L.problems != nullptr ? L.problems + pi : &L.single;
            if (threadIdx.x == 0) SP = *src;
            const int d = src->d;
            const int nfl = ((src->n_balls + kBallBlock - 1) / kBallBlock) * 2 * (d + 2);
            const float4 *bsrc = reinterpret_cast<const float4 *>(src->balls);
            for (int i = threadIdx.x; i < nfl; i += blockDim.x) smem_balls[i] = __ldg(bsrc + i);
            const int ng = geom_count(d);
            for (int i = threadIdx.x; i < ng; i += blockDim.x) S.geom[i] = __ldg(src->geom + i);
            __syncthreads();
            if (threadIdx.x == 0) S.problem = pi;
        }
        switch (SP.d) {
#define WOS_CASE(DD) \
    case DD:                                                                       \
        if (DD <= kMaxArmLinksMixed && SP.n_links > 0)                                 \
            run_item<DD, GRAD, (DD <= kMaxArmLinksMixed)>(L, SP, S, smem_balls);       \
        else                                                                           \
            run_item<DD, GRAD, false>(L, SP, S, smem_balls);                           \
        break;
            WOS_CASE(2) WOS_CASE(3) WOS_CASE(4) WOS_CASE(5) WOS_CASE(6) WOS_CASE(7)
            WOS_CASE(8) WOS_CASE(9) WOS_CASE(10) WOS_CASE(11) WOS_CASE(12)
#undef WOS_CASE
            default: break;
        }
    }
}

}  // namespace wos
