// Persistent mixed-precision Walk-on-Spheres walker (Sec. IV-A estimators, FP32 walkers).
//
// One launch serves many problems of uneven dimension, obstacle count and walk budget:
//   * a global work queue of items (problem, walk range) in longest-first order, pulled by
//     CTAs through an atomic cursor;
//   * the current problem's balls are staged in shared memory as 4-ball blocks
//     [m_0 x4][m_1 x4]...[m_{d-1} x4][e0 x4][e1 x4] with m = -2c, e0 = |c|^2 - r^2, e1 = -2r,
//     so one 128-bit shared load fetches one field of four balls;
//   * every lane runs walks back to back, refilling from the item's walk counter the moment
//     its walk ends (walk lengths vary, so lanes never wait for the slowest walk of a batch);
//   * per-lane FP32 partial sums over the walks of one query, flushed to FP64 per-query
//     sums in global memory (warp-reduced when the whole warp holds the same query).
//
// Distance to the balls (Sec. VI, |x - c| - r): a ball can only beat the current best
// distance b if |x-c|^2 < (r+b)^2, i.e. if
//     L = e0 + e1 b + x.m  <  b^2 - |x|^2.
// L is evaluated in FP32 for every ball (d+1 FMAs) and compared against the threshold plus a
// slack E that bounds the FP32 rounding of both sides, so no true candidate is ever missed;
// candidates are then refined with the direct form sqrt(sum (x_j - c_j)^2) - r.
// The radius used for the jump is the computed distance minus `shrink`, a bound on the FP32
// error of the distance evaluation and of the position update, so every sphere lies inside
// the FP64 domain.
#pragma once

#include <cuda_runtime.h>
#include <math_constants.h>

#include "wos_launch.h"

namespace wos {

struct MixedSmem {
    float geom[4 * kMaxD + kMaxExp + kMaxExp * kMaxD];
    int problem;
    int item_problem;
    unsigned next_walk;
    unsigned end_walk;
    unsigned begin_walk;
    long long item;
};

template <int D>
struct MixedWalker {
    float x[D];
    float logw, dsig, gfac0;  // gfac0 = alpha(R0) / C(R0); v0 is regenerated from its counter
    int k;
    unsigned j;      // walk index within the problem
    long long q;     // query
    bool active;
};

// geom layout in shared memory: [0,d) box lo, [d,2d) box hi, [2d,3d) goal c, [3d,4d) outer c,
// [4d, 4d+K) exp w, then K x d exp a.
template <int D>
__device__ __forceinline__ float distance_mixed(const MixedProblem &P, const float *geom,
                                                const float4 *balls, int nblk,
                                                const float (&x)[D], float slack, int &kind,
                                                int &idx) {
    float best = CUDART_INF_F;
    kind = -1;
    idx = -1;
    if (P.has_goal) {
        float s = 0.f;
#pragma unroll
        for (int j = 0; j < D; ++j) {
            const float t = x[j] - geom[2 * D + j];
            s = fmaf(t, t, s);
        }
        const float r = sqrtf(s) - P.goal_r;
        if (r < best) { best = r; kind = kGoal; idx = 0; }
    }
    // Balls are searched below; the other components go first so that `best` starts small.
    float other = CUDART_INF_F;
    int okind = -1, oidx = -1;
    if (P.has_outer) {
        float s = 0.f;
#pragma unroll
        for (int j = 0; j < D; ++j) {
            const float t = x[j] - geom[3 * D + j];
            s = fmaf(t, t, s);
        }
        const float r = P.outer_r - sqrtf(s);
        if (r < other) { other = r; okind = kOuter; oidx = 0; }
    }
    if (P.has_box) {
#pragma unroll
        for (int j = 0; j < D; ++j) {
            const float rlo = x[j] - geom[j];
            if (rlo < other) { other = rlo; okind = kFace; oidx = 2 * j; }
            const float rhi = geom[D + j] - x[j];
            if (rhi < other) { other = rhi; okind = kFace; oidx = 2 * j + 1; }
        }
    }
    // Running upper bound used by the ball screen (ties and ordering are resolved below).
    float b = fminf(best, other);
    float xx = 0.f;
#pragma unroll
    for (int j = 0; j < D; ++j) xx = fmaf(x[j], x[j], xx);
    float thr = fmaf(b, b, slack - xx);
    float bball = CUDART_INF_F;
    int bidx = -1;
#pragma unroll 1
    for (int blk = 0; blk < nblk; ++blk) {
        const float4 *B = balls + blk * (D + 2);
        const float4 e0 = B[D];
        const float4 e1 = B[D + 1];
        float4 L;
        L.x = fmaf(e1.x, b, e0.x);
        L.y = fmaf(e1.y, b, e0.y);
        L.z = fmaf(e1.z, b, e0.z);
        L.w = fmaf(e1.w, b, e0.w);
#pragma unroll
        for (int j = 0; j < D; ++j) {
            const float4 m = B[j];
            L.x = fmaf(x[j], m.x, L.x);
            L.y = fmaf(x[j], m.y, L.y);
            L.z = fmaf(x[j], m.z, L.z);
            L.w = fmaf(x[j], m.w, L.w);
        }
        const bool c0 = L.x < thr, c1 = L.y < thr, c2 = L.z < thr, c3 = L.w < thr;
        if (c0 | c1 | c2 | c3) {
            const float *Bf = reinterpret_cast<const float *>(B);
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                const bool ct = t == 0 ? c0 : (t == 1 ? c1 : (t == 2 ? c2 : c3));
                if (ct) {
                    float s = 0.f;
#pragma unroll
                    for (int j = 0; j < D; ++j) {
                        const float dj = fmaf(0.5f, Bf[4 * j + t], x[j]);  // x_j - c_j
                        s = fmaf(dj, dj, s);
                    }
                    const float r = -0.5f * Bf[4 * (D + 1) + t];
                    const float dist = sqrtf(s) - r;
                    if (dist < bball) {
                        bball = dist;
                        bidx = 4 * blk + t;
                        if (dist < b) {
                            b = dist;
                            thr = fmaf(b, b, slack - xx);
                        }
                    }
                }
            }
        }
    }
    // Combine in the component order goal, balls, outer, faces (strict '<').
    if (bball < best) { best = bball; kind = kBall; idx = bidx; }
    if (other < best) { best = other; kind = okind; idx = oidx; }
    return best;
}

// Closest boundary point and g there, in log space: returns log(g) + logw contributions as
// t = g * exp(logw) and e[k] = exp(a_k . xbar + logw).
template <int D>
__device__ __forceinline__ float terminal_value(const MixedProblem &P, const float *geom,
                                                const float4 *balls, const float (&x)[D],
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
        const float *Bf = reinterpret_cast<const float *>(balls + (idx >> 2) * (D + 2));
        const int t = idx & 3;
#pragma unroll
        for (int j = 0; j < D; ++j) cc[j] = -0.5f * Bf[4 * j + t];
        rad = -0.5f * Bf[4 * (D + 1) + t];
        sphere = true;
    }
    if (sphere) {
        float s = 0.f;
#pragma unroll
        for (int j = 0; j < D; ++j) {
            const float t = x[j] - cc[j];
            s = fmaf(t, t, s);
        }
        const float len = sqrtf(s);
        const float f = len > 0.f ? rad / len : 0.f;
#pragma unroll
        for (int j = 0; j < D; ++j)
            xb[j] = len > 0.f ? fmaf(f, x[j] - cc[j], cc[j]) : cc[j] + (j == 0 ? rad : 0.f);
    } else {
#pragma unroll
        for (int j = 0; j < D; ++j) xb[j] = x[j];
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

// Per-lane FP32 partial sums of one query: [u, u^2, du/dsigma, (grad[D], grad^2[D]), dw_0].
// Boundary-data derivatives dw_k for k >= 1 go straight to the FP64 sums at walk end.
template <int D, bool GRAD>
struct LaneAcc {
    static constexpr int kG = GRAD ? 2 * D : 0;  // gradient fields present
    static constexpr int kN = 3 + kG + 1;
    float s[kN];
    unsigned c[kCounters];
    long long q;
};

template <int D, bool GRAD>
__device__ __forceinline__ void lane_acc_clear(LaneAcc<D, GRAD> &A) {
#pragma unroll
    for (int f = 0; f < LaneAcc<D, GRAD>::kN; ++f) A.s[f] = 0.f;
#pragma unroll
    for (int f = 0; f < kCounters; ++f) A.c[f] = 0u;
}

// Global FP64 field index of lane-accumulator field f.
template <int D, bool GRAD>
__device__ __forceinline__ int acc_global_field(int f) {
    return f < 3 + LaneAcc<D, GRAD>::kG ? f : f - (3 + LaneAcc<D, GRAD>::kG) + 3 + 2 * D;
}

template <int D, bool GRAD>
__device__ __forceinline__ void lane_acc_flush(const MixedProblem &P, const LaneAcc<D, GRAD> &A) {
    const int nf = acc_fields(D, P.n_exp);
    double *acc = P.acc + A.q * nf;
    constexpr int kE = 3 + LaneAcc<D, GRAD>::kG;
#pragma unroll
    for (int f = 0; f < kE; ++f) atomicAdd(acc + f, (double)A.s[f]);
    if (P.n_exp > 0) atomicAdd(acc + 3 + 2 * D, (double)A.s[kE]);
    unsigned long long *cnt = P.counts + A.q * kCounters;
#pragma unroll
    for (int f = 0; f < kCounters; ++f)
        if (A.c[f]) atomicAdd(cnt + f, (unsigned long long)A.c[f]);
}

// End of an item: warp-reduce when all lanes hold the same query, else flush lane by lane.
template <int D, bool GRAD>
__device__ __forceinline__ void lane_acc_final(const MixedProblem &P, LaneAcc<D, GRAD> &A) {
    const unsigned peers = __match_any_sync(0xffffffffu, A.q);
    if (peers == 0xffffffffu) {
        if (A.q < 0) return;
        constexpr int kE = 3 + LaneAcc<D, GRAD>::kG;
        const int nf = acc_fields(D, P.n_exp);
#pragma unroll
        for (int f = 0; f < LaneAcc<D, GRAD>::kN; ++f) {
            if (f >= kE && f - kE >= P.n_exp) continue;  // warp-uniform
            double dv = (double)A.s[f];
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) dv += __shfl_xor_sync(0xffffffffu, dv, off);
            if ((threadIdx.x & 31) == 0) atomicAdd(P.acc + A.q * nf + acc_global_field<D, GRAD>(f), dv);
        }
#pragma unroll
        for (int f = 0; f < kCounters; ++f) {
            unsigned long long v = A.c[f];
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
            if ((threadIdx.x & 31) == 0 && v) atomicAdd(P.counts + A.q * kCounters + f, v);
        }
    } else if (A.q >= 0) {
        lane_acc_flush<D, GRAD>(P, A);
    }
    A.q = -1;
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
    for (int i = 0; i < D; ++i) W.x[i] = (float)__ldg(xq + i);
    W.logw = 0.f;
    W.dsig = 0.f;
    W.gfac0 = 0.f;
    W.k = 0;
}

template <int D, bool GRAD>
__device__ void run_item(const MixedLaunch &L, const MixedProblem &P, MixedSmem &S,
                         const float4 *balls) {
    const int nblk = (P.n_balls + 3) >> 2;
    const float *geom = S.geom;
    const unsigned end = S.end_walk;
    const float inv2d = 1.0f / (2.0f * (float)D);
    MixedWalker<D> W;
    LaneAcc<D, GRAD> A;
    lane_acc_clear<D, GRAD>(A);
    A.q = -1;
    {
        const unsigned j = grab_walk(S);
        W.active = j < end;
        if (W.active) start_walk<D, GRAD>(P, W, j);
    }
    while (__any_sync(0xffffffffu, W.active)) {
        if (!W.active) continue;
        int kind, idx;
        const float R =
            distance_mixed<D>(P, geom, balls, nblk, W.x, P.slack, kind, idx) - P.shrink;
        int outcome = 0;  // 0 jump, 1 boundary reached, 2 capped, 3 query outside
        if (W.k == 0 && !(R > 0.f))
            outcome = 3;
        else if (R < P.eps && !(GRAD && P.grad_mode && W.k == 0))
            outcome = 1;
        else if (W.k >= L.max_steps)
            outcome = 2;
        if (outcome == 0) {
            float v[D];
            direction_f32<D, true>(L.seed, (uint64_t)(P.walk_base + (long long)W.j),
                                   (uint32_t)W.k, v);
            const float2 t = table_lookup(P.table, R * P.sqrt_sigma);
            if (GRAD && W.k == 0) {
                // alpha(R0) u^(x_1) = (d/R0) C_{nu+1}(z0) term / C_nu(z0) = (d/R0) term / ratio(z0)
                W.gfac0 = P.laplace ? ((float)D / R) * __expf(-t.x) : ((float)D / R) / t.y;
            }
            W.logw += t.x;
            W.dsig = fmaf(-(R * R) * inv2d, t.y, W.dsig);
#pragma unroll
            for (int i = 0; i < D; ++i) W.x[i] = fmaf(R, v[i], W.x[i]);
            ++W.k;
            continue;
        }
        // ---- the walk ended: contribution, per-walk record, refill
        float term = 0.f;
        float e[kMaxExp];
#pragma unroll
        for (int k = 0; k < kMaxExp; ++k) e[k] = 0.f;
        if (outcome == 1) term = terminal_value<D>(P, geom, balls, W.x, kind, idx, W.logw, e);
        if (A.q != W.q) {
            if (A.q >= 0) lane_acc_flush<D, GRAD>(P, A);
            lane_acc_clear<D, GRAD>(A);
            A.q = W.q;
        }
        const bool has_grad = GRAD && outcome == 1 && W.k > 0;
        float v0[D];
        if constexpr (GRAD) {
            if (has_grad) {
                direction_f32<D, true>(L.seed, (uint64_t)(P.walk_base + (long long)W.j), 0u, v0);
            } else {
#pragma unroll
                for (int i = 0; i < D; ++i) v0[i] = 0.f;
            }
        }
        if (outcome != 3) {
            A.s[0] += term;
            A.s[1] = fmaf(term, term, A.s[1]);
            A.s[2] = fmaf(term, W.dsig, A.s[2]);
            if constexpr (GRAD) {
                const float gt = W.gfac0 * term;
#pragma unroll
                for (int i = 0; i < D; ++i) {
                    const float g = gt * v0[i];
                    A.s[3 + i] += g;
                    A.s[3 + D + i] = fmaf(g, g, A.s[3 + D + i]);
                }
            }
            A.s[3 + LaneAcc<D, GRAD>::kG] += e[0];
            if (P.n_exp > 1) {
                double *accq = P.acc + W.q * acc_fields(D, P.n_exp) + 3 + 2 * D;
#pragma unroll
                for (int k = 1; k < kMaxExp; ++k)
                    if (k < P.n_exp) atomicAdd(accq + k, (double)e[k]);
            }
        }
        A.c[0] += 1u;
        A.c[1] += (unsigned)(W.k + 1);
        A.c[2] += outcome == 2 ? 1u : 0u;
        A.c[3] += outcome == 3 ? 1u : 0u;
        if (P.w_term != nullptr) P.w_term[W.j] = outcome == 3 ? (double)CUDART_NAN : (double)term;
        if (P.w_jumps != nullptr) P.w_jumps[W.j] = W.k;
        if (P.w_dsigma != nullptr) P.w_dsigma[W.j] = (double)(term * W.dsig);
        if (P.w_grad != nullptr) {
            const float gt = has_grad ? W.gfac0 * term : 0.f;
#pragma unroll
            for (int i = 0; i < D; ++i)
                P.w_grad[(long long)W.j * D + i] = GRAD ? (double)(gt * v0[i]) : 0.0;
        }
        const unsigned nj = grab_walk(S);
        W.active = nj < end;
        if (W.active) start_walk<D, GRAD>(P, W, nj);
    }
    lane_acc_final<D, GRAD>(P, A);
}

template <bool GRAD>
__global__ void __launch_bounds__(512, 1) walk_mixed_kernel(const __grid_constant__ MixedLaunch L) {
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
            const int nfl = ((src->n_balls + 3) >> 2) * (d + 2);
            const float4 *bsrc = reinterpret_cast<const float4 *>(src->balls);
            for (int i = threadIdx.x; i < nfl; i += blockDim.x) smem_balls[i] = __ldg(bsrc + i);
            const int ng = 4 * d + kMaxExp + kMaxExp * d;
            for (int i = threadIdx.x; i < ng; i += blockDim.x) S.geom[i] = __ldg(src->geom + i);
            __syncthreads();
            if (threadIdx.x == 0) S.problem = pi;
        }
        switch (SP.d) {
#define WOS_CASE(DD) \
    case DD: run_item<DD, GRAD>(L, SP, S, smem_balls); break;
            WOS_CASE(2) WOS_CASE(3) WOS_CASE(4) WOS_CASE(5) WOS_CASE(6) WOS_CASE(7)
            WOS_CASE(8) WOS_CASE(9) WOS_CASE(10) WOS_CASE(11) WOS_CASE(12)
#undef WOS_CASE
            default: break;
        }
    }
}

}  // namespace wos
