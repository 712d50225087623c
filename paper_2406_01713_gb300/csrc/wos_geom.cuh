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

template <typename T, int D>
__device__ __forceinline__ T norm_diff(const T (&x)[D], const T *c) {
    T s = T(0);
#pragma unroll
    for (int j = 0; j < D; ++j) {
        const T t = x[j] - c[j];
        s += t * t;
    }
    return sqrt(s);
}

// Distance to the boundary (minimum over components, strict '<' keeps the lowest id).
template <typename T, int D>
__device__ __forceinline__ T distance(const DomainView<T> &dm, const T (&x)[D], int &kind, int64_t &idx) {
    T best = inf_of<T>();
    kind = -1;
    idx = -1;
    if (dm.has_goal) {
        const T r = norm_diff<T, D>(x, dm.goal_c) - dm.goal_r;
        if (r < best) { best = r; kind = kGoal; idx = 0; }
    }
    for (int i = 0; i < dm.n_balls; ++i) {
        const T r = norm_diff<T, D>(x, dm.ball_c + (int64_t)i * D) - dm.ball_r[i];
        if (r < best) { best = r; kind = kBall; idx = i; }
    }
    for (int64_t i = 0; i < dm.n_points; ++i) {
        const T r = norm_diff<T, D>(x, dm.points + i * D);
        if (r < best) { best = r; kind = kPoint; idx = i; }
    }
    if (dm.has_outer) {
        const T r = dm.outer_r - norm_diff<T, D>(x, dm.outer_c);
        if (r < best) { best = r; kind = kOuter; idx = 0; }
    }
    if (dm.has_box) {
#pragma unroll
        for (int j = 0; j < D; ++j) {
            const T rlo = x[j] - dm.box_lo[j];
            if (rlo < best) { best = rlo; kind = kFace; idx = 2 * j; }
            const T rhi = dm.box_hi[j] - x[j];
            if (rhi < best) { best = rhi; kind = kFace; idx = 2 * j + 1; }
        }
    }
    return best;
}

// g at the closest boundary point xbar (Fig. 2); e[k] = exp(a_k . xbar) for exp data.
template <typename T, int D>
__device__ __forceinline__ T boundary_value(const DomainView<T> &dm, const T (&x)[D], int kind, int64_t idx,
                            T (&e)[kMaxExp]) {
    T xb[D];
    const T *c = nullptr;
    T rad = T(0);
    if (kind == kGoal) { c = dm.goal_c; rad = dm.goal_r; }
    if (kind == kBall) { c = dm.ball_c + idx * D; rad = dm.ball_r[idx]; }
    if (kind == kOuter) { c = dm.outer_c; rad = dm.outer_r; }
    if (c != nullptr) {
        const T len = norm_diff<T, D>(x, c);
#pragma unroll
        for (int j = 0; j < D; ++j)
            xb[j] = len > T(0) ? c[j] + rad * (x[j] - c[j]) / len : c[j] + (j == 0 ? rad : T(0));
    } else if (kind == kPoint) {
#pragma unroll
        for (int j = 0; j < D; ++j) xb[j] = dm.points[idx * D + j];
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

}  // namespace wos
