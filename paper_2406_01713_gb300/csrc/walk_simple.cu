// One-thread-per-walk Walk-on-Spheres walkers (Sec. IV-A):
//   T = double : FP64 parity mode. Same component order, same Philox counters and the same
//                direct normaliser series as the definition, so every walk can be compared
//                with an FP64 reference walk by walk.
//   T = float  : the plain FP32 walker used as the speed baseline: obstacles read from global
//                memory, FP32 normaliser series evaluated every step, FP32 per-query sums.
#include <cuda_runtime.h>
#include <math_constants.h>

#include "wos_geom.cuh"
#include "wos_launch.h"

namespace wos {
namespace {

template <typename T, int D>
struct WalkResult {
    T term, dsig;
    T grad[D];
    T v0[D];   // first direction if the walk took its first sphere (control variate), else 0
    T G;       // alpha(R0)/C(R0) if the walk took its first sphere, else 0
    T s0;      // impulse source: value added at step 0 (the same for every walk of the query)
    T gsrc[D]; // impulse source: q grad_x G_B(x0, z), the source part of the gradient
    T dw[kMaxExp];
    int64_t jumps;
    int capped, outside, killed;
};

template <int D>
__device__ __forceinline__ void direction(uint64_t seed, uint64_t walk, uint32_t step,
                                          double (&v)[D]) {
    direction_f64<D>(seed, walk, step, v);
}
template <int D>
__device__ __forceinline__ void direction(uint64_t seed, uint64_t walk, uint32_t step,
                                          float (&v)[D]) {
    direction_f32<D, false>(seed, walk, step, v);
}

template <typename T, int D>
__device__ void run_walk(const SimpleParams<T> &p, const double *xq, uint64_t walk,
                         WalkResult<T, D> &res) {
    const DomainView<T> &dm = p.dom;
    const T nu = T(0.5) * T(D) - T(1);
    T x[D], v[D], v0[D];
#pragma unroll
    for (int j = 0; j < D; ++j) {
        x[j] = (T)xq[j];
        v0[j] = T(0);
    }
    T logw = T(0), dsig = T(0), R0 = T(0), logC0 = T(0), S1_0 = T(1);
    T src = T(0);   // impulse-source contributions of the steps so far
    T dsrc = T(0);  // their sigma derivatives
    int64_t k = 0;
    int kind = -1;
    int64_t idx = -1;
    res.term = T(0);
    res.dsig = T(0);
    res.capped = 0;
    res.outside = 0;
    res.killed = 0;
#pragma unroll
    for (int i = 0; i < kMaxExp; ++i) res.dw[i] = T(0);
#pragma unroll
    for (int j = 0; j < D; ++j) res.grad[j] = res.v0[j] = res.gsrc[j] = T(0);
    res.G = T(0);
    res.s0 = T(0);
    for (;;) {
        const T R = distance<T, D>(dm, x, kind, idx) - p.shrink;
        if (k == 0 && !(R > T(0))) {
            res.outside = 1;
            res.jumps = 0;
            return;
        }
        if (R < p.eps && !(p.grad_mode && k == 0)) {
            T e[kMaxExp];
            const T g = boundary_value<T, D>(dm, x, kind, idx, e);
            const T w = exp(logw);
            res.term = g * w + src;
#pragma unroll
            for (int i = 0; i < kMaxExp; ++i)
                if (i < dm.n_exp) res.dw[i] = w * e[i];
            break;
        }
        if (k == p.max_steps) {
            res.capped = 1;
            res.term = T(0);
            break;
        }
        if (p.roulette_w > 0.0 && k > 0) {
            // Russian roulette on the weight W: survive with probability W / w_min carrying w_min,
            // or end with the source contributions so far and no boundary value
            const T W = exp(logw);
            if (W < (T)p.roulette_w) {
                const T u = (T)roulette_uniform(p.seed, walk, (uint32_t)k);
                if (u < W / (T)p.roulette_w) {
                    logw = log((T)p.roulette_w);
                } else {
                    res.killed = 1;
                    res.term = src;
                    break;
                }
            }
        }
        if (dm.has_source) {
            // the ball B(x_k, R) contains the source: q G_B(x_k, z) times the weight so far
            // (evaluated in FP64 in both precisions)
            double rr = 0.0;
#pragma unroll
            for (int j = 0; j < D; ++j) {
                const double t = (double)dm.source_z[j] - (double)x[j];
                rr += t * t;
            }
            const double r = sqrt(rr);
            if (r > 0.0 && r < (double)R) {
                double G, F, dG;
                source_green_f64(D, (double)p.sqrt_sigma, r, (double)R, G, F, &dG);
                const double qw = (double)dm.source_q * exp((double)logw);
                const T c = (T)(qw * G);
                src += c;
                // d/dsigma: the weight's (the d log C / d sigma of the steps before) and G_B's
                dsrc += (T)(qw * ((double)dsig * G + dG));
                if (k == 0) {
                    res.s0 = c;
#pragma unroll
                    for (int j = 0; j < D; ++j)
                        res.gsrc[j] = (T)((double)dm.source_q * F * ((double)dm.source_z[j] - (double)x[j]) / r);
                }
            }
        }
        if (k == 0) {
            direction<D>(p.seed, first_direction_walk(walk, p.antithetic), 0u, v);
            if (first_direction_negated(walk, p.antithetic)) {
#pragma unroll
                for (int j = 0; j < D; ++j) v[j] = -v[j];
            }
        } else {
            direction<D>(p.seed, walk, (uint32_t)k, v);
        }
        const T z = R * p.sqrt_sigma;
        const T S0 = bessel_S<T>(nu, z);
        const T S1 = bessel_S<T>(nu + T(1), z);
        const T logC = -log(S0);
        if (k == 0) {
            R0 = R;
            logC0 = logC;
            S1_0 = S1;
#pragma unroll
            for (int j = 0; j < D; ++j) v0[j] = v[j];
        }
        logw += logC;
        dsig += -(R * R / (T(2) * T(D))) * S1 / S0;
#pragma unroll
        for (int j = 0; j < D; ++j) x[j] = x[j] + R * v[j];
        ++k;
    }
    res.jumps = k;
    // d/dsigma of the walk's value (the walk geometry does not depend on sigma): the boundary
    // part times the summed d log C / d sigma plus the source contributions' derivatives; a
    // capped walk contributes 0
    res.dsig = res.capped ? T(0) : (res.term - src) * dsig + dsrc;
    if (k > 0) {
        const T factor = p.laplace ? T(D) / R0 : (T(D) / R0) / S1_0;
        if (p.cv) {
            res.G = factor * exp(-logC0);
#pragma unroll
            for (int j = 0; j < D; ++j) res.v0[j] = v0[j];
        }
        if (!res.capped) {
            // u^(x_1) C(R0): the walk's value without its step-0 source part
            const T u1 = (res.term - res.s0) * exp(-logC0);
#pragma unroll
            for (int j = 0; j < D; ++j) res.grad[j] = factor * u1 * v0[j];
        }
    }
}

// Sum of v over the lanes of this lane's segment that follow it (segments = runs of equal
// query index in consecutive lanes); the first lane of a segment gets the segment total.
template <typename V>
__device__ __forceinline__ V segment_sum(V v, int lane, int seg_end) {
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const V o = __shfl_down_sync(0xffffffffu, v, off);
        if (lane + off <= seg_end) v += o;
    }
    return v;
}

template <typename T, int D>
__global__ void __launch_bounds__(128) walk_simple_kernel(const SimpleParams<T> p) {
    if (p.skip != nullptr && *p.skip != 0) return;
    const int lane = threadIdx.x & 31;
    const int64_t total = p.Q * p.N;
    const int K = p.dom.n_exp;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < total;
         base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = base + threadIdx.x;
        const bool active = j < total;
        const int64_t q = active ? j / p.N : -1;
        WalkResult<T, D> r;
        r.jumps = 0;
        r.term = T(0);
        r.killed = 0;
        if (active) {
            run_walk<T, D>(p, p.x + q * D, (uint64_t)(p.walk_offset + j), r);
            if (p.w_term) p.w_term[j] = r.outside ? (double)CUDART_NAN : (double)r.term;
            if (p.w_jumps) p.w_jumps[j] = r.jumps;
            if (p.w_dsigma) p.w_dsigma[j] = (double)r.dsig;
            if (p.w_grad)
                for (int i = 0; i < D; ++i) p.w_grad[j * D + i] = (double)r.grad[i] + (double)r.gsrc[i];
        } else {
            r.outside = 0;
            r.capped = 0;
        }
        __syncwarp();
        // Per-query reduction: consecutive walks share a query, so reduce runs of equal q.
        const unsigned peers = __match_any_sync(0xffffffffu, (long long)q);
        const int seg_end = 31 - __clz(peers);
        const bool leader = (lane == __ffs(peers) - 1) && q >= 0;
        const bool ok = active && !r.outside;
        // squares: of the walk's value, or with antithetic pairs (lanes 2i, 2i + 1 hold the walks
        // 2m, 2m + 1 of one query: N and the walk offset are even) of the pair mean, on the even lane
        auto square = [&](T v) -> T {
            if (!p.antithetic) return v * v;
            const T m = T(0.5) * (v + __shfl_xor_sync(0xffffffffu, v, 1));
            return (lane & 1) ? T(0) : m * m;
        };
        const T t_ok = ok ? r.term : T(0);
        T vals[3] = {t_ok, square(t_ok), ok ? r.dsig : T(0)};
        T *acc = p.acc + (q >= 0 ? q : 0) * p.nf;
#pragma unroll
        for (int f = 0; f < 3; ++f) {
            const T s = segment_sum(vals[f], lane, seg_end);
            if (leader) atomicAdd(acc + f, s);
        }
#pragma unroll
        for (int i = 0; i < D; ++i) {
            const T g = ok ? r.grad[i] : T(0);
            const T s1 = segment_sum(g, lane, seg_end);
            const T s2 = segment_sum(square(g), lane, seg_end);
            if (leader) {
                atomicAdd(acc + 3 + i, s1);
                atomicAdd(acc + 3 + D + i, s2);
            }
        }
        for (int k = 0; k < K; ++k) {
            const T s = segment_sum(ok ? r.dw[k] : T(0), lane, seg_end);
            if (leader) atomicAdd(acc + 3 + 2 * D + k, s);
        }
        if (p.cv) {
            // [sum v0, sum t v0^2, sum v0^2, G]; G is the same for every walk of the query
            T *cvp = acc + cv_field(D, K);
#pragma unroll
            for (int i = 0; i < D; ++i) {
                const T v = ok ? r.v0[i] : T(0);
                const T tt = ok ? r.term : T(0);
                const T s1 = segment_sum(v, lane, seg_end);
                const T s2 = segment_sum(tt * v * v, lane, seg_end);
                const T s3 = segment_sum(v * v, lane, seg_end);
                if (leader) {
                    atomicAdd(cvp + i, s1);
                    atomicAdd(cvp + D + i, s2);
                    atomicAdd(cvp + 2 * D + i, s3);
                }
            }
            if (ok && r.G != T(0)) cvp[3 * D] = r.G;
        }
        if (p.src && ok && r.jumps > 0) {
            // impulse source: step-0 value and gradient part, one per query (plain stores of
            // the same values)
            T *sp = acc + src_field(D, K, p.cv);
            sp[0] = r.s0;
#pragma unroll
            for (int i = 0; i < D; ++i) sp[1 + i] = r.gsrc[i];
        }
        const unsigned long long c[kCounters] = {active ? 1ull : 0ull,
                                                 active ? (unsigned long long)(r.jumps + 1) : 0ull,
                                                 (unsigned long long)(active && r.capped),
                                                 (unsigned long long)(active && r.outside),
                                                 (unsigned long long)(active && r.killed)};
        unsigned long long *cnt = p.counts + (q >= 0 ? q : 0) * kCounters;
#pragma unroll
        for (int f = 0; f < kCounters; ++f) {
            const unsigned long long s = segment_sum(c[f], lane, seg_end);
            if (leader) atomicAdd(cnt + f, s);
        }
    }
}

template <typename T>
cudaError_t launch_simple(const SimpleParams<T> &p, cudaStream_t s) {
    const int threads = 128;
    const int64_t total = p.Q * p.N;
    if (total <= 0) return cudaSuccess;
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int64_t blocks = (total + threads - 1) / threads;
    const int64_t cap = (int64_t)sms * 16;
    if (blocks > cap) blocks = cap;
    switch (p.dom.d) {
#define WOS_CASE(DD) \
    case DD: walk_simple_kernel<T, DD><<<(unsigned)blocks, threads, 0, s>>>(p); break;
        WOS_CASE(2) WOS_CASE(3) WOS_CASE(4) WOS_CASE(5) WOS_CASE(6) WOS_CASE(7)
        WOS_CASE(8) WOS_CASE(9) WOS_CASE(10) WOS_CASE(11) WOS_CASE(12)
#undef WOS_CASE
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_walk_simple_f64(const SimpleParams<double> &p, cudaStream_t s) {
    return launch_simple<double>(p, s);
}
cudaError_t launch_walk_simple_f32(const SimpleParams<float> &p, cudaStream_t s) {
    return launch_simple<float>(p, s);
}

}  // namespace wos
