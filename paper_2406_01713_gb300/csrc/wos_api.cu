// Host side of the C ABI declared in include/wos.h: domain objects, weight tables,
// walker launches, per-query finalisation, planner, backward and the batched persistent
// launch with its CUDA graph and autotuner.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "wos_geom.cuh"
#include "wos_launch.h"

using namespace wos;

// =====================================================================================
// errors
// =====================================================================================
namespace {

thread_local std::string g_err;

wos_status fail(wos_status s, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return s;
}

#define WOS_CUDA(call)                                                                    \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess)                                                            \
            return fail(WOS_ERR_CUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), \
                        __FILE__, __LINE__);                                              \
    } while (0)

#define WOS_TRY(expr)                     \
    do {                                  \
        wos_status s_ = (expr);           \
        if (s_ != WOS_OK) return s_;      \
    } while (0)

const double kU32 = 5.9604644775390625e-08;  // FP32 unit roundoff 2^-24

int device_sms() {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 1;
    return sms > 0 ? sms : 1;
}

}  // namespace

// =====================================================================================
// domain
// =====================================================================================
// Weight table on the fixed grid z_i = i / kTableNodesPerUnit, i = 0 .. kTableNodesPerUnit 2^level,
// covering z in [0, 2^level]. Every table of a dimension has the same nodes, so the interpolated
// weights depend on z alone: not on sigma, and not on which tables earlier calls built.
struct TableEntry {
    int level = 0;
    float2 *nodes = nullptr;
    cudaEvent_t built = nullptr;  // recorded after an asynchronous build; null once it completed
};

struct wos_domain_s {
    int d = 0, has_box = 0, has_outer = 0, has_goal = 0, n_balls = 0, n_exp = 0;
    int has_source = 0;
    int proj = 0;  // coordinates the components are measured in (d, or fewer when extruded)
    int n_links = 0;        // planar arm: joints 0..n_links-1 (0: none)
    int64_t n_arm_obs = 0;  // its task-space obstacle points
    double arm_K = 0;       // Lipschitz constant of its kinematics
    std::vector<double> link_l, arm_obs;
    int64_t n_points = 0;
    double outer_r = 0, goal_r = 0, source_q = 0;
    std::vector<double> box_lo, box_hi, outer_c, goal_c, exp_w, exp_a, ball_r, ball_c, points, source_z;
    double R_max = 0;     // upper bound of any distance to the boundary
    double shrink32 = 0;  // FP32 distance + jump error bound
    double slack32 = 0;   // FP32 ball-screen rounding bound
    double *f64 = nullptr;
    float *f32 = nullptr;
    DomainView<double> v64{};
    DomainView<float> v32{};
    float *balls_mixed = nullptr;  // 4-ball blocks for shared-memory staging
    float *geom_mixed = nullptr;   // box lo/hi, goal c, outer c, exp w (padded), exp a (padded)
    int nblk = 0;
    std::mutex mu;
    std::vector<TableEntry> tables;  // one per z-range level, built once
    PointCloudDev pcd{};  // tensor-core operands of the sphere set (point set or large ball set)
    bool has_pcd = false;
    float pc_delta = 0.f;
};

namespace {

template <typename T>
void layout_view(DomainView<T> &v, T *base, const wos_domain_s &D) {
    const int d = D.d, K = D.n_exp;
    const int64_t B = D.n_balls, M = D.n_points;
    T *p = base;
    v.d = d;
    v.n_balls = D.n_balls;
    v.n_exp = K;
    v.has_box = D.has_box;
    v.has_outer = D.has_outer;
    v.has_goal = D.has_goal;
    v.has_source = D.has_source;
    v.proj = D.proj;
    v.n_points = M;
    v.outer_r = (T)D.outer_r;
    v.goal_r = (T)D.goal_r;
    v.source_q = (T)D.source_q;
    v.box_lo = p; p += d;
    v.box_hi = p; p += d;
    v.outer_c = p; p += d;
    v.goal_c = p; p += d;
    v.exp_w = p; p += K;
    v.exp_a = p; p += (int64_t)K * d;
    v.ball_r = p; p += B;
    v.ball_c = p; p += B * d;
    v.points = p; p += M * d;
    v.source_z = p; p += d;
    v.n_links = D.n_links;
    v.n_arm_obs = D.n_arm_obs;
    v.arm_inv_K = D.n_links > 0 ? (T)(1.0 / D.arm_K) : T(0);
    v.link_l = p; p += D.n_links;
    v.arm_obs = p; p += 2 * D.n_arm_obs;
}

int64_t view_size(const wos_domain_s &D) {
    return 5LL * D.d + D.n_exp + (int64_t)D.n_exp * D.d + D.n_balls + (int64_t)D.n_balls * D.d +
           D.n_points * D.d + D.n_links + 2 * D.n_arm_obs;
}

template <typename T>
std::vector<T> pack_view(const wos_domain_s &D) {
    std::vector<T> h((size_t)view_size(D), T(0));
    size_t o = 0;
    auto put = [&](const std::vector<double> &v, size_t n) {
        for (size_t i = 0; i < n; ++i) h[o + i] = (T)(i < v.size() ? v[i] : 0.0);
        o += n;
    };
    const size_t d = D.d;
    put(D.box_lo, d);
    put(D.box_hi, d);
    put(D.outer_c, d);
    put(D.goal_c, d);
    put(D.exp_w, D.n_exp);
    put(D.exp_a, (size_t)D.n_exp * d);
    put(D.ball_r, D.n_balls);
    put(D.ball_c, (size_t)D.n_balls * d);
    put(D.points, (size_t)D.n_points * d);
    put(D.source_z, d);
    put(D.link_l, D.n_links);
    put(D.arm_obs, 2 * D.n_arm_obs);
    return h;
}

int geom_floats(int d) { return geom_count(d); }

// Error bounds of the FP32 walkers (rounding unit u = 2^-24):
//  * shrink: distance |x-c| - r evaluated in FP32 is within u((d+4)/2 (|x|+|c|) + R + |c| + r)
//    of the exact distance at the FP32 point; the jump x + R v moves by at most
//    R (1 + (d+5) u) + u |x|. Twice the sum keeps every sphere inside the FP64 domain.
//  * slack: the screen L = e0 + e1 b + x.m and the threshold b^2 - |x|^2 are FMA chains whose
//    partial sums are bounded by P = |c|^2 + r^2 + 2 r b + 2 |x||c| and b^2 + |x|^2.
//  An extruded domain measures its components in the first m = proj coordinates only, so the
//  position bounds L, |x_j| and the centre norms are taken over those (the free coordinates are
//  unbounded but never enter a distance); the jump term keeps the full dimension.
void error_bounds(wos_domain_s &D) {
    const int d = D.d, m = D.proj;
    double xabs = 0.0;  // bound of |x_j| inside the domain, j < m
    double xa_box = 0.0, xa_out = 0.0;
    if (D.has_box)
        for (int j = 0; j < m; ++j) xa_box = std::max({xa_box, std::fabs(D.box_lo[j]), std::fabs(D.box_hi[j])});
    if (D.has_outer)
        for (int j = 0; j < m; ++j) xa_out = std::max(xa_out, std::fabs(D.outer_c[j]) + D.outer_r);
    if (D.has_box && D.has_outer) xabs = std::min(xa_box, xa_out);
    else xabs = D.has_box ? xa_box : xa_out;
    const double L = std::sqrt((double)m) * xabs;
    double cmax = 0.0, rmax = 0.0, ccmax = 0.0;
    for (int i = 0; i < D.n_balls; ++i) {
        double cc = 0.0;
        for (int j = 0; j < m; ++j) cc += D.ball_c[(size_t)i * d + j] * D.ball_c[(size_t)i * d + j];
        ccmax = std::max(ccmax, cc);
        rmax = std::max(rmax, D.ball_r[i]);
    }
    for (int64_t i = 0; i < D.n_points; ++i) {
        double cc = 0.0;
        for (int j = 0; j < m; ++j) cc += D.points[(size_t)i * d + j] * D.points[(size_t)i * d + j];
        ccmax = std::max(ccmax, cc);
    }
    cmax = std::sqrt(ccmax);
    double cgo = 0.0;
    if (D.has_goal) {
        double cc = 0.0;
        for (int j = 0; j < m; ++j) cc += D.goal_c[j] * D.goal_c[j];
        cgo = std::sqrt(cc) + D.goal_r;
    }
    if (D.has_outer) {
        double cc = 0.0;
        for (int j = 0; j < m; ++j) cc += D.outer_c[j] * D.outer_c[j];
        cgo = std::max(cgo, std::sqrt(cc) + D.outer_r);
    }
    const double C = std::max(cmax, cgo);
    const double R = D.R_max;
    double dist_err = ((m + 4) / 2.0) * (L + C) + R + C + rmax + xabs;
    if (D.n_links > 0) {
        // the arm's safe-ball radius in FP32: the joint angles summed (n u sum |q|), sine and
        // cosine of angle / pi (the division: u |angle|; sincospi: 2 u), the link end points
        // (n u reach), the projection on each link and its square root (10 u (|obstacle| + reach)),
        // divided by K
        const int n = D.n_links;
        double reach = 0.0, omax = 0.0, qsum = 0.0;
        for (int i = 0; i < n; ++i) {
            reach += D.link_l[i];
            qsum += xabs;
        }
        for (int64_t o = 0; o < D.n_arm_obs; ++o)
            omax = std::max(omax, std::hypot(D.arm_obs[2 * o], D.arm_obs[2 * o + 1]));
        const double arm = reach * ((n + 1) * qsum + 2.0 + n) + 10.0 * (omax + reach);
        dist_err = std::max(dist_err, arm / D.arm_K);
    }
    const double jump_err = (d + 5) * R + L;
    D.shrink32 = 2.0 * kU32 * (dist_err + jump_err);
    const double P = ccmax + rmax * rmax + 2.0 * rmax * R + 2.0 * L * cmax;
    D.slack32 = 2.0 * (d + 4) * kU32 * (P + R * R + 2.0 * L * L);
}

// Table of log C_nu(z) and S_{nu+1}(z)/S_nu(z), built in FP64 on the device.
__global__ void build_table_kernel(int d, double h, int64_t n, float2 *out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double z = h * i;
    const double nu = 0.5 * d - 1.0;
    const double S0 = bessel_S<double>(nu, z);
    const double S1 = bessel_S<double>(nu + 1.0, z);
    out[i] = make_float2((float)(-log(S0)), (float)(S1 / S0));
}

// Copies device FP64 weights w[K] into the FP64, FP32 and mixed copies of the domain.
__global__ void set_exp_w_kernel(const double *w, int K, double *w64, float *w32, float *wg) {
    const int k = threadIdx.x;
    if (k < K) {
        w64[k] = w[k];
        w32[k] = (float)w[k];
        wg[k] = (float)w[k];
    }
}

constexpr int kTableNodesPerUnit = 1024;  // node spacing 2^-10 in z
constexpr int kTableMaxLevel = 12;        // z up to 4096 (4M nodes, 32 MB)
int64_t table_nodes(int level) { return ((int64_t)kTableNodesPerUnit << level) + 1; }

// The smallest level whose table covers every z = R sqrt(sigma) of the domain, or -1 if none does.
int table_level(const wos_domain_s &D, double sigma) {
    const double need = D.R_max * std::sqrt(sigma) * 1.0001 + 1e-9;
    for (int level = 0; level <= kTableMaxLevel; ++level)
        if (std::ldexp(1.0, level) >= need) return level;
    return -1;
}

// A weight table covering `level` (any built table of that level or above: they agree on their
// common nodes). The first call that needs a larger one allocates it (cudaMalloc) and builds it
// on stream s. With sync the call waits for the build; otherwise it records an event that later
// calls on other streams wait for (on the device) until the build is seen complete.
wos_status ensure_table_level(wos_domain_t dom, int level, WeightTable *out, cudaStream_t s, bool sync) {
    if (level < 0)
        return fail(WOS_ERR_UNSUPPORTED, "sigma too large for the weight tables: R_max sqrt(sigma) above %d",
                    1 << kTableMaxLevel);
    std::lock_guard<std::mutex> lk(dom->mu);
    TableEntry *T = nullptr;
    for (TableEntry &t : dom->tables)
        if (t.level >= level && (T == nullptr || t.level > T->level)) T = &t;
    if (T == nullptr) {
        TableEntry t;
        t.level = level;
        const int64_t n = table_nodes(level);
        WOS_CUDA(cudaMalloc(&t.nodes, sizeof(float2) * (size_t)n));
        build_table_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(dom->d, 1.0 / kTableNodesPerUnit, n,
                                                                     t.nodes);
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess) {
            if (sync) e = cudaStreamSynchronize(s);
            else if ((e = cudaEventCreateWithFlags(&t.built, cudaEventDisableTiming)) == cudaSuccess)
                e = cudaEventRecord(t.built, s);
        }
        if (e != cudaSuccess) {
            if (t.built) cudaEventDestroy(t.built);
            cudaFree(t.nodes);
            return fail(WOS_ERR_CUDA, "weight table build failed: %s", cudaGetErrorString(e));
        }
        dom->tables.push_back(t);
        T = &dom->tables.back();
    } else if (T->built != nullptr) {
        const cudaError_t q = cudaEventQuery(T->built);
        if (q == cudaSuccess) {
            cudaEventDestroy(T->built);
            T->built = nullptr;
        } else if (q == cudaErrorNotReady && sync) {
            WOS_CUDA(cudaEventSynchronize(T->built));
            cudaEventDestroy(T->built);
            T->built = nullptr;
        } else if (q == cudaErrorNotReady) {
            WOS_CUDA(cudaStreamWaitEvent(s, T->built, 0));
        } else {
            return fail(WOS_ERR_CUDA, "weight table build failed: %s", cudaGetErrorString(q));
        }
    }
    out->nodes = T->nodes;
    out->n = (int)table_nodes(T->level);
    out->inv_h = (float)kTableNodesPerUnit;
    return WOS_OK;
}

wos_status ensure_table(wos_domain_t dom, double sigma, WeightTable *out, cudaStream_t s, bool sync) {
    return ensure_table_level(dom, table_level(*dom, sigma), out, s, sync);
}

// =====================================================================================
// per-query finalisation (u = mean, SE of the mean, grad, derivatives)
// =====================================================================================
struct FinalizeRec {
    int d, K, acc_f32;
    int anti;        // antithetic pairs: the squared fields hold squared pair means (N/2 pairs)
    int cv;          // gradient control variate sums present
    int src;         // impulse-source fields present (gradient walks)
    int64_t Q, N, q_begin;
    const void *acc;
    const unsigned long long *counts;
    double *u, *u_se, *grad, *grad_se, *du_dsigma, *du_dw;
    int64_t *walk_steps;
};

struct FinalizeArgs {
    const FinalizeRec *recs;  // device, or nullptr to use `single`
    int n;
    int64_t total_q;
    FinalizeRec single;
    wos_stats *stats;
    const int *status;                   // nonzero: the walker gave up (timeout); NaN outputs
    const unsigned long long *shrinks;   // point-cloud radius-bound events (nullable)
};

__device__ __forceinline__ double se_mean(double s, double s2, double n) {
    if (n < 2.0) return 0.0;
    const double var = (s2 - s * s / n) / (n - 1.0);
    return var > 0.0 ? sqrt(var / n) : 0.0;
}

__global__ void finalize_kernel(const __grid_constant__ FinalizeArgs a) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < a.total_q;
         t += (int64_t)gridDim.x * blockDim.x) {
        const FinalizeRec *R = &a.single;
        if (a.recs != nullptr) {
            int lo = 0, hi = a.n - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (a.recs[mid].q_begin <= t) lo = mid;
                else hi = mid - 1;
            }
            R = a.recs + lo;
        }
        const int64_t q = t - R->q_begin;
        const int d = R->d, K = R->K, nf = acc_fields(d, K, R->cv, R->src);
        auto S = [&](int f) -> double {
            return R->acc_f32 ? (double)((const float *)R->acc)[q * nf + f]
                              : ((const double *)R->acc)[q * nf + f];
        };
        const unsigned long long *c = R->counts + q * kCounters;
        const double n = (double)R->N;
        const double inv = 1.0 / n;
        const bool out = c[3] > 0 || (a.status != nullptr && *a.status != 0);
        if (t == 0 && a.stats != nullptr && a.shrinks != nullptr)
            atomicAdd(reinterpret_cast<unsigned long long *>(a.stats) + 4, *a.shrinks);
        if (t == 0 && a.stats != nullptr && a.status != nullptr && *a.status != 0)
            reinterpret_cast<unsigned long long *>(a.stats)[6] = (unsigned long long)*a.status;
        const double nan = CUDART_NAN;
        // standard errors: from the walks, or from the N/2 antithetic pair means (their sum is
        // half the walks' sum)
        const double sh = R->anti ? 0.5 : 1.0, ns = R->anti ? 0.5 * n : n;
        if (R->u) R->u[q] = out ? nan : S(0) * inv;
        if (R->u_se) R->u_se[q] = out ? nan : se_mean(sh * S(0), S(1), ns);
        if (R->du_dsigma) R->du_dsigma[q] = out ? nan : S(2) * inv;
        const bool cv = R->cv && n >= 2.0;
        const int cf = cv_field(d, K);
        // impulse source: the gradient sums hold G (t - s0) v0; s0 and the source part of the
        // gradient are one per query
        const int sf = src_field(d, K, R->cv);
        const double s0 = R->src ? S(sf) : 0.0;
        for (int i = 0; i < d; ++i) {
            double g = S(3 + i) * inv, se = se_mean(sh * S(3 + i), S(3 + d + i), ns);
            if (cv)  // sum (t - s0) = sum t - n s0, sum (t - s0) v^2 = sum t v^2 - s0 sum v^2
                cv_estimate(S(3 + i), S(3 + d + i), S(cf + i), S(cf + d + i) - s0 * S(cf + 2 * d + i),
                            S(cf + 2 * d + i), S(cf + 3 * d), S(0) - n * s0, n, g, se);
            if (R->src) g += S(sf + 1 + i);
            if (R->grad) R->grad[q * d + i] = out ? nan : g;
            if (R->grad_se) R->grad_se[q * d + i] = out ? nan : se;
        }
        for (int k = 0; k < K; ++k)
            if (R->du_dw) R->du_dw[q * K + k] = out ? nan : S(3 + 2 * d + k) * inv;
        if (R->walk_steps) R->walk_steps[q] = (int64_t)c[1];
        if (a.stats != nullptr) {
            unsigned long long *st = reinterpret_cast<unsigned long long *>(a.stats);
            atomicAdd(st + 0, c[0]);
            atomicAdd(st + 1, c[1]);
            if (c[2]) atomicAdd(st + 2, c[2]);
            if (c[3]) atomicAdd(st + 3, c[3]);
            if (c[4]) atomicAdd(st + 5, c[4]);
        }
    }
}

// =====================================================================================
// per-query reduction of the mixed walkers' per-walk records (fixed order, FP64)
// =====================================================================================
// The estimates of a query are sample means over its walks (Sec. IV-A). The mixed-precision
// walkers leave one FP32 record per walk (rec_words, wos_launch.h); one CTA sums the records of
// a segment of at most kReduceSegment walks of one query in FP64 -- each thread its strided
// share in walk order, then each warp's shuffle tree, then the warps in order -- and writes the
// query's sums (one segment) or the segment's partial sums, which reduce_combine_kernel adds in
// segment order. Every sum is formed in the same order on every run, so the outputs repeat bit
// for bit. Sums, in the layout of the query's accumulator (acc_fields):
//   [u, u^2, du/dsigma, grad (d), grad^2 (d), du/dw (K)] and, with the control variate,
//   [sum v0 (d), sum t v0^2 (d), sum v0^2 (d)]; counters [walks, walk-steps, capped, outside].
constexpr int kReduceSegment = 4096;
constexpr int kReduceThreads = 128;
constexpr int kReduceMaxSums = 3 + 2 * kMaxD + kMaxExp + 3 * kMaxD;

__host__ __device__ inline int reduce_sums(int d, int K, int cv) { return 3 + 2 * d + K + (cv ? 3 * d : 0); }

struct ReduceRec {
    int d, K, grad, cv, nf;      // nf: accumulator fields per query (acc_fields)
    int anti;                    // antithetic pairs: squares of pair means
    int rw;                      // record words
    int64_t Q, N;
    int64_t nseg;                // segments per query
    int64_t blk_begin;           // first reduce CTA of this problem
    int64_t q_begin;             // first combine CTA (query) of this problem
    const float *rec;            // Q N x rw
    double *acc;                 // Q x nf
    unsigned long long *counts;  // Q x kCounters
    double *part;                // Q x nseg x (sums + kCounters) when nseg > 1
};

struct ReduceArgs {
    const ReduceRec *recs;  // device array, or nullptr: `single`
    int n;
    int64_t total_blocks;   // reduce: sum of Q nseg; combine: sum of Q
    ReduceRec single;
    const int *skip;        // nullable; nothing is done if *skip != 0
};

__device__ __forceinline__ const ReduceRec *reduce_find(const ReduceArgs &a, int64_t t, bool by_query) {
    if (a.recs == nullptr) return &a.single;
    int lo = 0, hi = a.n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if ((by_query ? a.recs[mid].q_begin : a.recs[mid].blk_begin) <= t) lo = mid;
        else hi = mid - 1;
    }
    return a.recs + lo;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <int D>
__device__ void reduce_segment(const ReduceRec &R, int64_t q, int64_t seg, double (*red)[kReduceMaxSums],
                               unsigned long long (*redc)[kCounters]) {
    const int t = threadIdx.x, lane = t & 31, wp = t >> 5;
    double u = 0.0, u2 = 0.0, ds = 0.0, g[D], g2[D], dw[kMaxExp], sv[D], stv2[D], sv2[D];
#pragma unroll
    for (int i = 0; i < D; ++i) g[i] = g2[i] = sv[i] = stv2[i] = sv2[i] = 0.0;
#pragma unroll
    for (int k = 0; k < kMaxExp; ++k) dw[k] = 0.0;
    unsigned long long c[kCounters] = {0ull, 0ull, 0ull, 0ull, 0ull};
    const int64_t w0 = seg * kReduceSegment;
    const int64_t w1 = w0 + kReduceSegment < R.N ? w0 + kReduceSegment : R.N;
    const float *base = R.rec + (q * R.N) * R.rw;
    const int eoff = 4 + (R.grad ? D : 0);
    // one record: counters and plain sums; returns the walk's value and gradient terms (the
    // squares are added by the caller: per walk, or per antithetic pair mean)
    auto one = [&](int64_t w, double &tv, double (&gv)[D]) {
        tv = 0.0;
#pragma unroll
        for (int i = 0; i < D; ++i) gv[i] = 0.0;
        const float *r = base + w * R.rw;
        const float4 h = __ldg(reinterpret_cast<const float4 *>(r));
        const unsigned info = __float_as_uint(h.w);
        const int outcome = (int)((info >> kRecOutcomeShift) & kRecOutcomeMask);
        c[0] += 1ull;
        c[1] += (unsigned long long)(info & kRecKMask) + 1ull;
        c[2] += outcome == 2 ? 1ull : 0ull;
        c[3] += outcome == 3 ? 1ull : 0ull;
        c[4] += outcome == 4 ? 1ull : 0ull;
        if (outcome == 3) return;
        const double term = (double)h.x;
        const bool has_v0 = (info & kRecHasV0) != 0u;
        float v0[D];
#pragma unroll
        for (int i = 0; i < D; ++i) v0[i] = 0.f;
        if (has_v0) {
#pragma unroll
            for (int i = 0; i + 3 < D; i += 4) {
                const float4 v = __ldg(reinterpret_cast<const float4 *>(r + 4 + i));
                v0[i] = v.x;
                v0[i + 1] = v.y;
                v0[i + 2] = v.z;
                v0[i + 3] = v.w;
            }
#pragma unroll
            for (int i = D & ~3; i < D; ++i) v0[i] = __ldg(r + 4 + i);
        }
        ds += (double)h.y;  // the walk's d term / d sigma
        if (term != 0.0) {
            tv = term;
            u += term;
            if (h.z != 0.f) {
#pragma unroll
                for (int i = 0; i < D; ++i) {
                    gv[i] = (double)h.z * (double)v0[i];
                    g[i] += gv[i];
                }
            }
#pragma unroll
            for (int k = 0; k < kMaxExp; ++k)
                if (k < R.K) dw[k] += (double)__ldg(r + eoff + k);
        }
        if (R.cv && has_v0) {
#pragma unroll
            for (int i = 0; i < D; ++i) {
                const double vi = (double)v0[i];
                sv[i] += vi;
                sv2[i] += vi * vi;
                stv2[i] += term * vi * vi;
            }
        }
    };
    if (!R.anti) {
        for (int64_t w = w0 + t; w < w1; w += kReduceThreads) {
            double tv, gv[D];
            one(w, tv, gv);
            u2 += tv * tv;
#pragma unroll
            for (int i = 0; i < D; ++i) g2[i] += gv[i] * gv[i];
        }
    } else {
        // antithetic pairs (2m, 2m + 1): the squares of the pair means (segments start even)
        for (int64_t w = w0 + 2 * t; w + 1 < w1; w += 2 * kReduceThreads) {
            double ta, ga[D], tb, gb[D];
            one(w, ta, ga);
            one(w + 1, tb, gb);
            const double m = 0.5 * (ta + tb);
            u2 += m * m;
#pragma unroll
            for (int i = 0; i < D; ++i) {
                const double mg = 0.5 * (ga[i] + gb[i]);
                g2[i] += mg * mg;
            }
        }
    }
    // the warps' shuffle trees, then the warps in order
    int f = 0;
    auto put = [&](double v) {
        v = warp_sum(v);
        if (lane == 0) red[wp][f] = v;
        ++f;
    };
    put(u);
    put(u2);
    put(ds);
#pragma unroll
    for (int i = 0; i < D; ++i) put(g[i]);
#pragma unroll
    for (int i = 0; i < D; ++i) put(g2[i]);
#pragma unroll
    for (int k = 0; k < kMaxExp; ++k)
        if (k < R.K) put(dw[k]);
    if (R.cv) {
#pragma unroll
        for (int i = 0; i < D; ++i) put(sv[i]);
#pragma unroll
        for (int i = 0; i < D; ++i) put(stv2[i]);
#pragma unroll
        for (int i = 0; i < D; ++i) put(sv2[i]);
    }
#pragma unroll
    for (int k = 0; k < kCounters; ++k) {
        const unsigned long long v = warp_sum_u64(c[k]);
        if (lane == 0) redc[wp][k] = v;
    }
    __syncthreads();
    const int nsum = f;
    constexpr int kWarps = kReduceThreads / 32;
    if (t < nsum + kCounters) {
        if (t < nsum) {
            double v = 0.0;
#pragma unroll
            for (int w = 0; w < kWarps; ++w) v += red[w][t];
            if (R.nseg == 1) R.acc[q * R.nf + t] = v;
            else R.part[(q * R.nseg + seg) * (nsum + kCounters) + t] = v;
        } else {
            unsigned long long v = 0;
#pragma unroll
            for (int w = 0; w < kWarps; ++w) v += redc[w][t - nsum];
            if (R.nseg == 1) R.counts[q * kCounters + (t - nsum)] = v;
            else
                reinterpret_cast<unsigned long long *>(R.part)[(q * R.nseg + seg) * (nsum + kCounters) + t] = v;
        }
    }
}

__global__ void __launch_bounds__(kReduceThreads) reduce_kernel(const __grid_constant__ ReduceArgs a) {
    __shared__ double red[kReduceThreads / 32][kReduceMaxSums];
    __shared__ unsigned long long redc[kReduceThreads / 32][kCounters];
    if (a.skip != nullptr && *a.skip != 0) return;
    for (int64_t b = blockIdx.x; b < a.total_blocks; b += gridDim.x) {
        const ReduceRec *R = reduce_find(a, b, false);
        const int64_t local = b - R->blk_begin;
        const int64_t q = local / R->nseg, seg = local % R->nseg;
        switch (R->d) {
#define WOS_CASE(DD) \
    case DD: reduce_segment<DD>(*R, q, seg, red, redc); break;
            WOS_CASE(2) WOS_CASE(3) WOS_CASE(4) WOS_CASE(5) WOS_CASE(6) WOS_CASE(7)
            WOS_CASE(8) WOS_CASE(9) WOS_CASE(10) WOS_CASE(11) WOS_CASE(12)
#undef WOS_CASE
            default: break;
        }
        __syncthreads();  // red is reused by the next segment
    }
}

// Queries with several segments: the segments' partial sums added in segment order (one CTA per
// query, one thread per sum).
__global__ void reduce_combine_kernel(const __grid_constant__ ReduceArgs a) {
    if (a.skip != nullptr && *a.skip != 0) return;
    for (int64_t b = blockIdx.x; b < a.total_blocks; b += gridDim.x) {
        const ReduceRec *R = reduce_find(a, b, true);
        if (R->nseg <= 1) continue;
        const int64_t q = b - R->q_begin;
        const int nsum = reduce_sums(R->d, R->K, R->cv);
        const int stride = nsum + kCounters;
        const double *p = R->part + q * R->nseg * stride;
        for (int f = threadIdx.x; f < stride; f += blockDim.x) {
            if (f < nsum) {
                double v = 0.0;
                for (int64_t s = 0; s < R->nseg; ++s) v += p[s * stride + f];
                R->acc[q * R->nf + f] = v;
            } else {
                const unsigned long long *pc = reinterpret_cast<const unsigned long long *>(p);
                unsigned long long v = 0;
                for (int64_t s = 0; s < R->nseg; ++s) v += pc[s * stride + f];
                R->counts[q * kCounters + (f - nsum)] = v;
            }
        }
    }
}

// Bytes of the records and segment partials of one problem (16-byte multiples).
size_t record_bytes(int d, int K, int grad, int64_t Q, int64_t N) {
    return ((size_t)(Q * N) * rec_words(d, K, grad) * sizeof(float) + 255) & ~(size_t)255;
}
int64_t reduce_segments(int64_t N) { return (N + kReduceSegment - 1) / kReduceSegment; }
size_t partial_bytes(int d, int K, int cv, int64_t Q, int64_t N) {
    const int64_t nseg = reduce_segments(N);
    if (nseg <= 1) return 0;
    return ((size_t)(Q * nseg) * (reduce_sums(d, K, cv) + kCounters) * sizeof(double) + 255) & ~(size_t)255;
}

ReduceRec make_reduce_rec(int d, int K, int grad, int cv, int src, int anti, int64_t Q, int64_t N,
                          const float *rec, double *acc, unsigned long long *counts, double *part) {
    ReduceRec r{};
    r.anti = anti;
    r.d = d;
    r.K = K;
    r.grad = grad;
    r.cv = grad && cv;
    r.nf = acc_fields(d, K, r.cv, grad && src);
    r.rw = rec_words(d, K, grad);
    r.Q = Q;
    r.N = N;
    r.nseg = reduce_segments(N);
    r.rec = rec;
    r.acc = acc;
    r.counts = counts;
    r.part = part;
    return r;
}

wos_status launch_reduce(const ReduceArgs &a_in, int64_t total_queries, bool any_segmented, cudaStream_t s) {
    if (a_in.total_blocks <= 0) return WOS_OK;
    ReduceArgs a = a_in;
    const unsigned grid = (unsigned)std::min<int64_t>(a.total_blocks, 1 << 20);
    reduce_kernel<<<grid, kReduceThreads, 0, s>>>(a);
    WOS_CUDA(cudaGetLastError());
    if (any_segmented) {
        a.total_blocks = total_queries;
        reduce_combine_kernel<<<(unsigned)std::min<int64_t>(total_queries, 1 << 20), 96, 0, s>>>(a);
        WOS_CUDA(cudaGetLastError());
    }
    return WOS_OK;
}

wos_status launch_finalize(const FinalizeArgs &a, cudaStream_t s) {
    if (a.total_q <= 0) return WOS_OK;
    const int threads = 128;
    const int64_t blocks = std::min<int64_t>((a.total_q + threads - 1) / threads, 4096);
    finalize_kernel<<<(unsigned)blocks, threads, 0, s>>>(a);
    WOS_CUDA(cudaGetLastError());
    return WOS_OK;
}

// =====================================================================================
// walker launches
// =====================================================================================
struct Opts {
    int precision, laplace;
    int cv;  // gradient control variate (gradient calls only)
    int cuda_core_balls;  // keep tensor-core ball sets on the CUDA-core screen
    int antithetic;       // walk pairs with opposite first directions
    uint64_t seed;
    int64_t walk_offset, max_steps;
    double roulette_w;    // > 0: Russian roulette on weights below it
    long long wait_cycles;  // tensor-core walker: main-loop wait budget (clock cycles)
};

Opts read_opts(const wos_options *o) {
    Opts r{WOS_MIXED, 0, 0, 0, 0, 0ull, 0, 10000, 0.0, kDefaultWaitBudget};
    if (o != nullptr) {
        r.precision = o->precision;
        r.laplace = (o->flags & WOS_FLAG_LAPLACE_FACTOR) ? 1 : 0;
        r.cv = (o->flags & WOS_FLAG_GRAD_CONTROL_VARIATE) ? 1 : 0;
        r.cuda_core_balls = (o->flags & WOS_FLAG_CUDA_CORE_BALLS) ? 1 : 0;
        r.antithetic = (o->flags & WOS_FLAG_ANTITHETIC) ? 1 : 0;
        r.seed = o->seed;
        r.walk_offset = o->walk_offset;
        r.max_steps = o->max_steps > 0 ? o->max_steps : 10000;
        r.roulette_w = o->roulette_w;
        r.wait_cycles = o->wait_cycles > 0 ? (long long)o->wait_cycles : kDefaultWaitBudget;
    }
    return r;
}

// Options that need checks against the call: the roulette threshold, and the antithetic pair
// layout (N and the walk offset even, not with the control variate).
wos_status check_opts(const Opts &o, int64_t N) {
    if (!(o.roulette_w >= 0.0) || !std::isfinite(o.roulette_w))
        return fail(WOS_ERR_INVALID_ARG, "roulette_w must be finite and >= 0");
    if (o.antithetic) {
        if (N % 2 != 0 || o.walk_offset % 2 != 0)
            return fail(WOS_ERR_INVALID_ARG, "antithetic pairs need n_walks and walk_offset even");
        if (o.cv) return fail(WOS_ERR_INVALID_ARG, "antithetic pairs are not combined with the control variate");
    }
    return WOS_OK;
}

struct PerWalk {
    double *term = nullptr;
    int64_t *jumps = nullptr;
    double *grad = nullptr;
    double *dsigma = nullptr;
};

struct Scratch {
    void *acc = nullptr;                    // Q x nf (double, or float for the plain walker)
    unsigned long long *counts = nullptr;   // Q x kCounters
    unsigned long long *cursor = nullptr;   // work-queue cursor (mixed walker)
    float *rec = nullptr;                   // mixed walkers: Q N per-walk records
    double *part = nullptr;                 // mixed walkers: segment partial sums (N > kReduceSegment)
};

size_t scratch_bytes(int precision, int64_t Q, int nf) {
    const size_t es = precision == WOS_FP32_PLAIN ? sizeof(float) : sizeof(double);
    size_t acc = ((size_t)Q * nf * es + 255) & ~(size_t)255;
    size_t cnt = ((size_t)Q * kCounters * 8 + 255) & ~(size_t)255;
    return acc + cnt + 256;
}

Scratch carve_scratch(void *base, int precision, int64_t Q, int nf) {
    const size_t es = precision == WOS_FP32_PLAIN ? sizeof(float) : sizeof(double);
    size_t acc = ((size_t)Q * nf * es + 255) & ~(size_t)255;
    size_t cnt = ((size_t)Q * kCounters * 8 + 255) & ~(size_t)255;
    Scratch s;
    s.acc = base;
    s.counts = reinterpret_cast<unsigned long long *>((char *)base + acc);
    s.cursor = reinterpret_cast<unsigned long long *>((char *)base + acc + cnt);
    return s;
}

// Records and segment partials of a mixed-precision call, after the scratch of scratch_bytes.
size_t mixed_extra_bytes(const wos_domain_s &D, int64_t Q, int64_t N, int grad_mode, int cv) {
    return record_bytes(D.d, D.n_exp, grad_mode, Q, N) + partial_bytes(D.d, D.n_exp, grad_mode && cv, Q, N);
}
void carve_mixed(Scratch &sc, void *extra, const wos_domain_s &D, int64_t Q, int64_t N, int grad_mode) {
    sc.rec = reinterpret_cast<float *>(extra);
    sc.part = reinterpret_cast<double *>((char *)extra + record_bytes(D.d, D.n_exp, grad_mode, Q, N));
}

size_t g_mixed_smem_configured = 0;
std::mutex g_mixed_mu;

wos_status ensure_mixed_smem(size_t bytes) {
    std::lock_guard<std::mutex> lk(g_mixed_mu);
    if (bytes > g_mixed_smem_configured) {
        WOS_CUDA(configure_walk_mixed(bytes));
        g_mixed_smem_configured = bytes;
    }
    return WOS_OK;
}

MixedProblem make_mixed_problem(wos_domain_t dom, const double *x, int64_t Q, int64_t N,
                                double eps, double sigma, int grad_mode, int laplace, int cv,
                                int64_t walk_base, const WeightTable &tab, double *acc,
                                unsigned long long *counts, const PerWalk &pw, float *rec) {
    MixedProblem P{};
    P.rec = rec;
    P.rec_words = rec_words(dom->d, dom->n_exp, grad_mode);
    P.d = dom->d;
    P.n_balls = dom->n_balls;
    P.n_exp = dom->n_exp;
    P.has_box = dom->has_box;
    P.has_outer = dom->has_outer;
    P.has_goal = dom->has_goal;
    P.grad_mode = grad_mode;
    P.has_source = dom->has_source;
    P.proj = dom->proj;
    P.n_links = dom->n_links;
    P.n_arm_obs = (int)std::min<int64_t>(dom->n_arm_obs, kMaxArmObs);
    P.arm_inv_K = dom->n_links > 0 ? (float)(1.0 / dom->arm_K) : 0.f;
    P.src = grad_mode && dom->has_source;
    if (dom->has_source) {
        const int d = dom->d;
        const double nu = 0.5 * d - 1.0, k = std::sqrt(sigma);
        P.source_q = (float)dom->source_q;
        for (int j = 0; j < d; ++j) P.source_z[j] = (float)dom->source_z[j];
        P.src_inv_omega = (float)(std::tgamma(0.5 * d) / (2.0 * std::pow(M_PI, 0.5 * d)));
        P.src_lc0 = k > 0.0 ? (float)(nu * std::log(k) - 0.5 * d * std::log(2.0 * M_PI)) : 0.0f;
    }
    P.laplace = laplace;
    P.cv = grad_mode && cv;
    P.antithetic = 0;
    P.roulette_w = 0.f;
    P.log_roulette_w = 0.f;
    P.eps = (float)eps;
    P.sqrt_sigma = (float)std::sqrt(sigma);
    P.shrink = (float)dom->shrink32;
    P.slack = (float)dom->slack32;
    P.goal_r = (float)dom->goal_r;
    P.outer_r = (float)dom->outer_r;
    P.Q = Q;
    P.N = N;
    P.walk_base = walk_base;
    P.balls = dom->balls_mixed;
    P.geom = dom->geom_mixed;
    P.x = x;
    P.table = tab;
    P.acc = acc;
    P.counts = counts;
    P.w_term = pw.term;
    P.w_jumps = pw.jumps;
    P.w_grad = pw.grad;
    P.w_dsigma = pw.dsigma;
    return P;
}

// The walk options every mixed-precision problem record carries: antithetic pairs, roulette.
void apply_walk_opts(MixedProblem &P, const Opts &o) {
    P.antithetic = o.antithetic;
    P.roulette_w = (float)o.roulette_w;
    P.log_roulette_w = o.roulette_w > 0.0 ? (float)std::log(o.roulette_w) : 0.f;
}

size_t mixed_smem_bytes(const wos_domain_s &D) {
    return (size_t)((D.n_balls + 7) / 8) * (D.d + 2) * 32;
}

// The per-query reduction of a single mixed-precision call (records in sc.rec).
wos_status launch_reduce_single(wos_domain_t dom, const Opts &o, int64_t Q, int64_t N, int grad_mode,
                                const Scratch &sc, const int *skip, cudaStream_t s) {
    ReduceArgs ra{};
    ra.single = make_reduce_rec(dom->d, dom->n_exp, grad_mode, o.cv, dom->has_source, o.antithetic, Q, N, sc.rec,
                                (double *)sc.acc, sc.counts, sc.part);
    ra.n = 1;
    ra.total_blocks = Q * ra.single.nseg;
    ra.skip = skip;
    return launch_reduce(ra, Q, ra.single.nseg > 1, s);
}

// Launches the walk kernel of the chosen precision for Q x N walks on zeroed scratch (mixed
// precision: then the per-query reduction of its records).
wos_status launch_walkers(wos_domain_t dom, const Opts &o, const double *x, int64_t Q, int64_t N,
                          double eps, double sigma, int grad_mode, const Scratch &sc,
                          const PerWalk &pw, const int *skip, cudaStream_t s) {
    const int cv = grad_mode && o.cv;
    const int src = grad_mode && dom->has_source;
    const int nf = acc_fields(dom->d, dom->n_exp, cv, src);
    if (o.precision == WOS_FP64) {
        SimpleParams<double> p{};
        p.dom = dom->v64;
        p.x = x;
        p.Q = Q;
        p.N = N;
        p.seed = o.seed;
        p.walk_offset = o.walk_offset;
        p.max_steps = o.max_steps;
        p.eps = eps;
        p.sqrt_sigma = std::sqrt(sigma);
        p.shrink = 0.0;
        p.grad_mode = grad_mode;
        p.laplace = o.laplace;
        p.cv = cv;
        p.src = src;
        p.antithetic = o.antithetic;
        p.roulette_w = o.roulette_w;
        p.acc = (double *)sc.acc;
        p.counts = sc.counts;
        p.nf = nf;
        p.w_term = pw.term;
        p.w_jumps = pw.jumps;
        p.w_grad = pw.grad;
        p.w_dsigma = pw.dsigma;
        p.skip = skip;
        WOS_CUDA(launch_walk_simple_f64(p, s));
        return WOS_OK;
    }
    if (o.precision == WOS_FP32_PLAIN) {
        SimpleParams<float> p{};
        p.dom = dom->v32;
        p.x = x;
        p.Q = Q;
        p.N = N;
        p.seed = o.seed;
        p.walk_offset = o.walk_offset;
        p.max_steps = o.max_steps;
        p.eps = (float)eps;
        p.sqrt_sigma = (float)std::sqrt(sigma);
        p.shrink = (float)dom->shrink32;
        p.grad_mode = grad_mode;
        p.laplace = o.laplace;
        p.cv = cv;
        p.src = src;
        p.antithetic = o.antithetic;
        p.roulette_w = o.roulette_w;
        p.acc = (float *)sc.acc;
        p.counts = sc.counts;
        p.nf = nf;
        p.w_term = pw.term;
        p.w_jumps = pw.jumps;
        p.w_grad = pw.grad;
        p.w_dsigma = pw.dsigma;
        p.skip = skip;
        WOS_CUDA(launch_walk_simple_f32(p, s));
        return WOS_OK;
    }
    if (o.precision != WOS_MIXED) return fail(WOS_ERR_INVALID_ARG, "unknown precision %d", o.precision);
    if (o.max_steps > (int64_t)kRecKMask)
        return fail(WOS_ERR_INVALID_ARG, "max_steps must be below 2^28 in mixed precision");
    if (dom->n_links > 0 && (dom->n_points > 0 || dom->n_arm_obs > kMaxArmObs || dom->d > kMaxArmLinksMixed))
        return fail(WOS_ERR_UNSUPPORTED,
                    "mixed precision runs an arm in d <= %d with at most %d obstacle points, and no point set",
                    kMaxArmLinksMixed, kMaxArmObs);
    WeightTable tab;
    WOS_TRY(ensure_table(dom, sigma, &tab, s, false));
    if (dom->n_points > 0 || (dom->has_pcd && !o.cuda_core_balls)) {
        if (!dom->has_pcd)
            return fail(WOS_ERR_UNSUPPORTED, "mixed-precision point clouds need d <= %d", kPointCloudMaxD);
        if (dom->n_balls > 0 && dom->n_points > 0)
            return fail(WOS_ERR_UNSUPPORTED, "a domain with both balls and points runs in FP64 or plain FP32");
        MixedProblem P = make_mixed_problem(dom, x, Q, N, eps, sigma, grad_mode, o.laplace, cv, o.walk_offset, tab,
                                            (double *)sc.acc, sc.counts, pw, sc.rec);
        apply_walk_opts(P, o);
        unsigned long long *shrinks = sc.cursor + 1;
        int *status = reinterpret_cast<int *>(sc.cursor + 2);
        P.done = skip;  // a planner step after the goal runs no walks
        WOS_CUDA(launch_pointcloud(dom->pcd, P, dom->pc_delta, sc.cursor, status, shrinks, o.seed, o.max_steps,
                                   o.wait_cycles, grad_mode, s));
        return launch_reduce_single(dom, o, Q, N, grad_mode, sc, skip, s);
    }
    const int64_t total = Q * N;
    if (total > (int64_t)0x7fffffff) return fail(WOS_ERR_UNSUPPORTED, "Q * n_walks must be < 2^31");
    const size_t smem = mixed_smem_bytes(*dom);
    WOS_TRY(ensure_mixed_smem(smem));
    // Launch shape. Few walks (a planner step): one walk per lane, as many lanes as walks, for
    // latency. Many walks: at least 8 walks per lane per item, so that the spread of walk
    // lengths averages out before an item ends, and at least as many items as CTAs.
    const int sms = device_sms();
    int threads;
    int64_t wpi;
    int grid;
    if (total <= (int64_t)sms * 512) {
        threads = (int)std::min<int64_t>(512, std::max<int64_t>(32, (total / sms + 31) / 32 * 32));
        if (max_active_mixed(threads, smem, grad_mode) < 1)
            return fail(WOS_ERR_UNSUPPORTED, "mixed walker does not fit (%zu B smem)", smem);
        wpi = threads;
        grid = (int)((total + wpi - 1) / wpi);
    } else {
        threads = (int)std::min<int64_t>(512, std::max<int64_t>(32, (total / (8LL * sms) + 31) / 32 * 32));
        const int occ = max_active_mixed(threads, smem, grad_mode);
        if (occ < 1) return fail(WOS_ERR_UNSUPPORTED, "mixed walker does not fit (%zu B smem)", smem);
        const int64_t grid_full = (int64_t)sms * occ;
        wpi = std::max<int64_t>(8LL * threads, (total + 4 * grid_full - 1) / (4 * grid_full));
        wpi = std::min<int64_t>(wpi, 1 << 22);
        wpi = (wpi + 31) / 32 * 32;
        grid = (int)std::min<int64_t>(grid_full, (total + wpi - 1) / wpi);
    }
    const int64_t n_items = (total + wpi - 1) / wpi;
    MixedLaunch L{};
    L.problems = nullptr;
    L.items = nullptr;
    L.n_items = n_items;
    L.walks_per_item = wpi;
    L.total_walks = total;
    L.cursor = sc.cursor;
    L.seed = o.seed;
    L.max_steps = o.max_steps;
    L.skip = skip;
    L.single = make_mixed_problem(dom, x, Q, N, eps, sigma, grad_mode, o.laplace, cv, o.walk_offset,
                                  tab, (double *)sc.acc, sc.counts, pw, sc.rec);
    apply_walk_opts(L.single, o);
    WOS_CUDA(launch_walk_mixed(L, grad_mode, grid, threads, smem, s));
    return launch_reduce_single(dom, o, Q, N, grad_mode, sc, skip, s);
}

wos_status check_common(wos_domain_t dom, const double *x, int64_t Q, int64_t N, double eps,
                        double sigma) {
    if (dom == nullptr) return fail(WOS_ERR_INVALID_ARG, "domain is NULL");
    if (Q < 0 || N < 1) return fail(WOS_ERR_INVALID_ARG, "Q must be >= 0 and n_walks >= 1");
    if (Q > 0 && x == nullptr) return fail(WOS_ERR_INVALID_ARG, "x is NULL");
    if (!(eps > 0.0) || !(sigma >= 0.0) || !std::isfinite(sigma))
        return fail(WOS_ERR_INVALID_ARG, "eps must be > 0 and sigma >= 0");
    if (Q > ((int64_t)1 << 40) / N) return fail(WOS_ERR_INVALID_ARG, "Q * n_walks too large");
    return WOS_OK;
}

struct Outputs {
    double *u = nullptr, *u_se = nullptr, *grad = nullptr, *grad_se = nullptr;
    double *du_dsigma = nullptr, *du_dw = nullptr;
};

wos_status run_estimator(wos_domain_t dom, const wos_options *opt, const double *x, int64_t Q,
                         int64_t N, double eps, double sigma, int grad_mode, const Outputs &out,
                         const PerWalk &pw, wos_stats *stats, cudaStream_t s) {
    WOS_TRY(check_common(dom, x, Q, N, eps, sigma));
    const Opts o = read_opts(opt);
    if (o.precision < WOS_FP64 || o.precision > WOS_MIXED)
        return fail(WOS_ERR_INVALID_ARG, "unknown precision %d", o.precision);
    {
        Opts oc = o;
        if (!grad_mode) oc.cv = 0;  // value calls ignore the control variate
        WOS_TRY(check_opts(oc, N));
    }
    if (stats != nullptr) WOS_CUDA(cudaMemsetAsync(stats, 0, sizeof(wos_stats), s));
    if (Q == 0) return WOS_OK;
    const int cv = grad_mode && o.cv;
    const int src = grad_mode && dom->has_source;
    const int nf = acc_fields(dom->d, dom->n_exp, cv, src);
    const size_t bytes = scratch_bytes(o.precision, Q, nf);
    const size_t extra = o.precision == WOS_MIXED ? mixed_extra_bytes(*dom, Q, N, grad_mode, o.cv) : 0;
    void *base = nullptr;
    WOS_CUDA(cudaMallocAsync(&base, bytes + extra, s));
    Scratch sc = carve_scratch(base, o.precision, Q, nf);
    if (o.precision == WOS_MIXED) carve_mixed(sc, (char *)base + bytes, *dom, Q, N, grad_mode);
    wos_status st = WOS_OK;
    if (cudaMemsetAsync(base, 0, bytes, s) != cudaSuccess)  // records and partials are written in full
        st = fail(WOS_ERR_CUDA, "scratch memset failed");
    if (st == WOS_OK) st = launch_walkers(dom, o, x, Q, N, eps, sigma, grad_mode, sc, pw, nullptr, s);
    if (st == WOS_OK) {
        FinalizeArgs a{};
        a.recs = nullptr;
        a.n = 1;
        a.total_q = Q;
        a.stats = stats;
        a.status = reinterpret_cast<const int *>(sc.cursor + 2);
        a.shrinks = sc.cursor + 1;
        FinalizeRec &r = a.single;
        r.d = dom->d;
        r.K = dom->n_exp;
        r.acc_f32 = o.precision == WOS_FP32_PLAIN;
        r.anti = o.antithetic;
        r.cv = cv;
        r.src = src;
        r.Q = Q;
        r.N = N;
        r.q_begin = 0;
        r.acc = sc.acc;
        r.counts = sc.counts;
        r.u = out.u;
        r.u_se = out.u_se;
        r.grad = out.grad;
        r.grad_se = out.grad_se;
        r.du_dsigma = out.du_dsigma;
        r.du_dw = out.du_dw;
        r.walk_steps = nullptr;
        st = launch_finalize(a, s);
    }
    cudaFreeAsync(base, s);
    return st;
}

}  // namespace

// =====================================================================================
// C ABI: domain
// =====================================================================================
extern "C" {

const char *wos_status_string(wos_status s) {
    switch (s) {
        case WOS_OK: return "ok";
        case WOS_ERR_INVALID_ARG: return "invalid argument";
        case WOS_ERR_UNSUPPORTED: return "unsupported";
        case WOS_ERR_OOM: return "out of memory";
        case WOS_ERR_CUDA: return "CUDA error";
        case WOS_ERR_TIMEOUT: return "device iteration budget exhausted";
        case WOS_ERR_OUTSIDE_DOMAIN: return "query outside the domain";
    }
    return "unknown status";
}

const char *wos_last_error(void) { return g_err.c_str(); }

wos_status wos_domain_create(const wos_domain_desc *desc, wos_domain_t *out) {
    if (out == nullptr) return fail(WOS_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (desc == nullptr) return fail(WOS_ERR_INVALID_ARG, "desc is NULL");
    const int d = desc->d;
    if (d < 2 || d > WOS_MAX_D) return fail(WOS_ERR_UNSUPPORTED, "d = %d outside 2..%d", d, WOS_MAX_D);
    if (desc->n_balls < 0 || desc->n_points < 0 || desc->n_exp < 0)
        return fail(WOS_ERR_INVALID_ARG, "negative count");
    if (!(desc->sigma_max >= 0) || desc->sigma_max > 1e12)
        return fail(WOS_ERR_INVALID_ARG, "sigma_max must be in [0, 1e12]");
    if (desc->proj_dims < 0 || desc->proj_dims > d)
        return fail(WOS_ERR_INVALID_ARG, "proj_dims = %d outside 0..%d", desc->proj_dims, d);
    const int proj = desc->proj_dims > 0 ? desc->proj_dims : d;
    if (proj < d && desc->n_points > 0) return fail(WOS_ERR_UNSUPPORTED, "extruded point sets");
    if (desc->n_exp > WOS_MAX_EXP) return fail(WOS_ERR_UNSUPPORTED, "n_exp > %d", WOS_MAX_EXP);
    if ((desc->box_lo == nullptr) != (desc->box_hi == nullptr))
        return fail(WOS_ERR_INVALID_ARG, "box_lo and box_hi must both be given");
    if (desc->box_lo == nullptr && desc->outer_c == nullptr)
        return fail(WOS_ERR_INVALID_ARG, "a box or an outer ball is required");
    if (desc->n_balls > 0 && (desc->ball_c == nullptr || desc->ball_r == nullptr))
        return fail(WOS_ERR_INVALID_ARG, "ball arrays missing");
    if (desc->n_points > 0 && desc->points == nullptr) return fail(WOS_ERR_INVALID_ARG, "points missing");
    if (desc->n_exp > 0 && (desc->exp_w == nullptr || desc->exp_a == nullptr))
        return fail(WOS_ERR_INVALID_ARG, "exp arrays missing");
    if (desc->outer_c != nullptr && !(desc->outer_r > 0)) return fail(WOS_ERR_INVALID_ARG, "outer_r <= 0");
    if (desc->goal_c != nullptr && !(desc->goal_r > 0)) return fail(WOS_ERR_INVALID_ARG, "goal_r <= 0");
    for (int i = 0; i < desc->n_balls; ++i)
        if (!(desc->ball_r[i] > 0) || !std::isfinite(desc->ball_r[i]))
            return fail(WOS_ERR_INVALID_ARG, "ball %d radius <= 0", i);
    if (desc->box_lo != nullptr)
        for (int j = 0; j < proj; ++j)
            if (!(desc->box_hi[j] > desc->box_lo[j])) return fail(WOS_ERR_INVALID_ARG, "empty box");
    if (desc->n_links < 0 || desc->n_links > d)
        return fail(WOS_ERR_INVALID_ARG, "n_links = %d outside 0..d", desc->n_links);
    if (desc->n_links > 0) {
        if (desc->link_l == nullptr || desc->arm_obs == nullptr || desc->n_arm_obs < 1)
            return fail(WOS_ERR_INVALID_ARG, "an arm needs link lengths and at least one obstacle point");
        for (int i = 0; i < desc->n_links; ++i)
            if (!(desc->link_l[i] > 0) || !std::isfinite(desc->link_l[i]))
                return fail(WOS_ERR_INVALID_ARG, "link %d length <= 0", i);
        if (proj < d) return fail(WOS_ERR_UNSUPPORTED, "an arm in an extruded domain");
    }

    wos_domain_s *D = new (std::nothrow) wos_domain_s();
    if (D == nullptr) return fail(WOS_ERR_OOM, "host allocation failed");
    D->d = d;
    D->has_box = desc->box_lo != nullptr;
    D->has_outer = desc->outer_c != nullptr;
    D->has_goal = desc->goal_c != nullptr;
    D->n_balls = desc->n_balls;
    D->n_points = desc->n_points;
    D->n_exp = desc->n_exp;
    D->outer_r = D->has_outer ? desc->outer_r : 0.0;
    D->goal_r = D->has_goal ? desc->goal_r : 0.0;
    D->has_source = desc->source_z != nullptr;
    D->source_q = D->has_source ? desc->source_q : 0.0;
    D->proj = proj;
    auto copy = [](std::vector<double> &v, const double *p, size_t n) {
        v.assign(n, 0.0);
        if (p) std::copy(p, p + n, v.begin());
    };
    copy(D->box_lo, desc->box_lo, d);
    copy(D->box_hi, desc->box_hi, d);
    copy(D->outer_c, desc->outer_c, d);
    copy(D->goal_c, desc->goal_c, d);
    copy(D->exp_w, desc->exp_w, desc->n_exp);
    copy(D->exp_a, desc->exp_a, (size_t)desc->n_exp * d);
    copy(D->ball_r, desc->ball_r, desc->n_balls);
    copy(D->ball_c, desc->ball_c, (size_t)desc->n_balls * d);
    copy(D->points, desc->points, (size_t)desc->n_points * d);
    copy(D->source_z, desc->source_z, d);
    D->n_links = desc->n_links;
    D->n_arm_obs = desc->n_links > 0 ? desc->n_arm_obs : 0;
    copy(D->link_l, desc->link_l, D->n_links);
    copy(D->arm_obs, desc->arm_obs, (size_t)(2 * D->n_arm_obs));
    if (D->n_links > 0) {
        double reach = 0.0, k2 = 0.0;  // K = sqrt(sum_n (sum_{i<=n} l_i)^2), Sec. V-A
        for (int i = 0; i < D->n_links; ++i) {
            reach += D->link_l[i];
            k2 += reach * reach;
        }
        D->arm_K = std::sqrt(k2);
    }
    // an extruded domain's box has no faces in the free coordinates: far away, never nearest
    for (int j = proj; j < d; ++j) {
        D->box_lo[j] = -1.0e30;
        D->box_hi[j] = 1.0e30;
    }
    double rmax = INFINITY;
    if (D->has_box)
        for (int j = 0; j < proj; ++j) rmax = std::min(rmax, 0.5 * (D->box_hi[j] - D->box_lo[j]));
    if (D->has_outer) rmax = std::min(rmax, D->outer_r);
    D->R_max = rmax;
    error_bounds(*D);

    // device copies
    const int64_t nv = view_size(*D);
    std::vector<double> h64 = pack_view<double>(*D);
    std::vector<float> h32 = pack_view<float>(*D);
    // 8-ball blocks [m_0 x8]...[m_{d-1} x8][e0 x8][e1 x8], m = -2c, e0 = |c|^2 - r^2, e1 = -2r;
    // an extruded domain has m_j = 0 in the free coordinates and |c|^2 over the first proj
    const int kB = 8;
    const int nblk = (D->n_balls + kB - 1) / kB;
    D->nblk = nblk;
    std::vector<float> hb((size_t)std::max(1, nblk) * (d + 2) * kB, 0.0f);
    for (int i = 0; i < nblk * kB; ++i) {
        const int blk = i / kB, t = i % kB;
        float *B = hb.data() + (size_t)blk * (d + 2) * kB;
        if (i < D->n_balls) {
            double cc = 0.0;
            for (int j = 0; j < d; ++j) {
                const float c = j < proj ? (float)D->ball_c[(size_t)i * d + j] : 0.0f;
                B[kB * j + t] = -2.0f * c;
                cc += (double)c * (double)c;
            }
            const float r = (float)D->ball_r[i];
            B[kB * d + t] = (float)(cc - (double)r * (double)r);
            B[kB * (d + 1) + t] = -2.0f * r;
        } else {
            // padding ball: far away (never passes the screen), radius 0
            for (int j = 0; j < d; ++j) B[kB * j + t] = 0.0f;
            B[kB * d + t] = 3.0e38f;
            B[kB * (d + 1) + t] = 0.0f;
        }
    }
    std::vector<float> hg((size_t)geom_floats(d), 0.0f);
    for (int j = 0; j < d; ++j) {
        hg[j] = (float)D->box_lo[j];
        hg[d + j] = (float)D->box_hi[j];
        hg[2 * d + j] = (float)D->goal_c[j];
        hg[3 * d + j] = (float)D->outer_c[j];
    }
    for (int k = 0; k < D->n_exp; ++k) {
        hg[4 * d + k] = (float)D->exp_w[k];
        for (int j = 0; j < d; ++j) hg[4 * d + kMaxExp + k * d + j] = (float)D->exp_a[(size_t)k * d + j];
    }
    for (int i = 0; i < D->n_links; ++i) hg[geom_link(d) + i] = (float)D->link_l[i];
    for (int64_t o = 0; o < std::min<int64_t>(D->n_arm_obs, kMaxArmObs); ++o) {
        hg[geom_arm_obs(d) + 2 * o] = (float)D->arm_obs[2 * o];
        hg[geom_arm_obs(d) + 2 * o + 1] = (float)D->arm_obs[2 * o + 1];
    }
    cudaError_t e = cudaMalloc(&D->f64, sizeof(double) * (size_t)nv);
    if (e == cudaSuccess) e = cudaMalloc(&D->f32, sizeof(float) * (size_t)nv);
    if (e == cudaSuccess) e = cudaMalloc(&D->balls_mixed, sizeof(float) * hb.size());
    if (e == cudaSuccess) e = cudaMalloc(&D->geom_mixed, sizeof(float) * hg.size());
    if (e == cudaSuccess) e = cudaMemcpy(D->f64, h64.data(), sizeof(double) * nv, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(D->f32, h32.data(), sizeof(float) * nv, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(D->balls_mixed, hb.data(), sizeof(float) * hb.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(D->geom_mixed, hg.data(), sizeof(float) * hg.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        const wos_status st = fail(e == cudaErrorMemoryAllocation ? WOS_ERR_OOM : WOS_ERR_CUDA,
                                   "domain upload failed: %s", cudaGetErrorString(e));
        wos_domain_destroy(D);
        return st;
    }
    layout_view<double>(D->v64, D->f64, *D);
    layout_view<float>(D->v32, D->f32, *D);
    // large ball sets run on the tensor-core sphere-set walker (not extruded domains or arms)
    const bool sphere_balls = D->n_points == 0 && D->n_balls >= sphere_min_balls(d) && d <= kPointCloudMaxD &&
                              D->proj == d && D->n_links == 0;
    if ((D->n_points > 0 && d <= kPointCloudMaxD) || sphere_balls) {
        e = sphere_balls ? pointcloud_prepare(D->ball_c.data(), D->ball_r.data(), D->n_balls, d, &D->pcd)
                         : pointcloud_prepare(D->points.data(), nullptr, D->n_points, d, &D->pcd);
        if (e != cudaSuccess) {
            const wos_status st = fail(e == cudaErrorMemoryAllocation ? WOS_ERR_OOM : WOS_ERR_CUDA,
                                       "point-cloud operand setup failed: %s", cudaGetErrorString(e));
            wos_domain_destroy(D);
            return st;
        }
        D->has_pcd = true;
        double xabs = 0.0;
        for (int j = 0; j < d; ++j)
            xabs = std::max({xabs, std::fabs(D->box_lo[j]), std::fabs(D->box_hi[j]),
                             std::fabs(D->outer_c[j]) + D->outer_r});
        D->pc_delta = pointcloud_delta(d, xabs, D->pcd.pmax);
    }
    // weight tables for every sigma up to sigma_max, so that no later call builds one
    if (desc->sigma_max > 0) {
        WeightTable t;
        const wos_status st = ensure_table_level(D, table_level(*D, desc->sigma_max), &t, nullptr, true);
        if (st != WOS_OK) {
            wos_domain_destroy(D);
            return st;
        }
    }
    *out = D;
    return WOS_OK;
}

wos_status wos_domain_destroy(wos_domain_t dom) {
    if (dom == nullptr) return WOS_OK;
    cudaDeviceSynchronize();
    cudaFree(dom->f64);
    cudaFree(dom->f32);
    cudaFree(dom->balls_mixed);
    cudaFree(dom->geom_mixed);
    for (TableEntry &t : dom->tables) {
        if (t.built) cudaEventDestroy(t.built);
        cudaFree(t.nodes);
    }
    if (dom->has_pcd) pointcloud_release(&dom->pcd);
    delete dom;
    return WOS_OK;
}

wos_status wos_domain_info(wos_domain_t dom, int32_t *tensor_sphere_set, int32_t *sphere_tiles) {
    if (dom == nullptr) return fail(WOS_ERR_INVALID_ARG, "domain is NULL");
    if (tensor_sphere_set != nullptr) *tensor_sphere_set = dom->has_pcd ? 1 : 0;
    if (sphere_tiles != nullptr) *sphere_tiles = dom->has_pcd ? dom->pcd.n_tiles : 0;
    return WOS_OK;
}

wos_status wos_domain_set_exp_w(wos_domain_t dom, const double *w_device, int32_t n, void *stream) {
    if (dom == nullptr || w_device == nullptr) return fail(WOS_ERR_INVALID_ARG, "NULL argument");
    if (n != dom->n_exp) return fail(WOS_ERR_INVALID_ARG, "n = %d but the domain has %d terms", n, dom->n_exp);
    if (n == 0) return WOS_OK;
    set_exp_w_kernel<<<1, 32, 0, (cudaStream_t)stream>>>(
        w_device, n, const_cast<double *>(dom->v64.exp_w), const_cast<float *>(dom->v32.exp_w),
        dom->geom_mixed + 4 * dom->d);
    WOS_CUDA(cudaGetLastError());
    return WOS_OK;
}

// =====================================================================================
// C ABI: estimators
// =====================================================================================
wos_status wos_solve(wos_domain_t dom, const wos_options *opt, const double *x, int64_t Q,
                     int64_t n_walks, double eps, double sigma, double *u, double *u_se,
                     wos_stats *stats, void *stream) {
    if (Q > 0 && u == nullptr) return fail(WOS_ERR_INVALID_ARG, "u is NULL");
    Outputs o;
    o.u = u;
    o.u_se = u_se;
    return run_estimator(dom, opt, x, Q, n_walks, eps, sigma, 0, o, PerWalk{}, stats,
                         (cudaStream_t)stream);
}

wos_status wos_grad(wos_domain_t dom, const wos_options *opt, const double *x, int64_t Q,
                    int64_t n_walks, double eps, double sigma, double *u, double *u_se,
                    double *grad, double *grad_se, double *du_dsigma, double *du_dw,
                    wos_stats *stats, void *stream) {
    if (Q > 0 && grad == nullptr) return fail(WOS_ERR_INVALID_ARG, "grad is NULL");
    Outputs o;
    o.u = u;
    o.u_se = u_se;
    o.grad = grad;
    o.grad_se = grad_se;
    o.du_dsigma = du_dsigma;
    o.du_dw = du_dw;
    return run_estimator(dom, opt, x, Q, n_walks, eps, sigma, 1, o, PerWalk{}, stats,
                         (cudaStream_t)stream);
}

wos_status wos_walks(wos_domain_t dom, const wos_options *opt, const double *x, int64_t Q,
                     int64_t n_walks, double eps, double sigma, int32_t grad_mode, double *term,
                     int64_t *jumps, double *grad, double *dsigma, void *stream) {
    PerWalk pw;
    pw.term = term;
    pw.jumps = jumps;
    pw.grad = grad;
    pw.dsigma = dsigma;
    return run_estimator(dom, opt, x, Q, n_walks, eps, sigma, grad_mode ? 1 : 0, Outputs{}, pw,
                         nullptr, (cudaStream_t)stream);
}

}  // extern "C"

// =====================================================================================
// planner
// =====================================================================================
namespace {

struct PlanArgs {
    DomainView<double> dom;
    double *x;
    double eps, s_ub;
    int64_t N;
    int *done;
    int *skip;
    int32_t *flag;
    void *acc;
    int acc_bytes;
    int acc_f32;
    int cv;  // control-variate gradient (sums after the du/dw fields)
    int src;  // impulse-source fields after those
    unsigned long long *counts;
    unsigned long long *cursor;  // single walker launch: [item cursor, shrinks, status]; nullable
    double *grad_row;
    double *path_row;
    const int *status;  // nullable: the tensor-core walker's status word (nonzero: it gave up)
    int *timed_out;     // nullable: set when a step found the status word set
};

// The goal test of a planner step (one thread): a path that has reached its goal skips the step
// (flag 1 at the step that finds it, 8 after).
__device__ void plan_pre_decide(const PlanArgs &a) {
    {
        int skip = 0;
        int32_t f = 0;
        if (*a.done) {
            skip = 1;
            f = 8;
        } else if (a.dom.has_goal) {
            double s = 0.0;
            for (int j = 0; j < a.dom.proj; ++j) {
                const double t = a.x[j] - a.dom.goal_c[j];
                s += t * t;
            }
            if (sqrt(s) - a.dom.goal_r < a.eps) {
                skip = 1;
                f = 1;
                *a.done = 1;
            }
        } else if (a.dom.has_source) {
            // the goal is the impulse source: reached once it is within one nominal step
            double s = 0.0;
            for (int j = 0; j < a.dom.d; ++j) {
                const double t = a.x[j] - a.dom.source_z[j];
                s += t * t;
            }
            if (sqrt(s) < a.s_ub) {
                skip = 1;
                f = 1;
                *a.done = 1;
            }
        }
        *a.skip = skip;
        *a.flag = f;
    }
}

__global__ void plan_pre_kernel(const __grid_constant__ PlanArgs a) {
    if (threadIdx.x == 0) {
        plan_pre_decide(a);
        a.cursor[0] = a.cursor[1] = a.cursor[2] = 0ull;
    }
    __syncthreads();
    unsigned char *acc = (unsigned char *)a.acc;
    for (int i = threadIdx.x; i < a.acc_bytes; i += blockDim.x) acc[i] = 0;
    for (int i = threadIdx.x; i < kCounters; i += blockDim.x) a.counts[i] = 0ull;
}

template <int D>
__device__ void plan_post_d(const PlanArgs &a) {
    double x[D];
    for (int j = 0; j < D; ++j) x[j] = a.x[j];
    if (!*a.skip && a.status != nullptr && *a.status != 0) {  // the walker gave up: stop the path
        *a.flag = 16;
        *a.done = 1;
        if (a.timed_out != nullptr) *a.timed_out = 1;
    } else if (!*a.skip) {
        int kind;
        int64_t idx;
        const double R = distance<double, D>(a.dom, x, kind, idx);
        const bool outside = a.counts[3] > 0;
        if (outside || !(R > 0.0)) {
            *a.flag = 4;
            *a.done = 1;
        } else {
            const double inv = 1.0 / (double)a.N;
            auto S = [&](int f) -> double {
                return a.acc_f32 ? (double)((const float *)a.acc)[f] : ((const double *)a.acc)[f];
            };
            const int cf = cv_field(D, a.dom.n_exp);
            const int sf = src_field(D, a.dom.n_exp, a.cv);
            const double s0 = a.src ? S(sf) : 0.0;
            double g[D];
            double gg = 0.0;
            for (int j = 0; j < D; ++j) {
                g[j] = S(3 + j) * inv;
                if (a.cv && a.N >= 2) {
                    double se;
                    cv_estimate(S(3 + j), S(3 + D + j), S(cf + j), S(cf + D + j) - s0 * S(cf + 2 * D + j),
                                S(cf + 2 * D + j), S(cf + 3 * D), S(0) - (double)a.N * s0, (double)a.N, g[j], se);
                }
                if (a.src) g[j] += S(sf + 1 + j);
                gg += g[j] * g[j];
            }
            if (a.grad_row)
                for (int j = 0; j < D; ++j) a.grad_row[j] = g[j];
            if (gg > 0.0) {
                const double gn = sqrt(gg);
                const double s = 0.5 * R < a.s_ub ? 0.5 * R : a.s_ub;
                for (int j = 0; j < D; ++j) x[j] = x[j] + s * (g[j] / gn);
                for (int j = 0; j < D; ++j) a.x[j] = x[j];
            } else {
                *a.flag = 2;
            }
        }
    }
    if (a.path_row)
        for (int j = 0; j < D; ++j) a.path_row[j] = x[j];
}

__global__ void plan_post_kernel(const __grid_constant__ PlanArgs a) {
    if (threadIdx.x != 0) return;
    switch (a.dom.d) {
#define WOS_CASE(DD) \
    case DD: plan_post_d<DD>(a); break;
        WOS_CASE(2) WOS_CASE(3) WOS_CASE(4) WOS_CASE(5) WOS_CASE(6) WOS_CASE(7)
        WOS_CASE(8) WOS_CASE(9) WOS_CASE(10) WOS_CASE(11) WOS_CASE(12)
#undef WOS_CASE
        default: break;
    }
}

// ---- many planner paths in one batch: per-path records of the step kernels ----------------
struct PathRec {
    PlanArgs a;                 // flag/grad_row/path_row hold the bases of the path's outputs
    int32_t *flags;             // n_steps
    double *grads;              // n_steps x d or nullptr
    double *path;               // (n_steps + 1) x d
    int64_t walk_offset;        // global walk index of walk 0 at step 0
    int64_t *walk_base_mixed;   // the walk base of the path's record in the batch's problem table
    int64_t *walk_base_sphere;  // ... and in the tensor-core problem table (nullptr if none)
};

// Step `step` of every path, before its walks: the goal test, and the walk offset of the step
// (walk_offset + step N, the walks wos_plan_path draws) in the problem tables. One block per path.
__global__ void paths_pre_kernel(const PathRec *recs, int n, int64_t step) {
    for (int p = blockIdx.x; p < n; p += gridDim.x) {
        if (threadIdx.x != 0) continue;
        const PathRec &R = recs[p];
        PlanArgs a = R.a;
        a.flag = R.flags + step;
        plan_pre_decide(a);
        const int64_t wb = R.walk_offset + step * a.N;
        *R.walk_base_mixed = wb;
        if (R.walk_base_sphere != nullptr) *R.walk_base_sphere = wb;
    }
}

// Step `step` of every path, after the reduction of its walks: grad u and the move.
__global__ void paths_post_kernel(const PathRec *recs, int n, int64_t step) {
    for (int p = blockIdx.x; p < n; p += gridDim.x) {
        if (threadIdx.x != 0) continue;
        const PathRec &R = recs[p];
        PlanArgs a = R.a;
        const int d = a.dom.d;
        a.flag = R.flags + step;
        a.grad_row = R.grads != nullptr ? R.grads + step * d : nullptr;
        a.path_row = R.path + (step + 1) * d;
        switch (d) {
#define WOS_CASE(DD) \
    case DD: plan_post_d<DD>(a); break;
            WOS_CASE(2) WOS_CASE(3) WOS_CASE(4) WOS_CASE(5) WOS_CASE(6) WOS_CASE(7)
            WOS_CASE(8) WOS_CASE(9) WOS_CASE(10) WOS_CASE(11) WOS_CASE(12)
#undef WOS_CASE
            default: break;
        }
    }
}

// One planner step: [pre: goal test, zero scratch] [gradient walkers] [post: step].
wos_status enqueue_plan_step(wos_domain_t dom, const Opts &o, double *x, int64_t N, double eps,
                             double sigma, double s_ub, int64_t step_idx, int *done, int *skip,
                             int32_t *flag, const Scratch &sc, double *grad_row, double *path_row,
                             cudaStream_t s) {
    const int nf = acc_fields(dom->d, dom->n_exp, o.cv, dom->has_source);
    PlanArgs a{};
    a.dom = dom->v64;
    a.x = x;
    a.eps = eps;
    a.s_ub = s_ub;
    a.N = N;
    a.done = done;
    a.skip = skip;
    a.flag = flag;
    a.acc = sc.acc;
    a.acc_f32 = o.precision == WOS_FP32_PLAIN;
    a.cv = o.cv;
    a.src = dom->has_source;
    a.acc_bytes = nf * (a.acc_f32 ? 4 : 8);
    a.counts = sc.counts;
    a.cursor = sc.cursor;
    a.grad_row = grad_row;
    a.path_row = path_row;
    a.status = reinterpret_cast<const int *>(sc.cursor + 2);
    a.timed_out = done + 2;  // the planner's ints: [done, skip, timed out]
    plan_pre_kernel<<<1, 128, 0, s>>>(a);
    WOS_CUDA(cudaGetLastError());
    Opts os = o;
    os.walk_offset = o.walk_offset + step_idx * N;
    WOS_TRY(launch_walkers(dom, os, x, 1, N, eps, sigma, 1, sc, PerWalk{}, skip, s));
    plan_post_kernel<<<1, 32, 0, s>>>(a);
    WOS_CUDA(cudaGetLastError());
    return WOS_OK;
}

}  // namespace

extern "C" {

wos_status wos_plan_step(wos_domain_t dom, const wos_options *opt, double *x, int64_t n_walks,
                         double eps, double sigma, double s_ub, int64_t step_idx, int32_t *flag,
                         double *grad_out, void *stream) {
    WOS_TRY(check_common(dom, x, 1, n_walks, eps, sigma));
    if (flag == nullptr || !(s_ub > 0)) return fail(WOS_ERR_INVALID_ARG, "flag NULL or s_ub <= 0");
    const Opts o = read_opts(opt);
    WOS_TRY(check_opts(o, n_walks));
    cudaStream_t s = (cudaStream_t)stream;
    if (o.precision == WOS_MIXED) {
        WeightTable t;
        WOS_TRY(ensure_table(dom, sigma, &t, s, false));
    }
    const int nf = acc_fields(dom->d, dom->n_exp, o.cv, dom->has_source);
    const size_t bytes = scratch_bytes(o.precision, 1, nf) + 256;
    const size_t extra = o.precision == WOS_MIXED ? mixed_extra_bytes(*dom, 1, n_walks, 1, o.cv) : 0;
    void *base = nullptr;
    WOS_CUDA(cudaMallocAsync(&base, bytes + extra, s));
    Scratch sc = carve_scratch(base, o.precision, 1, nf);
    if (o.precision == WOS_MIXED) carve_mixed(sc, (char *)base + bytes, *dom, 1, n_walks, 1);
    int *ints = reinterpret_cast<int *>((char *)base + bytes - 256);
    wos_status st = WOS_OK;
    if (cudaMemsetAsync(ints, 0, 3 * sizeof(int), s) != cudaSuccess) st = fail(WOS_ERR_CUDA, "memset");
    if (st == WOS_OK)
        st = enqueue_plan_step(dom, o, x, n_walks, eps, sigma, s_ub, step_idx, ints, ints + 1, flag,
                               sc, grad_out, nullptr, s);
    cudaFreeAsync(base, s);
    return st;
}

wos_status wos_plan_path(wos_domain_t dom, const wos_options *opt, const double *x0,
                         int64_t n_steps, int64_t n_walks, double eps, double sigma, double s_ub,
                         double *path, int32_t *flags, double *grads, void *stream) {
    WOS_TRY(check_common(dom, x0, 1, n_walks, eps, sigma));
    if (path == nullptr || flags == nullptr || n_steps < 0 || !(s_ub > 0))
        return fail(WOS_ERR_INVALID_ARG, "bad planner arguments");
    const Opts o = read_opts(opt);
    WOS_TRY(check_opts(o, n_walks));
    cudaStream_t s = (cudaStream_t)stream;
    const int d = dom->d;
    WOS_CUDA(cudaMemcpyAsync(path, x0, sizeof(double) * d, cudaMemcpyDeviceToDevice, s));
    if (n_steps == 0) return WOS_OK;
    if (o.precision == WOS_MIXED) {
        WeightTable t;
        WOS_TRY(ensure_table(dom, sigma, &t, s, true));
        WOS_TRY(ensure_mixed_smem(mixed_smem_bytes(*dom)));
    }
    const int nf = acc_fields(d, dom->n_exp, o.cv, dom->has_source);
    const size_t bytes = ((scratch_bytes(o.precision, 1, nf) + 256 + sizeof(double) * d) + 255) & ~(size_t)255;
    const size_t extra = o.precision == WOS_MIXED ? mixed_extra_bytes(*dom, 1, n_walks, 1, o.cv) : 0;
    void *base = nullptr;
    WOS_CUDA(cudaMalloc(&base, bytes + extra));
    Scratch sc = carve_scratch(base, o.precision, 1, nf);
    if (o.precision == WOS_MIXED) carve_mixed(sc, (char *)base + bytes, *dom, 1, n_walks, 1);
    int *ints = reinterpret_cast<int *>((char *)base + scratch_bytes(o.precision, 1, nf));
    double *x = reinterpret_cast<double *>((char *)ints + 256);
    wos_status st = WOS_OK;
    cudaStream_t cap = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    do {
        if (cudaMemsetAsync(ints, 0, 3 * sizeof(int), s) != cudaSuccess ||
            cudaMemcpyAsync(x, x0, sizeof(double) * d, cudaMemcpyDeviceToDevice, s) != cudaSuccess) {
            st = fail(WOS_ERR_CUDA, "planner setup failed");
            break;
        }
        if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess) {
            st = fail(WOS_ERR_CUDA, "stream create failed");
            break;
        }
        if (cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
            st = fail(WOS_ERR_CUDA, "graph capture failed to start");
            break;
        }
        for (int64_t i = 0; i < n_steps && st == WOS_OK; ++i)
            st = enqueue_plan_step(dom, o, x, n_walks, eps, sigma, s_ub, i, ints, ints + 1,
                                   flags + i, sc, grads ? grads + i * d : nullptr,
                                   path + (i + 1) * d, cap);
        cudaError_t e = cudaStreamEndCapture(cap, &graph);
        if (st != WOS_OK) break;
        if (e != cudaSuccess) {
            st = fail(WOS_ERR_CUDA, "graph capture failed: %s", cudaGetErrorString(e));
            break;
        }
        e = cudaGraphInstantiate(&exec, graph, 0);
        if (e != cudaSuccess) {
            st = fail(WOS_ERR_CUDA, "graph instantiate failed: %s", cudaGetErrorString(e));
            break;
        }
        e = cudaGraphLaunch(exec, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        int timed_out = 0;
        if (e == cudaSuccess) e = cudaMemcpy(&timed_out, ints + 2, sizeof(int), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) st = fail(WOS_ERR_CUDA, "planner graph failed: %s", cudaGetErrorString(e));
        else if (timed_out) st = fail(WOS_ERR_TIMEOUT, "a tensor-core walker wait ran out of its budget");
    } while (0);
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (cap) cudaStreamDestroy(cap);
    cudaStreamSynchronize(s);
    cudaFree(base);
    return st;
}

}  // extern "C"

// =====================================================================================
// backward
// =====================================================================================
namespace {

__global__ void backward_kernel(const double *gout, const double *grad, const double *dsig,
                                const double *dw, int64_t Q, int d, int K, double *gx,
                                double *gsigma, double *gw) {
    __shared__ double red[256];
    if (gx != nullptr)
        for (int64_t i = threadIdx.x; i < Q * d; i += blockDim.x) gx[i] = gout[i / d] * grad[i];
    for (int s = 0; s <= K; ++s) {
        const double *src = s == 0 ? dsig : dw;
        double *dst = s == 0 ? gsigma : gw + (s - 1);
        if (src == nullptr || (s == 0 && gsigma == nullptr) || (s > 0 && gw == nullptr)) continue;
        double acc = 0.0;
        for (int64_t q = threadIdx.x; q < Q; q += blockDim.x)
            acc += gout[q] * (s == 0 ? src[q] : src[q * K + (s - 1)]);
        red[threadIdx.x] = acc;
        __syncthreads();
        for (int w = 128; w > 0; w >>= 1) {
            if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
            __syncthreads();
        }
        if (threadIdx.x == 0) *dst = red[0];
        __syncthreads();
    }
}

}  // namespace

extern "C" wos_status wos_backward(const double *gout, const double *grad, const double *du_dsigma,
                                   const double *du_dw, int64_t Q, int32_t d, int32_t K,
                                   double *gx, double *gsigma, double *gw, void *stream) {
    if (Q < 0 || d < 1 || K < 0) return fail(WOS_ERR_INVALID_ARG, "bad sizes");
    if (Q > 0 && gout == nullptr) return fail(WOS_ERR_INVALID_ARG, "gout is NULL");
    if (gx != nullptr && grad == nullptr) return fail(WOS_ERR_INVALID_ARG, "grad is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    if (Q == 0) {
        if (gsigma) WOS_CUDA(cudaMemsetAsync(gsigma, 0, sizeof(double), s));
        if (gw && K) WOS_CUDA(cudaMemsetAsync(gw, 0, sizeof(double) * K, s));
        return WOS_OK;
    }
    backward_kernel<<<1, 256, 0, s>>>(gout, grad, du_dsigma, du_dw, Q, d, K, gx, gsigma, gw);
    WOS_CUDA(cudaGetLastError());
    return WOS_OK;
}

// =====================================================================================
// random-stream diagnostics
// =====================================================================================
namespace {
__global__ void philox_kernel(uint64_t seed, uint64_t walk0, int64_t n, uint32_t step, uint32_t block,
                              uint32_t *out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint4 r = philox_block(seed, walk0 + (uint64_t)i, step, block);
        out[4 * i + 0] = r.x;
        out[4 * i + 1] = r.y;
        out[4 * i + 2] = r.z;
        out[4 * i + 3] = r.w;
    }
}
}  // namespace

extern "C" wos_status wos_debug_philox(uint64_t seed, uint64_t walk0, int64_t n, uint32_t step,
                                       uint32_t block, uint32_t *out, void *stream) {
    if (n < 0 || (n > 0 && out == nullptr)) return fail(WOS_ERR_INVALID_ARG, "bad arguments");
    if (n == 0) return WOS_OK;
    const int64_t blocks = std::min<int64_t>((n + 255) / 256, 65535);
    philox_kernel<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(seed, walk0, n, step, block, out);
    WOS_CUDA(cudaGetLastError());
    return WOS_OK;
}

// =====================================================================================
// weight-table diagnostics
// =====================================================================================
extern "C" wos_status wos_debug_weight_table(int32_t d, double z_max, int32_t n, double *log_c,
                                             double *ratio) {
    if (d < 2 || d > WOS_MAX_D || n < 2 || !(z_max > 0) || !log_c || !ratio)
        return fail(WOS_ERR_INVALID_ARG, "bad arguments");
    float2 *t = nullptr;
    WOS_CUDA(cudaMalloc(&t, sizeof(float2) * n));
    build_table_kernel<<<(n + 255) / 256, 256>>>(d, z_max / (n - 1), n, t);
    std::vector<float2> h(n);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpy(h.data(), t, sizeof(float2) * n, cudaMemcpyDeviceToHost);
    cudaFree(t);
    if (e != cudaSuccess) return fail(WOS_ERR_CUDA, "table debug failed: %s", cudaGetErrorString(e));
    for (int i = 0; i < n; ++i) {
        log_c[i] = h[i].x;
        ratio[i] = h[i].y;
    }
    return WOS_OK;
}

// =====================================================================================
// batched uneven problems: one persistent launch, recorded as a CUDA graph
// =====================================================================================
struct wos_batch_s {
    std::vector<wos_problem> probs;
    std::vector<const int *> done;  // per problem: nonzero -> no walks (finished planner paths)
    int *sph_status = nullptr;      // the tensor-core launches' status word (zeroed every run)
    Opts o{};
    wos_batch_config cfg{};
    int grad_any = 0;
    size_t smem = 0;
    int grid = 0;
    int64_t n_items = 0, total_q = 0;
    int64_t n_sphere_items = 0;  // items of the tensor-core sphere-set launches
    void *dev = nullptr;       // problems | items | finalize records | records | zeroed region
    size_t zero_off = 0, zero_bytes = 0;
    size_t off_sph = 0;        // the tensor-core problem table in dev
    std::vector<int> sph_index;  // batch problem -> tensor-core problem (-1: CUDA-core walker)
    std::vector<double *> acc_ptr;                // per problem: its accumulators
    std::vector<unsigned long long *> cnt_ptr;    // ... and counters
    int min_walks_per_lane = 8;  // CUDA-core items hold at least this many walks per lane
    wos_stats *d_stats = nullptr;
    // one run: [memset zeroed region] [tensor-core launches per queue | CUDA-core walker]
    // [reduction] [finalize]
    MixedLaunch L{};
    std::vector<SphereLaunch> sph;
    std::vector<int> sph_grid, sph_dims, sph_src, sph_wide;
    ReduceArgs ra{};
    bool any_seg = false;
    FinalizeArgs fa{};
    bool no_graph = false;     // planner paths capture their own graph
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::string signature;
};

namespace {

std::mutex g_cache_mu;
std::string g_cache_path;

size_t align256(size_t n) { return (n + 255) & ~(size_t)255; }

// Relative cost of one walk step of a problem: ball screen B (d+3), plus the fixed per-step
// work (faces, sampling, weights).
double step_cost(const wos_domain_s &D) { return (double)D.n_balls * (D.d + 3) + 40.0 * D.d + 200.0; }

std::string batch_signature(const std::vector<wos_problem> &ps) {
    uint64_t h = 1469598103934665603ull;
    auto mix = [&](uint64_t v) {
        for (int i = 0; i < 8; ++i) {
            h ^= (v >> (8 * i)) & 0xff;
            h *= 1099511628211ull;
        }
    };
    mix(ps.size());
    for (const wos_problem &p : ps) {
        mix((uint64_t)p.domain->d);
        mix((uint64_t)p.domain->n_balls);
        mix((uint64_t)p.n_queries);
        mix((uint64_t)p.n_walks);
        mix(p.grad != nullptr);
    }
    int dev = 0;
    cudaDeviceProp prop{};
    cudaGetDevice(&dev);
    cudaGetDeviceProperties(&prop, dev);
    char buf[64];
    snprintf(buf, sizeof(buf), "%016llx", (unsigned long long)h);
    std::string name(prop.name);
    for (char &c : name)
        if (c == ' ') c = '_';
    return name + ":" + buf;
}

bool cache_lookup(const std::string &path, const std::string &sig, wos_batch_config *cfg) {
    if (path.empty()) return false;
    FILE *f = fopen(path.c_str(), "r");
    if (!f) return false;
    char line[512], key[256];
    int th, ct, sct;
    long long iw, siw;
    double ms;
    bool found = false;
    while (fgets(line, sizeof(line), f) != nullptr) {
        if (line[0] == '#') continue;  // candidate timings
        if (sscanf(line, "%255s %d %d %lld %d %lld %lf", key, &th, &ct, &iw, &sct, &siw, &ms) == 7 && sig == key) {
            cfg->threads = th;  // the last entry for a signature wins
            cfg->ctas_per_sm = ct;
            cfg->item_work = iw;
            cfg->sphere_ctas_per_sm = sct;
            cfg->sphere_item_walks = siw;
            found = true;
        }
    }
    fclose(f);
    return found;
}

void free_batch_device(wos_batch_s *b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->dev) cudaFree(b->dev);
    b->exec = nullptr;
    b->graph = nullptr;
    b->dev = nullptr;
}

// Side streams and events of a capture: one branch per tensor-core launch.
struct CaptureSide {
    std::vector<cudaStream_t> side;
    std::vector<cudaEvent_t> ev;  // one per branch, then the fork event
    wos_status init(size_t n) {
        side.assign(n, nullptr);
        ev.assign(n + 1, nullptr);
        for (size_t k = 0; k < n; ++k)
            if (cudaStreamCreateWithFlags(&side[k], cudaStreamNonBlocking) != cudaSuccess)
                return fail(WOS_ERR_CUDA, "stream creation failed");
        for (size_t k = 0; k < ev.size(); ++k)
            if (cudaEventCreateWithFlags(&ev[k], cudaEventDisableTiming) != cudaSuccess)
                return fail(WOS_ERR_CUDA, "event creation failed");
        return WOS_OK;
    }
    ~CaptureSide() {
        for (cudaStream_t x : side)
            if (x) cudaStreamDestroy(x);
        for (cudaEvent_t x : ev)
            if (x) cudaEventDestroy(x);
    }
};

// Enqueues one run of the batch's walkers and reduction (no finalize) on a capturing stream:
// zero the accumulators and queue cursors, fork the tensor-core launches onto the side streams,
// run the CUDA-core walker, join, reduce.
wos_status enqueue_batch_core(wos_batch_s *b, cudaStream_t cap, CaptureSide &cs) {
    char *zero = (char *)b->dev + b->zero_off;
    if (cudaMemsetAsync(zero, 0, b->zero_bytes, cap) != cudaSuccess) return fail(WOS_ERR_CUDA, "memset capture");
    const size_t ns = b->sph.size();
    if (ns > 0 && cudaEventRecord(cs.ev.back(), cap) != cudaSuccess) return fail(WOS_ERR_CUDA, "fork event capture");
    for (size_t k = 0; k < ns; ++k)
        if (cudaStreamWaitEvent(cs.side[k], cs.ev.back(), 0) != cudaSuccess ||
            launch_spheres(b->sph[k], b->sph_dims[k], b->grad_any, b->sph_src[k], b->sph_wide[k], b->sph_grid[k],
                           cs.side[k]) !=
                cudaSuccess ||
            cudaEventRecord(cs.ev[k], cs.side[k]) != cudaSuccess)
            return fail(WOS_ERR_CUDA, "sphere-set kernel capture failed");
    if (b->n_items > 0 && launch_walk_mixed(b->L, b->grad_any, b->grid, b->cfg.threads, b->smem, cap) != cudaSuccess)
        return fail(WOS_ERR_CUDA, "walk kernel capture failed");
    for (size_t k = 0; k < ns; ++k)
        if (cudaStreamWaitEvent(cap, cs.ev[k], 0) != cudaSuccess) return fail(WOS_ERR_CUDA, "join capture failed");
    return launch_reduce(b->ra, b->total_q, b->any_seg, cap);
}

wos_status batch_build(wos_batch_s *b, const wos_batch_config &cfg_in) {
    free_batch_device(b);
    wos_batch_config cfg = cfg_in;
    if (cfg.threads < 32 || cfg.threads > 768 || cfg.threads % 32)
        return fail(WOS_ERR_INVALID_ARG, "threads must be a multiple of 32 in 32..768");
    if (cfg.ctas_per_sm < 1 || cfg.ctas_per_sm > 8) return fail(WOS_ERR_INVALID_ARG, "ctas_per_sm in 1..8");
    if (cfg.item_work < 1) return fail(WOS_ERR_INVALID_ARG, "item_work must be positive");
    if (cfg.sphere_ctas_per_sm < 1 || cfg.sphere_ctas_per_sm > sphere_ctas_per_sm())
        return fail(WOS_ERR_INVALID_ARG, "sphere_ctas_per_sm in 1..%d", sphere_ctas_per_sm());
    if (cfg.sphere_item_walks < 128 || cfg.sphere_item_walks > (1 << 20) || cfg.sphere_item_walks % 128)
        return fail(WOS_ERR_INVALID_ARG, "sphere_item_walks: a multiple of 128 in 128..2^20");
    const int n = (int)b->probs.size();
    b->grad_any = 0;
    b->smem = 16;
    // problems whose obstacles are a tensor-core sphere set (large ball sets, point sets) run on
    // the sphere-set walker, the others on the CUDA-core persistent walker
    std::vector<char> tensor(n, 0);
    for (int i = 0; i < n; ++i) {
        const wos_problem &p = b->probs[i];
        b->grad_any |= p.grad != nullptr;
        if (p.domain->n_points > 0 && !p.domain->has_pcd)
            return fail(WOS_ERR_UNSUPPORTED, "problem %d: mixed-precision point sets need d <= %d", i, kPointCloudMaxD);
        if (p.domain->n_points > 0 && p.domain->n_balls > 0)
            return fail(WOS_ERR_UNSUPPORTED, "problem %d: a domain with both balls and points", i);
        if (p.domain->n_links > 0 &&
            (p.domain->n_points > 0 || p.domain->n_arm_obs > kMaxArmObs || p.domain->d > kMaxArmLinksMixed))
            return fail(WOS_ERR_UNSUPPORTED, "problem %d: an arm with a point set or over %d obstacle points", i,
                        kMaxArmObs);
        tensor[i] = p.domain->has_pcd && (p.domain->n_points > 0 || !b->o.cuda_core_balls);
        if (!tensor[i]) b->smem = std::max(b->smem, mixed_smem_bytes(*p.domain));
    }
    if (b->smem > 227 * 1024) return fail(WOS_ERR_UNSUPPORTED, "ball set needs %zu B of shared memory", b->smem);
    WOS_TRY(ensure_mixed_smem(b->smem));
    const int occ = max_active_mixed(cfg.threads, b->smem, b->grad_any);
    if (occ < 1) return fail(WOS_ERR_UNSUPPORTED, "persistent walker does not fit with %d threads", cfg.threads);
    cfg.ctas_per_sm = std::min(cfg.ctas_per_sm, occ);
    b->cfg = cfg;
    const int sms = device_sms();

    // problem records, accumulators and work items
    std::vector<MixedProblem> mp(n);
    std::vector<FinalizeRec> fr(n);
    size_t acc_bytes = 0;
    std::vector<size_t> acc_off(n), cnt_off(n);
    for (int i = 0; i < n; ++i) {
        const wos_problem &p = b->probs[i];
        const int nf = acc_fields(p.domain->d, p.domain->n_exp, p.grad != nullptr && b->o.cv,
                                  p.grad != nullptr && p.domain->has_source);
        acc_off[i] = acc_bytes;
        acc_bytes += align256((size_t)p.n_queries * nf * sizeof(double));
    }
    for (int i = 0; i < n; ++i) {
        cnt_off[i] = acc_bytes;
        acc_bytes += align256((size_t)b->probs[i].n_queries * kCounters * 8);
    }
    const size_t off_items = align256(sizeof(MixedProblem) * n);
    int64_t walk_base = b->o.walk_offset, q_begin = 0;
    // Items: at least 8 walks per lane (so the walk-length spread averages out before an item
    // ends), about item_work units of work otherwise. Problems in decreasing order of total
    // work, each problem's items consecutive: the long items go first, a CTA usually pulls its
    // next item from the problem it has staged, and the tail of the launch is made of short
    // items.
    std::vector<double> prob_cost(n);
    std::vector<int64_t> prob_wpi(n);
    for (int i = 0; i < n; ++i) {
        const wos_problem &p = b->probs[i];
        const double c = step_cost(*p.domain);
        int64_t wpi = (int64_t)((double)cfg.item_work / c);
        wpi = std::max<int64_t>((int64_t)b->min_walks_per_lane * cfg.threads, std::min<int64_t>(1 << 20, wpi));
        prob_wpi[i] = (wpi + 31) / 32 * 32;
        prob_cost[i] = c * (double)(p.n_queries * p.n_walks);
        walk_base += p.n_queries * p.n_walks;
        q_begin += p.n_queries;
    }
    std::vector<int> porder(n);
    for (int i = 0; i < n; ++i) porder[i] = i;
    std::stable_sort(porder.begin(), porder.end(),
                     [&](int a, int c) { return prob_cost[a] > prob_cost[c]; });
    std::vector<MixedItem> sorted;
    for (int i : porder) {
        if (tensor[i]) continue;
        const wos_problem &p = b->probs[i];
        const int64_t total = p.n_queries * p.n_walks;
        for (int64_t j0 = 0; j0 < total; j0 += prob_wpi[i]) {
            MixedItem it{};
            it.problem = i;
            it.j0 = j0;
            it.j1 = std::min(total, j0 + prob_wpi[i]);
            sorted.push_back(it);
        }
    }
    b->n_items = (int64_t)sorted.size();
    b->total_q = q_begin;
    // sphere-set items: one queue per dimension and set class (sphere_queue_class), problems by
    // decreasing cost, sphere_item_walks walks per item (a CTA continues into the next item of the
    // same problem without a pause, so items only matter for the balance at the end)
    const int64_t kSphereItemWalks = cfg.sphere_item_walks;
    std::vector<int> sph_index(n, -1);
    std::vector<int> sph_problem;  // sphere problem -> batch problem
    // one queue per (dimension, class): group kSphereQueueClasses d + sphere_queue_class(d, tiles)
    constexpr int kSphGroups = kSphereQueueClasses * (kPointCloudMaxD + 1);
    std::vector<std::vector<SphereItem>> sph_items(kSphGroups);
    for (int i : porder) {
        if (!tensor[i]) continue;
        sph_index[i] = (int)sph_problem.size();
        sph_problem.push_back(i);
        const wos_problem &p = b->probs[i];
        const int64_t total = p.n_queries * p.n_walks;
        for (int64_t j0 = 0; j0 < total; j0 += kSphereItemWalks) {
            SphereItem it{};
            it.problem = sph_index[i];
            it.j0 = j0;
            it.j1 = std::min(total, j0 + kSphereItemWalks);
            sph_items[kSphereQueueClasses * p.domain->d + sphere_queue_class(p.domain->d, p.domain->pcd.n_tiles)]
                .push_back(it);
        }
    }
    std::vector<SphereItem> sph_all;
    std::vector<size_t> sph_off(kSphGroups + 1, 0);
    for (int g = 0; g < kSphGroups; ++g) {
        sph_off[g] = sph_all.size();
        sph_all.insert(sph_all.end(), sph_items[g].begin(), sph_items[g].end());
    }
    sph_off[kSphGroups] = sph_all.size();
    b->n_sphere_items = (int64_t)sph_all.size();
    const int n_sph = (int)sph_problem.size();
    const size_t off_recs = off_items + align256(sizeof(MixedItem) * std::max<size_t>(1, sorted.size()));
    const size_t off_sph = off_recs + align256(sizeof(FinalizeRec) * n);
    const size_t off_sph_items = off_sph + align256(sizeof(SphereProblem) * std::max(1, n_sph));
    // per-walk records and segment partials of every problem, and the reduction's problem table
    const size_t off_red = off_sph_items + align256(sizeof(SphereItem) * std::max<size_t>(1, sph_all.size()));
    size_t off_rec = off_red + align256(sizeof(ReduceRec) * std::max(1, n));
    std::vector<size_t> rec_off(n), part_off(n);
    for (int i = 0; i < n; ++i) {
        const wos_problem &p = b->probs[i];
        const int g = p.grad != nullptr;
        rec_off[i] = off_rec;
        off_rec += record_bytes(p.domain->d, p.domain->n_exp, g, p.n_queries, p.n_walks);
        part_off[i] = off_rec;
        off_rec += partial_bytes(p.domain->d, p.domain->n_exp, g && b->o.cv, p.n_queries, p.n_walks);
    }
    const size_t off_zero = off_rec;
    // zeroed: accumulators | mixed cursor (8) + sphere status (8) + shrinks (8) + one cursor per
    // sphere queue | stats
    const size_t ctl_bytes = align256(8 * (3 + kSphGroups));
    const size_t zero_bytes = acc_bytes + ctl_bytes + align256(sizeof(wos_stats));
    const size_t total_bytes = off_zero + zero_bytes;
    WOS_CUDA(cudaMalloc(&b->dev, total_bytes));
    char *base = (char *)b->dev;
    char *zero = base + off_zero;
    unsigned long long *cursor = (unsigned long long *)(zero + acc_bytes);
    int *sph_status = reinterpret_cast<int *>(cursor + 1);
    b->sph_status = sph_status;
    unsigned long long *sph_shrinks = cursor + 2;
    unsigned long long *sph_cursors = cursor + 3;  // [queue group]
    b->d_stats = (wos_stats *)(zero + acc_bytes + ctl_bytes);
    b->zero_off = off_zero;
    b->zero_bytes = zero_bytes;
    walk_base = b->o.walk_offset;
    q_begin = 0;
    std::vector<ReduceRec> rr(n);
    int64_t red_blocks = 0;
    bool any_seg = false;
    b->acc_ptr.assign(n, nullptr);
    b->cnt_ptr.assign(n, nullptr);
    for (int i = 0; i < n; ++i) {
        const wos_problem &p = b->probs[i];
        WeightTable tab;
        WOS_TRY(ensure_table(p.domain, p.sigma, &tab, nullptr, true));
        double *acc = (double *)(zero + acc_off[i]);
        unsigned long long *cnt = (unsigned long long *)(zero + cnt_off[i]);
        b->acc_ptr[i] = acc;
        b->cnt_ptr[i] = cnt;
        mp[i] = make_mixed_problem(p.domain, p.x, p.n_queries, p.n_walks, p.eps, p.sigma,
                                   p.grad != nullptr, b->o.laplace, b->o.cv, walk_base, tab, acc, cnt,
                                   PerWalk{}, reinterpret_cast<float *>(base + rec_off[i]));
        apply_walk_opts(mp[i], b->o);
        mp[i].done = i < (int)b->done.size() ? b->done[i] : nullptr;
        rr[i] = make_reduce_rec(p.domain->d, p.domain->n_exp, p.grad != nullptr, b->o.cv, p.domain->has_source,
                                b->o.antithetic, p.n_queries, p.n_walks, reinterpret_cast<float *>(base + rec_off[i]), acc, cnt,
                                reinterpret_cast<double *>(base + part_off[i]));
        rr[i].blk_begin = red_blocks;
        rr[i].q_begin = q_begin;
        red_blocks += p.n_queries * rr[i].nseg;
        any_seg |= rr[i].nseg > 1;
        FinalizeRec &r = fr[i];
        r.d = p.domain->d;
        r.K = p.domain->n_exp;
        r.acc_f32 = 0;
        r.anti = b->o.antithetic;
        r.cv = mp[i].cv;
        r.src = mp[i].src;
        r.Q = p.n_queries;
        r.N = p.n_walks;
        r.q_begin = q_begin;
        r.acc = acc;
        r.counts = cnt;
        r.u = p.u;
        r.u_se = p.u_se;
        r.grad = p.grad;
        r.grad_se = p.grad_se;
        r.du_dsigma = nullptr;
        r.du_dw = nullptr;
        r.walk_steps = p.walk_steps;
        walk_base += p.n_queries * p.n_walks;
        q_begin += p.n_queries;
    }
    WOS_CUDA(cudaMemcpy(base, mp.data(), sizeof(MixedProblem) * n, cudaMemcpyHostToDevice));
    if (!sorted.empty())
        WOS_CUDA(cudaMemcpy(base + off_items, sorted.data(), sizeof(MixedItem) * sorted.size(),
                            cudaMemcpyHostToDevice));
    WOS_CUDA(cudaMemcpy(base + off_recs, fr.data(), sizeof(FinalizeRec) * n, cudaMemcpyHostToDevice));
    if (n > 0) WOS_CUDA(cudaMemcpy(base + off_red, rr.data(), sizeof(ReduceRec) * n, cudaMemcpyHostToDevice));
    ReduceArgs ra{};
    ra.recs = (const ReduceRec *)(base + off_red);
    ra.n = n;
    ra.total_blocks = red_blocks;
    ra.skip = nullptr;
    if (n_sph > 0) {
        std::vector<SphereProblem> sp(n_sph);
        for (int k = 0; k < n_sph; ++k) {
            const int i = sph_problem[k];
            const wos_domain_s &D = *b->probs[i].domain;
            sp[k].P = mp[i];
            sp[k].tiles = D.pcd.tiles;
            sp[k].soa = D.pcd.soa;
            sp[k].chunk_rhi = D.pcd.chunk_rhi;
            sp[k].n_tiles = D.pcd.n_tiles;
            sp[k].delta = D.pc_delta;
        }
        WOS_CUDA(cudaMemcpy(base + off_sph, sp.data(), sizeof(SphereProblem) * n_sph, cudaMemcpyHostToDevice));
        WOS_CUDA(cudaMemcpy(base + off_sph_items, sph_all.data(), sizeof(SphereItem) * sph_all.size(),
                            cudaMemcpyHostToDevice));
    }

    b->off_sph = off_sph;
    b->sph_index = sph_index;
    MixedLaunch &L = b->L;
    L = MixedLaunch{};
    L.problems = (const MixedProblem *)base;
    L.items = (const MixedItem *)(base + off_items);
    L.n_items = b->n_items;
    L.cursor = cursor;
    L.seed = b->o.seed;
    L.max_steps = b->o.max_steps;
    L.skip = nullptr;
    b->grid = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)sms * cfg.ctas_per_sm, b->n_items));
    b->ra = ra;
    b->any_seg = any_seg;
    FinalizeArgs &fa = b->fa;
    fa = FinalizeArgs{};
    fa.recs = (const FinalizeRec *)(base + off_recs);
    fa.n = n;
    fa.total_q = b->total_q;
    fa.stats = b->d_stats;
    fa.status = n_sph > 0 ? sph_status : nullptr;
    fa.shrinks = n_sph > 0 ? sph_shrinks : nullptr;
    // one sphere-set launch per queue (run on their own streams so that their CTAs and the
    // CUDA-core walker's share the GPU as each queue drains)
    b->sph.clear();
    b->sph_grid.clear();
    b->sph_dims.clear();
    b->sph_src.clear();
    b->sph_wide.clear();
    for (int g = 0; g < kSphGroups; ++g) {
        if (sph_off[g + 1] <= sph_off[g]) continue;
        const int dd = g / kSphereQueueClasses, cls = g % kSphereQueueClasses, wide = cls == 2 ? 1 : 0;
        SphereLaunch SL;
        memset(&SL, 0, sizeof(SL));
        SL.problems = (const SphereProblem *)(base + off_sph);
        SL.items = (const SphereItem *)(base + off_sph_items) + sph_off[g];
        SL.n_items = (int64_t)(sph_off[g + 1] - sph_off[g]);
        SL.item_cursor = sph_cursors + g;
        SL.status = sph_status;
        SL.shrinks = sph_shrinks;
        SL.seed = b->o.seed;
        SL.max_steps = b->o.max_steps;
        SL.wait_budget = b->o.wait_cycles > 0 ? b->o.wait_cycles : kDefaultWaitBudget;
        SL.wait_hint = wait_hint_ns(SL.wait_budget);
        b->sph.push_back(SL);
        b->sph_grid.push_back((int)std::min<int64_t>((int64_t)cfg.sphere_ctas_per_sm * sms, SL.n_items));
        b->sph_dims.push_back(dd);
        b->sph_wide.push_back(wide);
        int src_any = 0;  // the source variant of the kernel if a problem of this queue has one
        for (int k : sph_problem) {
            const wos_domain_t dk = b->probs[k].domain;
            src_any |= dk->d == dd && sphere_queue_class(dd, dk->pcd.n_tiles) == cls && dk->has_source;
        }
        b->sph_src.push_back(src_any);
    }
    if (b->no_graph) return WOS_OK;
    CaptureSide side;
    WOS_TRY(side.init(b->sph.size()));
    cudaStream_t cap = nullptr;
    WOS_CUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    if (cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaStreamDestroy(cap);
        return fail(WOS_ERR_CUDA, "batch capture failed to start");
    }
    wos_status st = enqueue_batch_core(b, cap, side);
    if (st == WOS_OK) st = launch_finalize(b->fa, cap);
    cudaError_t e = cudaStreamEndCapture(cap, &b->graph);
    cudaStreamDestroy(cap);
    if (st != WOS_OK) return st;
    if (e != cudaSuccess) return fail(WOS_ERR_CUDA, "batch capture failed: %s", cudaGetErrorString(e));
    WOS_CUDA(cudaGraphInstantiate(&b->exec, b->graph, 0));
    return WOS_OK;
}

wos_batch_config default_batch_config() {
    // the autotuner's choice for the 256-problem batched workload on GB300 (858 ms per run
    // against 963 ms for 512 threads and item_work 2^26)
    wos_batch_config c{};
    c.threads = 768;
    c.ctas_per_sm = 1;
    c.item_work = (int64_t)1 << 24;
    c.sphere_ctas_per_sm = sphere_ctas_per_sm();
    c.sphere_item_walks = 4096;
    return c;
}

}  // namespace

extern "C" {

wos_status wos_set_autotune_cache(const char *cache_path) {
    std::lock_guard<std::mutex> lk(g_cache_mu);
    g_cache_path = cache_path ? cache_path : "";
    return WOS_OK;
}

wos_status wos_batch_create(const wos_problem *probs, int32_t n_problems, const wos_options *opt,
                            const wos_batch_config *cfg, wos_batch_t *out) {
    if (out == nullptr) return fail(WOS_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (n_problems < 0 || (n_problems > 0 && probs == nullptr))
        return fail(WOS_ERR_INVALID_ARG, "bad problem array");
    const Opts o = read_opts(opt);
    if (opt != nullptr && o.precision != WOS_MIXED)
        return fail(WOS_ERR_UNSUPPORTED, "batched launches run the mixed-precision walker");
    if (o.max_steps > (int64_t)kRecKMask) return fail(WOS_ERR_INVALID_ARG, "max_steps must be below 2^28");
    for (int i = 0; i < n_problems; ++i) {
        const wos_problem &p = probs[i];
        WOS_TRY(check_common(p.domain, p.x, p.n_queries, p.n_walks, p.eps, p.sigma));
        if (p.n_queries > 0 && p.u == nullptr) return fail(WOS_ERR_INVALID_ARG, "problem %d: u is NULL", i);
        if (p.domain->n_points > 0 && !p.domain->has_pcd)
            return fail(WOS_ERR_UNSUPPORTED, "problem %d: mixed-precision point sets need d <= %d", i,
                        kPointCloudMaxD);
        if (p.n_queries * p.n_walks > (int64_t)0x7fffffff)
            return fail(WOS_ERR_UNSUPPORTED, "problem %d: n_queries * n_walks must be < 2^31", i);
        Opts oc = o;
        if (p.grad == nullptr) oc.cv = 0;
        WOS_TRY(check_opts(oc, p.n_walks));
    }
    wos_batch_s *b = new (std::nothrow) wos_batch_s();
    if (b == nullptr) return fail(WOS_ERR_OOM, "host allocation failed");
    b->probs.assign(probs, probs + n_problems);
    b->o = o;
    b->signature = batch_signature(b->probs);
    wos_batch_config c = default_batch_config();
    if (cfg != nullptr) {
        c = *cfg;
    } else {
        std::lock_guard<std::mutex> lk(g_cache_mu);
        cache_lookup(g_cache_path, b->signature, &c);
    }
    const wos_status st = batch_build(b, c);
    if (st != WOS_OK) {
        free_batch_device(b);
        delete b;
        return st;
    }
    *out = b;
    return WOS_OK;
}

wos_status wos_batch_run(wos_batch_t b, wos_stats *stats, void *stream) {
    if (b == nullptr || b->exec == nullptr) return fail(WOS_ERR_INVALID_ARG, "batch is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    WOS_CUDA(cudaGraphLaunch(b->exec, s));
    if (stats != nullptr)
        WOS_CUDA(cudaMemcpyAsync(stats, b->d_stats, sizeof(wos_stats), cudaMemcpyDeviceToDevice, s));
    return WOS_OK;
}

wos_status wos_batch_get_config(wos_batch_t b, wos_batch_config *cfg) {
    if (b == nullptr || cfg == nullptr) return fail(WOS_ERR_INVALID_ARG, "NULL argument");
    *cfg = b->cfg;
    return WOS_OK;
}

wos_status wos_batch_destroy(wos_batch_t b) {
    if (b == nullptr) return WOS_OK;
    cudaDeviceSynchronize();
    free_batch_device(b);
    delete b;
    return WOS_OK;
}

wos_status wos_solve_batch(const wos_problem *probs, int32_t n_problems, const wos_options *opt,
                           wos_stats *stats, void *stream) {
    wos_batch_t b = nullptr;
    WOS_TRY(wos_batch_create(probs, n_problems, opt, nullptr, &b));
    wos_status st = wos_batch_run(b, stats, stream);
    if (st == WOS_OK && cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess)
        st = fail(WOS_ERR_CUDA, "batch run failed");
    wos_batch_destroy(b);
    return st;
}

wos_status wos_batch_autotune(wos_batch_t b, const char *cache_path, wos_batch_config *best) {
    if (b == nullptr) return fail(WOS_ERR_INVALID_ARG, "batch is NULL");
    const wos_batch_config start = b->cfg;
    cudaStream_t s;
    WOS_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    double best_ms = 1e300;
    wos_batch_config best_cfg = start;
    std::vector<std::pair<wos_batch_config, float>> timed;
    auto same = [](const wos_batch_config &a, const wos_batch_config &c) {
        return a.threads == c.threads && a.ctas_per_sm == c.ctas_per_sm && a.item_work == c.item_work &&
               a.sphere_ctas_per_sm == c.sphere_ctas_per_sm && a.sphere_item_walks == c.sphere_item_walks;
    };
    // one timed run of a candidate (batch_build clamps CTAs per SM to what fits: candidates that
    // end up equal to one already timed are skipped)
    auto run = [&](const wos_batch_config &c) -> bool {
        if (batch_build(b, c) != WOS_OK) return true;
        for (auto &t : timed)
            if (same(t.first, b->cfg)) return true;
        cudaEventRecord(e0, s);
        cudaGraphLaunch(b->exec, s);
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess) return false;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        timed.push_back({b->cfg, ms});
        if (ms < best_ms) {
            best_ms = ms;
            best_cfg = b->cfg;
        }
        return true;
    };
    bool ok = true;
    // first pass: the CUDA-core walker's shapes, the tensor-core walker at its default
    {
        wos_batch_config c = default_batch_config();
        for (int th : {512, 768})
            for (int64_t iw : {(int64_t)1 << 24, (int64_t)1 << 26}) {
                c.threads = th;
                c.ctas_per_sm = 1;
                c.item_work = iw;
                if (ok) ok = run(c);
            }
        c.threads = 256;
        c.ctas_per_sm = 2;
        c.item_work = (int64_t)1 << 26;
        if (ok) ok = run(c);
    }
    // second pass: the tensor-core walker's shapes with the best CUDA-core shape
    if (ok && b->n_sphere_items > 0) {
        wos_batch_config c = best_cfg;
        for (int sct : {4, 3, 2})
            for (int64_t siw : {(int64_t)2048, (int64_t)4096, (int64_t)8192}) {
                if (sct > sphere_ctas_per_sm()) continue;
                c.sphere_ctas_per_sm = sct;
                c.sphere_item_walks = siw;
                if (ok) ok = run(c);
            }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamDestroy(s);
    WOS_TRY(batch_build(b, best_cfg));
    if (best) *best = b->cfg;
    if (cache_path != nullptr && best_ms < 1e300) {
        std::lock_guard<std::mutex> lk(g_cache_mu);
        FILE *f = fopen(cache_path, "a");
        if (f) {
            for (const auto &t : timed)
                fprintf(f, "# %s %d %d %lld %d %lld %.4f\n", b->signature.c_str(), t.first.threads,
                        t.first.ctas_per_sm, (long long)t.first.item_work, t.first.sphere_ctas_per_sm,
                        (long long)t.first.sphere_item_walks, t.second);
            fprintf(f, "%s %d %d %lld %d %lld %.4f\n", b->signature.c_str(), b->cfg.threads, b->cfg.ctas_per_sm,
                    (long long)b->cfg.item_work, b->cfg.sphere_ctas_per_sm, (long long)b->cfg.sphere_item_walks,
                    best_ms);
            fclose(f);
        }
    }
    return WOS_OK;
}

wos_status wos_plan_paths(const wos_path_problem *paths, int32_t n_paths, int64_t n_steps,
                          const wos_options *opt, void *stream) {
    if (n_paths < 0 || n_steps < 0 || (n_paths > 0 && paths == nullptr))
        return fail(WOS_ERR_INVALID_ARG, "bad path array or n_steps");
    const Opts o = read_opts(opt);
    if (opt != nullptr && o.precision != WOS_MIXED)
        return fail(WOS_ERR_UNSUPPORTED, "wos_plan_paths runs the mixed-precision walkers");
    if (o.max_steps > (int64_t)kRecKMask) return fail(WOS_ERR_INVALID_ARG, "max_steps must be below 2^28");
    for (int i = 0; i < n_paths; ++i) {
        const wos_path_problem &p = paths[i];
        WOS_TRY(check_common(p.domain, p.x0, 1, p.n_walks, p.eps, p.sigma));
        if (p.path == nullptr || p.flags == nullptr || !(p.s_ub > 0))
            return fail(WOS_ERR_INVALID_ARG, "path %d: path/flags NULL or s_ub <= 0", i);
        WOS_TRY(check_opts(o, p.n_walks));
        if (p.domain->n_points > 0 && (!p.domain->has_pcd || p.domain->n_balls > 0))
            return fail(WOS_ERR_UNSUPPORTED, "path %d: this point-set domain runs in FP64 or plain FP32", i);
    }
    cudaStream_t s = (cudaStream_t)stream;
    for (int i = 0; i < n_paths; ++i)
        WOS_CUDA(cudaMemcpyAsync(paths[i].path, paths[i].x0, sizeof(double) * paths[i].domain->d,
                                 cudaMemcpyDeviceToDevice, s));
    if (n_paths == 0 || n_steps == 0) return WOS_OK;
    // scratch: current points | u | grad u | [done, skip] per path | path records
    int64_t xs = 0;
    for (int i = 0; i < n_paths; ++i) xs += paths[i].domain->d;
    const size_t off_u = align256(sizeof(double) * xs), off_g = off_u + align256(sizeof(double) * n_paths);
    const size_t off_i = off_g + align256(sizeof(double) * xs);
    const size_t off_r = off_i + align256(sizeof(int) * (2 * n_paths + 1));
    const size_t bytes = off_r + sizeof(PathRec) * n_paths;
    char *scr = nullptr;
    WOS_CUDA(cudaMalloc(&scr, bytes));
    double *xc = (double *)scr, *uc = (double *)(scr + off_u), *gc = (double *)(scr + off_g);
    int *ints = (int *)(scr + off_i);
    wos_batch_s *b = new (std::nothrow) wos_batch_s();
    if (b == nullptr) {
        cudaFree(scr);
        return fail(WOS_ERR_OOM, "host allocation failed");
    }
    wos_status st = WOS_OK;
    cudaStream_t cap = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    do {
        if (cudaMemsetAsync(ints, 0, sizeof(int) * (2 * n_paths + 1), s) != cudaSuccess) {
            st = fail(WOS_ERR_CUDA, "memset failed");
            break;
        }
        int64_t ox = 0;
        for (int i = 0; i < n_paths; ++i) {
            const wos_path_problem &p = paths[i];
            const int d = p.domain->d;
            if (cudaMemcpyAsync(xc + ox, p.x0, sizeof(double) * d, cudaMemcpyDeviceToDevice, s) != cudaSuccess) {
                st = fail(WOS_ERR_CUDA, "copy failed");
                break;
            }
            wos_problem q{};
            q.domain = p.domain;
            q.x = xc + ox;
            q.n_queries = 1;
            q.n_walks = p.n_walks;
            q.eps = p.eps;
            q.sigma = p.sigma;
            q.u = uc + i;
            q.grad = gc + ox;
            b->probs.push_back(q);
            b->done.push_back(ints + 2 * i);
            ox += d;
        }
        if (st != WOS_OK) break;
        b->o = o;
        b->no_graph = true;
        b->min_walks_per_lane = 1;  // planner steps are latency-bound: one walk per lane
        b->signature = batch_signature(b->probs);
        wos_batch_config c = default_batch_config();
        c.threads = 128;
        c.ctas_per_sm = 4;
        c.item_work = 1;
        st = batch_build(b, c);
        if (st != WOS_OK) break;
        std::vector<PathRec> recs(n_paths);
        ox = 0;
        for (int i = 0; i < n_paths; ++i) {
            const wos_path_problem &p = paths[i];
            PathRec &R = recs[i];
            PlanArgs &a = R.a;
            a = PlanArgs{};
            a.dom = p.domain->v64;
            a.x = xc + ox;
            a.eps = p.eps;
            a.s_ub = p.s_ub;
            a.N = p.n_walks;
            a.done = ints + 2 * i;
            a.skip = ints + 2 * i + 1;
            a.acc = b->acc_ptr[i];
            a.acc_f32 = 0;
            a.cv = o.cv;
            a.src = p.domain->has_source;
            a.counts = b->cnt_ptr[i];
            a.status = b->sph_status;
            a.timed_out = ints + 2 * n_paths;
            R.flags = p.flags;
            R.grads = p.grads;
            R.path = p.path;
            R.walk_offset = o.walk_offset;
            R.walk_base_mixed = &(reinterpret_cast<MixedProblem *>(b->dev) + i)->walk_base;
            R.walk_base_sphere = b->sph_index[i] >= 0
                                     ? &(reinterpret_cast<SphereProblem *>((char *)b->dev + b->off_sph) +
                                         b->sph_index[i])->P.walk_base
                                     : nullptr;
            ox += p.domain->d;
        }
        PathRec *recs_dev = (PathRec *)(scr + off_r);
        if (cudaMemcpyAsync(recs_dev, recs.data(), sizeof(PathRec) * n_paths, cudaMemcpyHostToDevice, s) !=
                cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess) {
            st = fail(WOS_ERR_CUDA, "path setup failed");
            break;
        }
        CaptureSide cs;
        st = cs.init(b->sph.size());
        if (st != WOS_OK) break;
        if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess ||
            cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
            st = fail(WOS_ERR_CUDA, "graph capture failed to start");
            break;
        }
        const unsigned g = (unsigned)std::min(n_paths, 4096);
        for (int64_t i = 0; i < n_steps && st == WOS_OK; ++i) {
            paths_pre_kernel<<<g, 32, 0, cap>>>(recs_dev, n_paths, i);
            if (cudaGetLastError() != cudaSuccess) st = fail(WOS_ERR_CUDA, "pre kernel capture failed");
            if (st == WOS_OK) st = enqueue_batch_core(b, cap, cs);
            if (st == WOS_OK) {
                paths_post_kernel<<<g, 32, 0, cap>>>(recs_dev, n_paths, i);
                if (cudaGetLastError() != cudaSuccess) st = fail(WOS_ERR_CUDA, "post kernel capture failed");
            }
        }
        cudaError_t e = cudaStreamEndCapture(cap, &graph);
        if (st != WOS_OK) break;
        if (e != cudaSuccess) {
            st = fail(WOS_ERR_CUDA, "graph capture failed: %s", cudaGetErrorString(e));
            break;
        }
        e = cudaGraphInstantiate(&exec, graph, 0);
        if (e == cudaSuccess) e = cudaGraphLaunch(exec, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        int timed_out = 0;
        if (e == cudaSuccess) e = cudaMemcpy(&timed_out, ints + 2 * n_paths, sizeof(int), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) st = fail(WOS_ERR_CUDA, "paths graph failed: %s", cudaGetErrorString(e));
        else if (timed_out) st = fail(WOS_ERR_TIMEOUT, "a tensor-core walker wait ran out of its budget");
    } while (0);
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (cap) cudaStreamDestroy(cap);
    cudaStreamSynchronize(s);
    free_batch_device(b);
    delete b;
    cudaFree(scr);
    return st;
}

}  // extern "C"

// =====================================================================================
// allocation-free estimate: scratch in a static device array
// =====================================================================================
namespace {

// Per-query FP64 (or FP32) sums and int64 counters of wos_solve_noalloc. Every GPU that loads
// the library holds this array until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[WOS_NOALLOC_SCRATCH_BYTES];

// Device address of the array for the current device. Host code cannot use the symbol itself
// as a device address, so every call asks the runtime for it with the caller's device current:
// the lookup allocates nothing, and no address is cached across calls (a cached one would be
// stale after cudaDeviceReset or a new primary context).
wos_status noalloc_scratch(void **out) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr)
        return fail(WOS_ERR_CUDA, "cudaGetSymbolAddress(scratch) failed: %s", cudaGetErrorString(e));
    *out = p;
    return WOS_OK;
}

}  // namespace

extern "C" wos_status wos_solve_noalloc(wos_domain_t dom, const wos_options *opt, const double *x,
                                        int64_t Q, int64_t n_walks, double eps, double sigma,
                                        double *u, double *u_se, wos_stats *stats, void *stream) {
    WOS_TRY(check_common(dom, x, Q, n_walks, eps, sigma));
    if (Q > 0 && u == nullptr) return fail(WOS_ERR_INVALID_ARG, "u is NULL");
    const Opts o = read_opts(opt);
    {
        Opts oc = o;
        oc.cv = 0;  // value walks
        WOS_TRY(check_opts(oc, n_walks));
    }
    if (o.precision != WOS_FP64 && o.precision != WOS_FP32_PLAIN)
        return fail(WOS_ERR_UNSUPPORTED,
                    "wos_solve_noalloc runs WOS_FP64 or WOS_FP32_PLAIN (mixed precision allocates tables)");
    const int nf = acc_fields(dom->d, dom->n_exp);
    const size_t need = scratch_bytes(o.precision, Q, nf);
    if (need > (size_t)WOS_NOALLOC_SCRATCH_BYTES)
        return fail(WOS_ERR_INVALID_ARG,
                    "Q = %lld needs %zu bytes of scratch; the static array holds %u (at most %lld queries)",
                    (long long)Q, need, (unsigned)WOS_NOALLOC_SCRATCH_BYTES,
                    (long long)(((size_t)WOS_NOALLOC_SCRATCH_BYTES - 768) /
                                ((o.precision == WOS_FP32_PLAIN ? 4 : 8) * (size_t)nf + 8 * kCounters)));
    cudaStream_t s = (cudaStream_t)stream;
    void *base = nullptr;
    WOS_TRY(noalloc_scratch(&base));
    if (stats != nullptr) WOS_CUDA(cudaMemsetAsync(stats, 0, sizeof(wos_stats), s));
    if (Q == 0) return WOS_OK;
    WOS_CUDA(cudaMemsetAsync(base, 0, need, s));  // the array keeps the previous call's sums
    const Scratch sc = carve_scratch(base, o.precision, Q, nf);
    WOS_TRY(launch_walkers(dom, o, x, Q, n_walks, eps, sigma, 0, sc, PerWalk{}, nullptr, s));
    FinalizeArgs a{};
    a.recs = nullptr;
    a.n = 1;
    a.total_q = Q;
    a.stats = stats;
    FinalizeRec &r = a.single;
    r.d = dom->d;
    r.K = dom->n_exp;
    r.acc_f32 = o.precision == WOS_FP32_PLAIN;
    r.anti = o.antithetic;
    r.Q = Q;
    r.N = n_walks;
    r.q_begin = 0;
    r.acc = sc.acc;
    r.counts = sc.counts;
    r.u = u;
    r.u_se = u_se;
    return launch_finalize(a, s);
}

// =====================================================================================
// point-cloud distance diagnostics
// =====================================================================================
extern "C" wos_status wos_debug_pointcloud_radius(wos_domain_t dom, const double *x, int64_t Q,
                                                  double *radius, void *stream) {
    WOS_TRY(check_common(dom, x, Q, 1, 1e-30, 0.0));
    if (Q > 0 && radius == nullptr) return fail(WOS_ERR_INVALID_ARG, "radius is NULL");
    if (!dom->has_pcd) return fail(WOS_ERR_UNSUPPORTED, "the domain has no tensor-core sphere set");
    if (Q == 0) return WOS_OK;
    cudaStream_t s = (cudaStream_t)stream;
    WeightTable tab;
    WOS_TRY(ensure_table(dom, 0.0, &tab, s, false));
    const int nf = acc_fields(dom->d, dom->n_exp);
    const size_t bytes = scratch_bytes(WOS_MIXED, Q, nf);
    void *base = nullptr;
    WOS_CUDA(cudaMallocAsync(&base, bytes, s));
    const Scratch sc = carve_scratch(base, WOS_MIXED, Q, nf);
    wos_status st = WOS_OK;
    if (cudaMemsetAsync(base, 0, bytes, s) != cudaSuccess) st = fail(WOS_ERR_CUDA, "memset");
    if (st == WOS_OK) {
        // one distance evaluation per query: a walk capped at zero jumps
        MixedProblem P = make_mixed_problem(dom, x, Q, 1, 1e-30, 0.0, 0, 0, 0, 0, tab, (double *)sc.acc, sc.counts,
                                            PerWalk{}, nullptr);
        const cudaError_t e = launch_pointcloud(dom->pcd, P, dom->pc_delta, sc.cursor,
                                                reinterpret_cast<int *>(sc.cursor + 2), sc.cursor + 1, 0, 0, 0, 0,
                                                s, radius);
        if (e != cudaSuccess) st = fail(WOS_ERR_CUDA, "point-cloud probe failed: %s", cudaGetErrorString(e));
    }
    cudaFreeAsync(base, s);
    return st;
}
