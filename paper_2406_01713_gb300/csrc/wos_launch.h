// Internal launch interface between the host API (wos_api.cu) and the kernel translation
// units. Not part of the public C ABI.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "wos_device.cuh"

namespace wos {

// One-thread-per-walk walkers (FP64 parity mode and the plain FP32 baseline).
template <typename T>
struct SimpleParams {
    DomainView<T> dom;
    const double *x;  // Q x d queries (device)
    int64_t Q, N;
    uint64_t seed;
    int64_t walk_offset;
    int64_t max_steps;
    T eps, sqrt_sigma, shrink;
    int grad_mode, laplace;
    int cv;                      // gradient control variate: accumulate the 3d extra sums
    int src;                     // impulse source in gradient walks: store its per-query fields
    int antithetic;              // walk pairs (2m, 2m+1) with opposite first directions
    double roulette_w;           // > 0: Russian roulette on weights below it
    T *acc;                      // Q x nf sums
    unsigned long long *counts;  // Q x kCounters
    int nf;
    double *w_term;    // per-walk outputs (nullable)
    int64_t *w_jumps;
    double *w_grad;
    double *w_dsigma;
    const int *skip;   // nullable; the kernel does nothing if *skip != 0
};

cudaError_t launch_walk_simple_f64(const SimpleParams<double> &p, cudaStream_t s);
cudaError_t launch_walk_simple_f32(const SimpleParams<float> &p, cudaStream_t s);

// Problem record of the persistent mixed-precision walker.
struct MixedProblem {
    int d, n_balls, n_exp, has_box, has_outer, has_goal;
    int grad_mode, laplace;
    int cv;        // gradient control variate: accumulate the 3d extra sums
    int src;       // impulse source in gradient walks: store its per-query fields
    int has_source;
    int proj;      // components measured in coordinates 0..proj-1 (= d unless extruded)
    int n_links, n_arm_obs;  // planar arm (geom holds the link lengths and obstacle points)
    float arm_inv_K;         // 1 / Lipschitz constant of its kinematics
    int antithetic;        // walk pairs (2m, 2m+1) with opposite first directions
    float roulette_w;      // > 0: Russian roulette on weights below it
    float log_roulette_w;  // its logarithm (the walkers keep log weights)
    float source_q;
    float src_lc0;        // log(k^nu / (2 pi)^(d/2)), k = sqrt(sigma) > 0
    float src_inv_omega;  // 1 / |S^(d-1)| (sigma = 0)
    float source_z[kMaxD];
    float eps, sqrt_sigma;
    float shrink;  // FP32 error bound subtracted from every radius
    float slack;   // FP32 rounding bound of the ball screening test
    float goal_r, outer_r;
    int64_t Q, N;
    int64_t walk_base;            // global walk index of walk 0 of query 0
    const float *balls;           // packed ball records (see walk_mixed.cu)
    const float *geom;            // geom_count(d) floats, see geom_count
    const double *x;              // Q x d queries
    WeightTable table;
    double *acc;                  // Q x nf FP64 sums (the walkers store only the per-query G and
                                  // source fields; reduce_kernel writes the sums)
    unsigned long long *counts;   // Q x kCounters
    float *rec;                   // Q N x rec_words per-walk records (nullable: none written)
    int rec_words;
    const int *done;              // nullable; nonzero: the problem runs no walks (a finished path)
    double *w_term;               // per-walk outputs (nullable)
    int64_t *w_jumps;
    double *w_grad;
    double *w_dsigma;
};

struct MixedItem {
    int problem;
    int pad;
    int64_t j0, j1;  // walk range within the problem, j = q * N + w
};

struct MixedLaunch {
    const MixedProblem *problems;  // device array, or nullptr: problem 0 is `single`
    const MixedItem *items;        // device array, or nullptr: implicit items of problem 0
    int64_t n_items;
    int64_t walks_per_item;        // implicit items: item i = walks [i wpi, min((i+1) wpi, total))
    int64_t total_walks;
    unsigned long long *cursor;    // work-queue cursor (device, zero before the launch)
    uint64_t seed;
    int64_t max_steps;
    const int *skip;               // nullable; the kernel does nothing if *skip != 0
    MixedProblem single;
};

// Per-walk record of the mixed-precision walkers, the input of the per-query reduction
// (reduce_kernel): rec_words floats at walk index j = q N + w,
//   [term, dv, gt, info, v0 (d floats, gradient walks), e (K floats)]
// term: the walk's value estimate; dv: d term / d sigma (the boundary part times the summed
// d log C / d sigma, plus the derivatives of the source contributions); gt: alpha(R0) u^(x1),
// the factor of v0 in its gradient estimate (0 unless the walk reached the boundary after its
// first sphere); info: k (jumps) | outcome << 28 (0 jumped, 1 boundary, 2 capped, 3 outside) |
// has_v0 << 31; v0: the first direction (written when has_v0); e_k = exp(a_k . xbar) W (written
// when term != 0). Outcome 4: ended by the Russian roulette. A record is 16-byte aligned.
__host__ __device__ constexpr int rec_words(int d, int K, int grad) { return (4 + (grad ? d : 0) + K + 3) & ~3; }
constexpr unsigned kRecKMask = 0x0fffffffu;  // jumps per walk stay below 2^28
constexpr int kRecOutcomeShift = 28;
constexpr unsigned kRecOutcomeMask = 7u;
constexpr unsigned kRecHasV0 = 0x80000000u;

// Domain geometry of the mixed walkers in shared memory: box lo [d], box hi [d], goal c [d],
// outer c [d], exp w [kMaxExp], exp a [kMaxExp x d], arm link lengths [d], arm obstacle points
// [kMaxArmObs x 2].
__host__ __device__ constexpr int geom_count(int d) { return 4 * d + kMaxExp + kMaxExp * d + d + 2 * kMaxArmObs; }
__host__ __device__ constexpr int geom_link(int d) { return 4 * d + kMaxExp + kMaxExp * d; }
__host__ __device__ constexpr int geom_arm_obs(int d) { return 5 * d + kMaxExp + kMaxExp * d; }

// Floats per packed ball record for dimension d.
__host__ __device__ constexpr int ball_record_floats(int d) { return d + 2; }

cudaError_t configure_walk_mixed_val512(size_t smem_bytes);
int max_active_walk_mixed_val512(int threads, size_t smem_bytes);
cudaError_t launch_walk_mixed_val512(const MixedLaunch &L, int grid, int threads, size_t smem_bytes, cudaStream_t s);
cudaError_t configure_walk_mixed_val768(size_t smem_bytes);
int max_active_walk_mixed_val768(int threads, size_t smem_bytes);
cudaError_t launch_walk_mixed_val768(const MixedLaunch &L, int grid, int threads, size_t smem_bytes, cudaStream_t s);
cudaError_t configure_walk_mixed_grad512(size_t smem_bytes);
int max_active_walk_mixed_grad512(int threads, size_t smem_bytes);
cudaError_t launch_walk_mixed_grad512(const MixedLaunch &L, int grid, int threads, size_t smem_bytes, cudaStream_t s);
cudaError_t configure_walk_mixed_grad768(size_t smem_bytes);
int max_active_walk_mixed_grad768(int threads, size_t smem_bytes);
cudaError_t launch_walk_mixed_grad768(const MixedLaunch &L, int grid, int threads, size_t smem_bytes, cudaStream_t s);

// The persistent walker instantiations: value or gradient walks, CTAs of up to 512 or 768
// threads (the 768 variant trades registers for resident warps).
inline cudaError_t launch_walk_mixed(const MixedLaunch &L, int grad_any, int grid, int threads,
                                     size_t smem_bytes, cudaStream_t s) {
    if (threads <= 512)
        return grad_any ? launch_walk_mixed_grad512(L, grid, threads, smem_bytes, s)
                        : launch_walk_mixed_val512(L, grid, threads, smem_bytes, s);
    return grad_any ? launch_walk_mixed_grad768(L, grid, threads, smem_bytes, s)
                    : launch_walk_mixed_val768(L, grid, threads, smem_bytes, s);
}
inline cudaError_t configure_walk_mixed(size_t smem_bytes) {
    cudaError_t e = configure_walk_mixed_val512(smem_bytes);
    if (e == cudaSuccess) e = configure_walk_mixed_val768(smem_bytes);
    if (e == cudaSuccess) e = configure_walk_mixed_grad512(smem_bytes);
    if (e == cudaSuccess) e = configure_walk_mixed_grad768(smem_bytes);
    return e;
}
inline int max_active_mixed(int threads, size_t smem_bytes, int grad_any) {
    if (threads <= 512)
        return grad_any ? max_active_walk_mixed_grad512(threads, smem_bytes)
                        : max_active_walk_mixed_val512(threads, smem_bytes);
    return grad_any ? max_active_walk_mixed_grad768(threads, smem_bytes)
                    : max_active_walk_mixed_val768(threads, smem_bytes);
}

// Sphere set for the tensor-core walker (pointcloud.cu): points (radius 0) or balls, as
// BF16-split centre tiles in the MMA's core-matrix layout and FP32 records of 16 spheres for the
// exact pass. Balls are sorted by radius so that each record spans a narrow radius range;
// chunk_rhi bounds the radii of a record from above.
struct PointCloudDev {
    void *tiles = nullptr;      // n_tiles x 64 centres, BF16, already in the shared-memory layout
    float *soa = nullptr;       // per 16-sphere record: centres by coordinate quads, then 16 radii
    float *chunk_rhi = nullptr; // largest radius of each 16-sphere record (rounded up)
    int n_tiles = 0;
    int spheres = 0;            // 1: balls with radii; 0: points
    double pmax = 0.0;  // largest |coordinate| of a centre
};
// radii: NULL for a point set, else M ball radii (the set is reordered by radius).
cudaError_t pointcloud_prepare(const double *pts, const double *radii, int64_t M, int d, PointCloudDev *out);
void pointcloud_release(PointCloudDev *pcd);
float pointcloud_delta(int d, double xabs, double pmax);

// One problem of the tensor-core walker.
struct SphereProblem {
    MixedProblem P;
    const void *tiles;
    const float *soa;
    const float *chunk_rhi;
    int n_tiles;
    float delta;  // bound of |D~ - D| of the BF16 contraction (squared-distance units)
};
struct SphereItem {
    int problem;
    int pad;
    int64_t j0, j1;  // walk range within the problem
};
// A persistent launch over items (problem, walk range) of problems that share the dimension.
struct SphereLaunch {
    const SphereProblem *problems;    // device array, or nullptr: problem 0 is `single`
    const SphereItem *items;          // device array, or nullptr: implicit items of `single`
    int64_t n_items;
    int64_t walks_per_item;           // implicit items: item i = walks [i wpi, min((i+1) wpi, Q N))
    unsigned long long *item_cursor;  // zero before the launch
    int *status;                      // nonzero: a wait timed out (1: main loop, 2: teardown)
    unsigned long long *shrinks;      // steps whose radius came from a chunk bound
    long long wait_budget;            // clock cycles one main-loop wait may take
    uint32_t wait_hint;               // suspend-time hint of its tests (ns), wait_hint_ns(budget)
    uint64_t seed;
    int64_t max_steps;
    double *radius_out;  // nullable: distance bound at each walk's start (single problem only)
    SphereProblem single;
};
// src: a problem of the launch has an impulse source (selects the kernel variant with the source
// term); wide: 32-column candidate chunks instead of 16 (sphere_wide of every set of the launch;
// d <= kSphereWideMaxD)
cudaError_t launch_spheres(const SphereLaunch &L, int d, int grad, int src, int wide, int grid, cudaStream_t s);
int sphere_ctas_per_sm();
// Single problem: implicit items, grid sized to the work.
cudaError_t launch_pointcloud(const PointCloudDev &pcd, const MixedProblem &P, float delta,
                              unsigned long long *cursor, int *status, unsigned long long *shrinks,
                              uint64_t seed, int64_t max_steps, long long wait_budget, int grad,
                              cudaStream_t s, double *radius_out = nullptr);
constexpr long long kDefaultWaitBudget = 4000000000ll;  // clock cycles (~2 s at 2 GHz)
// Suspend-time hint of a wait's tests: at most 20 us, and about the budget for small budgets (a
// budget in cycles read as ns at ~2 GHz), so that one test does not outlast a small budget.
inline uint32_t wait_hint_ns(long long budget) {
    return budget >= 40000ll ? 20000u : (budget >= 64ll ? (uint32_t)(budget / 2) : 32u);
}
constexpr int kPointCloudMaxD = 12;  // 3d + 2 BF16 columns fit a 32- or 48-wide contraction
// Ball sets at least this large run on the tensor cores: the measured crossover of the two
// walkers (u and grad u with the control variate, 64 queries x 16384 walks per ball set; CUDA-core
// time over tensor-core time 1.13-1.31 at 96 balls for d <= 4, 1.05-1.15 at 160 balls for d = 5..9,
// 1.04-1.13 at 128 balls for d = 10..12).
constexpr int sphere_min_balls(int d) { return d <= 4 ? 96 : (d <= 9 ? 160 : 128); }
// Sets of at least kSphereWideTiles 64-centre tiles in d <= kSphereWideMaxD take 32-column
// candidate chunks: the per-tile bound work then outweighs the exact pass, which 16-column chunks
// halve. The width is a property of the domain, so that a problem takes the same walks alone and
// in a batch. Measured (u and grad u): 65536 points in d = 7, 17 % faster; 64 tiles in d = 8,
// 10 % faster alone at full occupancy but 4 % slower in the batched step, whose launches of
// large sets run few CTAs; 24-64 tiles in d = 12, 4-10 % slower.
constexpr int kSphereWideTiles = 128;
constexpr int kSphereWideMaxD = 8;
constexpr int sphere_wide(int d, int n_tiles) { return d <= kSphereWideMaxD && n_tiles >= kSphereWideTiles ? 1 : 0; }
// Batched sphere-set queues, per dimension: sets below kSphereLargeTiles tiles, larger 16-column
// sets, 32-column sets (each queue one launch; measured 640.5 vs 645.5 ms per batched step against
// one queue per dimension).
constexpr int kSphereLargeTiles = 24;
constexpr int kSphereQueueClasses = 3;
constexpr int sphere_queue_class(int d, int n_tiles) {
    return sphere_wide(d, n_tiles) ? 2 : (n_tiles >= kSphereLargeTiles ? 1 : 0);
}

}  // namespace wos
