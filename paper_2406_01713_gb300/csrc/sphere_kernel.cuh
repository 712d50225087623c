// Sphere-set Walk-on-Spheres walker on the 5th-generation tensor cores (sm_103a).
//
// Distance to a set of obstacle spheres: points (Sec. VII-A, d(q) = min_i |q - p_i|) or balls
// (Sec. VI, |q - c_i| - r_i), for 128 walkers at a time. The contraction
// D_wi = |c_i|^2 - 2 x_w . c_i runs as tcgen05.mma (BF16 inputs, FP32 accumulation in tensor
// memory) over centre tiles that bulk copies (cp.async.bulk) stream into shared memory; the
// walker warps take the minimum of each 16 columns of their rows with the reducing form of the
// tensor-memory load (tcgen05.ld.red .min). Per chunk of CH columns (16, or 32 for large sets, a
// template parameter), min D gives a lower bound of the chunk's distances,
// sqrt(min D + |x|^2 - delta) - r_hi (balls are sorted by radius, so r_hi, the chunk's largest
// radius, is close to every radius in it); each walker keeps the best, second and third chunk
// bounds. The best chunk is then recomputed exactly in FP32 (the second too when its bound is
// below that result), and every other sphere is bounded from below by the next chunk's bound, so
// the radius never exceeds the true distance (no sphere leaves the domain). Narrow chunks make
// the exact pass cheap; wide ones halve the per-tile bound work, which dominates on large sets.
//
// BF16 split: x = x_h + x_l and -2p = q_h + q_l (each a BF16), |p|^2 = n_h + n_l; the walker
// row [x_h, x_h, x_l, 1, 1] times the point row [q_h, q_l, q_h, n_h, n_l] gives
// |p|^2 - 2 x.p up to the dropped x_l q_l term and FP32 accumulation (3d + 2 columns, padded
// to K = 32 for d <= 10 and K = 48 for d = 11, 12).
//
// CTA: warps 0-3 own one walker per thread (TMEM lanes 0..127); warp 4, lane 0, issues the
// bulk copies of the centre tiles and the MMAs. The launch is persistent over a queue of items
// (problem, walk range) of problems with the same dimension: the walkers of a CTA draw walks
// from their item, take the next item when it runs out (continuing seamlessly if it belongs to
// the same problem), and switch problems once their last walks have ended. Every wait on an
// mbarrier is bounded by a clock budget; a timeout sets the launch's status word and every
// thread leaves through the same teardown, which waits for the issued MMAs and frees the
// tensor memory.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "walk_mixed.cuh"

namespace wos {
namespace pc {

constexpr int kRows = 128;       // walkers per CTA = MMA M = TMEM lanes
constexpr int kTileN = 64;       // centres per tile = MMA N
constexpr int kMaxStages = 6;
constexpr int kPairTiles = 2;  // centre tiles per bulk copy (consecutive in memory and in the ring)
constexpr int kCtasPerSm = 4;    // 4 x 128 TMEM columns; registers <= 102 per thread
constexpr int kChunk = 16;       // spheres per chunk record in memory (a candidate chunk is 1 or 2 records)
constexpr int kRefineGroup = 4;  // warp-wide chunk loads a lane keeps in flight together in the exact pass
// A chunk record in memory: its kChunk centres padded with zeros to a multiple of four
// coordinates and stored by coordinate quads (quad q: coordinates 4q..4q+3 of sphere 0, of
// sphere 1, ...), so that one 16-byte load per lane reads a quad of all 16 spheres in 256
// contiguous bytes (two records per warp-wide load); then its kChunk radii.
__host__ __device__ constexpr int chunk_pitch(int d) { return (d + 3) & ~3; }
__host__ __device__ constexpr int chunk_floats(int d) { return kChunk * (chunk_pitch(d) + 1); }
constexpr int kWalkerThreads = 128;
constexpr int kThreads = kWalkerThreads + 32;
constexpr uint32_t kTmemCols = 2 * kTileN;
// dynamic shared memory alignment: the operands use no swizzle, whose descriptors and bulk copies
// need 16-byte addresses
constexpr int kSmemAlign = 128;

// Contraction length: 3d + 2 BF16 columns padded to 32 (d <= 10) or 48 (d = 11, 12); the
// centre-tile ring is shorter for the wider tiles so that four CTAs still fit an SM.
__host__ __device__ constexpr int contraction_k(int d) { return 3 * d + 2 <= 32 ? 32 : 48; }
template <int K>
struct Geo {
    static constexpr int kK = K;
    static constexpr uint32_t kTileBytes = kTileN * K * 2;
    static constexpr uint32_t kABytes = kRows * K * 2;
    static constexpr uint32_t kSBO = (K / 8) * 128;  // to the next group of 8 rows
    static constexpr int kStages = K == 32 ? 6 : 4;  // centre-tile ring in shared memory (tiles)
    // the ring is filled kPairTiles tiles per bulk copy: kSlots slots, each with its own full
    // barrier (a slot is reused only after the MMAs that read it have completed, which the
    // accumulator waits already establish)
    static constexpr int kSlots = kStages / kPairTiles;
    static constexpr uint32_t kSlotBytes = kPairTiles * kTileBytes;
};
constexpr int kTrPitch = 34;  // transpose row: up to 32 spheres + 2 pad (8-byte aligned rows, no bank conflicts)
constexpr uint32_t kTransposeBytes = 4 * 32 * kTrPitch * 4;  // per walker warp: 32 walker rows
constexpr long long kDrainBudget = kDefaultWaitBudget;  // teardown waits, whatever the launch's budget

// Core-matrix layout (8 rows x 16 bytes), K-major, no swizzle: element (r, k) of a
// rows x K BF16 operand sits at byte (r/8) SBO + (k/8) LBO + (r%8) 16 + (k%8) 2, SBO = (K/8) 128.
constexpr uint32_t kLBO = 128;               // to the next core matrix along K

// tcgen05 instruction descriptor, kind::f16: D = F32 (bits 4-5), A = B = BF16 (7-9, 10-12),
// both K-major (15, 16 = 0), N >> 3 at bits 17-22, M >> 4 at bits 24-28.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kTileN >> 3) << 17) |
                            ((uint32_t)(kRows >> 4) << 24);

__device__ __forceinline__ uint32_t su32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t sbo) {
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((kLBO >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;  // descriptor version of tcgen05; base offset 0, no swizzle
    return d;
}

__device__ __forceinline__ void mbar_init(uint64_t *b, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *b) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(b)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *b, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(b)), "r"(bytes) : "memory");
}
// try_wait with a suspend-time hint (ns): a waiting thread is parked until the phase completes
// or the hint runs out, instead of spinning on the issue slots the MMA-issuing thread needs.
// hint_ns: the longest the thread may be suspended inside one test (suspend-time hint)
__device__ __forceinline__ bool mbar_test(uint64_t *b, uint32_t parity, uint32_t hint_ns = 20000u) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(su32(b)), "r"(parity), "r"(hint_ns)
        : "memory");
    return ok != 0;
}

struct Shared {
    uint64_t full[kMaxStages / kPairTiles];
    uint64_t tfull[2];
    uint64_t tempty[2];
    uint64_t a_ready;
    uint64_t drain;
    uint32_t tmem_base;
    volatile int abort_flag;
    volatile int stop;
    // work control: written by walker thread 0 between the two barriers of a step
    int cur, has_pend, queue_empty, skip, switched;
    unsigned long long j_next, j_end;  // walk range of the current item; j_next is the shared counter
    SphereItem pend;
};

// A slot of the centre-tile ring and the number of completed passes over the ring (whose
// parity is the phase a wait on that slot's barriers expects).
struct RingPos {
    int slot = 0;
    uint32_t round = 0;
    __device__ __forceinline__ void next(int n) {
        if (++slot == n) {
            slot = 0;
            ++round;
        }
    }
};

// Bounded wait of the main loop: false if the launch's budget ran out or another thread aborted.
// Bounded wait of the main loop (budget and suspend-time hint from the launch; the hint is
// scaled to the budget, so that a small budget is not outlasted by one test): false if the
// budget ran out or another thread aborted.
static __device__ __noinline__ bool wait_bar_slow(Shared &S, uint64_t *b, uint32_t parity, int *status, long long budget,
                                                  uint32_t hint) {
    const long long t0 = clock64();
    for (;;) {
        if (mbar_test(b, parity, hint)) return true;
        if (S.abort_flag) return false;
        if (clock64() - t0 > budget) {
            S.abort_flag = 1;
            atomicOr(status, 1);
            return false;
        }
    }
}
__device__ __forceinline__ bool wait_bar(Shared &S, uint64_t *b, uint32_t parity, const SphereLaunch &L) {
    if (mbar_test(b, parity, L.wait_hint)) return true;
    return wait_bar_slow(S, b, parity, L.status, L.wait_budget, L.wait_hint);
}

// Teardown wait for work already issued (products, copies): it does not stop at an abort, so
// that nothing is in flight when the tensor memory is freed and the CTA exits; bounded by the
// full budget.
__device__ __forceinline__ void drain_wait(uint64_t *b, uint32_t parity, int *status) {
    if (mbar_test(b, parity)) return;
    const long long t0 = clock64();
    while (!mbar_test(b, parity)) {
        if (clock64() - t0 > kDrainBudget) {
            atomicOr(status, 2);
            return;
        }
    }
}

// Warp-uniform bounded wait for the walker warps: every lane tests the phase once (a broadcast
// read, no divergence in the common case); if it is still open, lane 0 polls with the budget and
// every lane gets the result.
__device__ __forceinline__ bool warp_wait_bar(Shared &S, uint64_t *b, uint32_t parity, const SphereLaunch &L) {
    if (__any_sync(0xffffffffu, mbar_test(b, parity))) return true;
    int ok = 0;
    if ((threadIdx.x & 31) == 0) ok = wait_bar(S, b, parity, L) ? 1 : 0;
    return __shfl_sync(0xffffffffu, ok, 0) != 0;
}

// One centre tile (already in the core-matrix layout) by a bulk copy; both addresses are
// 16-byte aligned (tile sizes are multiples of 2 KB).
__device__ __forceinline__ void bulk_load_tile(uint32_t dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
        "l"((uint64_t)src), "r"(bytes), "r"(su32(bar))
        : "memory");
}

// Next item of the launch's queue; false when the queue is empty.
__device__ __forceinline__ bool next_item(const SphereLaunch &L, SphereItem &it) {
    const unsigned long long i = atomicAdd(L.item_cursor, 1ull);
    if (i >= (unsigned long long)L.n_items) return false;
    if (L.items != nullptr) {
        it = L.items[i];
        // a planner path that has reached its goal runs no walks
        const int *dn = L.problems != nullptr ? L.problems[it.problem].P.done : nullptr;
        if (dn != nullptr && *(volatile const int *)dn != 0) it.j1 = it.j0;
    } else {
        const int64_t total = L.single.P.Q * L.single.P.N;
        it.problem = 0;
        it.j0 = (int64_t)i * L.walks_per_item;
        it.j1 = it.j0 + L.walks_per_item < total ? it.j0 + L.walks_per_item : total;
        const int *dn = L.single.P.done;
        if (dn != nullptr && *(volatile const int *)dn != 0) it.j1 = it.j0;
    }
    return true;
}

// Copies problem p into shared memory (threads tid, tid + nt, ...).
__device__ __forceinline__ void load_problem(const SphereLaunch &L, int p, SphereProblem &SP, int tid, int nt) {
    const SphereProblem *src = L.problems != nullptr ? L.problems + p : &L.single;
    const int *s = reinterpret_cast<const int *>(src);
    int *d = reinterpret_cast<int *>(&SP);
    for (int i = tid; i < (int)(sizeof(SphereProblem) / 4); i += nt) d[i] = s[i];
}

__device__ __forceinline__ void walker_barrier() { asm volatile("barrier.cta.sync 2, 128;" ::: "memory"); }

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
            d_tmem),
        "l"(a), "l"(b), "r"(kIdesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(bar))
                 : "memory");
}

static_assert(kTileN == 64 && kChunk == 16, "the epilogue reads a 64-column tile as four 16-column minima");

// Minima of the two 16-column groups of 32 accumulator columns of this thread's TMEM lane, taken
// by the loads themselves (tcgen05.ld.red with .min, an sm_103a form: each load also returns the
// minimum of the columns it loads). The columns land in scratch registers declared inside the
// statement and are never read; both loads are waited for before it ends.
__device__ __forceinline__ void tmem_min16x2(uint32_t taddr, float &m0, float &m1) {
    asm volatile(
        "{\n .reg .f32 t<32>;\n"
        "tcgen05.ld.red.sync.aligned.32x32b.x16.min.f32 "
        "{t0,t1,t2,t3,t4,t5,t6,t7,t8,t9,t10,t11,t12,t13,t14,t15}, %0, [%2];\n"
        "tcgen05.ld.red.sync.aligned.32x32b.x16.min.f32 "
        "{t16,t17,t18,t19,t20,t21,t22,t23,t24,t25,t26,t27,t28,t29,t30,t31}, %1, [%3];\n"
        "tcgen05.wait::ld.sync.aligned;\n}\n"
        : "=f"(m0), "=f"(m1)
        : "r"(taddr), "r"(taddr + 16)
        : "memory");
}

// The same for two 32-column groups (the minima of 32-column chunks), one load at a time.
__device__ __forceinline__ void tmem_min32x2(uint32_t taddr, float &m0, float &m1) {
    asm volatile(
        "{\n .reg .f32 t<32>;\n"
        "tcgen05.ld.red.sync.aligned.32x32b.x32.min.f32 "
        "{t0,t1,t2,t3,t4,t5,t6,t7,t8,t9,t10,t11,t12,t13,t14,t15,"
        "t16,t17,t18,t19,t20,t21,t22,t23,t24,t25,t26,t27,t28,t29,t30,t31}, %0, [%1];\n"
        "tcgen05.wait::ld.sync.aligned;\n}\n"
        : "=f"(m0)
        : "r"(taddr)
        : "memory");
    asm volatile(
        "{\n .reg .f32 t<32>;\n"
        "tcgen05.ld.red.sync.aligned.32x32b.x32.min.f32 "
        "{t0,t1,t2,t3,t4,t5,t6,t7,t8,t9,t10,t11,t12,t13,t14,t15,"
        "t16,t17,t18,t19,t20,t21,t22,t23,t24,t25,t26,t27,t28,t29,t30,t31}, %0, [%1];\n"
        "tcgen05.wait::ld.sync.aligned;\n}\n"
        : "=f"(m1)
        : "r"(taddr + 32)
        : "memory");
}

// Lower bounds of sqrt(max(s, 0)) from the hardware approximation, whose excess over the exact
// root was measured below 2^-23.6 on every float in [2^-40, 2^40): scaled down by 2^-16 (chunk
// bounds) or 2^-22 (refined distances, which stay within an FP32 rounding of the exact value).
__device__ __forceinline__ float sqrt_approx(float s) {
    float r;
    asm("sqrt.approx.f32 %0, %1;" : "=f"(r) : "f"(fmaxf(s, 0.f)));
    return r;
}
__device__ __forceinline__ float sqrt_below(float s) { return sqrt_approx(s) * 0.9999847412109375f; }
__device__ __forceinline__ float sqrt_below_tight(float s) { return sqrt_approx(s) * 0.999999761581420898f; }

// Writes this walker's A row (BF16 split of x; zeros for an idle lane).
template <int D>
__device__ __forceinline__ void write_row(unsigned char *A, int r, const float (&x)[D], bool active) {
    constexpr int kK = contraction_k(D);
    constexpr uint32_t kSBO = Geo<kK>::kSBO;
    __nv_bfloat16 row[kK];
#pragma unroll
    for (int k = 0; k < kK; ++k) row[k] = __float2bfloat16_rn(0.f);
    if (active) {
#pragma unroll
        for (int j = 0; j < D; ++j) {
            const __nv_bfloat16 h = __float2bfloat16_rn(x[j]);
            const __nv_bfloat16 l = __float2bfloat16_rn(x[j] - __bfloat162float(h));
            row[j] = h;
            row[D + j] = h;
            row[2 * D + j] = l;
        }
        row[3 * D] = __float2bfloat16_rn(1.f);
        row[3 * D + 1] = __float2bfloat16_rn(1.f);
    }
#pragma unroll
    for (int kc = 0; kc < kK / 8; ++kc) {
        const uint32_t off = (r / 8) * kSBO + kc * kLBO + (r % 8) * 16;
        *reinterpret_cast<uint4 *>(A + off) = *reinterpret_cast<const uint4 *>(row + 8 * kc);
    }
}

// Impulse source (Sec. IV-A source term) in the ball B(x_k, R) of a walker at distance r from
// the source: returns q G_B(x_k, z) times the weight so far; at step 0 of a gradient walk it also
// stores the query's step-0 value and the source part of its gradient, q grad_x G_B(x_0, z)
// (x_0 is the query point; every walk of the query writes the same). Not inlined, scalar
// arguments: walkers without a source keep their registers, and the position never needs local
// memory.
template <int D>
__device__ __noinline__ float sphere_source(const MixedProblem &P, long long q, int k, float r, float R, float2 tR,
                                            float logw, float dsig, float &dc) {
    float G, F, dG;
    source_green_f32<D>(P, r, R, tR, G, F, dG);
    const float qw = P.source_q * expf(logw);
    const float c = qw * G;
    dc = qw * fmaf(dsig, G, dG);  // d c / d sigma: the weight's and G_B's
    if (k == 0 && P.src) {
        double *sp = P.acc + q * acc_fields(D, P.n_exp, P.cv, 1) + src_field(D, P.n_exp, P.cv);
        sp[0] = (double)c;
        for (int i = 0; i < D; ++i) {
            const float x0 = (float)P.x[q * D + i];
            sp[1 + i] = (double)(P.source_q * F * (P.source_z[i] - x0) / r);
        }
    }
    return c;
}

// SRC: the launch holds a problem with an impulse source (the variant without keeps the walkers'
// registers free of the source state). CH: candidate chunk width in columns, 16 or 32.
template <int D, bool GRAD, bool SRC, int CH>
__global__ void __launch_bounds__(kThreads, kCtasPerSm) sphere_kernel(const __grid_constant__ SphereLaunch L) {
    static_assert(CH == kChunk || CH == 2 * kChunk, "a candidate chunk is one or two records");
    constexpr int kChunksPerTile = kTileN / CH;
    constexpr int kRecs = CH / kChunk;  // records per candidate chunk
    using G = Geo<contraction_k(D)>;
    constexpr int kK = G::kK;
    constexpr uint32_t kTileBytes = G::kTileBytes, kABytes = G::kABytes, kSBO = G::kSBO;
    constexpr int kStages = G::kStages, kSlots = G::kSlots;
    constexpr uint32_t kSlotBytes = G::kSlotBytes;
    extern __shared__ __align__(kSmemAlign) unsigned char smem_raw[];
    __shared__ Shared S;
    __shared__ SphereProblem SP;  // the problem the CTA's walkers are on
    __shared__ float geom_s[4 * kMaxD + kMaxExp + kMaxExp * kMaxD];
    unsigned char *base =
        reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + kSmemAlign - 1) & ~(uintptr_t)(kSmemAlign - 1));
    unsigned char *A = base;
    unsigned char *Bst = base + kABytes;
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const MixedProblem &P = SP.P;
    constexpr int kGeom = 4 * D + kMaxExp + kMaxExp * D;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kSlots; ++s) {
            mbar_init(&S.full[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&S.tfull[b], 1);
            mbar_init(&S.tempty[b], 4);
        }
        mbar_init(&S.a_ready, 4);
        mbar_init(&S.drain, 1);
        S.abort_flag = 0;
        S.stop = 0;
        S.has_pend = 0;
        S.queue_empty = 0;
        S.skip = 0;
        S.switched = 0;
        SphereItem it;
        if (next_item(L, it)) {
            S.cur = it.problem;
            S.j_next = (unsigned long long)it.j0;
            S.j_end = (unsigned long long)it.j1;
        } else {
            S.cur = 0;
            S.j_next = S.j_end = 0ull;
            S.queue_empty = 1;
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    load_problem(L, S.cur, SP, threadIdx.x, blockDim.x);
    __syncthreads();
    for (int i = threadIdx.x; i < kGeom; i += blockDim.x) geom_s[i] = SP.P.geom[i];
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&S.tmem_base)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = S.tmem_base;

    if (warp == 4) {
        // ------------------------------------------------------------------ producer
        if (lane == 0) {
            long long g_mma = 0;  // tiles multiplied so far (their parity picks the accumulator buffer)
            // the operand descriptors, built once: a descriptor of (addr + off) is the descriptor of
            // addr plus off / 16 while the address stays below 256 KB (its 14-bit field)
            const uint64_t a_desc = smem_desc(su32(A), kSBO);
            const uint64_t b_desc0 = smem_desc(su32(Bst), kSBO);
            constexpr uint64_t kKStep = (2 * kLBO) >> 4, kStageStep = kTileBytes >> 4;
            RingPos lp, mp;  // ring slots of the next copy and of the next MMA's tile pair
            long long g_load = 0, g_pair = 0;  // tile pairs copied and consumed so far
            bool ok = true;
            for (int step = 0; ok; ++step) {
                if (!wait_bar(S, &S.a_ready, step & 1, L)) break;
                if (S.stop) break;
                // the problem of this step (the walkers change it only between steps)
                const int T = SP.n_tiles;
                const int n_pairs = (T + kPairTiles - 1) / kPairTiles;
                const unsigned char *tiles = reinterpret_cast<const unsigned char *>(SP.tiles);
                int p_load = 0;
                // copies pair p_load into the next slot, kSlots - 1 pairs ahead of the MMAs. The
                // MMAs that read the slot last (those of the pair before the one just released)
                // have completed: at a step start every walker has read the previous step's
                // accumulators; within a step the released pair had two tiles, and the wait on
                // the accumulator buffer of its second tile means the walkers have read the tile
                // two before it, the previous pair's last (an MMA completes before its
                // accumulators are signalled, and the MMAs of one thread complete in order)
                auto issue_load = [&]() -> bool {
                    const int s = lp.slot;
                    const int nt = T - kPairTiles * p_load < kPairTiles ? T - kPairTiles * p_load : kPairTiles;
                    mbar_expect_tx(&S.full[s], nt * kTileBytes);
                    bulk_load_tile(su32(Bst) + s * kSlotBytes, tiles + (size_t)p_load * kSlotBytes, nt * kTileBytes,
                                   &S.full[s]);
                    lp.next(kSlots);
                    ++g_load;
                    ++p_load;
                    return true;
                };
                while (ok && p_load < n_pairs && g_load < g_pair + kSlots - 1) ok = issue_load();
                for (int t = 0; ok && t < T; ++t) {
                    const int s = mp.slot, half = t % kPairTiles;
                    const int b = (int)(g_mma & 1);
                    if (half == 0 && !wait_bar(S, &S.full[s], mp.round & 1u, L)) { ok = false; break; }
                    if (g_mma >= 2 && !wait_bar(S, &S.tempty[b], (uint32_t)(((g_mma >> 1) - 1) & 1), L)) {
                        ok = false;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint64_t b_desc = b_desc0 + (uint64_t)(s * kPairTiles + half) * kStageStep;
#pragma unroll
                    for (int kk = 0; kk < kK / 16; ++kk)
                        mma_bf16(tmem + b * kTileN, a_desc + kk * kKStep, b_desc + kk * kKStep, kk > 0);
                    mma_commit(&S.tfull[b]);
                    ++g_mma;
                    if (half == kPairTiles - 1 || t == T - 1) {  // the pair's last tile: move on
                        mp.next(kSlots);
                        ++g_pair;
                        while (ok && p_load < n_pairs && g_load < g_pair + kSlots - 1) ok = issue_load();
                    }
                }
            }
            // drain: every issued MMA completes before the tensor memory is freed; every issued
            // copy was consumed by an MMA, except after an abort
            mma_commit(&S.drain);
            drain_wait(&S.drain, 0, L.status);
            for (long long g = g_pair; g < g_load; ++g) {
                drain_wait(&S.full[mp.slot], mp.round & 1u, L.status);
                mp.next(kSlots);
            }
        }
        __syncwarp();
    } else {
        // ------------------------------------------------------------------ walkers
        const int r = threadIdx.x;  // TMEM lane / A row
        const uint32_t trow = tmem + ((uint32_t)(32 * warp) << 16);
        const float inv2d = 1.0f / (2.0f * (float)D);
        float x[D];
#pragma unroll
        for (int i = 0; i < D; ++i) x[i] = 0.f;
        float logw = 0.f, dsig = 0.f, gfac0 = 0.f;
        float src = 0.f, src0 = 0.f;  // impulse source: contributions so far, and the step-0 one
        float dsrc = 0.f;             // and their d / d sigma
        int k = 0;
        long long j = -1, q = 0;
        bool active = false;
        uint32_t g_epi = 0;  // tiles read so far (only its two low bits are used: wrapping is harmless)
        for (int step = 0;; ++step) {
            // refill idle lanes from the CTA's item (warp-aggregated claim on its counter)
            {
                const bool need = !active;
                const unsigned m = __ballot_sync(0xffffffffu, need);
                unsigned long long basej = 0;
                if (m != 0) {
                    if (lane == __ffs(m) - 1) basej = atomicAdd(&S.j_next, (unsigned long long)__popc(m));
                    basej = __shfl_sync(0xffffffffu, basej, __ffs(m) - 1);
                }
                if (need) {
                    const unsigned long long jj = basej + __popc(m & ((1u << lane) - 1u));
                    if (jj < S.j_end) {
                        active = true;
                        j = (long long)jj;
                        q = j / P.N;
#pragma unroll
                        for (int i = 0; i < D; ++i) x[i] = (float)__ldg(P.x + q * D + i);
                        logw = dsig = gfac0 = src = src0 = dsrc = 0.f;
                        k = 0;
                    }
                }
            }
            // every walker thread reaches this reduction each step; then thread 0 manages the
            // item queue and the others learn its decision after the second barrier
            int any;
            asm volatile("{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n barrier.cta.red.or.pred q, 1, 128, p;\n selp.u32 %0, 1, 0, q;\n}\n"
                         : "=r"(any)
                         : "r"(active ? 1u : 0u)
                         : "memory");
            if (threadIdx.x == 0) {
                S.skip = 0;
                if (S.abort_flag) {
                    S.stop = 1;
                } else {
                    if (S.j_next >= S.j_end && !S.has_pend && !S.queue_empty) {
                        SphereItem it;
                        if (!next_item(L, it)) {
                            S.queue_empty = 1;
                        } else if (it.problem == S.cur) {  // same problem: walks continue without a pause
                            S.j_next = (unsigned long long)it.j0;
                            S.j_end = (unsigned long long)it.j1;
                        } else {
                            S.pend = it;
                            S.has_pend = 1;
                        }
                    }
                    if (!any) {
                        if (S.has_pend) {  // every walk of the old problem has ended: switch
                            S.cur = S.pend.problem;
                            S.j_next = (unsigned long long)S.pend.j0;
                            S.j_end = (unsigned long long)S.pend.j1;
                            S.has_pend = 0;
                            S.switched = 1;
                            S.skip = 1;
                        } else if (S.queue_empty) {
                            S.stop = 1;
                        } else {
                            S.skip = 1;  // the item was extended: refill first
                        }
                    }
                }
            }
            walker_barrier();
            if (S.stop) {
                if (lane == 0) mbar_arrive(&S.a_ready);
                break;
            }
            if (S.skip) {
                if (S.switched) {
                    load_problem(L, S.cur, SP, threadIdx.x, kWalkerThreads);
                    walker_barrier();
                    for (int i = threadIdx.x; i < kGeom; i += kWalkerThreads) geom_s[i] = SP.P.geom[i];
                    walker_barrier();
                    if (threadIdx.x == 0) S.switched = 0;
                }
                continue;
            }
            // the problem record lives in shared memory, which the waits' memory clobbers force to
            // be re-read at every use: its fields for this step go to registers once
            const int T = SP.n_tiles;
            const float *const soa = SP.soa;
            const float *const chunk_rhi = SP.chunk_rhi;
            write_row<D>(A, r, x, active);
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(&S.a_ready);

            // ---- epilogue: best and second-best CH-column chunk by the lower bound
            //      sqrt(min D~ + |x|^2 - delta) - r_hi, D~ = |c|^2 - 2 x.c (the square root
            //      rounded down); the TMEM loads return the 16-column minima
            float xx = 0.f;
#pragma unroll
            for (int i = 0; i < D; ++i) xx = fmaf(x[i], x[i], xx);
            const float xxd = xx - SP.delta;
            float m1 = CUDART_INF_F, m2 = CUDART_INF_F, m3 = CUDART_INF_F;
            int c1 = 0, c2 = 0;
            bool ok = true;
            // the record radius bounds of a tile (one 16-byte load): issued before the wait for
            // the tile's accumulators with 16-column chunks (fewer registers live across the tile
            // loop: fewer spills at the 96-register cap), fetched a tile ahead with 32-column ones
            // (no spill in d = 4..7 that way)
            const float4 *const rhi4 = reinterpret_cast<const float4 *>(chunk_rhi);
            float4 rhi_ahead = make_float4(0.f, 0.f, 0.f, 0.f);
            if constexpr (CH != kChunk) rhi_ahead = __ldg(rhi4);
            for (int t = 0; t < T; ++t, ++g_epi) {
                const int b = (int)(g_epi & 1);
                float rhi[kChunksPerTile];
                if constexpr (CH == kChunk) {
                    const float4 r4 = __ldg(rhi4 + t);
                    rhi[0] = r4.x;
                    rhi[1] = r4.y;
                    rhi[2] = r4.z;
                    rhi[3] = r4.w;
                } else {
                    rhi[0] = fmaxf(rhi_ahead.x, rhi_ahead.y);
                    rhi[1] = fmaxf(rhi_ahead.z, rhi_ahead.w);
                    rhi_ahead = __ldg(rhi4 + (t + 1 < T ? t + 1 : t));
                }
                if (!warp_wait_bar(S, &S.tfull[b], (uint32_t)((g_epi >> 1) & 1), L)) {
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                float cmin[kChunksPerTile];
                {
                    // the chunk minima (16 columns each, or 32)
                    if constexpr (CH == kChunk) {
                        tmem_min16x2(trow + b * kTileN, cmin[0], cmin[1]);
                        tmem_min16x2(trow + b * kTileN + 32, cmin[2], cmin[3]);
                    } else {
                        tmem_min32x2(trow + b * kTileN, cmin[0], cmin[1]);
                    }
                    // the accumulator buffer is free as soon as its minima are in registers
                    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&S.tempty[b]);
                }
#pragma unroll
                for (int c = 0; c < kChunksPerTile; ++c) {
                    const int id = t * kChunksPerTile + c;
                    const float cs = cmin[c] + xxd;
                    const float cm = sqrt_below(cs) - rhi[c];
                    // best, second and third bound; select form, no divergent branches
                    const bool lt1 = cm < m1, lt2 = cm < m2;
                    m3 = lt2 ? m2 : fminf(m3, cm);
                    m2 = lt1 ? m1 : (lt2 ? cm : m2);
                    c2 = lt1 ? c1 : (lt2 ? id : c2);
                    m1 = lt1 ? cm : m1;
                    c1 = lt1 ? id : c1;
                }
            }
            if (!ok) {
                active = false;  // abandon the walk; the next barrier reduction ends the loop
                continue;
            }

            // ---- exact FP32 distances |x - c| - r of the best chunk (and of the second-best
            //      one when its bound is below that); every other sphere is bounded below by the
            //      next chunk's bound. The warp refines the asking walkers one sphere per lane,
            //      32 / CH walkers per warp-wide load: a record stores its centres by coordinate
            //      quads, so every load is 512 contiguous bytes.
            float Rp = CUDART_INF_F;
            int pbest = c1 * CH;
            float *tr = reinterpret_cast<float *>(Bst + kStages * kTileBytes) + warp * 32 * kTrPitch;
            // the walkers' positions, padded like the chunk centres, in this warp's own rows of
            // the A operand: every MMA of the step has completed, and the next step rewrites them
            constexpr int kP = chunk_pitch(D);
            static_assert(32 * kP * 4 <= 4 * kSBO, "positions fit the warp's A rows");
            float *xs = reinterpret_cast<float *>(A + warp * 4 * kSBO);
#pragma unroll
            for (int i = 0; i < kP; i += 4)
                *reinterpret_cast<float4 *>(xs + lane * kP + i) =
                    make_float4(i < D ? x[i] : 0.f, i + 1 < D ? x[i + 1] : 0.f, i + 2 < D ? x[i + 2] : 0.f,
                                i + 3 < D ? x[i + 3] : 0.f);
            __syncwarp();
            auto refine = [&](int cc, bool want) {
                const unsigned todo = __ballot_sync(0xffffffffu, want);
                if (todo == 0u) return;
                // lane i: column i % CH of the chunk of walker w0 + (32 / CH) u + i / CH (sphere
                // i % 16 of its record i % CH / 16), kRefineGroup loads at a time so that they are
                // in flight together; a walker that does not ask still names a valid chunk, and its
                // row is not read
                constexpr int kPerLoad = 32 / CH;  // walkers per warp-wide load
                constexpr int kGroupWalkers = kPerLoad * kRefineGroup;
                const int wsub = lane / CH, col = lane % CH, rec = col / kChunk, sl = lane % kChunk;
#pragma unroll 1
                for (int w0 = 0; w0 < 32; w0 += kGroupWalkers) {
                    if (((todo >> w0) & ((1u << kGroupWalkers) - 1u)) == 0u) continue;
                    const float4 *cen[kRefineGroup];
                    float rr[kRefineGroup];
                    f32x2 s01[kRefineGroup], s23[kRefineGroup];  // packed partial sums of (x - c)^2
#pragma unroll
                    for (int u = 0; u < kRefineGroup; ++u) {
                        const int w = w0 + kPerLoad * u + wsub;
                        const float *ch =
                            soa + ((long long)__shfl_sync(0xffffffffu, cc, w) * kRecs + rec) * chunk_floats(D);
                        cen[u] = reinterpret_cast<const float4 *>(ch) + sl;
                        rr[u] = __ldg(ch + kChunk * kP + sl);
                        s01[u] = 0ull;
                        s23[u] = 0ull;
                    }
                    const f32x2 neg1 = pack2(-1.f, -1.f);
#pragma unroll
                    for (int i4 = 0; i4 < kP / 4; ++i4) {
#pragma unroll
                        for (int u = 0; u < kRefineGroup; ++u) {
                            const float4 c = __ldg(cen[u] + i4 * kChunk);
                            const float4 xv =
                                *reinterpret_cast<const float4 *>(xs + (w0 + kPerLoad * u + wsub) * kP + 4 * i4);
                            // x - c exactly rounded (fma with -1), squares summed in four packed
                            // lanes; zero padding adds exact zeros
                            const f32x2 t01 = ffma2(pack2(c.x, c.y), neg1, pack2(xv.x, xv.y));
                            const f32x2 t23 = ffma2(pack2(c.z, c.w), neg1, pack2(xv.z, xv.w));
                            s01[u] = ffma2(t01, t01, s01[u]);
                            s23[u] = ffma2(t23, t23, s23[u]);
                        }
                    }
#pragma unroll
                    for (int u = 0; u < kRefineGroup; ++u) {
                        const float2 a = unpack2(s01[u]), b = unpack2(s23[u]);
                        tr[(w0 + kPerLoad * u + wsub) * kTrPitch + col] =
                            sqrt_below_tight((a.x + b.x) + (a.y + b.y)) - rr[u];
                    }
                }
                __syncwarp();
                // walker w scans its own row (lowest index on ties)
                if (want) {
                    const float2 *row = reinterpret_cast<const float2 *>(tr + lane * kTrPitch);
#pragma unroll 4
                    for (int i = 0; i < CH / 2; ++i) {
                        const float2 di = row[i];
                        if (di.x < Rp) {
                            Rp = di.x;
                            pbest = cc * CH + 2 * i;
                        }
                        if (di.y < Rp) {
                            Rp = di.y;
                            pbest = cc * CH + 2 * i + 1;
                        }
                    }
                }
                __syncwarp();
            };
            refine(c1, active);
            float mrest = m2;
            const bool second = active && m2 < Rp;
            refine(c2, second);
            if (second) mrest = m3;
            if (!active) continue;
            if (mrest < Rp) {
                Rp = mrest;
                atomicAdd(L.shrinks, 1ull);
            }
            // other components: goal, outer ball, box faces (FP32 direct form)
            float best = Rp;
            int kind = kPoint, idx = pbest;
            if (P.has_goal) {
                float s = 0.f;
#pragma unroll
                for (int i = 0; i < D; ++i) {
                    const float t0 = x[i] - geom_s[2 * D + i];
                    s = fmaf(t0, t0, s);
                }
                const float rg = sqrtf(s) - P.goal_r;
                if (rg <= best) { best = rg; kind = kGoal; idx = 0; }
            }
            if (P.has_outer) {
                float s = 0.f;
#pragma unroll
                for (int i = 0; i < D; ++i) {
                    const float t0 = x[i] - geom_s[3 * D + i];
                    s = fmaf(t0, t0, s);
                }
                const float ro = P.outer_r - sqrtf(s);
                if (ro < best) { best = ro; kind = kOuter; idx = 0; }
            }
            if (P.has_box) {
#pragma unroll
                for (int i = 0; i < D; ++i) {
                    const float rlo = x[i] - geom_s[i];
                    if (rlo < best) { best = rlo; kind = kFace; idx = 2 * i; }
                    const float rhi = geom_s[D + i] - x[i];
                    if (rhi < best) { best = rhi; kind = kFace; idx = 2 * i + 1; }
                }
            }
            if (L.radius_out != nullptr && k == 0) L.radius_out[j] = (double)best;
            const float R = best - P.shrink;
            int outcome = 0;  // 0 jump, 1 boundary reached, 2 capped, 3 query outside, 4 roulette
            if (k == 0 && !(R > 0.f))
                outcome = 3;
            else if (R < P.eps && !(GRAD && P.grad_mode && k == 0))
                outcome = 1;
            else if (k >= L.max_steps)
                outcome = 2;
            else if (P.roulette_w > 0.f && k > 0 && logw < P.log_roulette_w) {
                // Russian roulette: survive with probability W / w_min carrying w_min
                if (roulette_uniform(L.seed, (uint64_t)(P.walk_base + j), (uint32_t)k) < expf(logw - P.log_roulette_w))
                    logw = P.log_roulette_w;
                else
                    outcome = 4;
            }
            if (outcome == 0) {
                float v[D];
                // antithetic pairs: the first direction of walk 2m + 1 is the negated one of walk 2m
                const uint64_t walk = (uint64_t)(P.walk_base + j);
                const bool first = k == 0;
                direction_f32<D, true>(L.seed, first ? first_direction_walk(walk, P.antithetic) : walk, (uint32_t)k, v);
                const float sgn = first && first_direction_negated(walk, P.antithetic) ? -1.f : 1.f;
                const float2 tb = table_lookup(P.table, R * P.sqrt_sigma);
                if (SRC && P.has_source) {
                    // the ball B(x_k, R) contains the source: q G_B(x_k, z) times the weight so far; at
                    // step 0 of a gradient walk also the query's step-0 value and the source part of
                    // the gradient, q grad_x G_B(x_0, z) (every walk of the query writes the same)
                    float rr = 0.f;
#pragma unroll
                    for (int i = 0; i < D; ++i) rr = fmaf(P.source_z[i] - x[i], P.source_z[i] - x[i], rr);
                    const float rz = sqrtf(rr);
                    if (rz > 0.f && rz < R) {
                        float dc;
                        const float c = sphere_source<D>(P, q, k, rz, R, tb, logw, dsig, dc);
                        src += c;
                        dsrc += dc;
                        if (k == 0) src0 = c;
                    }
                }
                if (GRAD && k == 0)
                    gfac0 = P.laplace ? ((float)D / R) * __expf(-tb.x) : ((float)D / R) / tb.y;
                logw += tb.x;
                dsig = fmaf(-(R * R) * inv2d, tb.y, dsig);
                const float Rs = sgn * R;
#pragma unroll
                for (int i = 0; i < D; ++i) x[i] = fmaf(Rs, v[i], x[i]);
                ++k;
                continue;
            }
            // ---- the walk ended
            float term = 0.f;
            float e[kMaxExp];
#pragma unroll
            for (int kk = 0; kk < kMaxExp; ++kk) e[kk] = 0.f;
            if (outcome == 1) {
                float xb[D];
#pragma unroll
                for (int i = 0; i < D; ++i) xb[i] = x[i];
                if (kind == kPoint) {
                    // closest point of the sphere (c, r): c + r (x - c)/|x - c|; c itself for a point
                    const float *ch = soa + (long long)(idx / kChunk) * chunk_floats(D);
                    const float *c = ch + (idx % kChunk) * 4;  // coordinate i at c[(i / 4) 4 kChunk + i % 4]
                    const float rad = __ldg(ch + kChunk * chunk_pitch(D) + idx % kChunk);
                    float cv[D];
#pragma unroll
                    for (int i = 0; i < D; ++i) cv[i] = __ldg(c + (i / 4) * 4 * kChunk + i % 4);
                    float s = 0.f;
#pragma unroll
                    for (int i = 0; i < D; ++i) s = fmaf(x[i] - cv[i], x[i] - cv[i], s);
                    const float len = sqrtf(s);
                    const float f = len > 0.f ? rad / len : 0.f;
#pragma unroll
                    for (int i = 0; i < D; ++i) xb[i] = fmaf(f, x[i] - cv[i], cv[i]);
                } else if (kind == kFace) {
#pragma unroll
                    for (int i = 0; i < D; ++i)
                        if (i == (idx >> 1)) xb[i] = (idx & 1) ? geom_s[D + i] : geom_s[i];
                } else {
                    const float *c = geom_s + (kind == kGoal ? 2 * D : 3 * D);
                    const float rad = kind == kGoal ? P.goal_r : P.outer_r;
                    float s = 0.f;
#pragma unroll
                    for (int i = 0; i < D; ++i) s = fmaf(x[i] - c[i], x[i] - c[i], s);
                    const float len = sqrtf(s);
#pragma unroll
                    for (int i = 0; i < D; ++i) xb[i] = len > 0.f ? fmaf(rad / len, x[i] - c[i], c[i]) : c[i];
                }
                if (P.n_exp > 0) {
                    const float *wv = geom_s + 4 * D;
                    const float *av = geom_s + 4 * D + kMaxExp;
#pragma unroll
                    for (int kk = 0; kk < kMaxExp; ++kk) {
                        if (kk < P.n_exp) {
                            float dot = logw;
#pragma unroll
                            for (int i = 0; i < D; ++i) dot = fmaf(av[kk * D + i], xb[i], dot);
                            e[kk] = expf(dot);
                            term = fmaf(wv[kk], e[kk], term);
                        }
                    }
                } else {
                    term = kind == kGoal ? expf(logw) : 0.f;
                }
                if (SRC) term += src;
            }
            if (outcome == 4) term = SRC ? src : 0.f;  // ended by the roulette: the source contributions so far
            // (a value-only problem in a gradient launch has no gradient terms)
            // (a walk ended by the roulette has a value only from the source)
            const bool has_grad = GRAD && P.grad_mode && (outcome == 1 || (SRC && outcome == 4)) && k > 0;
            const bool cv_walk = GRAD && P.cv && k > 0 && outcome != 3;  // capped walks count too
            float v0[D];
#pragma unroll
            for (int i = 0; i < D; ++i) v0[i] = 0.f;
            // the first direction: for the gradient terms, and for every walk that took its first
            // sphere when the control variate sums sum v0 and sum v0^2
            const bool need_v0 = (has_grad && (term != 0.f || (SRC && src0 != 0.f))) || cv_walk;
            if (GRAD && need_v0) {
                const uint64_t walk = (uint64_t)(P.walk_base + j);
                direction_f32<D, true>(L.seed, first_direction_walk(walk, P.antithetic), 0u, v0);
                const float sgn = first_direction_negated(walk, P.antithetic) ? -1.f : 1.f;
#pragma unroll
                for (int i = 0; i < D; ++i) v0[i] *= sgn;
            }
            // u^(x_1) C(R0): the walk's value without its step-0 source part
            const float gt = has_grad ? gfac0 * (SRC ? term - src0 : term) : 0.f;
            // control variate: G = alpha(R0)/C(R0), one number per query (every walk writes it)
            if (cv_walk && gfac0 != 0.f)
                P.acc[q * acc_fields(D, P.n_exp, P.cv, P.src) + cv_field(D, P.n_exp) + 3 * D] = (double)gfac0;
            // d term / d sigma: the boundary part times the summed d log C / d sigma, plus the
            // source contributions' derivatives (a capped walk has value 0)
            const float dv = SRC ? (outcome == 2 ? 0.f : fmaf(term - src, dsig, dsrc)) : term * dsig;
            write_record<D>(P, j, outcome, k, term, dv, gt, GRAD && need_v0, v0, e);
            if (P.w_term != nullptr) P.w_term[j] = outcome == 3 ? (double)CUDART_NAN : (double)term;
            if (P.w_jumps != nullptr) P.w_jumps[j] = k;
            if (P.w_dsigma != nullptr)
                P.w_dsigma[j] = outcome == 3 ? (double)CUDART_NAN : (double)dv;
            if (P.w_grad != nullptr) {
                // with a source, the per-query source part of the gradient (stored at step 0)
                const double *sp = (SRC && P.src) ? P.acc + q * acc_fields(D, P.n_exp, P.cv, 1) + src_field(D, P.n_exp, P.cv)
                                                  : nullptr;
#pragma unroll
                for (int i = 0; i < D; ++i) {
                    const double g = (double)(gt * v0[i]);
                    P.w_grad[j * D + i] = sp != nullptr ? g + sp[1 + i] : g;
                }
            }
            active = false;
        }
    }
    // ---------------------------------------------------------------------- teardown
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
}

// At least 48 KB: shared memory then also caps the residency at kCtasPerSm CTAs per SM, so the
// CTAs of an SM never ask for more than the 512 TMEM columns it has.
template <int K>
inline size_t smem_bytes_k() {
    using G = Geo<K>;
    return std::max<size_t>(48 * 1024, kSmemAlign + G::kABytes + (size_t)G::kStages * G::kTileBytes + kTransposeBytes);
}
inline size_t smem_bytes(int d) { return contraction_k(d) == 32 ? smem_bytes_k<32>() : smem_bytes_k<48>(); }


template <int D, bool GRAD, bool SRC, int CH>
inline cudaError_t configure_sphere_kernel() {
    cudaError_t e =
        cudaFuncSetAttribute(sphere_kernel<D, GRAD, SRC, CH>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes(D));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(sphere_kernel<D, GRAD, SRC, CH>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared);
    return e;
}

// Launch of the CH-column variants (each width is instantiated by one translation unit, so that
// the two sets of kernels compile in parallel; 32-column ones for d <= kSphereWideMaxD only). The
// shared-memory attributes are per device: the first launch on a device sets them for every
// variant of the width.
template <int CH>
cudaError_t launch_spheres_ch(const SphereLaunch &L, int d, int grad, int src, int grid, cudaStream_t s) {
    static std::mutex mu;
    static std::vector<int> configured;
    if (d < 2 || d > kPointCloudMaxD) return cudaErrorInvalidValue;
    const size_t smem = smem_bytes(d);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    {
        std::lock_guard<std::mutex> g(mu);
        if (std::find(configured.begin(), configured.end(), dev) == configured.end()) {
#define WOS_CFG(DD)                                                                      \
    if constexpr (CH == kChunk || DD <= kSphereWideMaxD) {                              \
        if (e == cudaSuccess) e = configure_sphere_kernel<DD, false, false, CH>();      \
        if (e == cudaSuccess) e = configure_sphere_kernel<DD, true, false, CH>();       \
        if (e == cudaSuccess) e = configure_sphere_kernel<DD, false, true, CH>();       \
        if (e == cudaSuccess) e = configure_sphere_kernel<DD, true, true, CH>();        \
    }
            WOS_CFG(2) WOS_CFG(3) WOS_CFG(4) WOS_CFG(5) WOS_CFG(6) WOS_CFG(7) WOS_CFG(8) WOS_CFG(9) WOS_CFG(10)
            WOS_CFG(11) WOS_CFG(12)
#undef WOS_CFG
            if (e != cudaSuccess) return e;
            configured.push_back(dev);
        }
    }
    if (grid < 1) return cudaSuccess;
    switch (d) {
#define WOS_LAUNCH(DD, G, S) sphere_kernel<DD, G, S, CH><<<grid, kThreads, smem, s>>>(L)
#define WOS_CASE(DD)                                                                   \
    case DD:                                                                           \
        if constexpr (CH == kChunk || DD <= kSphereWideMaxD) {                         \
            if (grad)                                                                  \
                src ? WOS_LAUNCH(DD, true, true) : WOS_LAUNCH(DD, true, false);        \
            else                                                                       \
                src ? WOS_LAUNCH(DD, false, true) : WOS_LAUNCH(DD, false, false);      \
            break;                                                                     \
        } else {                                                                       \
            return cudaErrorInvalidValue;                                              \
        }
        WOS_CASE(2) WOS_CASE(3) WOS_CASE(4) WOS_CASE(5) WOS_CASE(6) WOS_CASE(7) WOS_CASE(8) WOS_CASE(9)
        WOS_CASE(10) WOS_CASE(11) WOS_CASE(12)
#undef WOS_CASE
#undef WOS_LAUNCH
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}
extern template cudaError_t launch_spheres_ch<16>(const SphereLaunch &, int, int, int, int, cudaStream_t);
extern template cudaError_t launch_spheres_ch<32>(const SphereLaunch &, int, int, int, int, cudaStream_t);

}  // namespace pc
}  // namespace wos
