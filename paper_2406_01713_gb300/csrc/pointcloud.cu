// Host side of the sphere-set Walk-on-Spheres walker on the tensor cores (the kernel is in
// sphere_kernel.cuh): operand preparation (BF16-split centre tiles in the shared-memory layout,
// chunk records, radius bounds), the contraction error bound, and the launches. This unit
// instantiates the 16-column chunk kernels; pointcloud_wide.cu the 32-column ones.
#include "sphere_kernel.cuh"

namespace wos {

static inline uint16_t bf16_bits(float f) {
    const __nv_bfloat16 h = __float2bfloat16_rn(f);
    return *reinterpret_cast<const uint16_t *>(&h);
}
static inline float bf16_value(uint16_t b) {
    __nv_bfloat16 h;
    *reinterpret_cast<uint16_t *>(&h) = b;
    return __bfloat162float(h);
}

cudaError_t pointcloud_prepare(const double *pts, const double *radii, int64_t M, int d, PointCloudDev *out) {
    if (d < 2 || d > kPointCloudMaxD) return cudaErrorInvalidValue;
    const int K = pc::contraction_k(d);
    const uint32_t tile_bytes = (uint32_t)pc::kTileN * K * 2, sbo = (uint32_t)(K / 8) * 128;
    const int64_t n_tiles = (M + pc::kTileN - 1) / pc::kTileN;
    const int64_t Mp = n_tiles * pc::kTileN;
    std::vector<uint16_t> hb((size_t)n_tiles * tile_bytes / 2, 0);
    std::vector<float> hsoa((size_t)(Mp / pc::kChunk) * pc::chunk_floats(d), 0.f);
    std::vector<float> hrhi((size_t)(Mp / pc::kChunk), 0.f);
    // balls in increasing radius (ties by index), points in input order
    std::vector<int64_t> order((size_t)M);
    for (int64_t i = 0; i < M; ++i) order[(size_t)i] = i;
    if (radii != nullptr)
        std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t b) { return radii[a] < radii[b]; });
    double pmax = 0.0;
    for (int64_t i = 0; i < Mp; ++i) {
        const bool real = i < M;
        const int64_t src = real ? order[(size_t)i] : 0;
        float p[WOS_MAX_D];
        double nn = 0.0;
        float *chunk = hsoa.data() + (size_t)(i / pc::kChunk) * pc::chunk_floats(d);
        float *centre = chunk + (size_t)(i % pc::kChunk) * 4;  // coordinate j at [(j / 4) 4 kChunk + j % 4]
        if (real && radii != nullptr) {
            const float r32 = (float)radii[src];
            chunk[(size_t)pc::kChunk * pc::chunk_pitch(d) + (size_t)(i % pc::kChunk)] = r32;
            // chunk bound rounded up: never below the FP64 radius
            float up = r32 < radii[src] ? std::nextafter(r32, 3.0e38f) : r32;
            float &cb = hrhi[(size_t)(i / pc::kChunk)];
            cb = std::max(cb, up);
        }
        for (int j = 0; j < d; ++j) {
            // padding centres sit far outside any domain: they never win the minimum
            p[j] = real ? (float)pts[src * d + j] : 1.0e3f;
            centre[(size_t)(j / 4) * 4 * pc::kChunk + (size_t)(j % 4)] = p[j];
            nn += (double)p[j] * (double)p[j];
            if (real) pmax = std::max(pmax, std::fabs((double)p[j]));
        }
        uint16_t row[48] = {0};
        for (int j = 0; j < d; ++j) {
            const float qv = -2.0f * p[j];
            const uint16_t qh = bf16_bits(qv);
            const uint16_t ql = bf16_bits(qv - bf16_value(qh));
            row[j] = qh;
            row[d + j] = ql;
            row[2 * d + j] = qh;
        }
        const float n32 = (float)nn;
        const uint16_t nh = bf16_bits(n32);
        row[3 * d] = nh;
        row[3 * d + 1] = bf16_bits(n32 - bf16_value(nh));
        const int64_t t = i / pc::kTileN;
        const int r = (int)(i % pc::kTileN);
        uint16_t *tile = hb.data() + (size_t)t * tile_bytes / 2;
        for (int k = 0; k < K; ++k) {
            const uint32_t off = (r / 8) * sbo + (k / 8) * pc::kLBO + (r % 8) * 16 + (k % 8) * 2;
            tile[off / 2] = row[k];
        }
    }
    out->n_tiles = (int)n_tiles;
    out->pmax = pmax;
    out->spheres = radii != nullptr ? 1 : 0;
    cudaError_t e = cudaMalloc(&out->tiles, hb.size() * 2);
    if (e == cudaSuccess) e = cudaMalloc(&out->soa, hsoa.size() * 4);
    if (e == cudaSuccess) e = cudaMalloc(&out->chunk_rhi, hrhi.size() * 4);
    if (e == cudaSuccess) e = cudaMemcpy(out->tiles, hb.data(), hb.size() * 2, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(out->soa, hsoa.data(), hsoa.size() * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(out->chunk_rhi, hrhi.data(), hrhi.size() * 4, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return e;
    return cudaSuccess;
}

void pointcloud_release(PointCloudDev *pcd) {
    cudaFree(pcd->tiles);
    cudaFree(pcd->soa);
    cudaFree(pcd->chunk_rhi);
    pcd->tiles = nullptr;
    pcd->soa = nullptr;
    pcd->chunk_rhi = nullptr;
}

// Bound of |D~ - D| for the BF16-split contraction: representation of x and -2p (2^-18
// relative each), the dropped x_l q_l term (2^-18), |p|^2 in two BF16 (2^-16 relative), and
// FP32 accumulation of 3d + 2 terms (2^-23 relative per addition, covering truncation).
float pointcloud_delta(int d, double xabs, double pmax) {
    const double dot = 2.0 * d * xabs * pmax;  // sum_j |x_j| |2 p_j|
    const double nn = d * pmax * pmax;
    const double terms = 2.0 * dot + nn;
    const double u18 = 3.814697265625e-06, u16 = 1.52587890625e-05, u23 = 1.1920928955078125e-07;
    const double bound = 3.0 * u18 * dot + u16 * nn + (3 * d + 2) * u23 * terms;
    return (float)(2.0 * bound + 1e-6);
}

int sphere_ctas_per_sm() { return pc::kCtasPerSm; }

template cudaError_t pc::launch_spheres_ch<16>(const SphereLaunch &, int, int, int, int, cudaStream_t);

cudaError_t launch_spheres(const SphereLaunch &L, int d, int grad, int src, int wide, int grid, cudaStream_t s) {
    return wide ? pc::launch_spheres_ch<32>(L, d, grad, src, grid, s) : pc::launch_spheres_ch<16>(L, d, grad, src, grid, s);
}

// One problem: implicit items of about 64 walks per walker (at least 4 items per CTA slot
// when there is that much work), so that the item tails stay short against the item.
cudaError_t launch_pointcloud(const PointCloudDev &pcd, const MixedProblem &P, float delta,
                              unsigned long long *cursor, int *status, unsigned long long *shrinks,
                              uint64_t seed, int64_t max_steps, long long wait_budget, int grad,
                              cudaStream_t s, double *radius_out) {
    SphereLaunch L;
    memset(&L, 0, sizeof(L));
    L.single.P = P;
    L.single.tiles = pcd.tiles;
    L.single.soa = pcd.soa;
    L.single.chunk_rhi = pcd.chunk_rhi;
    L.single.n_tiles = pcd.n_tiles;
    L.single.delta = delta;
    L.item_cursor = cursor;
    L.status = status;
    L.shrinks = shrinks;
    L.seed = seed;
    L.max_steps = max_steps;
    L.wait_budget = wait_budget > 0 ? wait_budget : kDefaultWaitBudget;
    L.wait_hint = wait_hint_ns(L.wait_budget);
    L.radius_out = radius_out;
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t total = P.Q * P.N;
    if (total <= 0) return cudaSuccess;
    const int64_t slots = (int64_t)pc::kCtasPerSm * sms;
    int64_t wpi = (total + 4 * slots - 1) / (4 * slots);
    wpi = std::max<int64_t>(pc::kRows, std::min<int64_t>(wpi, (int64_t)pc::kRows * 64));
    L.walks_per_item = wpi;
    L.n_items = (total + wpi - 1) / wpi;
    const int grid = (int)std::min<int64_t>(slots, L.n_items);
    return launch_spheres(L, P.d, grad, P.has_source, sphere_wide(P.d, pcd.n_tiles), grid, s);
}

}  // namespace wos
