// Instantiation of the persistent mixed-precision walker: value walks, CTAs of up to 768 threads
// (see walk_mixed.cuh).
#include "walk_mixed.cuh"

namespace wos {

cudaError_t configure_walk_mixed_val768(size_t smem_bytes) {
    return cudaFuncSetAttribute(walk_mixed_kernel<false, 768>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem_bytes);
}

int max_active_walk_mixed_val768(int threads, size_t smem_bytes) {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, walk_mixed_kernel<false, 768>, threads, smem_bytes) !=
        cudaSuccess)
        return 0;
    return n;
}

cudaError_t launch_walk_mixed_val768(const MixedLaunch &L, int grid, int threads, size_t smem_bytes, cudaStream_t s) {
    walk_mixed_kernel<false, 768><<<grid, threads, smem_bytes, s>>>(L);
    return cudaGetLastError();
}

}  // namespace wos
