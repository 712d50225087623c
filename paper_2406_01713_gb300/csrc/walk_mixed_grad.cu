// Instantiation and launch of the persistent mixed-precision walker, gradient walks (first sphere always taken) (see walk_mixed.cuh).
#include "walk_mixed.cuh"

namespace wos {

cudaError_t configure_walk_mixed_grad(size_t smem_bytes) {
    return cudaFuncSetAttribute(walk_mixed_kernel<true>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes);
}

int max_active_mixed_grad(int threads, size_t smem_bytes) {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, walk_mixed_kernel<true>, threads,
                                                      smem_bytes) != cudaSuccess)
        return 0;
    return n;
}

cudaError_t launch_walk_mixed_grad(const MixedLaunch &L, int grid, int threads, size_t smem_bytes,
                                  cudaStream_t s) {
    walk_mixed_kernel<true><<<grid, threads, smem_bytes, s>>>(L);
    return cudaGetLastError();
}

}  // namespace wos
