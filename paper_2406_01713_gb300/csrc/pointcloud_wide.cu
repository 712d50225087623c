// The 32-column chunk variants of the sphere-set walker (sphere_kernel.cuh), for large sets: in
// a translation unit of their own so that they compile beside the 16-column ones.
#include "sphere_kernel.cuh"

namespace wos {
template cudaError_t pc::launch_spheres_ch<32>(const SphereLaunch &, int, int, int, int, cudaStream_t);
}  // namespace wos
