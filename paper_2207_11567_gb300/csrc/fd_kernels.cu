// Finite-difference, flame-sensor kernels for 2-D and 3-D grids, FP32 and FP64.
#include "fd_kernel.cuh"
namespace hlbm {
template cudaError_t launch_fd<2, float>(const FDArgs<float>&, cudaStream_t, bool);
template cudaError_t launch_fd<2, double>(const FDArgs<double>&, cudaStream_t, bool);
template cudaError_t launch_fd<3, float>(const FDArgs<float>&, cudaStream_t, bool);
template cudaError_t launch_fd<3, double>(const FDArgs<double>&, cudaStream_t, bool);
int fd_partial_blocks(int D, const Geo& g) { return D == 2 ? fd_blocks<2>(g) : fd_blocks<3>(g); }
}  // namespace hlbm
