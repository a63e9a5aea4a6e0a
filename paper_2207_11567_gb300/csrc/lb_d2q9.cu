// Stream-collide kernels for D2Q9, every storage type.
#include "lb_kernel.cuh"
namespace hlbm {
template cudaError_t launch_lb<2, double, double>(const LBArgs<double>&, int, int, cudaStream_t, bool);
template cudaError_t launch_lb<2, float, float>(const LBArgs<float>&, int, int, cudaStream_t, bool);
template cudaError_t launch_lb<2, __half, float>(const LBArgs<float>&, int, int, cudaStream_t, bool);
}  // namespace hlbm
