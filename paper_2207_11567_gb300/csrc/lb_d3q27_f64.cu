// Stream-collide kernels for D3Q27 with FP64 storage and arithmetic.
#include "lb_kernel.cuh"
namespace hlbm {
template cudaError_t launch_lb<3, double, double>(const LBArgs<double>&, int, int, cudaStream_t, bool);
}  // namespace hlbm
