// Stream-collide kernels for D3Q27 with FP32 storage and arithmetic.
#include "lb_kernel.cuh"
namespace hlbm {
template cudaError_t launch_lb<3, float, float>(const LBArgs<float>&, int, int, cudaStream_t, bool);
}  // namespace hlbm
