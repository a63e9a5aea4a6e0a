// Stream-collide kernels for D3Q27 with FP16 shifted storage and FP32 arithmetic.
#include "lb_kernel.cuh"
namespace hlbm {
template cudaError_t launch_lb<3, __half, float>(const LBArgs<float>&, int, int, cudaStream_t, bool);
}  // namespace hlbm
