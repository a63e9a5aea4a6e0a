// Finite-difference update with variable heat capacities (c_p,k(T) polynomials), 2-D and 3-D,
// FP32 and FP64: compiled apart from the constant-c_p kernels so that both build in parallel.
#include "fd_kernel.cuh"
namespace hlbm {
template <int D, typename R> cudaError_t launch_fd_vcp(const FDArgs<R>& a, cudaStream_t st) {
  const dim3 grid = fd_grid<D>(a.geo), block(FDShape<D>::X, FDShape<D>::Y, FDShape<D>::Z);
  // polynomial degree: linear c_p (the common case) or the full quartic
  const bool lin = a.c.varcp == 1;
  if (a.c.K == 6 && a.c.nrx == 2) {
    if (lin) fd_step_kernel<D, R, 6, 2, 1><<<grid, block, 0, st>>>(a);
    else fd_step_kernel<D, R, 6, 2, 4><<<grid, block, 0, st>>>(a);
  } else {
    if (lin) fd_step_kernel<D, R, 0, 0, 1><<<grid, block, 0, st>>>(a);
    else fd_step_kernel<D, R, 0, 0, 4><<<grid, block, 0, st>>>(a);
  }
  return cudaGetLastError();
}
template cudaError_t launch_fd_vcp<2, float>(const FDArgs<float>&, cudaStream_t);
template cudaError_t launch_fd_vcp<2, double>(const FDArgs<double>&, cudaStream_t);
template cudaError_t launch_fd_vcp<3, float>(const FDArgs<float>&, cudaStream_t);
template cudaError_t launch_fd_vcp<3, double>(const FDArgs<double>&, cudaStream_t);
}  // namespace hlbm
