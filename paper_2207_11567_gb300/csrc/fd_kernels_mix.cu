// Finite-difference update with mixture-averaged species diffusion, 2-D and 3-D, FP32 and FP64:
// a per-cell pass writes the Hirschfelder-Curtiss coefficients, then fd_step_kernel's MIX copy
// of the cell update forms the fluxes (compiled apart so that the variants build in parallel).
#include "fd_kernel.cuh"
namespace hlbm {

constexpr int AUX_THREADS_MIX = 256;

// Per fluid cell: G_k = F_loc mu(T) / (Pr Le_k^mix) into mix[k N + r] and W into mix[K N + r], with
// Le_k^mix = sum_{j != k} (X_j + d) Le_kj / sum_{j != k} (X_j + d), X_j = max(Y_j W / W_j, 0),
// d = 1e-10: the resistance 1 / D_k of Blanc's law, (1 - X_k) / D_k = sum_{j != k} X_j / D_kj.
template <typename R>
__global__ void __launch_bounds__(AUX_THREADS_MIX) mix_coeff_kernel(const FDArgs<R> a, R* __restrict__ mix) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  const int N = a.geo.N;
  if (r >= N || __ldg(a.mask + r)) return;
  const FDConst<R>& c = a.c;
  const int K = c.K;
  R Y[MAX_SP];
  R sW = R(0);
  for (int k = 0; k < K; ++k) {
    Y[k] = ldg(a.Y + (size_t)k * N + r);
    sW += Y[k] * c.inv_W[k];
  }
  const R W = R(1) / sW;
  R X[MAX_SP];
  for (int k = 0; k < K; ++k) X[k] = fmax(Y[k] * W * c.inv_W[k], R(0)) + R(1e-10);
  const R T = ldg(a.T + r);
  const R F = a.Floc ? ldg(a.Floc + r) : c.F;
  const R fm = F * c.nu_lat * powr<R>(T * c.T_ref_inv, c.mu_exp) * c.inv_Pr;
  for (int k = 0; k < K; ++k) {
    R num = R(0), den = R(0);
    for (int j = 0; j < K; ++j) {
      if (j == k) continue;
      num += X[j] * c.Le_pair[k][j];
      den += X[j];
    }
    mix[(size_t)k * N + r] = fm * den / num;
  }
  mix[(size_t)K * N + r] = W;
}

template <int D, typename R> cudaError_t launch_fd_mix(const FDArgs<R>& a, R* mix, cudaStream_t st) {
  if (!mix) return cudaErrorInvalidValue;
  mix_coeff_kernel<R><<<(a.geo.N + AUX_THREADS_MIX - 1) / AUX_THREADS_MIX, AUX_THREADS_MIX, 0, st>>>(a, mix);
  const dim3 grid = fd_grid<D>(a.geo), block(FDShape<D>::X, FDShape<D>::Y, FDShape<D>::Z);
  if (a.c.K == 6 && a.c.nrx == 2) fd_step_kernel<D, R, 6, 2, 0, true><<<grid, block, 0, st>>>(a);
  else if (a.c.K == 4 && a.c.nrx == 1) fd_step_kernel<D, R, 4, 1, 0, true><<<grid, block, 0, st>>>(a);
  else fd_step_kernel<D, R, 0, 0, 0, true><<<grid, block, 0, st>>>(a);
  return cudaGetLastError();
}
template cudaError_t launch_fd_mix<2, float>(const FDArgs<float>&, float*, cudaStream_t);
template cudaError_t launch_fd_mix<2, double>(const FDArgs<double>&, double*, cudaStream_t);
template cudaError_t launch_fd_mix<3, float>(const FDArgs<float>&, float*, cudaStream_t);
template cudaError_t launch_fd_mix<3, double>(const FDArgs<double>&, double*, cudaStream_t);
}  // namespace hlbm
