// Probe time series and their spectra (Section 3.2 finds the precessing vortex core from the
// pressure recorded at points in the burner and reads its frequency off the spectrum).
//
// Probes: after every sampled step one thread per (probe, field) copies u_x, u_y[, u_z], P_h[, T]
// of the probe cell into row `slot` of a ring buffer [capacity][n_probes][nf] of doubles.
// Spectrum: Welch's estimate of the one-sided power spectral density of a series x_0..x_{n-1}
// sampled every dt: segments of L samples advancing by L/2, each with its mean removed and the
// periodic Hann window w_j = (1 - cos(2 pi j / L)) / 2 applied, |DFT|^2 averaged over the
// segments and scaled by dt / sum_j w_j^2, doubled except at 0 and L/2. One block per frequency
// bin; the twiddle angle is reduced exactly in integers, (f j) mod L, before sincospi.
#include "launch.h"

namespace hlbm {

namespace {
constexpr int PSD_BLOCK = 256;

template <typename R>
__global__ void probe_kernel(const int* __restrict__ cells, int n, int nf, int D, int N, const R* __restrict__ u,
                             const R* __restrict__ ph, const R* __restrict__ T, double* __restrict__ row) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n * nf) return;
  const int p = i / nf, f = i % nf;
  const int r = cells[p];
  double v;
  if (f < D) v = (double)u[(size_t)f * N + r];
  else if (f == D) v = (double)ph[r];
  else v = (double)T[r];
  row[i] = v;
}

// ordered copy of the ring (oldest sample first) into dst
__global__ void ring_order_kernel(const double* __restrict__ ring, long long cap, long long first, long long count,
                                  long long row, double* __restrict__ dst) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count * row) return;
  const long long s = i / row, k = i % row;
  dst[i] = ring[((first + s) % cap) * row + k];
}

__device__ __forceinline__ double block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < PSD_BLOCK / 32; ++w) t += sh[w];
  return t;  // valid in thread 0
}

// mean of each segment
__global__ void segment_mean_kernel(const double* __restrict__ x, long long stride, int L, int hop,
                                    double* __restrict__ mean) {
  __shared__ double sh[PSD_BLOCK / 32];
  const long long s0 = (long long)blockIdx.x * hop;
  double v = 0.0;
  for (int j = threadIdx.x; j < L; j += PSD_BLOCK) v += x[(s0 + j) * stride];
  const double t = block_sum(v, sh);
  if (threadIdx.x == 0) mean[blockIdx.x] = t / L;
}

__global__ void welch_kernel(const double* __restrict__ x, long long stride, int L, int hop, int nseg,
                             const double* __restrict__ mean, double dt, double* __restrict__ psd) {
  __shared__ double sh[PSD_BLOCK / 32];
  const int f = blockIdx.x;
  double acc = 0.0, w2 = 0.0;
  for (int s = 0; s < nseg; ++s) {
    const long long s0 = (long long)s * hop;
    const double m = mean[s];
    double re = 0.0, im = 0.0, ww = 0.0;
    for (int j = threadIdx.x; j < L; j += PSD_BLOCK) {
      double sw, cw, sa, ca;
      sincospi(2.0 * j / L, &sw, &cw);
      const double w = 0.5 - 0.5 * cw;
      const double v = w * (x[(s0 + j) * stride] - m);
      const long long fj = ((long long)f * j) % L;
      sincospi(2.0 * (double)fj / L, &sa, &ca);
      re += v * ca;
      im -= v * sa;
      ww += w * w;
    }
    const double Xr = block_sum(re, sh);
    const double Xi = block_sum(im, sh);
    if (s == 0) w2 = block_sum(ww, sh);
    if (threadIdx.x == 0) acc += Xr * Xr + Xi * Xi;
  }
  if (threadIdx.x == 0) {
    const double one = acc / nseg * dt / w2;
    psd[f] = (f == 0 || 2 * f == L) ? one : 2.0 * one;
  }
}
}  // namespace

template <typename R>
cudaError_t launch_probes(const int* cells, int n, int nf, int D, int N, const R* u, const R* ph, const R* T,
                          double* row, cudaStream_t st) {
  const int tot = n * nf;
  probe_kernel<R><<<(tot + 127) / 128, 128, 0, st>>>(cells, n, nf, D, N, u, ph, T, row);
  return cudaGetLastError();
}

cudaError_t launch_ring_order(const double* ring, long long cap, long long first, long long count, long long row,
                              double* dst, cudaStream_t st) {
  const long long tot = count * row;
  if (tot == 0) return cudaSuccess;
  ring_order_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(ring, cap, first, count, row, dst);
  return cudaGetLastError();
}

cudaError_t launch_welch(const double* x, long long stride, long long n, int L, double dt, double* mean_ws,
                         double* psd, cudaStream_t st) {
  const int hop = L / 2;
  const int nseg = (int)((n - L) / hop + 1);
  segment_mean_kernel<<<nseg, PSD_BLOCK, 0, st>>>(x, stride, L, hop, mean_ws);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  welch_kernel<<<L / 2 + 1, PSD_BLOCK, 0, st>>>(x, stride, L, hop, nseg, mean_ws, dt, psd);
  return cudaGetLastError();
}

template cudaError_t launch_probes<float>(const int*, int, int, int, int, const float*, const float*, const float*,
                                          double*, cudaStream_t);
template cudaError_t launch_probes<double>(const int*, int, int, int, int, const double*, const double*,
                                           const double*, double*, cudaStream_t);

}  // namespace hlbm
