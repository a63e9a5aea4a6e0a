// Diagnostics on the device (Section 3: time-averaged and RMS fields, flame surface).
//
// Running statistics: per fluid cell and field (u components, P_h, T), Welford's update of the
// mean and of M2 = sum of squared deviations in FP32, once per sampled step:
//   mean_n = mean_{n-1} + (x - mean_{n-1}) / n,  M2_n = M2_{n-1} + (x - mean_{n-1}) (x - mean_n).
// Flame length (2-D): marching squares on the progress variable c = (T - T_u) / (T_b - T_u) over
// squares of four fluid cell centres; one thread per square (its lower-left cell), FP64 lengths,
// per-block partial sums added on the host in block order (deterministic).
#include "common.cuh"
#include "launch.h"

namespace hlbm {

namespace {
constexpr int ST_BLOCK = 256;

template <typename R>
__global__ void stats_kernel(int N, int nf, const uint32_t* __restrict__ links, const R* __restrict__ u, int D,
                             const R* __restrict__ ph, const R* __restrict__ T, float inv_n, float* __restrict__ mean,
                             float* __restrict__ m2) {
  const int r = blockIdx.x * ST_BLOCK + threadIdx.x;
  if (r >= N || !(__ldg(links + r) >> 31)) return;
  for (int f = 0; f < nf; ++f) {
    float x;
    if (f < D) x = (float)u[(size_t)f * N + r];
    else if (f == D) x = (float)ph[r];
    else x = (float)T[r];
    const size_t k = (size_t)f * N + r;
    const float m0 = mean[k];
    const float m1 = m0 + (x - m0) * inv_n;
    mean[k] = m1;
    m2[k] += (x - m0) * (x - m1);
  }
}

__device__ __forceinline__ double seg(double ax, double ay, double bx, double by) {
  const double dx = ax - bx, dy = ay - by;
  return sqrt(dx * dx + dy * dy);
}

template <typename R>
__global__ void flame_length_kernel(Geo g, const uint32_t* __restrict__ links, const R* __restrict__ T, double T_u,
                                    double inv_dT, double level, double* __restrict__ partials) {
  const int r = blockIdx.x * ST_BLOCK + threadIdx.x;
  double len = 0.0;
  if (r < g.N) {
    const int x = r % g.nx, y = r / g.nx;
    if (x < g.nx - 1 && y < g.ny - 1) {
      const int id[4] = {r, r + 1, r + 1 + g.nx, r + g.nx};
      bool ok = true;
      double v[4];
      for (int k = 0; k < 4; ++k) {
        ok = ok && (__ldg(links + id[k]) >> 31);
        v[k] = ((double)T[id[k]] - T_u) * inv_dT;
      }
      if (ok) {
        const double px[4] = {0.0, 1.0, 1.0, 0.0}, py[4] = {0.0, 0.0, 1.0, 1.0};
        bool ab[4];
        for (int k = 0; k < 4; ++k) ab[k] = v[k] >= level;
        double cxs[4], cys[4];
        int nc = 0;
        bool has[4];
        for (int e = 0; e < 4; ++e) {
          const int a = e, b = (e + 1) & 3;
          has[e] = ab[a] != ab[b];
          if (has[e]) {
            const double t = (level - v[a]) / (v[b] - v[a]);
            cxs[e] = px[a] + t * (px[b] - px[a]);
            cys[e] = py[a] + t * (py[b] - py[a]);
            ++nc;
          }
        }
        if (nc == 2) {
          int e0 = -1, e1 = -1;
          for (int e = 0; e < 4; ++e)
            if (has[e]) {
              if (e0 < 0) e0 = e;
              else e1 = e;
            }
          len = seg(cxs[e0], cys[e0], cxs[e1], cys[e1]);
        } else if (nc == 4) {
          const bool centre = 0.25 * (v[0] + v[1] + v[2] + v[3]) >= level;
          for (int k = 0; k < 4; ++k)
            if (ab[k] != centre) {
              const int ep = (k + 3) & 3;
              len += seg(cxs[ep], cys[ep], cxs[k], cys[k]);
            }
        }
      }
    }
  }
  __shared__ double sh[ST_BLOCK];
  sh[threadIdx.x] = len;
  __syncthreads();
  for (int o = ST_BLOCK / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) partials[blockIdx.x] = sh[0];
}
// mean and RMS fluctuation sqrt(M2 / n) as FP64 (layout: nf means, then nf RMS fields)
__global__ void stats_finalize_kernel(int N, int nf, const uint32_t* __restrict__ links, const float* __restrict__ mean,
                                      const float* __restrict__ m2, double inv_n, double* __restrict__ out) {
  const int r = blockIdx.x * ST_BLOCK + threadIdx.x;
  if (r >= N) return;
  const bool fl = (__ldg(links + r) >> 31) != 0u;
  for (int f = 0; f < nf; ++f) {
    const size_t k = (size_t)f * N + r;
    out[k] = fl ? (double)mean[k] : 0.0;
    out[(size_t)nf * N + k] = fl ? sqrt(fmax((double)m2[k] * inv_n, 0.0)) : 0.0;
  }
}
}  // namespace

int stats_block() { return ST_BLOCK; }

cudaError_t launch_stats_finalize(int N, int nf, const uint32_t* links, const float* mean, const float* m2,
                                  long long n, double* out, cudaStream_t st) {
  stats_finalize_kernel<<<(N + ST_BLOCK - 1) / ST_BLOCK, ST_BLOCK, 0, st>>>(N, nf, links, mean, m2,
                                                                            n > 0 ? 1.0 / (double)n : 0.0, out);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_stats(int N, int nf, const uint32_t* links, const R* u, int D, const R* ph, const R* T, long long n,
                         float* mean, float* m2, cudaStream_t st) {
  stats_kernel<R><<<(N + ST_BLOCK - 1) / ST_BLOCK, ST_BLOCK, 0, st>>>(N, nf, links, u, D, ph, T, 1.0f / (float)n, mean,
                                                                      m2);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_flame_length(const Geo& g, const uint32_t* links, const R* T, double T_u, double T_b, double level,
                                double* partials, cudaStream_t st) {
  flame_length_kernel<R><<<(g.N + ST_BLOCK - 1) / ST_BLOCK, ST_BLOCK, 0, st>>>(g, links, T, T_u, 1.0 / (T_b - T_u),
                                                                                level, partials);
  return cudaGetLastError();
}

template cudaError_t launch_stats<float>(int, int, const uint32_t*, const float*, int, const float*, const float*,
                                         long long, float*, float*, cudaStream_t);
template cudaError_t launch_stats<double>(int, int, const uint32_t*, const double*, int, const double*, const double*,
                                          long long, float*, float*, cudaStream_t);
template cudaError_t launch_flame_length<float>(const Geo&, const uint32_t*, const float*, double, double, double,
                                                double*, cudaStream_t);
template cudaError_t launch_flame_length<double>(const Geo&, const uint32_t*, const double*, double, double, double,
                                                 double*, cudaStream_t);

}  // namespace hlbm
