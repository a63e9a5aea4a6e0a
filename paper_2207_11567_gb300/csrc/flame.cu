// Planar-flame diagnostics (Section 3.1 sets the burnt state, adiabatic temperature and interface
// thickness of its initial fields from a 1-D freely propagating flame of the same scheme and
// mixture; Section 3.2.2 quotes that flame's speed S_L and its thickness
// delta_L = (T_max - T_min) / max dT/dx).
//
// For a flame that propagates along x, one block per x column sums over the cross-section (y, z)
// the fluid cells, T, Y_k and the fuel consumption rate -omega_F of the rate law the update uses;
// one thread then turns the column means into the flame properties:
//   S_c     = sum over fluid cells of (-omega_F / F_loc) dx / (rho_u Y_F,u A), A = ny nz
//             cross-section cells (consumption speed, m/s), rho_u = P_th W_u / (R T_u) from the
//             inlet state; the rate is divided by the local thickening factor as in the update
//             (the thickened flame keeps S_L: its rate is F times lower over an F times wider
//             front);
//   delta_L = (T_max - T_min) / max |dT/dx| over the column means (centred differences);
//   x_f     = first crossing of (T_min + T_max) / 2 by the column means from low x, linear in x;
//   burnt state = column means of T and Y_k at the last column holding fluid.
#include "fd_kernel.cuh"
#include "launch.h"

namespace hlbm {

namespace {
constexpr int FL_BLOCK = 128;
constexpr int FL_ROWS = 3 + MAX_SP;  // fluid count, T, -omega_F, Y_k

template <typename R> __global__ void to_field_kernel(const double* __restrict__ src, R* __restrict__ dst, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = (R)src[i];
}

// Column means (fluid cells of column x): rows [count, T, -omega_F / F_loc, Y_0 .. Y_K-1] of
// col [.][nx]; F_loc = F, or the flame sensor's value at the current state.
template <typename R>
__global__ void __launch_bounds__(FL_BLOCK) flame_columns_kernel(FDArgs<R> a, int fuel, double* __restrict__ col) {
  const FDConst<R>& c = a.c;
  const Geo& g = a.geo;
  const int x = blockIdx.x;
  const int rows = g.ny * g.nz;
  const size_t N = (size_t)g.N;
  const R fdr = sizeof(R) == 4 ? (R)a.pth->fd_rho : (R)a.pth->fd_rho_d;
  double acc[FL_ROWS];
#pragma unroll
  for (int f = 0; f < FL_ROWS; ++f) acc[f] = 0.0;
  for (int j = threadIdx.x; j < rows; j += FL_BLOCK) {
    const int r = x + g.nx * j;
    if (!(__ldg(a.sword + r) >> 31)) continue;
    const R Tr = a.T[r];
    R sW = R(0), Yr[MAX_SP];
#pragma unroll
    for (int k = 0; k < MAX_SP; ++k) {
      Yr[k] = R(0);
      if (k < c.K) {
        Yr[k] = a.Y[(size_t)k * N + r];
        sW += Yr[k] * c.inv_W[k];
        acc[3 + k] += (double)Yr[k];
      }
    }
    const R rho_phys = fdr / (sW * Tr) / c.inv_rho_ref;  // P_th W / (R T)
    R q[MAX_RX];
#pragma unroll
    for (int jr = 0; jr < MAX_RX; ++jr) q[jr] = R(0);
    reaction_rates<0, R, MAX_SP>(c, Tr, R(1) / Tr, Yr, rho_phys, q);
    R w = R(0);
    for (int jr = 0; jr < c.nrx; ++jr) w += c.nu[jr][fuel] * q[jr];
    const R Floc = c.sensor ? sensor_floc<R>(c, Tr, a.Y[(size_t)c.sensor_species * N + r],
                                             a.Y[(size_t)c.sensor_oxidizer * N + r])
                            : c.F;
    acc[0] += 1.0;
    acc[1] += (double)Tr;
    acc[2] -= (double)(c.W[fuel] * w / Floc);
  }
  __shared__ double sh[FL_ROWS][FL_BLOCK / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int f = 0; f < FL_ROWS; ++f) {
    double v = acc[f];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) sh[f][warp] = v;
  }
  __syncthreads();
  if (threadIdx.x < 3 + c.K) {
    const int f = threadIdx.x;
    double s = 0.0, n = 0.0;
    for (int w = 0; w < FL_BLOCK / 32; ++w) {
      s += sh[f][w];
      n += sh[0][w];
    }
    col[(size_t)f * g.nx + x] = f == 0 ? n : (n > 0.0 ? s / n : 0.0);
  }
}

// props: [S_c, delta_L, x_f, T_min, T_max, T_b, Y_b[K]].
__global__ void flame_finalize_kernel(Geo g, int K, const double* __restrict__ col, const PthState* __restrict__ pth,
                                      double rho_u_per_P, double Y_Fu, double dx, double* __restrict__ props) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int nx = g.nx;
  const double* n = col;
  const double* Tm = col + nx;
  const double* wm = col + 2 * (size_t)nx;
  double Tmin = 0.0, Tmax = 0.0, J = 0.0;
  int last = -1;
  for (int x = 0; x < nx; ++x) {
    if (!(n[x] > 0.0)) continue;
    if (last < 0) Tmin = Tmax = Tm[x];
    Tmin = fmin(Tmin, Tm[x]);
    Tmax = fmax(Tmax, Tm[x]);
    J += wm[x] * n[x];
    last = x;
  }
  double gmax = 0.0;
  for (int x = 1; x + 1 < nx; ++x)
    if (n[x - 1] > 0.0 && n[x + 1] > 0.0) gmax = fmax(gmax, fabs(Tm[x + 1] - Tm[x - 1]) / (2.0 * dx));
  const double Tmid = 0.5 * (Tmin + Tmax);
  double xf = -1.0;
  for (int x = 0; x + 1 < nx; ++x) {
    if (!(n[x] > 0.0 && n[x + 1] > 0.0)) continue;
    const double a = Tm[x] - Tmid, b = Tm[x + 1] - Tmid;
    if (a != b && ((a <= 0.0 && b >= 0.0) || (a >= 0.0 && b <= 0.0))) {
      xf = dx * (x + a / (a - b));
      break;
    }
  }
  const double rho_u = pth->P * rho_u_per_P;
  props[0] = J * dx / (rho_u * Y_Fu * (double)(g.ny * g.nz));
  props[1] = gmax > 0.0 ? (Tmax - Tmin) / gmax : 0.0;
  props[2] = xf;
  props[3] = Tmin;
  props[4] = Tmax;
  props[5] = last >= 0 ? Tm[last] : 0.0;
  for (int k = 0; k < K; ++k) props[6 + k] = last >= 0 ? col[(size_t)(3 + k) * nx + last] : 0.0;
}
}  // namespace

int flame_col_rows() { return FL_ROWS; }

template <typename R> cudaError_t launch_to_field(const double* src, R* dst, size_t n, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  to_field_kernel<R><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(src, dst, (int)n);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_flame_properties(const FDArgs<R>& a, int fuel, double rho_u_per_P, double Y_Fu, double dx,
                                    double* col, double* props, cudaStream_t st) {
  flame_columns_kernel<R><<<a.geo.nx, FL_BLOCK, 0, st>>>(a, fuel, col);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  flame_finalize_kernel<<<1, 32, 0, st>>>(a.geo, a.c.K, col, a.pth, rho_u_per_P, Y_Fu, dx, props);
  return cudaGetLastError();
}

template cudaError_t launch_to_field<float>(const double*, float*, size_t, cudaStream_t);
template cudaError_t launch_to_field<double>(const double*, double*, size_t, cudaStream_t);
template cudaError_t launch_flame_properties<float>(const FDArgs<float>&, int, double, double, double, double*,
                                                    double*, cudaStream_t);
template cudaError_t launch_flame_properties<double>(const FDArgs<double>&, int, double, double, double, double*,
                                                     double*, cudaStream_t);

}  // namespace hlbm
