// Adjoint step and objective of the 2-D hybrid step (not in the paper): the exact discrete
// reverse of one lbm_step (FD update -> LB stream-collide; the LB adjoint then the FD adjoint,
// which leaves the T and Y adjoints in slot form), and the fuel-consumption objective
// J = sum over fluid cells of the fuel consumption rate -omega_F with its gradient.
#include "adjoint_fd.cuh"
#include "adjoint_lb.cuh"
#include "fd_kernel.cuh"
#include "launch.h"

namespace hlbm {

namespace {

// J = sum_fluid -omega_F(T, Y) (kg/(m^3 s) per unit lattice volume) and dJ/dT, dJ/dY.
template <typename R>
__global__ void fuel_objective_kernel(FDArgs<R> a, int fuel, R* __restrict__ Tbar, R* __restrict__ Ybar,
                                      double* __restrict__ partials) {
  const FDConst<R>& c = a.c;
  const int r = blockIdx.x * FD_BLOCK + threadIdx.x;
  const int N = a.geo.N;
  double v = 0.0;
  if (r < N) {
    const uint32_t sw = __ldg(a.sword + r);
    R Tb = R(0);
    R Yb[MAX_SP];
    for (int k = 0; k < MAX_SP; ++k) Yb[k] = R(0);
    if (sw >> 31) {
      const R Tr = a.T[r];
      R Yr[MAX_SP];
      R sW = R(0);
      for (int k = 0; k < c.K; ++k) {
        Yr[k] = a.Y[k * N + r];
        sW += Yr[k] * c.inv_W[k];
      }
      const R W = R(1) / sW;
      const R fdr = sizeof(R) == 4 ? (R)a.pth->fd_rho : (R)a.pth->fd_rho_d;
      const R rho = fdr * W / Tr;
      const R rho_phys = rho / c.inv_rho_ref;
      R rpb = R(0), Wb = R(0);
      for (int j = 0; j < c.nrx; ++j) {
        R q = c.A[j] * exp(-(c.ER_hi[j] + c.ER_lo[j]) / Tr);
        if (c.beta[j] != R(0)) q *= pow(Tr, c.beta[j]);
        for (int m = 0; m < c.nord[j]; ++m) {
          const int k = c.ord_k[j][m];
          q *= Yr[k] > R(0) ? pow(rho_phys * Yr[k] * c.inv_W[k], c.ord_n[j][m]) : R(0);
        }
        const R wj = -c.W[fuel] * c.nu[j][fuel];  // J = sum_j wj q_j
        v += (double)(wj * q);
        const R qq = wj * q;
        Tb += qq * ((c.ER_hi[j] + c.ER_lo[j]) / (Tr * Tr) + c.beta[j] / Tr);
        for (int m = 0; m < c.nord[j]; ++m) {
          const int k = c.ord_k[j][m];
          if (Yr[k] > R(0)) {
            rpb += qq * c.ord_n[j][m] / rho_phys;
            Yb[k] += qq * c.ord_n[j][m] / Yr[k];
          }
        }
      }
      const R rhob = rpb / c.inv_rho_ref;
      Wb += rhob * fdr / Tr;
      Tb -= rhob * rho / Tr;
      const R sWb = -Wb * W * W;
      for (int k = 0; k < c.K; ++k) Yb[k] += sWb * c.inv_W[k];
    }
    Tbar[r] = Tb;
    for (int k = 0; k < c.K; ++k) Ybar[(size_t)k * N + r] = Yb[k];
  }
  __shared__ double sh[FD_BLOCK];
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int o = FD_BLOCK / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) partials[blockIdx.x] = sh[0];
}

// Reverse of lbm_set_fields with respect to T: the initial populations are the equilibrium
// q_i = (P_h - P_ref) + rho (c_i.u + 1.5 (c_i.u)^2 - 0.5 u^2) (shifted form) with
// rho = P_th W / (R T rho_ref), so dJ/dT = Tbar + sum_i qbar_i (c_i.u + 1.5 (c_i.u)^2 - 0.5 u^2) (-rho / T).
template <typename R>
__global__ void initial_T_adjoint_kernel(FDArgs<R> a, const R* __restrict__ adj0, R* __restrict__ gradT) {
  const int r = blockIdx.x * FD_BLOCK + threadIdx.x;
  const int N = a.geo.N;
  if (r >= N) return;
  const R Tb = adj0[(size_t)11 * N + r];
  if (!(__ldg(a.sword + r) >> 31)) {
    gradT[r] = Tb;
    return;
  }
  const FDConst<R>& c = a.c;
  const R Tr = a.T[r];
  R sW = R(0);
  for (int k = 0; k < c.K; ++k) sW += a.Y[(size_t)k * N + r] * c.inv_W[k];
  const R fdr = sizeof(R) == 4 ? (R)a.pth->fd_rho : (R)a.pth->fd_rho_d;
  const R rho = fdr / (sW * Tr);
  const R ux = a.u[r], uy = a.u[N + r];
  const R usq = ux * ux + uy * uy;
  R rb = R(0);
  for (int i = 0; i < 9; ++i) {
    const R cu = (R)cx(i) * ux + (R)cy(i) * uy;
    rb += adj0[(size_t)i * N + r] * (cu + R(1.5) * cu * cu - R(0.5) * usq);
  }
  gradT[r] = Tb - rb * rho / Tr;
}

}  // namespace

template <typename R>
cudaError_t launch_initial_T_adjoint(const FDArgs<R>& fdf, const R* adj0, R* gradT, cudaStream_t st) {
  initial_T_adjoint_kernel<R><<<(fdf.geo.N + FD_BLOCK - 1) / FD_BLOCK, FD_BLOCK, 0, st>>>(fdf, adj0, gradT);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_adjoint_step2d(const AdjBuffers<R>& b, const LBArgs<R>& lbf, const FDArgs<R>& fdf, bool thermal,
                                  bool pdl, cudaStream_t st) {
  const Geo& g = lbf.geo;
  const int N = g.N, K = thermal ? fdf.c.K : 0;
  LBAdjArgs<R> la{};
  la.f = lbf;
  la.u_prev = (const R*)lbf.u;
  la.gbar_out = b.in;
  la.ubar_out = b.in + 9 * (size_t)N;
  la.gbar_in = b.out;
  la.rho_bar = b.rho_own;
  la.lam_bar = b.lam_bar;
  la.T_bar = b.T_lb;
  la.u_bar = b.u_lb;
  la.rho_nb = b.rho_nb;
  la.inlet_bar = b.inlet_bar;
  const dim3 lgrid((g.nx + LB_BLOCK - 1) / LB_BLOCK, g.ny, 1);
  cudaError_t e = thermal ? launch_ex<LBAdjArgs<R>>(lb_adjoint_kernel<R, true>, lgrid, dim3(LB_BLOCK), st, pdl, la)
                          : launch_ex<LBAdjArgs<R>>(lb_adjoint_kernel<R, false>, lgrid, dim3(LB_BLOCK), st, false, la);
  if (e != cudaSuccess) return e;
  R* out_u = b.out + 9 * (size_t)N;
  if (!thermal) return cudaMemcpyAsync(out_u, b.u_lb, 2 * (size_t)N * sizeof(R), cudaMemcpyDeviceToDevice, st);
  FDAdjArgs<R> fa{};
  fa.f = fdf;
  if (!b.slots_in) {
    fa.Tbar_out = b.in + 11 * (size_t)N;
    fa.Ybar_out = b.in + 12 * (size_t)N;
  }
  fa.slots_in = b.slots_in;
  fa.rho_own = b.rho_own;
  fa.rho_nb = b.rho_nb;
  fa.lam_bar = b.lam_bar;
  fa.T_lb = b.T_lb;
  fa.u_lb = b.u_lb;
  fa.slots = b.slots;
  fa.u_out = out_u;
  const int fb = (N + FDA_BLOCK - 1) / FDA_BLOCK;
  // the LB adjoint of this step precedes it in the stream
  void (*fk)(FDAdjArgs<R>) = K == 6 ? fd_adjoint_kernel<R, 6> : (K == 4 ? fd_adjoint_kernel<R, 4> : fd_adjoint_kernel<R, 0>);
  return launch_ex<FDAdjArgs<R>>(fk, dim3(fb), dim3(FDA_BLOCK), st, true, fa);
}

namespace {
template <typename R> __global__ void zero_solid_pops_kernel(Geo g, const uint32_t* __restrict__ links, R* pops) {
  const int r = blockIdx.x * FD_BLOCK + threadIdx.x;
  if (r >= g.N || (__ldg(links + r) >> 31)) return;
  for (int i = 0; i < 9; ++i) pops[(size_t)i * g.N + r] = R(0);
}
}  // namespace

template <typename R> cudaError_t launch_zero_solid_pops(const Geo& g, const uint32_t* links, R* pops, cudaStream_t st) {
  zero_solid_pops_kernel<R><<<(g.N + FD_BLOCK - 1) / FD_BLOCK, FD_BLOCK, 0, st>>>(g, links, pops);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_adjoint_gather(const Geo& g, const uint32_t* sword, int K, const R* slots, R* Tbar, R* Ybar,
                                  cudaStream_t st) {
  fd_adjoint_gather<R><<<(g.N + FDA_BLOCK - 1) / FDA_BLOCK, FDA_BLOCK, 0, st>>>(g, sword, K, slots, Tbar, Ybar);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_fuel_objective(const FDArgs<R>& fdf, int fuel, R* Tbar, R* Ybar, double* partials, int nblocks,
                                  cudaStream_t st) {
  fuel_objective_kernel<R><<<nblocks, FD_BLOCK, 0, st>>>(fdf, fuel, Tbar, Ybar, partials);
  return cudaGetLastError();
}

template cudaError_t launch_adjoint_step2d<float>(const AdjBuffers<float>&, const LBArgs<float>&, const FDArgs<float>&, bool,
                                                  bool, cudaStream_t);
template cudaError_t launch_adjoint_step2d<double>(const AdjBuffers<double>&, const LBArgs<double>&,
                                                   const FDArgs<double>&, bool, bool, cudaStream_t);
template cudaError_t launch_adjoint_gather<float>(const Geo&, const uint32_t*, int, const float*, float*, float*,
                                                  cudaStream_t);
template cudaError_t launch_adjoint_gather<double>(const Geo&, const uint32_t*, int, const double*, double*, double*,
                                                   cudaStream_t);
template cudaError_t launch_zero_solid_pops<float>(const Geo&, const uint32_t*, float*, cudaStream_t);
template cudaError_t launch_zero_solid_pops<double>(const Geo&, const uint32_t*, double*, cudaStream_t);
template cudaError_t launch_initial_T_adjoint<float>(const FDArgs<float>&, const float*, float*, cudaStream_t);
template cudaError_t launch_initial_T_adjoint<double>(const FDArgs<double>&, const double*, double*, cudaStream_t);
template cudaError_t launch_fuel_objective<float>(const FDArgs<float>&, int, float*, float*, double*, int, cudaStream_t);
template cudaError_t launch_fuel_objective<double>(const FDArgs<double>&, int, double*, double*, double*, int,
                                                   cudaStream_t);

}  // namespace hlbm
