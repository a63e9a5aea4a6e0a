// Set-up, output and reduction kernels: boundary link words, initial equilibrium populations
// (Eq. 6), field output, and the thermodynamic-pressure update.
#include "launch.h"

namespace hlbm {

namespace {

// Link word of one cell: bit i set when the source r - c_i of direction i is a solid cell, lies
// beyond a wall face, the low-x inlet or the high-x outlet (any link that is not a plain pull);
// bit 31 marks a fluid cell; 0 for a solid cell.
__global__ void links_kernel(int D, Geo g, const uint8_t* __restrict__ mask, uint32_t* __restrict__ out) {
  const int r = blockIdx.x * AUX_BLOCK + threadIdx.x;
  if (r >= g.N) return;
  if (mask[r]) {
    out[r] = 0u;
    return;
  }
  const int x = r % g.nx, t = r / g.nx, y = t % g.ny, z = t / g.ny;
  const int pos[3] = {x, y, z};
  const int dims[3] = {g.nx, g.ny, g.nz};
  const int Q = D == 2 ? 9 : 27;
  uint32_t word = 1u << 31;
  for (int i = 0; i < Q; ++i) {
    const int c[3] = {cx(i), cy(i), D == 3 ? cz(i) : 0};
    bool inlet = false, outlet = false, wall = false;
    int s[3];
    for (int a = 0; a < 3; ++a) {
      if (a >= D) {
        s[a] = 0;
        continue;
      }
      const int n = dims[a];
      int v = pos[a] - c[a];
      const bool below = v < 0, above = v >= n;
      if (g.bc_lo[a] == BC_PERIODIC) { if (below) v += n; }
      else if (g.bc_lo[a] == BC_WALL) wall |= below;
      else if (g.bc_lo[a] == BC_INLET) inlet |= below;
      if (g.bc_hi[a] == BC_PERIODIC) { if (above) v -= n; }
      else if (g.bc_hi[a] == BC_WALL) wall |= above;
      else if (g.bc_hi[a] == BC_OUTLET) outlet |= above;
      s[a] = v < 0 ? 0 : (v > n - 1 ? n - 1 : v);
    }
    const int si = s[0] + g.nx * (s[1] + g.ny * s[2]);
    const bool bb = inlet || outlet || wall || mask[si] != 0;
    if (bb) word |= 1u << i;
  }
  out[r] = word;
}

// Stencil word of the FD update (per axis a and side s, 4 bits at 4 (2a + s)): bits 0-1 the kind
// of the distance-1 point (0 fluid, 1 wall or solid, 2 inlet, 3 outlet), bits 2-3 that of the
// distance-2 point (0 fluid, 1 zero-gradient copy of the distance-1 value, 2 inlet); bit 31
// marks a fluid cell, a solid cell has word 0.
__device__ int sw_kind(const Geo& g, const uint8_t* mask, int axis, int sigma, int* p) {
  const int n = axis == 0 ? g.nx : (axis == 1 ? g.ny : g.nz);
  int v = p[axis] + sigma;
  if (v < 0) {
    if (g.bc_lo[axis] == BC_PERIODIC) v += n;
    else return g.bc_lo[axis] == BC_INLET ? 2 : 1;
  } else if (v >= n) {
    if (g.bc_hi[axis] == BC_PERIODIC) v -= n;
    else return g.bc_hi[axis] == BC_OUTLET ? 3 : 1;
  }
  int q[3] = {p[0], p[1], p[2]};
  q[axis] = v;
  if (mask[q[0] + g.nx * (q[1] + g.ny * q[2])]) return 1;
  p[axis] = v;
  return 0;
}

__global__ void stencil_words_kernel(int D, Geo g, const uint8_t* __restrict__ mask, uint32_t* __restrict__ out) {
  const int r = blockIdx.x * AUX_BLOCK + threadIdx.x;
  if (r >= g.N) return;
  if (mask[r]) {
    out[r] = 0u;
    return;
  }
  const int x = r % g.nx, t = r / g.nx, y = t % g.ny, z = t / g.ny;
  uint32_t word = 1u << 31;
  for (int ax = 0; ax < D; ++ax) {
    for (int sd = 0; sd < 2; ++sd) {
      int p[3] = {x, y, z};
      const int sg = sd ? 1 : -1;
      const int k1 = sw_kind(g, mask, ax, sg, p);
      int k2;
      if (k1 != 0) {
        k2 = k1 == 2 ? 2 : 1;
      } else {
        const int kk = sw_kind(g, mask, ax, sg, p);
        k2 = kk == 0 ? 0 : (kk == 2 ? 2 : 1);
      }
      word |= (uint32_t)(k1 | (k2 << 2)) << (4 * (2 * ax + sd));
    }
  }
  out[r] = word;
}

// Equilibrium populations of Eq. 6 (with Eq. 4) for the given fields, in the arithmetic type R of
// the storage (FP64 for FP64 storage, FP32 otherwise; FP64 is slow on this part).
template <typename S, typename R>
__global__ void set_fields_kernel(int D, Geo g, const double* __restrict__ T, const double* __restrict__ Y,
                                  int K, const double* __restrict__ invW, const double* __restrict__ u,
                                  const double* __restrict__ P_h, const double* __restrict__ g_pert,
                                  double p_fac, double P_ref, int thermal, S* g_out, R* T_out, R* Y_out,
                                  R* u_out, R* rho_out, R* lam_out, R* ph_out) {
  const int r = blockIdx.x * AUX_BLOCK + threadIdx.x;
  if (r >= g.N) return;
  const size_t N = (size_t)g.N;
  R rho = R(1);
  if (thermal) {
    R s = R(0);
    for (int k = 0; k < K; ++k) {
      const R yk = (R)Y[k * N + r];
      s += yk * (R)invW[k];
      Y_out[k * N + r] = yk;
    }
    const R Tr = (R)T[r];
    rho = (R)p_fac / (s * Tr);  // P_th W / (R T rho_ref)
    T_out[r] = Tr;
  }
  const R ux = (R)u[r], uy = (R)u[N + r], uz = D == 3 ? (R)u[2 * N + r] : R(0);
  u_out[r] = ux;
  u_out[N + r] = uy;
  if (D == 3) u_out[2 * N + r] = uz;
  rho_out[r] = rho;
  lam_out[r] = R(0);
  const R ph = (R)P_h[r];
  ph_out[r] = ph;
  const int Q = D == 2 ? 9 : 27;
  const R usq = ux * ux + uy * uy + uz * uz;
  const R third = R(1) / R(3);
  for (int i = 0; i < Q; ++i) {
    // q_i = g_eq,i / w_i - P_ref = (P_h - P_ref) + rho/3 (3 cu + 4.5 cu^2 - 1.5 u^2)
    const R cu = (R)cx(i) * ux + (R)cy(i) * uy + (D == 3 ? (R)cz(i) * uz : R(0));
    R q = (ph - (R)P_ref) + rho * third * (R(3) * cu + R(4.5) * cu * cu - R(1.5) * usq);
    if (g_pert) {
      const R w = (R)(D == 2 ? wgt<2>(i) : wgt<3>(i));
      q += (R)g_pert[(size_t)i * N + r] / w;
    }
    g_out[(size_t)i * N + r] = (S)q;
  }
}

template <typename S, typename R>
__global__ void get_fields_kernel(int D, Geo g, unsigned bits, int K, const S* __restrict__ gp,
                                  const R* __restrict__ T, const R* __restrict__ Y, const R* __restrict__ u,
                                  const R* __restrict__ ph, const R* __restrict__ rho, const R* __restrict__ lam,
                                  const PthState* pth, double P_ref, double* __restrict__ dst) {
  const int r = blockIdx.x * AUX_BLOCK + threadIdx.x;
  if (r >= g.N) return;
  const size_t N = (size_t)g.N;
  size_t off = 0;
  if (bits & 1u) { dst[off + r] = (double)T[r]; off += N; }
  if (bits & 2u) {
    for (int k = 0; k < K; ++k) dst[off + k * N + r] = (double)Y[k * N + r];
    off += (size_t)K * N;
  }
  if (bits & 4u) {
    for (int a = 0; a < D; ++a) dst[off + a * N + r] = (double)u[a * N + r];
    off += (size_t)D * N;
  }
  if (bits & 8u) { dst[off + r] = (double)ph[r]; off += N; }
  if (bits & 16u) { dst[off + r] = (double)rho[r]; off += N; }
  if (bits & 32u) {
    const double extra = sizeof(R) == 8 ? pth->lb_lam_d : (double)pth->lb_lam;
    dst[off + r] = (double)lam[r] + extra;
    off += N;
  }
  if (bits & 64u) {
    const int Q = D == 2 ? 9 : 27;
    for (int i = 0; i < Q; ++i) {
      const double w = D == 2 ? wgt<2>(i) : wgt<3>(i);
      dst[off + (size_t)i * N + r] = w * ((double)(R)gp[(size_t)i * N + r] + P_ref);
    }
  }
}

// Thermodynamic-pressure integrand of the stored initial state, with the same arithmetic and
// the same partial layout as the per-step reduction of the finite-difference kernel.
template <typename R>
__global__ void init_integral_kernel(Geo g, const uint8_t* __restrict__ mask, const R* __restrict__ T,
                                     const R* __restrict__ Y, FDConst<R> c, void* __restrict__ partials,
                                     unsigned long long* __restrict__ bad) {
  const int r = blockIdx.x * AUX_BLOCK + threadIdx.x;
  R v = R(0);
  if (r < g.N && mask[r] == 0) {
    R s = R(0);
    for (int k = 0; k < c.K; ++k) s += Y[(size_t)k * g.N + r] * (R)c.inv_W[k];
    v = (R)c.I_scale / (s * T[r]);
    // bad: count of fluid cells whose term the fixed-point sum cannot hold (non-finite, |v| >= 2^30)
    if (sizeof(R) == 4 && bad && !fix32_in_range((float)v)) atomicAdd(bad, 1ull);
  }
  if constexpr (sizeof(R) == 4) {
    __shared__ long long sh[AUX_BLOCK];
    sh[threadIdx.x] = f32_to_fix32((float)v);
    __syncthreads();
    for (int o = AUX_BLOCK / 2; o > 0; o >>= 1) {
      if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      ((long long*)partials)[2 * blockIdx.x] = sh[0];
      ((long long*)partials)[2 * blockIdx.x + 1] = 0;
    }
  } else {
    __shared__ double sh[AUX_BLOCK];
    sh[threadIdx.x] = (double)v;
    __syncthreads();
    for (int o = AUX_BLOCK / 2; o > 0; o >>= 1) {
      if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      ((double*)partials)[2 * blockIdx.x] = sh[0];
      ((double*)partials)[2 * blockIdx.x + 1] = 0.0;
    }
  }
}

// One block: exact sum of the per-block partials, then the thermodynamic-pressure update
// P^{n+1} = M^{n+1} / I^{n+1} in FP64.
// Thermodynamic-pressure update: the per-block partial sums of the FD update (integral I and the
// boundary mass flux) are reduced by PTH_BLOCKS blocks, each over a fixed contiguous range; the
// block that finishes last (a counter in device memory) adds the block sums in block order and
// updates the pressure state, then resets the counter. The partition and the order of every sum
// are fixed, so the result does not depend on scheduling (the FP32 path's sums are exact integers
// anyway).
constexpr int PTH_BLOCKS = 152;
constexpr int PTH_THREADS = 256;

template <typename T> __device__ __forceinline__ void block_sum2(T& a, T& b, T* sa, T* sb) {
  const int t = threadIdx.x;
  sa[t] = a;
  sb[t] = b;
  __syncthreads();
  for (int o = PTH_THREADS / 2; o > 0; o >>= 1) {
    if (t < o) {
      sa[t] += sa[t + o];
      sb[t] += sb[t + o];
    }
    __syncthreads();
  }
  a = sa[0];
  b = sb[0];
}

__global__ void __launch_bounds__(PTH_THREADS) pth_update_kernel(PthUpdate pu, const void* __restrict__ partials,
                                                                 int nblocks, void* stage, unsigned int* counter,
                                                                 PthState* pth, int init) {
  __shared__ long long sI[PTH_THREADS], sM[PTH_THREADS];
  __shared__ double dI[PTH_THREADS], dM[PTH_THREADS];
  __shared__ bool last;
  // the stream-collide that follows may start now: it reads the state this kernel writes only
  // after its own pdl_wait
  pdl_trigger();
  const int t = threadIdx.x, b = blockIdx.x, nb = gridDim.x;
  const int chunk = (nblocks + nb - 1) / nb;
  const int i0 = b * chunk, i1 = min(nblocks, i0 + chunk);
  if (pu.fixed_point) {
    const long long* p = (const long long*)partials;
    long long a = 0, c = 0;
    for (int i = i0 + t; i < i1; i += PTH_THREADS) { a += p[2 * i]; c += p[2 * i + 1]; }
    block_sum2(a, c, sI, sM);
    if (t == 0) { ((long long*)stage)[2 * b] = a; ((long long*)stage)[2 * b + 1] = c; }
  } else {
    const double* p = (const double*)partials;
    double a = 0, c = 0;
    for (int i = i0 + t; i < i1; i += PTH_THREADS) { a += p[2 * i]; c += p[2 * i + 1]; }
    block_sum2(a, c, dI, dM);
    if (t == 0) { ((double*)stage)[2 * b] = a; ((double*)stage)[2 * b + 1] = c; }
  }
  __threadfence();
  __syncthreads();
  if (t == 0) last = atomicAdd(counter, 1u) == (unsigned int)(nb - 1);
  __syncthreads();
  if (!last) return;
  __threadfence();
  double I, mflux;
  if (pu.fixed_point) {
    long long a = t < nb ? __ldcg((const long long*)stage + 2 * t) : 0;
    long long c = t < nb ? __ldcg((const long long*)stage + 2 * t + 1) : 0;
    block_sum2(a, c, sI, sM);
    I = (double)a / (FIX_SCALE * pu.I_s);
    mflux = (double)c / (FIX_SCALE * pu.M_s);
  } else {
    double a = t < nb ? __ldcg((const double*)stage + 2 * t) : 0.0;
    double c = t < nb ? __ldcg((const double*)stage + 2 * t + 1) : 0.0;
    block_sum2(a, c, dI, dM);
    I = a / pu.I_s;
    mflux = c / pu.M_s;
  }
  if (t == 0) {
    const double P_old = pth->P;
    // set-up: M = P_th0 I0 and nothing moves; step: P^{n+1} = M^{n+1} / I^{n+1}, or, with a
    // pressure outlet (hold), P stays at the ambient value while M keeps the mass balance
    const double M_new = init ? P_old * I : pth->M + mflux;
    const double P_new = (init || pu.hold) ? P_old : M_new / I;
    const double dP = P_new - P_old;
    pth->M = M_new;
    pth->P = P_new;
    pth->dP = dP;
    pth->lb_lam_d = -dP / P_old;
    pth->fd_rho_d = P_new / pu.R_rho_ref;
    pth->fd_dT_d = dP / pu.cp_rho_ref;
    pth->rho_in_d = P_new * pu.rin_fac;
    pth->lb_lam = (float)pth->lb_lam_d;
    pth->fd_rho = (float)pth->fd_rho_d;
    pth->fd_dT = (float)pth->fd_dT_d;
    pth->rho_in = (float)pth->rho_in_d;
    *counter = 0u;  // ready for the next launch (stream order)
  }
}
}  // namespace

cudaError_t launch_links(int D, const Geo& g, const uint8_t* mask, uint32_t* out, cudaStream_t st) {
  links_kernel<<<(g.N + AUX_BLOCK - 1) / AUX_BLOCK, AUX_BLOCK, 0, st>>>(D, g, mask, out);
  return cudaGetLastError();
}

cudaError_t launch_stencil_words(int D, const Geo& g, const uint8_t* mask, uint32_t* out, cudaStream_t st) {
  stencil_words_kernel<<<(g.N + AUX_BLOCK - 1) / AUX_BLOCK, AUX_BLOCK, 0, st>>>(D, g, mask, out);
  return cudaGetLastError();
}

template <typename S, typename R>
cudaError_t launch_set_fields(int D, const Geo& g, const double* T, const double* Y, int K,
                              const double* invW, const double* u, const double* P_h,
                              const double* g_pert, double p_fac, double P_ref, int thermal, S* g_out,
                              R* T_out, R* Y_out, R* u_out, R* rho_out, R* lam_out, R* ph_out,
                              cudaStream_t st) {
  set_fields_kernel<S, R><<<(g.N + AUX_BLOCK - 1) / AUX_BLOCK, AUX_BLOCK, 0, st>>>(
      D, g, T, Y, K, invW, u, P_h, g_pert, p_fac, P_ref, thermal, g_out, T_out, Y_out, u_out, rho_out,
      lam_out, ph_out);
  return cudaGetLastError();
}

template <typename S, typename R>
cudaError_t launch_get_fields(int D, const Geo& g, unsigned bits, int K, const S* gp, const R* T,
                              const R* Y, const R* u, const R* ph, const R* rho, const R* lam,
                              const PthState* pth, double P_ref, double* dst, cudaStream_t st) {
  get_fields_kernel<S, R><<<(g.N + AUX_BLOCK - 1) / AUX_BLOCK, AUX_BLOCK, 0, st>>>(
      D, g, bits, K, gp, T, Y, u, ph, rho, lam, pth, P_ref, dst);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_init_integral(const Geo& g, const uint8_t* mask, const R* T, const R* Y, const FDConst<R>& c,
                                 void* partials, int nblocks, cudaStream_t st, unsigned long long* bad) {
  init_integral_kernel<R><<<nblocks, AUX_BLOCK, 0, st>>>(g, mask, T, Y, c, partials, bad);
  return cudaGetLastError();
}
template cudaError_t launch_init_integral<float>(const Geo&, const uint8_t*, const float*, const float*,
                                                 const FDConst<float>&, void*, int, cudaStream_t,
                                                 unsigned long long*);
template cudaError_t launch_init_integral<double>(const Geo&, const uint8_t*, const double*, const double*,
                                                  const FDConst<double>&, void*, int, cudaStream_t,
                                                  unsigned long long*);

int pth_stage_words() { return 2 * PTH_BLOCKS; }

cudaError_t launch_pth_update(const PthUpdate& pu, const void* partials, int nblocks, void* stage,
                              unsigned int* counter, PthState* pth, int init, cudaStream_t st) {
  const int nb = nblocks < PTH_BLOCKS ? (nblocks > 0 ? nblocks : 1) : PTH_BLOCKS;
  pth_update_kernel<<<nb, PTH_THREADS, 0, st>>>(pu, partials, nblocks, stage, counter, pth, init);
  return cudaGetLastError();
}

#define INST(S, R)                                                                                     \
  template cudaError_t launch_set_fields<S, R>(int, const Geo&, const double*, const double*, int,    \
                                               const double*, const double*, const double*,           \
                                               const double*, double, double, int, S*, R*, R*, R*, R*, \
                                               R*, R*, cudaStream_t);                                  \
  template cudaError_t launch_get_fields<S, R>(int, const Geo&, unsigned, int, const S*, const R*,    \
                                               const R*, const R*, const R*, const R*, const R*,       \
                                               const PthState*, double, double*, cudaStream_t);
INST(double, double)
INST(float, float)
INST(__half, float)
#undef INST

}  // namespace hlbm
