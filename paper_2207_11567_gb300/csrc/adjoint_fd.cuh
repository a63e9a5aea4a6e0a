// Adjoint (reverse mode) of the 2-D finite-difference update of fd_kernel.cuh (open domain,
// constant thickening factor): WENO3 faces, centred diffusion, chemistry, rho and Lambda. The
// adjoint step is not in the paper; it is the exact transpose of the discrete update written by
// hand. Upwind choices and the max(Y, 0) of the rate law are held fixed (their derivative is 0).
//
// Each fluid cell recomputes its forward update, reverses it, and writes the adjoint of every
// stencil value it read into one of 9 slots per field (center, distance-1 and distance-2 points
// on each side of each axis); a ghost value's adjoint is folded onto the cell it copies (inlet
// values are constants). fd_adjoint_gather then sums, for each cell, the slots of the cells
// whose stencils contain it.
#pragma once
#include "common.cuh"
#include "fd_kernel.cuh"

namespace hlbm {

template <typename R> struct FDAdjArgs {
  FDArgs<R> f;           // forward arguments of state n (T, Y, u, stencil words, constants)
  const R* Tbar_out;     // [N] adjoint of T^{n+1}
  const R* Ybar_out;     // [K][N] adjoint of Y^{n+1}
  const R* rho_own;      // [N] adjoint of rho^n used by the cell's own LB update
  const R* rho_nb;       // [4][N] adjoint of the +x, -x, +y, -y neighbour rho in a cell's LB update
  const R* lam_bar;      // [N] adjoint of Lambda^n (from the LB adjoint)
  R* slots;              // [9][1+K][N] stencil-value adjoints
  R* u_bar;              // [2][N] adjoint of u^n through the advection (center only)
};

// reverse of one WENO3 face b + (tbc dab + 2 tab dbc) / (2 (tbc + 2 tab)), t = (d^2 + eps)^2
template <typename R>
__device__ __forceinline__ void weno_face_rev(R dab, R dbc, R eps, R fb, R& bb, R& dabb, R& dbcb) {
  const R sab = dab * dab + eps, sbc = dbc * dbc + eps;
  const R tab = sab * sab, tbc = sbc * sbc;
  const R Nn = tbc * dab + R(2) * tab * dbc, Dn = tbc + R(2) * tab;
  const R iD = fdiv<R>(R(1), Dn);
  const R Nb = fb * R(0.5) * iD;
  const R Db = -Nb * Nn * iD;
  const R tabb = Nb * R(2) * dbc + Db * R(2);
  const R tbcb = Nb * dab + Db;
  bb = fb;
  dabb = Nb * tbc + tabb * R(4) * dab * sab;
  dbcb = Nb * R(2) * tab + tbcb * R(4) * dbc * sbc;
}
template <typename R> __device__ __forceinline__ R weno_face(R b, R dab, R dbc, R eps) {
  const R sab = dab * dab + eps, sbc = dbc * dbc + eps;
  const R tab = sab * sab, tbc = sbc * sbc;
  return b + R(0.5) * fdiv<R>(tbc * dab + R(2) * tab * dbc, tbc + R(2) * tab);
}

// slot numbering: 0 center, 1 + 2*(2a+s) distance-1 point, 2 + 2*(2a+s) distance-2 point
__device__ __forceinline__ int slot1(int ax, int sd) { return 1 + 2 * (2 * ax + sd); }
__device__ __forceinline__ int slot2(int ax, int sd) { return 2 + 2 * (2 * ax + sd); }

// Thread layout of the adjoint kernels: blockDim = (FDA_CELLS, K + 1), x the cell within the
// block, y the field (0: T, k + 1: Y_k), so that a cell's fields are reversed in parallel.
constexpr int FDA_CELLS = 32;
constexpr int FDA_THREADS = FDA_CELLS * (MAX_SP + 1);
// per-field partial adjoints of the quantities the fields share, summed over the fields
enum { PA_INVRHO = 0, PA_INVRPF, PA_QDOT, PA_TR, PA_W, PA_FM, PA_UR = PA_FM + 4, PA_Q = PA_UR + 2,
       PA_N = PA_Q + MAX_RX };

// Stencil of a cell: neighbour kinds and indices of the distance-1 and distance-2 points on each
// side of each axis (ghost points copy the cell or the distance-1 point; inlet ghosts are
// constants).
struct FDStencil2 {
  int k1[2][2], k2[2][2], i1[2][2], i2[2][2];
};
__device__ __forceinline__ void fd_stencil2(const Geo& g, uint32_t sw, int r, int x, int y, FDStencil2& S) {
  const int pos[2] = {x, y}, dims[2] = {g.nx, g.ny}, strides[2] = {1, g.nx};
#pragma unroll
  for (int ax = 0; ax < 2; ++ax)
#pragma unroll
    for (int sd = 0; sd < 2; ++sd) {
      const uint32_t bits = (sw >> (4 * (2 * ax + sd))) & 15u;
      const int kk1 = (int)(bits & 3u), kk2 = (int)(bits >> 2);
      const int sg = sd ? 1 : -1;
      int p1 = pos[ax] + sg;
      p1 = p1 < 0 ? p1 + dims[ax] : (p1 >= dims[ax] ? p1 - dims[ax] : p1);
      int p2 = p1 + sg;
      p2 = p2 < 0 ? p2 + dims[ax] : (p2 >= dims[ax] ? p2 - dims[ax] : p2);
      const int j1 = kk1 == NB_FLUID ? r + (p1 - pos[ax]) * strides[ax] : r;
      S.k1[ax][sd] = kk1;
      S.k2[ax][sd] = kk2;
      S.i1[ax][sd] = j1;
      S.i2[ax][sd] = kk2 == 0 ? r + (p2 - pos[ax]) * strides[ax] : j1;
    }
}

// Rate q_j of one cell, the same arithmetic as reaction_rates of the forward kernel.
template <typename R>
__device__ __forceinline__ R rate_of(const FDConst<R>& c, int j, R T, const R* __restrict__ Y, size_t N, int r,
                                     R rho_phys) {
  R v;
  if constexpr (sizeof(R) == 4) v = c.A[j] * arrhenius(c.ER_hi[j], c.ER_lo[j], T);
  else v = c.A[j] * exp(-c.ER_hi[j] / T);
  if (c.beta[j] != R(0)) v *= powr<R>(T, c.beta[j]);
#pragma unroll
  for (int m = 0; m < MAX_ORD; ++m) {
    if (m >= c.nord[j]) break;
    const int k = c.ord_k[j][m];
    const R n = c.ord_n[j][m];
    const R conc = rho_phys * fmax(Y[(size_t)k * N + r], R(0)) * c.inv_W[k];
    v *= (n == R(1)) ? conc : powr<R>(conc, n);
  }
  return v;
}

template <typename R>
__global__ void __launch_bounds__(FDA_THREADS) fd_adjoint_kernel(const FDAdjArgs<R> A) {
  __shared__ R part[MAX_SP + 1][PA_N][FDA_CELLS];
  __shared__ R sh_q[MAX_RX][FDA_CELLS];
  __shared__ R sh_mu[5][FDA_CELLS];  // mu(T_r), then mu at the distance-1 points (-x, +x, -y, +y)
  // inputs of the per-cell reverse of the shared terms, staged by all warps so that the one warp
  // that runs that dependent chain reads shared memory only: the field sums of the partial
  // adjoints, the cell's mass fractions and the adjoint of rho^n from the LB step
  __shared__ R sh_tot[PA_N][FDA_CELLS];
  __shared__ R sh_Y[MAX_SP][FDA_CELLS];
  __shared__ R sh_rhob[FDA_CELLS];
  const FDArgs<R>& a = A.f;
  const FDConst<R>& c = a.c;
  const Geo& g = a.geo;
  const int N = g.N, K = c.K;
  const int tx = threadIdx.x, fi = threadIdx.y;
  const int r = blockIdx.x * FDA_CELLS + tx;
  const uint32_t sw = r < N ? __ldg(a.sword + r) : 0u;
  const bool act = (sw >> 31) != 0u;  // every thread reaches the barriers below
  const int x = r % g.nx, y = r / g.nx;
  FDStencil2 S;
  fd_stencil2(g, sw, r, x, y, S);
  // adjoint of rho^n from the LB step: own part and the density-gradient parts of the cells that
  // hold this cell as their -x / +x / -y / +y neighbour (zero where that cell is solid or mirrored)
  if (act && fi == (K > 0 ? 1 : 0)) {
    R rhob = A.rho_own[r];
    const int xm = x > 0 ? r - 1 : (g.bc_lo[0] == BC_PERIODIC ? r + g.nx - 1 : -1);
    const int xp = x < g.nx - 1 ? r + 1 : (g.bc_hi[0] == BC_PERIODIC ? r - g.nx + 1 : -1);
    const int ym = y > 0 ? r - g.nx : (g.bc_lo[1] == BC_PERIODIC ? r + (g.ny - 1) * g.nx : -1);
    const int yp = y < g.ny - 1 ? r + g.nx : (g.bc_hi[1] == BC_PERIODIC ? r - (g.ny - 1) * g.nx : -1);
    if (xm >= 0) rhob += A.rho_nb[xm];
    if (xp >= 0) rhob += A.rho_nb[N + xp];
    if (ym >= 0) rhob += A.rho_nb[2 * N + ym];
    if (yp >= 0) rhob += A.rho_nb[3 * N + yp];
    sh_rhob[tx] = rhob;
  }

  // ------------------------------------------------------------ forward: shared quantities
  R Tr = R(1), W = R(1), rho = R(1), rho_phys = R(1), inv_rho = R(1);
  const R F = c.F;
  const R fdr = sizeof(R) == 4 ? (R)a.pth->fd_rho : (R)a.pth->fd_rho_d;
  R Tn[2][2];
  if (act) {
    Tr = a.T[r];
    R sW = R(0);
    for (int k = 0; k < K; ++k) sW += a.Y[(size_t)k * N + r] * c.inv_W[k];
    W = R(1) / sW;
    rho = fdr * W / Tr;
    rho_phys = rho / c.inv_rho_ref;
    inv_rho = R(1) / rho;
#pragma unroll
    for (int ax = 0; ax < 2; ++ax)
#pragma unroll
      for (int sd = 0; sd < 2; ++sd) {
        const int kk = S.k1[ax][sd];
        Tn[ax][sd] = kk == NB_FLUID ? a.T[S.i1[ax][sd]] : (kk == NB_INLET ? c.T_in : Tr);
      }
    // transcendental work shared out over the cell's threads: task 0 the rates, task 1 mu(T_r),
    // tasks 2..5 mu at the distance-1 points
    for (int t = fi; t < 6; t += K + 1) {
      if (t == 0) {
#pragma unroll
        for (int j = 0; j < MAX_RX; ++j)
          if (j < c.nrx) sh_q[j][tx] = rate_of<R>(c, j, Tr, a.Y, N, r, rho_phys);
      } else {
        const R Tt = t == 1 ? Tr : Tn[(t - 2) >> 1][(t - 2) & 1];
        sh_mu[t - 1][tx] = c.nu_lat * powr<R>(Tt * c.T_ref_inv, c.mu_exp);
      }
    }
  }
  __syncthreads();
  R q[MAX_RX], mun[2][2], FMf[2][2], uf[2][2], ur[2] = {R(0), R(0)};
  R mur = R(0), inv_rpF = R(0), qdot = R(0);
  if (act) {
#pragma unroll
    for (int j = 0; j < MAX_RX; ++j) {
      q[j] = j < c.nrx ? sh_q[j][tx] : R(0);
      qdot += c.heat[j] * q[j];
    }
    mur = sh_mu[0][tx];
    ur[0] = a.u[r];
    ur[1] = a.u[N + r];
#pragma unroll
    for (int ax = 0; ax < 2; ++ax)
#pragma unroll
      for (int sd = 0; sd < 2; ++sd) {
        const int kk = S.k1[ax][sd], j = S.i1[ax][sd];
        mun[ax][sd] = sh_mu[1 + 2 * ax + sd][tx];
        FMf[ax][sd] = R(0.5) * (F * mur + F * mun[ax][sd]);
        R un;
        if (kk == NB_FLUID) un = a.u[ax * N + j];
        else if (kk == NB_INLET) un = a.inlet_u[ax * g.ny + y];
        else if (kk == NB_OUTLET) un = ur[ax];
        else un = R(0);
        uf[ax][sd] = R(0.5) * (ur[ax] + un);
      }
    inv_rpF = R(1) / (rho_phys * F);
  }
  const R dt = c.dt_phys;

  // ------------------------------------------------------------- this thread's field
  // pointb: adjoints of the 9 stencil values (slot order), constant indices only
  R pointb[9];
#pragma unroll
  for (int p = 0; p < 9; ++p) pointb[p] = R(0);
  R pa[PA_N];
#pragma unroll
  for (int p = 0; p < PA_N; ++p) pa[p] = R(0);
  if (act) {
    const R* phi = fi == 0 ? a.T : a.Y + (size_t)(fi - 1) * N;
    const R phin = fi == 0 ? c.T_in : c.Y_in[fi - 1];
    const R eps = fi == 0 ? c.eps_T : c.eps_Y;
    const R gfac = c.inv_Pr * (fi == 0 ? R(1) : c.inv_Le[fi - 1]);
    const R pr = phi[r];
    if (fi > 0) sh_Y[fi - 1][tx] = pr;
    R pm2[2], pm1[2], pp1[2], pp2[2];
    R dif = R(0);
#pragma unroll
    for (int ax = 0; ax < 2; ++ax) {
      pm2[ax] = S.k2[ax][0] == 2 ? phin : phi[S.i2[ax][0]];
      pm1[ax] = S.k1[ax][0] == NB_INLET ? phin : phi[S.i1[ax][0]];
      pp1[ax] = S.k1[ax][1] == NB_INLET ? phin : phi[S.i1[ax][1]];
      pp2[ax] = S.k2[ax][1] == 2 ? phin : phi[S.i2[ax][1]];
      dif += FMf[ax][1] * (pp1[ax] - pr) - FMf[ax][0] * (pr - pm1[ax]);
    }
    R om = R(0), src;
    if (fi == 0) {
      src = dt * qdot * inv_rpF * c.inv_cp;
    } else {
#pragma unroll
      for (int j = 0; j < MAX_RX; ++j) om += c.nu[j][fi - 1] * q[j];
      src = dt * c.W[fi - 1] * om * inv_rpF;
    }
    const R NA = gfac * inv_rho * dif + src;
    // reverse. Lambda = NA_T / T + sum_k W / W_k NA_k; out = phi - adv + NA
    const R lamb = A.lam_bar[r];
    const R outb = fi == 0 ? A.Tbar_out[r] : A.Ybar_out[(size_t)(fi - 1) * N + r];
    R NAb;
    if (fi == 0) {
      pa[PA_TR] = -lamb * NA / (Tr * Tr);
      NAb = outb + lamb / Tr;
    } else {
      pa[PA_W] = lamb * c.inv_W[fi - 1] * NA;
      NAb = outb + lamb * W * c.inv_W[fi - 1];
    }
    pointb[0] = outb;
    pa[PA_INVRHO] = NAb * gfac * dif;
    const R gi = NAb * gfac * inv_rho;
#pragma unroll
    for (int ax = 0; ax < 2; ++ax) {
      const R m2 = pm2[ax], m1 = pm1[ax], p1 = pp1[ax], p2 = pp2[ax];
      R m2b = R(0), m1b = R(0), p1b = R(0), p2b = R(0), prb = R(0);
      pa[PA_FM + 2 * ax + 1] += gi * (p1 - pr);
      pa[PA_FM + 2 * ax] -= gi * (pr - m1);
      p1b += gi * FMf[ax][1];
      prb -= gi * (FMf[ax][1] + FMf[ax][0]);
      m1b += gi * FMf[ax][0];
      const bool up = uf[ax][1] >= R(0), um = uf[ax][0] >= R(0);
      const R dm2 = m1 - m2, dm1 = pr - m1, dp1 = p1 - pr, dp2 = p2 - p1;
      const R fp = up ? weno_face<R>(pr, dm1, dp1, eps) : weno_face<R>(p1, -dp2, -dp1, eps);
      const R fm = um ? weno_face<R>(m1, dm2, dm1, eps) : weno_face<R>(pr, -dp1, -dm1, eps);
      const R advb = -outb;
      pa[PA_UR + ax] += advb * (fp - fm);
      const R fpb = advb * ur[ax], fmb = -advb * ur[ax];
      R bb, dab, dbc;
      if (up) {
        weno_face_rev<R>(dm1, dp1, eps, fpb, bb, dab, dbc);
        prb += bb + dab - dbc; m1b -= dab; p1b += dbc;
      } else {
        weno_face_rev<R>(-dp2, -dp1, eps, fpb, bb, dab, dbc);
        p1b += bb + dab - dbc; p2b -= dab; prb += dbc;
      }
      if (um) {
        weno_face_rev<R>(dm2, dm1, eps, fmb, bb, dab, dbc);
        m1b += bb + dab - dbc; m2b -= dab; prb += dbc;
      } else {
        weno_face_rev<R>(-dp1, -dm1, eps, fmb, bb, dab, dbc);
        prb += bb + dab - dbc; p1b -= dab; m1b += dbc;
      }
      pointb[0] += prb;
      // distance-1 points: a fluid neighbour's slot, the cell itself (zero-gradient ghost) or
      // nothing (inlet constant); distance-2 points likewise, or the distance-1 point they copy
#pragma unroll
      for (int sd = 0; sd < 2; ++sd) {
        const R v1 = sd ? p1b : m1b, v2 = sd ? p2b : m2b;
        const int kk1 = S.k1[ax][sd], kk2 = S.k2[ax][sd];
        const R to1 = v1 + (kk2 == 1 ? v2 : R(0));
        if (kk1 == NB_FLUID) pointb[slot1(ax, sd)] += to1;
        else if (kk1 != NB_INLET) pointb[0] += to1;
        if (kk2 == 0) pointb[slot2(ax, sd)] += v2;
      }
    }
    if (fi == 0) {
      pa[PA_QDOT] = NAb * dt * inv_rpF * c.inv_cp;
      pa[PA_INVRPF] = NAb * dt * qdot * c.inv_cp;
    } else {
      const R omb = NAb * dt * c.W[fi - 1] * inv_rpF;
      pa[PA_INVRPF] = NAb * dt * c.W[fi - 1] * om;
#pragma unroll
      for (int j = 0; j < MAX_RX; ++j) pa[PA_Q + j] = c.nu[j][fi - 1] * omb;
    }
  }
#pragma unroll
  for (int p = 0; p < PA_N; ++p) part[fi][p][tx] = pa[p];
  __syncthreads();
  // field sums of the partial adjoints, spread over the block's warps
  if (act)
    for (int p = fi; p < PA_N; p += K + 1) {
      R v = R(0);
      for (int f = 0; f <= K; ++f) v += part[f][p][tx];
      sh_tot[p][tx] = v;
    }
  __syncthreads();
  // ---------------------- shared terms, once per cell (thread fi = 0): sums over the fields,
  // reverse of the rate law, rho = P W / (R T), W and mu(T); the center adjoint of each species
  // goes to the field threads through shared memory
  __shared__ R sh_add[MAX_SP][FDA_CELLS];
  if (act && fi == 0) {
    R tot[PA_N];
#pragma unroll
    for (int p = 0; p < PA_N; ++p) tot[p] = sh_tot[p][tx];
    R Trb = tot[PA_TR], Wb = tot[PA_W];
    R rho_physb = -tot[PA_INVRPF] * inv_rpF / rho_phys;
    for (int k = 0; k < K; ++k) sh_add[k][tx] = R(0);
#pragma unroll
    for (int j = 0; j < MAX_RX; ++j) {
      if (j >= c.nrx) break;
      const R qq = q[j] * (tot[PA_Q + j] + c.heat[j] * tot[PA_QDOT]);
      Trb += qq * ((c.ER_hi[j] + c.ER_lo[j]) / (Tr * Tr) + c.beta[j] / Tr);
#pragma unroll
      for (int m = 0; m < MAX_ORD; ++m) {
        if (m >= c.nord[j]) break;
        const int k = c.ord_k[j][m];
        const R yk = sh_Y[k][tx];
        if (yk > R(0)) {
          rho_physb += qq * c.ord_n[j][m] / rho_phys;
          sh_add[k][tx] += qq * c.ord_n[j][m] / yk;
        }
      }
    }
    // adjoint of rho^n: from the LB step (staged above) and this update
    R rhob = sh_rhob[tx];
    rhob += rho_physb / c.inv_rho_ref;
    rhob -= tot[PA_INVRHO] * inv_rho * inv_rho;
    Wb += rhob * fdr / Tr;
    Trb -= rhob * rho / Tr;
    const R sWb = -Wb * W * W;
    for (int k = 0; k < K; ++k) sh_add[k][tx] += sWb * c.inv_W[k];
    // face coefficients FM = F (mu_r + mu_n) / 2, mu = nu (T / T_ref)^mu_exp
    R murb = R(0);
#pragma unroll
    for (int ax = 0; ax < 2; ++ax)
#pragma unroll
      for (int sd = 0; sd < 2; ++sd) {
        const R munb = R(0.5) * F * tot[PA_FM + 2 * ax + sd];
        murb += munb;
        const R dmu = munb * c.mu_exp * mun[ax][sd] / Tn[ax][sd];
        const int kk = S.k1[ax][sd];
        if (kk == NB_FLUID) pointb[slot1(ax, sd)] += dmu;
        else if (kk != NB_INLET) Trb += dmu;
      }
    Trb += murb * c.mu_exp * mur / Tr;
    pointb[0] += Trb;
    A.u_bar[r] = tot[PA_UR];
    A.u_bar[N + r] = tot[PA_UR + 1];
  }
  __syncthreads();
  if (!act) return;
  if (fi > 0) pointb[0] += sh_add[fi - 1][tx];
  const size_t fs = (size_t)(K + 1) * N;  // stride between slots
  R* out = A.slots + (size_t)fi * N + r;
#pragma unroll
  for (int p = 0; p < 9; ++p) out[(size_t)p * fs] = pointb[p];
}

// Sum of the slot adjoints for every (cell, field): the cell's own center slot plus the
// distance-1 and distance-2 slots of the cells whose stencil points land on it. Same thread
// layout as fd_adjoint_kernel; the field-0 thread of each cell finds those cells once.
template <typename R>
__global__ void __launch_bounds__(FDA_THREADS)
    fd_adjoint_gather(Geo g, const uint32_t* __restrict__ sword, int K, const R* __restrict__ slots,
                      const R* __restrict__ T_lb, const R* __restrict__ u_fd, const R* __restrict__ u_lb,
                      R* __restrict__ Tbar, R* __restrict__ Ybar, R* __restrict__ ubar) {
  __shared__ int src[8][FDA_CELLS];  // cell whose (axis, side, distance) point is s, or -1
  const int tx = threadIdx.x, fi = threadIdx.y;
  const int s = blockIdx.x * FDA_CELLS + tx;
  const int N = g.N;
  const bool inside = s < N;
  const bool fluid = inside && (__ldg(sword + s) >> 31);
  if (fi == 0 && fluid) {
    const int x = s % g.nx, y = s / g.nx;
    const int pos[2] = {x, y}, dims[2] = {g.nx, g.ny}, strides[2] = {1, g.nx};
#pragma unroll
    for (int ax = 0; ax < 2; ++ax)
#pragma unroll
      for (int sd = 0; sd < 2; ++sd) {
        const int sg = sd ? 1 : -1;
        const bool per = g.bc_lo[ax] == BC_PERIODIC;
#pragma unroll
        for (int dist = 1; dist <= 2; ++dist) {
          int qd = pos[ax] - dist * sg;
          bool ok = true;
          if (qd < 0 || qd >= dims[ax]) {
            if (per) qd = ((qd % dims[ax]) + dims[ax]) % dims[ax];
            else ok = false;
          }
          int rc = -1;
          if (ok) {
            // that cell's stencil point is s only when the point is a real (fluid) neighbour
            const int cand = s + (qd - pos[ax]) * strides[ax];
            const uint32_t w = __ldg(sword + cand);
            if ((w >> 31) && ((w >> (4 * (2 * ax + sd) + 2 * (dist - 1))) & 3u) == 0u) rc = cand;
          }
          src[2 * (2 * ax + sd) + dist - 1][tx] = rc;
        }
      }
  }
  __syncthreads();
  if (!inside || fi > K) return;
  R* dst = fi == 0 ? Tbar + s : Ybar + (size_t)(fi - 1) * N + s;
  if (!fluid) {
    *dst = R(0);
    if (fi == 0) {
      ubar[s] = R(0);
      ubar[N + s] = R(0);
    }
    return;
  }
  const size_t fs = (size_t)(K + 1) * N;
  const R* sl = slots + (size_t)fi * N;
  R v = sl[s];
#pragma unroll
  for (int t = 0; t < 8; ++t) {
    const int rc = src[t][tx];
    if (rc >= 0) v += sl[(size_t)(1 + t) * fs + rc];  // slot 1 + t: distance 1 + (t & 1), side t >> 1
  }
  if (fi == 0) {
    *dst = v + T_lb[s];
    ubar[s] = u_fd[s] + u_lb[s];
    ubar[N + s] = u_fd[N + s] + u_lb[N + s];
  } else {
    *dst = v;
  }
}

}  // namespace hlbm
