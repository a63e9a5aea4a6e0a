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
  const R Nb = fb * R(0.5) / Dn;
  const R Db = -fb * R(0.5) * Nn / (Dn * Dn);
  const R tabb = Nb * R(2) * dbc + Db * R(2);
  const R tbcb = Nb * dab + Db;
  bb = fb;
  dabb = Nb * tbc + tabb * R(4) * dab * sab;
  dbcb = Nb * R(2) * tab + tbcb * R(4) * dbc * sbc;
}
template <typename R> __device__ __forceinline__ R weno_face(R b, R dab, R dbc, R eps) {
  const R sab = dab * dab + eps, sbc = dbc * dbc + eps;
  const R tab = sab * sab, tbc = sbc * sbc;
  return b + R(0.5) * (tbc * dab + R(2) * tab * dbc) / (tbc + R(2) * tab);
}

// slot numbering: 0 center, 1 + 2*(2a+s) distance-1 point, 2 + 2*(2a+s) distance-2 point
__device__ __forceinline__ int slot1(int ax, int sd) { return 1 + 2 * (2 * ax + sd); }
__device__ __forceinline__ int slot2(int ax, int sd) { return 2 + 2 * (2 * ax + sd); }

template <typename R>
__global__ void __launch_bounds__(FD_BLOCK) fd_adjoint_kernel(const FDAdjArgs<R> A) {
  const FDArgs<R>& a = A.f;
  const FDConst<R>& c = a.c;
  const Geo& g = a.geo;
  const int r = blockIdx.x * FD_BLOCK + threadIdx.x;
  if (r >= g.N) return;
  const uint32_t sw = __ldg(a.sword + r);
  if (!(sw >> 31)) return;
  const int N = g.N;
  const int K = c.K;
  const int x = r % g.nx, y = r / g.nx;
  const int pos[2] = {x, y}, dims[2] = {g.nx, g.ny}, strides[2] = {1, g.nx};
  int k1[2][2], k2[2][2], i1[2][2], i2[2][2];
#pragma unroll
  for (int ax = 0; ax < 2; ++ax)
#pragma unroll
    for (int sd = 0; sd < 2; ++sd) {
      const uint32_t bits = (sw >> (4 * (2 * ax + sd))) & 15u;
      k1[ax][sd] = (int)(bits & 3u);
      k2[ax][sd] = (int)(bits >> 2);
      const int sg = sd ? 1 : -1;
      int p1 = pos[ax] + sg;
      p1 = p1 < 0 ? p1 + dims[ax] : (p1 >= dims[ax] ? p1 - dims[ax] : p1);
      int p2 = p1 + sg;
      p2 = p2 < 0 ? p2 + dims[ax] : (p2 >= dims[ax] ? p2 - dims[ax] : p2);
      const int j1 = k1[ax][sd] == NB_FLUID ? r + (p1 - pos[ax]) * strides[ax] : r;
      i1[ax][sd] = j1;
      i2[ax][sd] = k2[ax][sd] == 0 ? r + (p2 - pos[ax]) * strides[ax] : j1;
    }
  // target slot of the adjoint of each stencil point (fold ghosts onto the cell they copy)
  int t1s[2][2], t2s[2][2];
#pragma unroll
  for (int ax = 0; ax < 2; ++ax)
#pragma unroll
    for (int sd = 0; sd < 2; ++sd) {
      t1s[ax][sd] = k1[ax][sd] == NB_FLUID ? slot1(ax, sd) : (k1[ax][sd] == NB_INLET ? -1 : 0);
      if (k2[ax][sd] == 0) t2s[ax][sd] = slot2(ax, sd);
      else if (k2[ax][sd] == 2) t2s[ax][sd] = -1;
      else t2s[ax][sd] = t1s[ax][sd];
    }

  // ------------------------------------------------------------ forward: shared quantities
  const R Tr = a.T[r];
  R Yr[MAX_SP];
  R sW = R(0);
  for (int k = 0; k < K; ++k) {
    Yr[k] = a.Y[k * N + r];
    sW += Yr[k] * c.inv_W[k];
  }
  const R W = R(1) / sW;
  const R fdr = sizeof(R) == 4 ? (R)a.pth->fd_rho : (R)a.pth->fd_rho_d;
  const R rho = fdr * W / Tr;
  const R rho_phys = rho / c.inv_rho_ref;
  const R inv_rho = R(1) / rho;
  R q[MAX_RX];
  for (int j = 0; j < c.nrx; ++j) {
    R v = c.A[j] * exp(-(c.ER_hi[j] + c.ER_lo[j]) / Tr);
    if (c.beta[j] != R(0)) v *= pow(Tr, c.beta[j]);
    for (int m = 0; m < c.nord[j]; ++m) {
      const int k = c.ord_k[j][m];
      const R y = Yr[k];
      v *= y > R(0) ? pow(rho_phys * y * c.inv_W[k], c.ord_n[j][m]) : R(0);
    }
    q[j] = v;
  }
  const R F = c.F;
  const R mur = c.nu_lat * pow(Tr * c.T_ref_inv, c.mu_exp);
  const R ur[2] = {a.u[r], a.u[N + r]};
  const int f = y;
  R FMf[2][2], uf[2][2], Tn[2][2], mun[2][2];
#pragma unroll
  for (int ax = 0; ax < 2; ++ax)
#pragma unroll
    for (int sd = 0; sd < 2; ++sd) {
      const int kk = k1[ax][sd], j = i1[ax][sd];
      Tn[ax][sd] = kk == NB_FLUID ? a.T[j] : (kk == NB_INLET ? c.T_in : Tr);
      mun[ax][sd] = c.nu_lat * pow(Tn[ax][sd] * c.T_ref_inv, c.mu_exp);
      FMf[ax][sd] = R(0.5) * (F * mur + F * mun[ax][sd]);
      R un;
      if (kk == NB_FLUID) un = a.u[ax * N + j];
      else if (kk == NB_INLET) un = a.inlet_u[ax * g.ny + f];
      else if (kk == NB_OUTLET) un = ur[ax];
      else un = R(0);
      uf[ax][sd] = R(0.5) * (ur[ax] + un);
    }
  const R dt = c.dt_phys;
  const R inv_rpF = R(1) / (rho_phys * F);
  R qdot = R(0);
  for (int j = 0; j < c.nrx; ++j) qdot += c.heat[j] * q[j];

  // per-field values: NA and the diffusion sum, needed by the Lambda reverse
  R NAv[MAX_SP + 1], difs[MAX_SP + 1];
  for (int fi = 0; fi <= K; ++fi) {
    const R* phi = fi == 0 ? a.T : a.Y + (size_t)(fi - 1) * N;
    const R phin = fi == 0 ? c.T_in : c.Y_in[fi - 1];
    const R gfac = c.inv_Pr * (fi == 0 ? R(1) : c.inv_Le[fi - 1]);
    const R pr = phi[r];
    R dif = R(0);
    for (int ax = 0; ax < 2; ++ax) {
      const R m1 = k1[ax][0] == NB_INLET ? phin : phi[i1[ax][0]];
      const R p1 = k1[ax][1] == NB_INLET ? phin : phi[i1[ax][1]];
      dif += FMf[ax][1] * (p1 - pr) - FMf[ax][0] * (pr - m1);
    }
    difs[fi] = dif;
    R src;
    if (fi == 0) {
      src = dt * qdot * inv_rpF * c.inv_cp;
    } else {
      R om = R(0);
      for (int j = 0; j < c.nrx; ++j) om += c.nu[j][fi - 1] * q[j];
      src = dt * c.W[fi - 1] * om * inv_rpF;
    }
    NAv[fi] = gfac * inv_rho * dif + src;
  }

  // ------------------------------------------------------------------------- reverse
  const R lamb = A.lam_bar[r];
  // adjoint of rho^n: the cell's own part plus the density-gradient parts of the cells that
  // hold it as their -x / +x / -y / +y neighbour (zero where that cell is solid or mirrored it)
  R rhob = A.rho_own[r];
  {
    const int xm = x > 0 ? r - 1 : (g.bc_lo[0] == BC_PERIODIC ? r + g.nx - 1 : -1);
    const int xp = x < g.nx - 1 ? r + 1 : (g.bc_hi[0] == BC_PERIODIC ? r - g.nx + 1 : -1);
    const int ym = y > 0 ? r - g.nx : (g.bc_lo[1] == BC_PERIODIC ? r + (g.ny - 1) * g.nx : -1);
    const int yp = y < g.ny - 1 ? r + g.nx : (g.bc_hi[1] == BC_PERIODIC ? r - (g.ny - 1) * g.nx : -1);
    if (xm >= 0) rhob += A.rho_nb[xm];
    if (xp >= 0) rhob += A.rho_nb[N + xp];
    if (ym >= 0) rhob += A.rho_nb[2 * N + ym];
    if (yp >= 0) rhob += A.rho_nb[3 * N + yp];
  }
  R Trb = R(0), Wb = R(0), inv_rhob = R(0), inv_rpFb = R(0), qdotb = R(0);
  R qb[MAX_RX];
  for (int j = 0; j < MAX_RX; ++j) qb[j] = R(0);
  R Ycb[MAX_SP];  // center adjoint of Y from shared terms
  for (int k = 0; k < MAX_SP; ++k) Ycb[k] = R(0);
  R FMb[2][2] = {{R(0), R(0)}, {R(0), R(0)}};
  R urb[2] = {R(0), R(0)};
  // Lambda = NA_T / T + sum_k W / W_k NA_k
  Trb -= lamb * NAv[0] / (Tr * Tr);
  for (int k = 0; k < K; ++k) Wb += lamb * c.inv_W[k] * NAv[k + 1];

  for (int fi = 0; fi <= K; ++fi) {
    const R* phi = fi == 0 ? a.T : a.Y + (size_t)(fi - 1) * N;
    const R phin = fi == 0 ? c.T_in : c.Y_in[fi - 1];
    const R eps = fi == 0 ? c.eps_T : c.eps_Y;
    const R gfac = c.inv_Pr * (fi == 0 ? R(1) : c.inv_Le[fi - 1]);
    const R outb = fi == 0 ? A.Tbar_out[r] : A.Ybar_out[(size_t)(fi - 1) * N + r];
    const R NAb = outb + (fi == 0 ? lamb / Tr : lamb * W * c.inv_W[fi - 1]);
    R pointb[9];
#pragma unroll
    for (int p = 0; p < 9; ++p) pointb[p] = R(0);
    pointb[0] = outb;  // out = pr - adv + NA
    const R pr = phi[r];
    // diffusion: NA += gfac inv_rho sum_a (FMp dp1 - FMm dm1)
    inv_rhob += NAb * gfac * difs[fi];
    const R gi = NAb * gfac * inv_rho;
    for (int ax = 0; ax < 2; ++ax) {
      const R m2 = k2[ax][0] == 2 ? phin : phi[i2[ax][0]];
      const R m1 = k1[ax][0] == NB_INLET ? phin : phi[i1[ax][0]];
      const R p1 = k1[ax][1] == NB_INLET ? phin : phi[i1[ax][1]];
      const R p2 = k2[ax][1] == 2 ? phin : phi[i2[ax][1]];
      R m2b = R(0), m1b = R(0), p1b = R(0), p2b = R(0), prb = R(0);
      FMb[ax][1] += gi * (p1 - pr);
      FMb[ax][0] -= gi * (pr - m1);
      p1b += gi * FMf[ax][1];
      prb -= gi * FMf[ax][1];
      prb -= gi * FMf[ax][0];
      m1b += gi * FMf[ax][0];
      // advection: out -= ur (fp - fm)
      const bool up = uf[ax][1] >= R(0), um = uf[ax][0] >= R(0);
      const R dm2 = m1 - m2, dm1 = pr - m1, dp1 = p1 - pr, dp2 = p2 - p1;
      const R fp = up ? weno_face<R>(pr, dm1, dp1, eps) : weno_face<R>(p1, -dp2, -dp1, eps);
      const R fm = um ? weno_face<R>(m1, dm2, dm1, eps) : weno_face<R>(pr, -dp1, -dm1, eps);
      const R advb = -outb;
      urb[ax] += advb * (fp - fm);
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
      if (t1s[ax][0] >= 0) pointb[t1s[ax][0]] += m1b;
      if (t1s[ax][1] >= 0) pointb[t1s[ax][1]] += p1b;
      if (t2s[ax][0] >= 0) pointb[t2s[ax][0]] += m2b;
      if (t2s[ax][1] >= 0) pointb[t2s[ax][1]] += p2b;
    }
    // sources
    if (fi == 0) {
      qdotb += NAb * dt * inv_rpF * c.inv_cp;
      inv_rpFb += NAb * dt * qdot * c.inv_cp;
    } else {
      R om = R(0);
      for (int j = 0; j < c.nrx; ++j) om += c.nu[j][fi - 1] * q[j];
      const R omb = NAb * dt * c.W[fi - 1] * inv_rpF;
      inv_rpFb += NAb * dt * c.W[fi - 1] * om;
      for (int j = 0; j < c.nrx; ++j) qb[j] += c.nu[j][fi - 1] * omb;
    }
    // the center adjoint of the shared terms (rho, W, chemistry) is added after the loop
#pragma unroll
    for (int p = 0; p < 9; ++p) A.slots[((size_t)p * (K + 1) + fi) * N + r] = pointb[p];
  }
  // chemistry and shared terms
  for (int j = 0; j < c.nrx; ++j) qb[j] += c.heat[j] * qdotb;
  R rho_physb = -inv_rpFb * inv_rpF / rho_phys;
  for (int j = 0; j < c.nrx; ++j) {
    const R qq = q[j] * qb[j];
    Trb += qq * ((c.ER_hi[j] + c.ER_lo[j]) / (Tr * Tr) + c.beta[j] / Tr);
    for (int m = 0; m < c.nord[j]; ++m) {
      const int k = c.ord_k[j][m];
      if (Yr[k] > R(0)) {
        rho_physb += qq * c.ord_n[j][m] / rho_phys;
        Ycb[k] += qq * c.ord_n[j][m] / Yr[k];
      }
    }
  }
  rhob += rho_physb / c.inv_rho_ref;
  rhob -= inv_rhob * inv_rho * inv_rho;
  Wb += rhob * fdr / Tr;
  Trb -= rhob * rho / Tr;
  const R sWb = -Wb * W * W;
  for (int k = 0; k < K; ++k) Ycb[k] += sWb * c.inv_W[k];
  // face coefficients: FM = F (mu_r + mu_n) / 2
  R murb = R(0);
#pragma unroll
  for (int ax = 0; ax < 2; ++ax)
#pragma unroll
    for (int sd = 0; sd < 2; ++sd) {
      murb += R(0.5) * F * FMb[ax][sd];
      const R munb = R(0.5) * F * FMb[ax][sd];
      const R dmu = munb * c.mu_exp * mun[ax][sd] / Tn[ax][sd];
      const int kk = k1[ax][sd];
      if (kk == NB_FLUID) A.slots[((size_t)slot1(ax, sd) * (K + 1) + 0) * N + r] += dmu;
      else if (kk != NB_INLET) Trb += dmu;
    }
  Trb += murb * c.mu_exp * mur / Tr;
  A.slots[(size_t)0 * N + r] += Trb;
  for (int k = 0; k < K; ++k) A.slots[((size_t)(k + 1)) * N + r] += Ycb[k];
  A.u_bar[r] = urb[0];
  A.u_bar[N + r] = urb[1];
}

// Sum of the slot adjoints for every cell: its own center slot plus the distance-1 and
// distance-2 slots of the cells whose stencil points land on it.
template <typename R>
__global__ void fd_adjoint_gather(Geo g, const uint32_t* __restrict__ sword, int K, const R* __restrict__ slots,
                                  const R* __restrict__ T_lb, const R* __restrict__ u_fd,
                                  const R* __restrict__ u_lb, R* __restrict__ Tbar, R* __restrict__ Ybar,
                                  R* __restrict__ ubar) {
  const int s = blockIdx.x * FD_BLOCK + threadIdx.x;
  if (s >= g.N) return;
  const int N = g.N;
  if (!(__ldg(sword + s) >> 31)) {
    Tbar[s] = R(0);
    for (int k = 0; k < K; ++k) Ybar[(size_t)k * N + s] = R(0);
    ubar[s] = R(0);
    ubar[N + s] = R(0);
    return;
  }
  const int x = s % g.nx, y = s / g.nx;
  const int pos[2] = {x, y}, dims[2] = {g.nx, g.ny}, strides[2] = {1, g.nx};
  const int lo[2] = {g.bc_lo[0], g.bc_lo[1]};
  // cells whose distance-1 / distance-2 point on side sd of axis ax is s
  int c1[2][2], c2[2][2];
#pragma unroll
  for (int ax = 0; ax < 2; ++ax)
#pragma unroll
    for (int sd = 0; sd < 2; ++sd) {
      const int sg = sd ? 1 : -1;
      const bool per = lo[ax] == BC_PERIODIC;
      int q1 = pos[ax] - sg, q2 = pos[ax] - 2 * sg;
      bool ok1 = true, ok2 = true;
      if (q1 < 0 || q1 >= dims[ax]) { if (per) q1 = (q1 + dims[ax]) % dims[ax]; else ok1 = false; }
      if (q2 < 0 || q2 >= dims[ax]) { if (per) q2 = ((q2 % dims[ax]) + dims[ax]) % dims[ax]; else ok2 = false; }
      int r1 = ok1 ? s + (q1 - pos[ax]) * strides[ax] : -1;
      int r2 = ok2 ? s + (q2 - pos[ax]) * strides[ax] : -1;
      // the cell's stencil point is s only when that point is a real (fluid) neighbour
      if (r1 >= 0) {
        const uint32_t w = __ldg(sword + r1);
        if (!(w >> 31) || ((w >> (4 * (2 * ax + sd))) & 3u) != 0u) r1 = -1;
      }
      if (r2 >= 0) {
        const uint32_t w = __ldg(sword + r2);
        if (!(w >> 31) || ((w >> (4 * (2 * ax + sd) + 2)) & 3u) != 0u) r2 = -1;
      }
      c1[ax][sd] = r1;
      c2[ax][sd] = r2;
    }
  for (int fi = 0; fi <= K; ++fi) {
    R v = slots[((size_t)0 * (K + 1) + fi) * N + s];
#pragma unroll
    for (int ax = 0; ax < 2; ++ax)
#pragma unroll
      for (int sd = 0; sd < 2; ++sd) {
        if (c1[ax][sd] >= 0) v += slots[((size_t)slot1(ax, sd) * (K + 1) + fi) * N + c1[ax][sd]];
        if (c2[ax][sd] >= 0) v += slots[((size_t)slot2(ax, sd) * (K + 1) + fi) * N + c2[ax][sd]];
      }
    if (fi == 0) Tbar[s] = v + T_lb[s];
    else Ybar[(size_t)(fi - 1) * N + s] = v;
  }
  ubar[s] = u_fd[s] + u_lb[s];
  ubar[N + s] = u_fd[N + s] + u_lb[N + s];
}

}  // namespace hlbm
