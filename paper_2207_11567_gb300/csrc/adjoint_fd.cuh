// Adjoint (reverse mode) of the 2-D finite-difference update of fd_kernel.cuh (open domain,
// constant thickening factor): WENO3 faces, centred diffusion, chemistry, rho and Lambda. The
// adjoint step is not in the paper; it is the exact transpose of the discrete update written by
// hand. Upwind choices and the max(Y, 0) of the rate law are held fixed (their derivative is 0).
//
// One thread per fluid cell recomputes its forward update and reverses it, field after field,
// writing the adjoint of every stencil value it read into one of 9 slots per field (center,
// distance-1 and distance-2 points on each side of each axis); a ghost value's adjoint is folded
// onto the cell it copies (inlet values are constants). The adjoint of a cell's T and Y_k is the
// sum of its own center slot and the slots of the cells whose stencils contain it: the next
// reverse step forms that sum for its own cell as it starts (slot form, double-buffered), and
// fd_adjoint_gather forms it for every cell where a reverse sweep ends.
#pragma once
#include "common.cuh"
#include "fd_kernel.cuh"

namespace hlbm {

template <typename R> struct FDAdjArgs {
  FDArgs<R> f;           // forward arguments of state n (T, Y, u, stencil words, constants)
  const R* Tbar_out;     // [N] adjoint of T^{n+1}, or null: slot form in slots_in
  const R* Ybar_out;     // [K][N] adjoint of Y^{n+1} (with Tbar_out)
  const R* slots_in;     // [9][1+K][N] slot form of the adjoint of T^{n+1}, Y^{n+1}
  const R* rho_own;      // [N] adjoint of rho^n used by the cell's own LB update
  const R* rho_nb;       // [4][N] adjoint of the +x, -x, +y, -y neighbour rho in a cell's LB update
  const R* lam_bar;      // [N] adjoint of Lambda^n (from the LB adjoint)
  const R* T_lb;         // [N] adjoint of T^n through the LB step's viscosity law
  const R* u_lb;         // [2][N] adjoint of u^n through the LB step's outlet rule
  R* slots;              // [9][1+K][N] stencil-value adjoints of this step (slot form of T^n, Y^n)
  R* u_out;              // [2][N] adjoint of u^n: advection part plus u_lb (0 on solid cells)
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

constexpr int FDA_BLOCK = 64;
// partial adjoints of the quantities the fields share, summed over the fields
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


// Cells whose stencil point (axis, side, distance) is the fluid cell s: src[2 (2 ax + sd) + dist - 1]
// is that cell, or -1 where it is not fluid or its point there is a ghost. Its slot 1 + t holds the
// adjoint of s read through that point. The stencil kinds are symmetric (a point is a real fluid
// point when both cells are fluid and inside the domain or across a periodic face), so s's own
// word tells: the cell at distance 1 (2) on the opposite side has s as its point exactly when s's
// distance-1 point (distance-1 and distance-2 points) on that side are real.
__device__ __forceinline__ void slot_sources(const Geo& g, uint32_t sw, int s, int x, int y, int src[8]) {
  const int pos[2] = {x, y}, dims[2] = {g.nx, g.ny}, strides[2] = {1, g.nx};
#pragma unroll
  for (int ax = 0; ax < 2; ++ax)
#pragma unroll
    for (int sd = 0; sd < 2; ++sd) {
      const int sg = sd ? 1 : -1;
      const uint32_t opp = (sw >> (4 * (2 * ax + (1 - sd)))) & 15u;  // s's kinds toward -sg
#pragma unroll
      for (int dist = 1; dist <= 2; ++dist) {
        const bool real = dist == 1 ? (opp & 3u) == 0u : opp == 0u;
        int rc = -1;
        if (real) {
          int qd = pos[ax] - dist * sg;
          if (qd < 0 || qd >= dims[ax]) qd = ((qd % dims[ax]) + dims[ax]) % dims[ax];  // periodic
          rc = s + (qd - pos[ax]) * strides[ax];
        }
        src[2 * (2 * ax + sd) + dist - 1] = rc;
      }
    }
}

// Sum of one field's slots for the fluid cell s: its own center slot, then slot 1 + t of src[t].
template <typename R>
__device__ __forceinline__ R slot_sum(const R* __restrict__ sl, size_t fs, int s, const int src[8]) {
  R v = sl[s];
#pragma unroll
  for (int t = 0; t < 8; ++t)
    if (src[t] >= 0) v += sl[(size_t)(1 + t) * fs + src[t]];
  return v;
}

// One thread per cell. NK > 0: that many species (fields unrolled); NK = 0: c.K <= MAX_SP.
template <typename R, int NK>
__global__ void __launch_bounds__(FDA_BLOCK, sizeof(R) == 4 ? 7 : 1) fd_adjoint_kernel(const FDAdjArgs<R> A) {
  constexpr int NF = (NK > 0 ? NK : MAX_SP) + 1;  // fields held in registers
  const FDArgs<R>& a = A.f;
  const FDConst<R>& c = a.c;
  const Geo& g = a.geo;
  const int N = g.N, K = NK > 0 ? NK : c.K;
  const int r = blockIdx.x * FDA_BLOCK + threadIdx.x;
  if (r >= N) return;
  const uint32_t sw = __ldg(a.sword + r);
  if (!(sw >> 31)) {
    pdl_wait();
    pdl_trigger();
    A.u_out[r] = R(0);
    A.u_out[N + r] = R(0);
    return;
  }
  const int x = r % g.nx, y = r / g.nx;
  FDStencil2 S;
  fd_stencil2(g, sw, r, x, y, S);
  const size_t fs = (size_t)(K + 1) * N;  // stride between slots

  // adjoints of T^{n+1}, Y^{n+1} at this cell
  R ob[NF];
  if (A.Tbar_out) {
#pragma unroll
    for (int f = 0; f < NF; ++f)
      if (f <= K) ob[f] = f == 0 ? A.Tbar_out[r] : A.Ybar_out[(size_t)(f - 1) * N + r];
  } else {
    int src[8];
    slot_sources(g, sw, r, x, y, src);
#pragma unroll
    for (int f = 0; f < NF; ++f)
      if (f <= K) ob[f] = slot_sum<R>(A.slots_in + (size_t)f * N, fs, r, src);
  }
  // ------------------------------------------------------------ forward: shared quantities
  const R F = c.F;
  const R fdr = sizeof(R) == 4 ? (R)a.pth->fd_rho : (R)a.pth->fd_rho_d;
  const R Tr = a.T[r];
  R Y[MAX_SP];
  R sW = R(0);
#pragma unroll
  for (int k = 0; k < MAX_SP; ++k) {
    Y[k] = (k < K) ? a.Y[(size_t)k * N + r] : R(0);
    if (k < K) sW += Y[k] * c.inv_W[k];
  }
  const R W = R(1) / sW;
  const R rho = fdr * W / Tr;
  const R rho_phys = rho / c.inv_rho_ref;
  const R inv_rho = R(1) / rho;
  R Tn[2][2], mun[2][2], FMf[2][2], uf[2][2];
  const R ur[2] = {a.u[r], a.u[N + r]};
  const R mur = c.nu_lat * powr<R>(Tr * c.T_ref_inv, c.mu_exp);
#pragma unroll
  for (int ax = 0; ax < 2; ++ax)
#pragma unroll
    for (int sd = 0; sd < 2; ++sd) {
      const int kk = S.k1[ax][sd], j = S.i1[ax][sd];
      Tn[ax][sd] = kk == NB_FLUID ? a.T[j] : (kk == NB_INLET ? c.T_in : Tr);
      mun[ax][sd] = c.nu_lat * powr<R>(Tn[ax][sd] * c.T_ref_inv, c.mu_exp);
      FMf[ax][sd] = R(0.5) * (F * mur + F * mun[ax][sd]);
      R un;
      if (kk == NB_FLUID) un = a.u[ax * N + j];
      else if (kk == NB_INLET) un = a.inlet_u[ax * g.ny + y];
      else if (kk == NB_OUTLET) un = ur[ax];
      else un = R(0);
      uf[ax][sd] = R(0.5) * (ur[ax] + un);
    }
  // rates q_j: the forward kernel's arithmetic
  R q[MAX_RX], qdot = R(0);
#pragma unroll
  for (int j = 0; j < MAX_RX; ++j) q[j] = R(0);
  reaction_rates<0, R, MAX_SP>(c, Tr, R(1) / Tr, Y, rho_phys, q);
#pragma unroll
  for (int j = 0; j < MAX_RX; ++j) qdot += c.heat[j] * q[j];
  const R inv_rpF = R(1) / (rho_phys * F);
  const R dt = c.dt_phys;

  // the LB adjoint of this step (the predecessor kernel) has completed: its outputs and every
  // write of this kernel after this point
  pdl_wait();
  pdl_trigger();
  // adjoint of rho^n from the LB step: own part and the density-gradient parts of the cells that
  // hold this cell as their -x / +x / -y / +y neighbour (zero where that cell is solid or mirrored)
  R rhob_lb = A.rho_own[r];
  {
    const int xm = x > 0 ? r - 1 : (g.bc_lo[0] == BC_PERIODIC ? r + g.nx - 1 : -1);
    const int xp = x < g.nx - 1 ? r + 1 : (g.bc_hi[0] == BC_PERIODIC ? r - g.nx + 1 : -1);
    const int ym = y > 0 ? r - g.nx : (g.bc_lo[1] == BC_PERIODIC ? r + (g.ny - 1) * g.nx : -1);
    const int yp = y < g.ny - 1 ? r + g.nx : (g.bc_hi[1] == BC_PERIODIC ? r - (g.ny - 1) * g.nx : -1);
    if (xm >= 0) rhob_lb += A.rho_nb[xm];
    if (xp >= 0) rhob_lb += A.rho_nb[N + xp];
    if (ym >= 0) rhob_lb += A.rho_nb[2 * N + ym];
    if (yp >= 0) rhob_lb += A.rho_nb[3 * N + yp];
  }
  const R lamb = A.lam_bar[r];

  // ------------------------------------------------------------- field after field
  R tot[PA_N];
#pragma unroll
  for (int p = 0; p < PA_N; ++p) tot[p] = R(0);
  R c0[NF];     // center slot of each field (before the shared terms)
  R pT[9];      // slots of T (the viscosity law adds to its distance-1 points below)
#pragma unroll
  for (int f = 0; f < NF; ++f) {
    if (f > K) break;
    const R* phi = f == 0 ? a.T : a.Y + (size_t)(f - 1) * N;
    const R phin = f == 0 ? c.T_in : c.Y_in[f - 1];
    const R eps = f == 0 ? c.eps_T : c.eps_Y;
    const R gfac = c.inv_Pr * (f == 0 ? R(1) : c.inv_Le[f - 1]);
    const R pr = f == 0 ? Tr : Y[f - 1];
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
    if (f == 0) {
      src = dt * qdot * inv_rpF * c.inv_cp;
    } else {
#pragma unroll
      for (int j = 0; j < MAX_RX; ++j) om += c.nu[j][f - 1] * q[j];
      src = dt * c.W[f - 1] * om * inv_rpF;
    }
    const R NA = gfac * inv_rho * dif + src;
    // reverse. Lambda = NA_T / T + sum_k W / W_k NA_k; out = phi - adv + NA
    const R outb = ob[f];
    R NAb;
    if (f == 0) {
      tot[PA_TR] += -lamb * NA / (Tr * Tr);
      NAb = outb + lamb / Tr;
    } else {
      tot[PA_W] += lamb * c.inv_W[f - 1] * NA;
      NAb = outb + lamb * W * c.inv_W[f - 1];
    }
    R pointb[9];
#pragma unroll
    for (int p = 1; p < 9; ++p) pointb[p] = R(0);
    pointb[0] = outb;
    tot[PA_INVRHO] += NAb * gfac * dif;
    const R gi = NAb * gfac * inv_rho;
#pragma unroll
    for (int ax = 0; ax < 2; ++ax) {
      const R m2 = pm2[ax], m1 = pm1[ax], p1 = pp1[ax], p2 = pp2[ax];
      R m2b = R(0), m1b = R(0), p1b = R(0), p2b = R(0), prb = R(0);
      tot[PA_FM + 2 * ax + 1] += gi * (p1 - pr);
      tot[PA_FM + 2 * ax] -= gi * (pr - m1);
      p1b += gi * FMf[ax][1];
      prb -= gi * (FMf[ax][1] + FMf[ax][0]);
      m1b += gi * FMf[ax][0];
      const bool up = uf[ax][1] >= R(0), um = uf[ax][0] >= R(0);
      const R dm2 = m1 - m2, dm1 = pr - m1, dp1 = p1 - pr, dp2 = p2 - p1;
      // each face from its upwind side: the stencil differences picked by selects and one
      // evaluation (one copy of the face code per field keeps the kernel in the instruction cache)
      const R pa = up ? dm1 : -dp2, pb = up ? dp1 : -dp1;  // + face
      const R ma = um ? dm2 : -dp1, mb = um ? dm1 : -dm1;  // - face
      const R fp = weno_face<R>(up ? pr : p1, pa, pb, eps);
      const R fm = weno_face<R>(um ? m1 : pr, ma, mb, eps);
      const R advb = -outb;
      tot[PA_UR + ax] += advb * (fp - fm);
      const R fpb = advb * ur[ax], fmb = -advb * ur[ax];
      R bb, dab, dbc;
      weno_face_rev<R>(pa, pb, eps, fpb, bb, dab, dbc);
      {
        // up: base pr, differences (m1 -> pr, pr -> p1); else base p1, (p2 -> p1, p1 -> pr)
        const R t = bb + dab - dbc;
        prb += up ? t : dbc;
        m1b -= up ? dab : R(0);
        p1b += up ? dbc : t;
        p2b -= up ? R(0) : dab;
      }
      weno_face_rev<R>(ma, mb, eps, fmb, bb, dab, dbc);
      {
        // um: base m1, differences (m2 -> m1, m1 -> pr); else base pr, (p1 -> pr, pr -> m1)
        const R t = bb + dab - dbc;
        m1b += um ? t : dbc;
        m2b -= um ? dab : R(0);
        prb += um ? dbc : t;
        p1b -= um ? R(0) : dab;
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
    if (f == 0) {
      tot[PA_QDOT] += NAb * dt * inv_rpF * c.inv_cp;
      tot[PA_INVRPF] += NAb * dt * qdot * c.inv_cp;
    } else {
      const R omb = NAb * dt * c.W[f - 1] * inv_rpF;
      tot[PA_INVRPF] += NAb * dt * c.W[f - 1] * om;
#pragma unroll
      for (int j = 0; j < MAX_RX; ++j) tot[PA_Q + j] += c.nu[j][f - 1] * omb;
    }
    c0[f] = pointb[0];
    if (f == 0) {
#pragma unroll
      for (int p = 1; p < 9; ++p) pT[p] = pointb[p];
    } else {
      R* out = A.slots + (size_t)f * N + r;
#pragma unroll
      for (int p = 1; p < 9; ++p) out[(size_t)p * fs] = pointb[p];
    }
  }

  // ---------------------- shared terms: reverse of the rate law, rho = P W / (R T), W and mu(T)
  R Trb = tot[PA_TR], Wb = tot[PA_W];
  R rho_physb = -tot[PA_INVRPF] * inv_rpF / rho_phys;
  R add[MAX_SP];  // center adjoint of each species from the shared terms
#pragma unroll
  for (int k = 0; k < MAX_SP; ++k) add[k] = R(0);
#pragma unroll
  for (int j = 0; j < MAX_RX; ++j) {
    if (j >= c.nrx) break;
    const R qq = q[j] * (tot[PA_Q + j] + c.heat[j] * tot[PA_QDOT]);
    Trb += qq * ((c.ER_hi[j] + c.ER_lo[j]) / (Tr * Tr) + c.beta[j] / Tr);
#pragma unroll
    for (int m = 0; m < MAX_ORD; ++m) {
      if (m >= c.nord[j]) break;
      const int k = c.ord_k[j][m];
      const R yk = pick_species<MAX_SP, R>(Y, k);
      if (yk > R(0)) {
        rho_physb += qq * c.ord_n[j][m] / rho_phys;
        const R d = qq * c.ord_n[j][m] / yk;
#pragma unroll
        for (int kk = 0; kk < MAX_SP; ++kk)
          if (kk == k) add[kk] += d;
      }
    }
  }
  // adjoint of rho^n: from the LB step and this update
  R rhob = rhob_lb;
  rhob += rho_physb / c.inv_rho_ref;
  rhob -= tot[PA_INVRHO] * inv_rho * inv_rho;
  Wb += rhob * fdr / Tr;
  Trb -= rhob * rho / Tr;
  const R sWb = -Wb * W * W;
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
      if (kk == NB_FLUID) pT[slot1(ax, sd)] += dmu;
      else if (kk != NB_INLET) Trb += dmu;
    }
  Trb += murb * c.mu_exp * mur / Tr;
  // center slots (T: with the LB step's adjoint of T^n), the slots of T, the velocity adjoint
  A.slots[r] = (c0[0] + Trb) + A.T_lb[r];
  {
    R* out = A.slots + r;
#pragma unroll
    for (int p = 1; p < 9; ++p) out[(size_t)p * fs] = pT[p];
  }
#pragma unroll
  for (int f = 1; f < NF; ++f)
    if (f <= K) A.slots[(size_t)f * N + r] = c0[f] + (add[f - 1] + sWb * c.inv_W[f - 1]);
  A.u_out[r] = tot[PA_UR] + A.u_lb[r];
  A.u_out[N + r] = tot[PA_UR + 1] + A.u_lb[N + r];
}

// Adjoint of T and Y_k from the slot form, for every cell (0 on solid cells): where a reverse
// sweep ends.
template <typename R>
__global__ void __launch_bounds__(FDA_BLOCK)
    fd_adjoint_gather(Geo g, const uint32_t* __restrict__ sword, int K, const R* __restrict__ slots,
                      R* __restrict__ Tbar, R* __restrict__ Ybar) {
  const int s = blockIdx.x * FDA_BLOCK + threadIdx.x;
  const int N = g.N;
  if (s >= N) return;
  const uint32_t sw = __ldg(sword + s);
  if (!(sw >> 31)) {
    Tbar[s] = R(0);
    for (int k = 0; k < K; ++k) Ybar[(size_t)k * N + s] = R(0);
    return;
  }
  int src[8];
  slot_sources(g, sw, s, s % g.nx, s / g.nx, src);
  const size_t fs = (size_t)(K + 1) * N;
  Tbar[s] = slot_sum<R>(slots, fs, s, src);
  for (int k = 0; k < K; ++k) Ybar[(size_t)k * N + s] = slot_sum<R>(slots + (size_t)(k + 1) * N, fs, s, src);
}

}  // namespace hlbm
