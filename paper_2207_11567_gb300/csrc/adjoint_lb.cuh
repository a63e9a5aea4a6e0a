// Adjoint (reverse mode) of the D2Q9 stream-collide update of lb_kernel.cuh for the thermal
// cumulant case with full relaxation of orders 3..4 (the default rates), Smagorinsky closure,
// bounce-back walls, moving-wall inlet and pressure outlet. The adjoint step is not in the paper;
// it is the exact transpose of the discrete update, written by hand operation by operation.
//
// Per fluid cell the forward is recomputed from state n, then every operation is reversed in
// the opposite order. Population adjoints go back to the unique place each pulled population
// came from (a pull has exactly one consumer per stored population), so no atomics are needed.
// Density-gradient adjoints are written per cell and neighbour side; the FD adjoint of the same
// step sums, for each cell, those of the cells that hold it as a neighbour.
#pragma once
#include "common.cuh"

namespace hlbm {

template <typename R> struct LBAdjArgs {
  LBArgs<R> f;        // forward arguments (g_in = state n populations; g_out unused)
  const R* u_prev;    // [2][N] velocity of state n (outlet rule)
  const R* gbar_out;  // [9][N] adjoint of the stored populations of state n+1
  const R* ubar_out;  // [2][N] adjoint of the velocity of state n+1
  R* gbar_in;         // [9][N] adjoint of the populations of state n (written once per slot)
  R* rho_bar;         // [N] adjoint of rho used by this cell (own part)
  R* lam_bar;         // [N] adjoint of Lambda (FD part)
  R* T_bar;           // [N] adjoint of T through the viscosity law
  R* u_bar;           // [2][N] adjoint of the state-n velocity through the outlet rule
  R* rho_nb;          // [4][N] adjoint of rho at the +x, -x, +y, -y neighbour (0 when mirrored)
  R* inlet_bar;       // [2][ny] adjoint of the inlet face velocity (one cell per face element)
};

template <typename R> __device__ __forceinline__ void fwd3(R a, R b, R c, R u, R& m0, R& m1, R& m2) {
  m0 = a + b + c;
  m1 = (c - a) - u * m0;
  m2 = (c + a) - R(2) * u * (c - a) + u * u * m0;
}
// reverse of fwd3: given the adjoints of (m0, m1, m2), accumulate those of (a, b, c) and u
template <typename R>
__device__ __forceinline__ void fwd3_rev(R a, R c, R u, R m0, R mb0, R mb1, R mb2, R& ab, R& bb, R& cb, R& ub) {
  const R m0t = mb0 - u * mb1 + u * u * mb2;
  const R db = mb1 - R(2) * u * mb2;  // adjoint of d = c - a
  const R sb = mb2;                   // adjoint of s = c + a
  ab = m0t - db + sb;
  bb = m0t;
  cb = m0t + db + sb;
  ub += -m0 * mb1 + (-R(2) * (c - a) + R(2) * u * m0) * mb2;
}
template <typename R> __device__ __forceinline__ void bwd3(R m0, R m1, R m2, R u, R& a, R& b, R& c) {
  const R k1 = m1 + u * m0;
  const R k2 = m2 + R(2) * u * m1 + u * u * m0;
  a = R(0.5) * (k2 - k1);
  b = m0 - k2;
  c = R(0.5) * (k2 + k1);
}
template <typename R>
__device__ __forceinline__ void bwd3_rev(R m0, R m1, R u, R ab, R bb, R cb, R& mb0, R& mb1, R& mb2, R& ub) {
  const R k1b = R(-0.5) * ab + R(0.5) * cb;
  const R k2b = R(0.5) * ab - bb + R(0.5) * cb;
  mb0 = bb + u * k1b + u * u * k2b;
  mb1 = k1b + R(2) * u * k2b;
  mb2 = k2b;
  ub += m0 * k1b + (R(2) * m1 + R(2) * u * m0) * k2b;
}

// Delta_eq of lb_kernel.cuh for D = 2: -(ex ky + kx ey + ex ey), ke = (1, 0, 1/3), dl = (0, -u, u^2)
template <typename R> __device__ __forceinline__ void deq2(R ux, R uy, R* dq, R* dqx, R* dqy) {
  const R ke[3] = {R(1), R(0), R(1) / R(3)};
  const R ex[3] = {R(0), -ux, ux * ux}, ey[3] = {R(0), -uy, uy * uy};
  const R dex[3] = {R(0), R(-1), R(2) * ux}, dey[3] = {R(0), R(-1), R(2) * uy};
#pragma unroll
  for (int J = 0; J < 9; ++J) {
    const int a = J % 3, b = J / 3;
    dq[J] = -(ex[a] * ke[b] + ke[a] * ey[b] + ex[a] * ey[b]);
    dqx[J] = -(dex[a] * ke[b] + dex[a] * ey[b]);
    dqy[J] = -(ke[a] * dey[b] + ex[a] * dey[b]);
  }
}

template <typename R, bool THERMAL>
__global__ void __launch_bounds__(LB_BLOCK, sizeof(R) == 4 ? 4 : 1) lb_adjoint_kernel(const LBAdjArgs<R> A) {
  const LBArgs<R>& a = A.f;
  constexpr int Q = 9;
  const int nx = a.geo.nx, ny = a.geo.ny;
  const int x = blockIdx.x * LB_BLOCK + threadIdx.x;
  const int y = blockIdx.y;
  if (x >= nx) return;
  const int r = x + nx * y;
  const int N = a.geo.N;
  const uint32_t lw = __ldg(a.links + r);
  if (!(lw >> 31)) return;
  const R third = R(1) / R(3);
  const R* gin = (const R*)a.g_in;

  // ---------------------------------------------------------------- forward recomputation
  R rho = R(1), lam = R(0);
  if constexpr (THERMAL) {
    rho = a.rho[r];
    lam = a.lam[r] + (sizeof(R) == 8 ? (R)a.pth->lb_lam_d : (R)a.pth->lb_lam);
  }
  R rho_p[2] = {rho, rho}, rho_m[2] = {rho, rho};
  bool real_p[2] = {false, false}, real_m[2] = {false, false};
  const int oxm = x > 0 ? -1 : nx - 1, oxp = x < nx - 1 ? 1 : 1 - nx;
  const int oym = y > 0 ? -nx : (ny - 1) * nx, oyp = y < ny - 1 ? nx : (1 - ny) * nx;
  int src[Q];
  R qin[Q];
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const int ci = cx(i), cj = cy(i);
    if ((lw >> i) & 1u) {
      src[i] = -1;
      qin[i] = ld_raw<R>(gin + (Q - 1 - i) * N + r);
    } else {
      const int s = r + (ci == 1 ? oxm : (ci == -1 ? oxp : 0)) + (cj == 1 ? oym : (cj == -1 ? oyp : 0));
      src[i] = s;
      qin[i] = ld_raw<R>(gin + i * N + s);
      if constexpr (THERMAL) {
        if (ci * ci + cj * cj == 1) {
          const R rs = a.rho[s];
          if (ci == -1) { rho_p[0] = rs; real_p[0] = true; }
          if (ci == 1) { rho_m[0] = rs; real_m[0] = true; }
          if (cj == -1) { rho_p[1] = rs; real_p[1] = true; }
          if (cj == 1) { rho_m[1] = rs; real_m[1] = true; }
        }
      }
    }
  }
  const bool inlet_cell = x == 0 && a.geo.bc_lo[0] == BC_INLET;
  const bool outlet_cell = x == nx - 1 && a.geo.bc_hi[0] == BC_OUTLET;
  R uw0 = R(0), uw1 = R(0), v0 = R(0), v1 = R(0);
  if (inlet_cell) { uw0 = a.inlet_u[y]; uw1 = a.inlet_u[ny + y]; }
  if (outlet_cell) { v0 = A.u_prev[r]; v1 = A.u_prev[N + r]; }
  R q[Q];
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    q[i] = qin[i];
    if (((lw >> i) & 1u) && inlet_cell && cx(i) == 1) q[i] += R(2) * rho * (uw0 + (R)cy(i) * uw1);
    if (((lw >> i) & 1u) && outlet_cell && cx(i) == -1) {
      const R cv = -v0 + (R)cy(i) * v1;
      q[i] = -q[i] + rho * (R(3) * cv * cv - (v0 * v0 + v1 * v1));
    }
  }
  R mx = R(0), my = R(0);
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    mx += (R)cx(i) * (R)wgt<2>(i) * q[i];
    my += (R)cy(i) * (R)wgt<2>(i) * q[i];
  }
  const R inv_rho = R(1) / rho;
  const R ux = R(3) * mx * inv_rho, uy = R(3) * my * inv_rho, usq = ux * ux + uy * uy;
  const R gx = THERMAL ? R(0.5) * (rho_p[0] - rho_m[0]) : R(0);
  const R gy = THERMAL ? R(0.5) * (rho_p[1] - rho_m[1]) : R(0);
  const R udg = ux * gx + uy * gy;
  const R rl3 = rho * lam * third;
  R xi[Q], e[Q], s[Q];
  R S = R(0);
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const R cu = (R)cx(i) * ux + (R)cy(i) * uy, cg = (R)cx(i) * gx + (R)cy(i) * gy;
    e[i] = cu + R(1.5) * cu * cu - R(0.5) * usq;
    xi[i] = THERMAL ? e[i] * (cg - udg) + rl3 : R(0);
    s[i] = q[i] + R(0.5) * xi[i];
    S += (R)wgt<2>(i) * s[i];
  }
  R d[Q], xv[Q];
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    d[i] = R(3) * inv_rho * (s[i] - S);
    xv[i] = (R)wgt<2>(i) * d[i];
  }
  R Tpow = R(1), tau0;
  if constexpr (THERMAL) {
    Tpow = pow(a.T[r] * a.T_ref_inv, a.mu_exp);
    tau0 = R(3) * a.nu_lat * Tpow * inv_rho + R(0.5);
  } else {
    tau0 = R(3) * a.nu_lat + R(0.5);
  }
  // chimera forward: x lines (slots 3j..3j+2) with ux, then y lines (ax, ax+3, ax+6) with uy
  R t1[Q];
#pragma unroll
  for (int j = 0; j < 3; ++j) fwd3(xv[3 * j], xv[3 * j + 1], xv[3 * j + 2], ux, t1[3 * j], t1[3 * j + 1], t1[3 * j + 2]);
  R mt[Q];
#pragma unroll
  for (int ax = 0; ax < 3; ++ax) fwd3(t1[ax], t1[ax + 3], t1[ax + 6], uy, mt[ax], mt[ax + 3], mt[ax + 6]);
  R dq[Q], dqx[Q], dqy[Q];
  deq2(ux, uy, dq, dqx, dqy);
  R n[Q];
#pragma unroll
  for (int J = 0; J < Q; ++J) n[J] = mt[J] - dq[J];
  const R tr = R(0.5) * (n[2] + n[6]);
  const R dd0 = n[2] - tr, dd1 = n[6] - tr;
  const R n2 = dd0 * dd0 + dd1 * dd1 + R(2) * n[4] * n[4];
  R tau = tau0, Rn = R(0), sqA = R(1);
  if (a.smag_k > R(0)) {
    Rn = sqrt(n2);
    sqA = sqrt(tau0 * tau0 + a.smag_k * Rn);
    tau = R(0.5) * (tau0 + sqA);
  }
  const R om = R(1) / tau;
  const R o1 = R(1) - om, ob = R(1) - a.omega_b;
  const R s20 = o1 * (n[2] - tr) + ob * tr, s02 = o1 * (n[6] - tr) + ob * tr, s11 = o1 * n[4];
  R ns[Q];
  ns[0] = n[0]; ns[1] = n[1]; ns[3] = n[3];
  ns[2] = s20; ns[6] = s02; ns[4] = s11; ns[5] = R(0); ns[7] = R(0);
  ns[8] = third * (s20 + s02) + s20 * s02 + R(2) * s11 * s11;
  R mts[Q];
#pragma unroll
  for (int J = 0; J < Q; ++J) mts[J] = ns[J] + dq[J];
  // chimera backward: y lines with uy, then x lines with ux
  R t2[Q];
#pragma unroll
  for (int ax = 0; ax < 3; ++ax) bwd3(mts[ax], mts[ax + 3], mts[ax + 6], uy, t2[ax], t2[ax + 3], t2[ax + 6]);
  R xs[Q];
#pragma unroll
  for (int j = 0; j < 3; ++j) bwd3(t2[3 * j], t2[3 * j + 1], t2[3 * j + 2], ux, xs[3 * j], xs[3 * j + 1], xs[3 * j + 2]);

  // ---------------------------------------------------------------- reverse
  // the adjoint of state n + 1 and every output: after the predecessor kernel (the FD adjoint of
  // the step after this one) has completed
  pdl_wait();
  pdl_trigger();
  R rhob = R(0), Sb = R(0), uxb = A.ubar_out[r], uyb = A.ubar_out[N + r];
  R xib[Q], xsb[Q];
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const R ob_ = ld_raw<R>(A.gbar_out + i * N + r);
    const R dstar = xs[i] / (R)wgt<2>(i);
    rhob += third * dstar * ob_;
    Sb += ob_;
    xib[i] = R(0.5) * ob_;
    xsb[i] = rho * third * ob_ / (R)wgt<2>(i);  // through d* = x* / w
  }
  // chimera backward, reversed: x lines first, then y lines
  R t2b[Q];
#pragma unroll
  for (int j = 0; j < 3; ++j)
    bwd3_rev(t2[3 * j], t2[3 * j + 1], ux, xsb[3 * j], xsb[3 * j + 1], xsb[3 * j + 2], t2b[3 * j], t2b[3 * j + 1],
             t2b[3 * j + 2], uxb);
  R mtsb[Q];
#pragma unroll
  for (int ax = 0; ax < 3; ++ax)
    bwd3_rev(mts[ax], mts[ax + 3], uy, t2b[ax], t2b[ax + 3], t2b[ax + 6], mtsb[ax], mtsb[ax + 3], mtsb[ax + 6], uyb);
  // mts = ns + dq
  R nsb[Q];
#pragma unroll
  for (int J = 0; J < Q; ++J) {
    nsb[J] = mtsb[J];
    uxb += mtsb[J] * dqx[J];
    uyb += mtsb[J] * dqy[J];
  }
  // relaxation, reversed
  R s20b = nsb[2] + nsb[8] * (third + s02);
  R s02b = nsb[6] + nsb[8] * (third + s20);
  R s11b = nsb[4] + nsb[8] * R(4) * s11;
  R nb[Q];
#pragma unroll
  for (int J = 0; J < Q; ++J) nb[J] = R(0);
  nb[0] = nsb[0]; nb[1] = nsb[1]; nb[3] = nsb[3];
  const R c1 = R(0.5) * o1 + R(0.5) * ob, c2 = -R(0.5) * o1 + R(0.5) * ob;
  nb[2] += c1 * s20b + c2 * s02b;
  nb[6] += c2 * s20b + c1 * s02b;
  nb[4] += o1 * s11b;
  const R omb = -(n[2] - tr) * s20b - (n[6] - tr) * s02b - n[4] * s11b;
  const R taub = -om * om * omb;
  R tau0b = taub;
  if (a.smag_k > R(0)) {
    tau0b = taub * R(0.5) * (R(1) + tau0 / sqA);
    const R Rb = taub * a.smag_k / (R(4) * sqA);
    const R n2b = Rn > R(0) ? Rb / (R(2) * Rn) : R(0);
    nb[2] += n2b * (dd0 - dd1);
    nb[6] += n2b * (dd1 - dd0);
    nb[4] += n2b * R(4) * n[4];
  }
  // n = mt - dq
  R mtb[Q];
#pragma unroll
  for (int J = 0; J < Q; ++J) {
    mtb[J] = nb[J];
    uxb -= nb[J] * dqx[J];
    uyb -= nb[J] * dqy[J];
  }
  // chimera forward, reversed: y lines first, then x lines
  R t1b[Q];
#pragma unroll
  for (int ax = 0; ax < 3; ++ax)
    fwd3_rev(t1[ax], t1[ax + 6], uy, mt[ax], mtb[ax], mtb[ax + 3], mtb[ax + 6], t1b[ax], t1b[ax + 3], t1b[ax + 6], uyb);
  R xvb[Q];
#pragma unroll
  for (int j = 0; j < 3; ++j)
    fwd3_rev(xv[3 * j], xv[3 * j + 2], ux, t1[3 * j], t1b[3 * j], t1b[3 * j + 1], t1b[3 * j + 2], xvb[3 * j],
             xvb[3 * j + 1], xvb[3 * j + 2], uxb);
  // tau0
  if constexpr (THERMAL) {
    const R Tr = a.T[r];
    A.T_bar[r] = tau0b * R(3) * a.nu_lat * a.mu_exp * Tpow / Tr * inv_rho;
    rhob -= tau0b * R(3) * a.nu_lat * Tpow * inv_rho * inv_rho;
  }
  // x = w d; d = 3/rho (s - S)
  R sb[Q];
  R dsum = R(0);
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const R db = (R)wgt<2>(i) * xvb[i];
    sb[i] = R(3) * inv_rho * db;
    dsum += db;
    rhob -= d[i] * db * inv_rho;
  }
  Sb -= R(3) * inv_rho * dsum;
  // S = sum w s; s = q + xi/2
  R qb[Q];
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    sb[i] += (R)wgt<2>(i) * Sb;
    qb[i] = sb[i];
    xib[i] += R(0.5) * sb[i];
  }
  // source
  R gxb = R(0), gyb = R(0);
  if constexpr (THERMAL) {
    R udgb = R(0), rl3b = R(0), usqb = R(0);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const R cu = (R)cx(i) * ux + (R)cy(i) * uy, cg = (R)cx(i) * gx + (R)cy(i) * gy;
      const R eb = xib[i] * (cg - udg);
      const R cgb = xib[i] * e[i];
      udgb -= xib[i] * e[i];
      rl3b += xib[i];
      const R cub = eb * (R(1) + R(3) * cu);
      usqb -= R(0.5) * eb;
      uxb += (R)cx(i) * cub;
      uyb += (R)cy(i) * cub;
      gxb += (R)cx(i) * cgb;
      gyb += (R)cy(i) * cgb;
    }
    uxb += udgb * gx + R(2) * ux * usqb;
    uyb += udgb * gy + R(2) * uy * usqb;
    gxb += udgb * ux;
    gyb += udgb * uy;
    rhob += rl3b * lam * third;
    A.lam_bar[r] = rl3b * rho * third;
  } else {
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const R cu = (R)cx(i) * ux + (R)cy(i) * uy;
      const R eb = R(0);
      (void)cu;
      (void)eb;
    }
  }
  // u = 3 m / rho
  const R mxb = R(3) * inv_rho * uxb, myb = R(3) * inv_rho * uyb;
  rhob -= (ux * uxb + uy * uyb) * inv_rho;
#pragma unroll
  for (int i = 0; i < Q; ++i) qb[i] += (R)wgt<2>(i) * ((R)cx(i) * mxb + (R)cy(i) * myb);
  // boundary terms and streaming
  R uw0b = R(0), uw1b = R(0), v0b = R(0), v1b = R(0);
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    R qinb = qb[i];
    if (((lw >> i) & 1u) && inlet_cell && cx(i) == 1) {
      rhob += R(2) * (uw0 + (R)cy(i) * uw1) * qb[i];
      uw0b += R(2) * rho * qb[i];
      uw1b += R(2) * rho * (R)cy(i) * qb[i];
    }
    if (((lw >> i) & 1u) && outlet_cell && cx(i) == -1) {
      const R cv = -v0 + (R)cy(i) * v1;
      qinb = -qb[i];
      rhob += (R(3) * cv * cv - (v0 * v0 + v1 * v1)) * qb[i];
      v0b += rho * (R(6) * cv * R(-1) - R(2) * v0) * qb[i];
      v1b += rho * (R(6) * cv * (R)cy(i) - R(2) * v1) * qb[i];
    }
    if (src[i] < 0) A.gbar_in[(Q - 1 - i) * N + r] = qinb;
    else A.gbar_in[i * N + src[i]] = qinb;
  }
  if (inlet_cell) {
    A.inlet_bar[y] += uw0b;
    A.inlet_bar[ny + y] += uw1b;
  }
  A.u_bar[r] = v0b;
  A.u_bar[N + r] = v1b;
  // density gradient: G = (rho_p - rho_m) / 2, mirrored neighbours are rho itself
  if constexpr (THERMAL) {
    const R gb[2] = {gxb, gyb};
#pragma unroll
    for (int ax = 0; ax < 2; ++ax) {
      const R pb = R(0.5) * gb[ax], mb = R(-0.5) * gb[ax];
      if (real_p[ax]) A.rho_nb[(2 * ax) * N + r] = pb; else { A.rho_nb[(2 * ax) * N + r] = R(0); rhob += pb; }
      if (real_m[ax]) A.rho_nb[(2 * ax + 1) * N + r] = mb; else { A.rho_nb[(2 * ax + 1) * N + r] = R(0); rhob += mb; }
    }
  }
  A.rho_bar[r] = rhob;
}

}  // namespace hlbm
