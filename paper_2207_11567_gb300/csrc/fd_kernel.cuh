// Finite-difference update of temperature and species (Section 2.3) with Arrhenius chemistry
// and the thickened-flame factor, the flame sensor, and the thermodynamic-pressure reduction.
// One thread per cell, lattice units of length and time (dr = dt = 1).
//
//   phi^{n+1} = phi^n - sum_a u_a (phi_hat(r + e_a/2) - phi_hat(r - e_a/2)) + N_phi
//   N_phi = (1/rho) sum_a [G(r+e/2)(phi(r+e) - phi(r)) - G(r-e/2)(phi(r) - phi(r-e))] + sources
// WENO3 face values (upwind side from the face velocity), centred diffusion with the arithmetic
// face mean of G = F_loc mu(T) / (Pr Le), chemistry divided by F_loc, pressure work on T.
// Lambda (Eq. 3) = N_T / T + sum_k (W / W_k) N_k, rho = P_th W / (R T).
// Stencil points outside the fluid take ghost values: zero gradient (walls, solids, outlet) or
// the inlet state (low-x inlet), velocity 0 at walls and solids, inlet velocity at the inlet;
// with sub-cell wall positions, ghost-point values from the wall fractions.
//
// Copies of the cell update (fd_cell): FAST for cells whose radius-2 stencil is all fluid and
// inside the grid, the general one, and GW for cells with ghost-point wall weights; each warp
// takes one copy for all its cells (the most general any of them needs). VDEG > 0 compiles the
// variable heat-capacity form of the temperature equation (fd_kernels_vcp.cu). The update also
// writes the flame sensor's F_loc of the state it produces, so the separate sensor pass is
// needed only after the state was set from outside.
#pragma once
#include "common.cuh"

namespace hlbm {

// Kind and index of the neighbour of (p[0], p[1], p[2]) at +sigma along `axis`.
// On return p holds the (wrapped) neighbour coordinates when the kind is fluid.
__device__ __forceinline__ int nb_classify(const Geo& g, const uint8_t* __restrict__ mask, int axis,
                                           int sigma, int* p, int base, int& idx) {
  const int n = axis == 0 ? g.nx : (axis == 1 ? g.ny : g.nz);
  int v = p[axis] + sigma;
  int kind = NB_FLUID;
  if (v < 0) {
    if (g.bc_lo[axis] == BC_PERIODIC) v += n;
    else kind = g.bc_lo[axis] == BC_INLET ? NB_INLET : NB_SOLID;
  } else if (v >= n) {
    if (g.bc_hi[axis] == BC_PERIODIC) v -= n;
    else kind = g.bc_hi[axis] == BC_OUTLET ? NB_OUTLET : NB_SOLID;
  }
  idx = base;
  if (kind == NB_FLUID) {
    int q[3] = {p[0], p[1], p[2]};
    q[axis] = v;
    const int j = q[0] + g.nx * (q[1] + g.ny * q[2]);
    if (__ldg(mask + j)) {
      kind = NB_SOLID;
    } else {
      idx = j;
      p[axis] = v;
    }
  }
  return kind;
}

// exp(-E / (R T)) with the exponent argument E/(R T) carried in float-float arithmetic
// (error ~1e-13 relative before the final float rounding of the exponential). r: 1 / T, correctly
// rounded (the caller's IEEE reciprocal, shared with its other uses).
__device__ __forceinline__ float arrhenius(float ER_hi, float ER_lo, float T, float r) {
  const float e = fmaf(-T, r, 1.0f);  // exact residual of the reciprocal
  const float rlo = r * e;
  const float hi = ER_hi * r;
  const float lo = fmaf(ER_hi, r, -hi) + ER_hi * rlo + ER_lo * r;
  return expf(-hi) * (1.0f - lo);
}

// x^y for x >= 0: FP32 as exp2(y log2 x) with the hardware log2 / exp2 (relative error a few
// 1e-7, against ~50 instructions for powf); FP64 with pow.
// Hardware reciprocal (PTX rcp.approx.ftz, relative error ~2^-23) for the WENO weights, whose
// denominators lie in [1e-12, 1e14]: far from denormals and from overflow, so no range handling.
__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

template <typename R> __device__ __forceinline__ R powr(R x, R y);
template <> __device__ __forceinline__ float powr<float>(float x, float y) { return exp2f(y * __log2f(x)); }
template <> __device__ __forceinline__ double powr<double>(double x, double y) { return pow(x, y); }

template <typename R> __device__ __forceinline__ R fdiv(R a, R b) { return a / b; }
template <> __device__ __forceinline__ float fdiv<float>(float a, float b) { return a * rcp_approx(b); }

template <typename R> __device__ __forceinline__ R weno3(R a, R b, R c, R eps) {
  const R q0 = R(-0.5) * a + R(1.5) * b;
  const R q1 = R(0.5) * (b + c);
  const R s0 = (eps + (b - a) * (b - a));
  const R s1 = (eps + (c - b) * (c - b));
  const R t0 = s0 * s0, t1 = s1 * s1;  // alpha_k = d_k / t_k
  // (d0/t0 q0 + d1/t1 q1) / (d0/t0 + d1/t1) with d0 = 1/3, d1 = 2/3
  // the denominator stays far below 2^126, the range where the fast division is exact enough
  return fdiv<R>(t1 * q0 + R(2) * t0 * q1, t1 + R(2) * t0);
}

// Y[k] for a run-time species index k, by selects over the KMAX register values (an indexed
// access would place the array in local memory).
template <int KMAX, typename R> __device__ __forceinline__ R pick_species(const R* Y, int k) {
  R v = Y[0];
#pragma unroll
  for (int i = 1; i < KMAX; ++i) v = (k == i) ? Y[i] : v;
  return v;
}

// Reaction rates q_j (mol/(m^3 s)) of one cell. NR > 0: reaction count known at compile time;
// NK > 0: species count known (Y then holds NK values in registers). Concentration powers: order 1
// as is, others as x^n (a separate square-root branch for order 1/2 measured 3% slower).
// inv_T: 1 / T, correctly rounded.
template <int NR, typename R, int NK = 0>
__device__ __forceinline__ void reaction_rates(const FDConst<R>& c, R T, R inv_T, const R* Y, R rho_phys, R* q) {
  const int nr = NR > 0 ? NR : c.nrx;
#pragma unroll
  for (int j = 0; j < (NR > 0 ? NR : MAX_RX); ++j) {
    if (NR == 0 && j >= nr) break;
    R v;
    if constexpr (sizeof(R) == 4) {
      v = c.A[j] * arrhenius(c.ER_hi[j], c.ER_lo[j], T, inv_T);
    } else {
      v = c.A[j] * exp(-c.ER_hi[j] / T);
    }
    if (c.beta[j] != R(0)) v *= powr<R>(T, c.beta[j]);
#pragma unroll
    for (int m = 0; m < MAX_ORD; ++m) {
      if (m >= c.nord[j]) break;
      const int k = c.ord_k[j][m];
      const R n = c.ord_n[j][m];
      const R yk = NK > 0 ? pick_species<NK, R>(Y, k) : Y[k];
      const R conc = rho_phys * fmax(yk, R(0)) * c.inv_W[k];
      v *= (n == R(1)) ? conc : powr<R>(conc, n);
    }
    q[j] = v;
  }
}

template <typename R> __device__ __forceinline__ R nu_of(const FDConst<R>& c, int j, int k) {
  return c.nu[j][k];
}

// Flame sensor: F_loc = 1 + (F - 1) tanh(beta Omega / Omega_0) with
// Omega = max(Y_F, 0) max(Y_O, 0) exp(-T_s / T), a function of the cell's own state.
template <typename R> __device__ __forceinline__ R sensor_floc(const FDConst<R>& c, R T, R yf, R yo) {
  const R om = fmax(yf, R(0)) * fmax(yo, R(0)) * exp(-c.sensor_Ta / T);
  return R(1) + (c.F - R(1)) * tanh(c.sensor_beta * om * c.inv_wref);
}

// F_loc of the current state, per fluid cell: needed once after the state is set from outside
// (fields, a checkpoint); each update then writes F_loc of the state it produces (Floc_out).
template <int D, typename R>
__global__ void __launch_bounds__(FD_BLOCK) flame_sensor_kernel(const FDArgs<R> a) {
  const int r = blockIdx.x * FD_BLOCK + threadIdx.x;
  if (r >= a.geo.N) return;
  if (__ldg(a.mask + r)) return;
  const FDConst<R>& c = a.c;
  const size_t N = (size_t)a.geo.N;
  a.Floc[r] = sensor_floc<R>(c, ldg(a.T + r), ldg(a.Y + c.sensor_species * N + r),
                             ldg(a.Y + c.sensor_oxidizer * N + r));
}

// Thread-block shape of the FD update: 32 x 4 x 2 cells in 3-D, 32 x 8 in 2-D (256 threads),
// so that the y and z neighbours of most stencils are loaded by the same block (L1 reuse).
template <int D> struct FDShape;
template <> struct FDShape<2> { static constexpr int X = 32, Y = 8, Z = 1; };
template <> struct FDShape<3> { static constexpr int X = 32, Y = 4, Z = 2; };

// One fluid cell of the FD update. FAST: the whole radius-2 stencil is fluid and inside the grid
// (no ghosts, no periodic wrap), so neighbour kinds are known at compile time and indices are
// plain offsets; the arithmetic is the same as the general path.
// Polynomials of the variable heat capacities (Horner, degree DEG of c_p known at compile time):
// c_p,k(T) and W_k h_k(T) (one degree higher).
template <int DEG, typename R> __device__ __forceinline__ R cp_eval(const R (&a)[5], R T) {
  R v = a[DEG];
#pragma unroll
  for (int m = DEG - 1; m >= 0; --m) v = fma(v, T, a[m]);
  return v;
}
template <int DEG, typename R> __device__ __forceinline__ R hW_eval(const R (&a)[6], R T) {
  R v = a[DEG + 1];
#pragma unroll
  for (int m = DEG; m >= 0; --m) v = fma(v, T, a[m]);
  return v;
}

// VDEG > 0: variable heat capacities, polynomials of degree VDEG. The temperature update becomes
//   N_T = [sum_faces lambda_face (T_n - T) + F mu/Pr sum_k (c_p,k - c_p)/Le_k grad Y_k . grad T]
//         / (rho c_p) + dt (-sum_k h_k omega_k) / (rho c_p F) + dP/(rho c_p),
// lambda = F mu c_p / Pr per cell (face value the arithmetic mean, a ghost neighbour's c_p from its
// ghost T and Y), centred gradients. The species fields run first so that the neighbours' c_p and
// the species-enthalpy flux are summed before the temperature field.
// MIX: mixture-averaged species diffusion. With G_k = F mu / (Pr Le_k^mix) and W per cell (from
// mix_coeff_kernel; ghosts: the own cell's values, the inlet state's at the inlet) and, per face,
// the arithmetic means G_k,f, Y_k,f and dlnW = (W_n - W_r) / mean W, the species term is
//   sum_faces [G_k,f (dY_k + Y_k,f dlnW) - Y_k,f C_f],  C_f = sum_j G_j,f (dY_j + Y_j,f dlnW)
// (differences neighbour minus cell), the Hirschfelder-Curtiss flux with its correction velocity.
template <int D, typename R, int NK, int NR, bool FAST, int VDEG, bool GW = false, bool MIX = false>
__device__ __forceinline__ void fd_cell(const FDArgs<R>& a, int x, int y, int z, int r, uint32_t sw, R& termI,
                                        R& termM) {
  const FDConst<R>& c = a.c;
  const Geo& g = a.geo;
  const int N = g.N;
  constexpr bool VCP = VDEG > 0;
  {
    const int pos[3] = {x, y, z};
    const int dims[3] = {g.nx, g.ny, g.nz};
    const int strides[3] = {1, g.nx, g.nx * g.ny};
    // neighbour kinds from the stencil word, indices with periodic wrap
    int k1[3][2], k2[3][2], i1[3][2], i2[3][2];
#pragma unroll
    for (int ax = 0; ax < D; ++ax) {
#pragma unroll
      for (int sd = 0; sd < 2; ++sd) {
        const int sg = sd ? 1 : -1;
        if constexpr (FAST) {
          // interior: every point of the radius-2 stencil is fluid and inside the grid
          k1[ax][sd] = NB_FLUID;
          k2[ax][sd] = 0;
          i1[ax][sd] = r + sg * strides[ax];
          i2[ax][sd] = r + 2 * sg * strides[ax];
        } else {
          const uint32_t bits = (sw >> (4 * (2 * ax + sd))) & 15u;
          k1[ax][sd] = (int)(bits & 3u);
          k2[ax][sd] = (int)(bits >> 2);
          int p1 = pos[ax] + sg;
          p1 = p1 < 0 ? p1 + dims[ax] : (p1 >= dims[ax] ? p1 - dims[ax] : p1);
          int p2 = p1 + sg;
          p2 = p2 < 0 ? p2 + dims[ax] : (p2 >= dims[ax] ? p2 - dims[ax] : p2);
          const int j1 = k1[ax][sd] == NB_FLUID ? r + (p1 - pos[ax]) * strides[ax] : r;
          i1[ax][sd] = j1;
          i2[ax][sd] = k2[ax][sd] == 0 ? r + (p2 - pos[ax]) * strides[ax] : j1;
        }
      }
    }
    // GW: ghost-point wall weights of this cell (0: the zero-gradient ghost); a separate copy of
    // the update, so that the other cells carry none of its registers
    R wg1[GW ? 3 : 1][2], wg2[GW ? 3 : 1][2];
    if constexpr (GW) {
      // a cell without weights (in a warp that takes this copy for another lane) gets zeros,
      // which reproduce the zero-gradient ghosts exactly
      const bool has = (sw & SW_WALL) != 0u;
      const R* wr = a.fd_w + (size_t)(has ? __ldg(a.fd_row + r) : 0) * (4 * D);
#pragma unroll
      for (int ax = 0; ax < D; ++ax)
#pragma unroll
        for (int sd = 0; sd < 2; ++sd) {
          wg1[ax][sd] = has ? wr[2 * ax + sd] : R(0);
          wg2[ax][sd] = has ? wr[2 * D + 2 * ax + sd] : R(0);
        }
    }
    // local state
    constexpr int KMAX = NK > 0 ? NK : MAX_SP;
    constexpr int RMAX = NR > 0 ? NR : MAX_RX;
    const int K = NK > 0 ? NK : c.K;
    const int nrx = NR > 0 ? NR : c.nrx;
    const R Tr = ldg(a.T + r);
    R Yr[KMAX];
    R sW = R(0);
#pragma unroll
    for (int k = 0; k < KMAX; ++k) {
      if (NK > 0 || k < K) {
        Yr[k] = ldg(a.Y + k * N + r);
        sW += Yr[k] * c.inv_W[k];
      } else {
        Yr[k] = R(0);
      }
    }
    const R W = R(1) / sW;
    const R fdr = sizeof(R) == 4 ? (R)a.pth->fd_rho : (R)a.pth->fd_rho_d;
    const R rho = fdr * W / Tr;  // lattice units
    const R rho_phys = rho / c.inv_rho_ref;
    const R inv_rho = R(1) / rho;
    R q[RMAX];
    reaction_rates<NR, R, NK>(c, Tr, R(1) / Tr, Yr, rho_phys, q);
    const R Fr = a.Floc ? ldg(a.Floc + r) : c.F;
    const R mur = c.nu_lat * powr<R>(Tr * c.T_ref_inv, c.mu_exp);
    // variable heat capacities: mixture c_p and the heat of each reaction at T_r
    R cp_r = R(0);
    R heatT[VCP ? RMAX : 1];
    if constexpr (VCP) {
      R hW[KMAX];
#pragma unroll
      for (int k = 0; k < KMAX; ++k) {
        if (NK > 0 || k < K) {
          cp_r += Yr[k] * cp_eval<VDEG, R>(c.cp_poly[k], Tr);
          hW[k] = hW_eval<VDEG, R>(c.hW_poly[k], Tr);
        } else {
          hW[k] = R(0);
        }
      }
#pragma unroll
      for (int j = 0; j < RMAX; ++j) {
        R h = R(0);
#pragma unroll
        for (int k = 0; k < KMAX; ++k) h -= c.nu[j][k] * hW[k];
        heatT[j] = h;
      }
    }
    R ur[3] = {ldg(a.u + r), ldg(a.u + N + r), D == 3 ? ldg(a.u + 2 * N + r) : R(0)};
    const int f = y + g.ny * z;
    const int nf = g.ny * g.nz;
    // face coefficients (F mu) and face velocities
    R FMf[3][2], uf[3][2];
    R Tnb[VCP ? 3 : 1][2], FMn[VCP ? 3 : 1][2];  // VCP: neighbour T and F mu
#pragma unroll
    for (int ax = 0; ax < D; ++ax) {
#pragma unroll
      for (int sd = 0; sd < 2; ++sd) {
        const int kk = k1[ax][sd];
        const int j = i1[ax][sd];
        R Tn = kk == NB_FLUID ? ldg(a.T + j) : (kk == NB_INLET ? c.T_in : Tr);
        if constexpr (GW) {
          if (kk == NB_SOLID) Tn = Tr + wg1[ax][sd] * (ldg(a.T + i1[ax][1 - sd]) - Tr);
        }
        const R Fn = (a.Floc && kk == NB_FLUID) ? ldg(a.Floc + j) : Fr;
        const R mun = c.nu_lat * powr<R>(Tn * c.T_ref_inv, c.mu_exp);
        FMf[ax][sd] = R(0.5) * (Fr * mur + Fn * mun);
        if constexpr (VCP) {
          Tnb[ax][sd] = Tn;
          FMn[ax][sd] = Fn * mun;
        }
        R un;
        if (kk == NB_FLUID) un = ldg(a.u + ax * N + j);
        else if (kk == NB_INLET) un = ldg(a.inlet_u + ax * nf + f);
        else if (kk == NB_OUTLET) un = ur[ax];
        else un = R(0);
        uf[ax][sd] = R(0.5) * (ur[ax] + un);
      }
    }
    // chemistry sources
    const R dt = c.dt_phys;
    const R inv_rpF = R(1) / (rho_phys * Fr);
    R qdot = R(0);
#pragma unroll
    for (int j = 0; j < RMAX; ++j)
      if (NR > 0 || j < nrx) qdot += (VCP ? heatT[j] : c.heat[j]) * q[j];
    const R fd_dT = sizeof(R) == 4 ? (R)a.pth->fd_dT : (R)a.pth->fd_dT_d;
    R lam = R(0);
    R sWn = R(0);
    R Tnew = Tr;
    R yf_new = R(0), yo_new = R(0);  // sensor species of the new state
    // VCP accumulators: neighbour c_p (sum over species of Y_k(n) c_p,k(T_n)) and, per axis,
    // sum_k (c_p,k - c_p)/Le_k (Y_k(r+e) - Y_k(r-e))
    R cpn[VCP ? 3 : 1][2], gYw[VCP ? 3 : 1];
    if constexpr (VCP) {
#pragma unroll
      for (int ax = 0; ax < D; ++ax) {
        cpn[ax][0] = cpn[ax][1] = R(0);
        gYw[ax] = R(0);
      }
    }
    R tflux = R(0);
    // MIX: per face dlnW and the correction sum C_f (ghost neighbours as in the species stencil)
    R mdl[MIX ? 3 : 1][2], mcr[MIX ? 3 : 1][2];
    R Wm = R(0);
    if constexpr (MIX) {
      Wm = a.mix[(size_t)K * N + r];
      const R muin = c.nu_lat * powr<R>(c.T_in * c.T_ref_inv, c.mu_exp);
#pragma unroll
      for (int ax = 0; ax < D; ++ax) {
#pragma unroll
        for (int sd = 0; sd < 2; ++sd) {
          const int kk = k1[ax][sd];
          const int j = i1[ax][sd];
          const R Wn = kk == NB_FLUID ? a.mix[(size_t)K * N + j] : (kk == NB_INLET ? c.W_in : Wm);
          const R dl = (Wn - Wm) / (R(0.5) * (Wn + Wm));
          R cr = R(0);
#pragma unroll
          for (int jj = 0; jj < KMAX; ++jj) {
            if (NK > 0 || jj < K) {
              const R Gr = a.mix[(size_t)jj * N + r];
              const R Gn = kk == NB_FLUID ? a.mix[(size_t)jj * N + j]
                                          : (kk == NB_INLET ? Fr * muin * c.inv_Pr * c.inv_Lemix_in[jj] : Gr);
              const R Yn = kk == NB_FLUID ? ldg(a.Y + (size_t)jj * N + j) : (kk == NB_INLET ? c.Y_in[jj] : Yr[jj]);
              const R Yb = R(0.5) * (Yr[jj] + Yn);
              cr += R(0.5) * (Gr + Gn) * ((Yn - Yr[jj]) + Yb * dl);
            }
          }
          mdl[ax][sd] = dl;
          mcr[ax][sd] = cr;
        }
      }
    }
    // fields: 0 = T, 1.. = Y_k (VCP: the species first, T last)
#pragma unroll 1
    for (int it = 0; it <= K; ++it) {
      const int fi = VCP ? (it == K ? 0 : it + 1) : it;
      R ckr = R(0);
      if constexpr (VCP) {
        if (fi > 0) ckr = cp_eval<VDEG, R>(c.cp_poly[fi - 1], Tr);
      }
      const R* phi = fi == 0 ? a.T : a.Y + (size_t)(fi - 1) * N;
      const R phin = fi == 0 ? c.T_in : c.Y_in[fi - 1];
      const R eps = fi == 0 ? c.eps_T : c.eps_Y;
      const R gfac = c.inv_Pr * (fi == 0 ? R(1) : c.inv_Le[fi - 1]);
      const R pr = ldg(phi + r);
      R adv = R(0), dif = R(0);
#pragma unroll
      for (int ax = 0; ax < D; ++ax) {
        // m1 = phi(r - e), m2 = phi(r - 2e), p1 = phi(r + e), p2 = phi(r + 2e)
        R m1 = k1[ax][0] == NB_INLET ? phin : ldg(phi + i1[ax][0]);
        R m2 = k2[ax][0] == 2 ? phin : ldg(phi + i2[ax][0]);
        R p1 = k1[ax][1] == NB_INLET ? phin : ldg(phi + i1[ax][1]);
        R p2 = k2[ax][1] == 2 ? phin : ldg(phi + i2[ax][1]);
        if constexpr (GW) {
          // ghost-point walls: a distance-1 wall ghost from the parabola through the cell and the
          // opposite point with zero slope at the wall; a distance-2 point copies it, or past a
          // fluid neighbour takes that neighbour's wall ghost
          const R m1r = m1, p1r = p1;
          if (k1[ax][0] == NB_SOLID) {
            m1 = pr + wg1[ax][0] * (p1r - pr);
            m2 = m1;
          } else if (wg2[ax][0] != R(0)) {
            m2 = m1r + wg2[ax][0] * (pr - m1r);
          }
          if (k1[ax][1] == NB_SOLID) {
            p1 = pr + wg1[ax][1] * (m1r - pr);
            p2 = p1;
          } else if (wg2[ax][1] != R(0)) {
            p2 = p1r + wg2[ax][1] * (pr - p1r);
          }
        }
        // WENO3 written with the one-sided differences around r, shared by both faces and the
        // diffusion flux: face = b + (t(d_bc) d_ab + 2 t(d_ab) d_bc) / (2 (t(d_bc) + 2 t(d_ab)))
        // with t(d) = (eps + d^2)^2 (b the upwind value, d_ab, d_bc its upwind-side differences)
        const R dm2 = m1 - m2, dm1 = pr - m1, dp1 = p1 - pr, dp2 = p2 - p1;
        const R sm2 = fma(dm2, dm2, eps), sm1 = fma(dm1, dm1, eps), sp1 = fma(dp1, dp1, eps), sp2 = fma(dp2, dp2, eps);
        const R tm2 = sm2 * sm2, tm1 = sm1 * sm1, tp1 = sp1 * sp1, tp2 = sp2 * sp2;
        const bool up = uf[ax][1] >= R(0), um = uf[ax][0] >= R(0);
        // face r + 1/2: upwind (m1, r, p1) or (p2, p1, r)
        const R bP = up ? pr : p1, dabP = up ? dm1 : -dp2, dbcP = up ? dp1 : -dp1;
        const R tabP = up ? tm1 : tp2, tbcP = up ? tp1 : tp1;
        // face r - 1/2: upwind (m2, m1, r) or (p1, r, m1)
        const R bM = um ? m1 : pr, dabM = um ? dm2 : -dp1, dbcM = um ? dm1 : -dm1;
        const R tabM = um ? tm2 : tp1, tbcM = um ? tm1 : tm1;
        const R fp = bP + R(0.5) * fdiv<R>(tbcP * dabP + R(2) * tabP * dbcP, tbcP + R(2) * tabP);
        const R fm = bM + R(0.5) * fdiv<R>(tbcM * dabM + R(2) * tabM * dbcM, tbcM + R(2) * tabM);
        adv += ur[ax] * (fp - fm);
        if constexpr (VCP) {
          if (fi > 0) {
            cpn[ax][0] += m1 * cp_eval<VDEG, R>(c.cp_poly[fi - 1], Tnb[ax][0]);
            cpn[ax][1] += p1 * cp_eval<VDEG, R>(c.cp_poly[fi - 1], Tnb[ax][1]);
            gYw[ax] += (ckr - cp_r) * c.inv_Le[fi - 1] * (p1 - m1);
            dif += FMf[ax][1] * dp1 - FMf[ax][0] * dm1;
          } else {
            const R Frm = Fr * mur * cp_r;
            dif += R(0.5) * (Frm + FMn[ax][1] * cpn[ax][1]) * dp1 - R(0.5) * (Frm + FMn[ax][0] * cpn[ax][0]) * dm1;
            tflux += gYw[ax] * (p1 - m1);
          }
        } else if (MIX && fi > 0) {
          const R Gr = a.mix[(size_t)(fi - 1) * N + r];
#pragma unroll
          for (int sd = 0; sd < 2; ++sd) {
            const int kk = k1[ax][sd];
            const R Gn = kk == NB_FLUID ? a.mix[(size_t)(fi - 1) * N + i1[ax][sd]]
                                        : (kk == NB_INLET ? Fr * c.nu_lat * powr<R>(c.T_in * c.T_ref_inv, c.mu_exp) *
                                                                c.inv_Pr * c.inv_Lemix_in[fi - 1]
                                                          : Gr);
            const R pn = sd ? p1 : m1;
            const R Yb = R(0.5) * (pr + pn);
            dif += R(0.5) * (Gr + Gn) * ((pn - pr) + Yb * mdl[ax][sd]) - Yb * mcr[ax][sd];
          }
        } else {
          dif += FMf[ax][1] * dp1 - FMf[ax][0] * dm1;
        }
      }
      R src;
      if (VCP && fi == 0) {
        const R inv_cpr = R(1) / cp_r;
        dif = (dif + R(0.25) * Fr * mur * tflux) * gfac * inv_rho * inv_cpr;
        src = (dt * qdot * inv_rpF + fd_dT * inv_rho / c.inv_cp) * inv_cpr;
      } else if (fi == 0) {
        dif *= gfac * inv_rho;
        src = dt * qdot * inv_rpF * c.inv_cp + fd_dT * inv_rho;
      } else {
        dif *= (MIX ? R(1) : gfac) * inv_rho;
        R om = R(0);
#pragma unroll
        for (int j = 0; j < RMAX; ++j)
          if (NR > 0 || j < nrx) om += c.nu[j][fi - 1] * q[j];
        src = dt * c.W[fi - 1] * om * inv_rpF;
      }
      const R NA = dif + src;
      const R pn = pr - adv + NA;
      if (fi == 0) {
        a.T_out[r] = pn;
        lam += NA / Tr;
        Tnew = pn;
      } else {
        a.Y_out[(size_t)(fi - 1) * N + r] = pn;
        lam += W * c.inv_W[fi - 1] * NA;
        sWn += pn * c.inv_W[fi - 1];
        if (fi - 1 == c.sensor_species) yf_new = pn;
        if (fi - 1 == c.sensor_oxidizer) yo_new = pn;
      }
    }
    // flame sensor of the new state (the separate sensor pass for the next step, fused)
    if (a.Floc_out) a.Floc_out[r] = sensor_floc<R>(c, Tnew, yf_new, yo_new);
    a.rho_out[r] = rho;
    a.lam_out[r] = lam;
    if (c.closed) {
      // W_new / (R T_new rho_ref), pre-scaled; gas constant folded into I_scale
      termI = c.I_scale / (sWn * Tnew);
      if (x == 0 && g.bc_lo[0] == BC_INLET) {
        const R rin = sizeof(R) == 4 ? (R)a.pth->rho_in : (R)a.pth->rho_in_d;
        termM += c.M_scale * rin * ldg(a.inlet_u + f);
      }
      if (x == g.nx - 1 && g.bc_hi[0] == BC_OUTLET) termM -= c.M_scale * rho * ur[0];
    }
    }
}

// NK, NR > 0: species and reaction counts known at compile time (loops unroll exactly);
// NK = NR = 0: counts read from the constants at run time.
#ifndef HLBM_FD_MIN_BLOCKS
#define HLBM_FD_MIN_BLOCKS 4  // FP32: resident blocks per SM the register budget is sized for
#endif
#ifndef HLBM_FD_VCP_MIN_BLOCKS
#define HLBM_FD_VCP_MIN_BLOCKS 4  // the same for the variable heat-capacity variant (measured: 2 blocks 2.24 ms, 3 blocks 1.72 ms, 4 blocks 1.60 ms per C4 launch)
#endif
template <int D, typename R, int NK, int NR, int VDEG = 0, bool MIX = false>
__global__ void __launch_bounds__(FD_BLOCK, sizeof(R) == 4 ? (VDEG > 0 ? HLBM_FD_VCP_MIN_BLOCKS : HLBM_FD_MIN_BLOCKS) : 1)
    fd_step_kernel(const FDArgs<R> a) {
  const FDConst<R>& c = a.c;
  const Geo& g = a.geo;
  int x, y, z, r;
  bool inside;
  if (a.wall_list) {
    // one thread per listed cell (a 1-D grid of blocks of the same shape)
    const int wrow = blockIdx.x * FD_BLOCK + threadIdx.x + FDShape<D>::X * (threadIdx.y + FDShape<D>::Y * threadIdx.z);
    inside = wrow < a.n_wall_list;
    r = inside ? __ldg(a.wall_list + wrow) : 0;
    x = r % g.nx;
    y = (r / g.nx) % g.ny;
    z = r / (g.nx * g.ny);
  } else {
    x = blockIdx.x * FDShape<D>::X + threadIdx.x;
    y = blockIdx.y * FDShape<D>::Y + threadIdx.y;
    z = blockIdx.z * FDShape<D>::Z + threadIdx.z;
    inside = x < g.nx && y < g.ny && z < g.nz;
    r = x + g.nx * (y + g.ny * z);
  }
  const uint32_t sw = inside ? __ldg(a.sword + r) : 0u;
  // walls_only: the launch after the tiled update, for the cells with ghost-point wall weights
  const bool active = (sw >> 31) != 0u && (!a.walls_only || (sw & SW_WALL) != 0u);
  R termI = R(0), termM = R(0);  // P_th integrand and boundary mass flux of this cell

  // interior fast path: stencil word without any non-fluid neighbour, cell 2 away from every face
  const uint32_t ghosts = sw & (D == 3 ? 0x00ffffffu : 0x0000ffffu);
  const bool fast = ghosts == 0u && x >= 2 && x < g.nx - 2 && y >= 2 && y < g.ny - 2 &&
                    (D == 2 || (z >= 2 && z < g.nz - 2));
  // one copy of the update per warp (a warp is a row of 32 cells along x): a warp whose cells
  // would take different copies takes the most general one any of them needs, rather than
  // issuing several in turn; the copies compute identical values
  const bool warp_fast = __all_sync(0xffffffffu, !active || fast);
  const bool warp_walls = __any_sync(0xffffffffu, active && (sw & SW_WALL) != 0u);
  if (active) {
    if constexpr (MIX) {
      // mixture-averaged diffusion has no ghost-point wall copy (lbm_set_transport refuses walls)
      if (warp_fast) fd_cell<D, R, NK, NR, true, 0, false, true>(a, x, y, z, r, sw, termI, termM);
      else fd_cell<D, R, NK, NR, false, 0, false, true>(a, x, y, z, r, sw, termI, termM);
    } else {
      if (warp_fast) fd_cell<D, R, NK, NR, true, VDEG>(a, x, y, z, r, sw, termI, termM);
      else if (warp_walls) fd_cell<D, R, NK, NR, false, VDEG, true>(a, x, y, z, r, sw, termI, termM);
      else fd_cell<D, R, NK, NR, false, VDEG>(a, x, y, z, r, sw, termI, termM);
    }
  }
  if (!c.closed) return;  // uniform across the grid
  // block reduction of the two terms into this block's partial slot
  __shared__ long long sI[FD_BLOCK / 32], sM[FD_BLOCK / 32];
  __shared__ double dI[FD_BLOCK / 32], dM[FD_BLOCK / 32];
  const int tid = threadIdx.x + FDShape<D>::X * (threadIdx.y + FDShape<D>::Y * threadIdx.z);
  const int lane = tid & 31, wid = tid >> 5;
  const int bid = a.part_offset + blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
  if constexpr (sizeof(R) == 4) {
    long long vI = warp_sum_ll(f32_to_fix32((float)termI));
    long long vM = warp_sum_ll(f32_to_fix32((float)termM));
    if (lane == 0) { sI[wid] = vI; sM[wid] = vM; }
    __syncthreads();
    if (tid == 0) {
      long long tI = 0, tM = 0;
      for (int w = 0; w < FD_BLOCK / 32; ++w) { tI += sI[w]; tM += sM[w]; }
      long long* out = (long long*)a.partials;
      out[2 * bid] = tI;
      out[2 * bid + 1] = tM;
    }
  } else {
    double vI = (double)termI, vM = (double)termM;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      vI += __shfl_down_sync(0xffffffffu, vI, o);
      vM += __shfl_down_sync(0xffffffffu, vM, o);
    }
    if (lane == 0) { dI[wid] = vI; dM[wid] = vM; }
    __syncthreads();
    if (tid == 0) {
      double tI = 0, tM = 0;
      for (int w = 0; w < FD_BLOCK / 32; ++w) { tI += dI[w]; tM += dM[w]; }
      double* out = (double*)a.partials;
      out[2 * bid] = tI;
      out[2 * bid + 1] = tM;
    }
  }
}

template <int D> inline dim3 fd_grid(const Geo& g) {
  return dim3((g.nx + FDShape<D>::X - 1) / FDShape<D>::X, (g.ny + FDShape<D>::Y - 1) / FDShape<D>::Y,
              (g.nz + FDShape<D>::Z - 1) / FDShape<D>::Z);
}
template <int D> inline int fd_blocks(const Geo& g) {
  const dim3 b = fd_grid<D>(g);
  return (int)(b.x * b.y * b.z);
}

// variable heat capacities: fd_kernels_vcp.cu
template <int D, typename R> cudaError_t launch_fd_vcp(const FDArgs<R>& a, cudaStream_t st);
// mixture-averaged species diffusion: fd_kernels_mix.cu (coefficient pass + update)
template <int D, typename R> cudaError_t launch_fd_mix(const FDArgs<R>& a, R* mix, cudaStream_t st);

template <int D, typename R>
cudaError_t launch_fd(const FDArgs<R>& a, cudaStream_t st, bool sensor_pass) {
  if (!sensor_pass && a.c.varcp) return launch_fd_vcp<D, R>(a, st);
  if (!sensor_pass && a.c.mixavg) return launch_fd_mix<D, R>(a, const_cast<R*>(a.mix), st);
  if (sensor_pass) {
    const int grid = (a.geo.N + FD_BLOCK - 1) / FD_BLOCK;
    flame_sensor_kernel<D, R><<<grid, FD_BLOCK, 0, st>>>(a);
  } else {
    const dim3 grid = a.wall_list ? dim3((a.n_wall_list + FD_BLOCK - 1) / FD_BLOCK) : fd_grid<D>(a.geo);
    const dim3 block(FDShape<D>::X, FDShape<D>::Y, FDShape<D>::Z);
    if (a.c.K == 6 && a.c.nrx == 2) fd_step_kernel<D, R, 6, 2><<<grid, block, 0, st>>>(a);
    else if (a.c.K == 4 && a.c.nrx == 1) fd_step_kernel<D, R, 4, 1><<<grid, block, 0, st>>>(a);
    else fd_step_kernel<D, R, 0, 0><<<grid, block, 0, st>>>(a);
  }
  return cudaGetLastError();
}

}  // namespace hlbm
