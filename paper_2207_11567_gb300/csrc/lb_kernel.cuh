// Fused pull-stream + collide kernel of the pressure/momentum lattice Boltzmann solver
// (Section 2.1-2.2), one thread per cell, lattice units (c_s^2 = 1/3).
//
// Per fluid cell:
//   stream   g_i(r) = g*_i(r - c_i) (Eq. 1, pull), bounce-back g_i = g*_{Q-1-i}(r) on links
//            marked in the cell's link word, plus 2 w_i rho (c_i . u_w) on low-x inlet links;
//   moments  P_h = sum g + rho Lambda / 6, u = 3 sum c g / rho (Eq. 7);
//   source   Xi_i = w_i [ (c.u/cs2 + (c.u)^2/(2 cs4) - u^2/(2 cs2)) cs2 (c_i - u).grad rho
//            + rho cs2 Lambda ] (Eq. 2 with Eq. 4 inserted);
//   precond  f'_i = 3 (g_i + Xi_i / 2) / rho (Eq. 13); p' = sum f'; h = f' - (p' - 1) w;
//   collide  cumulants of h about u (central moments by the axis-by-axis transform), shear rate
//            1/tau with tau from Eq. 12 plus the Smagorinsky closure, trace rate omega_b,
//            orders 3..6 with omega_hi; or the single-rate (BGK) relaxation of h to f^eq(1, u);
//   post     g*_i = rho/3 (h*_i + (p' - 1) w_i) + Xi_i / 2 (Eq. 8), stored shifted as
//            (g* - w P_ref) / w.
// Arithmetic is arranged so that no O(1) offset is ever added and cancelled again (which costs
// FP32 its precision): with q_i = g_i / w_i - P_ref, xi_i = Xi_i / w_i, s_i = q_i + xi_i / 2 and
// S = sum_j w_j s_j, one has h_i / w_i - 1 = 3 (s_i - S) / rho and
// g*_i / w_i - P_ref = rho/3 (h*_i / w_i - 1) + S + xi_i / 2; the cumulant collision works on
// h - h_eq with h_eq the product-form equilibrium, whose central moments are known exactly.
#pragma once
#include "common.cuh"

namespace hlbm {

// central-moment transform of one line of three values (c = -1, 0, +1) about velocity u
template <typename R> __device__ __forceinline__ void chim_fwd(R& a, R& b, R& c, const R u) {
  const R m0 = a + b + c;
  const R d = c - a;
  const R s = c + a;
  a = m0;
  b = d - u * m0;
  c = s - R(2) * u * d + u * u * m0;
}
template <typename R> __device__ __forceinline__ void chim_bwd(R& a, R& b, R& c, const R u) {
  const R m0 = a, m1 = b, m2 = c;
  const R k1 = m1 + u * m0;
  const R k2 = m2 + R(2) * u * m1 + u * u * m0;
  a = R(0.5) * (k2 - k1);
  b = m0 - k2;
  c = R(0.5) * (k2 + k1);
}

// x^y for x > 0: FP32 via the hardware log2 / exp2 (relative error a few 1e-7), FP64 with pow
template <typename R> __device__ __forceinline__ R pw(R x, R y);
template <> __device__ __forceinline__ float pw<float>(float x, float y) { return exp2f(y * __log2f(x)); }
template <> __device__ __forceinline__ double pw<double>(double x, double y) { return pow(x, y); }

// Cumulant relaxation in deviation form. n[] holds the central moments (slot a + 3b [+ 9c])
// of e = h - h_eq, where h_eq is the product-form equilibrium at the cell velocity; the central
// moments of h_eq are exactly 0 for any odd index and (1/3)^k for k indices equal to 2, so the
// full central moments are kappa = kappa_eq + n. All formulas below are the cumulant relations
// (partition formula, unit density) rewritten in n, so that every FP32 quantity is small.
template <bool FULL, typename R>
__device__ __forceinline__ void cumulant_relax2(R* n, const R om, const R omb, const R om3, const R om4) {
  const R third = R(1) / R(3);
  const R n20 = n[2], n02 = n[6], n11 = n[4];
  const R C22 = FULL ? R(0) : n[8] - third * (n20 + n02) - n20 * n02 - R(2) * n11 * n11;
  const R tr = R(0.5) * (n20 + n02);
  const R o1 = R(1) - om, ob = R(1) - omb;
  const R s20 = o1 * (n20 - tr) + ob * tr;
  const R s02 = o1 * (n02 - tr) + ob * tr;
  const R s11 = o1 * n11;
  n[2] = s20; n[6] = s02; n[4] = s11;
  if constexpr (FULL) {
    n[5] = R(0);
    n[7] = R(0);
    n[8] = third * (s20 + s02) + s20 * s02 + R(2) * s11 * s11;
  } else {
    n[5] *= (R(1) - om3);
    n[7] *= (R(1) - om3);
    n[8] = (R(1) - om4) * C22 + third * (s20 + s02) + s20 * s02 + R(2) * s11 * s11;
  }
}

template <bool FULL, typename R>
__device__ __forceinline__ void cumulant_relax3(R* n, const R om, const R omb, const R om3,
                                                const R om4, const R om5, const R om6) {
#define K(a, b, c) n[(a) + 3 * (b) + 9 * (c)]
  const R third = R(1) / R(3), ninth = R(1) / R(9);
  const R a = K(2, 0, 0), b = K(0, 2, 0), c = K(0, 0, 2);
  const R n110 = K(1, 1, 0), n101 = K(1, 0, 1), n011 = K(0, 1, 1);
  const R n210 = K(2, 1, 0), n201 = K(2, 0, 1), n120 = K(1, 2, 0);
  const R n021 = K(0, 2, 1), n102 = K(1, 0, 2), n012 = K(0, 1, 2), n111 = K(1, 1, 1);
  const R n211 = K(2, 1, 1), n121 = K(1, 2, 1), n112 = K(1, 1, 2);
  const R n220 = K(2, 2, 0), n202 = K(2, 0, 2), n022 = K(0, 2, 2);
  // forward cumulants of order 4, 5, 6 (not needed when those orders relax fully)
  R C211 = R(0), C121 = R(0), C112 = R(0), C220 = R(0), C202 = R(0), C022 = R(0);
  R C221 = R(0), C212 = R(0), C122 = R(0), C222 = R(0);
  if constexpr (!FULL) {
    C211 = n211 - third * n011 - a * n011 - R(2) * n110 * n101;
    C121 = n121 - third * n101 - b * n101 - R(2) * n110 * n011;
    C112 = n112 - third * n110 - c * n110 - R(2) * n101 * n011;
    C220 = n220 - third * (a + b) - a * b - R(2) * n110 * n110;
    C202 = n202 - third * (a + c) - a * c - R(2) * n101 * n101;
    C022 = n022 - third * (b + c) - b * c - R(2) * n011 * n011;
    C221 = K(2, 2, 1) - ((third + a) * n021 + (third + b) * n201 + R(4) * n110 * n111 +
                                 R(2) * n101 * n120 + R(2) * n011 * n210);
    C212 = K(2, 1, 2) - ((third + a) * n012 + (third + c) * n210 + R(4) * n101 * n111 +
                                 R(2) * n110 * n102 + R(2) * n011 * n201);
    C122 = K(1, 2, 2) - ((third + c) * n120 + (third + b) * n102 + R(4) * n011 * n111 +
                                 R(2) * n101 * n021 + R(2) * n110 * n012);
    C222 = K(2, 2, 2) + ninth * (a + b + c) - third * (n022 + n202 + n220) -
                   (a * n022 + b * n202 + c * n220) -
                   R(4) * (n110 * n112 + n101 * n121 + n011 * n211) -
                   (R(2) * (n210 * n012 + n201 * n021 + n120 * n102) + R(4) * n111 * n111) +
                   R(2) * third * (a * b + b * c + c * a) + R(2) * a * b * c +
                   R(4) * ((third + a) * n011 * n011 + (third + b) * n101 * n101 + (third + c) * n110 * n110) +
                   R(16) * n110 * n101 * n011;
  }
  // second order: trace deviation (rate omega_b) and deviatoric part (rate omega)
  const R tr = third * (a + b + c);
  const R o1 = R(1) - om, ob = R(1) - omb;
  const R s200 = o1 * (a - tr) + ob * tr;
  const R s020 = o1 * (b - tr) + ob * tr;
  const R s002 = o1 * (c - tr) + ob * tr;
  const R s110 = o1 * n110, s101 = o1 * n101, s011 = o1 * n011;
  const R o3 = FULL ? R(0) : R(1) - om3;
  const R s210 = FULL ? R(0) : o3 * n210, s201 = FULL ? R(0) : o3 * n201, s120 = FULL ? R(0) : o3 * n120;
  const R s021 = FULL ? R(0) : o3 * n021, s102 = FULL ? R(0) : o3 * n102, s012 = FULL ? R(0) : o3 * n012;
  const R s111 = FULL ? R(0) : o3 * n111;
  const R o4 = FULL ? R(0) : R(1) - om4, o5 = FULL ? R(0) : R(1) - om5, o6 = FULL ? R(0) : R(1) - om6;
  const R D211 = FULL ? R(0) : o4 * C211, D121 = FULL ? R(0) : o4 * C121, D112 = FULL ? R(0) : o4 * C112;
  const R D220 = FULL ? R(0) : o4 * C220, D202 = FULL ? R(0) : o4 * C202, D022 = FULL ? R(0) : o4 * C022;
  // back to central moments (deviation form)
  K(2, 0, 0) = s200; K(0, 2, 0) = s020; K(0, 0, 2) = s002;
  K(1, 1, 0) = s110; K(1, 0, 1) = s101; K(0, 1, 1) = s011;
  K(2, 1, 0) = s210; K(2, 0, 1) = s201; K(1, 2, 0) = s120;
  K(0, 2, 1) = s021; K(1, 0, 2) = s102; K(0, 1, 2) = s012; K(1, 1, 1) = s111;
  K(2, 1, 1) = D211 + (third + s200) * s011 + R(2) * s110 * s101;
  K(1, 2, 1) = D121 + (third + s020) * s101 + R(2) * s110 * s011;
  K(1, 1, 2) = D112 + (third + s002) * s110 + R(2) * s101 * s011;
  K(2, 2, 0) = D220 + third * (s200 + s020) + s200 * s020 + R(2) * s110 * s110;
  K(2, 0, 2) = D202 + third * (s200 + s002) + s200 * s002 + R(2) * s101 * s101;
  K(0, 2, 2) = D022 + third * (s020 + s002) + s020 * s002 + R(2) * s011 * s011;
  K(2, 2, 1) = (FULL ? R(0) : o5 * C221) + (third + s200) * s021 + (third + s020) * s201 + R(4) * s110 * s111 +
               R(2) * s101 * s120 + R(2) * s011 * s210;
  K(2, 1, 2) = (FULL ? R(0) : o5 * C212) + (third + s200) * s012 + (third + s002) * s210 + R(4) * s101 * s111 +
               R(2) * s110 * s102 + R(2) * s011 * s201;
  K(1, 2, 2) = (FULL ? R(0) : o5 * C122) + (third + s002) * s120 + (third + s020) * s102 + R(4) * s011 * s111 +
               R(2) * s101 * s021 + R(2) * s110 * s012;
  const R A = (third + s200) * D022 + (third + s020) * D202 + (third + s002) * D220;
  const R B = R(4) * (s110 * D112 + s101 * D121 + s011 * D211);
  const R C3 = R(2) * (s210 * s012 + s201 * s021 + s120 * s102) + R(4) * s111 * s111;
  const R Dd = ninth * (s200 + s020 + s002) + third * (s200 * s020 + s020 * s002 + s002 * s200) +
               s200 * s020 * s002 +
               R(2) * ((third + s200) * s011 * s011 + (third + s020) * s101 * s101 + (third + s002) * s110 * s110) +
               R(8) * s110 * s101 * s011;
  K(2, 2, 2) = (FULL ? R(0) : o6 * C222) + A + B + C3 + Dd;
#undef K
}

// Central moments of the product-form equilibrium minus those of the rest weights w, both
// about u, for the moment (a, b, c): prod ke - prod (ke + dl) with ke = (1, 0, 1/3) and
// dl = (0, -u, u^2) per axis, expanded so that only small terms are formed.
template <int D, int J, typename R>
__device__ __forceinline__ R delta_eq(const R* dx, const R* dy, const R* dz) {
  constexpr int a = J % 3, b = (J / 3) % 3, c = J / 9;
  const R kx = a == 0 ? R(1) : (a == 1 ? R(0) : R(1) / R(3));
  const R ky = b == 0 ? R(1) : (b == 1 ? R(0) : R(1) / R(3));
  const R kz = c == 0 ? R(1) : (c == 1 ? R(0) : R(1) / R(3));
  const R ex = dx[a], ey = dy[b], ez = (D == 3) ? dz[c] : R(0);
  if constexpr (D == 2) return -(ex * ky + kx * ey + ex * ey);
  return -(ex * ky * kz + kx * ey * kz + kx * ky * ez + ex * ey * kz + ex * ky * ez + kx * ey * ez + ex * ey * ez);
}

// m[J] += sign * delta_eq for the moments whose order a + b + c lies in [LO, HI]
template <int D, typename R, int J, int LO = 0, int HI = 6>
__device__ __forceinline__ void add_delta_eq(R* m, const R* dx, const R* dy, const R* dz, const R sign) {
  if constexpr (J < Lat<D>::Q) {
    constexpr int order = J % 3 + (J / 3) % 3 + J / 9;
    if constexpr (order >= LO && order <= HI) m[J] += sign * delta_eq<D, J, R>(dx, dy, dz);
    add_delta_eq<D, R, J + 1, LO, HI>(m, dx, dy, dz, sign);
  }
}

// WALLS = false: every fluid cell except those flagged LINK_WALL, one block row per (y, z).
// WALLS = true: the flagged cells only, one thread per entry of the wall list, with the
// interpolated bounce-back fix-up compiled in (so that it costs the other cells no registers).
template <int D, typename S, typename R, bool THERMAL, int COLL, bool WALLS>
__global__ void __launch_bounds__(LB_BLOCK, LB_MIN_BLOCKS) lb_step_kernel(const LBArgs<R> a) {
  constexpr int Q = Lat<D>::Q;
  const int nx = a.geo.nx, ny = a.geo.ny, nz = a.geo.nz;
  int x, y, z, r, wrow = 0;
  if constexpr (WALLS) {
    // one thread per cell of the interpolated-wall list (its position is the table row)
    wrow = blockIdx.x * LB_BLOCK + threadIdx.x;
    if (wrow >= a.n_wall) return;
    r = __ldg(a.wall_cells + wrow);
    x = r % nx;
    y = (r / nx) % ny;
    z = r / (nx * ny);
  } else {
    // one block row of LB_BLOCK cells along x; y and z come from the grid (no integer division)
    x = blockIdx.x * LB_BLOCK + threadIdx.x;
    y = blockIdx.y;
    z = blockIdx.z;
    if (x >= nx) return;
    r = x + nx * (y + ny * z);
  }
  // the cell's rho, Lambda and T are loaded together with its link word (every cell has them)
  R rho = R(1), lam = R(0), T_early = R(0);
  if constexpr (THERMAL) {
    rho = ldg(a.rho + r);
    lam = ldg(a.lam + r);
    T_early = ldg(a.T + r);
  }
  const uint32_t lw = __ldg(a.links + r);
  if (!(lw >> 31)) return;
  if (!WALLS && (lw & LINK_WALL)) return;  // done by the wall-list launch
  const size_t N = (size_t)a.geo.N;
  const S* __restrict__ gin = (const S*)a.g_in;
  const R third = R(1) / R(3);
  R rho_p[3] = {rho, rho, rho}, rho_m[3] = {rho, rho, rho};  // rho at r + e_a, r - e_a

  // ---------------------------------------------------------------- pull streaming
  // q_i = g_i / w_i - P_ref (the stored shifted form). Offsets fit in 32 bits (checked at init).
  // Per-axis offsets to the minus / plus neighbour, wrapped on periodic faces (a plain pull across
  // a non-periodic face never happens: those links are bounce-back, inlet or outlet links).
  // phase 1 issues every load into raw[] (storage type), phase 2 converts: all loads of a cell
  // are in flight together whatever the storage type
  S raw[Q];
  const int sy_ = nx, sz_ = nx * ny;
  const int Ni = a.geo.N;
  const int oxm = x > 0 ? -1 : nx - 1, oxp = x < nx - 1 ? 1 : 1 - nx;
  const int oym = y > 0 ? -sy_ : (ny - 1) * sy_, oyp = y < ny - 1 ? sy_ : (1 - ny) * sy_;
  const int ozm = z > 0 ? -sz_ : (nz - 1) * sz_, ozp = z < nz - 1 ? sz_ : (1 - nz) * sz_;
  const bool outlet_cell = x == nx - 1 && a.geo.bc_hi[0] == BC_OUTLET;
  // interior warp: no lane has a bounce-back, inlet or outlet link or sits on a periodic face, so
  // every pull is a plain offset (same loads as below, without the per-direction link tests)
  const bool interior = !WALLS && (lw & ((1u << Q) - 1u)) == 0u && x > 0 && x < nx - 1 && y > 0 &&
                        y < ny - 1 && (D == 2 || (z > 0 && z < nz - 1));
  if (!WALLS && __all_sync(__activemask(), interior)) {
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const int ci = cx(i), cj = cy(i), ck = (D == 3) ? cz(i) : 0;
      raw[i] = ld_raw<S>(gin + i * Ni + r - ci - cj * sy_ - ck * sz_);
    }
    if constexpr (THERMAL) {
      rho_p[0] = ldg(a.rho + r + 1);
      rho_m[0] = ldg(a.rho + r - 1);
      rho_p[1] = ldg(a.rho + r + sy_);
      rho_m[1] = ldg(a.rho + r - sy_);
      if (D == 3) {
        rho_p[2] = ldg(a.rho + r + sz_);
        rho_m[2] = ldg(a.rho + r - sz_);
      }
    }
  } else {
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const int ci = cx(i), cj = cy(i), ck = (D == 3) ? cz(i) : 0;
    if ((lw >> i) & 1u) {
      raw[i] = ld_raw<S>(gin + (Q - 1 - i) * Ni + r);
    } else {
      // source r - c_i
      const int s = r + (ci == 1 ? oxm : (ci == -1 ? oxp : 0)) + (cj == 1 ? oym : (cj == -1 ? oyp : 0)) +
                    (ck == 1 ? ozm : (ck == -1 ? ozp : 0));
      raw[i] = ld_raw<S>(gin + i * Ni + s);
      if constexpr (THERMAL) {
        if (ci * ci + cj * cj + ck * ck == 1) {
          // direction -e_a pulls from r + e_a; +e_a pulls from r - e_a
          const R rs = ldg(a.rho + s);
          if (ci == -1) rho_p[0] = rs;
          if (ci == 1) rho_m[0] = rs;
          if (cj == -1) rho_p[1] = rs;
          if (cj == 1) rho_m[1] = rs;
          if (D == 3 && ck == -1) rho_p[2] = rs;
          if (D == 3 && ck == 1) rho_m[2] = rs;
        }
      }
    }
  }
  }
  // the thermodynamic-pressure state of this step: after the kernel that updates it (launched just
  // before this one; the loads above read only what earlier kernels wrote)
  pdl_wait();
  if constexpr (THERMAL) {
    if constexpr (sizeof(R) == 8) lam += (R)a.pth->lb_lam_d;
    else lam += (R)a.pth->lb_lam;
  }
  R q[Q];
#pragma unroll
  for (int i = 0; i < Q; ++i) q[i] = cvt_pop<S, R>(raw[i]);
  // interpolated bounce-back (curved or offset walls) on flagged cells: for a link whose wall
  // lies at the fraction f of r -> r - c_i, with o the opposite direction and q_i = g*_o(r) above,
  //   f <  1/2:  g_i = 2 f g*_o(r) + (1 - 2 f) g*_o(r + c_i) = g*_o(r + c_i) + 2 f (g*_o(r) - g*_o(r + c_i))
  //   f >= 1/2:  g_i = g*_o(r) / (2 f) + (2 f - 1) / (2 f) g*_i(r) = g*_i(r) + (g*_o(r) - g*_i(r)) / (2 f)
  // (affine with weights summing to 1, so it holds for the shifted stored form as well; the
  // right-hand forms round once, on a difference of neighbouring populations)
  if constexpr (WALLS) {
    const R* __restrict__ wq = a.wall_q + (size_t)wrow * Q;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      if ((lw >> i) & 1u) {
        const R f = wq[i];
        if (f != R(0.5)) {
          const int ci = cx(i), cj = cy(i), ck = (D == 3) ? cz(i) : 0;
          if (f < R(0.5)) {
            // r + c_i: the pull source of the opposite direction (a fluid node, checked at set-up)
            const int s = r + (ci == -1 ? oxm : (ci == 1 ? oxp : 0)) + (cj == -1 ? oym : (cj == 1 ? oyp : 0)) +
                          (ck == -1 ? ozm : (ck == 1 ? ozp : 0));
            const R far_o = cvt_pop<S, R>(ld_raw<S>(gin + (Q - 1 - i) * Ni + s));
            q[i] = far_o + R(2) * f * (q[i] - far_o);  // one rounding on a small difference
          } else {
            const R own_i = cvt_pop<S, R>(ld_raw<S>(gin + i * Ni + r));
            q[i] = own_i + (q[i] - own_i) / (R(2) * f);
          }
        }
      }
    }
  }
  // moving-wall term of the low-x inlet: g_i += 2 w_i rho (c_i . u_w)
  if (x == 0 && a.geo.bc_lo[0] == BC_INLET) {
    const int f = y + ny * z;
    const int nf = ny * nz;
    const R uw0 = ldg(a.inlet_u + f), uw1 = ldg(a.inlet_u + nf + f);
    const R uw2 = (D == 3) ? ldg(a.inlet_u + 2 * nf + f) : R(0);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      if (cx(i) == 1) {
        if ((lw >> i) & 1u) {
          const R cu = uw0 + (R)cy(i) * uw1 + ((D == 3) ? (R)cz(i) * uw2 : R(0));
          q[i] += R(2) * rho * cu;
        }
      }
    }
  }
  // pressure outlet (anti-bounce-back at the half-way face, P_h = P_ref):
  // g_i = -g*_opp + 2 w_i (P_ref + rho (1.5 (c_i.u)^2 - 0.5 u^2)), u of the previous step
  if (outlet_cell) {
    const R vx = a.u_in[r], vy = a.u_in[N + r], vz = (D == 3) ? a.u_in[2 * N + r] : R(0);
    const R vv = vx * vx + vy * vy + vz * vz;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      if (cx(i) == -1) {
        if ((lw >> i) & 1u) {
          const R cu = -vx + (R)cy(i) * vy + ((D == 3) ? (R)cz(i) * vz : R(0));
          q[i] = -q[i] + rho * (R(3) * cu * cu - vv);
        }
      }
    }
  }

  // ---------------------------------------------------------------- moments (Eq. 7)
  R psum = R(0), mx = R(0), my = R(0), mz = R(0);
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const R wq = (R)wgt<D>(i) * q[i];
    psum += wq;
    if (cx(i) == 1) mx += wq;
    if (cx(i) == -1) mx -= wq;
    if (cy(i) == 1) my += wq;
    if (cy(i) == -1) my -= wq;
    if (D == 3) {
      if (cz(i) == 1) mz += wq;
      if (cz(i) == -1) mz -= wq;
    }
  }
  const R inv_rho = R(1) / rho;
  const R ux = R(3) * mx * inv_rho, uy = R(3) * my * inv_rho, uz = (D == 3) ? R(3) * mz * inv_rho : R(0);
  const R usq = ux * ux + uy * uy + uz * uz;
  R gx = R(0), gy = R(0), gz = R(0), udg = R(0);
  if constexpr (THERMAL) {
    gx = R(0.5) * (rho_p[0] - rho_m[0]);
    gy = R(0.5) * (rho_p[1] - rho_m[1]);
    if (D == 3) gz = R(0.5) * (rho_p[2] - rho_m[2]);
    udg = ux * gx + uy * gy + uz * gz;
  }
  const R rl3 = rho * lam * third;  // rho cs2 Lambda

  // ------------------------------ source xi_i = Xi_i / w_i (Eq. 2) and pre-conditioning (Eq. 13)
  // s_i = q_i + xi_i / 2, S = sum w s; d_i = h_i / w_i - 1 = 3 (s_i - S) / rho.
  // With full relaxation of orders 3..6 the collision reads the source only through the central
  // moments of w xi of orders 0..2 (the higher ones are overwritten), which have closed forms on
  // the product-weight lattices: with L = rho cs2 Lambda and G = u . grad rho,
  //   k_0 = L + G/3, k_a = -u_a k_0, k_aa = L u_a^2 + L/3 + (G + 2 g_a u_a)/9,
  //   k_ab = L u_a u_b + (g_a u_b + g_b u_a)/9 (a != b);
  // they are added to the moments after the forward transform (SRC_MOM); otherwise the source is
  // added per direction here.
  constexpr bool SRC_MOM = THERMAL && COLL == COLL_CUMULANT_FULL;
  R Ssum = R(0);
  R k0 = R(0);
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    if constexpr (THERMAL && !SRC_MOM) {
      const R cu = (R)cx(i) * ux + (R)cy(i) * uy + ((D == 3) ? (R)cz(i) * uz : R(0));
      const R cg = (R)cx(i) * gx + (R)cy(i) * gy + ((D == 3) ? (R)cz(i) * gz : R(0));
      const R e = cu + R(1.5) * cu * cu - R(0.5) * usq;  // (f^eq/rho - w)/w * cs2
      q[i] += R(0.5) * (e * (cg - udg) + rl3);
    }
    Ssum += (R)wgt<D>(i) * q[i];
  }
  if constexpr (SRC_MOM) {
    k0 = rl3 + third * udg;
    Ssum += R(0.5) * k0;
  }
  const R three_over_rho = R(3) * inv_rho;
  // d_i = h_i / w_i - 1; the cumulant path works on w_i d_i (w_i folded into the factor)
#pragma unroll
  for (int i = 0; i < Q; ++i)
    q[i] = (COLL == COLL_BGK ? three_over_rho : three_over_rho * (R)wgt<D>(i)) * (q[i] - Ssum);

  // ---------------------------------------------------------------- relaxation time
  R tau0;
  if constexpr (THERMAL) {
    const R Tr = T_early;
    tau0 = R(3) * a.nu_lat * pw<R>(Tr * a.T_ref_inv, a.mu_exp) * inv_rho + R(0.5);
  } else {
    tau0 = R(3) * a.nu_lat + R(0.5);
  }

  if constexpr (COLL != COLL_BGK) {
    constexpr bool FULL = COLL == COLL_CUMULANT_FULL;
    // central moments of w d (d = h/w - 1) about u, minus those of h_eq - w, give the central
    // moments n of h - h_eq (h_eq: product-form equilibrium); see delta_eq
    const R dlx[3] = {R(0), -ux, ux * ux}, dly[3] = {R(0), -uy, uy * uy}, dlz[3] = {R(0), -uz, uz * uz};
#pragma unroll
    for (int j = 0; j < Q / 3; ++j) chim_fwd(q[3 * j], q[3 * j + 1], q[3 * j + 2], ux);
#pragma unroll
    for (int kz = 0; kz < Q / 9; ++kz)
#pragma unroll
      for (int ax = 0; ax < 3; ++ax) chim_fwd(q[ax + 9 * kz], q[ax + 3 + 9 * kz], q[ax + 6 + 9 * kz], uy);
    if constexpr (D == 3) {
#pragma unroll
      for (int j = 0; j < 9; ++j) chim_fwd(q[j], q[j + 9], q[j + 18], uz);
    }
    if constexpr (SRC_MOM) {
      // (3 / rho) (1/2) times the moments k of w xi listed above, orders 0..2
      const R h = R(1.5) * inv_rho, ninth = R(1) / R(9);
      const R u3[3] = {ux, uy, uz}, g3[3] = {gx, gy, gz};
      q[0] += h * k0;
#pragma unroll
      for (int a = 0; a < D; ++a) {
        const int ja = a == 0 ? 1 : (a == 1 ? 3 : 9);  // index of the first-order moment along a
        q[ja] += h * (-u3[a] * k0);
        q[2 * ja] += h * (rl3 * (u3[a] * u3[a] + third) + ninth * (udg + R(2) * g3[a] * u3[a]));
#pragma unroll
        for (int b = a + 1; b < D; ++b) {
          const int jb = b == 1 ? 3 : 9;
          q[ja + jb] += h * (rl3 * u3[a] * u3[b] + ninth * (g3[a] * u3[b] + g3[b] * u3[a]));
        }
      }
    }
    // full relaxation of orders 3..6 reads only the second-order moments, and orders 0 and 1
    // pass through unchanged: there the deviation is removed and restored for order 2 and
    // restored for orders >= 2 only (the skipped terms cancel exactly in real arithmetic)
    if constexpr (FULL) add_delta_eq<D, R, 0, 2, 2>(q, dlx, dly, dlz, R(-1));
    else add_delta_eq<D, R, 0>(q, dlx, dly, dlz, R(-1));
    // Smagorinsky: deviatoric part of the second central moments (equilibrium is isotropic)
    R tau = tau0;
    if (a.smag_k > R(0)) {
      R n2;
      if constexpr (D == 2) {
        const R tr = R(0.5) * (q[2] + q[6]);
        const R d0 = q[2] - tr, d1 = q[6] - tr;
        n2 = d0 * d0 + d1 * d1 + R(2) * q[4] * q[4];
      } else {
        const R tr = third * (q[2] + q[6] + q[18]);
        const R d0 = q[2] - tr, d1 = q[6] - tr, d2 = q[18] - tr;
        n2 = d0 * d0 + d1 * d1 + d2 * d2 + R(2) * (q[4] * q[4] + q[10] * q[10] + q[12] * q[12]);
      }
      tau = R(0.5) * (tau0 + sqrt(tau0 * tau0 + a.smag_k * sqrt(n2)));
    }
    const R om = R(1) / tau;
    if constexpr (D == 2) cumulant_relax2<FULL, R>(q, om, a.omega_b, a.om3, a.om4);
    else cumulant_relax3<FULL, R>(q, om, a.omega_b, a.om3, a.om4, a.om5, a.om6);
    if constexpr (FULL) add_delta_eq<D, R, 0, 2, 6>(q, dlx, dly, dlz, R(1));
    else add_delta_eq<D, R, 0>(q, dlx, dly, dlz, R(1));
    if constexpr (D == 3) {
#pragma unroll
      for (int j = 0; j < 9; ++j) chim_bwd(q[j], q[j + 9], q[j + 18], uz);
    }
#pragma unroll
    for (int kz = 0; kz < Q / 9; ++kz)
#pragma unroll
      for (int ax = 0; ax < 3; ++ax) chim_bwd(q[ax + 9 * kz], q[ax + 3 + 9 * kz], q[ax + 6 + 9 * kz], uy);
#pragma unroll
    for (int j = 0; j < Q / 3; ++j) chim_bwd(q[3 * j], q[3 * j + 1], q[3 * j + 2], ux);
    // q now holds w_i d*_i; the 1 / w_i is folded into the store below
  } else {
    // single rate towards the polynomial equilibrium f^eq(1, u) of Eq. 4: E_i = f^eq_i / w_i - 1
    R tau = tau0;
    if (a.smag_k > R(0)) {
      R pxx = R(0), pyy = R(0), pzz = R(0), pxy = R(0), pxz = R(0), pyz = R(0);
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        const R cu = (R)cx(i) * ux + (R)cy(i) * uy + ((D == 3) ? (R)cz(i) * uz : R(0));
        const R ne = (R)wgt<D>(i) * (q[i] - (R(3) * cu + R(4.5) * cu * cu - R(1.5) * usq));
        const R c0 = (R)cx(i), c1 = (R)cy(i), c2 = (D == 3) ? (R)cz(i) : R(0);
        pxx += c0 * c0 * ne; pyy += c1 * c1 * ne; pxy += c0 * c1 * ne;
        if (D == 3) { pzz += c2 * c2 * ne; pxz += c0 * c2 * ne; pyz += c1 * c2 * ne; }
      }
      R n2;
      if (D == 2) {
        const R tr = R(0.5) * (pxx + pyy);
        n2 = (pxx - tr) * (pxx - tr) + (pyy - tr) * (pyy - tr) + R(2) * pxy * pxy;
      } else {
        const R tr = third * (pxx + pyy + pzz);
        n2 = (pxx - tr) * (pxx - tr) + (pyy - tr) * (pyy - tr) + (pzz - tr) * (pzz - tr) +
             R(2) * (pxy * pxy + pxz * pxz + pyz * pyz);
      }
      tau = R(0.5) * (tau0 + sqrt(tau0 * tau0 + a.smag_k * sqrt(n2)));
    }
    const R om = R(1) / tau;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const R cu = (R)cx(i) * ux + (R)cy(i) * uy + ((D == 3) ? (R)cz(i) * uz : R(0));
      const R E = R(3) * cu + R(4.5) * cu * cu - R(1.5) * usq;
      q[i] -= om * (q[i] - E);
    }
  }

  // ------------------------------------------------- post-collision (Eq. 8), stored shifted
  // g*_i / w_i - P_ref = rho/3 (h*_i / w_i - 1) + S + xi_i / 2
  S* __restrict__ gout = (S*)a.g_out;
  const R rho3 = rho * third;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    R half_xi = R(0);
    if constexpr (THERMAL) {
      const R cu = (R)cx(i) * ux + (R)cy(i) * uy + ((D == 3) ? (R)cz(i) * uz : R(0));
      const R cg = (R)cx(i) * gx + (R)cy(i) * gy + ((D == 3) ? (R)cz(i) * gz : R(0));
      const R e = cu + R(1.5) * cu * cu - R(0.5) * usq;
      half_xi = R(0.5) * (e * (cg - udg) + rl3);
    }
    const R fac = COLL == COLL_BGK ? rho3 : rho3 * (R)(1.0 / wgt<D>(i));
    st_pop<S, R>(gout + i * Ni + r, fac * q[i] + Ssum + half_xi);
  }
  if (a.write_u || outlet_cell) {
    a.u[r] = ux;
    a.u[N + r] = uy;
    if (D == 3) a.u[2 * N + r] = uz;
  }
  if (a.ph_out) a.ph_out[r] = a.P_ref + psum + R(0.5) * rl3;
  if (!isfinite(usq)) atomicOr(a.flag, 1);
}

// pdl: the kernel may start while the one before it in the stream (the thermodynamic-pressure
// update) runs; it reads that kernel's state after pdl_wait.
template <int D, typename S, typename R>
cudaError_t launch_lb(const LBArgs<R>& a, int thermal, int coll, cudaStream_t st, bool pdl) {
  const dim3 grid((a.geo.nx + LB_BLOCK - 1) / LB_BLOCK, a.geo.ny, a.geo.nz);
#define LB_LAUNCH(TH, CO)                                                                         \
  do {                                                                                            \
    cudaError_t e_ = launch_ex<LBArgs<R>>(lb_step_kernel<D, S, R, TH, CO, false>, grid, dim3(LB_BLOCK), st, pdl, a); \
    if (e_ != cudaSuccess) return e_;                                                             \
    if (a.n_wall > 0)                                                                             \
      lb_step_kernel<D, S, R, TH, CO, true><<<(a.n_wall + LB_BLOCK - 1) / LB_BLOCK, LB_BLOCK, 0, st>>>(a); \
  } while (0)
  if (thermal) {
    if (coll == COLL_CUMULANT_FULL) LB_LAUNCH(true, COLL_CUMULANT_FULL);
    else if (coll == COLL_CUMULANT) LB_LAUNCH(true, COLL_CUMULANT);
    else LB_LAUNCH(true, COLL_BGK);
  } else {
    if (coll == COLL_CUMULANT_FULL) LB_LAUNCH(false, COLL_CUMULANT_FULL);
    else if (coll == COLL_CUMULANT) LB_LAUNCH(false, COLL_CUMULANT);
    else LB_LAUNCH(false, COLL_BGK);
  }
#undef LB_LAUNCH
  return cudaGetLastError();
}

}  // namespace hlbm
