// Tiled finite-difference update of temperature and species (Section 2.3) for 3-D grids in FP32:
// the same cell update as fd_step_kernel (WENO3 advection, centred diffusion with the arithmetic
// face mean of F_loc mu(T), Arrhenius sources divided by F_loc, pressure work, Lambda of Eq. 3,
// rho, the flame sensor of the new state and the thermodynamic-pressure partial sums), organised
// so that every face quantity is computed once:
//
// * A block owns a 32 x 8 tile of (x, y) columns and marches along z over a chunk of planes.
//   Each plane of T, Y_k, u, F_loc and the stencil words, with a halo of 4 cells in x (16-byte
//   aligned TMA start) and 2 in y, arrives in shared memory by one TMA tile load per array into a
//   ring of four plane slots (planes z, z+1, z+2 in use, z+3 in flight), completion tracked by one
//   mbarrier per slot.
// * F_loc mu(T) is evaluated once per point of the plane (with a halo of 1) into shared memory.
// * Per field, each thread evaluates the WENO3 face value and the diffusive flux of its +x, +y and
//   +z faces; the -x and -y faces come from the neighbours through shared memory, the -z face is
//   the +z face of the plane below, carried in registers. Faces on the tile's low x and y edges are
//   evaluated by warps 0 and 1. Fields go in pairs, one barrier per pair, with the face buffers of
//   two pairs in shared memory.
// * A face between two cells is evaluated from the point of view of its low-side cell when that
//   cell is fluid, else from its high-side cell; the ghost rules of the stencil word (zero
//   gradient at walls, solids and the outlet, the inlet state at the inlet) give the same face
//   from either fluid side, so the shared face equals what each cell's own stencil gives.
// * Inlet and outlet ghosts have a single viewer each (the first and last column), so their
//   values are written into the x halo of the plane tile once the plane has arrived (inlet
//   state and inlet velocity at x = -1, -2; the last column's values at x = nx, nx + 1). Only
//   the zero-gradient ghosts of walls and solid cells remain view-dependent: per plane, each x or
//   y face turns its stencil word into four source indices into the plane tile (a ghost points at
//   the cell it copies), so that every field reads its face values with four plain loads; the
//   z face selects among its four register values.
//
// Cells flagged with ghost-point wall weights (SW_WALL) are left to fd_step_kernel (walls-only
// launch); the tiled kernel needs non-periodic faces and nx a multiple of 4 (TMA strides).
#pragma once
#include <cuda.h>
#include <type_traits>
#include "fd_kernel.cuh"

namespace hlbm {

constexpr int TT_X = 32, TT_Y = 8;          // cells of a tile; one warp per row
constexpr int TT_HX = 4, TT_HY = 2;         // halo of the plane tiles (x start 16-byte aligned)
constexpr int TT_PX = TT_X + 2 * TT_HX;     // 40
constexpr int TT_PY = TT_Y + 2 * TT_HY;     // 12
constexpr int TT_PLANE = TT_PX * TT_PY;     // 480 words per plane array
constexpr int TT_SLOTS = 4;
constexpr int TT_FX = TT_X + 2, TT_FY = TT_Y + 2;  // F mu tile, halo 1
// planes of one slot: T, Y_0..Y_{K-1}, u_x, u_y, u_z, F_loc, stencil word
template <int NK> struct TTLayout {
  static constexpr int NP = NK + 6;
  static constexpr int P_T = 0, P_Y = 1, P_U = NK + 1, P_F = NK + 4, P_S = NK + 5;
  static constexpr int RING = TT_SLOTS * NP * TT_PLANE;                 // words
  static constexpr int XF = RING;                                      // float2 [4][TT_Y][TT_X + 1]
  static constexpr int YF = XF + 4 * 2 * TT_Y * (TT_X + 1);            // float2 [4][TT_Y + 1][TT_X]
  static constexpr int FM = YF + 4 * 2 * (TT_Y + 1) * TT_X;            // [2][TT_FY][TT_FX]
  static constexpr int BAR = (FM + 2 * TT_FX * TT_FY + 1) & ~1;       // uint64 [TT_SLOTS]
  static constexpr int RED = BAR + 2 * TT_SLOTS;                       // int64 [8][2]
  static constexpr int WORDS = RED + 2 * 2 * 8;
  static constexpr size_t BYTES = (size_t)WORDS * 4;
};

// Tensor maps of the arrays the tiled update reads, for the two state parities.
struct FDTiledMaps {
  CUtensorMap T[2], Y[2], F[2], U, S;
  int lz = 0;              // planes per block along z
  dim3 grid;
  bool sensor = false;
};

// face recipe flags: upwind side, inlet values and zero-gradient copies of the four stencil points
// (a - e, a, b, b + e) of the face between a and b = a + e
enum : uint32_t {
  FR_UP = 1u, FR_IN_M = 2u, FR_IN_0 = 4u, FR_IN_1 = 8u, FR_IN_2 = 16u,
  FR_CP_M = 32u, FR_CP_0 = 64u, FR_CP_1 = 128u, FR_CP_2 = 256u
};

// Face velocity (upwind side), face coefficient 0.5 (F mu (a) + F mu (b)) and ghost recipe of the
// face between a and b along `ax`, from the view of a when a is fluid, else of b.
// GH = false: both cells and their radius-2 lines are fluid (no ghost).
template <bool GH>
__device__ __forceinline__ void face_recipe(uint32_t swa, uint32_t swb, int ax, float ua, float ub, float FMa,
                                            float FMb, float Fa, float Fb, float mu_in, float uin, float& FMf,
                                            uint32_t& fl) {
  if constexpr (!GH) {
    FMf = 0.5f * (FMa + FMb);
    fl = (0.5f * (ua + ub) >= 0.0f) ? FR_UP : 0u;
    return;
  } else {
    const int sm = 4 * (2 * ax), sp = 4 * (2 * ax + 1);
    float un, FMn, uown, FMown;
    uint32_t f = 0u;
    if (swa >> 31) {
      const uint32_t k1p = (swa >> sp) & 3u, d2p = (swa >> (sp + 2)) & 3u, k1m = (swa >> sm) & 3u;
      un = k1p == NB_FLUID ? ub : (k1p == NB_INLET ? uin : (k1p == NB_OUTLET ? ua : 0.0f));
      FMn = k1p == NB_FLUID ? FMb : (k1p == NB_INLET ? Fa * mu_in : FMa);
      uown = ua;
      FMown = FMa;
      if (k1p == NB_INLET) f |= FR_IN_1;
      else if (k1p != NB_FLUID) f |= FR_CP_1;
      if (d2p == 2u) f |= FR_IN_2;
      else if (d2p == 1u) f |= FR_CP_2;
      if (k1m == NB_INLET) f |= FR_IN_M;
      else if (k1m != NB_FLUID) f |= FR_CP_M;
    } else {
      const uint32_t k1m = (swb >> sm) & 3u, d2m = (swb >> (sm + 2)) & 3u, k1p = (swb >> sp) & 3u;
      un = k1m == NB_FLUID ? ua : (k1m == NB_INLET ? uin : (k1m == NB_OUTLET ? ub : 0.0f));
      FMn = k1m == NB_FLUID ? FMa : (k1m == NB_INLET ? Fb * mu_in : FMb);
      uown = ub;
      FMown = FMb;
      if (k1m == NB_INLET) f |= FR_IN_0;
      else if (k1m != NB_FLUID) f |= FR_CP_0;
      if (d2m == 2u) f |= FR_IN_M;
      else if (d2m == 1u) f |= FR_CP_M;
      if (k1p == NB_INLET) f |= FR_IN_2;
      else if (k1p != NB_FLUID) f |= FR_CP_2;
    }
    FMf = 0.5f * (FMown + FMn);
    fl = f | ((0.5f * (uown + un) >= 0.0f) ? FR_UP : 0u);
  }
}

// WENO3 value and diffusive flux (without the field's 1/(Pr Le)) of a face from the raw values of
// its four stencil points; the recipe replaces ghosts. Same formulas as fd_cell: with
// d1 = v0 - vm, d2 = v1 - v0, d3 = v2 - v1 and t(d) = (eps + d^2)^2, the face is
// v0 + (t(d2) d1 + 2 t(d1) d2) / (2 (t(d2) + 2 t(d1))) upwind from a, and
// v1 - (t(d2) d3 + 2 t(d3) d2) / (2 (t(d2) + 2 t(d3))) upwind from b.
template <bool GH>
__device__ __forceinline__ void face_eval(float vm, float v0, float v1, float v2, float phin, uint32_t fl,
                                          float FMf, float eps, float& Fv, float& Dv) {
  if constexpr (GH) {
    vm = (fl & FR_IN_M) ? phin : vm;
    v0 = (fl & FR_IN_0) ? phin : v0;
    v1 = (fl & FR_IN_1) ? phin : v1;
    v2 = (fl & FR_IN_2) ? phin : v2;
    const float c0 = (fl & FR_CP_0) ? v1 : v0;
    const float c1 = (fl & FR_CP_1) ? v0 : v1;
    v0 = c0;
    v1 = c1;
    vm = (fl & FR_CP_M) ? v0 : vm;
    v2 = (fl & FR_CP_2) ? v1 : v2;
  }
  const bool up = (fl & FR_UP) != 0u;
  const float d1 = v0 - vm, d2 = v1 - v0, d3 = v2 - v1;
  const float s = up ? d1 : d3;
  const float ss = fmaf(s, s, eps), s2 = fmaf(d2, d2, eps);
  const float ts = ss * ss, t2 = s2 * s2;
  const float num = fmaf(t2, s, 2.0f * ts * d2);
  const float q = num * rcp_approx(fmaf(2.0f, ts, t2));
  Fv = up ? fmaf(0.5f, q, v0) : fmaf(-0.5f, q, v1);
  Dv = FMf * d2;
}

// ------------------------------------------------------------------------ TMA and mbarriers
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
// Bounded wait for the phase with parity `parity` of the barrier; false after the limit.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  const uint32_t a = smem_u32(bar);
  for (int it = 0; it < (1 << 22); ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar, int c0, int c1, int c2) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
      ::"r"(smem_u32(dst)), "l"((uint64_t)map), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, uint64_t* bar, int c0, int c1, int c2,
                                            int c3) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], [%6];"
      ::"r"(smem_u32(dst)), "l"((uint64_t)map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(bar))
      : "memory");
}

constexpr int TT_THREADS = TT_X * TT_Y;

// WENO3 face value and diffusive flux (without the field's 1/(Pr Le)) from the four stencil values
// (a - e, a, b, b + e) of the face between a and b = a + e, ghosts already substituted. Same
// formulas as fd_cell: with d1 = v0 - vm, d2 = v1 - v0, d3 = v2 - v1 and t(d) = (eps + d^2)^2, the
// face is v0 + (t(d2) d1 + 2 t(d1) d2) / (2 (t(d2) + 2 t(d1))) upwind from a, and
// v1 - (t(d2) d3 + 2 t(d3) d2) / (2 (t(d2) + 2 t(d3))) upwind from b.
__device__ __forceinline__ void face_math(float vm, float v0, float v1, float v2, bool up, float FMf, float eps,
                                          float& Fv, float& Dv) {
  const float d1 = v0 - vm, d2 = v1 - v0, d3 = v2 - v1;
  const float s = up ? d1 : d3;
  const float ss = fmaf(s, s, eps), s2 = fmaf(d2, d2, eps);
  const float ts = ss * ss, t2 = s2 * s2;
  const float num = fmaf(t2, s, 2.0f * ts * d2);
  const float q = num * rcp_approx(fmaf(2.0f, ts, t2));
  Fv = up ? fmaf(0.5f, q, v0) : fmaf(-0.5f, q, v1);
  Dv = FMf * d2;
}

// A face of the plane tile: the plane indices of its four stencil values after ghost
// substitution, its upwind side and its diffusion coefficient 0.5 (F mu (a) + F mu (b)).
struct TFace {
  int im, i0, i1, i2;
  bool up;
  float FMf;
};

// Face between tile points ia and ia + st (plane indices; st = 1 along x, TT_PX along y), from the
// view of a when a is fluid, else of b. Inlet and outlet halo values are already in the tile, so
// only solid neighbours (kind 1) are ghosts: a distance-1 solid copies the viewer, a distance-2
// zero-gradient point copies the distance-1 value; a solid neighbour's velocity is 0 and its
// F mu is the viewer's.
__device__ __forceinline__ TFace tile_face(const float* __restrict__ sS, const float* __restrict__ sU,
                                           const float* __restrict__ FMt, int ia, int st, int fa, int fst, int ax) {
  const uint32_t swa = __float_as_uint(sS[ia]), swb = __float_as_uint(sS[ia + st]);
  const int sm = 4 * (2 * ax), sp = sm + 4;
  const float ua = sU[ia], ub = sU[ia + st], FMa = FMt[fa], FMb = FMt[fa + fst];
  TFace f;
  float uown, un, FMown, FMn;
  int om, o0, o1, o2;
  if (swa >> 31) {
    const bool s1p = ((swa >> sp) & 3u) == NB_SOLID, c2p = ((swa >> (sp + 2)) & 3u) == 1u;
    const bool s1m = ((swa >> sm) & 3u) == NB_SOLID;
    o0 = 0;
    o1 = s1p ? 0 : 1;
    o2 = c2p ? o1 : 2;
    om = s1m ? 0 : -1;
    uown = ua;
    un = s1p ? 0.0f : ub;
    FMown = FMa;
    FMn = s1p ? FMa : FMb;
  } else {
    const bool s1m = ((swb >> sm) & 3u) == NB_SOLID, c2m = ((swb >> (sm + 2)) & 3u) == 1u;
    const bool s1p = ((swb >> sp) & 3u) == NB_SOLID;
    o1 = 1;
    o0 = s1m ? 1 : 0;
    om = c2m ? o0 : -1;
    o2 = s1p ? 1 : 2;
    uown = ub;
    un = s1m ? 0.0f : ua;
    FMown = FMb;
    FMn = s1m ? FMb : FMa;
  }
  f.im = ia + om * st;
  f.i0 = ia + o0 * st;
  f.i1 = ia + o1 * st;
  f.i2 = ia + o2 * st;
  f.FMf = 0.5f * (FMown + FMn);
  f.up = 0.5f * (uown + un) >= 0.0f;
  return f;
}

template <int NK, int NR>
__global__ void __launch_bounds__(TT_THREADS, 2)
    fd_tiled_kernel(const FDArgs<float> a, const __grid_constant__ CUtensorMap mT, const __grid_constant__ CUtensorMap mY,
                    const __grid_constant__ CUtensorMap mU, const __grid_constant__ CUtensorMap mF,
                    const __grid_constant__ CUtensorMap mS, const int LZ, const int sensor) {
  using L = TTLayout<NK>;
  extern __shared__ __align__(128) float sm[];
  float* ring = sm;
  float2* XF = reinterpret_cast<float2*>(sm + L::XF);
  float2* YF = reinterpret_cast<float2*>(sm + L::YF);
  float* FMbuf = sm + L::FM;  // F mu tiles of planes z (z & 1) and z + 1
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm + L::BAR);
  long long* red = reinterpret_cast<long long*>(sm + L::RED);

  const FDConst<float>& c = a.c;
  const Geo& g = a.geo;
  const int nx = g.nx, ny = g.ny, nz = g.nz, N = g.N;
  const int tx = threadIdx.x, ty = threadIdx.y, tid = tx + TT_X * ty;
  const int x0 = blockIdx.x * TT_X, y0 = blockIdx.y * TT_Y, z0 = blockIdx.z * LZ;
  const int z1 = min(z0 + LZ, nz);
  const int x = x0 + tx, y = y0 + ty;
  const bool in_xy = x < nx && y < ny;
  const int own = (ty + TT_HY) * TT_PX + tx + TT_HX;  // index of this cell in a plane array
  const uint32_t bytes = (uint32_t)((1 + NK + 3 + (sensor ? 1 : 0) + 1) * TT_PLANE * 4);
  const int zlast = min(z1 + 1, nz - 1);             // last plane any step of this chunk reads
  // tiles whose x halo holds inlet or outlet ghost points (written after each plane arrives)
  const bool inlet_tile = x0 == 0 && g.bc_lo[0] == BC_INLET;
  const int xo = nx - x0 + TT_HX;  // plane column of x = nx
  const bool outlet_tile = g.bc_hi[0] == BC_OUTLET && xo >= 1 && xo < TT_PX;

  auto slot = [&](int zp) -> float* { return ring + ((zp - z0) & (TT_SLOTS - 1)) * L::NP * TT_PLANE; };
  auto issue = [&](int zp) {
    float* s = slot(zp);
    uint64_t* b = bar + ((zp - z0) & (TT_SLOTS - 1));
    mbar_expect_tx(b, bytes);
    const int cx = x0 - TT_HX, cy = y0 - TT_HY;
    tma_load_3d(s + L::P_T * TT_PLANE, &mT, b, cx, cy, zp);
    tma_load_4d(s + L::P_Y * TT_PLANE, &mY, b, cx, cy, zp, 0);
    tma_load_4d(s + L::P_U * TT_PLANE, &mU, b, cx, cy, zp, 0);
    if (sensor) tma_load_3d(s + L::P_F * TT_PLANE, &mF, b, cx, cy, zp);
    tma_load_3d(s + L::P_S * TT_PLANE, &mS, b, cx, cy, zp);
  };
  auto wait = [&](int zp) -> bool {
    if (zp >= nz) return true;
    return mbar_wait(bar + ((zp - z0) & (TT_SLOTS - 1)), (uint32_t)(((zp - z0) >> 2) & 1));
  };

  if (tid == 0) {
#pragma unroll
    for (int s = 0; s < TT_SLOTS; ++s) mbar_init(bar + s, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (tid == 0) {
    for (int zp = z0; zp <= min(z0 + 2, zlast); ++zp) issue(zp);
  }

  // constants of this launch
  const float fdr = a.pth->fd_rho, fd_dT = a.pth->fd_dT;
  const float rin = a.pth->rho_in;
  const float mu_in = c.nu_lat * powr<float>(c.T_in * c.T_ref_inv, c.mu_exp);
  const float dt = c.dt_phys;
  long long accI = 0, accM = 0;  // fixed-point P_th integrand and boundary mass flux of this thread

  // inlet / outlet ghost values into the x halo of plane zp, held in slot sp (single viewer each)
  auto ghosts = [&](int zp, float* sp) {
    if (tid < 2 * TT_PY) {
      const int row = tid % TT_PY, col = tid / TT_PY;  // col 0, 1: x = -1, -2 or x = nx, nx + 1
      const int yy = y0 - TT_HY + row;
      if (inlet_tile) {
        const int pi = row * TT_PX + TT_HX - 1 - col;
#pragma unroll
        for (int f = 0; f <= NK; ++f) sp[(L::P_T + f) * TT_PLANE + pi] = f == 0 ? c.T_in : c.Y_in[f - 1];
        sp[L::P_U * TT_PLANE + pi] = (yy >= 0 && yy < ny) ? __ldg(a.inlet_u + yy + ny * zp) : 0.0f;
        if (sensor) sp[L::P_F * TT_PLANE + pi] = sp[L::P_F * TT_PLANE + row * TT_PX + TT_HX];
      }
      if (outlet_tile && xo + col < TT_PX) {
        const int pi = row * TT_PX + xo + col, pl = row * TT_PX + xo - 1;
#pragma unroll
        for (int f = 0; f <= NK; ++f) sp[(L::P_T + f) * TT_PLANE + pi] = sp[(L::P_T + f) * TT_PLANE + pl];
        sp[L::P_U * TT_PLANE + pi] = sp[L::P_U * TT_PLANE + pl];
        if (sensor) sp[L::P_F * TT_PLANE + pi] = sp[L::P_F * TT_PLANE + pl];
      }
    }
  };
  // F mu(T) of the plane in slot sp on the tile and a halo of 1, into the tile buffer fm
  auto fm_tile = [&](const float* sp, float* fm) {
    for (int i = tid; i < TT_FX * TT_FY; i += TT_THREADS) {
      const int px = i % TT_FX, py = i / TT_FX;
      const int pi = (py + TT_HY - 1) * TT_PX + px + TT_HX - 1;
      const float Fp = sensor ? sp[L::P_F * TT_PLANE + pi] : c.F;
      fm[i] = Fp * (c.nu_lat * powr<float>(sp[L::P_T * TT_PLANE + pi] * c.T_ref_inv, c.mu_exp));
    }
  };

  // ---------------------------------------------------------------- prologue: the -z face of z0
  bool ok = wait(z0) && wait(z0 + 1);
  ok = __syncthreads_and(ok);
  if (!ok) {
    if (tid == 0) atomicOr(a.flag, 4);
    for (int zp = z0; zp <= min(z0 + 2, zlast); ++zp) wait(zp);
    return;
  }
  // ghosts and F mu tile of plane z0 (each step of the march prepares the plane above it)
  if (inlet_tile || outlet_tile) {
    ghosts(z0, slot(z0));
    __syncthreads();
  }
  fm_tile(slot(z0), FMbuf + (z0 & 1) * TT_FX * TT_FY);
  float carF[NK + 1], carD[NK + 1], phim[NK + 1];  // -z face of the plane, phi at z - 1
  {
    const float* s0 = slot(z0);
    const float* s1 = slot(z0 + 1);
    const int zm = z0 - 1, zmm = z0 - 2;
    const bool hm = in_xy && zm >= 0, hmm = in_xy && zmm >= 0;
    const int rm = hm ? x + nx * (y + ny * zm) : 0;
    const int rmm = hmm ? x + nx * (y + ny * zmm) : 0;
    const uint32_t swa = hm ? __ldg(a.sword + rm) : 0u;
    const uint32_t swb = __float_as_uint(s0[L::P_S * TT_PLANE + own]);
    const float ua = hm ? __ldg(a.u + 2 * (size_t)N + rm) : 0.0f;
    const float ub = s0[(L::P_U + 2) * TT_PLANE + own];
    const float Ta = hm ? __ldg(a.T + rm) : c.T_in;
    const float Fa = (sensor && hm) ? __ldg(a.Floc + rm) : c.F;
    const float Fb = sensor ? s0[L::P_F * TT_PLANE + own] : c.F;
    const float FMa = Fa * (c.nu_lat * powr<float>(Ta * c.T_ref_inv, c.mu_exp));
    const float FMb = Fb * (c.nu_lat * powr<float>(s0[L::P_T * TT_PLANE + own] * c.T_ref_inv, c.mu_exp));
    float FMf;
    uint32_t fl;
    face_recipe<true>(swa, swb, 2, ua, ub, FMa, FMb, Fa, Fb, mu_in, 0.0f, FMf, fl);
#pragma unroll
    for (int f = 0; f <= NK; ++f) {
      const float* pb = (f == 0 ? a.T : a.Y + (size_t)(f - 1) * N);
      const float vmm = hmm ? __ldg(pb + rmm) : 0.0f;
      const float vm = hm ? __ldg(pb + rm) : 0.0f;
      const float v0 = s0[(L::P_T + f) * TT_PLANE + own];
      const float v1 = s1[(L::P_T + f) * TT_PLANE + own];
      const float phin = f == 0 ? c.T_in : c.Y_in[f - 1];
      face_eval<true>(vmm, vm, v0, v1, phin, fl, FMf, f == 0 ? c.eps_T : c.eps_Y, carF[f], carD[f]);
      phim[f] = vm;
    }
  }

  // ---------------------------------------------------------------- march along z
  for (int z = z0; z < z1; ++z) {
    const bool okz = wait(z + 2);
    float* s0 = slot(z);
    float* s1 = slot(z + 1);
    const float* s2 = slot(z + 2);
    const float* FMs = FMbuf + (z & 1) * TT_FX * TT_FY;      // plane z (prepared one step earlier)
    float* FMn = FMbuf + ((z + 1) & 1) * TT_FX * TT_FY;      // plane z + 1
    // ghosts and F mu tile of plane z + 1: its z face with plane z reads them now, plane z + 1
    // itself in the next step
    if ((inlet_tile || outlet_tile) && z + 1 < nz) {
      ghosts(z + 1, s1);
      __syncthreads();
    }
    fm_tile(s1, FMn);
    // all threads leave together when a plane load did not arrive
    if (!__syncthreads_and(okz)) {
      if (tid == 0) atomicOr(a.flag, 4);
      for (int zp = z; zp <= min(z + 3, zlast); ++zp) wait(zp);
      return;
    }
    if (tid == 0 && z + 3 <= zlast) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      issue(z + 3);
    }

    // ---- per-cell state of plane z
    const uint32_t sw = __float_as_uint(s0[L::P_S * TT_PLANE + own]);
    const bool active = in_xy && (sw >> 31) != 0u && (sw & SW_WALL) == 0u;
    const int r = x + nx * (y + ny * z);
    const float Tr = s0[L::P_T * TT_PLANE + own];
    float Yr[NK];
    float sW = 0.0f;
#pragma unroll
    for (int k = 0; k < NK; ++k) {
      Yr[k] = s0[(L::P_Y + k) * TT_PLANE + own];
      sW += Yr[k] * c.inv_W[k];
    }
    const float ux = s0[L::P_U * TT_PLANE + own], uy = s0[(L::P_U + 1) * TT_PLANE + own];
    const float uz = s0[(L::P_U + 2) * TT_PLANE + own];
    const float Fr = sensor ? s0[L::P_F * TT_PLANE + own] : c.F;
    // chemistry and the update only where a cell is updated (solid cells hold arbitrary values)
    float W = 1.0f, rho = 1.0f, inv_rho = 1.0f, qdot = 0.0f, inv_rpF = 0.0f;
    float q[NR];
#pragma unroll
    for (int j = 0; j < NR; ++j) q[j] = 0.0f;
    float inv_T = 0.0f;
    if (active) {
      // one IEEE reciprocal each of T, sum Y/W and rho, reused where fd_cell divides
      inv_T = 1.0f / Tr;
      W = 1.0f / sW;
      rho = fdr * W * inv_T;
      const float rho_phys = rho * c.rho_ref_f;
      inv_rho = 1.0f / rho;
      reaction_rates<NR, float, NK>(c, Tr, inv_T, Yr, rho_phys, q);
#pragma unroll
      for (int j = 0; j < NR; ++j) qdot += c.heat[j] * q[j];
      inv_rpF = inv_rho * c.inv_rho_ref / Fr;
    }

    // ---- faces of this plane: +x, +y of this cell as source indices, +z as selects; the
    // tile-edge faces -y (warp 0, one per column) and -x (warp 1, lanes 0..7, one per row)
    const float* sS = s0 + L::P_S * TT_PLANE;
    const int fo = (ty + 1) * TT_FX + tx + 1;  // this cell in the F mu tile
    // a fluid cell whose radius-2 stencil is all fluid sees no ghost on its +x, +y, +z faces
    const bool plain = (sw >> 31) != 0u && (sw & 0x00ffffffu) == 0u;
    TFace fx, fy;
    if (plain) {
      fx = {own - 1, own, own + 1, own + 2, 0.5f * (ux + s0[L::P_U * TT_PLANE + own + 1]) >= 0.0f,
            0.5f * (FMs[fo] + FMs[fo + 1])};
      fy = {own - TT_PX, own, own + TT_PX, own + 2 * TT_PX,
            0.5f * (uy + s0[(L::P_U + 1) * TT_PLANE + own + TT_PX]) >= 0.0f, 0.5f * (FMs[fo] + FMs[fo + TT_FX])};
    } else {
      fx = tile_face(sS, s0 + L::P_U * TT_PLANE, FMs, own, 1, fo, 1, 0);
      fy = tile_face(sS, s0 + (L::P_U + 1) * TT_PLANE, FMs, own, TT_PX, fo, TT_FX, 1);
    }
    const bool edge_y = ty == 0, edge_x = ty == 1 && tx < TT_Y;
    TFace fe = fx;
    if (edge_y) fe = tile_face(sS, s0 + (L::P_U + 1) * TT_PLANE, FMs, own - TT_PX, TT_PX, tx + 1, TT_FX, 1);
    else if (edge_x) {
      const int ia = (tx + TT_HY) * TT_PX + TT_HX - 1;  // (x0 - 1, y0 + tx)
      fe = tile_face(sS, s0 + L::P_U * TT_PLANE, FMs, ia, 1, (tx + 1) * TT_FX, 1, 0);
    }
    bool upz, zcm, zc0, zc1, zc2;
    float FMz;
    {
      const uint32_t swb = (z + 1 < nz) ? __float_as_uint(s1[L::P_S * TT_PLANE + own]) : 0u;
      const float FMb = FMn[fo];
      const float FMa = FMs[fo];
      const float ub = s1[(L::P_U + 2) * TT_PLANE + own];
      float uown, un, FMown, FMn;
      if (plain) {
        zc0 = zc1 = zc2 = zcm = false;
        uown = uz;
        un = ub;
        FMown = FMa;
        FMn = FMb;
      } else if (sw >> 31) {
        const bool s1p = ((sw >> 20) & 3u) == NB_SOLID, c2p = ((sw >> 22) & 3u) == 1u;
        zc0 = false;
        zc1 = s1p;
        zc2 = c2p;
        zcm = ((sw >> 16) & 3u) == NB_SOLID;
        uown = uz;
        un = s1p ? 0.0f : ub;
        FMown = FMa;
        FMn = s1p ? FMa : FMb;
      } else {
        const bool s1m = ((swb >> 16) & 3u) == NB_SOLID;
        zc1 = false;
        zc0 = s1m;
        zcm = ((swb >> 18) & 3u) == 1u;
        zc2 = ((swb >> 20) & 3u) == NB_SOLID;
        uown = ub;
        un = s1m ? 0.0f : uz;
        FMown = FMb;
        FMn = s1m ? FMb : FMa;
      }
      FMz = 0.5f * (FMown + FMn);
      upz = 0.5f * (uown + un) >= 0.0f;
    }

    // ---- fields: 0 = T, 1.. = Y_k, in pairs (one barrier per pair)
    float lam = 0.0f, sWn = 0.0f, Tnew = Tr, yf_new = 0.0f, yo_new = 0.0f;
#pragma unroll
    for (int p = 0; p <= NK; p += 2) {
      float Fxp[2], Dxp[2], Fyp[2], Dyp[2], Fzp[2], Dzp[2];
      const int pb = (p >> 1) & 1;  // face buffers of this pair: 2 pb, 2 pb + 1
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int fi = p + h;
        if (fi > NK) break;
        const float* P = s0 + (L::P_T + fi) * TT_PLANE;
        const float eps = fi == 0 ? c.eps_T : c.eps_Y;
        float2* xf = XF + (2 * pb + h) * TT_Y * (TT_X + 1);
        float2* yf = YF + (2 * pb + h) * (TT_Y + 1) * TT_X;
        const float pr = P[own];
        face_math(P[fx.im], P[fx.i0], P[fx.i1], P[fx.i2], fx.up, fx.FMf, eps, Fxp[h], Dxp[h]);
        face_math(P[fy.im], P[fy.i0], P[fy.i1], P[fy.i2], fy.up, fy.FMf, eps, Fyp[h], Dyp[h]);
        {
          const float v1r = s1[(L::P_T + fi) * TT_PLANE + own], v2r = s2[(L::P_T + fi) * TT_PLANE + own];
          const float v0 = zc0 ? v1r : pr;
          const float v1 = zc1 ? pr : v1r;
          const float vm = zcm ? v0 : phim[fi];
          const float v2 = zc2 ? v1 : v2r;
          face_math(vm, v0, v1, v2, upz, FMz, eps, Fzp[h], Dzp[h]);
        }
        xf[ty * (TT_X + 1) + tx + 1] = make_float2(Fxp[h], Dxp[h]);
        yf[(ty + 1) * TT_X + tx] = make_float2(Fyp[h], Dyp[h]);
        if (edge_y || edge_x) {
          float Fe, De;
          face_math(P[fe.im], P[fe.i0], P[fe.i1], P[fe.i2], fe.up, fe.FMf, eps, Fe, De);
          if (edge_y) yf[tx] = make_float2(Fe, De);
          else xf[tx * (TT_X + 1)] = make_float2(Fe, De);
        }
      }
      __syncthreads();
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int fi = p + h;
        if (fi > NK) break;
        const float pr = s0[(L::P_T + fi) * TT_PLANE + own];
        const float2 xm = XF[(2 * pb + h) * TT_Y * (TT_X + 1) + ty * (TT_X + 1) + tx];
        const float2 ym = YF[(2 * pb + h) * (TT_Y + 1) * TT_X + ty * TT_X + tx];
        const float Fzm = carF[fi], Dzm = carD[fi];
        carF[fi] = Fzp[h];
        carD[fi] = Dzp[h];
        phim[fi] = pr;
        if (!active) continue;
        const float adv = ux * (Fxp[h] - xm.x) + uy * (Fyp[h] - ym.x) + uz * (Fzp[h] - Fzm);
        float dif = (Dxp[h] - xm.y) + (Dyp[h] - ym.y) + (Dzp[h] - Dzm);
        const float gfac = c.inv_Pr * (fi == 0 ? 1.0f : c.inv_Le[fi - 1]);
        float src;
        dif *= gfac * inv_rho;
        if (fi == 0) {
          src = dt * qdot * inv_rpF * c.inv_cp + fd_dT * inv_rho;
        } else {
          float om = 0.0f;
#pragma unroll
          for (int j = 0; j < NR; ++j) om += c.nu[j][fi - 1] * q[j];
          src = dt * c.W[fi - 1] * om * inv_rpF;
        }
        const float NA = dif + src;
        const float pn = pr - adv + NA;
        if (fi == 0) {
          a.T_out[r] = pn;
          lam += NA * inv_T;
          Tnew = pn;
        } else {
          a.Y_out[(size_t)(fi - 1) * N + r] = pn;
          lam += W * c.inv_W[fi - 1] * NA;
          sWn += pn * c.inv_W[fi - 1];
          if (fi - 1 == c.sensor_species) yf_new = pn;
          if (fi - 1 == c.sensor_oxidizer) yo_new = pn;
        }
      }
    }
    if (active) {
      if (a.Floc_out) a.Floc_out[r] = sensor_floc<float>(c, Tnew, yf_new, yo_new);
      a.rho_out[r] = rho;
      a.lam_out[r] = lam;
      if (c.closed) {
        accI += f32_to_fix32(c.I_scale / (sWn * Tnew));
        if (x == 0 && g.bc_lo[0] == BC_INLET) accM += f32_to_fix32(c.M_scale * rin * __ldg(a.inlet_u + y + ny * z));
        if (x == nx - 1 && g.bc_hi[0] == BC_OUTLET) accM += f32_to_fix32(-(c.M_scale * rho * ux));
      }
    }
  }

  // ---------------------------------------------------------------- P_th partial of this block
  if (!c.closed) return;
  long long vI = warp_sum_ll(accI), vM = warp_sum_ll(accM);
  if (tx == 0) {
    red[2 * ty] = vI;
    red[2 * ty + 1] = vM;
  }
  __syncthreads();
  if (tid == 0) {
    long long tI = 0, tM = 0;
    for (int w = 0; w < TT_Y; ++w) {
      tI += red[2 * w];
      tM += red[2 * w + 1];
    }
    const int bid = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
    long long* out = (long long*)a.partials;
    out[2 * bid] = tI;
    out[2 * bid + 1] = tM;
  }
}

}  // namespace hlbm
