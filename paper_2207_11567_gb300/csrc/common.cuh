// Shared device-side definitions of the GB300 library: lattice tables (compile-time),
// parameter blocks passed by value to the kernels, and small numeric helpers.
//
// Lattice (Section 2.1): D2Q9 / D3Q27 from the tensor product of the three-point rule with
// weights (1/6, 2/3, 1/6); direction i has c = ((i%3)-1, ((i/3)%3)-1, (i/9)-1); the opposite
// direction is Q-1-i. All constants below are derived from that rule at compile time.
#pragma once
#include <cstdint>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

namespace hlbm {

enum { BC_PERIODIC = 0, BC_WALL = 1, BC_INLET = 2, BC_OUTLET = 3 };
// COLL_CUMULANT_FULL: cumulant collision whose orders 3..6 relax fully (rate 1), the default
enum { COLL_BGK = 0, COLL_CUMULANT = 1, COLL_CUMULANT_FULL = 2 };
constexpr int MAX_SP = 8;
constexpr int MAX_RX = 4;
constexpr int MAX_ORD = 4;  // species with a nonzero order in one reaction

template <int D> struct Lat;
template <> struct Lat<2> { static constexpr int Q = 9; };
template <> struct Lat<3> { static constexpr int Q = 27; };

__host__ __device__ constexpr int cx(int i) { return i % 3 - 1; }
__host__ __device__ constexpr int cy(int i) { return (i / 3) % 3 - 1; }
__host__ __device__ constexpr int cz(int i) { return i / 9 - 1; }
__host__ __device__ constexpr double w1(int c) { return c == 0 ? 2.0 / 3.0 : 1.0 / 6.0; }
template <int D> __host__ __device__ constexpr double wgt(int i) {
  return D == 2 ? w1(cx(i)) * w1(cy(i)) : w1(cx(i)) * w1(cy(i)) * w1(cz(i));
}

// ---------------------------------------------------------------------------- geometry
struct Geo {
  int nx, ny, nz;
  int N;
  int bc_lo[3], bc_hi[3];
};

// Thermodynamic-pressure scalars, kept on the device and updated by the reduction kernel.
struct PthState {
  double P;        // thermodynamic pressure, Pa (level n during the FD update)
  double M;        // total mass, lattice units
  double dP;       // last increment of P (Pa per step)
  double steps;    // number of steps taken
  float fd_rho;    // P / (R rho_ref): rho_lat = fd_rho * W / T
  float fd_dT;     // dP_prev / (cp rho_ref): pressure-work increment of T is fd_dT / rho_lat
  float lb_lam;    // -dP / P_old, added to Lambda by the LB kernel of this step
  float rho_in;    // inlet density, lattice units
  double fd_rho_d, fd_dT_d, lb_lam_d, rho_in_d;  // same in FP64 for the FP64 storage path
};

// Fixed-point scales of the exact integer reduction (sum of per-cell FP32 terms).
constexpr double FIX_SCALE = 4294967296.0;  // 2^32

// Finite-difference / chemistry constants (lattice units unless noted), in the arithmetic type R.
template <typename R> struct FDConst {
  int K, nrx;
  int sensor, sensor_species, sensor_oxidizer;
  int closed;
  R nu_lat, T_ref_inv, mu_exp, inv_Pr;
  R inv_Le[MAX_SP];       // 1 / Le_k
  R inv_W[MAX_SP];        // 1 / W_k  (mol/kg)
  R W[MAX_SP];
  R hf_W[MAX_SP];         // h_f,k * W_k (J/mol)
  R dt_phys;              // s
  R inv_cp;               // 1 / cp
  R inv_rho_ref;
  R rho_ref_f;            // 1 / inv_rho_ref
  R F, sensor_beta, inv_wref, sensor_Ta;
  R eps_T, eps_Y;
  R T_in, Y_in[MAX_SP];
  // reactions: q = A exp(-E/(R T)) T^beta prod c^n. E/R is split into hi + lo parts for the
  // float path (float-float argument); the double path uses ER_hi = E/R and ER_lo = 0.
  R A[MAX_RX], beta[MAX_RX], ER_hi[MAX_RX], ER_lo[MAX_RX];
  R nu[MAX_RX][MAX_SP], order[MAX_RX][MAX_SP];
  // compact form: the species with a nonzero order in each reaction, and the heat released per
  // mole of each reaction, -sum_k h_f,k W_k nu_jk (J/mol)
  int nord[MAX_RX], ord_k[MAX_RX][MAX_ORD];
  R ord_n[MAX_RX][MAX_ORD];
  R heat[MAX_RX];
  R I_scale;              // integrand -> O(1) before the reduction
  R M_scale;              // mass flux -> O(1) before the reduction
  // variable heat capacities (lbm_set_thermo; varcp = 0: the constant inv_cp above, 1: c_p linear
  // in T, 4: higher powers present):
  // c_p,k(T) = sum_m cp_poly[k][m] T^m (J/(kg K)); W_k h_k(T) = hW_poly[k][0] + T (hW_poly[k][1]
  // + T (... hW_poly[k][5])) (J/mol); cp_in = c_p of the inlet state
  int varcp;
  R cp_poly[MAX_SP][5];
  R hW_poly[MAX_SP][6];
  R cp_in;
  // mixture-averaged species diffusion (lbm_set_transport; mixavg = 0: constant Lewis numbers):
  // pair Lewis numbers Le_kj (rho D_kj = mu / (Pr Le_kj)), the inlet state's 1 / Le_k^mix and W
  int mixavg;
  R Le_pair[MAX_SP][MAX_SP];
  R inv_Lemix_in[MAX_SP];
  R W_in;
};

// ---------------------------------------------------------------------------- storage
// Populations are stored shifted: h = (g - w P_ref) / w. Loads return g.
template <typename S, typename R> __device__ __forceinline__ R ld_pop(const S* p) { return (R)(*p); }
// FP16: read the raw 16-bit word through the read-only path and reinterpret it, so that the
// compiler can issue all loads of a cell back to back
template <> __device__ __forceinline__ float ld_pop<__half, float>(const __half* p) {
  return __half2float(__ushort_as_half(__ldg(reinterpret_cast<const unsigned short*>(p))));
}
template <> __device__ __forceinline__ float ld_pop<float, float>(const float* p) { return __ldg(p); }
template <> __device__ __forceinline__ double ld_pop<double, double>(const double* p) { return __ldg(p); }

// raw load of the stored value (no conversion) and its conversion, for two-phase streaming
// Population loads and stores (C4 stream-collide, A/B in one call each). Loads ask L2 for
// 256-byte prefetches: FP32 0.703 -> 0.697 ms, FP16 0.719 -> 0.708 ms (against the streaming
// hint); not allocating the FP32 loads in L1 made the kernel 5% slower (the x-shifted pulls of
// neighbouring warps share lines there), and the streaming hint on FP32 loads and stores 7%
// slower. The 2-byte stores keep the streaming hint (each population is written once per step).
template <typename S> __device__ __forceinline__ S ld_raw(const S* p) { return __ldg(p); }
template <> __device__ __forceinline__ float ld_raw<float>(const float* p) {
  float v;
  asm("ld.global.nc.L2::256B.f32 %0, [%1];" : "=f"(v) : "l"(p));
  return v;
}
template <> __device__ __forceinline__ __half ld_raw<__half>(const __half* p) {
  unsigned short v;
  asm("ld.global.nc.L2::256B.u16 %0, [%1];" : "=h"(v) : "l"(p));
  return __ushort_as_half(v);
}
template <typename S, typename R> __device__ __forceinline__ R cvt_pop(S v) { return (R)v; }
template <> __device__ __forceinline__ float cvt_pop<__half, float>(__half v) { return __half2float(v); }

template <typename S, typename R> __device__ __forceinline__ void st_pop(S* p, R v) { *p = (S)v; }
template <> __device__ __forceinline__ void st_pop<__half, float>(__half* p, float v) {
  __stcs(reinterpret_cast<unsigned short*>(p), __half_as_ushort(__float2half_rn(v)));
}

// Programmatic dependent launch: a kernel launched with programmatic stream serialization may
// start before its predecessor in the stream has finished. pdl_wait blocks until that predecessor
// has completed and its writes are visible (it returns at once without one); pdl_trigger lets the
// next such kernel start. Kernels call pdl_trigger only after pdl_wait, so that when a kernel
// starts, every kernel before its predecessor has completed.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Launch with programmatic stream serialization when pdl is set (see pdl_wait).
template <typename Arg>
cudaError_t launch_ex(void (*kern)(Arg), dim3 grid, dim3 block, cudaStream_t st, bool pdl, const Arg& arg) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kern, arg);
}
template <typename R> __device__ __forceinline__ R ldg(const R* p) { return __ldg(p); }

// ---------------------------------------------------------------------------- fixed point
// x * 2^32 as a 64-bit integer, using integer operations only (the value of a float is
// mantissa * 2^(exponent - 23), so the product is a shift of the mantissa). Bits below 2^-32
// are truncated. Summing these integers is exact and independent of the order, which makes the
// reductions deterministic. |x| >= 2^30, infinities and NaN saturate to +-2^62 (no shift past the
// word); callers that take terms from outside check the range themselves (fix32_in_range).
__device__ __forceinline__ bool fix32_in_range(float x) { return fabsf(x) < 1073741824.0f; }
__device__ __forceinline__ long long f32_to_fix32(float x) {
  const unsigned b = __float_as_uint(x);
  const int e = (int)((b >> 23) & 0xffu);
  if (e == 0) return 0;  // zero or subnormal: below the resolution
  if (e >= 127 + 30) return (b >> 31) ? -(1LL << 62) : (1LL << 62);
  const long long m = (long long)((b & 0x7fffffu) | 0x800000u);
  const int sh = e - 127 - 23 + 32;
  long long v = sh >= 0 ? (m << sh) : (sh > -64 ? (m >> (-sh)) : 0);
  return (b >> 31) ? -v : v;
}

// Warp-wide sum of a 64-bit integer (exact).
__device__ __forceinline__ long long warp_sum_ll(long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// ---------------------------------------------------------------------------- kernel arguments
constexpr int LB_BLOCK = 128;
// resident blocks per SM the register allocation aims for (C4, D3Q27 thermal: 6 blocks 80
// registers, LB 0.738 / 0.764 ms FP32 / FP16 storage; 7 blocks 0.736 / 0.737 ms; 8 blocks, 64
// registers with spills, 0.767 / 0.807 ms)
#ifndef LB_MIN_BLOCKS
#define LB_MIN_BLOCKS 7
#endif

// link word bit 30: the cell has interpolated bounce-back links (it is on the wall list)
constexpr uint32_t LINK_WALL = 1u << 30;

template <typename R> struct LBArgs {
  Geo geo;
  const void* g_in;
  void* g_out;
  const uint32_t* links;
  const int* wall_cells;  // [n_wall] cells flagged LINK_WALL (interpolated bounce-back)
  const R* wall_q;        // [n_wall][Q] their wall fraction per pull direction (0.5: half-way)
  int n_wall;
  const R* rho;      // thermal: density at level n (lattice units)
  const R* lam;      // thermal: Lambda from the FD update (without the P_th term)
  const R* T;        // thermal: temperature at level n (viscosity law)
  const R* inlet_u;  // [D][ny*nz], low-x face
  const R* u_in;     // [D][N]: velocity of the previous step, read at outlet cells
  R* u;              // [D][N]: written as below (may alias u_in)
  int write_u;       // 1: write u of every cell; 0: outlet cells only
  R* ph_out;         // [N] or nullptr
  const PthState* pth;
  int* flag;
  R nu_lat, T_ref_inv, mu_exp, smag_k, omega_b, om3, om4, om5, om6, P_ref;
};

constexpr int FD_BLOCK = 256;
enum { NB_FLUID = 0, NB_SOLID = 1, NB_INLET = 2, NB_OUTLET = 3 };
// Stencil-word flag: the cell has ghost-point wall weights (fd_row / fd_w of FDArgs).
constexpr uint32_t SW_WALL = 1u << 30;

template <typename R> struct FDArgs {
  Geo geo;
  const uint8_t* mask;
  const uint32_t* sword;  // [N] stencil words (neighbour kinds of the FD stencil)
  const R* T;         // [N] level n
  const R* Y;         // [K][N] level n
  R* T_out;           // [N] level n+1
  R* Y_out;           // [K][N]
  const R* u;         // [D][N]
  const R* inlet_u;   // [D][ny*nz]
  R* Floc;            // [N] flame sensor output (nullptr: F_loc = F)
  R* Floc_out;        // [N] F_loc of the state this update produces (sensor on), else nullptr
  R* rho_out;         // [N]
  R* lam_out;         // [N]
  void* partials;     // [grid][2] fixed-point int64 (float path) or double (double path)
  const PthState* pth;
  // ghost-point walls: for a cell flagged SW_WALL, row fd_row[r] of fd_w holds, per axis side
  // 2a + s, the weight w of the distance-1 wall ghost (phi_r + w (phi_opposite - phi_r)) and then
  // that of the distance-2 wall ghost seen past the fluid neighbour (phi_1 + w (phi_r - phi_1))
  const int* fd_row;
  const R* fd_w;      // [rows][2][2 D]
  int* flag;          // error bits: 4 = a plane load of the tiled update did not arrive in time
  const R* mix;       // mixture-averaged diffusion: per cell G_k [K][N] and W [N] (mix_coeff_kernel)
  int walls_only;     // fd_step_kernel: update only the cells flagged SW_WALL
  const int* wall_list;  // with walls_only: the flagged cells (ascending), one thread each
  int n_wall_list;
  int part_offset;    // fd_step_kernel: first partial slot it writes
  FDConst<R> c;
};

}  // namespace hlbm
