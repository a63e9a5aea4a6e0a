// Host-side declarations of the kernel launchers (one translation unit per lattice/storage,
// compiled in parallel) used by the C-ABI runtime in api.cu.
#pragma once
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include "common.cuh"

namespace hlbm {

template <int D, typename S, typename R>
cudaError_t launch_lb(const LBArgs<R>& a, int thermal, int coll, cudaStream_t st, bool pdl = false);
template <int D, typename R>
cudaError_t launch_fd(const FDArgs<R>& a, cudaStream_t st, bool sensor_pass);

// fd_tiled.cu: tiled FD update of 3-D FP32 grids (TMA plane tiles, faces evaluated once)
struct FDTiledMaps;
bool fd_tiled_eligible(const Geo& g, int D, int f64, int varcp, int K, int nrx);
FDTiledMaps* fd_tiled_create();
void fd_tiled_destroy(FDTiledMaps* m);
// T, Y, F: the two state parities (F nullptr without the flame sensor); n_sm: SMs of the device
cudaError_t fd_tiled_setup(FDTiledMaps& m, const Geo& g, int K, void* const T[2], void* const Y[2],
                           void* const F[2], const void* u, const uint32_t* sword, int n_sm);
int fd_tiled_blocks(const FDTiledMaps& m);
cudaError_t launch_fd_tiled(const FDArgs<float>& a, const FDTiledMaps& m, int cur, cudaStream_t st);

// aux_kernels.cu
cudaError_t launch_links(int D, const Geo& g, const uint8_t* mask, uint32_t* out, cudaStream_t st);
cudaError_t launch_stencil_words(int D, const Geo& g, const uint8_t* mask, uint32_t* out, cudaStream_t st);
int fd_partial_blocks(int D, const Geo& g);
template <typename S, typename R>
cudaError_t launch_set_fields(int D, const Geo& g, const double* T, const double* Y, int K,
                              const double* invW, const double* u, const double* P_h,
                              const double* g_pert, double P_th0_over_R_rho_ref, double P_ref,
                              int thermal, S* g_out, R* T_out, R* Y_out, R* u_out, R* rho_out,
                              R* lam_out, R* ph_out, cudaStream_t st);
template <typename S, typename R>
cudaError_t launch_get_fields(int D, const Geo& g, unsigned bits, int K, const S* gp, const R* T,
                              const R* Y, const R* u, const R* ph, const R* rho, const R* lam,
                              const PthState* pth, double P_ref, double* dst, cudaStream_t st);
template <typename R>
cudaError_t launch_init_integral(const Geo& g, const uint8_t* mask, const R* T, const R* Y, const FDConst<R>& c,
                                 void* partials, int nblocks, cudaStream_t st,
                                 unsigned long long* bad = nullptr);
struct PthUpdate {
  double I_s, M_s, R_rho_ref, cp_rho_ref, rin_fac;  // rin_fac = W_in / (R T_in rho_ref)
  int fixed_point;                                  // partials are int64 fixed point
  int hold;                                         // pressure outlet: P stays, M is still reduced
};
// stage: pth_stage_words() 8-byte words; counter: zero before the first launch (kept zero after)
int pth_stage_words();
cudaError_t launch_pth_update(const PthUpdate& pu, const void* partials, int nblocks, void* stage,
                              unsigned int* counter, PthState* pth, int init, cudaStream_t st);
constexpr int AUX_BLOCK = 256;

// adjoint.cu: one adjoint step. in: adjoint of state n+1, out: adjoint of state n, both in the
// lbm_save_state layout (g 9N, u 2N, T N, Y KN). In thermal runs the step leaves the T and Y parts
// of state n in slot form in `slots` ([9][K+1][N], see adjoint_fd.cuh) and does not write them in
// `out`; it reads those of state n+1 from slots_in, or from `in` where slots_in is null.
// launch_adjoint_gather writes the fields from the slot form. pdl: the LB adjoint may start as the
// previous step's FD adjoint ends (it must be the kernel just before it in the stream, with no
// other dependency in between); the FD adjoint always does so after the LB adjoint. Scratch arrays and the population
// part of out must hold zeros on solid cells (they are never written there): zero them once at
// allocation.
template <typename R> struct AdjBuffers {
  const R* in; R* out;
  R* rho_own; R* lam_bar; R* T_lb; R* u_lb; R* rho_nb;
  const R* slots_in; R* slots;
  R* inlet_bar;
};
// rho_own, lam_bar, T_lb (N each), u_lb (2N), rho_nb (4N), two slot arrays (9 (K + 1) N each)
template <typename R> constexpr size_t adj_scratch_words(size_t N, int K) {
  return (1 + 1 + 1 + 2 + 4 + 2 * 9 * (size_t)(K + 1)) * N;
}
template <typename R>
cudaError_t launch_adjoint_gather(const Geo& g, const uint32_t* sword, int K, const R* slots, R* Tbar, R* Ybar,
                                  cudaStream_t st);
template <typename R>
cudaError_t launch_adjoint_step2d(const AdjBuffers<R>& b, const LBArgs<R>& lbf, const FDArgs<R>& fdf, bool thermal,
                                  bool pdl, cudaStream_t st);
template <typename R> cudaError_t launch_zero_solid_pops(const Geo& g, const uint32_t* links, R* pops, cudaStream_t st);
template <typename R>
cudaError_t launch_initial_T_adjoint(const FDArgs<R>& fdf, const R* adj0, R* gradT, cudaStream_t st);
template <typename R>
cudaError_t launch_fuel_objective(const FDArgs<R>& fdf, int fuel, R* Tbar, R* Ybar, double* partials, int nblocks,
                                  cudaStream_t st);
// stats.cu: running statistics and flame length
int stats_block();
cudaError_t launch_stats_finalize(int N, int nf, const uint32_t* links, const float* mean, const float* m2,
                                  long long n, double* out, cudaStream_t st);
template <typename R>
cudaError_t launch_stats(int N, int nf, const uint32_t* links, const R* u, int D, const R* ph, const R* T, long long n,
                         float* mean, float* m2, cudaStream_t st);
template <typename R>
cudaError_t launch_flame_length(const Geo& g, const uint32_t* links, const R* T, double T_u, double T_b, double level,
                                double* partials, cudaStream_t st);
// flame.cu: inlet conversion and planar-flame properties
template <typename R> cudaError_t launch_to_field(const double* src, R* dst, size_t n, cudaStream_t st);
int flame_col_rows();
template <typename R>
cudaError_t launch_flame_properties(const FDArgs<R>& a, int fuel, double rho_u_per_P, double Y_Fu, double dx,
                                    double* col, double* props, cudaStream_t st);
// probes.cu: probe series and Welch spectra
template <typename R>
cudaError_t launch_probes(const int* cells, int n, int nf, int D, int N, const R* u, const R* ph, const R* T,
                          double* row, cudaStream_t st);
cudaError_t launch_ring_order(const double* ring, long long cap, long long first, long long count, long long row,
                              double* dst, cudaStream_t st);
cudaError_t launch_welch(const double* x, long long stride, long long n, int L, double dt, double* mean_ws,
                         double* psd, cudaStream_t st);
}  // namespace hlbm
