// C-ABI runtime of the library (declared in include/hlbm.h): configuration checks, unit
// conversion, device state, the per-step launch sequence (FD -> thermodynamic pressure -> LB,
// Section 2), CUDA-graph replay of step pairs, kernel timing and checkpoints.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/hlbm.h"
#include "launch.h"

using namespace hlbm;

namespace {
constexpr double R_GAS = 8.314462618;
enum { KIND_FD = 0, KIND_SENSOR = 1, KIND_PTH = 2, KIND_LB = 3 };
}  // namespace

struct lbm_ctx {
  lbm_config cfg;
  std::string err;
  int dev = 0;
  int D = 2, Q = 9, K = 0;
  size_t N = 0;
  bool f64 = false;  // FP64 fields and arithmetic
  size_t S = 4, F = 4;  // bytes per population / per field value
  cudaStream_t st = nullptr;
  bool own_stream = false;
  Geo geo{};
  // device buffers
  void* g[2] = {nullptr, nullptr};
  void* T[2] = {nullptr, nullptr};
  void* Y[2] = {nullptr, nullptr};
  void* u = nullptr;
  void* rho = nullptr;
  void* lam = nullptr;
  void* ph = nullptr;
  void* Floc[2] = {nullptr, nullptr};  // flame sensor F_loc of state cur / the next state
  bool floc_ok = false;                 // Floc[cur] belongs to the current state
  uint32_t* links = nullptr;
  int* wall_cells = nullptr;   // interpolated bounce-back list and table (lbm_set_wall_links)
  void* wall_q = nullptr;
  size_t wall_rows_cap = 0, n_wall = 0;
  int* fd_row = nullptr;        // ghost-point wall weights of the FD update: row per flagged cell
  void* fd_w = nullptr;         // [rows][2][2 D] in the field type
  size_t fd_rows_cap = 0;
  uint32_t* sword = nullptr;
  uint8_t* mask = nullptr;
  void* inlet_u = nullptr;
  void* partials = nullptr;
  int nblocks_fd = 0;    // partial slots written by fd_step_kernel over the whole grid
  FDTiledMaps* tiled = nullptr;  // tiled FD update (3-D FP32), nullptr where it does not apply
  int nblocks_tiled = 0;         // partial slots written by the tiled update
  size_t n_fd_wall_rows = 0;     // cells with ghost-point wall weights (fd_step_kernel, walls only)
  int* fd_wall_list = nullptr;   // those cells, ascending (the tiled update's walls-only launch)
  size_t fd_wall_list_cap = 0;
  void* mix = nullptr;           // mixture-averaged diffusion: per-cell G_k and W [(K + 1)][N]
  int nblocks_init = 0;  // partial slots written by the initial-integral kernel
  PthState* pth = nullptr;
  void* pth_stage = nullptr;            // block sums of the P_th reduction
  unsigned int* pth_counter = nullptr;  // blocks done in the P_th reduction (zero between launches)
  int* flag = nullptr;
  double* scratch_out = nullptr;  // staging for get_fields
  size_t scratch_out_n = 0;
  std::vector<void*> allocs;
  // lattice-unit constants
  FDConst<float> fdc_f{};
  FDConst<double> fdc_d{};
  PthUpdate pu{};
  double nu_lat = 0, W_in = 0;
  size_t n_fluid = 0;
  int cur = 0;
  long long steps = 0;
  bool have_geo = false, have_fields = false;
  // graphs
  bool use_graphs = true;
  cudaGraphExec_t gexec[2] = {nullptr, nullptr};
  // adjoint workspace (allocated zero-filled on the first adjoint call): scratch arrays and one
  // adjoint buffer; segment states (n slots of state + rho + Lambda) for lbm_adjoint_segment
  void* adj_ws = nullptr;
  void* seg_ws = nullptr;
  int seg_cap = 0;
  // second stream and events of the pipelined sweep (lbm_adjoint_sweep)
  cudaStream_t st2 = nullptr;
  cudaEvent_t sw_ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  double* obj_partials = nullptr;
  // running statistics (lbm_stats_control) and flame length
  float* st_mean = nullptr;
  float* st_m2 = nullptr;
  int st_nf = 0, st_interval = 1;
  long long st_n = 0;
  bool st_on = false;
  double* fl_partials = nullptr;
  // planar-flame properties: column means [rows][nx] and the property vector
  double* flame_col = nullptr;
  double* flame_props = nullptr;
  // staging of pageable inlet velocities (dim * ny * nz doubles)
  double* inlet_stage = nullptr;
  // probes: cells, ring buffer [cap][n][nf] of doubles, samples taken so far
  int* pr_cells = nullptr;
  double* pr_ring = nullptr;
  int pr_n = 0, pr_nf = 0, pr_interval = 1;
  long long pr_cap = 0, pr_count = 0;
  size_t pr_ring_words = 0;
  bool pr_on = false;
  // spectrum workspace: segment means, PSD, ordered series
  double* psd_ws = nullptr;
  size_t psd_ws_n = 0;
  // profiling
  bool prof = false;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> ev_used;
  double ms[LBM_KERNEL_KINDS] = {0, 0, 0, 0};
  long long cnt[LBM_KERNEL_KINDS] = {0, 0, 0, 0};
};

namespace {

lbm_status fail(lbm_ctx* c, lbm_status s, const std::string& msg) {
  if (c) c->err = msg;
  return s;
}

lbm_status cuda_fail(lbm_ctx* c, cudaError_t e, const char* where) {
  return fail(c, LBM_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define CK(call, where)                               \
  do {                                                \
    cudaError_t e_ = (call);                          \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, where); \
  } while (0)

void* dalloc(lbm_ctx* c, size_t bytes) {
  if (bytes == 0) bytes = 16;
  void* p = nullptr;
  if (c->cfg.alloc) {
    p = c->cfg.alloc(bytes, c->cfg.alloc_user);
  } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    p = nullptr;
  }
  if (p) c->allocs.push_back(p);
  return p;
}

// A pointer the device can dereference for this host pointer: pinned (page-locked) host memory
// through its device mapping, device or managed memory as it is; nullptr for pageable memory.
const double* device_view(const double* p) {
  if (!p) return nullptr;
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) return p;
  if (a.type == cudaMemoryTypeHost && a.devicePointer) return (const double*)a.devicePointer;
  return nullptr;
}

void dfree_all(lbm_ctx* c) {
  for (void* p : c->allocs) {
    if (c->cfg.free) c->cfg.free(p, c->cfg.alloc_user);
    else cudaFree(p);
  }
  c->allocs.clear();
}

void drop_graphs(lbm_ctx* c) {
  for (auto& ge : c->gexec)
    if (ge) {
      cudaGraphExecDestroy(ge);
      ge = nullptr;
    }
}

lbm_status validate(const lbm_config* cfg, std::string& msg) {
  auto bad = [&](const char* m) {
    msg = m;
    return LBM_ERR_ARG;
  };
  if (cfg->dim != 2 && cfg->dim != 3) return bad("dim must be 2 or 3");
  if (cfg->nx < 1 || cfg->ny < 1 || (cfg->dim == 3 && cfg->nz < 1)) return bad("grid sizes must be >= 1");
  const double N = (double)cfg->nx * cfg->ny * (cfg->dim == 3 ? cfg->nz : 1);
  if (N * (cfg->dim == 2 ? 9 : 27) > 2147483000.0) return bad("Q * cells must stay below 2^31");
  if (cfg->storage < LBM_STORE_F64 || cfg->storage > LBM_STORE_F16) return bad("unknown storage");
  if (cfg->collision != LBM_COLL_BGK && cfg->collision != LBM_COLL_CUMULANT) return bad("unknown collision");
  for (int a = 0; a < cfg->dim; ++a) {
    const int lo = cfg->bc_lo[a], hi = cfg->bc_hi[a];
    if (lo < 0 || lo > 3 || hi < 0 || hi > 3) return bad("unknown boundary code");
    if (lo == LBM_BC_OUTLET || hi == LBM_BC_INLET) return bad("inlet only on low x, outlet only on high x");
    if (a > 0 && (lo >= LBM_BC_INLET || hi >= LBM_BC_INLET)) return bad("inlet/outlet only on the x faces");
    if ((lo == LBM_BC_PERIODIC) != (hi == LBM_BC_PERIODIC)) return bad("periodic must pair with periodic");
  }
  if (!(cfg->dx > 0) || !(cfg->dt > 0) || !(cfg->nu_ref > 0)) return bad("dx, dt, nu_ref must be > 0");
  if (cfg->smag_cs < 0) return bad("smag_cs must be >= 0");
  if (cfg->thermal) {
    if (cfg->n_species < 1 || cfg->n_species > LBM_MAX_SPECIES) return bad("thermal needs 1..8 species");
    if (cfg->n_reactions < 0 || cfg->n_reactions > LBM_MAX_REACTIONS) return bad("at most 4 reactions");
    if (!(cfg->P_th0 > 0) || !(cfg->T_ref > 0) || !(cfg->cp > 0) || !(cfg->rho_ref > 0) || !(cfg->Pr > 0))
      return bad("P_th0, T_ref, cp, rho_ref, Pr must be > 0");
    for (int k = 0; k < cfg->n_species; ++k)
      if (!(cfg->sp[k].W > 0) || !(cfg->sp[k].Le > 0)) return bad("species W and Le must be > 0");
    if (cfg->flame_sensor && (cfg->sensor_species < 0 || cfg->sensor_species >= cfg->n_species ||
                              cfg->sensor_oxidizer < 0 || cfg->sensor_oxidizer >= cfg->n_species ||
                              !(cfg->sensor_wref > 0) || !(cfg->sensor_Ta >= 0)))
      return bad("invalid flame sensor parameters");
    if (!(cfg->thicken_F >= 1.0)) return bad("thicken_F must be >= 1");
    for (int j = 0; j < cfg->n_reactions; ++j) {
      int nz = 0;
      for (int k = 0; k < cfg->n_species; ++k) nz += cfg->rx[j].order[k] != 0.0;
      if (nz > 4) return bad("at most 4 species with a nonzero order per reaction");
    }
  } else if (cfg->closed_domain || cfg->flame_sensor) {
    return bad("closed_domain and flame_sensor need thermal");
  }
  return LBM_OK;
}

template <typename R> LBArgs<R> make_lb_args(lbm_ctx* c, int cur, bool want_out) {
  LBArgs<R> a{};
  a.geo = c->geo;
  a.g_in = c->g[cur];
  a.g_out = c->g[1 - cur];
  a.links = c->links;
  a.wall_cells = c->wall_cells;
  a.wall_q = (const R*)c->wall_q;
  a.n_wall = (int)c->n_wall;
  a.rho = (const R*)c->rho;
  a.lam = (const R*)c->lam;
  a.T = (const R*)c->T[cur];
  a.inlet_u = (const R*)c->inlet_u;
  a.u = (R*)c->u;
  a.u_in = a.u;
  a.write_u = (c->cfg.thermal || want_out) ? 1 : 0;
  a.ph_out = want_out ? (R*)c->ph : nullptr;
  a.pth = c->pth;
  a.flag = c->flag;
  a.nu_lat = (R)c->nu_lat;
  a.T_ref_inv = (R)(1.0 / c->cfg.T_ref);
  a.mu_exp = (R)c->cfg.mu_exp;
  a.smag_k = (R)(18.0 * std::sqrt(2.0) * c->cfg.smag_cs * c->cfg.smag_cs);
  a.omega_b = (R)c->cfg.omega_bulk;
  a.om3 = (R)c->cfg.omega_hi[0];
  a.om4 = (R)c->cfg.omega_hi[1];
  a.om5 = (R)c->cfg.omega_hi[2];
  a.om6 = (R)c->cfg.omega_hi[3];
  a.P_ref = (R)c->cfg.P_ref;
  return a;
}

template <typename R> const FDConst<R>& fdconst(const lbm_ctx* c);
template <> const FDConst<float>& fdconst<float>(const lbm_ctx* c) { return c->fdc_f; }
template <> const FDConst<double>& fdconst<double>(const lbm_ctx* c) { return c->fdc_d; }

// Lattice-unit constants of the finite-difference update in the arithmetic type R.
template <typename R> void fill_fdconst(FDConst<R>& f, const lbm_config& c, int K, double nu_lat, double I_unit) {
  f.K = K;
  f.nrx = c.thermal ? c.n_reactions : 0;
  f.sensor = c.flame_sensor;
  f.sensor_species = c.sensor_species;
  f.sensor_oxidizer = c.sensor_oxidizer;
  f.sensor_Ta = (R)c.sensor_Ta;
  f.closed = c.closed_domain;
  f.nu_lat = (R)nu_lat;
  f.T_ref_inv = (R)(1.0 / c.T_ref);
  f.mu_exp = (R)c.mu_exp;
  f.inv_Pr = (R)(1.0 / c.Pr);
  f.dt_phys = (R)c.dt;
  f.inv_cp = (R)(1.0 / c.cp);
  f.inv_rho_ref = (R)(1.0 / c.rho_ref);
  f.rho_ref_f = (R)c.rho_ref;
  f.F = (R)c.thicken_F;
  f.sensor_beta = (R)c.sensor_beta;
  f.inv_wref = (R)(c.sensor_wref > 0 ? 1.0 / c.sensor_wref : 0.0);
  f.eps_T = (R)(1e-6 * c.T_ref * c.T_ref);
  f.eps_Y = (R)1e-6;
  f.T_in = (R)c.T_in;
  for (int k = 0; k < K; ++k) {
    f.inv_Le[k] = (R)(1.0 / c.sp[k].Le);
    f.inv_W[k] = (R)(1.0 / c.sp[k].W);
    f.W[k] = (R)c.sp[k].W;
    f.hf_W[k] = (R)(c.sp[k].hf * c.sp[k].W);
    f.Y_in[k] = (R)c.Y_in[k];
  }
  for (int j = 0; j < f.nrx; ++j) {
    const lbm_reaction& rx = c.rx[j];
    f.A[j] = (R)rx.A;
    f.beta[j] = (R)rx.beta;
    const double ER = rx.E / R_GAS;
    f.ER_hi[j] = (R)ER;
    f.ER_lo[j] = (R)(ER - (double)f.ER_hi[j]);
    double heat = 0.0;
    f.nord[j] = 0;
    for (int k = 0; k < K; ++k) {
      f.nu[j][k] = (R)rx.nu[k];
      f.order[j][k] = (R)rx.order[k];
      heat -= c.sp[k].hf * c.sp[k].W * rx.nu[k];
      if (rx.order[k] != 0.0 && f.nord[j] < MAX_ORD) {
        f.ord_k[j][f.nord[j]] = k;
        f.ord_n[j][f.nord[j]] = (R)rx.order[k];
        ++f.nord[j];
      }
    }
    f.heat[j] = (R)heat;
  }
  f.I_scale = (R)I_unit;
  f.M_scale = (R)16.0;
}

template <typename R> FDArgs<R> make_fd_args(lbm_ctx* c, int cur) {
  FDArgs<R> a{};
  a.geo = c->geo;
  a.mask = c->mask;
  a.sword = c->sword;
  a.T = (const R*)c->T[cur];
  a.Y = (const R*)c->Y[cur];
  a.T_out = (R*)c->T[1 - cur];
  a.Y_out = (R*)c->Y[1 - cur];
  a.u = (const R*)c->u;
  a.inlet_u = (const R*)c->inlet_u;
  a.Floc = c->cfg.flame_sensor ? (R*)c->Floc[cur] : nullptr;
  a.Floc_out = c->cfg.flame_sensor ? (R*)c->Floc[1 - cur] : nullptr;
  a.rho_out = (R*)c->rho;
  a.lam_out = (R*)c->lam;
  a.partials = c->partials;
  a.pth = c->pth;
  a.fd_row = c->fd_row;
  a.fd_w = (const R*)c->fd_w;
  a.flag = c->flag;
  a.mix = (const R*)c->mix;
  a.walls_only = 0;
  a.part_offset = 0;
  a.c = fdconst<R>(c);
  return a;
}

cudaError_t run_lb(lbm_ctx* c, int cur, bool want_out) {
  const int th = c->cfg.thermal;
  // the cumulant kernel has a variant for the default case where orders 3..6 relax fully
  const bool hi1 = c->cfg.omega_hi[0] == 1.0 && c->cfg.omega_hi[1] == 1.0 && c->cfg.omega_hi[2] == 1.0 &&
                   c->cfg.omega_hi[3] == 1.0;
  const int co = c->cfg.collision == LBM_COLL_CUMULANT ? (hi1 ? COLL_CUMULANT_FULL : COLL_CUMULANT) : COLL_BGK;
  // in a closed domain the step launches the thermodynamic-pressure update just before: the
  // stream-collide may start with it and waits for its state (programmatic dependent launch)
  const bool pdl = th && c->cfg.closed_domain;
  if (c->f64) {
    auto a = make_lb_args<double>(c, cur, want_out);
    return c->D == 2 ? launch_lb<2, double, double>(a, th, co, c->st, pdl)
                     : launch_lb<3, double, double>(a, th, co, c->st, pdl);
  }
  auto a = make_lb_args<float>(c, cur, want_out);
  if (c->cfg.storage == LBM_STORE_F16)
    return c->D == 2 ? launch_lb<2, __half, float>(a, th, co, c->st, pdl)
                     : launch_lb<3, __half, float>(a, th, co, c->st, pdl);
  return c->D == 2 ? launch_lb<2, float, float>(a, th, co, c->st, pdl) : launch_lb<3, float, float>(a, th, co, c->st, pdl);
}

// the tiled update applies (3-D FP32, constant heat capacity, grid and chemistry it supports)
bool use_tiled(const lbm_ctx* c) { return c->tiled && !c->fdc_f.varcp && !c->fdc_f.mixavg; }

// partial slots of the P_th reduction written by one FD update
int fd_slots(const lbm_ctx* c) {
  if (!use_tiled(c)) return c->nblocks_fd;
  return c->nblocks_tiled + (int)((c->n_fd_wall_rows + FD_BLOCK - 1) / FD_BLOCK);
}

cudaError_t run_fd(lbm_ctx* c, int cur, bool sensor_pass) {
  if (c->f64) {
    auto a = make_fd_args<double>(c, cur);
    return c->D == 2 ? launch_fd<2, double>(a, c->st, sensor_pass) : launch_fd<3, double>(a, c->st, sensor_pass);
  }
  auto a = make_fd_args<float>(c, cur);
  if (!sensor_pass && use_tiled(c)) {
    cudaError_t e = launch_fd_tiled(a, *c->tiled, cur, c->st);
    if (e != cudaSuccess || !c->n_fd_wall_rows) return e;
    // cells with ghost-point wall weights: the general kernel over their list, partial slots after
    // the tiled ones
    a.walls_only = 1;
    a.wall_list = c->fd_wall_list;
    a.n_wall_list = (int)c->n_fd_wall_rows;
    a.part_offset = c->nblocks_tiled;
    return launch_fd<3, float>(a, c->st, false);
  }
  return c->D == 2 ? launch_fd<2, float>(a, c->st, sensor_pass) : launch_fd<3, float>(a, c->st, sensor_pass);
}

cudaError_t timed(lbm_ctx* c, int kind, cudaError_t (*fn)(lbm_ctx*, int, int), int cur, int arg) {
  if (!c->prof) return fn(c, cur, arg);
  cudaEvent_t e0, e1;
  if (c->ev_pool.size() >= 2) {
    e0 = c->ev_pool.back(); c->ev_pool.pop_back();
    e1 = c->ev_pool.back(); c->ev_pool.pop_back();
  } else {
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
  }
  cudaEventRecord(e0, c->st);
  cudaError_t e = fn(c, cur, arg);
  cudaEventRecord(e1, c->st);
  c->ev_used.push_back({kind, {e0, e1}});
  return e;
}

cudaError_t fd_thunk(lbm_ctx* c, int cur, int sensor) { return run_fd(c, cur, sensor != 0); }
cudaError_t lb_thunk(lbm_ctx* c, int cur, int want) { return run_lb(c, cur, want != 0); }
cudaError_t pth_thunk(lbm_ctx* c, int, int) {
  return launch_pth_update(c->pu, c->partials, fd_slots(c), c->pth_stage, c->pth_counter, c->pth, 0, c->st);
}

// One full step from parity `cur`: FD (+ sensor) -> P_th -> LB.
cudaError_t enqueue_step(lbm_ctx* c, int cur, bool want_out) {
  cudaError_t e;
  if (c->cfg.thermal) {
    // the FD update writes F_loc of the state it produces; the sensor pass runs only when the
    // state came from outside (lbm_step ensures it before any capture)
    if (c->cfg.flame_sensor && !c->floc_ok && (e = timed(c, KIND_SENSOR, fd_thunk, cur, 1)) != cudaSuccess)
      return e;
    if (c->cfg.flame_sensor) c->floc_ok = true;
    if ((e = timed(c, KIND_FD, fd_thunk, cur, 0)) != cudaSuccess) return e;
    if (c->cfg.closed_domain && (e = timed(c, KIND_PTH, pth_thunk, cur, 0)) != cudaSuccess) return e;
  }
  return timed(c, KIND_LB, lb_thunk, cur, want_out ? 1 : 0);
}

cudaError_t build_graph(lbm_ctx* c, int cur) {
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamBeginCapture(c->st, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return e;
  cudaError_t e1 = enqueue_step(c, cur, false);
  cudaError_t e2 = e1 == cudaSuccess ? enqueue_step(c, 1 - cur, false) : e1;
  e = cudaStreamEndCapture(c->st, &graph);
  if (e2 != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return e2;
  }
  if (e != cudaSuccess) return e;
  e = cudaGraphInstantiate(&c->gexec[cur], graph, 0);
  cudaGraphDestroy(graph);
  return e;
}

size_t fields_size(const lbm_ctx* c, unsigned bits) {
  size_t n = 0;
  if (bits & LBM_F_T) n += c->N;
  if (bits & LBM_F_Y) n += (size_t)c->K * c->N;
  if (bits & LBM_F_U) n += (size_t)c->D * c->N;
  if (bits & LBM_F_PH) n += c->N;
  if (bits & LBM_F_RHO) n += c->N;
  if (bits & LBM_F_LAM) n += c->N;
  if (bits & LBM_F_G) n += (size_t)c->Q * c->N;
  return n;
}

}  // namespace

extern "C" {

lbm_status lbm_init(const lbm_config* cfg, lbm_ctx** out) {
  if (!cfg || !out) return LBM_ERR_ARG;
  *out = nullptr;
  std::string msg;
  lbm_status s = validate(cfg, msg);
  lbm_ctx* ctx = new (std::nothrow) lbm_ctx();
  if (!ctx) return LBM_ERR_ALLOC;
  ctx->cfg = *cfg;
  *out = ctx;
  if (s != LBM_OK) return fail(ctx, s, msg);
  lbm_config& c = ctx->cfg;
  if (c.dim == 2) c.nz = 1;
  CK(cudaGetDevice(&ctx->dev), "cudaGetDevice");
  ctx->st = (cudaStream_t)c.stream;
  if (!ctx->st) {
    // graph capture needs a stream other than the legacy default stream; a blocking stream
    // still orders itself with the legacy default stream
    CK(cudaStreamCreate(&ctx->st), "cudaStreamCreate");
    ctx->own_stream = true;
  }
  ctx->D = c.dim;
  ctx->Q = c.dim == 2 ? 9 : 27;
  ctx->K = c.thermal ? c.n_species : 0;
  ctx->N = (size_t)c.nx * c.ny * c.nz;
  ctx->f64 = c.storage == LBM_STORE_F64;
  ctx->S = c.storage == LBM_STORE_F64 ? 8 : (c.storage == LBM_STORE_F32 ? 4 : 2);
  ctx->F = ctx->f64 ? 8 : 4;
  Geo& g = ctx->geo;
  g.nx = c.nx;
  g.ny = c.ny;
  g.nz = c.nz;
  g.N = (int)ctx->N;
  for (int a = 0; a < 3; ++a) {
    g.bc_lo[a] = a < c.dim ? c.bc_lo[a] : BC_PERIODIC;
    g.bc_hi[a] = a < c.dim ? c.bc_hi[a] : BC_PERIODIC;
  }
  // lattice units: nu_lat = nu dt / dx^2, tau = nu_lat / cs2 + 1/2 (Eq. 12)
  ctx->nu_lat = c.nu_ref * c.dt / (c.dx * c.dx);
  double sWin = 0.0;
  for (int k = 0; k < ctx->K; ++k) sWin += c.Y_in[k] / c.sp[k].W;
  ctx->W_in = sWin > 0 ? 1.0 / sWin : 0.0;
  // reduction scale: the integrand W / (R T rho_ref) ~ 1e-5 is computed as I_unit * W / T ~ 1
  const double I_unit = c.T_ref / 0.029;
  fill_fdconst<float>(ctx->fdc_f, c, ctx->K, ctx->nu_lat, I_unit);
  fill_fdconst<double>(ctx->fdc_d, c, ctx->K, ctx->nu_lat, I_unit);
  PthUpdate& pu = ctx->pu;
  // I = sum(I_unit W/T) / I_s with I_s = I_unit R rho_ref, using the exact scale of the kernels
  pu.I_s = (ctx->f64 ? (double)ctx->fdc_d.I_scale : (double)ctx->fdc_f.I_scale) * R_GAS * c.rho_ref;
  pu.M_s = 16.0;
  pu.R_rho_ref = R_GAS * c.rho_ref;
  pu.cp_rho_ref = c.cp * c.rho_ref;
  pu.rin_fac = c.thermal ? ctx->W_in / (R_GAS * c.T_in * c.rho_ref) : 0.0;
  pu.fixed_point = ctx->f64 ? 0 : 1;
  pu.hold = c.bc_hi[0] == LBM_BC_OUTLET ? 1 : 0;

  // device state
  const size_t N = ctx->N;
  bool ok = true;
  for (int b = 0; b < 2; ++b) ok = ok && (ctx->g[b] = dalloc(ctx, (size_t)ctx->Q * N * ctx->S));
  ok = ok && (ctx->u = dalloc(ctx, (size_t)ctx->D * N * ctx->F));
  ok = ok && (ctx->rho = dalloc(ctx, N * ctx->F));
  ok = ok && (ctx->lam = dalloc(ctx, N * ctx->F));
  ok = ok && (ctx->ph = dalloc(ctx, N * ctx->F));
  ok = ok && (ctx->links = (uint32_t*)dalloc(ctx, N * 4));
  ok = ok && (ctx->sword = (uint32_t*)dalloc(ctx, N * 4));
  ok = ok && (ctx->mask = (uint8_t*)dalloc(ctx, N));
  ok = ok && (ctx->inlet_u = dalloc(ctx, (size_t)ctx->D * c.ny * c.nz * ctx->F));
  ok = ok && (ctx->pth = (PthState*)dalloc(ctx, sizeof(PthState)));
  ok = ok && (ctx->flag = (int*)dalloc(ctx, 16));
  ctx->nblocks_fd = fd_partial_blocks(ctx->D, ctx->geo);
  ctx->nblocks_init = (int)((N + AUX_BLOCK - 1) / AUX_BLOCK);
  if (c.thermal && fd_tiled_eligible(ctx->geo, ctx->D, ctx->f64, 0, ctx->K, c.n_reactions)) {
    ctx->tiled = fd_tiled_create();
    if (!ctx->tiled) ok = false;
  }
  ok = ok && (ctx->partials = dalloc(ctx, (size_t)std::max(ctx->nblocks_fd * (ctx->tiled ? 2 : 1),
                                                           ctx->nblocks_init) * 16));
  ok = ok && (ctx->pth_stage = dalloc(ctx, (size_t)pth_stage_words() * 8));
  ok = ok && (ctx->pth_counter = (unsigned int*)dalloc(ctx, 16));
  if (c.thermal) {
    for (int b = 0; b < 2; ++b) {
      ok = ok && (ctx->T[b] = dalloc(ctx, N * ctx->F));
      ok = ok && (ctx->Y[b] = dalloc(ctx, (size_t)ctx->K * N * ctx->F));
    }
    if (c.flame_sensor)
      for (int b = 0; b < 2; ++b) ok = ok && (ctx->Floc[b] = dalloc(ctx, N * ctx->F));
  }
  if (!ok) {
    dfree_all(ctx);
    return fail(ctx, LBM_ERR_ALLOC, "device allocation failed");
  }
  CK(cudaMemsetAsync(ctx->flag, 0, 16, ctx->st), "memset");
  CK(cudaMemsetAsync(ctx->pth_counter, 0, 16, ctx->st), "memset");
  CK(cudaMemsetAsync(ctx->inlet_u, 0, (size_t)ctx->D * c.ny * c.nz * ctx->F, ctx->st), "memset");
  if (ctx->tiled) {
    int n_sm = 0;
    CK(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, ctx->dev), "device attribute");
    CK(fd_tiled_setup(*ctx->tiled, ctx->geo, ctx->K, ctx->T, ctx->Y, ctx->Floc, ctx->u, ctx->sword, n_sm),
       "tensor maps of the tiled FD update");
    ctx->nblocks_tiled = fd_tiled_blocks(*ctx->tiled);
    if (ctx->nblocks_tiled > ctx->nblocks_fd) return fail(ctx, LBM_ERR_ARG, "tiled FD grid too large");
  }
  for (int b = 0; b < 2; ++b)
    if (ctx->Floc[b]) CK(cudaMemsetAsync(ctx->Floc[b], 0, N * ctx->F, ctx->st), "memset");
  return LBM_OK;
}

void lbm_destroy(lbm_ctx* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->dev);
  if (ctx->st) cudaStreamSynchronize(ctx->st);
  else cudaDeviceSynchronize();
  drop_graphs(ctx);
  for (auto& e : ctx->ev_used) {
    cudaEventDestroy(e.second.first);
    cudaEventDestroy(e.second.second);
  }
  for (auto e : ctx->ev_pool) cudaEventDestroy(e);
  if (ctx->st2) cudaStreamSynchronize(ctx->st2);
  for (auto e : ctx->sw_ev)
    if (e) cudaEventDestroy(e);
  if (ctx->st2) cudaStreamDestroy(ctx->st2);
  dfree_all(ctx);
  fd_tiled_destroy(ctx->tiled);
  if (ctx->own_stream) cudaStreamDestroy(ctx->st);
  delete ctx;
}

const char* lbm_last_error(const lbm_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

namespace {
// Inlet-face velocities ([dim][ny nz] doubles) converted to the field type on the device. Input
// the device can read in place is converted directly; pageable host memory goes through a
// staging buffer the context keeps (cudaMemcpyAsync has taken the data when it returns).
lbm_status set_inlet_impl(lbm_ctx* ctx, const double* inlet_u, int on_device) {
  const size_t n = (size_t)ctx->D * ctx->cfg.ny * ctx->cfg.nz;
  const double* src = on_device ? inlet_u : device_view(inlet_u);
  if (!src) {
    if (!ctx->inlet_stage && !(ctx->inlet_stage = (double*)dalloc(ctx, n * 8)))
      return fail(ctx, LBM_ERR_ALLOC, "allocation failed");
    CK(cudaMemcpyAsync(ctx->inlet_stage, inlet_u, n * 8, cudaMemcpyHostToDevice, ctx->st), "copy inlet");
    src = ctx->inlet_stage;
  }
  if (ctx->f64) CK(launch_to_field<double>(src, (double*)ctx->inlet_u, n, ctx->st), "inlet kernel");
  else CK(launch_to_field<float>(src, (float*)ctx->inlet_u, n, ctx->st), "inlet kernel");
  return LBM_OK;
}
}  // namespace

extern "C++" {
namespace {
// Heat-capacity polynomials into the FD constants of type R: c_p,k and W_k h_k with
// h_k(T) = h_f,k + integral from T0 to T of c_p,k.
template <typename R> void fill_thermo(FDConst<R>& f, const lbm_config& c, int K, const double* cp, double T0) {
  f.varcp = 0;
  if (cp) {
    f.varcp = 1;  // degree of the kernel variant: 1 when every c_p,k is linear in T, else 4
    for (int k = 0; k < K; ++k)
      for (int m = 2; m < 5; ++m)
        if (cp[5 * k + m] != 0.0) f.varcp = 4;
  }
  for (int k = 0; k < MAX_SP; ++k) {
    for (int m = 0; m < 5; ++m) f.cp_poly[k][m] = R(0);
    for (int m = 0; m < 6; ++m) f.hW_poly[k][m] = R(0);
  }
  f.cp_in = (R)c.cp;
  if (!cp) return;
  double cp_in = 0.0;
  for (int k = 0; k < K; ++k) {
    const double* a = cp + 5 * k;
    const double W = c.sp[k].W;
    double h0 = c.sp[k].hf, Tp = T0, ck = 0.0, Tm = 1.0;
    for (int m = 0; m < 5; ++m) {
      h0 -= a[m] * Tp / (m + 1);  // minus the integral's value at T0
      Tp *= T0;
      f.cp_poly[k][m] = (R)a[m];
      f.hW_poly[k][m + 1] = (R)(W * a[m] / (m + 1));
      ck += a[m] * Tm;
      Tm *= c.T_in;
    }
    f.hW_poly[k][0] = (R)(W * h0);
    cp_in += c.Y_in[k] * ck;
  }
  f.cp_in = (R)cp_in;
}
}  // namespace
}  // extern "C++"

lbm_status lbm_set_thermo(lbm_ctx* ctx, const double* cp, double T0) {
  if (!ctx) return LBM_ERR_ARG;
  if (cp && ctx->fdc_d.mixavg)
    return fail(ctx, LBM_ERR_UNSUPPORTED, "variable heat capacities with mixture-averaged diffusion");
  if (cp && (!ctx->cfg.thermal || !(T0 > 0.0)))
    return fail(ctx, LBM_ERR_ARG, "variable heat capacities need a thermal run and T0 > 0");
  if (cp)
    for (int i = 0; i < 5 * ctx->K; ++i)
      if (!std::isfinite(cp[i])) return fail(ctx, LBM_ERR_ARG, "non-finite heat-capacity coefficient");
  fill_thermo<float>(ctx->fdc_f, ctx->cfg, ctx->K, cp, T0);
  fill_thermo<double>(ctx->fdc_d, ctx->cfg, ctx->K, cp, T0);
  drop_graphs(ctx);  // the captured launches hold the old constants
  return LBM_OK;
}

}  // extern "C"

namespace {
template <typename R> void fill_transport(FDConst<R>& f, const lbm_config& c, int K, const double* Le, double W_in) {
  f.mixavg = Le ? 1 : 0;
  f.W_in = (R)W_in;
  for (int k = 0; k < MAX_SP; ++k) {
    f.inv_Lemix_in[k] = R(0);
    for (int j = 0; j < MAX_SP; ++j) f.Le_pair[k][j] = (k < K && j < K && Le) ? (R)Le[k * K + j] : R(1);
  }
  if (!Le) return;
  // 1 / Le_k^mix of the inlet state (the inlet ghost's coefficient), same rule as mix_coeff_kernel
  double X[MAX_SP];
  for (int k = 0; k < K; ++k) X[k] = std::max(c.Y_in[k] * W_in / c.sp[k].W, 0.0) + 1e-10;
  for (int k = 0; k < K; ++k) {
    double num = 0.0, den = 0.0;
    for (int j = 0; j < K; ++j)
      if (j != k) {
        num += X[j] * Le[k * K + j];
        den += X[j];
      }
    f.inv_Lemix_in[k] = (R)(den / num);
  }
}
}  // namespace

extern "C" {

lbm_status lbm_set_transport(lbm_ctx* ctx, const double* Le_pair) {
  if (!ctx) return LBM_ERR_ARG;
  if (Le_pair) {
    if (!ctx->cfg.thermal || ctx->K < 2) return fail(ctx, LBM_ERR_ARG, "mixture-averaged diffusion needs species");
    for (int i = 0; i < ctx->K * ctx->K; ++i)
      if (!std::isfinite(Le_pair[i]) || !(Le_pair[i] > 0.0))
        return fail(ctx, LBM_ERR_ARG, "pair Lewis numbers must be finite and > 0");
    if (ctx->fdc_d.varcp)
      return fail(ctx, LBM_ERR_UNSUPPORTED, "mixture-averaged diffusion with variable heat capacities");
    if (ctx->n_fd_wall_rows)
      return fail(ctx, LBM_ERR_UNSUPPORTED, "mixture-averaged diffusion with ghost-point (curved) walls");
    if (!ctx->mix && !(ctx->mix = dalloc(ctx, (size_t)(ctx->K + 1) * ctx->N * ctx->F)))
      return fail(ctx, LBM_ERR_ALLOC, "allocation failed");
  }
  fill_transport<float>(ctx->fdc_f, ctx->cfg, ctx->K, Le_pair, ctx->W_in);
  fill_transport<double>(ctx->fdc_d, ctx->cfg, ctx->K, Le_pair, ctx->W_in);
  drop_graphs(ctx);  // the captured launches hold the old constants
  return LBM_OK;
}

lbm_status lbm_set_inlet(lbm_ctx* ctx, const double* inlet_u, int on_device) {
  if (!ctx || !inlet_u) return fail(ctx, LBM_ERR_ARG, "null argument");
  if (!ctx->have_geo) return fail(ctx, LBM_ERR_STATE, "set_geometry must come first");
  CK(cudaSetDevice(ctx->dev), "cudaSetDevice");
  return set_inlet_impl(ctx, inlet_u, on_device);
}

lbm_status lbm_set_geometry(lbm_ctx* ctx, const uint8_t* mask, const double* inlet_u, int on_device) {
  if (!ctx || !mask) return fail(ctx, LBM_ERR_ARG, "null argument");
  if (ctx->allocs.empty()) return fail(ctx, LBM_ERR_STATE, "context not initialised");
  CK(cudaSetDevice(ctx->dev), "cudaSetDevice");
  const size_t N = ctx->N;
  const auto kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  CK(cudaMemcpyAsync(ctx->mask, mask, N, kind, ctx->st), "copy mask");
  const size_t nf = (size_t)ctx->cfg.ny * ctx->cfg.nz;
  if (inlet_u) {
    lbm_status st = set_inlet_impl(ctx, inlet_u, on_device);
    if (st != LBM_OK) return st;
  }
  CK(launch_links(ctx->D, ctx->geo, ctx->mask, ctx->links, ctx->st), "links kernel");
  CK(launch_stencil_words(ctx->D, ctx->geo, ctx->mask, ctx->sword, ctx->st), "stencil words kernel");
  std::vector<uint8_t> hm(N);
  CK(cudaMemcpyAsync(hm.data(), ctx->mask, N, cudaMemcpyDeviceToHost, ctx->st), "copy mask");
  CK(cudaStreamSynchronize(ctx->st), "sync");
  size_t nfl = 0;
  for (size_t i = 0; i < N; ++i) nfl += hm[i] == 0;
  ctx->n_fluid = nfl;
  ctx->have_geo = true;
  ctx->floc_ok = false;
  ctx->n_wall = 0;  // the rebuilt link words carry no interpolated walls
  drop_graphs(ctx);
  return LBM_OK;
}

lbm_status lbm_set_fields(lbm_ctx* ctx, const double* T, const double* Y, const double* u, const double* P_h,
                          const double* g_pert, int on_device) {
  if (!ctx || !u || !P_h) return fail(ctx, LBM_ERR_ARG, "null argument");
  if (!ctx->have_geo) return fail(ctx, LBM_ERR_STATE, "set_geometry must come first");
  const lbm_config& c = ctx->cfg;
  if (c.thermal && (!T || !Y)) return fail(ctx, LBM_ERR_ARG, "thermal run needs T and Y");
  CK(cudaSetDevice(ctx->dev), "cudaSetDevice");
  const size_t N = ctx->N, K = ctx->K, D = ctx->D, Q = ctx->Q;
  // inputs the kernel can read in place (device memory, or pinned host memory through its device
  // mapping) are used directly; the others are staged in one device buffer
  const size_t nT = c.thermal ? N : 0, nY = c.thermal ? K * N : 0, nG = g_pert ? Q * N : 0;
  const double* vT = on_device ? T : device_view(T);
  const double* vY = on_device ? Y : device_view(Y);
  const double* vu = on_device ? u : device_view(u);
  const double* vP = on_device ? P_h : device_view(P_h);
  const double* vG = on_device ? g_pert : device_view(g_pert);
  const size_t total = (nT && !vT ? nT : 0) + (nY && !vY ? nY : 0) + (vu ? 0 : D * N) + (vP ? 0 : N) +
                       (nG && !vG ? nG : 0) + 8;
  double* buf = (double*)dalloc(ctx, total * 8);
  if (!buf) return fail(ctx, LBM_ERR_ALLOC, "allocation failed");
  double* next = buf;
  lbm_status st = LBM_OK;
  auto stage = [&](const double* view, const double* src, size_t n) -> const double* {
    if (!n || !src) return nullptr;
    if (view) return view;
    double* dst = next;
    next += n;
    if (st == LBM_OK) {
      cudaError_t e = cudaMemcpyAsync(dst, src, n * 8, cudaMemcpyHostToDevice, ctx->st);
      if (e != cudaSuccess) st = cuda_fail(ctx, e, "copy fields");
    }
    return dst;
  };
  const double* dT = stage(vT, T, nT);
  const double* dY = stage(vY, Y, nY);
  const double* du = stage(vu, u, D * N);
  const double* dP = stage(vP, P_h, N);
  const double* dG = stage(vG, g_pert, nG);
  double* dW = next;
  double invW[LBM_MAX_SPECIES] = {0};
  for (size_t k = 0; k < K; ++k) invW[k] = 1.0 / c.sp[k].W;
  if (st == LBM_OK) {
    cudaError_t e = cudaMemcpyAsync(dW, invW, 8 * LBM_MAX_SPECIES, cudaMemcpyHostToDevice, ctx->st);
    if (e != cudaSuccess) st = cuda_fail(ctx, e, "copy");
  }
  const double p_fac = c.thermal ? c.P_th0 / (R_GAS * c.rho_ref) : 0.0;
  if (st == LBM_OK) {
    cudaError_t e;
    const int cur = 0;
    if (ctx->f64)
      e = launch_set_fields<double, double>(ctx->D, ctx->geo, dT, dY, (int)K, dW, du, dP, dG,
                                            p_fac, c.P_ref, c.thermal, (double*)ctx->g[cur], (double*)ctx->T[cur],
                                            (double*)ctx->Y[cur], (double*)ctx->u, (double*)ctx->rho,
                                            (double*)ctx->lam, (double*)ctx->ph, ctx->st);
    else if (c.storage == LBM_STORE_F16)
      e = launch_set_fields<__half, float>(ctx->D, ctx->geo, dT, dY, (int)K, dW, du, dP, dG,
                                           p_fac, c.P_ref, c.thermal, (__half*)ctx->g[cur], (float*)ctx->T[cur],
                                           (float*)ctx->Y[cur], (float*)ctx->u, (float*)ctx->rho,
                                           (float*)ctx->lam, (float*)ctx->ph, ctx->st);
    else
      e = launch_set_fields<float, float>(ctx->D, ctx->geo, dT, dY, (int)K, dW, du, dP, dG,
                                          p_fac, c.P_ref, c.thermal, (float*)ctx->g[cur], (float*)ctx->T[cur],
                                          (float*)ctx->Y[cur], (float*)ctx->u, (float*)ctx->rho,
                                          (float*)ctx->lam, (float*)ctx->ph, ctx->st);
    if (e != cudaSuccess) st = cuda_fail(ctx, e, "set_fields kernel");
  }
  // the second buffer of each double-buffered field starts as a copy, so that cells a step
  // never writes (solid cells) hold defined values in both (saved states are then defined)
  if (st == LBM_OK) {
    cudaError_t e = cudaMemcpyAsync(ctx->g[1], ctx->g[0], Q * N * ctx->S, cudaMemcpyDeviceToDevice, ctx->st);
    if (e == cudaSuccess && c.thermal)
      e = cudaMemcpyAsync(ctx->T[1], ctx->T[0], N * ctx->F, cudaMemcpyDeviceToDevice, ctx->st);
    if (e == cudaSuccess && c.thermal)
      e = cudaMemcpyAsync(ctx->Y[1], ctx->Y[0], K * N * ctx->F, cudaMemcpyDeviceToDevice, ctx->st);
    if (e != cudaSuccess) st = cuda_fail(ctx, e, "copy fields");
  }
  // thermodynamic-pressure state: P = P_th0, M = P_th0 * I0 (same arithmetic as every step)
  PthState ps{};
  ps.P = c.P_th0;
  ps.fd_rho_d = c.thermal ? c.P_th0 / (R_GAS * c.rho_ref) : 0.0;
  ps.rho_in_d = c.P_th0 * ctx->pu.rin_fac;
  ps.fd_rho = (float)ps.fd_rho_d;
  ps.rho_in = (float)ps.rho_in_d;
  if (st == LBM_OK) {
    cudaError_t e = cudaMemcpyAsync(ctx->pth, &ps, sizeof(ps), cudaMemcpyHostToDevice, ctx->st);
    if (e != cudaSuccess) st = cuda_fail(ctx, e, "copy");
  }
  if (st == LBM_OK && c.thermal && c.closed_domain) {
    cudaError_t e = ctx->f64
        ? launch_init_integral<double>(ctx->geo, ctx->mask, (const double*)ctx->T[0], (const double*)ctx->Y[0],
                                       ctx->fdc_d, ctx->partials, ctx->nblocks_init, ctx->st)
        : launch_init_integral<float>(ctx->geo, ctx->mask, (const float*)ctx->T[0], (const float*)ctx->Y[0],
                                      ctx->fdc_f, ctx->partials, ctx->nblocks_init, ctx->st);
    if (e == cudaSuccess)
      e = launch_pth_update(ctx->pu, ctx->partials, ctx->nblocks_init, ctx->pth_stage, ctx->pth_counter, ctx->pth, 1,
                            ctx->st);
    if (e != cudaSuccess) st = cuda_fail(ctx, e, "initial integral");
  }
  cudaError_t e = cudaStreamSynchronize(ctx->st);
  if (st == LBM_OK && e != cudaSuccess) st = cuda_fail(ctx, e, "sync");
  // release the staging buffer
  for (size_t i = 0; i < ctx->allocs.size(); ++i)
    if (ctx->allocs[i] == buf) {
      ctx->allocs.erase(ctx->allocs.begin() + i);
      break;
    }
  if (ctx->cfg.free) ctx->cfg.free(buf, ctx->cfg.alloc_user);
  else cudaFree(buf);
  if (st != LBM_OK) return st;
  ctx->cur = 0;
  ctx->steps = 0;
  ctx->have_fields = true;
  ctx->floc_ok = false;
  CK(cudaMemsetAsync(ctx->flag, 0, 16, ctx->st), "memset");
  return LBM_OK;
}

lbm_status lbm_step(lbm_ctx* ctx, int n_steps) {
  if (!ctx) return LBM_ERR_ARG;
  if (n_steps < 0) return fail(ctx, LBM_ERR_ARG, "n_steps must be >= 0");
  if (!ctx->have_fields) return fail(ctx, LBM_ERR_STATE, "set_fields must come first");
  if (n_steps == 0) return LBM_OK;
  CK(cudaSetDevice(ctx->dev), "cudaSetDevice");
  if (ctx->cfg.thermal && ctx->cfg.flame_sensor && !ctx->floc_ok) {
    // F_loc of a state set from outside, before any graph is captured or replayed
    CK(timed(ctx, KIND_SENSOR, fd_thunk, ctx->cur, 1), "flame sensor");
    ctx->floc_ok = true;
  }
  if (ctx->st_on || ctx->pr_on) {
    // statistics and probes: direct launches; a sampled step also writes P_h, then the
    // accumulators update and the probe values are copied into the ring
    for (int k = 0; k < n_steps; ++k) {
      const bool sample = ctx->st_on && (ctx->steps + 1) % ctx->st_interval == 0;
      const bool probe = ctx->pr_on && (ctx->steps + 1) % ctx->pr_interval == 0;
      CK(enqueue_step(ctx, ctx->cur, sample || probe || k == n_steps - 1), "step launch");
      ctx->cur ^= 1;
      ++ctx->steps;
      if (probe) {
        const size_t row = (size_t)ctx->pr_n * ctx->pr_nf;
        double* dst = ctx->pr_ring + (size_t)(ctx->pr_count % ctx->pr_cap) * row;
        const int cur = ctx->cur;
        if (ctx->f64)
          CK(launch_probes<double>(ctx->pr_cells, ctx->pr_n, ctx->pr_nf, ctx->D, (int)ctx->N, (const double*)ctx->u,
                                   (const double*)ctx->ph, (const double*)ctx->T[cur], dst, ctx->st),
             "probes");
        else
          CK(launch_probes<float>(ctx->pr_cells, ctx->pr_n, ctx->pr_nf, ctx->D, (int)ctx->N, (const float*)ctx->u,
                                  (const float*)ctx->ph, (const float*)ctx->T[cur], dst, ctx->st),
             "probes");
        ++ctx->pr_count;
      }
      if (sample) {
        ++ctx->st_n;
        const int cur = ctx->cur;
        if (ctx->f64)
          CK(launch_stats<double>((int)ctx->N, ctx->st_nf, ctx->links, (const double*)ctx->u, ctx->D,
                                  (const double*)ctx->ph, (const double*)ctx->T[cur], ctx->st_n, ctx->st_mean,
                                  ctx->st_m2, ctx->st),
             "statistics");
        else
          CK(launch_stats<float>((int)ctx->N, ctx->st_nf, ctx->links, (const float*)ctx->u, ctx->D,
                                 (const float*)ctx->ph, (const float*)ctx->T[cur], ctx->st_n, ctx->st_mean,
                                 ctx->st_m2, ctx->st),
             "statistics");
      }
    }
    return LBM_OK;
  }
  int left = n_steps - 1;  // the last step also writes the output-only fields
  if (ctx->use_graphs && !ctx->prof) {
    while (left >= 2) {
      if (!ctx->gexec[ctx->cur]) CK(build_graph(ctx, ctx->cur), "graph capture");
      CK(cudaGraphLaunch(ctx->gexec[ctx->cur], ctx->st), "graph launch");
      left -= 2;
      ctx->steps += 2;
    }
  }
  while (left > 0) {
    CK(enqueue_step(ctx, ctx->cur, false), "step launch");
    ctx->cur ^= 1;
    --left;
    ++ctx->steps;
  }
  CK(enqueue_step(ctx, ctx->cur, true), "step launch");
  ctx->cur ^= 1;
  ++ctx->steps;
  return LBM_OK;
}

size_t lbm_fields_size(const lbm_ctx* ctx, unsigned bits) { return ctx ? fields_size(ctx, bits) : 0; }

lbm_status lbm_get_fields(lbm_ctx* ctx, unsigned bits, double* dst, int dst_on_device) {
  if (!ctx || !dst) return fail(ctx, LBM_ERR_ARG, "null argument");
  if (!ctx->have_fields) return fail(ctx, LBM_ERR_STATE, "no fields");
  if (!ctx->cfg.thermal && (bits & (LBM_F_T | LBM_F_Y | LBM_F_RHO | LBM_F_LAM)))
    return fail(ctx, LBM_ERR_ARG, "T, Y, rho, Lambda need a thermal run");
  if (bits & ~127u) return fail(ctx, LBM_ERR_ARG, "unknown field bits");
  CK(cudaSetDevice(ctx->dev), "cudaSetDevice");
  const size_t n = fields_size(ctx, bits);
  if (n == 0) return LBM_OK;
  double* out = dst;
  // pinned host memory is written in place through its device mapping; other host memory is
  // filled from a device scratch buffer
  double* view = dst_on_device ? dst : (double*)device_view(dst);
  const bool staged = view == nullptr;
  if (staged) {
    if (ctx->scratch_out_n < n) {
      double* p = (double*)dalloc(ctx, n * 8);
      if (!p) return fail(ctx, LBM_ERR_ALLOC, "allocation failed");
      ctx->scratch_out = p;
      ctx->scratch_out_n = n;
    }
    out = ctx->scratch_out;
  } else {
    out = view;
  }
  const int cur = ctx->cur;
  cudaError_t e;
  if (ctx->f64)
    e = launch_get_fields<double, double>(ctx->D, ctx->geo, bits, ctx->K, (const double*)ctx->g[cur],
                                          (const double*)ctx->T[cur], (const double*)ctx->Y[cur],
                                          (const double*)ctx->u, (const double*)ctx->ph, (const double*)ctx->rho,
                                          (const double*)ctx->lam, ctx->pth, ctx->cfg.P_ref, out, ctx->st);
  else if (ctx->cfg.storage == LBM_STORE_F16)
    e = launch_get_fields<__half, float>(ctx->D, ctx->geo, bits, ctx->K, (const __half*)ctx->g[cur],
                                         (const float*)ctx->T[cur], (const float*)ctx->Y[cur], (const float*)ctx->u,
                                         (const float*)ctx->ph, (const float*)ctx->rho, (const float*)ctx->lam,
                                         ctx->pth, ctx->cfg.P_ref, out, ctx->st);
  else
    e = launch_get_fields<float, float>(ctx->D, ctx->geo, bits, ctx->K, (const float*)ctx->g[cur],
                                        (const float*)ctx->T[cur], (const float*)ctx->Y[cur], (const float*)ctx->u,
                                        (const float*)ctx->ph, (const float*)ctx->rho, (const float*)ctx->lam,
                                        ctx->pth, ctx->cfg.P_ref, out, ctx->st);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "get_fields kernel");
  if (staged) CK(cudaMemcpyAsync(dst, out, n * 8, cudaMemcpyDeviceToHost, ctx->st), "copy out");
  int flag = 0;
  CK(cudaMemcpyAsync(&flag, ctx->flag, 4, cudaMemcpyDeviceToHost, ctx->st), "copy flag");
  CK(cudaStreamSynchronize(ctx->st), "sync");
  if (flag) {
    CK(cudaMemsetAsync(ctx->flag, 0, 4, ctx->st), "memset");
    if (flag & 4) return fail(ctx, LBM_ERR_TIMEOUT, "a plane load of the FD update did not arrive in time");
    return fail(ctx, LBM_ERR_NONFINITE, "a step produced a non-finite velocity");
  }
  return LBM_OK;
}

lbm_status lbm_get_scalars(lbm_ctx* ctx, double out[4]) {
  if (!ctx || !out) return fail(ctx, LBM_ERR_ARG, "null argument");
  if (!ctx->have_fields) return fail(ctx, LBM_ERR_STATE, "no fields");
  CK(cudaSetDevice(ctx->dev), "cudaSetDevice");
  PthState ps;
  CK(cudaMemcpyAsync(&ps, ctx->pth, sizeof(ps), cudaMemcpyDeviceToHost, ctx->st), "copy");
  CK(cudaStreamSynchronize(ctx->st), "sync");
  out[0] = ps.P;
  out[1] = ps.dP;
  out[2] = ps.M;
  out[3] = (double)ctx->steps;
  return LBM_OK;
}

lbm_status lbm_get_stencil_words(lbm_ctx* ctx, uint32_t* dst, int dst_on_device) {
  if (!ctx || !dst) return fail(ctx, LBM_ERR_ARG, "null argument");
  if (!ctx->have_geo) return fail(ctx, LBM_ERR_STATE, "no geometry");
  CK(cudaSetDevice(ctx->dev), "cudaSetDevice");
  CK(cudaMemcpyAsync(dst, ctx->sword, ctx->N * 4, dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                     ctx->st), "copy stencil words");
  CK(cudaStreamSynchronize(ctx->st), "sync");
  return LBM_OK;
}

lbm_status lbm_get_links(lbm_ctx* ctx, uint32_t* dst, int dst_on_device) {
  if (!ctx || !dst) return fail(ctx, LBM_ERR_ARG, "null argument");
  if (!ctx->have_geo) return fail(ctx, LBM_ERR_STATE, "no geometry");
  CK(cudaSetDevice(ctx->dev), "cudaSetDevice");
  CK(cudaMemcpyAsync(dst, ctx->links, ctx->N * 4, dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                     ctx->st), "copy links");
  CK(cudaStreamSynchronize(ctx->st), "sync");
  return LBM_OK;
}

size_t lbm_state_bytes(const lbm_ctx* ctx) {
  if (!ctx) return 0;
  const size_t N = ctx->N;
  size_t b = (size_t)ctx->Q * N * ctx->S + (size_t)ctx->D * N * ctx->F + sizeof(PthState);
  if (ctx->cfg.thermal) b += (1 + (size_t)ctx->K) * N * ctx->F;
  return b;
}

static lbm_status copy_state(lbm_ctx* ctx, char* dev, bool save) {
  if (!save) ctx->floc_ok = false;  // a new state: its F_loc is computed before the next step
  const size_t N = ctx->N;
  auto mv = [&](void* state, size_t bytes) -> cudaError_t {
    cudaError_t e = save ? cudaMemcpyAsync(dev, state, bytes, cudaMemcpyDeviceToDevice, ctx->st)
                         : cudaMemcpyAsync(state, dev, bytes, cudaMemcpyDeviceToDevice, ctx->st);
    dev += bytes;
    return e;
  };
  const int cur = ctx->cur;
  CK(mv(ctx->g[cur], (size_t)ctx->Q * N * ctx->S), "copy state");
  CK(mv(ctx->u, (size_t)ctx->D * N * ctx->F), "copy state");
  if (ctx->cfg.thermal) {
    CK(mv(ctx->T[cur], N * ctx->F), "copy state");
    CK(mv(ctx->Y[cur], (size_t)ctx->K * N * ctx->F), "copy state");
  }
  CK(mv(ctx->pth, sizeof(PthState)), "copy state");
  return LBM_OK;
}

lbm_status lbm_save_state(lbm_ctx* ctx, void* dst_device) {
  if (!ctx || !dst_device) return fail(ctx, LBM_ERR_ARG, "null argument");
  if (!ctx->have_fields) return fail(ctx, LBM_ERR_STATE, "no fields");
  CK(cudaSetDevice(ctx->dev), "cudaSetDevice");
  return copy_state(ctx, (char*)dst_device, true);
}

lbm_status lbm_load_state(lbm_ctx* ctx, const void* src_device) {
  if (!ctx || !src_device) return fail(ctx, LBM_ERR_ARG, "null argument");
  if (!ctx->have_fields) return fail(ctx, LBM_ERR_STATE, "set_fields must come first");
  CK(cudaSetDevice(ctx->dev), "cudaSetDevice");
  return copy_state(ctx, (char*)src_device, false);
}

lbm_status lbm_profile(lbm_ctx* ctx, int enable) {
  if (!ctx) return LBM_ERR_ARG;
  CK(cudaSetDevice(ctx->dev), "cudaSetDevice");
  CK(cudaStreamSynchronize(ctx->st), "sync");
  for (auto& e : ctx->ev_used) {
    ctx->ev_pool.push_back(e.second.first);
    ctx->ev_pool.push_back(e.second.second);
  }
  ctx->ev_used.clear();
  for (int k = 0; k < LBM_KERNEL_KINDS; ++k) {
    ctx->ms[k] = 0;
    ctx->cnt[k] = 0;
  }
  ctx->prof = enable != 0;
  return LBM_OK;
}

lbm_status lbm_kernel_times(lbm_ctx* ctx, double ms[LBM_KERNEL_KINDS], long long launches[LBM_KERNEL_KINDS]) {
  if (!ctx || !ms || !launches) return fail(ctx, LBM_ERR_ARG, "null argument");
  CK(cudaSetDevice(ctx->dev), "cudaSetDevice");
  CK(cudaStreamSynchronize(ctx->st), "sync");
  for (auto& e : ctx->ev_used) {
    float t = 0;
    CK(cudaEventElapsedTime(&t, e.second.first, e.second.second), "event time");
    ctx->ms[e.first] += t;
    ctx->cnt[e.first] += 1;
    ctx->ev_pool.push_back(e.second.first);
    ctx->ev_pool.push_back(e.second.second);
  }
  ctx->ev_used.clear();
  for (int k = 0; k < LBM_KERNEL_KINDS; ++k) {
    ms[k] = ctx->ms[k];
    launches[k] = ctx->cnt[k];
  }
  return LBM_OK;
}

lbm_status lbm_kernel_bytes(const lbm_ctx* ctx, double bytes[LBM_KERNEL_KINDS]) {
  if (!ctx || !bytes) return LBM_ERR_ARG;
  const double N = (double)ctx->N, Nf = (double)ctx->n_fluid, S = (double)ctx->S, F = (double)ctx->F;
  const double K = ctx->K, D = ctx->D, Q = ctx->Q;
  const bool th = ctx->cfg.thermal;
  // FD: read T, Y, u; write T, Y, rho, Lambda; stencil word per cell; with the sensor, read F_loc
  // of this state and write that of the next
  bytes[KIND_FD] = th ? Nf * ((2.0 * (1 + K) + D + 2.0 + (ctx->cfg.flame_sensor ? 2.0 : 0.0)) * F) + 4.0 * N : 0.0;
  bytes[KIND_SENSOR] = (th && ctx->cfg.flame_sensor) ? Nf * 4.0 * F + N : 0.0;
  bytes[KIND_PTH] = (th && ctx->cfg.closed_domain) ? 16.0 * fd_slots(ctx) : 0.0;
  // LB: populations read + written, link word, and (thermal) rho, Lambda, T read + u written
  bytes[KIND_LB] = Nf * (2.0 * Q * S + (th ? (3.0 + D) * F : 0.0)) + 4.0 * N;
  return LBM_OK;
}

}  // extern "C"

namespace {
size_t state_words(const lbm_ctx* c) {
  return ((size_t)c->Q + c->D + (c->cfg.thermal ? 1 + (size_t)c->K : 0)) * c->N;
}

// Scratch of the adjoint kernels plus one adjoint buffer, zero-filled once: the kernels never
// write solid-cell entries, which therefore stay zero.
template <typename R> lbm_status ensure_adj_ws(lbm_ctx* ctx, R** scratch, R** buf) {
  const size_t N = ctx->N;
  const size_t sw = adj_scratch_words<R>(N, ctx->K), bw = state_words(ctx);
  if (!ctx->adj_ws) {
    if (!(ctx->adj_ws = dalloc(ctx, (sw + bw) * sizeof(R))))
      return fail(ctx, LBM_ERR_ALLOC, "adjoint workspace allocation failed");
    CK(cudaMemsetAsync(ctx->adj_ws, 0, (sw + bw) * sizeof(R), ctx->st), "memset");
  }
  *scratch = (R*)ctx->adj_ws;
  *buf = *scratch + sw;
  return LBM_OK;
}

// Slot array i (0 or 1) of the adjoint scratch: the slot form of the T and Y adjoints, written by
// one reverse step and read by the next.
template <typename R> R* adj_slots(lbm_ctx* ctx, R* w, int i) {
  return w + (9 + (size_t)i * 9 * (ctx->K + 1)) * ctx->N;
}

template <typename R>
AdjBuffers<R> adj_buffers(lbm_ctx* ctx, R* w, const R* in, R* out, void* grad_inlet, const R* slots_in, R* slots) {
  const size_t N = ctx->N;
  AdjBuffers<R> b{};
  b.in = in;
  b.out = out;
  b.rho_own = w; w += N;
  b.lam_bar = w; w += N;
  b.T_lb = w; w += N;
  b.u_lb = w; w += 2 * N;
  b.rho_nb = w;
  b.slots_in = slots_in;
  b.slots = slots;
  b.inlet_bar = (R*)grad_inlet;
  return b;
}

// End of a reverse sweep: the T and Y adjoints from the slot form (slot array sp, when sp >= 0)
// into the adjoint buffer that holds the rest of it.
template <typename R> lbm_status adj_finish(lbm_ctx* ctx, R* scratch, int sp, R* adj_buf) {
  if (sp < 0) return LBM_OK;
  const size_t N = ctx->N;
  CK(launch_adjoint_gather<R>(ctx->geo, ctx->sword, ctx->K, adj_slots<R>(ctx, scratch, sp), adj_buf + 11 * N,
                              adj_buf + 12 * N, ctx->st),
     "adjoint gather");
  return LBM_OK;
}

template <typename R> lbm_status adjoint_step_impl(lbm_ctx* ctx, const void* state_n, void* adj, void* grad_inlet) {
  const bool th = ctx->cfg.thermal != 0;
  R *scratch, *buf;
  lbm_status st = ensure_adj_ws<R>(ctx, &scratch, &buf);
  if (st != LBM_OK) return st;
  if ((st = lbm_load_state(ctx, state_n)) != LBM_OK) return st;
  const int cur = ctx->cur;
  if (th) CK(run_fd(ctx, cur, false), "forward FD for the adjoint");  // rho^n, Lambda^n
  const AdjBuffers<R> b =
      adj_buffers<R>(ctx, scratch, (const R*)adj, buf, grad_inlet, nullptr, adj_slots<R>(ctx, scratch, 0));
  CK(launch_adjoint_step2d<R>(b, make_lb_args<R>(ctx, cur, false), make_fd_args<R>(ctx, cur), th, false, ctx->st),
     "adjoint kernels");
  if ((st = adj_finish<R>(ctx, scratch, th ? 0 : -1, buf)) != LBM_OK) return st;
  CK(cudaMemcpyAsync(adj, buf, state_words(ctx) * sizeof(R), cudaMemcpyDeviceToDevice, ctx->st), "copy adjoint");
  return LBM_OK;
}

// Segment workspace: slot k holds state k (k >= 1; state 0 is the checkpoint) then rho^k,
// Lambda^k. Grown to at least `slots` slots; the old block stays with the context's allocations
// until lbm_destroy.
template <typename R> lbm_status ensure_seg_ws(lbm_ctx* ctx, int slots, size_t slot_w) {
  if (slots > ctx->seg_cap) {
    if (!(ctx->seg_ws = dalloc(ctx, (size_t)slots * slot_w * sizeof(R))))
      return fail(ctx, LBM_ERR_ALLOC, "adjoint segment workspace allocation failed");
    ctx->seg_cap = slots;
  }
  return LBM_OK;
}

// Recompute of one segment on stream st: n steps from the checkpoint, state k + 1 written straight
// into slot k + 1 of ws, rho^k, Lambda^k into slot k; the last step needs its FD pass only (its
// state outputs go to the context's spare buffers, which nothing reads).
template <typename R>
lbm_status seg_recompute(lbm_ctx* ctx, const void* checkpoint, int n, R* ws, cudaStream_t st) {
  const size_t N = ctx->N;
  const bool th = ctx->cfg.thermal != 0;
  const size_t sw = state_words(ctx), slot_w = sw + (th ? 2 * N : 0);
  auto state_of = [&](int k) -> R* { return k == 0 ? (R*)checkpoint : ws + (size_t)k * slot_w; };
  auto rho_of = [&](int k) -> R* { return ws + (size_t)k * slot_w + sw; };
  const int other = 1 - ctx->cur;
  const bool hi1 = ctx->cfg.omega_hi[0] == 1.0 && ctx->cfg.omega_hi[1] == 1.0 && ctx->cfg.omega_hi[2] == 1.0 &&
                   ctx->cfg.omega_hi[3] == 1.0;
  const int co = hi1 ? COLL_CUMULANT_FULL : COLL_CUMULANT;
  for (int k = 0; k < n; ++k) {
    R* sk = state_of(k);
    const bool last = k + 1 == n;
    R* sk1 = last ? nullptr : state_of(k + 1);
    if (th) {
      FDArgs<R> fdf = make_fd_args<R>(ctx, ctx->cur);
      fdf.T = sk + 11 * N;
      fdf.Y = sk + 12 * N;
      fdf.u = sk + 9 * N;
      fdf.T_out = last ? (R*)ctx->T[other] : sk1 + 11 * N;
      fdf.Y_out = last ? (R*)ctx->Y[other] : sk1 + 12 * N;
      fdf.rho_out = rho_of(k);
      fdf.lam_out = rho_of(k) + N;
      CK((launch_fd<2, R>(fdf, st, false)), "segment recompute (FD)");
    }
    if (!last) {
      LBArgs<R> lbf = make_lb_args<R>(ctx, ctx->cur, false);
      lbf.g_in = sk;
      lbf.g_out = sk1;
      lbf.u_in = sk + 9 * N;
      lbf.u = sk1 + 9 * N;
      if (th) {
        lbf.rho = rho_of(k);
        lbf.lam = rho_of(k) + N;
        lbf.T = sk + 11 * N;
      } else {
        // isothermal: the step writes u at outlet cells only; carry the rest over
        CK(cudaMemcpyAsync(sk1 + 9 * N, sk + 9 * N, 2 * N * sizeof(R), cudaMemcpyDeviceToDevice, st),
           "segment recompute (u)");
      }
      CK((launch_lb<2, R, R>(lbf, th ? 1 : 0, co, st)), "segment recompute (LB)");
    }
  }
  return LBM_OK;
}

// Reverse of one recomputed segment on stream st: the adjoint step over the states n - 1 .. 0,
// read in place, alternating between the two buffers pp[0], pp[1]; *which selects the one that
// holds the incoming adjoint and, on return, the one that holds the adjoint of the segment's
// first state. *sp: slot array holding the T and Y adjoints of the incoming state in slot form,
// or -1 when they are in pp[*which]; on return, the slot array of the segment's first state.
template <typename R>
lbm_status seg_reverse(lbm_ctx* ctx, const void* checkpoint, int n, R* ws, R* scratch, R* const pp[2], int* which,
                       int* sp, void* grad_inlet, cudaStream_t st) {
  const size_t N = ctx->N;
  const bool th = ctx->cfg.thermal != 0;
  const size_t sw = state_words(ctx), slot_w = sw + (th ? 2 * N : 0);
  auto state_of = [&](int k) -> R* { return k == 0 ? (R*)checkpoint : ws + (size_t)k * slot_w; };
  auto rho_of = [&](int k) -> R* { return ws + (size_t)k * slot_w + sw; };
  for (int k = n - 1; k >= 0; --k) {
    R* sk = state_of(k);
    LBArgs<R> lbf = make_lb_args<R>(ctx, ctx->cur, false);
    lbf.g_in = sk;
    lbf.u = sk + 9 * N;
    lbf.u_in = lbf.u;
    FDArgs<R> fdf = make_fd_args<R>(ctx, ctx->cur);
    fdf.u = sk + 9 * N;
    if (th) {
      lbf.T = sk + 11 * N;
      lbf.rho = rho_of(k);
      lbf.lam = rho_of(k) + N;
      fdf.T = sk + 11 * N;
      fdf.Y = sk + 12 * N;
    }
    const int so = *sp >= 0 ? 1 - *sp : 0;
    const AdjBuffers<R> b = adj_buffers<R>(ctx, scratch, pp[*which], pp[1 - *which], grad_inlet,
                                           *sp >= 0 ? adj_slots<R>(ctx, scratch, *sp) : nullptr,
                                           adj_slots<R>(ctx, scratch, so));
    // within a segment, each LB adjoint follows the previous step's FD adjoint directly
    CK(launch_adjoint_step2d<R>(b, lbf, fdf, th, th && k < n - 1, st), "adjoint kernels");
    *which ^= 1;
    if (th) *sp = so;
  }
  return LBM_OK;
}

// Reverse sweep over one checkpoint segment: recompute then reverse, on the context's stream.
// The context's current state is not touched.
template <typename R>
lbm_status adjoint_segment_impl(lbm_ctx* ctx, const void* checkpoint, int n, void* adj, void* grad_inlet) {
  const size_t N = ctx->N;
  const bool th = ctx->cfg.thermal != 0;
  R *scratch, *buf;
  lbm_status st = ensure_adj_ws<R>(ctx, &scratch, &buf);
  if (st != LBM_OK) return st;
  const size_t sw = state_words(ctx), slot_w = sw + (th ? 2 * N : 0);
  if ((st = ensure_seg_ws<R>(ctx, n, slot_w)) != LBM_OK) return st;
  R* ws = (R*)ctx->seg_ws;
  // thermodynamic-pressure state of the checkpoint (constant in the supported open domain)
  CK(cudaMemcpyAsync(ctx->pth, (const char*)checkpoint + sw * sizeof(R), sizeof(PthState),
                     cudaMemcpyDeviceToDevice, ctx->st), "load P_th state");
  if ((st = seg_recompute<R>(ctx, checkpoint, n, ws, ctx->st)) != LBM_OK) return st;
  CK(launch_zero_solid_pops<R>(ctx->geo, ctx->links, (R*)adj, ctx->st), "zero solid adjoint");
  R* const pp[2] = {(R*)adj, buf};
  int which = 0, sp = -1;
  if ((st = seg_reverse<R>(ctx, checkpoint, n, ws, scratch, pp, &which, &sp, grad_inlet, ctx->st)) != LBM_OK)
    return st;
  if ((st = adj_finish<R>(ctx, scratch, sp, pp[which])) != LBM_OK) return st;
  if (which != 0)
    CK(cudaMemcpyAsync(adj, buf, sw * sizeof(R), cudaMemcpyDeviceToDevice, ctx->st), "copy adjoint");
  return LBM_OK;
}

// Whole-run sweep: segment s covers steps [s C, min((s + 1) C, K)). The recompute of segment s - 1
// runs on a second stream into the other half of a two-segment workspace while segment s is
// reversed on the context's stream; events order each half's reuse. Same kernels and arithmetic
// as lbm_adjoint_segment segment by segment, so the results are identical.
template <typename R>
lbm_status adjoint_sweep_impl(lbm_ctx* ctx, const void* const* ckpt, int S, int C, int K, void* adj,
                              void* grad_inlet) {
  const size_t N = ctx->N;
  const bool th = ctx->cfg.thermal != 0;
  R *scratch, *buf;
  lbm_status st = ensure_adj_ws<R>(ctx, &scratch, &buf);
  if (st != LBM_OK) return st;
  const size_t sw = state_words(ctx), slot_w = sw + (th ? 2 * N : 0);
  if ((st = ensure_seg_ws<R>(ctx, 2 * C, slot_w)) != LBM_OK) return st;
  if (!ctx->st2) CK(cudaStreamCreateWithFlags(&ctx->st2, cudaStreamNonBlocking), "cudaStreamCreate");
  for (auto& e : ctx->sw_ev)
    if (!e) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "cudaEventCreate");
  cudaEvent_t start = ctx->sw_ev[0], rec[2] = {ctx->sw_ev[1], ctx->sw_ev[2]}, rev[2] = {ctx->sw_ev[3], ctx->sw_ev[4]};
  R* half[2] = {(R*)ctx->seg_ws, (R*)ctx->seg_ws + (size_t)C * slot_w};
  auto len = [&](int s) { return (s + 1) * C <= K ? C : K - s * C; };
  // P_th state (the same in every checkpoint of the supported open domain) and the solid-cell
  // entries of the incoming adjoint, then the second stream joins
  CK(cudaMemcpyAsync(ctx->pth, (const char*)ckpt[0] + sw * sizeof(R), sizeof(PthState), cudaMemcpyDeviceToDevice,
                     ctx->st), "load P_th state");
  CK(launch_zero_solid_pops<R>(ctx->geo, ctx->links, (R*)adj, ctx->st), "zero solid adjoint");
  CK(cudaEventRecord(start, ctx->st), "event");
  CK(cudaStreamWaitEvent(ctx->st2, start, 0), "event wait");
  if ((st = seg_recompute<R>(ctx, ckpt[S - 1], len(S - 1), half[(S - 1) & 1], ctx->st2)) != LBM_OK) return st;
  CK(cudaEventRecord(rec[(S - 1) & 1], ctx->st2), "event");
  R* const pp[2] = {(R*)adj, buf};
  int which = 0, sp = -1;
  for (int s = S - 1; s >= 0; --s) {
    if (s >= 1) {
      // the half of segment s - 1 was last read by the reverse of segment s + 1
      if (s + 1 <= S - 1) CK(cudaStreamWaitEvent(ctx->st2, rev[(s + 1) & 1], 0), "event wait");
      if ((st = seg_recompute<R>(ctx, ckpt[s - 1], len(s - 1), half[(s - 1) & 1], ctx->st2)) != LBM_OK) return st;
      CK(cudaEventRecord(rec[(s - 1) & 1], ctx->st2), "event");
    }
    CK(cudaStreamWaitEvent(ctx->st, rec[s & 1], 0), "event wait");
    if ((st = seg_reverse<R>(ctx, ckpt[s], len(s), half[s & 1], scratch, pp, &which, &sp, grad_inlet, ctx->st)) !=
        LBM_OK)
      return st;
    CK(cudaEventRecord(rev[s & 1], ctx->st), "event");
  }
  if ((st = adj_finish<R>(ctx, scratch, sp, pp[which])) != LBM_OK) return st;
  if (which != 0)
    CK(cudaMemcpyAsync(adj, buf, sw * sizeof(R), cudaMemcpyDeviceToDevice, ctx->st), "copy adjoint");
  return LBM_OK;
}

template <typename R> lbm_status fuel_objective_impl(lbm_ctx* ctx, int fuel, double* J, void* adj_out) {
  const size_t N = ctx->N;
  const int nb = (int)((N + FD_BLOCK - 1) / FD_BLOCK);
  if (!ctx->obj_partials && !(ctx->obj_partials = (double*)dalloc(ctx, (size_t)nb * sizeof(double))))
    return fail(ctx, LBM_ERR_ALLOC, "allocation failed");
  R* o = (R*)adj_out;
  CK(cudaMemsetAsync(o, 0, 11 * N * sizeof(R), ctx->st), "memset");
  const FDArgs<R> fdf = make_fd_args<R>(ctx, ctx->cur);
  CK(launch_fuel_objective<R>(fdf, fuel, o + 11 * N, o + 12 * N, ctx->obj_partials, nb, ctx->st), "objective");
  std::vector<double> h(nb);
  CK(cudaMemcpyAsync(h.data(), ctx->obj_partials, nb * sizeof(double), cudaMemcpyDeviceToHost, ctx->st), "copy");
  CK(cudaStreamSynchronize(ctx->st), "sync");
  double s = 0.0;
  for (double v : h) s += v;
  *J = s;
  return LBM_OK;
}

template <typename R> lbm_status initial_T_adjoint_impl(lbm_ctx* ctx, const void* state0, const void* adj0, void* gT) {
  lbm_status st = lbm_load_state(ctx, state0);
  if (st != LBM_OK) return st;
  const FDArgs<R> fdf = make_fd_args<R>(ctx, ctx->cur);
  CK(launch_initial_T_adjoint<R>(fdf, (const R*)adj0, (R*)gT, ctx->st), "initial-temperature adjoint");
  return LBM_OK;
}

// Ghost-point weights of the FD update from the interpolated-wall rows (cells, Q fractions each,
// the half-way fallback already applied): for a fluid cell whose distance-1 point along axis a on
// side s is a wall or solid (stencil kind 1), whose opposite distance-1 point is fluid and whose
// link toward that wall (pull direction c = -s e_a) has fraction q, w = (1 - 2q) / (1 + 2q); the
// fluid cell on the opposite side gets the same weight for its distance-2 wall point. Flags the
// stencil words of the cells with weights (SW_WALL) and uploads the rows.
template <typename R> lbm_status set_fd_walls(lbm_ctx* ctx, const std::vector<int>& cells, const std::vector<R>& rows) {
  const size_t N = ctx->N;
  const int D = ctx->D, Q = ctx->Q;
  const Geo& g = ctx->geo;
  std::vector<uint32_t> sw(N);
  CK(cudaMemcpyAsync(sw.data(), ctx->sword, N * 4, cudaMemcpyDeviceToHost, ctx->st), "copy stencil words");
  CK(cudaStreamSynchronize(ctx->st), "sync");
  for (size_t r = 0; r < N; ++r) sw[r] &= ~SW_WALL;
  std::vector<int> frow(N, -1);
  std::vector<R> w;
  const int W = 4 * D;
  auto row_for = [&](int r) -> R* {
    if (frow[r] < 0) {
      frow[r] = (int)(w.size() / W);
      w.insert(w.end(), W, R(0));
    }
    return w.data() + (size_t)frow[r] * W;
  };
  const int dims[3] = {g.nx, g.ny, g.nz};
  const int strides[3] = {1, g.nx, g.nx * g.ny};
  for (size_t k = 0; k < cells.size(); ++k) {
    const int r = cells[k];
    const uint32_t word = sw[r];
    const int pos[3] = {r % g.nx, (r / g.nx) % g.ny, r / (g.nx * g.ny)};
    for (int ax = 0; ax < D; ++ax)
      for (int sd = 0; sd < 2; ++sd) {
        const int k1 = (int)((word >> (4 * (2 * ax + sd))) & 3u);
        const int ko = (int)((word >> (4 * (2 * ax + 1 - sd))) & 3u);
        if (k1 != NB_SOLID || ko != NB_FLUID) continue;
        int c[3] = {0, 0, 0};
        c[ax] = sd ? -1 : 1;  // pull direction whose source is the wall point
        const int i = (c[0] + 1) + 3 * (c[1] + 1) + (D == 3 ? 9 * (c[2] + 1) : 0);
        const double q = (double)rows[k * Q + i];
        if (q == 0.5) continue;
        const R wv = (R)((1.0 - 2.0 * q) / (1.0 + 2.0 * q));
        row_for(r)[2 * ax + sd] = wv;
        // the opposite fluid point (periodic wrap as in the stencil) sees this wall at distance 2
        int po = pos[ax] + (sd ? -1 : 1);
        po = po < 0 ? po + dims[ax] : (po >= dims[ax] ? po - dims[ax] : po);
        const int ro = r + (po - pos[ax]) * strides[ax];
        const uint32_t wo = sw[ro];
        if (((wo >> (4 * (2 * ax + sd))) & 15u) == (uint32_t)(NB_FLUID | (1 << 2))) row_for(ro)[2 * D + 2 * ax + sd] = wv;
      }
  }
  const size_t nr = w.size() / W;
  if (nr > 0 && ctx->fdc_d.mixavg)
    return fail(ctx, LBM_ERR_UNSUPPORTED, "ghost-point (curved) walls with mixture-averaged diffusion");
  ctx->n_fd_wall_rows = nr;
  if (nr > 0) {
    if (!ctx->fd_row && !(ctx->fd_row = (int*)dalloc(ctx, N * sizeof(int))))
      return fail(ctx, LBM_ERR_ALLOC, "allocation failed");
    if (nr > ctx->fd_rows_cap) {
      if (!(ctx->fd_w = dalloc(ctx, nr * W * sizeof(R)))) return fail(ctx, LBM_ERR_ALLOC, "allocation failed");
      ctx->fd_rows_cap = nr;
    }
    std::vector<int> list;
    list.reserve(nr);
    for (size_t r = 0; r < N; ++r)
      if (frow[r] >= 0) {
        sw[r] |= SW_WALL;
        list.push_back((int)r);
      }
    if (list.size() > ctx->fd_wall_list_cap) {
      if (!(ctx->fd_wall_list = (int*)dalloc(ctx, list.size() * sizeof(int))))
        return fail(ctx, LBM_ERR_ALLOC, "allocation failed");
      ctx->fd_wall_list_cap = list.size();
    }
    CK(cudaMemcpyAsync(ctx->fd_wall_list, list.data(), list.size() * sizeof(int), cudaMemcpyHostToDevice, ctx->st),
       "copy wall list");
    CK(cudaMemcpyAsync(ctx->fd_row, frow.data(), N * sizeof(int), cudaMemcpyHostToDevice, ctx->st), "copy rows");
    CK(cudaMemcpyAsync(ctx->fd_w, w.data(), nr * W * sizeof(R), cudaMemcpyHostToDevice, ctx->st), "copy weights");
  }
  CK(cudaMemcpyAsync(ctx->sword, sw.data(), N * 4, cudaMemcpyHostToDevice, ctx->st), "copy stencil words");
  CK(cudaStreamSynchronize(ctx->st), "sync");
  return LBM_OK;
}

// Build the interpolated-wall table from a list of links (cell, pull direction, fraction);
// later entries for the same link replace earlier ones.
template <typename R>
lbm_status set_wall_impl(lbm_ctx* ctx, long long n_links, const int* cell, const int* dir, const double* q) {
  const size_t N = ctx->N;
  const int Q = ctx->Q;
  const Geo& g = ctx->geo;
  std::vector<uint32_t> lw(N);
  CK(cudaMemcpyAsync(lw.data(), ctx->links, N * 4, cudaMemcpyDeviceToHost, ctx->st), "copy links");
  CK(cudaStreamSynchronize(ctx->st), "sync");
  for (size_t r = 0; r < N; ++r) lw[r] &= ~LINK_WALL;
  std::vector<int> row_of(N, -1);
  std::vector<R> rows;
  std::vector<int> cells;
  for (long long k = 0; k < n_links; ++k) {
    const int r = cell[k], i = dir[k];
    if (r < 0 || (size_t)r >= N || i < 0 || i >= Q) return fail(ctx, LBM_ERR_ARG, "wall link out of range");
    const double v = q[k];
    const uint32_t w = lw[r];
    if (!(w >> 31) || !((w >> i) & 1u) || !(v > 0.0 && v <= 1.0)) continue;
    const int x = r % g.nx;
    if ((x == 0 && g.bc_lo[0] == BC_INLET && cx(i) == 1) || (x == g.nx - 1 && g.bc_hi[0] == BC_OUTLET && cx(i) == -1))
      continue;
    R f = (R)v;
    // f < 1/2 needs r + c_i as a fluid pull source of the opposite direction
    if (f < R(0.5) && ((w >> (Q - 1 - i)) & 1u)) f = R(0.5);
    if (row_of[r] < 0) {
      if (f == R(0.5)) continue;
      row_of[r] = (int)cells.size();
      cells.push_back(r);
      rows.insert(rows.end(), Q, R(0.5));
    }
    rows[(size_t)row_of[r] * Q + i] = f;
  }
  const size_t n = cells.size();
  if (n > 0) {
    // list (and table rows) in cell order, so that the wall-list launch reads coalesced
    std::vector<size_t> order(n);
    for (size_t k = 0; k < n; ++k) order[k] = k;
    std::sort(order.begin(), order.end(), [&](size_t a, size_t b) { return cells[a] < cells[b]; });
    std::vector<int> sc(n);
    std::vector<R> sr(n * Q);
    for (size_t k = 0; k < n; ++k) {
      sc[k] = cells[order[k]];
      std::copy(rows.begin() + order[k] * Q, rows.begin() + (order[k] + 1) * Q, sr.begin() + k * Q);
    }
    cells.swap(sc);
    rows.swap(sr);
    if (n > ctx->wall_rows_cap) {
      // grow: the old blocks stay with the context's allocations until lbm_destroy
      if (!(ctx->wall_q = dalloc(ctx, n * Q * sizeof(R))) || !(ctx->wall_cells = (int*)dalloc(ctx, n * sizeof(int))))
        return fail(ctx, LBM_ERR_ALLOC, "wall table allocation failed");
      ctx->wall_rows_cap = n;
    }
    for (size_t k = 0; k < n; ++k) lw[cells[k]] |= LINK_WALL;
    CK(cudaMemcpyAsync(ctx->wall_cells, cells.data(), n * sizeof(int), cudaMemcpyHostToDevice, ctx->st), "copy wall list");
    CK(cudaMemcpyAsync(ctx->wall_q, rows.data(), n * Q * sizeof(R), cudaMemcpyHostToDevice, ctx->st), "copy wall table");
  }
  {
    lbm_status s2 = set_fd_walls<R>(ctx, cells, rows);
    if (s2 != LBM_OK) return s2;
  }
  CK(cudaMemcpyAsync(ctx->links, lw.data(), N * 4, cudaMemcpyHostToDevice, ctx->st), "copy links");
  CK(cudaStreamSynchronize(ctx->st), "sync");
  ctx->n_wall = n;
  drop_graphs(ctx);
  return LBM_OK;
}

lbm_status adjoint_supported(lbm_ctx* ctx) {
  const lbm_config& c = ctx->cfg;
  const bool hi1 = c.omega_hi[0] == 1.0 && c.omega_hi[1] == 1.0;
  if (c.dim != 2 || c.storage == LBM_STORE_F16 || c.collision != LBM_COLL_CUMULANT || !hi1 || c.closed_domain ||
      c.flame_sensor || ctx->n_wall > 0 || ctx->fdc_d.varcp || ctx->fdc_d.mixavg)
    return fail(ctx, LBM_ERR_UNSUPPORTED,
                "adjoint: 2-D, FP32/FP64 storage, cumulant collision with default higher-order rates, open domain, "
                "no flame sensor, half-way walls, constant heat capacity, constant Lewis numbers");
  return LBM_OK;
}
}  // namespace

extern "C" {

lbm_status lbm_adjoint_step(lbm_ctx* ctx, const void* state_n, void* adj, void* grad_inlet) {
  if (!ctx || !state_n || !adj || !grad_inlet) return fail(ctx, LBM_ERR_ARG, "null argument");
  if (!ctx->have_fields) return fail(ctx, LBM_ERR_STATE, "set_fields must come first");
  lbm_status s = adjoint_supported(ctx);
  if (s != LBM_OK) return s;
  CK(cudaSetDevice(ctx->dev), "cudaSetDevice");
  return ctx->f64 ? adjoint_step_impl<double>(ctx, state_n, adj, grad_inlet)
                  : adjoint_step_impl<float>(ctx, state_n, adj, grad_inlet);
}

lbm_status lbm_fuel_objective(lbm_ctx* ctx, int fuel_species, double* J, void* adj_out) {
  if (!ctx || !J || !adj_out) return fail(ctx, LBM_ERR_ARG, "null argument");
  if (!ctx->have_fields) return fail(ctx, LBM_ERR_STATE, "set_fields must come first");
  if (!ctx->cfg.thermal || fuel_species < 0 || fuel_species >= ctx->K)
    return fail(ctx, LBM_ERR_ARG, "objective needs a thermal run and a valid fuel index");
  lbm_status s = adjoint_supported(ctx);
  if (s != LBM_OK) return s;
  CK(cudaSetDevice(ctx->dev), "cudaSetDevice");
  return ctx->f64 ? fuel_objective_impl<double>(ctx, fuel_species, J, adj_out)
                  : fuel_objective_impl<float>(ctx, fuel_species, J, adj_out);
}

lbm_status lbm_adjoint_sweep(lbm_ctx* ctx, const void* const* checkpoints, int n_segments, int seg_len, int n_steps,
                             void* adj, void* grad_inlet) {
  if (!ctx || !checkpoints || !adj || !grad_inlet) return fail(ctx, LBM_ERR_ARG, "null argument");
  if (n_segments < 1 || seg_len < 1 || n_steps <= (long long)(n_segments - 1) * seg_len ||
      n_steps > (long long)n_segments * seg_len)
    return fail(ctx, LBM_ERR_ARG, "need (n_segments - 1) * seg_len < n_steps <= n_segments * seg_len");
  for (int s = 0; s < n_segments; ++s)
    if (!checkpoints[s]) return fail(ctx, LBM_ERR_ARG, "null checkpoint");
  if (!ctx->have_fields) return fail(ctx, LBM_ERR_STATE, "set_fields must come first");
  lbm_status s = adjoint_supported(ctx);
  if (s != LBM_OK) return s;
  CK(cudaSetDevice(ctx->dev), "cudaSetDevice");
  return ctx->f64 ? adjoint_sweep_impl<double>(ctx, checkpoints, n_segments, seg_len, n_steps, adj, grad_inlet)
                  : adjoint_sweep_impl<float>(ctx, checkpoints, n_segments, seg_len, n_steps, adj, grad_inlet);
}

lbm_status lbm_adjoint_segment(lbm_ctx* ctx, const void* checkpoint, int n_steps, void* adj, void* grad_inlet) {
  if (!ctx || !checkpoint || !adj || !grad_inlet) return fail(ctx, LBM_ERR_ARG, "null argument");
  if (n_steps < 1) return fail(ctx, LBM_ERR_ARG, "n_steps must be >= 1");
  if (!ctx->have_fields) return fail(ctx, LBM_ERR_STATE, "set_fields must come first");
  lbm_status s = adjoint_supported(ctx);
  if (s != LBM_OK) return s;
  CK(cudaSetDevice(ctx->dev), "cudaSetDevice");
  return ctx->f64 ? adjoint_segment_impl<double>(ctx, checkpoint, n_steps, adj, grad_inlet)
                  : adjoint_segment_impl<float>(ctx, checkpoint, n_steps, adj, grad_inlet);
}

lbm_status lbm_initial_T_adjoint(lbm_ctx* ctx, const void* state0, const void* adj0, void* grad_T0) {
  if (!ctx || !state0 || !adj0 || !grad_T0) return fail(ctx, LBM_ERR_ARG, "null argument");
  if (!ctx->have_fields) return fail(ctx, LBM_ERR_STATE, "set_fields must come first");
  if (!ctx->cfg.thermal) return fail(ctx, LBM_ERR_ARG, "initial-temperature adjoint needs a thermal run");
  lbm_status s = adjoint_supported(ctx);
  if (s != LBM_OK) return s;
  CK(cudaSetDevice(ctx->dev), "cudaSetDevice");
  return ctx->f64 ? initial_T_adjoint_impl<double>(ctx, state0, adj0, grad_T0)
                  : initial_T_adjoint_impl<float>(ctx, state0, adj0, grad_T0);
}

lbm_status lbm_set_wall_links(lbm_ctx* ctx, long long n_links, const int* cell, const int* dir, const double* q) {
  if (!ctx) return LBM_ERR_ARG;
  if (!ctx->have_geo) return fail(ctx, LBM_ERR_STATE, "set_geometry must come first");
  if (n_links < 0 || (n_links > 0 && (!cell || !dir || !q))) return fail(ctx, LBM_ERR_ARG, "null argument");
  if (n_links > 0 && ctx->fdc_d.mixavg)
    return fail(ctx, LBM_ERR_UNSUPPORTED, "interpolated walls with mixture-averaged diffusion");
  CK(cudaSetDevice(ctx->dev), "cudaSetDevice");
  return ctx->f64 ? set_wall_impl<double>(ctx, n_links, cell, dir, q)
                  : set_wall_impl<float>(ctx, n_links, cell, dir, q);
}

lbm_status lbm_set_wall_fractions(lbm_ctx* ctx, const double* q) {
  if (!ctx) return LBM_ERR_ARG;
  if (!ctx->have_geo) return fail(ctx, LBM_ERR_STATE, "set_geometry must come first");
  std::vector<int> cell, dir;
  std::vector<double> val;
  if (q) {
    for (int i = 0; i < ctx->Q; ++i)
      for (size_t r = 0; r < ctx->N; ++r) {
        const double v = q[(size_t)i * ctx->N + r];
        if (v > 0.0 && v <= 1.0 && v != 0.5) {
          cell.push_back((int)r);
          dir.push_back(i);
          val.push_back(v);
        }
      }
  }
  return lbm_set_wall_links(ctx, (long long)cell.size(), cell.data(), dir.data(), val.data());
}

lbm_status lbm_stats_control(lbm_ctx* ctx, int op, int interval) {
  if (!ctx) return LBM_ERR_ARG;
  if (op < 0 || op > 2 || (op == 1 && interval < 1)) return fail(ctx, LBM_ERR_ARG, "op 0|1|2, interval >= 1");
  if (!ctx->have_geo) return fail(ctx, LBM_ERR_STATE, "set_geometry must come first");
  CK(cudaSetDevice(ctx->dev), "cudaSetDevice");
  const int nf = ctx->D + 1 + (ctx->cfg.thermal ? 1 : 0);
  if (!ctx->st_mean) {
    if (!(ctx->st_mean = (float*)dalloc(ctx, (size_t)nf * ctx->N * sizeof(float))) ||
        !(ctx->st_m2 = (float*)dalloc(ctx, (size_t)nf * ctx->N * sizeof(float))))
      return fail(ctx, LBM_ERR_ALLOC, "statistics allocation failed");
    ctx->st_nf = nf;
    CK(cudaMemsetAsync(ctx->st_mean, 0, (size_t)nf * ctx->N * sizeof(float), ctx->st), "memset");
    CK(cudaMemsetAsync(ctx->st_m2, 0, (size_t)nf * ctx->N * sizeof(float), ctx->st), "memset");
  }
  if (op == 0) {
    CK(cudaMemsetAsync(ctx->st_mean, 0, (size_t)nf * ctx->N * sizeof(float), ctx->st), "memset");
    CK(cudaMemsetAsync(ctx->st_m2, 0, (size_t)nf * ctx->N * sizeof(float), ctx->st), "memset");
    ctx->st_n = 0;
  } else if (op == 1) {
    ctx->st_on = true;
    ctx->st_interval = interval;
  } else {
    ctx->st_on = false;
  }
  return LBM_OK;
}

lbm_status lbm_get_stats(lbm_ctx* ctx, double* dst, int dst_on_device, long long* n_samples) {
  if (!ctx || !dst) return fail(ctx, LBM_ERR_ARG, "null argument");
  if (!ctx->st_mean) return fail(ctx, LBM_ERR_STATE, "statistics were never started");
  CK(cudaSetDevice(ctx->dev), "cudaSetDevice");
  const size_t n = 2 * (size_t)ctx->st_nf * ctx->N;
  double* out = dst;
  if (!dst_on_device) {
    if (ctx->scratch_out_n < n) {
      if (!(ctx->scratch_out = (double*)dalloc(ctx, n * sizeof(double))))
        return fail(ctx, LBM_ERR_ALLOC, "allocation failed");
      ctx->scratch_out_n = n;
    }
    out = ctx->scratch_out;
  }
  CK(launch_stats_finalize((int)ctx->N, ctx->st_nf, ctx->links, ctx->st_mean, ctx->st_m2, ctx->st_n, out, ctx->st),
     "statistics");
  if (!dst_on_device) {
    CK(cudaMemcpyAsync(dst, out, n * sizeof(double), cudaMemcpyDeviceToHost, ctx->st), "copy statistics");
    CK(cudaStreamSynchronize(ctx->st), "sync");
  }
  if (n_samples) *n_samples = ctx->st_n;
  return LBM_OK;
}

lbm_status lbm_flame_length(lbm_ctx* ctx, double level, double T_u, double T_b, double* length) {
  if (!ctx || !length) return fail(ctx, LBM_ERR_ARG, "null argument");
  if (!ctx->have_fields) return fail(ctx, LBM_ERR_STATE, "set_fields must come first");
  if (ctx->D != 2 || !ctx->cfg.thermal) return fail(ctx, LBM_ERR_UNSUPPORTED, "flame length: 2-D thermal runs");
  if (!(T_b != T_u)) return fail(ctx, LBM_ERR_ARG, "T_b must differ from T_u");
  CK(cudaSetDevice(ctx->dev), "cudaSetDevice");
  const int nb = (int)((ctx->N + stats_block() - 1) / stats_block());
  if (!ctx->fl_partials && !(ctx->fl_partials = (double*)dalloc(ctx, (size_t)nb * sizeof(double))))
    return fail(ctx, LBM_ERR_ALLOC, "allocation failed");
  const int cur = ctx->cur;
  if (ctx->f64)
    CK(launch_flame_length<double>(ctx->geo, ctx->links, (const double*)ctx->T[cur], T_u, T_b, level, ctx->fl_partials,
                                   ctx->st),
       "flame length");
  else
    CK(launch_flame_length<float>(ctx->geo, ctx->links, (const float*)ctx->T[cur], T_u, T_b, level, ctx->fl_partials,
                                  ctx->st),
       "flame length");
  std::vector<double> h(nb);
  CK(cudaMemcpyAsync(h.data(), ctx->fl_partials, nb * sizeof(double), cudaMemcpyDeviceToHost, ctx->st), "copy");
  CK(cudaStreamSynchronize(ctx->st), "sync");
  double t = 0.0;
  for (double v : h) t += v;
  *length = t;
  return LBM_OK;
}

lbm_status lbm_flame_properties(lbm_ctx* ctx, int fuel_species, double* props, double* profile) {
  if (!ctx || !props) return fail(ctx, LBM_ERR_ARG, "null argument");
  if (!ctx->have_fields) return fail(ctx, LBM_ERR_STATE, "set_fields must come first");
  if (!ctx->cfg.thermal || fuel_species < 0 || fuel_species >= ctx->K)
    return fail(ctx, LBM_ERR_ARG, "flame properties need a thermal run and a valid fuel index");
  const double Y_Fu = ctx->cfg.Y_in[fuel_species];
  if (!(Y_Fu > 0.0)) return fail(ctx, LBM_ERR_ARG, "the inlet mixture holds no fuel");
  CK(cudaSetDevice(ctx->dev), "cudaSetDevice");
  const size_t nx = ctx->cfg.nx, rows = (size_t)flame_col_rows();
  if (!ctx->flame_col && !(ctx->flame_col = (double*)dalloc(ctx, rows * nx * 8)))
    return fail(ctx, LBM_ERR_ALLOC, "allocation failed");
  if (!ctx->flame_props && !(ctx->flame_props = (double*)dalloc(ctx, (6 + LBM_MAX_SPECIES) * 8)))
    return fail(ctx, LBM_ERR_ALLOC, "allocation failed");
  const double rho_u_per_P = ctx->W_in / (R_GAS * ctx->cfg.T_in);
  const double dx = ctx->cfg.dx;
  if (ctx->f64)
    CK(launch_flame_properties<double>(make_fd_args<double>(ctx, ctx->cur), fuel_species, rho_u_per_P, Y_Fu, dx,
                                       ctx->flame_col, ctx->flame_props, ctx->st),
       "flame properties");
  else
    CK(launch_flame_properties<float>(make_fd_args<float>(ctx, ctx->cur), fuel_species, rho_u_per_P, Y_Fu, dx,
                                      ctx->flame_col, ctx->flame_props, ctx->st),
       "flame properties");
  CK(cudaMemcpyAsync(props, ctx->flame_props, (6 + ctx->K) * 8, cudaMemcpyDeviceToHost, ctx->st), "copy");
  if (profile) {
    // rows T, -omega_F, Y_k of the column means (the fluid-count row is not returned)
    CK(cudaMemcpyAsync(profile, ctx->flame_col + nx, (2 + ctx->K) * nx * 8, cudaMemcpyDeviceToHost, ctx->st),
       "copy");
  }
  CK(cudaStreamSynchronize(ctx->st), "sync");
  return LBM_OK;
}

lbm_status lbm_set_probes(lbm_ctx* ctx, int n_probes, const int* cells, long long capacity, int interval) {
  if (!ctx) return LBM_ERR_ARG;
  if (!ctx->have_geo) return fail(ctx, LBM_ERR_STATE, "set_geometry must come first");
  if (n_probes < 0 || (n_probes > 0 && (!cells || capacity < 1 || interval < 1)))
    return fail(ctx, LBM_ERR_ARG, "n_probes >= 0, cells, capacity >= 1 and interval >= 1 needed");
  CK(cudaSetDevice(ctx->dev), "cudaSetDevice");
  ctx->pr_on = false;
  ctx->pr_count = 0;
  ctx->pr_n = 0;
  if (n_probes == 0) return LBM_OK;
  std::vector<uint8_t> hm(ctx->N);
  CK(cudaMemcpyAsync(hm.data(), ctx->mask, ctx->N, cudaMemcpyDeviceToHost, ctx->st), "copy mask");
  CK(cudaStreamSynchronize(ctx->st), "sync");
  for (int i = 0; i < n_probes; ++i)
    if (cells[i] < 0 || (size_t)cells[i] >= ctx->N || hm[cells[i]])
      return fail(ctx, LBM_ERR_ARG, "probe cell " + std::to_string(i) + " is outside the grid or solid");
  const int nf = ctx->D + 1 + (ctx->cfg.thermal ? 1 : 0);
  const size_t words = (size_t)capacity * n_probes * nf;
  if (words > ctx->pr_ring_words) {
    // grow: an older, smaller ring stays with the context's allocations until lbm_destroy
    if (!(ctx->pr_ring = (double*)dalloc(ctx, words * 8))) return fail(ctx, LBM_ERR_ALLOC, "allocation failed");
    ctx->pr_ring_words = words;
  }
  if (!(ctx->pr_cells = (int*)dalloc(ctx, (size_t)n_probes * sizeof(int))))
    return fail(ctx, LBM_ERR_ALLOC, "allocation failed");
  CK(cudaMemcpyAsync(ctx->pr_cells, cells, (size_t)n_probes * sizeof(int), cudaMemcpyHostToDevice, ctx->st),
     "copy probes");
  CK(cudaStreamSynchronize(ctx->st), "sync");
  ctx->pr_n = n_probes;
  ctx->pr_nf = nf;
  ctx->pr_cap = capacity;
  ctx->pr_interval = interval;
  ctx->pr_on = true;
  return LBM_OK;
}

namespace {
// device scratch of at least n doubles for the spectrum calls
double* psd_scratch(lbm_ctx* ctx, size_t n) {
  if (ctx->psd_ws_n < n) {
    double* p = (double*)dalloc(ctx, n * 8);
    if (!p) return nullptr;
    ctx->psd_ws = p;
    ctx->psd_ws_n = n;
  }
  return ctx->psd_ws;
}
}  // namespace

lbm_status lbm_get_probes(lbm_ctx* ctx, double* dst, int dst_on_device, long long* n_samples) {
  if (!ctx) return LBM_ERR_ARG;
  if (!ctx->pr_n) return fail(ctx, LBM_ERR_STATE, "no probes set");
  CK(cudaSetDevice(ctx->dev), "cudaSetDevice");
  const long long count = ctx->pr_count < ctx->pr_cap ? ctx->pr_count : ctx->pr_cap;
  const long long first = ctx->pr_count < ctx->pr_cap ? 0 : ctx->pr_count % ctx->pr_cap;
  const long long row = (long long)ctx->pr_n * ctx->pr_nf;
  if (n_samples) *n_samples = count;
  if (!dst || count == 0) return LBM_OK;
  double* view = dst_on_device ? dst : (double*)device_view(dst);
  double* out = view;
  if (!view && !(out = psd_scratch(ctx, (size_t)(count * row)))) return fail(ctx, LBM_ERR_ALLOC, "allocation failed");
  CK(launch_ring_order(ctx->pr_ring, ctx->pr_cap, first, count, row, out, ctx->st), "probe order");
  if (!view)
    CK(cudaMemcpyAsync(dst, out, (size_t)(count * row) * 8, cudaMemcpyDeviceToHost, ctx->st), "copy probes");
  if (!dst_on_device) CK(cudaStreamSynchronize(ctx->st), "sync");
  return LBM_OK;
}

namespace {
lbm_status welch_impl(lbm_ctx* ctx, const double* x, long long n, long long stride, double dt, int seg_len,
                      double* psd, size_t ws_offset) {
  const int nseg = (int)((n - seg_len) / (seg_len / 2) + 1);
  double* ws = psd_scratch(ctx, ws_offset + (size_t)nseg + seg_len / 2 + 1);
  if (!ws) return fail(ctx, LBM_ERR_ALLOC, "allocation failed");
  double* mean = ws + ws_offset;
  double* dpsd = mean + nseg;
  CK(launch_welch(x, stride, n, seg_len, dt, mean, dpsd, ctx->st), "spectrum");
  CK(cudaMemcpyAsync(psd, dpsd, (size_t)(seg_len / 2 + 1) * 8, cudaMemcpyDeviceToHost, ctx->st), "copy");
  CK(cudaStreamSynchronize(ctx->st), "sync");
  return LBM_OK;
}
bool bad_segment(long long n, int seg_len) { return seg_len < 4 || seg_len % 2 != 0 || n < seg_len; }
}  // namespace

lbm_status lbm_welch_psd(lbm_ctx* ctx, const double* x, long long n, long long stride, double dt, int seg_len,
                         double* psd) {
  if (!ctx || !x || !psd) return fail(ctx, LBM_ERR_ARG, "null argument");
  if (bad_segment(n, seg_len) || stride < 1 || !(dt > 0.0))
    return fail(ctx, LBM_ERR_ARG, "seg_len even and >= 4, n >= seg_len, stride >= 1, dt > 0");
  CK(cudaSetDevice(ctx->dev), "cudaSetDevice");
  return welch_impl(ctx, x, n, stride, dt, seg_len, psd, 0);
}

lbm_status lbm_probe_spectrum(lbm_ctx* ctx, int probe, int field, int seg_len, double* psd) {
  if (!ctx || !psd) return fail(ctx, LBM_ERR_ARG, "null argument");
  if (!ctx->pr_n) return fail(ctx, LBM_ERR_STATE, "no probes set");
  if (probe < 0 || probe >= ctx->pr_n || field < 0 || field >= ctx->pr_nf)
    return fail(ctx, LBM_ERR_ARG, "probe or field index out of range");
  const long long count = ctx->pr_count < ctx->pr_cap ? ctx->pr_count : ctx->pr_cap;
  if (bad_segment(count, seg_len)) return fail(ctx, LBM_ERR_ARG, "seg_len even, >= 4 and <= the samples recorded");
  CK(cudaSetDevice(ctx->dev), "cudaSetDevice");
  const long long first = ctx->pr_count < ctx->pr_cap ? 0 : ctx->pr_count % ctx->pr_cap;
  const long long row = (long long)ctx->pr_n * ctx->pr_nf;
  const size_t words = (size_t)(count * row);
  const int nseg = (int)((count - seg_len) / (seg_len / 2) + 1);
  double* ws = psd_scratch(ctx, words + (size_t)nseg + seg_len / 2 + 1);
  if (!ws) return fail(ctx, LBM_ERR_ALLOC, "allocation failed");
  CK(launch_ring_order(ctx->pr_ring, ctx->pr_cap, first, count, row, ws, ctx->st), "probe order");
  return welch_impl(ctx, ws + (size_t)probe * ctx->pr_nf + field, count, row, ctx->pr_interval * ctx->cfg.dt,
                    seg_len, psd, words);
}

lbm_status lbm_use_graphs(lbm_ctx* ctx, int enable) {
  if (!ctx) return LBM_ERR_ARG;
  ctx->use_graphs = enable != 0;
  return LBM_OK;
}

}  // extern "C"
