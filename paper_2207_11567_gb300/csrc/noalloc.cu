// Thermodynamic-pressure integral without any device allocation.
//
// Some callers cannot allocate device memory at the point where they need this quantity: a host
// framework that owns every allocation through its own pool, code running where cudaMalloc is
// forbidden or would synchronise the device, or a monitor that only holds pointers to fields
// produced elsewhere. For them, lbm_pth_integral_noalloc computes
//     I = sum over fluid cells of W / (R T rho_ref),  W = (sum_k Y_k / W_k)^-1,
// from FP32 temperature and mass-fraction fields already in device memory, with the same
// kernel and the same exact fixed-point per-block partial sums that lbm_step uses for the
// thermodynamic pressure. The partial sums live in g_noalloc_partials, a file-scope device
// array of fixed size: every GPU that loads this library holds that array (1 MiB) until the
// process exits. Its last two words count the fluid cells whose integrand the fixed-point sum
// cannot hold (a non-finite value, or 2^30 and above after scaling, e.g. T = 0); such a call
// writes NaN to I_out.
#include <cstring>
#include <mutex>

#include "../../include/hlbm.h"
#include "launch.h"

namespace {

constexpr int kMaxBlocks = 65536;  // partial slots: 2 int64 per block of AUX_BLOCK cells
constexpr double kRGas = 8.314462618;

// Shared by every call on a device; each call overwrites the slots it uses and clears the
// bad-cell counter (word 2 kMaxBlocks) first.
static __device__ __align__(256) long long g_noalloc_partials[2 * kMaxBlocks + 2];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
void* g_partials_ptr[kMaxDevices] = {nullptr};

// Exact sum of the int64 partials, scaled back to the integral (one block); NaN when a cell's
// integrand was out of the fixed-point range.
__global__ void noalloc_sum_kernel(const long long* __restrict__ partials, int nblocks, double scale,
                                   const unsigned long long* __restrict__ bad, double* __restrict__ out) {
  __shared__ long long s[1024];
  long long v = 0;
  for (int i = threadIdx.x; i < nblocks; i += blockDim.x) v += partials[2 * i];
  s[threadIdx.x] = v;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = *bad ? __longlong_as_double(0x7ff8000000000000LL) : (double)s[0] / scale;
}

void set_err(char* err, size_t err_len, const char* msg) {
  if (err && err_len) {
    std::strncpy(err, msg, err_len - 1);
    err[err_len - 1] = '\0';
  }
}

}  // namespace

extern "C" lbm_status lbm_pth_integral_noalloc(const float* T, const float* Y, const uint8_t* mask, int n_cells,
                                               int n_species, const double* W, double T_ref, double rho_ref,
                                               double* I_out, void* stream, char* err, size_t err_len) {
  if (!T || !Y || !mask || !W || !I_out || n_cells < 1 || n_species < 1 || n_species > LBM_MAX_SPECIES ||
      !(T_ref > 0) || !(rho_ref > 0)) {
    set_err(err, err_len, "invalid argument");
    return LBM_ERR_ARG;
  }
  const long long nblocks = ((long long)n_cells + hlbm::AUX_BLOCK - 1) / hlbm::AUX_BLOCK;
  if (nblocks > kMaxBlocks) {
    set_err(err, err_len, "n_cells exceeds the static scratch of lbm_pth_integral_noalloc (16777216 cells)");
    return LBM_ERR_ARG;
  }
  for (int k = 0; k < n_species; ++k)
    if (!(W[k] > 0)) {
      set_err(err, err_len, "molar masses must be > 0");
      return LBM_ERR_ARG;
    }
  // the work runs on the stream's device (the current device for the legacy default stream):
  // that device is made current for the call and the caller's current device restored after it
  cudaStream_t st = (cudaStream_t)stream;
  int cur = 0, dev = 0;
  if (cudaGetDevice(&cur) != cudaSuccess) {
    set_err(err, err_len, "no usable CUDA device");
    return LBM_ERR_CUDA;
  }
  dev = cur;
  if (st && cudaStreamGetDevice(st, &dev) != cudaSuccess) {
    set_err(err, err_len, "stream does not belong to a usable device");
    return LBM_ERR_ARG;
  }
  if (dev < 0 || dev >= kMaxDevices) {
    set_err(err, err_len, "device index beyond the supported range");
    return LBM_ERR_CUDA;
  }
  struct Restore {
    int d;
    bool on;
    ~Restore() {
      if (on) cudaSetDevice(d);
    }
  } restore{cur, dev != cur};
  if (dev != cur && cudaSetDevice(dev) != cudaSuccess) {
    set_err(err, err_len, "cannot make the stream's device current");
    return LBM_ERR_CUDA;
  }
  void* partials = nullptr;
  {
    // first call on this device: resolve the device address of the static array (with the
    // device current); host code cannot use the array's name as a device pointer
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_partials_ptr[dev]) {
      void* p = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_partials);
      if (e != cudaSuccess || !p) {
        set_err(err, err_len, cudaGetErrorString(e));
        return LBM_ERR_CUDA;
      }
      g_partials_ptr[dev] = p;
    }
    partials = g_partials_ptr[dev];
  }
  // per cell I_unit W / T in FP32, exact fixed-point sums as in the context's FP32 path; the
  // scale T_ref / max_k W_k keeps the terms of order T_ref / T whatever the molar masses
  hlbm::FDConst<float> c{};
  c.K = n_species;
  double Wmax = 0.0;
  for (int k = 0; k < n_species; ++k) {
    c.inv_W[k] = (float)(1.0 / W[k]);
    Wmax = W[k] > Wmax ? W[k] : Wmax;
  }
  c.I_scale = (float)(T_ref / Wmax);
  const double I_s = (double)c.I_scale * kRGas * rho_ref;
  hlbm::Geo g{};
  g.nx = n_cells;
  g.ny = 1;
  g.nz = 1;
  g.N = n_cells;
  unsigned long long* bad = reinterpret_cast<unsigned long long*>((long long*)partials + 2 * kMaxBlocks);
  cudaError_t e = cudaMemsetAsync(bad, 0, sizeof(unsigned long long), st);
  if (e == cudaSuccess) e = hlbm::launch_init_integral<float>(g, mask, T, Y, c, partials, (int)nblocks, st, bad);
  if (e == cudaSuccess) {
    noalloc_sum_kernel<<<1, 1024, 0, st>>>((const long long*)partials, (int)nblocks, hlbm::FIX_SCALE * I_s, bad,
                                           I_out);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) {
    set_err(err, err_len, cudaGetErrorString(e));
    return LBM_ERR_CUDA;
  }
  set_err(err, err_len, "");
  return LBM_OK;
}
