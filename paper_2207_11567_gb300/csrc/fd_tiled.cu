// Host side of the tiled FD update (fd_tiled.cuh): eligibility, TMA tensor maps, launch.
#include <algorithm>
#include <cstdlib>
#include <new>
#include "fd_tiled.cuh"
#include "launch.h"

namespace hlbm {

namespace {

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
  }
  return fn;
}

// Tensor over (x, y, z[, comp]) of a [comps][nz][ny][nx] array, box (40, 12, 1[, comps]).
bool make_map(CUtensorMap* m, CUtensorMapDataType dt, const void* base, const Geo& g, int comps) {
  const int rank = comps > 1 ? 4 : 3;
  cuuint64_t dims[4] = {(cuuint64_t)g.nx, (cuuint64_t)g.ny, (cuuint64_t)g.nz, (cuuint64_t)comps};
  cuuint64_t strides[3] = {(cuuint64_t)g.nx * 4, (cuuint64_t)g.nx * g.ny * 4, (cuuint64_t)g.N * 4};
  cuuint32_t box[4] = {(cuuint32_t)TT_PX, (cuuint32_t)TT_PY, 1u, (cuuint32_t)comps};
  cuuint32_t es[4] = {1, 1, 1, 1};
  const CUresult r = encode_fn()(m, dt, (cuuint32_t)rank, const_cast<void*>(base), dims, strides, box, es,
                                 CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                 CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

template <int NK, int NR> cudaError_t set_smem() {
  return cudaFuncSetAttribute(fd_tiled_kernel<NK, NR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)TTLayout<NK>::BYTES);
}

}  // namespace

bool fd_tiled_eligible(const Geo& g, int D, int f64, int varcp, int K, int nrx) {
  if (D != 3 || f64 || varcp) return false;
  if (!((K == 6 && nrx == 2) || (K == 4 && nrx == 1))) return false;
  for (int a = 0; a < 3; ++a)
    if (g.bc_lo[a] == BC_PERIODIC || g.bc_hi[a] == BC_PERIODIC) return false;
  if (g.nx % 4 != 0) return false;  // TMA: row strides are multiples of 16 bytes
  return encode_fn() != nullptr;
}

FDTiledMaps* fd_tiled_create() { return new (std::nothrow) FDTiledMaps(); }
void fd_tiled_destroy(FDTiledMaps* m) { delete m; }

cudaError_t fd_tiled_setup(FDTiledMaps& m, const Geo& g, int K, void* const T[2], void* const Y[2],
                           void* const F[2], const void* u, const uint32_t* sword, int n_sm) {
  m.sensor = F[0] != nullptr;
  bool ok = true;
  for (int b = 0; b < 2; ++b) {
    ok = ok && make_map(&m.T[b], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, T[b], g, 1);
    ok = ok && make_map(&m.Y[b], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, Y[b], g, K);
    m.F[b] = m.T[b];
    if (m.sensor) ok = ok && make_map(&m.F[b], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, F[b], g, 1);
  }
  ok = ok && make_map(&m.U, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, u, g, 3);
  ok = ok && make_map(&m.S, CU_TENSOR_MAP_DATA_TYPE_UINT32, sword, g, 1);
  if (!ok) return cudaErrorInvalidValue;
  // z chunks: about eleven waves of two resident blocks per SM (the last, partial wave then costs
  // little; on the 384x192x192 case 12 chunks of 16 planes ran 0.4% faster than 7 of 28, 4 chunks
  // 2% slower), at least 8 planes per chunk
  const int gx = (g.nx + TT_X - 1) / TT_X, gy = (g.ny + TT_Y - 1) / TT_Y;
  int nzc = (11 * 2 * n_sm + gx * gy - 1) / (gx * gy);
  nzc = std::max(1, std::min(nzc, g.nz / 8));
  if (const char* s = std::getenv("HLBM_FD_CHUNKS")) nzc = std::max(1, std::min(atoi(s), g.nz));
  m.lz = (g.nz + nzc - 1) / nzc;
  m.grid = dim3(gx, gy, (g.nz + m.lz - 1) / m.lz);
  cudaError_t e = set_smem<6, 2>();
  if (e == cudaSuccess) e = set_smem<4, 1>();
  return e;
}

int fd_tiled_blocks(const FDTiledMaps& m) { return (int)(m.grid.x * m.grid.y * m.grid.z); }

cudaError_t launch_fd_tiled(const FDArgs<float>& a, const FDTiledMaps& m, int cur, cudaStream_t st) {
  const dim3 block(TT_X, TT_Y);
  const int sensor = a.Floc ? 1 : 0;
  if (a.c.K == 6 && a.c.nrx == 2)
    fd_tiled_kernel<6, 2><<<m.grid, block, TTLayout<6>::BYTES, st>>>(a, m.T[cur], m.Y[cur], m.U, m.F[cur], m.S,
                                                                      m.lz, sensor);
  else
    fd_tiled_kernel<4, 1><<<m.grid, block, TTLayout<4>::BYTES, st>>>(a, m.T[cur], m.Y[cur], m.U, m.F[cur], m.S,
                                                                      m.lz, sensor);
  return cudaGetLastError();
}

}  // namespace hlbm
