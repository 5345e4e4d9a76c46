// pfc_residual_static: the 2D residual and its norm for callers that cannot
// allocate device memory at all (no cudaMalloc, no caching allocator, no
// workspace of their own) -- for example code running inside a host that
// forbids device allocations after start-up, or a plug-in that is handed
// only its input and output buffers.
//
// The kernel's scratch (one partial sum of F^2 per 32x16 tile and the reduced
// total) lives in a file-scope __device__ array of fixed size instead of a
// caller workspace.  Every GPU that loads this library holds the array until
// the process exits.  In host code the array's name is only a host-side
// stand-in for the symbol, never a device address: every call looks up the
// array's address on the current device with cudaGetSymbolAddress (cheap once
// the module is loaded, and never stale after the context is torn down and
// the module reloaded) and passes it to the kernels.
#include <cuda_runtime.h>

#include <cmath>

#include "../../include/pfc.h"
#include "pfc_internal.cuh"

namespace {

constexpr int kStaticTiles = 65536;  // 32 x 16 tiles: grids of up to 33,554,432 cells
// [0, kStaticTiles): per-tile partial sums; [kStaticTiles]: the reduced sum of F^2.
static __device__ __align__(256) double g_residual_scratch[kStaticTiles + 32];

// Device address of the scratch array on the current device.
int scratch_on_current_device(double** out) {
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_residual_scratch) != cudaSuccess || !p) return PFC_ECUDA;
  *out = static_cast<double*>(p);
  return PFC_OK;
}

}  // namespace

extern "C" int pfc_residual_static(const pfc_grid* grid, double h, double eps, const double* Phi,
                                   const double* phin, double dt, double* F_out, double* norm, void* cuda_stream) {
  // the grid and scalar checks of pfc_create (an infinite h would zero the stencil silently)
  if (!grid || !Phi || !phin || !F_out || grid->dim != 2 || grid->n[2] != 1 || !(h > 0.0) || !std::isfinite(h) ||
      !std::isfinite(eps) || !(dt > 0.0) || !std::isfinite(dt))
    return PFC_EINVAL;
  if (grid->n[0] < 1 || grid->n[1] < 1 || grid->n[0] > (1 << 20) || grid->n[1] > (1 << 20)) return PFC_EINVAL;
  const long long tiles = ((grid->n[0] + 31) / 32) * ((grid->n[1] + 15) / 16);
  if (tiles > kStaticTiles) return PFC_EINVAL;  // beyond the fixed scratch: use pfc_residual
  double* scratch = nullptr;
  int rc = scratch_on_current_device(&scratch);
  if (rc) return rc;
  pfc::Geo g{};
  g.nx = (int)grid->n[0];
  g.ny = (int)grid->n[1];
  g.nz = 1;
  g.n = (long long)g.nx * g.ny;
  g.ih2 = 1.0 / (h * h);
  g.gamma = eps;
  g.hd = h * h;
  pfc::geo_constants(&g);
  cudaStream_t st = (cudaStream_t)cuda_stream;
  int np = 0;
  // every tile writes its own partial and the reduction overwrites the total, so
  // no part of the scratch has to start at zero
  pfc::launch_residual2d(g, Phi, nullptr, 0.0, nullptr, phin, 1.0 / dt, F_out, nullptr, nullptr, scratch, &np, st);
  pfc::launch_reduce(scratch, 1, np, scratch + kStaticTiles, st);
  if (cudaGetLastError() != cudaSuccess) return PFC_ECUDA;
  double s2 = 0.0;
  if (cudaMemcpyAsync(&s2, scratch + kStaticTiles, sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return PFC_ECUDA;
  if (norm) *norm = std::sqrt(s2);
  return PFC_OK;
}
