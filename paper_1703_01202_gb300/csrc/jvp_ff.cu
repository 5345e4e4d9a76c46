// Jacobian-vector product of the mixed path in float-float arithmetic.
//
// J v = v/dt - Delta_d w,  w = L_gamma v / 2 + q v (Eq. Jacobi) is linear in v, so
// GMRES only needs it to the accuracy of its own stop test, not bit-for-bit
// FP64.  GB300 executes FP64 at 1/61 of the FP32 rate, so the FP64 stencil is
// bound by the FP64 pipe; here the stencil runs in the float-float arithmetic of
// ff.cuh on the FP32 pipe, and the output takes one FP64 addition.
//
// The plain FP64 path keeps k_jvp2d; this kernel serves F32/BF16-factor solves.
#include "../../include/pfc.h"
#include "ff.cuh"
#include "pfc_internal.cuh"
#include "pfc_tma.cuh"

namespace pfc {
namespace {

constexpr int TX = 32, TY = 16, R = 3;
constexpr int AX = TX + 2 * R, AY = TY + 2 * R;  // 38 x 22 staged points
constexpr int NT = 256;                          // 32 x 8 threads, 2 outputs each

// TMA staging of an interior tile: one thread issues the two tensor copies (the v box of
// kJvpBoxVX x kJvpBoxVY values from (x0 - 4, y0 - 3), the q box of kJvpBoxQX x kJvpBoxQY from
// (x0 - 2, y0 - 1); even x, as the copies need) onto one mbarrier; every thread waits, bounded.
// False (PFC_ETIMEOUT recorded, the copies drained) when the wait ran out.
__device__ __forceinline__ bool tma_stage(const JvpMaps& maps, int x0, int y0, int zj, double* tv, double* tq,
                                          uint64_t* bar, int* err) {
  const int tid = threadIdx.x + threadIdx.y * blockDim.x;
  if (tid == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (tid == 0) {
    mbar_expect_tx(bar, (kJvpBoxVX * kJvpBoxVY + kJvpBoxQX * kJvpBoxQY) * (uint32_t)sizeof(double));
    tma_load_3d(tv, &maps.z, x0 - 4, y0 - 3, zj, bar);
    tma_load_2d(tq, &maps.q, x0 - 2, y0 - 1, bar);
  }
  const bool ok = __syncthreads_and(mbar_wait_bounded(bar, 0u));
  if (!ok && tid == 0) {
    if (err) atomicExch(err, PFC_ETIMEOUT);
    mbar_wait_bounded(bar, 0u);  // the copies must land before the CTA leaves
  }
  return ok;
}
// Whether the tile at (x0, y0) stages by TMA: its boxes lie inside the grid (x0 is a multiple
// of 32, so x0 - 4 and x0 - 2 are even).
__device__ __forceinline__ bool tma_tile(const Geo& g, const JvpMaps& maps, int x0, int y0, int zj) {
  return maps.ok && zj >= 0 && x0 >= 4 && x0 - 4 + kJvpBoxVX <= g.nx && y0 >= 3 && y0 - 3 + kJvpBoxVY <= g.ny;
}
// Staging buffer shared by the TMA boxes (during staging) and later stage arrays.
constexpr int kJvpRaw = (kJvpBoxVX * kJvpBoxVY + kJvpBoxQX * kJvpBoxQY) * (int)sizeof(double);

// Global index of staged point (lx, ly) of the tile at (x0, y0) with halo r: direct when the
// whole staged region lies inside the grid (interior), else through the periodic or mirror image.
struct Stage {
  int x0, y0, r;
  bool interior;
  __device__ __forceinline__ Stage(const Geo& g, int x0_, int y0_, int tx, int ty, int r_)
      : x0(x0_), y0(y0_), r(r_), interior(x0_ - r_ >= 0 && x0_ + tx + r_ <= g.nx && y0_ - r_ >= 0 && y0_ + ty + r_ <= g.ny) {}
  __device__ __forceinline__ long long idx(const Geo& g, int lx, int ly) const {
    const int x = x0 + lx - r, y = y0 + ly - r;
    if (interior) return x + (long long)g.nx * y;
    return cell_index(x, g.nx, g.neumann) + (long long)g.nx * cell_index(y, g.ny, g.neumann);
  }
};

__global__ void __launch_bounds__(NT) k_jvp2d_ff(Geo g, const double* __restrict__ v,
                                                 const double* __restrict__ vscale, const double* __restrict__ q,
                                                 double idt, double* __restrict__ Jv, const int* __restrict__ skip,
                                                 const IterArgs* __restrict__ ia, const __grid_constant__ JvpMaps maps,
                                                 int zj, int* __restrict__ err, int pout) {
  pdl_wait();
  if (skip && *skip) return;
  if (ia) {  // graph mode: J Z_j into V_(j+1)
    v = ia->z;
    q = ia->q;
    idt = ia->idt;
    Jv = ia->w;
    zj = ia->zplane;
  }
  static_assert(kJvpRaw >= (int)sizeof(ff) * ((AY - 2) * (AX - 2) + (AY - 4) * (AX - 4)), "sL, sW fit the raw buffer");
  __shared__ ff sV[AY][AX];
  __shared__ ff sQ[AY - 4][AX - 4];
  __shared__ __align__(128) unsigned char raw[kJvpRaw];  // TMA boxes, then sL and sW
  __shared__ __align__(8) uint64_t tbar;
  ff(*sL)[AX - 2] = reinterpret_cast<ff(*)[AX - 2]>(raw);
  ff(*sW)[AX - 4] = reinterpret_cast<ff(*)[AX - 4]>(raw + sizeof(ff) * (AY - 2) * (AX - 2));
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
  const int tid = threadIdx.x + threadIdx.y * 32;
  if (!vscale && tma_tile(g, maps, x0, y0, zj)) {  // interior tile: the halo boxes by TMA
    double* tv = reinterpret_cast<double*>(raw);
    double* tq = tv + kJvpBoxVX * kJvpBoxVY;
    if (!tma_stage(maps, x0, y0, zj, tv, tq, &tbar, err)) return;
    for (int i = tid; i < AX * AY; i += NT) {
      const int ly = i / AX, lx = i - ly * AX;
      sV[ly][lx] = ff_split(tv[ly * kJvpBoxVX + lx + 1]);
    }
    for (int i = tid; i < (AX - 4) * (AY - 4); i += NT) {
      const int ly = i / (AX - 4), lx = i - ly * (AX - 4);
      sQ[ly][lx] = ff_split(tq[ly * kJvpBoxQX + lx + 1]);
    }
  } else {
    const double sc = vscale ? *vscale : 1.0;
    const Stage sv(g, x0, y0, TX, TY, R), sq(g, x0, y0, TX, TY, 1);
    for (int i = tid; i < AX * AY; i += NT) {
      const int ly = i / AX, lx = i - ly * AX;
      const long long idx = sv.idx(g, lx, ly);
      sV[ly][lx] = ff_split(vscale ? sc * v[idx] : v[idx]);
    }
    for (int i = tid; i < (AX - 4) * (AY - 4); i += NT) {
      const int ly = i / (AX - 4), lx = i - ly * (AX - 4);
      sQ[ly][lx] = ff_split(q[sq.idx(g, lx, ly)]);
    }
  }
  __shared__ ff s_k[4];  // the scheme's constants, split once per CTA
  if (tid == 0) {
    s_k[0] = ff_split(g.ih2);
    s_k[1] = ff_split(g.hih4);
    s_k[2] = ff_split(g.c0);
    s_k[3] = ff_split(idt);
  }
  __syncthreads();
  for (int i = tid; i < (AX - 2) * (AY - 2); i += NT) {
    const int ly = i / (AX - 2) + 1, lx = i - (ly - 1) * (AX - 2) + 1;
    sL[ly - 1][lx - 1] = ff_lap5(sV[ly][lx], sV[ly][lx + 1], sV[ly][lx - 1], sV[ly + 1][lx], sV[ly - 1][lx]);
  }
  __syncthreads();
  const ff ih2 = s_k[0], hih4 = s_k[1], c0 = s_k[2];
  for (int i = tid; i < (AX - 4) * (AY - 4); i += NT) {
    const int ly = i / (AX - 4) + 2, lx = i - (ly - 2) * (AX - 4) + 2;
    const int a = ly - 1, b = lx - 1;
    const ff Lv = sL[a][b];
    const ff LLv = ff_lap5(Lv, sL[a][b + 1], sL[a][b - 1], sL[a + 1][b], sL[a - 1][b]);
    const ff vv = sV[ly][lx];
    // w = c0 v + ih2 Lv + (ih4/2) LLv + q v
    sW[ly - 2][lx - 2] = ff_dot4(c0, vv, ih2, Lv, hih4, LLv, sQ[ly - 2][lx - 2], vv);
  }
  __syncthreads();
  const ff fidt = s_k[3];
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    const int tx = threadIdx.x, ty = threadIdx.y + 8 * r;
    const int gx = x0 + tx, gy = y0 + ty;
    if (gx < g.nx && gy < g.ny) {
      const int a = ty + 1, b = tx + 1;
      const ff Lw = ff_lap5(sW[a][b], sW[a][b + 1], sW[a][b - 1], sW[a + 1][b], sW[a - 1][b]);
      const ff jv = ff_dot2m(sV[ty + R][tx + R], fidt, ih2, Lw);
      if (pout)
        st_pair(Jv, gx + (long long)g.nx * gy, jv);
      else
        Jv[gx + (long long)g.nx * gy] = ff_to_double(jv);
    }
  }
}

}  // namespace

// The driver's tensor-map encoder (looked up at run time; the signature of cuTensorMapEncodeTiled).
using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

void encode_jvp_maps(const Geo& g, const double* Zbuf, size_t vstride, int m, const double* q, JvpMaps* maps) {
  *maps = JvpMaps{};
  if (g.nz != 1 || g.nx % 2 != 0 || g.nx < kJvpBoxVX + 8 || g.ny < kJvpBoxVY + 6 || m < 1 || vstride % 2 != 0)
    return;
  void* fn = nullptr;
  cudaDriverEntryPointQueryResult qr{};
  if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &qr) != cudaSuccess ||
      qr != cudaDriverEntryPointSuccess || !fn)
    return;
  const EncodeTiled enc = reinterpret_cast<EncodeTiled>(fn);
  const cuuint64_t zdim[3] = {(cuuint64_t)g.nx, (cuuint64_t)g.ny, (cuuint64_t)m};
  const cuuint64_t zstr[2] = {(cuuint64_t)g.nx * sizeof(double), (cuuint64_t)vstride * sizeof(double)};
  const cuuint32_t zbox[3] = {kJvpBoxVX, kJvpBoxVY, 1};
  const cuuint64_t qdim[2] = {(cuuint64_t)g.nx, (cuuint64_t)g.ny};
  const cuuint64_t qstr[1] = {(cuuint64_t)g.nx * sizeof(double)};
  const cuuint32_t qbox[2] = {kJvpBoxQX, kJvpBoxQY};
  const cuuint32_t ones[3] = {1, 1, 1};
  if (enc(&maps->z, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 3, const_cast<double*>(Zbuf), zdim, zstr, zbox, ones,
          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS ||
      enc(&maps->q, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, const_cast<double*>(q), qdim, qstr, qbox, ones,
          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS) {
    *maps = JvpMaps{};
    return;
  }
  maps->ok = 1;
}

void launch_jvp2d_ff(const Geo& g, const double* v, const double* vscale, const double* q, double idt, double* Jv,
                     const int* skip, cudaStream_t st, const IterArgs* ia, const JvpMaps* maps, int zj, int* err,
                     int pout) {
  dim3 grid((g.nx + TX - 1) / TX, (g.ny + TY - 1) / TY);
  JvpMaps m{};
  if (maps) m = *maps;
  launch_pdl(k_jvp2d_ff, grid, dim3(32, 8), 0, st, g, v, vscale, q, idt, Jv, skip, ia, m, zj, err, pout);
  count_launches(1);
}

}  // namespace pfc

// ---- The same product in plain FP32 (opt-in, pfc_params.jvp_fp32): v and q cut to floats, the
// stencil in FP32, the result widened to FP64 by its bit pattern.  About 2^-24 of the largest
// terms per point (the sixth-order stencil's cancellation makes that a larger part of J v for
// smooth v); GMRES still solves to its own tolerance against this operator, and Newton's FP64
// residual judges the step.
namespace pfc {
namespace {

constexpr int FTX = 32, FTY = 16, FR = 3;
constexpr int FAX = FTX + 2 * FR, FAY = FTY + 2 * FR;

__global__ void __launch_bounds__(256) k_jvp2d_f32(Geo g, const double* __restrict__ v, const double* __restrict__ q,
                                                   double idt, double* __restrict__ Jv, const int* __restrict__ skip,
                                                   const IterArgs* __restrict__ ia,
                                                   const __grid_constant__ JvpMaps maps, int zj,
                                                   int* __restrict__ err, int pout) {
  pdl_wait();
  if (skip && *skip) return;
  if (ia) {  // graph mode: J Z_j into V_(j+1)
    v = ia->z;
    q = ia->q;
    idt = ia->idt;
    Jv = ia->w;
    zj = ia->zplane;
  }
  __shared__ float sV[FAY][FAX];
  __shared__ float sQ[FAY - 4][FAX - 4];
  __shared__ float sL[FAY - 2][FAX - 2];
  __shared__ float sW[FAY - 4][FAX - 4];
  __shared__ __align__(128) unsigned char raw[kJvpRaw];  // the TMA boxes
  __shared__ __align__(8) uint64_t tbar;
  const int x0 = blockIdx.x * FTX, y0 = blockIdx.y * FTY;
  const int tid = threadIdx.x + threadIdx.y * 32;
  if (tma_tile(g, maps, x0, y0, zj)) {  // interior tile: the halo boxes by TMA
    double* tv = reinterpret_cast<double*>(raw);
    double* tq = tv + kJvpBoxVX * kJvpBoxVY;
    if (!tma_stage(maps, x0, y0, zj, tv, tq, &tbar, err)) return;
    for (int i = tid; i < FAX * FAY; i += 256) {
      const int ly = i / FAX, lx = i - ly * FAX;
      sV[ly][lx] = f32_cut(tv[ly * kJvpBoxVX + lx + 1]);
    }
    for (int i = tid; i < (FAX - 4) * (FAY - 4); i += 256) {
      const int ly = i / (FAX - 4), lx = i - ly * (FAX - 4);
      sQ[ly][lx] = f32_cut(tq[ly * kJvpBoxQX + lx + 1]);
    }
  } else {
    const Stage sv(g, x0, y0, FTX, FTY, FR), sq(g, x0, y0, FTX, FTY, 1);
    for (int i = tid; i < FAX * FAY; i += 256) {
      const int ly = i / FAX, lx = i - ly * FAX;
      sV[ly][lx] = f32_cut(v[sv.idx(g, lx, ly)]);
    }
    for (int i = tid; i < (FAX - 4) * (FAY - 4); i += 256) {
      const int ly = i / (FAX - 4), lx = i - ly * (FAX - 4);
      sQ[ly][lx] = f32_cut(q[sq.idx(g, lx, ly)]);
    }
  }
  __shared__ float s_k[4];  // the scheme's constants, cut to floats once per CTA
  if (tid == 0) {
    s_k[0] = f32_cut(g.ih2);
    s_k[1] = f32_cut(g.hih4);
    s_k[2] = f32_cut(g.c0);
    s_k[3] = f32_cut(idt);
  }
  __syncthreads();
  for (int i = tid; i < (FAX - 2) * (FAY - 2); i += 256) {
    const int ly = i / (FAX - 2) + 1, lx = i - (ly - 1) * (FAX - 2) + 1;
    sL[ly - 1][lx - 1] = (sV[ly][lx + 1] + sV[ly][lx - 1]) + (sV[ly + 1][lx] + sV[ly - 1][lx]) - 4.0f * sV[ly][lx];
  }
  __syncthreads();
  const float ih2 = s_k[0], hih4 = s_k[1], c0 = s_k[2];
  for (int i = tid; i < (FAX - 4) * (FAY - 4); i += 256) {
    const int ly = i / (FAX - 4) + 2, lx = i - (ly - 2) * (FAX - 4) + 2;
    const int a = ly - 1, b = lx - 1;
    const float Lv = sL[a][b];
    const float LLv = (sL[a][b + 1] + sL[a][b - 1]) + (sL[a + 1][b] + sL[a - 1][b]) - 4.0f * Lv;
    const float vv = sV[ly][lx];
    sW[ly - 2][lx - 2] = fmaf(c0 + sQ[ly - 2][lx - 2], vv, fmaf(ih2, Lv, hih4 * LLv));  // w = (c0 + q) v + ih2 Lv + ih4/2 LLv
  }
  __syncthreads();
  const float fidt = s_k[3];
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    const int tx = threadIdx.x, ty = threadIdx.y + 8 * r;
    const int gx = x0 + tx, gy = y0 + ty;
    if (gx < g.nx && gy < g.ny) {
      const int a = ty + 1, b = tx + 1;
      const float Lw = (sW[a][b + 1] + sW[a][b - 1]) + (sW[a + 1][b] + sW[a - 1][b]) - 4.0f * sW[a][b];
      const float jv = fmaf(sV[ty + FR][tx + FR], fidt, -ih2 * Lw);
      if (pout)
        st_pair(Jv, gx + (long long)g.nx * gy, ff{jv, 0.0f});
      else
        Jv[gx + (long long)g.nx * gy] = f2d_bits(jv);
    }
  }
}

}  // namespace

void launch_jvp2d_f32(const Geo& g, const double* v, const double* q, double idt, double* Jv, const int* skip,
                      cudaStream_t st, const IterArgs* ia, const JvpMaps* maps, int zj, int* err, int pout) {
  dim3 grid((g.nx + FTX - 1) / FTX, (g.ny + FTY - 1) / FTY);
  JvpMaps m{};
  if (maps) m = *maps;
  launch_pdl(k_jvp2d_f32, grid, dim3(32, 8), 0, st, g, v, q, idt, Jv, skip, ia, m, zj, err, pout);
  count_launches(1);
}

}  // namespace pfc
