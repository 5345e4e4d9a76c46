// Jacobian-vector product of the mixed path in float-float arithmetic.
//
// J v = v/dt - Delta_d w,  w = L_gamma v / 2 + q v (Eq. Jacobi) is linear in v, so
// GMRES only needs it to the accuracy of its own stop test, not bit-for-bit
// FP64.  GB300 executes FP64 at 1/61 of the FP32 rate, so the FP64 stencil is
// bound by the FP64 pipe; here the stencil runs in the float-float arithmetic of
// ff.cuh on the FP32 pipe, and the output takes one FP64 addition.
//
// The plain FP64 path keeps k_jvp2d; this kernel serves F32/BF16-factor solves.
#include "ff.cuh"
#include "pfc_internal.cuh"

namespace pfc {
namespace {

constexpr int TX = 32, TY = 16, R = 3;
constexpr int AX = TX + 2 * R, AY = TY + 2 * R;  // 38 x 22 staged points
constexpr int NT = 256;                          // 32 x 8 threads, 2 outputs each

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
                                              const IterArgs* __restrict__ ia) {
  if (skip && *skip) return;
  if (ia) {  // graph mode: J Z_j into V_(j+1)
    v = ia->z;
    q = ia->q;
    idt = ia->idt;
    Jv = ia->w;
  }
  __shared__ ff sV[AY][AX];
  __shared__ ff sQ[AY - 4][AX - 4];
  __shared__ ff sL[AY - 2][AX - 2];
  __shared__ ff sW[AY - 4][AX - 4];
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
  const int tid = threadIdx.x + threadIdx.y * 32;
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
  __syncthreads();
  for (int i = tid; i < (AX - 2) * (AY - 2); i += NT) {
    const int ly = i / (AX - 2) + 1, lx = i - (ly - 1) * (AX - 2) + 1;
    sL[ly - 1][lx - 1] = ff_lap5(sV[ly][lx], sV[ly][lx + 1], sV[ly][lx - 1], sV[ly + 1][lx], sV[ly - 1][lx]);
  }
  __syncthreads();
  const ff ih2 = ff_split(g.ih2), hih4 = ff_split(0.5 * g.ih2 * g.ih2), c0 = ff_split(0.5 * (1.0 - g.gamma));
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
  const ff fidt = ff_split(idt);
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    const int tx = threadIdx.x, ty = threadIdx.y + 8 * r;
    const int gx = x0 + tx, gy = y0 + ty;
    if (gx < g.nx && gy < g.ny) {
      const int a = ty + 1, b = tx + 1;
      const ff Lw = ff_lap5(sW[a][b], sW[a][b + 1], sW[a][b - 1], sW[a + 1][b], sW[a - 1][b]);
      Jv[gx + (long long)g.nx * gy] = ff_to_double(ff_dot2m(sV[ty + R][tx + R], fidt, ih2, Lw));
    }
  }
}

}  // namespace

void launch_jvp2d_ff(const Geo& g, const double* v, const double* vscale, const double* q, double idt, double* Jv,
                     const int* skip, cudaStream_t st, const IterArgs* ia) {
  dim3 grid((g.nx + TX - 1) / TX, (g.ny + TY - 1) / TY);
  k_jvp2d_ff<<<grid, dim3(32, 8), 0, st>>>(g, v, vscale, q, idt, Jv, skip, ia);
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
                                                   const IterArgs* __restrict__ ia) {
  if (skip && *skip) return;
  if (ia) {  // graph mode: J Z_j into V_(j+1)
    v = ia->z;
    q = ia->q;
    idt = ia->idt;
    Jv = ia->w;
  }
  __shared__ float sV[FAY][FAX];
  __shared__ float sQ[FAY - 4][FAX - 4];
  __shared__ float sL[FAY - 2][FAX - 2];
  __shared__ float sW[FAY - 4][FAX - 4];
  const int x0 = blockIdx.x * FTX, y0 = blockIdx.y * FTY;
  const int tid = threadIdx.x + threadIdx.y * 32;
  const Stage sv(g, x0, y0, FTX, FTY, FR), sq(g, x0, y0, FTX, FTY, 1);
  for (int i = tid; i < FAX * FAY; i += 256) {
    const int ly = i / FAX, lx = i - ly * FAX;
    sV[ly][lx] = f32_cut(v[sv.idx(g, lx, ly)]);
  }
  for (int i = tid; i < (FAX - 4) * (FAY - 4); i += 256) {
    const int ly = i / (FAX - 4), lx = i - ly * (FAX - 4);
    sQ[ly][lx] = f32_cut(q[sq.idx(g, lx, ly)]);
  }
  __syncthreads();
  for (int i = tid; i < (FAX - 2) * (FAY - 2); i += 256) {
    const int ly = i / (FAX - 2) + 1, lx = i - (ly - 1) * (FAX - 2) + 1;
    sL[ly - 1][lx - 1] = (sV[ly][lx + 1] + sV[ly][lx - 1]) + (sV[ly + 1][lx] + sV[ly - 1][lx]) - 4.0f * sV[ly][lx];
  }
  __syncthreads();
  const float ih2 = f32_cut(g.ih2), hih4 = f32_cut(0.5 * g.ih2 * g.ih2), c0 = f32_cut(0.5 * (1.0 - g.gamma));
  for (int i = tid; i < (FAX - 4) * (FAY - 4); i += 256) {
    const int ly = i / (FAX - 4) + 2, lx = i - (ly - 2) * (FAX - 4) + 2;
    const int a = ly - 1, b = lx - 1;
    const float Lv = sL[a][b];
    const float LLv = (sL[a][b + 1] + sL[a][b - 1]) + (sL[a + 1][b] + sL[a - 1][b]) - 4.0f * Lv;
    const float vv = sV[ly][lx];
    sW[ly - 2][lx - 2] = fmaf(c0 + sQ[ly - 2][lx - 2], vv, fmaf(ih2, Lv, hih4 * LLv));  // w = (c0 + q) v + ih2 Lv + ih4/2 LLv
  }
  __syncthreads();
  const float fidt = f32_cut(idt);
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    const int tx = threadIdx.x, ty = threadIdx.y + 8 * r;
    const int gx = x0 + tx, gy = y0 + ty;
    if (gx < g.nx && gy < g.ny) {
      const int a = ty + 1, b = tx + 1;
      const float Lw = (sW[a][b + 1] + sW[a][b - 1]) + (sW[a + 1][b] + sW[a - 1][b]) - 4.0f * sW[a][b];
      Jv[gx + (long long)g.nx * gy] = f2d_bits(fmaf(sV[ty + FR][tx + FR], fidt, -ih2 * Lw));
    }
  }
}

}  // namespace

void launch_jvp2d_f32(const Geo& g, const double* v, const double* q, double idt, double* Jv, const int* skip,
                      cudaStream_t st, const IterArgs* ia) {
  dim3 grid((g.nx + FTX - 1) / FTX, (g.ny + FTY - 1) / FTY);
  k_jvp2d_f32<<<grid, dim3(32, 8), 0, st>>>(g, v, q, idt, Jv, skip, ia);
  count_launches(1);
}

}  // namespace pfc
