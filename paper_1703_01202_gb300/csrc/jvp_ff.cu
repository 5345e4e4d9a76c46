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

// Unscaled 5-point Laplacian (e + w) + (n + s) - 4 c.
__device__ __forceinline__ ff ff_lap(ff c, ff e, ff w, ff n, ff s) {
  return ff_add(ff_add(ff_add(e, w), ff_add(n, s)), ff_neg(ff_scale(c, 4.0f)));
}

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
  for (int i = tid; i < AX * AY; i += NT) {
    const int ly = i / AX, lx = i - ly * AX;
    const long long idx = cell_index(x0 + lx - R, g.nx, g.neumann) + (long long)g.nx * cell_index(y0 + ly - R, g.ny, g.neumann);
    sV[ly][lx] = ff_split(vscale ? sc * v[idx] : v[idx]);
  }
  for (int i = tid; i < (AX - 4) * (AY - 4); i += NT) {
    const int ly = i / (AX - 4), lx = i - ly * (AX - 4);
    const long long idx = cell_index(x0 + lx - 1, g.nx, g.neumann) + (long long)g.nx * cell_index(y0 + ly - 1, g.ny, g.neumann);
    sQ[ly][lx] = ff_split(q[idx]);
  }
  __syncthreads();
  for (int i = tid; i < (AX - 2) * (AY - 2); i += NT) {
    const int ly = i / (AX - 2) + 1, lx = i - (ly - 1) * (AX - 2) + 1;
    sL[ly - 1][lx - 1] = ff_lap(sV[ly][lx], sV[ly][lx + 1], sV[ly][lx - 1], sV[ly + 1][lx], sV[ly - 1][lx]);
  }
  __syncthreads();
  const ff ih2 = ff_split(g.ih2), hih4 = ff_split(0.5 * g.ih2 * g.ih2), c0 = ff_split(0.5 * (1.0 - g.gamma));
  for (int i = tid; i < (AX - 4) * (AY - 4); i += NT) {
    const int ly = i / (AX - 4) + 2, lx = i - (ly - 2) * (AX - 4) + 2;
    const int a = ly - 1, b = lx - 1;
    const ff Lv = sL[a][b];
    const ff LLv = ff_lap(Lv, sL[a][b + 1], sL[a][b - 1], sL[a + 1][b], sL[a - 1][b]);
    const ff vv = sV[ly][lx];
    // w = c0 v + ih2 Lv + (ih4/2) LLv + q v
    sW[ly - 2][lx - 2] = ff_add(ff_add(ff_mul(c0, vv), ff_mul(ih2, Lv)),
                                ff_add(ff_mul(hih4, LLv), ff_mul(sQ[ly - 2][lx - 2], vv)));
  }
  __syncthreads();
  const ff fidt = ff_split(idt);
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    const int tx = threadIdx.x, ty = threadIdx.y + 8 * r;
    const int gx = x0 + tx, gy = y0 + ty;
    if (gx < g.nx && gy < g.ny) {
      const int a = ty + 1, b = tx + 1;
      const ff Lw = ff_lap(sW[a][b], sW[a][b + 1], sW[a][b - 1], sW[a + 1][b], sW[a - 1][b]);
      const ff out = ff_add(ff_mul(sV[ty + R][tx + R], fidt), ff_neg(ff_mul(ih2, Lw)));
      Jv[gx + (long long)g.nx * gy] = ff_to_double(out);
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
  for (int i = tid; i < FAX * FAY; i += 256) {
    const int ly = i / FAX, lx = i - ly * FAX;
    const long long idx =
        cell_index(x0 + lx - FR, g.nx, g.neumann) + (long long)g.nx * cell_index(y0 + ly - FR, g.ny, g.neumann);
    sV[ly][lx] = f32_cut(v[idx]);
  }
  for (int i = tid; i < (FAX - 4) * (FAY - 4); i += 256) {
    const int ly = i / (FAX - 4), lx = i - ly * (FAX - 4);
    const long long idx =
        cell_index(x0 + lx - 1, g.nx, g.neumann) + (long long)g.nx * cell_index(y0 + ly - 1, g.ny, g.neumann);
    sQ[ly][lx] = f32_cut(q[idx]);
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
