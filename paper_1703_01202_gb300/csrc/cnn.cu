// Learned Newton initial guess: a small periodic convolutional network
// (3x3 convolutions, channels 3 -> 32 -> 32 -> 32 -> 1, exact GELU after the
// first three) with hand-written forward, backward and Adam kernels.  Weights
// and activations are stored in BF16 and every sum accumulates in FP32; the
// Adam master weights and moments are FP32.  (The paper's own guess is the
// previous solution, Sec. 4; this network is the learned form's addition.)
//
// Layouts: activations planar [channel][pixel] (x fastest), parameters one flat
// FP32 vector, layer by layer [W (Cout, Cin, 3, 3), b (Cout)].
//
// Each convolution kernel works on 16x16 pixel tiles with a one-pixel periodic
// halo staged in shared memory and the layer's weights staged as FP32.  The
// weight gradient is a reduction over all pixels: a fixed number of CTAs walk
// the tiles, keep their partial sums in registers, write them out, and one
// fixed-order reduction kernel sums them (deterministic).
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <new>

#include "../../include/pfc.h"
#include "pfc_internal.cuh"
#include "pfc_tma.cuh"

namespace pfc {

constexpr int kCnnLayers = 4;
constexpr int kCin[kCnnLayers] = {3, 32, 32, 32};
constexpr int kCout[kCnnLayers] = {32, 32, 32, 1};
constexpr int kGradCtas = 304;  // CTAs of the weight-gradient reduction

__host__ __device__ constexpr int layer_offset(int l) {
  int o = 0;
  for (int i = 0; i < l; ++i) o += kCout[i] * kCin[i] * 9 + kCout[i];
  return o;
}
constexpr int kCnnParams = layer_offset(kCnnLayers);

namespace {

constexpr int T = 16;          // tile edge
constexpr int NT = T * T;      // threads per CTA, one pixel each
constexpr int TH = T + 2;      // tile with halo

__device__ __forceinline__ int wrapi(int i, int n) {
  i %= n;
  return i < 0 ? i + n : i;
}
__device__ __forceinline__ float gelu_f(float x) { return 0.5f * x * (1.0f + erff(x * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad_f(float x) {
  return 0.5f * (1.0f + erff(x * 0.70710678118654752f)) + x * expf(-0.5f * x * x) * 0.39894228040143268f;
}

template <typename TI>
__device__ __forceinline__ float ld(const TI* p, long long i);
template <>
__device__ __forceinline__ float ld<double>(const double* p, long long i) { return (float)p[i]; }
template <>
__device__ __forceinline__ float ld<float>(const float* p, long long i) { return p[i]; }
template <>
__device__ __forceinline__ float ld<__nv_bfloat16>(const __nv_bfloat16* p, long long i) { return __bfloat162float(p[i]); }

// Loads CIN channels of a TxT tile plus a one-pixel periodic halo into s[CIN][TH][TH].
template <int CIN, typename TI>
__device__ __forceinline__ void load_tile(float* s, const TI* __restrict__ in, int nx, int ny, int x0, int y0,
                                          const float* __restrict__ scale_by_pixel_grad, const TI* dummy) {
  const long long N = (long long)nx * ny;
  for (int i = threadIdx.x; i < CIN * TH * TH; i += NT) {
    const int c = i / (TH * TH), r = i - c * TH * TH;
    const int ly = r / TH, lx = r - ly * TH;
    const long long p = wrapi(x0 + lx - 1, nx) + (long long)nx * wrapi(y0 + ly - 1, ny);
    s[i] = ld<TI>(in, c * N + p);
  }
}

// z = conv(in, W) + b; a = GELU(z) when ACT.  Output types: z and a in BF16
// (the last layer writes z in FP32 and no a).
template <int CIN, int COUT, bool ACT, typename TI, typename TZ>
__global__ void __launch_bounds__(NT) k_conv_fwd(int nx, int ny, const TI* __restrict__ in,
                                                 const __nv_bfloat16* __restrict__ W, const float* __restrict__ b,
                                                 TZ* __restrict__ z, __nv_bfloat16* __restrict__ a) {
  extern __shared__ float sm[];
  float* s_in = sm;                    // CIN * TH * TH
  float* s_w = sm + CIN * TH * TH;     // [ci][tap][co]
  const int x0 = blockIdx.x * T, y0 = blockIdx.y * T;
  load_tile<CIN, TI>(s_in, in, nx, ny, x0, y0, nullptr, nullptr);
  for (int i = threadIdx.x; i < COUT * CIN * 9; i += NT) {  // W[co][ci][tap] -> s_w[ci][tap][co]
    const int co = i / (CIN * 9), r = i - co * CIN * 9;
    s_w[r * COUT + co] = __bfloat162float(W[i]);
  }
  __syncthreads();
  const int tx = threadIdx.x % T, ty = threadIdx.x / T;
  float acc[COUT];
#pragma unroll
  for (int co = 0; co < COUT; ++co) acc[co] = b[co];
  for (int ci = 0; ci < CIN; ++ci) {
#pragma unroll
    for (int tap = 0; tap < 9; ++tap) {
      const int dy = tap / 3 - 1, dx = tap % 3 - 1;
      const float v = s_in[ci * TH * TH + (ty + 1 + dy) * TH + (tx + 1 + dx)];
      const float* wv = s_w + (ci * 9 + tap) * COUT;
#pragma unroll
      for (int co = 0; co < COUT; ++co) acc[co] = fmaf(wv[co], v, acc[co]);
    }
  }
  const int gx = x0 + tx, gy = y0 + ty;
  if (gx < nx && gy < ny) {
    const long long N = (long long)nx * ny, p = gx + (long long)nx * gy;
#pragma unroll
    for (int co = 0; co < COUT; ++co) {
      if (ACT) {
        z[co * N + p] = (TZ)acc[co];
        a[co * N + p] = __float2bfloat16(gelu_f(acc[co]));
      } else {
        z[co * N + p] = (TZ)acc[co];
      }
    }
  }
}

// The 32 -> 32 convolutions of the forward pass as an implicit GEMM on the fifth-generation
// tensor cores (tcgen05): per 16 x 16 tile, D (256 pixels x 32 channels) = sum over the 9 taps
// of A_tap (the tile shifted by the tap, 32 input channels) times W_tap^T (32 x 32), BF16
// operands from shared memory, FP32 accumulators in tensor memory (TMEM).  The 256 pixels
// are two M = 128 halves: half h holds pixel columns 8h .. 8h + 7 of all 16 rows, so row i of
// the half (TMEM lane i) is pixel (i / 8, 8h + i % 8).  K runs over tap x channel in 18 steps
// of 16; one thread issues the 36 MMAs (N = 32) and commits them to an mbarrier.
//
// Shared-memory operands in the no-swizzle K-major layout of UMMA: 8 x 16-byte core matrices
// (8 rows of 8 BF16 channels).  The input tile with its periodic halo is stored
// [channel group g (4)][halo row (18)][halo column (18)][8 channels], so 8 consecutive pixels
// of a row are one core matrix wherever the tap shifts them; the next 8 rows of M (the next
// pixel row) lie 18 x 16 bytes further (stride-dimension offset), the next 8 channels of K
// 18 x 18 x 16 bytes further (leading-dimension offset).  The weights are stored
// [tap][g][co (32)][8 channels]: N-direction offset 128 bytes, K-direction 512 bytes.
//
// Epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31 of half w / 4 (32 columns = the 32
// output channels of its 32 pixels), adds the bias, stages z and GELU(z) in shared memory and
// writes coalesced 16-pixel rows of each channel plane.  The MMA completion wait is bounded:
// when it runs out the kernel stores nothing, records PFC_ETIMEOUT in *err and still frees
// its TMEM.
constexpr int kTcCols = 64;                       // TMEM columns: two halves x 32 channels (FP32)
constexpr int kTcInBytes = 4 * TH * TH * 16;      // input tile: 20,736 bytes
constexpr int kTcWBytes = 9 * 4 * 32 * 16;        // weights: 18,432 bytes
constexpr int kTcSmem = kTcInBytes + kTcWBytes + 32 * 4 + 16;

// Instruction descriptor of tcgen05.mma kind::f16: FP32 accumulator (bits 4-5 = 1), BF16 A
// and B (bits 7-9, 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 at bits 17-22, M >> 4
// at bits 24-28.
constexpr uint32_t kTcIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((32u >> 3) << 17) | ((128u >> 4) << 24);

// Shared-memory matrix descriptor, no swizzle: start address, leading-dimension (K) and
// stride-dimension (M/N) byte offsets, each >> 4 in 14 bits; bits 46-48 hold the fixed
// descriptor version 1.
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr >> 4) & 0x3fffu) | ((uint64_t)((lbo >> 4) & 0x3fffu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3fffu) << 32) | (1ull << 46);
}
__device__ __forceinline__ void tc_alloc(uint32_t* dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)), "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tc_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t adesc, uint64_t bdesc, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(adesc), "l"(bdesc), "r"(kTcIdesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void tc_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
// 32 consecutive FP32 columns of the calling thread's TMEM lane (warp-quarter lanes).
__device__ __forceinline__ void tc_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__global__ void __launch_bounds__(NT) k_conv32_fwd_tc(int nx, int ny, const __nv_bfloat16* __restrict__ in,
                                                      const __nv_bfloat16* __restrict__ W,
                                                      const float* __restrict__ b, __nv_bfloat16* __restrict__ z,
                                                      __nv_bfloat16* __restrict__ a, int* __restrict__ err) {
  extern __shared__ __align__(128) unsigned char smraw[];
  __nv_bfloat16* s_in = reinterpret_cast<__nv_bfloat16*>(smraw);                 // [4][TH][TH][8]
  __nv_bfloat16* s_w = reinterpret_cast<__nv_bfloat16*>(smraw + kTcInBytes);    // [9][4][32][8]
  float* s_b = reinterpret_cast<float*>(smraw + kTcInBytes + kTcWBytes);         // [32]
  uint64_t* s_bar = reinterpret_cast<uint64_t*>(smraw + kTcInBytes + kTcWBytes + 128);
  uint32_t* s_tmem = reinterpret_cast<uint32_t*>(smraw + kTcInBytes + kTcWBytes + 136);
  __shared__ int s_fail;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (warp == 0) tc_alloc(s_tmem, kTcCols);
  if (tid == 0) {
    mbar_init(s_bar, 1);
    fence_mbar_init();
    s_fail = 0;
  }
  const int x0 = blockIdx.x * T, y0 = blockIdx.y * T;
  const long long N = (long long)nx * ny;
  // Input planes -> [g][row][col][8]: one 16-byte row of the layout (8 channels of a pixel) per
  // item, gathered from the 8 planes (consecutive threads take consecutive pixels).
  // All of a thread's loads are issued before its stores (the item loops are unrolled), so the
  // gathers of a tile are in flight together.
  const bool inner = x0 >= 1 && y0 >= 1 && x0 + T + 1 <= nx && y0 + T + 1 <= ny;  // no periodic wrap
  constexpr int kInItems = 4 * TH * TH, kInPer = (kInItems + NT - 1) / NT;
  constexpr int kWItems = 9 * 4 * 32, kWPer = (kWItems + NT - 1) / NT;
  uint4 vin[kInPer], vw[kWPer];
#pragma unroll
  for (int u = 0; u < kInPer; ++u) {
    const int it = tid + u * NT;
    if (it < kInItems) {
      const int g = it / (TH * TH), r = it - g * (TH * TH);
      const int ly = r / TH, lx = r - ly * TH;
      const int gx = inner ? x0 + lx - 1 : wrapi(x0 + lx - 1, nx), gy = inner ? y0 + ly - 1 : wrapi(y0 + ly - 1, ny);
      const __nv_bfloat16* src = in + (long long)(8 * g) * N + gx + (long long)nx * gy;
      __nv_bfloat16* e = reinterpret_cast<__nv_bfloat16*>(&vin[u]);
#pragma unroll
      for (int k = 0; k < 8; ++k) e[k] = src[k * N];
    }
  }
  // W[co][ci][tap] -> [tap][ci / 8][co][ci % 8], one 16-byte row (8 input channels) per item.
#pragma unroll
  for (int u = 0; u < kWPer; ++u) {
    const int it = tid + u * NT;
    if (it < kWItems) {
      const int tap = it >> 7, g = (it >> 5) & 3, co = it & 31;
      const __nv_bfloat16* src = W + co * 288 + (8 * g) * 9 + tap;
      __nv_bfloat16* e = reinterpret_cast<__nv_bfloat16*>(&vw[u]);
#pragma unroll
      for (int k = 0; k < 8; ++k) e[k] = src[9 * k];
    }
  }
#pragma unroll
  for (int u = 0; u < kInPer; ++u)
    if (tid + u * NT < kInItems) reinterpret_cast<uint4*>(s_in)[tid + u * NT] = vin[u];
#pragma unroll
  for (int u = 0; u < kWPer; ++u)
    if (tid + u * NT < kWItems) reinterpret_cast<uint4*>(s_w)[tid + u * NT] = vw[u];
  if (tid < 32) s_b[tid] = b[tid];
  fence_proxy_async();  // the operands are read by the tensor cores (async proxy)
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *s_tmem;
  if (tid == 0) {
    const uint32_t in0 = smem_u32(s_in), w0 = smem_u32(s_w);
    for (int tap = 0; tap < 9; ++tap) {
      const int dy = tap / 3 - 1, dx = tap % 3 - 1;
      for (int kc = 0; kc < 2; ++kc) {  // channels 16 kc .. 16 kc + 15: groups 2 kc, 2 kc + 1
        const uint64_t bd = umma_desc(w0 + (uint32_t)((tap * 4 + 2 * kc) * 32 * 16), 32 * 16, 8 * 16);
        for (int h = 0; h < 2; ++h) {
          const uint32_t a_at = in0 + (uint32_t)(((2 * kc) * TH * TH + (1 + dy) * TH + 8 * h + 1 + dx) * 16);
          tc_mma(tmem + 32u * h, umma_desc(a_at, TH * TH * 16, TH * 16), bd, (tap | kc) ? 1u : 0u);
        }
      }
    }
    tc_commit(s_bar);
  }
  if (!mbar_wait_bounded(s_bar, 0)) s_fail = 1;
  tc_fence_after();
  __syncthreads();  // every warp past the wait: the operand tiles are free for the output staging
  const bool ok = s_fail == 0;
  __nv_bfloat16* s_z = s_in;            // [32][256], over the input and weight tiles
  __nv_bfloat16* s_a = s_in + 32 * NT;  // [32][256]
  if (ok) {
    const int q = warp & 3, h = warp >> 2;
    uint32_t r[32];
    tc_ld32(tmem + ((uint32_t)(32 * q) << 16) + 32u * h, r);
    const int i = 32 * q + lane;
    const int pix = (i >> 3) * T + 8 * h + (i & 7);
#pragma unroll
    for (int co = 0; co < 32; ++co) {
      const float v = __uint_as_float(r[co]) + s_b[co];
      s_z[co * NT + pix] = __float2bfloat16(v);
      s_a[co * NT + pix] = __float2bfloat16(gelu_f(v));
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tc_dealloc(tmem, kTcCols);
  }
  if (!ok) {
    if (tid == 0 && err) atomicExch(err, PFC_ETIMEOUT);
    return;
  }
  if (x0 + T <= nx && y0 + T <= ny && (nx & 7) == 0) {  // whole tile, 16-byte aligned rows: 8 pixels a store
    for (int i = tid; i < 32 * NT / 8; i += NT) {
      const int co = i >> 5, ty = (i >> 1) & 15, h = i & 1;
      const long long p = co * N + x0 + 8 * h + (long long)nx * (y0 + ty);
      reinterpret_cast<uint4*>(z + p)[0] = reinterpret_cast<const uint4*>(s_z)[i];
      reinterpret_cast<uint4*>(a + p)[0] = reinterpret_cast<const uint4*>(s_a)[i];
    }
    return;
  }
  for (int i = tid; i < 32 * NT; i += NT) {  // ragged tile: 16-pixel rows of every plane
    const int co = i / NT, r = i - co * NT;
    const int ty = r / T, tx = r - ty * T;
    const int gx = x0 + tx, gy = y0 + ty;
    if (gx < nx && gy < ny) {
      const long long p = co * N + gx + (long long)nx * gy;
      z[p] = s_z[i];
      a[p] = s_a[i];
    }
  }
}

// Gradient through a convolution to its input, times GELU'(z_prev):
// dz_prev[ci][p] = GELU'(z_prev[ci][p]) * sum_{co,tap} W[co][ci][tap] dz[co][p - off(tap)]
template <int CIN, int COUT, typename TD>
__global__ void __launch_bounds__(NT) k_conv_bwd_data(int nx, int ny, const TD* __restrict__ dz,
                                                      const __nv_bfloat16* __restrict__ W,
                                                      const __nv_bfloat16* __restrict__ zprev,
                                                      float* __restrict__ dzprev) {
  extern __shared__ float sm[];
  float* s_d = sm;                   // COUT * TH * TH
  float* s_w = sm + COUT * TH * TH;  // [co][tap][ci]
  const int x0 = blockIdx.x * T, y0 = blockIdx.y * T;
  load_tile<COUT, TD>(s_d, dz, nx, ny, x0, y0, nullptr, nullptr);
  for (int i = threadIdx.x; i < COUT * CIN * 9; i += NT) {
    const int co = i / (CIN * 9), r = i - co * CIN * 9;
    const int ci = r / 9, tap = r - ci * 9;
    s_w[(co * 9 + tap) * CIN + ci] = __bfloat162float(W[i]);
  }
  __syncthreads();
  const int tx = threadIdx.x % T, ty = threadIdx.x / T;
  float acc[CIN];
#pragma unroll
  for (int ci = 0; ci < CIN; ++ci) acc[ci] = 0.0f;
  for (int co = 0; co < COUT; ++co) {
#pragma unroll
    for (int tap = 0; tap < 9; ++tap) {
      const int dy = tap / 3 - 1, dx = tap % 3 - 1;  // out[y,x] read in[y+dy,x+dx]: adjoint reads dz[y-dy,x-dx]
      const float v = s_d[co * TH * TH + (ty + 1 - dy) * TH + (tx + 1 - dx)];
      const float* wv = s_w + (co * 9 + tap) * CIN;
#pragma unroll
      for (int ci = 0; ci < CIN; ++ci) acc[ci] = fmaf(wv[ci], v, acc[ci]);
    }
  }
  const int gx = x0 + tx, gy = y0 + ty;
  if (gx < nx && gy < ny) {
    const long long N = (long long)nx * ny, p = gx + (long long)nx * gy;
#pragma unroll
    for (int ci = 0; ci < CIN; ++ci) dzprev[ci * N + p] = acc[ci] * gelu_grad_f(__bfloat162float(zprev[ci * N + p]));
  }
}

// Per-CTA partial sums of dW[co][ci][tap] = sum_p dz[co][p] a[ci][p + off(tap)] and db[co].
// Thread t owns (co, ci) pairs t, t + NT, ... (all 9 taps); CTAs stride over the tiles.
template <int CIN, int COUT, typename TA, typename TD>
__global__ void __launch_bounds__(NT) k_conv_bwd_weight(int nx, int ny, const TA* __restrict__ a,
                                                        const TD* __restrict__ dz, float* __restrict__ partial) {
  extern __shared__ float sm[];
  float* s_a = sm;                 // CIN * TH * TH
  float* s_d = sm + CIN * TH * TH;  // COUT * NT
  constexpr int PAIRS = CIN * COUT;
  constexpr int PER = (PAIRS + NT - 1) / NT;
  float acc[PER][9];
  float accb = 0.0f;
#pragma unroll
  for (int j = 0; j < PER; ++j)
#pragma unroll
    for (int t = 0; t < 9; ++t) acc[j][t] = 0.0f;
  const int tilesx = (nx + T - 1) / T, tilesy = (ny + T - 1) / T;
  const long long N = (long long)nx * ny;
  for (int tile = blockIdx.x; tile < tilesx * tilesy; tile += gridDim.x) {
    const int x0 = (tile % tilesx) * T, y0 = (tile / tilesx) * T;
    __syncthreads();
    load_tile<CIN, TA>(s_a, a, nx, ny, x0, y0, nullptr, nullptr);
    for (int i = threadIdx.x; i < COUT * NT; i += NT) {
      const int co = i / NT, r = i - co * NT;
      const int gx = x0 + r % T, gy = y0 + r / T;
      s_d[i] = (gx < nx && gy < ny) ? ld<TD>(dz, co * N + gx + (long long)nx * gy) : 0.0f;
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < PER; ++j) {
      const int pair = threadIdx.x + j * NT;
      if (pair < PAIRS) {
        const int co = pair / CIN, ci = pair - co * CIN;
        const float* sa = s_a + ci * TH * TH;
        const float* sd = s_d + co * NT;
        for (int py = 0; py < T; ++py)
          for (int px = 0; px < T; ++px) {
            const float d = sd[py * T + px];
#pragma unroll
            for (int t = 0; t < 9; ++t) acc[j][t] = fmaf(d, sa[(py + 1 + t / 3 - 1) * TH + (px + 1 + t % 3 - 1)], acc[j][t]);
          }
      }
    }
    if (threadIdx.x < COUT)
      for (int pp = 0; pp < NT; ++pp) accb += s_d[threadIdx.x * NT + pp];
  }
  float* out = partial + (size_t)blockIdx.x * (COUT * CIN * 9 + COUT);
#pragma unroll
  for (int j = 0; j < PER; ++j) {
    const int pair = threadIdx.x + j * NT;
    if (pair < PAIRS) {
      const int co = pair / CIN, ci = pair - co * CIN;
#pragma unroll
      for (int t = 0; t < 9; ++t) out[(co * CIN + ci) * 9 + t] = acc[j][t];
    }
  }
  if (threadIdx.x < COUT) out[COUT * CIN * 9 + threadIdx.x] = accb;
}

// grad[i] = sum over CTAs of partial[cta][i] (fixed order)
__global__ void k_sum_partials(const float* __restrict__ partial, int len, int nparts, float* __restrict__ grad) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < len; i += gridDim.x * blockDim.x) {
    float s = 0.0f;
    for (int c = 0; c < nparts; ++c) s += partial[(size_t)c * len + i];
    grad[i] = s;
  }
}

// d = 2/N (o - t); per-CTA partial sums of (o - t)^2.
__global__ void k_mse(long long n, const float* __restrict__ o, const double* __restrict__ t, float* __restrict__ d,
                      double* __restrict__ partial) {
  __shared__ double red[8];
  double s = 0.0;
  const float inv = 2.0f / (float)n;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float e = o[i] - (float)t[i];
    d[i] = inv * e;
    s += (double)e * e;
  }
  for (int k = 16; k > 0; k >>= 1) s += __shfl_xor_sync(0xffffffffu, s, k);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double tot = 0.0;
    for (int w = 0; w < 8; ++w) tot += red[w];
    partial[blockIdx.x] = tot;
  }
}

// Adam (Kingma & Ba) on the FP32 master weights; refreshes the BF16 weight copy.
__global__ void k_adam(int n, float* __restrict__ theta, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, float lr, float b1, float b2, float eps, float c1, float c2,
                       __nv_bfloat16* __restrict__ wbf) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float th = theta[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    theta[i] = th;
    wbf[i] = __float2bfloat16(th);
  }
}

__global__ void k_to_bf16(int n, const float* __restrict__ x, __nv_bfloat16* __restrict__ y) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) y[i] = __float2bfloat16(x[i]);
}

__global__ void k_f32_to_f64(long long n, const float* __restrict__ x, double* __restrict__ y) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = (double)x[i];
}

template <int CIN, int COUT, bool ACT, typename TI, typename TZ>
void conv_fwd(int nx, int ny, const TI* in, const __nv_bfloat16* W, const float* b, TZ* z, __nv_bfloat16* a,
              cudaStream_t st) {
  const size_t smem = sizeof(float) * (CIN * TH * TH + COUT * CIN * 9);
  cudaFuncSetAttribute(k_conv_fwd<CIN, COUT, ACT, TI, TZ>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k_conv_fwd<CIN, COUT, ACT, TI, TZ><<<dim3((nx + T - 1) / T, (ny + T - 1) / T), NT, smem, st>>>(nx, ny, in, W, b, z, a);
  count_launches(1);
}

void conv32_fwd_tc(int nx, int ny, const __nv_bfloat16* in, const __nv_bfloat16* W, const float* b,
                   __nv_bfloat16* z, __nv_bfloat16* a, int* err, cudaStream_t st) {
  cudaFuncSetAttribute(k_conv32_fwd_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmem);
  k_conv32_fwd_tc<<<dim3((nx + T - 1) / T, (ny + T - 1) / T), NT, kTcSmem, st>>>(nx, ny, in, W, b, z, a, err);
  count_launches(1);
}

template <int CIN, int COUT, typename TD>
void conv_bwd_data(int nx, int ny, const TD* dz, const __nv_bfloat16* W, const __nv_bfloat16* zprev, float* dzprev,
                   cudaStream_t st) {
  const size_t smem = sizeof(float) * (COUT * TH * TH + COUT * CIN * 9);
  cudaFuncSetAttribute(k_conv_bwd_data<CIN, COUT, TD>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k_conv_bwd_data<CIN, COUT, TD><<<dim3((nx + T - 1) / T, (ny + T - 1) / T), NT, smem, st>>>(nx, ny, dz, W, zprev,
                                                                                          dzprev);
  count_launches(1);
}

template <int CIN, int COUT, typename TA, typename TD>
void conv_bwd_weight(int nx, int ny, const TA* a, const TD* dz, float* partial, float* grad, cudaStream_t st) {
  const size_t smem = sizeof(float) * (CIN * TH * TH + COUT * NT);
  cudaFuncSetAttribute(k_conv_bwd_weight<CIN, COUT, TA, TD>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k_conv_bwd_weight<CIN, COUT, TA, TD><<<kGradCtas, NT, smem, st>>>(nx, ny, a, dz, partial);
  const int len = COUT * CIN * 9 + COUT;
  k_sum_partials<<<(len + 255) / 256, 256, 0, st>>>(partial, len, kGradCtas, grad);
  count_launches(2);
}

}  // namespace

// ---------------------------------------------------------------- network object

struct Cnn {
  int nx, ny;
  long long n;
  cudaStream_t st;
  float* theta;            // FP32 master parameters
  float* m;                // Adam moments
  float* v;
  float* grad;
  __nv_bfloat16* wbf;      // BF16 copy of the parameters (the biases are read from theta)
  __nv_bfloat16* z[3];     // pre-activations of layers 0..2 (32 x n)
  __nv_bfloat16* a[3];     // activations of layers 0..2
  float* out;              // network output (n)
  float* d1;               // gradient buffers (32 x n)
  float* d2;
  float* partial;          // kGradCtas x (largest layer's parameter count)
  double* red;             // reduction partials of the loss
  int* err;                // PFC_ETIMEOUT when a bounded wait of a kernel ran out (0: none)
};

size_t cnn_workspace_bytes(long long n) {
  auto r = [](size_t b) { return (b + 255) & ~(size_t)255; };
  size_t t = 0;
  t += 4 * r(sizeof(float) * kCnnParams);
  t += r(sizeof(__nv_bfloat16) * kCnnParams);
  t += 6 * r(sizeof(__nv_bfloat16) * 32 * n);
  t += r(sizeof(float) * n);
  t += 2 * r(sizeof(float) * 32 * n);
  t += r(sizeof(float) * (size_t)kGradCtas * (32 * 32 * 9 + 32));
  t += r(sizeof(double) * 1024);
  t += r(sizeof(int));
  return t;
}

void cnn_bind(Cnn* c, void* ws) {
  char* p = (char*)ws;
  auto take = [&](size_t b) {
    void* q = p;
    p += (b + 255) & ~(size_t)255;
    return q;
  };
  const long long n = c->n;
  c->theta = (float*)take(sizeof(float) * kCnnParams);
  c->m = (float*)take(sizeof(float) * kCnnParams);
  c->v = (float*)take(sizeof(float) * kCnnParams);
  c->grad = (float*)take(sizeof(float) * kCnnParams);
  c->wbf = (__nv_bfloat16*)take(sizeof(__nv_bfloat16) * kCnnParams);
  for (int i = 0; i < 3; ++i) c->z[i] = (__nv_bfloat16*)take(sizeof(__nv_bfloat16) * 32 * n);
  for (int i = 0; i < 3; ++i) c->a[i] = (__nv_bfloat16*)take(sizeof(__nv_bfloat16) * 32 * n);
  c->out = (float*)take(sizeof(float) * n);
  c->d1 = (float*)take(sizeof(float) * 32 * n);
  c->d2 = (float*)take(sizeof(float) * 32 * n);
  c->partial = (float*)take(sizeof(float) * (size_t)kGradCtas * (32 * 32 * 9 + 32));
  c->red = (double*)take(sizeof(double) * 1024);
  c->err = (int*)take(sizeof(int));
}

// The error flag of the network's kernels (PFC_ETIMEOUT when a bounded wait ran out), cleared
// once read; waits for the work queued on the network's stream.
int cnn_status(Cnn* c) {
  int e = 0;
  if (cudaMemcpyAsync(&e, c->err, sizeof(int), cudaMemcpyDeviceToHost, c->st) != cudaSuccess ||
      cudaStreamSynchronize(c->st) != cudaSuccess)
    return PFC_ECUDA;
  if (e && cudaMemsetAsync(c->err, 0, sizeof(int), c->st) != cudaSuccess) return PFC_ECUDA;
  return e;
}

// Forward pass on 3 FP64 feature planes (3 x n, planar); result in c->out (FP32).
void cnn_forward(Cnn* c, const double* feat) {
  const int nx = c->nx, ny = c->ny;
  const __nv_bfloat16* W = c->wbf;
  const float* th = c->theta;
  conv_fwd<3, 32, true, double, __nv_bfloat16>(nx, ny, feat, W + layer_offset(0), th + layer_offset(0) + 32 * 3 * 9,
                                               c->z[0], c->a[0], c->st);
  conv32_fwd_tc(nx, ny, c->a[0], W + layer_offset(1), th + layer_offset(1) + 32 * 32 * 9, c->z[1], c->a[1], c->err,
                c->st);
  conv32_fwd_tc(nx, ny, c->a[1], W + layer_offset(2), th + layer_offset(2) + 32 * 32 * 9, c->z[2], c->a[2], c->err,
                c->st);
  conv_fwd<32, 1, false, __nv_bfloat16, float>(nx, ny, c->a[2], W + layer_offset(3), th + layer_offset(3) + 32 * 9,
                                               c->out, nullptr, c->st);
}

// Loss and gradient (into c->grad) for one sample; loss sum of squares in c->red[0..nparts).
int cnn_backward(Cnn* c, const double* feat, const double* target, int* nparts) {
  const int nx = c->nx, ny = c->ny;
  const long long n = c->n;
  cnn_forward(c, feat);
  int blocks = (int)std::min<long long>((n + 255) / 256, 512);
  k_mse<<<blocks, 256, 0, c->st>>>(n, c->out, target, c->d1, c->red);
  count_launches(1);
  *nparts = blocks;
  const __nv_bfloat16* W = c->wbf;
  float* g = c->grad;
  // layer 3 (32 -> 1): d1 = dL/dz3 (1 x n)
  conv_bwd_weight<32, 1, __nv_bfloat16, float>(nx, ny, c->a[2], c->d1, c->partial, g + layer_offset(3), c->st);
  conv_bwd_data<32, 1, float>(nx, ny, c->d1, W + layer_offset(3), c->z[2], c->d2, c->st);
  // layer 2: d2 = dL/dz2
  conv_bwd_weight<32, 32, __nv_bfloat16, float>(nx, ny, c->a[1], c->d2, c->partial, g + layer_offset(2), c->st);
  conv_bwd_data<32, 32, float>(nx, ny, c->d2, W + layer_offset(2), c->z[1], c->d1, c->st);
  // layer 1: d1 = dL/dz1
  conv_bwd_weight<32, 32, __nv_bfloat16, float>(nx, ny, c->a[0], c->d1, c->partial, g + layer_offset(1), c->st);
  conv_bwd_data<32, 32, float>(nx, ny, c->d1, W + layer_offset(1), c->z[0], c->d2, c->st);
  // layer 0 (3 -> 32): d2 = dL/dz0
  conv_bwd_weight<3, 32, double, float>(nx, ny, feat, c->d2, c->partial, g + layer_offset(0), c->st);
  return cudaGetLastError() == cudaSuccess ? PFC_OK : PFC_ECUDA;
}

void cnn_adam(Cnn* c, float lr, int t) {
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.0f - powf(b1, (float)t), c2 = 1.0f - powf(b2, (float)t);
  k_adam<<<(kCnnParams + 255) / 256, 256, 0, c->st>>>(kCnnParams, c->theta, c->grad, c->m, c->v, lr, b1, b2, 1e-8f,
                                                       c1, c2, c->wbf);
  count_launches(1);
}

void cnn_refresh_bf16(Cnn* c) {
  k_to_bf16<<<(kCnnParams + 255) / 256, 256, 0, c->st>>>(kCnnParams, c->theta, c->wbf);
  count_launches(1);
}

void cnn_out_to_f64(Cnn* c, double* out) {
  k_f32_to_f64<<<(int)std::min<long long>((c->n + 255) / 256, 2048), 256, 0, c->st>>>(c->n, c->out, out);
  count_launches(1);
}

}  // namespace pfc

// ---------------------------------------------------------------- guess assembly kernels
namespace pfc {
namespace {

__global__ void k_cnn_features(long long n, const double* __restrict__ phin, const double* __restrict__ phinm1,
                               const double* __restrict__ sum, double r, double c2, double* __restrict__ feat) {
  const double mean = *sum / (double)n;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double p = phin[i];
    feat[i] = p - mean;
    feat[n + i] = r * (p - phinm1[i]);
    feat[2 * n + i] = c2;
  }
}

// delta = feat1 + s_out * out; per-CTA partial sums of delta
__global__ void k_cnn_delta(long long n, const double* __restrict__ feat, const float* __restrict__ out, double s_out,
                            double* __restrict__ delta, double* __restrict__ partial) {
  __shared__ double red[8];
  double s = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double d = feat[n + i] + s_out * (double)out[i];
    delta[i] = d;
    s += d;
  }
  for (int k = 16; k > 0; k >>= 1) s += __shfl_xor_sync(0xffffffffu, s, k);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += red[w];
    partial[blockIdx.x] = t;
  }
}

// out = base + delta - mean(delta)  (the guess keeps the mass of base)
__global__ void k_add_centered(long long n, const double* __restrict__ base, const double* __restrict__ delta,
                               const double* __restrict__ dsum, double* __restrict__ out) {
  const double mean = *dsum / (double)n;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = base[i] + (delta[i] - mean);
}

int gridfor(long long n) { return (int)std::min<long long>((n + 255) / 256, 512); }

__global__ void k_sum(long long n, const double* __restrict__ x, double* __restrict__ partial) {
  __shared__ double red[8];
  double s = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    s += x[i];
  for (int k = 16; k > 0; k >>= 1) s += __shfl_xor_sync(0xffffffffu, s, k);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += red[w];
    partial[blockIdx.x] = t;
  }
}

// target = (phi^{n+1} - phi^n - c1) / s_out
__global__ void k_cnn_target(long long n, const double* __restrict__ phinp1, const double* __restrict__ phin,
                             const double* __restrict__ feat, double s_out, double* __restrict__ target) {
  const double inv = 1.0 / s_out;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    target[i] = (phinp1[i] - phin[i] - feat[n + i]) * inv;
}

}  // namespace

void launch_sum(long long n, const double* x, double* partial, int* nparts, cudaStream_t st) {
  const int b = gridfor(n);
  k_sum<<<b, 256, 0, st>>>(n, x, partial);
  count_launches(1);
  *nparts = b;
}
void launch_cnn_target(long long n, const double* phinp1, const double* phin, const double* feat, double s_out,
                       double* target, cudaStream_t st) {
  k_cnn_target<<<gridfor(n), 256, 0, st>>>(n, phinp1, phin, feat, s_out, target);
  count_launches(1);
}

const float* cnn_output(const Cnn* c) { return c->out; }
int cnn_nx(const Cnn* c) { return c->nx; }
int cnn_ny(const Cnn* c) { return c->ny; }
cudaStream_t cnn_swap_stream(Cnn* c, cudaStream_t st) {
  const cudaStream_t old = c->st;
  c->st = st;
  return old;
}

void launch_cnn_features(long long n, const double* phin, const double* phinm1, const double* mass_sum, double r,
                         double c2, double* feat, cudaStream_t st) {
  k_cnn_features<<<gridfor(n), 256, 0, st>>>(n, phin, phinm1, mass_sum, r, c2, feat);
  count_launches(1);
}
void launch_cnn_delta(long long n, const double* feat, const float* out, double s_out, double* delta,
                      double* partial, int* nparts, cudaStream_t st) {
  const int b = gridfor(n);
  k_cnn_delta<<<b, 256, 0, st>>>(n, feat, out, s_out, delta, partial);
  count_launches(1);
  *nparts = b;
}
void launch_add_centered(long long n, const double* base, const double* delta, const double* dsum, double* out,
                         cudaStream_t st) {
  k_add_centered<<<gridfor(n), 256, 0, st>>>(n, base, delta, dsum, out);
  count_launches(1);
}

}  // namespace pfc

// ---------------------------------------------------------------- C ABI of the network
struct pfc_cnn {
  pfc::Cnn c;
};

extern "C" {

int pfc_cnn_param_count(void) { return pfc::kCnnParams; }

int pfc_cnn_workspace_size(int64_t nx, int64_t ny, size_t* bytes) {
  if (!bytes || nx < 1 || ny < 1 || nx > (1 << 16) || ny > (1 << 16)) return PFC_EINVAL;
  *bytes = pfc::cnn_workspace_bytes(nx * ny);
  return PFC_OK;
}

int pfc_cnn_create(int64_t nx, int64_t ny, void* ws, size_t bytes, void* stream, pfc_cnn** out) {
  if (!out || !ws || nx < 1 || ny < 1 || nx > (1 << 16) || ny > (1 << 16)) return PFC_EINVAL;
  if (((uintptr_t)ws & 255) != 0) return PFC_EINVAL;
  if (bytes < pfc::cnn_workspace_bytes(nx * ny)) return PFC_ENOMEM;
  pfc_cnn* h = new (std::nothrow) pfc_cnn();
  if (!h) return PFC_ENOMEM;
  h->c.nx = (int)nx;
  h->c.ny = (int)ny;
  h->c.n = nx * ny;
  h->c.st = (cudaStream_t)stream;
  pfc::cnn_bind(&h->c, ws);
  if (cudaMemsetAsync(ws, 0, pfc::cnn_workspace_bytes(nx * ny), h->c.st) != cudaSuccess) {
    delete h;
    return PFC_ECUDA;
  }
  *out = h;
  return PFC_OK;
}

void pfc_cnn_destroy(pfc_cnn* h) { delete h; }

int pfc_cnn_set_params(pfc_cnn* h, const float* theta) {
  if (!h || !theta) return PFC_EINVAL;
  pfc::Cnn& c = h->c;
  if (cudaMemcpyAsync(c.theta, theta, sizeof(float) * pfc::kCnnParams, cudaMemcpyHostToDevice, c.st) != cudaSuccess ||
      cudaMemsetAsync(c.m, 0, sizeof(float) * pfc::kCnnParams, c.st) != cudaSuccess ||
      cudaMemsetAsync(c.v, 0, sizeof(float) * pfc::kCnnParams, c.st) != cudaSuccess)
    return PFC_ECUDA;
  pfc::cnn_refresh_bf16(&c);
  return cudaStreamSynchronize(c.st) == cudaSuccess ? PFC_OK : PFC_ECUDA;
}

int pfc_cnn_get_params(pfc_cnn* h, float* theta) {
  if (!h || !theta) return PFC_EINVAL;
  pfc::Cnn& c = h->c;
  if (cudaMemcpyAsync(theta, c.theta, sizeof(float) * pfc::kCnnParams, cudaMemcpyDeviceToHost, c.st) != cudaSuccess ||
      cudaStreamSynchronize(c.st) != cudaSuccess)
    return PFC_ECUDA;
  return PFC_OK;
}

int pfc_cnn_forward(pfc_cnn* h, const double* feat, double* out) {
  if (!h || !feat || !out) return PFC_EINVAL;
  pfc::cnn_forward(&h->c, feat);
  pfc::cnn_out_to_f64(&h->c, out);
  if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(h->c.st) != cudaSuccess) return PFC_ECUDA;
  return pfc::cnn_status(&h->c);
}

static int cnn_loss(pfc_cnn* h, int nparts, double* loss) {
  double* part = (double*)malloc(sizeof(double) * nparts);
  if (!part) return PFC_ENOMEM;
  int rc = PFC_OK;
  if (cudaMemcpyAsync(part, h->c.red, sizeof(double) * nparts, cudaMemcpyDeviceToHost, h->c.st) != cudaSuccess ||
      cudaStreamSynchronize(h->c.st) != cudaSuccess)
    rc = PFC_ECUDA;
  if (!rc && loss) {
    double s = 0.0;
    for (int i = 0; i < nparts; ++i) s += part[i];
    *loss = s / (double)h->c.n;
  }
  free(part);
  return rc ? rc : pfc::cnn_status(&h->c);
}

int pfc_cnn_loss_grad(pfc_cnn* h, const double* feat, const double* target, double* loss, float* grad) {
  if (!h || !feat || !target) return PFC_EINVAL;
  int np = 0;
  int rc = pfc::cnn_backward(&h->c, feat, target, &np);
  if (rc) return rc;
  if (grad && cudaMemcpyAsync(grad, h->c.grad, sizeof(float) * pfc::kCnnParams, cudaMemcpyDeviceToHost, h->c.st) !=
                  cudaSuccess)
    return PFC_ECUDA;
  return cnn_loss(h, np, loss);
}

int pfc_cnn_sample(pfc_cnn* h, const double* phinm1, const double* phin, const double* phinp1, double r, double c2,
                   double s_out, double* feat, double* target) {
  if (!h || !phinm1 || !phin || !phinp1 || !feat || !target || !(s_out > 0.0)) return PFC_EINVAL;
  pfc::Cnn& c = h->c;
  int np = 0;
  pfc::launch_sum(c.n, phin, c.red, &np, c.st);
  pfc::launch_reduce(c.red, 1, np, c.red + 1000, c.st);
  pfc::launch_cnn_features(c.n, phin, phinm1, c.red + 1000, r, c2, feat, c.st);
  pfc::launch_cnn_target(c.n, phinp1, phin, feat, s_out, target, c.st);
  if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(c.st) != cudaSuccess) return PFC_ECUDA;
  return PFC_OK;
}

int pfc_cnn_train_step(pfc_cnn* h, const double* feat, const double* target, double lr, int t, double* loss) {
  if (!h || !feat || !target || t < 1 || !(lr > 0.0)) return PFC_EINVAL;
  int np = 0;
  int rc = pfc::cnn_backward(&h->c, feat, target, &np);
  if (rc) return rc;
  pfc::cnn_adam(&h->c, (float)lr, t);
  if (!loss) return cudaGetLastError() == cudaSuccess ? pfc::cnn_status(&h->c) : PFC_ECUDA;
  return cnn_loss(h, np, loss);
}

}  // extern "C"
