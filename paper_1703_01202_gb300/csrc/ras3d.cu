// Restricted additive Schwarz preconditioner of Sec. 4 (left-RAS, Eq. ras) for
// 3D grids, with ILU(0) subdomain solves (the paper's 3D choice, Sec. 5.2,
// Table 1) on the 63-point block matrices A_k = R_k J R_k^T (Eq. Ak with the
// improved boundary condition).  ILU(0) of A_k breaks down at the 3D
// workload's time steps, so it factors A_k + sigma I with sigma a fixed
// fraction of the block's mean |a_ii| (the shifted incomplete factorisation).
//
// Rows are processed in wavefront levels: every lower offset (da, db, dc)
// lowers a + 3b + 7c, so all rows of one level depend only on earlier levels.
// One CTA owns one block.  Rows are stored in level order, 32 factor entries
// per row (L: offsets 0..30; U: the inverted diagonal then offsets 32..62),
// so each level's factor data is one contiguous chunk that a TMA bulk copy
// brings into shared memory while the previous level is being solved.  The
// solve vector lives in a padded copy of the block (3-cell zero ring), so a
// neighbour outside the block reads zero and needs no bounds test.
#include <cuda_bf16.h>

#include <algorithm>

#include "../../include/pfc.h"
#include "pfc_internal.cuh"
#include "pfc_tma.cuh"

namespace pfc {
namespace {

constexpr int NT = 256;

__device__ __forceinline__ int wrap(int i, int n) {
  i %= n;
  return i < 0 ? i + n : i;
}

template <typename T>
__device__ __forceinline__ T to_store(double v);
template <>
__device__ __forceinline__ double to_store<double>(double v) { return v; }
template <>
__device__ __forceinline__ float to_store<float>(double v) { return (float)v; }
template <>
__device__ __forceinline__ __nv_bfloat16 to_store<__nv_bfloat16>(double v) { return __float2bfloat16((float)v); }
template <typename TC, typename TS>
__device__ __forceinline__ TC from_store(TS v) { return (TC)v; }
template <>
__device__ __forceinline__ float from_store<float, __nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }

__device__ __forceinline__ void offset_of(int o, int* da, int* db, int* dc) {
  // o-th entry of the lexicographic (dc, db, da) list of |d|_1 <= 3
  int idx = 0;
  for (int c = -3; c <= 3; ++c)
    for (int b = -3; b <= 3; ++b)
      for (int a = -3; a <= 3; ++a) {
        if (abs(a) + abs(b) + abs(c) > 3) continue;
        if (idx == o) {
          *da = a;
          *db = b;
          *dc = c;
          return;
        }
        ++idx;
      }
}

template <typename TC, typename TS>
__global__ void __launch_bounds__(NT) k_factor3d(Geo g, const BlockDesc* __restrict__ blocks,
                                                 const double* __restrict__ q, double idt,
                                                 const double* __restrict__ lin343, Ras3D R,
                                                 int* __restrict__ status) {
  __shared__ int s_off[kNOff][3];
  __shared__ double s_red[NT / 32];
  __shared__ double s_sigma;
  extern __shared__ __align__(16) unsigned char smem[];
  TC* rowbuf = reinterpret_cast<TC*>(smem) + threadIdx.x * 64;  // this thread's working row
  const BlockDesc B = blocks[blockIdx.x];
  const Shape3 S = R.shapes[R.block_shape[blockIdx.x]];
  const int* rowpad = R.rowpad + S.row_off;
  const int* rowlin = R.rowlin + S.row_off;
  const int* rowof = R.rowof + S.pad_off;
  const int* lev = R.lev_start + S.lev_off;
  TC* W = (TC*)R.work + blockIdx.x * R.sWork;
  TS* Lp = (TS*)R.Lp + blockIdx.x * R.sLU;
  TS* Up = (TS*)R.Up + blockIdx.x * R.sLU;
  if (threadIdx.x < kNOff) offset_of(threadIdx.x, &s_off[threadIdx.x][0], &s_off[threadIdx.x][1], &s_off[threadIdx.x][2]);
  __syncthreads();
  const double ih2 = g.ih2;
  auto qat = [&](int a, int b, int c) {
    return q[wrap(B.x0 + a, g.nx) + (long long)g.nx * (wrap(B.y0 + b, g.ny) + (long long)g.ny * wrap(B.z0 + c, g.nz))];
  };
  // sigma = shift * mean |a_ii| of the block matrix
  double dsum = 0.0;
  for (int r = threadIdx.x; r < S.nrows; r += NT) {
    const int li = rowlin[r];
    const int a = li % S.bx, b = (li / S.bx) % S.by, c = li / (S.bx * S.by);
    dsum += fabs(idt + lin343[171] + 6.0 * ih2 * qat(a, b, c));
  }
  for (int o = 16; o > 0; o >>= 1) dsum += __shfl_xor_sync(0xffffffffu, dsum, o);
  if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = dsum;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < NT / 32; ++w) t += s_red[w];
    s_sigma = R.shift * t / (double)S.nrows;
  }
  __syncthreads();
  const double sigma = s_sigma;
  // rows of A_k + sigma I (zero outside the block)
  for (int r = threadIdx.x; r < S.nrows; r += NT) {
    const int li = rowlin[r];
    const int a = li % S.bx, b = (li / S.bx) % S.by, c = li / (S.bx * S.by);
    for (int o = 0; o < 64; ++o) {
      double v = 0.0;
      if (o < kNOff) {
        const int da = s_off[o][0], db = s_off[o][1], dc = s_off[o][2];
        const int a2 = a + da, b2 = b + db, c2 = c + dc;
        if (a2 >= 0 && a2 < S.bx && b2 >= 0 && b2 < S.by && c2 >= 0 && c2 < S.bz) {
          const int ad = abs(da) + abs(db) + abs(dc);
          v = lin343[(dc + 3) * 49 + (db + 3) * 7 + (da + 3)];
          if (ad <= 1) v -= (ad == 0 ? -6.0 * ih2 : ih2) * qat(a2, b2, c2);
          if (ad == 0) v += idt + sigma;
        }
      }
      W[(size_t)r * 64 + o] = (TC)v;
    }
  }
  __syncthreads();
  // ILU(0), row by row in level order: a_ik /= a_kk, a_ij -= a_ik a_kj on the pattern
  for (int l = 0; l < S.nlev; ++l) {
    for (int r = lev[l] + threadIdx.x; r < lev[l + 1]; r += NT) {
      for (int o = 0; o < 64; ++o) rowbuf[o] = W[(size_t)r * 64 + o];
      const int p = rowpad[r];
      for (int o1 = 0; o1 < 31; ++o1) {
        TC lik = rowbuf[o1];
        if (lik == (TC)0) continue;
        const int k = rowof[p + S.poff[o1]];
        if (k < 0) continue;
        const TC* Wk = W + (size_t)k * 64;
        lik *= Wk[31];  // inverted diagonal of the finished row k
        rowbuf[o1] = lik;
        const int cnt = R.upd_n[o1];
        for (int t = 0; t < cnt; ++t) {
          const int e = R.upd[o1 * 32 + t];
          rowbuf[e >> 8] -= lik * Wk[e & 255];
        }
      }
      TC d = rowbuf[31];
      if (d == (TC)0) {
        atomicExch(status, PFC_ESINGULAR);
        d = (TC)1;
      }
      rowbuf[31] = (TC)1 / d;
      for (int o = 0; o < 64; ++o) W[(size_t)r * 64 + o] = rowbuf[o];
    }
    __syncthreads();
  }
  // pack into the storage precision
  for (int r = threadIdx.x; r < S.nrows; r += NT) {
    const TC* Wr = W + (size_t)r * 64;
    for (int o = 0; o < 32; ++o) {
      Lp[(size_t)r * 32 + o] = to_store<TS>(o < 31 ? (double)Wr[o] : 0.0);
      Up[(size_t)r * 32 + o] = to_store<TS>((double)Wr[31 + o]);
    }
  }
}

// Levels of factor rows in flight per block (the ring's depth, at most kMaxStages3; the launch
// picks it, see apply3d_dispatch).
constexpr int kMaxStages3 = 8;

template <typename TC, typename TS>
__global__ void __launch_bounds__(NT) k_ras_apply3d(Geo g, const BlockDesc* __restrict__ blocks, Ras3D R,
                                                    const double* __restrict__ rin, const double* __restrict__ rscale,
                                                    double* __restrict__ z, const int* __restrict__ skip,
                                                    int* __restrict__ err, int stages) {
  if (skip && *skip) return;
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ uint64_t bar[kMaxStages3];
  __shared__ int s_poff[kNOff];
  __shared__ int s_fail;
  const BlockDesc B = blocks[blockIdx.x];
  const Shape3 S = R.shapes[R.block_shape[blockIdx.x]];
  const int* rowpad = R.rowpad + S.row_off;
  const int* rowlin = R.rowlin + S.row_off;
  const int* lev = R.lev_start + S.lev_off;
  TC* Y = (TC*)R.ypad + blockIdx.x * R.sPad;
  const TS* Lp = (const TS*)R.Lp + blockIdx.x * R.sLU;
  const TS* Up = (const TS*)R.Up + blockIdx.x * R.sLU;
  const size_t stage_elems = (size_t)R.max_level_rows * 32;
  TS* stage_base = reinterpret_cast<TS*>(smem);
  if (threadIdx.x < kNOff) s_poff[threadIdx.x] = S.poff[threadIdx.x];
  const int nl = S.nlev;
  const int total = 2 * nl;  // forward levels 0..nl-1, then backward levels nl-1..0
  auto issue = [&](int t) {  // level copy t into stage t % stages
    const int l = t < nl ? t : 2 * nl - 1 - t;
    const TS* src = (t < nl ? Lp : Up) + (size_t)lev[l] * 32;
    const uint32_t bytes = (uint32_t)((lev[l + 1] - lev[l]) * 32 * sizeof(TS));
    const int st = t % stages;
    fence_proxy_async();
    mbar_expect_tx(&bar[st], bytes);
    bulk_g2s(stage_base + st * stage_elems, src, bytes, &bar[st]);
  };
  if (threadIdx.x == 0) {
    s_fail = 0;
    for (int st = 0; st < stages; ++st) mbar_init(&bar[st], 1);
    fence_mbar_init();
    for (int t = 0; t < stages && t < total; ++t) issue(t);
  }
  // restriction R_k^delta into the padded block (the ring stays zero)
  for (int r = threadIdx.x; r < S.nrows; r += NT) {
    const int li = rowlin[r];
    const int a = li % S.bx, b = (li / S.bx) % S.by, c = li / (S.bx * S.by);
    Y[rowpad[r]] = (TC)rin[wrap(B.x0 + a, g.nx) +
                           (long long)g.nx * (wrap(B.y0 + b, g.ny) + (long long)g.ny * wrap(B.z0 + c, g.nz))];
  }
  __syncthreads();
  for (int t = 0; t < total; ++t) {
    const int st = t % stages;
    if (threadIdx.x == 0) {
      if (!mbar_wait_bounded(&bar[st], (uint32_t)((t / stages) & 1))) s_fail = 1;
    }
    __syncthreads();
    if (s_fail) {  // give up: record, drain the copies in flight (levels t .. t + stages - 1), leave
      if (threadIdx.x == 0) {
        atomicExch(err, PFC_ETIMEOUT);
        for (int u = t; u < t + stages && u < total; ++u)
          mbar_wait_bounded(&bar[u % stages], (uint32_t)((u / stages) & 1));
      }
      return;
    }
    const TS* data = stage_base + st * stage_elems;
    // every thread reads the stage the waiting thread saw complete
    if (t < nl) {  // forward: y_r = b_r - sum_lower l_ro y_(r+o)
      const int l = t;
      for (int r = lev[l] + threadIdx.x; r < lev[l + 1]; r += NT) {
        const TS* lr = data + (size_t)(r - lev[l]) * 32;
        const int p = rowpad[r];
        TC acc = Y[p];
#pragma unroll
        for (int o = 0; o < 31; ++o) acc -= from_store<TC, TS>(lr[o]) * Y[p + s_poff[o]];
        Y[p] = acc;
      }
    } else {  // backward: x_r = (y_r - sum_upper u_ro x_(r+o)) / u_rr
      const int l = 2 * nl - 1 - t;
      for (int r = lev[l] + threadIdx.x; r < lev[l + 1]; r += NT) {
        const TS* ur = data + (size_t)(r - lev[l]) * 32;
        const int p = rowpad[r];
        TC acc = Y[p];
#pragma unroll
        for (int o = 0; o < 31; ++o) acc -= from_store<TC, TS>(ur[1 + o]) * Y[p + s_poff[32 + o]];
        Y[p] = acc * from_store<TC, TS>(ur[0]);
      }
    }
    __syncthreads();  // level done, stage free
    if (threadIdx.x == 0 && t + stages < total) issue(t + stages);
  }
  const double sc = rscale ? *rscale : 1.0;
  for (int r = threadIdx.x; r < S.nrows; r += NT) {  // extension (R_k^0)^T: core rows only
    const int li = rowlin[r];
    const int a = li % S.bx, b = (li / S.bx) % S.by, c = li / (S.bx * S.by);
    if (a >= B.ox && a < B.ox + B.cx && b >= B.oy && b < B.oy + B.cy && c >= B.oz && c < B.oz + B.cz)
      z[wrap(B.x0 + a, g.nx) + (long long)g.nx * (wrap(B.y0 + b, g.ny) + (long long)g.ny * wrap(B.z0 + c, g.nz))] =
          sc * (double)Y[rowpad[r]];
  }
}

template <typename TC, typename TS>
void factor3d_dispatch(const Geo& g, const BlockDesc* blocks, int nblocks, const double* q, double idt,
                       const double* lin343, const Ras3D& R, int* status, cudaStream_t st) {
  const size_t smem = (size_t)NT * 64 * sizeof(TC);
  cudaFuncSetAttribute(k_factor3d<TC, TS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k_factor3d<TC, TS><<<nblocks, NT, smem, st>>>(g, blocks, q, idt, lin343, R, status);
  count_launches(1);
}

template <typename TC, typename TS>
void apply3d_dispatch(const Geo& g, const BlockDesc* blocks, int nblocks, const Ras3D& R, const double* r,
                      const double* rscale, double* z, const int* skip, int* err, cudaStream_t st) {
  // Two levels in flight.  Deeper rings were slower on GB300 (256^3, BF16: 3.3 ms per apply with 2
  // stages, 8.7 ms with 4, 6.4 ms with 7): the ring's shared memory comes out of the SM's L1, and
  // the solve vector's neighbour reads, which live in global memory, depend on L1 hits.
  const size_t stage = (size_t)R.max_level_rows * 32 * sizeof(TS);
  const int stages = 2;
  const size_t smem = stages * stage;
  cudaFuncSetAttribute(k_ras_apply3d<TC, TS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k_ras_apply3d<TC, TS><<<nblocks, NT, smem, st>>>(g, blocks, R, r, rscale, z, skip, err, stages);
  count_launches(1);
}

}  // namespace

void launch_factor3d(const Geo& g, const BlockDesc* blocks, int nblocks, const double* q, double idt,
                     const double* lin343, const Ras3D& R, int* status, cudaStream_t st) {
  if (R.prec == PFC_F64)
    factor3d_dispatch<double, double>(g, blocks, nblocks, q, idt, lin343, R, status, st);
  else if (R.prec == PFC_F32)
    factor3d_dispatch<float, float>(g, blocks, nblocks, q, idt, lin343, R, status, st);
  else
    factor3d_dispatch<float, __nv_bfloat16>(g, blocks, nblocks, q, idt, lin343, R, status, st);
}

void launch_ras_apply3d(const Geo& g, const BlockDesc* blocks, int nblocks, const Ras3D& R, const double* r,
                        const double* rscale, double* z, const int* skip, int* err, cudaStream_t st) {
  if (R.prec == PFC_F64)
    apply3d_dispatch<double, double>(g, blocks, nblocks, R, r, rscale, z, skip, err, st);
  else if (R.prec == PFC_F32)
    apply3d_dispatch<float, float>(g, blocks, nblocks, R, r, rscale, z, skip, err, st);
  else
    apply3d_dispatch<float, __nv_bfloat16>(g, blocks, nblocks, R, r, rscale, z, skip, err, st);
}

}  // namespace pfc
