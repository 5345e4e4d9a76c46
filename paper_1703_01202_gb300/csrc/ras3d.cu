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
// brings into shared memory while the previous level is being solved.  Inside
// a level the entries are stored 16 bytes of a row at a time, row after row
// (entry o of the level's row i at ((o / E) n_l + i) E + o % E, E entries per
// 16 bytes, n_l rows), so that threads reading the same 16 bytes of
// consecutive rows read consecutive addresses.
//
// Two apply kernels give identical results.  The general one keeps the solve
// vector in a padded copy of the block in global memory (3-cell zero ring, so
// a neighbour outside the block reads zero and needs no bounds test).  The
// window kernel (FP32 solves, levels of at most 255 rows) keeps in shared memory
// only the levels a row can still read: an offset moves at most 21 levels
// (dc = -3), so 22 level slots of 256 floats hold every value the solve reads,
// row i of level l at place i of slot l mod 22, and each row's neighbours come
// with their places from host tables (255, a place kept zero, for a neighbour
// outside the block).  Both sum a row's 31 products as four partial sums of 8
// entries, (s0 + s1) + (s2 + s3): four independent chains for the FMA pipeline.
#include <cuda_bf16.h>

#include <algorithm>

#include "../../include/pfc.h"
#include "pfc_internal.cuh"
#include "pfc_tma.cuh"

namespace pfc {
namespace {

constexpr int NT = 256;

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

// o-th entry of the lexicographic (dc, db, da) list of the offsets with |d|_1 <= 3: 0..30 lower,
// 31 the centre, 32..62 upper
struct Off3 {
  int a, b, c;
};
__host__ __device__ constexpr Off3 off63(int o) {
  int idx = 0;
  for (int c = -3; c <= 3; ++c)
    for (int b = -3; b <= 3; ++b)
      for (int a = -3; a <= 3; ++a)
        if ((a < 0 ? -a : a) + (b < 0 ? -b : b) + (c < 0 ? -c : c) <= 3) {
          if (idx == o) return Off3{a, b, c};
          ++idx;
        }
  return Off3{0, 0, 0};
}

__device__ __forceinline__ void abc_of(int v, int* a, int* b, int* c) {
  *a = v & 1023;
  *b = (v >> 10) & 1023;
  *c = v >> 20;
}
// Periodic image of a block cell's coordinate (blocks never reach a second period).
__device__ __forceinline__ int wrap1(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }
__device__ __forceinline__ long long gidx(const Geo& g, const BlockDesc& B, int a, int b, int c) {
  return wrap1(B.x0 + a, g.nx) + (long long)g.nx * (wrap1(B.y0 + b, g.ny) + (long long)g.ny * wrap1(B.z0 + c, g.nz));
}
// Element of entry o of row i (of n) inside a level's factor data (16-byte units row after row).
template <typename TS>
__device__ __forceinline__ int lev_elem(int o, int i, int n) {
  constexpr int E = 16 / (int)sizeof(TS);
  return ((o / E) * n + i) * E + (o % E);
}

// Element i of an input stored as float pairs (the mixed path's Krylov basis): the float nearest
// their sum.
__device__ __forceinline__ float pair_sum(const double* __restrict__ r, long long i) {
  const float2 t = reinterpret_cast<const float2*>(r)[i];
  return __fadd_rn(t.x, t.y);
}

template <typename TC>
__device__ __forceinline__ TC fma_tc(TC a, TC b, TC c);
template <>
__device__ __forceinline__ float fma_tc<float>(float a, float b, float c) { return __fmaf_rn(a, b, c); }
template <>
__device__ __forceinline__ double fma_tc<double>(double a, double b, double c) { return __fma_rn(a, b, c); }

// Conversions between the solve type and FP64 by integer operations on the bit patterns: the
// hardware's FP64 <-> FP32 conversions run on GB300's FP64 pipe (1/64 of the FP32 rate), which the
// level sweeps would otherwise wait on.  Both round as the hardware does (to nearest, ties to
// even); zeros, subnormals, infinities and NaNs take the hardware conversion.
__device__ __forceinline__ float d2f_rn(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
  if ((b << 1) == 0ull) return __uint_as_float(sign);  // +-0
  const int e = (int)((b >> 52) & 0x7ffu) - 1023;
  if (e < -126 || e > 127) return (float)x;
  const unsigned long long m = b & 0xfffffffffffffull;
  unsigned f = sign | ((unsigned)(e + 127) << 23) | (unsigned)(m >> 29);
  const unsigned long long rem = m & 0x1fffffffull, half = 0x10000000ull;
  if (rem > half || (rem == half && (f & 1u))) ++f;  // a carry into the exponent is the correct rounding
  return __uint_as_float(f);
}
__device__ __forceinline__ double f2d_exact(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned ex = (u >> 23) & 0xffu;
  if (ex == 0u && (u & 0x7fffffu) == 0u) return __longlong_as_double((long long)((unsigned long long)u << 32));
  if (ex == 0u || ex == 255u) return (double)f;
  return __longlong_as_double((long long)(((unsigned long long)(u & 0x80000000u) << 32) |
                                          ((unsigned long long)(ex - 127 + 1023) << 52) |
                                          ((unsigned long long)(u & 0x7fffffu) << 29)));
}
template <typename TC>
__device__ __forceinline__ TC tc_of(double x) { return (TC)x; }
template <>
__device__ __forceinline__ float tc_of<float>(double x) { return d2f_rn(x); }
__device__ __forceinline__ double wide(double x) { return x; }
__device__ __forceinline__ double wide(float x) { return f2d_exact(x); }

// ILU(0) of one block, level by level (the rows of a level depend only on earlier levels), one
// warp per row.  Row i's 63 pattern entries sit in the warp's shared-memory row; the U parts
// (inverted diagonal, 31 upper entries) of finished rows sit in global memory by block cell, so
// that lane j fetches entry j of every lower neighbour's U part at once before the eliminations.
// Elimination by lower offset o1 (ascending, i.e. ascending neighbour row k = i + o1):
// l_ik = a_ik / u_kk, then lane j takes the update a_io3 -= l_ik u_kj of its upper entry j,
// o3 = o1 + o2(j) inside the pattern; the targets of one o1 are distinct, so one step is one
// warp-wide update.
template <typename TC>
__host__ __device__ constexpr int factor_threads() { return sizeof(TC) == 8 ? 512 : 1024; }

template <typename TC, typename TS>
__global__ void __launch_bounds__(factor_threads<TC>()) k_factor3d(Geo g, const BlockDesc* __restrict__ blocks,
                                                                   const double* __restrict__ q, double idt,
                                                                   const double* __restrict__ lin343, Ras3D R,
                                                                   int* __restrict__ status) {
  constexpr int FT = factor_threads<TC>(), FW = FT / 32;
  __shared__ int s_off[kNOff][3];
  __shared__ short s_idx[343];           // pattern index of offset (da, db, dc), -1 outside it
  __shared__ signed char s_tgt[31][32];  // o3 of lower offset o1 and U entry j, -1: none
  __shared__ double s_red[FW];
  __shared__ double s_sigma;
  __shared__ TC s_row[FW][64];
  const BlockDesc B = blocks[blockIdx.x];
  const Shape3 S = R.shapes[R.block_shape[blockIdx.x]];
  const int* rowabc = R.rowabc + S.row_off;
  const int* lev = R.lev_start + S.lev_off;
  TC* WU = (TC*)R.work + blockIdx.x * R.sWork;  // 32 entries per block cell
  TS* Lp = (TS*)R.Lp + blockIdx.x * R.sLU;
  TS* Up = (TS*)R.Up + blockIdx.x * R.sLU;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  for (int i = tid; i < 343; i += FT) s_idx[i] = -1;
  if (tid < kNOff) {
    const Off3 d = off63(tid);
    s_off[tid][0] = d.a;
    s_off[tid][1] = d.b;
    s_off[tid][2] = d.c;
  }
  __syncthreads();
  if (tid < kNOff) s_idx[(s_off[tid][2] + 3) * 49 + (s_off[tid][1] + 3) * 7 + s_off[tid][0] + 3] = (short)tid;
  __syncthreads();
  for (int e = tid; e < 31 * 32; e += FT) {
    const int o1 = e >> 5, j = e & 31;
    int t3 = -1;
    if (j > 0) {
      const int a = s_off[o1][0] + s_off[31 + j][0], b = s_off[o1][1] + s_off[31 + j][1],
                c = s_off[o1][2] + s_off[31 + j][2];
      if (abs(a) + abs(b) + abs(c) <= 3) t3 = s_idx[(c + 3) * 49 + (b + 3) * 7 + a + 3];
    }
    s_tgt[o1][j] = (signed char)t3;
  }
  const double ih2 = g.ih2;
  auto qat = [&](int a, int b, int c) { return q[gidx(g, B, a, b, c)]; };
  // Between mirror walls (Sec. 2) a row within 3 cells of a wall has stencil entries beyond it;
  // the Neumann Jacobian folds each onto the column of its mirror image (the image of global
  // cell -1 - i is i, of n + i is n - 1 - i), and A_k keeps the folded entries whose columns lie
  // in the block.
  auto mir = [](int i, int n) { return i < 0 ? -1 - i : (i >= n ? 2 * n - 1 - i : i); };
  auto wall_row = [&](int a, int b, int c) {
    return g.neumann && (B.x0 + a < 3 || B.x0 + a + 3 >= g.nx || B.y0 + b < 3 || B.y0 + b + 3 >= g.ny ||
                         B.z0 + c < 3 || B.z0 + c + 3 >= g.nz);
  };
  // entry of row (a, b, c) of the wall-folded J (without the diagonal's 1/dt and shift) in the
  // column of block cell (a2, b2, c2): the sum, in offset order, of the stencil entries whose
  // mirror images land there
  auto folded = [&](int a, int b, int c, int a2, int b2, int c2) {
    double v = 0.0;
    for (int d = 0; d < kNOff; ++d) {
      const int X = mir(B.x0 + a + s_off[d][0], g.nx), Y = mir(B.y0 + b + s_off[d][1], g.ny),
                Z = mir(B.z0 + c + s_off[d][2], g.nz);
      if (X - B.x0 != a2 || Y - B.y0 != b2 || Z - B.z0 != c2) continue;
      const int ad = abs(s_off[d][0]) + abs(s_off[d][1]) + abs(s_off[d][2]);
      double t = lin343[(s_off[d][2] + 3) * 49 + (s_off[d][1] + 3) * 7 + (s_off[d][0] + 3)];
      if (ad <= 1) t -= (ad == 0 ? -6.0 * ih2 : ih2) * q[X + (long long)g.nx * (Y + (long long)g.ny * Z)];
      v += t;
    }
    return v;
  };
  // Variable mobility (Sec. 3, M = 1 - s^2 at s = (Phi + phi^n)/2): row i of
  // J = I/dt - D_M (L_gamma/2 + Q) - B, with D_M the 7-point (div M grad)_d (edge M the average of
  // its end nodes) and B the term of dM/dPhi = -s.  mob_row gathers what the row's entries need
  // (the 7-point coefficients of D_M, q at the 7 nodes, B's three kinds of entry); mob_entry gives
  // the entry in the column of offset (da, db, dc), without 1/dt and the shift.
  const bool mob = R.mob_mu != nullptr;
  struct MobRow {
    double cf[7];  // D_M coefficients of the centre and of +x, -x, +y, -y, +z, -z
    double qn[7];  // q at those nodes
    double bd;     // -B(i, i)
    double bn[6];  // -B(i, i + n_k)
  };
  auto lgh = [&](int da, int db, int dc) -> double {  // L_gamma / 2 at offset (da, db, dc)
    const int ad = abs(da) + abs(db) + abs(dc), nz = (da != 0) + (db != 0) + (dc != 0);
    if (ad == 0) return g.c0 - 6.0 * ih2 + 21.0 * g.ih4;
    if (ad == 1) return ih2 - 6.0 * g.ih4;
    if (ad == 2) return nz == 1 ? 0.5 * g.ih4 : g.ih4;
    return 0.0;
  };
  constexpr int kNb[7][3] = {{0, 0, 0}, {1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1}};
  auto mob_row = [&](int a, int b, int c, MobRow* m) {
    double sn[7], mn[7], un[7];
#pragma unroll
    for (int k = 0; k < 7; ++k) {
      const long long i = gidx(g, B, a + kNb[k][0], b + kNb[k][1], c + kNb[k][2]);
      sn[k] = R.mob_s[i];
      un[k] = R.mob_mu[i];
      m->qn[k] = q[i];
      mn[k] = 1.0 - sn[k] * sn[k];
    }
    double c0 = 0.0, bd = 0.0;
#pragma unroll
    for (int k = 1; k < 7; ++k) {
      m->cf[k] = ih2 * 0.5 * (mn[0] + mn[k]);
      c0 -= m->cf[k];
      // the gradient of mu on the edge to neighbour k, oriented along +axis
      const double gk = (k & 1) ? (un[k] - un[0]) * ih2 : (un[0] - un[k]) * ih2;
      bd += (k & 1) ? 0.5 * gk : -0.5 * gk;
      m->bn[k - 1] = (k & 1) ? 0.5 * gk * sn[k] : -0.5 * gk * sn[k];
    }
    m->cf[0] = c0;
    m->bd = bd * sn[0];
  };
  auto mob_entry = [&](const MobRow& m, int da, int db, int dc) -> double {
    double v = 0.0;
#pragma unroll
    for (int k = 0; k < 7; ++k) {
      const int ea = da - kNb[k][0], eb = db - kNb[k][1], ec = dc - kNb[k][2];
      double t = lgh(ea, eb, ec);
      if (ea == 0 && eb == 0 && ec == 0) t += m.qn[k];
      v = fma(-m.cf[k], t, v);
    }
    const int ad = abs(da) + abs(db) + abs(dc);
    if (ad == 0) v += m.bd;
    if (ad == 1) {
      const int k = da == 1 ? 1 : da == -1 ? 2 : db == 1 ? 3 : db == -1 ? 4 : dc == 1 ? 5 : 6;
      v += m.bn[k - 1];
    }
    return v;
  };
  // sigma = shift * mean |a_ii| of the block matrix
  double dsum = 0.0;
  for (int r = tid; r < S.nrows; r += FT) {
    int a, b, c;
    abc_of(rowabc[r], &a, &b, &c);
    if (mob) {
      MobRow m;
      mob_row(a, b, c, &m);
      dsum += fabs(mob_entry(m, 0, 0, 0) + idt);
    } else {
      dsum += wall_row(a, b, c) ? fabs(folded(a, b, c, a, b, c) + idt)
                                : fabs(idt + lin343[171] + 6.0 * ih2 * qat(a, b, c));
    }
  }
  for (int o = 16; o > 0; o >>= 1) dsum += __shfl_xor_sync(0xffffffffu, dsum, o);
  if (lane == 0) s_red[wid] = dsum;
  __syncthreads();
  if (tid == 0) {
    double t = 0.0;
    for (int w = 0; w < FW; ++w) t += s_red[w];
    s_sigma = R.shift * t / (double)S.nrows;
  }
  __syncthreads();
  const double sigma = s_sigma;
  TC* row = s_row[wid];
  auto cell = [&](int a, int b, int c) { return a + S.bx * (b + S.by * c); };
  for (int l = 0; l < S.nlev; ++l) {
    const int r0 = lev[l], n = lev[l + 1] - r0;
    for (int i = wid; i < n; i += FW) {
      int a, b, c;
      abc_of(rowabc[r0 + i], &a, &b, &c);
      // row i of A_k + sigma I (zero outside the block): lane j builds entries j and 32 + j
      const bool wall = wall_row(a, b, c);  // the same for the whole warp
      MobRow mr;
      if (mob) mob_row(a, b, c, &mr);
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int o = lane + 32 * h;
        double v = 0.0;
        if (o < kNOff) {
          const int da = s_off[o][0], db = s_off[o][1], dc = s_off[o][2];
          const int a2 = a + da, b2 = b + db, c2 = c + dc;
          if (a2 >= 0 && a2 < S.bx && b2 >= 0 && b2 < S.by && c2 >= 0 && c2 < S.bz) {
            const int ad = abs(da) + abs(db) + abs(dc);
            if (mob) {
              v = mob_entry(mr, da, db, dc);
            } else if (wall) {
              v = folded(a, b, c, a2, b2, c2);
            } else {
              v = lin343[(dc + 3) * 49 + (db + 3) * 7 + (da + 3)];
              if (ad <= 1) v -= (ad == 0 ? -6.0 * ih2 : ih2) * qat(a2, b2, c2);
            }
            if (ad == 0) v += idt + sigma;
          }
        }
        row[o] = (TC)v;
      }
      // entry `lane` of the U part of every lower neighbour inside the block
      TC u[31];
#pragma unroll
      for (int o1 = 0; o1 < 31; ++o1) {
        const int a2 = a + s_off[o1][0], b2 = b + s_off[o1][1], c2 = c + s_off[o1][2];
        const bool in = a2 >= 0 && a2 < S.bx && b2 >= 0 && b2 < S.by && c2 >= 0;  // c2 <= c < bz
        u[o1] = in ? WU[(size_t)cell(a2, b2, c2) * 32 + lane] : (TC)0;
      }
      __syncwarp();
#pragma unroll
      for (int o1 = 0; o1 < 31; ++o1) {
        const int a2 = a + s_off[o1][0], b2 = b + s_off[o1][1], c2 = c + s_off[o1][2];
        if (!(a2 >= 0 && a2 < S.bx && b2 >= 0 && b2 < S.by && c2 >= 0)) continue;  // k outside: no entry
        TC lik = row[o1];
        if (lik == (TC)0) continue;  // the same value in every lane
        lik *= __shfl_sync(0xffffffffu, u[o1], 0);  // a_ik / u_kk
        const int t3 = s_tgt[o1][lane];
        __syncwarp();  // every lane has read a_ik
        if (lane == 0) row[o1] = lik;
        if (t3 >= 0) row[t3] = fma_tc<TC>(-lik, u[o1], row[t3]);
        __syncwarp();
      }
      TC d = row[31];
      if (d == (TC)0) {
        if (lane == 0) atomicExch(status, PFC_ESINGULAR);
        d = (TC)1;
      }
      const TC inv = (TC)1 / d;
      // the finished row: its U part for the rows below, L and U in the storage type
      const TC uj = lane == 0 ? inv : row[31 + lane];
      WU[(size_t)cell(a, b, c) * 32 + lane] = uj;
      Lp[(size_t)r0 * 32 + lev_elem<TS>(lane, i, n)] = to_store<TS>(lane < 31 ? (double)row[lane] : 0.0);
      Up[(size_t)r0 * 32 + lev_elem<TS>(lane, i, n)] = to_store<TS>((double)uj);
      __syncwarp();  // the warp's row buffer is free for its next row
    }
    __syncthreads();  // level done: its U parts are visible to the next level's warps
  }
}

// Levels of factor rows in flight per block (the ring's depth, at most kMaxStages3).
constexpr int kMaxStages3 = 8;

// General apply: the solve vector in a padded copy of the block in global memory, one thread per
// row.
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
  const int* rowabc = R.rowabc + S.row_off;
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
    int a, b, c;
    abc_of(rowabc[r], &a, &b, &c);
    const long long gi = gidx(g, B, a, b, c);
    Y[rowpad[r]] = R.pin ? (TC)pair_sum(rin, gi) : tc_of<TC>(rin[gi]);
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
      const int l = t, n = lev[l + 1] - lev[l];
      for (int i = threadIdx.x; i < n; i += NT) {
        const int p = rowpad[lev[l] + i];
        TC part[4];
#pragma unroll
        for (int qq = 0; qq < 4; ++qq) {  // entries 8 qq .. 8 qq + 7, as the window kernel sums them
          TC acc = qq == 0 ? Y[p] : (TC)0;
#pragma unroll
          for (int k = 0; k < 8; ++k) {
            const int o = 8 * qq + k;
            if (o < 31) acc = fma_tc<TC>(-from_store<TC, TS>(data[lev_elem<TS>(o, i, n)]), Y[p + s_poff[o]], acc);
          }
          part[qq] = acc;
        }
        Y[p] = (part[0] + part[1]) + (part[2] + part[3]);
      }
    } else {  // backward: x_r = (y_r - sum_upper u_ro x_(r+o)) / u_rr
      const int l = 2 * nl - 1 - t, n = lev[l + 1] - lev[l];
      for (int i = threadIdx.x; i < n; i += NT) {
        const int p = rowpad[lev[l] + i];
        TC part[4];
#pragma unroll
        for (int qq = 0; qq < 4; ++qq) {  // U entry e = 8 qq + k >= 1 is offset 31 + e; entry 0 is 1 / u_rr
          TC acc = qq == 0 ? Y[p] : (TC)0;
#pragma unroll
          for (int k = 0; k < 8; ++k) {
            const int e = 8 * qq + k;
            if (e >= 1)
              acc = fma_tc<TC>(-from_store<TC, TS>(data[lev_elem<TS>(e, i, n)]), Y[p + s_poff[31 + e]], acc);
          }
          part[qq] = acc;
        }
        Y[p] = ((part[0] + part[1]) + (part[2] + part[3])) * from_store<TC, TS>(data[lev_elem<TS>(0, i, n)]);
      }
    }
    __syncthreads();  // level done, stage free
    if (threadIdx.x == 0 && t + stages < total) issue(t + stages);
  }
  const double sc = rscale ? *rscale : 1.0;
  for (int r = threadIdx.x; r < S.nrows; r += NT) {  // extension (R_k^0)^T: core rows only
    int a, b, c;
    abc_of(rowabc[r], &a, &b, &c);
    if (a >= B.ox && a < B.ox + B.cx && b >= B.oy && b < B.oy + B.cy && c >= B.oz && c < B.oz + B.cz)
      z[gidx(g, B, a, b, c)] = sc * wide(Y[rowpad[r]]);
  }
}

// ---- Window apply (FP32 solves).  The solve of a row reads rows of the 21 levels before it
// (forward) or after it (backward) only, so 22 level slots hold every value it reads: level l in
// slot l mod kWinLevels, row i of the level at place i.  Each row's neighbours come with their
// places in their own levels (host tables, 255 for a neighbour outside the block: a place no
// level writes, zero from the start).  A slot is rewritten at level l + 22 only, after the last
// level that reads it; neither direction reads a slot it has not written in that direction.
constexpr int kWinLevels = 22;   // the level itself and the 21 an offset reaches
constexpr int kWinSlot = 256;    // floats per slot: places 0..254 and the zero place 255
constexpr int kWinFloats = kWinLevels * kWinSlot;

// Levels an offset moves: a + 3b + 7c.
__host__ __device__ constexpr int lev_shift(int o) { return off63(o).a + 3 * off63(o).b + 7 * off63(o).c; }

// Byte e of the 32 neighbour places of a row (two 16-byte words).
__device__ __forceinline__ int place_of(const uint4& p0, const uint4& p1, int e) {
  const uint4& p = e < 16 ? p0 : p1;
  const int k = e & 15;
  const uint32_t w = k < 4 ? p.x : k < 8 ? p.y : k < 12 ? p.z : p.w;
  return (int)((w >> (8 * (k & 3))) & 0xffu);
}

// acc[O / 8] -= cf[O] y(neighbour O) for the lower offsets O..30: the neighbour sits sft =
// -lev_shift(O) in 1..21 levels back, in slot (lm - sft) mod kWinLevels.  Four accumulators
// (entries 8q..8q+7): the general kernel's order.
template <int O>
__device__ __forceinline__ void win_lower(float* acc, const float* __restrict__ win, int lm, const uint4& p0,
                                          const uint4& p1, const float* cf) {
  if constexpr (O < 31) {
    constexpr int sft = -lev_shift(O);
    static_assert(sft >= 1 && sft < kWinLevels, "a lower offset reaches 1..21 levels back");
    const int sl = lm < sft ? lm - sft + kWinLevels : lm - sft;
    acc[O / 8] = __fmaf_rn(-cf[O], win[sl * kWinSlot + place_of(p0, p1, O)], acc[O / 8]);
    win_lower<O + 1>(acc, win, lm, p0, p1, cf);
  }
}
// acc[e / 8] -= cf[e] x(neighbour 31 + e) for the upper offsets, U entry e = O - 31 (cf[0] is the
// inverted diagonal).
template <int O>
__device__ __forceinline__ void win_upper(float* acc, const float* __restrict__ win, int lm, const uint4& p0,
                                          const uint4& p1, const float* cf) {
  if constexpr (O < 63) {
    constexpr int sft = lev_shift(O);
    static_assert(sft >= 1 && sft < kWinLevels, "an upper offset reaches 1..21 levels ahead");
    constexpr int e = O - 31;
    const int sl = lm + sft >= kWinLevels ? lm + sft - kWinLevels : lm + sft;
    acc[e / 8] = __fmaf_rn(-cf[e], win[sl * kWinSlot + place_of(p0, p1, e)], acc[e / 8]);
    win_upper<O + 1>(acc, win, lm, p0, p1, cf);
  }
}

// The 32 entries of row i (of n) of a level's factor data, as floats.
template <typename TS>
__device__ __forceinline__ void load_row(const TS* data, int i, int n, float* cf);
template <>
__device__ __forceinline__ void load_row<__nv_bfloat16>(const __nv_bfloat16* data, int i, int n, float* cf) {
  const uint4* u = reinterpret_cast<const uint4*>(data);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const uint4 v = u[k * n + i];
    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      cf[8 * k + 2 * j] = __uint_as_float(w[j] << 16);
      cf[8 * k + 2 * j + 1] = __uint_as_float(w[j] & 0xffff0000u);
    }
  }
}
template <>
__device__ __forceinline__ void load_row<float>(const float* data, int i, int n, float* cf) {
  const float4* u = reinterpret_cast<const float4*>(data);
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const float4 v = u[k * n + i];
    cf[4 * k] = v.x;
    cf[4 * k + 1] = v.y;
    cf[4 * k + 2] = v.z;
    cf[4 * k + 3] = v.w;
  }
}

// One thread per row of a level (levels of at most 255 rows), one barrier per level.  The small
// window lets several blocks share an SM.  The last thread keeps the copy ring (its warp has no
// row at levels of fewer than 225 rows).
template <typename TS>
__global__ void __launch_bounds__(NT) k_ras_apply3d_win(Geo g, const BlockDesc* __restrict__ blocks, Ras3D R,
                                                        const double* __restrict__ rin,
                                                        const double* __restrict__ rscale, double* __restrict__ z,
                                                        const int* __restrict__ skip, int* __restrict__ err,
                                                        int stages) {
  if (skip && *skip) return;
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ uint64_t bar[kMaxStages3];
  __shared__ int s_fail;
  const BlockDesc B = blocks[blockIdx.x];
  const Shape3 S = R.shapes[R.block_shape[blockIdx.x]];
  const int* rowabc = R.rowabc + S.row_off;
  const uint8_t* posL = R.posL + (size_t)S.row_off * 32;
  const uint8_t* posU = R.posU + (size_t)S.row_off * 32;
  const int* lev = R.lev_start + S.lev_off;
  float* ybuf = (float*)R.ypad + blockIdx.x * R.sPad;  // r, then the forward solution, row order
  const TS* Lp = (const TS*)R.Lp + blockIdx.x * R.sLU;
  const TS* Up = (const TS*)R.Up + blockIdx.x * R.sLU;
  const size_t fbytes = (size_t)R.max_level_rows * 32 * sizeof(TS);  // factor part of a stage
  const size_t sbytes = fbytes + (size_t)R.max_level_rows * 32;       // + the places
  float* win = reinterpret_cast<float*>(smem);
  unsigned char* stage_base = smem + (size_t)kWinFloats * sizeof(float);
  int* lev_s = reinterpret_cast<int*>(stage_base + (size_t)stages * sbytes);
  const int nl = S.nlev, total = 2 * nl, tid = threadIdx.x, ring = NT - 1;
  auto level_of = [&](int t) { return t < nl ? t : 2 * nl - 1 - t; };
  const int* lv = lev;  // the level starts: global memory until the shared copy is made
  auto issue = [&](int t) {  // level copy t (factors and places) into stage t % stages
    const int l = level_of(t), r0 = lv[l], n = lv[l + 1] - r0;
    const int st = t % stages;
    unsigned char* dst = stage_base + (size_t)st * sbytes;
    const uint32_t fb = (uint32_t)(n * 32 * sizeof(TS)), pb = (uint32_t)(n * 32);
    fence_proxy_async();
    mbar_expect_tx(&bar[st], fb + pb);
    bulk_g2s(dst, (t < nl ? Lp : Up) + (size_t)r0 * 32, fb, &bar[st]);
    bulk_g2s(dst + fbytes, (t < nl ? posL : posU) + (size_t)r0 * 32, pb, &bar[st]);
  };
  if (tid == ring) {
    s_fail = 0;
    for (int st = 0; st < stages; ++st) mbar_init(&bar[st], 1);
    fence_mbar_init();
    for (int t = 0; t < stages && t < total; ++t) issue(t);
  }
  // level starts in shared memory; the restriction R_k^delta r of every row, rounded to the solve
  // type, into ybuf (row order) with all loads in flight at once: no level waits on a gather
  for (int i = tid; i <= nl; i += NT) lev_s[i] = lev[i];
  for (int r = tid; r < S.nrows; r += NT) {
    int a, b, c;
    abc_of(rowabc[r], &a, &b, &c);
    const long long gi = gidx(g, B, a, b, c);
    ybuf[r] = R.pin ? pair_sum(rin, gi) : d2f_rn(rin[gi]);
  }
  for (int i = tid; i < kWinFloats; i += NT) win[i] = 0.f;
  __syncthreads();
  lv = lev_s;
  // The thread's row of a level (r < 0: none), the level's row count, its input (r of the
  // forward level, y of the backward one; both in ybuf) and its cell (backward, for the output).
  // Loads run ahead: the cell of level t + 2 and the input of level t + 1 are fetched while level t
  // is solved; the loop body runs three times per iteration with the rows' roles rotated, so no
  // register is moved while its load is in flight.
  struct Row {
    int r, n, abc;
    float val;
  };
  auto rows = [&](int t, Row& w) {
    const int l = level_of(t), r0 = lev_s[l];
    w.n = lev_s[l + 1] - r0;
    w.r = tid < w.n ? r0 + tid : -1;
    w.abc = (w.r >= 0 && t >= nl) ? rowabc[w.r] : 0;
  };
  auto input = [&](int t, Row& w) {  // not for the first backward level (its y is computed just before)
    if (w.r >= 0 && t != nl) w.val = ybuf[w.r];
  };
  const double sc = rscale ? *rscale : 1.0;
  auto level = [&](int t, Row& w0, Row& w1, Row& w2) -> bool {  // false: give up
    const int st = t % stages;
    const bool fwd = t < nl;
    if (t + 1 < total) input(t + 1, w1);
    if (t + 2 < total) rows(t + 2, w2);
    if (tid == ring && !mbar_wait_bounded(&bar[st], (uint32_t)((t / stages) & 1))) s_fail = 1;
    __syncthreads();  // level t - 1 done: its slot written, its stage free
    if (s_fail) {  // give up: record, drain the copies in flight (levels t .. last), leave
      if (tid == ring) {
        atomicExch(err, PFC_ETIMEOUT);
        const int last = t == 0 ? stages - 1 : t - 2 + stages;
        for (int u = t; u <= last && u < total; ++u)
          mbar_wait_bounded(&bar[u % stages], (uint32_t)((u / stages) & 1));
      }
      return false;
    }
    if (tid == ring && t >= 1 && t - 1 + stages < total) issue(t - 1 + stages);
    if (w0.r >= 0) {
      const unsigned char* data = stage_base + (size_t)st * sbytes;
      float cf[32];
      load_row<TS>(reinterpret_cast<const TS*>(data), tid, w0.n, cf);
      const uint4* pu = reinterpret_cast<const uint4*>(data + fbytes);
      const uint4 p0 = pu[tid], p1 = pu[w0.n + tid];
      const int lm = level_of(t) % kWinLevels;
      float acc[4] = {w0.val, 0.f, 0.f, 0.f};
      if (fwd) {  // y_r = b_r - sum_lower l_ro y_(r+o)
        win_lower<0>(acc, win, lm, p0, p1, cf);
        const float y = (acc[0] + acc[1]) + (acc[2] + acc[3]);
        win[lm * kWinSlot + tid] = y;
        ybuf[w0.r] = y;
        if (t == nl - 1) w1.val = y;  // the first backward level is this level: the same rows
      } else {  // x_r = (y_r - sum_upper u_ro x_(r+o)) / u_rr; the core goes out (R_k^0)^T
        win_upper<32>(acc, win, lm, p0, p1, cf);
        const float x = ((acc[0] + acc[1]) + (acc[2] + acc[3])) * cf[0];
        win[lm * kWinSlot + tid] = x;
        int a, b, c;
        abc_of(w0.abc, &a, &b, &c);
        if (a >= B.ox && a < B.ox + B.cx && b >= B.oy && b < B.oy + B.cy && c >= B.oz && c < B.oz + B.cz)
          z[gidx(g, B, a, b, c)] = sc * f2d_exact(x);
      }
    }
    return true;
  };
  Row ra{}, rb{}, rc{};
  rows(0, ra);
  input(0, ra);
  if (total > 1) rows(1, rb);
  for (int t = 0; t < total; t += 3) {
    if (!level(t, ra, rb, rc)) return;
    if (t + 1 < total && !level(t + 1, rb, rc, ra)) return;
    if (t + 2 < total && !level(t + 2, rc, ra, rb)) return;
  }
}

template <typename TC, typename TS>
void factor3d_dispatch(const Geo& g, const BlockDesc* blocks, int nblocks, const double* q, double idt,
                       const double* lin343, const Ras3D& R, int* status, cudaStream_t st) {
  k_factor3d<TC, TS><<<nblocks, factor_threads<TC>(), 0, st>>>(g, blocks, q, idt, lin343, R, status);
  count_launches(1);
}

template <typename TC, typename TS>
void apply3d_dispatch(const Geo& g, const BlockDesc* blocks, int nblocks, const Ras3D& R, const double* r,
                      const double* rscale, double* z, const int* skip, int* err, cudaStream_t st) {
  // Two levels in flight: the ring's shared memory comes out of the SM's L1, on which this
  // kernel's neighbour reads of the solve vector depend (deeper rings measured slower).
  const size_t stage = (size_t)R.max_level_rows * 32 * sizeof(TS);
  const int stages = 2;
  const size_t smem = stages * stage;
  cudaFuncSetAttribute(k_ras_apply3d<TC, TS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k_ras_apply3d<TC, TS><<<nblocks, NT, smem, st>>>(g, blocks, R, r, rscale, z, skip, err, stages);
  count_launches(1);
}

constexpr size_t kSmemCap = 227 * 1024 - 1024;  // dynamic shared memory a CTA may take (static use aside)

// Bytes of the window kernel's level-start table (padded to 16).
size_t win_lev_bytes(const Ras3D& R) { return ((size_t)(R.max_nlev + 1) * sizeof(int) + 15) / 16 * 16; }
size_t win_stage_bytes(const Ras3D& R) {
  return (size_t)R.max_level_rows * 32 * ((R.prec == PFC_BF16 ? 2 : 4) + 1);
}

// Stages of the window kernel's copy ring: as many as fit while three blocks share an SM (two
// levels at least), else while two do; 0 when the blocks' levels are too wide for it.
int win_stages(const Ras3D& R) {
  if (R.prec == PFC_F64 || R.max_level_rows > 255) return 0;
  const size_t fixed = (size_t)kWinFloats * sizeof(float) + win_lev_bytes(R), stage = win_stage_bytes(R);
  for (int per_sm = 3; per_sm >= 1; --per_sm) {
    // the SM's 228 KB of shared memory, less each CTA's 1 KB reserve and its static arrays
    const size_t cap = std::min<size_t>((size_t)228 * 1024 / per_sm - 1024 - 512, kSmemCap);
    if (fixed + 2 * stage <= cap) return (int)std::min<size_t>(kMaxStages3, (cap - fixed) / stage);
  }
  return 0;
}

template <typename TS>
void apply3d_win_dispatch(const Geo& g, const BlockDesc* blocks, int nblocks, const Ras3D& R, const double* r,
                          const double* rscale, double* z, const int* skip, int* err, cudaStream_t st) {
  const int stages = win_stages(R);
  const size_t smem = (size_t)kWinFloats * sizeof(float) + (size_t)stages * win_stage_bytes(R) + win_lev_bytes(R);
  cudaFuncSetAttribute(k_ras_apply3d_win<TS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k_ras_apply3d_win<TS><<<nblocks, NT, smem, st>>>(g, blocks, R, r, rscale, z, skip, err, stages);
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

bool apply3d_window_ok(const Ras3D& R) { return win_stages(R) >= 2; }

void launch_ras_apply3d(const Geo& g, const BlockDesc* blocks, int nblocks, const Ras3D& R, const double* r,
                        const double* rscale, double* z, const int* skip, int* err, cudaStream_t st) {
  if (R.window && R.prec == PFC_F32)
    apply3d_win_dispatch<float>(g, blocks, nblocks, R, r, rscale, z, skip, err, st);
  else if (R.window && R.prec == PFC_BF16)
    apply3d_win_dispatch<__nv_bfloat16>(g, blocks, nblocks, R, r, rscale, z, skip, err, st);
  else if (R.prec == PFC_F64)
    apply3d_dispatch<double, double>(g, blocks, nblocks, R, r, rscale, z, skip, err, st);
  else if (R.prec == PFC_F32)
    apply3d_dispatch<float, float>(g, blocks, nblocks, R, r, rscale, z, skip, err, st);
  else
    apply3d_dispatch<float, __nv_bfloat16>(g, blocks, nblocks, R, r, rscale, z, skip, err, st);
}

}  // namespace pfc
