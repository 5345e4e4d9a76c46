// Restricted additive Schwarz preconditioner of Sec. 4 (left-RAS, Eq. ras) for
// 2D grids: batched assembly + factorisation of every subdomain matrix A_k
// (Eq. Ak with the improved boundary condition: phi = 0 on the 3-layer ring,
// which makes A_k the principal submatrix of J on the block), and the batched
// apply z = sum_k (R_k^0)^T A_k^{-1} R_k^delta r.
//
// Design (GB300): A_k of a bx x by block ordered x-fastest is banded with
// half-bandwidth kl = 3 bx (the radius-3 stencil reaches 3 rows up/down).  LU
// with partial pivoting keeps L inside kl sub-diagonals and U inside 2 kl
// super-diagonals, so each block is factored by a sliding-window band LU: one
// CTA holds only the kl+1 active rows in shared memory (columns in a ring of
// RING slots), generating each new row of A_k on the fly from the stencil
// table and q, and streams L (one row of lrow >= kl multipliers per step) and U
// (one column of ucol >= 2kl+1 entries per step, diagonal stored inverted) out
// in the storage precision, pivots as 8-bit offsets.  This is the dense LU with
// partial pivoting of A_k restricted to its band: same pivots, same factors.
//
// The apply is a batched pair of banded triangular solves, one warp per block.
// The solve itself is a chain of n dependent steps, so the factor stream is
// decoupled from it: each warp runs a two-stage ring of TMA bulk copies
// (cp.async.bulk global->shared, completion on an mbarrier) that fetches the
// next chunk of L rows / U columns while the current chunk is consumed.  The
// kernel is bound by the factor bytes it streams from HBM.
#include <cuda_bf16.h>

#include "../../include/pfc.h"
#include "pfc_internal.cuh"
#include "pfc_tma.cuh"

namespace pfc {
namespace {

// Element i of the apply's input in the compute type; pin: r is stored as float pairs (the mixed
// path's Krylov basis), read as the float nearest their sum.
template <typename TC>
__device__ __forceinline__ TC ld_r(const double* __restrict__ r, long long i, int pin) {
  if (pin) {
    const float2 t = reinterpret_cast<const float2*>(r)[i];
    return (TC)__fadd_rn(t.x, t.y);
  }
  return (TC)r[i];
}

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

// Compute type -> storage type without a detour through double (double <-> float
// conversions run on GB300's FP64 pipe).
template <typename TS, typename TC>
__device__ __forceinline__ TS to_store_t(TC v) { return (TS)v; }
template <>
__device__ __forceinline__ __nv_bfloat16 to_store_t<__nv_bfloat16, float>(float v) { return __float2bfloat16(v); }

template <typename TC, typename TS>
__device__ __forceinline__ TC from_store(TS v) { return (TC)v; }
template <>
__device__ __forceinline__ float from_store<float, __nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }

__host__ __device__ inline size_t rup(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Four consecutive values from a 16-byte aligned shared-memory address.
__device__ __forceinline__ void load4(const float* p, float* out) {
  const float4 v = *reinterpret_cast<const float4*>(p);
  out[0] = v.x;
  out[1] = v.y;
  out[2] = v.z;
  out[3] = v.w;
}
__device__ __forceinline__ void load4(const double* p, double* out) {
  const double2 a = *reinterpret_cast<const double2*>(p), b = *reinterpret_cast<const double2*>(p + 2);
  out[0] = a.x;
  out[1] = a.y;
  out[2] = b.x;
  out[3] = b.y;
}

// Entry (r, c) of A_k = R_k J R_k^T, J = I/dt - (1/2) Delta_d L_gamma - Delta_d diag(q) (Eq. Jacobi).
// qb: q on the block (block-local order), lin: the 7x7 table of -(1/2) Delta_d L_gamma.
__device__ __forceinline__ double jac_entry(int bx, double ih2, const double* qb, double idt, const double* lin,
                                            int r, int c) {
  const int ar = r % bx, br = r / bx, ac = c % bx, bc = c / bx;
  const int dx = ac - ar, dy = bc - br;
  const int ad = abs(dx) + abs(dy);
  if (ad > 3) return 0.0;
  double v = lin[(dy + 3) * 7 + (dx + 3)];
  if (ad <= 1) v -= (ad == 0 ? -4.0 * ih2 : ih2) * qb[c];
  if (ad == 0) v += idt;
  return v;
}

// Entry (r, c) of A_k with variable mobility (the principal submatrix of J of the mobility
// form): J = I/dt - D_M K - B, K = (1/2) L_gamma + diag q, D_M = (div M grad)_d with M = 1 - s^2
// averaged onto edges, B = (div (-s v) grad)_d mu (derivative of M_d).  Row r collects, over
// the 4 edges (r, nb): M_e (K(nb, c) - K(r, c)) for D_M K, and the two ends' dM terms for B.
// sx, mx: s and mu on the block plus a one-cell ring ((bx+2) x (by+2), x fastest); l13: the 5 x 5
// table of (1/2) L_gamma (offset (dx, dy) at (dy+2)*5 + dx+2).
__device__ __forceinline__ double jac_entry_mob(int bx, int by, double ih2, const double* qb, double idt,
                                                const double* l13, const double* sx, const double* mx, int r,
                                                int c) {
  const int ar = r % bx, br = r / bx, ac = c % bx, bc = c / bx;
  const int dx = ac - ar, dy = bc - br;
  if (abs(dx) + abs(dy) > 3) return 0.0;
  const int ex = bx + 2;
  auto ext = [&](int a, int b) { return (b + 1) * ex + (a + 1); };
  auto K = [&](int a, int b) -> double {  // K(node (a, b), c): (1/2) L_gamma offset + q on the diagonal
    const int ox = ac - a, oy = bc - b;
    if (abs(ox) + abs(oy) > 2) return 0.0;
    double v = l13[(oy + 2) * 5 + (ox + 2)];
    if (ox == 0 && oy == 0) v += qb[c];
    return v;
  };
  const double sr = sx[ext(ar, br)], mur = mx[ext(ar, br)];
  const double Mr = 1.0 - sr * sr, Kr = K(ar, br);
  const int nbx[4] = {-1, 1, 0, 0}, nby[4] = {0, 0, -1, 1};
  double dmk = 0.0, bdiag = 0.0, boff = 0.0;
  for (int e = 0; e < 4; ++e) {
    const int na = ar + nbx[e], nb = br + nby[e];
    const double sn = sx[ext(na, nb)], mun = mx[ext(na, nb)];
    const double Me = 0.5 * (Mr + (1.0 - sn * sn));
    dmk += Me * (K(na, nb) - Kr);
    bdiag += mun - mur;
    if (na == ac && nb == bc) boff += sn * (mun - mur);
  }
  double v = -ih2 * dmk + 0.5 * ih2 * boff;
  if (dx == 0 && dy == 0) v += idt + 0.5 * ih2 * sr * bdiag;
  return v;
}

// Entry (r, c) of A_k between Neumann walls: J of the evenly extended grid summed over the mirror
// images of column c's cell (x images jx, -1 - jx, 2 nx - 1 - jx; likewise in y) that lie within
// the radius-3 stencil of row r's cell; q of an image is q of the cell.  An image is never
// nearer than the cell itself, so the band of A_k is that of the periodic case.
__device__ __forceinline__ double jac_entry_neu(const BlockDesc& B, const Geo& g, double ih2, const double* qb,
                                                double idt, const double* lin, int r, int c) {
  const int bx = B.bx;
  const int ar = r % bx, br = r / bx, ac = c % bx, bc = c / bx;
  if (abs(ac - ar) + abs(bc - br) > 3) return 0.0;
  const int gx = B.x0 + ar, gy = B.y0 + br, jx = B.x0 + ac, jy = B.y0 + bc;
  const int xs[3] = {jx - gx, -1 - jx - gx, 2 * g.nx - 1 - jx - gx};
  const int ys[3] = {jy - gy, -1 - jy - gy, 2 * g.ny - 1 - jy - gy};
  double v = 0.0;
  for (int iy = 0; iy < 3; ++iy)
    for (int ix = 0; ix < 3; ++ix) {
      const int dx = xs[ix], dy = ys[iy], ad = abs(dx) + abs(dy);
      if (ad > 3) continue;
      v += lin[(dy + 3) * 7 + (dx + 3)];
      if (ad <= 1) v -= (ad == 0 ? -4.0 * ih2 : ih2) * qb[c];
    }
  if (r == c) v += idt;
  return v;
}

template <typename TC, typename TS, int RING>
__global__ void __launch_bounds__(256) k_factor2d(Geo g, const BlockDesc* __restrict__ blocks,
                                                  const double* __restrict__ q, double idt,
                                                  const double* __restrict__ lin, FactorStore fs,
                                                  int* __restrict__ status, const double* __restrict__ idt_dev) {
  if (idt_dev) idt = *idt_dev;  // a captured step graph: this step's 1/dt
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ TC s_dinv;
  const BlockDesc B = blocks[blockIdx.x];
  const int n = B.bx * B.by;
  const int kl = min(3 * B.bx, n - 1);
  const int ku2 = min(2 * kl, n - 1);
  const int W = kl + 1;
  const int lrow = fs.lrow, ucol = fs.ucol;
  double* qb = reinterpret_cast<double*>(smem);  // q on the block, block-local order
  double* lin_s = qb + fs.n_max;                 // 7 x 7 stencil table
  constexpr int PM = RING / 2 - 1;               // window positions (<= RING/2 of them) map by pos & PM
  // Row stride RS = RING + 1 (odd): the column walks (pivot search, multipliers, zeroing) touch
  // one entry per row and would otherwise put every lane on the same shared-memory bank.
  constexpr int RS = RING + 1;
  // lv / roff 16-byte aligned so that the rank-1 update can read them 4 at a time
  TC* lv = reinterpret_cast<TC*>(smem + rup((size_t)(fs.n_max + 49) * sizeof(double), 16));  // multipliers
  TC* uv = lv + RING;                             // U row of the current step
  int* slot = reinterpret_cast<int*>(uv + RING);  // window position & PM -> row slot
  int* roff = slot + RING / 2;                    // row offsets (slot * RS) of positions k+1..k+kl
  TC* A = reinterpret_cast<TC*>(roff + RING / 2);  // W rows x RING column slots, stride RS
  TS* L = (TS*)fs.L + blockIdx.x * fs.strideL;
  TS* U = (TS*)fs.U + blockIdx.x * fs.strideU;
  uint8_t* piv = fs.piv + blockIdx.x * fs.strideP;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int bx = B.bx, by = B.by;
  const double ih2 = g.ih2;
  const float inv_bx = 1.0f / (float)bx;

  // variable mobility: s and mu on the block plus a ring, the (1/2) L_gamma table (after A)
  const bool mob = fs.mob_mu != nullptr;
  double* sx = reinterpret_cast<double*>(
      smem + rup((size_t)(reinterpret_cast<unsigned char*>(A + (size_t)W * RS) - smem), 16));
  double* mx = sx + fs.ext_max;
  double* l13 = mx + fs.ext_max;
  for (int t = tid; t < n; t += nt)
    qb[t] = q[wrap(B.x0 + t % bx, g.nx) + (long long)g.nx * wrap(B.y0 + t / bx, g.ny)];
  for (int t = tid; t < 49; t += nt) lin_s[t] = lin[t];
  for (int w = tid; w < W; w += nt) slot[w] = w;
  if (mob) {
    const int ex = bx + 2, ne = ex * (by + 2);
    for (int t = tid; t < ne; t += nt) {
      const long long gi = wrap(B.x0 - 1 + t % ex, g.nx) + (long long)g.nx * wrap(B.y0 - 1 + t / ex, g.ny);
      sx[t] = fs.mob_s[gi];
      mx[t] = fs.mob_mu[gi];
    }
    if (tid < 25) {  // (1/2) L_gamma = (1/2) [(1 - gamma) + 2 Delta_d + Delta_d^2]
      const int ox = tid % 5 - 2, oy = tid / 5 - 2, ad = abs(ox) + abs(oy);
      const double ih4 = ih2 * ih2;
      double v = 0.0;
      if (ad == 0) v = 0.5 * ((1.0 - g.gamma) - 8.0 * ih2 + 20.0 * ih4);
      else if (ad == 1) v = 0.5 * (2.0 * ih2 - 8.0 * ih4);
      else if (ad == 2) v = (ox != 0 && oy != 0) ? ih4 : 0.5 * ih4;
      l13[tid] = v;
    }
  }
  __syncthreads();
  const bool neu = g.neumann != 0;
  for (int idx = tid; idx < W * RING; idx += nt) {
    const int pos = idx / RING, col = idx - pos * RING;
    A[pos * RS + col] = (pos < n && col < n)
                            ? (TC)(mob   ? jac_entry_mob(bx, by, ih2, qb, idt, l13, sx, mx, pos, col)
                                   : neu ? jac_entry_neu(B, g, ih2, qb, idt, lin_s, pos, col)
                                         : jac_entry(bx, ih2, qb, idt, lin_s, pos, col))
                            : (TC)0;
  }
  __syncthreads();

  for (int k = 0; k < n; ++k) {
    const int kw = k & (RING - 1);
    const int last = min(k + kl, n - 1);
    if (tid < 32) {  // partial pivoting: largest |a_ik| over the window, first on ties
      TC best = (TC)-1;
      int bp = k;
      for (int pos = k + tid; pos <= last; pos += 32) {
        const TC v = abs(A[slot[pos & PM] * RS + kw]);
        if (v > best) {
          best = v;
          bp = pos;
        }
      }
      for (int o = 16; o > 0; o >>= 1) {
        const TC ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int op = __shfl_xor_sync(0xffffffffu, bp, o);
        if (ob > best || (ob == best && op < bp)) {
          best = ob;
          bp = op;
        }
      }
      if (tid == 0) {
        const int sk = slot[k & PM], sp = slot[bp & PM];
        slot[k & PM] = sp;
        slot[bp & PM] = sk;
        piv[k] = (uint8_t)(bp - k);
        TC d = A[sp * RS + kw];
        if (d == (TC)0) {
          atomicExch(status, PFC_ESINGULAR);
          d = (TC)1;
        }
        s_dinv = (TC)1 / d;
      }
    }
    __syncthreads();
    const int sk = slot[k & PM];
    const TC dinv = s_dinv;
    for (int i = tid; i < lrow; i += nt) {
      const int pos = k + 1 + i;
      TC l = (TC)0;
      if (i < kl) {
        const int off = slot[pos & PM] * RS;
        roff[i] = off;
        if (pos < n) l = A[off + kw] * dinv;
        lv[i] = l;
      }
      L[(size_t)k * lrow + i] = to_store_t<TS>(l);
    }
    for (int j = tid; j < ucol; j += nt) {
      const int col = k + j;
      TC u = (TC)0;
      if (j <= ku2 && col < n) {
        u = A[sk * RS + (col & (RING - 1))];
        U[(size_t)col * ucol + j] = to_store_t<TS>((TC)(j == 0 ? dinv : u));
      }
      if (j <= ku2) uv[j] = u;
    }
    // U column k's entries above the band (j > ku2) stay zero for the bulk copies
    for (int j = ku2 + 1 + tid; j < ucol; j += nt) U[(size_t)k * ucol + j] = to_store_t<TS>((TC)0);
    __syncthreads();
    // rank-1 update of the active window; multipliers and row offsets are read four at a time
    // (16-byte loads), so shared memory carries about half the traffic of one load per row
    // threads split the (row, column) rectangle: 128 column lanes x nt / 128 row bands
    const int rows = min(kl, n - 1 - k);
    const int bands = nt / 128, band = tid / 128;
    const int per = ((rows + bands - 1) / bands + 3) & ~3;  // rows per band, a multiple of 4
    const int i0 = min(rows, band * per), i1 = min(rows, i0 + per);
    const int i4 = i0 + ((i1 - i0) & ~3);
    for (int j = 1 + (tid & 127); j <= ku2; j += 128) {
      const TC u = uv[j];
      if (u != (TC)0 && k + j < n) {
        const int cw = (k + j) & (RING - 1);
        for (int i = i0; i < i4; i += 4) {
          const int4 o = *reinterpret_cast<const int4*>(roff + i);
          TC l[4];
          load4(lv + i, l);
          A[o.x + cw] -= l[0] * u;
          A[o.y + cw] -= l[1] * u;
          A[o.z + cw] -= l[2] * u;
          A[o.w + cw] -= l[3] * u;
        }
        for (int i = i4; i < i1; ++i) A[roff[i] + cw] -= lv[i] * u;
      }
    }
    // the column entering the band must start at zero in the rows that stay
    const int cz = (k + 1 + ku2) & (RING - 1);
    for (int i = tid; i < kl; i += nt) A[roff[i] + cz] = (TC)0;
    // next row of A_k enters the slot the pivot row leaves
    const int rnew = k + 1 + kl;
    if (rnew < n) {
      if (tid == 0) slot[rnew & PM] = sk;
      TC* row = &A[sk * RS];
      const int base = k + 1;
      const int ar = rnew % bx, br = rnew / bx;
      for (int t = tid; t < RING; t += nt) {
        const int col = base + ((t - base) & (RING - 1));
        TC v = (TC)0;
        if (col < n && mob) {
          v = (TC)jac_entry_mob(bx, by, ih2, qb, idt, l13, sx, mx, rnew, col);
        } else if (col < n && neu) {
          v = (TC)jac_entry_neu(B, g, ih2, qb, idt, lin_s, rnew, col);
        } else if (col < n) {
          if (bx >= 7) {  // col - rnew = dx + bx dy has a unique split with |dx| <= 3
            const int d = col - rnew;
            const int dy = __float2int_rn((float)d * inv_bx);
            const int dx = d - dy * bx;
            const int ad = abs(dx) + abs(dy);
            if (ad <= 3 && ar + dx >= 0 && ar + dx < bx && br + dy >= 0 && br + dy < by) {
              double e = lin_s[(dy + 3) * 7 + (dx + 3)];
              if (ad <= 1) e -= (ad == 0 ? -4.0 * ih2 : ih2) * qb[col];
              if (ad == 0) e += idt;
              v = (TC)e;
            }
          } else {
            v = (TC)jac_entry(bx, ih2, qb, idt, lin_s, rnew, col);
          }
        }
        row[t] = v;
      }
    }
    __syncthreads();
  }
}

// ---- Column-owned band LU (compute type float, kl <= 63).
//
// The same elimination as k_factor2d (same pivots, same multipliers, same rank-1
// updates with the same operations, so the same factors), arranged by columns:
// thread t of the 128 owns ring column slot t and keeps that column's entries for
// the 64 row slots of the window in its own row of shared memory (68 floats apart,
// so 16-byte accesses of 8 neighbouring threads hit distinct banks).  Per step warp
// 0 reads column k, picks the pivot and forms the multipliers; every thread then
// updates its column with 16-byte loads and stores (one load of its entries, one
// of the multipliers, four FMAs, one store per four rows).  New rows come from
// per-column tables of the q-dependent entries (evaluated in double as jac_entry
// does, then rounded).
constexpr int kColRows = 64;     // row slots (window of kl + 1 <= 64 rows)
constexpr int kColRing = 128;    // column slots (2 kl + 2 <= 128)
constexpr int kColStride = 68;   // floats per column row in shared memory

size_t factor_col_smem_bytes(int n_max) {
  const size_t cols = (size_t)kColRing * kColStride * sizeof(float);
  const size_t qtmp = (size_t)n_max * sizeof(double);  // q on the block, only while the tables are made
  return (cols > qtmp ? cols : qtmp) + (size_t)n_max * 5 * sizeof(float) + 49 * sizeof(double);
}

template <typename TS>
__global__ void __launch_bounds__(kColRing) k_factor2d_col(Geo g, const BlockDesc* __restrict__ blocks,
                                                         const double* __restrict__ q, double idt,
                                                         const double* __restrict__ lin, FactorStore fs,
                                                         int* __restrict__ status,
                                                         const double* __restrict__ idt_dev) {
  if (idt_dev) idt = *idt_dev;  // a captured step graph: this step's 1/dt
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ __align__(16) float lslot[kColRows];  // multipliers by row slot (0 off the window)
  __shared__ int slot[kColRows];                   // window position & 63 -> row slot
  __shared__ int posof[kColRows];                  // row slot -> window position (-1: free)
  __shared__ float linf[49];                       // the stencil table, rounded
  __shared__ float s_dinv;
  __shared__ int s_sk;
  constexpr int PM = kColRows - 1;
  const BlockDesc B = blocks[blockIdx.x];
  const int n = B.bx * B.by, bx = B.bx;
  const int kl = min(3 * bx, n - 1);
  const int ku2 = min(2 * kl, n - 1);
  const int W = kl + 1;
  // A row enters the slot its pivot row leaves, so only row slots 0 .. W - 1 ever hold rows: the
  // column updates stop at W rounded up to whole 16-byte groups.
  const int Wp = (W + 3) & ~3;
  const int lrow = fs.lrow, ucol = fs.ucol;
  const size_t cols = (size_t)kColRing * kColStride * sizeof(float);
  const size_t qtmp = (size_t)fs.n_max * sizeof(double);
  float* colA = reinterpret_cast<float*>(smem);  // column slot t: colA[t * kColStride + row slot]
  double* qb = reinterpret_cast<double*>(smem);  // q on the block (before the columns are filled)
  double* lin_s = reinterpret_cast<double*>(smem + (cols > qtmp ? cols : qtmp));  // 7 x 7 stencil table
  float* tabq = reinterpret_cast<float*>(lin_s + 49);                            // per column: 5 entries
  TS* L = (TS*)fs.L + blockIdx.x * fs.strideL;
  TS* U = (TS*)fs.U + blockIdx.x * fs.strideU;
  uint8_t* piv = fs.piv + blockIdx.x * fs.strideP;
  const int t = threadIdx.x, lane = t & 31;
  const double ih2 = g.ih2;

  for (int i = t; i < n; i += kColRing)
    qb[i] = q[wrap(B.x0 + i % bx, g.nx) + (long long)g.nx * wrap(B.y0 + i / bx, g.ny)];
  for (int i = t; i < 49; i += kColRing) {
    lin_s[i] = lin[i];
    linf[i] = (float)lin[i];
  }
  if (t < kColRows) {
    slot[t] = t;
    posof[t] = t < W ? t : -1;
  }
  __syncthreads();
  for (int i = t; i < n; i += kColRing) {  // the entries jac_entry gives for ad <= 1, same expressions
    const int dirs[5] = {24, 23, 25, 17, 31};  // (dx, dy) = (0,0), (-1,0), (1,0), (0,-1), (0,1)
#pragma unroll
    for (int d = 0; d < 5; ++d) {
      double e = lin_s[dirs[d]];
      e -= (d == 0 ? -4.0 * ih2 : ih2) * qb[i];
      if (d == 0) e += idt;
      tabq[5 * i + d] = (float)e;
    }
  }
  __syncthreads();  // qb is dead: its bytes become the columns
  // entry (row r, column col) of A_k from the tables: (ar, br), (ac, bc) block coordinates
  auto entry = [&](int ar, int br, int ac, int bc, int col) -> float {
    const int dx = ac - ar, dy = bc - br, ad = abs(dx) + abs(dy);
    if (ad > 3) return 0.0f;
    if (ad == 0) return tabq[5 * col];
    if (ad == 1) return tabq[5 * col + (dx == -1 ? 1 : dx == 1 ? 2 : dy == -1 ? 3 : 4)];
    return linf[(dy + 3) * 7 + dx + 3];
  };
  float* mine = colA + (size_t)t * kColStride;
  int ac = t % bx, bc = t / bx;  // block coordinates of this thread's column (t, then t + 128, ...)
  for (int r = 0; r < kColRows; ++r)
    mine[r] = (r < W && r < n && t < n) ? entry(r % bx, r / bx, ac, bc, t) : 0.0f;
  const int da = kColRing % bx, db = kColRing / bx;
  int ar = (kl + 1) % bx, br = (kl + 1) / bx;  // block coordinates of the entering row
  __syncthreads();

  for (int k = 0; k < n; ++k) {
    const int kw = k & (kColRing - 1);
    const int last = min(k + kl, n - 1);
    if (t < 32) {  // partial pivoting: largest |a_ik| over the window, first on ties
      const float* colk = colA + (size_t)kw * kColStride;
      // lane candidates: positions k + lane and k + lane + 32 (window <= 64 rows); |a| compares as
      // its bit pattern, a warp max of the bits and two ballots give the first maximal position
      const int p0 = k + lane, p1 = k + lane + 32;
      const unsigned b0 = p0 <= last ? __float_as_uint(fabsf(colk[slot[p0 & PM]])) : 0u;
      const unsigned b1 = p1 <= last ? __float_as_uint(fabsf(colk[slot[p1 & PM]])) : 0u;
      const bool second = b1 > b0 && p1 <= last;  // ties keep the earlier position
      const unsigned bb = second ? b1 : b0;
      const unsigned mx = __reduce_max_sync(0xffffffffu, bb);
      const unsigned first_set = __ballot_sync(0xffffffffu, bb == mx && !second && p0 <= last);
      const unsigned second_set = __ballot_sync(0xffffffffu, bb == mx && second);
      const int bp = first_set ? k + __ffs(first_set) - 1 : k + 32 + __ffs(second_set) - 1;
      const int sk0 = slot[k & PM], sp = slot[bp & PM];
      const float d0 = colk[sp];
      const float dinv = 1.0f / (d0 == 0.0f ? 1.0f : d0);
      __syncwarp();
      if (lane == 0) {
        slot[k & PM] = sp;
        slot[bp & PM] = sk0;
        posof[sk0] = bp;
        posof[sp] = k;
        piv[k] = (uint8_t)(bp - k);
        if (d0 == 0.0f) atomicExch(status, PFC_ESINGULAR);
        s_dinv = dinv;
        s_sk = sp;
      }
      __syncwarp();
      for (int r = lane; r < kColRows; r += 32) {  // multipliers by slot: rows k+1 .. last
        const int pos = posof[r];
        lslot[r] = (pos > k && pos <= last) ? colk[r] * dinv : 0.0f;
      }
    }
    __syncthreads();
    if (t >= 32 && t < 64) {  // L row k (the multipliers in window order), off warp 0's path
      const int ln = t - 32, last = min(k + kl, n - 1);
      for (int i = ln; i < lrow; i += 32)
        L[(size_t)k * lrow + i] = to_store_t<TS>(i < kl && k + 1 + i <= last ? lslot[slot[(k + 1 + i) & PM]] : 0.0f);
    }
    const int sk = s_sk;
    const float u = mine[sk];  // the pivot row's entry in this column
    const int j = (t - k) & (kColRing - 1), c = k + j;
    if (j <= ku2 && c < n) U[(size_t)c * ucol + j] = to_store_t<TS>(j == 0 ? s_dinv : u);
    if (j == 0)  // U column k's entries above the band stay zero for the bulk copies
      for (int jj = ku2 + 1; jj < ucol; ++jj) U[(size_t)k * ucol + jj] = to_store_t<TS>(0.0f);
    if (j >= 1 && j <= ku2 && c < n) {  // rank-1 update of this column (row slots < W hold the rows)
#pragma unroll 4
      for (int r = 0; r < Wp; r += 4) {
        const float4 l4 = *reinterpret_cast<const float4*>(&lslot[r]);
        float4 a4 = *reinterpret_cast<const float4*>(&mine[r]);
        a4.x -= l4.x * u;
        a4.y -= l4.y * u;
        a4.z -= l4.z * u;
        a4.w -= l4.w * u;
        *reinterpret_cast<float4*>(&mine[r]) = a4;
      }
    }
    if (j == ku2 + 1)  // the column entering the band starts at zero
      for (int r = 0; r < Wp; r += 4) *reinterpret_cast<float4*>(&mine[r]) = make_float4(0.f, 0.f, 0.f, 0.f);
    if (j == 0) {  // this slot now holds column k + 128
      ac += da;
      bc += db;
      if (ac >= bx) {
        ac -= bx;
        ++bc;
      }
    }
    const int rnew = k + 1 + kl;
    if (rnew < n) {  // the next row of A_k enters the pivot row's slot
      const int colw = k + 1 + ((t - k - 1) & (kColRing - 1));
      mine[sk] = colw < n ? entry(ar, br, ac, bc, colw) : 0.0f;
      if (t == 0) {
        slot[rnew & PM] = sk;
        posof[sk] = rnew;
      }
      if (++ar == bx) {
        ar = 0;
        ++br;
      }
    } else if (t == 0) {
      posof[sk] = -1;
    }
    __syncthreads();
  }
}

// Shared-memory carve-out of one warp of the apply kernel.
struct ApplySmem {
  size_t stage, buf, piv, total;
};
template <typename TC, typename TS, int CH>
__host__ __device__ inline ApplySmem apply_smem(int lrow, int ucol, int nmax) {
  ApplySmem s;
  const int row = lrow > ucol ? lrow : ucol;
  s.stage = rup((size_t)CH * row * sizeof(TS), 128);
  s.buf = rup((size_t)nmax * sizeof(TC), 16);
  s.piv = rup((size_t)nmax, 16);
  s.total = 2 * s.stage + s.buf + s.piv + 16;
  s.total = rup(s.total, 128);
  return s;
}

template <typename TC, typename TS, int CH, int WPC, int NW, int LB>
__global__ void __launch_bounds__(32 * WPC) k_ras_apply2d(Geo g, const BlockDesc* __restrict__ blocks, int nblocks,
                                                          FactorStore fs, const double* __restrict__ r,
                                                          const double* __restrict__ rscale, double* __restrict__ z,
                                                          const int* __restrict__ skip, int* __restrict__ err,
                                                          const IterArgs* __restrict__ ia) {
  constexpr int G = 32 / LB;  // subdomains per warp, LB lanes each
  static_assert(G * LB == 32 && (G == 1 || G == 2), "one or two subdomains per warp");
  if (skip && *skip) return;
  if (ia) {  // graph mode: this Arnoldi iteration's vectors
    r = ia->v;
    rscale = ia->scale;
    z = ia->z;
  }
  extern __shared__ __align__(128) unsigned char smem[];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int gi = lane / LB, li = lane % LB;
  // subdomain of this lane group: consecutive blocks for one per warp; for two per warp the
  // order of fs.order (blocks grouped by extent, every group padded to an even count with -1)
  const int wslot = (blockIdx.x * WPC + w) * G;
  int b;
  bool valid = true;
  if (G == 1) {
    b = wslot;
    if (b >= nblocks) return;  // warp-uniform; no CTA-wide barrier follows
  } else {
    if (wslot >= fs.norder || fs.order[wslot] < 0) return;  // warp-uniform
    b = fs.order[wslot + gi];
    valid = b >= 0;
    if (!valid) b = fs.order[wslot];  // a padding group shadows its partner (same extent), stores nothing
  }
  const int lrow = fs.lrow, ucol = fs.ucol;
  const ApplySmem lay = apply_smem<TC, TS, CH>(lrow, ucol, fs.n_max);
  // groups of one warp are skewed by LB storage elements: their lanes read the same row
  // offsets and would otherwise hit the same shared-memory banks
  const size_t gstride = lay.total + (G > 1 ? LB * sizeof(TS) : 0);
  unsigned char* base = smem + (size_t)w * rup(G * gstride, 128) + gi * gstride;
  auto stage = [&](int st) { return reinterpret_cast<TS*>(base + st * lay.stage); };
  TC* buf = reinterpret_cast<TC*>(base + 2 * lay.stage);
  uint8_t* pv = base + 2 * lay.stage + lay.buf;
  uint64_t* bar = reinterpret_cast<uint64_t*>(base + 2 * lay.stage + lay.buf + lay.piv);

  const BlockDesc B = blocks[b];
  const int bx = B.bx, n = B.bx * B.by;
  const int kl = min(3 * bx, n - 1), ku2 = min(2 * kl, n - 1);
  const TS* L = (const TS*)fs.L + b * fs.strideL;
  const TS* U = (const TS*)fs.U + b * fs.strideU;
  const uint8_t* piv = fs.piv + b * fs.strideP;
  const int nc = (n + CH - 1) / CH;
  const int total = 2 * nc;  // forward chunks 0..nc-1, then backward chunks nc-1..0

  auto issue = [&](int t) {  // group lane 0: bulk-copy chunk t into stage t & 1
    const int st = t & 1;
    const int c = t < nc ? t : 2 * nc - 1 - t;
    const int rows = min(CH, n - c * CH);
    const TS* src = t < nc ? L + (size_t)c * CH * lrow : U + (size_t)c * CH * ucol;
    const uint32_t bytes = (uint32_t)(rows * (t < nc ? lrow : ucol) * sizeof(TS));
    fence_proxy_async();
    mbar_expect_tx(&bar[st], bytes);
    bulk_g2s(stage(st), src, bytes, &bar[st]);
  };
  if (valid && li == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_mbar_init();
    issue(0);
    if (total > 1) issue(1);
  }
  for (int t = li; t < n; t += LB) {  // restriction R_k^delta (periodic wrap) and pivots
    const int a = t % bx, c = t / bx;
    buf[t] = valid ? ld_r<TC>(r, wrap(B.x0 + a, g.nx) + (long long)g.nx * wrap(B.y0 + c, g.ny), fs.pin) : (TC)0;
    pv[t] = valid ? piv[t] : (uint8_t)0;
  }
  __syncwarp();
  // The active window of each triangular solve lives in registers: lane li of a group
  // holds the entries congruent to li mod LB, one register per LB-entry block.  Forward
  // window [k, k+kl] (kl <= LB (NW - 1)): blocks mf..mf+NW-1 in wf[], mf = k / LB.
  // Backward window [k-ku2, k] (ku2 <= LB (NB - 1)): blocks mb..mb-NB+1 in wb[],
  // mb = k / LB.  A chunk of CH steps never crosses an LB-step block (CH divides LB),
  // so the registers rotate only between chunks, when the finished block (final y or
  // x values) goes to shared memory.  Inside a block, step k = LB m + s touches
  // register q of lane li exactly when li passes one threshold in s, and the row
  // interchange is one predicated write into the lane holding the pivot row; the
  // pivot and y_k / x_k values reach the group's lanes by shuffles of width LB.
  // Entries past n - 1 (forward) or below 0 (backward) may hold junk: no step reads
  // them into a valid entry and they are never stored.  A padding group (valid ==
  // false) runs the same instructions on zeros and unread stage memory.
  constexpr int NB = 2 * NW - 1;
  static_assert(LB % CH == 0, "a chunk stays inside one LB-step block");
  const unsigned FULL = 0xffffffffu;
  int mf = 0, mb = 0;
  TC wf[NW], wb[NB];
#pragma unroll
  for (int q = 0; q < NW; ++q) wf[q] = li + LB * q < n ? buf[li + LB * q] : (TC)0;
#pragma unroll
  for (int q = 0; q < NB; ++q) wb[q] = (TC)0;
  uint32_t phase0 = 0, phase1 = 0;
  for (int t = 0; t < total; ++t) {
    const int st = t & 1;
    const bool ok = valid ? mbar_wait_bounded(&bar[st], st ? phase1 : phase0) : true;
    if (st) phase1 ^= 1; else phase0 ^= 1;
    if (!__all_sync(FULL, ok)) {  // give up: record, drain the copies in flight, leave
      if (valid && li == 0) {
        atomicExch(err, PFC_ETIMEOUT);
        mbar_wait_bounded(&bar[st], st ? phase1 ^ 1 : phase0 ^ 1);
        if (t + 1 < total) mbar_wait_bounded(&bar[st ^ 1], st ? phase0 : phase1);
      }
      return;
    }
    const TS* data = stage(st);
    if (t < nc) {  // forward: row interchange P_k, then elimination L_k
      const int c = t, k0 = c * CH, rows = min(CH, n - k0);
      if (k0 / LB != mf) {  // entered block mf + 1: block mf holds final y
        if (LB * mf + li < n) buf[LB * mf + li] = wf[0];
        ++mf;
#pragma unroll
        for (int q = 0; q < NW - 1; ++q) wf[q] = wf[q + 1];
        const int tn = LB * (mf + NW - 1) + li;
        wf[NW - 1] = tn < n ? buf[tn] : (TC)0;
      }
      const int s0 = k0 % LB;
      auto fstep = [&](int kk) {
        const int s = s0 + kk, k = k0 + kk;
        const TS* lk = data + kk * lrow - s - 1;  // lk[LB q + li] multiplies row LB (mf + q) + li
        const int sp = s + pv[k];                 // pivot row p = LB mf + sp
        const int dp = sp / LB, lp = sp % LB;
        const TC bk = __shfl_sync(FULL, wf[0], s, LB);
        TC src = wf[0];
#pragma unroll
        for (int q = 1; q < NW; ++q)
          if (dp == q) src = wf[q];
        const TC bp = __shfl_sync(FULL, src, lp, LB);
        if (li == lp) {  // interchange: row p receives b_k
#pragma unroll
          for (int q = 0; q < NW; ++q)
            if (dp == q) wf[q] = bk;
        }
        if (li == s) wf[0] = bp;  // y_k
        if (li > s && li <= s + kl) wf[0] -= from_store<TC, TS>(lk[li]) * bp;
#pragma unroll
        for (int q = 1; q < NW; ++q)
          if (s + kl - LB * q >= 0) {  // warp-uniform: the band reaches register q at all
            if (li <= s + kl - LB * q) wf[q] -= from_store<TC, TS>(lk[LB * q + li]) * bp;
          }
      };
      if (rows == CH) {
#pragma unroll
        for (int kk = 0; kk < CH; ++kk) fstep(kk);
      } else {
        for (int kk = 0; kk < rows; ++kk) fstep(kk);
      }
      if (t == nc - 1) {  // forward done: the remaining blocks are final
#pragma unroll
        for (int q = 0; q < NW; ++q)
          if (LB * (mf + q) + li < n) buf[LB * (mf + q) + li] = wf[q];
      }
    } else {  // backward, column oriented: x_k = y_k / u_kk, y_{k-j} -= u_{k-j,k} x_k
      const int c = 2 * nc - 1 - t, k0 = c * CH, rows = min(CH, n - k0);
      if (t == nc) {  // y complete: load the top of the backward window
        __syncwarp();
        mb = (n - 1) / LB;
#pragma unroll
        for (int q = 0; q < NB; ++q) {
          const int tb = LB * (mb - q) + li;
          wb[q] = (tb >= 0 && tb < n) ? buf[tb] : (TC)0;
        }
      } else if (k0 / LB != mb) {  // entered block mb - 1: block mb holds final x
        if (LB * mb + li < n) buf[LB * mb + li] = wb[0];
        --mb;
#pragma unroll
        for (int q = 0; q < NB - 1; ++q) wb[q] = wb[q + 1];
        const int tn = LB * (mb - NB + 1) + li;
        wb[NB - 1] = tn >= 0 ? buf[tn] : (TC)0;
      }
      const int s0 = k0 % LB;
      auto bstep = [&](int kk) {
        const int s = s0 + kk;
        const TS* uk = data + kk * ucol + s;  // uk[LB q - li] multiplies row LB (mb - q) + li
        const TC xk = __shfl_sync(FULL, wb[0], s, LB) * from_store<TC, TS>(uk[-s]);
        if (li == s) wb[0] = xk;
        if (li < s && li >= s - ku2) wb[0] -= from_store<TC, TS>(uk[-li]) * xk;
#pragma unroll
        for (int q = 1; q < NB; ++q)
          if (s + LB * q - ku2 <= LB - 1) {  // warp-uniform: the band reaches register q at all
            if (li >= s + LB * q - ku2) wb[q] -= from_store<TC, TS>(uk[LB * q - li]) * xk;
          }
      };
      if (rows == CH) {
#pragma unroll
        for (int kk = CH - 1; kk >= 0; --kk) bstep(kk);
      } else {
        for (int kk = rows - 1; kk >= 0; --kk) bstep(kk);
      }
      if (t == total - 1 && li < n) buf[li] = wb[0];  // block 0
    }
    __syncwarp();  // every lane is done with this stage before it is refilled
    if (valid && li == 0 && t + 2 < total) issue(t + 2);
  }
  __syncwarp();
  if (!valid) return;
  const double sc = rscale ? *rscale : 1.0;
  for (int t = li; t < n; t += LB) {  // extension (R_k^0)^T: core points only
    const int a = t % bx, c = t / bx;
    if (a >= B.ox && a < B.ox + B.cx && c >= B.oy && c < B.oy + B.cy)
      z[wrap(B.x0 + a, g.nx) + (long long)g.nx * wrap(B.y0 + c, g.ny)] = sc * (double)buf[t];
  }
}

// ---- Chunked form of the factors and the chunked apply.
//
// The per-step solves above carry one dependent step per row.  Grouping kChunk
// elimination steps removes the chain inside a group except for a kChunk x
// kChunk triangle, which is applied as a small dense product with its inverse;
// the rest of the group's work is one gather (the group's row interchanges) and
// one product with the factor entries of the group's columns.  k_chunk2d
// rearranges L, U and the pivots into these records after each factorisation.

// One warp per chunk (warps of a CTA take chunks c = w, w + WPC, ...; one CTA per block).
template <typename TC, typename TS, int WPC>
__global__ void __launch_bounds__(32 * WPC) k_chunk2d(const BlockDesc* __restrict__ blocks, FactorStore fs) {
  constexpr int KC = kChunk;
  extern __shared__ __align__(16) unsigned char smem[];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int b = blockIdx.x;
  const BlockDesc B = blocks[b];
  const ChunkGeom cg = chunk_geom(B.bx, B.by, (int)sizeof(TS), (int)sizeof(TC));
  const int n = cg.n, kl = cg.kl, ku2 = cg.ku2, W = cg.W;
  const size_t xrows = (size_t)(KC + fs.kl_max);  // >= W
  TC* X = reinterpret_cast<TC*>(smem) + (size_t)w * xrows * KC;
  int* perm = reinterpret_cast<int*>(reinterpret_cast<TC*>(smem) + (size_t)WPC * xrows * KC) + (size_t)w * xrows;
  const TS* L = (const TS*)fs.L + b * fs.strideL;
  const TS* U = (const TS*)fs.U + b * fs.strideU;
  const uint8_t* piv = fs.piv + b * fs.strideP;
  for (int c = w; c < cg.nc; c += WPC) {
    const int k0 = c * KC, bc = min(KC, n - k0);
    // forward: perm[p] = window row whose value ends at p after the chunk's interchanges;
    // column m of X = the multipliers of step m, moved by the interchanges of steps > m
    if (lane == 0)
      for (int p = 0; p < W; ++p) perm[p] = p;
    for (int idx = lane; idx < W * KC; idx += 32) X[idx] = (TC)0;
    __syncwarp();
    for (int m = 0; m < bc; ++m) {
      const int sp = m + piv[k0 + m];
      if (sp != m) {
        if (lane < m) {  // interchange m moves the multipliers of the earlier steps
          const TC tmp = X[m * KC + lane];
          X[m * KC + lane] = X[sp * KC + lane];
          X[sp * KC + lane] = tmp;
        }
        if (lane == 0) {
          const int tmp = perm[m];
          perm[m] = perm[sp];
          perm[sp] = tmp;
        }
      }
      __syncwarp();
      const TS* lk = L + (size_t)(k0 + m) * fs.lrow;  // lk[i] multiplies window row m + 1 + i
      for (int i = lane; i < kl; i += 32)
        if (k0 + m + 1 + i < n) X[(m + 1 + i) * KC + m] = from_store<TC, TS>(lk[i]);
      __syncwarp();
    }
    unsigned char* rec = fs.X + chunk_rec_off(fs, b, cg.nc, c);
    const int wp = (W + 15) & ~15;
    for (int p = lane; p < wp; p += 32) rec[p] = p < W ? (unsigned char)perm[p] : (unsigned char)0;
    TC* E11 = reinterpret_cast<TC*>(rec + wp);
    if (lane < KC) {  // column lane of the inverse of the unit lower KC x KC block
      TC e[KC];
#pragma unroll
      for (int r = 0; r < KC; ++r) {
        TC v = r == lane ? (TC)1 : (TC)0;
        for (int q = 0; q < r; ++q) v -= X[r * KC + q] * e[q];
        e[r] = v;
      }
#pragma unroll
      for (int r = 0; r < KC; ++r) E11[r * KC + lane] = e[r];
    }
    TS* L21 = reinterpret_cast<TS*>(rec + wp + KC * KC * sizeof(TC));
    for (int idx = lane; idx < kl * KC; idx += 32) L21[idx] = to_store_t<TS>(-X[KC * KC + idx]);
    // backward: U11^{-1} (column lane by back substitution with the stored 1 / u_kk) and -U_a
    TC* U11i = reinterpret_cast<TC*>(fs.X + chunk_rec_off(fs, b, cg.nc, 2 * cg.nc - 1 - c));
    if (lane < KC) {
      TC x[KC];
#pragma unroll
      for (int r = KC - 1; r >= 0; --r) {
        TC v = r == lane ? (TC)1 : (TC)0;
        if (r < bc) {
          const TS* ur = U + (size_t)(k0 + r) * fs.ucol;  // ur[0] = 1 / u_rr
#pragma unroll
          for (int q = r + 1; q < KC; ++q)
            if (q < bc) v -= from_store<TC, TS>(U[(size_t)(k0 + q) * fs.ucol + (q - r)]) * x[q];
          v *= from_store<TC, TS>(ur[0]);
        }
        x[r] = v;
      }
#pragma unroll
      for (int r = 0; r < KC; ++r) U11i[r * KC + lane] = x[r];
    }
    TS* Ua = reinterpret_cast<TS*>(reinterpret_cast<unsigned char*>(U11i) + KC * KC * sizeof(TC));
    for (int idx = lane; idx < ku2 * KC; idx += 32) {
      const int i = idx / KC, j = idx % KC, jj = ku2 + j - i;  // u(k0 - ku2 + i, k0 + j) at U column k0 + j
      TC v = (TC)0;
      if (j < bc && jj <= ku2 && k0 - ku2 + i >= 0) v = -from_store<TC, TS>(U[(size_t)(k0 + j) * fs.ucol + jj]);
      Ua[idx] = to_store_t<TS>(v);
    }
    __syncwarp();
  }
}

// One row of kChunk stored entries in the compute type.
template <typename TC, typename TS>
__device__ __forceinline__ void load_row8(const TS* row, TC* e);
template <>
__device__ __forceinline__ void load_row8<float, __nv_bfloat16>(const __nv_bfloat16* row, float* e) {
  const uint4 v = *reinterpret_cast<const uint4*>(row);
  const uint32_t u[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    e[2 * i] = __uint_as_float(u[i] << 16);
    e[2 * i + 1] = __uint_as_float(u[i] & 0xffff0000u);
  }
}
template <>
__device__ __forceinline__ void load_row8<float, float>(const float* row, float* e) {
  load4(row, e);
  load4(row + 4, e + 4);
}
template <>
__device__ __forceinline__ void load_row8<double, double>(const double* row, double* e) {
  load4(row, e);
  load4(row + 4, e + 4);
}

// Shared memory of one warp of the chunked apply: STAGES record buffers, the
// block vector (rounded up to whole chunks), the stage barriers.
struct ChunkSmem {
  size_t stage, ybytes, total;
};
template <typename TC, int STAGES>
__host__ __device__ inline ChunkSmem chunk_smem(int xstage, int n_max) {
  ChunkSmem c;
  c.stage = rup((size_t)xstage, 128);
  c.ybytes = rup((size_t)((n_max + kChunk - 1) / kChunk * kChunk) * sizeof(TC), 16);
  c.total = rup(STAGES * c.stage + c.ybytes + 8 * STAGES, 128);
  return c;
}

// Periodic index for -n <= i < 2n (a block is never wider than the grid).
__device__ __forceinline__ int wrap1(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

// z = sum_k (R_k^0)^T A_k^{-1} R_k^delta r with the chunked factors: one warp per
// block, the block's records streamed through a ring of STAGES bulk copies.  Lanes
// 0..KC-1 apply the chunk's small inverse; then every lane takes one of the kl rows
// below (forward) or ku2 rows above (backward) per round (QF >= kl / 32 rounds,
// QB >= ku2 / 32).
template <typename TC, typename TS, int WPC, int STAGES, int QF, int QB>
__global__ void __launch_bounds__(32 * WPC)
    k_ras_apply2d_chunked(Geo g, const BlockDesc* __restrict__ blocks, int nblocks, FactorStore fs,
                          const double* __restrict__ r, const double* __restrict__ rscale, double* __restrict__ z,
                          const int* __restrict__ skip, int* __restrict__ err, const IterArgs* __restrict__ ia) {
  constexpr int KC = kChunk;
  static_assert(KC == 8, "rows of 8 entries (16-byte loads)");
  if (skip && *skip) return;
  if (ia) {  // graph mode: this Arnoldi iteration's vectors
    r = ia->v;
    rscale = ia->scale;
    z = ia->z;
  }
  extern __shared__ __align__(128) unsigned char smem[];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int b = blockIdx.x * WPC + w;
  if (b >= nblocks) return;  // warp-uniform; no CTA-wide barrier follows
  const ChunkSmem lay = chunk_smem<TC, STAGES>(fs.xstage, fs.n_max);
  unsigned char* base = smem + (size_t)w * lay.total;
  TC* y = reinterpret_cast<TC*>(base + STAGES * lay.stage);
  uint64_t* bar = reinterpret_cast<uint64_t*>(base + STAGES * lay.stage + lay.ybytes);
  const BlockDesc B = blocks[b];
  const ChunkGeom cg = chunk_geom(B.bx, B.by, (int)sizeof(TS), (int)sizeof(TC));
  const int n = cg.n, nc = cg.nc, total = 2 * nc;
  auto issue = [&](int t) {  // lane 0: record t into stage t % STAGES
    const int st = t % STAGES;
    const unsigned char* src = fs.X + chunk_rec_off(fs, b, nc, t);
    const uint32_t bytes = (uint32_t)(t < nc ? cg.fwd : cg.bwd);
    fence_proxy_async();
    mbar_expect_tx(&bar[st], bytes);
    bulk_g2s(base + st * lay.stage, src, bytes, &bar[st]);
  };
  if (lane == 0) {
#pragma unroll
    for (int st = 0; st < STAGES; ++st) mbar_init(&bar[st], 1);
    fence_mbar_init();
    for (int t = 0; t < STAGES && t < total; ++t) issue(t);
  }
  // block-local (a, c) of element t = lane + 32 i, advanced without divisions
  const int da = 32 % B.bx, dc = 32 / B.bx, a0 = lane % B.bx, c0 = lane / B.bx;
  {
    int a = a0, c = c0;
    const bool core_only = fs.ras_kind == PFC_RIGHT_RAS;
    for (int t = lane; t < nc * KC; t += 32) {  // restriction R_k^delta (R_k^0 for right-RAS); zeros past n
      const bool in = t < n && (!core_only || (a >= B.ox && a < B.ox + B.cx && c >= B.oy && c < B.oy + B.cy));
      y[t] = in ? ld_r<TC>(r, wrap1(B.x0 + a, g.nx) + (long long)g.nx * wrap1(B.y0 + c, g.ny), fs.pin) : (TC)0;
      a += da;
      c += dc;
      if (a >= B.bx) {
        a -= B.bx;
        ++c;
      }
    }
  }
  __syncwarp();
  const unsigned FULL = 0xffffffffu;
  for (int t = 0; t < total; ++t) {
    const int st = t % STAGES;
    const bool ok = mbar_wait_bounded(&bar[st], (uint32_t)((t / STAGES) & 1));
    if (!__all_sync(FULL, ok)) {  // give up: record, drain the copies in flight, leave
      if (lane == 0) {
        atomicExch(err, PFC_ETIMEOUT);
        for (int u = t; u < t + STAGES && u < total; ++u)
          mbar_wait_bounded(&bar[u % STAGES], (uint32_t)((u / STAGES) & 1));
      }
      return;
    }
    const unsigned char* rec = base + st * lay.stage;
    if (t < nc) {  // forward chunk t on the window [k0, k0 + W): gather, y_c = E11 t_c, y_b = t_b - L21 y_c
      const int k0 = t * KC, W = cg.W, kl = cg.kl;
      const unsigned char* perm = rec;
      const TC* E11 = reinterpret_cast<const TC*>(rec + ((W + 15) & ~15));
      const TS* L21 = reinterpret_cast<const TS*>(E11 + KC * KC);  // negated
      const TC tc = (lane < KC && k0 + lane < n) ? y[min(k0 + (int)perm[lane], n - 1)] : (TC)0;
      TC tv[QF];  // rows KC + i of the window, i = lane + 32 q
#pragma unroll
      for (int q = 0; q < QF; ++q) {
        const int i = lane + 32 * q, R = KC + i;
        tv[q] = (i < kl && k0 + R < n) ? y[min(k0 + (int)perm[R], n - 1)] : (TC)0;
      }
      TC t1[KC];
#pragma unroll
      for (int j = 0; j < KC; ++j) t1[j] = __shfl_sync(FULL, tc, j);
      TC yc = (TC)0;
      if (lane < KC) {
        TC e[KC];
        load_row8<TC, TC>(E11 + lane * KC, e);
#pragma unroll
        for (int j = 0; j < KC; ++j) yc = fma(e[j], t1[j], yc);
      }
      TC y1[KC];
#pragma unroll
      for (int j = 0; j < KC; ++j) y1[j] = __shfl_sync(FULL, yc, j);
      __syncwarp();  // every gather is done before any row is written
      if (lane < KC && k0 + lane < n) y[k0 + lane] = yc;
#pragma unroll
      for (int q = 0; q < QF; ++q) {
        const int i = lane + 32 * q, R = KC + i;
        if (i < kl && k0 + R < n) {
          TC e[KC];
          load_row8<TC, TS>(L21 + i * KC, e);
          TC acc = tv[q];
#pragma unroll
          for (int j = 0; j < KC; ++j) acc = fma(e[j], y1[j], acc);
          y[k0 + R] = acc;
        }
      }
    } else {  // backward chunk c: x_c = U11^{-1} y_c, y_a -= U_a x_c (a = the ku2 rows above)
      const int c = 2 * nc - 1 - t, k0 = c * KC, ku2 = cg.ku2;
      const TC* U11i = reinterpret_cast<const TC*>(rec);
      const TS* Ua = reinterpret_cast<const TS*>(U11i + KC * KC);  // negated
      TC t1[KC];
      load_row8<TC, TC>(y + k0, t1);  // zeros past n
      TC xc = (TC)0;
      if (lane < KC) {
        TC e[KC];
        load_row8<TC, TC>(U11i + lane * KC, e);
#pragma unroll
        for (int j = 0; j < KC; ++j) xc = fma(e[j], t1[j], xc);
      }
      TC x1[KC];
#pragma unroll
      for (int j = 0; j < KC; ++j) x1[j] = __shfl_sync(FULL, xc, j);
      __syncwarp();  // every lane holds y_c before x_c overwrites it
      if (lane < KC && k0 + lane < n) y[k0 + lane] = xc;
      // one row per lane and round; written as a loop over the lane's rows of the round
      // (at most one), which measured faster than the equivalent predicated body
#pragma unroll
      for (int qb = 0; qb < QB; ++qb)
        for (int i = lane + 32 * qb; i < ku2; i += 1 << 20) {
          const int pos = k0 - ku2 + i;
          if (pos >= 0) {
            TC e[KC];
            load_row8<TC, TS>(Ua + i * KC, e);
            TC acc = y[pos];
#pragma unroll
            for (int j = 0; j < KC; ++j) acc = fma(e[j], x1[j], acc);
            y[pos] = acc;
          }
        }
    }
    __syncwarp();  // every lane is done with this stage (and with y) before it is refilled
    if (lane == 0 && t + STAGES < total) issue(t + STAGES);
  }
  const double sc = rscale ? *rscale : 1.0;
  if (fs.ras_kind != PFC_LEFT_RAS) {  // extension over the whole block: to the block's scratch row
    for (int t = lane; t < n; t += 32) fs.Yb[(size_t)b * fs.n_max + t] = sc * (double)y[t];
    return;
  }
  pdl_trigger();  // the solves are done: the next kernel (the JVP) may be scheduled
  int a = a0, c = c0;
  for (int t = lane; t < n; t += 32) {  // extension (R_k^0)^T: core points only
    if (a >= B.ox && a < B.ox + B.cx && c >= B.oy && c < B.oy + B.cy)
      z[wrap1(B.x0 + a, g.nx) + (long long)g.nx * wrap1(B.y0 + c, g.ny)] = sc * (double)y[t];
    a += da;
    c += dc;
    if (a >= B.bx) {
      a -= B.bx;
      ++c;
    }
  }
}

// Core index along an axis of n cells in p cores (the first rem = n mod p hold base + 1).
__device__ __forceinline__ int core_of(int x, int base, int rem) {
  const int big = rem * (base + 1);
  return x < big ? x / (base + 1) : rem + (x - big) / base;
}
__device__ __forceinline__ int core_start(int i, int base, int rem) { return i * base + min(i, rem); }

// z(p) = sum over the blocks whose extended region holds p of their solution at p (Eq. invM /
// Eq. ash extension (R_k^delta)^T), blocks visited in a fixed order: deterministic sums.
__global__ void __launch_bounds__(256) k_schwarz_sum(Geo g, Decomp2 dc, const BlockDesc* __restrict__ blocks,
                                                     FactorStore fs, double* __restrict__ z,
                                                     const int* __restrict__ skip, const IterArgs* __restrict__ ia) {
  if (skip && *skip) return;
  if (ia) z = ia->z;
  const long long n = (long long)g.nx * g.ny;
  // cores within reach of a point (each distinct block once, in a fixed order)
  const int kx = (dc.ov + dc.base_x - 1) / dc.base_x, ky = (dc.ov + dc.base_y - 1) / dc.base_y;
  const int mx = min(2 * kx + 1, dc.px), my = min(2 * ky + 1, dc.py);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(i % g.nx), y = (int)(i / g.nx);
    const int ix = core_of(x, dc.base_x, dc.rem_x), iy = core_of(y, dc.base_y, dc.rem_y);
    double s = 0.0;
    for (int tj = 0; tj < my; ++tj) {
      const int by = my == dc.py ? tj : ((iy - ky + tj) % dc.py + dc.py) % dc.py;
      for (int ti = 0; ti < mx; ++ti) {
        const int bxi = mx == dc.px ? ti : ((ix - kx + ti) % dc.px + dc.px) % dc.px;
        const int b = by * dc.px + bxi;
        const BlockDesc B = blocks[b];
        const int a = ((x - B.x0) % g.nx + g.nx) % g.nx, c = ((y - B.y0) % g.ny + g.ny) % g.ny;
        if (a < B.bx && c < B.by) s += fs.Yb[(size_t)b * fs.n_max + a + B.bx * c];
      }
    }
    z[i] = s;
  }
}

template <typename TC, typename TS, int WPC, int STAGES, int QF, int QB>
void chunked_launch(const Geo& g, const BlockDesc* blocks, int nblocks, const FactorStore& fs, const double* r,
                    const double* rscale, double* z, const int* skip, int* err, cudaStream_t st, const IterArgs* ia,
                    size_t smem) {
  cudaFuncSetAttribute(k_ras_apply2d_chunked<TC, TS, WPC, STAGES, QF, QB>,
                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k_ras_apply2d_chunked<TC, TS, WPC, STAGES, QF, QB><<<(nblocks + WPC - 1) / WPC, 32 * WPC, smem, st>>>(
      g, blocks, nblocks, fs, r, rscale, z, skip, err, ia);
}

template <typename TC, typename TS, int WPC, int STAGES>
void chunked_dispatch(const Geo& g, const BlockDesc* blocks, int nblocks, const FactorStore& fs, const double* r,
                      const double* rscale, double* z, const int* skip, int* err, cudaStream_t st,
                      const IterArgs* ia) {
  const size_t smem = WPC * chunk_smem<TC, STAGES>(fs.xstage, fs.n_max).total;
  // rounds of 32 rows: kl rows forward, ku2 <= 2 kl rows backward
  if (fs.kl_max <= 64)
    chunked_launch<TC, TS, WPC, STAGES, 2, 4>(g, blocks, nblocks, fs, r, rscale, z, skip, err, st, ia, smem);
  else if (fs.kl_max <= 96)
    chunked_launch<TC, TS, WPC, STAGES, 3, 6>(g, blocks, nblocks, fs, r, rscale, z, skip, err, st, ia, smem);
  else
    chunked_launch<TC, TS, WPC, STAGES, 4, 8>(g, blocks, nblocks, fs, r, rscale, z, skip, err, st, ia, smem);
  count_launches(1);
}

template <typename TC, typename TS>
void factor_dispatch(const Geo& g, const BlockDesc* blocks, int nblocks, const double* q, double idt,
                     const double* lin, const FactorStore& fs, int* status, cudaStream_t st, const double* idt_dev) {
  if (sizeof(TC) == 4 && !fs.mob_mu && !g.neumann && fs.kl_max + 1 <= kColRows && 2 * fs.kl_max + 2 <= kColRing &&
      factor_col_smem_bytes(fs.n_max) <= 227 * 1024) {
    const size_t smem = factor_col_smem_bytes(fs.n_max);
    cudaFuncSetAttribute(k_factor2d_col<TS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_factor2d_col<TS><<<nblocks, kColRing, smem, st>>>(g, blocks, q, idt, lin, fs, status, idt_dev);
    count_launches(1);
    return;
  }
  const size_t smem = factor_smem_bytes(fs.prec, fs.kl_max, fs.n_max, fs.mob_mu ? fs.ext_max : 0);
  if (2 * fs.kl_max + 2 <= 128) {
    cudaFuncSetAttribute(k_factor2d<TC, TS, 128>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_factor2d<TC, TS, 128><<<nblocks, 256, smem, st>>>(g, blocks, q, idt, lin, fs, status, idt_dev);
  } else {
    cudaFuncSetAttribute(k_factor2d<TC, TS, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_factor2d<TC, TS, 256><<<nblocks, 256, smem, st>>>(g, blocks, q, idt, lin, fs, status, idt_dev);
  }
  count_launches(1);
}

template <typename TC, typename TS, int CH, int WPC, int NW = 3, int LB = 32>
void apply_dispatch(const Geo& g, const BlockDesc* blocks, int nblocks, const FactorStore& fs, const double* r,
                    const double* rscale, double* z, const int* skip, int* err, cudaStream_t st,
                    const IterArgs* ia) {
  constexpr int G = 32 / LB;
  const ApplySmem lay = apply_smem<TC, TS, CH>(fs.lrow, fs.ucol, fs.n_max);
  const size_t gstride = lay.total + (G > 1 ? LB * sizeof(TS) : 0);
  const size_t smem = WPC * rup(G * gstride, 128);
  const int warps = G == 1 ? nblocks : fs.norder / G;
  cudaFuncSetAttribute(k_ras_apply2d<TC, TS, CH, WPC, NW, LB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)smem);
  k_ras_apply2d<TC, TS, CH, WPC, NW, LB><<<(warps + WPC - 1) / WPC, 32 * WPC, smem, st>>>(g, blocks, nblocks, fs, r,
                                                                                       rscale, z, skip, err, ia);
  count_launches(1);
}

}  // namespace

// Chunked apply shapes per storage type (warps per CTA, stages).
constexpr int kChunkWpcF64 = 2, kChunkStF64 = 2;
constexpr int kChunkWpcF32 = 4, kChunkStF32 = 2;
constexpr int kChunkWpcB16 = 4, kChunkStB16 = 3;

size_t chunked_smem_bytes(int prec, int xstage, int n_max) {
  if (prec == PFC_F64) return kChunkWpcF64 * chunk_smem<double, kChunkStF64>(xstage, n_max).total;
  if (prec == PFC_F32) return kChunkWpcF32 * chunk_smem<float, kChunkStF32>(xstage, n_max).total;
  return kChunkWpcB16 * chunk_smem<float, kChunkStB16>(xstage, n_max).total;
}

static size_t chunk_build_smem(int prec, int kl_max) {
  const size_t tc = prec == PFC_F64 ? 8 : 4;
  return (size_t)4 * (kChunk + kl_max) * (kChunk * tc + sizeof(int));
}

bool apply_variant_ok(int v, int prec, int kl_max, int xstage, int n_max) {
  if (v == kChunkedVariant)
    return kl_max <= 128 && chunked_smem_bytes(prec, xstage, n_max) <= 227 * 1024 &&
           chunk_build_smem(prec, kl_max) <= 227 * 1024;
  if (kl_max <= 64) return v >= 0 && v < kChunkedVariant;  // 3 + 5 window registers per lane
  return v == 0 && kl_max <= 128;                           // 5 + 9 window registers, default shape
}

void launch_chunk2d(const BlockDesc* blocks, int nblocks, const FactorStore& fs, cudaStream_t st) {
  const size_t smem = chunk_build_smem(fs.prec, fs.kl_max);
  if (fs.prec == PFC_F64) {
    cudaFuncSetAttribute(k_chunk2d<double, double, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_chunk2d<double, double, 4><<<nblocks, 128, smem, st>>>(blocks, fs);
  } else if (fs.prec == PFC_F32) {
    cudaFuncSetAttribute(k_chunk2d<float, float, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_chunk2d<float, float, 4><<<nblocks, 128, smem, st>>>(blocks, fs);
  } else {
    cudaFuncSetAttribute(k_chunk2d<float, __nv_bfloat16, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    k_chunk2d<float, __nv_bfloat16, 4><<<nblocks, 128, smem, st>>>(blocks, fs);
  }
  count_launches(1);
}

// Dynamic shared memory of the factor kernel: q on the block and the stencil
// table (FP64), the (kl+1) x (RING+1) window plus the multiplier and U-row
// buffers (compute type), the position map and the row offsets.
size_t factor_smem_bytes(int prec, int kl, int n_max, int ext_max) {
  const int ring = (2 * kl + 2 <= 128) ? 128 : 256;
  const size_t tc = prec == PFC_F64 ? 8 : 4;
  size_t b = rup((size_t)(n_max + 49) * 8, 16) + (size_t)((kl + 1) * (ring + 1) + 2 * ring) * tc +
             ring * sizeof(int) + 16;
  if (ext_max > 0) b = rup(b, 16) + 16 + (size_t)(2 * ext_max + 25) * 8;  // mobility: s, mu with ring, table
  return b;
}

void launch_factor2d(const Geo& g, const BlockDesc* blocks, int nblocks, const double* q, double idt,
                     const double* lin, const FactorStore& fs, int* status, cudaStream_t st, const double* idt_dev) {
  if (fs.prec == PFC_F64)
    factor_dispatch<double, double>(g, blocks, nblocks, q, idt, lin, fs, status, st, idt_dev);
  else if (fs.prec == PFC_F32)
    factor_dispatch<float, float>(g, blocks, nblocks, q, idt, lin, fs, status, st, idt_dev);
  else
    factor_dispatch<float, __nv_bfloat16>(g, blocks, nblocks, q, idt, lin, fs, status, st, idt_dev);
}

void launch_ras_apply2d(const Geo& g, const BlockDesc* blocks, int nblocks, const FactorStore& fs, const double* r,
                        const double* rscale, double* z, const int* skip, int* err, cudaStream_t st,
                        const IterArgs* ia, const Decomp2* dc) {
  // Launch shapes (chunk length CH = steps per bulk copy, WPC = warps per CTA):
  // variant 0: stages of about 3.5 KB for every storage type, 4 warps per CTA;
  // 1: half the chunk (twice the resident warps per SM), 2: half the chunk and
  // 2 warps per CTA (finer packing), 3: twice the chunk (fewer, larger copies);
  // 4: two subdomains per warp, 16 lanes each (5 + 9 window registers per lane);
  // 5: the chunked solves (one warp per block, records of kChunk steps).
  if (fs.variant == kChunkedVariant) {
    if (fs.ras_kind != PFC_LEFT_RAS && dc) {  // solutions to the block scratch, then the overlap sums
      launch_ras_apply2d(g, blocks, nblocks, fs, r, rscale, z, skip, err, st, ia, nullptr);
      const long long n = (long long)g.nx * g.ny;
      const int grid = (int)((n + 255) / 256 < 4 * 152 ? (n + 255) / 256 : 4 * 152);
      k_schwarz_sum<<<grid, 256, 0, st>>>(g, *dc, blocks, fs, z, skip, ia);
      count_launches(1);
      return;
    }
    if (fs.prec == PFC_F64)
      chunked_dispatch<double, double, kChunkWpcF64, kChunkStF64>(g, blocks, nblocks, fs, r, rscale, z, skip, err,
                                                                   st, ia);
    else if (fs.prec == PFC_F32)
      chunked_dispatch<float, float, kChunkWpcF32, kChunkStF32>(g, blocks, nblocks, fs, r, rscale, z, skip, err, st,
                                                                 ia);
    else
      chunked_dispatch<float, __nv_bfloat16, kChunkWpcB16, kChunkStB16>(g, blocks, nblocks, fs, r, rscale, z, skip,
                                                                         err, st, ia);
  } else if (fs.kl_max > 64) {  // blocks wider than 21 cells: the wide-window kernel, default shape
    if (fs.prec == PFC_F64)
      apply_dispatch<double, double, 4, 4, 5>(g, blocks, nblocks, fs, r, rscale, z, skip, err, st, ia);
    else if (fs.prec == PFC_F32)
      apply_dispatch<float, float, 8, 4, 5>(g, blocks, nblocks, fs, r, rscale, z, skip, err, st, ia);
    else
      apply_dispatch<float, __nv_bfloat16, 16, 4, 5>(g, blocks, nblocks, fs, r, rscale, z, skip, err, st, ia);
  } else if (fs.prec == PFC_F64) {
    switch (fs.variant) {
      case 1: apply_dispatch<double, double, 2, 4>(g, blocks, nblocks, fs, r, rscale, z, skip, err, st, ia); break;
      case 2: apply_dispatch<double, double, 2, 2>(g, blocks, nblocks, fs, r, rscale, z, skip, err, st, ia); break;
      case 3: apply_dispatch<double, double, 8, 4>(g, blocks, nblocks, fs, r, rscale, z, skip, err, st, ia); break;
      case 4: apply_dispatch<double, double, 4, 4, 5, 16>(g, blocks, nblocks, fs, r, rscale, z, skip, err, st, ia);
        break;
      default: apply_dispatch<double, double, 4, 4>(g, blocks, nblocks, fs, r, rscale, z, skip, err, st, ia);
    }
  } else if (fs.prec == PFC_F32) {
    switch (fs.variant) {
      case 1: apply_dispatch<float, float, 4, 4>(g, blocks, nblocks, fs, r, rscale, z, skip, err, st, ia); break;
      case 2: apply_dispatch<float, float, 4, 2>(g, blocks, nblocks, fs, r, rscale, z, skip, err, st, ia); break;
      case 3: apply_dispatch<float, float, 16, 4>(g, blocks, nblocks, fs, r, rscale, z, skip, err, st, ia); break;
      case 4: apply_dispatch<float, float, 8, 4, 5, 16>(g, blocks, nblocks, fs, r, rscale, z, skip, err, st, ia);
        break;
      default: apply_dispatch<float, float, 8, 4>(g, blocks, nblocks, fs, r, rscale, z, skip, err, st, ia);
    }
  } else {
    using B16 = __nv_bfloat16;
    switch (fs.variant) {
      case 1: apply_dispatch<float, B16, 8, 4>(g, blocks, nblocks, fs, r, rscale, z, skip, err, st, ia); break;
      case 2: apply_dispatch<float, B16, 8, 2>(g, blocks, nblocks, fs, r, rscale, z, skip, err, st, ia); break;
      case 3: apply_dispatch<float, B16, 32, 4>(g, blocks, nblocks, fs, r, rscale, z, skip, err, st, ia); break;
      case 4: apply_dispatch<float, B16, 8, 4, 5, 16>(g, blocks, nblocks, fs, r, rscale, z, skip, err, st, ia);
        break;
      default: apply_dispatch<float, B16, 16, 4>(g, blocks, nblocks, fs, r, rscale, z, skip, err, st, ia);
    }
  }
}

}  // namespace pfc
