// FP64 vector kernels of right-preconditioned restarted GMRES (Sec. 4, Eq.
// hjacobi): fused multi-dot products and multi-axpys for classical Gram-Schmidt
// with one conditional re-orthogonalisation pass (Daniel-Gragg-Kaufman-Stewart
// criterion), and the Arnoldi/Givens bookkeeping, all on the device.
//
// Reductions are deterministic: every CTA writes its partial sums (fixed
// order inside the CTA), and the last CTA to finish -- found with an atomic
// ticket -- sums the partials in a fixed order and then runs the single-thread
// bookkeeping step (Hessenberg column, Givens rotation, residual estimate,
// convergence flag).  So one Gram-Schmidt pass costs one kernel per vector
// sweep, with no separate reduction launch.
//
// On the mixed path (F32/BF16 factors) the Arnoldi sweeps run on the FP32 pipe.
// There the Krylov basis V is stored as normalised float pairs (hi, lo) in the
// 8 bytes of each element (the JVP writes them, the sweeps and the Schwarz apply
// read them), so no sweep splits an FP64 value.  The multi-axpy w -= sum c_k V_k
// uses the float-float arithmetic of ff.cuh (about 2^-46 relative) and stores w
// as a pair: the Arnoldi relation J Z_j = V H holds to that accuracy whatever
// the coefficients are.  The coefficients (the multi-dot products) are
// float-float too by default (Dot::kFF: products with their exact rounding error
// and the cross terms, running sums with two-sum), so the orthogonalisation keeps
// FP64-class accuracy.  (The same sweeps over FP64-stored vectors, for the
// mobility form whose JVP stays FP64, split each element and send part of every
// tile to the FP64 pipe, kPd below.)  Dot::kF32 -- FP32 products of the leading
// floats, about 2^-24 of |V_i| |w| per product -- is a faster opt-in form
// (pfc_params.gmres_fast_dots) that leaves the orthogonality of the new vector
// to the conditional second (DGKS) pass.
//
// The basis is kept unnormalised: V_i = scale_i * Vraw_i with scale_i held on
// the device, so no kernel pass is spent on normalising.  Every kernel takes
// the cycle's "done" flag and returns at once when it is set, which lets the
// host queue several iterations ahead and synchronise rarely.
#include <algorithm>
#include <cstdio>
#include <cmath>

#include "../../include/pfc.h"
#include "ff.cuh"
#include "pfc_internal.cuh"
#include "pfc_tma.cuh"

namespace pfc {
namespace {

constexpr int G = 8;     // vectors per multi-dot pass
constexpr int NT = 256;  // threads per CTA

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Vector i of a list: v0 for i = 0, tab[i] otherwise (tab is a device pointer table).
__device__ __forceinline__ const double* vec_at(const double* v0, const double* const* tab, int i) {
  return i == 0 ? v0 : tab[i];
}

// ---- single-thread GMRES bookkeeping

__device__ void gmres_finalize(GmresCtl* c, int j, int m, double wn2) {
  const int m1 = kMaxRestart + 1;
  double* Hj = c->H + m1 * j;
  const double hn = sqrt(wn2);
  Hj[j + 1] = hn;
  c->scale[j + 1] = hn > 0.0 ? 1.0 / hn : 0.0;
  for (int i = 0; i < j; ++i) {  // previous Givens rotations
    const double t = c->cs[i] * Hj[i] + c->sn[i] * Hj[i + 1];
    Hj[i + 1] = -c->sn[i] * Hj[i] + c->cs[i] * Hj[i + 1];
    Hj[i] = t;
  }
  const double den = hypot(Hj[j], Hj[j + 1]);
  const double cs = den > 0.0 ? Hj[j] / den : 1.0;
  const double sn = den > 0.0 ? Hj[j + 1] / den : 0.0;
  c->cs[j] = cs;
  c->sn[j] = sn;
  Hj[j] = den;
  Hj[j + 1] = 0.0;
  c->g[j + 1] = -sn * c->g[j];
  c->g[j] = cs * c->g[j];
  c->est = fabs(c->g[j + 1]);
  c->its = j + 1;
  if (!(hn > 0.0)) c->breakdown = 1;
  if (c->est <= c->tol || !(hn > 0.0) || j + 1 >= m || !(c->est == c->est)) c->done = 1;
}

// After the multi-axpy w -= sum coef_i Vraw_i, with wn2 = w.w afterwards.
__device__ void gmres_after_axpy(GmresCtl* c, int j, int pass, int m, double wn2) {
  if (pass == 0) {
    if (wn2 < c->reorth_eta2 * c->wnorm2_before) {  // ||w'|| < eta ||w||: orthogonalise once more
      c->reorth = 1;
      c->n_reorth += 1;
      return;
    }
    c->reorth = 0;
    gmres_finalize(c, j, m, wn2);
  } else {
    c->reorth = 0;
    gmres_finalize(c, j, m, wn2);
  }
}

// ---- fused last-CTA reduction

// The last CTA of the grid (atomic ticket on t.counter) sums nvals partial rows
// of nparts entries each, in a fixed order, then runs the tail step.
__device__ __noinline__ void last_cta_tail(const Tail& t, const double* __restrict__ partial, int nvals,
                                          int nparts) {
  __shared__ bool s_last;
  __shared__ double s_sum[kMaxVecs + 2];
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned total = gridDim.x * gridDim.y;
    s_last = atomicAdd(t.counter, 1u) == total - 1;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int v = wid; v < nvals; v += (int)(blockDim.x / 32)) {
    double s = 0.0;
    for (int p = lane; p < nparts; p += 32) s += __ldcg(partial + (size_t)v * nparts + p);
    s = warp_sum(s);
    if (lane == 0) s_sum[v] = s;
  }
  __syncthreads();
  if (t.kind == Tail::kDot) {  // one thread per Hessenberg entry: the FP64 products run side by side
    GmresCtl* c = t.ctl;
    const int j = t.ia ? t.ia->j : t.j;
    const int m1 = kMaxRestart + 1;
    for (int i = threadIdx.x; i <= j + 1 && i < nvals; i += blockDim.x) c->red[i] = s_sum[i];
    for (int i = threadIdx.x; i <= j; i += blockDim.x) {
      const double sc = c->scale[i];
      const double h = sc * s_sum[i];
      if (t.pass == 0)
        c->H[i + m1 * j] = h;
      else
        c->H[i + m1 * j] += h;
      c->coef[i] = h * sc;
    }
    if (threadIdx.x == 0) {
      if (t.pass == 0) c->wnorm2_before = s_sum[j + 1];
      *t.counter = 0u;  // ready for the next kernel on this stream
    }
    return;
  }
  if (threadIdx.x == 0) {
    GmresCtl* c = t.ctl;
    const int j = t.ia ? t.ia->j : t.j;
    if (t.kind == Tail::kAxpy) {
      gmres_after_axpy(c, j, t.pass, t.m, s_sum[0]);
      if (t.set_reorth) cudaGraphSetConditional(t.h_reorth, c->reorth ? 1u : 0u);
    } else {
      for (int v = 0; v < nvals; ++v) t.out[v] = s_sum[v];
    }
    *t.counter = 0u;  // ready for the next kernel on this stream
  }
}

// ---- Streamed sweeps.  Each CTA takes tiles of kTile points round-robin and
// brings every vector's tile into shared memory with one bulk copy (TMA) through
// a ring of kStages buffers.  One producer warp issues the copies; the NT
// consumer threads wait for a buffer's "full" barrier (the copy's bytes), work
// from shared memory (kPts points each) and release it warp by warp on its
// "empty" barrier, so no CTA-wide barrier sits in the loop and a CTA keeps up to
// kStages x 8 KB in flight.  Element q of a CTA's copy sequence is (local tile
// q / per, vector q % per).
constexpr int kTile = 1024;
constexpr int kStages = 6;
constexpr int kPts = kTile / NT;
// Float-float sweeps (the mixed path) send the first kPd of a thread's kPts points of every
// tile to the FP64 pipe (one FMA each) and the rest to float-float on the FP32 pipe: both
// give FP64-class sums, and the two pipes, each too slow alone for the HBM rate on GB300
// (FP64 at 1/64 of FP32; float-float at ~30 instructions per element), run side by side.
constexpr int kPd = 2;
constexpr int kSweepThreads = NT + 32;  // consumers + the producer warp
constexpr int kSweepMinCtas = 4;        // CTAs per SM the register budget allows (__launch_bounds__)

struct Ring {
  double* buf;      // kStages x kTile
  uint64_t* full;   // kStages: the copy landed (1 arrival + bytes)
  uint64_t* empty;  // kStages: every consumer warp is done with it (NT / 32 arrivals)
};

__device__ __forceinline__ Ring ring_at(unsigned char* smem) {
  double* buf = reinterpret_cast<double*>(smem);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + (size_t)kStages * kTile * sizeof(double));
  return Ring{buf, bars, bars + kStages};
}

// Producer lane: the copy of element q (vector vp, local tile lt of CTA cta of P) into buffer
// q % kStages.
__device__ __forceinline__ void ring_issue(const Ring& rg, int q, const double* vp, long long n, int lt, int cta,
                                           int P) {
  const int st = q % kStages;
  const long long base = (long long)(cta + (long long)lt * P) * kTile;
  const long long cnt = min((long long)kTile, n - base);
  const uint32_t bytes = (uint32_t)((cnt * 8 + 15) & ~15ll);  // an odd count reads the 8-byte pad
  fence_proxy_async();
  mbar_expect_tx(&rg.full[st], bytes);
  bulk_g2s(rg.buf + (size_t)st * kTile, vp + base, bytes, &rg.full[st]);
}

// Producer (lane 0 of the last warp): issues elements 0 .. total-1, each once its buffer is
// free; vec(q) gives the source vector.  On a wait that runs out it records the error and
// waits for every copy it issued before returning.
template <typename VecOf>
__device__ __forceinline__ void ring_produce(const Ring& rg, int total, long long n, int per, VecOf vec, int* err,
                                             int cta, int P) {
  int issued = 0;
  bool ok = true;
  for (int q = 0; q < total; ++q) {
    const int st = q % kStages;
    if (q >= kStages && !(ok = mbar_wait_bounded(&rg.empty[st], (uint32_t)((q / kStages - 1) & 1)))) break;
    ring_issue(rg, q, vec(q % per), n, q / per, cta, P);
    issued = q + 1;
  }
  if (!ok) {
    if (err) atomicExch(err, PFC_ETIMEOUT);
    for (int u = max(0, issued - kStages); u < issued; ++u)  // the last copy issued into each buffer
      mbar_wait_bounded(&rg.full[u % kStages], (uint32_t)((u / kStages) & 1));
  }
}

// The skip flags of a sweep (cycle done; second Gram-Schmidt pass not wanted), read by one
// thread per CTA: a skipped sweep costs one load per CTA instead of one per thread.
__device__ __forceinline__ bool sweep_skipped(const int* skip, const int* only_if) {
  __shared__ int s_skip;
  if (threadIdx.x == 0) s_skip = (skip && *skip) || (only_if && !*only_if);
  __syncthreads();
  return s_skip != 0;
}

// Consumer side: wait for element q (false when the wait ran out) and release it.
__device__ __forceinline__ bool ring_wait(const Ring& rg, int q) {
  return mbar_wait_bounded(&rg.full[q % kStages], (uint32_t)((q / kStages) & 1));
}
__device__ __forceinline__ void ring_release(const Ring& rg, int q) {
  __syncwarp();
  if ((threadIdx.x & 31) == 0) mbar_arrive(&rg.empty[q % kStages]);
}

__device__ __forceinline__ void ring_init(const Ring& rg) {
  if (threadIdx.x == 0) {
    for (int st = 0; st < kStages; ++st) {
      mbar_init(&rg.full[st], 1);
      mbar_init(&rg.empty[st], NT / 32);
    }
    fence_mbar_init();
  }
  __syncthreads();
}

// Arithmetic of the multi-dot products: FP64, float-float, or FP32 from values cut to floats.
enum Dot { kF64 = 0, kFF = 1, kF32 = 2 };

// The multi-dot of this CTA's group of up to G vectors against w (wv: w in FP64,
// wff: w split into float pairs, wf: w cut to floats).
// PR: the vectors are stored as float pairs (the mixed path's basis): every point in
// float-float (or FP32 from the leading floats), no split and no FP64 part.
template <int D, bool PR>
__device__ __forceinline__ void dot_tile(const double* tb, int cntp, const double* wv, const ff* wff, const float* wf,
                                         double* acc, ff* aff, float* af, int k) {
#pragma unroll
  for (int p = 0; p < kPts; ++p) {
    const int i = threadIdx.x + p * NT;
    if (i < cntp) {
      if (PR) {
        const ff v = ld_pair(tb, i);
        if (D == kF32)
          af[k] = __fmaf_rn(v.hi, wf[p], af[k]);
        else
          aff[k] = ff_acc(aff[k], ff_prod(v, wff[p]));
        continue;
      }
      const double v = tb[i];
      if (D == kF32)
        af[k] = __fmaf_rn(f32_cut(v), wf[p], af[k]);
      else if (D == kFF && p >= kPd)
        aff[k] = ff_acc(aff[k], ff_prod(ff_split(v), wff[p]));
      else
        acc[k] = fma(v, wv[p], acc[k]);
    }
  }
}

// partial[(g0 + k) * P + cta] = sum_i V_{g0+k}[i] * w[i] over this CTA's tiles (P CTAs per group).
// PR: V and w stored as float pairs (D = kFF or kF32).
template <int D, bool PR>
__global__ void __launch_bounds__(kSweepThreads, kSweepMinCtas)
    k_multidot(const double* v0, const double* const* __restrict__ tab, int nv, const double* w, long long n,
               double* __restrict__ partial, const int* __restrict__ skip, const int* __restrict__ only_if, Tail tail) {
  pdl_wait();
  if (sweep_skipped(skip, only_if)) return;
  if (tail.ia) {  // graph mode: this iteration's vector count and w
    nv = tail.ia->j + 2;
    w = tail.ia->w;
  }
  extern __shared__ __align__(128) unsigned char smem[];
  const Ring rg = ring_at(smem);
  __shared__ double red[NT / 32][G];
  __shared__ const double* sp[G + 1];
  // The 1D grid is split evenly over the gy = ceil(nv / G) groups this sweep has (however
  // many the grid was sized for): P CTAs per group, CTA c of group g takes tiles c, c + P, ...;
  // CTAs past gy * P only take a ticket.  The nv vectors are dealt to the groups in sizes that
  // differ by at most one (9 vectors as 5 + 4, not 8 + 1), so that no group's CTAs wait idle
  // on the others.
  const int gy = (nv + G - 1) / G, P = gridDim.x / gy;
  const int grp = blockIdx.x / P, cta = blockIdx.x - grp * P;
  const int gbase = nv / gy, grem = nv - gbase * gy;
  const int g0 = grp * gbase + min(grp, grem);
  const int cnt = grp < gy ? gbase + (grp < grem ? 1 : 0) : 0;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  if (tid <= G) sp[tid] = tid == 0 ? w : (tid - 1 < cnt ? vec_at(v0, tab, g0 + tid - 1) : w);
  const long long ntile = (n + kTile - 1) / kTile;
  const int my_tiles = cnt > 0 && cta < ntile ? (int)((ntile - 1 - cta) / P + 1) : 0;
  const int per = 1 + cnt, total = my_tiles * per;
  ring_init(rg);  // also makes sp visible
  double acc[G];
  float af[G];
  ff aff[G];
#pragma unroll
  for (int k = 0; k < G; ++k) {
    acc[k] = 0.0;
    af[k] = 0.0f;
    aff[k] = {0.0f, 0.0f};
  }
  if (wid == NT / 32) {  // producer warp
    if (lane == 0) ring_produce(rg, total, n, per, [&](int k) { return sp[k]; }, tail.err, cta, P);
  } else {
    bool ok = true;
    int q = 0;
    for (int lt = 0; lt < my_tiles && ok; ++lt) {
      const long long base = (long long)(cta + (long long)lt * P) * kTile;
      const int cntp = (int)min((long long)kTile, n - base);
      double wv[kPts];
      float wf[kPts];
      ff wff[kPts];
      if (!(ok = ring_wait(rg, q))) break;
      {
        const double* tb = rg.buf + (size_t)(q % kStages) * kTile;
#pragma unroll
        for (int p = 0; p < kPts; ++p) {
          const int i = tid + p * NT;
          if (PR) {
            wff[p] = i < cntp ? ld_pair(tb, i) : ff{0.0f, 0.0f};
            wf[p] = wff[p].hi;
            continue;
          }
          wv[p] = i < cntp ? tb[i] : 0.0;
          if (D == kF32) wf[p] = f32_cut(wv[p]);
          if (D == kFF && p >= kPd) wff[p] = ff_split(wv[p]);
        }
      }
      ring_release(rg, q++);
#pragma unroll
      for (int k = 0; k < G; ++k) {
        if (k < cnt) {  // block-uniform
          if (!(ok = ring_wait(rg, q))) break;
          dot_tile<D, PR>(rg.buf + (size_t)(q % kStages) * kTile, cntp, wv, wff, wf, acc, aff, af, k);
          ring_release(rg, q++);
        }
      }
    }
    if (!ok && lane == 0 && tail.err) atomicExch(tail.err, PFC_ETIMEOUT);
    if (D == kF32) {
#pragma unroll
      for (int k = 0; k < G; ++k) acc[k] = f2d_bits(af[k]);
    }
    if (D == kFF) {  // the FP64 part plus the pair's sum (two FP64 adds per value and thread)
#pragma unroll
      for (int k = 0; k < G; ++k) acc[k] += ff_to_double(aff[k]);
    }
    // Warp reduce-scatter of the G = 8 sums: each halving step sends the half of the
    // values a lane does not keep, so a lane adds 4 + 2 + 1 values and then
    // finishes one value over the remaining 4 lanes of its quarter (9 FP64 adds
    // per lane instead of 8 full butterflies).  Lane l ends with the sum of value
    // 4 b4 + 2 b3 + b2 (b_i = bit i of l).
    static_assert(G == 8, "reduce-scatter written for 8 values");
    const unsigned FULL = 0xffffffffu;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const bool up = lane & 16;
      const double send = up ? acc[i] : acc[i + 4];
      const double keep = up ? acc[i + 4] : acc[i];
      acc[i] = keep + __shfl_xor_sync(FULL, send, 16);
    }
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const bool up = lane & 8;
      const double send = up ? acc[i] : acc[i + 2];
      const double keep = up ? acc[i + 2] : acc[i];
      acc[i] = keep + __shfl_xor_sync(FULL, send, 8);
    }
    {
      const bool up = lane & 4;
      const double send = up ? acc[0] : acc[1];
      const double keep = up ? acc[1] : acc[0];
      acc[0] = keep + __shfl_xor_sync(FULL, send, 4);
    }
    acc[0] += __shfl_xor_sync(FULL, acc[0], 2);
    acc[0] += __shfl_xor_sync(FULL, acc[0], 1);
    if ((lane & 3) == 0) red[wid][((lane >> 4) & 1) * 4 + ((lane >> 3) & 1) * 2 + ((lane >> 2) & 1)] = acc[0];
  }
  pdl_trigger();
  __syncthreads();  // also keeps the CTA alive until the producer has drained its copies
  if (tid < cnt) {
    double s = 0.0;
    for (int qq = 0; qq < NT / 32; ++qq) s += red[qq][tid];
    partial[(size_t)(g0 + tid) * P + cta] = s;
  }
  if (tail.counter) last_cta_tail(tail, partial, nv, P);
}

// w = w + sign * sum_k coef[k] X_k over this CTA's tiles (the tile of w comes last);
// partial[0..] = sum w^2, and with SUM partial[gridDim..] = sum w.  FF: the sum over
// k in float-float, one FP64 addition per point to store w.  PR (with FF, without SUM): X
// and w stored as float pairs, every point in float-float, w stored as a normalised pair and
// sum w^2 taken in float-float.
template <bool SUM, bool FF, bool PR>
__global__ void __launch_bounds__(kSweepThreads, kSweepMinCtas)
    k_multiaxpy(double* __restrict__ w, const double* x0, const double* const* __restrict__ tab, int nx,
                const double* __restrict__ coef, double sign, long long n, double* __restrict__ partial,
                const int* __restrict__ skip, const int* __restrict__ only_if, Tail tail) {
  pdl_wait();
  if (sweep_skipped(skip, only_if)) return;
  if (tail.ia) {  // graph mode: this iteration's vector count and w
    nx = tail.ia->j + 1;
    w = tail.ia->w;
  }
  if (tail.nx_dev) nx = *tail.nx_dev;  // graph mode: the count of a finished cycle
  extern __shared__ __align__(128) unsigned char smem[];
  const Ring rg = ring_at(smem);
  __shared__ double red[2][NT / 32];
  __shared__ double c[kMaxVecs];
  __shared__ ff cf[kMaxVecs];
  __shared__ const double* sp[kMaxVecs + 1];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  for (int k = tid; k <= nx; k += kSweepThreads) {
    if (k < nx) {
      c[k] = sign * coef[k];
      cf[k] = ff_of(sign * coef[k]);
    }
    sp[k] = k < nx ? vec_at(x0, tab, k) : w;
  }
  const long long ntile = (n + kTile - 1) / kTile;
  const int my_tiles = blockIdx.x < ntile ? (int)((ntile - 1 - blockIdx.x) / gridDim.x + 1) : 0;
  const int per = nx + 1, total = my_tiles * per;
  ring_init(rg);  // also makes c, cf, sp visible
  double s2 = 0.0, s1 = 0.0;
  ff s2f = {0.0f, 0.0f};
  if (wid == NT / 32) {  // producer warp
    if (lane == 0) ring_produce(rg, total, n, per, [&](int k) { return sp[k]; }, tail.err, blockIdx.x, gridDim.x);
  } else {
    bool ok = true;
    int q = 0;
    for (int lt = 0; lt < my_tiles && ok; ++lt) {
      const long long base = (long long)(blockIdx.x + (long long)lt * gridDim.x) * kTile;
      const int cntp = (int)min((long long)kTile, n - base);
      double acc[kPts];
      ff af[kPts];
#pragma unroll
      for (int p = 0; p < kPts; ++p) {
        acc[p] = 0.0;
        af[p] = {0.0f, 0.0f};
      }
      for (int k = 0; k <= nx; ++k) {
        if (!(ok = ring_wait(rg, q))) break;
        const double* tb = rg.buf + (size_t)(q % kStages) * kTile;
        if (k < nx) {
          const double ck = c[k];
          const ff cfk = cf[k];
#pragma unroll
          for (int p = 0; p < kPts; ++p) {
            const int i = tid + p * NT;
            if (i < cntp) {
              if (PR)
                af[p] = ff_acc(af[p], ff_prod(cfk, ld_pair(tb, i)));
              else if (FF && p >= kPd)
                af[p] = ff_acc(af[p], ff_prod(cfk, ff_split(tb[i])));
              else
                acc[p] = fma(ck, tb[i], acc[p]);
            }
          }
        } else {  // the tile of w: add and store
#pragma unroll
          for (int p = 0; p < kPts; ++p) {
            const int i = tid + p * NT;
            if (i < cntp) {
              if (PR) {
                const ff a = ff_acc(ld_pair(tb, i), af[p]);
                const ff wn = fast_two_sum(a.hi, a.lo);
                st_pair(w, base + i, wn);
                s2f = ff_acc(s2f, ff_prod(wn, wn));
                continue;
              }
              const double wn = FF && p >= kPd ? ff_to_double(ff_acc(ff_split(tb[i]), af[p])) : tb[i] + acc[p];
              w[base + i] = wn;
              s2 = fma(wn, wn, s2);
              if (SUM) s1 += wn;
            }
          }
        }
        ring_release(rg, q++);
      }
    }
    if (!ok && lane == 0 && tail.err) atomicExch(tail.err, PFC_ETIMEOUT);
    if (PR) s2 = ff_to_double(s2f);
    s2 = warp_sum(s2);
    s1 = warp_sum(s1);
    if (lane == 0) {
      red[0][wid] = s2;
      red[1][wid] = s1;
    }
  }
  pdl_trigger();
  __syncthreads();  // also keeps the CTA alive until the producer has drained its copies
  if (tid < (SUM ? 2 : 1)) {
    double s = 0.0;
    for (int qq = 0; qq < NT / 32; ++qq) s += red[tid][qq];
    partial[(size_t)tid * gridDim.x + blockIdx.x] = s;
  }
  if (tail.counter) last_cta_tail(tail, partial, SUM ? 2 : 1, gridDim.x);
}

// out[v] = sum_p partial[v * nparts + p], fixed order.
__global__ void __launch_bounds__(1024) k_reduce(const double* __restrict__ partial, int nvals, int nparts,
                                                 double* __restrict__ out) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int v = wid; v < nvals; v += 32) {
    double s = 0.0;
    for (int p = lane; p < nparts; p += 32) s += partial[(size_t)v * nparts + p];
    s = warp_sum(s);
    if (lane == 0) out[v] = s;
  }
}

__global__ void k_gmres_init(GmresCtl* c, const double* __restrict__ nrm2, double sign, double tol, double eta2) {
  const double beta = sqrt(*nrm2);
  c->done = 0;
  c->its = 0;
  c->reorth = 0;
  c->breakdown = 0;
  c->tol = tol;
  c->reorth_eta2 = eta2;
  c->beta = beta;
  c->est = beta;
  c->g[0] = beta;
  c->scale[0] = beta > 0.0 ? sign / beta : 0.0;
  if (!(beta > tol)) c->done = 1;
}

// y = R^{-1} g over the completed iterations (R = rotated Hessenberg).
// Back substitution R y = g of the rotated Hessenberg system (k <= kMaxRestart = 60 rows), by
// one warp, column by column: lane l keeps rows l and l + 32 of g and subtracts H(i, j) y_j from
// them as each y_j becomes final (FP64).
__global__ void __launch_bounds__(32) k_gmres_solve(GmresCtl* c) {
  static_assert(kMaxRestart <= 64, "two rows per lane");
  const int m1 = kMaxRestart + 1;
  const int k = c->its;
  const int lane = threadIdx.x;
  double g0 = lane < k ? c->g[lane] : 0.0, g1 = lane + 32 < k ? c->g[lane + 32] : 0.0;
  for (int j = k - 1; j >= 0; --j) {
    const double gj = __shfl_sync(0xffffffffu, j < 32 ? g0 : g1, j & 31);
    const double yj = gj / c->H[j + m1 * j];
    if (lane == (j & 31)) c->y[j] = yj;
    if (lane < j) g0 = fma(-c->H[lane + m1 * j], yj, g0);
    if (lane + 32 < j) g1 = fma(-c->H[lane + 32 + m1 * j], yj, g1);
  }
}

__global__ void k_axpby(double* __restrict__ y, const double* __restrict__ x, double a, double b, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = fma(a, y[i], b * x[i]);
}

__global__ void k_extrapolate(double* __restrict__ out, const double* __restrict__ a, const double* __restrict__ b,
                              double ratio, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = fma(ratio, a[i] - b[i], a[i]);
}

// The Arnoldi loop's condition, and the vectors of the iteration it lets run.
__global__ void k_arnoldi_next(const GmresCtl* __restrict__ ctl, const double* const* __restrict__ vtab,
                               const double* const* __restrict__ ztab, IterArgs* __restrict__ ia, int m,
                               cudaGraphConditionalHandle h) {
  pdl_wait();
  const int j = ctl->its;
  const bool go = !ctl->done && j < m;
  if (go) {
    ia->j = j;
    ia->v = vtab[j];
    ia->z = const_cast<double*>(ztab[j]);
    ia->zplane = j;
    ia->w = const_cast<double*>(vtab[j + 1]);
    ia->scale = &ctl->scale[j];
  }
  cudaGraphSetConditional(h, go ? 1u : 0u);
}

int red_ctas(long long n) {
  long long b = (n + NT - 1) / NT;
  return (int)(b < kRedCtas ? (b < 1 ? 1 : b) : kRedCtas);
}

}  // namespace

void launch_multidot(const double* v0, const double* const* tab, int nv, const double* w, long long n,
                     double* partial, const int* skip, const int* only_if, const Tail& tail, cudaStream_t st,
                     int dot, int nv_grid, bool pairs) {
  // groups of G vectors in y; about kSweepMinCtas CTAs per SM in all.  The grid is sized for
  // nv_grid vectors (>= nv): a sweep then splits the points over CTAs as the graph form's
  // sweeps do (sized for the restart length), so both sum in the same order.
  const int gy = (std::max(nv, nv_grid) + G - 1) / G;
  const long long ntile = (n + kTile - 1) / kTile;
  const int bx = (int)std::max(1ll, std::min(ntile, (long long)(kRedCtas / gy)));
  const dim3 grid(bx * gy);  // split over the groups the sweep has inside the kernel
  const size_t smem = (size_t)kStages * kTile * sizeof(double) + 2 * kStages * 8;
#define PFC_DOT(D, PR)                                                                                    \
  do {                                                                                                    \
    cudaFuncSetAttribute(k_multidot<D, PR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);      \
    launch_pdl(k_multidot<D, PR>, grid, dim3(kSweepThreads), smem, st, v0, tab, nv, w, n, partial, skip, only_if, \
               tail);                                                                                       \
  } while (0)
  if (dot == kDotFF && pairs)
    PFC_DOT(kFF, true);
  else if (dot == kDotF32 && pairs)
    PFC_DOT(kF32, true);
  else if (dot == kDotFF)
    PFC_DOT(kFF, false);
  else if (dot == kDotF32)
    PFC_DOT(kF32, false);
  else
    PFC_DOT(kF64, false);
#undef PFC_DOT
  count_launches(1);
}

void launch_multiaxpy(double* w, const double* x0, const double* const* tab, int nx, const double* coef, double sign,
                      long long n, double* partial, const int* skip, const int* only_if, const Tail& tail,
                      cudaStream_t st, bool ff, bool pairs) {
  const long long ntile = (n + kTile - 1) / kTile;
  const int bx = (int)std::max(1ll, std::min(ntile, (long long)kRedCtas));
  const size_t smem = (size_t)kStages * kTile * sizeof(double) + 2 * kStages * 8;
  // the sum of w is read only by the kSums tail (and by callers of partials-only sweeps)
  const bool sum = !(tail.counter && tail.kind != Tail::kSums);
#define PFC_AXPY(S, F, PR)                                                                              \
  do {                                                                                                  \
    cudaFuncSetAttribute(k_multiaxpy<S, F, PR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
    launch_pdl(k_multiaxpy<S, F, PR>, dim3(bx), dim3(kSweepThreads), smem, st, w, x0, tab, nx, coef, sign, n,   \
               partial, skip, only_if, tail);                                                           \
  } while (0)
  if (pairs && sum) {  // float-pair vectors come with no sum of w (the Gram-Schmidt sweeps only)
    fprintf(stderr, "libpfc: float-pair multi-axpy with the sum of w\n");
    static const int kInvalid = PFC_EINVAL;  // the step then fails with this status
    if (tail.err) cudaMemcpyAsync(tail.err, &kInvalid, sizeof kInvalid, cudaMemcpyHostToDevice, st);
    return;
  }
  if (pairs)
    PFC_AXPY(false, true, true);
  else if (sum && ff)
    PFC_AXPY(true, true, false);
  else if (sum)
    PFC_AXPY(true, false, false);
  else if (ff)
    PFC_AXPY(false, true, false);
  else
    PFC_AXPY(false, false, false);
#undef PFC_AXPY
  count_launches(1);
}

void launch_arnoldi_next(const GmresCtl* ctl, const double* const* vtab, const double* const* ztab, IterArgs* ia,
                         int m, cudaGraphConditionalHandle h, cudaStream_t st) {
  launch_pdl(k_arnoldi_next, dim3(1), dim3(1), 0, st, ctl, vtab, ztab, ia, m, h);
  count_launches(1);
}

void launch_reduce(const double* partial, int nvals, int nparts, double* out, cudaStream_t st) {
  k_reduce<<<1, 1024, 0, st>>>(partial, nvals, nparts, out);
  count_launches(1);
}

void launch_gmres_init(GmresCtl* ctl, const double* nrm2, double sign, double tol, double reorth_eta2,
                       cudaStream_t st) {
  k_gmres_init<<<1, 1, 0, st>>>(ctl, nrm2, sign, tol, reorth_eta2);
  count_launches(1);
}
void launch_gmres_solve(GmresCtl* ctl, cudaStream_t st) {
  k_gmres_solve<<<1, 32, 0, st>>>(ctl);
  count_launches(1);
}

void launch_axpby(double* y, const double* x, double a, double b, long long n, cudaStream_t st) {
  k_axpby<<<red_ctas(n), NT, 0, st>>>(y, x, a, b, n);
  count_launches(1);
}
void launch_extrapolate(double* out, const double* a, const double* b, double ratio, long long n, cudaStream_t st) {
  k_extrapolate<<<red_ctas(n), NT, 0, st>>>(out, a, b, ratio, n);
  count_launches(1);
}

}  // namespace pfc
