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
// On the mixed path (F32/BF16 factors) the Arnoldi sweeps run in the float-float
// arithmetic of ff.cuh on the FP32 pipe (FF = true): the multi-dot products and the
// multi-axpy w -= sum c_k V_k carry 48-bit significands and the new w is stored
// in FP64.  The Arnoldi relation J Z_j = V H holds to that accuracy whatever the
// coefficients, so GMRES sees FP64-grade vectors at FP32-pipe cost.
//
// The basis is kept unnormalised: V_i = scale_i * Vraw_i with scale_i held on
// the device, so no kernel pass is spent on normalising.  Every kernel takes
// the cycle's "done" flag and returns at once when it is set, which lets the
// host queue several iterations ahead and synchronise rarely.
#include <algorithm>
#include <cmath>

#include "ff.cuh"
#include "pfc_internal.cuh"

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

// After a multi-dot of V_0..V_j against w (c->red[0..j]) and w.w (c->red[j+1]).
__device__ void gmres_after_dot(GmresCtl* c, int j, int pass) {
  const int m1 = kMaxRestart + 1;
  for (int i = 0; i <= j; ++i) {
    const double h = c->scale[i] * c->red[i];
    if (pass == 0)
      c->H[i + m1 * j] = h;
    else
      c->H[i + m1 * j] += h;
    c->coef[i] = h * c->scale[i];
  }
  if (pass == 0) c->wnorm2_before = c->red[j + 1];
}

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
  for (int v = wid; v < nvals; v += NT / 32) {
    double s = 0.0;
    for (int p = lane; p < nparts; p += 32) s += __ldcg(partial + (size_t)v * nparts + p);
    s = warp_sum(s);
    if (lane == 0) s_sum[v] = s;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    GmresCtl* c = t.ctl;
    const int j = t.ia ? t.ia->j : t.j;
    if (t.kind == Tail::kDot) {
      for (int v = 0; v < nvals; ++v) c->red[v] = s_sum[v];
      gmres_after_dot(c, j, t.pass);
    } else if (t.kind == Tail::kAxpy) {
      gmres_after_axpy(c, j, t.pass, t.m, s_sum[0]);
    } else {
      for (int v = 0; v < nvals; ++v) t.out[v] = s_sum[v];
    }
    *t.counter = 0u;  // ready for the next kernel on this stream
  }
}

// acc[k] += sum over this thread's pairs of points of V_k . w, for exactly C vectors
// (a compile-time count: no predicated-off FP64 work for a partial group).
template <int C>
__device__ __forceinline__ void dot_sweep(const double* const* p, const double2* __restrict__ w2, long long n2,
                                          long long start, long long stride, double* acc) {
  for (long long i = start; i < n2; i += stride) {
    const double2 wi = w2[i];
#pragma unroll
    for (int k = 0; k < C; ++k) {
      const double2 a = reinterpret_cast<const double2*>(p[k])[i];
      acc[k] = fma(a.y, wi.y, fma(a.x, wi.x, acc[k]));
    }
  }
}

// The same sweep in float-float: acc[k] (hi) and accl[k] (lo).
template <int C>
__device__ __forceinline__ void dot_sweep_ff(const double* const* p, const double2* __restrict__ w2, long long n2,
                                             long long start, long long stride, double* acc) {
  ff a[C];
#pragma unroll
  for (int k = 0; k < C; ++k) a[k] = {0.0f, 0.0f};
  for (long long i = start; i < n2; i += stride) {
    const double2 wi = w2[i];
    const ff wx = ff_of(wi.x), wy = ff_of(wi.y);
#pragma unroll
    for (int k = 0; k < C; ++k) {
      const double2 v = reinterpret_cast<const double2*>(p[k])[i];
      a[k] = ff_acc(a[k], ff_prod(ff_of(v.x), wx));
      a[k] = ff_acc(a[k], ff_prod(ff_of(v.y), wy));
    }
  }
#pragma unroll
  for (int k = 0; k < C; ++k) acc[k] = ff_to_double(a[k]);
}

// partial[(g0 + k) * gridDim.x + blockIdx.x] = sum_i V_{g0+k}[i] * w[i]; pairs of points per
// 16-byte load (every vector starts 256-byte aligned).
template <bool FF>
__global__ void __launch_bounds__(NT) k_multidot(const double* v0, const double* const* __restrict__ tab, int nv,
                                                 const double* __restrict__ w, long long n,
                                                 double* __restrict__ partial, const int* __restrict__ skip,
                                                 const int* __restrict__ only_if, Tail tail) {
  if ((skip && *skip) || (only_if && !*only_if)) return;
  if (tail.ia) {  // graph mode: this iteration's vector count and w
    nv = tail.ia->j + 2;
    w = tail.ia->w;
  }
  __shared__ double red[NT / 32][G];
  __shared__ const double* sp[G];
  const int g0 = blockIdx.y * G;
  const int cnt = min(G, nv - g0);  // <= 0 for spare groups of a graph-mode grid: they only take a ticket
  if (threadIdx.x < G) sp[threadIdx.x] = threadIdx.x < cnt ? vec_at(v0, tab, g0 + threadIdx.x) : w;
  __syncthreads();
  const double* p[G];
#pragma unroll
  for (int k = 0; k < G; ++k) p[k] = sp[k];
  double acc[G];
#pragma unroll
  for (int k = 0; k < G; ++k) acc[k] = 0.0;
  const long long n2 = n >> 1;
  const long long stride = (long long)gridDim.x * NT;
  const double2* w2 = reinterpret_cast<const double2*>(w);
  const long long start = blockIdx.x * (long long)NT + threadIdx.x;
  if (FF) {
    switch (cnt) {  // block-uniform
      case 0: break;
      case 1: dot_sweep_ff<1>(p, w2, n2, start, stride, acc); break;
      case 2: dot_sweep_ff<2>(p, w2, n2, start, stride, acc); break;
      case 3: dot_sweep_ff<3>(p, w2, n2, start, stride, acc); break;
      case 4: dot_sweep_ff<4>(p, w2, n2, start, stride, acc); break;
      case 5: dot_sweep_ff<5>(p, w2, n2, start, stride, acc); break;
      case 6: dot_sweep_ff<6>(p, w2, n2, start, stride, acc); break;
      case 7: dot_sweep_ff<7>(p, w2, n2, start, stride, acc); break;
      default:
        if (cnt > 0) dot_sweep_ff<G>(p, w2, n2, start, stride, acc);
    }
  } else {
    switch (cnt) {  // block-uniform
      case 0: break;
      case 1: dot_sweep<1>(p, w2, n2, start, stride, acc); break;
      case 2: dot_sweep<2>(p, w2, n2, start, stride, acc); break;
      case 3: dot_sweep<3>(p, w2, n2, start, stride, acc); break;
      case 4: dot_sweep<4>(p, w2, n2, start, stride, acc); break;
      case 5: dot_sweep<5>(p, w2, n2, start, stride, acc); break;
      case 6: dot_sweep<6>(p, w2, n2, start, stride, acc); break;
      case 7: dot_sweep<7>(p, w2, n2, start, stride, acc); break;
      default:
        if (cnt > 0) dot_sweep<G>(p, w2, n2, start, stride, acc);
    }
  }
  if ((n & 1) && blockIdx.x == 0 && threadIdx.x == 0) {  // odd tail
    const double wi = w[n - 1];
#pragma unroll
    for (int k = 0; k < G; ++k)
      if (k < cnt) acc[k] = fma(p[k][n - 1], wi, acc[k]);
  }
  // Warp reduce-scatter of the G = 8 sums: each halving step sends the half of the
  // values a lane does not keep, so a lane adds 4 + 2 + 1 values and then
  // finishes one value over the remaining 4 lanes of its quarter (9 FP64 adds
  // per lane instead of 8 full butterflies).  Lane l ends with the sum of value
  // 4 b4 + 2 b3 + b2 (b_i = bit i of l).
  static_assert(G == 8, "reduce-scatter written for 8 values");
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
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
  __syncthreads();
  if ((int)threadIdx.x < cnt) {
    double s = 0.0;
    for (int q = 0; q < NT / 32; ++q) s += red[q][threadIdx.x];
    partial[(size_t)(g0 + threadIdx.x) * gridDim.x + blockIdx.x] = s;
  }
  if (tail.counter) last_cta_tail(tail, partial, nv, gridDim.x);
}

// w = w + sign * sum_k coef[k] X_k ; partial[0..] = sum w^2, and with SUM partial[gridDim..] = sum w
// (FF: the sum over k in float-float, one FP64 addition per point to store w)
template <bool SUM, bool FF>
__global__ void __launch_bounds__(NT) k_multiaxpy(double* __restrict__ w, const double* x0,
                                                  const double* const* __restrict__ tab, int nx,
                                                  const double* __restrict__ coef, double sign, long long n,
                                                  double* __restrict__ partial, const int* __restrict__ skip,
                                                  const int* __restrict__ only_if, Tail tail) {
  if ((skip && *skip) || (only_if && !*only_if)) return;
  if (tail.ia) {  // graph mode: this iteration's vector count and w
    nx = tail.ia->j + 1;
    w = tail.ia->w;
  }
  __shared__ double red[2][NT / 32];
  __shared__ double c[kMaxVecs];
  __shared__ ff cf[kMaxVecs];
  __shared__ const double* sp[kMaxVecs];
  for (int k = threadIdx.x; k < nx; k += NT) {
    c[k] = sign * coef[k];
    cf[k] = ff_of(sign * coef[k]);
    sp[k] = vec_at(x0, tab, k);
  }
  __syncthreads();
  double s2 = 0.0, s1 = 0.0;
  const long long n2 = n >> 1;
  const long long stride = (long long)gridDim.x * NT;
  double2* w2 = reinterpret_cast<double2*>(w);
  for (long long i = blockIdx.x * (long long)NT + threadIdx.x; i < n2; i += stride) {
    double2 acc = w2[i];
    if (FF) {
      ff ax = ff_of(acc.x), ay = ff_of(acc.y);
#pragma unroll 4
      for (int k = 0; k < nx; ++k) {
        const double2 a = reinterpret_cast<const double2*>(sp[k])[i];
        const ff ck = cf[k];
        ax = ff_acc(ax, ff_prod(ck, ff_of(a.x)));
        ay = ff_acc(ay, ff_prod(ck, ff_of(a.y)));
      }
      acc.x = ff_to_double(ax);
      acc.y = ff_to_double(ay);
    } else {
#pragma unroll 4
      for (int k = 0; k < nx; ++k) {
        const double2 a = reinterpret_cast<const double2*>(sp[k])[i];
        acc.x = fma(c[k], a.x, acc.x);
        acc.y = fma(c[k], a.y, acc.y);
      }
    }
    w2[i] = acc;
    s2 = fma(acc.y, acc.y, fma(acc.x, acc.x, s2));
    if (SUM) s1 += acc.x + acc.y;
  }
  if ((n & 1) && blockIdx.x == 0 && threadIdx.x == 0) {  // odd tail
    double acc = w[n - 1];
    for (int k = 0; k < nx; ++k) acc = fma(c[k], sp[k][n - 1], acc);
    w[n - 1] = acc;
    s2 = fma(acc, acc, s2);
    s1 += acc;
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  s2 = warp_sum(s2);
  s1 = warp_sum(s1);
  if (lane == 0) {
    red[0][wid] = s2;
    red[1][wid] = s1;
  }
  __syncthreads();
  if (threadIdx.x < (SUM ? 2 : 1)) {
    double s = 0.0;
    for (int q = 0; q < NT / 32; ++q) s += red[threadIdx.x][q];
    partial[(size_t)threadIdx.x * gridDim.x + blockIdx.x] = s;
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
__global__ void k_gmres_solve(GmresCtl* c) {
  const int m1 = kMaxRestart + 1;
  const int k = c->its;
  for (int i = k - 1; i >= 0; --i) {
    double s = c->g[i];
    for (int l = i + 1; l < k; ++l) s -= c->H[i + m1 * l] * c->y[l];
    c->y[i] = s / c->H[i + m1 * i];
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

__global__ void k_iter_setup(const GmresCtl* __restrict__ ctl, const double* const* __restrict__ vtab,
                             const double* const* __restrict__ ztab, IterArgs* __restrict__ ia) {
  const int j = ctl->its;
  ia->j = j;
  ia->v = vtab[j];
  ia->z = const_cast<double*>(ztab[j]);
  ia->w = const_cast<double*>(vtab[j + 1]);
  ia->scale = &ctl->scale[j];
}

// Keeps the graph's while loop running until the cycle is done (converged, broken
// down or at the restart length).
__global__ void k_cycle_cond(const GmresCtl* __restrict__ ctl, int m, cudaGraphConditionalHandle h) {
  cudaGraphSetConditional(h, (!ctl->done && ctl->its < m) ? 1u : 0u);
}

int red_ctas(long long n) {
  long long b = (n + NT - 1) / NT;
  return (int)(b < kRedCtas ? (b < 1 ? 1 : b) : kRedCtas);
}

}  // namespace

void launch_multidot(const double* v0, const double* const* tab, int nv, const double* w, long long n,
                     double* partial, const int* skip, const int* only_if, const Tail& tail, cudaStream_t st,
                     bool ff) {
  // half the CTAs of the other sweeps: each thread covers twice the points, so the
  // per-CTA reduction of 8 sums is a smaller share of the FP64 work
  const int bx = std::max(1, red_ctas((n + 1) / 2) / 2);
  dim3 grid(bx, (nv + G - 1) / G);
  if (ff)
    k_multidot<true><<<grid, NT, 0, st>>>(v0, tab, nv, w, n, partial, skip, only_if, tail);
  else
    k_multidot<false><<<grid, NT, 0, st>>>(v0, tab, nv, w, n, partial, skip, only_if, tail);
  count_launches(1);
}

void launch_multiaxpy(double* w, const double* x0, const double* const* tab, int nx, const double* coef, double sign,
                      long long n, double* partial, const int* skip, const int* only_if, const Tail& tail,
                      cudaStream_t st, bool ff) {
  const int bx = red_ctas((n + 1) / 2);
  // the sum of w is read only by the kSums tail (and by callers of partials-only sweeps)
  const bool sum = !(tail.counter && tail.kind != Tail::kSums);
  if (sum && ff)
    k_multiaxpy<true, true><<<bx, NT, 0, st>>>(w, x0, tab, nx, coef, sign, n, partial, skip, only_if, tail);
  else if (sum)
    k_multiaxpy<true, false><<<bx, NT, 0, st>>>(w, x0, tab, nx, coef, sign, n, partial, skip, only_if, tail);
  else if (ff)
    k_multiaxpy<false, true><<<bx, NT, 0, st>>>(w, x0, tab, nx, coef, sign, n, partial, skip, only_if, tail);
  else
    k_multiaxpy<false, false><<<bx, NT, 0, st>>>(w, x0, tab, nx, coef, sign, n, partial, skip, only_if, tail);
  count_launches(1);
}

void launch_iter_setup(GmresCtl* ctl, const double* const* vtab, const double* const* ztab, IterArgs* ia,
                       cudaStream_t st) {
  k_iter_setup<<<1, 1, 0, st>>>(ctl, vtab, ztab, ia);
  count_launches(1);
}

void launch_cycle_cond(const GmresCtl* ctl, int m, cudaGraphConditionalHandle h, cudaStream_t st) {
  k_cycle_cond<<<1, 1, 0, st>>>(ctl, m, h);
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
  k_gmres_solve<<<1, 1, 0, st>>>(ctl);
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
