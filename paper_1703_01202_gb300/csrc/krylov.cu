// FP64 vector kernels of right-preconditioned restarted GMRES (Sec. 4, Eq.
// hjacobi): fused multi-dot products and multi-axpys for classical Gram-Schmidt
// with one conditional re-orthogonalisation pass (Daniel-Gragg-Kaufman-Stewart
// criterion), deterministic two-level reductions (per-CTA partial sums in a
// fixed order, then one CTA per reduction), and the single-thread kernels that
// keep the Arnoldi/Givens bookkeeping on the device.
//
// The basis is kept unnormalised: V_i = scale_i * Vraw_i with scale_i held on
// the device, so no kernel pass is spent on normalising.  Every kernel takes
// the cycle's "done" flag and returns at once when it is set, which lets the
// host queue several iterations ahead and synchronise rarely.
#include <cmath>

#include "pfc_internal.cuh"

namespace pfc {
namespace {

constexpr int G = 8;     // vectors per multi-dot pass
constexpr int NT = 256;  // threads per CTA

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// partial[(g0 + k) * gridDim.x + blockIdx.x] = sum_i V_{g0+k}[i] * w[i]
__global__ void __launch_bounds__(NT) k_multidot(VecList V, int nv, const double* __restrict__ w, long long n,
                                                 double* __restrict__ partial, const int* __restrict__ skip,
                                                 const int* __restrict__ only_if) {
  if ((skip && *skip) || (only_if && !*only_if)) return;
  __shared__ double red[NT / 32][G];
  const int g0 = blockIdx.y * G;
  const int cnt = min(G, nv - g0);
  double acc[G];
#pragma unroll
  for (int k = 0; k < G; ++k) acc[k] = 0.0;
  const long long stride = (long long)gridDim.x * NT;
  for (long long i = blockIdx.x * (long long)NT + threadIdx.x; i < n; i += stride) {
    const double wi = w[i];
#pragma unroll
    for (int k = 0; k < G; ++k)
      if (k < cnt) acc[k] = fma(V.p[g0 + k][i], wi, acc[k]);
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < G; ++k) {
    const double s = warp_sum(acc[k]);
    if (lane == 0) red[wid][k] = s;
  }
  __syncthreads();
  if (threadIdx.x < cnt) {
    double s = 0.0;
    for (int q = 0; q < NT / 32; ++q) s += red[q][threadIdx.x];
    partial[(size_t)(g0 + threadIdx.x) * gridDim.x + blockIdx.x] = s;
  }
}

// w = w + sign * sum_k coef[k] X_k ; partial[0..] = sum w^2, partial[gridDim..] = sum w
__global__ void __launch_bounds__(NT) k_multiaxpy(double* __restrict__ w, VecList X, int nx,
                                                  const double* __restrict__ coef, double sign, long long n,
                                                  double* __restrict__ partial, const int* __restrict__ skip,
                                                  const int* __restrict__ only_if) {
  if ((skip && *skip) || (only_if && !*only_if)) return;
  __shared__ double red[2][NT / 32];
  __shared__ double c[kMaxVecs];
  for (int k = threadIdx.x; k < nx; k += NT) c[k] = sign * coef[k];
  __syncthreads();
  double s2 = 0.0, s1 = 0.0;
  const long long stride = (long long)gridDim.x * NT;
  for (long long i = blockIdx.x * (long long)NT + threadIdx.x; i < n; i += stride) {
    double acc = w[i];
    for (int k = 0; k < nx; ++k) acc = fma(c[k], X.p[k][i], acc);
    w[i] = acc;
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
  if (threadIdx.x < 2) {
    double s = 0.0;
    for (int q = 0; q < NT / 32; ++q) s += red[threadIdx.x][q];
    partial[(size_t)threadIdx.x * gridDim.x + blockIdx.x] = s;
  }
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

__global__ void k_gmres_init(GmresCtl* c, const double* __restrict__ nrm2, double sign, double tol) {
  const double beta = sqrt(*nrm2);
  c->done = 0;
  c->its = 0;
  c->reorth = 0;
  c->breakdown = 0;
  c->tol = tol;
  c->beta = beta;
  c->est = beta;
  c->g[0] = beta;
  c->scale[0] = beta > 0.0 ? sign / beta : 0.0;
  if (!(beta > tol)) c->done = 1;
}

// After a multi-dot of V_0..V_j against w (red[0..j]) and w.w (red[j+1]).
__global__ void k_gmres_after_dot(GmresCtl* c, int j, int pass) {
  if (c->done) return;
  if (pass == 1 && !c->reorth) return;
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

// After the multi-axpy w -= sum coef_i Vraw_i; red[0] = w.w afterwards.
__global__ void k_gmres_after_axpy(GmresCtl* c, const double* __restrict__ red2, int j, int pass, int m) {
  if (c->done) return;
  const double wn2 = red2[0];
  if (pass == 0) {
    if (wn2 < 0.5 * c->wnorm2_before) {  // ||w'|| < ||w|| / sqrt(2): orthogonalise once more
      c->reorth = 1;
      return;
    }
    c->reorth = 0;
    gmres_finalize(c, j, m, wn2);
  } else {
    if (!c->reorth) return;
    c->reorth = 0;
    gmres_finalize(c, j, m, wn2);
  }
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

int red_ctas(long long n) {
  long long b = (n + NT - 1) / NT;
  return (int)(b < kRedCtas ? (b < 1 ? 1 : b) : kRedCtas);
}

}  // namespace

void launch_multidot(const VecList& V, int nv, const double* w, long long n, double* partial, const int* skip,
                     const int* only_if, cudaStream_t st, int* nparts) {
  const int bx = red_ctas(n);
  dim3 grid(bx, (nv + G - 1) / G);
  k_multidot<<<grid, NT, 0, st>>>(V, nv, w, n, partial, skip, only_if);
  count_launches(1);
  *nparts = bx;
}

void launch_multiaxpy(double* w, const VecList& X, int nx, const double* coef, double sign, long long n,
                      double* partial, const int* skip, const int* only_if, cudaStream_t st, int* nparts) {
  const int bx = red_ctas(n);
  k_multiaxpy<<<bx, NT, 0, st>>>(w, X, nx, coef, sign, n, partial, skip, only_if);
  count_launches(1);
  *nparts = bx;
}

void launch_reduce(const double* partial, int nvals, int nparts, double* out, cudaStream_t st) {
  k_reduce<<<1, 1024, 0, st>>>(partial, nvals, nparts, out);
  count_launches(1);
}

void launch_gmres_init(GmresCtl* ctl, const double* nrm2, double sign, double tol, cudaStream_t st) {
  k_gmres_init<<<1, 1, 0, st>>>(ctl, nrm2, sign, tol);
  count_launches(1);
}
void launch_gmres_after_dot(GmresCtl* ctl, int j, int pass, cudaStream_t st) {
  k_gmres_after_dot<<<1, 1, 0, st>>>(ctl, j, pass);
  count_launches(1);
}
void launch_gmres_after_axpy(GmresCtl* ctl, const double* red2, int j, int pass, int m, cudaStream_t st) {
  k_gmres_after_axpy<<<1, 1, 0, st>>>(ctl, red2, j, pass, m);
  count_launches(1);
}
void launch_gmres_solve(GmresCtl* ctl, cudaStream_t st) { k_gmres_solve<<<1, 1, 0, st>>>(ctl);
  count_launches(1); }

void launch_axpby(double* y, const double* x, double a, double b, long long n, cudaStream_t st) {
  k_axpby<<<red_ctas(n), NT, 0, st>>>(y, x, a, b, n);
  count_launches(1);
}
void launch_extrapolate(double* out, const double* a, const double* b, double ratio, long long n, cudaStream_t st) {
  k_extrapolate<<<red_ctas(n), NT, 0, st>>>(out, a, b, ratio, n);
  count_launches(1);
}

}  // namespace pfc
