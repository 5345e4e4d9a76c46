// FP64 stencil kernels of the 3D scheme: the DVDM residual (Eq. NSOP with the
// variational derivative of Eq. discretedG), the Jacobian-vector product (Eq.
// Jacobi), the discrete energy (Eqs. relations, freeenergy) and mass, on a
// periodic nx x ny x nz grid (x fastest), or between mirror walls (Sec. 2: each
// pass reads the mirror image of a cell beyond a wall, which makes the composed
// operators those of the evenly extended fields).
//
// The radius-3 composed operators are evaluated in three 7-point passes with
// two scratch fields (T1, T2): a Laplacian pass, a pass that forms mu (or the
// JVP's w) from it, and a final Laplacian pass that writes F (or J v).  Every
// pass reads its neighbours through L1/L2; the FP64 issue rate, not HBM, bounds
// them on GB300, so the extra passes cost little next to a fused 3D tile.
#include "ff.cuh"
#include "pfc_internal.cuh"

namespace pfc {
namespace {

constexpr int NT = 256;

// Neighbour index along an axis: the periodic image, or between mirror walls the cell itself
// (the mirror image of the cell beyond the wall).
__device__ __forceinline__ int wrap_up(int i, int n, int neu) { return i + 1 == n ? (neu ? i : 0) : i + 1; }
__device__ __forceinline__ int wrap_dn(int i, int n, int neu) { return i == 0 ? (neu ? 0 : n - 1) : i - 1; }

// unscaled 7-point Laplacian of u (+ u2 if given) at point idx = (x, y, z)
__device__ __forceinline__ double lap7(const double* __restrict__ u, const double* __restrict__ u2, const Geo& g,
                                       int x, int y, int z) {
  const long long sx = 1, sy = g.nx, sz = (long long)g.nx * g.ny;
  const long long c = x + sy * y + sz * z;
  const long long xp = c + (wrap_up(x, g.nx, g.neumann) - x) * sx, xm = c + (wrap_dn(x, g.nx, g.neumann) - x) * sx;
  const long long yp = c + (wrap_up(y, g.ny, g.neumann) - y) * sy, ym = c + (wrap_dn(y, g.ny, g.neumann) - y) * sy;
  const long long zp = c + (wrap_up(z, g.nz, g.neumann) - z) * sz, zm = c + (wrap_dn(z, g.nz, g.neumann) - z) * sz;
  if (u2) {
    const double cc = u[c] + u2[c];
    return ((u[xp] + u2[xp]) + (u[xm] + u2[xm])) + ((u[yp] + u2[yp]) + (u[ym] + u2[ym])) +
           ((u[zp] + u2[zp]) + (u[zm] + u2[zm])) - 6.0 * cc;
  }
  return (u[xp] + u[xm]) + (u[yp] + u[ym]) + (u[zp] + u[zm]) - 6.0 * u[c];
}

__device__ __forceinline__ void coords(const Geo& g, long long i, int* x, int* y, int* z) {
  const long long nxy = (long long)g.nx * g.ny;
  *z = (int)(i / nxy);
  const long long r = i - (long long)(*z) * nxy;
  *y = (int)(r / g.nx);
  *x = (int)(r - (long long)(*y) * g.nx);
}

__device__ __forceinline__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < NT / 32; ++w) s += red[w];  // fixed order: deterministic
  return s;
}

// out = scale * Lap_u(a [+ b])   (scale applied to the unscaled Laplacian)
__global__ void __launch_bounds__(NT) k_lap3d(Geo g, const double* __restrict__ a, const double* __restrict__ b,
                                              const double* __restrict__ ascale, double* __restrict__ out,
                                              const int* __restrict__ skip) {
  if (skip && *skip) return;
  const double sc = ascale ? *ascale : 1.0;
  for (long long i = blockIdx.x * (long long)NT + threadIdx.x; i < g.n; i += (long long)gridDim.x * NT) {
    int x, y, z;
    coords(g, i, &x, &y, &z);
    out[i] = sc * lap7(a, b, g, x, y, z);
  }
}

// mode 0 (residual): out = mu = c0 s + ih2 T1 + ih4/2 Lap(T1) + (P^2 + N^2) s / 4, s = P + N
// mode 1 (JVP):      out = w  = c0 v + ih2 T1 + ih4/2 Lap(T1) + q v,  v = sc * P
__global__ void __launch_bounds__(NT) k_mid3d(Geo g, int mode, const double* __restrict__ P,
                                              const double* __restrict__ N, const double* __restrict__ vscale,
                                              const double* __restrict__ T1, double* __restrict__ out,
                                              const int* __restrict__ skip) {
  if (skip && *skip) return;
  const double ih2 = g.ih2, ih4 = g.ih4, c0 = g.c0;
  const double sc = vscale ? *vscale : 1.0;
  for (long long i = blockIdx.x * (long long)NT + threadIdx.x; i < g.n; i += (long long)gridDim.x * NT) {
    int x, y, z;
    coords(g, i, &x, &y, &z);
    const double L1 = T1[i];
    const double LL = lap7(T1, nullptr, g, x, y, z);
    if (mode == 0) {
      const double p = P[i], nn = N[i], s = p + nn;
      out[i] = fma(0.25 * fma(p, p, nn * nn), s, fma(0.5 * ih4, LL, fma(ih2, L1, c0 * s)));
    } else {
      const double v = sc * P[i];
      out[i] = fma(N[i], v, fma(0.5 * ih4, LL, fma(ih2, L1, c0 * v)));
    }
  }
}

// The six neighbours of (x, y, z) in the order +x, -x, +y, -y, +z, -z (periodic grid).
__device__ __forceinline__ void nbrs6(const Geo& g, int x, int y, int z, long long c, long long* nb) {
  const long long sy = g.nx, sz = (long long)g.nx * g.ny;
  nb[0] = c + (wrap_up(x, g.nx, g.neumann) - x);
  nb[1] = c + (wrap_dn(x, g.nx, g.neumann) - x);
  nb[2] = c + (wrap_up(y, g.ny, g.neumann) - y) * sy;
  nb[3] = c + (wrap_dn(y, g.ny, g.neumann) - y) * sy;
  nb[4] = c + (wrap_up(z, g.nz, g.neumann) - z) * sz;
  nb[5] = c + (wrap_dn(z, g.nz, g.neumann) - z) * sz;
}
// Variable mobility (Sec. 3, M = 1 - s^2 at the midpoint s = (Phi + phi^n)/2, node by node):
// (div M grad)_d u at c = ih2 sum over the six edges M_edge (u_nb - u_c), M_edge the average of
// the edge's two end nodes.  m[k] are the nodal M of the neighbours, mc that of c.
__device__ __forceinline__ double div_m_grad6(const double* __restrict__ u, long long c, const long long* nb,
                                              double mc, const double* m, double ih2) {
  const double uc = u[c];
  double acc = 0.0;
#pragma unroll
  for (int k = 0; k < 6; ++k) acc = fma(0.5 * (mc + m[k]), u[nb[k]] - uc, acc);
  return ih2 * acc;
}

// F = (P - N) idt - ih2 Lap(mu); q = (3P^2 + 2PN + N^2)/4; per-CTA sum of F^2.
// MOB: F = (P - N) idt - (div M grad)_d mu with M = 1 - s^2, s = (P + N)/2; mu and s of every node
// written to mu_out, s_out when given (the JVP and the factor of this iterate read them).
template <bool MOB>
__global__ void __launch_bounds__(NT) k_res_out3d(Geo g, const double* __restrict__ P, const double* __restrict__ N,
                                                  const double* __restrict__ mu, double idt, double* __restrict__ F,
                                                  double* __restrict__ qout, double* __restrict__ partial,
                                                  double* __restrict__ mu_out, double* __restrict__ s_out) {
  __shared__ double red[NT / 32];
  double acc = 0.0;
  for (long long i = blockIdx.x * (long long)NT + threadIdx.x; i < g.n; i += (long long)gridDim.x * NT) {
    int x, y, z;
    coords(g, i, &x, &y, &z);
    const double p = P[i], nn = N[i];
    double f;
    if (MOB) {
      long long nb[6];
      nbrs6(g, x, y, z, i, nb);
      double m[6];
#pragma unroll
      for (int k = 0; k < 6; ++k) {
        const double sk = 0.5 * (P[nb[k]] + N[nb[k]]);
        m[k] = 1.0 - sk * sk;
      }
      const double sc = 0.5 * (p + nn);
      f = (p - nn) * idt - div_m_grad6(mu, i, nb, 1.0 - sc * sc, m, g.ih2);
      if (mu_out) mu_out[i] = mu[i];
      if (s_out) s_out[i] = sc;
    } else {
      f = fma(-g.ih2, lap7(mu, nullptr, g, x, y, z), (p - nn) * idt);
    }
    F[i] = f;
    if (qout) qout[i] = 0.25 * fma(3.0 * p, p, nn * fma(2.0, p, nn));
    acc = fma(f, f, acc);
  }
  const double s = block_sum(acc, red);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

// J v = sc v idt - ih2 Lap(w)
// MOB: J v = sc v idt - (div M grad)_d w - (div dM grad)_d mu, with M = 1 - s^2 and its derivative
// dM = -s (sc v) at the nodes (edge values the averages), mu and s of the iterate.
template <bool MOB>
__global__ void __launch_bounds__(NT) k_jvp_out3d(Geo g, const double* __restrict__ v,
                                                  const double* __restrict__ vscale, const double* __restrict__ w,
                                                  double idt, double* __restrict__ Jv, const int* __restrict__ skip,
                                                  const double* __restrict__ mu, const double* __restrict__ sm) {
  if (skip && *skip) return;
  const double sc = vscale ? *vscale : 1.0;
  for (long long i = blockIdx.x * (long long)NT + threadIdx.x; i < g.n; i += (long long)gridDim.x * NT) {
    int x, y, z;
    coords(g, i, &x, &y, &z);
    if (MOB) {
      long long nb[6];
      nbrs6(g, x, y, z, i, nb);
      double m[6], dm[6];
#pragma unroll
      for (int k = 0; k < 6; ++k) {
        const double sk = sm[nb[k]];
        m[k] = 1.0 - sk * sk;
        dm[k] = -sk * (sc * v[nb[k]]);
      }
      const double s0 = sm[i];
      const double vi = sc * v[i];
      Jv[i] = vi * idt - div_m_grad6(w, i, nb, 1.0 - s0 * s0, m, g.ih2) - div_m_grad6(mu, i, nb, -s0 * vi, dm, g.ih2);
    } else {
      Jv[i] = fma(-g.ih2, lap7(w, nullptr, g, x, y, z), sc * v[i] * idt);
    }
  }
}

// trial point Pout = Pb + lam (S - mean S)
__global__ void k_trial(long long n, const double* __restrict__ Pb, const double* __restrict__ S, double lam,
                        const double* __restrict__ ssum, double* __restrict__ Pout) {
  const double sm = ssum ? *ssum / (double)n : 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    Pout[i] = Pb[i] + lam * (S[i] - sm);
}

// Per-CTA sums of G_d (Eq. relations, three axes) and of phi.
__global__ void __launch_bounds__(NT) k_energy3d(Geo g, const double* __restrict__ phi,
                                                 double* __restrict__ partial) {
  __shared__ double red[NT / 32];
  const double c0 = g.c0, ih2 = g.ih2;
  const long long sy = g.nx, sz = (long long)g.nx * g.ny;
  double e = 0.0, m = 0.0;
  for (long long i = blockIdx.x * (long long)NT + threadIdx.x; i < g.n; i += (long long)gridDim.x * NT) {
    int x, y, z;
    coords(g, i, &x, &y, &z);
    const double p = phi[i];
    const double xp = phi[i + (wrap_up(x, g.nx, g.neumann) - x)], xm = phi[i + (wrap_dn(x, g.nx, g.neumann) - x)];
    const double yp = phi[i + (wrap_up(y, g.ny, g.neumann) - y) * sy], ym = phi[i + (wrap_dn(y, g.ny, g.neumann) - y) * sy];
    const double zp = phi[i + (wrap_up(z, g.nz, g.neumann) - z) * sz], zm = phi[i + (wrap_dn(z, g.nz, g.neumann) - z) * sz];
    const double lap = ih2 * ((xp + xm) + (yp + ym) + (zp + zm) - 6.0 * p);
    const double grad = (xp - p) * (xp - p) + (p - xm) * (p - xm) + (yp - p) * (yp - p) + (p - ym) * (p - ym) +
                        (zp - p) * (zp - p) + (p - zm) * (p - zm);
    const double p2 = p * p;
    e += c0 * p2 + 0.25 * p2 * p2 + 0.5 * lap * lap - 0.5 * ih2 * grad;
    m += p;
  }
  const double se = block_sum(e, red);
  __syncthreads();
  const double sm = block_sum(m, red);
  if (threadIdx.x == 0) {
    partial[blockIdx.x] = se;
    partial[gridDim.x + blockIdx.x] = sm;
  }
}

int ctas(long long n) {
  long long b = (n + NT - 1) / NT;
  const long long cap = 152LL * 8;
  return (int)(b < cap ? (b < 1 ? 1 : b) : cap);
}

}  // namespace

void launch_trial(const Geo& g, const double* Pb, const double* S, double lam, const double* ssum, double* Pout,
                  cudaStream_t st) {
  k_trial<<<ctas(g.n), NT, 0, st>>>(g.n, Pb, S, lam, ssum, Pout);
  count_launches(1);
}

void launch_residual3d(const Geo& g, const double* P, const double* phin, double idt, double* F, double* q_out,
                       double* T1, double* T2, double* partial, int* nparts, cudaStream_t st, bool mob,
                       double* mu_out, double* s_out) {
  const int b = ctas(g.n);
  k_lap3d<<<b, NT, 0, st>>>(g, P, phin, nullptr, T1, nullptr);
  k_mid3d<<<b, NT, 0, st>>>(g, 0, P, phin, nullptr, T1, T2, nullptr);
  if (mob)
    k_res_out3d<true><<<b, NT, 0, st>>>(g, P, phin, T2, idt, F, q_out, partial, mu_out, s_out);
  else
    k_res_out3d<false><<<b, NT, 0, st>>>(g, P, phin, T2, idt, F, q_out, partial, nullptr, nullptr);
  count_launches(3);
  *nparts = b;
}

void launch_jvp3d(const Geo& g, const double* v, const double* vscale, const double* q, double idt, double* Jv,
                  double* T1, double* T2, const int* skip, cudaStream_t st, const double* mu, const double* sm) {
  const int b = ctas(g.n);
  k_lap3d<<<b, NT, 0, st>>>(g, v, nullptr, vscale, T1, skip);
  k_mid3d<<<b, NT, 0, st>>>(g, 1, v, q, vscale, T1, T2, skip);
  if (mu)
    k_jvp_out3d<true><<<b, NT, 0, st>>>(g, v, vscale, T2, idt, Jv, skip, mu, sm);
  else
    k_jvp_out3d<false><<<b, NT, 0, st>>>(g, v, vscale, T2, idt, Jv, skip, nullptr, nullptr);
  count_launches(3);
}

void launch_energy3d(const Geo& g, const double* phi, double* partial, int* nparts, cudaStream_t st) {
  const int b = ctas(g.n);
  k_energy3d<<<b, NT, 0, st>>>(g, phi, partial);
  count_launches(1);
  *nparts = b;
}

}  // namespace pfc

// ---- The Jacobian-vector product of the mixed path in float-float arithmetic (FP32 pipe): the
// same three 7-point passes, with the scratch fields holding float pairs (8 bytes a point, as an
// FP64 value).  J v is linear in v, so GMRES needs it only to its own stop test; float-float keeps
// it to about 2^-44 of its terms, and GB300's FP64 pipe, which bounds the FP64 passes, idles.
// One thread per point, CTAs of 32 x 8 points of one z plane (no index divisions).
namespace pfc {
namespace {

constexpr int FX = 32, FY = 8;

// ((xp + xm) + (yp + ym)) + (zp + zm) - 6 c, with one two-sum per leading part (as ff_lap5).
__device__ __forceinline__ ff ff_lap7(ff c, ff xp, ff xm, ff yp, ff ym, ff zp, ff zm) {
  const ff a = two_sum(xp.hi, xm.hi), b = two_sum(yp.hi, ym.hi), d = two_sum(zp.hi, zm.hi);
  const ff t = two_sum(a.hi, b.hi);
  const ff t2 = two_sum(t.hi, d.hi);
  const float p = __fmul_rn(-6.0f, c.hi), pe = __fmaf_rn(-6.0f, c.hi, -p);  // -6 c.hi = p + pe exactly
  const ff u = two_sum(t2.hi, p);
  const float lo = __fadd_rn(
      __fadd_rn(__fadd_rn(__fadd_rn(xp.lo, xm.lo), __fadd_rn(yp.lo, ym.lo)), __fadd_rn(zp.lo, zm.lo)),
      __fadd_rn(__fadd_rn(__fadd_rn(a.lo, b.lo), __fadd_rn(d.lo, t.lo)),
                __fadd_rn(__fadd_rn(t2.lo, u.lo), __fadd_rn(pe, __fmul_rn(-6.0f, c.lo)))));
  return fast_two_sum(u.hi, lo);
}

struct Nb {  // the point and its six periodic neighbours
  long long c, xp, xm, yp, ym, zp, zm;
};
__device__ __forceinline__ bool nb_of(const Geo& g, Nb* o) {
  const int x = blockIdx.x * FX + threadIdx.x, y = blockIdx.y * FY + threadIdx.y, z = blockIdx.z;
  if (x >= g.nx || y >= g.ny) return false;
  const long long sy = g.nx, sz = (long long)g.nx * g.ny;
  o->c = x + sy * y + sz * z;
  o->xp = o->c + (wrap_up(x, g.nx, g.neumann) - x);
  o->xm = o->c + (wrap_dn(x, g.nx, g.neumann) - x);
  o->yp = o->c + (wrap_up(y, g.ny, g.neumann) - y) * sy;
  o->ym = o->c + (wrap_dn(y, g.ny, g.neumann) - y) * sy;
  o->zp = o->c + (wrap_up(z, g.nz, g.neumann) - z) * sz;
  o->zm = o->c + (wrap_dn(z, g.nz, g.neumann) - z) * sz;
  return true;
}
__device__ __forceinline__ ff ldff(const float2* p, long long i) {
  const float2 v = p[i];
  return {v.x, v.y};
}

// T1 = Lap v (unscaled)
__global__ void __launch_bounds__(FX* FY) k_lap3d_ff(Geo g, const double* __restrict__ v, float2* __restrict__ T1,
                                                     const int* __restrict__ skip) {
  if (skip && *skip) return;
  Nb o;
  if (!nb_of(g, &o)) return;
  const ff L = ff_lap7(ff_split(v[o.c]), ff_split(v[o.xp]), ff_split(v[o.xm]), ff_split(v[o.yp]),
                       ff_split(v[o.ym]), ff_split(v[o.zp]), ff_split(v[o.zm]));
  T1[o.c] = make_float2(L.hi, L.lo);
}
// T2 = w = c0 v + ih2 T1 + ih4/2 Lap T1 + q v
__global__ void __launch_bounds__(FX* FY) k_mid3d_ff(Geo g, const double* __restrict__ v,
                                                     const double* __restrict__ q, const float2* __restrict__ T1,
                                                     float2* __restrict__ T2, const int* __restrict__ skip) {
  if (skip && *skip) return;
  Nb o;
  if (!nb_of(g, &o)) return;
  const ff L1 = ldff(T1, o.c);
  const ff LL = ff_lap7(L1, ldff(T1, o.xp), ldff(T1, o.xm), ldff(T1, o.yp), ldff(T1, o.ym), ldff(T1, o.zp),
                        ldff(T1, o.zm));
  const ff vv = ff_split(v[o.c]);
  const ff ih2 = ff_split(g.ih2), hih4 = ff_split(g.hih4), c0 = ff_split(g.c0);
  const ff w = ff_dot4(c0, vv, ih2, L1, hih4, LL, ff_split(q[o.c]), vv);
  T2[o.c] = make_float2(w.hi, w.lo);
}
// J v = v idt - ih2 Lap w
__global__ void __launch_bounds__(FX* FY) k_jvp_out3d_ff(Geo g, const double* __restrict__ v,
                                                         const float2* __restrict__ T2, double idt,
                                                         double* __restrict__ Jv, const int* __restrict__ skip, int pout) {
  if (skip && *skip) return;
  Nb o;
  if (!nb_of(g, &o)) return;
  const ff Lw = ff_lap7(ldff(T2, o.c), ldff(T2, o.xp), ldff(T2, o.xm), ldff(T2, o.yp), ldff(T2, o.ym),
                        ldff(T2, o.zp), ldff(T2, o.zm));
  const ff jv = ff_dot2m(ff_split(v[o.c]), ff_split(idt), ff_split(g.ih2), Lw);
  if (pout)
    st_pair(Jv, o.c, jv);
  else
    Jv[o.c] = ff_to_double(jv);
}

// The same three passes in plain FP32 (opt-in on the mixed path, pfc_params.jvp_fp32): inputs cut
// to floats, FP32 scratch fields, the 2D FP32 JVP's arithmetic with 7-point Laplacians.  The
// scheme's constants are cut once per CTA.
__device__ __forceinline__ float lap7f(float c, float xp, float xm, float yp, float ym, float zp, float zm) {
  return ((xp + xm) + (yp + ym)) + (zp + zm) - 6.0f * c;
}
__device__ __forceinline__ void consts_f32(const Geo& g, double idt, float* k) {
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    k[0] = f32_cut(g.ih2);
    k[1] = f32_cut(g.hih4);
    k[2] = f32_cut(g.c0);
    k[3] = f32_cut(idt);
  }
  __syncthreads();
}
// T1 = Lap v (unscaled)
__global__ void __launch_bounds__(FX* FY) k_lap3d_f32(Geo g, const double* __restrict__ v, float* __restrict__ T1,
                                                      const int* __restrict__ skip) {
  if (skip && *skip) return;
  Nb o;
  if (!nb_of(g, &o)) return;
  T1[o.c] = lap7f(f32_cut(v[o.c]), f32_cut(v[o.xp]), f32_cut(v[o.xm]), f32_cut(v[o.yp]), f32_cut(v[o.ym]),
                  f32_cut(v[o.zp]), f32_cut(v[o.zm]));
}
// T2 = w = (c0 + q) v + ih2 T1 + ih4/2 Lap T1
__global__ void __launch_bounds__(FX* FY) k_mid3d_f32(Geo g, const double* __restrict__ v,
                                                      const double* __restrict__ q, const float* __restrict__ T1,
                                                      float* __restrict__ T2, const int* __restrict__ skip) {
  if (skip && *skip) return;
  __shared__ float k[4];
  consts_f32(g, 0.0, k);
  Nb o;
  if (!nb_of(g, &o)) return;
  const float L1 = T1[o.c];
  const float LL = lap7f(L1, T1[o.xp], T1[o.xm], T1[o.yp], T1[o.ym], T1[o.zp], T1[o.zm]);
  T2[o.c] = fmaf(k[2] + f32_cut(q[o.c]), f32_cut(v[o.c]), fmaf(k[0], L1, k[1] * LL));
}
// J v = v idt - ih2 Lap w
__global__ void __launch_bounds__(FX* FY) k_jvp_out3d_f32(Geo g, const double* __restrict__ v,
                                                          const float* __restrict__ T2, double idt,
                                                          double* __restrict__ Jv, const int* __restrict__ skip,
                                                          int pout) {
  if (skip && *skip) return;
  __shared__ float k[4];
  consts_f32(g, idt, k);
  Nb o;
  if (!nb_of(g, &o)) return;
  const float Lw = lap7f(T2[o.c], T2[o.xp], T2[o.xm], T2[o.yp], T2[o.ym], T2[o.zp], T2[o.zm]);
  const float jv = fmaf(f32_cut(v[o.c]), k[3], -k[0] * Lw);
  if (pout)
    st_pair(Jv, o.c, ff{jv, 0.0f});
  else
    Jv[o.c] = f2d_bits(jv);
}

}  // namespace

void launch_jvp3d_f32(const Geo& g, const double* v, const double* q, double idt, double* Jv, double* T1, double* T2,
                      const int* skip, cudaStream_t st, int pout) {
  const dim3 grid((g.nx + FX - 1) / FX, (g.ny + FY - 1) / FY, g.nz), blk(FX, FY);
  float* t1 = reinterpret_cast<float*>(T1);
  float* t2 = reinterpret_cast<float*>(T2);
  k_lap3d_f32<<<grid, blk, 0, st>>>(g, v, t1, skip);
  k_mid3d_f32<<<grid, blk, 0, st>>>(g, v, q, t1, t2, skip);
  k_jvp_out3d_f32<<<grid, blk, 0, st>>>(g, v, t2, idt, Jv, skip, pout);
  count_launches(3);
}

void launch_jvp3d_ff(const Geo& g, const double* v, const double* q, double idt, double* Jv, double* T1, double* T2,
                     const int* skip, cudaStream_t st, int pout) {
  const dim3 grid((g.nx + FX - 1) / FX, (g.ny + FY - 1) / FY, g.nz), blk(FX, FY);
  float2* t1 = reinterpret_cast<float2*>(T1);
  float2* t2 = reinterpret_cast<float2*>(T2);
  k_lap3d_ff<<<grid, blk, 0, st>>>(g, v, t1, skip);
  k_mid3d_ff<<<grid, blk, 0, st>>>(g, v, q, t1, t2, skip);
  k_jvp_out3d_ff<<<grid, blk, 0, st>>>(g, v, t2, idt, Jv, skip, pout);
  count_launches(3);
}

}  // namespace pfc
