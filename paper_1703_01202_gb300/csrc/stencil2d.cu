// Fused FP64 stencil kernels of the 2D scheme: the DVDM residual (Eq. NSOP with
// the variational derivative of Eq. discretedG), the Jacobian-vector product
// (Eq. Jacobi), the discrete energy (Eqs. relations, freeenergy) and mass.
//
// The residual and the JVP are radius-3 composed stencils, Delta_d applied to a
// radius-2 operator.  Each CTA stages a (32+6) x (16+6) tile of its inputs in
// shared memory (periodic wrap, or mirror images across Neumann walls, at the grid
// edges: the operators are then those of the evenly extended grid) and evaluates the stages in
// place: Laplacian of the halo-2 ring, then mu (or w) on the halo-1 ring, then
// Delta_d of that on the tile.  All arithmetic is FP64; on GB300 these kernels
// are bound by the FP64 issue rate, not by HBM (about 25 FP64 ops per 24 bytes).
#include "pfc_internal.cuh"

namespace pfc {
namespace {

constexpr int TX = 32, TY = 16, R = 3;
constexpr int AX = TX + 2 * R, AY = TY + 2 * R;  // 38 x 22 staged points
constexpr int NT = 256;                          // 32 x 8 threads, 2 outputs each

__device__ __forceinline__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int tid = threadIdx.x + threadIdx.y * blockDim.x;
  const int nw = (blockDim.x * blockDim.y) >> 5;
  if ((tid & 31) == 0) red[tid >> 5] = v;
  __syncthreads();
  double s = 0.0;
  if (tid == 0)
    for (int w = 0; w < nw; ++w) s += red[w];  // fixed order: deterministic
  return s;
}

// F(Phi) = (Phi - phi^n)/dt - Delta_d mu,  mu = L_gamma (Phi+phi^n)/2 + (Phi+phi^n)(Phi^2+phi^n^2)/4.
// MOB: (div M grad)_d instead of Delta_d, M = 1 - s^2 at the midpoint s = (Phi+phi^n)/2 of each node
// and the average of its two ends on an edge (Sec. 3); with qout also writes mu and s (muout, sout).
// Phi = Pb + lam (S - mean S) when S != nullptr (line-search trial point, also written to Pout);
// smean points at sum(S), or is null when the update is not projected.
// Writes q = (3 Phi^2 + 2 Phi phi^n + phi^n^2)/4 when qout != nullptr, and the CTA's sum of F^2.
template <bool MOB>
__global__ void __launch_bounds__(NT) k_residual2d(Geo g, const double* __restrict__ Pb,
                                                   const double* __restrict__ S, double lam,
                                                   const double* __restrict__ smean,
                                                   const double* __restrict__ phin, double idt,
                                                   double* __restrict__ F, double* __restrict__ Pout,
                                                   double* __restrict__ qout, double* __restrict__ partial,
                                                   double* __restrict__ muout, double* __restrict__ sout,
                                                   const double* __restrict__ idt_dev,
                                                   const double* __restrict__ lam_dev) {
  __shared__ double sP[AY][AX], sN[AY][AX], sS[AY][AX];
  if (idt_dev) idt = *idt_dev;  // a captured step graph: this step's 1/dt and line-search step
  if (lam_dev) lam = *lam_dev;
  __shared__ double sL[AY - 2][AX - 2];
  __shared__ double sM[AY - 4][AX - 4];
  __shared__ double red[NT / 32];
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
  const int tid = threadIdx.x + threadIdx.y * 32;
  const double sm = (S && smean) ? *smean / (double)g.n : 0.0;  // mean of S (mass projection)
  for (int i = tid; i < AX * AY; i += NT) {
    const int ly = i / AX, lx = i - ly * AX;
    const long long idx = cell_index(x0 + lx - R, g.nx, g.neumann) + (long long)g.nx * cell_index(y0 + ly - R, g.ny, g.neumann);
    double p = Pb[idx];
    if (S) p = p + lam * (S[idx] - sm);
    const double nn = phin[idx];
    sP[ly][lx] = p;
    sN[ly][lx] = nn;
    sS[ly][lx] = p + nn;
  }
  __syncthreads();
  // unscaled Laplacian of s = Phi + phi^n on the halo-2 region
  for (int i = tid; i < (AX - 2) * (AY - 2); i += NT) {
    const int ly = i / (AX - 2) + 1, lx = i - (ly - 1) * (AX - 2) + 1;
    sL[ly - 1][lx - 1] = (sS[ly][lx - 1] + sS[ly][lx + 1]) + (sS[ly - 1][lx] + sS[ly + 1][lx]) - 4.0 * sS[ly][lx];
  }
  __syncthreads();
  const double ih2 = g.ih2, ih4 = g.ih4, c0 = g.c0;
  // mu on the halo-1 region
  for (int i = tid; i < (AX - 4) * (AY - 4); i += NT) {
    const int ly = i / (AX - 4) + 2, lx = i - (ly - 2) * (AX - 4) + 2;
    const int a = ly - 1, b = lx - 1;  // index into sL
    const double Ls = sL[a][b];
    const double LLs = (sL[a][b - 1] + sL[a][b + 1]) + (sL[a - 1][b] + sL[a + 1][b]) - 4.0 * Ls;
    const double s = sS[ly][lx], p = sP[ly][lx], nn = sN[ly][lx];
    const double cub = 0.25 * fma(p, p, nn * nn);
    sM[ly - 2][lx - 2] = fma(cub, s, fma(0.5 * ih4, LLs, fma(ih2, Ls, c0 * s)));
  }
  __syncthreads();
  double acc = 0.0;
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    const int tx = threadIdx.x, ty = threadIdx.y + 8 * r;
    const int gx = x0 + tx, gy = y0 + ty;
    if (gx < g.nx && gy < g.ny) {
      const int a = ty + 1, b = tx + 1;  // index into sM
      const double mu = sM[a][b];
      double Lmu;
      if (MOB) {  // sum over the 4 edges of M_edge (mu_nb - mu), M_edge = (M_c + M_nb)/2, M = 1 - (sS/2)^2
        const int ly = ty + R, lx = tx + R;
        auto mob = [&](int y, int x) { const double h = 0.5 * sS[y][x]; return 1.0 - h * h; };
        const double mc = mob(ly, lx);
        Lmu = 0.5 * ((mc + mob(ly, lx - 1)) * (sM[a][b - 1] - mu) + (mc + mob(ly, lx + 1)) * (sM[a][b + 1] - mu)) +
              0.5 * ((mc + mob(ly - 1, lx)) * (sM[a - 1][b] - mu) + (mc + mob(ly + 1, lx)) * (sM[a + 1][b] - mu));
      } else {
        Lmu = (sM[a][b - 1] + sM[a][b + 1]) + (sM[a - 1][b] + sM[a + 1][b]) - 4.0 * mu;
      }
      const double p = sP[ty + R][tx + R], nn = sN[ty + R][tx + R];
      const double f = fma(-ih2, Lmu, (p - nn) * idt);
      const long long idx = gx + (long long)g.nx * gy;
      F[idx] = f;
      if (Pout) Pout[idx] = p;
      if (qout) qout[idx] = 0.25 * fma(3.0 * p, p, nn * fma(2.0, p, nn));
      if (MOB && qout) {
        muout[idx] = mu;
        sout[idx] = 0.5 * sS[ty + R][tx + R];
      }
      acc = fma(f, f, acc);
    }
  }
  const double s = block_sum(acc, red);
  if (tid == 0) partial[blockIdx.x + gridDim.x * blockIdx.y] = s;
}

// J v = v/dt - Delta_d w,  w = L_gamma v / 2 + q v (Eq. Jacobi).
// J v = v/dt - Delta_d w, w = L_gamma v/2 + q v (Eq. Jacobi).  MOB: J v = v/dt - (div M grad)_d w
// - (div dM grad)_d mu with M = 1 - s^2 and dM = -s v at the nodes, both averaged onto the edges.
template <bool MOB>
__global__ void __launch_bounds__(NT) k_jvp2d(Geo g, const double* __restrict__ v,
                                              const double* __restrict__ vscale, const double* __restrict__ q,
                                              double idt, double* __restrict__ Jv, const int* __restrict__ skip,
                                              const IterArgs* __restrict__ ia, const double* __restrict__ mug,
                                              const double* __restrict__ smg) {
  if (skip && *skip) return;
  if (ia) {  // graph mode: J Z_j into V_(j+1)
    v = ia->z;
    q = ia->q;
    idt = ia->idt;
    Jv = ia->w;
    mug = ia->mu;
    smg = ia->sm;
  }
  __shared__ double sV[AY][AX];
  __shared__ double sQ[AY - 4][AX - 4];
  __shared__ double sL[AY - 2][AX - 2];
  __shared__ double sW[AY - 4][AX - 4];
  __shared__ double sMu[MOB ? AY - 4 : 1][MOB ? AX - 4 : 1], sSm[MOB ? AY - 4 : 1][MOB ? AX - 4 : 1];
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
  const int tid = threadIdx.x + threadIdx.y * 32;
  const double sc = vscale ? *vscale : 1.0;
  for (int i = tid; i < AX * AY; i += NT) {
    const int ly = i / AX, lx = i - ly * AX;
    const long long idx = cell_index(x0 + lx - R, g.nx, g.neumann) + (long long)g.nx * cell_index(y0 + ly - R, g.ny, g.neumann);
    sV[ly][lx] = sc * v[idx];
  }
  for (int i = tid; i < (AX - 4) * (AY - 4); i += NT) {
    const int ly = i / (AX - 4), lx = i - ly * (AX - 4);
    const long long idx = cell_index(x0 + lx - 1, g.nx, g.neumann) + (long long)g.nx * cell_index(y0 + ly - 1, g.ny, g.neumann);
    sQ[ly][lx] = q[idx];
    if (MOB) {
      sMu[ly][lx] = mug[idx];
      sSm[ly][lx] = smg[idx];
    }
  }
  __syncthreads();
  for (int i = tid; i < (AX - 2) * (AY - 2); i += NT) {
    const int ly = i / (AX - 2) + 1, lx = i - (ly - 1) * (AX - 2) + 1;
    sL[ly - 1][lx - 1] = (sV[ly][lx - 1] + sV[ly][lx + 1]) + (sV[ly - 1][lx] + sV[ly + 1][lx]) - 4.0 * sV[ly][lx];
  }
  __syncthreads();
  const double ih2 = g.ih2, ih4 = g.ih4, c0 = g.c0;
  for (int i = tid; i < (AX - 4) * (AY - 4); i += NT) {
    const int ly = i / (AX - 4) + 2, lx = i - (ly - 2) * (AX - 4) + 2;
    const int a = ly - 1, b = lx - 1;
    const double Lv = sL[a][b];
    const double LLv = (sL[a][b - 1] + sL[a][b + 1]) + (sL[a - 1][b] + sL[a + 1][b]) - 4.0 * Lv;
    const double vv = sV[ly][lx];
    sW[ly - 2][lx - 2] = fma(sQ[ly - 2][lx - 2], vv, fma(0.5 * ih4, LLv, fma(ih2, Lv, c0 * vv)));
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    const int tx = threadIdx.x, ty = threadIdx.y + 8 * r;
    const int gx = x0 + tx, gy = y0 + ty;
    if (gx < g.nx && gy < g.ny) {
      const int a = ty + 1, b = tx + 1;
      const double w = sW[a][b];
      double Lw;
      if (MOB) {  // edge (c, nb): M_e (w_nb - w_c) + dM_e (mu_nb - mu_c), averages of the two ends
        const int ly = ty + R, lx = tx + R;
        const double sc = sSm[a][b], mc = 1.0 - sc * sc, dc = -sc * sV[ly][lx], muc = sMu[a][b];
        auto edge = [&](int ya, int xb, int vy, int vx) {
          const double sn = sSm[ya][xb];
          return 0.5 * ((mc + (1.0 - sn * sn)) * (sW[ya][xb] - w) + (dc - sn * sV[vy][vx]) * (sMu[ya][xb] - muc));
        };
        Lw = (edge(a, b - 1, ly, lx - 1) + edge(a, b + 1, ly, lx + 1)) + (edge(a - 1, b, ly - 1, lx) + edge(a + 1, b, ly + 1, lx));
      } else {
        Lw = (sW[a][b - 1] + sW[a][b + 1]) + (sW[a - 1][b] + sW[a + 1][b]) - 4.0 * w;
      }
      Jv[gx + (long long)g.nx * gy] = fma(-ih2, Lw, sV[ty + R][tx + R] * idt);
    }
  }
}

// Per-CTA sums of G_d (Eq. relations) and of phi.
__global__ void __launch_bounds__(256) k_energy2d(Geo g, const double* __restrict__ phi,
                                                  double* __restrict__ partial) {
  __shared__ double red[8];
  const double c0 = g.c0, ih2 = g.ih2;
  double e = 0.0, m = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < g.n; i += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(i % g.nx), y = (int)(i / g.nx);
    const double p = phi[i];
    const double pe = phi[cell_index(x + 1, g.nx, g.neumann) + (long long)g.nx * y];
    const double pw = phi[cell_index(x - 1, g.nx, g.neumann) + (long long)g.nx * y];
    const double pn = phi[x + (long long)g.nx * cell_index(y + 1, g.ny, g.neumann)];
    const double ps = phi[x + (long long)g.nx * cell_index(y - 1, g.ny, g.neumann)];
    const double lap = ih2 * ((pe + pw) + (pn + ps) - 4.0 * p);
    const double grad = (pe - p) * (pe - p) + (p - pw) * (p - pw) + (pn - p) * (pn - p) + (p - ps) * (p - ps);
    const double p2 = p * p;
    e += c0 * p2 + 0.25 * p2 * p2 + 0.5 * lap * lap - 0.5 * ih2 * grad;
    m += p;
  }
  const double se = block_sum(e, red);
  __syncthreads();
  const double smm = block_sum(m, red);
  if (threadIdx.x == 0) {
    partial[blockIdx.x] = se;
    partial[gridDim.x + blockIdx.x] = smm;
  }
}

__global__ void k_qcoef(long long n, const double* __restrict__ P, const double* __restrict__ N,
                        double* __restrict__ q) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double p = P[i], nn = N[i];
    q[i] = 0.25 * fma(3.0 * p, p, nn * fma(2.0, p, nn));
  }
}

}  // namespace

void launch_residual2d(const Geo& g, const double* Pb, const double* S, double lam, const double* smean,
                       const double* phin, double idt, double* F, double* Pout, double* qout, double* partial,
                       int* nparts, cudaStream_t st, bool mob, double* mu_out, double* s_out, const double* idt_dev,
                       const double* lam_dev) {
  dim3 grid((g.nx + TX - 1) / TX, (g.ny + TY - 1) / TY);
  if (mob)
    k_residual2d<true><<<grid, dim3(32, 8), 0, st>>>(g, Pb, S, lam, smean, phin, idt, F, Pout, qout, partial,
                                                      mu_out, s_out, idt_dev, lam_dev);
  else
    k_residual2d<false><<<grid, dim3(32, 8), 0, st>>>(g, Pb, S, lam, smean, phin, idt, F, Pout, qout, partial,
                                                       nullptr, nullptr, idt_dev, lam_dev);
  count_launches(1);
  *nparts = grid.x * grid.y;
}

void launch_jvp2d(const Geo& g, const double* v, const double* vscale, const double* q, double idt, double* Jv,
                  const int* skip, cudaStream_t st, const IterArgs* ia, const double* mu, const double* sm) {
  dim3 grid((g.nx + TX - 1) / TX, (g.ny + TY - 1) / TY);
  if (mu)
    k_jvp2d<true><<<grid, dim3(32, 8), 0, st>>>(g, v, vscale, q, idt, Jv, skip, ia, mu, sm);
  else
    k_jvp2d<false><<<grid, dim3(32, 8), 0, st>>>(g, v, vscale, q, idt, Jv, skip, ia, nullptr, nullptr);
  count_launches(1);
}

void launch_energy2d(const Geo& g, const double* phi, double* partial, int* nparts, cudaStream_t st) {
  int blocks = (int)((g.n + 255) / 256);
  if (blocks > kRedCtas) blocks = kRedCtas;
  k_energy2d<<<blocks, 256, 0, st>>>(g, phi, partial);
  count_launches(1);
  *nparts = blocks;
}

void launch_qcoef(const Geo& g, const double* Phi, const double* phin, double* q, cudaStream_t st) {
  int blocks = (int)((g.n + 255) / 256);
  if (blocks > kRedCtas) blocks = kRedCtas;
  k_qcoef<<<blocks, 256, 0, st>>>(g.n, Phi, phin, q);
  count_launches(1);
}

}  // namespace pfc
