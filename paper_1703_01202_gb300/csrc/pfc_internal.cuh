// Internal declarations shared by the CUDA translation units of libpfc.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

namespace pfc {

constexpr int kMaxRestart = 60;   // GMRES restart length limit
constexpr int kMaxVecs = kMaxRestart + 2;
constexpr int kRedCtas = 4 * 152;  // CTAs of the grid-stride reduction kernels

// Geometry of a periodic grid (x fastest) and the scheme's constants.
struct Geo {
  int nx, ny, nz;
  long long n;      // nx * ny * nz
  double ih2;       // 1 / h^2
  double gamma;     // quench depth of Eq. (GE)
  double hd;        // h^d (cell volume)
};

// One overlapped subdomain Omega_k^delta and its core Omega_k (Sec. 4).
struct BlockDesc {
  int x0, y0, z0;  // global cell of block-local (0,0,0); may be negative (periodic wrap)
  int bx, by, bz;  // block extent
  int ox, oy, oz;  // core offset inside the block (= overlap)
  int cx, cy, cz;  // core extent
};

// Device-resident state of one GMRES cycle (Arnoldi relation + Givens QR).
struct GmresCtl {
  int done;      // 1 once the cycle has converged or broken down
  int its;       // iterations completed in this cycle
  int reorth;    // second Gram-Schmidt pass requested for the current column
  int breakdown;
  double tol, beta, est;
  double wnorm2_before;
  double H[(kMaxRestart + 1) * kMaxRestart];  // column-major: H[i + (m+1) j]
  double cs[kMaxRestart], sn[kMaxRestart], g[kMaxRestart + 1], y[kMaxRestart];
  double scale[kMaxRestart + 2];  // V_i = scale_i * Vraw_i
  double coef[kMaxRestart + 2];   // coefficients of the pending multi-axpy
  double red[kMaxVecs + 2];       // reduced sums of the last multi-dot / axpy
};

// Scalars the host reads back after a reduction.
struct Scalars {
  double sum[8];
};

struct VecList {
  const double* p[kMaxVecs];
};

// Constant stencil tables of the Jacobian's linear part, -(1/2) Delta_d L_gamma,
// with the h scaling folded in.  2D: 7x7 (index (dy+3)*7 + dx+3); 3D: 7x7x7.
struct LinStencil {
  double c[343];
};

// Process-wide count of kernels launched by this library (for launch reports).
void count_launches(long long n);
long long launches_so_far();

// ---- stencil kernels (stencil2d.cu)
void launch_residual2d(const Geo& g, const double* Phi_base, const double* S, double lam, const double* smean,
                       const double* phin, double idt, double* F, double* Phi_out, double* q_out, double* partial,
                       int* nparts, cudaStream_t st);
void launch_jvp2d(const Geo& g, const double* v, const double* vscale, const double* q, double idt, double* Jv,
                  const int* skip, cudaStream_t st);
void launch_energy2d(const Geo& g, const double* phi, double* partial, int* nparts, cudaStream_t st);
void launch_qcoef(const Geo& g, const double* Phi, const double* phin, double* q, cudaStream_t st);

// ---- Schwarz preconditioner (ras2d.cu)
struct FactorStore {
  void* L;       // per block: n_max rows of lrow multipliers (row k = step k of the elimination)
  void* U;       // per block: n_max columns of ucol entries, U(k-j, k) at j; diagonal stored inverted
  uint8_t* piv;  // per block: pivot row of step k as the offset p - k (< 2^8)
  size_t strideL, strideU, strideP;  // elements (bytes for piv) per block
  int lrow, ucol;                    // kl_max and 2 kl_max + 1 rounded up to 8 elements (16-byte rows)
  int prec;                          // PFC_F64 / PFC_F32 / PFC_BF16
  int kl_max;
  int n_max;
};
void launch_factor2d(const Geo& g, const BlockDesc* blocks, int nblocks, const double* q, double idt,
                     const double* lin, const FactorStore& fs, int* status, cudaStream_t st);
void launch_ras_apply2d(const Geo& g, const BlockDesc* blocks, int nblocks, const FactorStore& fs, const double* r,
                        const double* rscale, double* z, const int* skip, int* err, cudaStream_t st);
size_t factor_smem_bytes(int prec, int kl, int n_max);

// ---- Krylov vector kernels (krylov.cu)
void launch_multidot(const VecList& V, int nv, const double* w, long long n, double* partial, const int* skip,
                     const int* only_if, cudaStream_t st, int* nparts);
void launch_multiaxpy(double* w, const VecList& X, int nx, const double* coef, double sign, long long n,
                      double* partial, const int* skip, const int* only_if, cudaStream_t st, int* nparts);
void launch_reduce(const double* partial, int nvals, int nparts, double* out, cudaStream_t st);
void launch_gmres_init(GmresCtl* ctl, const double* nrm2, double sign, double tol, cudaStream_t st);
void launch_gmres_after_dot(GmresCtl* ctl, int j, int pass, cudaStream_t st);
void launch_gmres_after_axpy(GmresCtl* ctl, const double* red2, int j, int pass, int m, cudaStream_t st);
void launch_gmres_solve(GmresCtl* ctl, cudaStream_t st);
void launch_axpby(double* y, const double* x, double a, double b, long long n, cudaStream_t st);
void launch_extrapolate(double* out, const double* a, const double* b, double ratio, long long n,
                        cudaStream_t st);

}  // namespace pfc
