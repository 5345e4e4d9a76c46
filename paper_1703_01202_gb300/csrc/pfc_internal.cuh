// Internal declarations shared by the CUDA translation units of libpfc.
#pragma once
#include <cuda.h>  // CUtensorMap (the type only; the driver's encoder is looked up at run time)
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstddef>
#include <cstdint>

namespace pfc {

constexpr int kMaxRestart = 60;   // GMRES restart length limit
constexpr int kMaxVecs = kMaxRestart + 2;
constexpr int kRedCtas = 4 * 152;  // CTAs of the grid-stride reduction kernels

// Programmatic dependent launch between the kernels of an Arnoldi iteration: a kernel launched
// with launch_pdl may be scheduled while the kernel before it on the stream drains; it calls
// pdl_wait() before reading anything (every earlier kernel has then completed and its writes are
// visible).  A kernel calls pdl_trigger() once its main work is done, so that the next one can be
// scheduled during its tail (the last CTA's reduction).  Both are no-ops for kernels launched
// without the attribute.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                              Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// Geometry of the grid (x fastest; periodic or between mirror walls) and the scheme's constants.
struct Geo {
  int nx, ny, nz;
  long long n;      // nx * ny * nz
  double ih2;       // 1 / h^2
  double gamma;     // quench depth of Eq. (GE)
  double hd;        // h^d (cell volume)
  int neumann;      // 0: periodic grid; 1: mirror walls half a cell outside the end cells (Sec. 2)
  // derived on the host by geo_constants (kernels read them instead of computing them per thread)
  double ih4;       // ih2 * ih2
  double hih4;      // 0.5 * ih2 * ih2
  double c0;        // 0.5 * (1 - gamma)
};
inline void geo_constants(Geo* g) {
  g->ih4 = g->ih2 * g->ih2;
  g->hih4 = 0.5 * g->ih2 * g->ih2;
  g->c0 = 0.5 * (1.0 - g->gamma);
}

// Cell that index i (any integer) of an axis of n cells reads: the periodic image, or, between
// mirror walls, the image in the evenly extended grid of period 2n (ghost -1 -> 0, n -> n - 1).
__device__ __forceinline__ int cell_index(int i, int n, int neumann) {
  if (!neumann) {
    i %= n;
    return i < 0 ? i + n : i;
  }
  const int p = 2 * n;
  i %= p;
  if (i < 0) i += p;
  return i < n ? i : p - 1 - i;
}

// One overlapped subdomain Omega_k^delta and its core Omega_k (Sec. 4).
struct BlockDesc {
  int x0, y0, z0;  // global cell of block-local (0,0,0); may be negative (periodic wrap; >= 0 between walls)
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
  int n_reorth;  // second passes run in this cycle
  double tol, beta, est;
  double wnorm2_before;
  double reorth_eta2;  // second pass when ||w'||^2 < reorth_eta2 ||w||^2 (0: never)
  double H[(kMaxRestart + 1) * kMaxRestart];  // column-major: H[i + (m+1) j]
  double cs[kMaxRestart], sn[kMaxRestart], g[kMaxRestart + 1], y[kMaxRestart];
  double scale[kMaxRestart + 2];  // V_i = scale_i * Vraw_i
  double coef[kMaxRestart + 2];   // coefficients of the pending multi-axpy
  double red[kMaxVecs + 2];       // reduced sums of the last multi-dot / axpy
};

// Arguments of one Arnoldi iteration read from device memory, so that a captured
// CUDA graph can loop over iterations: j and the vectors of step j are written by
// the loop-condition kernel before every iteration; q and idt by the host once per
// GMRES solve.
struct IterArgs {
  int j;
  const double* v;      // V_j (preconditioner input)
  double* z;            // Z_j = M^-1 V_j
  double* w;            // V_{j+1} = J Z_j before orthogonalisation
  const double* scale;  // &scale[j]
  const double* q;      // Jacobian coefficient of this Newton iteration
  double idt;           // 1 / dt
  const double* mu;     // variable mobility: mu and the midpoint s = (Phi + phi^n)/2 of this
  const double* sm;     // Newton iteration (null with M = 1)
  int zplane;           // z = Z_zplane of the basis (the JVP may stage it by TMA); -1: z is not
};

// Device-side control of one time step (inexact Newton, Sec. 4): every decision of
// the Newton loop, the GMRES restart loop and the backtracking line search is taken
// by a one-thread kernel on these fields, so that a whole step can run as one CUDA
// graph (conditional nodes driven by the *_go fields) or from the host, which reads
// the same fields back; both execute the same kernels in the same order.
struct StepCtl {
  // set by the host before the step
  double idt;       // 1 / dt
  double ref_norm;  // ||F(phi^n)|| for the stop test with another guess (< 0: ||F(Phi_0)||)
  double newton_rtol, newton_atol, gmres_rtol, gmres_atol, ls_alpha, reorth_eta2;
  int newton_max_it, ls_max_cuts, gmres_max_it, refactor;
  // state of the step
  double r0, target, rnorm, f0, ft, lam, gtol;
  int m, gm_total, gm_its, cuts_total, cut, status;
  // branch and loop conditions
  int newton_go, factor_go, cycle_go, restart_go, ls_go, commit_go;
  // what ran (the host counts the launches of a graph step from these)
  int n_factor, n_cycles, n_restarts, n_trials, n_reorth;
  // time loop of the batch form (pfc_run_batch): the adaptive step of Eq. (sencondt), retries
  // with dt / 2, per-step records, all on the device
  double dt, dt_prev, E_n, E_nm1;   // controller state
  double dt_min, dt_max, eta, escale, hd;
  int have_Em1, have_prev_dt;
  int steps_target, steps_done, cuts, dt_halvings, failed, loop_go;
  int body_kernels, chunked;        // kernels of one Arnoldi iteration; 1: factor + chunk records
  long long kernels;                // kernels the time loop has run
};
// Conditional handles of a step graph (unused when the host drives the step).
struct StepHandles {
  cudaGraphConditionalHandle newton, factor, cycle, arnoldi, restart, ls, commit, mloop, reorth;
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
void count_pause(bool on);  // the calling thread is capturing a graph: its launches run later
void count_graph_launch();
extern long long g_graph_launches;
long long launches_so_far();

// ---- stencil kernels (stencil2d.cu)
// mob: variable mobility M = 1 - s^2 at the midpoint s = (Phi + phi^n)/2 (Eq. NSOP's M_d); the
// residual then also writes mu and s beside q (mu_out, s_out), and the JVP reads them (mu, sm).
// idt_dev / lam_dev (optional): 1/dt and the line-search step read from device memory instead of
// idt / lam (a captured step graph serves every time step).
void launch_residual2d(const Geo& g, const double* Phi_base, const double* S, double lam, const double* smean,
                       const double* phin, double idt, double* F, double* Phi_out, double* q_out, double* partial,
                       int* nparts, cudaStream_t st, bool mob = false, double* mu_out = nullptr,
                       double* s_out = nullptr, const double* idt_dev = nullptr, const double* lam_dev = nullptr);
void launch_jvp2d(const Geo& g, const double* v, const double* vscale, const double* q, double idt, double* Jv,
                  const int* skip, cudaStream_t st, const IterArgs* ia = nullptr, const double* mu = nullptr,
                  const double* sm = nullptr);
void launch_energy2d(const Geo& g, const double* phi, double* partial, int* nparts, cudaStream_t st);
// Tensor maps of the mixed path's JVP (jvp_ff.cu): the basis Z_0..Z_(m-1) as an nx x ny x m
// tensor (planes vstride doubles apart) and the Jacobian coefficient q as an nx x ny one.  An
// interior tile stages its halo boxes of Z_j and q with two TMA tensor copies.
struct JvpMaps {
  CUtensorMap z;
  CUtensorMap q;
  int ok;
};
constexpr int kJvpBoxVX = 40, kJvpBoxVY = 22, kJvpBoxQX = 36, kJvpBoxQY = 18;
// Encodes the two maps; maps->ok stays 0 (plain loads) when the grid is too small for the boxes,
// nx is odd (row strides must be multiples of 16 bytes) or the driver's encoder is unavailable.
void encode_jvp_maps(const Geo& g, const double* Zbuf, size_t vstride, int m, const double* q, JvpMaps* maps);
// The same JVP in float-float arithmetic on the FP32 pipe (jvp_ff.cu), for the mixed path.  With
// maps (ok) and v = Z_zj of the basis (zj >= 0, or ia->zplane in graph mode) and q the mapped
// one, interior tiles stage by TMA; a staging wait that runs out records PFC_ETIMEOUT in *err.
void launch_jvp2d_ff(const Geo& g, const double* v, const double* vscale, const double* q, double idt, double* Jv,
                     const int* skip, cudaStream_t st, const IterArgs* ia = nullptr, const JvpMaps* maps = nullptr,
                     int zj = -1, int* err = nullptr, int pout = 0);
// The same JVP in plain FP32 (opt-in on the mixed path, pfc_params.jvp_fp32).
// pout (both): Jv is stored as float pairs (ff.cuh), the form of the mixed path's Krylov basis.
void launch_jvp2d_f32(const Geo& g, const double* v, const double* q, double idt, double* Jv, const int* skip,
                      cudaStream_t st, const IterArgs* ia = nullptr, const JvpMaps* maps = nullptr, int zj = -1,
                      int* err = nullptr, int pout = 0);
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
  int variant;       // apply launch shape, 0 .. kApplyVariants - 1
  const int* order;  // two-per-warp shape: blocks grouped by extent, each group padded to an even count with -1
  int norder;
  // Chunked form of the same factors (apply variant kChunkedVariant); built from L, U, piv
  // by launch_chunk2d.  Record-major: record t of every block (in the order the apply
  // consumes them: forward chunks 0 .. nc-1, then backward chunks nc-1 .. 0) lies next to
  // record t of the neighbouring blocks, so the warps of one apply stream through
  // memory together.
  unsigned char* X;
  size_t xfw, xbw;  // stride of the forward / backward records (the largest of each)
  int xnc;          // chunks of the largest block
  int nblk;         // blocks
  int xstage;       // bytes of the largest record (one TMA stage)
  int x_valid;      // X holds the chunks of the current factors
  // Schwarz form (Sec. 4): PFC_LEFT_RAS writes block cores only; PFC_AS (Eq. invM) and
  // PFC_RIGHT_RAS (Eq. ash) extend over the whole block, so the chunked apply writes every
  // block's solution to Yb (n_max doubles per block) and k_schwarz_sum adds the overlapping
  // parts point by point; PFC_RIGHT_RAS also restricts r to the core (R_k^0).
  int ras_kind;
  double* Yb;
  int pin;  // the apply's input r is stored as float pairs (the mixed path's Krylov basis)
  // variable mobility: mu and s = (Phi + phi^n)/2 at the factored iterate (null: M = 1), and the
  // largest (bx + 2)(by + 2) of a block with its one-cell ring
  const double* mob_mu;
  const double* mob_s;
  int ext_max;
};
// Axis splits of the 2D decomposition (the first n mod p cores one cell larger).
struct Decomp2 {
  int px, py, ov;
  int base_x, rem_x, base_y, rem_y;
};
constexpr int kApplyVariants = 6;
constexpr int kChunkedVariant = 5;

// Chunked triangular solves.  The forward solve P/L of a block advances kChunk
// elimination steps at a time: the steps k0 .. k0+bc-1 (bc = min(kChunk, n-k0))
// act on the window of positions [k0, k0+W), W = kChunk + kl, as a row permutation
// (their interchanges combined) followed by the unit lower triangular factor with
// the chunk's multipliers, each moved by the interchanges after its own step:
// y_c = E11 t_c on the chunk's rows (E11 = inverse of its kChunk x kChunk block)
// and y_b = t_b - L21 y_c on the kl rows below.  The backward solve takes the same
// chunks from the bottom: x_c = U11^{-1} y_c, then y_a -= U_a x_c on the ku2 rows
// above.  L21 and U_a are entries of the factors themselves (storage type); the
// small inverses are kept in the compute type.
// Records (16-byte multiples): forward = W permutation bytes rounded up to 16,
// E11 (kChunk^2, compute type, row-major), -L21 (kl rows of kChunk); backward =
// U11^{-1} (kChunk^2, compute type), -U_a (ku2 rows of kChunk, positions
// k0-ku2 .. k0-1).
constexpr int kChunk = 8;
struct ChunkGeom {
  int n, kl, ku2, nc, W;
  size_t fwd, bwd;  // record bytes
};
// es: bytes of a stored factor entry; tc: bytes of the compute type
__host__ __device__ inline ChunkGeom chunk_geom(int bx, int by, int es, int tc) {
  ChunkGeom c;
  c.n = bx * by;
  c.kl = 3 * bx < c.n - 1 ? 3 * bx : c.n - 1;
  c.ku2 = 2 * c.kl < c.n - 1 ? 2 * c.kl : c.n - 1;
  c.nc = (c.n + kChunk - 1) / kChunk;
  c.W = kChunk + c.kl;
  c.fwd = (size_t)(c.W + 15) / 16 * 16 + (size_t)kChunk * kChunk * tc + (size_t)c.kl * kChunk * es;
  c.bwd = (size_t)kChunk * kChunk * tc + (size_t)c.ku2 * kChunk * es;
  return c;
}
// Byte offset in X of record t (consumption order) of block b with nc chunks.
__host__ __device__ inline size_t chunk_rec_off(const FactorStore& fs, int b, int nc, int t) {
  if (t < nc) return ((size_t)t * fs.nblk + b) * fs.xfw;
  return (size_t)fs.xnc * fs.nblk * fs.xfw + ((size_t)(t - nc) * fs.nblk + b) * fs.xbw;
}
void launch_chunk2d(const BlockDesc* blocks, int nblocks, const FactorStore& fs, cudaStream_t st);
void launch_factor2d(const Geo& g, const BlockDesc* blocks, int nblocks, const double* q, double idt,
                     const double* lin, const FactorStore& fs, int* status, cudaStream_t st,
                     const double* idt_dev = nullptr);
void launch_ras_apply2d(const Geo& g, const BlockDesc* blocks, int nblocks, const FactorStore& fs, const double* r,
                        const double* rscale, double* z, const int* skip, int* err, cudaStream_t st,
                        const IterArgs* ia = nullptr, const Decomp2* dc = nullptr);
size_t factor_smem_bytes(int prec, int kl, int n_max, int ext_max = 0);
// Whether apply variant v runs blocks of half-bandwidth kl_max at precision prec
// (xstage: bytes of the largest chunk record, n_max: rows of the largest block).
bool apply_variant_ok(int v, int prec, int kl_max, int xstage, int n_max);

// ---- 3D stencils (stencil3d.cu)
void launch_trial(const Geo& g, const double* Pb, const double* S, double lam, const double* ssum, double* Pout,
                  cudaStream_t st);
// mob: variable mobility M = 1 - s^2, s = (P + phin)/2; mu and s written to mu_out, s_out when given.
void launch_residual3d(const Geo& g, const double* P, const double* phin, double idt, double* F, double* q_out,
                       double* T1, double* T2, double* partial, int* nparts, cudaStream_t st, bool mob = false,
                       double* mu_out = nullptr, double* s_out = nullptr);
// mu, sm (variable mobility): mu and s of the iterate q belongs to; null: M = 1.
void launch_jvp3d(const Geo& g, const double* v, const double* vscale, const double* q, double idt, double* Jv,
                  double* T1, double* T2, const int* skip, cudaStream_t st, const double* mu = nullptr,
                  const double* sm = nullptr);
// The same product in float-float arithmetic (the mixed path); T1, T2 hold float pairs.
void launch_jvp3d_ff(const Geo& g, const double* v, const double* q, double idt, double* Jv, double* T1, double* T2,
                     const int* skip, cudaStream_t st, int pout = 0);  // pout: Jv as float pairs
// The same product in plain FP32 (opt-in on the mixed path, pfc_params.jvp_fp32); T1, T2 hold floats.
void launch_jvp3d_f32(const Geo& g, const double* v, const double* q, double idt, double* Jv, double* T1, double* T2,
                      const int* skip, cudaStream_t st, int pout = 0);
void launch_energy3d(const Geo& g, const double* phi, double* partial, int* nparts, cudaStream_t st);

// ---- 3D Schwarz preconditioner with shifted ILU(0) subdomain solves (ras3d.cu)
// The 63 offsets (da, db, dc) with |da|+|db|+|dc| <= 3 in lexicographic (dc, db, da)
// order: 0..30 lower, 31 the diagonal, 32..62 upper.
constexpr int kNOff = 63;
// Blocks of equal extent share one shape: rows in level order (level = a + 3b + 7c,
// which every lower offset strictly decreases), padded positions (3-cell zero ring).
struct Shape3 {
  int bx, by, bz, px, py, pz;
  int nrows, nlev;
  int lev_off;  // level starts: lev_start[lev_off .. lev_off + nlev]
  int row_off;  // rowpad / rowabc: [row_off .. row_off + nrows)
  int poff[kNOff];
};
struct Ras3D {
  const Shape3* shapes;
  const int* block_shape;
  const int* lev_start;
  const int* rowpad;  // padded linear position of each row
  const int* rowabc;  // block-local cell (a, b, c) of each row, packed a | b << 10 | c << 20
  void* Lp;           // per block nrows_max x 32: L multipliers of offsets 0..30 (storage type)
  void* Up;           // per block nrows_max x 32: [0] inverted diagonal, [1..31] offsets 32..62
  void* work;         // per block nrows_max x 32: U parts of factored rows by block cell (compute type)
  void* ypad;         // per block pad_max (compute type): solve vector with zero ring
  size_t sLU, sWork, sPad;
  int prec;
  int max_level_rows;
  int max_nlev;       // most levels of a block
  int window;         // 1: FP32 solves in the shared-memory level window (apply3d_window_ok)
  const uint8_t* posL;  // per row, 32 bytes in the level layout: place of each lower / upper
  const uint8_t* posU;  // neighbour in its level's row list (255: outside the block)
  double shift;       // diagonal shift, relative to the block's mean |a_ii|
  int pin;            // the apply's input r is stored as float pairs (the mixed path's Krylov basis)
  const double* mob_mu;  // variable mobility: mu and s = (Phi + phi^n)/2 at the factored iterate
  const double* mob_s;   // (null: M = 1)
};
// Whether the window apply can run these blocks: FP32/BF16 factors and levels of at most 255 rows.
bool apply3d_window_ok(const Ras3D& R);
void launch_factor3d(const Geo& g, const BlockDesc* blocks, int nblocks, const double* q, double idt,
                     const double* lin343, const Ras3D& R, int* status, cudaStream_t st);
void launch_ras_apply3d(const Geo& g, const BlockDesc* blocks, int nblocks, const Ras3D& R, const double* r,
                        const double* rscale, double* z, const int* skip, int* err, cudaStream_t st);

// ---- learned initial guess network (cnn.cu)
struct Cnn;
size_t cnn_workspace_bytes(long long n);
void cnn_bind(Cnn* c, void* ws);
void cnn_forward(Cnn* c, const double* feat);
int cnn_status(Cnn* c);  // PFC_ETIMEOUT if a bounded wait of the network's kernels ran out (then cleared)
int cnn_backward(Cnn* c, const double* feat, const double* target, int* nparts);
void cnn_adam(Cnn* c, float lr, int t);
void cnn_refresh_bf16(Cnn* c);
void cnn_out_to_f64(Cnn* c, double* out);
const float* cnn_output(const Cnn* c);
int cnn_nx(const Cnn* c);
cudaStream_t cnn_swap_stream(Cnn* c, cudaStream_t st);  // returns the previous stream
int cnn_ny(const Cnn* c);
// features (phi^n - mean, r (phi^n - phi^{n-1}), dt / dt_max) as 3 planes; guess pieces
void launch_cnn_features(long long n, const double* phin, const double* phinm1, const double* mass_sum, double r,
                         double c2, double* feat, cudaStream_t st);
void launch_cnn_delta(long long n, const double* feat, const float* out, double s_out, double* delta,
                      double* partial, int* nparts, cudaStream_t st);
void launch_add_centered(long long n, const double* base, const double* delta, const double* dsum, double* out,
                         cudaStream_t st);
void launch_sum(long long n, const double* x, double* partial, int* nparts, cudaStream_t st);
void launch_cnn_target(long long n, const double* phinp1, const double* phin, const double* feat, double s_out,
                       double* target, cudaStream_t st);

// ---- Krylov vector kernels (krylov.cu)
// What the last CTA of a multi-dot / multi-axpy does after the fixed-order
// reduction of all CTAs' partial sums (counter: a device ticket that is zero
// between launches; a null counter means "partials only").
struct Tail {
  enum { kSums = 0, kDot = 1, kAxpy = 2 };
  int kind;
  int j, pass, m;           // Arnoldi column, Gram-Schmidt pass, restart length
  GmresCtl* ctl;
  unsigned int* counter;
  double* out;              // kSums: reduced values
  const IterArgs* ia;       // when set, j comes from ia->j (graph mode)
  int* err = nullptr;       // PFC_ETIMEOUT is stored here when a bounded wait runs out
  const int* nx_dev = nullptr;  // multi-axpy: the vector count read from device memory (graph mode)
  // graph mode, first Gram-Schmidt pass: the kAxpy tail sets this conditional handle to
  // "second pass wanted" (the IF node around the second pass's sweeps)
  cudaGraphConditionalHandle h_reorth = 0;
  int set_reorth = 0;
};

// Vector lists: entry 0 is v0 (x0), entry i > 0 is tab[i] (a device array of pointers).
// With tail.ia set (graph mode) the vector count is ia->j + 2 (dot) / ia->j + 1 (axpy), w is
// ia->w, and nv / nx only bound the grid.
// dot: arithmetic of the products -- kDotF64, kDotFF (float-float on the FP32 pipe, the mixed
// path's default) or kDotF32 (FP32 products of values cut to floats, opt-in).
// ff: float-float multi-axpy on the FP32 pipe (the mixed path's Arnoldi sweeps)
// pairs: the vectors (and w) are stored as float pairs (ff.cuh), the mixed path's Krylov
// basis; with dot = kDotFF / kDotF32 and, for the multi-axpy, ff and a tail other than kSums
constexpr int kDotF64 = 0, kDotFF = 1, kDotF32 = 2;
void launch_multidot(const double* v0, const double* const* tab, int nv, const double* w, long long n,
                     double* partial, const int* skip, const int* only_if, const Tail& tail, cudaStream_t st,
                     int dot = kDotF64, int nv_grid = 0, bool pairs = false);
void launch_multiaxpy(double* w, const double* x0, const double* const* tab, int nx, const double* coef, double sign,
                      long long n, double* partial, const int* skip, const int* only_if, const Tail& tail,
                      cudaStream_t st, bool ff = false, bool pairs = false);
// Graph-mode helpers: ia <- the vectors of iteration j = ctl->its; loop condition of a GMRES cycle.
// Graph mode, before the Arnoldi loop and at the end of each iteration: the loop's
// conditional handle h = (cycle not done and fewer than m iterations), and when it goes on,
// the next iteration's vectors in ia (j = its; V_j, Z_j, V_{j+1} from the pointer tables).
void launch_arnoldi_next(const GmresCtl* ctl, const double* const* vtab, const double* const* ztab, IterArgs* ia,
                         int m, cudaGraphConditionalHandle h, cudaStream_t st);
void launch_reduce(const double* partial, int nvals, int nparts, double* out, cudaStream_t st);
// ---- step control (newton.cu); graph = 1 also sets the conditional handles in h
void launch_newton_begin(StepCtl* c, const double* nrm2, IterArgs* ia, IterArgs* ia_restart, const StepHandles& h,
                         int graph, cudaStream_t st);
void launch_set_factor_cond(StepCtl* c, const StepHandles& h, int graph, cudaStream_t st);
void launch_factor_done(StepCtl* c, cudaStream_t st);
void launch_gmres_begin(StepCtl* c, GmresCtl* g, const StepHandles& h, int graph, cudaStream_t st);
void launch_cycle_decide(StepCtl* c, GmresCtl* g, const StepHandles& h, int graph, cudaStream_t st);
void launch_gmres_restart(StepCtl* c, GmresCtl* g, const double* nrm2, cudaStream_t st);
void launch_gmres_end(StepCtl* c, const int* status_dev, const StepHandles& h, int graph, cudaStream_t st);
void launch_ls_decide(StepCtl* c, const double* nrm2, const StepHandles& h, int graph, cudaStream_t st);
// Copies src[k] -> dst[k] (k < npairs, N doubles each) when the step's status is still PFC_OK.
// Bit k of to_pairs: dst[k] receives src[k] as float pairs (ff.cuh) instead of a copy.
struct CopyPairs {
  const double* src[5];
  double* dst[5];
  int n;
  unsigned to_pairs;
};
void launch_copy_if_ok(const StepCtl* c, const CopyPairs& cp, long long n, cudaStream_t st);
// GMRES start: S = 0, red2[0..1] = 0 (|S|^2, sum S), V0 <- F (as float pairs with pairs).
void launch_gmres_prep(double* S, double* red2, const double* F, double* V0, long long n, cudaStream_t st,
                       bool pairs = false);
void launch_newton_next(StepCtl* c, const StepHandles& h, int graph, cudaStream_t st);
void launch_step_end(StepCtl* c, const StepHandles& h, int graph, cudaStream_t st);
// Batch form's device time loop: the loop test, the next step's dt (or the halved retry), and
// the bookkeeping after a step (record into rec[steps_done], energy history, retry or stop).
// rec points to pfc_step_info records (include/pfc.h).
void launch_mloop_begin(StepCtl* c, const StepHandles& h, cudaStream_t st);
void launch_mstep_prep(StepCtl* c, cudaStream_t st);
void launch_mstep_end(StepCtl* c, const double* red45, void* rec, const StepHandles& h, cudaStream_t st);
// The time step Eq. (sencondt) gives (the same arithmetic on host and device).
__host__ __device__ inline double controller_dt(double E_n, double E_nm1, double dt_prev, double escale, double dt_min,
                                                double dt_max, double eta, bool have) {
  if (!have) return dt_min;
#ifdef __CUDA_ARCH__
  const double fp = __ddiv_rn(__dmul_rn(__dsub_rn(E_n, E_nm1), escale), dt_prev);
  const double d = __ddiv_rn(dt_max, __dsqrt_rn(__dadd_rn(1.0, __dmul_rn(__dmul_rn(eta, fp), fp))));
#else
  const double fp = (E_n - E_nm1) * escale / dt_prev;
  const double d = dt_max / std::sqrt(1.0 + eta * fp * fp);
#endif
  return d > dt_min ? d : dt_min;
}
void launch_gmres_init(GmresCtl* ctl, const double* nrm2, double sign, double tol, double reorth_eta2,
                       cudaStream_t st);
void launch_gmres_solve(GmresCtl* ctl, cudaStream_t st);
void launch_axpby(double* y, const double* x, double a, double b, long long n, cudaStream_t st);
void launch_extrapolate(double* out, const double* a, const double* b, double ratio, long long n,
                        cudaStream_t st);

}  // namespace pfc
