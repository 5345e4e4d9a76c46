/*
 * pfc.h -- C ABI of the GB300 phase-field-crystal time stepper.
 *
 * One call of pfc_step advances the density field phi^n by one time step of
 * the energy-stable DVDM semi-implicit scheme (Eq. NSOP with the discrete
 * variational derivative of Eq. discretedG; mobility M = 1 or 1 - phi^2,
 * periodic grid or Neumann-type walls, see pfc_params),
 * solving the nonlinear system F(Phi) = 0 (Eq. NLS) by inexact Newton
 * (Eq. newton) with right-preconditioned GMRES (Eq. hjacobi) and a restricted
 * additive Schwarz preconditioner with the paper's "improved" subdomain
 * boundary condition (Sec. 4, Eqs. ras, Ak).  pfc_run adds the adaptive time
 * step of Eq. (sencondt).
 *
 * Conventions shared by every entry point
 *  - Fields are float64, one value per cell of an Nx x Ny (x Nz) cell-centred
 *    grid (periodic unless pfc_params.boundary says otherwise) with isotropic
 *    spacing h, row-major with x fastest:
 *    idx = i + Nx * (j + Ny * k).
 *  - The library never allocates device memory.  The caller allocates one
 *    device workspace of pfc_workspace_size() bytes (256-byte aligned) and
 *    passes it, together with the CUDA stream all work is queued on, to
 *    pfc_create.  The workspace and the stream stay owned by the caller and
 *    must outlive the state.  Host arrays are caller-owned and are never
 *    retained past the call.
 *  - Every function returns a pfc_status (0 = success).  On any error pfc_step
 *    and pfc_run leave phi^n, phi^{n-1} and the energy history unchanged.
 *  - Calls on one state are not thread-safe; distinct states are independent.
 */
#ifndef PFC_H
#define PFC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  PFC_OK = 0,
  PFC_EINVAL = -1,     /* bad argument (sizes, parameters, null pointers)        */
  PFC_ENOMEM = -2,     /* workspace smaller than pfc_workspace_size()             */
  PFC_ECUDA = -3,      /* a CUDA runtime call failed                              */
  PFC_ENEWTON = -4,    /* Newton reached newton_max_it without meeting its test   */
  PFC_EGMRES = -5,     /* GMRES reached gmres_max_it without meeting its test     */
  PFC_ESINGULAR = -6,  /* a subdomain factorisation met a zero pivot              */
  PFC_ENAN = -7,       /* a residual norm became NaN or Inf                       */
  PFC_ETIMEOUT = -8    /* a bounded device-side wait ran out                      */
} pfc_status;

/* Subdomain factor storage precision. */
enum { PFC_F64 = 0, PFC_F32 = 1, PFC_BF16 = 2 };
/* Schwarz variant (Sec. 4): Eq. invM, Eq. ras, Eq. ash. */
enum { PFC_AS = 0, PFC_LEFT_RAS = 1, PFC_RIGHT_RAS = 2 };
/* Domain boundary (pfc_params.boundary). */
enum { PFC_PERIODIC = 0, PFC_NEUMANN = 1 };
/* Newton initial guess: phi^n (Sec. 4), linear extrapolation, caller-supplied,
   or the learned network (pfc_set_guess_net).  EXTRAP and LEARNED are
   safeguarded: the residual norm of every candidate (phi^n, the extrapolation,
   and the network's guess for LEARNED) is evaluated and Newton starts from the
   smallest; pfc_step_info.guess_used reports the pick. */
enum { PFC_GUESS_PREV = 0, PFC_GUESS_EXTRAP = 1, PFC_GUESS_USER = 2, PFC_GUESS_LEARNED = 3 };

typedef struct {
  int dim;       /* 2 or 3                                        */
  int64_t n[3];  /* Nx, Ny, Nz (n[2] = 1 when dim == 2)          */
} pfc_grid;

typedef struct {
  /* Newton stop test ||F(Phi_{m+1})|| <= max(newton_rtol ||F(Phi_0)||, newton_atol)
     (Sec. 4, Newton stopping condition); 2-norms.  With the EXTRAP / LEARNED
     guesses ||F(Phi_0)|| is that of Phi_0 = phi^n, the paper's start, so the
     tolerance does not depend on the guess. */
  double newton_rtol, newton_atol;
  int newton_max_it;
  /* GMRES stop test ||r_m|| <= max(gmres_rtol ||F(Phi_m)||, gmres_atol) (Sec. 4). */
  double gmres_rtol, gmres_atol;
  int gmres_restart, gmres_max_it;
  /* Decomposition: sub[a] cores along x, y, z (uneven splits give the first
     cores one extra cell); overlap = cells added per side (Sec. 4). */
  int sub[3];
  int overlap;
  int ras_kind;      /* Schwarz form (Sec. 4): PFC_LEFT_RAS (default, Eq. ras:
                        solve on the overlapped block, keep the core), PFC_AS
                        (Eq. invM: keep the whole block, overlaps summed) or
                        PFC_RIGHT_RAS (Eq. ash: core of r in, whole block out).
                        AS and right-RAS: 2D grids, apply_variant -1 or 5.   */
  int factor_prec;   /* PFC_F64 (plain path), PFC_F32 or PFC_BF16 storage    */
  int guess;         /* PFC_GUESS_*                                          */
  int mass_projection; /* 1: Newton update projected to zero mean            */
  double ls_alpha;   /* Armijo constant of the backtracking line search      */
  int ls_max_cuts;
  /* Adaptive time step, Eq. (sencondt); energy_scaled = 1 feeds F_d/|Omega|. */
  double dt_min, dt_max, eta;
  int energy_scaled;
  /* 2D Schwarz apply kernel.  Per-step triangular solves (steps per bulk copy
     x warps per CTA): 0 default, 1 half-length copies, 2 half-length copies and
     2-warp CTAs, 3 double-length copies, 4 two subdomains per warp (16 lanes
     each); these five give bitwise identical results.  5: chunked solves, the
     same factors regrouped 8 elimination steps at a time (a row permutation and
     a dense 8-column product per group, built after each factorisation; equal
     to 0-4 up to rounding in the storage type).
     -1 (default) times every kernel on the first factorisation and keeps the
     fastest (pfc_get_tuning reports the pick).
     Blocks wider than 21 cells in x (kl = 3 bx > 64) accept only 0 and 5.
     3D grids: 0 solves with the block's solve vector in global memory; 1 keeps
     the 22 wavefront levels a solve reads in shared memory (F32/BF16 factors,
     at most 255 rows per level; otherwise pfc_create fails with PFC_EINVAL);
     -1 takes 1 where it can run, else 0.
     The two give bitwise identical results; 2..5 are refused in 3D. */
  int apply_variant;
  /* pfc_run only: a step whose Newton or GMRES iteration fails (PFC_ENEWTON,
     PFC_EGMRES) is retried with half the time step, at most dt_halvings times
     (default 0: the failure is returned).  The paper is silent on failures. */
  int dt_halvings;
  /* Classical Gram-Schmidt re-orthogonalisation test (Daniel-Gragg-Kaufman-
     Stewart): a second pass when ||w'|| < gmres_reorth_eta ||w||; default 0.3
     (a second pass only under strong cancellation); 1/sqrt(2) is the classical
     choice; 0 = one pass only.  Both sweeps have FP64-class accuracy (FP64 on
     the plain path, float-float on the mixed path; see gmres_fast_dots). */
  double gmres_reorth_eta;
  /* 2D: run every time step as one CUDA graph launch (default 1).  The step --
     Newton loop with its stop test, factor branch, GMRES restart loop, Arnoldi
     loop, restart branch, backtracking line search and the commit of the new
     field -- is captured once as nested conditional nodes whose conditions are
     set by one-thread control kernels on the device; the host only writes the
     step's inputs (dt, tolerances) and reads back one control block per step.
     Used once the apply kernel is fixed (after the first factorisation when
     apply_variant = -1), on a stream other than the legacy default stream and
     while pfc_profile is off; otherwise, or if the graph cannot be built, the
     host drives the same kernels, reading the control block after each
     decision.  Both forms give identical results. */
  int use_graph;
  /* Factor reuse across time steps (extends the paper's reuse within a step,
     Sec. 5.2): 0 (default) factors the subdomain matrices at the first Newton
     iteration of every step; k > 0 keeps them for up to k further steps while
     dt stays within 1e-3 (relative) of the dt they were made with.  Changes
     the preconditioner only, not the converged phi^{n+1}. */
  int reuse_factor;
  /* Mobility of Eq. (NSOP): 0 (default) M = 1; 1: M(phi) = 1 - phi^2 evaluated at
     (Phi + phi^n)/2 and averaged onto edges (Sec. 3), with the Jacobian's
     dM/dPhi term.  2D and 3D periodic grids; the JVP then runs in FP64 on every
     path. */
  int mobility;
  /* Boundary of the domain: PFC_PERIODIC (0, default) or PFC_NEUMANN (1), the
     homogeneous Neumann-type conditions of Sec. 2 (n.grad phi = n.grad Delta phi =
     n.grad Delta^2 phi = 0) as mirror walls half a cell outside the end cells: every
     stencil reads the mirror image of a cell beyond a wall.  The overlapped
     subdomains stop at the walls and A_k is the principal submatrix of the Neumann
     Jacobian (the mirror images folded into the block's own columns).  Grids of
     at least 4 cells per axis (2D and 3D), left-RAS, mobility 0; 3D blocks at least
     7 cells per axis; pfc_residual_static stays periodic. */
  int boundary;
  /* Arnoldi dot products of the mixed path (F32/BF16 factors): 0 (default)
     float-float products and sums on the FP32 pipe (about 2^-46 relative, like
     the multi-axpy, so the orthogonalisation keeps FP64-class accuracy); 1: FP32
     products of the vectors cut to 24-bit significands (faster; the
     re-orthogonalisation pass then carries more of the orthogonality).  The
     plain path (F64 factors) always uses FP64 sweeps. */
  int gmres_fast_dots;
  /* JVP of the mixed path (F32/BF16 factors, M = 1, 2D and 3D): 0 (default)
     float-float on the FP32 pipe (about 2^-46 relative, so GMRES sees the FP64
     operator); 1: plain FP32 (v and q cut to floats; much cheaper, about 2^-24 of
     the largest stencil terms per point).  The Newton residual stays FP64, so the
     converged phi^{n+1} meets the same tolerance either way; the iteration
     counts tell whether the cheaper operator pays.  The plain path (F64
     factors) and variable mobility always use the FP64 JVP. */
  int jvp_fp32;
} pfc_params;

typedef struct {
  int status;        /* pfc_status of the step                                */
  int newton_its;    /* Newton iterations taken                               */
  int gmres_its;     /* GMRES iterations summed over the Newton iterations    */
  int ls_cuts;       /* line-search step reductions summed over the step      */
  double dt;         /* time step used                                        */
  double energy;     /* F_d(phi^{n+1}), Eq. (freeenergy)                      */
  double mass;       /* h^d sum phi^{n+1}                                      */
  double res_norm0;  /* ||F(Phi_0)||                                          */
  double res_norm;   /* ||F(phi^{n+1})||                                      */
  int guess_used;    /* PFC_GUESS_* actually used for Phi_0 (safeguard pick)   */
  int dt_cuts;       /* pfc_run: halvings of the controller's dt before success */
} pfc_step_info;

typedef struct pfc_cnn pfc_cnn;

typedef struct pfc_state pfc_state;

/* Fills *p with the defaults: Newton rtol 1e-10, GMRES rtol 1e-6, restart 30,
   left-RAS, overlap 1, F64 factors, guess = phi^n, mass projection on,
   Armijo 1e-4 with 10 cuts, dt in [1e-2, 10], eta 5000, scaled energy. */
int pfc_default_params(pfc_params* p);

/* Bytes of device workspace a state for this grid and these parameters needs.
   Errors: PFC_EINVAL for an invalid grid or decomposition (a block, core plus
   2*overlap, wider than the grid along an axis). */
int pfc_workspace_size(const pfc_grid* g, const pfc_params* p, size_t* bytes);

/* Host only (no device work): the overlapped subdomains Omega_k^delta of Sec. 4 that
   a state with this grid and these parameters factors, in its block order (x
   fastest, then y, then z).  Block k is 12 ints at out[12 k]: first cell x0, y0, z0
   (negative, or reaching past the grid's end, where a periodic block wraps; never
   between Neumann walls, where blocks stop at the walls), extent bx, by, bz, core
   offset inside the block ox, oy, oz and core extent cx, cy, cz (2D: z0 = oz = 0,
   bz = cz = 1).  Writes min(cap, count) blocks (out may be NULL when cap is 0) and
   the count to *nblocks.  Errors: PFC_EINVAL as pfc_workspace_size, or cap < 0. */
int pfc_block_layout(const pfc_grid* g, const pfc_params* p, int* out, int cap, int* nblocks);

/* Creates a state on the current CUDA device.  h: grid spacing; eps: the
   quench depth gamma of Eq. (GE).  dev_workspace: caller-owned device buffer
   of `bytes` >= pfc_workspace_size (256-byte aligned); cuda_stream: a
   cudaStream_t (NULL = legacy default stream).  phi^n starts at zero. */
int pfc_create(const pfc_grid* g, double h, double eps, const pfc_params* p, void* dev_workspace,
               size_t bytes, void* cuda_stream, pfc_state** out);
void pfc_destroy(pfc_state* s);

/* Sets phi^n = phi^{n-1} = phi (N values) and clears the energy history.
   on_device = 1: phi is a device pointer; 0: a host pointer. */
int pfc_set_field(pfc_state* s, const double* phi, int on_device);
/* Copies phi^n out (N values) to a device (on_device = 1) or host buffer. */
int pfc_get_field(pfc_state* s, double* out, int on_device);
/* Checkpoint and resume of the time stepping: pfc_save writes phi^n,
   phi^{n-1} and the adaptive-step history (energies of the last two steps,
   previous dt) with the grid, h and eps to the host file `path` (binary, host
   byte order); pfc_load restores them into a state created with the same grid,
   h and eps, so that the following steps equal those of the saved run.
   PFC_EINVAL on a file that cannot be written or read, a foreign or corrupt
   file, or a different grid / h / eps (pfc_load then changes nothing).  Not
   part of the paper's method. */
int pfc_save(pfc_state* s, const char* path);
int pfc_load(pfc_state* s, const char* path);

/* Caller-supplied Newton initial guess for the next pfc_step when
   params.guess == PFC_GUESS_USER (N values, device or host). */
int pfc_set_guess(pfc_state* s, const double* guess, int on_device);

/* One time step of size dt (Eq. NSOP solved by NKS, Sec. 4).  On success
   phi^{n-1} <- phi^n, phi^n <- phi^{n+1}.  info may be NULL. */
int pfc_step(pfc_state* s, double dt, pfc_step_info* info);

/* nsteps steps with dt from Eq. (sencondt); the first step of a fresh field
   uses dt_min.  per_step: caller-owned array of nsteps records, or NULL.
   Stops at the first failing step and returns its status. */
int pfc_run(pfc_state* s, int nsteps, pfc_step_info* per_step);

/* Batched form (independent runs, e.g. an ensemble of small grids): runs
   pfc_run(states[i], nsteps, ...) for every i.  When every state is 2D with the
   graph form on (use_graph), the phi^n guess, one device and streams of their
   own, each ensemble step is one CUDA graph launch: a graph captured once that
   holds every state's step graph as a parallel branch (each with its own dt,
   convergence and line search), so the states' kernels overlap on the GPU with
   no host work in between.  The first step of states that still have to tune
   their apply kernel, and every other case, run on one host thread per state.
   A state's failed step (PFC_ENEWTON, PFC_EGMRES) is retried alone with half the
   time step (dt_halvings), as in pfc_run; a state that fails for good is left
   unchanged by the later ensemble steps.  The paper runs one problem at a time;
   this entry point has no counterpart there.
   per_step: count x nsteps records (state i at per_step[i * nsteps + n]) or
   NULL; status: count ints or NULL.  Returns PFC_OK when every run succeeded,
   else the status of the lowest-numbered failing state.  No two entries may be
   the same state (PFC_EINVAL). */
int pfc_run_batch(pfc_state** states, int count, int nsteps, pfc_step_info* per_step, int* status);

/* F_d(phi^n) (Eq. freeenergy) and h^d sum phi^n. */
int pfc_energy(pfc_state* s, double* F);
int pfc_mass(pfc_state* s, double* m);

/* Test hooks on caller device arrays of N values (no state change):
   residual F(Phi) of Eq. (NSOP) for the given phi^n and dt; its 2-norm in
   *norm (may be NULL). */
int pfc_residual(pfc_state* s, const double* Phi, const double* phin, double dt, double* F_out,
                 double* norm);
/* J v = v/dt - Delta_d(L_gamma v / 2 + q v), q = (3 Phi^2 + 2 Phi phi^n + phi^n^2)/4 (Eq. Jacobi).
   On the 2D mixed path (F32/BF16 factors, M = 1) the product runs as GMRES takes it: v is
   copied into the state's first Krylov scratch vector and interior tiles stage v and q by TMA
   tensor copies; a staging wait that runs out returns PFC_ETIMEOUT.  The field and the time-step
   state are untouched. */
int pfc_jvp(pfc_state* s, const double* Phi, const double* phin, const double* v, double dt,
            double* Jv);
/* Builds the subdomain factors of J(Phi, phi^n, dt) (Eq. Ak, improved BC) and
   applies the Schwarz preconditioner (Eq. ras) to r: z = sum_k (R_k^0)^T A_k^{-1} R_k^delta r. */
int pfc_precond_apply(pfc_state* s, const double* Phi, const double* phin, double dt, const double* r,
                      double* z);

/* The time step Eq. (sencondt) gives from the state's energy history:
   max(dt_min, dt_max / sqrt(1 + eta F'^2)), F' = (E^n - E^{n-1}) / dt_{n-1}, E the
   energy (or the energy density when energy_scaled); dt_min on a fresh field.
   pfc_run uses exactly this value. */
int pfc_next_dt(pfc_state* s, double* dt);

/* One step through host buffers: copies phin_host (N values, pinned memory
   recommended) into phi^n keeping the energy history -- pass the field the
   previous step returned -- advances by dt as pfc_step does, and copies
   phi^{n+1} back into out_host.  The copies run on the state's stream. */
int pfc_step_host(pfc_state* s, const double* phin_host, double dt, double* out_host, pfc_step_info* info);

/* Kernel timing for roofline reports.  pfc_profile(s, 1) creates a pool of CUDA
   events and from then on brackets, with a pair of events on the state's
   stream, every executed launch of the kernel families below; pfc_profile(s, 0)
   releases them; both clear the sums.  While profiling is on, GMRES cycles run
   from the host loop (event records cannot sit inside the cycle graph).
   Families (index into the pfc_profile_kernels array):
     PFC_PROF_APPLY     Schwarz apply (Eq. ras), one per GMRES iteration
     PFC_PROF_JVP       Jacobian-vector product (Eq. Jacobi), one per GMRES iteration
     PFC_PROF_DOT       first Gram-Schmidt pass, multi-dot of V_0..V_j against w
     PFC_PROF_AXPY      first Gram-Schmidt pass, multi-axpy w -= sum c_i V_i
     PFC_PROF_FACTOR    subdomain factorisation (Eq. Ak), once per time step
     PFC_PROF_RESIDUAL  residual F (Eq. NSOP) with its norm and q
     PFC_PROF_RECORDS   2D chunked records of the factors (chunked apply only)
   Algorithmic work per launch: apply = the method's band factor entries (2D band
   LU with partial pivoting, kl = 3 bx multipliers and 2 kl U entries per step,
   shortened at the block's end; 3D: 63 ILU(0) entries per row) in the storage
   precision, 1-byte pivots, the gather of r over the block and the write of z
   on the core; JVP 24 bytes per point (v, q in, Jv out); multi-dot (j + 2) and
   multi-axpy (j + 3) vectors of 8 bytes per point at Arnoldi column j; residual
   3 vectors (+2 for a line-search trial point, +1 with q); factor: band factors
   written plus q read, and 2 r c + r flops per elimination step (r multipliers,
   c updated columns).  bytes_stored: what the kernels in use actually move
   (padded rows, chunk records, scratch passes). */
enum {
  PFC_PROF_APPLY = 0,
  PFC_PROF_JVP = 1,
  PFC_PROF_DOT = 2,
  PFC_PROF_AXPY = 3,
  PFC_PROF_FACTOR = 4,
  PFC_PROF_RESIDUAL = 5,
  PFC_PROF_RECORDS = 6,
  PFC_PROF_KINDS = 7
};
typedef struct {
  long long launches;   /* timed launches                                         */
  double ms;            /* summed device milliseconds between each launch's events */
  double bytes;         /* summed algorithmic bytes                               */
  double flops;         /* summed algorithmic floating-point operations           */
  double bytes_stored;  /* summed bytes of the storage format in use              */
} pfc_kernel_prof;
int pfc_profile(pfc_state* s, int enable);
/* Sums since profiling was enabled, one record per family for the first
   min(cap, PFC_PROF_KINDS) families (out may be NULL when cap is 0).
   Synchronises the state's stream when launches are still waiting. */
int pfc_profile_kernels(pfc_state* s, pfc_kernel_prof* out, int cap);
/* The apply family's launches and milliseconds, the algorithmic bytes of one
   apply, and the number of kernels this library launched in the process so
   far (all kinds, profiled or not). */
int pfc_profile_read(pfc_state* s, long long* apply_launches, double* apply_ms, double* apply_bytes,
                     long long* kernel_launches);

/* Process-wide counts: kernels this library has run (a graph step's kernels are
   counted from what its control kernels recorded) and CUDA graph launches (each a
   whole time step of one state, or one step of a whole ensemble). */
int pfc_launch_counts(long long* kernels, long long* graphs);

/* Autotuner report.  *apply_variant: the Schwarz apply kernel in use
   (pfc_params.apply_variant numbering; 3D: 0 or 1, fixed at pfc_create).  apply_ms (optional, 6 floats): the
   mean device milliseconds of one apply measured per kernel at the first
   factorisation, -1 for kernels not timed (not tuned yet, an explicit variant,
   or one that cannot run the blocks).  *graph (optional): 1 once GMRES cycles
   run as captured CUDA graphs (use_graph), 0 otherwise.  Not part of the
   paper's method. */
int pfc_get_tuning(const pfc_state* s, int* apply_variant, float* apply_ms, int* graph);

/* ---- Learned Newton initial guess (2D).  The paper starts Newton from phi^n
   (Sec. 4); the learned form adds a periodic 3x3 convolutional network
   (channels 3 -> 32 -> 32 -> 32 -> 1, GELU, BF16 weights and activations,
   FP32 accumulation) on the features
     c0 = phi^n - mean(phi^n), c1 = r (phi^n - phi^{n-1}), c2 = dt / dt_max,
   r = dt / dt_prev, and takes Phi_0 = phi^n + c1 + s_out * net(c), shifted to
   the mass of phi^n.  Parameters: one flat FP32 vector, layer by layer
   [W (Cout, Cin, 3, 3) row-major, b (Cout)].  Fields on device, planar. */
int pfc_cnn_param_count(void);
/* Workspace bytes of a network object for an nx x ny grid (activations,
   gradients, Adam state). */
int pfc_cnn_workspace_size(int64_t nx, int64_t ny, size_t* bytes);
int pfc_cnn_create(int64_t nx, int64_t ny, void* dev_workspace, size_t bytes, void* cuda_stream, pfc_cnn** out);
void pfc_cnn_destroy(pfc_cnn* c);
/* Host arrays of pfc_cnn_param_count() floats; set also clears the Adam moments. */
int pfc_cnn_set_params(pfc_cnn* c, const float* theta);
int pfc_cnn_get_params(pfc_cnn* c, float* theta);
/* out (N doubles) = net(feat), feat = 3 planes of N doubles. */
int pfc_cnn_forward(pfc_cnn* c, const double* feat, double* out);
/* Mean squared error against target (N doubles) and its gradient (host array
   of pfc_cnn_param_count() floats, may be NULL). */
int pfc_cnn_loss_grad(pfc_cnn* c, const double* feat, const double* target, double* loss, float* grad);
/* One Adam step (lr, step count t >= 1) on one sample; *loss (may be NULL) is
   the loss before the step. */
int pfc_cnn_train_step(pfc_cnn* c, const double* feat, const double* target, double lr, int t, double* loss);
/* One training sample from three consecutive fields of a trajectory (device
   arrays of N doubles): feat (3 x N) = the features above with r = dt / dt_prev
   and c2 = dt / dt_max, target (N) = (phi^{n+1} - phi^n - c1) / s_out. */
int pfc_cnn_sample(pfc_cnn* c, const double* phinm1, const double* phin, const double* phinp1, double r,
                   double c2, double s_out, double* feat, double* target);
/* Lets PFC_GUESS_LEARNED use network c (same grid as s; c stays owned by the
   caller and must outlive its use; during a step its forward pass runs on the
   state's stream, so c must not be used concurrently on another stream).  Each step compares the residual norms of
   the learned guess, the extrapolated guess and phi^n and starts Newton from
   the smallest. */
int pfc_set_guess_net(pfc_state* s, pfc_cnn* c, double s_out);

/* The 2D residual F(Phi) of pfc_residual, for callers that cannot allocate
   device memory at all: it needs no pfc_state and no workspace.  (The paper
   has no counterpart; this is a deployment convenience.)  The caller still
   passes the inputs Phi, phin and the output F_out (device arrays of
   Nx*Ny doubles) and the stream; *norm (may be NULL) receives ||F||_2.
   Its scratch -- one partial sum per 32x16 tile plus the total -- is a
   fixed array inside the library (65,536 tiles, 512 KiB, held on every GPU
   that loads the library until the process exits), so grids with more than
   65,536 tiles (more than 33,554,432 cells) are rejected with PFC_EINVAL.
   Every call looks up the array's address on the current device.  All calls
   share the one array: calls that overlap on the GPU (other streams, other
   threads) race and must be serialised by the caller.  The call synchronises
   its stream to return the norm, so it cannot be used inside a stream
   capture.  Errors: PFC_EINVAL for a grid or scalar pfc_create would refuse
   (dim != 2, n[2] != 1, h or eps not finite, h <= 0), dt <= 0 or not finite,
   null pointers, or too many tiles; PFC_ECUDA when a CUDA call fails. */
int pfc_residual_static(const pfc_grid* g, double h, double eps, const double* Phi, const double* phin,
                        double dt, double* F_out, double* norm, void* cuda_stream);

/* Failure-detection self-test of the bounded device-side wait that guards every
   mbarrier wait of the library's TMA copy rings (a wait gives up after a cycle
   limit, records PFC_ETIMEOUT and returns instead of hanging).  Launches one
   CTA on cuda_stream that initialises an mbarrier with one expected arrival,
   arrives on it when `arrive` is 1 (the wait then succeeds) or not at all (the
   phase never completes and the wait runs out), and waits with a limit of
   limit_cycles SM clock cycles (1 .. 4e9).  No copy is ever in flight, so the
   kernel always returns.  The outcome (PFC_OK or PFC_ETIMEOUT) is written to
   the caller's device int *dev_status and returned after the stream is
   synchronised.  Not part of the paper's method.  Errors: PFC_EINVAL for a null
   dev_status, arrive not 0/1 or a limit out of range; PFC_ECUDA. */
int pfc_wait_selftest(int arrive, long long limit_cycles, int* dev_status, void* cuda_stream);

/* Human-readable name of a status code (static string). */
const char* pfc_status_str(int status);

#ifdef __cplusplus
}
#endif
#endif /* PFC_H */
