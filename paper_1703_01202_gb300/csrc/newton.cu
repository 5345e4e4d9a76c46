// Device-side control of one time step: inexact Newton with a backtracking line
// search (Sec. 4, Eq. newton) around right-preconditioned restarted GMRES (Eq.
// hjacobi).  Each decision is a one-thread kernel on the step's StepCtl:
//   Newton stop test   ||F(Phi_m)|| <= max(eps_r ||F(Phi_0)||, eps_a)  (or eps_r ||F(phi^n)||
//                      when another initial guess was taken),
//   GMRES stop test    ||r|| <= max(xi_r ||F(Phi_m)||, xi_a), restarts, the iteration cap,
//   line search        Armijo test ||F(Phi + lam S)||^2 <= (1 - 2 alpha lam) ||F(Phi)||^2 with the
//                      quadratic-model step clamped to [0.1 lam, 0.5 lam], at most ls_max_cuts cuts.
// With graph = 1 a kernel also sets the conditional handle of the loop or branch it
// decides, so that a captured graph runs the whole step with no host round trip;
// with graph = 0 the host reads the same fields back and drives the loops.
#include <cmath>

#include "../../include/pfc.h"
#include "ff.cuh"
#include "pfc_internal.cuh"

namespace pfc {
namespace {

__device__ __forceinline__ void set_cond(cudaGraphConditionalHandle h, int graph, int v) {
  if (graph) cudaGraphSetConditional(h, v ? 1u : 0u);
}

__device__ __forceinline__ bool bad(double x) { return !(x == x) || isinf(x); }

__global__ void k_newton_begin(StepCtl* c, const double* nrm2, IterArgs* ia, IterArgs* ia2, StepHandles h,
                               int graph) {
  const double r0 = sqrt(*nrm2);
  c->r0 = r0;
  c->rnorm = r0;
  c->m = 0;
  c->gm_total = 0;
  c->cuts_total = 0;
  c->status = bad(r0) ? PFC_ENAN : PFC_OK;
  c->target = fmax(c->newton_rtol * (c->ref_norm >= 0.0 ? c->ref_norm : r0), c->newton_atol);
  ia->idt = c->idt;
  ia2->idt = c->idt;
  c->newton_go = c->status == PFC_OK && r0 > c->target && c->newton_max_it > 0;
  c->factor_go = c->refactor;
  c->commit_go = 0;
  c->n_factor = c->n_cycles = c->n_restarts = c->n_trials = c->n_reorth = 0;
  set_cond(h.newton, graph, c->newton_go);
}

__global__ void k_set_factor_cond(StepCtl* c, StepHandles h, int graph) { set_cond(h.factor, graph, c->factor_go); }

__global__ void k_factor_done(StepCtl* c) {
  c->factor_go = 0;
  c->n_factor += 1;
}

// GMRES for J S = -F from S = 0: V_0 = -F / ||F|| (the basis vector is stored as F, scaled by -1/beta).
__global__ void k_gmres_begin(StepCtl* c, GmresCtl* g, StepHandles h, int graph) {
  const double tol = fmax(c->gmres_rtol * c->rnorm, c->gmres_atol);
  const double beta = c->rnorm;
  c->gtol = tol;
  c->gm_its = 0;
  g->done = 0;
  g->its = 0;
  g->reorth = 0;
  g->breakdown = 0;
  g->n_reorth = 0;
  g->tol = tol;
  g->reorth_eta2 = c->reorth_eta2;
  g->beta = beta;
  g->est = beta;
  g->g[0] = beta;
  g->scale[0] = beta > 0.0 ? -1.0 / beta : 0.0;
  if (!(beta > tol)) g->done = 1;
  c->cycle_go = !g->done;
  c->restart_go = 0;
  set_cond(h.cycle, graph, c->cycle_go);
}

// After a cycle (its iterations, S updated): converged, failed, or restart.
__global__ void k_cycle_decide(StepCtl* c, GmresCtl* g, StepHandles h, int graph) {
  c->gm_its += g->its;
  c->n_reorth += g->n_reorth;
  const double est = g->est;
  int go = 0;
  if (!(est == est)) {
    c->status = PFC_ENAN;
  } else if (est <= g->tol || g->breakdown) {
    go = 0;
  } else if (c->gm_its >= c->gmres_max_it) {
    c->status = PFC_EGMRES;
  } else {
    go = 1;
  }
  c->cycle_go = go;
  c->restart_go = go;
  c->n_cycles += 1;
  c->n_restarts += go;
  set_cond(h.cycle, graph, go);
  set_cond(h.restart, graph, go);
}

// Restart: r = -F - J S has been formed with ||r||^2 in *nrm2; V_0 = r / ||r||.
__global__ void k_gmres_restart(StepCtl* c, GmresCtl* g, const double* nrm2) {
  const double beta = sqrt(*nrm2);
  g->done = 0;
  g->its = 0;
  g->reorth = 0;
  g->breakdown = 0;
  g->n_reorth = 0;
  g->tol = c->gtol;
  g->reorth_eta2 = c->reorth_eta2;
  g->beta = beta;
  g->est = beta;
  g->g[0] = beta;
  g->scale[0] = beta > 0.0 ? 1.0 / beta : 0.0;
  if (!(beta > c->gtol)) g->done = 1;
}

// After GMRES: fold in the device-side error flags of the factorisation (zero pivot) and of
// the bounded waits, then start the line search at lam = 1.
__global__ void k_gmres_end(StepCtl* c, const int* status_dev, StepHandles h, int graph) {
  c->gm_total += c->gm_its;
  if (c->status == PFC_OK && status_dev[0]) c->status = status_dev[0];
  if (c->status == PFC_OK && status_dev[1]) c->status = status_dev[1];
  c->lam = 1.0;
  c->cut = 0;
  c->f0 = 0.5 * c->rnorm * c->rnorm;
  c->ls_go = c->status == PFC_OK;
  set_cond(h.ls, graph, c->ls_go);
}

// One line-search trial evaluated (||F(Phi + lam S)||^2 in *nrm2): accept or cut.
__global__ void k_ls_decide(StepCtl* c, const double* nrm2, StepHandles h, int graph) {
  const double ft = 0.5 * *nrm2;
  const double lam = c->lam, f0 = c->f0;
  c->ft = ft;
  c->n_trials += 1;
  int go = 0;
  if (bad(ft)) {
    c->status = PFC_ENAN;
  } else if (!(ft <= (1.0 - 2.0 * c->ls_alpha * lam) * f0 || c->cut == c->ls_max_cuts)) {
    const double lq = lam * lam * f0 / (ft - f0 + 2.0 * lam * f0);
    c->lam = fmin(fmax(lq, 0.1 * lam), 0.5 * lam);
    c->cut += 1;
    c->cuts_total += 1;
    go = 1;
  }
  c->ls_go = go;
  set_cond(h.ls, graph, go);
}

__global__ void k_copy_if_ok(const StepCtl* c, CopyPairs cp, long long n) {
  if (c->status != PFC_OK) return;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (int k = 0; k < cp.n; ++k) {
    if ((cp.to_pairs >> k) & 1u) {
      for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += stride)
        st_pair(cp.dst[k], i, ff_pair_of(cp.src[k][i]));
      continue;
    }
    const double2* __restrict__ s = reinterpret_cast<const double2*>(cp.src[k]);
    double2* __restrict__ d = reinterpret_cast<double2*>(cp.dst[k]);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n / 2; i += stride) d[i] = s[i];
    if ((n & 1) && blockIdx.x == 0 && threadIdx.x == 0) cp.dst[k][n - 1] = cp.src[k][n - 1];
  }
}

__global__ void k_gmres_prep(double* __restrict__ S, double* __restrict__ red2, const double* __restrict__ F,
                             double* __restrict__ V0, long long n, int pairs) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += stride) {
    S[i] = 0.0;
    if (pairs)
      st_pair(V0, i, ff_pair_of(F[i]));
    else
      V0[i] = F[i];
  }
  if (blockIdx.x == 0 && threadIdx.x < 2) red2[threadIdx.x] = 0.0;
}

__global__ void k_newton_next(StepCtl* c, StepHandles h, int graph) {
  if (c->status == PFC_OK) {
    c->rnorm = sqrt(2.0 * c->ft);
    c->m += 1;
  }
  c->newton_go = c->status == PFC_OK && c->rnorm > c->target && c->m < c->newton_max_it;
  set_cond(h.newton, graph, c->newton_go);
}

__global__ void k_step_end(StepCtl* c, StepHandles h, int graph) {
  if (c->status == PFC_OK && c->rnorm > c->target) c->status = PFC_ENEWTON;
  c->commit_go = c->status == PFC_OK;
  set_cond(h.commit, graph, c->commit_go);
}

__global__ void k_mloop_begin(StepCtl* c, StepHandles h) {
  c->loop_go = c->steps_done < c->steps_target && !c->failed;
  c->cuts = 0;
  c->dt = controller_dt(c->E_n, c->E_nm1, c->dt_prev, c->escale, c->dt_min, c->dt_max, c->eta,
                        c->have_Em1 && c->have_prev_dt);
  cudaGraphSetConditional(h.mloop, c->loop_go ? 1u : 0u);
}

__global__ void k_mstep_prep(StepCtl* c) {
  c->idt = 1.0 / c->dt;
  c->refactor = 1;
}

// After one attempt of a step (the graph step's status in c): keep it and go on, retry with
// dt / 2 (Newton or GMRES failed and halvings remain), or stop the loop with the failure.
__global__ void k_mstep_end(StepCtl* c, const double* red45, pfc_step_info* rec, StepHandles h) {
  // kernels of the attempt (as the host counts a graph step) and this loop's own two per attempt
  c->kernels += 2 + 4 + (c->commit_go ? 3 : 0) + 6LL * c->m + (long long)c->n_factor * (2 + c->chunked) +
                4LL * c->n_cycles + 5LL * c->n_restarts + 3LL * c->n_trials + (long long)c->gm_total * c->body_kernels +
                2LL * c->n_reorth;
  const int st = c->status;
  if ((st == PFC_ENEWTON || st == PFC_EGMRES) && c->cuts < c->dt_halvings) {
    c->dt *= 0.5;
    c->cuts += 1;
  } else {
    pfc_step_info& r = rec[c->steps_done];
    r.status = st;
    r.newton_its = c->m;
    r.gmres_its = c->gm_total;
    r.ls_cuts = c->cuts_total;
    r.dt = c->dt;
    r.res_norm0 = c->r0;
    r.res_norm = c->rnorm;
    r.guess_used = PFC_GUESS_PREV;
    r.dt_cuts = c->cuts;
    r.energy = 0.0;
    r.mass = 0.0;
    if (st == PFC_OK) {
      const double E = red45[0] * c->hd;
      r.energy = E;
      r.mass = red45[1] * c->hd;
      c->E_nm1 = c->E_n;
      c->E_n = E;
      c->have_Em1 = 1;
      c->dt_prev = c->dt;
      c->have_prev_dt = 1;
      c->steps_done += 1;
      c->cuts = 0;
      c->dt = controller_dt(c->E_n, c->E_nm1, c->dt_prev, c->escale, c->dt_min, c->dt_max, c->eta, true);
    } else {
      c->failed = st;
    }
  }
  c->loop_go = c->steps_done < c->steps_target && !c->failed;
  cudaGraphSetConditional(h.mloop, c->loop_go ? 1u : 0u);
}

}  // namespace

void launch_mloop_begin(StepCtl* c, const StepHandles& h, cudaStream_t st) {
  k_mloop_begin<<<1, 1, 0, st>>>(c, h);
  count_launches(1);
}
void launch_mstep_prep(StepCtl* c, cudaStream_t st) {
  k_mstep_prep<<<1, 1, 0, st>>>(c);
  count_launches(1);
}
void launch_mstep_end(StepCtl* c, const double* red45, void* rec, const StepHandles& h, cudaStream_t st) {
  k_mstep_end<<<1, 1, 0, st>>>(c, red45, static_cast<pfc_step_info*>(rec), h);
  count_launches(1);
}

void launch_newton_begin(StepCtl* c, const double* nrm2, IterArgs* ia, IterArgs* ia2, const StepHandles& h,
                         int graph, cudaStream_t st) {
  k_newton_begin<<<1, 1, 0, st>>>(c, nrm2, ia, ia2, h, graph);
  count_launches(1);
}
void launch_set_factor_cond(StepCtl* c, const StepHandles& h, int graph, cudaStream_t st) {
  k_set_factor_cond<<<1, 1, 0, st>>>(c, h, graph);
  count_launches(1);
}
void launch_factor_done(StepCtl* c, cudaStream_t st) {
  k_factor_done<<<1, 1, 0, st>>>(c);
  count_launches(1);
}
void launch_gmres_begin(StepCtl* c, GmresCtl* g, const StepHandles& h, int graph, cudaStream_t st) {
  k_gmres_begin<<<1, 1, 0, st>>>(c, g, h, graph);
  count_launches(1);
}
void launch_cycle_decide(StepCtl* c, GmresCtl* g, const StepHandles& h, int graph, cudaStream_t st) {
  k_cycle_decide<<<1, 1, 0, st>>>(c, g, h, graph);
  count_launches(1);
}
void launch_gmres_restart(StepCtl* c, GmresCtl* g, const double* nrm2, cudaStream_t st) {
  k_gmres_restart<<<1, 1, 0, st>>>(c, g, nrm2);
  count_launches(1);
}
void launch_gmres_end(StepCtl* c, const int* status_dev, const StepHandles& h, int graph, cudaStream_t st) {
  k_gmres_end<<<1, 1, 0, st>>>(c, status_dev, h, graph);
  count_launches(1);
}
void launch_ls_decide(StepCtl* c, const double* nrm2, const StepHandles& h, int graph, cudaStream_t st) {
  k_ls_decide<<<1, 1, 0, st>>>(c, nrm2, h, graph);
  count_launches(1);
}
void launch_copy_if_ok(const StepCtl* c, const CopyPairs& cp, long long n, cudaStream_t st) {
  const long long b = (n / 2 + 255) / 256;
  k_copy_if_ok<<<(int)(b < kRedCtas ? (b < 1 ? 1 : b) : kRedCtas), 256, 0, st>>>(c, cp, n);
  count_launches(1);
}
void launch_gmres_prep(double* S, double* red2, const double* F, double* V0, long long n, cudaStream_t st,
                       bool pairs) {
  const long long b = (n + 255) / 256;
  k_gmres_prep<<<(int)(b < kRedCtas ? (b < 1 ? 1 : b) : kRedCtas), 256, 0, st>>>(S, red2, F, V0, n, pairs ? 1 : 0);
  count_launches(1);
}
void launch_newton_next(StepCtl* c, const StepHandles& h, int graph, cudaStream_t st) {
  k_newton_next<<<1, 1, 0, st>>>(c, h, graph);
  count_launches(1);
}
void launch_step_end(StepCtl* c, const StepHandles& h, int graph, cudaStream_t st) {
  k_step_end<<<1, 1, 0, st>>>(c, h, graph);
  count_launches(1);
}

}  // namespace pfc
