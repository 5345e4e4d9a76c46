// C ABI of libpfc (include/pfc.h): state, workspace layout and the host-side
// control of one time step -- inexact Newton with backtracking line search
// (Sec. 4, Eq. newton), right-preconditioned restarted GMRES (Eq. hjacobi)
// whose Arnoldi bookkeeping lives on the device, the left-RAS preconditioner
// with factors built once per step and reused by every Newton iteration
// (Sec. 5.2), and the adaptive time step of Eq. (sencondt).
//
// Every numeric step runs in the CUDA kernels of this library; the host only
// sequences launches on the caller's stream and reads back a few scalars
// (residual norms, GMRES iteration counts) to take the Newton and GMRES
// decisions.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <thread>
#include <utility>
#include <vector>

#include "../../include/pfc.h"
#include "pfc_internal.cuh"

using pfc::BlockDesc;
using pfc::Geo;
using pfc::GmresCtl;
using pfc::VecList;

// One timed launch waiting for its events: its family, its Arnoldi column (-1: not part of a
// GMRES cycle) and its algorithmic work.
struct ProfPair {
  int kind, j;
  double bytes, flops, stored;
};
constexpr int kProfSlots = 256;

struct pfc_state {
  pfc_grid grid;
  pfc_params p;
  Geo g;
  double h, gamma;
  cudaStream_t st;
  int dim;
  // fields (device, N doubles each)
  double *phin, *phinm1, *Phi, *F, *q, *Pt, *Ft, *qt, *S, *W, *guess;
  double *Vbuf, *Zbuf;  // (m+1) and m vectors of vstride doubles
  size_t vstride;       // N rounded up to 32 doubles: every basis vector starts 256-byte aligned
  const double** vtab;  // device pointer tables: vtab[i] = Vbuf + i vstride, ztab[i] = Zbuf + i vstride
  const double** ztab;
  // preconditioner
  BlockDesc* blocks_dev;
  int nblocks;
  pfc::FactorStore fs;
  pfc::JvpMaps jmaps{};  // TMA maps of the basis Z and of q for the mixed path's JVP
  pfc::Decomp2 dc;  // 2D decomposition (AS / right-RAS overlap sums)
  // variable mobility: mu and s = (Phi + phi^n)/2 at the iterate of q (mu, sm) and of the trial q (mut, smt)
  double *mu = nullptr, *mut = nullptr, *sm = nullptr, *smt = nullptr;
  // factors kept across steps (reuse_factor): valid, the dt they were made with, steps reused since
  bool factors_ok = false;
  double factor_dt = 0.0;
  int factor_age = 0;
  double* lin_dev;
  // 3D: scratch fields of the three-pass stencils and the ILU(0) Schwarz data
  double *T1, *T2;
  pfc::Ras3D r3;
  // learned initial guess
  pfc_cnn* cnn;
  double s_out;
  double* feat;  // 3 x N feature planes
  // reductions and control
  GmresCtl* ctl;
  double* partial;
  double* red;   // device scalars: [0..7] general, [8..15] axpy reductions
  int* status_dev;
  // host mirrors (pinned)
  GmresCtl* ctl_h;
  // host loop: control-block heads read back after every chunk of iterations, two in flight
  GmresCtl* ctl_hb[2];
  cudaEvent_t ctl_ev[2];
  double* red_h;
  int* status_h;
  // history for the adaptive step and the extrapolated guess
  bool have_E, have_Em1, have_prev_dt, have_user_guess;
  double E_n, E_nm1, dt_prev;
  // kernel timing (pfc_profile): a pool of event pairs bracketing launches, resolved at
  // synchronisation points into per-family sums
  bool prof;
  std::vector<cudaEvent_t> pev;  // 2 per slot
  std::vector<ProfPair> ppend;   // slots in use, in record order
  pfc_kernel_prof pk[PFC_PROF_KINDS];
  double apply_bytes;        // the method's band factors + gather + core write (one apply)
  double apply_bytes_step;   // what the per-step apply kernels (variants 0-4) read and write
  double apply_bytes_chunk;  // what the chunked apply (variant 5) reads and writes
  double factor_flops;       // one factorisation of every block (band LU with partial pivoting)
  double factor_bytes;       // its band factors written + q read
  double record_bytes;       // one chunk-record build: factors read + records written
  // apply kernel picked by timing at the first 2D factorisation (apply_variant = -1)
  bool tuned;
  float tune_ms[pfc::kApplyVariants];
  // ||F(phi^n)|| of the current step when a safeguarded guess was chosen (< 0: none)
  double ref_norm;
  int device;  // CUDA device current at pfc_create
  // device-side control of a step and its graph form (2D): the whole step captured once
  pfc::StepCtl* sc;     // device
  pfc::StepCtl* sc_h;   // pinned host mirror
  pfc::IterArgs* ia;    // Arnoldi iteration arguments (device): vectors of iteration j, q, 1/dt
  pfc::IterArgs* ia2;   // the restart's J S -> W with this step's 1/dt (device)
  pfc::StepHandles hs;  // conditional handles of the step graph
  cudaStream_t cs[5];   // capture streams of the nested bodies (graph form; one more level in a batch graph)
  pfc_step_info* recs;  // device records of the batch form's time loop (kBatchRecs)
  cudaGraph_t sgraph;
  cudaGraphExec_t sexec;
  bool graph_failed;    // capture or instantiation failed once: keep the host-driven step
};

namespace pfc {
namespace {
long long g_launches = 0;        // host-side count; launches come from the calling thread
thread_local bool g_paused = false;  // this thread is capturing a graph (nothing runs)
}
void count_launches(long long n) {
  if (!g_paused) __atomic_add_fetch(&g_launches, n, __ATOMIC_RELAXED);
}
void count_pause(bool on) { g_paused = on; }
long long g_graph_launches = 0;  // graph launches (each a whole time step, or a whole ensemble step)
void count_graph_launch() { __atomic_add_fetch(&g_graph_launches, 1, __ATOMIC_RELAXED); }
long long launches_so_far() { return __atomic_load_n(&g_launches, __ATOMIC_RELAXED); }
}  // namespace pfc

namespace {

#define CU(call)                                         \
  do {                                                   \
    cudaError_t e_ = (call);                             \
    if (e_ != cudaSuccess) {                             \
      fprintf(stderr, "libpfc: %s failed: %s (%s:%d)\n", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
      return PFC_ECUDA;                                  \
    }                                                    \
  } while (0)

struct Layout {
  size_t total = 0;
  size_t take(size_t bytes) {
    size_t off = total;
    total += (bytes + 255) & ~(size_t)255;
    return off;
  }
};

struct Split {
  int start, size;
};

std::vector<Split> split_axis(int n, int p) {
  std::vector<Split> out;
  const int base = n / p, extra = n % p;
  int s = 0;
  for (int r = 0; r < p; ++r) {
    const int sz = base + (r < extra ? 1 : 0);
    out.push_back({s, sz});
    s += sz;
  }
  return out;
}

int validate(const pfc_grid* g, const pfc_params* p) {
  if (!g || !p) return PFC_EINVAL;
  if (g->dim != 2 && g->dim != 3) return PFC_EINVAL;
  for (int a = 0; a < g->dim; ++a)
    if (g->n[a] < 1 || g->n[a] > (1 << 20)) return PFC_EINVAL;
  if (g->dim == 2 && g->n[2] != 1) return PFC_EINVAL;
  if (p->gmres_restart < 1 || p->gmres_restart > pfc::kMaxRestart) return PFC_EINVAL;
  if (p->newton_max_it < 0 || p->gmres_max_it < 1 || p->overlap < 0) return PFC_EINVAL;
  // left-RAS everywhere; AS and right-RAS (full-block extension) on 2D grids, with the chunked apply
  if (p->ras_kind != PFC_LEFT_RAS && p->ras_kind != PFC_AS && p->ras_kind != PFC_RIGHT_RAS) return PFC_EINVAL;
  if (p->ras_kind != PFC_LEFT_RAS && (g->dim != 2 || (p->apply_variant != -1 && p->apply_variant != 5)))
    return PFC_EINVAL;
  if (p->factor_prec < PFC_F64 || p->factor_prec > PFC_BF16) return PFC_EINVAL;
  if (p->apply_variant < -1 || p->apply_variant >= pfc::kApplyVariants) return PFC_EINVAL;
  if (g->dim == 3 && p->apply_variant > 1) return PFC_EINVAL;
  if (p->dt_halvings < 0 || p->dt_halvings > 30) return PFC_EINVAL;
  if (!(p->gmres_reorth_eta >= 0.0 && p->gmres_reorth_eta < 1.0)) return PFC_EINVAL;
  if (p->use_graph != 0 && p->use_graph != 1) return PFC_EINVAL;
  if (p->gmres_fast_dots != 0 && p->gmres_fast_dots != 1) return PFC_EINVAL;
  if (p->jvp_fp32 != 0 && p->jvp_fp32 != 1) return PFC_EINVAL;
  if (p->reuse_factor < 0 || p->reuse_factor > 1000000) return PFC_EINVAL;
  if (p->mobility != 0 && p->mobility != 1) return PFC_EINVAL;
  // Neumann walls: left-RAS, M = 1, at least 4 cells per axis (the radius-3 stencils then never
  // see a second mirror image)
  if (p->boundary != PFC_PERIODIC &&
      (p->boundary != PFC_NEUMANN || p->ras_kind != PFC_LEFT_RAS || p->mobility != 0 || g->n[0] < 4 ||
       g->n[1] < 4 || (g->dim == 3 && g->n[2] < 4)))
    return PFC_EINVAL;
  for (int a = 0; a < g->dim; ++a) {
    if (p->sub[a] < 1 || p->sub[a] > g->n[a]) return PFC_EINVAL;
    const int core_max = (int)((g->n[a] + p->sub[a] - 1) / p->sub[a]);
    const int core_min = (int)(g->n[a] / p->sub[a]);
    // a periodic block must not reach its own image (3D blocks between walls are clipped instead)
    if (core_max + 2 * p->overlap > g->n[a] && !(g->dim == 3 && p->boundary == PFC_NEUMANN)) return PFC_EINVAL;
    if (g->dim == 3) {
      // 3D blocks: at least 7 cells per axis (offset order = row order); periodic blocks plus their
      // 3-cell ring must not wrap onto themselves (A_k = R J R^T pattern); between walls a block at
      // a wall has one overlap (or none, when one block spans the axis)
      const int ext_min = p->boundary == PFC_NEUMANN ? (p->sub[a] == 1 ? (int)g->n[a] : core_min + p->overlap)
                                                     : core_min + 2 * p->overlap;
      if (ext_min < 7) return PFC_EINVAL;
      if (p->boundary != PFC_NEUMANN && core_max + 2 * p->overlap + 3 > g->n[a]) return PFC_EINVAL;
      if (core_max + 2 * p->overlap > 1023) return PFC_EINVAL;  // row cells packed in 10 bits per axis
    }
  }
  return PFC_OK;
}

void build_blocks(const pfc_grid* g, const pfc_params* p, std::vector<BlockDesc>* out, int* n_max, int* kl_max) {
  auto sx = split_axis((int)g->n[0], p->sub[0]);
  auto sy = split_axis((int)g->n[1], p->sub[1]);
  const int nz_parts = g->dim == 3 ? p->sub[2] : 1;
  auto sz = split_axis(g->dim == 3 ? (int)g->n[2] : 1, nz_parts);
  const int ov = p->overlap;
  const int ovz = g->dim == 3 ? ov : 0;
  *n_max = 0;
  *kl_max = 0;
  for (int bz = 0; bz < nz_parts; ++bz)
    for (int by = 0; by < p->sub[1]; ++by)
      for (int bx = 0; bx < p->sub[0]; ++bx) {
        BlockDesc b{};
        b.x0 = sx[bx].start - ov;
        b.y0 = sy[by].start - ov;
        b.z0 = sz[bz].start - ovz;
        b.bx = sx[bx].size + 2 * ov;
        b.by = sy[by].size + 2 * ov;
        b.bz = sz[bz].size + 2 * ovz;
        b.ox = ov;
        b.oy = ov;
        b.oz = ovz;
        b.cx = sx[bx].size;
        b.cy = sy[by].size;
        b.cz = sz[bz].size;
        if (p->boundary == PFC_NEUMANN) {  // the overlap stops at the walls: blocks are clipped
          const int x1 = std::min((int)g->n[0], b.x0 + b.bx), y1 = std::min((int)g->n[1], b.y0 + b.by);
          b.x0 = std::max(0, b.x0);
          b.y0 = std::max(0, b.y0);
          b.bx = x1 - b.x0;
          b.by = y1 - b.y0;
          b.ox = sx[bx].start - b.x0;
          b.oy = sy[by].start - b.y0;
          if (g->dim == 3) {
            const int z1 = std::min((int)g->n[2], b.z0 + b.bz);
            b.z0 = std::max(0, b.z0);
            b.bz = z1 - b.z0;
            b.oz = sz[bz].start - b.z0;
          }
        }
        out->push_back(b);
        const int n = b.bx * b.by * b.bz;
        const int kl = std::min(3 * b.bx, n - 1);
        *n_max = std::max(*n_max, n);
        *kl_max = std::max(*kl_max, kl);
      }
}

// 3D shape tables: one entry per distinct block extent.
struct Shapes3 {
  std::vector<pfc::Shape3> shapes;
  std::vector<int> block_shape, lev_start, rowpad, rowabc;
  // per row, in each level's 16-bytes-per-row layout: the place of each lower (posL) / upper
  // (posU) neighbour in its own level's row list, 255 where the neighbour is outside the block
  std::vector<uint8_t> posL, posU;
  int nrows_max = 0, pad_max = 0, max_level_rows = 0;
};

void offsets63(int off[63][3]) {
  int idx = 0;
  for (int c = -3; c <= 3; ++c)
    for (int b = -3; b <= 3; ++b)
      for (int a = -3; a <= 3; ++a)
        if (std::abs(a) + std::abs(b) + std::abs(c) <= 3) {
          off[idx][0] = a;
          off[idx][1] = b;
          off[idx][2] = c;
          ++idx;
        }
}

void build_shapes3(const std::vector<BlockDesc>& blocks, Shapes3* S) {
  int off[63][3];
  offsets63(off);
  for (const BlockDesc& b : blocks) {
    int found = -1;
    for (size_t i = 0; i < S->shapes.size(); ++i)
      if (S->shapes[i].bx == b.bx && S->shapes[i].by == b.by && S->shapes[i].bz == b.bz) found = (int)i;
    if (found < 0) {
      pfc::Shape3 sh{};
      sh.bx = b.bx;
      sh.by = b.by;
      sh.bz = b.bz;
      sh.px = b.bx + 6;
      sh.py = b.by + 6;
      sh.pz = b.bz + 6;
      sh.nrows = b.bx * b.by * b.bz;
      sh.nlev = (b.bx - 1) + 3 * (b.by - 1) + 7 * (b.bz - 1) + 1;
      sh.lev_off = (int)S->lev_start.size();
      sh.row_off = (int)S->rowpad.size();
      for (int o = 0; o < 63; ++o) sh.poff[o] = off[o][0] + sh.px * (off[o][1] + sh.py * off[o][2]);
      // rows in level order, ascending linear index inside a level
      std::vector<std::vector<int>> bylev(sh.nlev);
      for (int c = 0; c < b.bz; ++c)
        for (int bb = 0; bb < b.by; ++bb)
          for (int a = 0; a < b.bx; ++a) bylev[a + 3 * bb + 7 * c].push_back(a + b.bx * (bb + b.by * c));
      int r = 0;
      for (int l = 0; l < sh.nlev; ++l) {
        S->lev_start.push_back(r);
        S->max_level_rows = std::max(S->max_level_rows, (int)bylev[l].size());
        for (int li : bylev[l]) {
          const int a = li % b.bx, bb = (li / b.bx) % b.by, c = li / (b.bx * b.by);
          const int pp = (a + 3) + sh.px * ((bb + 3) + sh.py * (c + 3));
          S->rowpad.push_back(pp);
          S->rowabc.push_back(a | (bb << 10) | (c << 20));
          ++r;
        }
      }
      S->lev_start.push_back(r);
      {  // neighbour places for the compact-window apply (levels of at most 255 rows)
        const int r0s = sh.row_off;
        std::vector<int> place(sh.nrows);
        std::vector<int> rowof_cell((size_t)sh.nrows);
        for (int l = 0; l < sh.nlev; ++l)
          for (int rr = S->lev_start[sh.lev_off + l]; rr < S->lev_start[sh.lev_off + l + 1]; ++rr) {
            place[rr] = rr - S->lev_start[sh.lev_off + l];
            const int v = S->rowabc[r0s + rr];
            rowof_cell[(v & 1023) + b.bx * (((v >> 10) & 1023) + b.by * (v >> 20))] = rr;
          }
        S->posL.resize((size_t)(r0s + sh.nrows) * 32, 255);
        S->posU.resize((size_t)(r0s + sh.nrows) * 32, 255);
        for (int l = 0; l < sh.nlev; ++l) {
          const int l0 = S->lev_start[sh.lev_off + l], n = S->lev_start[sh.lev_off + l + 1] - l0;
          for (int i = 0; i < n; ++i) {
            const int v = S->rowabc[r0s + l0 + i];
            const int a = v & 1023, bb = (v >> 10) & 1023, c = v >> 20;
            for (int e = 0; e < 32; ++e) {
              const size_t at = (size_t)(r0s + l0) * 32 + (size_t)((e / 16) * n + i) * 16 + e % 16;
              for (int pass = 0; pass < 2; ++pass) {
                const int o = pass == 0 ? e : 31 + e;  // lower offset e (e < 31) / upper offset 31 + e (e >= 1)
                if ((pass == 0 && e >= 31) || (pass == 1 && e < 1)) continue;
                const int a2 = a + off[o][0], b2 = bb + off[o][1], c2 = c + off[o][2];
                uint8_t pl = 255;
                if (a2 >= 0 && a2 < b.bx && b2 >= 0 && b2 < b.by && c2 >= 0 && c2 < b.bz) {
                  const int r2 = rowof_cell[a2 + b.bx * (b2 + b.by * c2)];
                  if (place[r2] < 255) pl = (uint8_t)place[r2];
                }
                (pass == 0 ? S->posL : S->posU)[at] = pl;
              }
            }
          }
        }
      }
      S->nrows_max = std::max(S->nrows_max, sh.nrows);
      S->pad_max = std::max(S->pad_max, sh.px * sh.py * sh.pz);
      found = (int)S->shapes.size();
      S->shapes.push_back(sh);
    }
    S->block_shape.push_back(found);
  }
}

// ILU(0) update lists: for lower offset o1 and upper offset o2 of row k = i + o1,
// the entry o3 = o1 + o2 of row i when |o3|_1 <= 3.
void update_lists(std::vector<int>* upd, std::vector<int>* upd_n) {
  int off[63][3];
  offsets63(off);
  upd->assign(31 * 32, 0);
  upd_n->assign(32, 0);
  for (int o1 = 0; o1 < 31; ++o1) {
    int cnt = 0;
    for (int o2 = 32; o2 < 63; ++o2) {
      const int a = off[o1][0] + off[o2][0], b = off[o1][1] + off[o2][1], c = off[o1][2] + off[o2][2];
      if (std::abs(a) + std::abs(b) + std::abs(c) > 3) continue;
      int o3 = -1;
      for (int t = 0; t < 63; ++t)
        if (off[t][0] == a && off[t][1] == b && off[t][2] == c) o3 = t;
      (*upd)[o1 * 32 + cnt] = o2 | (o3 << 8);
      ++cnt;
    }
    (*upd_n)[o1] = cnt;
  }
}

// Doubles between consecutive Krylov basis vectors: N rounded up to 32 (every vector
// 256-byte aligned, for 16-byte loads and bulk copies) plus 17 x 256 bytes, so that
// the vectors of a power-of-two grid do not all start at the same offset modulo a
// large power of two (the Gram-Schmidt sweeps read all of them at the same offsets).
size_t basis_stride(long long N) { return ((size_t)N + 31) / 32 * 32 + 17 * 32; }

// Steps the batch form's device time loop runs per graph launch (records kept on the device).
constexpr int kBatchRecs = 64;

struct Plan {
  size_t phin, phinm1, Phi, F, q, Pt, Ft, qt, S, W, guess, V, Z, L, U, piv, blocks, lin, ctl, partial, red, status,
      tabs, feat, iargs, iargs2, sctl, recs, order, X, Yb, mu, mut, smid, smidt;
  // 3D
  size_t T1, T2, shapes, block_shape, lev_start, rowpad, rowabc, posL, posU, Lp, Up, work, ypad;
  size_t total;
  int nblocks, n_max, kl_max;
  size_t sL, sU, sP;
  int lrow, ucol;
  size_t xfw, xbw;  // strides of the chunked forward / backward records (2D)
  int xnc;          // chunks of the largest block
  int xstage;       // bytes of the largest chunked record
  size_t partial_len;
  Shapes3 sh3;
  size_t sLU3, sWork3, sPad3;
};

int make_plan(const pfc_grid* g, const pfc_params* p, Plan* pl) {
  int rc = validate(g, p);
  if (rc) return rc;
  const bool d3 = g->dim == 3;
  const long long N = g->n[0] * g->n[1] * (d3 ? g->n[2] : 1);
  std::vector<BlockDesc> blocks;
  build_blocks(g, p, &blocks, &pl->n_max, &pl->kl_max);
  pl->nblocks = (int)blocks.size();
  const size_t es = p->factor_prec == PFC_F64 ? 8 : (p->factor_prec == PFC_F32 ? 4 : 2);
  const size_t tc = p->factor_prec == PFC_F64 ? 8 : 4;
  if (!d3) {
    // rows of L and columns of U padded to 8 elements: every block, row and chunk
    // of rows starts on a 16-byte boundary and spans a multiple of 16 bytes (bulk copies)
    pl->lrow = (pl->kl_max + 7) / 8 * 8;
    pl->ucol = (2 * pl->kl_max + 1 + 7) / 8 * 8;
    pl->sL = (size_t)pl->n_max * pl->lrow;
    pl->sU = (size_t)pl->n_max * pl->ucol;
    pl->sP = ((size_t)pl->n_max + 15) / 16 * 16;
    pl->xfw = pl->xbw = 0;
    pl->xnc = 0;
    for (const BlockDesc& b : blocks) {
      const pfc::ChunkGeom cg = pfc::chunk_geom(b.bx, b.by, (int)es, (int)tc);
      pl->xfw = std::max(pl->xfw, cg.fwd);
      pl->xbw = std::max(pl->xbw, cg.bwd);
      pl->xnc = std::max(pl->xnc, cg.nc);
    }
    pl->xstage = (int)std::max(pl->xfw, pl->xbw);
  } else {
    pl->lrow = pl->ucol = 0;
    pl->sL = pl->sU = pl->sP = 0;
    pl->xfw = pl->xbw = 0;
    pl->xnc = 0;
    pl->xstage = 0;
    build_shapes3(blocks, &pl->sh3);
    pl->sLU3 = (size_t)pl->sh3.nrows_max * 32;
    pl->sWork3 = (size_t)pl->sh3.nrows_max * 32;  // U part of every block cell
    pl->sPad3 = ((size_t)pl->sh3.pad_max + 31) / 32 * 32;
  }
  const size_t vec = (size_t)N * 8;
  const int m = p->gmres_restart;
  const size_t tiles = (size_t)((g->n[0] + 31) / 32) * ((g->n[1] + 15) / 16);
  pl->partial_len = std::max<size_t>(tiles * 2, (size_t)pfc::kRedCtas * (pfc::kMaxVecs + 2));
  pl->partial_len = std::max<size_t>(pl->partial_len, 152 * 8 * 2);
  Layout L;
  pl->phin = L.take(vec);
  pl->phinm1 = L.take(vec);
  pl->Phi = L.take(vec);
  pl->F = L.take(vec);
  pl->q = L.take(vec);
  pl->Pt = L.take(vec);
  pl->Ft = L.take(vec);
  pl->qt = L.take(vec);
  pl->S = L.take(vec);
  pl->W = L.take(vec);
  pl->guess = L.take(vec);
  const size_t vstride = basis_stride(N);
  pl->V = L.take(vstride * 8 * (m + 1));
  pl->Z = L.take(vstride * 8 * m);
  pl->L = L.take(pl->sL * es * pl->nblocks);
  pl->U = L.take(pl->sU * es * pl->nblocks);
  pl->piv = L.take(pl->sP * pl->nblocks);
  pl->X = L.take((size_t)pl->xnc * pl->nblocks * (pl->xfw + pl->xbw));
  pl->Yb = L.take(!d3 && p->ras_kind != PFC_LEFT_RAS ? sizeof(double) * (size_t)pl->n_max * pl->nblocks : 0);
  const size_t mvec = p->mobility ? vec : 0;  // mu and s = (Phi + phi^n)/2 beside q and the trial q
  pl->mu = L.take(mvec);
  pl->mut = L.take(mvec);
  pl->smid = L.take(mvec);
  pl->smidt = L.take(mvec);
  pl->blocks = L.take(sizeof(BlockDesc) * pl->nblocks);
  pl->lin = L.take(sizeof(double) * 343);
  pl->ctl = L.take(sizeof(GmresCtl));
  pl->partial = L.take(sizeof(double) * pl->partial_len);
  pl->red = L.take(sizeof(double) * 16);
  pl->status = L.take(sizeof(int) * 4);
  pl->tabs = L.take(sizeof(double*) * 2 * pfc::kMaxVecs);
  pl->iargs = L.take(sizeof(pfc::IterArgs));
  pl->iargs2 = L.take(sizeof(pfc::IterArgs));
  pl->sctl = L.take(sizeof(pfc::StepCtl));
  pl->recs = L.take(sizeof(pfc_step_info) * kBatchRecs);
  pl->order = L.take(sizeof(int) * (pl->nblocks + 16));
  pl->feat = d3 ? 0 : L.take(vec * 3);
  if (d3) {
    const Shapes3& S = pl->sh3;
    pl->T1 = L.take(vec);
    pl->T2 = L.take(vec);
    pl->shapes = L.take(sizeof(pfc::Shape3) * S.shapes.size());
    pl->block_shape = L.take(sizeof(int) * S.block_shape.size());
    pl->lev_start = L.take(sizeof(int) * S.lev_start.size());
    pl->rowpad = L.take(sizeof(int) * S.rowpad.size());
    pl->rowabc = L.take(sizeof(int) * S.rowabc.size());
    pl->posL = L.take(S.posL.size());
    pl->posU = L.take(S.posU.size());
    pl->Lp = L.take(pl->sLU3 * es * pl->nblocks);
    pl->Up = L.take(pl->sLU3 * es * pl->nblocks);
    pl->work = L.take(pl->sWork3 * tc * pl->nblocks);
    pl->ypad = L.take(pl->sPad3 * tc * pl->nblocks);
  }
  pl->total = L.total;
  return PFC_OK;
}

// 7-point (or 5-point) stencil convolution on a 7x7x7 table, centre (3,3,3).
void conv3(const double* a, const double* b, double* c) {
  for (int i = 0; i < 343; ++i) c[i] = 0.0;
  for (int i = 0; i < 343; ++i) {
    if (a[i] == 0.0) continue;
    const int az = i / 49 - 3, ay = (i / 7) % 7 - 3, ax = i % 7 - 3;
    for (int j = 0; j < 343; ++j) {
      if (b[j] == 0.0) continue;
      const int z = az + j / 49 - 3, y = ay + (j / 7) % 7 - 3, x = ax + j % 7 - 3;
      if (std::abs(x) <= 3 && std::abs(y) <= 3 && std::abs(z) <= 3) c[(z + 3) * 49 + (y + 3) * 7 + (x + 3)] += a[i] * b[j];
    }
  }
}

// -(1/2) Delta_d L_gamma with L_gamma = (1-gamma) + 2 Delta_d + Delta_d^2, as a
// 7x7x7 table (index (dz+3)*49 + (dy+3)*7 + dx+3); a 2D grid uses its dz = 0 plane.
void lin_stencil(int dim, double h, double gamma, double* out343, double* out49) {
  double P1[343] = {}, P2[343], P3[343];
  const int c = 171;
  P1[c] = -2.0 * dim;
  P1[c - 1] = P1[c + 1] = P1[c - 7] = P1[c + 7] = 1.0;
  if (dim == 3) P1[c - 49] = P1[c + 49] = 1.0;
  conv3(P1, P1, P2);
  conv3(P2, P1, P3);
  const double ih2 = 1.0 / (h * h), ih4 = ih2 * ih2, ih6 = ih4 * ih2;
  for (int i = 0; i < 343; ++i)
    out343[i] = -0.5 * ((1.0 - gamma) * ih2 * P1[i] + 2.0 * ih4 * P2[i] + ih6 * P3[i]);
  for (int i = 0; i < 49; ++i) out49[i] = out343[3 * 49 + i];
}

// ---------------------------------------------------------------- building blocks of a step
int sync_read(pfc_state* s, void* dst, const void* src, size_t bytes) {
  CU(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, s->st));
  CU(cudaStreamSynchronize(s->st));
  return PFC_OK;
}

// ---- kernel timing (pfc_profile)
// Adds every waiting pair whose launch ran to its family's sums (pairs of Arnoldi column
// j >= its_run belong to iterations queued after the cycle converged: their kernels
// returned at once) and empties the pool.  The stream must have passed every pair.
int prof_resolve(pfc_state* s, int its_run) {
  for (size_t i = 0; i < s->ppend.size(); ++i) {
    const ProfPair& pp = s->ppend[i];
    if (pp.j >= 0 && pp.j >= its_run) continue;
    float ms = 0.f;
    CU(cudaEventElapsedTime(&ms, s->pev[2 * i], s->pev[2 * i + 1]));
    pfc_kernel_prof& k = s->pk[pp.kind];
    k.launches += 1;
    k.ms += ms;
    k.bytes += pp.bytes;
    k.flops += pp.flops;
    k.bytes_stored += pp.stored;
  }
  s->ppend.clear();
  return PFC_OK;
}
// Opens a timed launch (returns its slot, -1 when profiling is off); a full pool is first
// drained with a stream synchronisation.
int prof_begin(pfc_state* s, int* slot) {
  *slot = -1;
  if (!s->prof) return PFC_OK;
  if (s->ppend.size() >= (size_t)kProfSlots) {
    CU(cudaStreamSynchronize(s->st));
    int rc = prof_resolve(s, 1 << 30);
    if (rc) return rc;
  }
  *slot = (int)s->ppend.size();
  CU(cudaEventRecord(s->pev[2 * *slot], s->st));
  s->ppend.push_back(ProfPair{-1, -1, 0.0, 0.0, 0.0});
  return PFC_OK;
}
int prof_end(pfc_state* s, int slot, int kind, int j, double bytes, double flops = 0.0, double stored = -1.0) {
  if (slot < 0) return PFC_OK;
  CU(cudaEventRecord(s->pev[2 * slot + 1], s->st));
  s->ppend[slot] = ProfPair{kind, j, bytes, flops, stored < 0.0 ? bytes : stored};
  return PFC_OK;
}
#define PROF_BEGIN(slot)                \
  do {                                  \
    int rc_ = prof_begin(s, &(slot));   \
    if (rc_) return rc_;                \
  } while (0)
#define PROF_END(...)                   \
  do {                                  \
    int rc_ = prof_end(s, __VA_ARGS__); \
    if (rc_) return rc_;                \
  } while (0)

// F, q at Phi (or at the trial point Phi + lam (S - mean S)); returns ||F||^2 on the device in red[slot].
// dev (2D): 1/dt and the line-search step lam are read from the step's StepCtl on the device.
int eval_residual(pfc_state* s, const double* Pb, const double* S, double lam, bool project, const double* phin,
                  double idt, double* F, double* Pout, double* qout, int slot, bool dev = false) {
  int np = 0;
  int ps;
  PROF_BEGIN(ps);
  if (s->dim == 2) {
    // with variable mobility, mu and s go beside q: (mu, sm) with q, (mut, smt) with the trial q
    const bool mob = s->p.mobility != 0;
    double* muo = qout == s->q ? s->mu : s->mut;
    double* so = qout == s->q ? s->sm : s->smt;
    pfc::launch_residual2d(s->g, Pb, S, lam, project ? s->red + 9 : nullptr, phin, idt, F, Pout, qout, s->partial,
                           &np, s->st, mob, mob && qout ? muo : nullptr, mob && qout ? so : nullptr,
                           dev ? &s->sc->idt : nullptr, dev && S ? &s->sc->lam : nullptr);
  } else {
    const double* P = Pb;
    if (S) {  // the trial point is needed at neighbours: materialise it first
      pfc::launch_trial(s->g, Pb, S, lam, project ? s->red + 9 : nullptr, Pout, s->st);
      P = Pout;
    }
    const bool mob = s->p.mobility != 0;  // mu and s beside q, as in 2D
    double* muo = qout == s->q ? s->mu : s->mut;
    double* so = qout == s->q ? s->sm : s->smt;
    pfc::launch_residual3d(s->g, P, phin, idt, F, qout, s->T1, s->T2, s->partial, &np, s->st, mob,
                           mob && qout ? muo : nullptr, mob && qout ? so : nullptr);
  }
  // reads Phi (or Phi_b and S), phi^n; writes F (and the trial Phi, q)
  PROF_END(ps, PFC_PROF_RESIDUAL, -1, 8.0 * s->g.n * (3 + (S ? 2 : 0) + (qout ? 1 : 0)));
  pfc::launch_reduce(s->partial, 1, np, s->red + slot, s->st);
  CU(cudaGetLastError());
  return PFC_OK;
}

// The mixed path (F32/BF16 factors) runs the Arnoldi sweeps in float-float arithmetic
// (the dot products too, unless gmres_fast_dots asks for FP32 ones).
bool ff_sweeps(const pfc_state* s) { return s->p.factor_prec != PFC_F64; }
// The mixed path keeps its Krylov basis V as float pairs (ff.cuh): the JVP writes them, the
// sweeps and the Schwarz apply read them without a split.  Not with variable mobility, whose JVP
// stays FP64.
bool pair_basis(const pfc_state* s) { return ff_sweeps(s) && !s->p.mobility; }
// Bytes the apply kernel in use reads and writes per launch (its storage format).
double apply_stored(const pfc_state* s) {
  return s->dim == 2 && s->fs.variant == pfc::kChunkedVariant ? s->apply_bytes_chunk : s->apply_bytes_step;
}
int dot_mode(const pfc_state* s) {
  if (!ff_sweeps(s)) return pfc::kDotF64;
  return s->p.gmres_fast_dots ? pfc::kDotF32 : pfc::kDotFF;
}

// zplane: v = Z_zplane of the basis and q = s->q, so the product may stage both by TMA (-1: not).
// pout: out (or ia->w) is a basis vector stored as float pairs (pair_basis).
void jvp(pfc_state* s, const double* v, const double* q, double idt, double* out, const int* skip,
         const pfc::IterArgs* ia = nullptr, int zplane = -1, bool pout = false) {
  if (s->p.mobility) {  // variable mobility: FP64 on every path; mu, s of q's iterate
    const bool trial = q != nullptr && q == s->qt;
    if (s->dim == 2)
      pfc::launch_jvp2d(s->g, v, nullptr, q, idt, out, skip, s->st, ia, trial ? s->mut : s->mu,
                        trial ? s->smt : s->sm);
    else
      pfc::launch_jvp3d(s->g, v, nullptr, q, idt, out, s->T1, s->T2, skip, s->st, trial ? s->mut : s->mu,
                        trial ? s->smt : s->sm);
  } else if (s->dim == 2 && s->fs.prec != PFC_F64 && s->p.jvp_fp32)  // mixed path, opt-in: plain FP32
    pfc::launch_jvp2d_f32(s->g, v, q, idt, out, skip, s->st, ia, &s->jmaps, zplane, s->status_dev + 1, pout);
  else if (s->dim == 2 && s->fs.prec != PFC_F64)  // mixed path: float-float JVP on the FP32 pipe
    pfc::launch_jvp2d_ff(s->g, v, nullptr, q, idt, out, skip, s->st, ia, &s->jmaps, zplane, s->status_dev + 1,
                         pout);
  else if (s->dim == 2)
    pfc::launch_jvp2d(s->g, v, nullptr, q, idt, out, skip, s->st, ia);
  else if (s->fs.prec != PFC_F64 && s->p.jvp_fp32)  // 3D mixed path, opt-in: plain FP32 passes
    pfc::launch_jvp3d_f32(s->g, v, q, idt, out, s->T1, s->T2, skip, s->st, pout);
  else if (s->fs.prec != PFC_F64)  // 3D mixed path: float-float passes on the FP32 pipe
    pfc::launch_jvp3d_ff(s->g, v, q, idt, out, s->T1, s->T2, skip, s->st, pout);
  else
    pfc::launch_jvp3d(s->g, v, nullptr, q, idt, out, s->T1, s->T2, skip, s->st);
}

// pin: r (or ia->v) is a basis vector stored as float pairs (pair_basis).
void precond(pfc_state* s, const double* r, const double* rscale, double* z, const int* skip,
             const pfc::IterArgs* ia = nullptr, bool pin = false) {
  s->fs.pin = pin ? 1 : 0;
  s->r3.pin = pin ? 1 : 0;
  if (s->dim == 2)
    pfc::launch_ras_apply2d(s->g, s->blocks_dev, s->nblocks, s->fs, r, rscale, z, skip, s->status_dev + 1, s->st,
                            ia, &s->dc);
  else
    pfc::launch_ras_apply3d(s->g, s->blocks_dev, s->nblocks, s->r3, r, rscale, z, skip, s->status_dev + 1, s->st);
}

// Times every apply kernel that can run the blocks on the factors just made
// (r = F, z = W: both free at this point) and keeps the fastest.
bool variant_ok(const pfc_state* s, int v) {
  return pfc::apply_variant_ok(v, s->fs.prec, s->fs.kl_max, s->fs.xstage, s->fs.n_max);
}

constexpr int kTuneReps = 10;  // timed applies per kernel

int tune_apply(pfc_state* s) {
  cudaEvent_t e0, e1;
  CU(cudaEventCreate(&e0));
  CU(cudaEventCreate(&e1));
  int best = -1;
  float best_ms = 0.f;
  int rc = PFC_OK;
  for (int v = 0; v < pfc::kApplyVariants && rc == PFC_OK; ++v) {
    s->tune_ms[v] = -1.f;
    if (!variant_ok(s, v) || (v == pfc::kChunkedVariant && !s->fs.x_valid)) continue;
    s->fs.variant = v;
    for (int i = 0; i < 2; ++i) precond(s, s->F, nullptr, s->W, nullptr);  // warm-up
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventRecord(e0, s->st);
    for (int i = 0; i < kTuneReps && e == cudaSuccess; ++i) {
      precond(s, s->F, nullptr, s->W, nullptr);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, s->st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e != cudaSuccess) {
      fprintf(stderr, "libpfc: timing apply kernel %d failed: %s\n", v, cudaGetErrorString(e));
      rc = PFC_ECUDA;
      break;
    }
    s->tune_ms[v] = ms / kTuneReps;
    if (best < 0 || ms < best_ms) {
      best = v;
      best_ms = ms;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != PFC_OK) return rc;
  if (best < 0) return PFC_EINVAL;
  for (int v = 0; v < best; ++v)  // timing noise: prefer the lowest-numbered shape within 1 % of the best
    if (s->tune_ms[v] > 0.f && s->tune_ms[v] <= 1.01f * s->tune_ms[best]) {
      best = v;
      break;
    }
  s->fs.variant = best;
  s->tuned = true;
  return PFC_OK;
}

// dev: 1/dt read from the step's StepCtl (a captured step graph).
int factor_blocks(pfc_state* s, const double* q, double idt, bool dev = false) {
  if (s->p.mobility) {  // the mobility fields of q's iterate
    const bool trial = q == s->qt;
    s->fs.mob_mu = s->r3.mob_mu = trial ? s->mut : s->mu;
    s->fs.mob_s = s->r3.mob_s = trial ? s->smt : s->sm;
  }
  if (s->dim == 2) {
    // the sliding factor window holds 2 kl + 2 <= 256 column slots (kl = 3 bx: blocks at most 42 cells
    // wide in x); blocks wider than 21 cells run the wide-window apply kernel in its default shape or
    // the chunked apply
    if (2 * s->fs.kl_max + 2 > 256 ||
        pfc::factor_smem_bytes(s->fs.prec, s->fs.kl_max, s->fs.n_max, s->p.mobility ? s->fs.ext_max : 0) > 227 * 1024)
      return PFC_EINVAL;
    if (s->p.apply_variant >= 0 && !variant_ok(s, s->p.apply_variant)) return PFC_EINVAL;
    if (s->p.apply_variant < 0 && !variant_ok(s, 0)) return PFC_EINVAL;
  }
  CU(cudaMemsetAsync(s->status_dev, 0, 2 * sizeof(int), s->st));
  int ps;
  PROF_BEGIN(ps);
  if (s->dim == 2)
    pfc::launch_factor2d(s->g, s->blocks_dev, s->nblocks, q, idt, s->lin_dev, s->fs, s->status_dev, s->st,
                         dev ? &s->sc->idt : nullptr);
  else
    pfc::launch_factor3d(s->g, s->blocks_dev, s->nblocks, q, idt, s->lin_dev, s->r3, s->status_dev, s->st);
  PROF_END(ps, PFC_PROF_FACTOR, -1, s->factor_bytes, s->factor_flops);
  CU(cudaGetLastError());
  if (s->dim == 2) {  // chunked records for the chunked apply (in use, or about to be timed)
    const bool tuning = s->p.apply_variant < 0 && !s->tuned && variant_ok(s, pfc::kChunkedVariant);
    s->fs.x_valid = 0;
    if (tuning || s->fs.variant == pfc::kChunkedVariant) {
      PROF_BEGIN(ps);
      pfc::launch_chunk2d(s->blocks_dev, s->nblocks, s->fs, s->st);
      PROF_END(ps, PFC_PROF_RECORDS, -1, s->record_bytes);
      CU(cudaGetLastError());
      s->fs.x_valid = 1;
    }
  }
  if (s->dim == 2 && s->p.apply_variant < 0 && !s->tuned) return tune_apply(s);
  return PFC_OK;
}

// ---------------------------------------------------------------- one time step
// Every decision of a step is taken on the device by the control kernels of
// newton.cu on the step's StepCtl (s->sc).  The emitters below queue the kernels of
// each part of the step on s->st.  The host-driven form (step_host) reads StepCtl
// back after each decision and runs the loops itself; the graph form captures the
// same emitters once into the bodies of nested conditional nodes (Newton loop,
// factor branch, GMRES restart loop, Arnoldi loop, restart branch, line-search
// loop, commit branch), so that a whole step is one graph launch.  Both forms run
// the same kernels in the same order on the same data.

int read_ctl(pfc_state* s) { return sync_read(s, s->sc_h, s->sc, sizeof(pfc::StepCtl)); }

unsigned int* ticket(pfc_state* s) { return reinterpret_cast<unsigned int*>(s->status_dev + 2); }

// Factors of J(Phi_0) (Eq. Ak) at the first Newton iteration of a step, reused by the
// later ones (Sec. 5.2).
int emit_factor(pfc_state* s, double idt) {
  int rc = factor_blocks(s, s->q, idt, s->dim == 2);
  if (rc) return rc;
  pfc::launch_factor_done(s->sc, s->st);
  CU(cudaGetLastError());
  return PFC_OK;
}

// GMRES for J S = -F from S = 0 (Eq. hjacobi): S and the sums of S cleared, V_0 <- F
// (scaled by -1/||F|| on the device), the cycle's tolerance and state.
int emit_gmres_begin(pfc_state* s, int gm) {
  pfc::launch_gmres_prep(s->S, s->red + 8, s->F, s->Vbuf, s->g.n, s->st, pair_basis(s));
  pfc::launch_gmres_begin(s->sc, s->ctl, s->hs, gm, s->st);
  CU(cudaGetLastError());
  return PFC_OK;
}

int gs_passes(const pfc_state* s) { return s->p.gmres_reorth_eta > 0.0 ? 2 : 1; }

// The Arnoldi iterations of one cycle driven by the host: iterations are queued a chunk at a
// time; after each chunk the head of the control block is copied back asynchronously, and the
// host waits for a chunk's head only once the next chunk is queued, so the GPU never idles on
// the host.  A chunk queued after the cycle ended runs its kernels as immediate returns (the
// done flag).  Basis V_0 = Vbuf, V_i = Vbuf + i vstride (s->vtab); Z_i = Zbuf + i vstride.
int arnoldi_host(pfc_state* s, double idt) {
  const long long N = s->g.n;
  const int m = s->p.gmres_restart;
  const int* done = &s->ctl->done;
  const int* reorth = &s->ctl->reorth;
  const double* v0 = s->Vbuf;
  const bool pairs = pair_basis(s);
  int j = 0;
  const int chunk = 3;
  int c = 0, pend = -1;  // chunks queued; buffer of the pending chunk
  bool stop = false;
  while (!stop) {
    const int q0 = j, q1 = std::min(m, j + chunk);
    const bool more = q0 < q1;
    for (; j < q1; ++j) {
      const double* vj = s->Vbuf + (size_t)j * s->vstride;
      double* zj = s->Zbuf + (size_t)j * s->vstride;
      double* w = s->Vbuf + (size_t)(j + 1) * s->vstride;
      // (pfc_profile: apply, JVP and the first Gram-Schmidt pass are timed; the second pass
      // runs only on the DGKS test, which the host does not see)
      int ps;
      PROF_BEGIN(ps);
      precond(s, vj, &s->ctl->scale[j], zj, done, nullptr, pairs);
      PROF_END(ps, PFC_PROF_APPLY, j, s->apply_bytes, 0.0, apply_stored(s));
      PROF_BEGIN(ps);
      jvp(s, zj, s->q, idt, w, done, nullptr, j, pairs);
      PROF_END(ps, PFC_PROF_JVP, j, 24.0 * N);  // reads v, q; writes Jv
      for (int pass = 0; pass < gs_passes(s); ++pass) {
        pfc::Tail td{pfc::Tail::kDot, j, pass, m, s->ctl, ticket(s), nullptr};
        td.err = s->status_dev + 1;
        if (pass == 0) PROF_BEGIN(ps);
        pfc::launch_multidot(v0, s->vtab, j + 2, w, N, s->partial, done, pass ? reorth : nullptr, td, s->st,
                             dot_mode(s), m + 1, pairs);
        if (pass == 0) PROF_END(ps, PFC_PROF_DOT, j, 8.0 * N * (j + 2));  // reads V_0..V_j and w
        pfc::Tail ta{pfc::Tail::kAxpy, j, pass, m, s->ctl, ticket(s), nullptr};
        ta.err = s->status_dev + 1;
        if (pass == 0) PROF_BEGIN(ps);
        pfc::launch_multiaxpy(w, v0, s->vtab, j + 1, s->ctl->coef, -1.0, N, s->partial, done,
                              pass ? reorth : nullptr, ta, s->st, ff_sweeps(s), pairs);
        if (pass == 0) PROF_END(ps, PFC_PROF_AXPY, j, 8.0 * N * (j + 3));  // reads V_0..V_j, w; writes w
      }
    }
    if (more) {
      CU(cudaGetLastError());
      CU(cudaMemcpyAsync(s->ctl_hb[c & 1], s->ctl, offsetof(GmresCtl, H), cudaMemcpyDeviceToHost, s->st));
      CU(cudaEventRecord(s->ctl_ev[c & 1], s->st));
    }
    if (pend >= 0) {  // the chunk before this one: did the cycle end there?
      CU(cudaEventSynchronize(s->ctl_ev[pend]));
      if (s->ctl_hb[pend]->done) stop = true;
    }
    if (more) {
      pend = c & 1;
      ++c;
    } else {
      pend = -1;
      stop = true;
    }
  }
  // the cycle's final head (every queued kernel has finished after this)
  int rc = sync_read(s, s->ctl_h, s->ctl, offsetof(GmresCtl, H));
  if (rc) return rc;
  if (s->prof && (rc = prof_resolve(s, s->ctl_h->its))) return rc;
  return PFC_OK;
}

// After a cycle: y from the rotated Hessenberg system, S += sum_j y_j Z_j over the cycle's
// iterations (|S|^2 and sum S into red[8..9]), then converged / failed / restart.
int emit_cycle_end(pfc_state* s, int gm) {
  pfc::launch_gmres_solve(s->ctl, s->st);
  pfc::Tail tsum{pfc::Tail::kSums, 0, 0, 0, s->ctl, ticket(s), s->red + 8};
  tsum.err = s->status_dev + 1;
  tsum.nx_dev = &s->ctl->its;
  pfc::launch_multiaxpy(s->S, s->Zbuf, s->ztab, s->p.gmres_restart, s->ctl->y, 1.0, s->g.n, s->partial, nullptr,
                        nullptr, tsum, s->st);
  pfc::launch_cycle_decide(s->sc, s->ctl, s->hs, gm, s->st);
  CU(cudaGetLastError());
  return PFC_OK;
}

// Restart: r = -F - J S into W, ||r||^2 into red[10], V_0 <- r (scaled by 1/||r||).
int emit_restart(pfc_state* s, double idt, int gm) {
  const long long N = s->g.n;
  if (gm)
    jvp(s, nullptr, nullptr, 0.0, nullptr, nullptr, s->ia2);  // S -> W with this step's 1/dt
  else
    jvp(s, s->S, s->q, idt, s->W, nullptr);
  pfc::launch_axpby(s->W, s->F, -1.0, -1.0, N, s->st);
  pfc::Tail tnrm{pfc::Tail::kSums, 0, 0, 0, s->ctl, ticket(s), s->red + 10};
  tnrm.err = s->status_dev + 1;
  pfc::launch_multidot(s->W, s->vtab, 1, s->W, N, s->partial, nullptr, nullptr, tnrm, s->st);
  pfc::launch_gmres_restart(s->sc, s->ctl, s->red + 10, s->st);
  pfc::CopyPairs cp{};
  cp.src[0] = s->W;
  cp.dst[0] = s->Vbuf;
  cp.n = 1;
  cp.to_pairs = pair_basis(s) ? 1u : 0u;
  pfc::launch_copy_if_ok(s->sc, cp, N, s->st);
  CU(cudaGetLastError());
  return PFC_OK;
}

// One line-search trial Phi + lam (S - mean S) (Armijo backtracking on ||F||^2 / 2) and its decision.
int emit_ls_trial(pfc_state* s, double lam, double idt, int gm) {
  int rc = eval_residual(s, s->Phi, s->S, lam, s->p.mass_projection != 0, s->phin, idt, s->Ft, s->Pt, s->qt, 1,
                         s->dim == 2);
  if (rc) return rc;
  pfc::launch_ls_decide(s->sc, s->red + 1, s->hs, gm, s->st);
  CU(cudaGetLastError());
  return PFC_OK;
}

// The accepted trial point becomes the Newton iterate (Phi, F, q and the mobility fields), then
// the Newton stop test.
int emit_accept(pfc_state* s, int gm) {
  pfc::CopyPairs cp{};
  cp.src[0] = s->Pt;
  cp.dst[0] = s->Phi;
  cp.src[1] = s->Ft;
  cp.dst[1] = s->F;
  cp.src[2] = s->qt;
  cp.dst[2] = s->q;
  cp.n = 3;
  if (s->p.mobility) {
    cp.src[3] = s->mut;
    cp.dst[3] = s->mu;
    cp.src[4] = s->smt;
    cp.dst[4] = s->sm;
    cp.n = 5;
  }
  pfc::launch_copy_if_ok(s->sc, cp, s->g.n, s->st);
  pfc::launch_newton_next(s->sc, s->hs, gm, s->st);
  CU(cudaGetLastError());
  return PFC_OK;
}

// A converged step: phi^{n-1} <- phi^n, phi^n <- Phi, and the energy and mass of the new
// phi^n (Eq. freeenergy; h^d sum phi) into red[4..5].
int emit_commit(pfc_state* s) {
  pfc::CopyPairs cp{};
  cp.src[0] = s->phin;
  cp.dst[0] = s->phinm1;
  cp.src[1] = s->Phi;
  cp.dst[1] = s->phin;
  cp.n = 2;
  pfc::launch_copy_if_ok(s->sc, cp, s->g.n, s->st);
  int np = 0;
  if (s->dim == 2)
    pfc::launch_energy2d(s->g, s->phin, s->partial, &np, s->st);
  else
    pfc::launch_energy3d(s->g, s->phin, s->partial, &np, s->st);
  pfc::launch_reduce(s->partial, 2, np, s->red + 4, s->st);
  CU(cudaGetLastError());
  return PFC_OK;
}

// One step driven by the host (3D, per-kernel profiling, the step that tunes the apply, no
// capturable stream, or use_graph = 0): Newton from the guess in s->Phi.
int step_host(pfc_state* s, double dt) {
  const double idt = 1.0 / dt;
  int rc = eval_residual(s, s->Phi, nullptr, 0.0, false, s->phin, idt, s->F, nullptr, s->q, 0, s->dim == 2);
  if (rc) return rc;
  pfc::launch_newton_begin(s->sc, s->red, s->ia, s->ia2, s->hs, 0, s->st);
  if ((rc = read_ctl(s))) return rc;
  const pfc::StepCtl* c = s->sc_h;
  while (c->newton_go) {
    if (c->factor_go && (rc = emit_factor(s, idt))) return rc;
    if ((rc = emit_gmres_begin(s, 0)) || (rc = read_ctl(s))) return rc;
    while (c->cycle_go) {
      if ((rc = arnoldi_host(s, idt))) return rc;
      if ((rc = emit_cycle_end(s, 0)) || (rc = read_ctl(s))) return rc;
      if (c->restart_go && (rc = emit_restart(s, idt, 0))) return rc;
    }
    pfc::launch_gmres_end(s->sc, s->status_dev, s->hs, 0, s->st);
    if ((rc = read_ctl(s))) return rc;
    while (c->ls_go)
      if ((rc = emit_ls_trial(s, c->lam, idt, 0)) || (rc = read_ctl(s))) return rc;
    if ((rc = emit_accept(s, 0)) || (rc = read_ctl(s))) return rc;
  }
  pfc::launch_step_end(s->sc, s->hs, 0, s->st);
  if ((rc = read_ctl(s))) return rc;
  if (c->commit_go) rc = emit_commit(s);
  return rc;
}

// ---- the graph form
// A conditional handle on the graph being captured on st (the graph that will hold its node).
bool new_handle(cudaStream_t st, cudaGraphConditionalHandle* h) {
  cudaStreamCaptureStatus cs;
  cudaGraph_t g = nullptr;
  if (cudaStreamGetCaptureInfo(st, &cs, nullptr, &g, nullptr, nullptr, nullptr) != cudaSuccess ||
      cs != cudaStreamCaptureStatusActive || !g)
    return false;
  return cudaGraphConditionalHandleCreate(h, g, 0, cudaGraphCondAssignDefault) == cudaSuccess;
}

// Adds a conditional node after the work captured so far on st; returns its body graph.
bool add_cond(cudaStream_t st, cudaGraphConditionalHandle h, cudaGraphConditionalNodeType type, cudaGraph_t* body) {
  cudaStreamCaptureStatus cs;
  cudaGraph_t g = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  size_t nd = 0;
  if (cudaStreamGetCaptureInfo(st, &cs, nullptr, &g, &deps, nullptr, &nd) != cudaSuccess ||
      cs != cudaStreamCaptureStatusActive || !g)
    return false;
  cudaGraphNodeParams p = {};
  p.type = cudaGraphNodeTypeConditional;
  p.conditional.handle = h;
  p.conditional.type = type;
  p.conditional.size = 1;
  cudaGraphNode_t node;
  if (cudaGraphAddNode(&node, g, deps, nullptr, nd, &p) != cudaSuccess) return false;
  if (cudaStreamUpdateCaptureDependencies(st, &node, nullptr, 1, cudaStreamSetCaptureDependencies) != cudaSuccess)
    return false;
  *body = p.conditional.phGraph_out[0];
  return true;
}

// Captures what `emit` queues into `body` on the helper stream cs (s->st is switched to cs
// meanwhile, so that every emitter queues there).
template <class F>
bool capture_body(pfc_state* s, cudaGraph_t body, cudaStream_t cs, F emit) {
  if (cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
    return false;
  cudaStream_t saved = s->st;
  s->st = cs;
  bool ok = emit();
  s->st = saved;
  cudaGraph_t out = nullptr;
  ok = cudaStreamEndCapture(cs, &out) == cudaSuccess && ok;
  return ok;
}

// Kernels of one Arnoldi iteration of the graph form without a second Gram-Schmidt pass (each
// second pass adds its two sweeps; StepCtl counts them).
int arnoldi_body_kernels(const pfc_state* s) { return 5 + (s->fs.ras_kind != PFC_LEFT_RAS ? 1 : 0); }

// One Arnoldi iteration (graph form): Schwarz apply, JVP, the first Gram-Schmidt pass, the
// second pass inside an IF node that the first pass's last CTA sets (DGKS test), and the loop
// test, which also writes the next iteration's vectors to s->ia.  The IF body is captured on
// cs_if.
bool emit_arnoldi_body(pfc_state* s, cudaStream_t cs_if) {
  const long long N = s->g.n;
  const int m = s->p.gmres_restart;
  const int* done = &s->ctl->done;
  const int* reorth = &s->ctl->reorth;
  const double* v0 = s->Vbuf;
  const bool two = gs_passes(s) == 2;
  const bool pairs = pair_basis(s);
  if (two && !new_handle(s->st, &s->hs.reorth)) return false;
  precond(s, nullptr, nullptr, nullptr, done, s->ia, pairs);
  jvp(s, nullptr, nullptr, 0.0, nullptr, done, s->ia, -1, pairs);
  auto pass = [&](int p) {
    pfc::Tail td{pfc::Tail::kDot, 0, p, m, s->ctl, ticket(s), nullptr, s->ia};
    td.err = s->status_dev + 1;
    pfc::launch_multidot(v0, s->vtab, m + 1, nullptr, N, s->partial, done, p ? reorth : nullptr, td, s->st,
                         dot_mode(s), 0, pairs);
    pfc::Tail ta{pfc::Tail::kAxpy, 0, p, m, s->ctl, ticket(s), nullptr, s->ia};
    ta.err = s->status_dev + 1;
    if (two && p == 0) {
      ta.h_reorth = s->hs.reorth;
      ta.set_reorth = 1;
    }
    pfc::launch_multiaxpy(nullptr, v0, s->vtab, m, s->ctl->coef, -1.0, N, s->partial, done, p ? reorth : nullptr,
                          ta, s->st, ff_sweeps(s), pairs);
    return cudaGetLastError() == cudaSuccess;
  };
  bool ok = pass(0);
  if (ok && two) {
    cudaGraph_t body;
    ok = add_cond(s->st, s->hs.reorth, cudaGraphCondTypeIf, &body) && capture_body(s, body, cs_if, [&] { return pass(1); });
  }
  pfc::launch_arnoldi_next(s->ctl, s->vtab, s->ztab, s->ia, m, s->hs.arnoldi, s->st);
  return ok && cudaGetLastError() == cudaSuccess;
}

// Queues the whole step of the graph form on s->st (which is being captured): every 1/dt
// and line-search step is read from s->sc, every decision sets a conditional handle.
bool emit_step_graph(pfc_state* s, int depth0 = 0) {
  pfc::StepHandles& h = s->hs;
  const int m = s->p.gmres_restart;
  cudaStream_t* cs = s->cs + depth0;  // nested bodies at depth d are captured on cs[d]
  if (!new_handle(s->st, &h.newton) || !new_handle(s->st, &h.commit)) return false;
  if (eval_residual(s, s->Phi, nullptr, 0.0, false, s->phin, 1.0, s->F, nullptr, s->q, 0, true)) return false;
  pfc::launch_newton_begin(s->sc, s->red, s->ia, s->ia2, h, 1, s->st);
  cudaGraph_t newton_body;
  bool ok = add_cond(s->st, h.newton, cudaGraphCondTypeWhile, &newton_body) &&
            capture_body(s, newton_body, cs[0], [&] {
              if (!new_handle(s->st, &h.factor) || !new_handle(s->st, &h.cycle) || !new_handle(s->st, &h.ls))
                return false;
              pfc::launch_set_factor_cond(s->sc, h, 1, s->st);
              cudaGraph_t factor_body, cycle_body, ls_body;
              bool k = add_cond(s->st, h.factor, cudaGraphCondTypeIf, &factor_body) &&
                       capture_body(s, factor_body, cs[1], [&] { return emit_factor(s, 1.0) == PFC_OK; });
              k = k && emit_gmres_begin(s, 1) == PFC_OK;
              k = k && add_cond(s->st, h.cycle, cudaGraphCondTypeWhile, &cycle_body) &&
                  capture_body(s, cycle_body, cs[1], [&] {
                    if (!new_handle(s->st, &h.arnoldi) || !new_handle(s->st, &h.restart)) return false;
                    pfc::launch_arnoldi_next(s->ctl, s->vtab, s->ztab, s->ia, m, h.arnoldi, s->st);
                    cudaGraph_t arnoldi_body, restart_body;
                    bool q = add_cond(s->st, h.arnoldi, cudaGraphCondTypeWhile, &arnoldi_body) &&
                             capture_body(s, arnoldi_body, cs[2], [&] { return emit_arnoldi_body(s, cs[3]); });
                    q = q && emit_cycle_end(s, 1) == PFC_OK;
                    q = q && add_cond(s->st, h.restart, cudaGraphCondTypeIf, &restart_body) &&
                        capture_body(s, restart_body, cs[2], [&] { return emit_restart(s, 1.0, 1) == PFC_OK; });
                    return q;
                  });
              pfc::launch_gmres_end(s->sc, s->status_dev, h, 1, s->st);
              k = k && add_cond(s->st, h.ls, cudaGraphCondTypeWhile, &ls_body) &&
                  capture_body(s, ls_body, cs[1], [&] { return emit_ls_trial(s, 1.0, 1.0, 1) == PFC_OK; });
              k = k && emit_accept(s, 1) == PFC_OK;
              return k;
            });
  pfc::launch_step_end(s->sc, h, 1, s->st);
  cudaGraph_t commit_body;
  ok = ok && add_cond(s->st, h.commit, cudaGraphCondTypeIf, &commit_body) &&
       capture_body(s, commit_body, cs[0], [&] { return emit_commit(s) == PFC_OK; });
  return ok && cudaGetLastError() == cudaSuccess;
}

// Kernels a graph step ran, from what the step's control kernels counted.
long long graph_step_launches(const pfc_state* s, const pfc::StepCtl& c) {
  const int m = c.m;
  const bool chunked = s->dim == 2 && s->fs.variant == pfc::kChunkedVariant;
  long long n = 4 + (c.commit_go ? 3 : 0);               // residual, reduce, begin, end; commit
  n += 6LL * m;                                          // per Newton iteration
  n += (long long)c.n_factor * (2 + (chunked ? 1 : 0));  // factor (+ records), done
  n += 4LL * c.n_cycles + 5LL * c.n_restarts + 3LL * c.n_trials;
  n += (long long)c.gm_total * arnoldi_body_kernels(s) + 2LL * c.n_reorth;
  return n;
}

bool graph_ready(const pfc_state* s) {
  return s->p.use_graph && s->dim == 2 && s->st != nullptr && !s->prof && !s->graph_failed &&
         (s->tuned || s->p.apply_variant >= 0);
}

// Captures s's step graph (helper streams created on first use); false if it cannot be built.
bool build_step_graph(pfc_state* s) {
  for (cudaStream_t& c : s->cs)
    if (!c && cudaStreamCreateWithFlags(&c, cudaStreamNonBlocking) != cudaSuccess) return false;
  pfc::count_pause(true);  // the capture launches nothing; replays are counted from StepCtl
  bool ok = cudaStreamBeginCapture(s->st, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
  if (ok) ok = emit_step_graph(s);
  cudaGraph_t g = nullptr;
  ok = cudaStreamEndCapture(s->st, &g) == cudaSuccess && ok && g;
  pfc::count_pause(false);
  cudaGraphExec_t ge = nullptr;
  if (ok) ok = cudaGraphInstantiate(&ge, g, 0) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    if (ge) cudaGraphExecDestroy(ge);
    if (g) cudaGraphDestroy(g);
    return false;
  }
  s->sgraph = g;
  s->sexec = ge;
  return true;
}

// The step's inputs in StepCtl: 1/dt, the stop-test reference, the tolerances, refactor.
int write_ctl_inputs(pfc_state* s, double dt, bool refactor) {
  pfc::StepCtl* c = s->sc_h;
  const pfc_params& p = s->p;
  c->idt = 1.0 / dt;
  c->ref_norm = s->ref_norm;
  c->newton_rtol = p.newton_rtol;
  c->newton_atol = p.newton_atol;
  c->gmres_rtol = p.gmres_rtol;
  c->gmres_atol = p.gmres_atol;
  c->ls_alpha = p.ls_alpha;
  c->reorth_eta2 = p.gmres_reorth_eta * p.gmres_reorth_eta;
  c->newton_max_it = p.newton_max_it;
  c->ls_max_cuts = p.ls_max_cuts;
  c->gmres_max_it = p.gmres_max_it;
  c->refactor = refactor ? 1 : 0;
  CU(cudaMemcpyAsync(s->sc, c, offsetof(pfc::StepCtl, r0), cudaMemcpyHostToDevice, s->st));
  return PFC_OK;
}

// Whether this step factors the subdomain matrices (or reuses those of an earlier step at the
// same dt, reuse_factor).
bool needs_factor(pfc_state* s, double dt) {
  const pfc_params& p = s->p;
  return !(p.reuse_factor > 0 && s->factors_ok && s->factor_age < p.reuse_factor &&
           std::fabs(dt / s->factor_dt - 1.0) <= 1e-3);
}

// One Newton solve from the guess in s->Phi, by the graph or by the host; on success phi^n and
// phi^{n-1} have been advanced on the device and red[4..5] hold E and M of the new phi^n.
int newton(pfc_state* s, double dt, pfc_step_info* info) {
  const bool refactor = needs_factor(s, dt);
  int rc = write_ctl_inputs(s, dt, refactor);
  if (rc) return rc;
  bool graph = graph_ready(s);
  if (graph && !s->sexec && !build_step_graph(s)) {
    s->graph_failed = true;
    graph = false;
  }
  if (graph) {
    CU(cudaGraphLaunch(s->sexec, s->st));
    pfc::count_graph_launch();
    CU(cudaMemcpyAsync(s->red_h + 4, s->red + 4, 2 * sizeof(double), cudaMemcpyDeviceToHost, s->st));
    if ((rc = read_ctl(s))) return rc;
    pfc::count_launches(graph_step_launches(s, *s->sc_h));
  } else {
    if ((rc = step_host(s, dt))) return rc;
    if (s->sc_h->commit_go && (rc = sync_read(s, s->red_h + 4, s->red + 4, 2 * sizeof(double)))) return rc;
  }
  const pfc::StepCtl& c = *s->sc_h;
  if (refactor && c.n_factor > 0) {  // factors of this dt, reusable while it lasts
    s->factors_ok = c.status != PFC_ESINGULAR;
    s->factor_dt = dt;
    s->factor_age = 0;
  } else if (!refactor) {
    ++s->factor_age;
  }
  info->newton_its = c.m;
  info->gmres_its = c.gm_total;
  info->ls_cuts = c.cuts_total;
  info->res_norm0 = c.r0;
  info->res_norm = c.rnorm;
  return c.status;
}

int energy_mass(pfc_state* s, const double* phi, double* E, double* M);

// Safeguarded initial guess.  Candidates: phi^n (the paper's start, Sec. 4), the
// extrapolation Phi_E = phi^n + c1, c1 = (dt / dt_prev)(phi^n - phi^{n-1}), and in
// the learned form Phi_L = phi^n + c1 + s_out net(c) shifted to the mass of phi^n.
// Newton starts from the candidate with the smallest ||F|| (ties keep Phi_E, then
// phi^n): a step-size jump makes c1 large, and the extrapolation can then be far
// worse than phi^n.  Leaves the choice in s->Phi.
int safeguarded_guess(pfc_state* s, double dt, bool learned, int* used) {
  const long long N = s->g.n;
  const double idt = 1.0 / dt;
  int rc = PFC_OK;
  if (learned) {
    if ((rc = energy_mass(s, s->phin, nullptr, nullptr))) return rc;  // red[5] = sum phi^n
    pfc::launch_cnn_features(N, s->phin, s->phinm1, s->red + 5, dt / s->dt_prev, dt / s->p.dt_max, s->feat, s->st);
    pfc::Cnn* c = reinterpret_cast<pfc::Cnn*>(s->cnn);
    const cudaStream_t own = pfc::cnn_swap_stream(c, s->st);  // the forward pass joins the step's stream
    pfc::cnn_forward(c, s->feat);
    pfc::cnn_swap_stream(c, own);
    int np = 0;
    pfc::launch_cnn_delta(N, s->feat, pfc::cnn_output(c), s->s_out, s->W, s->partial, &np, s->st);
    pfc::launch_reduce(s->partial, 1, np, s->red + 11, s->st);
    pfc::launch_add_centered(N, s->phin, s->W, s->red + 11, s->Pt, s->st);  // Phi_L
    if ((rc = eval_residual(s, s->Pt, nullptr, 0.0, false, s->phin, idt, s->Ft, nullptr, nullptr, 2))) return rc;
  }
  pfc::launch_extrapolate(s->Phi, s->phin, s->phinm1, dt / s->dt_prev, N, s->st);  // Phi_E
  if ((rc = eval_residual(s, s->Phi, nullptr, 0.0, false, s->phin, idt, s->Ft, nullptr, nullptr, 3))) return rc;
  if ((rc = eval_residual(s, s->phin, nullptr, 0.0, false, s->phin, idt, s->Ft, nullptr, nullptr, 6))) return rc;
  if ((rc = sync_read(s, s->red_h + 2, s->red + 2, 5 * sizeof(double)))) return rc;
  if (learned) {
    pfc::Cnn* c = reinterpret_cast<pfc::Cnn*>(s->cnn);
    const cudaStream_t own = pfc::cnn_swap_stream(c, s->st);
    rc = pfc::cnn_status(c);
    pfc::cnn_swap_stream(c, own);
    if (rc) return rc;
  }
  const double rl = learned ? s->red_h[2] : NAN, re = s->red_h[3], rp = s->red_h[6];
  s->ref_norm = std::sqrt(rp);
  double best = re;
  *used = PFC_GUESS_EXTRAP;
  if (rp < best) {
    best = rp;
    *used = PFC_GUESS_PREV;
  }
  if (rl == rl && rl < best) *used = PFC_GUESS_LEARNED;
  if (*used == PFC_GUESS_LEARNED) CU(cudaMemcpyAsync(s->Phi, s->Pt, sizeof(double) * N, cudaMemcpyDeviceToDevice, s->st));
  if (*used == PFC_GUESS_PREV) CU(cudaMemcpyAsync(s->Phi, s->phin, sizeof(double) * N, cudaMemcpyDeviceToDevice, s->st));
  return PFC_OK;
}

// ---- batched steps of independent states (pfc_run_batch): one captured graph holds every
// state's step graph as a parallel branch, so one graph launch steps the whole ensemble.
struct BatchGraph {
  cudaStream_t st = nullptr;
  cudaEvent_t fork = nullptr;
  std::vector<cudaEvent_t> join;
  cudaGraph_t g = nullptr;
  cudaGraphExec_t ge = nullptr;
};

// States that can share a batch graph: 2D, graph form on, the paper's phi^n guess, one device,
// distinct streams other than the legacy default stream.
bool batch_graph_ok(pfc_state** states, int count) {
  if (count < 2) return false;
  for (int i = 0; i < count; ++i) {
    const pfc_state* s = states[i];
    if (s->dim != 2 || !s->p.use_graph || s->st == nullptr || s->prof || s->graph_failed ||
        s->p.guess != PFC_GUESS_PREV || s->p.reuse_factor != 0 || s->device != states[0]->device)
      return false;
    for (int k = 0; k < i; ++k)
      if (states[k]->st == s->st) return false;
  }
  return true;
}

bool all_graph_ready(pfc_state** states, int count, const std::vector<int>& rc) {
  for (int i = 0; i < count; ++i)
    if (rc[i] == PFC_OK && !graph_ready(states[i])) return false;
  return true;
}

void destroy_batch_graph(BatchGraph* b) {
  if (b->ge) cudaGraphExecDestroy(b->ge);
  if (b->g) cudaGraphDestroy(b->g);
  for (cudaEvent_t e : b->join)
    if (e) cudaEventDestroy(e);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->st) cudaStreamDestroy(b->st);
  *b = BatchGraph();
}

// One state's branch of a batch graph, queued on s->st (being captured): a while loop over its
// time steps -- the step's dt from Eq. (sencondt) on the device, Phi_0 = phi^n, the whole step
// graph, then record, retry with dt / 2 or stop -- so that every state advances through its
// own steps, however long its Newton and GMRES iterations take, within one graph launch.
bool emit_time_loop(pfc_state* s) {
  if (!new_handle(s->st, &s->hs.mloop)) return false;
  pfc::launch_mloop_begin(s->sc, s->hs, s->st);
  cudaGraph_t body;
  return add_cond(s->st, s->hs.mloop, cudaGraphCondTypeWhile, &body) &&
         capture_body(s, body, s->cs[0], [&] {
           pfc::launch_mstep_prep(s->sc, s->st);
           if (cudaMemcpyAsync(s->Phi, s->phin, sizeof(double) * s->g.n, cudaMemcpyDeviceToDevice, s->st) !=
               cudaSuccess)
             return false;
           if (!emit_step_graph(s, 1)) return false;
           pfc::launch_mstep_end(s->sc, s->red + 4, s->recs, s->hs, s->st);
           return cudaGetLastError() == cudaSuccess;
         });
}

// Captures every state's time loop into one graph: the batch stream forks into each state's
// stream, which records its loop (nested bodies on its own helper streams), and joins back.
int build_batch_graph(pfc_state** states, int count, BatchGraph* b) {
  CU(cudaSetDevice(states[0]->device));
  CU(cudaStreamCreateWithFlags(&b->st, cudaStreamNonBlocking));
  CU(cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming));
  b->join.assign(count, nullptr);
  for (int i = 0; i < count; ++i) {
    CU(cudaEventCreateWithFlags(&b->join[i], cudaEventDisableTiming));
    CU(cudaStreamSynchronize(states[i]->st));
    for (cudaStream_t& c : states[i]->cs)
      if (!c) CU(cudaStreamCreateWithFlags(&c, cudaStreamNonBlocking));
  }
  pfc::count_pause(true);
  bool ok = cudaStreamBeginCapture(b->st, cudaStreamCaptureModeThreadLocal) == cudaSuccess &&
            cudaEventRecord(b->fork, b->st) == cudaSuccess;
  for (int i = 0; i < count && ok; ++i) {
    pfc_state* s = states[i];
    ok = cudaStreamWaitEvent(s->st, b->fork, 0) == cudaSuccess && emit_time_loop(s) &&
         cudaEventRecord(b->join[i], s->st) == cudaSuccess && cudaStreamWaitEvent(b->st, b->join[i], 0) == cudaSuccess;
  }
  cudaGraph_t g = nullptr;
  ok = cudaStreamEndCapture(b->st, &g) == cudaSuccess && ok && g;
  pfc::count_pause(false);
  b->g = g;
  if (ok) ok = cudaGraphInstantiate(&b->ge, g, 0) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    return PFC_ECUDA;
  }
  return PFC_OK;
}

// k steps of every live state with one graph launch: each state's branch runs its own time loop
// on the device (controller, retries with dt / 2 as pfc_run does, records).  The host uploads the
// states' controller state and tolerances, launches once, and reads back the control blocks and
// records.  Records of state i go to rec[i * stride + t], t < its steps done (and its failure).
int batch_chunk(pfc_state** states, int count, BatchGraph* b, std::vector<int>& rc, pfc_step_info* rec, int stride,
                int k) {
  for (int i = 0; i < count; ++i) {
    pfc_state* s = states[i];
    pfc::StepCtl* c = s->sc_h;
    memset(c, 0, sizeof(*c));
    c->ref_norm = -1.0;
    c->newton_rtol = s->p.newton_rtol;
    c->newton_atol = s->p.newton_atol;
    c->gmres_rtol = s->p.gmres_rtol;
    c->gmres_atol = s->p.gmres_atol;
    c->ls_alpha = s->p.ls_alpha;
    c->reorth_eta2 = s->p.gmres_reorth_eta * s->p.gmres_reorth_eta;
    c->newton_max_it = s->p.newton_max_it;
    c->ls_max_cuts = s->p.ls_max_cuts;
    c->gmres_max_it = s->p.gmres_max_it;
    c->refactor = 1;
    c->E_n = s->E_n;
    c->E_nm1 = s->E_nm1;
    c->dt_prev = s->dt_prev;
    c->have_Em1 = s->have_Em1;
    c->have_prev_dt = s->have_prev_dt;
    c->dt_min = s->p.dt_min;
    c->dt_max = s->p.dt_max;
    c->eta = s->p.eta;
    c->escale = s->p.energy_scaled ? 1.0 / (s->g.hd * (double)s->g.n) : 1.0;
    c->hd = s->g.hd;
    c->steps_target = rc[i] == PFC_OK ? k : 0;
    c->dt_halvings = s->p.dt_halvings;
    c->body_kernels = arnoldi_body_kernels(s);
    c->chunked = s->fs.variant == pfc::kChunkedVariant;
    CU(cudaMemcpyAsync(s->sc, c, sizeof(*c), cudaMemcpyHostToDevice, b->st));
  }
  CU(cudaGraphLaunch(b->ge, b->st));
  pfc::count_graph_launch();
  std::vector<std::vector<pfc_step_info>> recs(count);
  for (int i = 0; i < count; ++i) {
    pfc_state* s = states[i];
    recs[i].resize(k);
    CU(cudaMemcpyAsync(s->sc_h, s->sc, sizeof(pfc::StepCtl), cudaMemcpyDeviceToHost, b->st));
    CU(cudaMemcpyAsync(recs[i].data(), s->recs, sizeof(pfc_step_info) * k, cudaMemcpyDeviceToHost, b->st));
  }
  CU(cudaStreamSynchronize(b->st));
  for (int i = 0; i < count; ++i) {
    pfc_state* s = states[i];
    const pfc::StepCtl& c = *s->sc_h;
    pfc::count_launches(c.kernels + 1);  // the loop's kernels and its first loop test
    if (rc[i] != PFC_OK) continue;
    s->E_n = c.E_n;
    s->E_nm1 = c.E_nm1;
    s->dt_prev = c.dt_prev;
    s->have_Em1 = c.have_Em1 != 0;
    s->have_prev_dt = c.have_prev_dt != 0;
    s->factors_ok = false;  // the loop refactors every step
    const int done = c.steps_done + (c.failed ? 1 : 0);
    if (rec)
      for (int t = 0; t < done && t < k; ++t) rec[(size_t)i * stride + t] = recs[i][t];
    if (c.failed) rc[i] = c.failed;
  }
  return PFC_OK;
}

int energy_mass(pfc_state* s, const double* phi, double* E, double* M) {
  int np = 0;
  if (s->dim == 2)
    pfc::launch_energy2d(s->g, phi, s->partial, &np, s->st);
  else
    pfc::launch_energy3d(s->g, phi, s->partial, &np, s->st);
  pfc::launch_reduce(s->partial, 2, np, s->red + 4, s->st);
  CU(cudaGetLastError());
  int rc = sync_read(s, s->red_h + 4, s->red + 4, 2 * sizeof(double));
  if (rc) return rc;
  if (E) *E = s->red_h[4] * s->g.hd;
  if (M) *M = s->red_h[5] * s->g.hd;
  return PFC_OK;
}

}  // namespace

extern "C" {

int pfc_default_params(pfc_params* p) {
  if (!p) return PFC_EINVAL;
  memset(p, 0, sizeof(*p));
  p->newton_rtol = 1e-10;
  p->newton_atol = 0.0;
  p->newton_max_it = 50;
  p->gmres_rtol = 1e-6;
  p->gmres_atol = 0.0;
  p->gmres_restart = 30;
  p->gmres_max_it = 10000;
  p->sub[0] = p->sub[1] = p->sub[2] = 1;
  p->overlap = 1;
  p->ras_kind = PFC_LEFT_RAS;
  p->factor_prec = PFC_F64;
  p->guess = PFC_GUESS_PREV;
  p->mass_projection = 1;
  p->ls_alpha = 1e-4;
  p->ls_max_cuts = 10;
  p->dt_min = 1e-2;
  p->dt_max = 10.0;
  p->eta = 5000.0;
  p->energy_scaled = 1;
  p->apply_variant = -1;
  p->gmres_reorth_eta = 0.3;
  p->use_graph = 1;
  p->reuse_factor = 0;
  p->mobility = 0;
  return PFC_OK;
}

int pfc_workspace_size(const pfc_grid* g, const pfc_params* p, size_t* bytes) {
  if (!bytes) return PFC_EINVAL;
  Plan pl;
  int rc = make_plan(g, p, &pl);
  if (rc) return rc;
  *bytes = pl.total;
  return PFC_OK;
}

int pfc_block_layout(const pfc_grid* g, const pfc_params* p, int* out, int cap, int* nblocks) {
  if (!nblocks || cap < 0 || (cap > 0 && !out)) return PFC_EINVAL;
  int rc = validate(g, p);
  if (rc) return rc;
  std::vector<BlockDesc> blocks;
  int n_max = 0, kl_max = 0;
  build_blocks(g, p, &blocks, &n_max, &kl_max);
  static_assert(sizeof(BlockDesc) == 12 * sizeof(int), "BlockDesc is 12 ints");
  for (int k = 0; k < cap && k < (int)blocks.size(); ++k) memcpy(out + 12 * k, &blocks[k], sizeof(BlockDesc));
  *nblocks = (int)blocks.size();
  return PFC_OK;
}

int pfc_create(const pfc_grid* g, double h, double eps, const pfc_params* p, void* ws, size_t bytes,
               void* cuda_stream, pfc_state** out) {
  if (!out || !ws || !(h > 0.0) || !std::isfinite(h) || !std::isfinite(eps)) return PFC_EINVAL;
  *out = nullptr;
  Plan pl;
  int rc = make_plan(g, p, &pl);
  if (rc) return rc;
  if (bytes < pl.total) return PFC_ENOMEM;
  if (((uintptr_t)ws & 255) != 0) return PFC_EINVAL;
  pfc_state* s = new (std::nothrow) pfc_state();
  if (!s) return PFC_ENOMEM;
  s->grid = *g;
  s->p = *p;
  s->h = h;
  s->gamma = eps;
  s->dim = g->dim;
  s->st = (cudaStream_t)cuda_stream;
  s->g.nx = (int)g->n[0];
  s->g.ny = (int)g->n[1];
  s->g.nz = g->dim == 3 ? (int)g->n[2] : 1;
  s->g.n = (long long)s->g.nx * s->g.ny * s->g.nz;
  s->g.ih2 = 1.0 / (h * h);
  s->g.gamma = eps;
  s->g.hd = g->dim == 3 ? h * h * h : h * h;
  s->g.neumann = p->boundary == PFC_NEUMANN ? 1 : 0;
  pfc::geo_constants(&s->g);
  char* base = (char*)ws;
  auto at = [&](size_t off) { return (void*)(base + off); };
  s->phin = (double*)at(pl.phin);
  s->phinm1 = (double*)at(pl.phinm1);
  s->Phi = (double*)at(pl.Phi);
  s->F = (double*)at(pl.F);
  s->q = (double*)at(pl.q);
  s->Pt = (double*)at(pl.Pt);
  s->Ft = (double*)at(pl.Ft);
  s->qt = (double*)at(pl.qt);
  s->S = (double*)at(pl.S);
  s->W = (double*)at(pl.W);
  s->guess = (double*)at(pl.guess);
  s->Vbuf = (double*)at(pl.V);
  s->Zbuf = (double*)at(pl.Z);
  s->vstride = basis_stride(s->g.n);
  s->fs.L = at(pl.L);
  s->fs.U = at(pl.U);
  s->fs.piv = (uint8_t*)at(pl.piv);
  s->fs.strideL = pl.sL;
  s->fs.strideU = pl.sU;
  s->fs.strideP = pl.sP;
  s->fs.lrow = pl.lrow;
  s->fs.ucol = pl.ucol;
  s->fs.X = (unsigned char*)at(pl.X);
  s->fs.ras_kind = p->ras_kind;
  if (p->mobility) {
    s->mu = (double*)at(pl.mu);
    s->mut = (double*)at(pl.mut);
    s->sm = (double*)at(pl.smid);
    s->smt = (double*)at(pl.smidt);
    int em = 0;
    std::vector<BlockDesc> bl;
    int nm0, km0;
    build_blocks(g, p, &bl, &nm0, &km0);
    for (const BlockDesc& b : bl) em = std::max(em, (b.bx + 2) * (b.by + 2));
    s->fs.ext_max = em;
  }
  s->fs.mob_mu = nullptr;
  s->fs.mob_s = nullptr;
  s->r3.mob_mu = nullptr;
  s->r3.mob_s = nullptr;
  s->fs.Yb = (double*)at(pl.Yb);
  if (g->dim == 2) {
    s->dc.px = p->sub[0];
    s->dc.py = p->sub[1];
    s->dc.ov = p->overlap;
    s->dc.base_x = (int)(g->n[0] / p->sub[0]);
    s->dc.rem_x = (int)(g->n[0] % p->sub[0]);
    s->dc.base_y = (int)(g->n[1] / p->sub[1]);
    s->dc.rem_y = (int)(g->n[1] % p->sub[1]);
  }
  s->fs.xfw = pl.xfw;
  s->fs.xbw = pl.xbw;
  s->fs.xnc = pl.xnc;
  s->fs.nblk = pl.nblocks;
  s->fs.xstage = pl.xstage;
  s->fs.x_valid = 0;
  s->fs.prec = p->factor_prec;
  s->fs.kl_max = pl.kl_max;
  s->fs.n_max = pl.n_max;
  s->fs.variant = p->apply_variant >= 0 ? p->apply_variant : 0;
  s->tuned = false;
  if (p->ras_kind != PFC_LEFT_RAS) {  // AS / right-RAS: the chunked apply only
    s->fs.variant = pfc::kChunkedVariant;
    s->tuned = true;
  }
  s->ref_norm = -1.0;
  if (cudaGetDevice(&s->device) != cudaSuccess) {
    pfc_destroy(s);
    return PFC_ECUDA;
  }
  for (int v = 0; v < pfc::kApplyVariants; ++v) s->tune_ms[v] = -1.f;
  s->nblocks = pl.nblocks;
  s->blocks_dev = (BlockDesc*)at(pl.blocks);
  s->lin_dev = (double*)at(pl.lin);
  s->ctl = (GmresCtl*)at(pl.ctl);
  s->partial = (double*)at(pl.partial);
  s->red = (double*)at(pl.red);
  s->status_dev = (int*)at(pl.status);
  s->feat = g->dim == 2 ? (double*)at(pl.feat) : nullptr;
  s->ia = (pfc::IterArgs*)at(pl.iargs);
  s->ia2 = (pfc::IterArgs*)at(pl.iargs2);
  s->sc = (pfc::StepCtl*)at(pl.sctl);
  s->recs = (pfc_step_info*)at(pl.recs);
  s->fs.order = (const int*)at(pl.order);
  if (cudaMallocHost((void**)&s->ctl_h, sizeof(GmresCtl)) != cudaSuccess ||
      cudaMallocHost((void**)&s->ctl_hb[0], sizeof(GmresCtl)) != cudaSuccess ||
      cudaMallocHost((void**)&s->ctl_hb[1], sizeof(GmresCtl)) != cudaSuccess ||
      cudaEventCreateWithFlags(&s->ctl_ev[0], cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&s->ctl_ev[1], cudaEventDisableTiming) != cudaSuccess ||
      cudaMallocHost((void**)&s->red_h, 16 * sizeof(double)) != cudaSuccess ||
      cudaMallocHost((void**)&s->status_h, 4 * sizeof(int)) != cudaSuccess ||
      cudaMallocHost((void**)&s->sc_h, sizeof(pfc::StepCtl)) != cudaSuccess) {
    pfc_destroy(s);
    return PFC_ECUDA;
  }
  std::vector<BlockDesc> blocks;
  int nm, km;
  build_blocks(g, p, &blocks, &nm, &km);
  // two-subdomains-per-warp order: blocks grouped by extent, each group padded to an even count with -1,
  // so the first slot of every warp is a real block and both slots of a warp share the extent
  std::vector<int> order;
  {
    std::vector<int> idx(blocks.size());
    for (size_t i = 0; i < idx.size(); ++i) idx[i] = (int)i;
    std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) {
      return std::make_pair(blocks[a].by, blocks[a].bx) < std::make_pair(blocks[b].by, blocks[b].bx);
    });
    for (size_t i = 0; i < idx.size(); ++i) {
      order.push_back(idx[i]);
      const bool last = i + 1 == idx.size() || blocks[idx[i + 1]].bx != blocks[idx[i]].bx ||
                        blocks[idx[i + 1]].by != blocks[idx[i]].by;
      if (last && order.size() % 2) order.push_back(-1);
    }
  }
  s->fs.norder = (int)order.size();
  {  // algorithmic work of the Schwarz kernels, per launch
    const double es = p->factor_prec == PFC_F64 ? 8.0 : (p->factor_prec == PFC_F32 ? 4.0 : 2.0);
    double bytes = 0.0, bytes_step = 0.0, bytes_chunk = 0.0, fflops = 0.0, fbytes = 0.0, rbytes = 0.0;
    std::vector<int> upd3, upd3_n;
    if (g->dim == 3) update_lists(&upd3, &upd3_n);
    for (const BlockDesc& b : blocks) {
      const double core = (double)b.cx * b.cy * b.cz * 8.0;
      if (g->dim == 2) {
        // the method's band LU with partial pivoting: step k has min(kl, n-1-k) multipliers and
        // U row k min(ku2, n-1-k) entries right of the diagonal (ku2 = 2 kl with the pivots' fill)
        const int n = b.bx * b.by;
        const int kl = std::min(3 * b.bx, n - 1), ku2 = std::min(2 * kl, n - 1);
        double entries = 0.0, fl = 0.0;
        for (int k = 0; k < n; ++k) {
          const int r = std::min(kl, n - 1 - k), c = std::min(ku2, n - 1 - k);
          entries += r + c + 1;
          fl += r + 2.0 * r * c;  // multipliers, then the rank-1 update of the window
        }
        bytes += entries * es + n * 1.0 + n * 8.0 + core;  // band entries, pivots, gather of r, core of z
        bytes_step += (double)n * (kl + ku2 + 1) * es + n * 1.0 + n * 8.0 + core;
        const pfc::ChunkGeom cg = pfc::chunk_geom(b.bx, b.by, (int)es, p->factor_prec == PFC_F64 ? 8 : 4);
        bytes_chunk += (double)cg.nc * (cg.fwd + cg.bwd) + n * 8.0 + core;
        fflops += fl;
        fbytes += entries * es + n * 1.0 + (double)(b.bx + 6) * (b.by + 6) * 8.0;  // factors out, q in
        rbytes += (double)n * (pl.lrow + pl.ucol) * es + n + (double)cg.nc * (cg.fwd + cg.bwd);
      } else {  // ILU(0): 63 entries per row (64 stored), gather, core write
        const double n = (double)b.bx * b.by * b.bz;
        bytes += n * 63.0 * es + n * 8.0 + core;
        bytes_step += n * 64.0 * es + n * 8.0 * 2 + core;
        double per_row = 0.0;
        for (int o = 0; o < 31; ++o) per_row += 1.0 + 2.0 * upd3_n[o];  // multiplier + row updates
        fflops += n * per_row;
        fbytes += n * 64.0 * es + (double)(b.bx + 6) * (b.by + 6) * (b.bz + 6) * 8.0;
      }
    }
    s->apply_bytes = bytes;
    s->apply_bytes_step = bytes_step;
    s->apply_bytes_chunk = bytes_chunk;
    s->factor_flops = fflops;
    s->factor_bytes = fbytes;
    s->record_bytes = rbytes;
  }
  if (g->dim == 3) {
    const Shapes3& S = pl.sh3;
    s->T1 = (double*)at(pl.T1);
    s->T2 = (double*)at(pl.T2);
    pfc::Ras3D& R = s->r3;
    R.shapes = (const pfc::Shape3*)at(pl.shapes);
    R.block_shape = (const int*)at(pl.block_shape);
    R.lev_start = (const int*)at(pl.lev_start);
    R.rowpad = (const int*)at(pl.rowpad);
    R.rowabc = (const int*)at(pl.rowabc);
    R.posL = (const uint8_t*)at(pl.posL);
    R.posU = (const uint8_t*)at(pl.posU);
    R.Lp = at(pl.Lp);
    R.Up = at(pl.Up);
    R.work = at(pl.work);
    R.ypad = at(pl.ypad);
    R.sLU = pl.sLU3;
    R.sWork = pl.sWork3;
    R.sPad = pl.sPad3;
    R.prec = p->factor_prec;
    R.max_level_rows = S.max_level_rows;
    R.max_nlev = 0;
    for (const pfc::Shape3& sh : S.shapes) R.max_nlev = std::max(R.max_nlev, sh.nlev);
    R.window = 0;
    if (p->apply_variant != 0) {  // -1: the window kernel where it fits; 1: only the window kernel
      R.window = pfc::apply3d_window_ok(R) ? 1 : 0;
      if (p->apply_variant == 1 && !R.window) {
        pfc_destroy(s);
        return PFC_EINVAL;
      }
    }
    s->fs.variant = R.window;  // reported by pfc_get_tuning
    R.shift = 0.1;  // fraction of the block's mean |a_ii| added to the diagonal before ILU(0)
    const size_t tc = p->factor_prec == PFC_F64 ? 8 : 4;
    auto put = [&](const void* dst, const void* src, size_t bytes) {
      return cudaMemcpyAsync((void*)dst, src, bytes, cudaMemcpyHostToDevice, s->st) == cudaSuccess;
    };
    if (!put(R.shapes, S.shapes.data(), sizeof(pfc::Shape3) * S.shapes.size()) ||
        !put(R.block_shape, S.block_shape.data(), sizeof(int) * S.block_shape.size()) ||
        !put(R.lev_start, S.lev_start.data(), sizeof(int) * S.lev_start.size()) ||
        !put(R.rowpad, S.rowpad.data(), sizeof(int) * S.rowpad.size()) ||
        !put(R.rowabc, S.rowabc.data(), sizeof(int) * S.rowabc.size()) ||
        !put(R.posL, S.posL.data(), S.posL.size()) || !put(R.posU, S.posU.data(), S.posU.size()) ||
        cudaMemsetAsync(R.ypad, 0, pl.sPad3 * tc * pl.nblocks, s->st) != cudaSuccess ||
        cudaStreamSynchronize(s->st) != cudaSuccess) {
      pfc_destroy(s);
      return PFC_ECUDA;
    }
  }
  double lin343[343], lin49[49];
  lin_stencil(g->dim, h, eps, lin343, lin49);
  const double* lin = g->dim == 2 ? lin49 : lin343;
  const size_t lin_bytes = sizeof(double) * (g->dim == 2 ? 49 : 343);
  s->vtab = (const double**)at(pl.tabs);
  s->ztab = s->vtab + pfc::kMaxVecs;
  std::vector<const double*> tabs(2 * pfc::kMaxVecs, nullptr);
  for (int i = 0; i <= p->gmres_restart; ++i) tabs[i] = s->Vbuf + (size_t)i * s->vstride;
  for (int i = 0; i < p->gmres_restart; ++i) tabs[pfc::kMaxVecs + i] = s->Zbuf + (size_t)i * s->vstride;
  // iteration arguments whose pointers never change (q, the mobility fields; the restart's S -> W)
  pfc::IterArgs ia0{}, ia20{};
  ia0.q = ia20.q = s->q;
  ia0.mu = ia20.mu = s->mu;
  ia0.sm = ia20.sm = s->sm;
  ia20.z = s->S;
  ia20.w = s->W;
  ia0.zplane = ia20.zplane = -1;
  if (g->dim == 2 && !p->mobility) pfc::encode_jvp_maps(s->g, s->Zbuf, s->vstride, p->gmres_restart, s->q, &s->jmaps);
  if (cudaMemcpyAsync(s->ia, &ia0, sizeof ia0, cudaMemcpyHostToDevice, s->st) != cudaSuccess ||
      cudaMemcpyAsync(s->ia2, &ia20, sizeof ia20, cudaMemcpyHostToDevice, s->st) != cudaSuccess ||
      cudaMemsetAsync(s->sc, 0, sizeof(pfc::StepCtl), s->st) != cudaSuccess ||
      cudaMemcpyAsync(s->blocks_dev, blocks.data(), sizeof(BlockDesc) * blocks.size(), cudaMemcpyHostToDevice,
                      s->st) != cudaSuccess ||
      cudaMemcpyAsync((void*)s->fs.order, order.data(), sizeof(int) * order.size(), cudaMemcpyHostToDevice, s->st) !=
          cudaSuccess ||
      cudaMemcpyAsync(s->lin_dev, lin, lin_bytes, cudaMemcpyHostToDevice, s->st) != cudaSuccess ||
      cudaMemcpyAsync((void*)s->vtab, tabs.data(), sizeof(double*) * tabs.size(), cudaMemcpyHostToDevice, s->st) !=
          cudaSuccess ||
      cudaMemsetAsync(s->phin, 0, sizeof(double) * s->g.n, s->st) != cudaSuccess ||
      cudaMemsetAsync(s->phinm1, 0, sizeof(double) * s->g.n, s->st) != cudaSuccess ||
      cudaMemsetAsync(s->red, 0, sizeof(double) * 16, s->st) != cudaSuccess ||
      cudaMemsetAsync(s->status_dev, 0, sizeof(int) * 4, s->st) != cudaSuccess ||
      cudaStreamSynchronize(s->st) != cudaSuccess) {
    pfc_destroy(s);
    return PFC_ECUDA;
  }
  *out = s;
  return PFC_OK;
}

int pfc_get_tuning(const pfc_state* s, int* apply_variant, float* apply_ms, int* graph) {
  if (!s || !apply_variant) return PFC_EINVAL;
  *apply_variant = s->fs.variant;
  if (graph) *graph = s->sexec != nullptr;
  if (apply_ms)
    for (int v = 0; v < pfc::kApplyVariants; ++v) apply_ms[v] = s->tune_ms[v];
  return PFC_OK;
}

void pfc_destroy(pfc_state* s) {
  if (!s) return;
  pfc_profile(s, 0);
  if (s->ctl_h) cudaFreeHost(s->ctl_h);
  for (int b = 0; b < 2; ++b) {
    if (s->ctl_hb[b]) cudaFreeHost(s->ctl_hb[b]);
    if (s->ctl_ev[b]) cudaEventDestroy(s->ctl_ev[b]);
  }
  if (s->red_h) cudaFreeHost(s->red_h);
  if (s->status_h) cudaFreeHost(s->status_h);
  if (s->sc_h) cudaFreeHost(s->sc_h);
  if (s->sexec) cudaGraphExecDestroy(s->sexec);
  if (s->sgraph) cudaGraphDestroy(s->sgraph);
  for (cudaStream_t c : s->cs)
    if (c) cudaStreamDestroy(c);
  delete s;
}

int pfc_set_field(pfc_state* s, const double* phi, int on_device) {
  if (!s || !phi) return PFC_EINVAL;
  const size_t b = sizeof(double) * s->g.n;
  CU(cudaMemcpyAsync(s->phin, phi, b, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s->st));
  CU(cudaMemcpyAsync(s->phinm1, s->phin, b, cudaMemcpyDeviceToDevice, s->st));
  CU(cudaStreamSynchronize(s->st));
  s->have_E = s->have_Em1 = s->have_prev_dt = s->have_user_guess = false;
  s->factors_ok = false;
  return PFC_OK;
}

// Checkpoint layout: magic, grid (dim, n[3]), h, gamma, the history flags and
// scalars, then phi^n and phi^{n-1} (N doubles each), all in host byte order.
namespace {
constexpr char kCkptMagic[8] = {'P', 'F', 'C', 'C', 'K', 'P', 'T', '1'};
struct CkptHeader {
  char magic[8];
  int32_t dim, pad;
  int64_t n[3];
  double h, gamma;
  int32_t have_E, have_Em1, have_prev_dt, pad2;
  double E_n, E_nm1, dt_prev;
};
}  // namespace

int pfc_save(pfc_state* s, const char* path) {
  if (!s || !path) return PFC_EINVAL;
  CkptHeader hd{};
  memcpy(hd.magic, kCkptMagic, 8);
  hd.dim = s->dim;
  hd.n[0] = s->g.nx;
  hd.n[1] = s->g.ny;
  hd.n[2] = s->g.nz;
  hd.h = s->h;
  hd.gamma = s->gamma;
  hd.have_E = s->have_E;
  hd.have_Em1 = s->have_Em1;
  hd.have_prev_dt = s->have_prev_dt;
  hd.E_n = s->E_n;
  hd.E_nm1 = s->E_nm1;
  hd.dt_prev = s->dt_prev;
  std::vector<double> host((size_t)s->g.n);
  FILE* f = fopen(path, "wb");
  if (!f) return PFC_EINVAL;
  bool ok = fwrite(&hd, sizeof hd, 1, f) == 1;
  for (const double* src : {s->phin, s->phinm1}) {
    if (!ok) break;
    ok = cudaMemcpyAsync(host.data(), src, sizeof(double) * host.size(), cudaMemcpyDeviceToHost, s->st) ==
             cudaSuccess &&
         cudaStreamSynchronize(s->st) == cudaSuccess &&
         fwrite(host.data(), sizeof(double), host.size(), f) == host.size();
  }
  if (fclose(f) != 0) ok = false;
  return ok ? PFC_OK : PFC_EINVAL;
}

int pfc_load(pfc_state* s, const char* path) {
  if (!s || !path) return PFC_EINVAL;
  FILE* f = fopen(path, "rb");
  if (!f) return PFC_EINVAL;
  CkptHeader hd{};
  bool ok = fread(&hd, sizeof hd, 1, f) == 1 && memcmp(hd.magic, kCkptMagic, 8) == 0 && hd.dim == s->dim &&
            hd.n[0] == s->g.nx && hd.n[1] == s->g.ny && hd.n[2] == s->g.nz && hd.h == s->h && hd.gamma == s->gamma;
  std::vector<double> a, b;
  if (ok) {
    a.resize((size_t)s->g.n);
    b.resize((size_t)s->g.n);
    ok = fread(a.data(), sizeof(double), a.size(), f) == a.size() &&
         fread(b.data(), sizeof(double), b.size(), f) == b.size();
  }
  fclose(f);
  if (!ok) return PFC_EINVAL;  // the state is left unchanged
  CU(cudaMemcpyAsync(s->phin, a.data(), sizeof(double) * a.size(), cudaMemcpyHostToDevice, s->st));
  CU(cudaMemcpyAsync(s->phinm1, b.data(), sizeof(double) * b.size(), cudaMemcpyHostToDevice, s->st));
  CU(cudaStreamSynchronize(s->st));
  s->factors_ok = false;
  s->have_E = hd.have_E;
  s->have_Em1 = hd.have_Em1;
  s->have_prev_dt = hd.have_prev_dt;
  s->E_n = hd.E_n;
  s->E_nm1 = hd.E_nm1;
  s->dt_prev = hd.dt_prev;
  s->have_user_guess = false;
  return PFC_OK;
}

int pfc_get_field(pfc_state* s, double* out, int on_device) {
  if (!s || !out) return PFC_EINVAL;
  CU(cudaMemcpyAsync(out, s->phin, sizeof(double) * s->g.n,
                     on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s->st));
  CU(cudaStreamSynchronize(s->st));
  return PFC_OK;
}

int pfc_set_guess(pfc_state* s, const double* guess, int on_device) {
  if (!s || !guess) return PFC_EINVAL;
  CU(cudaMemcpyAsync(s->guess, guess, sizeof(double) * s->g.n,
                     on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s->st));
  s->have_user_guess = true;
  return PFC_OK;
}

int pfc_step(pfc_state* s, double dt, pfc_step_info* info_out) {
  if (!s || !(dt > 0.0) || std::isinf(dt)) return PFC_EINVAL;
  pfc_step_info info{};
  info.dt = dt;
  const size_t b = sizeof(double) * s->g.n;
  // initial guess Phi_0
  int rc = PFC_OK;
  info.guess_used = PFC_GUESS_PREV;
  s->ref_norm = -1.0;
  if ((s->p.guess == PFC_GUESS_EXTRAP || s->p.guess == PFC_GUESS_LEARNED) && s->have_prev_dt) {
    if ((rc = safeguarded_guess(s, dt, s->p.guess == PFC_GUESS_LEARNED && s->cnn, &info.guess_used))) return rc;
  } else if (s->p.guess == PFC_GUESS_USER && s->have_user_guess) {
    CU(cudaMemcpyAsync(s->Phi, s->guess, b, cudaMemcpyDeviceToDevice, s->st));
    info.guess_used = PFC_GUESS_USER;
  } else {
    CU(cudaMemcpyAsync(s->Phi, s->phin, b, cudaMemcpyDeviceToDevice, s->st));
  }
  CU(cudaGetLastError());
  if (!s->have_E) {  // E^n of the first field, for the time-step controller
    if ((rc = energy_mass(s, s->phin, &s->E_n, nullptr))) return rc;
    s->have_E = true;
  }
  // Newton on the device; a converged step also moves phi^n to phi^{n-1} and phi^{n+1} to phi^n
  rc = newton(s, dt, &info);
  s->have_user_guess = false;
  if (rc) {
    info.status = rc;
    if (info_out) *info_out = info;
    return rc;
  }
  const double E = s->red_h[4] * s->g.hd, M = s->red_h[5] * s->g.hd;
  s->E_nm1 = s->E_n;
  s->E_n = E;
  s->have_Em1 = true;
  s->dt_prev = dt;
  s->have_prev_dt = true;
  info.energy = E;
  info.mass = M;
  info.status = PFC_OK;
  if (info_out) *info_out = info;
  return PFC_OK;
}

int pfc_set_guess_net(pfc_state* s, pfc_cnn* c, double s_out) {
  if (!s || s->dim != 2 || !(s_out > 0.0)) return PFC_EINVAL;
  if (c) {
    const pfc::Cnn* cc = reinterpret_cast<const pfc::Cnn*>(c);
    if (pfc::cnn_nx(cc) != s->g.nx || pfc::cnn_ny(cc) != s->g.ny) return PFC_EINVAL;
  }
  s->cnn = c;
  s->s_out = s_out;
  return PFC_OK;
}

int pfc_next_dt(pfc_state* s, double* dt_out) {
  if (!s || !dt_out) return PFC_EINVAL;
  const double area = s->g.hd * (double)s->g.n;
  const double scale = s->p.energy_scaled ? 1.0 / area : 1.0;
  // Eq. (sencondt); the same arithmetic as the batch form's device time loop
  *dt_out = pfc::controller_dt(s->E_n, s->E_nm1, s->dt_prev, scale, s->p.dt_min, s->p.dt_max, s->p.eta,
                               s->have_Em1 && s->have_prev_dt);
  return PFC_OK;
}

int pfc_step_host(pfc_state* s, const double* phin_host, double dt, double* out_host, pfc_step_info* info) {
  if (!s || !phin_host || !out_host) return PFC_EINVAL;
  const size_t b = sizeof(double) * s->g.n;
  CU(cudaMemcpyAsync(s->phin, phin_host, b, cudaMemcpyHostToDevice, s->st));
  int rc = pfc_step(s, dt, info);
  if (rc) return rc;
  CU(cudaMemcpyAsync(out_host, s->phin, b, cudaMemcpyDeviceToHost, s->st));
  CU(cudaStreamSynchronize(s->st));
  return PFC_OK;
}

int pfc_profile(pfc_state* s, int enable) {
  if (!s) return PFC_EINVAL;
  if (enable && !s->prof) {
    s->pev.assign(2 * kProfSlots, nullptr);
    for (cudaEvent_t& e : s->pev) CU(cudaEventCreate(&e));
    s->prof = true;
  } else if (!enable && s->prof) {
    cudaStreamSynchronize(s->st);
    for (cudaEvent_t& e : s->pev)
      if (e) cudaEventDestroy(e);
    s->pev.clear();
    s->prof = false;
  }
  s->ppend.clear();
  memset(s->pk, 0, sizeof(s->pk));
  return PFC_OK;
}

int pfc_profile_kernels(pfc_state* s, pfc_kernel_prof* out, int cap) {
  if (!s || cap < 0 || (cap > 0 && !out)) return PFC_EINVAL;
  if (s->prof && !s->ppend.empty()) {  // launches since the last GMRES cycle ended
    CU(cudaStreamSynchronize(s->st));
    int rc = prof_resolve(s, 1 << 30);
    if (rc) return rc;
  }
  for (int k = 0; k < cap && k < PFC_PROF_KINDS; ++k) out[k] = s->pk[k];
  return PFC_OK;
}

int pfc_launch_counts(long long* kernels, long long* graphs) {
  if (kernels) *kernels = pfc::launches_so_far();
  if (graphs) *graphs = __atomic_load_n(&pfc::g_graph_launches, __ATOMIC_RELAXED);
  return PFC_OK;
}

int pfc_profile_read(pfc_state* s, long long* apply_launches, double* apply_ms, double* apply_bytes,
                     long long* kernel_launches) {
  if (!s) return PFC_EINVAL;
  pfc_kernel_prof pk[PFC_PROF_KINDS];
  int rc = pfc_profile_kernels(s, pk, PFC_PROF_KINDS);
  if (rc) return rc;
  if (apply_launches) *apply_launches = pk[PFC_PROF_APPLY].launches;
  if (apply_ms) *apply_ms = pk[PFC_PROF_APPLY].ms;
  if (apply_bytes) *apply_bytes = s->apply_bytes;
  if (kernel_launches) *kernel_launches = pfc::launches_so_far();
  return PFC_OK;
}

int pfc_run(pfc_state* s, int nsteps, pfc_step_info* per_step) {
  if (!s || nsteps < 0) return PFC_EINVAL;
  for (int n = 0; n < nsteps; ++n) {
    double dt = 0.0;
    pfc_next_dt(s, &dt);
    pfc_step_info info{};
    int rc = PFC_OK, cuts = 0;
    for (;;) {  // a failed step leaves the state unchanged: retry with dt / 2
      rc = pfc_step(s, dt, &info);
      if ((rc == PFC_ENEWTON || rc == PFC_EGMRES) && cuts < s->p.dt_halvings) {
        dt *= 0.5;
        ++cuts;
        continue;
      }
      break;
    }
    info.dt_cuts = cuts;
    if (per_step) per_step[n] = info;
    if (rc) return rc;
  }
  return PFC_OK;
}

int pfc_run_batch(pfc_state** states, int count, int nsteps, pfc_step_info* per_step, int* status) {
  if (!states || count < 1 || nsteps < 0) return PFC_EINVAL;
  for (int i = 0; i < count; ++i) {
    if (!states[i]) return PFC_EINVAL;
    for (int k = 0; k < i; ++k)
      if (states[k] == states[i]) return PFC_EINVAL;
  }
  std::vector<int> rc(count, PFC_OK);
  int n = 0;
  // steps of every live state on host threads (one per state, each on its state's stream); the
  // batch graph takes over once every state can run its step as a graph
  auto threaded_steps = [&](int k) {
    std::vector<std::thread> pool;
    pool.reserve(count);
    for (int i = 0; i < count; ++i)
      pool.emplace_back([&, i]() {
        if (rc[i] != PFC_OK) return;
        if (cudaSetDevice(states[i]->device) != cudaSuccess) {
          rc[i] = PFC_ECUDA;
          return;
        }
        std::vector<pfc_step_info> rec(k);
        rc[i] = pfc_run(states[i], k, rec.data());
        if (per_step)
          for (int t = 0; t < k; ++t) per_step[(size_t)i * nsteps + n + t] = rec[t];
      });
    for (std::thread& t : pool) t.join();
    n += k;
  };
  if (!batch_graph_ok(states, count)) {
    threaded_steps(nsteps);
  } else {
    while (n < nsteps && !all_graph_ready(states, count, rc)) threaded_steps(1);
    if (n < nsteps) {
      BatchGraph bg;
      int brc = build_batch_graph(states, count, &bg);
      while (brc == PFC_OK && n < nsteps) {
        const int k = std::min(kBatchRecs, nsteps - n);
        brc = batch_chunk(states, count, &bg, rc, per_step ? per_step + n : nullptr, nsteps, k);
        n += k;
      }
      destroy_batch_graph(&bg);
      if (brc != PFC_OK) return brc;
    }
  }
  int first = PFC_OK;
  for (int i = 0; i < count; ++i) {
    if (status) status[i] = rc[i];
    if (first == PFC_OK) first = rc[i];
  }
  return first;
}

int pfc_energy(pfc_state* s, double* F) {
  if (!s || !F) return PFC_EINVAL;
  return energy_mass(s, s->phin, F, nullptr);
}

int pfc_mass(pfc_state* s, double* m) {
  if (!s || !m) return PFC_EINVAL;
  return energy_mass(s, s->phin, nullptr, m);
}

int pfc_residual(pfc_state* s, const double* Phi, const double* phin, double dt, double* F_out, double* norm) {
  if (!s || !Phi || !phin || !F_out || !(dt > 0.0)) return PFC_EINVAL;
  int rc = eval_residual(s, Phi, nullptr, 0.0, false, phin, 1.0 / dt, F_out, nullptr, nullptr, 2);
  if (rc) return rc;
  if ((rc = sync_read(s, s->red_h + 2, s->red + 2, sizeof(double)))) return rc;
  if (norm) *norm = std::sqrt(s->red_h[2]);
  return PFC_OK;
}

int pfc_jvp(pfc_state* s, const double* Phi, const double* phin, const double* v, double dt, double* Jv) {
  if (!s || !Phi || !phin || !v || !Jv || !(dt > 0.0)) return PFC_EINVAL;
  if (s->p.mobility) {  // q, mu and s of (Phi, phi^n) from the residual (F into scratch)
    int rc = eval_residual(s, Phi, nullptr, 0.0, false, phin, 1.0 / dt, s->Ft, nullptr, s->qt, 2);
    if (rc) return rc;
  } else if (s->dim == 2 && s->fs.prec != PFC_F64) {
    // the mixed path's product as GMRES takes it: v as basis vector Z_0 and q in s->q, so that
    // interior tiles stage by TMA (both are scratch between steps)
    pfc::launch_qcoef(s->g, Phi, phin, s->q, s->st);
    CU(cudaMemcpyAsync(s->Zbuf, v, sizeof(double) * (size_t)s->g.n, cudaMemcpyDeviceToDevice, s->st));
    CU(cudaMemsetAsync(s->status_dev, 0, 2 * sizeof(int), s->st));
    jvp(s, s->Zbuf, s->q, 1.0 / dt, Jv, nullptr, nullptr, 0);
    CU(cudaGetLastError());
    int st[2];
    CU(cudaMemcpyAsync(st, s->status_dev, sizeof st, cudaMemcpyDeviceToHost, s->st));
    CU(cudaStreamSynchronize(s->st));
    return st[1] ? st[1] : PFC_OK;
  } else {
    pfc::launch_qcoef(s->g, Phi, phin, s->qt, s->st);
  }
  jvp(s, v, s->qt, 1.0 / dt, Jv, nullptr);
  CU(cudaGetLastError());
  CU(cudaStreamSynchronize(s->st));
  return PFC_OK;
}

int pfc_precond_apply(pfc_state* s, const double* Phi, const double* phin, double dt, const double* r, double* z) {
  if (!s || !Phi || !phin || !r || !z || !(dt > 0.0)) return PFC_EINVAL;
  if (s->p.mobility) {  // q, mu and s of (Phi, phi^n) from the residual (F into scratch)
    int rc = eval_residual(s, Phi, nullptr, 0.0, false, phin, 1.0 / dt, s->Ft, nullptr, s->qt, 2);
    if (rc) return rc;
  } else {
    pfc::launch_qcoef(s->g, Phi, phin, s->qt, s->st);
  }
  s->factors_ok = false;  // the factors below belong to this call's arguments, not to a step
  int rc = factor_blocks(s, s->qt, 1.0 / dt);
  if (rc) return rc;
  precond(s, r, nullptr, z, nullptr);
  CU(cudaGetLastError());
  if ((rc = sync_read(s, s->status_h, s->status_dev, 2 * sizeof(int)))) return rc;
  if (s->status_h[0]) return s->status_h[0];
  return s->status_h[1] ? s->status_h[1] : PFC_OK;
}

const char* pfc_status_str(int st) {
  switch (st) {
    case PFC_OK: return "ok";
    case PFC_EINVAL: return "invalid argument";
    case PFC_ENOMEM: return "workspace too small";
    case PFC_ECUDA: return "CUDA error";
    case PFC_ENEWTON: return "Newton did not converge";
    case PFC_EGMRES: return "GMRES did not converge";
    case PFC_ESINGULAR: return "zero pivot in a subdomain factorisation";
    case PFC_ENAN: return "NaN or Inf in a residual norm";
    case PFC_ETIMEOUT: return "device wait timed out";
    default: return "unknown status";
  }
}

}  // extern "C"
