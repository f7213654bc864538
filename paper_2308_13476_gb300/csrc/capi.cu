// C-ABI of the helmmg library: hierarchy setup, the cycle driver (recursive
// V/W schedule captured once into a CUDA graph), the FP64 and the mixed
// (complex64 cycles in FP64 iterative refinement) solve loops, the adjoint
// solve and the misfit gradient.  See include/helmmg.h for the contract.
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <numeric>
#include <string>
#include <thread>
#include <vector>

#include "../../include/helmmg.h"
#include "internal.h"
#include "ragged_api.h"

using namespace hmg;

static thread_local std::string g_err;

namespace hmg {
void hmg_set_error(const char* msg) { g_err = msg; }
}  // namespace hmg

#define FAIL(code, ...)                                          \
  do {                                                           \
    char _b[512];                                                \
    snprintf(_b, sizeof(_b), __VA_ARGS__);                       \
    g_err = _b;                                                  \
    return code;                                                 \
  } while (0)

#define CK(call)                                                                          \
  do {                                                                                    \
    cudaError_t _e = (call);                                                              \
    if (_e != cudaSuccess) FAIL(MG_ECUDA, "%s failed: %s", #call, cudaGetErrorString(_e)); \
  } while (0)

namespace {

template <class T> struct LevelVec {
  cx<T>* x = nullptr;   // iterate / correction
  cx<T>* b = nullptr;   // right-hand side / restricted residual
  cx<T>* t = nullptr;   // Jacobi ping-pong partner of x
  cx<T>* r = nullptr;   // residual before restriction
  cx<T>* st = nullptr;  // stored stencil planes (levels >= 1)
  cx<T>* dinv = nullptr;
  GmresBufs gb{};
};

template <class T> struct CoarsePlan {
  CLevel<T>* levels = nullptr;   // device, one per level
  CStep* steps = nullptr;        // device
  int nsteps = 0;
};

struct Level {
  Grid g;
  int radius;                 // 1 on level 0 (matrix free), 2, then 3
  int kind = 1;               // OpView kind of the level's operator
  double2* st = nullptr;      // FP64 Galerkin stencil (variable k), levels >= 1
  double2* dinv = nullptr;
  long long plane = 0;
  // constant k: Kronecker factors [n+1][2r+1] (FP64 and float copies)
  double2 *gx = nullptr, *hy = nullptr;
  double *wx = nullptr, *wy = nullptr;
  float2 *gx32 = nullptr, *hy32 = nullptr;
  float *wx32 = nullptr, *wy32 = nullptr;
  float2* dinv32 = nullptr;
  // constant k: rows [ty0, ty1) whose y-factor rows (hy, wy) all equal the
  // middle row's, and that row (the translation-invariant interior)
  int ty0 = 0, ty1 = 0;
  double2 hyc[7] = {};
  double wyc[7] = {};
};

}  // namespace

struct mg_ctx {
  mg_options opt;
  long long peer_nodes = 0;   // ragged sub-handle: fine-level nodes of the problems solved beside it
  int nx = 0, ny = 0, B = 1, nlev = 0, ncoarse = 0;
  double h = 0, kconst = 0, beta2 = 0;
  Xfer xw = xfer_of(0);   // inter-grid transfer weights (opt.transfer)
  std::vector<Level> lev;
  std::vector<LevelVec<double>> v64;
  std::vector<LevelVec<float>> v32;
  Op0Consts<double>* c0d = nullptr;   // device copies (written by the setup kernel)
  Op0Consts<float>* c0f = nullptr;
  Op0Consts<double> hc0d{};            // host copies, passed to the kernels by value
  Op0Consts<float> hc0f{};
  double* kf64 = nullptr;
  float* kf32 = nullptr;
  FFConsts* ffc = nullptr;   // mixed path: float-float constants (device) and host copy
  FFConsts hffc{};
  float2* ffdiag = nullptr;  // mixed path, variable k: per-node float-float diagonal
  double2* cinv = nullptr;
  double* partial = nullptr;
  unsigned* tickets = nullptr;
  double* gst = nullptr;   // GMRES scalars
  int* active = nullptr;
  int* state = nullptr;
  int* cycles = nullptr;
  double* relres = nullptr;
  double* hist = nullptr;
  int hist_len = 0;
  double* bnorm = nullptr;
  double* tolp = nullptr;  // {tol, divergence threshold}
  int* n_active = nullptr;
  int* h_n_active = nullptr;  // pinned
  int* status = nullptr;
  cudaStream_t cap = nullptr;        // capture stream
  cudaStream_t side = nullptr;       // second stream of the fine-level row marches
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  cudaGraphExec_t gexec = nullptr;
  cudaGraph_t graph = nullptr;
  std::vector<void*> allocs;
  int lc = 1 << 30;                  // first level run by the coarse-cycle interpreter
  int coop_grid = 0;                 // > 0: cooperative interpreter with this many blocks
  CoopCtl coop{};
  CoarsePlan<double> plan64;
  CoarsePlan<float> plan32;
  long long graph_kernels = 0;     // kernel nodes in the cycle graph
  long long last_launches = 0, last_graphs = 0;
  int done = 0;                    // cycles of the current solve
  std::vector<mg_ctx*> sub;        // ragged batch: one handle per group of identical problems
  std::vector<std::vector<int>> members;  // ragged batch: the problems (caller's indices) of each handle
  std::vector<double2*> stage;     // ragged batch: per handle of several problems, their rhs and x side by side
  cudaStream_t own_stream = nullptr;
  bool flat = false;               // ragged batch: one flattened launch per kernel over all problems
  int* d_counts = nullptr;         // ragged flat: [2 P] active counts and barrier flags (device)
  int* h_counts = nullptr;         // and their pinned host copy
  std::vector<cudaStream_t> cstreams;  // ragged flat: per level, the stream of the coarse-cycle launches
  std::vector<cudaEvent_t> cfork, cjoin;
  // FGMRES(m) outer loop (opt.krylov = m > 0)
  FgArgs fg{};                     // buffers and geometry; per-solve fields set in solve_fgmres
  cudaGraph_t pgraph = nullptr;    // one preconditioning cycle (no test, no update)
  cudaGraphExec_t pexec = nullptr;
  long long pgraph_kernels = 0;

  ~mg_ctx() {
    for (mg_ctx* p : sub) delete p;
    if (gexec) cudaGraphExecDestroy(gexec);
    if (graph) cudaGraphDestroy(graph);
    if (pexec) cudaGraphExecDestroy(pexec);
    if (pgraph) cudaGraphDestroy(pgraph);
    for (void* p : allocs) cudaFree(p);
    if (h_n_active) cudaFreeHost(h_n_active);
    if (h_counts) cudaFreeHost(h_counts);
    if (cap) cudaStreamDestroy(cap);
    if (side) cudaStreamDestroy(side);
    if (ev_fork) cudaEventDestroy(ev_fork);
    if (ev_join) cudaEventDestroy(ev_join);
    if (own_stream) cudaStreamDestroy(own_stream);
    for (cudaStream_t q : cstreams) cudaStreamDestroy(q);
    for (cudaEvent_t e : cfork) cudaEventDestroy(e);
    for (cudaEvent_t e : cjoin) cudaEventDestroy(e);
  }
};

static cudaError_t dalloc(mg_ctx* c, void** p, size_t bytes) {
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) return e;
  c->allocs.push_back(*p);
  return cudaMemset(*p, 0, bytes);
}

// Rows per thread: several on big grids (fewer, fuller blocks and fewer
// reduction partials), one on small grids (more threads to hide latency);
// tile_rows > 0 forces the value (the autotuner's knob).
static Grid make_grid(int nx, int ny, int B, int tile_rows = 0) {
  Grid g;
  g.nx = nx;
  g.ny = ny;
  g.pitch = ((nx + 1 + 2 * HALO) + 3) / 4 * 4;
  g.rows = ny + 1 + 2 * HALO;
  g.vstride = (long long)g.pitch * g.rows;
  const long long nodes = (long long)(nx + 1) * (ny + 1) * B;
  g.ry = nodes >= (1LL << 20) ? 4 : (nodes >= (1LL << 18) ? 2 : 1);
  if (tile_rows > 0) g.ry = std::min(tile_rows, RYMAX);
  return g;
}

static long long node_blocks(const Grid& g) { return (long long)cdiv(g.nx + 1, BX) * cdiv(g.ny + 1, BY * g.ry); }

static OpView<double> op64(const mg_ctx* c, int l) {
  OpView<double> v{};
  const Level& L = c->lev[l];
  v.kind = L.kind;
  if (l == 0) {
    v.c0 = c->hc0d;
    v.kf = c->kf64;
  } else {
    v.st = L.st;
    v.dinv = L.dinv;
    v.plane = L.plane;
    v.gx = L.gx;
    v.wx = L.wx;
    v.hy = L.hy;
    v.wy = L.wy;
    v.ty0 = L.ty0;
    v.ty1 = L.ty1;
    for (int k = 0; k < 7; ++k) {
      v.hyc[k] = L.hyc[k];
      v.wyc[k] = L.wyc[k];
    }
  }
  return v;
}

static OpView<float> op32(const mg_ctx* c, int l) {
  OpView<float> v{};
  const Level& L = c->lev[l];
  v.kind = L.kind;
  if (l == 0) {
    v.c0 = c->hc0f;
    v.kf = c->kf32;
  } else {
    v.st = c->v32[l].st;
    v.dinv = L.kind >= 4 ? L.dinv32 : c->v32[l].dinv;
    v.plane = L.plane;
    v.gx = L.gx32;
    v.wx = L.wx32;
    v.hy = L.hy32;
    v.wy = L.wy32;
    v.ty0 = L.ty0;   // the float copies round the same FP64 rows: equal rows stay equal
    v.ty1 = L.ty1;
    for (int k = 0; k < 7; ++k) {
      v.hyc[k] = make_float2((float)L.hyc[k].x, (float)L.hyc[k].y);
      v.wyc[k] = (float)L.wyc[k];
    }
  }
  return v;
}

template <class T> static OpView<T> opT(const mg_ctx* c, int l);
template <> OpView<double> opT<double>(const mg_ctx* c, int l) { return op64(c, l); }
template <> OpView<float> opT<float>(const mg_ctx* c, int l) { return op32(c, l); }
template <class T> static std::vector<LevelVec<T>>& vecs(mg_ctx* c);
template <> std::vector<LevelVec<double>>& vecs<double>(mg_ctx* c) { return c->v64; }
template <> std::vector<LevelVec<float>>& vecs<float>(mg_ctx* c) { return c->v32; }

template <class T> static cudaError_t alloc_vectors(mg_ctx* c, LevelVec<T>& v, const Grid& g, bool gmres, bool kron) {
  const size_t bytes = sizeof(cx<T>) * (size_t)g.vstride * c->B;
  cudaError_t e;
  if ((e = dalloc(c, (void**)&v.x, bytes))) return e;
  if ((e = dalloc(c, (void**)&v.b, bytes))) return e;
  if ((e = dalloc(c, (void**)&v.t, bytes))) return e;
  if ((e = dalloc(c, (void**)&v.r, bytes))) return e;
  if (gmres) {
    for (int q = 0; q < 3; ++q)
      if ((e = dalloc(c, &v.gb.u[q], bytes))) return e;
    if ((e = dalloc(c, &v.gb.w, bytes))) return e;
    if (kron && sizeof(T) == 4 && (e = dalloc(c, &v.gb.w2, bytes))) return e;   // fused column marches' second w
    v.gb.partial = c->partial;
    v.gb.tickets = c->tickets;
    v.gb.st = c->gst;
  }
  return cudaSuccess;
}

// ----------------------------------------------------------------- cycle emission

// nu GMRES(3) smoothing steps on level l: the fine level as row marches, the
// Kronecker-form levels with column-march operator kernels (both with
// fuse = 1), stored stencils (or fuse = 0) with the node-parallel kernels.
// Whether level l runs its GMRES(3) kernels as marches (option march).
// Automatic: the Kronecker-form levels always (their column marches cut the
// arithmetic of every apply); the fine level when it holds at least 4 M nodes
// over all right-hand sides, counting those of the other problems of a
// ragged batch, which run beside it (a row march keeps each warp on one
// strip, and less work leaves the GPU under-filled).
static bool use_march(const mg_ctx* c, int l) {
  if (!c->opt.fuse || c->opt.march == 0) return false;
  if (c->opt.march == 1 || c->lev[l].kind >= 4) return true;
  const Grid& g = c->lev[l].g;
  return (long long)(g.nx + 1) * (g.ny + 1) * c->B + c->peer_nodes >= (4LL << 20);
}

template <class T>
static void gmres_level(mg_ctx* c, int l, cx<T>* x, const cx<T>* b, int nu, const int* active, cudaStream_t s,
                        double2* outer = nullptr, bool x_zero = false) {
  const Grid& g = c->lev[l].g;
  const OpView<T> op = opT<T>(c, l);
  GmresBufs gb = vecs<T>(c)[l].gb;
  gb.side = c->side;
  gb.kron_ch = c->opt.kron_chunk;
  gb.ev_fork = c->ev_fork;
  gb.ev_join = c->ev_join;
  gb.outer = outer;
  gb.x_zero = x_zero;
  const bool m = use_march(c, l);
  if (m && op.kind == 1) gmres_smooth_march<T>(g, op, x, b, nu, c->B, active, gb, s);
  else if (m && op.kind >= 4) gmres_smooth_kron<T>(g, op, x, b, nu, c->B, active, gb, s);
  else gmres_smooth<T>(g, op, x, b, nu, c->B, active, gb, s);
}

template <class T> struct Emit {
  mg_ctx* c;
  cudaStream_t s;
  std::vector<cx<T>*> cur, oth;
  int lc;                        // first level run by the coarse-cycle interpreter
  const CoarsePlan<T>* plan;
  // complex64 cycle of the FP64 refinement: the FP64 iterate that the
  // level-0 post-smoothing's last GMRES(3) update adds the cycle's result to
  // (the fused refinement update); null: the caller adds it
  double2* outer0 = nullptr;
  // zx[l]: level l's x is zero (just cleared) until its next smoothing, whose
  // first GMRES(3) step then takes u0 = b without applying A
  std::vector<char> zx;

  void smooth(int l, int nu, double2* outer = nullptr) {
    const bool z = zx[l] != 0;
    zx[l] = 0;
    if (nu <= 0) return;
    auto& V = vecs<T>(c)[l];
    const Grid& g = c->lev[l].g;
    const OpView<T> op = opT<T>(c, l);
    if (c->opt.smoother == 0 && l == 0 && c->opt.fuse && nu > 1) {   // temporal blocking on the fine level
      for (int q = 0; q < nu; q += jacobi_fused_max_nu()) {
        const int m = std::min(nu - q, jacobi_fused_max_nu());
        launch_jacobi_fused<T>(g, op, cur[l], V.b, oth[l], m, c->B, c->active, s);
        std::swap(cur[l], oth[l]);
      }
    } else if (c->opt.smoother == 0) {
      for (int q = 0; q < nu; ++q) {
        launch_jacobi<T>(g, op, cur[l], V.b, oth[l], c->B, c->active, s);
        std::swap(cur[l], oth[l]);
      }
    } else {
      gmres_level<T>(c, l, cur[l], V.b, nu, c->active, s, outer, z);
    }
  }

  void coarse_solve(int l) {
    auto& V = vecs<T>(c)[l];
    launch_coarse_solve<T>(c->lev[l].g, c->cinv, c->ncoarse, V.b, cur[l], c->B, c->active, s);
  }

  void cycle(int l) {
    const int L = c->nlev;
    if (l >= lc) {   // one visit of the sub-cycle below, in one launch
      if (c->coop_grid > 0)
        launch_cycle_coop<T>(plan->levels, c->nlev, plan->steps, plan->nsteps, c->cinv, c->ncoarse, c->active,
                             c->B, c->coop_grid, c->coop, s);
      else
        launch_coarse_cycle<T>(plan->levels, plan->steps, plan->nsteps, c->cinv, c->ncoarse, c->B, c->active, s);
      return;
    }
    if (l == L - 1) {
      coarse_solve(l);
      return;
    }
    auto& V = vecs<T>(c);
    const Grid& g = c->lev[l].g;
    const Grid& gc = c->lev[l + 1].g;
    smooth(l, c->opt.nu_pre);
    if (c->opt.fuse && c->lev[l].kind >= 4 && use_march(c, l)) {
      // a Kronecker-form level: the residual as a column march (about a
      // twelfth of OpK::apply's arithmetic), then the restriction
      launch_kron_residual<T>(g, opT<T>(c, l), cur[l], V[l].b, V[l].r, c->B, c->active, c->opt.kron_chunk, s);
      launch_restrict<T>(g, gc, V[l].r, V[l + 1].b, c->B, c->active, c->xw, s);
    } else if (c->opt.fuse) {
      launch_resid_restrict<T>(g, gc, opT<T>(c, l), cur[l], V[l].b, V[l + 1].b, c->B, c->active, c->xw, s);
    } else {
      launch_residual<T>(g, opT<T>(c, l), cur[l], V[l].b, V[l].r, c->B, c->active, s);
      launch_restrict<T>(g, gc, V[l].r, V[l + 1].b, c->B, c->active, c->xw, s);
    }
    if (l + 1 == L - 1 && lc > l + 1) {
      coarse_solve(l + 1);
    } else {
      cudaMemsetAsync(cur[l + 1], 0, sizeof(cx<T>) * (size_t)gc.vstride * c->B, s);
      zx[l + 1] = 1;
      for (int q = 0; q < c->opt.cycle; ++q) cycle(l + 1);
    }
    launch_prolong_add<T>(g, gc, cur[l + 1], cur[l], c->B, c->active, c->xw, s);
    smooth(l, c->opt.nu_post, l == 0 ? outer0 : nullptr);
  }

  void init() {
    auto& V = vecs<T>(c);
    cur.resize(c->nlev);
    oth.resize(c->nlev);
    for (int l = 0; l < c->nlev; ++l) {
      cur[l] = V[l].x;
      oth[l] = V[l].t;
    }
    zx.assign(c->nlev, 0);
  }
};

static Ctl ctl(const mg_ctx* c) {
  return Ctl{c->bnorm, c->tolp, c->active, c->state, c->cycles, c->relres, c->hist, c->hist_len, c->n_active,
             c->partial, c->tickets};
}

// Records the steps of one visit of level lc (the same recursion as
// Emit::cycle) for the coarse-cycle interpreter.
template <class T> struct Plan {
  mg_ctx* c;
  std::vector<cx<T>*> cur, oth;
  std::vector<CStep> steps;
  void push(int op, int l, int arg, void* p0, void* p1) { steps.push_back(CStep{op, l, arg, 0, p0, p1}); }
  void smooth(int l, int nu) {
    if (nu <= 0) return;
    if (c->opt.smoother == 0) {
      for (int q = 0; q < nu; ++q) {
        push(C_JACOBI, l, 0, cur[l], oth[l]);
        std::swap(cur[l], oth[l]);
      }
    } else {
      push(C_GMRES, l, nu, cur[l], nullptr);
    }
  }
  void cycle(int l) {
    const int L = c->nlev;
    if (l == L - 1) {
      push(C_COARSE, l, 0, cur[l], nullptr);
      return;
    }
    smooth(l, c->opt.nu_pre);
    push(C_RESTRICT, l, 0, cur[l], nullptr);
    if (l + 1 == L - 1) {
      push(C_COARSE, l + 1, 0, cur[l + 1], nullptr);
    } else {
      push(C_ZERO, l + 1, 0, cur[l + 1], nullptr);
      for (int q = 0; q < c->opt.cycle; ++q) cycle(l + 1);
    }
    push(C_PROLONG, l, 0, cur[l], cur[l + 1]);
    smooth(l, c->opt.nu_post);
  }
};

template <class T> static cudaError_t build_plan(mg_ctx* c, int lc, CoarsePlan<T>& P) {
  auto& V = vecs<T>(c);
  const int L = c->nlev;
  std::vector<CLevel<T>> lv(L);
  for (int l = 0; l < L; ++l) {
    CLevel<T> d{};
    const OpView<T> op = opT<T>(c, l);
    d.g = c->lev[l].g;
    d.xw = c->xw;
    d.kind = op.kind;
    d.c0 = op.c0;
    d.kf = op.kf;
    d.st = op.st;
    d.dinv = op.dinv;
    d.plane = op.plane;
    d.gx = op.gx;
    d.wx = op.wx;
    d.hy = op.hy;
    d.wy = op.wy;
    d.b = V[l].b;
    d.r = V[l].r;
    for (int q = 0; q < 3; ++q) d.u[q] = (cx<T>*)V[l].gb.u[q];
    d.w = (cx<T>*)V[l].gb.w;
    lv[l] = d;
  }
  Plan<T> pl{c};
  pl.cur.resize(L);
  pl.oth.resize(L);
  for (int l = 0; l < L; ++l) {
    pl.cur[l] = V[l].x;
    pl.oth[l] = V[l].t;
  }
  pl.cycle(lc);
  if (pl.cur[lc] != V[lc].x) pl.push(C_COPY, lc, 0, pl.cur[lc], V[lc].x);
  P.nsteps = (int)pl.steps.size();
  cudaError_t e;
  if ((e = dalloc(c, (void**)&P.levels, sizeof(CLevel<T>) * L))) return e;
  if ((e = dalloc(c, (void**)&P.steps, sizeof(CStep) * P.nsteps))) return e;
  if ((e = cudaMemcpy(P.levels, lv.data(), sizeof(CLevel<T>) * L, cudaMemcpyHostToDevice))) return e;
  return cudaMemcpy(P.steps, pl.steps.data(), sizeof(CStep) * P.nsteps, cudaMemcpyHostToDevice);
}

// One FP64 cycle followed by the stopping test (graph body of the FP64 path).
static void emit_fp64_iteration(mg_ctx* c, cudaStream_t s) {
  Emit<double> e{c, s, {}, {}, c->lc, &c->plan64};
  e.init();
  e.cycle(0);
  if (e.cur[0] != c->v64[0].x) launch_copy_masked<double>(c->lev[0].g, e.cur[0], c->v64[0].x, c->B, c->active, s);
  launch_resnorm_stop<double>(c->lev[0].g, op64(c, 0), c->v64[0].x, c->v64[0].b, c->B, ctl(c), 1, s);
}

// One refinement step of the mixed path: e = 0, one complex64 cycle on the
// float residual, x += e and the new outer residual (cast to float) with the
// stopping test -- in FP64 (precision 1) or float-float (precision 2).
static void emit_mixed_iteration(mg_ctx* c, cudaStream_t s) {
  Emit<float> e{c, s, {}, {}, c->lc, &c->plan32};
  e.init();
  const Grid& g0 = c->lev[0].g;
  // the refinement update x64 += e fused into the cycle's last kernel: the
  // level-0 post-smoothing's last GMRES(3) update (a level-0 smoothing run by
  // the cycle's own kernels, precision 1)
  const bool fused = c->opt.precision == 1 && c->opt.smoother == 1 && c->opt.nu_post > 0 && c->lc > 0 &&
                     c->nlev > 1;
  if (fused) e.outer0 = c->v64[0].x;
  cudaMemsetAsync(c->v32[0].x, 0, sizeof(float2) * (size_t)g0.vstride * c->B, s);
  e.zx[0] = 1;
  e.cycle(0);
  if (c->opt.precision == 2) {
    launch_ff_update(g0, c->v64[0].x, e.cur[0], c->B, c->active, s);
    launch_ff_resid_cast_stop(g0, c->hffc, c->kf64, c->h, c->ffdiag, c->v64[0].x, c->v64[0].b, c->v32[0].b, c->B,
                              ctl(c), 1, s);
  } else {
    if (!fused) launch_update_mixed(g0, c->v64[0].x, e.cur[0], c->B, c->active, s);
    launch_resid_cast_stop(g0, op64(c, 0), c->v64[0].x, c->v64[0].b, c->v32[0].b, c->B, ctl(c), 1, s);
  }
}

// The FGMRES kernels' arguments: the handle's buffers and control arrays.
static FgArgs fg_args(const mg_ctx* c, double tol) {
  FgArgs a = c->fg;
  a.c0 = c->hc0d;
  a.kf = c->kf64;
  a.c0f = c->hc0f;
  a.kf32 = c->kf32;
  a.active = c->active;
  a.state = c->state;
  a.cycles = c->cycles;
  a.relres = c->relres;
  a.hist = c->hist;
  a.hist_len = c->hist_len;
  a.n_active = c->n_active;
  a.bnorm = c->bnorm;
  a.tol = tol;
  a.max_cycles = c->opt.max_cycles;
  return a;
}

// Throughput probe of the FP64 FMA pipe (instrumentation for the FP64
// roofline, no step of the method).  Every thread runs eight independent
// FMA chains; the sum is stored only if it equals a value it cannot reach,
// so nothing is written and nothing can be folded away.
__global__ void __launch_bounds__(256) k_fp64_fma_probe(int iters, double* __restrict__ sink) {
  double a[8];
  const double m = 1.0 + 1e-12 * (threadIdx.x + 1), c = 1e-13;
#pragma unroll
  for (int q = 0; q < 8; ++q) a[q] = 1.0 + 1e-3 * q + 1e-7 * blockIdx.x;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int q = 0; q < 8; ++q) a[q] = fma(a[q], m, c);
  }
  double t = 0.0;
#pragma unroll
  for (int q = 0; q < 8; ++q) t += a[q];
  if (t == -1.0) sink[0] = t;
}

static double launch_fp64_fma_probe(int iters, double* sink, cudaStream_t s) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int blocks = sms * 8;
  k_fp64_fma_probe<<<blocks, 256, 0, s>>>(iters, sink);
  return 2.0 * 8.0 * (double)iters * blocks * 256.0;   // FP64 flops of one launch
}

template <class T> static mg_status profile_t(mg_ctx* h, int what, int level, int reps, double* ms, double* bytes) {
  cudaStream_t s = (cudaStream_t)h->opt.stream;
  auto& V = vecs<T>(h);
  if (level < 0 || level >= (int)V.size() || ((what == 2 || what == 3) && level + 1 >= h->nlev))
    FAIL(MG_EINVAL, "bad level");
  if (what == 4 && h->opt.smoother != 1) FAIL(MG_EINVAL, "what = 4 needs the GMRES(3) smoother");
  if (what == 5 && (h->opt.krylov < 1 || level != 0)) FAIL(MG_EINVAL, "what = 5 needs krylov > 0 and level 0");
  const Grid& g = h->lev[level].g;
  const OpView<T> op = opT<T>(h, level);
  const double nodes = (double)(g.nx + 1) * (g.ny + 1) * h->B;
  const double e = sizeof(cx<T>);
  double opbytes = 0;   // per node: stored stencil and inverse diagonal, or the k field
  if (level > 0 && h->lev[level].kind <= 3) {
    const int r = h->lev[level].radius;
    opbytes = e * ((2 * r + 1) * (2 * r + 1) + 1) / h->B;
  } else if (level > 0) {
    opbytes = e / h->B;   // Kronecker form: only the inverse diagonal per node
  } else if (op.kf) {
    opbytes = sizeof(T) / (double)h->B;
  }
  const std::vector<int> ones(h->B, 1);
  const FgArgs fa = what == 5 ? fg_args(h, 0.0) : FgArgs{};
  double probe_flops = 0.0;
  auto launch = [&]() {
    switch (what) {
      case 6: probe_flops = launch_fp64_fma_probe(4096, reinterpret_cast<double*>(V[0].t), s); break;
      case 0: launch_jacobi<T>(g, op, V[level].x, V[level].b, V[level].t, h->B, nullptr, s); break;
      case 1: launch_residual<T>(g, op, V[level].x, V[level].b, V[level].r, h->B, nullptr, s); break;
      case 2: launch_restrict<T>(g, h->lev[level + 1].g, V[level].r, V[level + 1].b, h->B, nullptr, h->xw, s); break;
      case 3: launch_prolong_add<T>(g, h->lev[level + 1].g, V[level + 1].x, V[level].x, h->B, nullptr, h->xw, s); break;
      case 4: gmres_level<T>(h, level, V[level].x, V[level].b, 1, nullptr, s); break;
      default: {   // the last Arnoldi step of a restart cycle (j = m - 1): both passes, every RHS active
        const int j = h->opt.krylov - 1;
        cudaMemcpyAsync(h->active, ones.data(), sizeof(int) * h->B, cudaMemcpyHostToDevice, s);
        launch_fg_dots<T>(fa, j, V[0].x, s);
        launch_fg_orth<T>(fa, j, V[0].b, V[0].x, s);
        break;
      }
    }
  };
  if (what == 6) *bytes = 0.0;   // set from the probe's flop count below
  else if (what == 0 || what == 1) *bytes = nodes * (3 * e + opbytes);
  else if (what == 2) *bytes = nodes * e * 1.25;     // read fine r, write coarse r
  else if (what == 3) *bytes = nodes * e * 2.25;     // read+write fine x, read coarse e
  else if (what == 5)   // z, Z_j twice; u_0..u_j twice; u_{j+1}, cycle rhs, cycle x (all in the cycle's precision); k twice
    *bytes = nodes * (e * (2.0 * h->opt.krylov + 6.0) + (op.kf ? 2 * sizeof(T) / (double)h->B : 0.0));
  else {   // GMRES(3) step: four passes that read the operator, plus vectors
    double gop = 0;   // operator bytes per node and RHS read by one pass
    if (level == 0) gop = op.kf ? sizeof(T) / (double)h->B : 0.0;
    else if (h->lev[level].kind <= 3) gop = opbytes - e / h->B;   // stencil without the inverse diagonal
    // fine-level row marches + update 16, complex64 13 (no M3: u3's norm from the Gram form); Kronecker column
    // marches, complex64 (two fused passes, no closing g_arn_b<2>) 19; else 28, complex64 23 (no g_arn_b<2>,
    // and g_arn_a<2> stores no w)
    const bool mr = use_march(h, level);
    const bool c64 = sizeof(T) == 4;
    const int vec = (mr && h->lev[level].kind == 1) ? (c64 ? 13 : 16)
                                                     : (mr && h->lev[level].kind >= 4 && c64) ? 19 : (c64 ? 23 : 28);
    *bytes = nodes * (vec * e + 4 * gop);
  }
  launch();
  cudaEvent_t a, b;
  CK(cudaEventCreate(&a));
  CK(cudaEventCreate(&b));
  CK(cudaEventRecord(a, s));
  for (int q = 0; q < reps; ++q) launch();
  CK(cudaEventRecord(b, s));
  CK(cudaEventSynchronize(b));
  float t = 0;
  CK(cudaEventElapsedTime(&t, a, b));
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  CK(cudaGetLastError());
  *ms = t / reps;
  if (what == 6) *bytes = probe_flops;
  return MG_OK;
}

// ----------------------------------------------------------------- C ABI

// ---------------------------------------------------------- ragged, flattened
//
// The cycle of every problem of a ragged batch as one graph whose kernels are
// single launches over all problems (ragged.cuh).  The recursion is the one
// of Emit::cycle, run on the set of problems that visit a level: problems
// whose coarse-cycle launch starts at this level take it here (one CTA per
// problem), the others smooth, restrict, recurse gamma times, prolong and
// smooth.  Every problem sees its own kernels in the order Emit gives them.
template <class T> struct EmitR {
  mg_ctx* c;
  cudaStream_t s;
  int P() const { return (int)c->sub.size(); }
  mg_ctx* q(int p) const { return c->sub[p]; }
  cx<T>* cur(int p, int l) const { return vecs<T>(c->sub[p])[l].x; }   // GMRES(3) smoothing keeps x in place

  void smooth(int l, const std::vector<int>& G, int nu) {
    if (nu <= 0 || G.empty()) return;
    std::vector<RagLevel<T>> v;
    for (int p : G) {
      mg_ctx* h = q(p);
      GmresBufs gb = vecs<T>(h)[l].gb;
      gb.kron_ch = h->opt.kron_chunk;
      v.push_back(RagLevel<T>{h->lev[l].g, opT<T>(h, l), cur(p, l), vecs<T>(h)[l].b, gb, h->active});
    }
    if (l == 0) gmres_smooth_march_rag<T>(v, nu, s, c->side, c->ev_fork, c->ev_join);
    else gmres_smooth_kron_rag<T>(v, nu, s);
  }

  void cycle(int l, const std::vector<int>& S) {
    std::vector<int> G, I;
    for (int p : S) (l >= q(p)->lc ? I : G).push_back(p);
    if (!I.empty()) {   // one visit of each one's coarse sub-cycle, beside the deeper work of the others
      std::vector<RagCoarse<T>> v;
      for (int p : I) {
        mg_ctx* h = q(p);
        const CoarsePlan<T>* pl = sizeof(T) == 8 ? (const CoarsePlan<T>*)&h->plan64 : (const CoarsePlan<T>*)&h->plan32;
        v.push_back(RagCoarse<T>{pl->levels, pl->steps, pl->nsteps, h->cinv, h->ncoarse, h->active});
      }
      if (G.empty()) {
        launch_coarse_cycle_rag<T>(v, s);
      } else {
        cudaEventRecord(c->cfork[l], s);
        cudaStreamWaitEvent(c->cstreams[l], c->cfork[l], 0);
        launch_coarse_cycle_rag<T>(v, c->cstreams[l]);
        cudaEventRecord(c->cjoin[l], c->cstreams[l]);
      }
    }
    if (G.empty()) return;
    struct Join {   // the caller's next kernel (a prolongation) reads the coarse launch's result
      mg_ctx* c;
      cudaStream_t s;
      int l;
      bool on;
      ~Join() {
        if (on) cudaStreamWaitEvent(s, c->cjoin[l], 0);
      }
    } join{c, s, l, !I.empty()};
    smooth(l, G, c->opt.nu_pre);
    std::vector<RagXfer<T>> xf;
    std::vector<RagVec> zv;
    for (int p : G) {
      mg_ctx* h = q(p);
      auto& V = vecs<T>(h);
      xf.push_back(RagXfer<T>{h->lev[l].g, h->lev[l + 1].g, opT<T>(h, l), cur(p, l), V[l].b, V[l + 1].b, cur(p, l),
                              h->active});
      zv.push_back(RagVec{h->lev[l + 1].g, cur(p, l + 1), h->active});
    }
    launch_resid_restrict_rag<T>(xf, c->sub[0]->xw, s);
    launch_zero_rag<T>(zv, s);
    for (int g = 0; g < c->opt.cycle; ++g) cycle(l + 1, G);
    for (size_t k = 0; k < G.size(); ++k) xf[k].rc = cur(G[k], l + 1);   // the coarse correction
    launch_prolong_add_rag<T>(xf, c->sub[0]->xw, s);
    smooth(l, G, c->opt.nu_post);
  }

  std::vector<int> all() const {
    std::vector<int> v(P());
    for (int p = 0; p < P(); ++p) v[p] = p;
    return v;
  }
};

// One cycle of every problem and its stopping test, then the active counts
// gathered into the pinned host array (graph body of the flattened batch).
static void emit_ragged_iteration(mg_ctx* c, cudaStream_t s) {
  const int P = (int)c->sub.size();
  std::vector<RagOuter> outer;
  std::vector<const int*> counts;
  for (mg_ctx* h : c->sub) {
    const Grid& g0 = h->lev[0].g;
    const OpView<double> o = op64(h, 0);
    outer.push_back(RagOuter{g0, Op0<double>{o.c0, o.kf, g0.nx, g0.ny}, h->v64[0].x, h->v64[0].b,
                             h->opt.precision == 1 ? h->v32[0].x : nullptr, h->opt.precision == 1 ? h->v32[0].b : nullptr,
                             ctl(h)});
    counts.push_back(h->n_active);
  }
  if (c->opt.precision == 1) {
    std::vector<RagVec> zv;
    for (mg_ctx* h : c->sub) zv.push_back(RagVec{h->lev[0].g, h->v32[0].x, h->active});
    launch_zero_rag<float>(zv, s);
    EmitR<float> e{c, s};
    e.cycle(0, e.all());
    launch_update_mixed_rag(outer, s);
    launch_resid_cast_stop_rag(outer, 1, s);
  } else {
    EmitR<double> e{c, s};
    e.cycle(0, e.all());
    launch_resnorm_stop_rag(outer, 1, s);
  }
  launch_gather_counts(counts, c->d_counts, s);
  cudaMemcpyAsync(c->h_counts, c->d_counts, sizeof(int) * 2 * P, cudaMemcpyDeviceToHost, s);
}

// Instantiates a captured graph and counts its kernel nodes.
static mg_status instantiate_graph(cudaGraph_t g, cudaGraphExec_t* exec, long long* kernels) {
  CK(cudaGraphInstantiate(exec, g, 0));
  size_t n = 0;
  CK(cudaGraphGetNodes(g, nullptr, &n));
  std::vector<cudaGraphNode_t> nodes(n);
  CK(cudaGraphGetNodes(g, nodes.data(), &n));
  *kernels = 0;
  for (auto nd : nodes) {
    cudaGraphNodeType t;
    CK(cudaGraphNodeGetType(nd, &t));
    *kernels += t == cudaGraphNodeTypeKernel;
  }
  return MG_OK;
}

static mg_status capture_ragged(mg_ctx* c) {
  if (c->gexec) return MG_OK;
  CK(cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal));
  emit_ragged_iteration(c, c->cap);
  cudaGraph_t g;
  cudaError_t e = cudaStreamEndCapture(c->cap, &g);
  if (e != cudaSuccess) FAIL(MG_ECUDA, "graph capture of the flattened ragged cycle failed: %s", cudaGetErrorString(e));
  c->graph = g;
  return instantiate_graph(g, &c->gexec, &c->graph_kernels);
}

extern "C" {

void mg_default_options(mg_options* o) {
  if (!o) return;
  o->cycle = 1;
  o->smoother = 0;
  o->nu_pre = 1;
  o->nu_post = 1;
  o->omega = 4.5;
  o->precision = 0;
  o->max_cycles = 10000;
  o->min_coarse = 10;
  o->batch = 1;
  o->coarse_nodes = 1100;
  o->coarse_mode = 0;
  o->fuse = 1;
  o->tile_rows = 0;
  o->march = -1;
  o->krylov = 0;
  o->transfer = 0;
  o->flat = 0;
  o->kron_chunk = 0;
  o->abc = 1;
  o->stream = nullptr;
}

const char* mg_last_error(void) { return g_err.c_str(); }

mg_status mg_destroy(mg_handle h) {
  delete h;
  return MG_OK;
}

static mg_status setup_impl(mg_ctx* c, const double* k_field) {
  const mg_options& o = c->opt;
  cudaStream_t s = (cudaStream_t)o.stream;
  c->xw = xfer_of(o.transfer);
  // level list: halve while both counts are even and the grid has >= min_coarse nodes
  std::vector<std::pair<int, int>> sizes{{c->nx, c->ny}};
  while (true) {
    auto [cx_, cy_] = sizes.back();
    if (c->nlev > 0 && (int)sizes.size() >= c->nlev) break;
    if (cx_ % 2 || cy_ % 2 || (long long)(cx_ + 1) * (cy_ + 1) < o.min_coarse) break;
    sizes.push_back({cx_ / 2, cy_ / 2});
  }
  c->nlev = (int)sizes.size();
  c->ncoarse = (sizes.back().first + 1) * (sizes.back().second + 1);
  if (c->ncoarse > 2048) FAIL(MG_EINVAL, "coarsest grid has %d nodes (> 2048); use more levels", c->ncoarse);
  c->lev.resize(c->nlev);
  for (int l = 0; l < c->nlev; ++l) {
    c->lev[l].g = make_grid(sizes[l].first, sizes[l].second, c->B, o.tile_rows);
    c->lev[l].radius = l == 0 ? 1 : (l == 1 ? 2 : 3);
    c->lev[l].plane = (long long)(sizes[l].first + 1) * (sizes[l].second + 1);
  }
  const bool mixed = o.precision >= 1;
  const bool ffo = o.precision == 2;   // float-float outer loop
  const bool gm = o.smoother == 1;
  const Grid& g0 = c->lev[0].g;
  CK(configure_fused_kernels());
  CK(dalloc(c, (void**)&c->c0d, sizeof(Op0Consts<double>)));
  if (mixed) CK(dalloc(c, (void**)&c->c0f, sizeof(Op0Consts<float>)));
  const long long N0 = c->lev[0].plane;
  if (k_field) {
    CK(dalloc(c, (void**)&c->kf64, sizeof(double) * N0));
    CK(cudaMemcpyAsync(c->kf64, k_field, sizeof(double) * N0, cudaMemcpyDefault, s));
    if (mixed) {
      CK(dalloc(c, (void**)&c->kf32, sizeof(float) * N0));
      launch_to_float_real(c->kf64, c->kf32, N0, s);
    }
  }
  launch_op0consts(c->c0d, c->c0f, c->h, c->kconst, o.omega, c->beta2, o.abc, s);
  CK(cudaMemcpyAsync(&c->hc0d, c->c0d, sizeof(Op0Consts<double>), cudaMemcpyDeviceToHost, s));
  if (mixed) CK(cudaMemcpyAsync(&c->hc0f, c->c0f, sizeof(Op0Consts<float>), cudaMemcpyDeviceToHost, s));
  if (ffo) {
    CK(dalloc(c, (void**)&c->ffc, sizeof(FFConsts)));
    if (k_field) CK(dalloc(c, (void**)&c->ffdiag, sizeof(float2) * N0));
    launch_ff_setup(c->h, c->kconst, c->kf64, g0.nx, g0.ny, c->ffc, c->ffdiag, s);
    CK(cudaMemcpyAsync(&c->hffc, c->ffc, sizeof(FFConsts), cudaMemcpyDeviceToHost, s));
  }
  CK(cudaStreamSynchronize(s));
  // Galerkin operators A_{l+1} = R_l C_l P_l.  Constant k: Kronecker form,
  // A_l = W_y (x) G_x + H_y (x) W_x, each factor coarsened in 1D.  Variable
  // k, or the second-order absorbing rows (whose tangential boundary terms
  // are not of that two-term form): per-node stencils from the 2D product.
  const bool kron = k_field == nullptr && o.abc == 1;
  if (kron && c->nlev > 1) {
    // fine-level 1D factors (radius 1) in scratch, then coarsen level by level
    double2 *g0, *h0, *wx0, *wy0, *tmp;
    const int nx = c->nx, ny = c->ny, nmax = std::max(nx, ny);
    CK(dalloc(c, (void**)&g0, sizeof(double2) * 3 * (nx + 1)));
    CK(dalloc(c, (void**)&wx0, sizeof(double2) * 3 * (nx + 1)));
    CK(dalloc(c, (void**)&h0, sizeof(double2) * 3 * (ny + 1)));
    CK(dalloc(c, (void**)&wy0, sizeof(double2) * 3 * (ny + 1)));
    CK(dalloc(c, (void**)&tmp, sizeof(double2) * 3 * (nmax + 1)));
    launch_factors0(nx, c->h, c->kconst, c->beta2, g0, tmp, wx0, s);
    launch_factors0(ny, c->h, c->kconst, c->beta2, tmp, h0, wy0, s);
    const double2 *pg = g0, *ph = h0, *pwx = wx0, *pwy = wy0;
    std::vector<double2*> cwx(c->nlev), cwy(c->nlev);
    for (int l = 1; l < c->nlev; ++l) {
      Level& L = c->lev[l];
      const int r = L.radius, rf = c->lev[l - 1].radius, w = 2 * r + 1;
      const int fx = c->lev[l - 1].g.nx, fy = c->lev[l - 1].g.ny, cx_ = L.g.nx, cy_ = L.g.ny;
      L.kind = 2 + r;
      CK(dalloc(c, (void**)&L.gx, sizeof(double2) * w * (cx_ + 1)));
      CK(dalloc(c, (void**)&L.hy, sizeof(double2) * w * (cy_ + 1)));
      CK(dalloc(c, (void**)&cwx[l], sizeof(double2) * w * (cx_ + 1)));
      CK(dalloc(c, (void**)&cwy[l], sizeof(double2) * w * (cy_ + 1)));
      CK(dalloc(c, (void**)&L.wx, sizeof(double) * w * (cx_ + 1)));
      CK(dalloc(c, (void**)&L.wy, sizeof(double) * w * (cy_ + 1)));
      launch_galerkin_1d(pg, fx, rf, L.gx, r, c->xw, s);
      launch_galerkin_1d(pwx, fx, rf, cwx[l], r, c->xw, s);
      launch_galerkin_1d(ph, fy, rf, L.hy, r, c->xw, s);
      launch_galerkin_1d(pwy, fy, rf, cwy[l], r, c->xw, s);
      launch_real_part(cwx[l], L.wx, (long long)w * (cx_ + 1), s);
      launch_real_part(cwy[l], L.wy, (long long)w * (cy_ + 1), s);
      CK(dalloc(c, (void**)&L.dinv, sizeof(double2) * L.plane));
      launch_diaginv_op(op64(c, l), cx_, cy_, o.omega, L.dinv, s);
      // rows of the y-factors equal to the middle row (translation-invariant interior)
      {
        const int K = w, ny1 = cy_ + 1, mid = cy_ / 2;
        std::vector<double2> hh((size_t)K * ny1);
        std::vector<double> ww((size_t)K * ny1);
        CK(cudaMemcpyAsync(hh.data(), L.hy, sizeof(double2) * hh.size(), cudaMemcpyDeviceToHost, s));
        CK(cudaMemcpyAsync(ww.data(), L.wy, sizeof(double) * ww.size(), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        auto same = [&](int j) {
          for (int k = 0; k < K; ++k) {
            const double2 a = hh[(size_t)j * K + k], b = hh[(size_t)mid * K + k];
            if (a.x != b.x || a.y != b.y || ww[(size_t)j * K + k] != ww[(size_t)mid * K + k]) return false;
          }
          return true;
        };
        int j0 = mid, j1 = mid + 1;
        while (j0 > 0 && same(j0 - 1)) --j0;
        while (j1 < ny1 && same(j1)) ++j1;
        L.ty0 = j0;
        L.ty1 = j1;
        for (int k = 0; k < K; ++k) {
          L.hyc[k] = hh[(size_t)mid * K + k];
          L.wyc[k] = ww[(size_t)mid * K + k];
        }
      }
      pg = L.gx;
      ph = L.hy;
      pwx = cwx[l];
      pwy = cwy[l];
      if (mixed) {
        CK(dalloc(c, (void**)&L.gx32, sizeof(float2) * w * (cx_ + 1)));
        CK(dalloc(c, (void**)&L.hy32, sizeof(float2) * w * (cy_ + 1)));
        CK(dalloc(c, (void**)&L.wx32, sizeof(float) * w * (cx_ + 1)));
        CK(dalloc(c, (void**)&L.wy32, sizeof(float) * w * (cy_ + 1)));
        CK(dalloc(c, (void**)&L.dinv32, sizeof(float2) * L.plane));
        launch_to_float(L.gx, L.gx32, (long long)w * (cx_ + 1), s);
        launch_to_float(L.hy, L.hy32, (long long)w * (cy_ + 1), s);
        launch_to_float_real(L.wx, L.wx32, (long long)w * (cx_ + 1), s);
        launch_to_float_real(L.wy, L.wy32, (long long)w * (cy_ + 1), s);
        launch_to_float(L.dinv, L.dinv32, L.plane, s);
      }
    }
  } else {
    for (int l = 1; l < c->nlev; ++l) {
      Level& L = c->lev[l];
      const int r = L.radius;
      const long long S = (long long)(2 * r + 1) * (2 * r + 1);
      L.kind = r;
      CK(dalloc(c, (void**)&L.st, sizeof(double2) * S * L.plane));
      CK(dalloc(c, (void**)&L.dinv, sizeof(double2) * L.plane));
      launch_galerkin(op64(c, l - 1), c->lev[l - 1].g.nx, c->lev[l - 1].g.ny, L.st, L.g.nx, L.g.ny, r, c->beta2, c->xw,
                      s);
      launch_diaginv(L.st, r, L.plane, o.omega, L.dinv, s);
    }
  }
  CK(cudaGetLastError());
  // coarsest direct solver
  {
    const int N = c->ncoarse;
    double2* M;
    CK(dalloc(c, (void**)&M, sizeof(double2) * (size_t)N * N));
    CK(dalloc(c, (void**)&c->cinv, sizeof(double2) * (size_t)N * N));
    CK(dalloc(c, (void**)&c->status, sizeof(int) * 4));
    const int lc = c->nlev - 1;
    launch_dense(op64(c, lc), c->lev[lc].g.nx, c->lev[lc].g.ny, M, s);
    launch_gauss_jordan(M, c->cinv, N, c->status, s);
    CK(cudaGetLastError());
    int st = 0;
    CK(cudaMemcpyAsync(&st, c->status, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (st) FAIL(MG_ESTATE, "coarsest operator is singular");
  }
  // work arrays
  long long nblk_max = 0;   // reduction partials: the most blocks of any level
  for (int l = 0; l < c->nlev; ++l) {
    nblk_max = std::max(nblk_max, node_blocks(c->lev[l].g));
    if (c->lev[l].kind == 1)
      nblk_max = std::max({nblk_max, gmres_march_blocks(c->lev[l].g, true, c->B),
                           gmres_march_blocks(c->lev[l].g, false, c->B)});
    if (c->lev[l].kind >= 4) nblk_max = std::max(nblk_max, kron_march_blocks(c->lev[l].g, c->B));
  }
  CK(dalloc(c, (void**)&c->partial, sizeof(double) * (size_t)nblk_max * c->B * NVMAX));
  CK(dalloc(c, (void**)&c->tickets, sizeof(unsigned) * c->B));
  CK(dalloc(c, (void**)&c->gst, sizeof(double) * 96 * c->B));
  CK(dalloc(c, (void**)&c->active, sizeof(int) * c->B));
  CK(dalloc(c, (void**)&c->state, sizeof(int) * c->B));
  CK(dalloc(c, (void**)&c->cycles, sizeof(int) * c->B));
  CK(dalloc(c, (void**)&c->relres, sizeof(double) * c->B));
  CK(dalloc(c, (void**)&c->bnorm, sizeof(double) * c->B));
  CK(dalloc(c, (void**)&c->tolp, sizeof(double) * 2));
  CK(dalloc(c, (void**)&c->n_active, sizeof(int) * 2));   // {active count, cooperative-barrier error}
  c->hist_len = std::min(o.max_cycles, 4096);
  CK(dalloc(c, (void**)&c->hist, sizeof(double) * (size_t)c->hist_len * c->B));
  CK(cudaMallocHost((void**)&c->h_n_active, sizeof(int) * 2));
  // vectors
  if (!mixed) {
    c->v64.resize(c->nlev);
    for (int l = 0; l < c->nlev; ++l) CK(alloc_vectors<double>(c, c->v64[l], c->lev[l].g, gm, c->lev[l].kind >= 4));
  } else {
    c->v64.resize(1);
    const size_t bytes = sizeof(double2) * (size_t)g0.vstride * c->B;
    CK(dalloc(c, (void**)&c->v64[0].x, bytes));
    CK(dalloc(c, (void**)&c->v64[0].b, bytes));
    c->v32.resize(c->nlev);
    for (int l = 0; l < c->nlev; ++l) {
      CK(alloc_vectors<float>(c, c->v32[l], c->lev[l].g, gm, c->lev[l].kind >= 4));
      if (l > 0 && c->lev[l].kind <= 3) {
        const Level& L = c->lev[l];
        const long long S = (long long)(2 * L.radius + 1) * (2 * L.radius + 1);
        CK(dalloc(c, (void**)&c->v32[l].st, sizeof(float2) * S * L.plane));
        CK(dalloc(c, (void**)&c->v32[l].dinv, sizeof(float2) * L.plane));
        launch_to_float(L.st, c->v32[l].st, S * L.plane, s);
        launch_to_float(L.dinv, c->v32[l].dinv, L.plane, s);
      }
    }
  }
  // coarse-cycle interpreter: every level from the first one with at most
  // opt.coarse_nodes nodes down to the coarsest grid
  c->lc = 1 << 30;
  if (o.coarse_nodes > 0)
    for (int l = 0; l < c->nlev; ++l)
      if (c->lev[l].plane <= o.coarse_nodes) {
        c->lc = l;
        break;
      }
  CK(cudaStreamSynchronize(s));
  if (c->lc < c->nlev) {
    if (!mixed) CK(build_plan<double>(c, c->lc, c->plan64));
    else CK(build_plan<float>(c, c->lc, c->plan32));
    if (o.coarse_mode == 1 && c->nlev <= COOP_MAXLEV) {   // cooperative grid: all co-resident blocks, split evenly over the RHS
      const int gmax = mixed ? coop_max_blocks<float>(c->ncoarse) : coop_max_blocks<double>(c->ncoarse);
      if (gmax >= c->B) {
        c->coop_grid = (gmax / c->B) * c->B;
        CK(dalloc(c, (void**)&c->coop.bar, sizeof(unsigned) * 2));
        CK(dalloc(c, (void**)&c->coop.partial, sizeof(double) * (size_t)c->coop_grid * NVMAX));
        c->coop.err = c->n_active + 1;
        c->coop.spin_limit = 1LL << 22;
      }
    }
  }
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(s));
  if (o.krylov > 0) {   // FGMRES(m) basis, preconditioned vectors and scalars
    FgArgs& a = c->fg;
    const int m = o.krylov;
    a.g = g0;
    a.B = c->B;
    a.m = m;
    a.vlen = g0.vstride * c->B;
    fg_geometry(g0, c->B, !mixed, a);
    const size_t zb = mixed ? sizeof(float2) : sizeof(double2);
    CK(dalloc(c, &a.V, zb * (size_t)a.vlen * (m + 1)));
    CK(dalloc(c, &a.Z, zb * (size_t)a.vlen * m));
    CK(dalloc(c, (void**)&a.X, sizeof(double2) * (size_t)a.vlen));
    CK(dalloc(c, (void**)&a.b, sizeof(double2) * (size_t)a.vlen));
    a.sd = FgLayout{m}.size();
    CK(dalloc(c, (void**)&a.S, sizeof(double) * (size_t)a.sd * c->B));
    CK(dalloc(c, (void**)&a.kst, sizeof(int) * 2 * c->B));
    CK(dalloc(c, (void**)&a.partial, sizeof(double) * (size_t)a.nvp * a.nbr * c->B));
    CK(dalloc(c, (void**)&a.tickets, sizeof(unsigned) * c->B));
  }
  CK(cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking));
  if (o.smoother == 1) {   // the side stream takes the priority of the handle's stream
    int sprio = 0;
    if (o.stream) CK(cudaStreamGetPriority((cudaStream_t)o.stream, &sprio));
    CK(cudaStreamCreateWithPriority(&c->side, cudaStreamNonBlocking, sprio));
    CK(cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming));
  }
  return MG_OK;
}

mg_status mg_setup(mg_handle* out, int nx, int ny, double h, const double* k_field, double k_const, double beta2,
                   int levels, const mg_options* opt) {
  if (!out) FAIL(MG_EINVAL, "out is NULL");
  *out = nullptr;
  mg_options o;
  if (opt) o = *opt; else mg_default_options(&o);
  if (nx < 2 || ny < 2) FAIL(MG_EINVAL, "grid needs nx, ny >= 2 (got %d, %d)", nx, ny);
  if (!(h > 0) || !(beta2 >= 0) || levels < 0) FAIL(MG_EINVAL, "need h > 0, beta2 >= 0, levels >= 0");
  if (!k_field && !(k_const >= 0)) FAIL(MG_EINVAL, "k_const must be >= 0");
  if (o.cycle != 1 && o.cycle != 2) FAIL(MG_EINVAL, "cycle must be 1 (V) or 2 (W)");
  if (o.smoother != 0 && o.smoother != 1) FAIL(MG_EINVAL, "smoother must be 0 (Jacobi) or 1 (GMRES(3))");
  if (o.nu_pre < 0 || o.nu_post < 0 || o.nu_pre + o.nu_post > 64) FAIL(MG_EINVAL, "bad nu_pre / nu_post");
  if (!(o.omega > 0)) FAIL(MG_EINVAL, "omega must be > 0");
  if (o.precision < 0 || o.precision > 2) FAIL(MG_EINVAL, "precision must be 0, 1 or 2");
  if (o.max_cycles < 1 || o.min_coarse < 1) FAIL(MG_EINVAL, "max_cycles and min_coarse must be >= 1");
  if (o.batch < 1 || o.batch > 65535) FAIL(MG_EINVAL, "batch must be in 1..65535");
  if (o.coarse_nodes < 0) FAIL(MG_EINVAL, "coarse_nodes must be >= 0");
  if (o.coarse_mode != 0 && o.coarse_mode != 1) FAIL(MG_EINVAL, "coarse_mode must be 0 or 1");
  if (o.fuse != 0 && o.fuse != 1) FAIL(MG_EINVAL, "fuse must be 0 or 1");
  if (o.tile_rows < 0 || o.tile_rows > RYMAX) FAIL(MG_EINVAL, "tile_rows must be in 0..4");
  if (o.march < -1 || o.march > 1) FAIL(MG_EINVAL, "march must be -1, 0 or 1");
  if (o.krylov < 0 || o.krylov > FG_MAXM) FAIL(MG_EINVAL, "krylov must be in 0..%d", FG_MAXM);
  if (o.krylov > 0 && o.precision == 2) FAIL(MG_EINVAL, "the FGMRES outer loop needs precision 0 or 1");
  if (o.transfer != 0 && o.transfer != 1) FAIL(MG_EINVAL, "transfer must be 0 (Eq. (xex)) or 1 (linear)");
  if (o.flat != 0 && o.flat != 1) FAIL(MG_EINVAL, "flat must be 0 or 1");
  if (o.kron_chunk < 0 || o.kron_chunk > 1024) FAIL(MG_EINVAL, "kron_chunk must be in 0..1024");
  if (o.abc != 1 && o.abc != 2) FAIL(MG_EINVAL, "abc must be 1 or 2");
  if (o.abc == 2 && o.precision == 2)
    FAIL(MG_EINVAL, "the second-order absorbing rows need precision 0 or 1 (the float-float loop keeps the first-order rows)");
  if ((long long)(nx + 1) * (ny + 1) > (1LL << 31) / 8) FAIL(MG_EINVAL, "grid too large");
  mg_ctx* c = new mg_ctx();
  c->opt = o;
  c->nx = nx;
  c->ny = ny;
  c->h = h;
  c->kconst = k_field ? 0.0 : k_const;
  c->beta2 = beta2;
  c->B = o.batch;
  c->nlev = levels;
  mg_status st = setup_impl(c, k_field);
  if (st != MG_OK) {
    delete c;
    return st;
  }
  *out = c;
  return MG_OK;
}

mg_status mg_setup_ragged(mg_handle* out, int nprob, const int* nx, const int* ny, const double* h,
                          const double* k_const, const double* beta2, const mg_options* opt) {
  if (!out) FAIL(MG_EINVAL, "out is NULL");
  *out = nullptr;
  if (nprob < 1 || !nx || !ny || !h || !k_const || !beta2)
    FAIL(MG_EINVAL, "ragged batch needs nprob >= 1 and its arrays");
  mg_options o;
  if (opt) o = *opt; else mg_default_options(&o);
  if (o.batch != 1) FAIL(MG_EINVAL, "a ragged batch solves one right-hand side per problem (batch must be 1)");
  mg_ctx* c = new mg_ctx();
  c->opt = o;
  // Problems with the same grid, cell size, wavenumber and shift (compared
  // bit for bit) share one hierarchy and are solved as the right-hand sides
  // of one batched handle (flat = 0); with flat = 1 every problem has its
  // own handle, as the flattened launches need.
  std::vector<std::vector<int>> groups;
  for (int p = 0; p < nprob; ++p) {
    int gi = -1;
    if (o.flat == 0)
      for (int q = 0; q < (int)groups.size() && gi < 0; ++q) {
        const int r = groups[q][0];
        if (nx[r] == nx[p] && ny[r] == ny[p] && h[r] == h[p] && k_const[r] == k_const[p] && beta2[r] == beta2[p])
          gi = q;
      }
    if (gi < 0) {
      gi = (int)groups.size();
      groups.emplace_back();
    }
    groups[gi].push_back(p);
  }
  const int ng = (int)groups.size();
  // stream priorities by problem size: the largest problems (the longest
  // chains of cycles) get the highest priority, so their blocks are
  // scheduled first whenever the problems compete for the GPU
  int prio_least = 0, prio_greatest = 0;
  cudaDeviceGetStreamPriorityRange(&prio_least, &prio_greatest);
  const int nprio = prio_least - prio_greatest + 1;
  auto nodes_of = [&](int q) { return (long long)(nx[groups[q][0]] + 1) * (ny[groups[q][0]] + 1); };
  std::vector<int> order(ng);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return nodes_of(a) > nodes_of(b); });
  std::vector<int> prio(ng, prio_least);
  for (int r = 0; r < ng; ++r) prio[order[r]] = prio_greatest + (int)((long long)r * nprio / ng);
  for (int q = 0; q < ng; ++q) {
    const int p = groups[q][0];
    cudaStream_t sp;
    if (cudaStreamCreateWithPriority(&sp, cudaStreamNonBlocking, prio[q]) != cudaSuccess) {
      delete c;
      FAIL(MG_ECUDA, "stream creation failed");
    }
    mg_options op = o;
    op.stream = sp;
    op.batch = (int)groups[q].size();
    mg_handle hp = nullptr;
    mg_status st = mg_setup(&hp, nx[p], ny[p], h[p], nullptr, k_const[p], beta2[p], 0, &op);
    if (st != MG_OK) {
      cudaStreamDestroy(sp);
      std::string m = g_err;
      delete c;
      FAIL(st, "problem %d of the ragged batch: %s", p, m.c_str());
    }
    hp->own_stream = sp;
    c->sub.push_back(hp);
    c->members.push_back(groups[q]);
    double2* stg = nullptr;
    if (groups[q].size() > 1 &&
        dalloc(c, (void**)&stg, sizeof(double2) * 2 * groups[q].size() * (size_t)nodes_of(q)) != cudaSuccess) {
      delete c;
      FAIL(MG_ENOMEM, "ragged batch: staging buffers of problem %d's group", p);
    }
    c->stage.push_back(stg);
  }
  long long total = 0;
  for (mg_ctx* q : c->sub) total += (long long)(q->nx + 1) * (q->ny + 1) * q->B;
  // The fine-level kernels (use_march) are chosen for the whole batch's
  // load, except on the largest problems: they run the most cycles, their
  // chain of cycles is the batch's critical path, and they decide by their
  // own size (a single large right-hand side runs its fine level faster
  // node-parallel than as row marches).
  long long nmax = 0;
  for (mg_ctx* q : c->sub) nmax = std::max(nmax, (long long)(q->nx + 1) * (q->ny + 1));
  for (mg_ctx* q : c->sub) {
    const long long own = (long long)(q->nx + 1) * (q->ny + 1);
    q->peer_nodes = own == nmax ? 0 : total - own * q->B;
  }
  c->nx = c->sub[0]->nx;
  c->ny = c->sub[0]->ny;
  c->nlev = c->sub[0]->nlev;
  // one flattened launch per kernel over all problems: GMRES(3) smoothing
  // with the march kernels, precision 0 or 1, the stand-alone cycle, and
  // every problem's coarsest grid inside its coarse-cycle launch
  bool flat = o.flat == 1 && o.smoother == 1 && o.fuse == 1 && o.march != 0 && o.precision <= 1 && o.krylov == 0 && o.abc == 1 &&
              o.coarse_mode == 0;
  for (mg_ctx* q : c->sub) flat = flat && q->lc <= q->nlev - 1 && q->coop_grid == 0;
  if (flat) {
    mg_status fs = MG_OK;
    if (cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithPriority(&c->side, cudaStreamNonBlocking, prio_greatest) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming) != cudaSuccess ||
        dalloc(c, (void**)&c->d_counts, sizeof(int) * 2 * nprob) != cudaSuccess ||
        cudaMallocHost((void**)&c->h_counts, sizeof(int) * 2 * nprob) != cudaSuccess)
      fs = MG_ENOMEM;
    int lmax = 0;
    for (mg_ctx* q : c->sub) lmax = std::max(lmax, q->nlev);
    for (int l = 0; l < lmax && fs == MG_OK; ++l) {
      cudaStream_t cs;
      cudaEvent_t ef, ej;
      if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) { fs = MG_ECUDA; break; }
      c->cstreams.push_back(cs);
      if (cudaEventCreateWithFlags(&ef, cudaEventDisableTiming) != cudaSuccess) { fs = MG_ECUDA; break; }
      c->cfork.push_back(ef);
      if (cudaEventCreateWithFlags(&ej, cudaEventDisableTiming) != cudaSuccess) { fs = MG_ECUDA; break; }
      c->cjoin.push_back(ej);
    }
    if (fs != MG_OK) {
      delete c;
      FAIL(fs, "ragged batch: allocation of the flattened cycle failed");
    }
    c->flat = true;
  }
  *out = c;
  return MG_OK;
}

static mg_status capture(mg_ctx* c) {
  if (c->gexec) return MG_OK;
  CK(cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal));
  if (c->opt.precision == 0) emit_fp64_iteration(c, c->cap);
  else emit_mixed_iteration(c, c->cap);
  cudaGraph_t g;
  cudaError_t e = cudaStreamEndCapture(c->cap, &g);
  if (e != cudaSuccess) FAIL(MG_ECUDA, "graph capture failed: %s", cudaGetErrorString(e));
  c->graph = g;
  return instantiate_graph(g, &c->gexec, &c->graph_kernels);
}

// Graph of one preconditioning cycle for the FGMRES outer loop: the cycle
// from the level-0 iterate (zeroed by the prep kernel) on the level-0
// right-hand side, the result left in the level-0 iterate.
static mg_status capture_precond(mg_ctx* c) {
  if (c->pexec) return MG_OK;
  CK(cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal));
  if (c->opt.precision == 0) {
    Emit<double> e{c, c->cap, {}, {}, c->lc, &c->plan64};
    e.init();
    e.zx[0] = 1;   // the FGMRES restart and orthogonalisation kernels clear the cycle's x
    e.cycle(0);
    if (e.cur[0] != c->v64[0].x) launch_copy_masked<double>(c->lev[0].g, e.cur[0], c->v64[0].x, c->B, c->active, c->cap);
  } else {
    Emit<float> e{c, c->cap, {}, {}, c->lc, &c->plan32};
    e.init();
    e.zx[0] = 1;
    e.cycle(0);
    if (e.cur[0] != c->v32[0].x) launch_copy_masked<float>(c->lev[0].g, e.cur[0], c->v32[0].x, c->B, c->active, c->cap);
  }
  cudaGraph_t g;
  cudaError_t e = cudaStreamEndCapture(c->cap, &g);
  if (e != cudaSuccess) FAIL(MG_ECUDA, "graph capture failed: %s", cudaGetErrorString(e));
  c->pgraph = g;
  return instantiate_graph(g, &c->pexec, &c->pgraph_kernels);
}

// FGMRES(m) with the cycle as the right preconditioner (fgmres.cu): every
// right-hand side runs its own restart cycles; the steps of one restart
// cycle run in lockstep over the batch, a RHS leaving it (residual estimate
// at tol, breakdown, or its step allowance used) is masked out of the
// remaining steps, and all of them take the update and the restart test
// together.  The host polls the count of RHS still inside the restart cycle
// after every step.
static mg_status solve_fgmres(mg_ctx* c, const void* rhs, void* x, double tol, int conj, int* cycles_out,
                              double* relres_out) {
  if (!rhs || !x) FAIL(MG_EINVAL, "rhs and x must be device pointers");
  if (!(tol > 0)) FAIL(MG_EINVAL, "tol must be > 0");
  cudaStream_t s = (cudaStream_t)c->opt.stream;
  const Grid& g0 = c->lev[0].g;
  const int B = c->B, m = c->opt.krylov;
  const bool mixed = c->opt.precision == 1;
  mg_status st = capture_precond(c);
  if (st != MG_OK) return st;
  const FgArgs a = fg_args(c, tol);
  launch_pack<double>(g0, (const double2*)rhs, (double2*)a.b, B, conj, s);
  launch_pack<double>(g0, (const double2*)x, a.X, B, conj, s);
  launch_vecnorm_fin<double>(g0, a.b, B, c->bnorm, c->partial, c->tickets, s);
  std::vector<double> bn(B);
  CK(cudaMemcpyAsync(bn.data(), c->bnorm, sizeof(double) * B, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  std::vector<int> zero(B, 0), stt(B);
  std::vector<double> bsafe(B);
  for (int b = 0; b < B; ++b) {
    bsafe[b] = bn[b] > 0 ? bn[b] : 1.0;
    stt[b] = bn[b] > 0 ? 0 : 1;
    if (bn[b] == 0.0) CK(cudaMemsetAsync(a.X + (size_t)b * g0.vstride, 0, sizeof(double2) * g0.vstride, s));
  }
  CK(cudaMemcpyAsync(c->active, zero.data(), sizeof(int) * B, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(c->state, stt.data(), sizeof(int) * B, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(c->cycles, zero.data(), sizeof(int) * B, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(c->bnorm, bsafe.data(), sizeof(double) * B, cudaMemcpyHostToDevice, s));
  CK(cudaMemsetAsync(a.kst, 0, sizeof(int) * 2 * B, s));
  if (c->coop.bar) CK(cudaMemsetAsync(c->coop.bar, 0, sizeof(unsigned) * 2, s));
  CK(cudaMemsetAsync(c->relres, 0, sizeof(double) * B, s));
  CK(cudaMemsetAsync(c->hist, 0, sizeof(double) * (size_t)c->hist_len * B, s));
  long long launches = 3, graphs = 0;   // 2 pack + norm
  cx<float>* cb32 = mixed ? c->v32[0].b : nullptr;
  cx<float>* cx32 = mixed ? c->v32[0].x : nullptr;
  while (true) {
    CK(cudaMemsetAsync(c->n_active, 0, sizeof(int) * 2, s));
    if (mixed) launch_fg_restart<float>(a, cb32, cx32, s);
    else launch_fg_restart<double>(a, c->v64[0].b, c->v64[0].x, s);
    ++launches;
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(c->h_n_active, c->n_active, sizeof(int) * 2, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (c->h_n_active[0] == 0) break;
    for (int j = 0; j < m; ++j) {
      CK(cudaGraphLaunch(c->pexec, s));
      if (mixed) {
        launch_fg_dots<float>(a, j, cx32, s);
        launch_fg_orth<float>(a, j, cb32, cx32, s);
      } else {
        launch_fg_dots<double>(a, j, c->v64[0].x, s);
        launch_fg_orth<double>(a, j, c->v64[0].b, c->v64[0].x, s);
      }
      launches += 2 + c->pgraph_kernels;
      ++graphs;
      CK(cudaGetLastError());
      CK(cudaMemcpyAsync(c->h_n_active, c->n_active, sizeof(int) * 2, cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      if (c->h_n_active[1] != 0) FAIL(MG_ETIMEOUT, "a grid-wide barrier of the cooperative cycle kernel timed out");
      if (c->h_n_active[0] == 0) break;
    }
    if (mixed) launch_fg_update<float>(a, s);
    else launch_fg_update<double>(a, s);
    ++launches;
  }
  launch_unpack<double>(g0, a.X, (double2*)x, B, conj, s);
  ++launches;
  c->last_launches = launches;
  c->last_graphs = graphs;
  std::vector<int> cyc(B);
  std::vector<double> rr(B);
  CK(cudaMemcpyAsync(stt.data(), c->state, sizeof(int) * B, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(cyc.data(), c->cycles, sizeof(int) * B, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(rr.data(), c->relres, sizeof(double) * B, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  CK(cudaGetLastError());
  bool div = false, maxit = false;
  for (int b = 0; b < B; ++b) {
    if (cycles_out) cycles_out[b] = cyc[b];
    if (relres_out) relres_out[b] = rr[b];
    div |= stt[b] == 2;
    maxit |= stt[b] == 0;
  }
  if (div) FAIL(MG_EDIVERGED, "relative residual not finite");
  if (maxit) FAIL(MG_EMAXIT, "max_cycles (%d) reached before tol", c->opt.max_cycles);
  return MG_OK;
}

// A solve in four phases, so that several handles (the problems of a ragged
// batch) can run their cycles side by side on their own streams:
// solve_begin packs the inputs, sets up the per-RHS control arrays and runs
// the initial stopping test; solve_launch issues one cycle (graph) and the
// asynchronous read-back of the active count; solve_more says, after the
// stream is synchronised, whether another cycle is needed; solve_end
// unpacks x and reports.
static mg_status solve_begin(mg_ctx* c, const void* rhs, void* x, double tol, int conj) {
  if (!rhs || !x) FAIL(MG_EINVAL, "rhs and x must be device pointers");
  if (!(tol > 0)) FAIL(MG_EINVAL, "tol must be > 0");
  cudaStream_t s = (cudaStream_t)c->opt.stream;
  const Grid& g0 = c->lev[0].g;
  const int B = c->B;
  const bool mixed = c->opt.precision >= 1, ffo = c->opt.precision == 2;
  mg_status st = capture(c);
  if (st != MG_OK) return st;
  if (ffo) {   // level-0 outer vectors in float-float
    launch_ff_pack(g0, (const double2*)rhs, c->v64[0].b, B, conj, s);
    launch_ff_pack(g0, (const double2*)x, c->v64[0].x, B, conj, s);
    launch_ff_norm(g0, c->v64[0].b, B, c->bnorm, c->partial, c->tickets, s);
  } else {
    launch_pack<double>(g0, (const double2*)rhs, c->v64[0].b, B, conj, s);
    launch_pack<double>(g0, (const double2*)x, c->v64[0].x, B, conj, s);
    launch_vecnorm_fin<double>(g0, c->v64[0].b, B, c->bnorm, c->partial, c->tickets, s);
  }
  std::vector<double> bn(B);
  CK(cudaMemcpyAsync(bn.data(), c->bnorm, sizeof(double) * B, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  std::vector<int> act(B), zero(B, 0), stt(B);
  std::vector<double> bsafe(B);
  const double tolv[2] = {tol, 1e6};
  int nact = 0;
  for (int b = 0; b < B; ++b) {
    act[b] = bn[b] > 0.0;
    nact += act[b];
    bsafe[b] = bn[b] > 0 ? bn[b] : 1.0;
    stt[b] = act[b] ? 0 : 1;
    if (bn[b] == 0.0) CK(cudaMemsetAsync(c->v64[0].x + (size_t)b * g0.vstride, 0, sizeof(double2) * g0.vstride, s));
  }
  CK(cudaMemcpyAsync(c->active, act.data(), sizeof(int) * B, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(c->state, stt.data(), sizeof(int) * B, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(c->cycles, zero.data(), sizeof(int) * B, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(c->bnorm, bsafe.data(), sizeof(double) * B, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(c->tolp, tolv, sizeof(double) * 2, cudaMemcpyHostToDevice, s));
  const int ctl2[2] = {nact, 0};
  CK(cudaMemcpyAsync(c->n_active, ctl2, sizeof(int) * 2, cudaMemcpyHostToDevice, s));
  if (c->coop.bar) CK(cudaMemsetAsync(c->coop.bar, 0, sizeof(unsigned) * 2, s));
  CK(cudaMemsetAsync(c->relres, 0, sizeof(double) * B, s));
  CK(cudaMemsetAsync(c->hist, 0, sizeof(double) * (size_t)c->hist_len * B, s));
  if (ffo)   // initial test on x0
    launch_ff_resid_cast_stop(g0, c->hffc, c->kf64, c->h, c->ffdiag, c->v64[0].x, c->v64[0].b, c->v32[0].b, B,
                              ctl(c), 0, s);
  else if (mixed)
    launch_resid_cast_stop(g0, op64(c, 0), c->v64[0].x, c->v64[0].b, c->v32[0].b, B, ctl(c), 0, s);
  else
    launch_resnorm_stop<double>(g0, op64(c, 0), c->v64[0].x, c->v64[0].b, B, ctl(c), 0, s);
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(c->h_n_active, c->n_active, sizeof(int) * 2, cudaMemcpyDeviceToHost, s));
  c->done = 0;
  c->last_launches = 5;   // 2 pack + norm + initial residual test + unpack
  c->last_graphs = 0;
  return MG_OK;
}

static bool solve_more(const mg_ctx* c) {
  return c->h_n_active[0] > 0 && c->h_n_active[1] == 0 && c->done < c->opt.max_cycles;
}

static mg_status solve_launch(mg_ctx* c) {
  cudaStream_t s = (cudaStream_t)c->opt.stream;
  CK(cudaGraphLaunch(c->gexec, s));
  ++c->done;
  c->last_graphs += 1;
  c->last_launches += c->graph_kernels;
  CK(cudaMemcpyAsync(c->h_n_active, c->n_active, sizeof(int) * 2, cudaMemcpyDeviceToHost, s));
  return MG_OK;
}

static mg_status solve_end(mg_ctx* c, void* x, int conj, int* cycles_out, double* relres_out) {
  cudaStream_t s = (cudaStream_t)c->opt.stream;
  const Grid& g0 = c->lev[0].g;
  const int B = c->B;
  if (c->opt.precision == 2)
    launch_ff_unpack(g0, c->v64[0].x, (double2*)x, B, conj, s);
  else
    launch_unpack<double>(g0, c->v64[0].x, (double2*)x, B, conj, s);
  if (c->h_n_active[1] != 0) {
    cudaStreamSynchronize(s);
    FAIL(MG_ETIMEOUT, "a grid-wide barrier of the cooperative cycle kernel timed out");
  }
  std::vector<int> cyc(B), stt(B);
  std::vector<double> rr(B);
  CK(cudaMemcpyAsync(stt.data(), c->state, sizeof(int) * B, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(cyc.data(), c->cycles, sizeof(int) * B, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(rr.data(), c->relres, sizeof(double) * B, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  CK(cudaGetLastError());
  bool div = false, maxit = false;
  for (int b = 0; b < B; ++b) {
    if (cycles_out) cycles_out[b] = cyc[b];
    if (relres_out) relres_out[b] = rr[b];
    div |= stt[b] == 2;
    maxit |= stt[b] == 0;
  }
  if (div) FAIL(MG_EDIVERGED, "relative residual diverged (> 1e6 or not finite)");
  if (maxit) FAIL(MG_EMAXIT, "max_cycles (%d) reached before tol", c->opt.max_cycles);
  return MG_OK;
}

// Ragged batch: every problem on its own stream, one cycle graph per
// unconverged problem per round, all problems polled after each round.
static mg_status solve_ragged(mg_ctx* c, const void* rhs, void* x, double tol, int* cycles_out, double* relres_out,
                              int conj) {
  if (!rhs || !x) FAIL(MG_EINVAL, "rhs and x must be device pointers");
  CK(cudaStreamSynchronize((cudaStream_t)c->opt.stream));   // the caller's inputs are ready
  const int P = (int)c->sub.size();   // handles; handle p solves the problems members[p]
  int nprob = 0;
  for (const auto& m : c->members) nprob += (int)m.size();
  std::vector<size_t> pn(nprob), off(nprob + 1, 0);   // each problem's nodes and offset in rhs and x
  for (int p = 0; p < P; ++p)
    for (int m : c->members[p]) pn[m] = (size_t)(c->sub[p]->nx + 1) * (c->sub[p]->ny + 1);
  for (int m = 0; m < nprob; ++m) off[m + 1] = off[m] + pn[m];
  const double2* R = (const double2*)rhs;
  double2* X = (double2*)x;
  // handle p's right-hand sides and iterates: the caller's arrays for a
  // single problem, else the staging buffer (rhs of every member, then x)
  // filled on the handle's stream
  auto in_rhs = [&](int p) -> const double2* {
    return c->members[p].size() == 1 ? R + off[c->members[p][0]] : c->stage[p];
  };
  auto in_x = [&](int p) -> double2* {
    const size_t B = c->members[p].size();
    return B == 1 ? X + off[c->members[p][0]] : c->stage[p] + B * pn[c->members[p][0]];
  };
  for (int p = 0; p < P; ++p) {
    const size_t B = c->members[p].size();
    if (B == 1) continue;
    cudaStream_t sp = (cudaStream_t)c->sub[p]->opt.stream;
    for (size_t i = 0; i < B; ++i) {
      const int m = c->members[p][i];
      CK(cudaMemcpyAsync(c->stage[p] + i * pn[m], R + off[m], sizeof(double2) * pn[m], cudaMemcpyDeviceToDevice, sp));
      CK(cudaMemcpyAsync(in_x(p) + i * pn[m], X + off[m], sizeof(double2) * pn[m], cudaMemcpyDeviceToDevice, sp));
    }
  }
  // handle p's results back into the caller's arrays
  auto scatter = [&](int p, const int* cb, const double* rb) -> mg_status {
    const size_t B = c->members[p].size();
    for (size_t i = 0; i < B; ++i) {
      const int m = c->members[p][i];
      if (cycles_out) cycles_out[m] = cb[i];
      if (relres_out) relres_out[m] = rb[i];
    }
    if (B == 1) return MG_OK;
    cudaStream_t sp = (cudaStream_t)c->sub[p]->opt.stream;
    for (size_t i = 0; i < B; ++i) {
      const int m = c->members[p][i];
      CK(cudaMemcpyAsync(X + off[m], in_x(p) + i * pn[m], sizeof(double2) * pn[m], cudaMemcpyDeviceToDevice, sp));
    }
    CK(cudaStreamSynchronize(sp));
    return MG_OK;
  };
  mg_status worst = MG_OK;
  std::string msg;
  auto note = [&](mg_status st) {
    if (st != MG_OK && (worst == MG_OK || st == MG_EDIVERGED)) {
      worst = st;
      msg = g_err;
    }
  };
  long long launches = 0;
  if (c->opt.krylov > 0) {   // FGMRES: the handles one after the other
    for (int p = 0; p < P; ++p) {
      const size_t B = c->members[p].size();
      std::vector<int> cb(B);
      std::vector<double> rb(B);
      mg_status st = solve_fgmres(c->sub[p], in_rhs(p), in_x(p), tol, conj, cb.data(), rb.data());
      launches += c->sub[p]->last_launches;
      note(st);
      if (st != MG_OK && st != MG_EMAXIT && st != MG_EDIVERGED) return st;
      mg_status sc = scatter(p, cb.data(), rb.data());
      if (sc != MG_OK) return sc;
    }
    c->last_launches = launches;
    if (worst != MG_OK) FAIL(worst, "problem(s) of the ragged batch: %s", msg.c_str());
    return MG_OK;
  }
  for (int p = 0; p < P; ++p) {
    mg_status st = solve_begin(c->sub[p], in_rhs(p), in_x(p), tol, conj);
    if (st != MG_OK) return st;
  }
  if (c->flat) {   // every cycle one graph over all problems (emit_ragged_iteration)
    for (int p = 0; p < P; ++p) CK(cudaStreamSynchronize((cudaStream_t)c->sub[p]->opt.stream));
    mg_status st = capture_ragged(c);
    if (st != MG_OK) return st;
    cudaStream_t s = (cudaStream_t)c->opt.stream;
    int left = 0;
    for (int p = 0; p < P; ++p) left += c->sub[p]->h_n_active[0] > 0;
    for (int round = 0; left > 0 && round < c->opt.max_cycles; ++round) {
      CK(cudaGraphLaunch(c->gexec, s));
      CK(cudaStreamSynchronize(s));
      launches += c->graph_kernels;
      left = 0;
      for (int p = 0; p < P; ++p) left += c->h_counts[p] > 0;
    }
  } else {
    // Each handle runs its own cycles: a handle whose stream has drained (its
    // active count read back) gets its next cycle at once, without waiting
    // for the slower ones, so the small problems finish early and the
    // largest one, on the highest-priority stream, is never held back by a
    // round barrier.
    std::vector<char> running(P, 1);
    int left = P;
    while (left > 0) {
      bool progressed = false;
      for (int p = 0; p < P; ++p) {
        if (!running[p]) continue;
        const cudaError_t q = cudaStreamQuery((cudaStream_t)c->sub[p]->opt.stream);
        if (q == cudaErrorNotReady) continue;
        CK(q);
        progressed = true;
        if (solve_more(c->sub[p])) {
          mg_status st = solve_launch(c->sub[p]);
          if (st != MG_OK) return st;
        } else {
          running[p] = 0;
          --left;
        }
      }
      if (!progressed) std::this_thread::yield();
    }
  }
  for (int p = 0; p < P; ++p) {
    const size_t B = c->members[p].size();
    std::vector<int> cb(B);
    std::vector<double> rb(B);
    mg_status st = solve_end(c->sub[p], in_x(p), conj, cb.data(), rb.data());
    launches += c->sub[p]->last_launches;
    note(st);
    if (st != MG_OK && st != MG_EMAXIT && st != MG_EDIVERGED) return st;
    mg_status sc = scatter(p, cb.data(), rb.data());
    if (sc != MG_OK) return sc;
  }
  c->last_launches = launches;
  if (worst != MG_OK) FAIL(worst, "problem(s) of the ragged batch: %s", msg.c_str());
  return MG_OK;
}

static mg_status solve_impl(mg_ctx* c, const void* rhs, void* x, double tol, int* cycles_out, double* relres_out,
                            int conj) {
  if (!c->sub.empty()) return solve_ragged(c, rhs, x, tol, cycles_out, relres_out, conj);
  if (c->opt.krylov > 0) return solve_fgmres(c, rhs, x, tol, conj, cycles_out, relres_out);
  mg_status st = solve_begin(c, rhs, x, tol, conj);
  if (st != MG_OK) return st;
  cudaStream_t s = (cudaStream_t)c->opt.stream;
  CK(cudaStreamSynchronize(s));
  while (solve_more(c)) {
    st = solve_launch(c);
    if (st != MG_OK) return st;
    CK(cudaStreamSynchronize(s));
  }
  return solve_end(c, x, conj, cycles_out, relres_out);
}

mg_status mg_solve(mg_handle h, const void* rhs, void* x, double tol, int* cycles_out, double* relres_out) {
  if (!h) FAIL(MG_EINVAL, "NULL handle");
  return solve_impl(h, rhs, x, tol, cycles_out, relres_out, 0);
}

mg_status mg_adjoint(mg_handle h, const void* rhs_adj, void* lam, double tol, int* cycles_out, double* relres_out) {
  if (!h) FAIL(MG_EINVAL, "NULL handle");
  return solve_impl(h, rhs_adj, lam, tol, cycles_out, relres_out, 1);
}

mg_status mg_gradient(mg_handle h, const void* u, const void* lam, int nsrc, const double* m, double omega_f,
                      double* g) {
  if (h && !h->sub.empty()) FAIL(MG_ESTATE, "not available on a ragged-batch handle");
  if (!h) FAIL(MG_EINVAL, "NULL handle");
  if (!u || !lam || !m || !g || nsrc < 1 || !(omega_f > 0)) FAIL(MG_EINVAL, "bad gradient arguments");
  if (h->opt.abc != 1) FAIL(MG_EINVAL, "the gradient differentiates the first-order absorbing rows only (abc 1)");
  cudaStream_t s = (cudaStream_t)h->opt.stream;
  launch_gradient(h->nx, h->ny, h->h, m, omega_f, (const double2*)u, (const double2*)lam, nsrc, g, s);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(s));
  return MG_OK;
}

mg_status mg_level_info(mg_handle h, int level, int* nx, int* ny, int* radius, int* nlevels) {
  if (h && !h->sub.empty()) FAIL(MG_ESTATE, "not available on a ragged-batch handle");
  if (!h) FAIL(MG_EINVAL, "NULL handle");
  if (nlevels) *nlevels = h->nlev;
  if (level < 0 || level >= h->nlev) FAIL(MG_EINVAL, "level %d out of range", level);
  if (nx) *nx = h->lev[level].g.nx;
  if (ny) *ny = h->lev[level].g.ny;
  if (radius) *radius = h->lev[level].radius;
  return MG_OK;
}

mg_status mg_apply(mg_handle h, int level, const void* x, void* y) {
  if (h && !h->sub.empty()) FAIL(MG_ESTATE, "not available on a ragged-batch handle");
  if (!h) FAIL(MG_EINVAL, "NULL handle");
  if (level < 0 || level >= h->nlev || !x || !y) FAIL(MG_EINVAL, "bad mg_apply arguments");
  cudaStream_t s = (cudaStream_t)h->opt.stream;
  const Grid& g = h->lev[level].g;
  const size_t bytes = sizeof(double2) * (size_t)g.vstride * h->B;
  double2 *a = nullptr, *b = nullptr;
  CK(cudaMalloc(&a, bytes));
  cudaError_t e = cudaMalloc(&b, bytes);
  if (e != cudaSuccess) { cudaFree(a); FAIL(MG_ENOMEM, "mg_apply scratch allocation failed"); }
  cudaMemsetAsync(a, 0, bytes, s);
  cudaMemsetAsync(b, 0, bytes, s);
  launch_pack<double>(g, (const double2*)x, a, h->B, 0, s);
  launch_apply<double>(g, op64(h, level), a, b, h->B, nullptr, s);
  launch_unpack<double>(g, b, (double2*)y, h->B, 0, s);
  e = cudaStreamSynchronize(s);
  cudaFree(a);
  cudaFree(b);
  if (e != cudaSuccess) FAIL(MG_ECUDA, "mg_apply: %s", cudaGetErrorString(e));
  CK(cudaGetLastError());
  return MG_OK;
}

mg_status mg_get_stencil(mg_handle h, int level, void* out) {
  if (h && !h->sub.empty()) FAIL(MG_ESTATE, "not available on a ragged-batch handle");
  if (!h) FAIL(MG_EINVAL, "NULL handle");
  if (level < 0 || level >= h->nlev || !out) FAIL(MG_EINVAL, "bad mg_get_stencil arguments");
  cudaStream_t s = (cudaStream_t)h->opt.stream;
  launch_export_stencil(op64(h, level), h->lev[level].g.nx, h->lev[level].g.ny, h->lev[level].radius, (double2*)out,
                        s);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(s));
  return MG_OK;
}

mg_status mg_counters(mg_handle h, long long* kernel_launches, long long* graph_launches) {
  if (!h) FAIL(MG_EINVAL, "NULL handle");
  if (kernel_launches) *kernel_launches = h->last_launches;
  if (graph_launches) *graph_launches = h->last_graphs;
  return MG_OK;
}

mg_status mg_profile(mg_handle h, int what, int level, int reps, double* ms, double* bytes) {
  if (h && !h->sub.empty()) FAIL(MG_ESTATE, "not available on a ragged-batch handle");
  if (!h) FAIL(MG_EINVAL, "NULL handle");
  if (what < 0 || what > 6 || reps < 1 || !ms || !bytes) FAIL(MG_EINVAL, "bad mg_profile arguments");
  if (h->opt.precision >= 1) return profile_t<float>(h, what, level, reps, ms, bytes);
  return profile_t<double>(h, what, level, reps, ms, bytes);
}

mg_status mg_two_grid(mg_handle h, int nu, int max_iter, double* out) {
  if (h && !h->sub.empty()) FAIL(MG_ESTATE, "not available on a ragged-batch handle");
  if (!h || !out) FAIL(MG_EINVAL, "NULL handle or output");
  if (nu < 1 || nu > 8 || max_iter < 200 || max_iter > 1000000) FAIL(MG_EINVAL, "need 1 <= nu <= 8 and 200 <= max_iter <= 1e6");
  if (h->nlev < 2) FAIL(MG_EINVAL, "the two-grid analysis needs a hierarchy with two levels");
  const Grid& g0 = h->lev[0].g;
  const Grid& g1 = h->lev[1].g;
  if ((long long)(g0.nx + 1) * (g0.ny + 1) > 4096) FAIL(MG_EINVAL, "the two-grid analysis is dense: at most 4096 fine nodes");
  cudaError_t e = two_grid_analysis(op64(h, 0), op64(h, 1), g0.nx, g0.ny, g1.nx, g1.ny, h->opt.omega, h->xw, nu,
                                    max_iter, out, (cudaStream_t)h->opt.stream);
  if (e == cudaErrorMemoryAllocation) FAIL(MG_ENOMEM, "two-grid analysis: device allocation failed");
  if (e != cudaSuccess) FAIL(MG_ECUDA, "two-grid analysis: %s", cudaGetErrorString(e));
  return MG_OK;
}

mg_status mg_history(mg_handle h, double* hist, int cap) {
  if (h && !h->sub.empty()) FAIL(MG_ESTATE, "not available on a ragged-batch handle");
  if (!h) FAIL(MG_EINVAL, "NULL handle");
  if (!hist || cap < 1) FAIL(MG_EINVAL, "bad history buffer");
  cudaStream_t s = (cudaStream_t)h->opt.stream;
  std::vector<double> tmp((size_t)h->hist_len * h->B);
  CK(cudaMemcpyAsync(tmp.data(), h->hist, sizeof(double) * tmp.size(), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  for (int b = 0; b < h->B; ++b)
    for (int q = 0; q < cap; ++q) hist[(size_t)b * cap + q] = q < h->hist_len ? tmp[(size_t)b * h->hist_len + q] : 0.0;
  return MG_OK;
}

}  // extern "C"
