// Host-side declarations shared by the helmmg translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace hmg {

// Operator of one level in precision T, as handed to the launch wrappers.
// kind 1: matrix-free fine-level operator (c0, kf); kind 2 / 3: stored
// Galerkin stencil of that radius (st, dinv, plane); kind 4 / 5: constant-k
// Kronecker form of radius 2 / 3 (gx, wx, hy, wy, dinv).
template <class T> struct OpView {
  int kind;
  Op0Consts<T> c0;
  const T* kf;
  const cx<T>* st;
  const cx<T>* dinv;
  long long plane;
  const cx<T>* gx;
  const T* wx;
  const cx<T>* hy;
  const T* wy;
  // constant-k levels: rows [ty0, ty1) whose y-factor rows are hyc / wyc
  int ty0, ty1;
  cx<T> hyc[7];
  T wyc[7];
};
__host__ __device__ inline int op_radius(int kind) { return kind == 1 ? 1 : (kind == 2 || kind == 4) ? 2 : 3; }

// Dispatch a generic lambda on the operator functor of a view.
// The Kronecker-form operator of a view, with its translation-invariant
// y-factor rows (parameter-bank copies) when it has them.
template <class T, int R> inline OpK<T, R> kron_op(const OpView<T>& v, int nx, int ny) {
  OpK<T, R> o{v.gx, v.wx, v.hy, v.wy, v.dinv, nx, ny};
  o.ty0 = v.ty0;
  o.ty1 = v.ty1;
  for (int k = 0; k < 2 * R + 1; ++k) {
    o.hyc[k] = v.hyc[k];
    o.wyc[k] = v.wyc[k];
    if constexpr (sizeof(T) == 4) {
      o.pk.hyr[k] = make_float2(v.hyc[k].x, v.hyc[k].x);
      o.pk.hyi[k] = make_float2(v.hyc[k].y, v.hyc[k].y);
      o.pk.wyb[k] = make_float2(v.wyc[k], v.wyc[k]);
    }
  }
  return o;
}

template <class T, class F> inline void with_op(const OpView<T>& v, int nx, int ny, F&& f) {
  switch (v.kind) {
    case 1:   // the second-order absorbing rows are a separate instantiation
      if (v.c0.abc2) f(Op0<T, true>{v.c0, v.kf, nx, ny});
      else f(Op0<T>{v.c0, v.kf, nx, ny});
      break;
    case 2: f(OpS<T, 2>{v.st, v.dinv, v.plane, nx, ny}); break;
    case 3: f(OpS<T, 3>{v.st, v.dinv, v.plane, nx, ny}); break;
    case 4: f(kron_op<T, 2>(v, nx, ny)); break;
    default: f(kron_op<T, 3>(v, nx, ny)); break;
  }
}

// Node-parallel kernels (kernels_level.cu).  `active[b]` == 0 skips RHS b.
// B = number of right-hand sides.
template <class T> void launch_residual(const Grid& g, const OpView<T>& op, const cx<T>* x, const cx<T>* b,
                                        cx<T>* r, int B, const int* active, cudaStream_t s);
template <class T> void launch_apply(const Grid& g, const OpView<T>& op, const cx<T>* x, cx<T>* y, int B,
                                     const int* active, cudaStream_t s);
template <class T> void launch_jacobi(const Grid& g, const OpView<T>& op, const cx<T>* x, const cx<T>* b,
                                      cx<T>* xout, int B, const int* active, cudaStream_t s);
// Per-solve control block of the stopping test (device arrays, one entry per
// RHS unless noted).  tolp = {tol, divergence threshold}; partial/tickets are
// the scratch of the fused reductions (reduce_last).
struct Ctl {
  const double* bnorm;
  const double* tolp;
  int* active;
  int* state;
  int* cycles;
  double* relres;
  double* hist;
  int hist_len;
  int* n_active;        // one int
  double* partial;
  unsigned* tickets;
};
// Stopping test for one right-hand side, run by the last block of a norm
// reduction: relres = sqrt(sumsq) / ||b||; count != 0 means a cycle has just
// finished.  A RHS that meets tol (state 1) or diverges (state 2: not finite
// or above the threshold) is deactivated.
__device__ __forceinline__ void stop_update(const Ctl& c, int rhs, double sumsq, int count) {
  const double tol = c.tolp[0], diverge = c.tolp[1];
  const double rr = sqrt(sumsq) / c.bnorm[rhs];
  c.relres[rhs] = rr;
  if (count) {
    const int cy = ++c.cycles[rhs];
    if (cy <= c.hist_len) c.hist[(long long)rhs * c.hist_len + cy - 1] = rr;
  }
  int st = 0;
  if (!(rr == rr) || rr > diverge) st = 2;
  else if (rr <= tol) st = 1;
  if (st) {
    c.state[rhs] = st;
    c.active[rhs] = 0;
    atomicSub(c.n_active, 1);
  }
}

// ||b - A x|| per RHS with the stopping test fused (count != 0: a cycle just finished).
template <class T> void launch_resnorm_stop(const Grid& g, const OpView<T>& op, const cx<T>* x, const cx<T>* b,
                                            int B, const Ctl& c, int count, cudaStream_t s);
// Mixed path, FP64 outer loop: r = b - A x in FP64, written as float into r32
// (same Grid), stopping test fused; and x += e (FP64 += float), masked.
void launch_resid_cast_stop(const Grid& g, const OpView<double>& op, const double2* x, const double2* b,
                            float2* r32, int B, const Ctl& c, int count, cudaStream_t s);
void launch_update_mixed(const Grid& g, double2* x, const float2* e, int B, const int* active, cudaStream_t s);
// out[b] = ||v_b|| (one kernel).
template <class T> void launch_vecnorm_fin(const Grid& g, const cx<T>* v, int B, double* out, double* partial,
                                           unsigned* tickets, cudaStream_t s);
// Transfers (weights xw, Eq. (xex) or linear): r_c = R r_f and x_f += P e_c.
template <class T> void launch_restrict(const Grid& gf, const Grid& gc, const cx<T>* rf, cx<T>* rc, int B,
                                        const int* active, const Xfer& xw, cudaStream_t s);
template <class T> void launch_prolong_add(const Grid& gf, const Grid& gc, const cx<T>* ec, cx<T>* xf, int B,
                                           const int* active, const Xfer& xw, cudaStream_t s);
template <class T> void launch_copy_masked(const Grid& g, const cx<T>* src, cx<T>* dst, int B, const int* active,
                                           cudaStream_t s);
// Dense user array [B][ny+1][nx+1] complex128 <-> padded vector; conj != 0 conjugates.
template <class T> void launch_pack(const Grid& g, const double2* user, cx<T>* v, int B, int conj, cudaStream_t s);
template <class T> void launch_unpack(const Grid& g, const cx<T>* v, double2* user, int B, int conj, cudaStream_t s);
// Coarsest-grid solve with the stored FP64 inverse (setup.cu).
template <class T> void launch_coarse_solve(const Grid& g, const double2* inv, int N, const cx<T>* r, cx<T>* e,
                                            int B, const int* active, cudaStream_t s);

// Setup kernels (setup.cu).  All FP64.
void launch_op0consts(Op0Consts<double>* c64, Op0Consts<float>* c32, double h, double k, double omega,
                      double beta2, int abc, cudaStream_t s);
// Galerkin coarse stencil (radius rc) from the fine operator: fine kind 1 uses
// the matrix-free definition with the CSL shift beta2; kind 2/3 a stored stencil.
void launch_galerkin(const OpView<double>& fine, int fnx, int fny, double2* coarse_st, int cnx, int cny, int rc,
                     double beta2, const Xfer& xw, cudaStream_t s);
void launch_diaginv(const double2* st, int rc, long long plane, double omega, double2* dinv, cudaStream_t s);
void launch_to_float(const double2* src, float2* dst, long long n, cudaStream_t s);
void launch_to_float_real(const double* src, float* dst, long long n, cudaStream_t s);
// 1D factors of the constant-k fine operator (radius 1, rows [n+1][3]):
// g = L1/h^2 - (1 + i beta2) k^2 W1 - i (k/h) B1 (the x factor) when shifted,
// h = L1/h^2 - i (k/h) B1 (the y factor), w = W1.
void launch_factors0(int n, double h, double k, double beta2, double2* g, double2* hf, double2* w, cudaStream_t s);
// 1D Galerkin coarsening X_c = (P1^T / 2) X P1 of a banded [nf+1][2rf+1] row
// array into [nc+1][2rc+1] (nc = nf / 2).
void launch_galerkin_1d(const double2* X, int nf, int rf, double2* Xc, int rc, const Xfer& xw, cudaStream_t s);
// Real parts of a complex row array (the W factors are real).
void launch_real_part(const double2* a, double* b, long long n, cudaStream_t s);
// Per-node 1/(omega * diagonal) of a level operator (any kind).
void launch_diaginv_op(const OpView<double>& op, int nx, int ny, double omega, double2* dinv, cudaStream_t s);
// Dense matrix of a level operator (N = (nx+1)(ny+1) <= 4096) and its inverse.
void launch_dense(const OpView<double>& op, int nx, int ny, double2* M, cudaStream_t s);
void launch_gauss_jordan(double2* M, double2* inv, int N, int* status, cudaStream_t s);
// Per-node stencil export [ny+1][nx+1][2r+1][2r+1] complex128 of a level operator.
void launch_export_stencil(const OpView<double>& op, int nx, int ny, int r, double2* out, cudaStream_t s);

// GMRES(3) smoother (kernels_gmres.cu).  State layout per RHS in `gs`.
struct GmresBufs {
  void* u[3];          // Arnoldi vectors (unnormalised), precision T
  void* w;             // A v_j
  void* w2;            // second w of the fused Kronecker-level marches (null: unfused)
  double* partial;     // block partials of the fused reductions
  unsigned* tickets;   // one per RHS, 0 at rest
  double* st;          // per-RHS scalars, see kernels_gmres.cu
  cudaStream_t side;   // optional second stream (with the two events) on
  cudaEvent_t ev_fork; // which the fine level's boundary launches run beside
  cudaEvent_t ev_join; // the interior ones; null: one stream
  double2* outer;      // complex64 level 0 inside the FP64 refinement: the FP64
                       // iterate to which the last smoothing step's result is
                       // added by the fused update (null: none)
  int kron_ch;         // rows per chunk of the Kronecker-level column marches
                       // (0: chosen from the kernel's occupancy)
  int x_zero;          // x is zero on entry: the first step takes b itself as
                       // u0 = b - A x (no apply, no u0 write; b is read-only
                       // in every pass) and only sums |b|^2 for its norm
};
// The last GMRES(3) update of a complex64 level-0 smoothing fused with the
// FP64 refinement update x64 += x (kernels_gmres.cu).
void launch_gmres_update_outer(const Grid& g, const float2* x, const GmresBufs& gb, int B, const int* active,
                               cudaStream_t s);
template <class T> void gmres_smooth(const Grid& g, const OpView<T>& op, cx<T>* x, const cx<T>* b, int nu, int B,
                                     const int* active, const GmresBufs& gb, cudaStream_t s);

// The same smoother on the fine level (kind 1) in four row-marching passes
// plus the update (gmres_march.cu); the partial buffer must hold
// gmres_march_blocks() records per RHS.
long long gmres_march_blocks(const Grid& g, bool fp64, int B);
template <class T> void gmres_smooth_march(const Grid& g, const OpView<T>& op, cx<T>* x, const cx<T>* b, int nu,
                                           int B, const int* active, const GmresBufs& gb, cudaStream_t s);

// The same smoother on a Kronecker-form level (kinds 4, 5) with the kernels
// that apply A written as column marches (kron_march.cu); the partial buffer
// must hold kron_march_blocks() records per RHS.
long long kron_march_blocks(const Grid& g, int B);
template <class T> void gmres_smooth_kron(const Grid& g, const OpView<T>& op, cx<T>* x, const cx<T>* b, int nu, int B,
                                          const int* active, const GmresBufs& gb, cudaStream_t s);
// r = b - A x on a Kronecker-form level as a column march (the residual that
// the restriction then reads; kron_ch as in GmresBufs).
template <class T> void launch_kron_residual(const Grid& g, const OpView<T>& op, const cx<T>* x, const cx<T>* b,
                                             cx<T>* r, int B, const int* active, int kron_ch, cudaStream_t s);

// Single-CTA coarse-cycle interpreter (coarse.cu).  One CTA per RHS walks a
// host-recorded list of steps over the levels lc..L-1.
constexpr int CTA_THREADS = 512;
enum { C_JACOBI = 0, C_GMRES = 1, C_RESTRICT = 2, C_ZERO = 3, C_COARSE = 4, C_PROLONG = 5, C_COPY = 6 };
template <class T> struct CLevel {
  Grid g;
  Xfer xw;                  // transfers between this level and the next
  int kind;                 // as OpView::kind
  Op0Consts<T> c0;
  const T* kf;
  const cx<T>* st;
  const cx<T>* dinv;
  long long plane;
  const cx<T>* gx;
  const T* wx;
  const cx<T>* hy;
  const T* wy;
  cx<T>* b;                 // right-hand side of the level
  cx<T>* r;                 // residual scratch
  cx<T>* u[3];              // GMRES(3) basis (null without GMRES)
  cx<T>* w;
};
struct CStep {
  int op, level, arg, pad;  // arg: GMRES steps
  void* p0;                 // iterate of `level` (in place), or source
  void* p1;                 // destination (Jacobi, copy) or coarse correction (prolong)
};
template <class T> void launch_coarse_cycle(const CLevel<T>* levels, const CStep* steps, int nsteps,
                                            const double2* inv, int N, int B, const int* active, cudaStream_t s);

// Cooperative multi-CTA interpreter (coop.cu): the same steps, all blocks of
// the GPU, grid-wide barriers between phases.
constexpr int COOP_THREADS = 256;
constexpr int COOP_MAXLEV = 16;
struct CoopCtl {
  unsigned* bar;          // {arrival count, generation}, zero at rest
  int* err;               // set to 1 when a barrier wait gave up
  long long spin_limit;   // polls per barrier wait
  double* partial;        // [B * bpr][NVMAX] block sums
};
template <class T> int coop_max_blocks(int N);
template <class T> cudaError_t launch_cycle_coop(const CLevel<T>* levels, int nlev, const CStep* steps, int nsteps,
                                                 const double2* inv, int N, const int* active, int B, int grid,
                                                 const CoopCtl& c, cudaStream_t s);

// Fused halo-tile kernels (fused.cu): r_c = R (b - A x) in one pass (any
// level), and up to jacobi_fused_max_nu() fine-level Jacobi sweeps in one pass.
template <class T> void launch_resid_restrict(const Grid& gf, const Grid& gc, const OpView<T>& op, const cx<T>* x,
                                              const cx<T>* b, cx<T>* rc, int B, const int* active, const Xfer& xw,
                                              cudaStream_t s);
template <class T> void launch_jacobi_fused(const Grid& g, const OpView<T>& op, const cx<T>* x, const cx<T>* b,
                                            cx<T>* xo, int nu, int B, const int* active, cudaStream_t s);
int jacobi_fused_max_nu();
cudaError_t configure_fused_kernels();

// Outer iterate of the mixed path in float-float arithmetic (mixed_ff.cu):
// level-0 vectors hold each node as the float4 {re.hi, im.hi, re.lo, im.lo}
// in the space of a complex128 vector.
struct FF {
  float h, l;
};
struct FFConsts {
  FF d, ih2, sb;   // 4/h^2 - k^2, 1/h^2, k/h (constant k)
};
// Constants, and for variable k the per-node diagonal w (4/h^2 - k^2) into dP.
void launch_ff_setup(double h, double k, const double* kf, int nx, int ny, FFConsts* consts, float2* dP,
                     cudaStream_t s);
// r = b - A x in float-float, written as float into r32, stopping test fused.
void launch_ff_resid_cast_stop(const Grid& g, const FFConsts& K, const double* kf, double h, const float2* dP,
                               const void* x, const void* b, float2* r32, int B, const Ctl& c, int count,
                               cudaStream_t s);
// x += e (float-float += float), masked.
void launch_ff_update(const Grid& g, void* x, const float2* e, int B, const int* active, cudaStream_t s);
void launch_ff_pack(const Grid& g, const double2* user, void* v, int B, int conj, cudaStream_t s);
void launch_ff_unpack(const Grid& g, const void* v, double2* user, int B, int conj, cudaStream_t s);
void launch_ff_norm(const Grid& g, const void* v, int B, double* out, double* partial, unsigned* tickets,
                    cudaStream_t s);

// Flexible GMRES(m) outer loop with one cycle as the right preconditioner
// (fgmres.cu).  V: m+1 basis vectors and Z: m preconditioned vectors, both
// in the cycle's precision; vector q of RHS b at base + q * vlen + b * vstride.
constexpr int FG_MAXM = 32;
// Per-RHS FP64 scalars of the restart cycle: the rotated Hessenberg columns
// (column j, row i), the Gram matrix of V (row a, column b: <v_a, v_b>), the
// rotations (cs real, sn complex), g, y, beta and the scales s_j of the
// unnormalised basis (v_j = s_j u_j); complex values as (re, im).
struct FgLayout {
  int m;
  __host__ __device__ int h(int j, int i) const { return 2 * (j * (m + 1) + i); }
  __host__ __device__ int gram(int a, int b) const { return 2 * m * (m + 1) + 2 * (a * (m + 1) + b); }
  __host__ __device__ int cs(int i) const { return 2 * m * (m + 1) + 2 * (m + 1) * (m + 1) + i; }
  __host__ __device__ int sn(int i) const { return cs(m) + 2 * i; }
  __host__ __device__ int g(int i) const { return sn(m) + 2 * i; }
  __host__ __device__ int y(int i) const { return g(m + 1) + 2 * i; }
  __host__ __device__ int beta() const { return y(m); }
  __host__ __device__ int s(int j) const { return beta() + 1 + j; }
  __host__ __device__ int size() const { return s(m + 1); }
};
struct FgArgs {
  Grid g;                  // fine level
  Op0Consts<double> c0;    // fine operator (FP64: restart residual)
  const double* kf;
  Op0Consts<float> c0f;    // and in FP32 (Arnoldi passes of the mixed path)
  const float* kf32;
  int B, m;
  int nbr, ncx, ns, nvp;   // blocks per RHS, strip columns, strips, values per partial record
  long long vlen;          // g.vstride * B
  void* V;
  void* Z;
  double2* X;
  const double2* b;
  double* S;               // [B][sd] scalars (FgLayout)
  int sd;
  int* kst;                // [B][2]: steps of the current restart cycle, steps allowed in it
  int* active;             // 1 while the RHS is inside a restart cycle
  int* state;              // 0 running, 1 converged, 2 not finite
  int* cycles;             // preconditioner applications
  double* relres;          // true relative residual at the last restart
  double* hist;            // residual estimate after every application
  int hist_len;
  int* n_active;
  const double* bnorm;
  double tol;
  int max_cycles;
  double* partial;         // [B][nvp][nbr]
  unsigned* tickets;       // [B], 0 at rest
};
// Strip geometry and blocks per RHS (nbr, ncx, ns, nvp) for a fine grid.
void fg_geometry(const Grid& g, int B, bool fp64z, FgArgs& a);
// cb, cxv: the cycle's level-0 right-hand side and iterate (the restart and
// orth passes write the next basis vector into cb and zero cxv).
template <class T> void launch_fg_restart(const FgArgs& a, cx<T>* cb, cx<T>* cxv, cudaStream_t s);
template <class T> void launch_fg_dots(const FgArgs& a, int j, const cx<T>* z, cudaStream_t s);
template <class T> void launch_fg_orth(const FgArgs& a, int j, cx<T>* cb, cx<T>* cxv, cudaStream_t s);
template <class T> void launch_fg_update(const FgArgs& a, cudaStream_t s);

// Dense two-grid analysis of the two finest levels (analysis.cu).  out[0] =
// ||T0||_2, out[1] = 1 if Gamma~ is Hermitian positive definite, out[2] =
// ||Gamma~||_1 / kappa_1(Gamma~), out[3] = power iterations, out[4] = 1 if
// the power method met its stopping test, out[5] = 1 if A_1 was singular.
cudaError_t two_grid_analysis(const OpView<double>& fine, const OpView<double>& coarse, int fnx, int fny, int cnx,
                              int cny, double omega, const Xfer& xw, int nu, int max_iter, double* out,
                              cudaStream_t s);

// Gradient of the receiver misfit (kernels_level.cu).
void launch_gradient(int nx, int ny, double h, const double* m, double omega_f, const double2* u,
                     const double2* lam, int nsrc, double* g, cudaStream_t s);

inline int cdiv(long long a, long long b) { return (int)((a + b - 1) / b); }

// Sets the message mg_last_error() returns on this host thread (capi.cu).
void hmg_set_error(const char* msg);

}  // namespace hmg
