// Host-side declarations shared by the helmmg translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace hmg {

// Operator of one level in precision T, as handed to the launch wrappers.
// kind 1: matrix-free fine-level operator (c0, kf); kind 2 / 3: stored
// Galerkin stencil of that radius (st, dinv, plane).
template <class T> struct OpView {
  int kind;
  const Op0Consts<T>* c0;
  const T* kf;
  const cx<T>* st;
  const cx<T>* dinv;
  long long plane;
};

// Node-parallel kernels (kernels_level.cu).  `active[b]` == 0 skips RHS b.
// B = number of right-hand sides.
template <class T> void launch_residual(const Grid& g, const OpView<T>& op, const cx<T>* x, const cx<T>* b,
                                        cx<T>* r, int B, const int* active, cudaStream_t s);
template <class T> void launch_apply(const Grid& g, const OpView<T>& op, const cx<T>* x, cx<T>* y, int B,
                                     const int* active, cudaStream_t s);
template <class T> void launch_jacobi(const Grid& g, const OpView<T>& op, const cx<T>* x, const cx<T>* b,
                                      cx<T>* xout, int B, const int* active, cudaStream_t s);
// Per-block partial sums of |b - A x|^2 into partial[b * nblk + blk]; returns nblk.
template <class T> int launch_resnorm(const Grid& g, const OpView<T>& op, const cx<T>* x, const cx<T>* b,
                                      double* partial, int B, const int* active, cudaStream_t s);
// r = b - A x in FP64 with |r|^2 partials, r written in float (mixed path).
int launch_resid_cast_norm(const Grid& g, const OpView<double>& op, const double2* x, const double2* b,
                           float2* r32, double* partial, int B, const int* active, cudaStream_t s);
// x += e (FP64 += float), masked.
void launch_update_mixed(const Grid& g, double2* x, const float2* e, int B, const int* active, cudaStream_t s);
template <class T> void launch_restrict(const Grid& gf, const Grid& gc, const cx<T>* rf, cx<T>* rc, int B,
                                        const int* active, cudaStream_t s);
template <class T> void launch_prolong_add(const Grid& gf, const Grid& gc, const cx<T>* ec, cx<T>* xf, int B,
                                           const int* active, cudaStream_t s);
template <class T> void launch_copy_masked(const Grid& g, const cx<T>* src, cx<T>* dst, int B, const int* active,
                                           cudaStream_t s);
// Dense user array [B][ny+1][nx+1] complex128 <-> padded vector; conj != 0 conjugates.
template <class T> void launch_pack(const Grid& g, const double2* user, cx<T>* v, int B, int conj, cudaStream_t s);
template <class T> void launch_unpack(const Grid& g, const cx<T>* v, double2* user, int B, int conj, cudaStream_t s);
// Stopping test for every active RHS b: relres[b] = sqrt(sum partial) / bnorm[b];
// tolp = {tol, divergence threshold} in device memory.  count != 0: a cycle
// has just finished (cycles[b] += 1, history entry written).  A RHS that meets
// tol (state 1) or diverges (state 2) is deactivated and n_active decremented.
void launch_stop(const double* partial, int nblk, int B, const double* bnorm, const double* tolp,
                 int* active, int* state, int* cycles, double* relres, double* hist, int hist_len,
                 int* n_active, int count, cudaStream_t s);
// ||b||: sum partials into bnorm (sqrt), one block per RHS.
void launch_norm_finish(const double* partial, int nblk, int B, double* out, cudaStream_t s);
template <class T> int launch_vecnorm(const Grid& g, const cx<T>* v, double* partial, int B, cudaStream_t s);

// Coarsest-grid solve with the stored FP64 inverse (setup.cu).
template <class T> void launch_coarse_solve(const Grid& g, const double2* inv, int N, const cx<T>* r, cx<T>* e,
                                            int B, const int* active, cudaStream_t s);

// Setup kernels (setup.cu).  All FP64.
void launch_op0consts(Op0Consts<double>* c64, Op0Consts<float>* c32, double h, double k, double omega,
                      double beta2, cudaStream_t s);
// Galerkin coarse stencil (radius rc) from the fine operator: fine kind 1 uses
// the matrix-free definition with the CSL shift beta2; kind 2/3 a stored stencil.
void launch_galerkin(const OpView<double>& fine, int fnx, int fny, double2* coarse_st, int cnx, int cny, int rc,
                     double beta2, cudaStream_t s);
void launch_diaginv(const double2* st, int rc, long long plane, double omega, double2* dinv, cudaStream_t s);
void launch_to_float(const double2* src, float2* dst, long long n, cudaStream_t s);
void launch_to_float_real(const double* src, float* dst, long long n, cudaStream_t s);
// Dense matrix of a level operator (N = (nx+1)(ny+1) <= 4096) and its inverse.
void launch_dense(const OpView<double>& op, int nx, int ny, double2* M, cudaStream_t s);
void launch_gauss_jordan(double2* M, double2* inv, int N, int* status, cudaStream_t s);
// Per-node stencil export [ny+1][nx+1][2r+1][2r+1] complex128 of a level operator.
void launch_export_stencil(const OpView<double>& op, int nx, int ny, int r, double2* out, cudaStream_t s);

// GMRES(3) smoother (kernels_gmres.cu).  State layout per RHS in `gs`.
struct GmresBufs {
  void* u[4];       // Arnoldi vectors (unnormalised), precision T
  void* w;          // A v_j
  double* partial;  // block partials
  double* st;       // per-RHS scalars, see kernels_gmres.cu
  int nblk_cap;
};
template <class T> void gmres_smooth(const Grid& g, const OpView<T>& op, cx<T>* x, const cx<T>* b, int nu, int B,
                                     const int* active, const GmresBufs& gb, cudaStream_t s);

// Gradient of the receiver misfit (kernels_level.cu).
void launch_gradient(int nx, int ny, double h, const double* m, double omega_f, const double2* u,
                     const double2* lam, int nsrc, double* g, cudaStream_t s);

inline int cdiv(long long a, long long b) { return (int)((a + b - 1) / b); }

}  // namespace hmg
