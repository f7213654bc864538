// Node-parallel kernels of one multigrid level: operator apply, residual,
// weighted-Jacobi sweep, residual norms, Bezier restriction / prolongation,
// layout conversion and the stopping test.
//
// Paper references: the operator is the 5-point discretisation of Sec. 2
// (matrix-free on the fine level, Galerkin stencils below, Sec. 3); the
// Jacobi sweep is S = I - X^{-1} A with X = omega * diag(A) (Sec. 3); the
// transfers are Eq. (xex) and its transpose; the stopping test is the
// relative residual of Sec. 5.
#include <math.h>

#include <algorithm>

#include "internal.h"
#include "ragged.cuh"
#include "ragged_api.h"
#include "pack.cuh"

namespace hmg {

// ------------------------------------------------------------------ helpers

static inline dim3 node_grid(const Grid& g, int B) {
  return dim3(cdiv(g.nx + 1, BX), cdiv(g.ny + 1, BY * g.ry), B);
}
static inline dim3 pack_grid(const Grid& g, int B, int np) {
  return dim3(cdiv(g.nx + 1, BX * np), cdiv(g.ny + 1, BY * g.ry), B);
}

// Thread (tx, ty) of block (bx, by, rhs) handles node column i and the g.ry
// rows j = by*BY*ry + r*BY + ty, r = 0..ry-1 (warps stay on one row).
// Arguments of the flattened launches over a ragged batch (one per problem).
template <class T, class Op>
struct RsA {
  Grid g;
  Op op;
  const cx<T>* x;
  const cx<T>* b;
  Ctl c;
  int count;
};


struct RcA {
  Grid g;
  Op0<double> op;
  const double2* x;
  const double2* b;
  float2* r32;
  Ctl c;
  int count;
};


struct UmA {
  Grid g;
  double2* x;
  const float2* e;
  const int* active;
};

template <class T>
struct PaA {
  Grid g;
  Grid gc;
  const cx<T>* ec;
  cx<T>* xf;
  const int* active;
  Xfer xw;
};

#define NODE_INDEX                                       \
  const int rhs = blockIdx.z;                            \
  const int i = blockIdx.x * BX + threadIdx.x;           \
  const long long off = (long long)rhs * g.vstride;
#define FOR_ROWS for (int r_ = 0, j = blockIdx.y * BY * g.ry + threadIdx.y; r_ < g.ry; ++r_, j += BY)
// Pack kernels: the thread's pack starts at column i0 and holds nv nodes
// inside the grid.
#define PACK_INDEX(T)                                          \
  constexpr int NP = PK<T>::NP;                                \
  const int rhs = blockIdx.z;                                  \
  const int i0 = (blockIdx.x * BX + threadIdx.x) * NP;         \
  const int nv = min(NP, g.nx + 1 - i0);                       \
  const long long off = (long long)rhs * g.vstride;

// ------------------------------------------------------------------ operator kernels

template <class T, class Op>
__global__ void __launch_bounds__(BX * BY) k_residual(Grid g, Op op, const cx<T>* __restrict__ x,
                                                      const cx<T>* __restrict__ b, cx<T>* __restrict__ r,
                                                      const int* __restrict__ active) {
  PACK_INDEX(T)
  if (active && !active[rhs]) return;
  if (nv <= 0) return;
  FOR_ROWS {
    if (j > g.ny) break;
    const int p = g.at(i0, j);
    const Pack<T> ax = apply_pack<T>(op, x + off, p, g.pitch, i0, j);
    Pack<T> bb = load_pack(b + off, p);
#pragma unroll
    for (int n = 0; n < NP; ++n) bb.v[n] = sub<T>(bb.v[n], ax.v[n]);
    store_pack(r + off, p, bb, nv);
  }
}

template <class T, class Op>
__global__ void __launch_bounds__(BX * BY) k_apply(Grid g, Op op, const cx<T>* __restrict__ x,
                                                   cx<T>* __restrict__ y, const int* __restrict__ active) {
  PACK_INDEX(T)
  if (active && !active[rhs]) return;
  if (nv <= 0) return;
  FOR_ROWS {
    if (j > g.ny) break;
    const int p = g.at(i0, j);
    store_pack(y + off, p, apply_pack<T>(op, x + off, p, g.pitch, i0, j), nv);
  }
}

// x_out = x + (omega diag A)^{-1} (b - A x)   (one weighted-Jacobi sweep)
template <class T, class Op>
__global__ void __launch_bounds__(BX * BY) k_jacobi(Grid g, Op op, const cx<T>* __restrict__ x,
                                                    const cx<T>* __restrict__ b, cx<T>* __restrict__ xo,
                                                    const int* __restrict__ active) {
  PACK_INDEX(T)
  if (active && !active[rhs]) return;
  if (nv <= 0) return;
  FOR_ROWS {
    if (j > g.ny) break;
    const int p = g.at(i0, j);
    const Pack<T> ax = apply_pack<T>(op, x + off, p, g.pitch, i0, j);
    const Pack<T> bb = load_pack(b + off, p);
    Pack<T> xv = load_pack(x + off, p);
#pragma unroll
    for (int n = 0; n < NP; ++n)
      xv.v[n] = fma_c<T>(op.diag_inv(min(i0 + n, g.nx), j), sub<T>(bb.v[n], ax.v[n]), xv.v[n]);
    store_pack(xo + off, p, xv, nv);
  }
}


template <class T, class Op>
__device__ __forceinline__ void k_resnorm_stop_body(uint3 vblk, dim3 vgrid, Grid g, Op op, const cx<T>* __restrict__ x, const cx<T>* __restrict__ b, Ctl c, int count) {
  const uint3 blockIdx = vblk;   // the block and grid inside this problem's launch
  const dim3 gridDim = vgrid;
  (void)blockIdx;
  (void)gridDim;
  __shared__ double sh[32];
  PACK_INDEX(T)
  if (!c.active[rhs]) return;   // block-uniform
  T a0[1] = {T(0)};   // per-thread sum in the working precision
  if (nv > 0) {
    FOR_ROWS {
      if (j > g.ny) break;
      const int p = g.at(i0, j);
      const Pack<T> ax = apply_pack<T>(op, x + off, p, g.pitch, i0, j);
      const Pack<T> bb = load_pack(b + off, p);
#pragma unroll
      for (int n = 0; n < NP; ++n)
        if (n < nv) a0[0] += abs2<T>(sub<T>(bb.v[n], ax.v[n]));
    }
  }
  double v[1];
  if (reduce_last<1, T>(a0, v, sh, c.partial, c.tickets, rhs, gridDim.x * gridDim.y, blockIdx.y * gridDim.x + blockIdx.x) &&
      threadIdx.x == 0 && threadIdx.y == 0)
    stop_update(c, rhs, v[0], count);
}

template <class T, class Op>
__global__ void __launch_bounds__(BX * BY) k_resnorm_stop(Grid g, Op op, const cx<T>* __restrict__ x, const cx<T>* __restrict__ b, Ctl c, int count) {
  k_resnorm_stop_body<T, Op>(blockIdx, gridDim, g, op, x, b, c, count);
}

template <class T, class Op>
__global__ void __launch_bounds__(BX * BY) k_resnorm_stop_rag(const __grid_constant__ RagLaunch<RsA<T, Op>> L) {
  uint3 vb;
  dim3 vg;
  const RsA<T, Op>& a = L.a[rag_problem(L, blockIdx.x, vb, vg)];
  k_resnorm_stop_body<T, Op>(vb, vg, a.g, a.op, a.x, a.b, a.c, a.count);
}

// FP64 residual of the refinement loop, written in float for the next
// complex64 correction cycle, with the stopping test fused.  This pass runs
// at the FP64 rate, so its FP64 work is kept small: on interior nodes
// b - A x is two FMAs per component after the neighbour sum,
// b - d x_P + (1/h^2)(x_E + x_W + x_N + x_S), d = 4/h^2 - k^2 (boundary nodes
// take Op0::apply5); and the norm is summed from the float residual the
// pass writes anyway (FP32 within a thread and a warp, FP64 across warps and
// blocks), which resolves the stopping test's relative residual to about
// 1e-7 of itself.  The conversions to float take the integer pipe
// (f32_from_f64_rn, the same rounding as the hardware's).
template <bool A2>
__device__ __forceinline__ void k_resid_cast_stop_body(uint3 vblk, dim3 vgrid, Grid g, Op0<double, A2> op, const double2* __restrict__ x, const double2* __restrict__ b, float2* __restrict__ r32, Ctl c, int count) {
  const uint3 blockIdx = vblk;   // the block and grid inside this problem's launch
  const dim3 gridDim = vgrid;
  (void)blockIdx;
  (void)gridDim;
  __shared__ double sh[32];
  NODE_INDEX
  if (!c.active[rhs]) return;
  float af = 0.f;
  const double ih2 = op.c.inv_h2;
  const double dconst = fma(-op.c.k, op.c.k, 4.0 * ih2);
  if (i <= g.nx) {
    const double2* xs = x + off;
    FOR_ROWS {
      if (j > g.ny) break;
      const int p = g.at(i, j);
      const double2 bb = b[off + p];
      double2 r;
      if (i > 0 && i < g.nx && j > 0 && j < g.ny) {
        const double2 xp = xs[p], xe = xs[p + 1], xw = xs[p - 1], xn = xs[p + g.pitch], xd = xs[p - g.pitch];
        double d = dconst;
        if (op.kf) {
          const double k = op.kf[j * (g.nx + 1) + i];
          d = fma(-k, k, 4.0 * ih2);
        }
        const double sr = (xe.x + xw.x) + (xn.x + xd.x), si = (xe.y + xw.y) + (xn.y + xd.y);
        r = make_double2(fma(ih2, sr, fma(-d, xp.x, bb.x)), fma(ih2, si, fma(-d, xp.y, bb.y)));
      } else {
        r = sub<double>(bb, op.apply(xs, p, g.pitch, i, j));
      }
      const float2 rf = make_float2(f32_from_f64_rn(r.x), f32_from_f64_rn(r.y));
      r32[off + p] = rf;
      af = fmaf(rf.x, rf.x, fmaf(rf.y, rf.y, af));
    }
  }
  const float a0[1] = {af};
  double v[1];
  if (reduce_last<1, float>(a0, v, sh, c.partial, c.tickets, rhs, gridDim.x * gridDim.y, blockIdx.y * gridDim.x + blockIdx.x) &&
      threadIdx.x == 0 && threadIdx.y == 0)
    stop_update(c, rhs, v[0], count);
}

template <bool A2>
__global__ void __launch_bounds__(BX * BY) k_resid_cast_stop(Grid g, Op0<double, A2> op, const double2* __restrict__ x, const double2* __restrict__ b, float2* __restrict__ r32, Ctl c, int count) {
  k_resid_cast_stop_body<A2>(blockIdx, gridDim, g, op, x, b, r32, c, count);
}

__global__ void __launch_bounds__(BX * BY) k_resid_cast_stop_rag(const __grid_constant__ RagLaunch<RcA> L) {
  uint3 vb;
  dim3 vg;
  const RcA& a = L.a[rag_problem(L, blockIdx.x, vb, vg)];
  k_resid_cast_stop_body(vb, vg, a.g, a.op, a.x, a.b, a.r32, a.c, a.count);
}

__device__ __forceinline__ void k_update_mixed_body(uint3 vblk, dim3 vgrid, Grid g, double2* __restrict__ x, const float2* __restrict__ e, const int* __restrict__ active) {
  const uint3 blockIdx = vblk;   // the block and grid inside this problem's launch
  const dim3 gridDim = vgrid;
  (void)blockIdx;
  (void)gridDim;
  NODE_INDEX
  if (active && !active[rhs]) return;
  if (i > g.nx) return;
  FOR_ROWS {
    if (j > g.ny) break;
    const long long p = off + g.at(i, j);
    const float2 d = e[p];
    double2 xv = x[p];
    xv.x += f64_from_f32(d.x);
    xv.y += f64_from_f32(d.y);
    x[p] = xv;
  }
}

__global__ void __launch_bounds__(BX * BY) k_update_mixed(Grid g, double2* __restrict__ x, const float2* __restrict__ e, const int* __restrict__ active) {
  k_update_mixed_body(blockIdx, gridDim, g, x, e, active);
}

__global__ void __launch_bounds__(BX * BY) k_update_mixed_rag(const __grid_constant__ RagLaunch<UmA> L) {
  uint3 vb;
  dim3 vg;
  const UmA& a = L.a[rag_problem(L, blockIdx.x, vb, vg)];
  k_update_mixed_body(vb, vg, a.g, a.x, a.e, a.active);
}

// ||v|| per RHS into out[rhs] (one kernel, last-block finish).
template <class T>
__global__ void __launch_bounds__(BX * BY) k_vecnorm_fin(Grid g, const cx<T>* __restrict__ v_, double* __restrict__ out,
                                                         double* partial, unsigned* tickets) {
  __shared__ double sh[32];
  NODE_INDEX
  T a0[1] = {T(0)};
  if (i <= g.nx) {
    FOR_ROWS {
      if (j > g.ny) break;
      a0[0] += abs2<T>(v_[off + g.at(i, j)]);
    }
  }
  double v[1];
  if (reduce_last<1, T>(a0, v, sh, partial, tickets, rhs, gridDim.x * gridDim.y, blockIdx.y * gridDim.x + blockIdx.x) &&
      threadIdx.x == 0 && threadIdx.y == 0)
    out[rhs] = sqrt(v[0]);
}

// ------------------------------------------------------------------ transfers

// r_c(I,J) = 1/4 sum_{a,b=-2..2} w(a) w(b) r_f(2I+a, 2J+b)   (R = P^T / 4)
template <class T>
__global__ void __launch_bounds__(BX * BY) k_restrict(Grid gf, Grid g, const cx<T>* __restrict__ rf,
                                                      cx<T>* __restrict__ rc, const int* __restrict__ active,
                                                      Xfer xw) {
  NODE_INDEX
  const T c0 = T(xw.w0), c1 = T(xw.w1), c2 = T(xw.w2);
  if (active && !active[rhs]) return;
  if (i > g.nx) return;
  const cx<T>* f = rf + (long long)rhs * gf.vstride;
  FOR_ROWS {
    if (j > g.ny) break;
    const int pc = gf.at(2 * i, 2 * j);
    cx<T> acc = mk<T>(0, 0);
#pragma unroll
    for (int b = -2; b <= 2; ++b) {
      const cx<T>* row = f + pc + b * gf.pitch;
      cx<T> t = scl<T>(c2, add<T>(row[-2], row[2]));
      t = add<T>(t, scl<T>(c1, add<T>(row[-1], row[1])));
      t = add<T>(t, scl<T>(c0, row[0]));
      acc = add<T>(acc, scl<T>(xw.w<T>(b), t));
    }
    rc[off + g.at(i, j)] = scl<T>(T(0.25), acc);
  }
}

// x_f(i,j) += sum_{I,J} P(i,I) P(j,J) e_c(I,J)   (Eq. (xex) in each direction)
template <class T>
__device__ __forceinline__ void k_prolong_add_body(uint3 vblk, dim3 vgrid, Grid g, Grid gc, const cx<T>* __restrict__ ec, cx<T>* __restrict__ xf, const int* __restrict__ active, Xfer xw) {
  const uint3 blockIdx = vblk;   // the block and grid inside this problem's launch
  const dim3 gridDim = vgrid;
  (void)blockIdx;
  (void)gridDim;
  PACK_INDEX(T)
  const T c0 = T(xw.w0), c1 = T(xw.w1), c2 = T(xw.w2);
  if (active && !active[rhs]) return;
  if (nv <= 0) return;
  const cx<T>* c = ec + (long long)rhs * gc.vstride;
  FOR_ROWS {
    if (j > g.ny) break;
    const int J = j >> 1;
    const int p = g.at(i0, j);
    Pack<T> xv = load_pack(xf + off, p);
#pragma unroll
    for (int n = 0; n < NP; ++n) {
      const int i = i0 + n, I = i >> 1;
      auto rowval = [&](int JJ) -> cx<T> {
        const cx<T>* row = c + gc.at(I, JJ);
        if (i & 1) return scl<T>(c1, add<T>(row[0], row[1]));
        return add<T>(scl<T>(c2, add<T>(row[-1], row[1])), scl<T>(c0, row[0]));
      };
      cx<T> v;
      if (j & 1) {
        v = scl<T>(c1, add<T>(rowval(J), rowval(J + 1)));
      } else {
        v = add<T>(scl<T>(c2, add<T>(rowval(J - 1), rowval(J + 1))), scl<T>(c0, rowval(J)));
      }
      xv.v[n] = add<T>(xv.v[n], v);
    }
    store_pack(xf + off, p, xv, nv);
  }
}

template <class T>
__global__ void __launch_bounds__(BX * BY) k_prolong_add(Grid g, Grid gc, const cx<T>* __restrict__ ec, cx<T>* __restrict__ xf, const int* __restrict__ active, Xfer xw) {
  k_prolong_add_body<T>(blockIdx, gridDim, g, gc, ec, xf, active, xw);
}

template <class T>
__global__ void __launch_bounds__(BX * BY) k_prolong_add_rag(const __grid_constant__ RagLaunch<PaA<T>> L) {
  uint3 vb;
  dim3 vg;
  const PaA<T>& a = L.a[rag_problem(L, blockIdx.x, vb, vg)];
  k_prolong_add_body<T>(vb, vg, a.g, a.gc, a.ec, a.xf, a.active, a.xw);
}

template <class T>
__global__ void __launch_bounds__(BX * BY) k_copy_masked(Grid g, const cx<T>* __restrict__ src, cx<T>* __restrict__ dst,
                                                         const int* __restrict__ active) {
  PACK_INDEX(T)
  if (active && !active[rhs]) return;
  if (nv <= 0) return;
  FOR_ROWS {
    if (j > g.ny) break;
    const int p = g.at(i0, j);
    store_pack(dst + off, p, load_pack(src + off, p), nv);
  }
}

template <class T>
__global__ void __launch_bounds__(BX * BY) k_pack(Grid g, const double2* __restrict__ user, cx<T>* __restrict__ v, int conj) {
  NODE_INDEX
  if (i > g.nx) return;
  FOR_ROWS {
    if (j > g.ny) break;
    double2 u = user[((long long)rhs * (g.ny + 1) + j) * (g.nx + 1) + i];
    if (conj) u.y = -u.y;
    v[off + g.at(i, j)] = mk<T>((T)u.x, (T)u.y);
  }
}

template <class T>
__global__ void __launch_bounds__(BX * BY) k_unpack(Grid g, const cx<T>* __restrict__ v, double2* __restrict__ user, int conj) {
  NODE_INDEX
  if (i > g.nx) return;
  FOR_ROWS {
    if (j > g.ny) break;
    const cx<T> a = v[off + g.at(i, j)];
    user[((long long)rhs * (g.ny + 1) + j) * (g.nx + 1) + i] =
        make_double2((double)a.x, conj ? -(double)a.y : (double)a.y);
  }
}

// ------------------------------------------------------------------ gradient

// g = -Re sum_s conj(lam_s) (dA_pp/dm_p) u_s with
// dA_pp/dm_p = -w_p omega_f^2 - i b_p omega_f / (2 h sqrt(m_p)).
__global__ void k_gradient(int nx, int ny, double h, const double* __restrict__ m, double omega_f,
                           const double2* __restrict__ u, const double2* __restrict__ lam, int nsrc,
                           double* __restrict__ g) {
  const int i = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y * BY + threadIdx.y;
  if (i > nx || j > ny) return;
  const long long q = (long long)j * (nx + 1) + i;
  const long long N = (long long)(nx + 1) * (ny + 1);
  const int bx = (i == 0 || i == nx), by = (j == 0 || j == ny);
  const double wx = bx ? 0.5 : 1.0, wy = by ? 0.5 : 1.0;
  const double bnd = bx * wy + wx * by;
  const double2 da = make_double2(-wx * wy * omega_f * omega_f, -bnd * omega_f / (2.0 * h * sqrt(m[q])));
  double acc = 0.0;
  for (int s = 0; s < nsrc; ++s) {
    const double2 t = cmul<double>(lam[s * N + q], mul<double>(da, u[s * N + q]));
    acc += t.x;
  }
  g[q] = -acc;
}

// ------------------------------------------------------------------ launch wrappers

template <class T>
void launch_residual(const Grid& g, const OpView<T>& v, const cx<T>* x, const cx<T>* b, cx<T>* r, int B,
                     const int* active, cudaStream_t s) {
  with_op<T>(v, g.nx, g.ny, [&](auto op) {
    k_residual<T, decltype(op)><<<pack_grid(g, B, PK<T>::NP), dim3(BX, BY), 0, s>>>(g, op, x, b, r, active);
  });
}
template <class T>
void launch_apply(const Grid& g, const OpView<T>& v, const cx<T>* x, cx<T>* y, int B, const int* active,
                  cudaStream_t s) {
  with_op<T>(v, g.nx, g.ny, [&](auto op) {
    k_apply<T, decltype(op)><<<pack_grid(g, B, PK<T>::NP), dim3(BX, BY), 0, s>>>(g, op, x, y, active);
  });
}
template <class T>
void launch_jacobi(const Grid& g, const OpView<T>& v, const cx<T>* x, const cx<T>* b, cx<T>* xo, int B,
                   const int* active, cudaStream_t s) {
  with_op<T>(v, g.nx, g.ny, [&](auto op) {
    k_jacobi<T, decltype(op)><<<pack_grid(g, B, PK<T>::NP), dim3(BX, BY), 0, s>>>(g, op, x, b, xo, active);
  });
}
template <class T>
void launch_resnorm_stop(const Grid& g, const OpView<T>& v, const cx<T>* x, const cx<T>* b, int B, const Ctl& c,
                         int count, cudaStream_t s) {
  with_op<T>(v, g.nx, g.ny, [&](auto op) {
    k_resnorm_stop<T, decltype(op)><<<pack_grid(g, B, PK<T>::NP), dim3(BX, BY), 0, s>>>(g, op, x, b, c, count);
  });
}
void launch_resid_cast_stop(const Grid& g, const OpView<double>& v, const double2* x, const double2* b, float2* r32,
                            int B, const Ctl& c, int count, cudaStream_t s) {
  if (v.c0.abc2)   // constants by value
    k_resid_cast_stop<true><<<node_grid(g, B), dim3(BX, BY), 0, s>>>(g, Op0<double, true>{v.c0, v.kf, g.nx, g.ny}, x, b,
                                                                     r32, c, count);
  else
    k_resid_cast_stop<false><<<node_grid(g, B), dim3(BX, BY), 0, s>>>(g, Op0<double>{v.c0, v.kf, g.nx, g.ny}, x, b, r32,
                                                                      c, count);
}
void launch_update_mixed(const Grid& g, double2* x, const float2* e, int B, const int* active, cudaStream_t s) {
  k_update_mixed<<<node_grid(g, B), dim3(BX, BY), 0, s>>>(g, x, e, active);
}
template <class T>
void launch_vecnorm_fin(const Grid& g, const cx<T>* v, int B, double* out, double* partial, unsigned* tickets,
                        cudaStream_t s) {
  k_vecnorm_fin<T><<<node_grid(g, B), dim3(BX, BY), 0, s>>>(g, v, out, partial, tickets);
}
template <class T>
void launch_restrict(const Grid& gf, const Grid& gc, const cx<T>* rf, cx<T>* rc, int B, const int* active,
                     const Xfer& xw, cudaStream_t s) {
  k_restrict<T><<<node_grid(gc, B), dim3(BX, BY), 0, s>>>(gf, gc, rf, rc, active, xw);
}
template <class T>
void launch_prolong_add(const Grid& gf, const Grid& gc, const cx<T>* ec, cx<T>* xf, int B, const int* active,
                        const Xfer& xw, cudaStream_t s) {
  k_prolong_add<T><<<pack_grid(gf, B, PK<T>::NP), dim3(BX, BY), 0, s>>>(gf, gc, ec, xf, active, xw);
}
template <class T>
void launch_copy_masked(const Grid& g, const cx<T>* src, cx<T>* dst, int B, const int* active, cudaStream_t s) {
  k_copy_masked<T><<<pack_grid(g, B, PK<T>::NP), dim3(BX, BY), 0, s>>>(g, src, dst, active);
}
template <class T> void launch_pack(const Grid& g, const double2* user, cx<T>* v, int B, int conj, cudaStream_t s) {
  k_pack<T><<<node_grid(g, B), dim3(BX, BY), 0, s>>>(g, user, v, conj);
}
template <class T> void launch_unpack(const Grid& g, const cx<T>* v, double2* user, int B, int conj, cudaStream_t s) {
  k_unpack<T><<<node_grid(g, B), dim3(BX, BY), 0, s>>>(g, v, user, conj);
}
// ---- flattened launches over the problems of a ragged batch (ragged.cuh) ----

template <class T>
__global__ void __launch_bounds__(256) k_zero_rag(const __grid_constant__ RagLaunch<RagVec> L) {
  uint3 vb;
  dim3 vg;
  const RagVec& a = L.a[rag_problem(L, blockIdx.x, vb, vg)];
  if (a.active && !a.active[0]) return;
  cx<T>* v = (cx<T>*)a.v;
  const long long i0 = (long long)vb.x * 1024 + threadIdx.x;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const long long i = i0 + 256 * k;
    if (i < a.g.vstride) v[i] = mk<T>(T(0), T(0));
  }
}

template <class T> void launch_zero_rag(const std::vector<RagVec>& v, cudaStream_t s) {
  rag_launch<RagVec>((int)v.size(), k_zero_rag<T>, dim3(256), 0, s, [&](int q, RagVec& a, int& gx, int&) {
    a = v[q];
    gx = (int)cdiv(v[q].g.vstride, (long long)1024);
    return true;
  });
}
template void launch_zero_rag<double>(const std::vector<RagVec>&, cudaStream_t);
template void launch_zero_rag<float>(const std::vector<RagVec>&, cudaStream_t);

template <class T> void launch_prolong_add_rag(const std::vector<RagXfer<T>>& v, const Xfer& xw, cudaStream_t s) {
  rag_launch<PaA<T>>((int)v.size(), k_prolong_add_rag<T>, dim3(BX, BY), 0, s, [&](int q, PaA<T>& a, int& gx, int& gy) {
    const RagXfer<T>& X = v[q];
    a = PaA<T>{X.gf, X.gc, X.rc, X.xf, X.active, xw};
    const dim3 d = pack_grid(X.gf, 1, PK<T>::NP);
    gx = (int)d.x;
    gy = (int)d.y;
    return true;
  });
}
template void launch_prolong_add_rag<double>(const std::vector<RagXfer<double>>&, const Xfer&, cudaStream_t);
template void launch_prolong_add_rag<float>(const std::vector<RagXfer<float>>&, const Xfer&, cudaStream_t);

void launch_update_mixed_rag(const std::vector<RagOuter>& v, cudaStream_t s) {
  rag_launch<UmA>((int)v.size(), k_update_mixed_rag, dim3(BX, BY), 0, s, [&](int q, UmA& a, int& gx, int& gy) {
    const RagOuter& O = v[q];
    a = UmA{O.g, O.x, O.e, O.c.active};
    const dim3 d = node_grid(O.g, 1);
    gx = (int)d.x;
    gy = (int)d.y;
    return true;
  });
}

void launch_resid_cast_stop_rag(const std::vector<RagOuter>& v, int count, cudaStream_t s) {
  rag_launch<RcA>((int)v.size(), k_resid_cast_stop_rag, dim3(BX, BY), 0, s, [&](int q, RcA& a, int& gx, int& gy) {
    const RagOuter& O = v[q];
    a = RcA{O.g, O.op, O.x, O.b, O.r32, O.c, count};
    const dim3 d = node_grid(O.g, 1);
    gx = (int)d.x;
    gy = (int)d.y;
    return true;
  });
}

void launch_resnorm_stop_rag(const std::vector<RagOuter>& v, int count, cudaStream_t s) {
  using A = RsA<double, Op0<double>>;
  rag_launch<A>((int)v.size(), k_resnorm_stop_rag<double, Op0<double>>, dim3(BX, BY), 0, s,
                [&](int q, A& a, int& gx, int& gy) {
                  const RagOuter& O = v[q];
                  a = A{O.g, O.op, O.x, O.b, O.c, count};
                  const dim3 d = pack_grid(O.g, 1, PK<double>::NP);
                  gx = (int)d.x;
                  gy = (int)d.y;
                  return true;
                });
}

struct GatherArgs {
  int np;
  const int* counts[RMAXP];
};
__global__ void k_gather_counts(const __grid_constant__ GatherArgs a, int* __restrict__ out, int stride) {
  const int p = threadIdx.x;
  if (p < a.np) {
    out[p] = a.counts[p][0];
    out[stride + p] = a.counts[p][1];
  }
}
void launch_gather_counts(const std::vector<const int*>& counts, int* out, cudaStream_t s) {
  const int n = (int)counts.size();
  for (int q0 = 0; q0 < n; q0 += RMAXP) {
    GatherArgs a{};
    a.np = std::min(RMAXP, n - q0);
    for (int q = 0; q < a.np; ++q) a.counts[q] = counts[q0 + q];
    k_gather_counts<<<1, RMAXP, 0, s>>>(a, out + q0, n);
  }
}

void launch_gradient(int nx, int ny, double h, const double* m, double omega_f, const double2* u, const double2* lam,
                     int nsrc, double* g, cudaStream_t s) {
  k_gradient<<<dim3(cdiv(nx + 1, BX), cdiv(ny + 1, BY)), dim3(BX, BY), 0, s>>>(nx, ny, h, m, omega_f, u, lam, nsrc, g);
}

#define INST(T)                                                                                                   \
  template void launch_residual<T>(const Grid&, const OpView<T>&, const cx<T>*, const cx<T>*, cx<T>*, int,         \
                                   const int*, cudaStream_t);                                                      \
  template void launch_apply<T>(const Grid&, const OpView<T>&, const cx<T>*, cx<T>*, int, const int*, cudaStream_t); \
  template void launch_jacobi<T>(const Grid&, const OpView<T>&, const cx<T>*, const cx<T>*, cx<T>*, int,           \
                                 const int*, cudaStream_t);                                                        \
  template void launch_resnorm_stop<T>(const Grid&, const OpView<T>&, const cx<T>*, const cx<T>*, int, const Ctl&, \
                                       int, cudaStream_t);                                                         \
  template void launch_restrict<T>(const Grid&, const Grid&, const cx<T>*, cx<T>*, int, const int*, const Xfer&,   \
                                   cudaStream_t);                                                                  \
  template void launch_prolong_add<T>(const Grid&, const Grid&, const cx<T>*, cx<T>*, int, const int*,            \
                                      const Xfer&, cudaStream_t);                                                  \
  template void launch_copy_masked<T>(const Grid&, const cx<T>*, cx<T>*, int, const int*, cudaStream_t);          \
  template void launch_pack<T>(const Grid&, const double2*, cx<T>*, int, int, cudaStream_t);                      \
  template void launch_unpack<T>(const Grid&, const cx<T>*, double2*, int, int, cudaStream_t);                    \
  template void launch_vecnorm_fin<T>(const Grid&, const cx<T>*, int, double*, double*, unsigned*, cudaStream_t);
INST(double)
INST(float)

}  // namespace hmg
