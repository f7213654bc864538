// GMRES(3) smoother, Sec. 5.3 of the paper: every smoothing step runs three
// GMRES iterations from the current iterate (a polynomial smoother).
//
// One step, per right-hand side:
//   u0 = b - A x,  beta = ||u0||,  v0 = u0 / beta
//   for j = 0..2:  w = A v_j
//                  h_ij = <v_i, w> - sum_{l<i} h_lj <v_i, v_l>   (i <= j)
//                  u_{j+1} = w - sum_{i<=j} h_ij v_i,  h_{j+1,j} = ||u_{j+1}||
//                  stop early if h_{j+1,j} <= 1e-14 beta
//   y = argmin || beta e1 - Hbar y ||   (Givens rotations, FP64)
//   x += sum_i y_i v_i
// The h_ij formula is modified Gram-Schmidt written with the Gram matrix of
// the basis, which lets one pass over the grid produce all dots of step j.
// Vectors are kept unnormalised (v_i = s_i u_i); all scalars are FP64.
#include <math.h>

#include "gmres.cuh"
#include "internal.h"
#include "pack.cuh"
#include "ragged.cuh"
#include "ragged_api.h"

namespace hmg {

// Arguments of the flattened launches over a ragged batch (one per problem).
template <class T>
struct GbA {
  Grid g;
  const cx<T>* u0;
  const cx<T>* u1;
  const cx<T>* u2;
  cx<T>* un;
  const cx<T>* w;
  double* st;
  double* partial;
  unsigned* tickets;
  const int* active;
  int ws;
};

template <class T>
struct GuA {
  Grid g;
  cx<T>* x;
  const cx<T>* u0;
  const cx<T>* u1;
  const cx<T>* u2;
  const double* st;
  const int* active;
};

// The thread's pack starts at column i0 and holds nv nodes inside the grid.
#define GNODE                                            \
  constexpr int NP = PK<T>::NP;                          \
  const int rhs = blockIdx.z;                            \
  const int i0 = (blockIdx.x * BX + threadIdx.x) * NP;   \
  const int nv = min(NP, g.nx + 1 - i0);                 \
  const long long off = (long long)rhs * g.vstride;      \
  const int nblk = gridDim.x * gridDim.y;                \
  const int blk = blockIdx.y * gridDim.x + blockIdx.x;   \
  const bool t0 = threadIdx.x == 0 && threadIdx.y == 0;
#define GROWS for (int r_ = 0, j = blockIdx.y * BY * g.ry + threadIdx.y; r_ < g.ry; ++r_, j += BY)

// u0 = b - A x, partial |u0|^2
template <class T, class Op>
__global__ void __launch_bounds__(BX * BY) g_init(Grid g, Op op, const cx<T>* __restrict__ x, const cx<T>* __restrict__ b,
                                                  cx<T>* __restrict__ u0, double* __restrict__ st, double* partial,
                                                  unsigned* tickets, const int* __restrict__ active) {
  __shared__ double sh[NVMAX * 32];
  GNODE
  if (active && !active[rhs]) return;
  T a0[1] = {T(0)};   // per-thread sums in the working precision
  if (nv > 0) {
    GROWS {
      if (j > g.ny) break;
      const int p = g.at(i0, j);
      const Pack<T> ax = apply_pack<T>(op, x + off, p, g.pitch, i0, j);
      Pack<T> r = load_pack(b + off, p);
#pragma unroll
      for (int n = 0; n < NP; ++n) {
        r.v[n] = sub<T>(r.v[n], ax.v[n]);
        if (n < nv) a0[0] += abs2<T>(r.v[n]);
      }
      store_pack(u0 + off, p, r, nv);
    }
  }
  double v[1];
  if (reduce_last<1, T>(a0, v, sh, partial, tickets, rhs, nblk, blk) && t0) fin_init<T>(gstate<T>(st, rhs), v);
}

// g_init with x = 0: u0 = b (the caller takes b as u0), partial |b|^2 in
// g_init's order, so the state equals g_init's on a zero x.
template <class T>
__global__ void __launch_bounds__(BX * BY) g_init_zero(Grid g, const cx<T>* __restrict__ b, double* __restrict__ st,
                                                       double* partial, unsigned* tickets,
                                                       const int* __restrict__ active) {
  __shared__ double sh[NVMAX * 32];
  GNODE
  if (active && !active[rhs]) return;
  T a0[1] = {T(0)};
  if (nv > 0) {
    GROWS {
      if (j > g.ny) break;
      const Pack<T> r = load_pack(b + off, g.at(i0, j));
#pragma unroll
      for (int n = 0; n < NP; ++n)
        if (n < nv) a0[0] += abs2<T>(r.v[n]);
    }
  }
  double v[1];
  if (reduce_last<1, T>(a0, v, sh, partial, tickets, rhs, nblk, blk) && t0) fin_init<T>(gstate<T>(st, rhs), v);
}

// w = A v_J (v_J = s_J u_J); partial dots <u_i, w> for i <= J
template <class T, class Op, int J>
__global__ void __launch_bounds__(BX * BY) g_arn_a(Grid g, Op op, const cx<T>* __restrict__ u0, const cx<T>* __restrict__ u1,
                                                   const cx<T>* __restrict__ u2, cx<T>* __restrict__ w,
                                                   double* __restrict__ st, double* partial, unsigned* tickets,
                                                   const int* __restrict__ active) {
  __shared__ double sh[NVMAX * 32];
  GNODE
  if (active && !active[rhs]) return;
  T* S = gstate<T>(st, rhs);
  if (S[G_BRK] != 0 || S[G_M] < J) return;   // block-uniform
  const cx<T>* uJ = J == 0 ? u0 : (J == 1 ? u1 : u2);
  // complex64, J = 2: |w|^2 as well, for the Gram form of u3's norm
  // (fin_b2_gram); w is then not stored (no g_arn_b<2> pass reads it)
  constexpr int NG = (sizeof(T) == 4 && J == 2) ? 1 : 0;
  T acc[2 * (J + 1) + NG];
#pragma unroll
  for (int k = 0; k < 2 * (J + 1) + NG; ++k) acc[k] = T(0);
  if (nv > 0) {
    const T sJ = (T)S[G_S + J];
    const cx<T>* us[3] = {u0, u1, u2};
    GROWS {
      if (j > g.ny) break;
      const int p = g.at(i0, j);
      Pack<T> a = apply_pack<T>(op, uJ + off, p, g.pitch, i0, j);
#pragma unroll
      for (int n = 0; n < NP; ++n) a.v[n] = scl<T>(sJ, a.v[n]);
      if constexpr (NG == 1) {
#pragma unroll
        for (int n = 0; n < NP; ++n)
          if (n < nv) acc[2 * (J + 1)] += abs2<T>(a.v[n]);
      } else {
        store_pack(w + off, p, a, nv);
      }
#pragma unroll
      for (int l = 0; l <= J; ++l) {
        const Pack<T> ul = load_pack(us[l] + off, p);
#pragma unroll
        for (int n = 0; n < NP; ++n) {
          if (n < nv) {
            const cx<T> d = cmul<T>(ul.v[n], a.v[n]);
            acc[2 * l] += d.x;
            acc[2 * l + 1] += d.y;
          }
        }
      }
    }
  }
  double v[2 * (J + 1) + NG];
  if (reduce_last<2 * (J + 1) + NG, T>(acc, v, sh, partial, tickets, rhs, nblk, blk))
    staged<T>(S, v, [](auto* s, const double* q) {
      fin_a<J, T>(s, q);
      if constexpr (NG == 1) fin_b2_gram<T>(s, q[2 * (J + 1)]);
    });
}

// u_{J+1} = w - sum_{i<=J} h_iJ s_i u_i ; partials |u_{J+1}|^2 and <u_{J+1}, u_l>, l <= J (J < 2)
template <class T, int J>
__device__ __forceinline__ void g_arn_b_body(uint3 vblk, dim3 vgrid, Grid g, const cx<T>* __restrict__ u0, const cx<T>* __restrict__ u1, const cx<T>* __restrict__ u2, cx<T>* __restrict__ un, const cx<T>* __restrict__ w, double* __restrict__ st, double* partial, unsigned* tickets, const int* __restrict__ active, int ws) {
  const uint3 blockIdx = vblk;   // the block and grid inside this problem's launch
  const dim3 gridDim = vgrid;
  (void)blockIdx;
  (void)gridDim;
  constexpr int NV = (J < 2) ? 1 + 2 * (J + 1) : 1;
  __shared__ double sh[NVMAX * 32];
  GNODE
  if (active && !active[rhs]) return;
  T* S = gstate<T>(st, rhs);
  if (S[G_BRK] != 0 || S[G_M] < J) return;
  T acc[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) acc[k] = T(0);
  if (nv > 0) {
    const cx<T>* us[3] = {u0, u1, u2};
    cx<T> c[J + 1];
#pragma unroll
    for (int l = 0; l <= J; ++l) {
      const T hr = S[G_H + 2 * (l * 3 + J)], hi = S[G_H + 2 * (l * 3 + J) + 1];
      const T sl = S[G_S + l];
      c[l] = mk<T>((T)(hr * sl), (T)(hi * sl));
    }
    // ws >= 0: w was stored without its scale s_ws (fused Kronecker marches)
    const T wsc = ws >= 0 ? (T)S[G_S + ws] : T(1);
    GROWS {
      if (j > g.ny) break;
      const int p = g.at(i0, j);
      Pack<T> a = load_pack(w + off, p);
      if (ws >= 0) {
#pragma unroll
        for (int n = 0; n < NP; ++n) a.v[n] = scl<T>(wsc, a.v[n]);
      }
      Pack<T> uu[J + 1];
#pragma unroll
      for (int l = 0; l <= J; ++l) {
        uu[l] = load_pack(us[l] + off, p);
#pragma unroll
        for (int n = 0; n < NP; ++n) a.v[n] = sub<T>(a.v[n], mul<T>(c[l], uu[l].v[n]));
      }
      if (un) store_pack(un + off, p, a, nv);
#pragma unroll
      for (int n = 0; n < NP; ++n) {
        if (n >= nv) continue;
        acc[0] += abs2<T>(a.v[n]);
        if (J < 2) {
#pragma unroll
          for (int l = 0; l <= J && 1 + 2 * l + 1 < NV; ++l) {
            const cx<T> d = cmul<T>(a.v[n], uu[l].v[n]);
            acc[1 + 2 * l] += d.x;
            acc[2 + 2 * l] += d.y;
          }
        }
      }
    }
  }
  double v[NV];
  if (reduce_last<NV, T>(acc, v, sh, partial, tickets, rhs, nblk, blk)) staged<T>(S, v, [](auto* s, const double* q) { fin_b<J, T>(s, q); });
}

template <class T, int J>
__global__ void __launch_bounds__(BX * BY) g_arn_b(Grid g, const cx<T>* __restrict__ u0, const cx<T>* __restrict__ u1, const cx<T>* __restrict__ u2, cx<T>* __restrict__ un, const cx<T>* __restrict__ w, double* __restrict__ st, double* partial, unsigned* tickets, const int* __restrict__ active, int ws) {
  g_arn_b_body<T, J>(blockIdx, gridDim, g, u0, u1, u2, un, w, st, partial, tickets, active, ws);
}

template <class T, int J>
__global__ void __launch_bounds__(BX * BY) g_arn_b_rag(const __grid_constant__ RagLaunch<GbA<T>> L) {
  uint3 vb;
  dim3 vg;
  const GbA<T>& a = L.a[rag_problem(L, blockIdx.x, vb, vg)];
  g_arn_b_body<T, J>(vb, vg, a.g, a.u0, a.u1, a.u2, a.un, a.w, a.st, a.partial, a.tickets, a.active, a.ws);
}

// x += sum_{i<m} y_i s_i u_i
template <class T>
__device__ __forceinline__ void g_update_body(uint3 vblk, dim3 vgrid, Grid g, cx<T>* __restrict__ x, const cx<T>* __restrict__ u0, const cx<T>* __restrict__ u1, const cx<T>* __restrict__ u2, const double* __restrict__ st, const int* __restrict__ active) {
  const uint3 blockIdx = vblk;   // the block and grid inside this problem's launch
  const dim3 gridDim = vgrid;
  (void)blockIdx;
  (void)gridDim;
  constexpr int NP = PK<T>::NP;
  const int rhs = blockIdx.z;
  const int i0 = (blockIdx.x * BX + threadIdx.x) * NP;
  const int nv = min(NP, g.nx + 1 - i0);
  const long long off = (long long)rhs * g.vstride;
  if (active && !active[rhs]) return;
  if (nv <= 0) return;
  const T* S = gstate<T>(st, rhs);
  const int m = (int)S[G_M];
  if (m <= 0) return;
  const cx<T>* us[3] = {u0, u1, u2};
  cx<T> c[3];
#pragma unroll
  for (int l = 0; l < 3; ++l) {
    const T sl = S[G_S + l];
    c[l] = mk<T>((T)(S[G_Y + 2 * l] * sl), (T)(S[G_Y + 2 * l + 1] * sl));
  }
  GROWS {
    if (j > g.ny) break;
    const int p = g.at(i0, j);
    Pack<T> a = load_pack(x + off, p);
#pragma unroll
    for (int l = 0; l < 3; ++l) {
      if (l < m) {
        const Pack<T> ul = load_pack(us[l] + off, p);
#pragma unroll
        for (int n = 0; n < NP; ++n) a.v[n] = fma_c<T>(c[l], ul.v[n], a.v[n]);
      }
    }
    store_pack(x + off, p, a, nv);
  }
}

template <class T>
__global__ void __launch_bounds__(BX * BY) g_update(Grid g, cx<T>* __restrict__ x, const cx<T>* __restrict__ u0, const cx<T>* __restrict__ u1, const cx<T>* __restrict__ u2, const double* __restrict__ st, const int* __restrict__ active) {
  g_update_body<T>(blockIdx, gridDim, g, x, u0, u1, u2, st, active);
}

// The last GMRES(3) update of the level-0 post-smoothing of a complex64
// cycle inside the FP64 refinement, fused with the refinement's update: the
// updated complex64 iterate is the cycle's correction e, added to the FP64
// iterate at once (x64 += e, the widening on the integer pipe) instead of
// being stored and read back by a separate pass.  The complex64 iterate is
// not stored (the next cycle starts from zero).  With no Arnoldi column
// (m = 0) e is the iterate as it stands.
__global__ void __launch_bounds__(BX * BY) g_update_outer(Grid g, const float2* __restrict__ x,
                                                          const float2* __restrict__ u0, const float2* __restrict__ u1,
                                                          const float2* __restrict__ u2, const double* __restrict__ st,
                                                          double2* __restrict__ x64, const int* __restrict__ active) {
  using T = float;
  constexpr int NP = PK<T>::NP;
  const int rhs = blockIdx.z;
  const int i0 = (blockIdx.x * BX + threadIdx.x) * NP;
  const int nv = min(NP, g.nx + 1 - i0);
  const long long off = (long long)rhs * g.vstride;
  if (active && !active[rhs]) return;
  if (nv <= 0) return;
  const T* S = gstate<T>(st, rhs);
  const int m = (int)S[G_M];
  const cx<T>* us[3] = {u0, u1, u2};
  cx<T> c[3];
#pragma unroll
  for (int l = 0; l < 3; ++l) {
    const T sl = S[G_S + l];
    c[l] = mk<T>((T)(S[G_Y + 2 * l] * sl), (T)(S[G_Y + 2 * l + 1] * sl));
  }
  GROWS {
    if (j > g.ny) break;
    const int p = g.at(i0, j);
    Pack<T> a = load_pack(x + off, p);
#pragma unroll
    for (int l = 0; l < 3; ++l) {
      if (l < m) {
        const Pack<T> ul = load_pack(us[l] + off, p);
#pragma unroll
        for (int n = 0; n < NP; ++n) a.v[n] = fma_c<T>(c[l], ul.v[n], a.v[n]);
      }
    }
#pragma unroll
    for (int n = 0; n < NP; ++n) {
      if (n < nv) {
        double2 xv = x64[off + p + n];
        xv.x += f64_from_f32(a.v[n].x);
        xv.y += f64_from_f32(a.v[n].y);
        x64[off + p + n] = xv;
      }
    }
  }
}

template <class T>
__global__ void __launch_bounds__(BX * BY) g_update_rag(const __grid_constant__ RagLaunch<GuA<T>> L) {
  uint3 vb;
  dim3 vg;
  const GuA<T>& a = L.a[rag_problem(L, blockIdx.x, vb, vg)];
  g_update_body<T>(vb, vg, a.g, a.x, a.u0, a.u1, a.u2, a.st, a.active);
}

template <class T>
void gmres_smooth(const Grid& g, const OpView<T>& opv, cx<T>* x, const cx<T>* b, int nu, int B, const int* active,
                  const GmresBufs& gb, cudaStream_t s) {
  dim3 grd(cdiv(g.nx + 1, BX * PK<T>::NP), cdiv(g.ny + 1, BY * g.ry), B);
  cx<T>* u0 = (cx<T>*)gb.u[0];
  cx<T>* u1 = (cx<T>*)gb.u[1];
  cx<T>* u2 = (cx<T>*)gb.u[2];
  cx<T>* w = (cx<T>*)gb.w;
  double* P = gb.partial;
  unsigned* tk = gb.tickets;
  double* st = gb.st;
  const dim3 blk(BX, BY);
  with_op<T>(opv, g.nx, g.ny, [&](auto op) {
    using Op = decltype(op);
    for (int step = 0; step < nu; ++step) {
      // a zero x: u0 = b itself (read-only in every later pass), no apply
      const bool z = step == 0 && gb.x_zero;
      const cx<T>* v0 = z ? b : u0;
      if (z) g_init_zero<T><<<grd, blk, 0, s>>>(g, b, st, P, tk, active);
      else g_init<T, Op><<<grd, blk, 0, s>>>(g, op, x, b, u0, st, P, tk, active);
      g_arn_a<T, Op, 0><<<grd, blk, 0, s>>>(g, op, v0, u1, u2, w, st, P, tk, active);
      g_arn_b<T, 0><<<grd, blk, 0, s>>>(g, v0, u1, u2, u1, w, st, P, tk, active, -1);
      g_arn_a<T, Op, 1><<<grd, blk, 0, s>>>(g, op, v0, u1, u2, w, st, P, tk, active);
      g_arn_b<T, 1><<<grd, blk, 0, s>>>(g, v0, u1, u2, u2, w, st, P, tk, active, -1);
      g_arn_a<T, Op, 2><<<grd, blk, 0, s>>>(g, op, v0, u1, u2, w, st, P, tk, active);
      if constexpr (sizeof(T) == 8)   // complex64: u3's norm came from the Gram form in g_arn_a<2>
        g_arn_b<T, 2><<<grd, blk, 0, s>>>(g, v0, u1, u2, nullptr, w, st, P, tk, active, -1);
      GmresBufs gs = gb;
      gs.u[0] = (void*)v0;
      if constexpr (sizeof(T) == 4) {
        if (step == nu - 1 && gb.outer) {
          launch_gmres_update_outer(g, x, gs, B, active, s);
          continue;
        }
      }
      g_update<T><<<grd, blk, 0, s>>>(g, x, v0, u1, u2, st, active);
    }
  });
}


template <class T>
void launch_gmres_update(const Grid& g, cx<T>* x, const GmresBufs& gb, int B, const int* active, cudaStream_t s) {
  dim3 grd(cdiv(g.nx + 1, BX * PK<T>::NP), cdiv(g.ny + 1, BY * g.ry), B);
  g_update<T><<<grd, dim3(BX, BY), 0, s>>>(g, x, (const cx<T>*)gb.u[0], (const cx<T>*)gb.u[1],
                                          (const cx<T>*)gb.u[2], gb.st, active);
}

void launch_gmres_update_outer(const Grid& g, const float2* x, const GmresBufs& gb, int B, const int* active,
                               cudaStream_t s) {
  dim3 grd(cdiv(g.nx + 1, BX * PK<float>::NP), cdiv(g.ny + 1, BY * g.ry), B);
  g_update_outer<<<grd, dim3(BX, BY), 0, s>>>(g, x, (const float2*)gb.u[0], (const float2*)gb.u[1],
                                              (const float2*)gb.u[2], gb.st, gb.outer, active);
}

template <class T, int J>
void launch_arn_b(const Grid& g, const GmresBufs& gb, cx<T>* un, int B, const int* active, cudaStream_t s, int ws) {
  dim3 grd(cdiv(g.nx + 1, BX * PK<T>::NP), cdiv(g.ny + 1, BY * g.ry), B);
  g_arn_b<T, J><<<grd, dim3(BX, BY), 0, s>>>(g, (const cx<T>*)gb.u[0], (const cx<T>*)gb.u[1], (const cx<T>*)gb.u[2],
                                            un, (const cx<T>*)gb.w, gb.st, gb.partial, gb.tickets, active, ws);
}

template <class T> void launch_gmres_update_rag(const std::vector<RagLevel<T>>& v, cudaStream_t s) {
  rag_launch<GuA<T>>((int)v.size(), g_update_rag<T>, dim3(BX, BY), 0, s, [&](int q, GuA<T>& a, int& gx, int& gy) {
    const RagLevel<T>& L = v[q];
    a = GuA<T>{L.g, L.x, (const cx<T>*)L.gb.u[0], (const cx<T>*)L.gb.u[1], (const cx<T>*)L.gb.u[2], L.gb.st, L.active};
    gx = cdiv(L.g.nx + 1, BX * PK<T>::NP);
    gy = cdiv(L.g.ny + 1, BY * L.g.ry);
    return true;
  });
}

template <class T, int J>
void launch_arn_b_rag(const std::vector<RagLevel<T>>& v, bool un_next, int ws, cudaStream_t s) {
  rag_launch<GbA<T>>((int)v.size(), g_arn_b_rag<T, J>, dim3(BX, BY), 0, s, [&](int q, GbA<T>& a, int& gx, int& gy) {
    const RagLevel<T>& L = v[q];
    cx<T>* un = un_next && J < 2 ? (cx<T>*)L.gb.u[J + 1] : nullptr;
    a = GbA<T>{L.g, (const cx<T>*)L.gb.u[0], (const cx<T>*)L.gb.u[1], (const cx<T>*)L.gb.u[2], un,
               (const cx<T>*)L.gb.w, L.gb.st, L.gb.partial, L.gb.tickets, L.active, ws};
    gx = cdiv(L.g.nx + 1, BX * PK<T>::NP);
    gy = cdiv(L.g.ny + 1, BY * L.g.ry);
    return true;
  });
}

template void launch_gmres_update_rag<double>(const std::vector<RagLevel<double>>&, cudaStream_t);
template void launch_gmres_update_rag<float>(const std::vector<RagLevel<float>>&, cudaStream_t);
template void launch_arn_b_rag<double, 0>(const std::vector<RagLevel<double>>&, bool, int, cudaStream_t);
template void launch_arn_b_rag<double, 1>(const std::vector<RagLevel<double>>&, bool, int, cudaStream_t);
template void launch_arn_b_rag<double, 2>(const std::vector<RagLevel<double>>&, bool, int, cudaStream_t);
template void launch_arn_b_rag<float, 0>(const std::vector<RagLevel<float>>&, bool, int, cudaStream_t);
template void launch_arn_b_rag<float, 1>(const std::vector<RagLevel<float>>&, bool, int, cudaStream_t);
template void launch_arn_b_rag<float, 2>(const std::vector<RagLevel<float>>&, bool, int, cudaStream_t);
template void launch_arn_b<double, 0>(const Grid&, const GmresBufs&, double2*, int, const int*, cudaStream_t, int);
template void launch_arn_b<double, 1>(const Grid&, const GmresBufs&, double2*, int, const int*, cudaStream_t, int);
template void launch_arn_b<double, 2>(const Grid&, const GmresBufs&, double2*, int, const int*, cudaStream_t, int);
template void launch_arn_b<float, 0>(const Grid&, const GmresBufs&, float2*, int, const int*, cudaStream_t, int);
template void launch_arn_b<float, 1>(const Grid&, const GmresBufs&, float2*, int, const int*, cudaStream_t, int);
template void launch_arn_b<float, 2>(const Grid&, const GmresBufs&, float2*, int, const int*, cudaStream_t, int);
template void launch_gmres_update<double>(const Grid&, double2*, const GmresBufs&, int, const int*, cudaStream_t);
template void launch_gmres_update<float>(const Grid&, float2*, const GmresBufs&, int, const int*, cudaStream_t);
template void gmres_smooth<double>(const Grid&, const OpView<double>&, double2*, const double2*, int, int, const int*,
                                   const GmresBufs&, cudaStream_t);
template void gmres_smooth<float>(const Grid&, const OpView<float>&, float2*, const float2*, int, int, const int*,
                                  const GmresBufs&, cudaStream_t);

}  // namespace hmg
