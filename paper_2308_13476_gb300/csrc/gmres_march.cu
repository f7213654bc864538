// GMRES(3) smoothing step (Sec. 5.3 of the paper) on the fine level in four
// row-marching passes plus the update.
//
// The node-parallel version (kernels_gmres.cu) stores w = A v_j and needs
// eight grid passes, about 28 vector reads and writes per step.  Here each
// warp owns a strip of columns and walks down a chunk of rows, keeping the
// last three rows of every field it needs in registers (horizontal
// neighbours come from the adjacent lanes by shuffles).  Row m of the next
// Arnoldi vector is formed as soon as rows m-1..m+1 of its input are in
// registers (w = A v_j is recomputed, never stored), and A is applied to
// the new vector one row behind, so the dots of Arnoldi step j+1 come out of
// the pass that creates u_{j+1}:
//   M0: u0 = b - A x                      |u0|^2, <u0, A u0>
//   M1: u1 = s0 A u0 - c00 u0             |u1|^2, <u1, u0>, <u_l, A u1>
//   M2: u2 = s1 A u1 - sum c_l1 u_l       |u2|^2, <u2, u_l>, <u_l, A u2>
//   M3: u3 = s2 A u2 - sum c_l2 u_l       |u3|^2 (not stored)
//   then x += sum y_l s_l u_l (g_update).
// That is 16 vector passes per step.  The scalar steps between passes are the
// same FP64 Gram-matrix updates and Givens solve (gmres.cuh) in the same order
// as the node-parallel version; only the dots of A u_{j+1} are taken before
// the scale s_{j+1} is known, and scaled afterwards.
//
// Geometry: a lane holds NP adjacent nodes (two for complex64, one 16-byte
// load; one for complex128).  A warp loads 32 NP columns starting two left of
// its strip; after the two stencil applications of a pass the outer two
// columns on each side are invalid, so a strip is 32 NP - 4 columns wide and
// neighbouring strips overlap by four loaded columns.  Rows: a warp covers a
// chunk of CH rows and reads two rows above and below it.  Nodes outside the
// grid are zero in every produced vector (they are not unknowns).
#include "gmres.cuh"
#include "internal.h"

namespace hmg {

namespace {

constexpr int MW = 4;   // warps per block

template <class T> struct MNP { static constexpr int NP = 1; };
template <> struct MNP<float> { static constexpr int NP = 2; };

template <class T> struct Row { cx<T> v[MNP<T>::NP]; };

template <class T> __device__ __forceinline__ cx<T> zc() { return mk<T>(T(0), T(0)); }
template <class T> __device__ __forceinline__ Row<T> zrow() {
  Row<T> r;
#pragma unroll
  for (int n = 0; n < MNP<T>::NP; ++n) r.v[n] = zc<T>();
  return r;
}

// Row j of a slice at this lane's nodes i.. (zero right of the grid; the
// padded layout makes the two columns left of the grid and the rows
// -2..ny+2 readable zeros).
__device__ __forceinline__ Row<float> mload(const float2* __restrict__ s, const Grid& g, int i, int j) {
  Row<float> r;
  if (i > g.nx) return zrow<float>();
  const float4 q = __ldg(reinterpret_cast<const float4*>(s + g.at(i, j)));
  r.v[0] = make_float2(q.x, q.y);
  r.v[1] = make_float2(q.z, q.w);
  return r;
}
__device__ __forceinline__ Row<double> mload(const double2* __restrict__ s, const Grid& g, int i, int j) {
  Row<double> r;
  r.v[0] = i > g.nx ? zc<double>() : __ldg(s + g.at(i, j));
  return r;
}
__device__ __forceinline__ void mstore(float2* __restrict__ d, const Grid& g, int i, int j, const Row<float>& r) {
  if (i + 1 <= g.nx)
    *reinterpret_cast<float4*>(d + g.at(i, j)) = make_float4(r.v[0].x, r.v[0].y, r.v[1].x, r.v[1].y);
  else if (i <= g.nx)
    d[g.at(i, j)] = r.v[0];
}
__device__ __forceinline__ void mstore(double2* __restrict__ d, const Grid& g, int i, int j, const Row<double>& r) {
  if (i <= g.nx) d[g.at(i, j)] = r.v[0];
}

template <class T> __device__ __forceinline__ cx<T> shfl_up1(cx<T> a) {
  return mk<T>(__shfl_up_sync(0xffffffffu, a.x, 1), __shfl_up_sync(0xffffffffu, a.y, 1));
}
template <class T> __device__ __forceinline__ cx<T> shfl_dn1(cx<T> a) {
  return mk<T>(__shfl_down_sync(0xffffffffu, a.x, 1), __shfl_down_sync(0xffffffffu, a.y, 1));
}

// (A v) on row m at this lane's nodes from rows m-1, m, m+1 of v; zero for
// nodes outside the grid.  All lanes must call it (shuffles).
template <class T>
__device__ __forceinline__ Row<T> mapply(const Op0<T>& op, const Row<T>& dn, const Row<T>& c, const Row<T>& up,
                                         int i, int m) {
  constexpr int NP = MNP<T>::NP;
  const cx<T> west = shfl_up1<T>(c.v[NP - 1]);
  const cx<T> east = shfl_dn1<T>(c.v[0]);
  Row<T> r;
  const bool rowin = m >= 0 && m <= op.ny;
#pragma unroll
  for (int n = 0; n < NP; ++n) {
    const int in = i + n;
    const cx<T> xe = n + 1 < NP ? c.v[n + 1 < NP ? n + 1 : 0] : east;
    const cx<T> xw = n > 0 ? c.v[n > 0 ? n - 1 : 0] : west;
    r.v[n] = (rowin && in >= 0 && in <= op.nx) ? op.apply5(c.v[n], xe, xw, up.v[n], dn.v[n], in, m) : zc<T>();
  }
  return r;
}

// Per-warp geometry inside one right-hand side.
struct MGeo {
  int nstrips, ch, nchunks;
};
template <class T> __host__ __device__ constexpr int strip_w() { return 32 * MNP<T>::NP - 4; }

// Common prologue.  `has`: the warp owns a (strip, chunk); i: first node of
// this lane; outl: the lane's nodes are in the strip's output columns.
#define MPRO                                                                  \
  constexpr int NP = MNP<T>::NP;                                              \
  __shared__ double sh[NVMAX * 32];                                           \
  const int rhs = blockIdx.z;                                                 \
  if (active && !active[rhs]) return;                                         \
  const long long off = (long long)rhs * g.vstride;                           \
  const int lane = threadIdx.x & 31;                                          \
  const int gw = blockIdx.x * MW + (threadIdx.x >> 5);                        \
  const bool has = gw < mg.nstrips * mg.nchunks;                              \
  const int strip = has ? gw % mg.nstrips : 0, chunk = has ? gw / mg.nstrips : 0; \
  const int i = strip * strip_w<T>() - 2 + NP * lane;                         \
  const bool outl = NP * lane >= 2 && NP * lane + NP <= 32 * NP - 2;          \
  const int j0 = chunk * mg.ch, j1 = min(j0 + mg.ch, g.ny + 1);               \
  const int nblk = gridDim.x, blk = blockIdx.x;                               \
  double* S = st + (long long)rhs * GS;

// node n of the lane counts in the dots of row m
#define MCOUNT(n, m) (outl && i + (n) <= g.nx && (m) >= j0 && (m) < j1)

// M0: u0 = b - A x; |u0|^2 and <u0, A u0>.
template <class T>
__global__ void __launch_bounds__(MW * 32) gm_init(Grid g, MGeo mg, Op0<T> op, const cx<T>* __restrict__ x,
                                                   const cx<T>* __restrict__ b, cx<T>* __restrict__ u0, double* st,
                                                   double* partial, unsigned* tickets,
                                                   const int* __restrict__ active) {
  MPRO
  T acc[3] = {T(0), T(0), T(0)};
  if (has) {
    const cx<T>* xs = x + off;
    const cx<T>* bs = b + off;
    cx<T>* us = u0 + off;
    // x rows t-2..t, b row t-1 (prefetched one row ahead); u0 rows t-3..t-1
    Row<T> x0, x1 = mload(xs, g, i, j0 - 2), x2 = mload(xs, g, i, j0 - 1);
    Row<T> xq = mload(xs, g, i, j0), bq = mload(bs, g, i, j0 - 1);
    Row<T> a0 = zrow<T>(), a1 = zrow<T>(), a2 = zrow<T>();
    for (int t = j0; t <= j1 + 1; ++t) {
      x0 = x1;
      x1 = x2;
      x2 = xq;
      const Row<T> bt = bq;
      if (t + 1 <= j1 + 1) {
        xq = mload(xs, g, i, t + 1);
        bq = mload(bs, g, i, t);
      }
      const Row<T> ax = mapply<T>(op, x0, x1, x2, i, t - 1);
      Row<T> u;
#pragma unroll
      for (int n = 0; n < NP; ++n) u.v[n] = sub<T>(bt.v[n], ax.v[n]);   // b and A x are zero outside the grid
      if (t - 1 >= j0 && t - 1 < j1 && outl) mstore(us, g, i, t - 1, u);
#pragma unroll
      for (int n = 0; n < NP; ++n)
        if (MCOUNT(n, t - 1)) acc[0] += abs2<T>(u.v[n]);
      a0 = a1;
      a1 = a2;
      a2 = u;
      if (t - 2 >= j0) {
        const Row<T> au = mapply<T>(op, a0, a1, a2, i, t - 2);
#pragma unroll
        for (int n = 0; n < NP; ++n)
          if (MCOUNT(n, t - 2)) {
            const cx<T> d = cmul<T>(a1.v[n], au.v[n]);
            acc[1] += d.x;
            acc[2] += d.y;
          }
      }
    }
  }
  double v[3];
  if (reduce_last<3, T>(acc, v, sh, partial, tickets, rhs, nblk, blk))
    staged<T>(S, v, [](double* s, const double* q) {
      fin_init<T>(s, q);
      if (s[G_BRK] == 0.0) {   // <u0, w> with w = s0 A u0
        const double d[2] = {q[1] * s[G_S], q[2] * s[G_S]};
        fin_a<0, T>(s, d);
      }
    });
}

// M1: u1 = s0 A u0 - c00 u0; |u1|^2, <u1, u0>, then <u0, A u1>, <u1, A u1>.
template <class T>
__global__ void __launch_bounds__(MW * 32) gm_step1(Grid g, MGeo mg, Op0<T> op, const cx<T>* __restrict__ u0,
                                                    cx<T>* __restrict__ u1, double* st, double* partial,
                                                    unsigned* tickets, const int* __restrict__ active) {
  MPRO
  if (S[G_BRK] != 0.0) return;   // uniform per RHS
  const T s0 = (T)S[G_S];
  const cx<T> c0 = mk<T>((T)(S[G_H] * S[G_S]), (T)(S[G_H + 1] * S[G_S]));
  T acc[7];
#pragma unroll
  for (int k = 0; k < 7; ++k) acc[k] = T(0);
  if (has) {
    const cx<T>* vs = u0 + off;
    cx<T>* ws = u1 + off;
    Row<T> a0, a1 = mload(vs, g, i, j0 - 2), a2 = mload(vs, g, i, j0 - 1), aq = mload(vs, g, i, j0);
    Row<T> b0 = zrow<T>(), b1 = zrow<T>(), b2 = zrow<T>();
    for (int t = j0; t <= j1 + 1; ++t) {
      a0 = a1;
      a1 = a2;
      a2 = aq;
      if (t + 1 <= j1 + 1) aq = mload(vs, g, i, t + 1);
      const Row<T> av = mapply<T>(op, a0, a1, a2, i, t - 1);
      Row<T> u;
#pragma unroll
      for (int n = 0; n < NP; ++n) u.v[n] = sub<T>(scl<T>(s0, av.v[n]), mul<T>(c0, a1.v[n]));
      if (t - 1 < 0 || t - 1 > g.ny) u = zrow<T>();
      else if (t - 1 >= j0 && t - 1 < j1 && outl) mstore(ws, g, i, t - 1, u);
#pragma unroll
      for (int n = 0; n < NP; ++n)
        if (MCOUNT(n, t - 1)) {
          acc[0] += abs2<T>(u.v[n]);
          const cx<T> d = cmul<T>(u.v[n], a1.v[n]);
          acc[1] += d.x;
          acc[2] += d.y;
        }
      b0 = b1;
      b1 = b2;
      b2 = u;
      if (t - 2 >= j0) {
        const Row<T> au = mapply<T>(op, b0, b1, b2, i, t - 2);
#pragma unroll
        for (int n = 0; n < NP; ++n)
          if (MCOUNT(n, t - 2)) {
            const cx<T> d0 = cmul<T>(a0.v[n], au.v[n]), d1 = cmul<T>(b1.v[n], au.v[n]);
            acc[3] += d0.x;
            acc[4] += d0.y;
            acc[5] += d1.x;
            acc[6] += d1.y;
          }
      }
    }
  }
  double v[7];
  if (reduce_last<7, T>(acc, v, sh, partial, tickets, rhs, nblk, blk))
    staged<T>(S, v, [](double* s, const double* q) {
      fin_b<0, T>(s, q);
      if (s[G_BRK] == 0.0) {
        const double s1 = s[G_S + 1];
        const double d[4] = {q[3] * s1, q[4] * s1, q[5] * s1, q[6] * s1};
        fin_a<1, T>(s, d);
      }
    });
}

// M2: u2 = s1 A u1 - c01 u0 - c11 u1; |u2|^2, <u2, u0>, <u2, u1>, then
// <u_l, A u2> for l = 0, 1, 2.
template <class T>
__global__ void __launch_bounds__(MW * 32) gm_step2(Grid g, MGeo mg, Op0<T> op, const cx<T>* __restrict__ u0,
                                                    const cx<T>* __restrict__ u1, cx<T>* __restrict__ u2, double* st,
                                                    double* partial, unsigned* tickets,
                                                    const int* __restrict__ active) {
  MPRO
  if (S[G_BRK] != 0.0 || S[G_M] < 1) return;
  const T s1 = (T)S[G_S + 1];
  const cx<T> c0 = mk<T>((T)(S[G_H + 2 * 1] * S[G_S]), (T)(S[G_H + 2 * 1 + 1] * S[G_S]));
  const cx<T> c1 = mk<T>((T)(S[G_H + 2 * 4] * S[G_S + 1]), (T)(S[G_H + 2 * 4 + 1] * S[G_S + 1]));
  T acc[11];
#pragma unroll
  for (int k = 0; k < 11; ++k) acc[k] = T(0);
  if (has) {
    const cx<T>* zs = u0 + off;
    const cx<T>* vs = u1 + off;
    cx<T>* ws = u2 + off;
    // u1 rows t-2..t, u0 rows t-2..t-1 (+ prefetch), u2 rows t-3..t-1
    Row<T> a0, a1 = mload(vs, g, i, j0 - 2), a2 = mload(vs, g, i, j0 - 1), aq = mload(vs, g, i, j0);
    Row<T> z0, z1 = mload(zs, g, i, j0 - 2), zq = mload(zs, g, i, j0 - 1);
    Row<T> b0 = zrow<T>(), b1 = zrow<T>(), b2 = zrow<T>();
    for (int t = j0; t <= j1 + 1; ++t) {
      a0 = a1;
      a1 = a2;
      a2 = aq;
      z0 = z1;
      z1 = zq;
      if (t + 1 <= j1 + 1) {
        aq = mload(vs, g, i, t + 1);
        zq = mload(zs, g, i, t);
      }
      const Row<T> av = mapply<T>(op, a0, a1, a2, i, t - 1);
      Row<T> u;
#pragma unroll
      for (int n = 0; n < NP; ++n) {
        u.v[n] = sub<T>(scl<T>(s1, av.v[n]), mul<T>(c0, z1.v[n]));
        u.v[n] = sub<T>(u.v[n], mul<T>(c1, a1.v[n]));
      }
      if (t - 1 < 0 || t - 1 > g.ny) u = zrow<T>();
      else if (t - 1 >= j0 && t - 1 < j1 && outl) mstore(ws, g, i, t - 1, u);
#pragma unroll
      for (int n = 0; n < NP; ++n)
        if (MCOUNT(n, t - 1)) {
          acc[0] += abs2<T>(u.v[n]);
          const cx<T> d0 = cmul<T>(u.v[n], z1.v[n]), d1 = cmul<T>(u.v[n], a1.v[n]);
          acc[1] += d0.x;
          acc[2] += d0.y;
          acc[3] += d1.x;
          acc[4] += d1.y;
        }
      b0 = b1;
      b1 = b2;
      b2 = u;
      if (t - 2 >= j0) {
        const Row<T> au = mapply<T>(op, b0, b1, b2, i, t - 2);
#pragma unroll
        for (int n = 0; n < NP; ++n)
          if (MCOUNT(n, t - 2)) {
            const cx<T> d0 = cmul<T>(z0.v[n], au.v[n]), d1 = cmul<T>(a0.v[n], au.v[n]),
                        d2 = cmul<T>(b1.v[n], au.v[n]);
            acc[5] += d0.x;
            acc[6] += d0.y;
            acc[7] += d1.x;
            acc[8] += d1.y;
            acc[9] += d2.x;
            acc[10] += d2.y;
          }
      }
    }
  }
  double v[11];
  if (reduce_last<11, T>(acc, v, sh, partial, tickets, rhs, nblk, blk))
    staged<T>(S, v, [](double* s, const double* q) {
      fin_b<1, T>(s, q);
      if (s[G_BRK] == 0.0) {
        const double s2 = s[G_S + 2];
        const double d[6] = {q[5] * s2, q[6] * s2, q[7] * s2, q[8] * s2, q[9] * s2, q[10] * s2};
        fin_a<2, T>(s, d);
      }
    });
}

// M3: |u3|^2 with u3 = s2 A u2 - sum_l c_l2 u_l; then the least-squares
// solve (fin_b<2>).
template <class T>
__global__ void __launch_bounds__(MW * 32) gm_step3(Grid g, MGeo mg, Op0<T> op, const cx<T>* __restrict__ u0,
                                                    const cx<T>* __restrict__ u1, const cx<T>* __restrict__ u2,
                                                    double* st, double* partial, unsigned* tickets,
                                                    const int* __restrict__ active) {
  MPRO
  if (S[G_BRK] != 0.0 || S[G_M] < 2) return;
  const T s2 = (T)S[G_S + 2];
  cx<T> cl[3];
#pragma unroll
  for (int l = 0; l < 3; ++l)
    cl[l] = mk<T>((T)(S[G_H + 2 * (l * 3 + 2)] * S[G_S + l]), (T)(S[G_H + 2 * (l * 3 + 2) + 1] * S[G_S + l]));
  T acc[1] = {T(0)};
  if (has) {
    const cx<T>* zs = u0 + off;
    const cx<T>* ys = u1 + off;
    const cx<T>* vs = u2 + off;
    // u2 rows t-2..t; u0, u1 row t-1 (all prefetched one row ahead)
    Row<T> a0, a1 = mload(vs, g, i, j0 - 1), a2 = mload(vs, g, i, j0), aq = mload(vs, g, i, j0 + 1);
    Row<T> zq = mload(zs, g, i, j0), yq = mload(ys, g, i, j0);
    for (int t = j0 + 1; t <= j1; ++t) {
      a0 = a1;
      a1 = a2;
      a2 = aq;
      const Row<T> z = zq, y = yq;
      if (t + 1 <= j1) {
        aq = mload(vs, g, i, t + 1);
        zq = mload(zs, g, i, t);
        yq = mload(ys, g, i, t);
      }
      const Row<T> av = mapply<T>(op, a0, a1, a2, i, t - 1);
#pragma unroll
      for (int n = 0; n < NP; ++n)
        if (MCOUNT(n, t - 1)) {
          cx<T> u = sub<T>(scl<T>(s2, av.v[n]), mul<T>(cl[0], z.v[n]));
          u = sub<T>(u, mul<T>(cl[1], y.v[n]));
          u = sub<T>(u, mul<T>(cl[2], a1.v[n]));
          acc[0] += abs2<T>(u);
        }
    }
  }
  double v[1];
  if (reduce_last<1, T>(acc, v, sh, partial, tickets, rhs, nblk, blk))
    staged<T>(S, v, [](double* s, const double* q) { fin_b<2, T>(s, q); });
}

// Rows per warp: tall chunks (few halo rows) unless the grid has too few
// strips to give every SM several warps.
template <class T> MGeo march_geo(const Grid& g, int B) {
  MGeo m;
  m.nstrips = cdiv(g.nx + 1, strip_w<T>());
  const long long want = 152LL * 48;   // warps to fill the GPU a few times over
  int ch = 64;
  while (ch > 8 && (long long)m.nstrips * cdiv(g.ny + 1, ch) * B < want) ch /= 2;
  m.ch = ch;
  m.nchunks = cdiv(g.ny + 1, ch);
  return m;
}

}  // namespace

// The x update of the node-parallel smoother (kernels_gmres.cu).
template <class T> void launch_gmres_update(const Grid& g, cx<T>* x, const GmresBufs& gb, int B, const int* active,
                                            cudaStream_t s);

long long gmres_march_blocks(const Grid& g, bool fp64, int B) {
  const MGeo m = fp64 ? march_geo<double>(g, B) : march_geo<float>(g, B);
  return cdiv((long long)m.nstrips * m.nchunks, MW);
}

template <class T>
void gmres_smooth_march(const Grid& g, const OpView<T>& opv, cx<T>* x, const cx<T>* b, int nu, int B,
                        const int* active, const GmresBufs& gb, cudaStream_t s) {
  cx<T>* u0 = (cx<T>*)gb.u[0];
  cx<T>* u1 = (cx<T>*)gb.u[1];
  cx<T>* u2 = (cx<T>*)gb.u[2];
  double* P = gb.partial;
  unsigned* tk = gb.tickets;
  double* st = gb.st;
  const Op0<T> op{opv.c0, opv.kf, g.nx, g.ny};
  const MGeo mg = march_geo<T>(g, B);
  const dim3 grd(cdiv((long long)mg.nstrips * mg.nchunks, MW), 1, B);
  for (int step = 0; step < nu; ++step) {
    gm_init<T><<<grd, MW * 32, 0, s>>>(g, mg, op, x, b, u0, st, P, tk, active);
    gm_step1<T><<<grd, MW * 32, 0, s>>>(g, mg, op, u0, u1, st, P, tk, active);
    gm_step2<T><<<grd, MW * 32, 0, s>>>(g, mg, op, u0, u1, u2, st, P, tk, active);
    gm_step3<T><<<grd, MW * 32, 0, s>>>(g, mg, op, u0, u1, u2, st, P, tk, active);
    launch_gmres_update<T>(g, x, gb, B, active, s);
  }
}

template void gmres_smooth_march<double>(const Grid&, const OpView<double>&, double2*, const double2*, int, int,
                                         const int*, const GmresBufs&, cudaStream_t);
template void gmres_smooth_march<float>(const Grid&, const OpView<float>&, float2*, const float2*, int, int,
                                        const int*, const GmresBufs&, cudaStream_t);

}  // namespace hmg
