// GMRES(3) smoothing step (Sec. 5.3 of the paper) on the fine level in four
// row-marching passes plus the update.
//
// The node-parallel version (kernels_gmres.cu) stores w = A v_j and needs
// eight grid passes, about 28 vector reads and writes per step.  Here each
// warp owns a strip of columns and walks down a chunk of rows, keeping the
// rows it needs of every field in registers (horizontal neighbours come from
// the adjacent lanes by shuffles).  Row m of the next Arnoldi vector is
// formed as soon as rows m-1..m+1 of its input are in registers (w = A v_j is
// recomputed, never stored), and A is applied to the new vector one row
// behind, so the dots of Arnoldi step j+1 come out of the pass that creates
// u_{j+1}:
//   M0: u0 = b - A x                      |u0|^2, <u0, A u0>
//   M1: u1 = s0 A u0 - c00 u0             |u1|^2, <u1, u0>, <u_l, A u1>
//   M2: u2 = s1 A u1 - sum c_l1 u_l       |u2|^2, <u2, u_l>, <u_l, A u2>
//   M3: u3 = s2 A u2 - sum c_l2 u_l       |u3|^2 (not stored)
//   then x += sum y_l s_l u_l (g_update).
// That is 16 vector passes per step.  complex64 steps skip M3: M2 also sums
// |A u2|^2, and |u3|^2 follows from the Gram form (13 vector passes).  The scalar steps between passes are the
// same FP64 Gram-matrix updates and Givens solve (gmres.cuh) in the same order
// as the node-parallel version; only the dots of A u_{j+1} are taken before
// the scale s_{j+1} is known, and scaled afterwards.
//
// Geometry: a lane holds NP adjacent nodes (two for complex64, one 16-byte
// load; one for complex128).  A warp loads 32 NP columns starting two left of
// its strip; after the two stencil applications of a pass the outer two
// columns on each side are invalid, so a strip is 32 NP - 4 columns wide and
// neighbouring strips overlap by four loaded columns.  Rows: a warp covers a
// chunk of rows (see MGeo) and reads two rows above and below it.  Nodes outside the
// grid are zero in every produced vector (they are not unknowns).
//
// Rows arrive through a per-lane ring of NS 16-byte shared-memory slots per
// field, filled by cp.async NS - 1 rows ahead of use (each lane reads back
// only what it copied, so no barrier is needed).  A pass with fewer input
// fields keeps more rows in flight (NS = 8, 6, 4 for one, two, three fields),
// so that every pass has about the same bytes in flight per SM: with one warp
// per block and at most 32 blocks per SM, a one-field pass staging three rows
// ahead ran at half the bandwidth of the three-field pass.  Every field keeps
// the rows it uses in a ring of four registers; row r sits in register slot
// (r - j0 + 2) mod 4, and the march is unrolled by four so that these slots
// are compile-time names (no copies as the ring advances).  The block's
// reduction scratch reuses the staging ring once the march has ended.  A warp whose loaded
// columns and computed rows hold no boundary node takes the interior path:
// the stencil without boundary tests (the same arithmetic as Op0::apply5's
// interior case).
#include <algorithm>

#include "gmres.cuh"
#include "internal.h"
#include "ragged.cuh"
#include "ragged_api.h"

namespace hmg {

namespace {

// staging slots per field of a pass with NF input fields
template <int NF> struct Ring { static constexpr int NS = NF == 1 ? 8 : NF == 2 ? 6 : 4; };
// shared memory of a pass: the staging ring, and afterwards the [NVMAX][32]
// doubles of the block reduction
template <int NF> constexpr int ring_bytes() {
  return NF * Ring<NF>::NS * 32 * 16 > NVMAX * 32 * 8 ? NF * Ring<NF>::NS * 32 * 16 : NVMAX * 32 * 8;
}

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

// Asynchronous copy of this lane's 16 bytes of row j (nodes i..) into a
// shared-memory slot; columns right of the grid are zero-filled (the padded
// layout makes the two columns left of the grid and the rows -2..ny+2
// readable zeros).
template <class T>
__device__ __forceinline__ void stage_row(uint32_t dst, const cx<T>* __restrict__ s, const Grid& g, int i, int j) {
  const bool ok = i <= g.nx;
  const cx<T>* src = s + g.at(ok ? i : 0, j);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src), "r"(ok ? 16 : 0) : "memory");
}
__device__ __forceinline__ void stage_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N> __device__ __forceinline__ void stage_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}
__device__ __forceinline__ Row<float> stage_read(const float4* p) {
  const float4 q = *p;
  Row<float> r;
  r.v[0] = make_float2(q.x, q.y);
  r.v[1] = make_float2(q.z, q.w);
  return r;
}
__device__ __forceinline__ Row<double> stage_read(const double2* p) {
  Row<double> r;
  r.v[0] = *p;
  return r;
}
template <class T> struct SlotT { using type = double2; };
template <> struct SlotT<float> { using type = float4; };

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

// March modes: MD = 1 interior strips (branch-free stencil), MD = 2 edge
// strips over interior rows (the same stencil, with the boundary row of
// Op0::apply5 on columns 0 and nx and zero off the grid), MD = 0 everything
// else (the 3-row bands; every warp on grids of fewer than 7 rows).  MD + 4
// (modes 0 and 2 only): the same with the second-order absorbing rows of
// Op0<T, true> on the boundary nodes (interior strips touch none).
template <int MD> constexpr int MM = MD & 3;
template <int MD> constexpr bool MA2 = (MD & 4) != 0;
// Per-warp march context.
template <class T, int MD> struct MCtx {
  static constexpr int NP = MNP<T>::NP;
  Op0<T, MA2<MD>> op;
  Grid g;
  int i;       // first node of this lane
  int j0, j1;  // chunk rows [j0, j1)
  bool outl;   // the lane's nodes are in the strip's output columns

  // (A v) on row m from rows m-1, m, m+1 of v; zero for nodes outside the
  // grid.  All lanes must call it (shuffles).
  __device__ __forceinline__ Row<T> apply(const Row<T>& dn, const Row<T>& c, const Row<T>& up, int m) const {
    const cx<T> west = shfl_up1<T>(c.v[NP - 1]);
    const cx<T> east = shfl_dn1<T>(c.v[0]);
    Row<T> r;
#pragma unroll
    for (int n = 0; n < NP; ++n) {
      const cx<T> xe = n + 1 < NP ? c.v[n + 1 < NP ? n + 1 : 0] : east;
      const cx<T> xw = n > 0 ? c.v[n > 0 ? n - 1 : 0] : west;
      const int in = i + n;
      if (MM<MD> != 0) {   // Op0::apply5, interior case
        const cx<T> xn = up.v[n], xs = dn.v[n], xp = c.v[n];
        const int ik = MM<MD> == 2 ? min(max(in, 0), op.nx) : in;   // edge strips: k of an in-grid node
        const T k = op.kf ? op.kf[m * (op.nx + 1) + ik] : op.c.k;
        const T d = fma(-k, k, T(4) * op.c.inv_h2);
        if constexpr (sizeof(T) == 4) {   // the same operations, both components per instruction
          const float2 sn = add2(add2(xe, xw), add2(xn, xs));
          r.v[n] = fma2(bc2(d), xp, mul2(bc2(-op.c.inv_h2), sn));
        } else {
          const T sr = (xe.x + xw.x) + (xn.x + xs.x), si = (xe.y + xw.y) + (xn.y + xs.y);
          r.v[n] = mk<T>(fma(d, xp.x, -op.c.inv_h2 * sr), fma(d, xp.y, -op.c.inv_h2 * si));
        }
        if (MM<MD> == 2) {   // rows are interior here; columns 0 and nx take the
                         // boundary row of Op0::apply5, columns off the grid zero
          const bool bcol = in == 0 || in == op.nx, inside = in >= 0 && in <= op.nx;
          if (bcol) r.v[n] = op.apply5(xp, xe, xw, xn, xs, in, m);
          if (!inside) r.v[n] = zc<T>();
        }
      } else {
        r.v[n] = (m >= 0 && m <= op.ny && in >= 0 && in <= op.nx)
                     ? op.apply5(c.v[n], xe, xw, up.v[n], dn.v[n], in, m)
                     : zc<T>();
      }
    }
    return r;
  }
  // node n of the lane counts in the dots of row m
  __device__ __forceinline__ bool cnt(int n, int m) const {
    return outl && (MM<MD> == 1 || i + n <= g.nx) && m >= j0 && m < j1;
  }
  __device__ __forceinline__ bool own_row(int m) const { return outl && m >= j0 && m < j1; }
};

// Register slot of row t + d at unroll phase S (the march starts at t0 = j0 -
// 2 with phase 0, so row r sits in slot (r - j0 + 2) mod 4).
template <int S, int D> struct Sl { static constexpr int v = (S + D + 8) & 3; };

// The NF input fields of a pass: shared-memory staging and register rings.
// Staging slot (f, k) of a lane is at sbase + (f NS + k) 512 bytes.
template <class T, int MD, int NF> struct MIn {
  static constexpr int NS = Ring<NF>::NS, AH = NS - 1;   // AH: rows in flight ahead of use
  MCtx<T, MD> c;
  const cx<T>* src[NF];
  uint32_t sbase;   // shared address of this lane's slot 0 of field 0
  Row<T> F[NF][4];  // register ring: row r in slot (r - j0 + 2) mod 4
  int t1;           // last row the march reads
  int sw, sr;       // staging slots of the next row to issue and to read

  __device__ __forceinline__ void issue(int r, int slot) {
#pragma unroll
    for (int f = 0; f < NF; ++f) stage_row<T>(sbase + (f * NS + slot) * 32 * 16, src[f], c.g, c.i, r);
  }
  // rows t0 .. t0 + AH - 1 in flight, in slots 0 .. AH - 1
  __device__ __forceinline__ void prime(int t0) {
#pragma unroll
    for (int d = 0; d < AH; ++d) {
      if (t0 + d <= t1) issue(t0 + d, d);
      stage_commit();
    }
    sw = AH;
    sr = 0;
  }
  // row t + AH in flight (into the slot row t - 1 left), row t into the
  // register ring
  template <int S> __device__ __forceinline__ void fetch(int t) {
    if (t + AH <= t1) issue(t + AH, sw);
    sw = sw + 1 == NS ? 0 : sw + 1;
    stage_commit();
    stage_wait<AH>();
#pragma unroll
    for (int f = 0; f < NF; ++f)
      F[f][Sl<S, 0>::v] = stage_read(reinterpret_cast<const typename SlotT<T>::type*>(
          __cvta_shared_to_generic(sbase + (f * NS + sr) * 32 * 16)));
    sr = sr + 1 == NS ? 0 : sr + 1;
  }
};

// Runs p.step<S>(t) for t = t0..t1, S = (t - t0) mod 4.
template <class P> __device__ __forceinline__ void march(P& p, int t0, int t1) {
#pragma unroll 1
  for (int t = t0; t <= t1; t += 4) {
    p.template step<0>(t);
    if (t + 1 > t1) break;
    p.template step<1>(t + 1);
    if (t + 2 > t1) break;
    p.template step<2>(t + 2);
    if (t + 3 > t1) break;
    p.template step<3>(t + 3);
  }
}

// complex64 steps take the norm of the last Arnoldi vector u3 = A v2 -
// sum_l h_l2 v_l from the Gram form instead of a fourth pass: with unit
// v_l the modified Gram-Schmidt steps give |u3|^2 = |A v2|^2 - sum_l
// |h_l2|^2 exactly, so M2 also sums |A u2|^2 (s_2 A u2 = A v2) and M3 is
// not run.  complex128 steps keep M3 (their iterates follow the oracle's
// explicit norm to rounding).
template <class T> constexpr bool G3 = sizeof(T) == 4;
template <class T> constexpr int NV2 = G3<T> ? 12 : 11;

// M0 at iteration t: x and b rows t arrive; u0 row t-1 = b - A x formed from
// x rows t-2..t; A u0 on row t-2.
template <class T, int MD> struct P0 {
  static constexpr int NP = MNP<T>::NP;
  MIn<T, MD, 2> m;   // 0: x, 1: b
  cx<T>* us;
  Row<T> U[4];
  T acc[3];
  template <int S> __device__ __forceinline__ void step(int t) {
    m.template fetch<S>(t);
    const MCtx<T, MD>& c = m.c;
    if (t < c.j0) return;
    const Row<T> ax = c.apply(m.F[0][Sl<S, -2>::v], m.F[0][Sl<S, -1>::v], m.F[0][Sl<S, 0>::v], t - 1);
    Row<T> u;
#pragma unroll
    for (int n = 0; n < NP; ++n) u.v[n] = psub<T>(m.F[1][Sl<S, -1>::v].v[n], ax.v[n]);   // both zero outside the grid
    U[Sl<S, -1>::v] = u;
    if (c.own_row(t - 1)) mstore(us, c.g, c.i, t - 1, u);
#pragma unroll
    for (int n = 0; n < NP; ++n)
      if (c.cnt(n, t - 1)) acc[0] += abs2<T>(u.v[n]);
    if (t - 2 >= c.j0) {
      const Row<T> au = c.apply(U[Sl<S, -3>::v], U[Sl<S, -2>::v], U[Sl<S, -1>::v], t - 2);
#pragma unroll
      for (int n = 0; n < NP; ++n)
        if (c.cnt(n, t - 2)) {
          const cx<T> d = cmul<T>(U[Sl<S, -2>::v].v[n], au.v[n]);
          acc[1] += d.x;
          acc[2] += d.y;
        }
    }
  }
};

// M0 on a zero x (u0 = b, not stored): b row t arrives; |u0|^2 on row t-1
// and A u0 on row t-2, in P0's order (the same sums as P0 with x = 0).
template <class T, int MD> struct P0Z {
  static constexpr int NP = MNP<T>::NP;
  MIn<T, MD, 1> m;   // 0: b
  T acc[3];
  template <int S> __device__ __forceinline__ void step(int t) {
    m.template fetch<S>(t);
    const MCtx<T, MD>& c = m.c;
    if (t < c.j0) return;
    const Row<T>(&U)[4] = m.F[0];
#pragma unroll
    for (int n = 0; n < NP; ++n)
      if (c.cnt(n, t - 1)) acc[0] += abs2<T>(U[Sl<S, -1>::v].v[n]);
    if (t - 2 >= c.j0) {
      const Row<T> au = c.apply(U[Sl<S, -3>::v], U[Sl<S, -2>::v], U[Sl<S, -1>::v], t - 2);
#pragma unroll
      for (int n = 0; n < NP; ++n)
        if (c.cnt(n, t - 2)) {
          const cx<T> d = cmul<T>(U[Sl<S, -2>::v].v[n], au.v[n]);
          acc[1] += d.x;
          acc[2] += d.y;
        }
    }
  }
};

// M1 at iteration t: u0 row t arrives; u1 row t-1 formed; A u1 on row t-2.
template <class T, int MD> struct P1 {
  static constexpr int NP = MNP<T>::NP;
  MIn<T, MD, 1> m;   // 0: u0
  cx<T>* ws;
  T s0;
  cx<T> c0;
  Row<T> U[4];
  T acc[7];
  template <int S> __device__ __forceinline__ void step(int t) {
    m.template fetch<S>(t);
    const MCtx<T, MD>& c = m.c;
    if (t < c.j0) return;
    const Row<T>(&V)[4] = m.F[0];
    const Row<T> av = c.apply(V[Sl<S, -2>::v], V[Sl<S, -1>::v], V[Sl<S, 0>::v], t - 1);
    Row<T> u;
#pragma unroll
    for (int n = 0; n < NP; ++n) {
      const cx<T> c[1] = {c0};
      const cx<T> v[1] = {V[Sl<S, -1>::v].v[n]};
      u.v[n] = scl_minus<T, 1>(s0, av.v[n], c, v);
    }
    U[Sl<S, -1>::v] = u;
    if (c.own_row(t - 1)) mstore(ws, c.g, c.i, t - 1, u);
#pragma unroll
    for (int n = 0; n < NP; ++n)
      if (c.cnt(n, t - 1)) {
        acc[0] += abs2<T>(u.v[n]);
        const cx<T> d = cmul<T>(u.v[n], V[Sl<S, -1>::v].v[n]);
        acc[1] += d.x;
        acc[2] += d.y;
      }
    if (t - 2 >= c.j0) {
      const Row<T> au = c.apply(U[Sl<S, -3>::v], U[Sl<S, -2>::v], U[Sl<S, -1>::v], t - 2);
#pragma unroll
      for (int n = 0; n < NP; ++n)
        if (c.cnt(n, t - 2)) {
          const cx<T> d0 = cmul<T>(V[Sl<S, -2>::v].v[n], au.v[n]), d1 = cmul<T>(U[Sl<S, -2>::v].v[n], au.v[n]);
          acc[3] += d0.x;
          acc[4] += d0.y;
          acc[5] += d1.x;
          acc[6] += d1.y;
        }
    }
  }
};

// M2 at iteration t: u1 and u0 rows t arrive; u2 row t-1 formed; A u2 on
// row t-2.
template <class T, int MD> struct P2 {
  static constexpr int NP = MNP<T>::NP;
  MIn<T, MD, 2> m;   // 0: u1, 1: u0
  cx<T>* ws;
  T s1;
  cx<T> c0, c1;
  Row<T> U[4];
  T acc[NV2<T>];
  template <int S> __device__ __forceinline__ void step(int t) {
    m.template fetch<S>(t);
    const MCtx<T, MD>& c = m.c;
    if (t < c.j0) return;
    const Row<T>(&V)[4] = m.F[0];
    const Row<T>(&Z)[4] = m.F[1];
    const Row<T> av = c.apply(V[Sl<S, -2>::v], V[Sl<S, -1>::v], V[Sl<S, 0>::v], t - 1);
    Row<T> u;
#pragma unroll
    for (int n = 0; n < NP; ++n) {
      const cx<T> c[2] = {c0, c1};
      const cx<T> v[2] = {Z[Sl<S, -1>::v].v[n], V[Sl<S, -1>::v].v[n]};
      u.v[n] = scl_minus<T, 2>(s1, av.v[n], c, v);
    }
    U[Sl<S, -1>::v] = u;
    if (c.own_row(t - 1)) mstore(ws, c.g, c.i, t - 1, u);
#pragma unroll
    for (int n = 0; n < NP; ++n)
      if (c.cnt(n, t - 1)) {
        acc[0] += abs2<T>(u.v[n]);
        const cx<T> d0 = cmul<T>(u.v[n], Z[Sl<S, -1>::v].v[n]), d1 = cmul<T>(u.v[n], V[Sl<S, -1>::v].v[n]);
        acc[1] += d0.x;
        acc[2] += d0.y;
        acc[3] += d1.x;
        acc[4] += d1.y;
      }
    if (t - 2 >= c.j0) {
      const Row<T> au = c.apply(U[Sl<S, -3>::v], U[Sl<S, -2>::v], U[Sl<S, -1>::v], t - 2);
#pragma unroll
      for (int n = 0; n < NP; ++n)
        if (c.cnt(n, t - 2)) {
          const cx<T> d0 = cmul<T>(Z[Sl<S, -2>::v].v[n], au.v[n]), d1 = cmul<T>(V[Sl<S, -2>::v].v[n], au.v[n]),
                      d2 = cmul<T>(U[Sl<S, -2>::v].v[n], au.v[n]);
          acc[5] += d0.x;
          acc[6] += d0.y;
          acc[7] += d1.x;
          acc[8] += d1.y;
          acc[9] += d2.x;
          acc[10] += d2.y;
          if constexpr (G3<T>) acc[11] += abs2<T>(au.v[n]);   // |A u2|^2: u3's norm without M3
        }
    }
  }
};

// M3 at iteration t: u2, u0 and u1 rows t arrive; u3 on row t-1.
template <class T, int MD> struct P3 {
  static constexpr int NP = MNP<T>::NP;
  MIn<T, MD, 3> m;   // 0: u2, 1: u0, 2: u1
  T s2;
  cx<T> cl[3];
  T acc[1];
  template <int S> __device__ __forceinline__ void step(int t) {
    m.template fetch<S>(t);
    const MCtx<T, MD>& c = m.c;
    if (t < c.j0 + 1) return;
    const Row<T>(&V)[4] = m.F[0];
    const Row<T> av = c.apply(V[Sl<S, -2>::v], V[Sl<S, -1>::v], V[Sl<S, 0>::v], t - 1);
#pragma unroll
    for (int n = 0; n < NP; ++n)
      if (c.cnt(n, t - 1)) {
        const cx<T> v[3] = {m.F[1][Sl<S, -1>::v].v[n], m.F[2][Sl<S, -1>::v].v[n], V[Sl<S, -1>::v].v[n]};
        const cx<T> u = scl_minus<T, 3>(s2, av.v[n], cl, v);
        acc[0] += abs2<T>(u);
      }
  }
};

// Per-warp geometry inside one right-hand side.  With band = 1 (grids of at
// least 7 rows) the interior set is every strip over rows [3, ny-2) in chunks
// of ch rows: strips [e_lo, e_hi), whose loaded columns hold no boundary
// column, take the branch-free stencil; the others (the edge strips) take it
// too and replace it by the boundary row of Op0::apply5 on columns 0 and nx
// and by zero off the grid (lane-constant choices: their rows are interior).
// The boundary set is the 3-row bands at the top (rows 0..2) and bottom (rows
// ny-2..ny) of every strip.  With band = 0 every warp is a boundary warp, in
// chunks of chb rows from row 0.
struct MGeo {
  int nstrips, ny, band, ch, chb;
  int e_lo, e_hi;   // strips of the interior set without a boundary column
  int nci;          // chunks per strip over rows [3, ny-2)
  int ni, nb;       // warps of the interior strips and of the 3-row bands (or of the whole grid)
  // strip and rows [j0, j1) of warp w of the set
  // interior strips [e_lo, e_hi), the edge strips outside that range, each
  // over rows [3, ny-2) in chunks of ch rows
  __host__ __device__ __forceinline__ int ne() const { return (nstrips - (e_hi - e_lo)) * nci; }
  template <int MD> __host__ __device__ __forceinline__ void map(int w, int& strip, int& j0, int& j1) const {
    if (MD != 0) {
      const int nse = nstrips - (e_hi - e_lo), nsm = MD == 1 ? e_hi - e_lo : nse;
      const int sidx = w % nsm;
      strip = MD == 1 ? e_lo + sidx : (sidx < e_lo ? sidx : e_hi + (sidx - e_lo));
      j0 = 3 + (w / nsm) * ch;
      j1 = j0 + ch < ny - 2 ? j0 + ch : ny - 2;
      return;
    }
    if (!band) {
      strip = w % nstrips;
      j0 = (w / nstrips) * chb;
      j1 = j0 + chb < ny + 1 ? j0 + chb : ny + 1;
      return;
    }
    strip = w % nstrips;
    j0 = w < nstrips ? 0 : ny - 2;
    j1 = j0 + 3;
  }
  // first reduction record of a mode's warps: interior, then edge, then the rest
  template <int MD> __host__ __device__ __forceinline__ int rec0() const {
    return MD == 1 ? 0 : (MD == 2 ? ni : ni + ne());
  }
  __host__ __device__ __forceinline__ int nrec() const { return ni + ne() + nb; }
};

template <class T> __host__ __device__ constexpr int strip_w() { return 32 * MNP<T>::NP - 4; }

// Arguments of the march kernels for one problem (the flattened launches of a
// ragged batch carry one per problem).
template <class T> struct GmA {
  Grid g;
  MGeo mg;
  Op0<T> op;
  const cx<T>* x;
  const cx<T>* b;
  cx<T>* u0;
  cx<T>* u1;
  cx<T>* u2;
  double* st;
  double* partial;
  unsigned* tickets;
  const int* active;
};

// Common prologue (one warp per block).  i: first node of this lane; outl:
// the lane's nodes are in the strip's output columns.
#define MPRO                                                                  \
  constexpr int NP = MNP<T>::NP;                                              \
  const int rhs = blockIdx.z;                                                 \
  if (active && !active[rhs]) return;                                         \
  const long long off = (long long)rhs * g.vstride;                           \
  const int lane = threadIdx.x & 31;                                          \
  int strip, j0, j1;                                                          \
  mg.template map<MM<MD>>(blockIdx.x, strip, j0, j1);                         \
  const int cs = strip * strip_w<T>() - 2;                                    \
  const int i = cs + NP * lane;                                               \
  const bool outl = NP * lane >= 2 && NP * lane + NP <= 32 * NP - 2;          \
  T* S = gstate<T>(st, rhs);                                                  \
  const MCtx<T, MD> ctx{op, g, i, j0, j1, outl};

// Runs pass P on the warp's strip and chunk (rows j0-2 .. t1 read) and
// returns its sums in acc.  stg: the warp's staging area, [NF][NS slots][32
// lanes] of 16 bytes, free again (every copy landed, the warp converged) on
// return.
template <template <class, int> class P, class T, int MD, int NV, class Init>
__device__ __forceinline__ void run_pass(const MCtx<T, MD>& c, int t1, const void* stg, T (&acc)[NV], Init&& init) {
  P<T, MD> p;
  p.m.c = c;
  p.m.sbase = (uint32_t)__cvta_generic_to_shared(stg) + (threadIdx.x & 31) * 16;
  p.m.t1 = t1;
  init(p);
#pragma unroll
  for (int k = 0; k < NV; ++k) p.acc[k] = T(0);
  p.m.prime(c.j0 - 2);
  march(p, c.j0 - 2, t1);
  asm volatile("cp.async.wait_all;\n" ::: "memory");
  __syncwarp();
#pragma unroll
  for (int k = 0; k < NV; ++k) acc[k] = p.acc[k];
}

// The interior and boundary launches of a pass may run one after the other
// or side by side: every block publishes its sums (interior blocks in
// records 0 .. ni-1, boundary blocks after them) and takes a ticket counted
// over both launches; the block holding the last ticket sums all records in
// record order and runs the scalar step F.
// blk: the block's index inside its own launch (the body's blockIdx.x).
template <int MD, int NV, class T, class F>
__device__ __forceinline__ void finish(const T (&acc)[NV], double* sh, double* partial, unsigned* tickets, int rhs,
                                       int blk, const MGeo& mg, T* S, F f) {
  double v[NV];
  const int nrec = mg.nrec();
  if (reduce_last_at<NV, T>(acc, v, sh, partial, tickets, rhs, nrec, blk, mg.template rec0<MM<MD>>(), nrec))
    staged<T>(S, v, f);
}

// M0: u0 = b - A x; |u0|^2 and <u0, A u0>.
template <class T, int MD>
__device__ __forceinline__ void gm_init_body(uint3 vblk, Grid g, MGeo mg, Op0<T, MA2<MD>> op, const cx<T>* __restrict__ x,
                                              const cx<T>* __restrict__ b, cx<T>* __restrict__ u0, double* st,
                                              double* partial, unsigned* tickets, const int* __restrict__ active) {
  const uint3 blockIdx = vblk;   // the block index inside this problem's launch
  MPRO
  T acc[3];
  __shared__ __align__(16) unsigned char stg[ring_bytes<2>()];
  double* sh = reinterpret_cast<double*>(stg);
  run_pass<P0>(ctx, j1 + 1, stg, acc, [&](auto& p) {
    p.m.src[0] = x + off;
    p.m.src[1] = b + off;
    p.us = u0 + off;
  });
  finish<MD>(acc, sh, partial, tickets, rhs, (int)blockIdx.x, mg, S, [](auto* s, const double* q) {
    fin_init<T>(s, q);
    if (s[G_BRK] == 0) {   // <u0, w> with w = s0 A u0
      const double d[2] = {q[1] * s[G_S], q[2] * s[G_S]};
      fin_a<0, T>(s, d);
    }
  });
}

template <class T, int MD>
__global__ void __launch_bounds__(32) gm_init(Grid g, MGeo mg, Op0<T, MA2<MD>> op, const cx<T>* __restrict__ x,
                                              const cx<T>* __restrict__ b, cx<T>* __restrict__ u0, double* st,
                                              double* partial, unsigned* tickets, const int* __restrict__ active) {
  gm_init_body<T, MD>(blockIdx, g, mg, op, x, b, u0, st, partial, tickets, active);
}

template <class T, int MD>
__global__ void __launch_bounds__(32) gm_init_rag(const __grid_constant__ RagLaunch<GmA<T>> L) {
  uint3 vb;
  dim3 vg;
  const GmA<T>& a = L.a[rag_problem(L, blockIdx.x, vb, vg)];
  gm_init_body<T, MD>(vb, a.g, a.mg, a.op, a.x, a.b, a.u0, a.st, a.partial, a.tickets, a.active);
}

// M0 on a zero x: u0 = b (the caller passes b as u0 to the later passes).
template <class T, int MD>
__global__ void __launch_bounds__(32) gm_init_zero(Grid g, MGeo mg, Op0<T, MA2<MD>> op, const cx<T>* __restrict__ b,
                                                   double* st, double* partial, unsigned* tickets,
                                                   const int* __restrict__ active) {
  MPRO
  T acc[3];
  __shared__ __align__(16) unsigned char stg[ring_bytes<1>()];
  double* sh = reinterpret_cast<double*>(stg);
  run_pass<P0Z>(ctx, j1 + 1, stg, acc, [&](auto& p) { p.m.src[0] = b + off; });
  finish<MD>(acc, sh, partial, tickets, rhs, (int)blockIdx.x, mg, S, [](auto* s, const double* q) {
    fin_init<T>(s, q);
    if (s[G_BRK] == 0) {
      const double d[2] = {q[1] * s[G_S], q[2] * s[G_S]};
      fin_a<0, T>(s, d);
    }
  });
}

// M1: u1 = s0 A u0 - c00 u0; |u1|^2, <u1, u0>, then <u0, A u1>, <u1, A u1>.
template <class T, int MD>
__device__ __forceinline__ void gm_step1_body(uint3 vblk, Grid g, MGeo mg, Op0<T, MA2<MD>> op, const cx<T>* __restrict__ u0,
                                               cx<T>* __restrict__ u1, double* st, double* partial,
                                               unsigned* tickets, const int* __restrict__ active) {
  const uint3 blockIdx = vblk;   // the block index inside this problem's launch
  MPRO
  if (S[G_BRK] != 0) return;   // uniform per RHS
  const T s0 = (T)S[G_S];
  const cx<T> c0 = mk<T>((T)(S[G_H] * S[G_S]), (T)(S[G_H + 1] * S[G_S]));
  T acc[7];
  __shared__ __align__(16) unsigned char stg[ring_bytes<1>()];
  double* sh = reinterpret_cast<double*>(stg);
  run_pass<P1>(ctx, j1 + 1, stg, acc, [&](auto& p) {
    p.m.src[0] = u0 + off;
    p.ws = u1 + off;
    p.s0 = s0;
    p.c0 = c0;
  });
  finish<MD>(acc, sh, partial, tickets, rhs, (int)blockIdx.x, mg, S, [](auto* s, const double* q) {
    fin_b<0, T>(s, q);
    if (s[G_BRK] == 0) {
      const double s1 = s[G_S + 1];
      const double d[4] = {q[3] * s1, q[4] * s1, q[5] * s1, q[6] * s1};
      fin_a<1, T>(s, d);
    }
  });
}

template <class T, int MD>
__global__ void __launch_bounds__(32) gm_step1(Grid g, MGeo mg, Op0<T, MA2<MD>> op, const cx<T>* __restrict__ u0,
                                               cx<T>* __restrict__ u1, double* st, double* partial,
                                               unsigned* tickets, const int* __restrict__ active) {
  gm_step1_body<T, MD>(blockIdx, g, mg, op, u0, u1, st, partial, tickets, active);
}

template <class T, int MD>
__global__ void __launch_bounds__(32) gm_step1_rag(const __grid_constant__ RagLaunch<GmA<T>> L) {
  uint3 vb;
  dim3 vg;
  const GmA<T>& a = L.a[rag_problem(L, blockIdx.x, vb, vg)];
  gm_step1_body<T, MD>(vb, a.g, a.mg, a.op, a.u0, a.u1, a.st, a.partial, a.tickets, a.active);
}

// M2: u2 = s1 A u1 - c01 u0 - c11 u1; |u2|^2, <u2, u0>, <u2, u1>, then
// <u_l, A u2> for l = 0, 1, 2.
template <class T, int MD>
__device__ __forceinline__ void gm_step2_body(uint3 vblk, Grid g, MGeo mg, Op0<T, MA2<MD>> op, const cx<T>* __restrict__ u0,
                                               const cx<T>* __restrict__ u1, cx<T>* __restrict__ u2, double* st,
                                               double* partial, unsigned* tickets, const int* __restrict__ active) {
  const uint3 blockIdx = vblk;   // the block index inside this problem's launch
  MPRO
  if (S[G_BRK] != 0 || S[G_M] < 1) return;
  const T s1 = (T)S[G_S + 1];
  const cx<T> c0 = mk<T>((T)(S[G_H + 2 * 1] * S[G_S]), (T)(S[G_H + 2 * 1 + 1] * S[G_S]));
  const cx<T> c1 = mk<T>((T)(S[G_H + 2 * 4] * S[G_S + 1]), (T)(S[G_H + 2 * 4 + 1] * S[G_S + 1]));
  T acc[NV2<T>];
  __shared__ __align__(16) unsigned char stg[ring_bytes<2>()];
  double* sh = reinterpret_cast<double*>(stg);
  run_pass<P2>(ctx, j1 + 1, stg, acc, [&](auto& p) {
    p.m.src[0] = u1 + off;
    p.m.src[1] = u0 + off;
    p.ws = u2 + off;
    p.s1 = s1;
    p.c0 = c0;
    p.c1 = c1;
  });
  finish<MD>(acc, sh, partial, tickets, rhs, (int)blockIdx.x, mg, S, [](auto* s, const double* q) {
    fin_b<1, T>(s, q);
    if (s[G_BRK] == 0) {
      const double s2 = s[G_S + 2];
      const double d[6] = {q[5] * s2, q[6] * s2, q[7] * s2, q[8] * s2, q[9] * s2, q[10] * s2};
      fin_a<2, T>(s, d);
      if constexpr (G3<T>) fin_b2_gram<T>(s, q[11] * s2 * s2);
    }
  });
}

template <class T, int MD>
__global__ void __launch_bounds__(32) gm_step2(Grid g, MGeo mg, Op0<T, MA2<MD>> op, const cx<T>* __restrict__ u0,
                                               const cx<T>* __restrict__ u1, cx<T>* __restrict__ u2, double* st,
                                               double* partial, unsigned* tickets, const int* __restrict__ active) {
  gm_step2_body<T, MD>(blockIdx, g, mg, op, u0, u1, u2, st, partial, tickets, active);
}

template <class T, int MD>
__global__ void __launch_bounds__(32) gm_step2_rag(const __grid_constant__ RagLaunch<GmA<T>> L) {
  uint3 vb;
  dim3 vg;
  const GmA<T>& a = L.a[rag_problem(L, blockIdx.x, vb, vg)];
  gm_step2_body<T, MD>(vb, a.g, a.mg, a.op, a.u0, a.u1, a.u2, a.st, a.partial, a.tickets, a.active);
}

// M3: |u3|^2 with u3 = s2 A u2 - sum_l c_l2 u_l; then the least-squares
// solve (fin_b<2>).
template <class T, int MD>
__device__ __forceinline__ void gm_step3_body(uint3 vblk, Grid g, MGeo mg, Op0<T, MA2<MD>> op, const cx<T>* __restrict__ u0,
                                               const cx<T>* __restrict__ u1, const cx<T>* __restrict__ u2,
                                               double* st, double* partial, unsigned* tickets,
                                               const int* __restrict__ active) {
  const uint3 blockIdx = vblk;   // the block index inside this problem's launch
  MPRO
  if (S[G_BRK] != 0 || S[G_M] < 2) return;
  const T s2 = (T)S[G_S + 2];
  cx<T> cl[3];
#pragma unroll
  for (int l = 0; l < 3; ++l)
    cl[l] = mk<T>((T)(S[G_H + 2 * (l * 3 + 2)] * S[G_S + l]), (T)(S[G_H + 2 * (l * 3 + 2) + 1] * S[G_S + l]));
  T acc[1];
  __shared__ __align__(16) unsigned char stg[ring_bytes<3>()];
  double* sh = reinterpret_cast<double*>(stg);
  run_pass<P3>(ctx, j1, stg, acc, [&](auto& p) {
    p.m.src[0] = u2 + off;
    p.m.src[1] = u0 + off;
    p.m.src[2] = u1 + off;
    p.s2 = s2;
    p.cl[0] = cl[0];
    p.cl[1] = cl[1];
    p.cl[2] = cl[2];
  });
  finish<MD>(acc, sh, partial, tickets, rhs, (int)blockIdx.x, mg, S, [](auto* s, const double* q) { fin_b<2, T>(s, q); });
}

template <class T, int MD>
__global__ void __launch_bounds__(32) gm_step3(Grid g, MGeo mg, Op0<T, MA2<MD>> op, const cx<T>* __restrict__ u0,
                                               const cx<T>* __restrict__ u1, const cx<T>* __restrict__ u2,
                                               double* st, double* partial, unsigned* tickets,
                                               const int* __restrict__ active) {
  gm_step3_body<T, MD>(blockIdx, g, mg, op, u0, u1, u2, st, partial, tickets, active);
}

template <class T, int MD>
__global__ void __launch_bounds__(32) gm_step3_rag(const __grid_constant__ RagLaunch<GmA<T>> L) {
  uint3 vb;
  dim3 vg;
  const GmA<T>& a = L.a[rag_problem(L, blockIdx.x, vb, vg)];
  gm_step3_body<T, MD>(vb, a.g, a.mg, a.op, a.u0, a.u1, a.u2, a.st, a.partial, a.tickets, a.active);
}

// Interior chunks are tall (few halo rows) unless the grid has too few
// strips to give every SM several warps.  Interior strips: loaded columns in
// 1..nx-1.
template <class T> MGeo march_geo(const Grid& g, int B) {
  constexpr int NP = MNP<T>::NP, SW = strip_w<T>();
  MGeo m;
  m.nstrips = cdiv(g.nx + 1, SW);
  m.ny = g.ny;
  m.band = g.ny >= 6;
  m.chb = 16;
  m.e_lo = m.e_hi = 0;
  for (int s = 0; s < m.nstrips; ++s) {
    const int cs = s * SW - 2;
    if (cs >= 1 && cs + 32 * NP - 1 <= g.nx - 1) {
      if (m.e_hi == 0) m.e_lo = s;
      m.e_hi = s + 1;
    }
  }
  const int inner_rows = g.ny - 5;
  const long long want = 152LL * 48;   // warps to fill the GPU a few times over
  int ch = 64;
  while (ch > 8 && (long long)m.nstrips * cdiv(inner_rows, ch) * B < want) ch /= 2;
  m.ch = ch;
  if (m.band) {
    m.nci = cdiv(inner_rows, ch);
    m.ni = (m.e_hi - m.e_lo) * m.nci;
    m.nb = 2 * m.nstrips;
  } else {
    m.e_lo = m.e_hi = 0;
    m.nci = m.ni = 0;
    m.nb = m.nstrips * cdiv(g.ny + 1, m.chb);
  }
  return m;
}

}  // namespace

// The x update of the node-parallel smoother (kernels_gmres.cu).
template <class T> void launch_gmres_update(const Grid& g, cx<T>* x, const GmresBufs& gb, int B, const int* active,
                                            cudaStream_t s);

long long gmres_march_blocks(const Grid& g, bool fp64, int B) {
  const MGeo m = fp64 ? march_geo<double>(g, B) : march_geo<float>(g, B);
  return (long long)m.nrec();
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
  const dim3 gi(mg.ni, 1, B), ge(mg.ne(), 1, B), gbd(mg.nb, 1, B);
  // the edge-strip and band launches of each pass on the side stream, beside
  // the interior one (their few warps then overlap the interior launch)
  const bool fork = gb.side && mg.ni;
  cudaStream_t sb = fork ? gb.side : s;
  auto pass = [&](auto interior, auto edge, auto bands) {
    if (fork) {
      cudaEventRecord(gb.ev_fork, s);
      cudaStreamWaitEvent(gb.side, gb.ev_fork, 0);
    }
    if (mg.ne()) edge();
    bands();
    if (mg.ni) interior();
    if (fork) {
      cudaEventRecord(gb.ev_join, gb.side);
      cudaStreamWaitEvent(s, gb.ev_join, 0);
    }
  };
  // the edge-strip and band launches take the boundary operator: with the
  // second-order absorbing rows its compile-time variant (modes 6 and 4)
  auto body = [&](auto opb, auto a2) {
    constexpr int ME = decltype(a2)::value ? 6 : 2, MB = decltype(a2)::value ? 4 : 0;
    for (int step = 0; step < nu; ++step) {
      // a zero x: u0 = b itself (read-only in every later pass)
      const bool z = step == 0 && gb.x_zero;
      if (z) {
        pass([&] { gm_init_zero<T, 1><<<gi, 32, 0, s>>>(g, mg, op, b, st, P, tk, active); },
             [&] { gm_init_zero<T, ME><<<ge, 32, 0, sb>>>(g, mg, opb, b, st, P, tk, active); },
             [&] { gm_init_zero<T, MB><<<gbd, 32, 0, sb>>>(g, mg, opb, b, st, P, tk, active); });
      } else {
        pass([&] { gm_init<T, 1><<<gi, 32, 0, s>>>(g, mg, op, x, b, u0, st, P, tk, active); },
             [&] { gm_init<T, ME><<<ge, 32, 0, sb>>>(g, mg, opb, x, b, u0, st, P, tk, active); },
             [&] { gm_init<T, MB><<<gbd, 32, 0, sb>>>(g, mg, opb, x, b, u0, st, P, tk, active); });
      }
      const cx<T>* v0 = z ? b : u0;
      GmresBufs gs = gb;
      gs.u[0] = (void*)v0;
      pass([&] { gm_step1<T, 1><<<gi, 32, 0, s>>>(g, mg, op, v0, u1, st, P, tk, active); },
           [&] { gm_step1<T, ME><<<ge, 32, 0, sb>>>(g, mg, opb, v0, u1, st, P, tk, active); },
           [&] { gm_step1<T, MB><<<gbd, 32, 0, sb>>>(g, mg, opb, v0, u1, st, P, tk, active); });
      pass([&] { gm_step2<T, 1><<<gi, 32, 0, s>>>(g, mg, op, v0, u1, u2, st, P, tk, active); },
           [&] { gm_step2<T, ME><<<ge, 32, 0, sb>>>(g, mg, opb, v0, u1, u2, st, P, tk, active); },
           [&] { gm_step2<T, MB><<<gbd, 32, 0, sb>>>(g, mg, opb, v0, u1, u2, st, P, tk, active); });
      if constexpr (!G3<T>) {   // complex64: u3's norm came from the Gram form in M2
        pass([&] { gm_step3<T, 1><<<gi, 32, 0, s>>>(g, mg, op, v0, u1, u2, st, P, tk, active); },
             [&] { gm_step3<T, ME><<<ge, 32, 0, sb>>>(g, mg, opb, v0, u1, u2, st, P, tk, active); },
             [&] { gm_step3<T, MB><<<gbd, 32, 0, sb>>>(g, mg, opb, v0, u1, u2, st, P, tk, active); });
      }
      if constexpr (sizeof(T) == 4) {
        if (step == nu - 1 && gb.outer) {
          launch_gmres_update_outer(g, x, gs, B, active, s);
          continue;
        }
      }
      launch_gmres_update<T>(g, x, gs, B, active, s);
    }
  };
  if (opv.c0.abc2) body(Op0<T, true>{opv.c0, opv.kf, g.nx, g.ny}, std::true_type{});
  else body(op, std::false_type{});
}

// The same smoothing steps on every problem of a ragged batch: each pass is
// one flattened launch per kind of warp (interior strips; edge strips and
// bands on the side stream), over the problems' own geometries.
template <class T>
void gmres_smooth_march_rag(const std::vector<RagLevel<T>>& v, int nu, cudaStream_t s, cudaStream_t side,
                            cudaEvent_t fork, cudaEvent_t join) {
  const int n = (int)v.size();
  std::vector<GmA<T>> A(n);
  bool any_interior = false;
  for (int q = 0; q < n; ++q) {
    const RagLevel<T>& L = v[q];
    const MGeo mg = march_geo<T>(L.g, 1);
    any_interior |= mg.ni > 0;
    A[q] = GmA<T>{L.g, mg, Op0<T>{L.op.c0, L.op.kf, L.g.nx, L.g.ny}, L.x, L.b, (cx<T>*)L.gb.u[0],
                  (cx<T>*)L.gb.u[1], (cx<T>*)L.gb.u[2], L.gb.st, L.gb.partial, L.gb.tickets, L.active};
  }
  const bool fk = side && any_interior;
  cudaStream_t sb = fk ? side : s;
  auto launch = [&](auto kern, int md, cudaStream_t st) {
    rag_launch<GmA<T>>(n, kern, dim3(32), 0, st, [&](int q, GmA<T>& a, int& gx, int&) {
      a = A[q];
      gx = md == 1 ? a.mg.ni : (md == 2 ? a.mg.ne() : a.mg.nb);
      return true;
    });
  };
  auto pass = [&](auto ki, auto ke, auto kb) {
    if (fk) {
      cudaEventRecord(fork, s);
      cudaStreamWaitEvent(side, fork, 0);
    }
    launch(ke, 2, sb);
    launch(kb, 0, sb);
    launch(ki, 1, s);
    if (fk) {
      cudaEventRecord(join, side);
      cudaStreamWaitEvent(s, join, 0);
    }
  };
  for (int step = 0; step < nu; ++step) {
    pass(gm_init_rag<T, 1>, gm_init_rag<T, 2>, gm_init_rag<T, 0>);
    pass(gm_step1_rag<T, 1>, gm_step1_rag<T, 2>, gm_step1_rag<T, 0>);
    pass(gm_step2_rag<T, 1>, gm_step2_rag<T, 2>, gm_step2_rag<T, 0>);
    if constexpr (!G3<T>) pass(gm_step3_rag<T, 1>, gm_step3_rag<T, 2>, gm_step3_rag<T, 0>);
    launch_gmres_update_rag<T>(v, s);
  }
}

template void gmres_smooth_march_rag<double>(const std::vector<RagLevel<double>>&, int, cudaStream_t, cudaStream_t,
                                             cudaEvent_t, cudaEvent_t);
template void gmres_smooth_march_rag<float>(const std::vector<RagLevel<float>>&, int, cudaStream_t, cudaStream_t,
                                            cudaEvent_t, cudaEvent_t);
template void gmres_smooth_march<double>(const Grid&, const OpView<double>&, double2*, const double2*, int, int,
                                         const int*, const GmresBufs&, cudaStream_t);
template void gmres_smooth_march<float>(const Grid&, const OpView<float>&, float2*, const float2*, int, int,
                                        const int*, const GmresBufs&, cudaStream_t);

}  // namespace hmg
