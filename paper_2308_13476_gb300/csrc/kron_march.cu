// GMRES(3) kernels that apply A on the constant-k coarse levels (Kronecker
// form A = W_y (x) G_x + H_y (x) W_x, radius R = 2 or 3), as column marches.
//
// OpK::apply evaluates, for every output node, the 2R+1 row sums
// s1 = G_x v and s2 = W_x v of the rows around it and then combines them
// along y: about 6 (2R+1)^2 FMAs per node, which makes these levels
// arithmetic-bound.  Here a thread owns one column and walks down a chunk of
// rows: each row's two sums are formed once, kept in a ring of 2R+1 rows in
// registers, and combined for the output row R behind.  The sums and the
// combination run in the same order as OpK::apply, so A v is the same value;
// the work drops to about 12 (2R+1) FMAs per node and the kernels become
// bandwidth-bound.  Outputs, reductions and scalar steps are those of
// g_init and g_arn_a (kernels_gmres.cu); g_arn_b and g_update, which do not
// apply A, are shared.
#include <algorithm>
#include <type_traits>

#include "gmres.cuh"
#include "internal.h"
#include "ragged.cuh"
#include "ragged_api.h"

namespace hmg {

namespace {

constexpr int KW = 4;   // warps per block; a warp covers 32 columns of one chunk of rows

struct KGeo {
  int ncw;      // 32-column groups
  int ch;       // rows per chunk
  int nchunks;
};

// Arguments of the column marches for one problem (the flattened launches of a
// ragged batch carry one per problem); each kernel reads the fields it takes.
template <class T, int R> struct KmA {
  Grid g;
  KGeo kg;
  OpK<T, R> op;
  const cx<T>* x;
  const cx<T>* b;
  cx<T>* u0;
  cx<T>* u1;
  cx<T>* u2;
  cx<T>* w;
  const cx<T>* win;
  cx<T>* uJ;
  cx<T>* wout;
  double* st;
  double* partial;
  unsigned* tickets;
  const int* active;
};

template <int P, int K, class F> __device__ __forceinline__ void kmarch_phases(int r, int last, F& f) {
  if constexpr (P < K) {
    if (r + P > last) return;
    f(std::integral_constant<int, P>{}, r + P);
    kmarch_phases<P + 1, K>(r, last, f);
  }
}
// Runs f(phase, r) for r = r0 .. last, phase = (r - r0) mod K as an
// std::integral_constant.
template <int K, class F> __device__ __forceinline__ void kmarch(int r0, int last, F&& f) {
#pragma unroll 1
  for (int r = r0; r <= last; r += K) kmarch_phases<0, K>(r, last, f);
}

// Whether the march over a radius-R level is unrolled so that its register
// ring never moves (KU = 2R+1 phases), or keeps one phase and shifts the ring
// by a row per step (KU = 1).  complex64 unrolls both radii (with the y
// coefficients of the interior rows in the parameter bank the radius-3
// passes stay within their launch bounds); the complex128 radius-3 marches
// would spill unrolled and keep the shifting ring.
template <class T, int R> constexpr int KU = (R == 2 || sizeof(T) == 4) ? 2 * R + 1 : 1;

// A v down column i: the input rows arrive in order through a per-warp
// shared-memory ring (each row's 32 + 2RA columns around the warp's columns,
// RA >= R, copied by cp.async KD rows ahead of use, so the 2R+1 neighbours of a lane
// are read from shared memory instead of being loaded from L2 2R+1 times);
// advance<P>() forms the two row sums of the lane's column and puts them in
// slot P of the register ring of the last 2R+1 rows, and combine<P>() returns
// (A v)(i, m) once that ring holds rows m-R..m+R.  With R = 2 the march over
// rows is unrolled by 2R+1 (kmarch, KU), so that row r sits in the
// compile-time slot P = (r - r0) mod (2R+1) and the ring never moves; with
// R = 3 the ring shifts by one row per step.
constexpr int KD = 4;    // rows in flight ahead of use
constexpr int KSL = 8;   // ring slots (a power of two > KD)

// Staged columns left (and right) of a warp's 32: R, rounded up to even for
// complex64 so that a staged row starts on a 16-byte boundary (the warp's
// first column is a multiple of 32, the row pitch a multiple of 4).
template <class T, int R> constexpr int kron_ra() { return sizeof(T) == 4 ? (R + 1) & ~1 : R; }

// Copy row r's staged columns cw0 - RA .. cw0 + 31 + RA of vs into dst.
// complex64: one 16-byte copy of a column pair per lane, for the first
// 16 + RA lanes; a pair that starts at column nx takes the zero halo column
// nx + 1 with it, a pair right of it is zero-filled.  complex128: one
// 16-byte element per copy.  The padded layout covers the columns left of
// the grid and the rows past either edge.
template <class T, int RA>
__device__ __forceinline__ void stage_kron_row(cx<T>* dst, const cx<T>* vs, const Grid& g, int cw0, int lane,
                                               int r) {
  constexpr int WD = 32 + 2 * RA;
  if constexpr (sizeof(cx<T>) == 8) {
    if (lane < WD / 2) {
      const int col = cw0 - RA + 2 * lane;
      const bool ok = col <= g.nx;
      const cx<T>* src = vs + g.at(ok ? col : 0, r);
      const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst + 2 * lane);
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src), "r"(ok ? 16 : 0) : "memory");
    }
  } else {
#pragma unroll
    for (int e = lane; e < WD; e += 32) {
      const int col = cw0 - RA + e;
      const bool ok = col <= g.nx;
      const cx<T>* src = vs + g.at(ok ? col : 0, r);
      const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst + e);
      asm volatile("cp.async.ca.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src), "r"(ok ? 16 : 0) : "memory");
    }
  }
}

// Copy row r's own 32 columns cw0 .. cw0 + 31 of vs into dst (no halo): a
// vector read only at the lane's own node, staged with the applied one so
// that its loads are in flight KD rows ahead too.
template <class T>
__device__ __forceinline__ void stage_own_row(cx<T>* dst, const cx<T>* vs, const Grid& g, int cw0, int lane, int r) {
  if constexpr (sizeof(cx<T>) == 8) {
    if (lane < 16) {
      const int col = cw0 + 2 * lane;
      const bool ok = col <= g.nx;
      const cx<T>* src = vs + g.at(ok ? col : 0, r);
      const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst + 2 * lane);
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src), "r"(ok ? 16 : 0) : "memory");
    }
  } else {
    const int col = cw0 + lane;
    const bool ok = col <= g.nx;
    const cx<T>* src = vs + g.at(ok ? col : 0, r);
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst + lane);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src), "r"(ok ? 16 : 0) : "memory");
  }
}

// combination along y for output row m = r - R, r the row just taken in
// slot P of a ring of the last K = 2R+1 row sums: row m + dy sits in slot
// (P + 1 + R + dy) mod K, or in slot dy + R of a shifting ring (KU = 1).
// Rows whose y-factors are the translation-invariant interior ones take the
// coefficients from the operator's parameter-bank copy (the same values);
// the others load their row's coefficients.
template <class T, int R, int K, int KUR, int P>
__device__ __forceinline__ cx<T> kcombine(const OpK<T, R>& op, int m, const cx<T> (&s1)[K], const cx<T> (&s2)[K]) {
  cx<T> acc = mk<T>(T(0), T(0));
  if (m >= op.ty0 && m < op.ty1) {
    if constexpr (sizeof(T) == 4 && R == 2) {   // packed: Re h and w_y with s, Im h apart, joined once
      float2 pr = make_float2(0.f, 0.f), pi = make_float2(0.f, 0.f);
#pragma unroll
      for (int dy = -R; dy <= R; ++dy) {
        const int q = KUR == 1 ? dy + R : (P + 1 + R + dy) % K;
        pr = fma2(op.pk.wyb[dy + R], s1[q], pr);
        pr = fma2(op.pk.hyr[dy + R], s2[q], pr);
        pi = fma2(op.pk.hyi[dy + R], s2[q], pi);
      }
      return make_float2(pr.x - pi.y, pr.y + pi.x);
    }
#pragma unroll
    for (int dy = -R; dy <= R; ++dy) {
      const int q = KUR == 1 ? dy + R : (P + 1 + R + dy) % K;
      const T wy = op.wyc[dy + R];
      acc = mk<T>(fma(wy, s1[q].x, acc.x), fma(wy, s1[q].y, acc.y));
      acc = fma_c<T>(op.hyc[dy + R], s2[q], acc);
    }
    return acc;
  }
  const cx<T>* H = op.hy + m * K;
  const T* Wy = op.wy + m * K;
#pragma unroll
  for (int dy = -R; dy <= R; ++dy) {
    const int q = KUR == 1 ? dy + R : (P + 1 + R + dy) % K;
    const T wy = __ldg(Wy + dy + R);
    acc = mk<T>(fma(wy, s1[q].x, acc.x), fma(wy, s1[q].y, acc.y));
    acc = fma_c<T>(__ldg(H + dy + R), s2[q], acc);
  }
  return acc;
}

template <class T, int R> struct KRing {
  static constexpr int K = 2 * R + 1;
  static constexpr int RA = kron_ra<T, R>();
  static constexpr int WD = 32 + 2 * RA;   // staged row width
  cx<T> G[K];
  T Wx[K];
  cx<T> s1[K], s2[K];
  const cx<T>* vs;   // slice of the applied vector
  Grid g;
  int cw0, lane;     // the warp's first column, the lane
  cx<T>* sm;         // the warp's ring, [KSL][WD]
  int r0;            // first row of the march (slot 0)
  const cx<T>* os = nullptr;   // optional vector read at the lane's own nodes (no halo)
  cx<T>* osm = nullptr;        // its ring, [KSL][32]

  __device__ __forceinline__ void init(const OpK<T, R>& op, int i, bool col) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      G[k] = col ? op.gx[i * K + k] : mk<T>(T(0), T(0));
      Wx[k] = col ? op.wx[i * K + k] : T(0);
      s1[k] = mk<T>(T(0), T(0));
      s2[k] = mk<T>(T(0), T(0));
    }
  }
  // copy row r's staged columns into its slot
  __device__ __forceinline__ void issue(int r) {
    stage_kron_row<T, RA>(sm + ((r - r0) & (KSL - 1)) * WD, vs, g, cw0, lane, r);
    if (os) stage_own_row<T>(osm + ((r - r0) & (KSL - 1)) * 32, os, g, cw0, lane, r);
  }
  // the applied vector and the own-node vector at row m (m >= r - KSL + KD,
  // r the row last taken: the slot is not yet reused), the lane's column
  __device__ __forceinline__ cx<T> staged_at(int m) const { return sm[((m - r0) & (KSL - 1)) * WD + lane + RA]; }
  __device__ __forceinline__ cx<T> own_at(int m) const { return osm[((m - r0) & (KSL - 1)) * 32 + lane]; }
  __device__ __forceinline__ static void commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
  // rows r0 .. r0 + KD - 1 in flight
  __device__ __forceinline__ void prime(int last) {
#pragma unroll
    for (int d = 0; d < KD; ++d) {
      if (r0 + d <= last) issue(r0 + d);
      commit();
    }
  }
  // take input row r (rows up to `last` exist): row r + KD in flight, row r's
  // sums into the register ring.  All lanes of the warp call it.
  template <int P> __device__ __forceinline__ void advance(int r, int last) {
    __syncwarp();   // every lane is done with the slot row r + KD reuses
    if (r + KD <= last) issue(r + KD);
    commit();
    asm volatile("cp.async.wait_group %0;\n" ::"n"(KD) : "memory");
    __syncwarp();   // row r, copied by all lanes, is visible to all
    const cx<T>* row = sm + ((r - r0) & (KSL - 1)) * WD + lane + RA;
    cx<T> a = mk<T>(T(0), T(0)), c = mk<T>(T(0), T(0));
#pragma unroll
    for (int dx = -R; dx <= R; ++dx) {
      const cx<T> xv = row[dx];
      a = fma_c<T>(G[dx + R], xv, a);
      c = mk<T>(fma(Wx[dx + R], xv.x, c.x), fma(Wx[dx + R], xv.y, c.y));
    }
    if constexpr (KU<T, R> == 1) {
#pragma unroll
      for (int k = 0; k < K - 1; ++k) {
        s1[k] = s1[k + 1];
        s2[k] = s2[k + 1];
      }
    }
    s1[KU<T, R> == 1 ? K - 1 : P] = a;
    s2[KU<T, R> == 1 ? K - 1 : P] = c;
  }
  // combination along y for output row m = r - R, r the row just taken in
  // slot P: row m + dy sits in slot (P + 1 + R + dy) mod K, or in slot dy + R
  // of the shifting ring (KU = 1)
  template <int P> __device__ __forceinline__ cx<T> combine(const OpK<T, R>& op, int m) const {
    return kcombine<T, R, K, KU<T, R>, P>(op, m, s1, s2);
  }
};

// Common prologue.  A warp owns 32 columns of one chunk of rows; `has`: the
// warp has work; `col`: the lane's column is inside the grid.
#define KPRO                                                                  \
  __shared__ double sh[NVMAX * 32];                                           \
  __shared__ __align__(16) cx<T> ksm[KW][KSL][KRing<T, R>::WD];              \
  const int rhs = blockIdx.z;                                                 \
  if (active && !active[rhs]) return;                                         \
  const long long off = (long long)rhs * g.vstride;                           \
  const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;                  \
  const int gw = blockIdx.x * KW + wib;                                       \
  const bool has = gw < kg.ncw * kg.nchunks;                                  \
  const int cw0 = (has ? gw % kg.ncw : 0) * 32, i = cw0 + lane;               \
  const int j0 = (has ? gw / kg.ncw : 0) * kg.ch, j1 = min(j0 + kg.ch, g.ny + 1); \
  const bool col = has && i <= g.nx;                                          \
  const int nblk = gridDim.x, blk = blockIdx.x;

#define KMARCH_SETUP(vsrc)                                                    \
  KRing<T, R> ring;                                                           \
  ring.init(op, i, col);                                                      \
  ring.vs = (vsrc);                                                           \
  ring.g = g;                                                                 \
  ring.cw0 = cw0;                                                             \
  ring.lane = lane;                                                           \
  ring.sm = &ksm[wib][0][0];                                                  \
  ring.r0 = j0 - R;                                                           \
  const int last = j1 + R - 1;                                                \
  ring.prime(last);

// u0 = b - A x, partial |u0|^2 (as g_init)
// NRM = false: only u0 = b - A x (the residual before the restriction; no
// norm, no state)
template <class T, int R, bool NRM = true>
__device__ __forceinline__ void km_init_body(uint3 vblk, dim3 vgrid, Grid g, KGeo kg, OpK<T, R> op, const cx<T>* __restrict__ x, const cx<T>* __restrict__ b, cx<T>* __restrict__ u0, double* st, double* partial, unsigned* tickets, const int* __restrict__ active) {
  const uint3 blockIdx = vblk;   // the block and grid inside this problem's launch
  const dim3 gridDim = vgrid;
  (void)blockIdx;
  (void)gridDim;
  KPRO
  T a0[1] = {T(0)};
  __shared__ __align__(16) cx<T> kbsm[KW][KSL][32];   // b, staged with x
  if (has) {
    KRing<T, R> ring;
    ring.init(op, i, col);
    ring.vs = x + off;
    ring.g = g;
    ring.cw0 = cw0;
    ring.lane = lane;
    ring.sm = &ksm[wib][0][0];
    ring.r0 = j0 - R;
    ring.os = b + off;
    ring.osm = &kbsm[wib][0][0];
    const int last = j1 + R - 1;
    ring.prime(last);
    kmarch<KU<T, R>>(j0 - R, last, [&](auto ph, int r) {
      constexpr int P = decltype(ph)::value;
      ring.template advance<P>(r, last);
      const int m = r - R;
      if (m >= j0 && col) {
        const int p = g.at(i, m);
        const cx<T> res = sub<T>(ring.own_at(m), ring.template combine<P>(op, m));
        u0[off + p] = res;
        a0[0] += abs2<T>(res);
      }
    });
    asm volatile("cp.async.wait_all;\n" ::: "memory");
  }
  if constexpr (NRM) {
    double v[1];
    if (reduce_last<1, T>(a0, v, sh, partial, tickets, rhs, nblk, blk) && threadIdx.x == 0)
      fin_init<T>(gstate<T>(st, rhs), v);
  }
}

// km_init on a zero x: u0 = b (the caller passes b as u0 to the later
// passes); each lane sums |b|^2 down its column of the chunk, in km_init's
// order and over its blocks, so the state equals km_init's on a zero x.
template <class T>
__global__ void __launch_bounds__(KW * 32) km_init_zero(Grid g, KGeo kg, const cx<T>* __restrict__ b, double* st,
                                                        double* partial, unsigned* tickets,
                                                        const int* __restrict__ active) {
  __shared__ double sh[NVMAX * 32];
  const int rhs = blockIdx.z;
  if (active && !active[rhs]) return;
  const long long off = (long long)rhs * g.vstride;
  const int lane = threadIdx.x & 31;
  const int gw = blockIdx.x * KW + (threadIdx.x >> 5);
  const bool has = gw < kg.ncw * kg.nchunks;
  const int i = (has ? gw % kg.ncw : 0) * 32 + lane;
  const int j0 = (has ? gw / kg.ncw : 0) * kg.ch, j1 = min(j0 + kg.ch, g.ny + 1);
  T a0[1] = {T(0)};
  if (has && i <= g.nx) {
    const cx<T>* bs = b + off;
#pragma unroll 4
    for (int m = j0; m < j1; ++m) a0[0] += abs2<T>(bs[g.at(i, m)]);
  }
  double v[1];
  if (reduce_last<1, T>(a0, v, sh, partial, tickets, rhs, gridDim.x, blockIdx.x) && threadIdx.x == 0)
    fin_init<T>(gstate<T>(st, rhs), v);
}

template <class T, int R, bool NRM = true>
__global__ void __launch_bounds__(KW * 32) km_init(Grid g, KGeo kg, OpK<T, R> op, const cx<T>* __restrict__ x, const cx<T>* __restrict__ b, cx<T>* __restrict__ u0, double* st, double* partial, unsigned* tickets, const int* __restrict__ active) {
  km_init_body<T, R, NRM>(blockIdx, gridDim, g, kg, op, x, b, u0, st, partial, tickets, active);
}

template <class T, int R>
__global__ void __launch_bounds__(KW * 32) km_init_rag(const __grid_constant__ RagLaunch<KmA<T, R>> L) {
  uint3 vb;
  dim3 vg;
  const KmA<T, R>& a = L.a[rag_problem(L, blockIdx.x, vb, vg)];
  km_init_body<T, R>(vb, vg, a.g, a.kg, a.op, a.x, a.b, a.u0, a.st, a.partial, a.tickets, a.active);
}

// w = s_J A u_J; partial dots <u_l, w>, l <= J (as g_arn_a)
template <class T, int R, int J>
__device__ __forceinline__ void km_arn_a_body(uint3 vblk, dim3 vgrid, Grid g, KGeo kg, OpK<T, R> op, const cx<T>* __restrict__ u0, const cx<T>* __restrict__ u1, const cx<T>* __restrict__ u2, cx<T>* __restrict__ w, double* __restrict__ st, double* partial, unsigned* tickets, const int* __restrict__ active) {
  const uint3 blockIdx = vblk;   // the block and grid inside this problem's launch
  const dim3 gridDim = vgrid;
  (void)blockIdx;
  (void)gridDim;
  KPRO
  T* S = gstate<T>(st, rhs);
  if (S[G_BRK] != 0 || S[G_M] < J) return;   // uniform per RHS
  const cx<T>* uJ = J == 0 ? u0 : (J == 1 ? u1 : u2);
  T acc[2 * (J + 1)];
#pragma unroll
  for (int k = 0; k < 2 * (J + 1); ++k) acc[k] = T(0);
  if (has) {
    const T sJ = (T)S[G_S + J];
    const cx<T>* us[3] = {u0 + off, u1 + off, u2 + off};
    KMARCH_SETUP(uJ + off)
    kmarch<KU<T, R>>(j0 - R, last, [&](auto ph, int r) {
      constexpr int P = decltype(ph)::value;
      ring.template advance<P>(r, last);
      const int m = r - R;
      if (m >= j0 && col) {
        const int p = g.at(i, m);
        const cx<T> a = scl<T>(sJ, ring.template combine<P>(op, m));
        w[off + p] = a;
#pragma unroll
        for (int l = 0; l <= J; ++l) {   // u_J is the staged vector
          const cx<T> d = cmul<T>(l == J ? ring.staged_at(m) : us[l][p], a);
          acc[2 * l] += d.x;
          acc[2 * l + 1] += d.y;
        }
      }
    });
    asm volatile("cp.async.wait_all;\n" ::: "memory");
  }
  double v[2 * (J + 1)];
  if (reduce_last<2 * (J + 1), T>(acc, v, sh, partial, tickets, rhs, nblk, blk))
    staged<T>(S, v, [](auto* s, const double* q) { fin_a<J, T>(s, q); });
}

template <class T, int R, int J>
__global__ void __launch_bounds__(KW * 32) km_arn_a(Grid g, KGeo kg, OpK<T, R> op, const cx<T>* __restrict__ u0, const cx<T>* __restrict__ u1, const cx<T>* __restrict__ u2, cx<T>* __restrict__ w, double* __restrict__ st, double* partial, unsigned* tickets, const int* __restrict__ active) {
  km_arn_a_body<T, R, J>(blockIdx, gridDim, g, kg, op, u0, u1, u2, w, st, partial, tickets, active);
}

template <class T, int R, int J>
__global__ void __launch_bounds__(KW * 32) km_arn_a_rag(const __grid_constant__ RagLaunch<KmA<T, R>> L) {
  uint3 vb;
  dim3 vg;
  const KmA<T, R>& a = L.a[rag_problem(L, blockIdx.x, vb, vg)];
  km_arn_a_body<T, R, J>(vb, vg, a.g, a.kg, a.op, a.u0, a.u1, a.u2, a.w, a.st, a.partial, a.tickets, a.active);
}

// ---------------------------------------------------------------- fused passes
//
// km_arn_ab<J> (J = 1, 2) is g_arn_b<J-1> and km_arn_a<J> in one march: the
// ring stages the rows of w and u_0..u_{J-1}, each lane forms
// u_J = c_w w - sum_{l<J} (h_{l,J-1} s_l) u_l for its staged columns into a
// second ring, writes u_J on its own rows and sums |u_J|^2 and <u_J, u_l>
// there (the inputs of fin_b<J-1>), and the column march applies A to the
// formed rows: w' = A u_J, stored unscaled (s_J = 1 / |u_J| is known only
// after this kernel's reduction), with the dots <u_l, w'> of the output rows.
// The last block runs fin_b<J-1> and, unless it found a breakdown, fin_a<J>
// on the dots scaled by s_J.  w' cannot overwrite the staged w (neighbouring
// chunks read its rows as halo), so J = 1 writes w2 and J = 2 reads w2 and
// writes w; the closing g_arn_b<2> scales w by s_2.  Per smoothing step this
// saves 7 of 28 vector passes and two launches.
template <class T, int R, int NS> struct KRingF {
  static constexpr int K = 2 * R + 1;
  static constexpr int RA = kron_ra<T, R>();
  static constexpr int WD = 32 + 2 * RA;
  cx<T> G[K];
  T Wx[K];
  cx<T> s1[K], s2[K];
  const cx<T>* vs[NS];   // staged slices: w, u_0, .., u_{NS-2}
  Grid g;
  int cw0, lane;
  cx<T>* sm;             // the warp's staged rings, [NS][KSL][WD]
  cx<T>* fm;             // the warp's ring of formed rows, [KSL][WD]
  int r0;

  __device__ __forceinline__ void init(const OpK<T, R>& op, int i, bool col) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      G[k] = col ? op.gx[i * K + k] : mk<T>(T(0), T(0));
      Wx[k] = col ? op.wx[i * K + k] : T(0);
      s1[k] = mk<T>(T(0), T(0));
      s2[k] = mk<T>(T(0), T(0));
    }
  }
  __device__ __forceinline__ int slot(int r) const { return (r - r0) & (KSL - 1); }
  __device__ __forceinline__ void issue(int r) {
#pragma unroll
    for (int v = 0; v < NS; ++v) stage_kron_row<T, RA>(sm + (v * KSL + slot(r)) * WD, vs[v], g, cw0, lane, r);
  }
  __device__ __forceinline__ static void commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
  __device__ __forceinline__ void prime(int last) {
#pragma unroll
    for (int d = 0; d < KD; ++d) {
      if (r0 + d <= last) issue(r0 + d);
      commit();
    }
  }
  // take input row r: form u_J on it (returned for the lane's column), its
  // two row sums into the register ring.  All lanes of the warp call it.
  template <int P> __device__ __forceinline__ cx<T> advance(int r, int last, T cw, const cx<T> (&c)[NS - 1]) {
    __syncwarp();
    if (r + KD <= last) issue(r + KD);
    commit();
    asm volatile("cp.async.wait_group %0;\n" ::"n"(KD) : "memory");
    __syncwarp();
    const int sl = slot(r);
    if constexpr (sizeof(cx<T>) == 8) {   // a column pair per lane, 16-byte accesses
      if (lane < WD / 2) {
        const int e = 2 * lane;
        const float4 wv = *reinterpret_cast<const float4*>(sm + sl * WD + e);
        cx<T> ua[NS - 1], ub[NS - 1];
#pragma unroll
        for (int l = 0; l < NS - 1; ++l) {
          const float4 q = *reinterpret_cast<const float4*>(sm + ((1 + l) * KSL + sl) * WD + e);
          ua[l] = mk<T>(q.x, q.y);
          ub[l] = mk<T>(q.z, q.w);
        }
        cx<T> a, b;
        if constexpr (R == 2) {   // packed (the radius-3 passes keep their register budget)
          a = scl_minus<T, NS - 1>(cw, mk<T>(wv.x, wv.y), c, ua);
          b = scl_minus<T, NS - 1>(cw, mk<T>(wv.z, wv.w), c, ub);
        } else {
          a = scl<T>(cw, mk<T>(wv.x, wv.y));
          b = scl<T>(cw, mk<T>(wv.z, wv.w));
#pragma unroll
          for (int l = 0; l < NS - 1; ++l) {
            a = sub<T>(a, mul<T>(c[l], ua[l]));
            b = sub<T>(b, mul<T>(c[l], ub[l]));
          }
        }
        *reinterpret_cast<float4*>(fm + sl * WD + e) = make_float4(a.x, a.y, b.x, b.y);
      }
    } else {
#pragma unroll
      for (int e = lane; e < WD; e += 32) {
        cx<T> u = scl<T>(cw, sm[sl * WD + e]);
#pragma unroll
        for (int l = 0; l < NS - 1; ++l) u = sub<T>(u, mul<T>(c[l], sm[((1 + l) * KSL + sl) * WD + e]));
        fm[sl * WD + e] = u;
      }
    }
    __syncwarp();
    const cx<T>* row = fm + sl * WD + lane + RA;
    cx<T> a = mk<T>(T(0), T(0)), b = mk<T>(T(0), T(0));
#pragma unroll
    for (int dx = -R; dx <= R; ++dx) {
      const cx<T> xv = row[dx];
      a = fma_c<T>(G[dx + R], xv, a);
      b = mk<T>(fma(Wx[dx + R], xv.x, b.x), fma(Wx[dx + R], xv.y, b.y));
    }
    if constexpr (KU<T, R> == 1) {
#pragma unroll
      for (int k = 0; k < K - 1; ++k) {
        s1[k] = s1[k + 1];
        s2[k] = s2[k + 1];
      }
    }
    s1[KU<T, R> == 1 ? K - 1 : P] = a;
    s2[KU<T, R> == 1 ? K - 1 : P] = b;
    return row[0];
  }
  // staged vector v (1 + l for u_l) and the formed u_J at row m, lane's column
  __device__ __forceinline__ cx<T> staged(int v, int m) const { return sm[(v * KSL + slot(m)) * WD + lane + RA]; }
  __device__ __forceinline__ cx<T> formed(int m) const { return fm[slot(m) * WD + lane + RA]; }
  template <int P> __device__ __forceinline__ cx<T> combine(const OpK<T, R>& op, int m) const {
    return kcombine<T, R, K, KU<T, R>, P>(op, m, s1, s2);
  }
};

// Resident blocks per SM the register budget must allow: as many as the
// shared memory holds (six for radius 2 with J = 1, five otherwise).
template <class T, int R, int J>
__device__ __forceinline__ void km_arn_ab_body(uint3 vblk, dim3 vgrid, Grid g, KGeo kg, OpK<T, R> op, const cx<T>* __restrict__ win, const cx<T>* __restrict__ u0, const cx<T>* __restrict__ u1, cx<T>* __restrict__ uJ, cx<T>* __restrict__ wout, double* __restrict__ st, double* partial, unsigned* tickets, const int* __restrict__ active) {
  const uint3 blockIdx = vblk;   // the block and grid inside this problem's launch
  const dim3 gridDim = vgrid;
  (void)blockIdx;
  (void)gridDim;
  constexpr int NS = J + 1;             // staged: w, u_0 .. u_{J-1}
  constexpr int NB = 1 + 2 * J;         // fin_b<J-1>: |u_J|^2, <u_J, u_l> (l < J)
  constexpr int NA = 2 * (J + 1);       // fin_a<J>: <u_l, w'> (l <= J)
  // complex64, J = 2: |w'|^2 too, and u3's norm from the Gram form
  // (fin_b2_gram) instead of the closing g_arn_b<2> pass
  constexpr int NG = (sizeof(T) == 4 && J == 2) ? 1 : 0;
  __shared__ double sh[NVMAX * 32];
  __shared__ __align__(16) cx<T> ksm[KW][NS][KSL][KRingF<T, R, NS>::WD];
  __shared__ __align__(16) cx<T> kfm[KW][KSL][KRingF<T, R, NS>::WD];
  const int rhs = blockIdx.z;
  if (active && !active[rhs]) return;
  const long long off = (long long)rhs * g.vstride;
  const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int gw = blockIdx.x * KW + wib;
  const bool has = gw < kg.ncw * kg.nchunks;
  const int cw0 = (has ? gw % kg.ncw : 0) * 32, i = cw0 + lane;
  const int j0 = (has ? gw / kg.ncw : 0) * kg.ch, j1 = min(j0 + kg.ch, g.ny + 1);
  const bool col = has && i <= g.nx;
  const int nblk = gridDim.x, blk = blockIdx.x;
  T* S = gstate<T>(st, rhs);
  if (S[G_BRK] != 0 || S[G_M] < J - 1) return;   // the guard of g_arn_b<J-1>; uniform per RHS
  T acc[NB + NA + NG];
#pragma unroll
  for (int k = 0; k < NB + NA + NG; ++k) acc[k] = T(0);
  if (has) {
    // u_J = c_w w - sum_l c_l u_l: w from km_arn_a<0> carries s_0 (c_w = 1);
    // w2 from km_arn_ab<1> is unscaled (c_w = s_1)
    const T cw = J == 1 ? T(1) : (T)S[G_S + J - 1];
    cx<T> c[NS - 1];
#pragma unroll
    for (int l = 0; l < J; ++l) {
      const T sl = S[G_S + l];
      c[l] = mk<T>((T)(S[G_H + 2 * (l * 3 + J - 1)] * sl), (T)(S[G_H + 2 * (l * 3 + J - 1) + 1] * sl));
    }
    KRingF<T, R, NS> ring;
    ring.init(op, i, col);
    ring.vs[0] = win + off;
    ring.vs[1] = u0 + off;
    if (NS > 2) ring.vs[NS - 1] = u1 + off;
    ring.g = g;
    ring.cw0 = cw0;
    ring.lane = lane;
    ring.sm = &ksm[wib][0][0][0];
    ring.fm = &kfm[wib][0][0];
    ring.r0 = j0 - R;
    const int last = j1 + R - 1;
    ring.prime(last);
    kmarch<KU<T, R>>(j0 - R, last, [&](auto ph, int r) {
      constexpr int P = decltype(ph)::value;
      const cx<T> u = ring.template advance<P>(r, last, cw, c);
      if (r >= j0 && r < j1 && col) {   // own row: store u_J, the inputs of fin_b<J-1>
        uJ[off + g.at(i, r)] = u;
        acc[0] += abs2<T>(u);
#pragma unroll
        for (int l = 0; l < J; ++l) {
          const cx<T> d = cmul<T>(u, ring.staged(1 + l, r));
          acc[1 + 2 * l] += d.x;
          acc[2 + 2 * l] += d.y;
        }
      }
      const int m = r - R;
      if (m >= j0 && col) {
        const int p = g.at(i, m);
        const cx<T> a = ring.template combine<P>(op, m);
        wout[off + p] = a;
#pragma unroll
        for (int l = 0; l <= J; ++l) {
          const cx<T> ul = l < J ? ring.staged(1 + l, m) : ring.formed(m);
          const cx<T> d = cmul<T>(ul, a);
          acc[NB + 2 * l] += d.x;
          acc[NB + 2 * l + 1] += d.y;
        }
        if constexpr (NG == 1) acc[NB + NA] += abs2<T>(a);
      }
    });
    asm volatile("cp.async.wait_all;\n" ::: "memory");
  }
  double v[NB + NA + NG];
  if (reduce_last<NB + NA + NG, T>(acc, v, sh, partial, tickets, rhs, nblk, blk))
    staged<T>(S, v, [](auto* s, const double* q) {
      fin_b<J - 1, T>(s, q);
      if (s[G_BRK] == 0) {
        double d[NA];
        const double sJ = s[G_S + J];
#pragma unroll
        for (int k = 0; k < NA; ++k) d[k] = sJ * q[NB + k];
        fin_a<J, T>(s, d);
        if constexpr (NG == 1) fin_b2_gram<T>(s, q[NB + NA] * sJ * sJ);
      }
    });
}

template <class T, int R, int J>
__global__ void __launch_bounds__(KW * 32, R == 2 && J == 1 ? 6 : 5) km_arn_ab(Grid g, KGeo kg, OpK<T, R> op, const cx<T>* __restrict__ win, const cx<T>* __restrict__ u0, const cx<T>* __restrict__ u1, cx<T>* __restrict__ uJ, cx<T>* __restrict__ wout, double* __restrict__ st, double* partial, unsigned* tickets, const int* __restrict__ active) {
  km_arn_ab_body<T, R, J>(blockIdx, gridDim, g, kg, op, win, u0, u1, uJ, wout, st, partial, tickets, active);
}

template <class T, int R, int J>
__global__ void __launch_bounds__(KW * 32, R == 2 && J == 1 ? 6 : 5) km_arn_ab_rag(const __grid_constant__ RagLaunch<KmA<T, R>> L) {
  uint3 vb;
  dim3 vg;
  const KmA<T, R>& a = L.a[rag_problem(L, blockIdx.x, vb, vg)];
  km_arn_ab_body<T, R, J>(vb, vg, a.g, a.kg, a.op, a.win, a.u0, a.u1, a.uJ, a.wout, a.st, a.partial, a.tickets, a.active);
}

constexpr int KCH[] = {64, 48, 32, 24, 16, 12, 8};   // candidate rows per chunk

// Rows per chunk for a level: each warp marches ch + 2R rows, and the
// launch runs in ceil(blocks / cap) rounds of the cap blocks the GPU holds
// at once, so the chunk height minimising rounds x (ch + 2R) is taken (the
// tallest on ties).  A fixed height can leave a last round of a few blocks:
// 64-row chunks of a 513^2 level with 64 right-hand sides give 2.05 rounds.
KGeo kron_geo(const Grid& g, int B, int R, long long cap, int forced = 0) {
  KGeo k;
  k.ncw = cdiv(g.nx + 1, 32);
  if (forced > 0) {   // a fixed height (the autotuner's axis), at least the shortest candidate
    k.ch = std::max(forced, KCH[sizeof(KCH) / sizeof(KCH[0]) - 1]);
    k.nchunks = cdiv(g.ny + 1, k.ch);
    return k;
  }
  long long best = -1;
  for (int ch : KCH) {
    const long long blocks = (long long)cdiv((long long)k.ncw * cdiv(g.ny + 1, ch), KW) * B;
    const long long cost = (long long)cdiv(blocks, cap) * (ch + 2 * R);
    if (best < 0 || cost < best) {
      best = cost;
      k.ch = ch;
    }
  }
  k.nchunks = cdiv(g.ny + 1, k.ch);
  return k;
}

// The fused marches stage three vectors per row in shared memory; their
// double variants would need more static shared memory than a block may
// declare, so only the complex64 path fuses.
template <class T> constexpr bool KFUSE = sizeof(T) == 4;

// Blocks of the level's heaviest march (km_arn_ab<T, R, 2> when fused, else
// km_arn_a<T, R, 2>) resident on the device at once.
template <class T, int R> long long kron_capacity(bool fused) {
  static long long cap[2] = {0, 0};
  if (!cap[fused]) {
    int dev = 0, sms = 1, per = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if constexpr (KFUSE<T>) {
      if (fused) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, km_arn_ab<T, R, 2>, KW * 32, 0);
      else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, km_arn_a<T, R, 2>, KW * 32, 0);
    } else {
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, km_arn_a<T, R, 2>, KW * 32, 0);
    }
    cudaGetLastError();
    cap[fused] = (long long)std::max(per, 1) * std::max(sms, 1);
  }
  return cap[fused];
}

}  // namespace

template <class T> void launch_gmres_update(const Grid& g, cx<T>* x, const GmresBufs& gb, int B, const int* active,
                                            cudaStream_t s);
template <class T, int J> void launch_arn_b(const Grid& g, const GmresBufs& gb, cx<T>* un, int B, const int* active,
                                            cudaStream_t s, int ws);

long long kron_march_blocks(const Grid& g, int B) {   // the most for any chunk height: the shortest
  (void)B;
  return cdiv((long long)cdiv(g.nx + 1, 32) * cdiv(g.ny + 1, KCH[sizeof(KCH) / sizeof(KCH[0]) - 1]), KW);
}

template <class T>
void gmres_smooth_kron(const Grid& g, const OpView<T>& opv, cx<T>* x, const cx<T>* b, int nu, int B,
                       const int* active, const GmresBufs& gb, cudaStream_t s) {
  cx<T>* u0 = (cx<T>*)gb.u[0];
  cx<T>* u1 = (cx<T>*)gb.u[1];
  cx<T>* u2 = (cx<T>*)gb.u[2];
  cx<T>* w = (cx<T>*)gb.w;
  cx<T>* w2 = (cx<T>*)gb.w2;
  double* P = gb.partial;
  unsigned* tk = gb.tickets;
  double* st = gb.st;
  auto run = [&](auto op, auto rad) {
    constexpr int R = decltype(rad)::value;
    const bool fused = KFUSE<T> && w2 != nullptr;
    const KGeo kg = kron_geo(g, B, R, kron_capacity<T, R>(fused), gb.kron_ch);
    const dim3 grd(cdiv((long long)kg.ncw * kg.nchunks, KW), 1, B);
    for (int step = 0; step < nu; ++step) {
      // a zero x: u0 = b itself (read-only in every later pass)
      const bool z = step == 0 && gb.x_zero;
      const cx<T>* v0 = z ? b : u0;
      GmresBufs gs = gb;
      gs.u[0] = (void*)v0;
      if (z) km_init_zero<T><<<grd, KW * 32, 0, s>>>(g, kg, b, st, P, tk, active);
      else km_init<T, R><<<grd, KW * 32, 0, s>>>(g, kg, op, x, b, u0, st, P, tk, active);
      km_arn_a<T, R, 0><<<grd, KW * 32, 0, s>>>(g, kg, op, v0, u1, u2, w, st, P, tk, active);
      bool done = false;
      if constexpr (KFUSE<T>) {
        if (fused) {   // arn_b<0> + arn_a<1>, arn_b<1> + arn_a<2>
          km_arn_ab<T, R, 1><<<grd, KW * 32, 0, s>>>(g, kg, op, w, v0, v0, u1, w2, st, P, tk, active);
          km_arn_ab<T, R, 2><<<grd, KW * 32, 0, s>>>(g, kg, op, w2, v0, u1, u2, w, st, P, tk, active);
          done = true;   // u3's norm from the Gram form: no closing g_arn_b<2>
        }
      }
      if (!done) {
        launch_arn_b<T, 0>(g, gs, u1, B, active, s, -1);
        km_arn_a<T, R, 1><<<grd, KW * 32, 0, s>>>(g, kg, op, v0, u1, u2, w, st, P, tk, active);
        launch_arn_b<T, 1>(g, gs, u2, B, active, s, -1);
        km_arn_a<T, R, 2><<<grd, KW * 32, 0, s>>>(g, kg, op, v0, u1, u2, w, st, P, tk, active);
        launch_arn_b<T, 2>(g, gs, nullptr, B, active, s, -1);
      }
      launch_gmres_update<T>(g, x, gs, B, active, s);
    }
  };
  if (opv.kind == 4) run(kron_op<T, 2>(opv, g.nx, g.ny), std::integral_constant<int, 2>{});
  else run(kron_op<T, 3>(opv, g.nx, g.ny), std::integral_constant<int, 3>{});
}

template <class T>
void launch_kron_residual(const Grid& g, const OpView<T>& opv, const cx<T>* x, const cx<T>* b, cx<T>* r, int B,
                          const int* active, int kron_ch, cudaStream_t s) {
  auto run = [&](auto op, auto rad) {
    constexpr int R = decltype(rad)::value;
    const KGeo kg = kron_geo(g, B, R, kron_capacity<T, R>(KFUSE<T>), kron_ch);
    const dim3 grd(cdiv((long long)kg.ncw * kg.nchunks, KW), 1, B);
    km_init<T, R, false><<<grd, KW * 32, 0, s>>>(g, kg, op, x, b, r, nullptr, nullptr, nullptr, active);
  };
  if (opv.kind == 4) run(kron_op<T, 2>(opv, g.nx, g.ny), std::integral_constant<int, 2>{});
  else run(kron_op<T, 3>(opv, g.nx, g.ny), std::integral_constant<int, 3>{});
}

// The same smoothing steps on every problem of a ragged batch (the problems'
// levels at the same depth share the radius): each kernel of a step is one
// flattened launch over the problems' own chunk geometries.
template <class T>
void gmres_smooth_kron_rag(const std::vector<RagLevel<T>>& v, int nu, cudaStream_t s) {
  if (v.empty()) return;
  const int n = (int)v.size();
  auto run = [&](auto rad) {
    constexpr int R = decltype(rad)::value;
    const bool fused = KFUSE<T> && v[0].gb.w2 != nullptr;
    std::vector<KmA<T, R>> A(n);
    for (int q = 0; q < n; ++q) {
      const RagLevel<T>& L = v[q];
      const OpView<T>& o = L.op;
      const OpK<T, R> op = kron_op<T, R>(o, L.g.nx, L.g.ny);
      const KGeo kg = kron_geo(L.g, 1, R, kron_capacity<T, R>(fused), L.gb.kron_ch);
      A[q] = KmA<T, R>{L.g, kg, op, L.x, L.b, (cx<T>*)L.gb.u[0], (cx<T>*)L.gb.u[1], (cx<T>*)L.gb.u[2],
                       (cx<T>*)L.gb.w, nullptr, nullptr, nullptr, L.gb.st, L.gb.partial, L.gb.tickets, L.active};
    }
    auto launch = [&](auto kern, auto set) {
      rag_launch<KmA<T, R>>(n, kern, dim3(KW * 32), 0, s, [&](int q, KmA<T, R>& a, int& gx, int&) {
        a = A[q];
        set(a, v[q]);
        gx = cdiv((long long)a.kg.ncw * a.kg.nchunks, KW);
        return true;
      });
    };
    auto none = [](KmA<T, R>&, const RagLevel<T>&) {};
    for (int step = 0; step < nu; ++step) {
      launch(km_init_rag<T, R>, none);
      launch(km_arn_a_rag<T, R, 0>, none);
      bool done = false;
      if constexpr (KFUSE<T>) {
        if (fused) {   // arn_b<0> + arn_a<1>, arn_b<1> + arn_a<2>, as gmres_smooth_kron
          launch(km_arn_ab_rag<T, R, 1>, [](KmA<T, R>& a, const RagLevel<T>& L) {
            a.win = (const cx<T>*)L.gb.w;
            a.uJ = (cx<T>*)L.gb.u[1];
            a.wout = (cx<T>*)L.gb.w2;
          });
          launch(km_arn_ab_rag<T, R, 2>, [](KmA<T, R>& a, const RagLevel<T>& L) {
            a.win = (const cx<T>*)L.gb.w2;
            a.uJ = (cx<T>*)L.gb.u[2];
            a.wout = (cx<T>*)L.gb.w;
          });
          done = true;   // u3's norm from the Gram form: no closing g_arn_b<2>
        }
      }
      if (!done) {
        launch_arn_b_rag<T, 0>(v, true, -1, s);
        launch(km_arn_a_rag<T, R, 1>, none);
        launch_arn_b_rag<T, 1>(v, true, -1, s);
        launch(km_arn_a_rag<T, R, 2>, none);
        launch_arn_b_rag<T, 2>(v, false, -1, s);
      }
      launch_gmres_update_rag<T>(v, s);
    }
  };
  if (v[0].op.kind == 4) run(std::integral_constant<int, 2>{});
  else run(std::integral_constant<int, 3>{});
}

template void gmres_smooth_kron_rag<double>(const std::vector<RagLevel<double>>&, int, cudaStream_t);
template void gmres_smooth_kron_rag<float>(const std::vector<RagLevel<float>>&, int, cudaStream_t);
template void launch_kron_residual<double>(const Grid&, const OpView<double>&, const double2*, const double2*,
                                           double2*, int, const int*, int, cudaStream_t);
template void launch_kron_residual<float>(const Grid&, const OpView<float>&, const float2*, const float2*, float2*,
                                          int, const int*, int, cudaStream_t);
template void gmres_smooth_kron<double>(const Grid&, const OpView<double>&, double2*, const double2*, int, int,
                                        const int*, const GmresBufs&, cudaStream_t);
template void gmres_smooth_kron<float>(const Grid&, const OpView<float>&, float2*, const float2*, int, int,
                                       const int*, const GmresBufs&, cudaStream_t);

}  // namespace hmg
