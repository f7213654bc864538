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
#include <type_traits>

#include "gmres.cuh"
#include "internal.h"

namespace hmg {

namespace {

constexpr int KW = 4;   // warps per block; a warp covers 32 columns of one chunk of rows

struct KGeo {
  int ncw;      // 32-column groups
  int ch;       // rows per chunk
  int nchunks;
};

// A v down column i: sums() forms the two row sums of one input row,
// shift_in() appends them to the ring of the last 2R+1 rows, and combine()
// returns (A v)(i, m) once the ring holds rows m-R..m+R.  The next input row
// is fetched one iteration ahead (prime / advance).
template <class T, int R> struct KRing {
  static constexpr int K = 2 * R + 1;
  cx<T> G[K];
  T Wx[K];
  cx<T> s1[K], s2[K];

  __device__ __forceinline__ void init(const OpK<T, R>& op, int i) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      G[k] = op.gx[i * K + k];
      Wx[k] = op.wx[i * K + k];
      s1[k] = mk<T>(T(0), T(0));
      s2[k] = mk<T>(T(0), T(0));
    }
  }
  // the 2R+1 values of one input row around column i (slice pointer vs,
  // node offset p of (i, row))
  __device__ __forceinline__ static void fetch(const cx<T>* __restrict__ vs, int p, cx<T> (&xv)[K]) {
#pragma unroll
    for (int dx = -R; dx <= R; ++dx) xv[dx + R] = __ldg(vs + p + dx);
  }
  // row sums of one input row
  __device__ __forceinline__ void sums(const cx<T> (&xv)[K], cx<T>& a, cx<T>& c) const {
    a = mk<T>(T(0), T(0));
    c = mk<T>(T(0), T(0));
#pragma unroll
    for (int dx = -R; dx <= R; ++dx) {
      a = fma_c<T>(G[dx + R], xv[dx + R], a);
      c = mk<T>(fma(Wx[dx + R], xv[dx + R].x, c.x), fma(Wx[dx + R], xv[dx + R].y, c.y));
    }
  }
  // march prologue: rows j0-R .. j0+R-1 into the ring, row j0+R fetched into nx
  __device__ __forceinline__ void prime(const cx<T>* __restrict__ vs, const Grid& g, int i, int j0, cx<T> (&nx)[K]) {
    cx<T> a, c;
#pragma unroll 1
    for (int r = j0 - R; r < j0 + R; ++r) {
      fetch(vs, g.at(i, r), nx);
      sums(nx, a, c);
      shift_in(a, c);
    }
    fetch(vs, g.at(i, j0 + R), nx);
  }
  // ring advance for output row m: uses the fetched row m+R, fetches row
  // m+R+1 (the next iteration's) before the arithmetic
  __device__ __forceinline__ void advance(const cx<T>* __restrict__ vs, const Grid& g, int i, int m, int j1,
                                          cx<T> (&nx)[K]) {
    cx<T> cur[K];
#pragma unroll
    for (int k = 0; k < K; ++k) cur[k] = nx[k];
    if (m + 1 < j1) fetch(vs, g.at(i, m + R + 1), nx);
    cx<T> a, c;
    sums(cur, a, c);
    shift_in(a, c);
  }
  __device__ __forceinline__ void shift_in(cx<T> a, cx<T> c) {
#pragma unroll
    for (int k = 0; k < K - 1; ++k) {
      s1[k] = s1[k + 1];
      s2[k] = s2[k + 1];
    }
    s1[K - 1] = a;
    s2[K - 1] = c;
  }
  // combination along y for output row m (ring holds rows m-R..m+R)
  __device__ __forceinline__ cx<T> combine(const OpK<T, R>& op, int m) const {
    const cx<T>* H = op.hy + m * K;
    const T* Wy = op.wy + m * K;
    cx<T> acc = mk<T>(T(0), T(0));
#pragma unroll
    for (int dy = -R; dy <= R; ++dy) {
      const T wy = __ldg(Wy + dy + R);
      acc = mk<T>(fma(wy, s1[dy + R].x, acc.x), fma(wy, s1[dy + R].y, acc.y));
      acc = fma_c<T>(__ldg(H + dy + R), s2[dy + R], acc);
    }
    return acc;
  }
};

#define KPRO                                                                  \
  __shared__ double sh[NVMAX * 32];                                           \
  const int rhs = blockIdx.z;                                                 \
  if (active && !active[rhs]) return;                                         \
  const long long off = (long long)rhs * g.vstride;                           \
  const int gw = blockIdx.x * KW + (threadIdx.x >> 5);                       \
  const bool has = gw < kg.ncw * kg.nchunks;                                  \
  const int i = (has ? gw % kg.ncw : 0) * 32 + (threadIdx.x & 31);            \
  const int j0 = (has ? gw / kg.ncw : 0) * kg.ch, j1 = min(j0 + kg.ch, g.ny + 1); \
  const bool col = has && i <= g.nx;                                          \
  const int nblk = gridDim.x, blk = blockIdx.x;                               \
  const bool t0 = threadIdx.x == 0;

// u0 = b - A x, partial |u0|^2 (as g_init)
template <class T, int R>
__global__ void __launch_bounds__(KW * 32) km_init(Grid g, KGeo kg, OpK<T, R> op, const cx<T>* __restrict__ x,
                                              const cx<T>* __restrict__ b, cx<T>* __restrict__ u0, double* st,
                                              double* partial, unsigned* tickets, const int* __restrict__ active) {
  KPRO
  T a0[1] = {T(0)};
  if (col) {
    const cx<T>* xs = x + off;
    KRing<T, R> ring;
    ring.init(op, i);
    cx<T> nx[KRing<T, R>::K];
    ring.prime(xs, g, i, j0, nx);
#pragma unroll 1
    for (int m = j0; m < j1; ++m) {
      ring.advance(xs, g, i, m, j1, nx);
      const int p = g.at(i, m);
      const cx<T> r = sub<T>(b[off + p], ring.combine(op, m));
      u0[off + p] = r;
      a0[0] += abs2<T>(r);
    }
  }
  double v[1];
  if (reduce_last<1, T>(a0, v, sh, partial, tickets, rhs, nblk, blk) && t0) fin_init<T>(st + (long long)rhs * GS, v);
}

// w = s_J A u_J; partial dots <u_l, w>, l <= J (as g_arn_a)
template <class T, int R, int J>
__global__ void __launch_bounds__(KW * 32) km_arn_a(Grid g, KGeo kg, OpK<T, R> op, const cx<T>* __restrict__ u0,
                                               const cx<T>* __restrict__ u1, const cx<T>* __restrict__ u2,
                                               cx<T>* __restrict__ w, double* __restrict__ st, double* partial,
                                               unsigned* tickets, const int* __restrict__ active) {
  KPRO
  double* S = st + (long long)rhs * GS;
  if (S[G_BRK] != 0.0 || S[G_M] < J) return;   // uniform per RHS
  const cx<T>* uJ = J == 0 ? u0 : (J == 1 ? u1 : u2);
  T acc[2 * (J + 1)];
#pragma unroll
  for (int k = 0; k < 2 * (J + 1); ++k) acc[k] = T(0);
  if (col) {
    const T sJ = (T)S[G_S + J];
    const cx<T>* us[3] = {u0 + off, u1 + off, u2 + off};
    const cx<T>* vs = uJ + off;
    KRing<T, R> ring;
    ring.init(op, i);
    cx<T> nx[KRing<T, R>::K];
    ring.prime(vs, g, i, j0, nx);
#pragma unroll 1
    for (int m = j0; m < j1; ++m) {
      ring.advance(vs, g, i, m, j1, nx);
      const int p = g.at(i, m);
      const cx<T> a = scl<T>(sJ, ring.combine(op, m));
      w[off + p] = a;
#pragma unroll
      for (int l = 0; l <= J; ++l) {
        const cx<T> d = cmul<T>(us[l][p], a);
        acc[2 * l] += d.x;
        acc[2 * l + 1] += d.y;
      }
    }
  }
  double v[2 * (J + 1)];
  if (reduce_last<2 * (J + 1), T>(acc, v, sh, partial, tickets, rhs, nblk, blk))
    staged<T>(S, v, [](double* s, const double* q) { fin_a<J, T>(s, q); });
}

KGeo kron_geo(const Grid& g, int B) {
  KGeo k;
  k.ncw = cdiv(g.nx + 1, 32);
  const long long want = 152LL * 64;   // warps to fill the GPU a few times over
  int ch = 64;
  while (ch > 8 && (long long)k.ncw * cdiv(g.ny + 1, ch) * B < want) ch /= 2;
  k.ch = ch;
  k.nchunks = cdiv(g.ny + 1, ch);
  return k;
}

}  // namespace

template <class T> void launch_gmres_update(const Grid& g, cx<T>* x, const GmresBufs& gb, int B, const int* active,
                                            cudaStream_t s);
template <class T, int J> void launch_arn_b(const Grid& g, const GmresBufs& gb, cx<T>* un, int B, const int* active,
                                            cudaStream_t s);

long long kron_march_blocks(const Grid& g, int B) {
  const KGeo k = kron_geo(g, B);
  return cdiv((long long)k.ncw * k.nchunks, KW);
}

template <class T>
void gmres_smooth_kron(const Grid& g, const OpView<T>& opv, cx<T>* x, const cx<T>* b, int nu, int B,
                       const int* active, const GmresBufs& gb, cudaStream_t s) {
  cx<T>* u0 = (cx<T>*)gb.u[0];
  cx<T>* u1 = (cx<T>*)gb.u[1];
  cx<T>* u2 = (cx<T>*)gb.u[2];
  cx<T>* w = (cx<T>*)gb.w;
  double* P = gb.partial;
  unsigned* tk = gb.tickets;
  double* st = gb.st;
  const KGeo kg = kron_geo(g, B);
  const dim3 grd(cdiv((long long)kg.ncw * kg.nchunks, KW), 1, B);
  auto run = [&](auto op, auto rad) {
    constexpr int R = decltype(rad)::value;
    for (int step = 0; step < nu; ++step) {
      km_init<T, R><<<grd, KW * 32, 0, s>>>(g, kg, op, x, b, u0, st, P, tk, active);
      km_arn_a<T, R, 0><<<grd, KW * 32, 0, s>>>(g, kg, op, u0, u1, u2, w, st, P, tk, active);
      launch_arn_b<T, 0>(g, gb, u1, B, active, s);
      km_arn_a<T, R, 1><<<grd, KW * 32, 0, s>>>(g, kg, op, u0, u1, u2, w, st, P, tk, active);
      launch_arn_b<T, 1>(g, gb, u2, B, active, s);
      km_arn_a<T, R, 2><<<grd, KW * 32, 0, s>>>(g, kg, op, u0, u1, u2, w, st, P, tk, active);
      launch_arn_b<T, 2>(g, gb, nullptr, B, active, s);
      launch_gmres_update<T>(g, x, gb, B, active, s);
    }
  };
  if (opv.kind == 4)
    run(OpK<T, 2>{opv.gx, opv.wx, opv.hy, opv.wy, opv.dinv, g.nx, g.ny}, std::integral_constant<int, 2>{});
  else
    run(OpK<T, 3>{opv.gx, opv.wx, opv.hy, opv.wy, opv.dinv, g.nx, g.ny}, std::integral_constant<int, 3>{});
}

template void gmres_smooth_kron<double>(const Grid&, const OpView<double>&, double2*, const double2*, int, int,
                                        const int*, const GmresBufs&, cudaStream_t);
template void gmres_smooth_kron<float>(const Grid&, const OpView<float>&, float2*, const float2*, int, int,
                                       const int*, const GmresBufs&, cudaStream_t);

}  // namespace hmg
