// Flexible GMRES(m) outer loop with one multigrid cycle as the right
// preconditioner: the Krylov use of multigrid recalled in Sec. 1 of the
// paper (the cycle inverts an approximation of A inside GMRES), around the
// stand-alone cycle of this library.  Restarted FGMRES (Saad 1993): one
// restart cycle from x is
//   r = b - A x, beta = ||r||, v_0 = r / beta, g = beta e_1
//   step j: z_j = M(v_j) (one cycle from zero on A e = v_j), w = A z_j,
//           h_ij = <v_i, w^(i)> (modified Gram-Schmidt), h_{j+1,j} = ||w'||,
//           v_{j+1} = w' / h_{j+1,j}, Givens rotations on column j and on g;
//           |g_{j+1}| is the residual norm of x + Z_{j+1} y
//   x += Z_k y (triangular solve)
// Precision: x, b, the restart residual r = b - A x, the update and every
// scalar (Hessenberg, Gram matrix, rotations, y) are FP64.  The basis V,
// the preconditioned vectors Z and the arithmetic of the Arnoldi passes
// (w = A z, the dots, v_{j+1}) take the cycle's precision T: FP64 for the
// complex128 path; FP32 for the mixed path, where each restart cycle is then
// an FP32 FGMRES correction of the FP64 residual (iterative refinement with
// FGMRES as the inner solver), and the true FP64 residual at the restart
// decides convergence.  GB300's FP64 pipe runs at about 1/58 of FP32, and an
// FP64 Arnoldi step costs ~180 FP64 FMAs per node, which made it ALU-bound.
//
// The basis is kept unnormalised: u_j with v_j = s_j u_j, s_0 = 1/beta and
// s_j = 1/h_{j,j-1} among the scalars.  The cycle from zero is homogeneous
// (M(u) = M(v)/s), so it runs directly on u_j, which the pass that forms u_j
// also writes as the cycle's right-hand side, and the dots pass scales its
// output: z_j = s_j M(u_j).  Kernels (the captured cycle graph runs between
// the restart or orth pass and the next dots pass):
//   restart  r = b - A x (FP64) into u_0 and the cycle rhs, cycle x = 0,
//            ||r||, restart test                                (last block)
//   dots     Z_j = s_j z', w = A Z_j, <u_i, w> (i <= j) and <u_i, u_j> (i < j);
//            the last block scales them by the s_i and turns them into the
//            MGS coefficients (Gram form: h_i = <v_i, w> - sum_{l<i} h_l
//            <v_i, v_l>, MGS in exact arithmetic for any V) in one pass over
//            the j+1 vectors
//   orth     u_{j+1} = w - sum_i h_i s_i u_i (w recomputed from Z_j) into the
//            basis and the cycle rhs, cycle x = 0, ||u_{j+1}||; the last block
//            finishes the Arnoldi step, the rotations and the per-RHS exit
//   update   x += sum_i y_i z_i (FP64)
// Every kernel walks strips of 32 columns x 64 rows (8 rows per thread,
// warps along rows) with a fixed number of blocks per right-hand side;
// per-strip sums in T are widened to FP64 per warp, block sums go to a
// value-major partial array and the block holding the last ticket adds them
// in block order (bitwise reproducible).
#include <math.h>

#include <algorithm>

#include "internal.h"

namespace hmg {

namespace {

constexpr int FBX = 32, FBY = 8, FR = 8;   // strip: 32 columns x (8 warps x 8 rows)
constexpr int FTHREADS = FBX * FBY;
constexpr int FNV = 4 * FG_MAXM + 2;       // values per block record of the dots pass

__device__ __forceinline__ double2 to_d(double2 a) { return a; }
__device__ __forceinline__ double2 to_d(float2 a) { return make_double2((double)a.x, (double)a.y); }
template <class T> __device__ __forceinline__ cx<T> from_d(double2 a);
template <> __device__ __forceinline__ double2 from_d<double>(double2 a) { return a; }
template <> __device__ __forceinline__ float2 from_d<float>(double2 a) { return make_float2((float)a.x, (float)a.y); }

__device__ __forceinline__ double warp_sum(double t) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
  return t;
}

// The fine operator in precision T (the cycle's level-0 operator).
// A2 selects the second-order absorbing rows at compile time.
template <class T, bool A2> __device__ __forceinline__ Op0<T, A2> op_t(const FgArgs& a) {
  if constexpr (std::is_same<T, double>::value) return Op0<T, A2>{a.c0, a.kf, a.g.nx, a.g.ny};
  else return Op0<T, A2>{a.c0f, a.kf32, a.g.nx, a.g.ny};
}

// Sums four values over a warp in six shuffles: the first two rounds halve
// the values each lane carries (lanes 0-15 keep a, b and 16-31 keep c, d;
// then lanes with bit 3 clear keep the first of their pair), the last three
// are plain butterflies.  Lane 8w + u (u < 8) returns the total of value w
// (a, b, c, d for w = 0..3).  Fixed order: bitwise reproducible.
template <class T> __device__ __forceinline__ T warp_sum4(T a, T b, T c, T d, int lane) {
  const bool hi16 = lane & 16;
  T k0 = hi16 ? c : a, k1 = hi16 ? d : b;
  const T s0 = hi16 ? a : c, s1 = hi16 ? b : d;
  k0 += __shfl_xor_sync(0xffffffffu, s0, 16);
  k1 += __shfl_xor_sync(0xffffffffu, s1, 16);
  const bool hi8 = lane & 8;
  T k = hi8 ? k1 : k0;
  k += __shfl_xor_sync(0xffffffffu, hi8 ? k0 : k1, 8);
#pragma unroll
  for (int o = 4; o > 0; o >>= 1) k += __shfl_xor_sync(0xffffffffu, k, o);
  return k;
}

template <class T> constexpr bool PREFETCH = sizeof(T) == 4;
// resident blocks per SM the Arnoldi passes are compiled for (FP32: 24 warps)
template <class T> constexpr int FG_MINB = sizeof(T) == 4 ? 3 : 2;

// The thread's FR rows of one vector (zero where pr < 0: outside the grid).
template <class T>
__device__ __forceinline__ void load_rows(const cx<T>* __restrict__ v, const int (&pr)[FR], cx<T> (&out)[FR]) {
#pragma unroll
  for (int r = 0; r < FR; ++r) out[r] = pr[r] >= 0 ? v[pr[r]] : mk<T>(T(0), T(0));
}

struct StripPos {
  int i, j0;
};
__device__ __forceinline__ StripPos strip_pos(const FgArgs& a, int s) {
  return StripPos{(s % a.ncx) * FBX + (int)threadIdx.x, (s / a.ncx) * (FBY * FR) + (int)threadIdx.y};
}

// Publishes this block's nval sums (thread t < nval holds value t) and takes
// a ticket; returns true, block-uniformly, in the block holding the last
// ticket, after which tot[0 .. nval-1] hold the sums over all blocks.
__device__ bool fg_reduce(const FgArgs& a, int rhs, int nval, const double* mine, double* tot) {
  __shared__ int s_last;
  const int tid = threadIdx.x + threadIdx.y * FBX, lane = threadIdx.x, warp = threadIdx.y;
  if (tid < nval) a.partial[((long long)rhs * a.nvp + tid) * a.nbr + blockIdx.x] = mine[tid];
  __threadfence();
  __syncthreads();
  if (tid == 0) s_last = atomicAdd(&a.tickets[rhs], 1u) == (unsigned)(a.nbr - 1);
  __syncthreads();
  if (!s_last) return false;
  __threadfence();
  for (int q = warp; q < nval; q += FBY) {
    const double* pq = a.partial + ((long long)rhs * a.nvp + q) * a.nbr;
    double t = 0.0;
    for (int b = lane; b < a.nbr; b += 32) t += __ldcg(pq + b);
    t = warp_sum(t);
    if (lane == 0) tot[q] = t;
  }
  __syncthreads();
  if (tid == 0) a.tickets[rhs] = 0u;
  return true;
}

// ------------------------------------------------------------------ restart

template <class T, bool A2>
__global__ void __launch_bounds__(FTHREADS) k_fg_restart(FgArgs a, cx<T>* __restrict__ cb, cx<T>* __restrict__ cxv) {
  const Op0<double, A2> op = op_t<double, A2>(a);
  __shared__ double red[FBY], tot[1], mine[1];
  const int rhs = blockIdx.z;
  if (a.state[rhs] != 0) return;   // block-uniform
  const Grid& g = a.g;
  const long long off = (long long)rhs * g.vstride;
  const double2* x = a.X + off;
  const double2* b = a.b + off;
  cx<T>* v0 = (cx<T>*)a.V + off;
  double acc = 0.0;
  for (int s = blockIdx.x; s < a.ns; s += a.nbr) {
    const StripPos sp = strip_pos(a, s);
    if (sp.i > g.nx) continue;
#pragma unroll
    for (int r = 0; r < FR; ++r) {
      const int j = sp.j0 + r * FBY;
      if (j > g.ny) break;
      const int p = g.at(sp.i, j);
      const double2 rr = sub<double>(b[p], op.apply(x, p, g.pitch, sp.i, j));
      const cx<T> u = from_d<T>(rr);
      v0[p] = u;
      cb[off + p] = u;
      cxv[off + p] = mk<T>(T(0), T(0));
      acc += abs2<double>(rr);
    }
  }
  acc = warp_sum(acc);
  if (threadIdx.x == 0) red[threadIdx.y] = acc;
  __syncthreads();
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    double t = 0.0;
    for (int w = 0; w < FBY; ++w) t += red[w];
    mine[0] = t;
  }
  __syncthreads();
  if (!fg_reduce(a, rhs, 1, mine, tot)) return;
  if (threadIdx.x || threadIdx.y) return;
  // restart test and the start of a restart cycle
  const FgLayout L{a.m};
  double* S = a.S + (long long)rhs * a.sd;
  const double beta = sqrt(tot[0]);
  const double rr = beta / a.bnorm[rhs];
  a.relres[rhs] = rr;
  a.kst[2 * rhs] = 0;
  if (!(rr == rr) || isinf(rr)) {
    a.state[rhs] = 2;
  } else if (rr <= a.tol) {
    a.state[rhs] = 1;
  } else if (a.cycles[rhs] < a.max_cycles) {
    a.kst[2 * rhs + 1] = min(a.m, a.max_cycles - a.cycles[rhs]);
    for (int q = 0; q <= a.m; ++q) S[L.g(q)] = S[L.g(q) + 1] = 0.0;
    S[L.g(0)] = beta;
    S[L.beta()] = beta;
    S[L.s(0)] = 1.0 / beta;
    a.active[rhs] = 1;
    atomicAdd(a.n_active, 1);
  }
}

// ------------------------------------------------------------------ dots (MGS coefficients)

template <class T, bool A2>
__global__ void __launch_bounds__(FTHREADS, FG_MINB<T>) k_fg_dots(FgArgs a, const cx<T>* __restrict__ z, int jj) {
  __shared__ double red[FNV][FBY];
  __shared__ double mine[FNV], tot[FNV];
  const int rhs = blockIdx.z;
  if (!a.active[rhs]) return;
  const int tid = threadIdx.x + threadIdx.y * FBX, lane = threadIdx.x, warp = threadIdx.y;
  const int nval = 4 * jj + 2;   // <v_i, w> for i <= jj, then <v_i, v_jj> for i < jj (re, im)
  for (int q = tid; q < nval * FBY; q += FTHREADS) red[q / FBY][q % FBY] = 0.0;
  __syncthreads();
  const Grid& g = a.g;
  const long long off = (long long)rhs * g.vstride;
  const Op0<T, A2> op = op_t<T, A2>(a);
  const cx<T>* zs = z + off;
  cx<T>* zj = (cx<T>*)a.Z + jj * a.vlen + off;
  const cx<T>* vj = (const cx<T>*)a.V + jj * a.vlen + off;
  const T sj = (T)a.S[(long long)rhs * a.sd + FgLayout{a.m}.s(jj)];   // z_j = s_j M(u_j)
  for (int s = blockIdx.x; s < a.ns; s += a.nbr) {
    const StripPos sp = strip_pos(a, s);
    cx<T> w[FR], u[FR];
    int pr[FR];
#pragma unroll
    for (int r = 0; r < FR; ++r) {
      const int j = sp.j0 + r * FBY;
      pr[r] = -1;
      w[r] = u[r] = mk<T>(T(0), T(0));
      if (sp.i <= g.nx && j <= g.ny) {
        const int p = g.at(sp.i, j);
        pr[r] = p;
        zj[p] = scl<T>(sj, zs[p]);
        w[r] = scl<T>(sj, op.apply(zs, p, g.pitch, sp.i, j));
        u[r] = vj[p];
      }
    }
    // v_q at the thread's rows; FP32 fetches v_{q+1} before v_q is used
    // (FP64 is bound by its arithmetic and has no registers to spare)
    cx<T> cur[FR], nxt[FR];
    load_rows<T>((const cx<T>*)a.V + off, pr, cur);
    for (int q = 0; q <= jj; ++q) {
      if (PREFETCH<T> && q < jj) load_rows<T>((const cx<T>*)a.V + (q + 1) * a.vlen + off, pr, nxt);
      T dr = T(0), di = T(0), gr = T(0), gi = T(0);
#pragma unroll
      for (int r = 0; r < FR; ++r) {
        const cx<T> v = cur[r];   // zero outside the grid
        dr = fma(v.x, w[r].x, fma(v.y, w[r].y, dr));
        di = fma(v.x, w[r].y, fma(-v.y, w[r].x, di));
        gr = fma(v.x, u[r].x, fma(v.y, u[r].y, gr));
        gi = fma(v.x, u[r].y, fma(-v.y, u[r].x, gi));
      }
      // the warp's four sums; lanes 0, 8, 16, 24 then hold dr, di, gr, gi,
      // widened to FP64 into the warp's column of red
      const T t = warp_sum4<T>(dr, di, gr, gi, lane);
      if ((lane & 7) == 0) {
        const int which = lane >> 3;   // 0 dr, 1 di, 2 gr, 3 gi
        if (which < 2) red[2 * q + which][warp] += (double)t;
        else if (q < jj) red[2 * (jj + 1) + 2 * q + which - 2][warp] += (double)t;
      }
      if (PREFETCH<T>) {
#pragma unroll
        for (int r = 0; r < FR; ++r) cur[r] = nxt[r];
      } else if (q < jj) {
        load_rows<T>((const cx<T>*)a.V + (q + 1) * a.vlen + off, pr, cur);
      }
    }
  }
  __syncthreads();
  if (tid < nval) {
    double t = 0.0;
    for (int w = 0; w < FBY; ++w) t += red[tid][w];
    mine[tid] = t;
  }
  __syncthreads();
  if (!fg_reduce(a, rhs, nval, mine, tot)) return;
  if (tid) return;
  // Gram row jj, then the MGS coefficients of column jj (v_i = s_i u_i)
  const FgLayout L{a.m};
  double* S = a.S + (long long)rhs * a.sd;
  const double sjj = S[L.s(jj)];
  for (int l = 0; l < jj; ++l) {   // <v_jj, v_l> = s_jj s_l conj(<u_l, u_jj>)
    const double f = sjj * S[L.s(l)];
    S[L.gram(jj, l)] = f * tot[2 * (jj + 1) + 2 * l];
    S[L.gram(jj, l) + 1] = -f * tot[2 * (jj + 1) + 2 * l + 1];
  }
  for (int q = 0; q <= jj; ++q) {
    const double sq = S[L.s(q)];
    double hr = sq * tot[2 * q], hi = sq * tot[2 * q + 1];
    for (int l = 0; l < q; ++l) {
      const double ar = S[L.h(jj, l)], ai = S[L.h(jj, l) + 1];
      const double gr = S[L.gram(q, l)], gi = S[L.gram(q, l) + 1];
      hr -= ar * gr - ai * gi;
      hi -= ar * gi + ai * gr;
    }
    S[L.h(jj, q)] = hr;
    S[L.h(jj, q) + 1] = hi;
  }
}

// ------------------------------------------------------------------ orth (new basis vector, Givens)

// (c, s), c real, with [[c, s], [-conj(s), c]] (a, b)^T = (r, 0)^T.
__device__ void givens(double2 a, double2 b, double& c, double2& s) {
  const double na = hypot(a.x, a.y), nb = hypot(b.x, b.y);
  const double nr = hypot(na, nb);
  if (nr == 0.0) {
    c = 1.0;
    s = make_double2(0.0, 0.0);
  } else if (na == 0.0) {
    c = 0.0;
    s = make_double2(b.x / nb, -b.y / nb);
  } else {
    c = na / nr;
    // (a / |a|) conj(b) / r
    const double ux = a.x / na, uy = a.y / na;
    s = make_double2((ux * b.x + uy * b.y) / nr, (uy * b.x - ux * b.y) / nr);
  }
}

__device__ void fg_finish_step(const FgArgs& a, int rhs, int jj, double sumsq) {
  const FgLayout L{a.m};
  double* S = a.S + (long long)rhs * a.sd;
  const double nrm = sqrt(sumsq);
  const double beta = S[L.beta()];
  const bool brk = nrm <= 1e-14 * beta;
  double2 hc[FG_MAXM + 1];
  for (int i = 0; i <= jj; ++i) hc[i] = make_double2(S[L.h(jj, i)], S[L.h(jj, i) + 1]);
  hc[jj + 1] = make_double2(nrm, 0.0);
  for (int i = 0; i < jj; ++i) {   // the earlier rotations on the new column
    const double c = S[L.cs(i)];
    const double2 sn = make_double2(S[L.sn(i)], S[L.sn(i) + 1]);
    const double2 x0 = hc[i], x1 = hc[i + 1];
    hc[i] = add<double>(scl<double>(c, x0), mul<double>(sn, x1));
    hc[i + 1] = sub<double>(scl<double>(c, x1), cmul<double>(sn, x0));   // -conj(s) a + c b
  }
  double c;
  double2 sn;
  givens(hc[jj], hc[jj + 1], c, sn);
  hc[jj] = add<double>(scl<double>(c, hc[jj]), mul<double>(sn, hc[jj + 1]));
  hc[jj + 1] = make_double2(0.0, 0.0);
  S[L.cs(jj)] = c;
  S[L.sn(jj)] = sn.x;
  S[L.sn(jj) + 1] = sn.y;
  for (int i = 0; i <= jj; ++i) {
    S[L.h(jj, i)] = hc[i].x;
    S[L.h(jj, i) + 1] = hc[i].y;
  }
  const double2 gj = make_double2(S[L.g(jj)], S[L.g(jj) + 1]);
  const double2 g1 = cmul<double>(sn, gj);   // conj(s) g_j
  S[L.g(jj + 1)] = -g1.x;
  S[L.g(jj + 1) + 1] = -g1.y;
  S[L.g(jj)] = c * gj.x;
  S[L.g(jj) + 1] = c * gj.y;
  const double est = hypot(g1.x, g1.y) / a.bnorm[rhs];
  const int k = jj + 1;
  a.kst[2 * rhs] = k;
  const int cy = ++a.cycles[rhs];
  if (cy <= a.hist_len) a.hist[(long long)rhs * a.hist_len + cy - 1] = est;
  if (brk || est <= a.tol || k >= a.kst[2 * rhs + 1]) {
    // y = R^{-1} g by back substitution over the k rotated columns
    for (int i = k - 1; i >= 0; --i) {
      double2 t = make_double2(S[L.g(i)], S[L.g(i) + 1]);
      for (int l = i + 1; l < k; ++l) {
        const double2 r = make_double2(S[L.h(l, i)], S[L.h(l, i) + 1]);
        const double2 yl = make_double2(S[L.y(l)], S[L.y(l) + 1]);
        t = sub<double>(t, mul<double>(r, yl));
      }
      const double2 d = make_double2(S[L.h(i, i)], S[L.h(i, i) + 1]);
      const double dd = d.x * d.x + d.y * d.y;
      const double2 yi = make_double2((t.x * d.x + t.y * d.y) / dd, (t.y * d.x - t.x * d.y) / dd);
      S[L.y(i)] = yi.x;
      S[L.y(i) + 1] = yi.y;
    }
    a.active[rhs] = 0;
    atomicSub(a.n_active, 1);
  } else {
    S[L.s(k)] = 1.0 / nrm;
  }
}

template <class T, bool A2>
__global__ void __launch_bounds__(FTHREADS, FG_MINB<T>) k_fg_orth(FgArgs a, int jj, cx<T>* __restrict__ cb,
                                                                  cx<T>* __restrict__ cxv) {
  __shared__ cx<T> hs[FG_MAXM + 1];
  __shared__ double red[FBY], mine[1], tot[1];
  const int rhs = blockIdx.z;
  if (!a.active[rhs]) return;
  const int tid = threadIdx.x + threadIdx.y * FBX;
  const FgLayout L{a.m};
  const double* S = a.S + (long long)rhs * a.sd;
  if (tid <= jj) {   // h_i s_i: the coefficient of u_i
    const double si = S[L.s(tid)];
    hs[tid] = mk<T>((T)(S[L.h(jj, tid)] * si), (T)(S[L.h(jj, tid) + 1] * si));
  }
  __syncthreads();
  const Op0<T, A2> op = op_t<T, A2>(a);
  const Grid& g = a.g;
  const long long off = (long long)rhs * g.vstride;
  const cx<T>* zj = (const cx<T>*)a.Z + jj * a.vlen + off;
  cx<T>* vn = (cx<T>*)a.V + (jj + 1) * a.vlen + off;
  double acc = 0.0;
  for (int s = blockIdx.x; s < a.ns; s += a.nbr) {
    const StripPos sp = strip_pos(a, s);
    cx<T> w[FR];
    int pr[FR];
#pragma unroll
    for (int r = 0; r < FR; ++r) {
      const int j = sp.j0 + r * FBY;
      pr[r] = -1;
      w[r] = mk<T>(T(0), T(0));
      if (sp.i <= g.nx && j <= g.ny) {
        pr[r] = g.at(sp.i, j);
        w[r] = op.apply(zj, pr[r], g.pitch, sp.i, j);
      }
    }
    cx<T> cur[FR], nxt[FR];
    load_rows<T>((const cx<T>*)a.V + off, pr, cur);
    for (int q = 0; q <= jj; ++q) {
      if (PREFETCH<T> && q < jj) load_rows<T>((const cx<T>*)a.V + (q + 1) * a.vlen + off, pr, nxt);
      const cx<T> h = hs[q];
#pragma unroll
      for (int r = 0; r < FR; ++r) {
        w[r].x -= h.x * cur[r].x - h.y * cur[r].y;
        w[r].y -= h.x * cur[r].y + h.y * cur[r].x;
      }
      if (PREFETCH<T>) {
#pragma unroll
        for (int r = 0; r < FR; ++r) cur[r] = nxt[r];
      } else if (q < jj) {
        load_rows<T>((const cx<T>*)a.V + (q + 1) * a.vlen + off, pr, cur);
      }
    }
    T part = T(0);   // this strip's sum in T, widened once
#pragma unroll
    for (int r = 0; r < FR; ++r) {
      if (pr[r] < 0) continue;
      vn[pr[r]] = w[r];
      cb[off + pr[r]] = w[r];
      cxv[off + pr[r]] = mk<T>(T(0), T(0));
      part += abs2<T>(w[r]);
    }
    acc += (double)part;
  }
  acc = warp_sum(acc);
  if (threadIdx.x == 0) red[threadIdx.y] = acc;
  __syncthreads();
  if (tid == 0) {
    double t = 0.0;
    for (int w = 0; w < FBY; ++w) t += red[w];
    mine[0] = t;
  }
  __syncthreads();
  if (!fg_reduce(a, rhs, 1, mine, tot)) return;
  if (tid == 0) fg_finish_step(a, rhs, jj, tot[0]);
}

// ------------------------------------------------------------------ update

// x += sum_q y_q z_q: the correction is summed in T (for the mixed path an
// FP32 correction, like the refinement loop's x += e) and added to x in FP64.
template <class T> __global__ void __launch_bounds__(FTHREADS) k_fg_update(FgArgs a) {
  __shared__ cx<T> ys[FG_MAXM];
  const int rhs = blockIdx.z;
  const int k = a.kst[2 * rhs];
  if (k == 0) return;   // block-uniform
  const int tid = threadIdx.x + threadIdx.y * FBX;
  const FgLayout L{a.m};
  const double* S = a.S + (long long)rhs * a.sd;
  if (tid < k) ys[tid] = mk<T>((T)S[L.y(tid)], (T)S[L.y(tid) + 1]);
  __syncthreads();
  const Grid& g = a.g;
  const long long off = (long long)rhs * g.vstride;
  double2* x = a.X + off;
  for (int s = blockIdx.x; s < a.ns; s += a.nbr) {
    const StripPos sp = strip_pos(a, s);
    if (sp.i > g.nx) continue;
    cx<T> acc[FR];
    int pr[FR];
#pragma unroll
    for (int r = 0; r < FR; ++r) {
      const int j = sp.j0 + r * FBY;
      pr[r] = j <= g.ny ? g.at(sp.i, j) : -1;
      acc[r] = mk<T>(T(0), T(0));
    }
    for (int q = 0; q < k; ++q) {
      const cx<T>* zq = (const cx<T>*)a.Z + q * a.vlen + off;
      const cx<T> y = ys[q];
#pragma unroll
      for (int r = 0; r < FR; ++r) {
        if (pr[r] < 0) continue;
        acc[r] = fma_c<T>(zq[pr[r]], y, acc[r]);
      }
    }
#pragma unroll
    for (int r = 0; r < FR; ++r)
      if (pr[r] >= 0) x[pr[r]] = add<double>(x[pr[r]], to_d(acc[r]));
  }
}

inline dim3 fg_grid(const FgArgs& a) { return dim3(a.nbr, 1, a.B); }

}  // namespace

void fg_geometry(const Grid& g, int B, bool fp64z, FgArgs& a) {
  a.ncx = cdiv(g.nx + 1, FBX);
  a.ns = a.ncx * cdiv(g.ny + 1, FBY * FR);
  int dev = 0, sms = 148, per = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (fp64z) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_fg_dots<double, false>, FTHREADS, 0);
  else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_fg_dots<float, false>, FTHREADS, 0);
  cudaGetLastError();
  per = per < 1 ? 1 : per;
  // about four waves of blocks over all right-hand sides
  const long long want = (4LL * sms * per + B - 1) / B;
  a.nbr = (int)std::max(1LL, std::min<long long>(want, a.ns));
  a.nvp = FNV;
}

template <class T> void launch_fg_restart(const FgArgs& a, cx<T>* cb, cx<T>* cxv, cudaStream_t s) {
  if (a.c0.abc2) k_fg_restart<T, true><<<fg_grid(a), dim3(FBX, FBY), 0, s>>>(a, cb, cxv);
  else k_fg_restart<T, false><<<fg_grid(a), dim3(FBX, FBY), 0, s>>>(a, cb, cxv);
}
template <class T> void launch_fg_dots(const FgArgs& a, int j, const cx<T>* z, cudaStream_t s) {
  if (a.c0.abc2) k_fg_dots<T, true><<<fg_grid(a), dim3(FBX, FBY), 0, s>>>(a, z, j);
  else k_fg_dots<T, false><<<fg_grid(a), dim3(FBX, FBY), 0, s>>>(a, z, j);
}
template <class T> void launch_fg_orth(const FgArgs& a, int j, cx<T>* cb, cx<T>* cxv, cudaStream_t s) {
  if (a.c0.abc2) k_fg_orth<T, true><<<fg_grid(a), dim3(FBX, FBY), 0, s>>>(a, j, cb, cxv);
  else k_fg_orth<T, false><<<fg_grid(a), dim3(FBX, FBY), 0, s>>>(a, j, cb, cxv);
}
template <class T> void launch_fg_update(const FgArgs& a, cudaStream_t s) {
  k_fg_update<T><<<fg_grid(a), dim3(FBX, FBY), 0, s>>>(a);
}

#define INST(T)                                                                                  \
  template void launch_fg_restart<T>(const FgArgs&, cx<T>*, cx<T>*, cudaStream_t);               \
  template void launch_fg_dots<T>(const FgArgs&, int, const cx<T>*, cudaStream_t);               \
  template void launch_fg_orth<T>(const FgArgs&, int, cx<T>*, cx<T>*, cudaStream_t);             \
  template void launch_fg_update<T>(const FgArgs&, cudaStream_t);
INST(double)
INST(float)
#undef INST

}  // namespace hmg
