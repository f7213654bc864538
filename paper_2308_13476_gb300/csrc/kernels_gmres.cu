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

#include "internal.h"

namespace hmg {

// Per-RHS scalar state, GS doubles each.
constexpr int GS = 96;
constexpr int G_BETA = 0;
constexpr int G_S = 1;      // s_0..s_3
constexpr int G_H = 8;      // Hbar[i][j] complex, i < 4, j < 3: 8 + 2*(i*3+j)
constexpr int G_G = 32;     // Gram <v_i, v_l> complex 4x4: 32 + 2*(i*4+l)
constexpr int G_Y = 64;     // y complex, 3
constexpr int G_M = 70;     // number of Arnoldi columns
constexpr int G_BRK = 71;   // 1 = stop (breakdown or beta == 0)
constexpr int NVMAX = 8;    // partial values per block

template <class T, class F>
static void with_op_g(const OpView<T>& v, int nx, int ny, F&& f) {
  if (v.kind == 1) {
    Op0<T> op{v.c0, v.kf, nx, ny};
    f(op);
  } else if (v.kind == 2) {
    OpS<T, 2> op{v.st, v.dinv, v.plane, nx, ny};
    f(op);
  } else {
    OpS<T, 3> op{v.st, v.dinv, v.plane, nx, ny};
    f(op);
  }
}

#define GNODE                                            \
  const int rhs = blockIdx.z;                            \
  const int i = blockIdx.x * BX + threadIdx.x;           \
  const int j = blockIdx.y * BY + threadIdx.y;           \
  const long long off = (long long)rhs * g.vstride;      \
  const long long blk = (long long)rhs * gridDim.x * gridDim.y + blockIdx.y * gridDim.x + blockIdx.x;

template <int NV>
__device__ __forceinline__ void store_partial(double (&v)[NV], double* sh, double* partial, long long blk) {
  block_sum<NV>(v, sh);
  if (threadIdx.x == 0 && threadIdx.y == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) partial[blk * NVMAX + k] = v[k];
  }
}

// u0 = b - A x, partial |u0|^2
template <class T, class Op>
__global__ void __launch_bounds__(BX * BY) g_init(Grid g, Op op, const cx<T>* __restrict__ x, const cx<T>* __restrict__ b,
                                                  cx<T>* __restrict__ u0, double* __restrict__ partial,
                                                  const int* __restrict__ active) {
  __shared__ double sh[NVMAX * 32];
  GNODE
  if (active && !active[rhs]) return;
  double v[1] = {0.0};
  if (i <= g.nx && j <= g.ny) {
    const long long p = g.at(i, j);
    const cx<T> r = sub<T>(b[off + p], op.apply(x + off, p, g.pitch, i, j));
    u0[off + p] = r;
    v[0] = (double)abs2<T>(r);
  }
  store_partial<1>(v, sh, partial, blk);
}

// w = A v_J (v_J = s_J u_J); partial dots <u_i, w> for i <= J
template <class T, class Op, int J>
__global__ void __launch_bounds__(BX * BY) g_arn_a(Grid g, Op op, const cx<T>* __restrict__ u0, const cx<T>* __restrict__ u1,
                                                   const cx<T>* __restrict__ u2, cx<T>* __restrict__ w,
                                                   const double* __restrict__ st, double* __restrict__ partial,
                                                   const int* __restrict__ active) {
  __shared__ double sh[NVMAX * 32];
  GNODE
  if (active && !active[rhs]) return;
  const double* S = st + (long long)rhs * GS;
  if (S[G_BRK] != 0.0 || S[G_M] < J) return;   // block-uniform
  const cx<T>* uJ = J == 0 ? u0 : (J == 1 ? u1 : u2);
  double v[2 * (J + 1)];
#pragma unroll
  for (int k = 0; k < 2 * (J + 1); ++k) v[k] = 0.0;
  if (i <= g.nx && j <= g.ny) {
    const long long p = g.at(i, j);
    const T sJ = (T)S[G_S + J];
    const cx<T> a = scl<T>(sJ, op.apply(uJ + off, p, g.pitch, i, j));
    w[off + p] = a;
    const cx<T>* us[3] = {u0, u1, u2};
#pragma unroll
    for (int l = 0; l <= J; ++l) {
      const cx<T> d = cmul<T>(us[l][off + p], a);
      v[2 * l] = (double)d.x;
      v[2 * l + 1] = (double)d.y;
    }
  }
  store_partial<2 * (J + 1)>(v, sh, partial, blk);
}

// u_{J+1} = w - sum_{i<=J} h_iJ s_i u_i ; partials |u_{J+1}|^2 and <u_{J+1}, u_l>, l <= J (J < 2)
template <class T, int J>
__global__ void __launch_bounds__(BX * BY) g_arn_b(Grid g, const cx<T>* __restrict__ u0, const cx<T>* __restrict__ u1,
                                                   const cx<T>* __restrict__ u2, cx<T>* __restrict__ un,
                                                   const cx<T>* __restrict__ w, const double* __restrict__ st,
                                                   double* __restrict__ partial, const int* __restrict__ active) {
  constexpr int NV = (J < 2) ? 1 + 2 * (J + 1) : 1;
  __shared__ double sh[NVMAX * 32];
  GNODE
  if (active && !active[rhs]) return;
  const double* S = st + (long long)rhs * GS;
  if (S[G_BRK] != 0.0 || S[G_M] < J) return;
  double v[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) v[k] = 0.0;
  if (i <= g.nx && j <= g.ny) {
    const long long p = g.at(i, j);
    const cx<T>* us[3] = {u0, u1, u2};
    cx<T> a = w[off + p];
    cx<T> uu[J + 1];
#pragma unroll
    for (int l = 0; l <= J; ++l) {
      uu[l] = us[l][off + p];
      const double hr = S[G_H + 2 * (l * 3 + J)], hi = S[G_H + 2 * (l * 3 + J) + 1];
      const double sl = S[G_S + l];
      const cx<T> c = mk<T>((T)(hr * sl), (T)(hi * sl));
      a = sub<T>(a, mul<T>(c, uu[l]));
    }
    un[off + p] = a;
    v[0] = (double)abs2<T>(a);
    if (J < 2) {
#pragma unroll
      for (int l = 0; l <= J && 1 + 2 * l + 1 < NV; ++l) {
        const cx<T> d = cmul<T>(a, uu[l]);
        v[1 + 2 * l] = (double)d.x;
        v[2 + 2 * l] = (double)d.y;
      }
    }
  }
  store_partial<NV>(v, sh, partial, blk);
}

// x += sum_{i<m} y_i s_i u_i
template <class T>
__global__ void __launch_bounds__(BX * BY) g_update(Grid g, cx<T>* __restrict__ x, const cx<T>* __restrict__ u0,
                                                    const cx<T>* __restrict__ u1, const cx<T>* __restrict__ u2,
                                                    const double* __restrict__ st, const int* __restrict__ active) {
  const int rhs = blockIdx.z;
  const int i = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y * BY + threadIdx.y;
  const long long off = (long long)rhs * g.vstride;
  if (active && !active[rhs]) return;
  if (i > g.nx || j > g.ny) return;
  const double* S = st + (long long)rhs * GS;
  const int m = (int)S[G_M];
  if (m <= 0) return;
  const long long p = off + g.at(i, j);
  const cx<T>* us[3] = {u0, u1, u2};
  cx<T> a = x[p];
#pragma unroll
  for (int l = 0; l < 3; ++l) {
    if (l < m) {
      const double sl = S[G_S + l];
      const cx<T> c = mk<T>((T)(S[G_Y + 2 * l] * sl), (T)(S[G_Y + 2 * l + 1] * sl));
      a = fma_c<T>(c, us[l][p], a);
    }
  }
  x[p] = a;
}

// ----------------------------------------------------------------- scalar kernels (one block per RHS)

template <int NV>
__device__ __forceinline__ void sum_partials(const double* partial, int nblk, int rhs, double (&v)[NV], double* sh) {
#pragma unroll
  for (int k = 0; k < NV; ++k) v[k] = 0.0;
  for (int b = threadIdx.x; b < nblk; b += blockDim.x) {
    const double* q = partial + ((long long)rhs * nblk + b) * NVMAX;
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] += q[k];
  }
  block_sum<NV>(v, sh);
}

__global__ void __launch_bounds__(256) g_fin_init(const double* __restrict__ partial, int nblk, double* __restrict__ st,
                                                  const int* __restrict__ active) {
  __shared__ double sh[NVMAX * 32];
  const int rhs = blockIdx.x;
  if (active && !active[rhs]) return;
  double v[1];
  sum_partials<1>(partial, nblk, rhs, v, sh);
  if (threadIdx.x == 0) {
    double* S = st + (long long)rhs * GS;
    for (int k = 0; k < GS; ++k) S[k] = 0.0;
    const double beta = sqrt(v[0]);
    S[G_BETA] = beta;
    S[G_M] = 0;
    if (beta == 0.0) {
      S[G_BRK] = 1.0;
    } else {
      S[G_S + 0] = 1.0 / beta;
    }
  }
}

template <int J>
__global__ void __launch_bounds__(256) g_fin_a(const double* __restrict__ partial, int nblk, double* __restrict__ st,
                                               const int* __restrict__ active) {
  __shared__ double sh[NVMAX * 32];
  const int rhs = blockIdx.x;
  if (active && !active[rhs]) return;
  double* S = st + (long long)rhs * GS;
  if (S[G_BRK] != 0.0 || S[G_M] < J) return;
  double v[2 * (J + 1)];
  sum_partials<2 * (J + 1)>(partial, nblk, rhs, v, sh);
  if (threadIdx.x == 0) {
    double hr[J + 1], hi[J + 1];
    for (int l = 0; l <= J; ++l) {
      // <v_l, w> = s_l <u_l, w>
      double dr = S[G_S + l] * v[2 * l], di = S[G_S + l] * v[2 * l + 1];
      for (int q = 0; q < l; ++q) {   // - sum_{q<l} h_q <v_l, v_q>
        const double gr = S[G_G + 2 * (l * 4 + q)], gi = S[G_G + 2 * (l * 4 + q) + 1];
        dr -= hr[q] * gr - hi[q] * gi;
        di -= hr[q] * gi + hi[q] * gr;
      }
      hr[l] = dr;
      hi[l] = di;
      S[G_H + 2 * (l * 3 + J)] = dr;
      S[G_H + 2 * (l * 3 + J) + 1] = di;
    }
  }
}

template <int J>
__global__ void __launch_bounds__(256) g_fin_b(const double* __restrict__ partial, int nblk, double* __restrict__ st,
                                               const int* __restrict__ active) {
  constexpr int NV = (J < 2) ? 1 + 2 * (J + 1) : 1;
  __shared__ double sh[NVMAX * 32];
  const int rhs = blockIdx.x;
  if (active && !active[rhs]) return;
  double* S = st + (long long)rhs * GS;
  if (S[G_BRK] != 0.0 || S[G_M] < J) return;
  double v[NV];
  sum_partials<NV>(partial, nblk, rhs, v, sh);
  if (threadIdx.x == 0) {
    const double hn = sqrt(v[0]);
    S[G_H + 2 * ((J + 1) * 3 + J)] = hn;
    S[G_H + 2 * ((J + 1) * 3 + J) + 1] = 0.0;
    S[G_M] = J + 1;
    if (hn <= 1e-14 * S[G_BETA]) {
      S[G_BRK] = 1.0;
    } else {
      const double sn = 1.0 / hn;
      S[G_S + J + 1] = sn;
      if (J < 2) {
        for (int l = 0; l <= J; ++l) {   // <v_{J+1}, v_l> = s_{J+1} s_l <u_{J+1}, u_l>
          S[G_G + 2 * ((J + 1) * 4 + l)] = sn * S[G_S + l] * v[1 + 2 * l];
          S[G_G + 2 * ((J + 1) * 4 + l) + 1] = sn * S[G_S + l] * v[2 + 2 * l];
        }
      }
    }
  }
}

// min || beta e1 - Hbar y || by Givens rotations; Hbar is (m+1) x m.
__global__ void g_lsq(double* __restrict__ st, int B, const int* __restrict__ active) {
  const int rhs = blockIdx.x * blockDim.x + threadIdx.x;
  if (rhs >= B) return;
  if (active && !active[rhs]) return;
  double* S = st + (long long)rhs * GS;
  const int m = (int)S[G_M];
  if (m <= 0) return;
  double Hr[4][3], Hi[4][3], gr[4], gi[4];
  for (int a = 0; a < 4; ++a) {
    gr[a] = gi[a] = 0.0;
    for (int c = 0; c < 3; ++c) {
      Hr[a][c] = S[G_H + 2 * (a * 3 + c)];
      Hi[a][c] = S[G_H + 2 * (a * 3 + c) + 1];
    }
  }
  gr[0] = S[G_BETA];
  for (int c = 0; c < m; ++c) {
    // rotation zeroing Hbar[c+1][c] against Hbar[c][c]
    const double ar = Hr[c][c], ai = Hi[c][c], br = Hr[c + 1][c], bi = Hi[c + 1][c];
    const double na = sqrt(ar * ar + ai * ai), nb = sqrt(br * br + bi * bi);
    const double nr = sqrt(na * na + nb * nb);
    if (nr == 0.0) continue;
    // G = [[cs, sn], [-conj(sn), cs]] with cs = |a|/r real, sn = (a/|a|) conj(b) / r
    double cs, snr, sni;
    if (na == 0.0) {
      cs = 0.0; snr = 1.0; sni = 0.0;
      // rows swap up to phase: sn = conj(b)/|b|
      snr = br / nb; sni = -bi / nb;
    } else {
      cs = na / nr;
      const double pr = ar / na, pi = ai / na;     // a/|a|
      snr = (pr * br + pi * bi) / nr;              // (a/|a|) * conj(b) / r
      sni = (pi * br - pr * bi) / nr;
    }
    for (int col = c; col < m; ++col) {
      const double xr = Hr[c][col], xi = Hi[c][col], yr = Hr[c + 1][col], yi = Hi[c + 1][col];
      // new_c = cs x + sn y ; new_{c+1} = -conj(sn) x + cs y
      Hr[c][col] = cs * xr + (snr * yr - sni * yi);
      Hi[c][col] = cs * xi + (snr * yi + sni * yr);
      Hr[c + 1][col] = -(snr * xr + sni * xi) + cs * yr;
      Hi[c + 1][col] = -(snr * xi - sni * xr) + cs * yi;
    }
    const double xr = gr[c], xi = gi[c], yr = gr[c + 1], yi = gi[c + 1];
    gr[c] = cs * xr + (snr * yr - sni * yi);
    gi[c] = cs * xi + (snr * yi + sni * yr);
    gr[c + 1] = -(snr * xr + sni * xi) + cs * yr;
    gi[c + 1] = -(snr * xi - sni * xr) + cs * yi;
  }
  double yr[3] = {0, 0, 0}, yi[3] = {0, 0, 0};
  for (int c = m - 1; c >= 0; --c) {
    double tr = gr[c], ti = gi[c];
    for (int q = c + 1; q < m; ++q) {
      tr -= Hr[c][q] * yr[q] - Hi[c][q] * yi[q];
      ti -= Hr[c][q] * yi[q] + Hi[c][q] * yr[q];
    }
    const double dr = Hr[c][c], di = Hi[c][c], dd = dr * dr + di * di;
    yr[c] = (tr * dr + ti * di) / dd;
    yi[c] = (ti * dr - tr * di) / dd;
  }
  for (int c = 0; c < 3; ++c) {
    S[G_Y + 2 * c] = c < m ? yr[c] : 0.0;
    S[G_Y + 2 * c + 1] = c < m ? yi[c] : 0.0;
  }
}

template <class T>
void gmres_smooth(const Grid& g, const OpView<T>& opv, cx<T>* x, const cx<T>* b, int nu, int B, const int* active,
                  const GmresBufs& gb, cudaStream_t s) {
  dim3 grd(cdiv(g.nx + 1, BX), cdiv(g.ny + 1, BY), B);
  const int nblk = grd.x * grd.y;
  cx<T>* u0 = (cx<T>*)gb.u[0];
  cx<T>* u1 = (cx<T>*)gb.u[1];
  cx<T>* u2 = (cx<T>*)gb.u[2];
  cx<T>* u3 = (cx<T>*)gb.u[3];
  cx<T>* w = (cx<T>*)gb.w;
  double* P = gb.partial;
  double* st = gb.st;
  with_op_g<T>(opv, g.nx, g.ny, [&](auto op) {
    using Op = decltype(op);
    for (int step = 0; step < nu; ++step) {
      g_init<T, Op><<<grd, dim3(BX, BY), 0, s>>>(g, op, x, b, u0, P, active);
      g_fin_init<<<B, 256, 0, s>>>(P, nblk, st, active);
      g_arn_a<T, Op, 0><<<grd, dim3(BX, BY), 0, s>>>(g, op, u0, u1, u2, w, st, P, active);
      g_fin_a<0><<<B, 256, 0, s>>>(P, nblk, st, active);
      g_arn_b<T, 0><<<grd, dim3(BX, BY), 0, s>>>(g, u0, u1, u2, u1, w, st, P, active);
      g_fin_b<0><<<B, 256, 0, s>>>(P, nblk, st, active);
      g_arn_a<T, Op, 1><<<grd, dim3(BX, BY), 0, s>>>(g, op, u0, u1, u2, w, st, P, active);
      g_fin_a<1><<<B, 256, 0, s>>>(P, nblk, st, active);
      g_arn_b<T, 1><<<grd, dim3(BX, BY), 0, s>>>(g, u0, u1, u2, u2, w, st, P, active);
      g_fin_b<1><<<B, 256, 0, s>>>(P, nblk, st, active);
      g_arn_a<T, Op, 2><<<grd, dim3(BX, BY), 0, s>>>(g, op, u0, u1, u2, w, st, P, active);
      g_fin_a<2><<<B, 256, 0, s>>>(P, nblk, st, active);
      g_arn_b<T, 2><<<grd, dim3(BX, BY), 0, s>>>(g, u0, u1, u2, u3, w, st, P, active);
      g_fin_b<2><<<B, 256, 0, s>>>(P, nblk, st, active);
      g_lsq<<<cdiv(B, 64), 64, 0, s>>>(st, B, active);
      g_update<T><<<grd, dim3(BX, BY), 0, s>>>(g, x, u0, u1, u2, st, active);
    }
  });
}

template void gmres_smooth<double>(const Grid&, const OpView<double>&, double2*, const double2*, int, int, const int*,
                                   const GmresBufs&, cudaStream_t);
template void gmres_smooth<float>(const Grid&, const OpView<float>&, float2*, const float2*, int, int, const int*,
                                  const GmresBufs&, cudaStream_t);

}  // namespace hmg
