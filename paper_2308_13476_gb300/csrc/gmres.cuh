// Scalar part of the GMRES(3) smoother (Sec. 5.3 of the paper), shared by
// the grid-wide kernels and the single-CTA coarse-cycle interpreter: the
// per-RHS state layout, the Hessenberg updates of one Arnoldi step (modified
// Gram-Schmidt written with the Gram matrix of the basis) and the FP64 Givens
// least-squares solve.  Each function runs in one thread.
#pragma once
#include "common.cuh"

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


// min || beta e1 - Hbar y || by Givens rotations; Hbar is (m+1) x m.  The
// arithmetic runs in Ts (FP64 for the complex128 path, FP32 for the
// complex64 cycles of the mixed path); the state S is stored in St: FP64 in
// global memory, or Ts where one thread block owns the state (every stored
// value is a Ts value, so both storages give the same results).  The summed
// inputs v of the fin_* steps come in V: FP64 from the grid-wide sums, Ts
// from the block sums of the coarse-cycle interpreter.
template <class Ts, class St = double> __device__ __forceinline__ void lsq(St* S) {
  const int m = (int)S[G_M];
  if (m <= 0) return;
  Ts Hr[4][3], Hi[4][3], gr[4], gi[4];
  for (int a = 0; a < 4; ++a) {
    gr[a] = gi[a] = Ts(0);
    for (int c = 0; c < 3; ++c) {
      Hr[a][c] = (Ts)S[G_H + 2 * (a * 3 + c)];
      Hi[a][c] = (Ts)S[G_H + 2 * (a * 3 + c) + 1];
    }
  }
  gr[0] = (Ts)S[G_BETA];
  for (int c = 0; c < m; ++c) {
    // rotation zeroing Hbar[c+1][c] against Hbar[c][c]:
    // G = [[cs, sn], [-conj(sn), cs]], cs = |a|/r real, sn = (a/|a|) conj(b) / r
    const Ts ar = Hr[c][c], ai = Hi[c][c], br = Hr[c + 1][c], bi = Hi[c + 1][c];
    const Ts na = sqrt(ar * ar + ai * ai), nb = sqrt(br * br + bi * bi);
    const Ts nr = sqrt(na * na + nb * nb);
    if (nr == Ts(0)) continue;
    Ts cs, snr, sni;
    if (na == Ts(0)) {
      cs = Ts(0);
      snr = br / nb;
      sni = -bi / nb;
    } else {
      cs = na / nr;
      const Ts pr = ar / na, pi = ai / na;
      snr = (pr * br + pi * bi) / nr;
      sni = (pi * br - pr * bi) / nr;
    }
    for (int col = c; col < m; ++col) {
      const Ts xr = Hr[c][col], xi = Hi[c][col], yr = Hr[c + 1][col], yi = Hi[c + 1][col];
      Hr[c][col] = cs * xr + (snr * yr - sni * yi);
      Hi[c][col] = cs * xi + (snr * yi + sni * yr);
      Hr[c + 1][col] = -(snr * xr + sni * xi) + cs * yr;
      Hi[c + 1][col] = -(snr * xi - sni * xr) + cs * yi;
    }
    const Ts xr = gr[c], xi = gi[c], yr = gr[c + 1], yi = gi[c + 1];
    gr[c] = cs * xr + (snr * yr - sni * yi);
    gi[c] = cs * xi + (snr * yi + sni * yr);
    gr[c + 1] = -(snr * xr + sni * xi) + cs * yr;
    gi[c + 1] = -(snr * xi - sni * xr) + cs * yi;
  }
  Ts yr[3] = {0, 0, 0}, yi[3] = {0, 0, 0};
  for (int c = m - 1; c >= 0; --c) {
    Ts tr = gr[c], ti = gi[c];
    for (int q = c + 1; q < m; ++q) {
      tr -= Hr[c][q] * yr[q] - Hi[c][q] * yi[q];
      ti -= Hr[c][q] * yi[q] + Hi[c][q] * yr[q];
    }
    const Ts dr = Hr[c][c], di = Hi[c][c], dd = dr * dr + di * di;
    yr[c] = (tr * dr + ti * di) / dd;
    yi[c] = (ti * dr - tr * di) / dd;
  }
  for (int c = 0; c < 3; ++c) {
    S[G_Y + 2 * c] = c < m ? (St)yr[c] : St(0);
    S[G_Y + 2 * c + 1] = c < m ? (St)yi[c] : St(0);
  }
}

// ---- scalar steps of one Arnoldi pass, run by one thread ----

template <class Ts, class St = double, class V = double> __device__ __forceinline__ void fin_init(St* S, const V* v) {
  for (int k = 0; k < GS; ++k) S[k] = St(0);
  const Ts beta = sqrt((Ts)v[0]);
  S[G_BETA] = (St)beta;
  S[G_M] = St(0);
  if (beta == Ts(0)) S[G_BRK] = St(1);
  else S[G_S + 0] = (St)(Ts(1) / beta);
}

// h_lJ = <v_l, w> - sum_{q<l} h_qJ <v_l, v_q>, with <v_l, w> = s_l <u_l, w>
template <int J, class Ts, class St = double, class V = double> __device__ __forceinline__ void fin_a(St* S, const V* v) {
  Ts hr[J + 1], hi[J + 1];
  for (int l = 0; l <= J; ++l) {
    const Ts sl = (Ts)S[G_S + l];
    Ts dr = sl * (Ts)v[2 * l], di = sl * (Ts)v[2 * l + 1];
    for (int q = 0; q < l; ++q) {
      const Ts gr = (Ts)S[G_G + 2 * (l * 4 + q)], gi = (Ts)S[G_G + 2 * (l * 4 + q) + 1];
      dr -= hr[q] * gr - hi[q] * gi;
      di -= hr[q] * gi + hi[q] * gr;
    }
    hr[l] = dr;
    hi[l] = di;
    S[G_H + 2 * (l * 3 + J)] = (St)dr;
    S[G_H + 2 * (l * 3 + J) + 1] = (St)di;
  }
}

// h_{J+1,J} = ||u_{J+1}||, breakdown test, Gram entries of v_{J+1}; the least
// squares problem is solved once the Arnoldi process stops.
template <int J, class Ts, class St = double, class V = double> __device__ __forceinline__ void fin_b(St* S, const V* v) {
  const Ts hn = sqrt((Ts)v[0]);
  S[G_H + 2 * ((J + 1) * 3 + J)] = (St)hn;
  S[G_H + 2 * ((J + 1) * 3 + J) + 1] = St(0);
  S[G_M] = St(J + 1);
  if (hn <= Ts(1e-14) * (Ts)S[G_BETA]) {
    S[G_BRK] = St(1);
  } else {
    const Ts sn = Ts(1) / hn;
    S[G_S + J + 1] = (St)sn;
    if (J < 2) {
      for (int l = 0; l <= J; ++l) {   // <v_{J+1}, v_l> = s_{J+1} s_l <u_{J+1}, u_l>
        const Ts f = sn * (Ts)S[G_S + l];
        S[G_G + 2 * ((J + 1) * 4 + l)] = (St)(f * (Ts)v[1 + 2 * l]);
        S[G_G + 2 * ((J + 1) * 4 + l) + 1] = (St)(f * (Ts)v[2 + 2 * l]);
      }
    }
  }
  if (J == 2 || S[G_BRK] != St(0)) lsq<Ts, St>(S);
}

// fin_b<2> with |u3|^2 from the Gram form: u3 = A v2 - sum_{l<=2} h_l2 v_l
// with unit v_l, and each modified Gram-Schmidt step removes |h_l2|^2 from
// the squared norm, so |u3|^2 = |A v2|^2 - sum_l |h_l2|^2 (aw2 = |A v2|^2).
// Computed in FP64; a cancellation to zero or below is a breakdown.
template <class Ts, class St = double> __device__ __forceinline__ void fin_b2_gram(St* S, double aw2) {
  double r = aw2;
  for (int l = 0; l <= 2; ++l) {
    const double hr = (double)S[G_H + 2 * (l * 3 + 2)], hi = (double)S[G_H + 2 * (l * 3 + 2) + 1];
    r -= hr * hr + hi * hi;
  }
  const double v[1] = {r > 0.0 ? r : 0.0};
  fin_b<2, Ts, St>(S, v);
}

// The per-RHS state in global memory: GS values of the cycle's working
// precision T per right-hand side (the scalar steps compute in T and store T
// values, so FP32 storage gives what FP64 storage would; kernels of a
// complex64 cycle then read their coefficients without FP64 instructions).
template <class T> __device__ __forceinline__ T* gstate(double* st, int rhs) {
  return reinterpret_cast<T*>(st) + (long long)rhs * GS;
}
template <class T> __device__ __forceinline__ const T* gstate(const double* st, int rhs) {
  return reinterpret_cast<const T*>(st) + (long long)rhs * GS;
}

// Runs a scalar step on the RHS state in shared memory (all threads of the
// block copy it in and out; thread 0 computes), so its many dependent reads
// and writes stay on chip.
template <class T, class St, class F>
__device__ __forceinline__ void staged(St* S, const double* v, F f) {
  __shared__ St Ssh[GS];
  const int tid = threadIdx.x + threadIdx.y * blockDim.x, nt = blockDim.x * blockDim.y;
  for (int k = tid; k < GS; k += nt) Ssh[k] = S[k];
  __syncthreads();
  if (tid == 0) f(Ssh, v);
  __syncthreads();
  for (int k = tid; k < GS; k += nt) S[k] = Ssh[k];
}

}  // namespace hmg
