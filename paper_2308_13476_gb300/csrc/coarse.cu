// Single-CTA coarse-cycle interpreter.
//
// The levels of the hierarchy with few nodes (all levels from `lc` down to
// the coarsest grid) cost almost nothing in arithmetic but, launched as
// separate grid-wide kernels, dozens of launches per level and cycle.  Here
// one CTA per right-hand side runs the whole sub-cycle below level lc-1:
// the host records the V/W schedule of those levels once (the same
// recursion as the grid-wide driver, Sec. 3 of the paper) as a list of
// steps, and the kernel walks it, with a __syncthreads() between dependent
// phases.  Every step computes exactly what the grid-wide kernels compute:
// the same stencils, the same Jacobi sweep, the same GMRES(3) arithmetic
// (gmres.cuh), the same transfers of Eq. (xex) and the same FP64 coarsest
// solve; only the reductions are block-wide instead of grid-wide.
#include <algorithm>

#include "gmres.cuh"
#include "internal.h"
#include "ragged.cuh"
#include "ragged_api.h"
#include "levelops.cuh"

namespace hmg {

// Node loop over one level: q -> (i, j, p).
#define CTA_NODES(L)                                                         \
  for (int q = tid, n1_ = (L).g.nx + 1, nn_ = n1_ * ((L).g.ny + 1); q < nn_; q += nt)
#define CTA_IJP(L)                 \
  const int i = q % n1_;           \
  const int j = q / n1_;           \
  const int p = (L).g.at(i, j);

// Block-wide sum in the working precision T: a shuffle tree within each warp,
// then one over the warps' sums in warp 0.  Fixed shape and order
// (reproducible); with T = float the interpreter's reductions issue no FP64
// instructions (the FP64 pipe is narrow and its latency would sit on the
// interpreter's serial path).  out is valid in thread 0.
template <int NV, class T>
__device__ __forceinline__ void cta_sum(const T (&v)[NV], T* sh /* [NV][32] */, T (&out)[NV]) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    T t = v[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    if (lane == 0) sh[k * 32 + warp] = t;
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      T t = lane < nwarps ? sh[k * 32 + lane] : T(0);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
      out[k] = t;
    }
  }
}

// Arnoldi step J of GMRES(3) inside one CTA: w = s_J A u_J, the Gram-form
// MGS coefficients (fin_a), u_{J+1} = w - sum_l h_lJ v_l and its norm and
// Gram entries (fin_b).  The per-RHS state S lives in shared memory in the
// working precision T, and the block sums run in T (cta_sum): with T = float
// the interpreter's GMRES(3) issues no FP64 instruction.  Returns false, block-uniformly, once the Arnoldi process has
// stopped (breakdown, or fewer than J columns).
template <int J, class T>
__device__ __forceinline__ bool cta_arnoldi(const CLevel<T>& L, cx<T>* const (&u)[3], cx<T>* w, T* S, double* sh) {
  const int tid = threadIdx.x, nt = blockDim.x;
  if (S[G_BRK] != T(0) || S[G_M] < T(J)) return false;   // uniform: shared state after a barrier
  const T sJ = S[G_S + J];
  constexpr int ND = 2 * (J + 1);
  T dt[ND];
#pragma unroll
  for (int l = 0; l < ND; ++l) dt[l] = T(0);
  CTA_NODES(L) {
    CTA_IJP(L)
    const cx<T> a = scl<T>(sJ, lv_apply<T>(L, u[J], p, i, j));
    w[p] = a;
#pragma unroll
    for (int l = 0; l <= J; ++l) {
      const cx<T> e = cmul<T>(u[l][p], a);
      dt[2 * l] += e.x;
      dt[2 * l + 1] += e.y;
    }
  }
  {
    T d[ND];
    cta_sum<ND, T>(dt, reinterpret_cast<T*>(sh), d);
    if (tid == 0) fin_a<J, T, T, T>(S, d);
    __syncthreads();
  }
  cx<T> c[J + 1];
#pragma unroll
  for (int l = 0; l <= J; ++l) {
    const T sl = S[G_S + l];
    c[l] = mk<T>(S[G_H + 2 * (l * 3 + J)] * sl, S[G_H + 2 * (l * 3 + J) + 1] * sl);
  }
  constexpr int NE = J < 2 ? 1 + 2 * (J + 1) : 1;
  T et[NE];
#pragma unroll
  for (int l = 0; l < NE; ++l) et[l] = T(0);
  CTA_NODES(L) {
    CTA_IJP(L)
    cx<T> a = w[p];
    cx<T> uu[J + 1];
#pragma unroll
    for (int l = 0; l <= J; ++l) {
      uu[l] = u[l][p];
      a = sub<T>(a, mul<T>(c[l], uu[l]));
    }
    et[0] += abs2<T>(a);
    if constexpr (J < 2) {
      u[J + 1][p] = a;
#pragma unroll
      for (int l = 0; l <= J; ++l) {
        const cx<T> e = cmul<T>(a, uu[l]);
        et[1 + 2 * l] += e.x;
        et[2 + 2 * l] += e.y;
      }
    }
  }
  {
    T e[NE];
    cta_sum<NE, T>(et, reinterpret_cast<T*>(sh), e);
    if (tid == 0) fin_b<J, T, T, T>(S, e);
    __syncthreads();
  }
  return true;
}

template <class T>
__device__ void cta_gmres(const CLevel<T>& L, cx<T>* x, long long off, int nu, T* S, double* sh) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const cx<T>* b = L.b + off;
  cx<T>* const u[3] = {L.u[0] + off, L.u[1] + off, L.u[2] + off};
  cx<T>* w = L.w + off;
  for (int step = 0; step < nu; ++step) {
    T a0[1] = {T(0)};
    CTA_NODES(L) {
      CTA_IJP(L)
      const cx<T> r = sub<T>(b[p], lv_apply<T>(L, x, p, i, j));
      u[0][p] = r;
      a0[0] += abs2<T>(r);
    }
    {
      T t[1];
      cta_sum<1, T>(a0, reinterpret_cast<T*>(sh), t);
      if (tid == 0) fin_init<T, T, T>(S, t);
      __syncthreads();
    }
    if (cta_arnoldi<0, T>(L, u, w, S, sh) && cta_arnoldi<1, T>(L, u, w, S, sh)) cta_arnoldi<2, T>(L, u, w, S, sh);
    const int m = (int)S[G_M];
    if (m > 0) {
      cx<T> c[3];
#pragma unroll
      for (int l = 0; l < 3; ++l) {
        const T sl = S[G_S + l];
        c[l] = mk<T>(S[G_Y + 2 * l] * sl, S[G_Y + 2 * l + 1] * sl);
      }
      CTA_NODES(L) {
        CTA_IJP(L)
        cx<T> a = x[p];
#pragma unroll
        for (int l = 0; l < 3; ++l)
          if (l < m) a = fma_c<T>(c[l], u[l][p], a);
        x[p] = a;
      }
    }
    __syncthreads();
  }
}

template <class T>
__device__ __forceinline__ void k_coarse_cycle_body(uint3 vblk, dim3 vgrid, const CLevel<T>* __restrict__ levels, const CStep* __restrict__ steps, int nsteps, const double2* __restrict__ inv, int N, const int* __restrict__ active) {
  const uint3 blockIdx = vblk;   // the block and grid inside this problem's launch
  const dim3 gridDim = vgrid;
  (void)blockIdx;
  (void)gridDim;
  extern __shared__ double2 rs[];            // coarsest right-hand side, N entries
  __shared__ double sh[NVMAX * 32];
  __shared__ T S[GS];
  const int rhs = blockIdx.x;
  if (active && !active[rhs]) return;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int s = 0; s < nsteps; ++s) {
    const CStep st = steps[s];
    const CLevel<T>& L = levels[st.level];
    const long long off = (long long)rhs * L.g.vstride;
    cx<T>* p0 = (cx<T>*)st.p0 + off;
    switch (st.op) {
      case C_JACOBI: {   // p1 = p0 + (omega diag A)^-1 (b - A p0)
        cx<T>* p1 = (cx<T>*)st.p1 + off;
        const cx<T>* b = L.b + off;
        CTA_NODES(L) {
          CTA_IJP(L)
          const cx<T> r = sub<T>(b[p], lv_apply<T>(L, p0, p, i, j));
          p1[p] = fma_c<T>(lv_dinv<T>(L, i, j), r, p0[p]);
        }
        __syncthreads();
        break;
      }
      case C_GMRES:
        cta_gmres<T>(L, p0, off, st.arg, S, sh);
        break;
      case C_RESTRICT: {  // r = b - A p0 on this level, then b_{l+1} = R r
        cx<T>* r = L.r + off;
        const cx<T>* b = L.b + off;
        CTA_NODES(L) {
          CTA_IJP(L)
          r[p] = sub<T>(b[p], lv_apply<T>(L, p0, p, i, j));
        }
        __syncthreads();
        const CLevel<T>& C = levels[st.level + 1];
        cx<T>* bc = C.b + (long long)rhs * C.g.vstride;
        CTA_NODES(C) {
          CTA_IJP(C)
          const int pc = L.g.at(2 * i, 2 * j);
          cx<T> acc = mk<T>(0, 0);
          for (int bb = -2; bb <= 2; ++bb) {
            const cx<T>* row = r + pc + bb * L.g.pitch;
            cx<T> t = scl<T>(T(L.xw.w2), add<T>(row[-2], row[2]));
            t = add<T>(t, scl<T>(T(L.xw.w1), add<T>(row[-1], row[1])));
            t = add<T>(t, scl<T>(T(L.xw.w0), row[0]));
            acc = add<T>(acc, scl<T>(L.xw.template w<T>(bb), t));
          }
          bc[p] = scl<T>(T(0.25), acc);
        }
        __syncthreads();
        break;
      }
      case C_ZERO: {
        CTA_NODES(L) {
          CTA_IJP(L)
          p0[p] = mk<T>(0, 0);
        }
        __syncthreads();
        break;
      }
      case C_COARSE: {   // p0 = A_c^{-1} b, FP64
        const cx<T>* b = L.b + off;
        CTA_NODES(L) {
          CTA_IJP(L)
          const cx<T> a = b[p];
          rs[q] = make_double2((double)a.x, (double)a.y);
        }
        __syncthreads();
        CTA_NODES(L) {
          CTA_IJP(L)
          double2 acc = make_double2(0, 0);
          const double2* row = inv + (long long)q * N;
          for (int c2 = 0; c2 < N; ++c2) acc = fma_c<double>(row[c2], rs[c2], acc);
          p0[p] = mk<T>((T)acc.x, (T)acc.y);
        }
        __syncthreads();
        break;
      }
      case C_PROLONG: {  // p0 += P p1 (p1 on level + 1)
        const CLevel<T>& C = levels[st.level + 1];
        const cx<T>* ec = (const cx<T>*)st.p1 + (long long)rhs * C.g.vstride;
        CTA_NODES(L) {
          CTA_IJP(L)
          const int I = i >> 1, J = j >> 1;
          auto rowval = [&](int JJ) -> cx<T> {
            const cx<T>* row = ec + C.g.at(I, JJ);
            if (i & 1) return scl<T>(T(L.xw.w1), add<T>(row[0], row[1]));
            return add<T>(scl<T>(T(L.xw.w2), add<T>(row[-1], row[1])), scl<T>(T(L.xw.w0), row[0]));
          };
          cx<T> v;
          if (j & 1) v = scl<T>(T(L.xw.w1), add<T>(rowval(J), rowval(J + 1)));
          else v = add<T>(scl<T>(T(L.xw.w2), add<T>(rowval(J - 1), rowval(J + 1))), scl<T>(T(L.xw.w0), rowval(J)));
          p0[p] = add<T>(p0[p], v);
        }
        __syncthreads();
        break;
      }
      default: {   // C_COPY p1 = p0
        cx<T>* p1 = (cx<T>*)st.p1 + off;
        CTA_NODES(L) {
          CTA_IJP(L)
          p1[p] = p0[p];
        }
        __syncthreads();
        break;
      }
    }
  }
}

template <class T>
__global__ void __launch_bounds__(CTA_THREADS) k_coarse_cycle(const CLevel<T>* __restrict__ levels, const CStep* __restrict__ steps, int nsteps, const double2* __restrict__ inv, int N, const int* __restrict__ active) {
  k_coarse_cycle_body<T>(blockIdx, gridDim, levels, steps, nsteps, inv, N, active);
}

template <class T>
__global__ void __launch_bounds__(CTA_THREADS) k_coarse_cycle_rag(const __grid_constant__ RagLaunch<RagCoarse<T>> L) {
  uint3 vb;
  dim3 vg;
  const RagCoarse<T>& a = L.a[rag_problem(L, blockIdx.x, vb, vg)];
  k_coarse_cycle_body<T>(vb, vg, a.levels, a.steps, a.nsteps, a.inv, a.N, a.active);
}

template <class T>
void launch_coarse_cycle(const CLevel<T>* levels, const CStep* steps, int nsteps, const double2* inv, int N, int B,
                         const int* active, cudaStream_t s) {
  k_coarse_cycle<T><<<B, CTA_THREADS, (size_t)N * sizeof(double2), s>>>(levels, steps, nsteps, inv, N, active);
}

// One CTA per problem of a ragged batch, each walking its own plan.
template <class T> void launch_coarse_cycle_rag(const std::vector<RagCoarse<T>>& v, cudaStream_t s) {
  int nmax = 0;
  for (const auto& c : v) nmax = std::max(nmax, c.N);
  rag_launch<RagCoarse<T>>((int)v.size(), k_coarse_cycle_rag<T>, dim3(CTA_THREADS), (size_t)nmax * sizeof(double2), s,
                           [&](int q, RagCoarse<T>& a, int& gx, int&) {
                             a = v[q];
                             gx = 1;
                             return true;
                           });
}
template void launch_coarse_cycle_rag<double>(const std::vector<RagCoarse<double>>&, cudaStream_t);
template void launch_coarse_cycle_rag<float>(const std::vector<RagCoarse<float>>&, cudaStream_t);

template void launch_coarse_cycle<double>(const CLevel<double>*, const CStep*, int, const double2*, int, int,
                                          const int*, cudaStream_t);
template void launch_coarse_cycle<float>(const CLevel<float>*, const CStep*, int, const double2*, int, int,
                                         const int*, cudaStream_t);

}  // namespace hmg
