// Cooperative multi-CTA cycle interpreter.
//
// One persistent cooperative launch walks the host-recorded V/W schedule of
// the levels lc..L-1 (the same steps as the single-CTA interpreter of
// coarse.cu, the same recursion as the grid-wide driver, Sec. 3 of the
// paper), with every block of the GPU working on every step: the blocks are
// split evenly over the right-hand sides (bpr blocks per RHS) and phases are
// separated by a grid-wide barrier instead of kernel boundaries.  A norm or
// dot-product reduction is a block sum per block, a barrier, and then every
// block of the RHS summing the bpr block sums itself in the same fixed order,
// so all of them hold bitwise-identical scalars (the GMRES(3) state lives in
// each block's shared memory) and no second barrier or broadcast is needed.
//
// Every block passes the same barriers in the same order whatever its work
// (idle blocks, converged right-hand sides, an Arnoldi breakdown): only the
// work inside a phase is skipped.  Each barrier wait is bounded; a block that
// gives up sets the error word and every block leaves at its next barrier,
// so a lost block can delay but never hang the launch.
#include "gmres.cuh"
#include "internal.h"
#include "levelops.cuh"

namespace hmg {

// Grid-wide barrier of a cooperative launch on a monotonic arrival counter:
// barrier number n completes when the counter reaches n * gridDim.x.  Each
// block adds one arrival and polls the counter (acquire loads), at most
// spin_limit polls.  Returns false (all threads) once any block has given up.
// The counter is zeroed before every solve.
__device__ __forceinline__ bool grid_sync(const CoopCtl& c) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned nb = gridDim.x;
    __threadfence();
    const unsigned old = atomicAdd(c.bar, 1u);
    const unsigned target = (old / nb + 1u) * nb;
    int ok = 1;
    long long it = 0;
    while (true) {
      unsigned cur;
      asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(cur) : "l"(c.bar) : "memory");
      if ((int)(cur - target) >= 0) break;
      if (++it > c.spin_limit) {
        atomicExch(c.err, 1);
        ok = 0;
        break;
      }
    }
    __threadfence();
    s_ok = ok && *(volatile int*)c.err == 0;
  }
  __syncthreads();
  return s_ok != 0;
}

// Block partial -> barrier -> every block of the RHS sums the bpr partials of
// its RHS in block order.  tot valid in all threads afterwards.
template <int NV>
__device__ __forceinline__ bool coop_reduce(double (&v)[NV], double* sh, double* tot_sh, const CoopCtl& c, bool work,
                                            int rhs, int part, int bpr) {
  if (work) {
    block_sum<NV>(v, sh);
    if (threadIdx.x == 0) {
      double* q = c.partial + ((long long)rhs * bpr + part) * NVMAX;
      for (int k = 0; k < NV; ++k) q[k] = v[k];
    }
  }
  if (!grid_sync(c)) return false;
  if (work) {
    double a[NV];
    for (int k = 0; k < NV; ++k) a[k] = 0.0;
    for (int p = threadIdx.x; p < bpr; p += blockDim.x) {
      const double* q = c.partial + ((long long)rhs * bpr + p) * NVMAX;
      for (int k = 0; k < NV; ++k) a[k] += __ldcg(q + k);
    }
    block_sum<NV>(a, sh);
    if (threadIdx.x == 0)
      for (int k = 0; k < NV; ++k) tot_sh[k] = a[k];
    __syncthreads();
  }
  return true;
}

#define COOP_NODES(L)\
  for (int q = part * nt + tid, n1_ = (L).g.nx + 1, nn_ = n1_ * ((L).g.ny + 1); q < nn_; q += stride)
#define COOP_IJP(L)     \
  const int i = q % n1_;\
  const int j = q / n1_;\
  const int p = (L).g.at(i, j);

template <class T>
__device__ bool coop_gmres(const CLevel<T>& L, cx<T>* x, long long off, int nu, double* S, double* sh, double* tot,
                           const CoopCtl& c, bool work, int rhs, int part, int bpr) {
  const int tid = threadIdx.x, nt = blockDim.x, stride = bpr * nt;
  const cx<T>* b = L.b + off;
  cx<T>* u[3] = {L.u[0] + off, L.u[1] + off, L.u[2] + off};
  cx<T>* w = L.w + off;
  for (int step = 0; step < nu; ++step) {
    {
      T a0 = T(0);
      if (work) {
        COOP_NODES(L) {
          COOP_IJP(L)
          const cx<T> r = sub<T>(b[p], lv_apply<T>(L, x, p, i, j));
          u[0][p] = r;
          a0 += abs2<T>(r);
        }
      }
      double v[1] = {(double)a0};
      if (!coop_reduce<1>(v, sh, tot, c, work, rhs, part, bpr)) return false;
      if (work && tid == 0) fin_init<T>(S, tot);
      __syncthreads();
    }
    for (int J = 0; J < 3; ++J) {
      // every block runs both phases of every J; work is skipped after a breakdown
      const bool go = work && S[G_BRK] == 0.0 && S[G_M] >= J;
      T dt[6] = {0, 0, 0, 0, 0, 0};
      if (go) {
        const T sJ = (T)S[G_S + J];
        COOP_NODES(L) {
          COOP_IJP(L)
          const cx<T> a = scl<T>(sJ, lv_apply<T>(L, u[J], p, i, j));
          w[p] = a;
          for (int l = 0; l <= J; ++l) {
            const cx<T> e = cmul<T>(u[l][p], a);
            dt[2 * l] += e.x;
            dt[2 * l + 1] += e.y;
          }
        }
      }
      double d[6];
      for (int l = 0; l < 6; ++l) d[l] = (double)dt[l];
      if (!coop_reduce<6>(d, sh, tot, c, go, rhs, part, bpr)) return false;
      if (go && tid == 0) {
        if (J == 0) fin_a<0, T>(S, tot);
        else if (J == 1) fin_a<1, T>(S, tot);
        else fin_a<2, T>(S, tot);
      }
      __syncthreads();
      T et[5] = {0, 0, 0, 0, 0};
      if (go) {
        cx<T> cf[3];
        for (int l = 0; l < 3; ++l) {
          const double sl = S[G_S + l];
          cf[l] = l <= J ? mk<T>((T)(S[G_H + 2 * (l * 3 + J)] * sl), (T)(S[G_H + 2 * (l * 3 + J) + 1] * sl))
                         : mk<T>(0, 0);
        }
        COOP_NODES(L) {
          COOP_IJP(L)
          cx<T> a = w[p];
          cx<T> uu[3];
          for (int l = 0; l <= J; ++l) {
            uu[l] = u[l][p];
            a = sub<T>(a, mul<T>(cf[l], uu[l]));
          }
          if (J < 2) u[J + 1][p] = a;
          et[0] += abs2<T>(a);
          if (J < 2)
            for (int l = 0; l <= J; ++l) {
              const cx<T> e = cmul<T>(a, uu[l]);
              et[1 + 2 * l] += e.x;
              et[2 + 2 * l] += e.y;
            }
        }
      }
      double e5[5];
      for (int l = 0; l < 5; ++l) e5[l] = (double)et[l];
      if (!coop_reduce<5>(e5, sh, tot, c, go, rhs, part, bpr)) return false;
      if (go && tid == 0) {
        if (J == 0) fin_b<0, T>(S, tot);
        else if (J == 1) fin_b<1, T>(S, tot);
        else fin_b<2, T>(S, tot);
      }
      __syncthreads();
    }
    const int m = work ? (int)S[G_M] : 0;
    if (m > 0) {
      cx<T> cf[3];
      for (int l = 0; l < 3; ++l) {
        const double sl = S[G_S + l];
        cf[l] = mk<T>((T)(S[G_Y + 2 * l] * sl), (T)(S[G_Y + 2 * l + 1] * sl));
      }
      COOP_NODES(L) {
        COOP_IJP(L)
        cx<T> a = x[p];
        for (int l = 0; l < 3; ++l)
          if (l < m) a = fma_c<T>(cf[l], u[l][p], a);
        x[p] = a;
      }
    }
    if (!grid_sync(c)) return false;
  }
  return true;
}

template <class T>
__global__ void __launch_bounds__(COOP_THREADS) k_cycle_coop(const CLevel<T>* __restrict__ levels,
                                                            const CStep* __restrict__ steps, int nsteps,
                                                            const double2* __restrict__ inv, int N,
                                                            const int* __restrict__ active, int B, int bpr,
                                                            int nlev, CoopCtl c) {
  extern __shared__ double2 rs[];   // coarsest right-hand side, N entries
  __shared__ double sh[NVMAX * 32];
  __shared__ double S[GS];
  __shared__ double tot[NVMAX];
  __shared__ CLevel<T> lvs[COOP_MAXLEV];   // level descriptors, read once
  for (int q = threadIdx.x; q < nlev * (int)(sizeof(CLevel<T>) / 8); q += blockDim.x)
    reinterpret_cast<long long*>(lvs)[q] = reinterpret_cast<const long long*>(levels)[q];
  __syncthreads();
  const int slot = blockIdx.x;
  const bool has = slot < B * bpr;
  const int rhs = has ? slot / bpr : 0, part = has ? slot % bpr : 0;
  const bool work = has && (active == nullptr || active[rhs] != 0);
  const int tid = threadIdx.x, nt = blockDim.x, stride = bpr * nt;
  for (int s = 0; s < nsteps; ++s) {
    const CStep st = steps[s];
    const CLevel<T>& L = lvs[st.level];
    const long long off = (long long)rhs * L.g.vstride;
    cx<T>* p0 = (cx<T>*)st.p0 + off;
    bool ok = true;
    switch (st.op) {
      case C_JACOBI: {
        if (work) {
          cx<T>* p1 = (cx<T>*)st.p1 + off;
          const cx<T>* b = L.b + off;
          COOP_NODES(L) {
            COOP_IJP(L)
            const cx<T> r = sub<T>(b[p], lv_apply<T>(L, p0, p, i, j));
            p1[p] = fma_c<T>(lv_dinv<T>(L, i, j), r, p0[p]);
          }
        }
        ok = grid_sync(c);
        break;
      }
      case C_GMRES:
        ok = coop_gmres<T>(L, p0, off, st.arg, S, sh, tot, c, work, rhs, part, bpr);
        break;
      case C_RESTRICT: {
        cx<T>* r = L.r + off;
        if (work) {
          const cx<T>* b = L.b + off;
          COOP_NODES(L) {
            COOP_IJP(L)
            r[p] = sub<T>(b[p], lv_apply<T>(L, p0, p, i, j));
          }
        }
        if (!(ok = grid_sync(c))) break;
        const CLevel<T>& C = lvs[st.level + 1];
        if (work) {
          cx<T>* bc = C.b + (long long)rhs * C.g.vstride;
          COOP_NODES(C) {
            COOP_IJP(C)
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
        }
        ok = grid_sync(c);
        break;
      }
      case C_ZERO: {
        if (work) {
          COOP_NODES(L) {
            COOP_IJP(L)
            p0[p] = mk<T>(0, 0);
          }
        }
        ok = grid_sync(c);
        break;
      }
      case C_COARSE: {   // p0 = A_c^{-1} b (FP64), rows split over the RHS's blocks
        if (work) {
          const cx<T>* b = L.b + off;
          for (int q = tid, n1_ = L.g.nx + 1; q < N; q += nt) {
            const int i = q % n1_, j = q / n1_;
            const cx<T> a = b[L.g.at(i, j)];
            rs[q] = make_double2((double)a.x, (double)a.y);
          }
          __syncthreads();
          for (int q = part * nt + tid, n1_ = L.g.nx + 1; q < N; q += stride) {
            double2 acc = make_double2(0, 0);
            const double2* row = inv + (long long)q * N;
            for (int c2 = 0; c2 < N; ++c2) acc = fma_c<double>(row[c2], rs[c2], acc);
            const int i = q % n1_, j = q / n1_;
            p0[L.g.at(i, j)] = mk<T>((T)acc.x, (T)acc.y);
          }
        }
        ok = grid_sync(c);
        break;
      }
      case C_PROLONG: {
        if (work) {
          const CLevel<T>& C = lvs[st.level + 1];
          const cx<T>* ec = (const cx<T>*)st.p1 + (long long)rhs * C.g.vstride;
          COOP_NODES(L) {
            COOP_IJP(L)
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
        }
        ok = grid_sync(c);
        break;
      }
      default: {   // C_COPY
        if (work) {
          cx<T>* p1 = (cx<T>*)st.p1 + off;
          COOP_NODES(L) {
            COOP_IJP(L)
            p1[p] = p0[p];
          }
        }
        ok = grid_sync(c);
        break;
      }
    }
    if (!ok) return;
  }
}

template <class T> int coop_max_blocks(int N) {
  int dev = 0, sms = 0, per = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_cycle_coop<T>, COOP_THREADS, (size_t)N * sizeof(double2)) !=
      cudaSuccess)
    return 0;
  return sms * per;
}

template <class T>
cudaError_t launch_cycle_coop(const CLevel<T>* levels, int nlev, const CStep* steps, int nsteps, const double2* inv,
                              int N, const int* active, int B, int grid, const CoopCtl& c, cudaStream_t s) {
  const int bpr = grid / B;
  void* args[] = {(void*)&levels, (void*)&steps, (void*)&nsteps, (void*)&inv, (void*)&N,
                  (void*)&active, (void*)&B, (void*)&bpr, (void*)&nlev, (void*)&c};
  return cudaLaunchCooperativeKernel((const void*)k_cycle_coop<T>, dim3(grid), dim3(COOP_THREADS), args,
                                     (size_t)N * sizeof(double2), s);
}

template int coop_max_blocks<double>(int);
template int coop_max_blocks<float>(int);
template cudaError_t launch_cycle_coop<double>(const CLevel<double>*, int, const CStep*, int, const double2*, int,
                                               const int*, int, int, const CoopCtl&, cudaStream_t);
template cudaError_t launch_cycle_coop<float>(const CLevel<float>*, int, const CStep*, int, const double2*, int,
                                              const int*, int, int, const CoopCtl&, cudaStream_t);

}  // namespace hmg
