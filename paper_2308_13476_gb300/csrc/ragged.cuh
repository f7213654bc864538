// One launch of a kernel over the problems of a ragged batch.
//
// A ragged batch holds independent problems of different sizes.  Launching
// every kernel once per problem costs one launch per kernel, level and
// problem.  Here the blocks of all problems' launches of one kernel are
// numbered one after the other in a single 1D grid: block b belongs to the
// problem p with b0[p] <= b < b0[p + 1], found by binary search, and runs the
// kernel body with its block index inside that problem's own launch (grid
// gx[p] x gy[p] x 1).  The per-problem arguments travel by value in the
// parameter bank (a __grid_constant__ struct), at most RMAXP problems per
// launch; larger batches take several launches.
//
// The kernel bodies are written as kernels: they read blockIdx and gridDim.
// A body function takes the block index and the grid it should see and
// declares them under those names, so the same body text serves the plain
// launch (with the real values) and the flattened one.
#pragma once
#include "common.cuh"

namespace hmg {

constexpr int RMAXP = 32;

template <class A> struct RagLaunch {
  int np;
  int b0[RMAXP + 1];          // first flattened block of each problem; b0[np] = all blocks
  int gx[RMAXP], gy[RMAXP];   // each problem's own grid
  A a[RMAXP];                 // each problem's kernel arguments
};

// The problem of flattened block `bid`, and the block's index and grid
// inside that problem's launch.
template <class A>
__device__ __forceinline__ int rag_problem(const RagLaunch<A>& L, int bid, uint3& blk, dim3& grd) {
  int lo = 0, hi = L.np - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (L.b0[mid] <= bid) lo = mid;
    else hi = mid - 1;
  }
  const int loc = bid - L.b0[lo], gx = L.gx[lo];
  blk = make_uint3(loc % gx, loc / gx, 0);
  grd = dim3(gx, L.gy[lo], 1);
  return lo;
}

// Host side: fills the block offsets of a launch from the problems' grids
// and returns the number of flattened blocks.
template <class A> inline int rag_finish(RagLaunch<A>& L) {
  int b = 0;
  for (int p = 0; p < L.np; ++p) {
    L.b0[p] = b;
    b += L.gx[p] * L.gy[p];
  }
  L.b0[L.np] = b;
  return b;
}

// Launches kern once per group of at most RMAXP problems.  fill(q, a, gx, gy)
// sets problem q's arguments and grid (gy = 1 if untouched) and returns
// false to leave the problem out; problems without blocks are left out.
template <class A, class K, class F>
inline void rag_launch(int n, K kern, dim3 block, size_t smem, cudaStream_t s, F&& fill) {
  static thread_local RagLaunch<A> L;   // large: kept off the stack
  for (int q0 = 0; q0 < n; q0 += RMAXP) {
    L.np = 0;
    for (int q = q0; q < n && q < q0 + RMAXP; ++q) {
      int gx = 0, gy = 1;
      if (!fill(q, L.a[L.np], gx, gy) || gx <= 0 || gy <= 0) continue;
      L.gx[L.np] = gx;
      L.gy[L.np] = gy;
      ++L.np;
    }
    if (!L.np) continue;
    const int tot = rag_finish(L);
    kern<<<tot, block, smem, s>>>(L);
  }
}

}  // namespace hmg
