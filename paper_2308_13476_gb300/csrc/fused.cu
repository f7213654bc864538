// Shared-memory halo-tile kernels that fuse steps of the cycle:
//
//  * k_resid_restrict: r_c = R (b - A x) in one pass.  A block owns a tile
//    of CTX x CTY coarse nodes; it computes the fine residual on the tile's
//    fine footprint plus the 2-node halo the restriction needs (Eq. (xex)
//    transposed: fine offsets -2..2 around node 2I) into shared memory, then
//    every thread restricts one coarse node from it.  The fine residual never
//    goes to HBM.  How the footprint residual is formed depends on the
//    operator: the matrix-free fine level takes a fixed, unrolled set of
//    nodes per thread; the Kronecker-form levels (complex64) form their row
//    sums once per footprint row and combine them along y; the stored
//    stencils (and complex128 Kronecker levels) apply the operator per node.
//  * k_jacobi_fused: nu weighted-Jacobi sweeps (Sec. 3) of the fine level in
//    one pass.  A block loads its tile of x with a nu-node halo and of b
//    with a (nu-1)-node halo once, runs the sweeps in shared memory on a
//    region that shrinks by one node per sweep, and writes the tile.  Nodes
//    outside the grid stay zero (they are not unknowns); nodes computed in
//    two tiles' halos get identical values, so the result equals nu separate
//    sweeps node for node.
#include <type_traits>

#include "internal.h"
#include "ragged.cuh"
#include "ragged_api.h"

namespace hmg {

constexpr int CTX = 32, CTY = 8;                  // coarse tile of k_resid_restrict
constexpr int RFX = 2 * CTX + 3, RFY = 2 * CTY + 3;  // fine footprint incl. restriction halo

// radius of a Kronecker-form operator, 0 for the others
template <class Op> struct KronRadius { static constexpr int R = 0; };
template <class T, int R_> struct KronRadius<OpK<T, R_>> { static constexpr int R = R_; };

// Arguments of the residual-restriction for one problem (flattened ragged launches).
template <class T, class Op>
struct RrA {
  Grid gf;
  Grid gc;
  Op op;
  const cx<T>* x;
  const cx<T>* b;
  cx<T>* rc;
  const int* active;
  Xfer xw;
};

template <class T, class Op>
__device__ __forceinline__ void k_resid_restrict_body(uint3 vblk, dim3 vgrid, Grid gf, Grid gc, Op op, const cx<T>* __restrict__ x, const cx<T>* __restrict__ b, cx<T>* __restrict__ rc, const int* __restrict__ active, Xfer xw) {
  const uint3 blockIdx = vblk;   // the block and grid inside this problem's launch
  const dim3 gridDim = vgrid;
  (void)blockIdx;
  (void)gridDim;
  __shared__ cx<T> rt[RFY][RFX];
  const int rhs = blockIdx.z;
  if (active && !active[rhs]) return;
  const cx<T>* xs = x + (long long)rhs * gf.vstride;
  const cx<T>* bs = b + (long long)rhs * gf.vstride;
  const int I0 = blockIdx.x * CTX, J0 = blockIdx.y * CTY;
  const int fx0 = 2 * I0 - 2, fy0 = 2 * J0 - 2;   // fine origin of the footprint
  const int tid = threadIdx.y * CTX + threadIdx.x;
  if constexpr (std::is_same<Op, Op0<T>>::value || std::is_same<Op, Op0<T, true>>::value) {
    // matrix-free fine level: a fixed, unrolled count of footprint nodes per
    // thread, each evaluated at its node clamped into the grid (every load is
    // in bounds and unconditional, so the loads of all of them can be in
    // flight together) and replaced by zero outside the grid
    constexpr int NQ = (RFX * RFY + CTX * CTY - 1) / (CTX * CTY);
#pragma unroll
    for (int k = 0; k < NQ; ++k) {
      const int q = tid + k * CTX * CTY;
      if (k + 1 < NQ || q < RFX * RFY) {
        const int li = q % RFX, lj = q / RFX;
        const int i = fx0 + li, j = fy0 + lj;
        const int ic = min(max(i, 0), gf.nx), jc = min(max(j, 0), gf.ny);
        const int p = gf.at(ic, jc);
        const cx<T> r = sub<T>(bs[p], op.apply(xs, p, gf.pitch, ic, jc));
        const bool in = i == ic && j == jc;
        rt[lj][li] = in ? r : mk<T>(0, 0);   // outside the grid the fine residual is zero
      }
    }
  } else if constexpr (KronRadius<Op>::R > 0 && sizeof(T) == 4) {
    // Kronecker form A = W_y (x) G_x + H_y (x) W_x (complex64): the two row
    // sums s1 = G_x x and s2 = W_x x of every footprint column are formed
    // once per row (rows fy0 - R .. fy0 + RFY - 1 + R) into shared memory,
    // and each footprint node combines the 2R + 1 rows around it along y.
    // The sums and the combination run in the order of OpK::apply, so every
    // residual is the same value; the work per node drops from 6 (2R+1)^2
    // to about 12 (2R+1) FMAs, and each thread loads the operator's
    // coefficients of one column (row) once.
    constexpr int KR = KronRadius<Op>::R, K = 2 * KR + 1, SR = RFY + 2 * KR;
    constexpr int NT = CTX * CTY;
    __shared__ cx<T> s1t[SR][RFX], s2t[SR][RFX];
    // row sums: a thread keeps one footprint column (and its column's x
    // coefficients in registers) and takes every CG-th row
    constexpr int CG = NT / RFX;
    if (tid < CG * RFX) {
      const int li = tid % RFX, i = fx0 + li;
      const bool icol = i >= 0 && i <= gf.nx;
      cx<T> G[K];
      T Wx[K];
#pragma unroll
      for (int k = 0; k < K; ++k) {
        G[k] = icol ? op.gx[i * K + k] : mk<T>(0, 0);
        Wx[k] = icol ? op.wx[i * K + k] : T(0);
      }
#pragma unroll
      for (int kk = 0; kk < (SR + CG - 1) / CG; ++kk) {   // a fixed trip count: the loads of all rows in flight together
        const int lr = tid / RFX + kk * CG;
        if (lr >= SR) break;
        const int j = fy0 - KR + lr;
        cx<T> a = mk<T>(0, 0), c = mk<T>(0, 0);   // unused outside the grid's columns and their row halo
        if (icol && j >= -KR && j <= gf.ny + KR) {
          const cx<T>* row = xs + gf.at(i, j);
#pragma unroll
          for (int dx = -KR; dx <= KR; ++dx) {
            const cx<T> xv = row[dx];
            a = fma_c<T>(G[dx + KR], xv, a);
            c = mk<T>(fma(Wx[dx + KR], xv.x, c.x), fma(Wx[dx + KR], xv.y, c.y));
          }
        }
        s1t[lr][li] = a;
        s2t[lr][li] = c;
      }
    }
    __syncthreads();
    // combination along y: a thread keeps one footprint row (and its row's y
    // coefficients in registers, the parameter bank's copy for the
    // translation-invariant interior rows) and takes every RG-th column
    constexpr int RG = NT / RFY;
    if (tid < RG * RFY) {
      const int lj = tid % RFY, j = fy0 + lj;
      const bool jrow = j >= 0 && j <= gf.ny;
      cx<T> H[K];
      T Wy[K];
      const bool inv = j >= op.ty0 && j < op.ty1;
#pragma unroll
      for (int k = 0; k < K; ++k) {
        H[k] = inv ? op.hyc[k] : jrow ? op.hy[j * K + k] : mk<T>(0, 0);
        Wy[k] = inv ? op.wyc[k] : jrow ? op.wy[j * K + k] : T(0);
      }
#pragma unroll
      for (int kk = 0; kk < (RFX + RG - 1) / RG; ++kk) {
        const int li = tid / RFY + kk * RG;
        if (li >= RFX) break;
        const int i = fx0 + li;
        cx<T> r = mk<T>(0, 0);   // outside the grid the fine residual is zero
        if (jrow && i >= 0 && i <= gf.nx) {
          cx<T> acc = mk<T>(0, 0);
#pragma unroll
          for (int dy = -KR; dy <= KR; ++dy) {
            const cx<T> a = s1t[lj + KR + dy][li], c = s2t[lj + KR + dy][li];
            acc = mk<T>(fma(Wy[dy + KR], a.x, acc.x), fma(Wy[dy + KR], a.y, acc.y));
            acc = fma_c<T>(H[dy + KR], c, acc);
          }
          r = sub<T>(bs[gf.at(i, j)], acc);
        }
        rt[lj][li] = r;
      }
    }
  } else {
    for (int q = tid; q < RFX * RFY; q += CTX * CTY) {
      const int li = q % RFX, lj = q / RFX;
      const int i = fx0 + li, j = fy0 + lj;
      cx<T> r = mk<T>(0, 0);   // outside the grid the fine residual is zero
      if (i >= 0 && i <= gf.nx && j >= 0 && j <= gf.ny) {
        const int p = gf.at(i, j);
        r = sub<T>(bs[p], op.apply(xs, p, gf.pitch, i, j));
      }
      rt[lj][li] = r;
    }
  }
  __syncthreads();
  const int I = I0 + threadIdx.x, J = J0 + threadIdx.y;
  if (I > gc.nx || J > gc.ny) return;
  const int ci = 2 * threadIdx.x + 2, cj = 2 * threadIdx.y + 2;   // fine node 2I in the tile
  cx<T> acc = mk<T>(0, 0);
#pragma unroll
  for (int bb = -2; bb <= 2; ++bb) {
    const cx<T>* row = &rt[cj + bb][ci];
    cx<T> t = scl<T>(T(xw.w2), add<T>(row[-2], row[2]));
    t = add<T>(t, scl<T>(T(xw.w1), add<T>(row[-1], row[1])));
    t = add<T>(t, scl<T>(T(xw.w0), row[0]));
    acc = add<T>(acc, scl<T>(xw.w<T>(bb), t));
  }
  rc[(long long)rhs * gc.vstride + gc.at(I, J)] = scl<T>(T(0.25), acc);
}

template <class T, class Op>
__global__ void __launch_bounds__(CTX * CTY) k_resid_restrict(Grid gf, Grid gc, Op op, const cx<T>* __restrict__ x, const cx<T>* __restrict__ b, cx<T>* __restrict__ rc, const int* __restrict__ active, Xfer xw) {
  k_resid_restrict_body<T, Op>(blockIdx, gridDim, gf, gc, op, x, b, rc, active, xw);
}

template <class T, class Op>
__global__ void __launch_bounds__(CTX * CTY) k_resid_restrict_rag(const __grid_constant__ RagLaunch<RrA<T, Op>> L) {
  uint3 vb;
  dim3 vg;
  const RrA<T, Op>& a = L.a[rag_problem(L, blockIdx.x, vb, vg)];
  k_resid_restrict_body<T, Op>(vb, vg, a.gf, a.gc, a.op, a.x, a.b, a.rc, a.active, a.xw);
}

constexpr int JTX = 64, JTY = 16;        // output tile of k_jacobi_fused
constexpr int JMAXNU = 4;                // sweeps fused in one launch (more: several launches)

template <class T, bool A2 = false>
__global__ void __launch_bounds__(256) k_jacobi_fused(Grid g, Op0<T, A2> op, const cx<T>* __restrict__ x,
                                                      const cx<T>* __restrict__ b, cx<T>* __restrict__ xo, int nu,
                                                      const int* __restrict__ active) {
  extern __shared__ unsigned char smem_raw[];
  const int rhs = blockIdx.z;
  if (active && !active[rhs]) return;
  const int H = nu;                                 // halo of x
  const int WX = JTX + 2 * H, WY = JTY + 2 * H;
  cx<T>* A = reinterpret_cast<cx<T>*>(smem_raw);   // x, ping
  cx<T>* Bf = A + WX * WY;                          // x, pong
  cx<T>* Bt = Bf + WX * WY;                         // b on the same window
  const cx<T>* xs = x + (long long)rhs * g.vstride;
  const cx<T>* bs = b + (long long)rhs * g.vstride;
  const int i0 = blockIdx.x * JTX - H, j0 = blockIdx.y * JTY - H;   // window origin
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int q = tid; q < WX * WY; q += nt) {
    const int li = q % WX, lj = q / WX, i = i0 + li, j = j0 + lj;
    const bool in = i >= 0 && i <= g.nx && j >= 0 && j <= g.ny;
    const int p = in ? g.at(i, j) : 0;
    A[q] = in ? xs[p] : mk<T>(0, 0);
    Bt[q] = in ? bs[p] : mk<T>(0, 0);
    Bf[q] = mk<T>(0, 0);
  }
  __syncthreads();
  cx<T>* src = A;
  cx<T>* dst = Bf;
  for (int s = 1; s <= nu; ++s) {
    // sweep s is valid on the window shrunk by s nodes
    const int lo = s, hix = WX - 1 - s, hiy = WY - 1 - s;
    const int w = hix - lo + 1, hgt = hiy - lo + 1;
    for (int q = tid; q < w * hgt; q += nt) {
      const int li = lo + q % w, lj = lo + q / w, i = i0 + li, j = j0 + lj;
      const int c = lj * WX + li;
      if (i < 0 || i > g.nx || j < 0 || j > g.ny) {
        dst[c] = mk<T>(0, 0);
        continue;
      }
      const cx<T> ax = op.apply5(src[c], src[c + 1], src[c - 1], src[c + WX], src[c - WX], i, j);
      dst[c] = fma_c<T>(op.diag_inv(i, j), sub<T>(Bt[c], ax), src[c]);
    }
    __syncthreads();
    cx<T>* t = src;
    src = dst;
    dst = t;
  }
  cx<T>* xd = xo + (long long)rhs * g.vstride;
  for (int q = tid; q < JTX * JTY; q += nt) {
    const int li = H + q % JTX, lj = H + q / JTX, i = i0 + li, j = j0 + lj;
    if (i <= g.nx && j <= g.ny) xd[g.at(i, j)] = src[lj * WX + li];
  }
}

template <class T>
void launch_resid_restrict(const Grid& gf, const Grid& gc, const OpView<T>& v, const cx<T>* x, const cx<T>* b,
                           cx<T>* rc, int B, const int* active, const Xfer& xw, cudaStream_t s) {
  const dim3 grd(cdiv(gc.nx + 1, CTX), cdiv(gc.ny + 1, CTY), B);
  with_op<T>(v, gf.nx, gf.ny, [&](auto op) {
    k_resid_restrict<T, decltype(op)><<<grd, dim3(CTX, CTY), 0, s>>>(gf, gc, op, x, b, rc, active, xw);
  });
}

template <class T> size_t jacobi_fused_smem(int nu) {
  return sizeof(cx<T>) * 3 * (size_t)(JTX + 2 * nu) * (JTY + 2 * nu);
}

template <class T>
void launch_jacobi_fused(const Grid& g, const OpView<T>& v, const cx<T>* x, const cx<T>* b, cx<T>* xo, int nu, int B,
                         const int* active, cudaStream_t s) {
  const dim3 grd(cdiv(g.nx + 1, JTX), cdiv(g.ny + 1, JTY), B);
  if (v.c0.abc2)
    k_jacobi_fused<T, true><<<grd, 256, jacobi_fused_smem<T>(nu), s>>>(g, Op0<T, true>{v.c0, v.kf, g.nx, g.ny}, x, b, xo,
                                                                       nu, active);
  else
    k_jacobi_fused<T><<<grd, 256, jacobi_fused_smem<T>(nu), s>>>(g, Op0<T>{v.c0, v.kf, g.nx, g.ny}, x, b, xo, nu, active);
}

int jacobi_fused_max_nu() { return JMAXNU; }

cudaError_t configure_fused_kernels() {   // allow the complex128 window (> 48 KiB) on the current device
  cudaError_t e = cudaFuncSetAttribute(k_jacobi_fused<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)jacobi_fused_smem<double>(JMAXNU));
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_jacobi_fused<double, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)jacobi_fused_smem<double>(JMAXNU));
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_jacobi_fused<float, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)jacobi_fused_smem<float>(JMAXNU));
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_jacobi_fused<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)jacobi_fused_smem<float>(JMAXNU));
}

template <class T>
void launch_resid_restrict_rag(const std::vector<RagXfer<T>>& v, const Xfer& xw, cudaStream_t s) {
  if (v.empty()) return;
  const RagXfer<T>& v0 = v[0];
  with_op<T>(v0.op, v0.gf.nx, v0.gf.ny, [&](auto op0) {   // the problems' levels at one depth share the operator kind
    using Op = decltype(op0);
    rag_launch<RrA<T, Op>>((int)v.size(), k_resid_restrict_rag<T, Op>, dim3(CTX, CTY), 0, s,
                           [&](int q, RrA<T, Op>& a, int& gx, int& gy) {
                             const RagXfer<T>& X = v[q];
                             Op op = op0;
                             with_op<T>(X.op, X.gf.nx, X.gf.ny, [&](auto o) {
                               if constexpr (std::is_same<decltype(o), Op>::value) op = o;
                             });
                             a = RrA<T, Op>{X.gf, X.gc, op, X.x, X.b, X.rc, X.active, xw};
                             gx = cdiv(X.gc.nx + 1, CTX);
                             gy = cdiv(X.gc.ny + 1, CTY);
                             return true;
                           });
  });
}

template void launch_resid_restrict_rag<double>(const std::vector<RagXfer<double>>&, const Xfer&, cudaStream_t);
template void launch_resid_restrict_rag<float>(const std::vector<RagXfer<float>>&, const Xfer&, cudaStream_t);
template void launch_resid_restrict<double>(const Grid&, const Grid&, const OpView<double>&, const double2*,
                                            const double2*, double2*, int, const int*, const Xfer&, cudaStream_t);
template void launch_resid_restrict<float>(const Grid&, const Grid&, const OpView<float>&, const float2*,
                                           const float2*, float2*, int, const int*, const Xfer&, cudaStream_t);
template void launch_jacobi_fused<double>(const Grid&, const OpView<double>&, const double2*, const double2*,
                                          double2*, int, int, const int*, cudaStream_t);
template void launch_jacobi_fused<float>(const Grid&, const OpView<float>&, const float2*, const float2*, float2*,
                                         int, int, const int*, cudaStream_t);

}  // namespace hmg
