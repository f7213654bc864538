// Shared device definitions of the helmmg library: padded grid layout,
// complex arithmetic, the two operator kinds (matrix-free fine level, stored
// Galerkin stencils) and deterministic block reductions.
//
// Layout of every grid vector: one (ny+1) x (nx+1) grid per right-hand side,
// stored row-major with a zero halo of HALO nodes on every side, rows of
// `pitch` elements (nx+1+2*HALO rounded up to a multiple of 4), RHS after RHS
// `vstride` elements apart.  The halo is zero-filled at allocation and never
// written, so stencils and transfers read neighbours without bounds tests.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace hmg {

constexpr int HALO = 4;
constexpr int BX = 32;   // block shape of the node-parallel kernels
constexpr int BY = 8;
constexpr int RYMAX = 4; // largest number of grid rows per thread (Grid::ry)
constexpr int MAXR = 3;  // largest Galerkin stencil radius (7 x 7)
constexpr int NVMAX = 12; // values per block partial record

template <class T> struct cvec;
template <> struct cvec<double> { using type = double2; };
template <> struct cvec<float> { using type = float2; };
template <class T> using cx = typename cvec<T>::type;

template <class T> __host__ __device__ __forceinline__ cx<T> mk(T re, T im) {
  cx<T> r; r.x = re; r.y = im; return r;
}
template <class T> __device__ __forceinline__ cx<T> add(cx<T> a, cx<T> b) { return mk<T>(a.x + b.x, a.y + b.y); }
template <class T> __device__ __forceinline__ cx<T> sub(cx<T> a, cx<T> b) { return mk<T>(a.x - b.x, a.y - b.y); }
template <class T> __device__ __forceinline__ cx<T> scl(T s, cx<T> a) { return mk<T>(s * a.x, s * a.y); }
template <class T> __device__ __forceinline__ cx<T> mul(cx<T> a, cx<T> b) {
  return mk<T>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a + b*c
template <class T> __device__ __forceinline__ cx<T> fma_c(cx<T> b, cx<T> c, cx<T> a) {
  return mk<T>(fma(b.x, c.x, fma(-b.y, c.y, a.x)), fma(b.x, c.y, fma(b.y, c.x, a.y)));
}
// conj(a) * b
template <class T> __device__ __forceinline__ cx<T> cmul(cx<T> a, cx<T> b) {
  return mk<T>(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
template <class T> __device__ __forceinline__ T abs2(cx<T> a) { return a.x * a.x + a.y * a.y; }

// Packed complex64 arithmetic: one .f32x2 instruction of the FP32 pipe for
// both components, each rounded as by the scalar instruction (so add2, sub2,
// mul2 and fma2 give the bits of the scalar add, sub, mul and fma).
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
  float2 d;
  asm("{\n .reg .b64 pa, pb, pd;\n mov.b64 pa, {%2, %3};\n mov.b64 pb, {%4, %5};\n"
      " sub.rn.f32x2 pd, pa, pb;\n mov.b64 {%0, %1}, pd;\n}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
}
__device__ __forceinline__ float2 bc2(float s) { return make_float2(s, s); }

// a - b; complex64 in one packed instruction
template <class T> __device__ __forceinline__ cx<T> psub(cx<T> a, cx<T> b) {
  if constexpr (sizeof(T) == 4) return sub2(a, b);
  else return sub<T>(a, b);
}

// s a - sum_l c_l v_l (the Arnoldi vector of a pass).  complex64: the real
// parts of the coefficients scale v_l in one packed accumulator and the
// imaginary parts in another, which are joined once (packed instructions
// need no component swap that way); complex128 in the scalar order.
template <class T, int L>
__device__ __forceinline__ cx<T> scl_minus(T s, cx<T> a, const cx<T> (&c)[L], const cx<T> (&v)[L]) {
  if constexpr (sizeof(T) == 4) {
    float2 p = mul2(bc2(s), a), q = mul2(bc2(c[0].y), v[0]);
    p = fma2(bc2(-c[0].x), v[0], p);
#pragma unroll
    for (int l = 1; l < L; ++l) {
      p = fma2(bc2(-c[l].x), v[l], p);
      q = fma2(bc2(c[l].y), v[l], q);
    }
    return make_float2(p.x + q.y, p.y - q.x);
  } else {
    cx<T> u = sub<T>(scl<T>(s, a), mul<T>(c[0], v[0]));
#pragma unroll
    for (int l = 1; l < L; ++l) u = sub<T>(u, mul<T>(c[l], v[l]));
    return u;
  }
}

// IEEE 754 conversions between binary64 and binary32 in integer arithmetic.
// The hardware conversions execute on the FP64 pipe, which is narrow on this
// GPU and is what bounds the FP64 refinement passes; these take the integer
// pipe for normal numbers and give the same results: binary64 to binary32
// rounds to nearest, ties to even (the fraction keeps its 23 leading bits and
// the 29 dropped bits decide the rounding; a carry out of the fraction raises
// the exponent, up to infinity), and binary32 to binary64 is exact (the
// exponent rebiased by 1023 - 127, the fraction shifted into place).  Zeros,
// subnormal inputs or results, infinities and NaNs take the hardware
// conversion.
__device__ __forceinline__ float f32_from_f64_rn(double d) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(d);
  const unsigned hi = (unsigned)(u >> 32);
  const int e = (int)((hi >> 20) & 0x7ffu) - (1023 - 127);   // biased binary32 exponent
  if (e >= 1 && e <= 254) {
    const unsigned long long frac = u & 0x000fffffffffffffull;
    unsigned f = ((unsigned)e << 23) | (unsigned)(frac >> 29);
    const unsigned rem = (unsigned)frac & 0x1fffffffu;
    f += (unsigned)(rem > 0x10000000u) | ((unsigned)(rem == 0x10000000u) & f & 1u);
    return __uint_as_float((hi & 0x80000000u) | f);
  }
  return __double2float_rn(d);
}
__device__ __forceinline__ double f64_from_f32(float v) {
  const unsigned u = __float_as_uint(v);
  const unsigned e = (u >> 23) & 0xffu;
  if (e - 1u < 254u) {   // normal
    const unsigned long long r = ((unsigned long long)(u & 0x80000000u) << 32) |
                                 ((unsigned long long)(e + (1023 - 127)) << 52) |
                                 ((unsigned long long)(u & 0x007fffffu) << 29);
    return __longlong_as_double((long long)r);
  }
  return (double)v;
}
template <class T> __device__ __forceinline__ cx<T> cinv(cx<T> a) {
  T d = a.x * a.x + a.y * a.y;
  return mk<T>(a.x / d, -a.y / d);
}
template <class T, class U> __device__ __forceinline__ cx<T> cvt(cx<U> a) {
  return mk<T>((T)a.x, (T)a.y);
}

// Geometry of one level's padded vectors.
struct Grid {
  int nx, ny;          // interval counts; nodes 0..nx, 0..ny
  int pitch;           // padded row length (elements)
  int rows;            // padded row count
  long long vstride;   // elements per right-hand side
  int ry;              // grid rows per thread of the node kernels (1..RYMAX):
                       // a block covers BX x (BY * ry) nodes
  // offset of node (i, j) inside one right-hand side's slice (< 2^31)
  __host__ __device__ __forceinline__ int at(int i, int j) const { return (j + HALO) * pitch + (i + HALO); }
};

// Inter-grid transfer in one direction as the column stencil of P: coarse
// node I reaches fine node 2I + d with weight w(d).  Eq. (xex) (the paper's
// higher-order transfer) gives w(0) = 3/4, w(+-1) = 1/2, w(+-2) = 1/8;
// linear interpolation (the "Linear" column of Table conv1) gives 1, 1/2, 0.
// 2D transfers are the tensor product, and R = P^T / 4.
struct Xfer {
  double w0, w1, w2;
  template <class T> __host__ __device__ __forceinline__ T w(int d) const {
    return d == 0 ? T(w0) : (d == 1 || d == -1) ? T(w1) : (d == 2 || d == -2) ? T(w2) : T(0);
  }
};
// kind 0: Eq. (xex); kind 1: linear interpolation.
inline Xfer xfer_of(int kind) { return kind == 1 ? Xfer{1.0, 0.5, 0.0} : Xfer{0.75, 0.5, 0.125}; }

// Fine-level (level 0) constants, computed on the device by the setup kernel
// and passed to the kernels by value (copied back once at setup).
// dinv[by*2+bx] = 1/(omega * A_PP) for constant k and the four boundary
// classes (bx = node on a vertical boundary line, by = on a horizontal one).
// abc2 = 1: the second-order absorbing rows (a variant the paper does not
// use, below), ih3q = 1 / (4 h^3), tang = 1 / (2 k h^3).
template <class T> struct Op0Consts {
  T inv_h2, inv_h, k, k2, omega, beta2;
  cx<T> dinv[4];
  int abc2;
  T ih3q;
  T tang;   // 2 ih3q / k (constant k)
};

// Matrix-free fine-level operator: ghost-eliminated Sommerfeld rows scaled
// by 1/2 (edge) and 1/4 (corner), Sec. 2 of the paper.  With wx = 1/2 on a
// vertical boundary line (else 1) and wy likewise,
//   (A x)_P = [4 wx wy x_P - wy (x_E + x_W) - wx (x_N + x_S)] / h^2
//             - wx wy k_P^2 x_P - i (k_P / h)(bx wy + wx by) x_P
// and halo nodes read as zero.  With c.abc2 the boundary rows carry the
// second-order absorbing condition of Engquist and Majda, d u/dn - i k u -
// (i/2k) d^2 u/dtau^2 = 0: its tangential term, in the weak form the
// boundary stiffness (i/2k) int dtau u dtau v with natural corners, adds
// for every boundary segment P-Q of a side through P
//   i c_PQ (x_P - x_Q),  c_PQ = (1/k_P + 1/k_Q) / (4 h^3)
// (an edge node has two such segments, a corner one on each of its sides).
// The term is compiled only into the A2 = true operator, which handles with
// the second-order rows use (c.abc2); the first-order kernels carry none of
// its registers.
template <class T, bool A2 = false> struct Op0 {
  Op0Consts<T> c;
  const T* kf;     // per-node k, dense (ny+1)*(nx+1), or null for constant k
  int nx, ny;

  __device__ __forceinline__ void geom(int i, int j, T& wx, T& wy, int& bx, int& by) const {
    bx = (i == 0 || i == nx);
    by = (j == 0 || j == ny);
    wx = bx ? T(0.5) : T(1);
    wy = by ? T(0.5) : T(1);
  }
  __device__ __forceinline__ T kval(int i, int j) const {
    return kf ? kf[j * (nx + 1) + i] : c.k;
  }
  __device__ __forceinline__ cx<T> apply(const cx<T>* __restrict__ x, int p, int pitch, int i, int j) const {
    return apply5(x[p], x[p + 1], x[p - 1], x[p + pitch], x[p - pitch], i, j);
  }
  // the stencil given the node's value and its E, W, N, S neighbours:
  // A x = d x_P - (wy (x_E + x_W) + wx (x_N + x_S)) / h^2 - i sb x_P with the
  // diagonal coefficient d = w (4 / h^2 - k^2); interior nodes (w = 1, no
  // boundary term) take the short path
  __device__ __forceinline__ cx<T> apply5(cx<T> xp, cx<T> xe, cx<T> xw, cx<T> xn, cx<T> xs, int i, int j) const {
    const T k = kval(i, j);
    const bool bx = (i == 0 || i == nx), by = (j == 0 || j == ny);
    if (!(bx || by)) {
      const T sr = (xe.x + xw.x) + (xn.x + xs.x), si = (xe.y + xw.y) + (xn.y + xs.y);
      const T d = fma(-k, k, T(4) * c.inv_h2);
      return mk<T>(fma(d, xp.x, -c.inv_h2 * sr), fma(d, xp.y, -c.inv_h2 * si));
    }
    const T wx = bx ? T(0.5) : T(1), wy = by ? T(0.5) : T(1), w = wx * wy;
    const T sr = wy * (xe.x + xw.x) + wx * (xn.x + xs.x), si = wy * (xe.y + xw.y) + wx * (xn.y + xs.y);
    const T d = w * fma(-k, k, T(4) * c.inv_h2);
    const T sb = (k * c.inv_h) * (T(bx) * wy + wx * T(by));
    const cx<T> a = mk<T>(fma(d, xp.x, fma(sb, xp.y, -c.inv_h2 * sr)), fma(d, xp.y, fma(-sb, xp.x, -c.inv_h2 * si)));
    if constexpr (!A2) {
      return a;
    } else {
      return add<T>(a, abc2_term(xp, xe, xw, xn, xs, i, j, bx, by));
    }
  }
  // the tangential term: i sum_Q c_PQ (x_P - x_Q)
  __device__ __forceinline__ cx<T> abc2_term(cx<T> xp, cx<T> xe, cx<T> xw, cx<T> xn, cx<T> xs, int i, int j, bool bx,
                                             bool by) const {
    if (kf) return abc2_var(xp, xe, xw, xn, xs, i, j, bx, by);
    // constant k: every segment has c_PQ = 2 ih3q / k = c.tang
    const bool sw = by && i > 0, se = by && i < nx, ss = bx && j > 0, sn = bx && j < ny;
    const T cnt = T(sw) + T(se) + T(ss) + T(sn);
    const T qr = (sw ? xw.x : T(0)) + (se ? xe.x : T(0)) + (ss ? xs.x : T(0)) + (sn ? xn.x : T(0));
    const T qi = (sw ? xw.y : T(0)) + (se ? xe.y : T(0)) + (ss ? xs.y : T(0)) + (sn ? xn.y : T(0));
    const T tr = c.tang * fma(cnt, xp.x, -qr), ti = c.tang * fma(cnt, xp.y, -qi);
    return mk<T>(-ti, tr);
  }
  // the tangential term i sum_Q c_PQ (x_P - x_Q) for variable k
  __device__ __forceinline__ cx<T> abc2_var(cx<T> xp, cx<T> xe, cx<T> xw, cx<T> xn, cx<T> xs, int i, int j, bool bx,
                                         bool by) const {
    T tr = T(0), ti = T(0);
    const T ik = T(1) / kval(i, j);
    auto seg = [&](cx<T> xq, int iq, int jq) {
      const T cs = c.ih3q * (ik + T(1) / kval(iq, jq));
      tr = fma(cs, xp.x - xq.x, tr);
      ti = fma(cs, xp.y - xq.y, ti);
    };
    if (by) {   // bottom or top side: neighbours along x
      if (i > 0) seg(xw, i - 1, j);
      if (i < nx) seg(xe, i + 1, j);
    }
    if (bx) {   // left or right side: neighbours along y
      if (j > 0) seg(xs, i, j - 1);
      if (j < ny) seg(xn, i, j + 1);
    }
    return mk<T>(-ti, tr);
  }
  // the second-order absorbing rows' diagonal contribution at (i, j): sum of
  // c_PQ over the node's boundary segments (times i); 0 off the boundary
  __device__ __forceinline__ T abc2_diag(int i, int j, int bx, int by) const {
    if constexpr (!A2) return T(0);
    const T ik = T(1) / kval(i, j);
    T s = T(0);
    if (by) {
      if (i > 0) s += c.ih3q * (ik + T(1) / kval(i - 1, j));
      if (i < nx) s += c.ih3q * (ik + T(1) / kval(i + 1, j));
    }
    if (bx) {
      if (j > 0) s += c.ih3q * (ik + T(1) / kval(i, j - 1));
      if (j < ny) s += c.ih3q * (ik + T(1) / kval(i, j + 1));
    }
    return s;
  }
  __device__ __forceinline__ cx<T> diag_inv(int i, int j) const {
    T wx, wy; int bx, by;
    geom(i, j, wx, wy, bx, by);
    if (!kf) return c.dinv[by * 2 + bx];
    const T k = kval(i, j);
    const T w = wx * wy;
    const T dr = (T(4) * w) * c.inv_h2 - w * (k * k);
    const T di = -(k * c.inv_h) * (T(bx) * wy + wx * T(by)) + abc2_diag(i, j, bx, by);
    return cinv<T>(mk<T>(c.omega * dr, c.omega * di));
  }
};

// Stored Galerkin stencil of radius R: st[e][j][i] (dense planes of
// (ny+1)*(nx+1) nodes) with e = (dy+R)*(2R+1) + (dx+R) the coupling of node
// (i,j) to node (i+dx, j+dy); dinv[j][i] = 1/(omega * centre entry).
template <class T, int R> struct OpS {
  const cx<T>* st;
  const cx<T>* dinvp;
  long long plane;
  int nx, ny;
  __device__ __forceinline__ cx<T> apply(const cx<T>* __restrict__ x, int p, int pitch, int i, int j) const {
    const long long q = (long long)j * (nx + 1) + i;
    cx<T> acc = mk<T>(0, 0);
#pragma unroll
    for (int dy = -R; dy <= R; ++dy) {
#pragma unroll
      for (int dx = -R; dx <= R; ++dx) {
        const int e = (dy + R) * (2 * R + 1) + (dx + R);
        acc = fma_c<T>(st[e * plane + q], x[p + dy * pitch + dx], acc);
      }
    }
    return acc;
  }
  __device__ __forceinline__ cx<T> diag_inv(int i, int j) const {
    return dinvp[(long long)j * (nx + 1) + i];
  }
};

// Constant-k Galerkin operator in Kronecker form (radius R):
//   A = W_y (x) G_x + H_y (x) W_x,
// with G_x, H_y complex and W_x, W_y real banded 1D operators, each the 1D
// Galerkin coarsening of its fine-level factor (the fine operator is
// W1 (x) (L1/h^2 - (1 + i beta2) k^2 W1 - i k/h B1) + (L1/h^2 - i k/h B1) (x) W1
// in terms of the 1D Neumann Laplacian L1, boundary weights W1 and boundary
// indicator B1).  Rows are [n+1][2R+1], entry R + d the coupling to node + d.
// Broadcast copies (value, value) of the translation-invariant y-factor row,
// for the packed complex64 column marches: a .f32x2 multiply-add takes such
// a pair straight from the parameter bank.  complex128 keeps none.
template <class T, int K> struct KBank {};
template <int K> struct KBank<float, K> {
  float2 hyr[K], hyi[K], wyb[K];   // Re h, Im h, w
};

template <class T, int R> struct OpK {
  const cx<T>* gx;
  const T* wx;
  const cx<T>* hy;
  const T* wy;
  const cx<T>* dinvp;
  int nx, ny;
  // Rows [ty0, ty1) whose y-factor rows equal hyc / wyc bit for bit (away
  // from the boundary the constant-k factors are translation invariant):
  // kernels that take the operator by value read them from the parameter
  // bank instead of loading the row's coefficients (ty0 = ty1 = 0: none).
  int ty0, ty1;
  cx<T> hyc[2 * R + 1];
  T wyc[2 * R + 1];
  KBank<T, 2 * R + 1> pk;   // broadcast copies of hyc / wyc
  static constexpr int radius = R;
  __device__ __forceinline__ cx<T> apply(const cx<T>* __restrict__ x, int p, int pitch, int i, int j) const {
    const cx<T>* G = gx + i * (2 * R + 1);
    const T* Wx = wx + i * (2 * R + 1);
    const cx<T>* H = hy + j * (2 * R + 1);
    const T* Wy = wy + j * (2 * R + 1);
    cx<T> acc = mk<T>(0, 0);
#pragma unroll
    for (int dy = -R; dy <= R; ++dy) {
      const cx<T>* row = x + p + dy * pitch;
      cx<T> s1 = mk<T>(0, 0), s2 = mk<T>(0, 0);
#pragma unroll
      for (int dx = -R; dx <= R; ++dx) {
        const cx<T> xv = row[dx];
        s1 = fma_c<T>(G[dx + R], xv, s1);
        s2 = mk<T>(fma(Wx[dx + R], xv.x, s2.x), fma(Wx[dx + R], xv.y, s2.y));
      }
      acc = mk<T>(fma(Wy[dy + R], s1.x, acc.x), fma(Wy[dy + R], s1.y, acc.y));
      acc = fma_c<T>(H[dy + R], s2, acc);
    }
    return acc;
  }
  __device__ __forceinline__ cx<T> diag_inv(int i, int j) const {
    return dinvp[(long long)j * (nx + 1) + i];
  }
};

// Final stage of the block sums below: value k of the block is the sum of
// the warps' partial sums sh[k][0..nwarps) added in warp order.  Lane k of
// warp 0 adds value k, all NV values at once (one FP64 add instruction per
// warp instead of one per warp and value: the FP64 pipe is narrow), and the
// totals are shuffled to lane 0.  out is valid in thread 0.
template <int NV>
__device__ __forceinline__ void warp_sums_to_thread0(const double* sh, int nwarps, int warp, int lane,
                                                     double (&out)[NV]) {
  static_assert(NV <= 32, "one lane per value");
  if (warp != 0) return;
  double t = 0;
  if (lane < NV)
    for (int w = 0; w < nwarps; ++w) t += sh[lane * 32 + w];
#pragma unroll
  for (int k = 0; k < NV; ++k) out[k] = __shfl_sync(0xffffffffu, t, k);
}

// Block-wide sum of NV doubles; result valid in thread 0.  Fixed shape and
// order, so results are bitwise reproducible run to run.
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double* sh /* [NV][32] */) {
  const int tid = threadIdx.x + threadIdx.y * blockDim.x;
  const int lane = tid & 31, warp = tid >> 5;
  const int nwarps = (blockDim.x * blockDim.y) >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    double t = v[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    if (lane == 0) sh[k * 32 + warp] = t;
  }
  __syncthreads();
  warp_sums_to_thread0<NV>(sh, nwarps, warp, lane, v);
  __syncthreads();
}

// Block-wide sum of NV values of the working precision T: the warp stage runs
// in T (shuffles), each warp's sum is widened to double once, and thread 0
// adds the warps in double.  Fixed shape and order (reproducible).
template <int NV, class T>
__device__ __forceinline__ void block_sum_t(const T (&v)[NV], double* sh /* [NV][32] */, double (&out)[NV]) {
  const int tid = threadIdx.x + threadIdx.y * blockDim.x;
  const int lane = tid & 31, warp = tid >> 5;
  const int nwarps = (blockDim.x * blockDim.y) >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    T t = v[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    if (lane == 0) sh[k * 32 + warp] = (double)t;
  }
  __syncthreads();
  warp_sums_to_thread0<NV>(sh, nwarps, warp, lane, out);
  __syncthreads();
}

// The last block's sum over few partial records (nrec <= 32), run by warp 0:
// the records are staged in shared memory and lane k adds value k over the
// records in order, all NV values at once (nrec FP64 adds in sequence instead
// of a shuffle tree of 5 adds per value).  v is valid in thread 0.
template <int NV>
__device__ __forceinline__ void last_block_sum_few(double (&v)[NV], const double* q, int nrec, double* sh, int lane) {
  static_assert(NV <= NVMAX, "record size");
  for (int e = lane; e < nrec * NV; e += 32) {
    const int b = e / NV, k = e - b * NV;
    sh[e] = __ldcg(q + (long long)b * NVMAX + k);
  }
  __syncwarp();
  double t = 0.0;
  if (lane < NV) {
    t = sh[lane];
    for (int b = 1; b < nrec; ++b) t += sh[b * NV + lane];
  }
#pragma unroll
  for (int k = 0; k < NV; ++k) v[k] = __shfl_sync(0xffffffffu, t, k);
}

// Thread tid's share of the partial records q[0..nrec) (NVMAX doubles
// each) summed in record order tid, tid + nt, ...; the first record is taken
// as it is rather than added to zero.
template <int NV>
__device__ __forceinline__ void last_block_partials(double (&acc)[NV], const double* q, int nrec, int tid, int nt) {
#pragma unroll
  for (int k = 0; k < NV; ++k) acc[k] = tid < nrec ? __ldcg(q + (long long)tid * NVMAX + k) : 0.0;
  for (int b = tid + nt; b < nrec; b += nt) {
#pragma unroll
    for (int k = 0; k < NV; ++k) acc[k] += __ldcg(q + (long long)b * NVMAX + k);
  }
}

// Grid-wide deterministic sum of NV doubles for one right-hand side, inside
// the producing kernel: every block publishes its block sum, takes a ticket,
// and the block holding the last ticket sums all partials in block order
// (fixed, so results are bitwise reproducible) and resets the ticket.
// vin: this thread's sums in the working precision.  Returns true,
// block-uniformly, in that last block; the totals are then valid in thread
// 0's v.  partial: [rhs][nblk][NVMAX]; tickets: [rhs], 0 at rest.  Must be
// reached by every thread of every block of the RHS.
template <int NV, class T>
__device__ __forceinline__ bool reduce_last(const T (&vin)[NV], double (&v)[NV], double* sh, double* partial,
                                            unsigned* tickets, int rhs, int nblk, int blk) {
  __shared__ int s_last;
  block_sum_t<NV, T>(vin, sh, v);
  const int tid = threadIdx.x + threadIdx.y * blockDim.x;
  const int nt = blockDim.x * blockDim.y;
  if (tid == 0) {
    double* q = partial + ((long long)rhs * nblk + blk) * NVMAX;
#pragma unroll
    for (int k = 0; k < NV; ++k) q[k] = v[k];
    __threadfence();
    const unsigned t = atomicAdd(&tickets[rhs], 1u);
    s_last = (t == (unsigned)(nblk - 1));
  }
  __syncthreads();
  if (!s_last) return false;
  __threadfence();
  if (nblk <= 32) {   // block-uniform
    if (tid < 32) last_block_sum_few<NV>(v, partial + (long long)rhs * nblk * NVMAX, nblk, sh, tid);
    if (tid == 0) tickets[rhs] = 0u;
    return true;
  }
  double acc[NV];
  last_block_partials<NV>(acc, partial + (long long)rhs * nblk * NVMAX, nblk, tid, nt);
  block_sum<NV>(acc, sh);
  if (tid == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] = acc[k];
    tickets[rhs] = 0u;
  }
  return true;
}

// The same sum split over two launches on one stream: the first launch's
// blocks only publish their block sums (publish, records 0 .. rec0-1); the
// second launch's blocks publish after them (records rec0 + blk) and take
// tickets, and its last block sums all nrec records in record order.
// partial: [rhs][nrec][NVMAX].
template <int NV, class T>
__device__ __forceinline__ void publish(const T (&vin)[NV], double* sh, double* partial, int rhs, int nrec, int rec) {
  double v[NV];
  block_sum_t<NV, T>(vin, sh, v);
  if (threadIdx.x + threadIdx.y * blockDim.x == 0) {
    double* q = partial + ((long long)rhs * nrec + rec) * NVMAX;
#pragma unroll
    for (int k = 0; k < NV; ++k) q[k] = v[k];
  }
}
template <int NV, class T>
__device__ __forceinline__ bool reduce_last_at(const T (&vin)[NV], double (&v)[NV], double* sh, double* partial,
                                               unsigned* tickets, int rhs, int nblk, int blk, int rec0, int nrec) {
  __shared__ int s_last;
  block_sum_t<NV, T>(vin, sh, v);
  const int tid = threadIdx.x + threadIdx.y * blockDim.x;
  const int nt = blockDim.x * blockDim.y;
  if (tid == 0) {
    double* q = partial + ((long long)rhs * nrec + rec0 + blk) * NVMAX;
#pragma unroll
    for (int k = 0; k < NV; ++k) q[k] = v[k];
    __threadfence();
    const unsigned t = atomicAdd(&tickets[rhs], 1u);
    s_last = (t == (unsigned)(nblk - 1));
  }
  __syncthreads();
  if (!s_last) return false;
  __threadfence();
  if (nrec <= 32) {   // block-uniform
    if (tid < 32) last_block_sum_few<NV>(v, partial + (long long)rhs * nrec * NVMAX, nrec, sh, tid);
    if (tid == 0) tickets[rhs] = 0u;
    return true;
  }
  double acc[NV];
  last_block_partials<NV>(acc, partial + (long long)rhs * nrec * NVMAX, nrec, tid, nt);
  block_sum<NV>(acc, sh);
  if (tid == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] = acc[k];
    tickets[rhs] = 0u;
  }
  return true;
}

}  // namespace hmg
