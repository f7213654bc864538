// Node packs: the complex64 kernels handle two horizontally adjacent nodes
// per thread (one 16-byte load or store per vector and pair), the complex128
// kernels one node.  A pack starts at an even node index, so with the padded
// layout (even halo, pitch a multiple of 4) its first element is 16-byte
// aligned.  Packs that straddle the grid's right edge store only their nodes
// inside the grid, so the zero halo is never written.
#pragma once
#include "common.cuh"

namespace hmg {

template <class T> struct PK;
template <> struct PK<float> { static constexpr int NP = 2; };
template <> struct PK<double> { static constexpr int NP = 1; };

template <class T> struct Pack {
  cx<T> v[PK<T>::NP];
};

__device__ __forceinline__ Pack<float> load_pack(const float2* a, int p) {
  const float4 q = *reinterpret_cast<const float4*>(a + p);
  Pack<float> r;
  r.v[0] = make_float2(q.x, q.y);
  r.v[1] = make_float2(q.z, q.w);
  return r;
}
__device__ __forceinline__ Pack<double> load_pack(const double2* a, int p) {
  Pack<double> r;
  r.v[0] = a[p];
  return r;
}
__device__ __forceinline__ void store_pack(float2* a, int p, const Pack<float>& v, int nvalid) {
  if (nvalid >= 2) {
    *reinterpret_cast<float4*>(a + p) = make_float4(v.v[0].x, v.v[0].y, v.v[1].x, v.v[1].y);
  } else {
    a[p] = v.v[0];
  }
}
__device__ __forceinline__ void store_pack(double2* a, int p, const Pack<double>& v, int) { a[p] = v.v[0]; }

// Operator applied to the pack of nodes (i0.., j) starting at offset p.
template <class T, class Op> struct PackApply {
  __device__ __forceinline__ static Pack<T> run(const Op& op, const cx<T>* x, int p, int pitch, int i0, int j) {
    // a node past the grid's right edge has no coefficients: it is not evaluated
    Pack<T> r;
#pragma unroll
    for (int n = 0; n < PK<T>::NP; ++n)
      r.v[n] = i0 + n <= op.nx ? op.apply(x, p + n, pitch, i0 + n, j) : mk<T>(0, 0);
    return r;
  }
};
// Fine level, complex64: three 16-byte row loads and two 8-byte edge loads
// serve both nodes' 5-point stencils.
template <> struct PackApply<float, Op0<float>> {
  __device__ __forceinline__ static Pack<float> run(const Op0<float>& op, const float2* x, int p, int pitch, int i0,
                                                    int j) {
    const Pack<float> c = load_pack(x, p), n = load_pack(x, p + pitch), s = load_pack(x, p - pitch);
    const float2 l = x[p - 1], r = x[p + 2];
    Pack<float> out;
    out.v[0] = op.apply5(c.v[0], c.v[1], l, n.v[0], s.v[0], i0, j);
    out.v[1] = i0 + 1 <= op.nx ? op.apply5(c.v[1], r, c.v[0], n.v[1], s.v[1], i0 + 1, j) : make_float2(0.f, 0.f);
    return out;
  }
};

template <class T, class Op>
__device__ __forceinline__ Pack<T> apply_pack(const Op& op, const cx<T>* x, int p, int pitch, int i0, int j) {
  return PackApply<T, Op>::run(op, x, p, pitch, i0, j);
}

}  // namespace hmg
