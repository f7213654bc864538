// Outer iterate of the mixed-precision path in float-float arithmetic.
//
// The refinement loop keeps x and b at level 0 in a format with a 48-bit
// significand and forms r = b - A x to that accuracy, so that the complex64
// correction cycles converge to an FP64-accurate solution.  On this GPU the
// FP64 units run at a small fraction of the FP32 rate and an FP64 stencil
// pass is arithmetic-bound, so the outer values are stored as unevaluated
// sums hi + lo of two floats (each complex node as the float4
// {re.hi, im.hi, re.lo, im.lo}, in the same 16 bytes per node as a complex128
// value) and the residual uses the error-free transformations of Dekker
// (1971) and Knuth (TAOCP vol. 2, 4.2.2): two_sum, fast_two_sum and the
// FMA-based exact product.  The additions are the "sloppy" double-single
// sums, whose absolute error is about 2^-44 of the operands' magnitude --
// close to the FP64 evaluation's 2^-53 and far below the residuals the
// stopping test resolves.
//
// Kernels: pack (complex128 -> hi/lo) and unpack, ||b||, the residual with
// the float cast for the next correction cycle and the fused stopping test,
// and x += e.  The stencil is Op0::apply5's (Sec. 2 of the paper: the
// ghost-eliminated Sommerfeld rows scaled by 1/2 on edges and 1/4 at
// corners), with every coefficient held as a float-float constant.
#include "internal.h"

namespace hmg {

namespace {

using ff = FF;

__device__ __forceinline__ ff two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  return {s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ ff fast_two_sum(float a, float b) {   // |a| >= |b|
  const float s = a + b;
  return {s, b - (s - a)};
}
__device__ __forceinline__ ff ff_add(ff a, ff b) {
  const ff s = two_sum(a.h, b.h);
  return fast_two_sum(s.h, s.l + (a.l + b.l));
}
__device__ __forceinline__ ff ff_neg(ff a) { return {-a.h, -a.l}; }
__device__ __forceinline__ ff ff_scale(ff a, float w) { return {a.h * w, a.l * w}; }   // w a power of two
__device__ __forceinline__ ff ff_mul(ff a, ff b) {
  const float p = a.h * b.h;
  float e = fmaf(a.h, b.h, -p);
  e = fmaf(a.h, b.l, fmaf(a.l, b.h, e));
  return fast_two_sum(p, e);
}
__device__ __forceinline__ ff ff_from(double v) {
  const float h = __double2float_rn(v);
  return {h, __double2float_rn(v - (double)h)};
}
__device__ __forceinline__ double ff_to(ff a) { return (double)a.h + (double)a.l; }

// a complex node
struct cff {
  ff re, im;
};
__device__ __forceinline__ cff ld(const float4* p) {
  const float4 q = *p;
  return {{q.x, q.z}, {q.y, q.w}};
}
__device__ __forceinline__ void st(float4* p, cff v) { *p = make_float4(v.re.h, v.im.h, v.re.l, v.im.l); }


// r = b - A x at node (i, j) (slice pointers at the node's offset p).
__device__ __forceinline__ cff ff_residual(const FFConsts& K, const double* kf, int nx, int ny, double inv_h,
                                           const float2* dP, const float4* x, const float4* b, int p, int pitch, int i,
                                           int j) {
  const cff xp = ld(x + p), xe = ld(x + p + 1), xw = ld(x + p - 1), xn = ld(x + p + pitch), xs = ld(x + p - pitch);
  const bool bx = (i == 0 || i == nx), by = (j == 0 || j == ny);
  const float wx = bx ? 0.5f : 1.f, wy = by ? 0.5f : 1.f;
  ff d = K.d, sb = K.sb;
  if (kf) {   // per-node diagonal w (4/h^2 - k^2) and k/h
    const float2 q = dP[(long long)j * (nx + 1) + i];
    d = {q.x, q.y};
    if (bx || by) sb = ff_from(kf[(long long)j * (nx + 1) + i] * inv_h);
  } else if (bx || by) {
    d = ff_scale(d, wx * wy);
  }
  const ff sr = ff_add(ff_scale(ff_add(xe.re, xw.re), wy), ff_scale(ff_add(xn.re, xs.re), wx));
  const ff si = ff_add(ff_scale(ff_add(xe.im, xw.im), wy), ff_scale(ff_add(xn.im, xs.im), wx));
  ff are = ff_add(ff_mul(d, xp.re), ff_neg(ff_mul(K.ih2, sr)));
  ff aim = ff_add(ff_mul(d, xp.im), ff_neg(ff_mul(K.ih2, si)));
  if (bx || by) {   // - i (k/h) x_P
    are = ff_add(are, ff_mul(sb, xp.im));
    aim = ff_add(aim, ff_neg(ff_mul(sb, xp.re)));
  }
  const cff bb = ld(b + p);
  return {ff_add(bb.re, ff_neg(are)), ff_add(bb.im, ff_neg(aim))};
}

#define FF_NODE                                                \
  const int rhs = blockIdx.z;                                  \
  const int i = blockIdx.x * BX + threadIdx.x;                 \
  const long long off = (long long)rhs * g.vstride;
#define FF_ROWS for (int r_ = 0, j = blockIdx.y * BY * g.ry + threadIdx.y; r_ < g.ry; ++r_, j += BY)

__global__ void __launch_bounds__(BX * BY) k_ff_resid_cast_stop(Grid g, FFConsts K, const double* __restrict__ kf,
                                                                double inv_h, const float2* __restrict__ dP,
                                                                const float4* __restrict__ x,
                                                                const float4* __restrict__ b, float2* __restrict__ r32,
                                                                Ctl c, int count) {
  __shared__ double sh[NVMAX * 32];
  FF_NODE
  if (!c.active[rhs]) return;   // block-uniform
  float a = 0.f;
  if (i <= g.nx) {
    FF_ROWS {
      if (j > g.ny) break;
      const int p = g.at(i, j);
      const cff r = ff_residual(K, kf, g.nx, g.ny, inv_h, dP, x + off, b + off, p, g.pitch, i, j);
      r32[off + p] = make_float2(r.re.h, r.im.h);
      a = fmaf(r.re.h, r.re.h, fmaf(r.im.h, r.im.h, a));
    }
  }
  const double ad[1] = {(double)a};
  double v[1];
  if (reduce_last<1, double>(ad, v, sh, c.partial, c.tickets, rhs, gridDim.x * gridDim.y,
                             blockIdx.y * gridDim.x + blockIdx.x) &&
      threadIdx.x == 0 && threadIdx.y == 0)
    stop_update(c, rhs, v[0], count);
}

__global__ void __launch_bounds__(BX * BY) k_ff_update(Grid g, float4* __restrict__ x, const float2* __restrict__ e,
                                                       const int* __restrict__ active) {
  FF_NODE
  if (active && !active[rhs]) return;
  if (i > g.nx) return;
  FF_ROWS {
    if (j > g.ny) break;
    const long long p = off + g.at(i, j);
    const float2 d = e[p];
    cff v = ld(x + p);
    v.re = ff_add(v.re, {d.x, 0.f});
    v.im = ff_add(v.im, {d.y, 0.f});
    st(x + p, v);
  }
}

// Dense complex128 [B][ny+1][nx+1] <-> padded float-float; conj != 0
// conjugates.
__global__ void __launch_bounds__(BX * BY) k_ff_pack(Grid g, const double2* __restrict__ user, float4* __restrict__ v,
                                                     int conj) {
  FF_NODE
  if (i > g.nx) return;
  FF_ROWS {
    if (j > g.ny) break;
    const double2 u = user[((long long)rhs * (g.ny + 1) + j) * (g.nx + 1) + i];
    st(v + off + g.at(i, j), {ff_from(u.x), ff_from(conj ? -u.y : u.y)});
  }
}
__global__ void __launch_bounds__(BX * BY) k_ff_unpack(Grid g, const float4* __restrict__ v, double2* __restrict__ user,
                                                       int conj) {
  FF_NODE
  if (i > g.nx) return;
  FF_ROWS {
    if (j > g.ny) break;
    const cff a = ld(v + off + g.at(i, j));
    const double im = ff_to(a.im);
    user[((long long)rhs * (g.ny + 1) + j) * (g.nx + 1) + i] = make_double2(ff_to(a.re), conj ? -im : im);
  }
}

// out[rhs] = ||v|| of a float-float vector (one kernel, last-block finish).
__global__ void __launch_bounds__(BX * BY) k_ff_norm(Grid g, const float4* __restrict__ v, double* __restrict__ out,
                                                     double* partial, unsigned* tickets) {
  __shared__ double sh[NVMAX * 32];
  FF_NODE
  double a[1] = {0.0};
  if (i <= g.nx) {
    FF_ROWS {
      if (j > g.ny) break;
      const cff q = ld(v + off + g.at(i, j));
      const double re = ff_to(q.re), im = ff_to(q.im);
      a[0] += re * re + im * im;
    }
  }
  double s[1];
  if (reduce_last<1, double>(a, s, sh, partial, tickets, rhs, gridDim.x * gridDim.y,
                             blockIdx.y * gridDim.x + blockIdx.x) &&
      threadIdx.x == 0 && threadIdx.y == 0)
    out[rhs] = sqrt(s[0]);
}

// Per-node float-float diagonal w (4/h^2 - k^2) for variable k (dense).
__global__ void k_ff_diag(int nx, int ny, double h, const double* __restrict__ kf, float2* __restrict__ dP) {
  const long long n = (long long)(nx + 1) * (ny + 1);
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(q % (nx + 1)), j = (int)(q / (nx + 1));
    const double w = ((i == 0 || i == nx) ? 0.5 : 1.0) * ((j == 0 || j == ny) ? 0.5 : 1.0);
    const double k = kf[q];
    const ff d = ff_from(w * (4.0 / (h * h) - k * k));
    dP[q] = make_float2(d.h, d.l);
  }
}

__global__ void k_ff_consts(double h, double k, FFConsts* out) {
  out->d = ff_from(4.0 / (h * h) - k * k);
  out->ih2 = ff_from(1.0 / (h * h));
  out->sb = ff_from(k / h);
}

dim3 ff_grid(const Grid& g, int B) { return dim3(cdiv(g.nx + 1, BX), cdiv(g.ny + 1, BY * g.ry), B); }

}  // namespace

void launch_ff_setup(double h, double k, const double* kf, int nx, int ny, FFConsts* consts, float2* dP,
                     cudaStream_t s) {
  k_ff_consts<<<1, 1, 0, s>>>(h, k, consts);
  if (kf) k_ff_diag<<<cdiv((long long)(nx + 1) * (ny + 1), 256), 256, 0, s>>>(nx, ny, h, kf, dP);
}

void launch_ff_resid_cast_stop(const Grid& g, const FFConsts& K, const double* kf, double h, const float2* dP,
                               const void* x, const void* b, float2* r32, int B, const Ctl& c, int count,
                               cudaStream_t s) {
  k_ff_resid_cast_stop<<<ff_grid(g, B), dim3(BX, BY), 0, s>>>(g, K, kf, 1.0 / h, dP, (const float4*)x,
                                                                (const float4*)b, r32, c, count);
}

void launch_ff_update(const Grid& g, void* x, const float2* e, int B, const int* active, cudaStream_t s) {
  k_ff_update<<<ff_grid(g, B), dim3(BX, BY), 0, s>>>(g, (float4*)x, e, active);
}

void launch_ff_pack(const Grid& g, const double2* user, void* v, int B, int conj, cudaStream_t s) {
  k_ff_pack<<<ff_grid(g, B), dim3(BX, BY), 0, s>>>(g, user, (float4*)v, conj);
}

void launch_ff_unpack(const Grid& g, const void* v, double2* user, int B, int conj, cudaStream_t s) {
  k_ff_unpack<<<ff_grid(g, B), dim3(BX, BY), 0, s>>>(g, (const float4*)v, user, conj);
}

void launch_ff_norm(const Grid& g, const void* v, int B, double* out, double* partial, unsigned* tickets,
                    cudaStream_t s) {
  k_ff_norm<<<ff_grid(g, B), dim3(BX, BY), 0, s>>>(g, (const float4*)v, out, partial, tickets);
}

}  // namespace hmg
