// Setup kernels: fine-level constants, Galerkin coarse operators
// A_{l+1} = R_l C_l P_l (Sec. 3; coarsening on the CSL, Sec. 4), Jacobi
// inverse diagonals, and the coarsest-grid direct solver (Sec. 5: coarsen
// until fewer than 10 unknowns remain, solve there exactly).  All FP64.
#include <math.h>

#include "internal.h"

namespace hmg {


// Coupling of node (i, j) to node (i+dx, j+dy) in a level operator; for the
// matrix-free fine operator the mass term carries the shift (1 + i beta2).
__device__ double2 op_coef(const OpView<double>& v, int nx, int ny, int i, int j, int dy, int dx, double beta2) {
  const int i2 = i + dx, j2 = j + dy;
  if (i2 < 0 || i2 > nx || j2 < 0 || j2 > ny) return make_double2(0, 0);
  if (v.kind == 2 || v.kind == 3) {
    const int r = v.kind;
    if (dx < -r || dx > r || dy < -r || dy > r) return make_double2(0, 0);
    const int e = (dy + r) * (2 * r + 1) + (dx + r);
    return v.st[e * v.plane + (long long)j * (nx + 1) + i];
  }
  if (v.kind >= 4) {   // W_y[j][dy] G_x[i][dx] + H_y[j][dy] W_x[i][dx]
    const int r = v.kind - 2, w = 2 * r + 1;
    if (dx < -r || dx > r || dy < -r || dy > r) return make_double2(0, 0);
    const double2 G = v.gx[i * w + dx + r], H = v.hy[j * w + dy + r];
    const double Wx = v.wx[i * w + dx + r], Wy = v.wy[j * w + dy + r];
    return make_double2(Wy * G.x + H.x * Wx, Wy * G.y + H.y * Wx);
  }
  const Op0Consts<double>* c = &v.c0;
  const int bx = (i == 0 || i == nx), by = (j == 0 || j == ny);
  const double wx = bx ? 0.5 : 1.0, wy = by ? 0.5 : 1.0, w = wx * wy;
  const double k = v.kf ? v.kf[(long long)j * (nx + 1) + i] : c->k;
  // the second-order absorbing rows (Op0): i c_PQ on the diagonal and -i c_PQ
  // to Q for every boundary segment P-Q of a side through P
  auto kat = [&](int a, int b) { return v.kf ? v.kf[(long long)b * (nx + 1) + a] : c->k; };
  auto cseg = [&](int a, int b) { return c->ih3q * (1.0 / k + 1.0 / kat(a, b)); };
  if (dx == 0 && dy == 0) {
    const double k2 = k * k;
    double tang = 0.0;
    if (c->abc2) {
      if (by && i > 0) tang += cseg(i - 1, j);
      if (by && i < nx) tang += cseg(i + 1, j);
      if (bx && j > 0) tang += cseg(i, j - 1);
      if (bx && j < ny) tang += cseg(i, j + 1);
    }
    return make_double2(4.0 * w * c->inv_h2 - w * k2,
                        -w * (beta2 * k2) - (k * c->inv_h) * (bx * wy + wx * by) + tang);
  }
  if (dy == 0 && (dx == 1 || dx == -1))
    return make_double2(-wy * c->inv_h2, c->abc2 && by ? -cseg(i2, j2) : 0.0);
  if (dx == 0 && (dy == 1 || dy == -1))
    return make_double2(-wx * c->inv_h2, c->abc2 && bx ? -cseg(i2, j2) : 0.0);
  return make_double2(0, 0);
}

__global__ void s_op0consts(Op0Consts<double>* c64, Op0Consts<float>* c32, double h, double k, double omega,
                            double beta2, int abc) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  Op0Consts<double> c;
  c.inv_h2 = 1.0 / (h * h);
  c.inv_h = 1.0 / h;
  c.k = k;
  c.k2 = k * k;
  c.omega = omega;
  c.beta2 = beta2;
  c.abc2 = abc == 2;
  c.ih3q = 1.0 / (4.0 * h * h * h);
  c.tang = k > 0 ? 2.0 * c.ih3q / k : 0.0;
  for (int by = 0; by < 2; ++by)
    for (int bx = 0; bx < 2; ++bx) {
      const double wx = bx ? 0.5 : 1.0, wy = by ? 0.5 : 1.0, w = wx * wy;
      const double dr = 4.0 * w * c.inv_h2 - w * (k * k);
      // second-order absorbing rows: an edge node and a corner both have two
      // boundary segments, each c_PQ = 2 / (4 h^3 k) at constant k
      const double di = -(k * c.inv_h) * (bx * wy + wx * by) + (c.abc2 && (bx || by) ? 2.0 * (2.0 * c.ih3q / k) : 0.0);
      const double2 d = make_double2(omega * dr, omega * di);
      const double dd = d.x * d.x + d.y * d.y;
      c.dinv[by * 2 + bx] = make_double2(d.x / dd, -d.y / dd);
    }
  *c64 = c;
  if (c32) {
    Op0Consts<float> f;
    f.inv_h2 = (float)c.inv_h2;
    f.inv_h = (float)c.inv_h;
    f.k = (float)c.k;
    f.k2 = (float)c.k2;
    f.omega = (float)c.omega;
    f.beta2 = (float)c.beta2;
    f.abc2 = c.abc2;
    f.ih3q = (float)c.ih3q;
    f.tang = (float)c.tang;
    for (int q = 0; q < 4; ++q) f.dinv[q] = make_float2((float)c.dinv[q].x, (float)c.dinv[q].y);
    *c32 = f;
  }
}

// One thread per (coarse node, stencil entry):
// A_c[(I,J),(I2,J2)] = sum 1/4 w(fa-2I) w(fb-2J) * A_f[(fa,fb),(fa2,fb2)] * w(fa2-2I2) w(fb2-2J2)
__global__ void s_galerkin(OpView<double> fine, int fnx, int fny, int rf, double2* __restrict__ cst, int cnx, int cny,
                           int rc, double beta2, Xfer xw) {
  const int S = (2 * rc + 1) * (2 * rc + 1);
  const long long plane = (long long)(cnx + 1) * (cny + 1);
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= plane * S) return;
  const int e = (int)(idx % S);
  const long long q = idx / S;
  const int I = (int)(q % (cnx + 1)), J = (int)(q / (cnx + 1));
  const int dy = e / (2 * rc + 1) - rc, dx = e % (2 * rc + 1) - rc;
  const int I2 = I + dx, J2 = J + dy;
  double2 acc = make_double2(0, 0);
  if (I2 >= 0 && I2 <= cnx && J2 >= 0 && J2 <= cny) {
    for (int b = -2; b <= 2; ++b) {
      const int fb = 2 * J + b;
      if (fb < 0 || fb > fny) continue;
      for (int a = -2; a <= 2; ++a) {
        const int fa = 2 * I + a;
        if (fa < 0 || fa > fnx) continue;
        const double wr = 0.25 * xw.w<double>(a) * xw.w<double>(b);
        for (int b2 = -2; b2 <= 2; ++b2) {
          const int fb2 = 2 * J2 + b2;
          const int ey = fb2 - fb;
          if (fb2 < 0 || fb2 > fny || ey < -rf || ey > rf) continue;
          for (int a2 = -2; a2 <= 2; ++a2) {
            const int fa2 = 2 * I2 + a2;
            const int ex = fa2 - fa;
            if (fa2 < 0 || fa2 > fnx || ex < -rf || ex > rf) continue;
            const double2 cf = op_coef(fine, fnx, fny, fa, fb, ey, ex, beta2);
            const double wgt = wr * xw.w<double>(a2) * xw.w<double>(b2);
            acc.x += wgt * cf.x;
            acc.y += wgt * cf.y;
          }
        }
      }
    }
  }
  cst[e * plane + q] = acc;
}

__global__ void s_diaginv(const double2* __restrict__ st, int rc, long long plane, double omega, double2* __restrict__ dinv) {
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= plane) return;
  const int ec = rc * (2 * rc + 1) + rc;
  const double2 d = st[ec * plane + q];
  const double2 x = make_double2(omega * d.x, omega * d.y);
  const double dd = x.x * x.x + x.y * x.y;
  dinv[q] = make_double2(x.x / dd, -x.y / dd);
}

__global__ void s_to_float(const double2* __restrict__ a, float2* __restrict__ b, long long n) {
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q < n) b[q] = make_float2((float)a[q].x, (float)a[q].y);
}
__global__ void s_to_float_real(const double* __restrict__ a, float* __restrict__ b, long long n) {
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q < n) b[q] = (float)a[q];
}

__global__ void s_dense(OpView<double> v, int nx, int ny, double2* __restrict__ M) {
  const long long N = (long long)(nx + 1) * (ny + 1);
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= N * N) return;
  const long long r = idx / N, c = idx % N;
  const int i = (int)(r % (nx + 1)), j = (int)(r / (nx + 1));
  const int i2 = (int)(c % (nx + 1)), j2 = (int)(c / (nx + 1));
  const int R = op_radius(v.kind);
  const int dx = i2 - i, dy = j2 - j;
  double2 val = make_double2(0, 0);
  if (dx >= -R && dx <= R && dy >= -R && dy <= R) val = op_coef(v, nx, ny, i, j, dy, dx, 0.0);
  M[idx] = val;
}

__global__ void s_export(OpView<double> v, int nx, int ny, int r, double2* __restrict__ out) {
  const int S = (2 * r + 1) * (2 * r + 1);
  const long long plane = (long long)(nx + 1) * (ny + 1);
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= plane * S) return;
  const long long q = idx / S;
  const int e = (int)(idx % S);
  const int i = (int)(q % (nx + 1)), j = (int)(q / (nx + 1));
  const int dy = e / (2 * r + 1) - r, dx = e % (2 * r + 1) - r;
  out[idx] = op_coef(v, nx, ny, i, j, dy, dx, 0.0);
}

// In-place Gauss-Jordan with partial pivoting, one block: inv = M^{-1}.
// fac: dynamic shared memory, N double2.  status[0] = 1 on a zero pivot.
__global__ void s_gauss_jordan(double2* __restrict__ M, double2* __restrict__ inv, int N, int* status) {
  extern __shared__ double2 fac[];
  __shared__ int piv;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (long long q = tid; q < (long long)N * N; q += nt) {
    const long long r = q / N, c = q % N;
    inv[q] = make_double2(r == c ? 1.0 : 0.0, 0.0);
  }
  __syncthreads();
  for (int k = 0; k < N; ++k) {
    if (tid == 0) {
      int p = k;
      double best = -1.0;
      for (int r = k; r < N; ++r) {
        const double2 a = M[(long long)r * N + k];
        const double m = a.x * a.x + a.y * a.y;
        if (m > best) { best = m; p = r; }
      }
      piv = p;
      if (best == 0.0) status[0] = 1;
    }
    __syncthreads();
    const int p = piv;
    if (p != k) {
      for (int c = tid; c < N; c += nt) {
        double2 t = M[(long long)k * N + c]; M[(long long)k * N + c] = M[(long long)p * N + c]; M[(long long)p * N + c] = t;
        t = inv[(long long)k * N + c]; inv[(long long)k * N + c] = inv[(long long)p * N + c]; inv[(long long)p * N + c] = t;
      }
    }
    __syncthreads();
    const double2 d = M[(long long)k * N + k];
    const double dd = d.x * d.x + d.y * d.y;
    const double2 di = dd > 0 ? make_double2(d.x / dd, -d.y / dd) : make_double2(0, 0);
    __syncthreads();
    for (int c = tid; c < N; c += nt) {
      M[(long long)k * N + c] = mul<double>(di, M[(long long)k * N + c]);
      inv[(long long)k * N + c] = mul<double>(di, inv[(long long)k * N + c]);
    }
    for (int r = tid; r < N; r += nt) fac[r] = M[(long long)r * N + k];
    __syncthreads();
    for (long long q = tid; q < (long long)N * N; q += nt) {
      const int r = (int)(q / N), c = (int)(q % N);
      if (r == k) continue;
      const double2 f = fac[r];
      M[q] = sub<double>(M[q], mul<double>(f, M[(long long)k * N + c]));
      inv[q] = sub<double>(inv[q], mul<double>(f, inv[(long long)k * N + c]));
    }
    __syncthreads();
  }
}

// e = A_coarsest^{-1} r, one block per RHS, FP64 arithmetic.
template <class T>
__global__ void s_coarse_solve(Grid g, const double2* __restrict__ inv, int N, const cx<T>* __restrict__ r,
                               cx<T>* __restrict__ e, const int* __restrict__ active) {
  extern __shared__ double2 rs[];
  const int rhs = blockIdx.x;
  if (active && !active[rhs]) return;
  const long long off = (long long)rhs * g.vstride;
  for (int q = threadIdx.x; q < N; q += blockDim.x) {
    const int i = q % (g.nx + 1), j = q / (g.nx + 1);
    const cx<T> a = r[off + g.at(i, j)];
    rs[q] = make_double2((double)a.x, (double)a.y);
  }
  __syncthreads();
  for (int q = threadIdx.x; q < N; q += blockDim.x) {
    double2 acc = make_double2(0, 0);
    const double2* row = inv + (long long)q * N;
    for (int c = 0; c < N; ++c) acc = fma_c<double>(row[c], rs[c], acc);
    const int i = q % (g.nx + 1), j = q / (g.nx + 1);
    e[off + g.at(i, j)] = mk<T>((T)acc.x, (T)acc.y);
  }
}

// 1D factors of the fine operator, rows [n+1][3] (offsets -1, 0, +1):
// L1 = Neumann Laplacian (row 0: [0, 1, -1], row n: [-1, 1, 0]), W1 = diag(1/2,
// 1, ..., 1, 1/2), B1 = diag(1, 0, ..., 0, 1);  g = L1/h^2 - (1 + i beta2) k^2 W1
// - i (k/h) B1, hf = L1/h^2 - i (k/h) B1, w = W1.
__global__ void s_factors0(int n, double h, double k, double beta2, double2* g, double2* hf, double2* w) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i > n) return;
  const double ih2 = 1.0 / (h * h);
  const bool bnd = (i == 0 || i == n);
  const double lm = i > 0 ? -1.0 : 0.0, lp = i < n ? -1.0 : 0.0, lc = bnd ? 1.0 : 2.0;
  const double wi = bnd ? 0.5 : 1.0, bi = bnd ? 1.0 : 0.0;
  const double k2 = k * k;
  g[i * 3 + 0] = make_double2(lm * ih2, 0);
  g[i * 3 + 1] = make_double2(lc * ih2 - wi * k2, -wi * (beta2 * k2) - bi * (k / h));
  g[i * 3 + 2] = make_double2(lp * ih2, 0);
  hf[i * 3 + 0] = make_double2(lm * ih2, 0);
  hf[i * 3 + 1] = make_double2(lc * ih2, -bi * (k / h));
  hf[i * 3 + 2] = make_double2(lp * ih2, 0);
  w[i * 3 + 0] = make_double2(0, 0);
  w[i * 3 + 1] = make_double2(wi, 0);
  w[i * 3 + 2] = make_double2(0, 0);
}

// X_c[I][d] = sum_{a, a2} 1/2 w(a - 2I) X[a][a2 - a] w(a2 - 2(I + d)), one thread per (I, d).
__global__ void s_galerkin_1d(const double2* __restrict__ X, int nf, int rf, double2* __restrict__ Xc, int rc,
                              Xfer xw) {
  const int nc = nf / 2, wc = 2 * rc + 1, wf = 2 * rf + 1;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (nc + 1) * wc) return;
  const int I = idx / wc, d = idx % wc - rc, I2 = I + d;
  double2 acc = make_double2(0, 0);
  if (I2 >= 0 && I2 <= nc) {
    for (int a = 2 * I - 2; a <= 2 * I + 2; ++a) {
      if (a < 0 || a > nf) continue;
      for (int a2 = 2 * I2 - 2; a2 <= 2 * I2 + 2; ++a2) {
        const int e = a2 - a;
        if (a2 < 0 || a2 > nf || e < -rf || e > rf) continue;
        const double wgt = 0.5 * xw.w<double>(a - 2 * I) * xw.w<double>(a2 - 2 * I2);
        const double2 xv = X[a * wf + e + rf];
        acc.x += wgt * xv.x;
        acc.y += wgt * xv.y;
      }
    }
  }
  Xc[idx] = acc;
}

__global__ void s_real_part(const double2* __restrict__ a, double* __restrict__ b, long long n) {
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q < n) b[q] = a[q].x;
}

__global__ void s_diaginv_op(OpView<double> v, int nx, int ny, double omega, double2* __restrict__ dinv) {
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (long long)(nx + 1) * (ny + 1)) return;
  const int i = (int)(q % (nx + 1)), j = (int)(q / (nx + 1));
  const double2 d = op_coef(v, nx, ny, i, j, 0, 0, 0.0);
  const double2 x = make_double2(omega * d.x, omega * d.y);
  const double dd = x.x * x.x + x.y * x.y;
  dinv[q] = make_double2(x.x / dd, -x.y / dd);
}

// ------------------------------------------------------------------ wrappers

void launch_factors0(int n, double h, double k, double beta2, double2* g, double2* hf, double2* w, cudaStream_t s) {
  s_factors0<<<cdiv(n + 1, 128), 128, 0, s>>>(n, h, k, beta2, g, hf, w);
}
void launch_galerkin_1d(const double2* X, int nf, int rf, double2* Xc, int rc, const Xfer& xw, cudaStream_t s) {
  const int n = (nf / 2 + 1) * (2 * rc + 1);
  s_galerkin_1d<<<cdiv(n, 128), 128, 0, s>>>(X, nf, rf, Xc, rc, xw);
}
void launch_real_part(const double2* a, double* b, long long n, cudaStream_t s) {
  if (n > 0) s_real_part<<<cdiv(n, 256), 256, 0, s>>>(a, b, n);
}
void launch_diaginv_op(const OpView<double>& op, int nx, int ny, double omega, double2* dinv, cudaStream_t s) {
  const long long n = (long long)(nx + 1) * (ny + 1);
  s_diaginv_op<<<cdiv(n, 256), 256, 0, s>>>(op, nx, ny, omega, dinv);
}

void launch_op0consts(Op0Consts<double>* c64, Op0Consts<float>* c32, double h, double k, double omega, double beta2,
                      int abc, cudaStream_t s) {
  s_op0consts<<<1, 32, 0, s>>>(c64, c32, h, k, omega, beta2, abc);
}
void launch_galerkin(const OpView<double>& fine, int fnx, int fny, double2* cst, int cnx, int cny, int rc, double beta2,
                     const Xfer& xw, cudaStream_t s) {
  const int rf = fine.kind == 1 ? 1 : fine.kind;
  const long long n = (long long)(cnx + 1) * (cny + 1) * (2 * rc + 1) * (2 * rc + 1);
  s_galerkin<<<cdiv(n, 128), 128, 0, s>>>(fine, fnx, fny, rf, cst, cnx, cny, rc, beta2, xw);
}
void launch_diaginv(const double2* st, int rc, long long plane, double omega, double2* dinv, cudaStream_t s) {
  s_diaginv<<<cdiv(plane, 256), 256, 0, s>>>(st, rc, plane, omega, dinv);
}
void launch_to_float(const double2* src, float2* dst, long long n, cudaStream_t s) {
  if (n > 0) s_to_float<<<cdiv(n, 256), 256, 0, s>>>(src, dst, n);
}
void launch_to_float_real(const double* src, float* dst, long long n, cudaStream_t s) {
  if (n > 0) s_to_float_real<<<cdiv(n, 256), 256, 0, s>>>(src, dst, n);
}
void launch_dense(const OpView<double>& op, int nx, int ny, double2* M, cudaStream_t s) {
  const long long N = (long long)(nx + 1) * (ny + 1);
  s_dense<<<cdiv(N * N, 256), 256, 0, s>>>(op, nx, ny, M);
}
void launch_gauss_jordan(double2* M, double2* inv, int N, int* status, cudaStream_t s) {
  s_gauss_jordan<<<1, 256, (size_t)N * sizeof(double2), s>>>(M, inv, N, status);
}
void launch_export_stencil(const OpView<double>& op, int nx, int ny, int r, double2* out, cudaStream_t s) {
  const long long n = (long long)(nx + 1) * (ny + 1) * (2 * r + 1) * (2 * r + 1);
  s_export<<<cdiv(n, 256), 256, 0, s>>>(op, nx, ny, r, out);
}
template <class T>
void launch_coarse_solve(const Grid& g, const double2* inv, int N, const cx<T>* r, cx<T>* e, int B, const int* active,
                         cudaStream_t s) {
  s_coarse_solve<T><<<B, 128, (size_t)N * sizeof(double2), s>>>(g, inv, N, r, e, active);
}
template void launch_coarse_solve<double>(const Grid&, const double2*, int, const double2*, double2*, int, const int*,
                                          cudaStream_t);
template void launch_coarse_solve<float>(const Grid&, const double2*, int, const float2*, float2*, int, const int*,
                                         cudaStream_t);

}  // namespace hmg
