// Dense two-grid analysis of a hierarchy's two finest levels (Sec. 3 of the
// paper), on small grids: the two-grid iteration matrix
//   T0 = (I - P A_1^{-1} R A)(I - X^{-1} A)^nu,   X = omega diag(A),
// (Eq. (tgi1); as an error propagator the sweeps act first, the paper's
// post-smoothing), its spectral norm (Table conv1), and the simplified
// operator of Definition def2s
//   D~ = X^{-1} + P A_1^{-1} R,   Gamma~ = A^H D~^H + D~ A - A^H D~^H D~ A,
// with the Hermitian-positive-definite test by Cholesky (Sec. 3, after
// Cor. mgc1) and ||Gamma~||_1 / kappa_1(Gamma~) (Cor. mgc2, Table opt1).
// A is the fine operator, A_1 the level-1 Galerkin operator of the handle
// (built on the CSL with the handle's shift), P and R = P^T / 4 the handle's
// transfers.  With E = D~ A = P A_1^{-1} R A + X^{-1} A, Gamma~ = E + E^H -
// E^H E, so E costs no extra product.
//
// Everything is FP64 complex on CUDA cores (GB300's tensor cores offer no
// fast FP64): a tiled complex GEMM with conjugate-transpose operands, a
// multi-block Gauss-Jordan inverse with partial pivoting (one pivot kernel
// and one elimination kernel per column), a right-looking Cholesky (one
// pivot kernel and one trailing-update kernel per column; a non-positive
// pivot stops it), and the power method on T0^H T0 for ||T0||_2.
#include <math.h>

#include <algorithm>
#include <vector>

#include "internal.h"

namespace hmg {

namespace {

// ------------------------------------------------------------------ GEMM

// C = alpha * op(A) op(B), all row-major; op 0 = as stored, 1 = conjugate
// transpose.  op(A) is M x K, op(B) is K x N.  64 x 64 output tile per
// block of 256 threads, 4 x 4 outputs per thread, K staged 16 at a time.
constexpr int GT = 64, GK = 16;

template <int OPA, int OPB>
__global__ void __launch_bounds__(256) k_zgemm(int M, int N, int K, double alpha, const double2* __restrict__ A,
                                               int lda, const double2* __restrict__ B, int ldb, double2* __restrict__ C,
                                               int ldc) {
  __shared__ double2 As[GK][GT + 1];
  __shared__ double2 Bs[GK][GT + 1];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int m0 = blockIdx.y * GT, n0 = blockIdx.x * GT;
  double2 acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = make_double2(0.0, 0.0);
  for (int k0 = 0; k0 < K; k0 += GK) {
    // consecutive threads read consecutive addresses of each stored matrix
    for (int q = threadIdx.x; q < GK * GT; q += 256) {
      {   // As[kk][mm] = op(A)[m0 + mm][k0 + kk]
        const int kk = OPA == 0 ? q % GK : q / GT, mm = OPA == 0 ? q / GK : q % GT;
        const int m = m0 + mm, k = k0 + kk;
        double2 v = make_double2(0.0, 0.0);
        if (m < M && k < K) {
          if (OPA == 0) v = A[(long long)m * lda + k];
          else { v = A[(long long)k * lda + m]; v.y = -v.y; }
        }
        As[kk][mm] = v;
      }
      {   // Bs[kk][nn] = op(B)[k0 + kk][n0 + nn]
        const int kk = OPB == 0 ? q / GT : q % GK, nn = OPB == 0 ? q % GT : q / GK;
        const int n = n0 + nn, k = k0 + kk;
        double2 w = make_double2(0.0, 0.0);
        if (n < N && k < K) {
          if (OPB == 0) w = B[(long long)k * ldb + n];
          else { w = B[(long long)n * ldb + k]; w.y = -w.y; }
        }
        Bs[kk][nn] = w;
      }
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < GK; ++kk) {
      double2 av[4], bv[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) av[a] = As[kk][ty + 16 * a];
#pragma unroll
      for (int b = 0; b < 4; ++b) bv[b] = Bs[kk][tx + 16 * b];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = fma_c<double>(av[a], bv[b], acc[a][b]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int m = m0 + ty + 16 * a, n = n0 + tx + 16 * b;
      if (m < M && n < N) C[(long long)m * ldc + n] = make_double2(alpha * acc[a][b].x, alpha * acc[a][b].y);
    }
}

void zgemm(int opa, int opb, int M, int N, int K, double alpha, const double2* A, int lda, const double2* B, int ldb,
           double2* C, int ldc, cudaStream_t s) {
  const dim3 grid(cdiv(N, GT), cdiv(M, GT));
  if (opa == 0 && opb == 0) k_zgemm<0, 0><<<grid, 256, 0, s>>>(M, N, K, alpha, A, lda, B, ldb, C, ldc);
  else if (opa == 0) k_zgemm<0, 1><<<grid, 256, 0, s>>>(M, N, K, alpha, A, lda, B, ldb, C, ldc);
  else if (opb == 0) k_zgemm<1, 0><<<grid, 256, 0, s>>>(M, N, K, alpha, A, lda, B, ldb, C, ldc);
  else k_zgemm<1, 1><<<grid, 256, 0, s>>>(M, N, K, alpha, A, lda, B, ldb, C, ldc);
}

// ------------------------------------------------------------------ elementwise builders

// P[r][c]: fine node r = i + j (fnx+1), coarse node c = I + J (cnx+1),
// weight w(i - 2I) w(j - 2J) (tensor product of the 1D column stencils).
__global__ void k_dense_p(int fnx, int fny, int cnx, int cny, Xfer xw, double2* __restrict__ P) {
  const long long Nf = (long long)(fnx + 1) * (fny + 1), Nc = (long long)(cnx + 1) * (cny + 1);
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= Nf * Nc) return;
  const long long r = q / Nc, c = q % Nc;
  const int i = (int)(r % (fnx + 1)), j = (int)(r / (fnx + 1));
  const int I = (int)(c % (cnx + 1)), J = (int)(c / (cnx + 1));
  P[q] = make_double2(xw.w<double>(i - 2 * I) * xw.w<double>(j - 2 * J), 0.0);
}

// S = I - X^{-1} A, X = omega diag(A)
__global__ void k_smoother(int N, double omega, const double2* __restrict__ A, double2* __restrict__ S) {
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (long long)N * N) return;
  const long long r = q / N, c = q % N;
  const double2 xi = cinv<double>(scl<double>(omega, A[r * N + r]));
  const double2 v = mul<double>(xi, A[q]);
  S[q] = make_double2((r == c ? 1.0 : 0.0) - v.x, -v.y);
}

// CGC = I - CG (in place)
__global__ void k_identity_minus(int N, double2* __restrict__ X) {
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (long long)N * N) return;
  const long long r = q / N, c = q % N;
  X[q] = make_double2((r == c ? 1.0 : 0.0) - X[q].x, -X[q].y);
}

// E = CG + (I - S) = D~ A  (CG = P A_1^{-1} R A, I - S = X^{-1} A)
__global__ void k_e_matrix(int N, const double2* __restrict__ CG, const double2* __restrict__ S,
                           double2* __restrict__ E) {
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (long long)N * N) return;
  const long long r = q / N, c = q % N;
  E[q] = make_double2(CG[q].x + (r == c ? 1.0 : 0.0) - S[q].x, CG[q].y - S[q].y);
}

// Gamma~ = E + E^H - EHE (EHE holds E^H E; overwritten by Gamma~)
__global__ void k_gamma(int N, const double2* __restrict__ E, double2* __restrict__ G) {
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (long long)N * N) return;
  const long long r = q / N, c = q % N;
  const double2 e = E[q], et = E[c * N + r];
  G[q] = make_double2(e.x + et.x - G[q].x, e.y - et.y - G[q].y);
}

// max |B - B^H| and max |B| (one block; out[0], out[1])
__global__ void k_herm_check(int N, const double2* __restrict__ B, double* out) {
  __shared__ double sh[2][32];
  double d = 0.0, m = 0.0;
  for (long long q = threadIdx.x; q < (long long)N * N; q += blockDim.x) {
    const long long r = q / N, c = q % N;
    const double2 b = B[q], t = B[c * N + r];
    d = fmax(d, hypot(b.x - t.x, b.y + t.y));
    m = fmax(m, hypot(b.x, b.y));
  }
  for (int o = 16; o > 0; o >>= 1) {
    d = fmax(d, __shfl_down_sync(0xffffffffu, d, o));
    m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
  }
  if ((threadIdx.x & 31) == 0) {
    sh[0][threadIdx.x >> 5] = d;
    sh[1][threadIdx.x >> 5] = m;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
      d = fmax(d, sh[0][w]);
      m = fmax(m, sh[1][w]);
    }
    d = fmax(d, sh[0][0]);
    m = fmax(m, sh[1][0]);
    out[0] = d;
    out[1] = m;
  }
}

// H = (B + B^H) / 2
__global__ void k_hermitian_part(int N, const double2* __restrict__ B, double2* __restrict__ H) {
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (long long)N * N) return;
  const long long r = q / N, c = q % N;
  const double2 b = B[q], t = B[c * N + r];
  H[q] = make_double2(0.5 * (b.x + t.x), 0.5 * (b.y - t.y));
}

// out = max_c sum_r |B[r][c]| (1-norm), one block per 32 columns then a max
__global__ void k_col_abs_sums(int N, const double2* __restrict__ B, double* __restrict__ colsum) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= N) return;
  double s = 0.0;
  for (int r = 0; r < N; ++r) {
    const double2 b = B[(long long)r * N + c];
    s += hypot(b.x, b.y);
  }
  colsum[c] = s;
}
__global__ void k_max(int N, const double* __restrict__ v, double* out) {
  __shared__ double sh[32];
  double m = 0.0;
  for (int q = threadIdx.x; q < N; q += blockDim.x) m = fmax(m, v[q]);
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = fmax(m, sh[w]);
    *out = m;
  }
}

// ------------------------------------------------------------------ Gauss-Jordan (multi-block)

// Column k: the pivot row p >= k of largest modulus, swapped into row k of
// M and of W (W starts as the identity), then row k scaled by 1/M[k][k].
// One block.  st[0] = 1 on a zero pivot.
__global__ void k_gj_pivot(int N, int k, double2* __restrict__ M, double2* __restrict__ W, int* st) {
  __shared__ double bv[32];
  __shared__ int bi[32];
  __shared__ int piv;
  __shared__ double2 dinv;
  double best = -1.0;
  int arg = k;
  for (int r = k + threadIdx.x; r < N; r += blockDim.x) {
    const double2 a = M[(long long)r * N + k];
    const double m = a.x * a.x + a.y * a.y;
    if (m > best) { best = m; arg = r; }
  }
  for (int o = 16; o > 0; o >>= 1) {
    const double b2 = __shfl_down_sync(0xffffffffu, best, o);
    const int a2 = __shfl_down_sync(0xffffffffu, arg, o);
    if (b2 > best || (b2 == best && a2 < arg)) { best = b2; arg = a2; }
  }
  if ((threadIdx.x & 31) == 0) { bv[threadIdx.x >> 5] = best; bi[threadIdx.x >> 5] = arg; }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
      if (bv[w] > bv[0] || (bv[w] == bv[0] && bi[w] < bi[0])) { bv[0] = bv[w]; bi[0] = bi[w]; }
    piv = bi[0];
    if (!(bv[0] > 0.0)) st[0] = 1;
  }
  __syncthreads();
  const int p = piv;
  if (p != k)
    for (int c = threadIdx.x; c < N; c += blockDim.x) {
      double2 t = M[(long long)k * N + c]; M[(long long)k * N + c] = M[(long long)p * N + c]; M[(long long)p * N + c] = t;
      t = W[(long long)k * N + c]; W[(long long)k * N + c] = W[(long long)p * N + c]; W[(long long)p * N + c] = t;
    }
  __syncthreads();
  if (threadIdx.x == 0) {
    const double2 d = M[(long long)k * N + k];
    const double dd = d.x * d.x + d.y * d.y;
    dinv = dd > 0 ? make_double2(d.x / dd, -d.y / dd) : make_double2(0.0, 0.0);
  }
  __syncthreads();
  for (int c = threadIdx.x; c < N; c += blockDim.x) {
    M[(long long)k * N + c] = mul<double>(dinv, M[(long long)k * N + c]);
    W[(long long)k * N + c] = mul<double>(dinv, W[(long long)k * N + c]);
  }
}

// Every row r != k: row_r -= M[r][k] row_k, in M (columns > k; column k is
// set to zero) and in W.  fac[r] = M[r][k] is read before the update.
__global__ void k_gj_eliminate(int N, int k, double2* __restrict__ M, double2* __restrict__ W,
                               const double2* __restrict__ fac) {
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= 2LL * N * N) return;
  const bool inW = q >= (long long)N * N;
  const long long e = inW ? q - (long long)N * N : q;
  const long long r = e / N, c = e % N;
  if (r == k) return;
  double2* X = inW ? W : M;
  const double2 f = fac[r];
  if (!inW && c == k) { X[e] = make_double2(0.0, 0.0); return; }
  if (!inW && c < k) return;   // columns left of k are already eliminated
  X[e] = sub<double>(X[e], mul<double>(f, X[(long long)k * N + c]));
}
__global__ void k_copy_col(int N, int k, const double2* __restrict__ M, double2* __restrict__ fac) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r < N) fac[r] = M[(long long)r * N + k];
}
__global__ void k_identity(int N, double2* __restrict__ W) {
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (long long)N * N) return;
  W[q] = make_double2((q / N == q % N) ? 1.0 : 0.0, 0.0);
}

// ------------------------------------------------------------------ Cholesky (HPD test)

// Column k of H = L L^H (lower part, in place): pivot d = Re H[k][k] (> 0,
// else st[0] = 1 and the factorisation stops), L[k][k] = sqrt(d), and
// L[r][k] = H[r][k] / L[k][k] for r > k.  One block.
__global__ void k_chol_pivot(int N, int k, double2* __restrict__ H, int* st) {
  __shared__ double l;
  if (st[0]) return;
  if (threadIdx.x == 0) {
    const double d = H[(long long)k * N + k].x;
    if (!(d > 0.0)) st[0] = 1;
    l = d > 0.0 ? sqrt(d) : 0.0;
    H[(long long)k * N + k] = make_double2(l, 0.0);
  }
  __syncthreads();
  if (st[0] || l == 0.0) return;
  for (int r = k + 1 + threadIdx.x; r < N; r += blockDim.x) {
    const double2 v = H[(long long)r * N + k];
    H[(long long)r * N + k] = make_double2(v.x / l, v.y / l);
  }
}
// Trailing update H[r][c] -= L[r][k] conj(L[c][k]) for k < c <= r.
__global__ void k_chol_update(int N, int k, double2* __restrict__ H, const int* st) {
  if (st[0]) return;
  const int m = N - k - 1;
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (long long)m * m) return;
  const int r = k + 1 + (int)(q / m), c = k + 1 + (int)(q % m);
  if (c > r) return;
  const double2 a = H[(long long)r * N + k], b = H[(long long)c * N + k];
  const double2 ab = make_double2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);   // a conj(b)
  H[(long long)r * N + c] = sub<double>(H[(long long)r * N + c], ab);
}

// ------------------------------------------------------------------ power method on B = T0^H T0

// y = B v (one warp per row)
__global__ void k_gemv(int N, const double2* __restrict__ B, const double2* __restrict__ v, double2* __restrict__ y) {
  const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (row >= N) return;
  double2 acc = make_double2(0.0, 0.0);
  for (int c = lane; c < N; c += 32) acc = fma_c<double>(B[(long long)row * N + c], v[c], acc);
  for (int o = 16; o > 0; o >>= 1) {
    acc.x += __shfl_down_sync(0xffffffffu, acc.x, o);
    acc.y += __shfl_down_sync(0xffffffffu, acc.y, o);
  }
  if (lane == 0) y[row] = acc;
}
// lam[it] = Re(v^H y) (Rayleigh quotient, ||v|| = 1), then v = y / ||y||.  One block.
__global__ void k_power_step(int N, double2* __restrict__ v, const double2* __restrict__ y, double* lam, int it) {
  __shared__ double sh[2][32];
  __shared__ double s_nrm;
  double rq = 0.0, nn = 0.0;
  for (int q = threadIdx.x; q < N; q += blockDim.x) {
    rq += v[q].x * y[q].x + v[q].y * y[q].y;
    nn += abs2<double>(y[q]);
  }
  for (int o = 16; o > 0; o >>= 1) {
    rq += __shfl_down_sync(0xffffffffu, rq, o);
    nn += __shfl_down_sync(0xffffffffu, nn, o);
  }
  if ((threadIdx.x & 31) == 0) { sh[0][threadIdx.x >> 5] = rq; sh[1][threadIdx.x >> 5] = nn; }
  __syncthreads();
  if (threadIdx.x == 0) {
    rq = nn = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { rq += sh[0][w]; nn += sh[1][w]; }
    lam[it] = rq;
    s_nrm = sqrt(nn);
  }
  __syncthreads();
  const double s = s_nrm > 0.0 ? 1.0 / s_nrm : 0.0;
  for (int q = threadIdx.x; q < N; q += blockDim.x) v[q] = make_double2(y[q].x * s, y[q].y * s);
}
// A fixed start vector with every component nonzero: v_q = (1 + (q mod 7)/7) / norm.
__global__ void k_power_init(int N, double2* __restrict__ v) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q < N) v[q] = make_double2((1.0 + (q % 7) / 7.0) / sqrt((double)N), 0.0);
}

inline int nb(long long n, int t = 256) { return cdiv(n, t); }

}  // namespace

// Host driver, see internal.h.  Device scratch is allocated here and freed on return.
cudaError_t two_grid_analysis(const OpView<double>& fine, const OpView<double>& coarse, int fnx, int fny, int cnx,
                              int cny, double omega, const Xfer& xw, int nu, int max_iter, double* out,
                              cudaStream_t s) {
  const int N = (fnx + 1) * (fny + 1), Nc = (cnx + 1) * (cny + 1);
  const size_t NN = (size_t)N * N;
  std::vector<void*> mem;
  cudaError_t e = cudaSuccess;
  auto alloc = [&](size_t bytes) -> void* {
    void* p = nullptr;
    if (e == cudaSuccess) e = cudaMalloc(&p, bytes);
    if (e == cudaSuccess) mem.push_back(p);
    return p;
  };
  double2* A = (double2*)alloc(NN * 16);
  double2* S = (double2*)alloc(NN * 16);
  double2* T = (double2*)alloc(NN * 16);
  double2* U = (double2*)alloc(NN * 16);
  double2* V = (double2*)alloc(NN * 16);
  double2* Ac = (double2*)alloc((size_t)Nc * Nc * 16);
  double2* Aci = (double2*)alloc((size_t)Nc * Nc * 16);
  double2* P = (double2*)alloc((size_t)N * Nc * 16);
  double2* Y = (double2*)alloc((size_t)Nc * N * 16);
  double2* fac = (double2*)alloc((size_t)N * 16);
  double2* pv = (double2*)alloc((size_t)N * 16);
  double2* py = (double2*)alloc((size_t)N * 16);
  double* colsum = (double*)alloc((size_t)N * 8);
  double* scal = (double*)alloc(8 * 8);
  double* lam = (double*)alloc((size_t)max_iter * 8);
  int* st = (int*)alloc(4 * sizeof(int));
  auto release = [&]() {
    for (void* p : mem) cudaFree(p);
  };
  if (e != cudaSuccess) {
    release();
    return e;
  }
  cudaMemsetAsync(st, 0, 4 * sizeof(int), s);
  auto inverse = [&](double2* M, double2* W, int n, int* flag) {   // W = M^{-1}, M destroyed
    k_identity<<<nb((long long)n * n), 256, 0, s>>>(n, W);
    for (int k = 0; k < n; ++k) {
      k_gj_pivot<<<1, 256, 0, s>>>(n, k, M, W, flag);
      k_copy_col<<<nb(n), 256, 0, s>>>(n, k, M, fac);
      k_gj_eliminate<<<nb(2LL * n * n), 256, 0, s>>>(n, k, M, W, fac);
    }
  };
  // A, S = I - X^{-1} A, A_1^{-1}, P, Y = A_1^{-1} R = A_1^{-1} P^T / 4
  launch_dense(fine, fnx, fny, A, s);
  k_smoother<<<nb(NN), 256, 0, s>>>(N, omega, A, S);
  launch_dense(coarse, cnx, cny, Ac, s);
  inverse(Ac, Aci, Nc, st + 1);
  k_dense_p<<<nb((long long)N * Nc), 256, 0, s>>>(fnx, fny, cnx, cny, xw, P);
  zgemm(0, 1, Nc, N, Nc, 0.25, Aci, Nc, P, Nc, Y, N, s);
  // U = P Y = P A_1^{-1} R;  V = CG = U A;  T = S^nu;  U = CGC = I - CG;  then T0 = CGC S^nu in A's slot
  zgemm(0, 0, N, N, Nc, 1.0, P, Nc, Y, N, U, N, s);
  zgemm(0, 0, N, N, N, 1.0, U, N, A, N, V, N, s);
  cudaMemcpyAsync(T, S, NN * 16, cudaMemcpyDeviceToDevice, s);
  for (int q = 1; q < nu; ++q) {   // T = S T
    zgemm(0, 0, N, N, N, 1.0, S, N, T, N, U, N, s);
    std::swap(T, U);
  }
  cudaMemcpyAsync(U, V, NN * 16, cudaMemcpyDeviceToDevice, s);
  k_identity_minus<<<nb(NN), 256, 0, s>>>(N, U);
  double2* T0 = A;   // A is no longer needed
  zgemm(0, 0, N, N, N, 1.0, U, N, T, N, T0, N, s);
  // B = T0^H T0 (in T), power method
  zgemm(1, 0, N, N, N, 1.0, T0, N, T0, N, T, N, s);
  k_power_init<<<nb(N), 256, 0, s>>>(N, pv);
  std::vector<double> lh(max_iter);
  int it = 0;
  double lam_last = 0.0;
  bool conv = false;
  while (it < max_iter && !conv) {
    const int chunk = std::min(100, max_iter - it);
    for (int q = 0; q < chunk; ++q, ++it) {
      k_gemv<<<nb((long long)N * 32), 256, 0, s>>>(N, T, pv, py);
      k_power_step<<<1, 256, 0, s>>>(N, pv, py, lam, it);
    }
    if ((e = cudaMemcpyAsync(lh.data(), lam, sizeof(double) * it, cudaMemcpyDeviceToHost, s)) != cudaSuccess) break;
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) break;
    const double l = lh[it - 1];
    conv = it >= 200 && fabs(l - lam_last) <= 1e-14 * fabs(l);
    lam_last = l;
  }
  // E = CG + X^{-1} A (S still holds I - X^{-1} A, V holds CG), in U; Gamma~ in V
  k_e_matrix<<<nb(NN), 256, 0, s>>>(N, V, S, U);
  zgemm(1, 0, N, N, N, 1.0, U, N, U, N, V, N, s);
  k_gamma<<<nb(NN), 256, 0, s>>>(N, U, V);
  // Hermitian check, Cholesky of the Hermitian part (in T)
  k_herm_check<<<1, 1024, 0, s>>>(N, V, scal);
  k_hermitian_part<<<nb(NN), 256, 0, s>>>(N, V, T);
  for (int k = 0; k < N; ++k) {
    k_chol_pivot<<<1, 256, 0, s>>>(N, k, T, st + 2);
    if (k + 1 < N) k_chol_update<<<nb((long long)(N - k - 1) * (N - k - 1)), 256, 0, s>>>(N, k, T, st + 2);
  }
  // ||Gamma~||_1 and ||Gamma~^{-1}||_1 (Gamma~ copied to S, inverted into T)
  k_col_abs_sums<<<nb(N, 128), 128, 0, s>>>(N, V, colsum);
  k_max<<<1, 256, 0, s>>>(N, colsum, scal + 2);
  cudaMemcpyAsync(S, V, NN * 16, cudaMemcpyDeviceToDevice, s);
  inverse(S, T, N, st + 3);
  k_col_abs_sums<<<nb(N, 128), 128, 0, s>>>(N, T, colsum);
  k_max<<<1, 256, 0, s>>>(N, colsum, scal + 3);
  double hs[4];
  int hst[4];
  if (e == cudaSuccess) e = cudaMemcpyAsync(hs, scal, sizeof(hs), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(hst, st, sizeof(hst), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = cudaGetLastError();
  release();
  if (e != cudaSuccess) return e;
  out[0] = sqrt(std::max(lam_last, 0.0));
  const bool herm = hs[0] <= 1e-10 * hs[1];
  out[1] = (herm && hst[2] == 0) ? 1.0 : 0.0;
  out[2] = hst[3] ? NAN : hs[2] / (hs[2] * hs[3]);
  out[3] = it;
  out[4] = conv ? 1.0 : 0.0;
  out[5] = hst[1] ? 1.0 : 0.0;   // singular coarse operator
  return cudaSuccess;
}

}  // namespace hmg
