// mg_residual_norm_static: the fine-level residual norm without any device
// allocation.
//
// Every other entry point of this library works through a handle whose
// mg_setup allocates device memory, and the norm reductions inside them
// keep their block partials in that memory.  Some callers cannot allocate
// device memory at the point where they need a residual: code that runs
// while another framework's memory pool owns the device (its caching
// allocator has reserved what it needs and raw allocations would fight it or
// fail), code on a latency-critical loop where an allocation's implicit
// device-wide synchronisation is not acceptable, or code in a context where
// allocation is simply not permitted.  This entry point keeps its scratch (the
// per-block partial sums and the completion ticket) in one file-scope device
// array instead, sized for a fixed maximum number of thread blocks.
//
// Set-up: the first call on each device looks up the array's device address
// with cudaGetSymbolAddress (the array's name in host code is only a host-side
// stand-in, not a device address) and caches it; make that first call on a
// device before any stream capture.  Calls share the array and it keeps the
// last call's contents, so each call clears its ticket first; calls whose
// kernels overlap on the GPU (different streams, or different host threads
// on the same device) race on the array and must be serialised by the caller.
#include <mutex>

#include "../../include/helmmg.h"
#include "internal.h"

namespace hmg {

namespace {
constexpr int NA_BX = 32, NA_BY = 8, NA_RY = 4;      // a block covers 32 x 32 grid nodes
constexpr int NA_MAX_BLOCKS = 16384;                  // -> at most 16.7 M nodes
constexpr int NA_MAX_DEVICES = 64;
}  // namespace

// [blk][2] partial sums (|r|^2, |b|^2) followed by the ticket; 256 KiB + 256 B.
static __device__ __align__(256) double g_noalloc_scratch[2 * NA_MAX_BLOCKS + 32];

// Same operator as Op0 (ghost-eliminated Sommerfeld rows scaled by 1/2 and
// 1/4), on the caller's dense [ny+1][nx+1] layout, neighbours off the grid
// read as zero.
__global__ void __launch_bounds__(NA_BX * NA_BY)
    k_resnorm_dense(int nx, int ny, double inv_h2, double inv_h, double kc, const double* __restrict__ kf,
                    const double2* __restrict__ x, const double2* __restrict__ b, double* scratch,
                    double* __restrict__ out) {
  __shared__ double sh[2 * 32];
  __shared__ int s_last;
  const int i = blockIdx.x * NA_BX + threadIdx.x;
  const int nblk = gridDim.x * gridDim.y, blk = blockIdx.y * gridDim.x + blockIdx.x;
  double v[2] = {0.0, 0.0};
  if (i <= nx) {
    for (int r_ = 0, j = blockIdx.y * NA_BY * NA_RY + threadIdx.y; r_ < NA_RY; ++r_, j += NA_BY) {
      if (j > ny) break;
      const long long q = (long long)j * (nx + 1) + i;
      const int bx = (i == 0 || i == nx), by = (j == 0 || j == ny);
      const double wx = bx ? 0.5 : 1.0, wy = by ? 0.5 : 1.0, w = wx * wy;
      const double k = kf ? kf[q] : kc;
      const double2 xp = x[q];
      const double2 z = make_double2(0.0, 0.0);
      const double2 xe = i < nx ? x[q + 1] : z, xw = i > 0 ? x[q - 1] : z;
      const double2 xn = j < ny ? x[q + nx + 1] : z, xs = j > 0 ? x[q - nx - 1] : z;
      const double sr = wy * (xe.x + xw.x) + wx * (xn.x + xs.x), si = wy * (xe.y + xw.y) + wx * (xn.y + xs.y);
      const double re = (4.0 * w * xp.x - sr) * inv_h2 - (w * (k * k)) * xp.x;
      const double im = (4.0 * w * xp.y - si) * inv_h2 - (w * (k * k)) * xp.y;
      const double sb = (k * inv_h) * (bx * wy + wx * by);
      const double2 bq = b[q];
      const double rx = bq.x - (re + sb * xp.y), ry = bq.y - (im - sb * xp.x);
      v[0] += rx * rx + ry * ry;
      v[1] += bq.x * bq.x + bq.y * bq.y;
    }
  }
  block_sum<2>(v, sh);
  const int tid = threadIdx.x + threadIdx.y * blockDim.x;
  unsigned* ticket = reinterpret_cast<unsigned*>(scratch + 2 * NA_MAX_BLOCKS);
  if (tid == 0) {
    scratch[2 * blk] = v[0];
    scratch[2 * blk + 1] = v[1];
    __threadfence();
    s_last = atomicAdd(ticket, 1u) == (unsigned)(nblk - 1);
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  double a[2] = {0.0, 0.0};
  for (int q = tid; q < nblk; q += blockDim.x * blockDim.y) {
    a[0] += __ldcg(scratch + 2 * q);
    a[1] += __ldcg(scratch + 2 * q + 1);
  }
  block_sum<2>(a, sh);
  if (tid == 0) {
    out[0] = sqrt(a[0]);
    out[1] = sqrt(a[1]);
    *ticket = 0u;
  }
}

}  // namespace hmg

using namespace hmg;

static std::mutex g_noalloc_mu;
static double* g_noalloc_ptr[NA_MAX_DEVICES] = {};

extern "C" mg_status mg_residual_norm_static(int nx, int ny, double h, const double* k_field, double k_const,
                                             const void* x, const void* b, double* out, void* stream) {
  if (nx < 2 || ny < 2 || !(h > 0) || !x || !b || !out || (!k_field && !(k_const >= 0))) {
    hmg_set_error("mg_residual_norm_static: need nx, ny >= 2, h > 0, k >= 0 and non-NULL x, b, out");
    return MG_EINVAL;
  }
  const long long nbx = (nx + 1 + NA_BX - 1) / NA_BX, nby = (ny + 1 + NA_BY * NA_RY - 1) / (NA_BY * NA_RY);
  if (nbx * nby > NA_MAX_BLOCKS) {
    hmg_set_error("mg_residual_norm_static: grid too large for the static scratch (at most 16384 blocks of 32 x 32 "
                  "nodes, about 16.7 M nodes)");
    return MG_EINVAL;
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= NA_MAX_DEVICES) {
    hmg_set_error("mg_residual_norm_static: no usable current device");
    return MG_ECUDA;
  }
  double* scratch;
  {
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {   // once per device: the array's device address
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess || !p) {
        hmg_set_error("mg_residual_norm_static: cudaGetSymbolAddress failed");
        return MG_ECUDA;
      }
      g_noalloc_ptr[dev] = (double*)p;
    }
    scratch = g_noalloc_ptr[dev];
  }
  cudaStream_t s = (cudaStream_t)stream;
  e = cudaMemsetAsync(scratch + 2 * NA_MAX_BLOCKS, 0, sizeof(unsigned), s);   // ticket starts at zero
  if (e != cudaSuccess) {
    hmg_set_error("mg_residual_norm_static: clearing the ticket failed");
    return MG_ECUDA;
  }
  k_resnorm_dense<<<dim3((unsigned)nbx, (unsigned)nby), dim3(NA_BX, NA_BY), 0, s>>>(
      nx, ny, 1.0 / (h * h), 1.0 / h, k_field ? 0.0 : k_const, k_field, (const double2*)x, (const double2*)b, scratch,
      out);
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    hmg_set_error("mg_residual_norm_static: kernel launch failed");
    return MG_ECUDA;
  }
  return MG_OK;
}
