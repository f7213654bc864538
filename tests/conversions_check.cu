// Test harness (compiled by tests/test_gpu_conversions.py): runs the
// library's integer-pipe IEEE conversions and the hardware conversions on
// the same inputs and returns both results' bit patterns.
#include <cuda_runtime.h>

#include "../paper_2308_13476_gb300/csrc/common.cuh"

using namespace hmg;

__global__ void k_d2f(const double* __restrict__ in, unsigned* __restrict__ lib, unsigned* __restrict__ hw, int n) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  lib[t] = __float_as_uint(f32_from_f64_rn(in[t]));
  hw[t] = __float_as_uint(__double2float_rn(in[t]));
}

__global__ void k_f2d(const float* __restrict__ in, unsigned long long* __restrict__ lib,
                      unsigned long long* __restrict__ hw, int n) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  lib[t] = (unsigned long long)__double_as_longlong(f64_from_f32(in[t]));
  hw[t] = (unsigned long long)__double_as_longlong((double)in[t]);
}

// Host arrays in and out; returns 0, or the CUDA error code.
extern "C" int check_d2f(const double* in, unsigned* lib, unsigned* hw, int n) {
  double* d_in = nullptr;
  unsigned *d_lib = nullptr, *d_hw = nullptr;
  cudaError_t e = cudaMalloc(&d_in, sizeof(double) * n);
  if (e == cudaSuccess) e = cudaMalloc(&d_lib, sizeof(unsigned) * n);
  if (e == cudaSuccess) e = cudaMalloc(&d_hw, sizeof(unsigned) * n);
  if (e == cudaSuccess) e = cudaMemcpy(d_in, in, sizeof(double) * n, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    k_d2f<<<(n + 255) / 256, 256>>>(d_in, d_lib, d_hw, n);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(lib, d_lib, sizeof(unsigned) * n, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(hw, d_hw, sizeof(unsigned) * n, cudaMemcpyDeviceToHost);
  cudaFree(d_in);
  cudaFree(d_lib);
  cudaFree(d_hw);
  return (int)e;
}

extern "C" int check_f2d(const float* in, unsigned long long* lib, unsigned long long* hw, int n) {
  float* d_in = nullptr;
  unsigned long long *d_lib = nullptr, *d_hw = nullptr;
  cudaError_t e = cudaMalloc(&d_in, sizeof(float) * n);
  if (e == cudaSuccess) e = cudaMalloc(&d_lib, sizeof(unsigned long long) * n);
  if (e == cudaSuccess) e = cudaMalloc(&d_hw, sizeof(unsigned long long) * n);
  if (e == cudaSuccess) e = cudaMemcpy(d_in, in, sizeof(float) * n, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    k_f2d<<<(n + 255) / 256, 256>>>(d_in, d_lib, d_hw, n);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(lib, d_lib, sizeof(unsigned long long) * n, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(hw, d_hw, sizeof(unsigned long long) * n, cudaMemcpyDeviceToHost);
  cudaFree(d_in);
  cudaFree(d_lib);
  cudaFree(d_hw);
  return (int)e;
}
