// Test-only probe: evaluates the sampler's table-driven exp/log on given inputs.
// Compiled by tests/test_gpu_math.py with nvcc; not part of the library.
#include <cuda_runtime.h>

#include "fp64_math.cuh"

namespace {
__global__ void probe_kernel(int which, const double* x, double* y, int n, const double* T) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  y[i] = (which == 0) ? chm::exp_tab(x[i], T) : chm::log_tab(x[i], T);
}
}  // namespace

extern "C" int probe_fp64_math(int which, const double* x_host, double* y_host, int n) {
  double *x = nullptr, *y = nullptr, *T = nullptr;
  if (cudaMalloc(&x, sizeof(double) * n) != cudaSuccess) return -1;
  if (cudaMalloc(&y, sizeof(double) * n) != cudaSuccess) return -1;
  if (cudaMalloc(&T, sizeof(double) * chm::kMathWords) != cudaSuccess) return -1;
  chm::math_table_kernel<<<2, 128>>>(T);
  cudaMemcpy(x, x_host, sizeof(double) * n, cudaMemcpyHostToDevice);
  probe_kernel<<<(n + 255) / 256, 256>>>(which, x, y, n, T);
  cudaMemcpy(y_host, y, sizeof(double) * n, cudaMemcpyDeviceToHost);
  const cudaError_t e = cudaGetLastError();
  cudaFree(x);
  cudaFree(y);
  cudaFree(T);
  return e == cudaSuccess ? 0 : -2;
}
