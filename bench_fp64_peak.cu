// Benchmark tool (built and loaded by bench.py; not part of the library): the FP64 pipe peak of
// the current GPU, as the DFMA throughput of a dependent-free stream (8 independent FMA chains
// per thread, a few waves of blocks per SM). This is the denominator of the ALU roofline the
// FP64 sampler is bound by.
#include <cuda_runtime.h>

namespace {

__global__ void dfma_stream(double* out, int iters, double a, double b) {
  double x0 = threadIdx.x * 1e-3, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3;
  double x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6, x7 = x0 + 7;
  for (int i = 0; i < iters; ++i) {
    x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
    x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}

}  // namespace

// DFMA operations per second (one DFMA = 2 FP64 flops) on `device`; 0 on success.
extern "C" int chm_fp64_dfma_rate(int device, double* dfma_per_s) {
  if (!dfma_per_s) return -1;
  if (cudaSetDevice(device) != cudaSuccess) return -3;
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return -3;
  const int block = 256, grid = sms * 8, iters = 20000;
  double* out = nullptr;
  if (cudaMalloc(&out, sizeof(double) * grid * block) != cudaSuccess) return -2;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  dfma_stream<<<grid, block>>>(out, iters / 10, 0.999999, 1e-6);  // warm-up
  cudaEventRecord(e0);
  dfma_stream<<<grid, block>>>(out, iters, 0.999999, 1e-6);
  cudaEventRecord(e1);
  cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  const cudaError_t err = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (err != cudaSuccess || ms <= 0.f) return -3;
  *dfma_per_s = static_cast<double>(grid) * block * iters * 8.0 / (ms * 1e-3);
  return 0;
}
