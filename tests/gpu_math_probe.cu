// Test-only probe: evaluates the sampler's table-driven exp/log/sincospi on given inputs.
// Compiled by tests/test_gpu_math.py with nvcc; not part of the library.
#include <cuda_runtime.h>

#include "fp64_math.cuh"

namespace {
__global__ void probe_kernel(int which, const double* x, double* y, int n, const double* T) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double sn, cs;
  switch (which) {
    case 0: y[i] = chm::exp_tab(x[i], T); break;
    case 1: y[i] = chm::log_tab(x[i], T); break;
    case 2: chm::sincospi_tab(x[i], T, &sn, &cs); y[i] = sn; break;
    case 3: chm::sincospi_tab(x[i], T, &sn, &cs); y[i] = cs; break;
    case 4: sincospi(x[i], &sn, &cs); y[i] = sn; break;
    default: sincospi(x[i], &sn, &cs); y[i] = cs; break;
  }
}
}  // namespace

extern "C" int probe_fp64_math(int which, const double* x_host, double* y_host, int n) {
  double *x = nullptr, *y = nullptr, *T = nullptr;
  if (cudaMalloc(&x, sizeof(double) * n) != cudaSuccess) return -1;
  if (cudaMalloc(&y, sizeof(double) * n) != cudaSuccess) return -1;
  if (cudaMalloc(&T, sizeof(double) * chm::kMathWords) != cudaSuccess) return -1;
  chm::math_table_kernel<<<4, 128>>>(T);
  cudaMemcpy(x, x_host, sizeof(double) * n, cudaMemcpyHostToDevice);
  probe_kernel<<<(n + 255) / 256, 256>>>(which, x, y, n, T);
  cudaMemcpy(y_host, y, sizeof(double) * n, cudaMemcpyDeviceToHost);
  const cudaError_t e = cudaGetLastError();
  cudaFree(x);
  cudaFree(y);
  cudaFree(T);
  return e == cudaSuccess ? 0 : -2;
}

// The FP32 form's binary32 exponentials next to CUDA's expf / expm1f on the same arguments.
#include "fp32_math.cuh"

namespace {
__global__ void probe32_kernel(int which, const float* x, float* y, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  switch (which) {
    case 0: y[i] = chm::exp32(x[i]); break;
    case 1: y[i] = chm::expm1_32(x[i]); break;
    case 2: y[i] = expf(x[i]); break;
    default: y[i] = expm1f(x[i]); break;
  }
}
}  // namespace

extern "C" int probe_fp32_math(int which, const float* x_host, float* y_host, int n) {
  float *x = nullptr, *y = nullptr;
  if (cudaMalloc(&x, sizeof(float) * n) != cudaSuccess) return -1;
  if (cudaMalloc(&y, sizeof(float) * n) != cudaSuccess) return -1;
  cudaMemcpy(x, x_host, sizeof(float) * n, cudaMemcpyHostToDevice);
  probe32_kernel<<<(n + 255) / 256, 256>>>(which, x, y, n);
  cudaMemcpy(y_host, y, sizeof(float) * n, cudaMemcpyDeviceToHost);
  const cudaError_t e = cudaGetLastError();
  cudaFree(x);
  cudaFree(y);
  return e == cudaSuccess ? 0 : -2;
}

// The sampler's Philox4x32-10 block next to cuRAND's Philox4_32_10 generator (its device API),
// for the same key and 128-bit counter: curand_init(seed = key1:key0, subsequence = c3:c2,
// offset = 4 (c1:c0)) puts the generator at counter (c0, c1, c2, c3) (c1 < 2^30, so that the
// offset fits 64 bits), and curand4 returns that block.
#include <cstdint>
#include <curand_kernel.h>

#include "device_common.cuh"

namespace {
__global__ void philox_kernel(const uint32_t* ctr, uint32_t k0, uint32_t k1, uint32_t* mine, uint32_t* ref, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint4 c = make_uint4(ctr[4 * i], ctr[4 * i + 1], ctr[4 * i + 2], ctr[4 * i + 3]);
  const uint4 m = chm::philox4x32_10(c, k0, k1);
  mine[4 * i] = m.x;
  mine[4 * i + 1] = m.y;
  mine[4 * i + 2] = m.z;
  mine[4 * i + 3] = m.w;
  curandStatePhilox4_32_10_t st;
  const unsigned long long seed = (static_cast<unsigned long long>(k1) << 32) | k0;
  const unsigned long long subseq = (static_cast<unsigned long long>(c.w) << 32) | c.z;
  const unsigned long long off = ((static_cast<unsigned long long>(c.y) << 32) | c.x) * 4ull;
  curand_init(seed, subseq, off, &st);
  const uint4 r = curand4(&st);
  ref[4 * i] = r.x;
  ref[4 * i + 1] = r.y;
  ref[4 * i + 2] = r.z;
  ref[4 * i + 3] = r.w;
}
}  // namespace

extern "C" int probe_philox(const uint32_t* ctr_host, uint32_t k0, uint32_t k1, uint32_t* mine_host, uint32_t* ref_host,
                            int n) {
  uint32_t *ctr = nullptr, *mine = nullptr, *ref = nullptr;
  if (cudaMalloc(&ctr, sizeof(uint32_t) * 4 * n) != cudaSuccess) return -1;
  if (cudaMalloc(&mine, sizeof(uint32_t) * 4 * n) != cudaSuccess) return -1;
  if (cudaMalloc(&ref, sizeof(uint32_t) * 4 * n) != cudaSuccess) return -1;
  cudaMemcpy(ctr, ctr_host, sizeof(uint32_t) * 4 * n, cudaMemcpyHostToDevice);
  philox_kernel<<<(n + 127) / 128, 128>>>(ctr, k0, k1, mine, ref, n);
  cudaMemcpy(mine_host, mine, sizeof(uint32_t) * 4 * n, cudaMemcpyDeviceToHost);
  cudaMemcpy(ref_host, ref, sizeof(uint32_t) * 4 * n, cudaMemcpyDeviceToHost);
  const cudaError_t e = cudaGetLastError();
  cudaFree(ctr);
  cudaFree(mine);
  cudaFree(ref);
  return e == cudaSuccess ? 0 : -2;
}

// The theta' partial's exact sum of binary32 addends, two ways: xacc_add_float alone, and the
// 64-bit fast path (xacc_add_float_q, folded every `fold_every` additions) that the FP32 kernels
// use. One thread adds the n values in order. out: the two 192-bit sums (limbs w0, w1, w2 each)
// and their flag counts (nan, neg_inf, big each).
namespace {
__global__ void xacc32_kernel(const float* v, int n, int fold_every, unsigned long long* out, unsigned int* flags) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  chm::Xacc a, b;
  chm::xacc_zero(a);
  chm::xacc_zero(b);
  chm::XFlags fa = {0u, 0u, 0u}, fb = {0u, 0u, 0u};
  long long q = 0;
  for (int i = 0; i < n; ++i) {
    chm::xacc_add_float(a, v[i], fa);
    chm::xacc_add_float_q(b, q, v[i], fb);
    if ((i + 1) % fold_every == 0) chm::xacc_fold_q(b, q);
  }
  chm::xacc_fold_q(b, q);
  out[0] = a.w0; out[1] = a.w1; out[2] = a.w2;
  out[3] = b.w0; out[4] = b.w1; out[5] = b.w2;
  flags[0] = fa.nan; flags[1] = fa.neg_inf; flags[2] = fa.big;
  flags[3] = fb.nan; flags[4] = fb.neg_inf; flags[5] = fb.big;
}
}  // namespace

extern "C" int probe_xacc_f32(const float* v_host, int n, int fold_every, unsigned long long* out_host,
                              unsigned int* flags_host) {
  if (n < 1 || fold_every < 1 || fold_every > 127) return -3;
  float* v = nullptr;
  unsigned long long* out = nullptr;
  unsigned int* flags = nullptr;
  if (cudaMalloc(&v, sizeof(float) * n) != cudaSuccess) return -1;
  if (cudaMalloc(&out, sizeof(unsigned long long) * 6) != cudaSuccess) return -1;
  if (cudaMalloc(&flags, sizeof(unsigned int) * 6) != cudaSuccess) return -1;
  cudaMemcpy(v, v_host, sizeof(float) * n, cudaMemcpyHostToDevice);
  xacc32_kernel<<<1, 32>>>(v, n, fold_every, out, flags);
  cudaMemcpy(out_host, out, sizeof(unsigned long long) * 6, cudaMemcpyDeviceToHost);
  cudaMemcpy(flags_host, flags, sizeof(unsigned int) * 6, cudaMemcpyDeviceToHost);
  const cudaError_t e = cudaGetLastError();
  cudaFree(v);
  cudaFree(out);
  cudaFree(flags);
  return e == cudaSuccess ? 0 : -2;
}
