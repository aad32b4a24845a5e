// Test model of the member accept rule: independent Metropolis chains on two states.
//
// Sec. 2.2's member step accepts a proposal with probability min(1, pi(Y)/pi(X)). On a target
// with two states and a proposal that always flips to the other state (symmetric), the chain's
// transition probabilities are P01 = min(1, pi1/pi0) and P10 = min(1, pi0/pi1), which satisfy
// detailed balance pi0 P01 = pi1 P10 and leave (pi0, pi1) stationary. This kernel runs the
// member step's own accept routine (mh_accept, mh_accept32) and the member's own accept uniform
// of each sweep on such chains and counts the transitions, so that the rule can be checked
// against those identities and, in binary64, against the oracle's chains draw for draw.
#include <cmath>
#include <cstdint>

#include "cudahm.h"
#include "sweep_common.cuh"

namespace chm {
namespace {

// Chain i starts in state i mod 2. Sweep k (1-based) proposes the other state with
// Delta = ln pi(other) - ln pi(current) and the member step's accept uniform of sweep k:
// binary64, Philox block (1, stream 0, i, k) as for every d = 1 member; binary32, word 2 (odd
// k) or 3 (even k) of block (0, stream 2, i, odd sweep) as in the bulk form. counts[2 from + to].
template <bool F32>
__global__ void twostate_kernel(long long n, long long T, double lp0, double lp1, uint32_t key0, uint32_t key1,
                                const double* math_tab, unsigned long long* counts) {
  extern __shared__ double s_math[];
  for (int q = threadIdx.x; q < kMathWords; q += blockDim.x) s_math[q] = math_tab[q];
  __syncthreads();
  unsigned long long c[4] = {0ull, 0ull, 0ull, 0ull};
  const long long stride = static_cast<long long>(gridDim.x) * blockDim.x;
  for (long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride) {
    int x = static_cast<int>(i & 1);
    for (long long k = 1; k <= T; ++k) {
      const uint32_t kk = static_cast<uint32_t>(k);
      bool acc;
      if constexpr (F32) {
        const float delta = x ? static_cast<float>(lp0 - lp1) : static_cast<float>(lp1 - lp0);
        const bool odd = (kk & 1u) != 0u;
        const uint4 w = philox4x32_10(make_uint4(0u, 2u, static_cast<uint32_t>(i), odd ? kk : kk - 1u), key0, key1);
        const float u = uniform23(odd ? w.z : w.w);
        float alpha;
        acc = mh_accept32(delta, u, alpha);
      } else {
        const double delta = x ? lp0 - lp1 : lp1 - lp0;
        const uint4 w = philox4x32_10(make_uint4(1u, 0u, static_cast<uint32_t>(i), kk), key0, key1);
        const double u = uniform53(w.x, w.y);
        double alpha;
        acc = mh_accept(delta, u, s_math, alpha);
      }
      const int y = acc ? 1 - x : x;
      c[2 * x + y]++;
      x = y;
    }
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    unsigned long long v = c[q];
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    if ((threadIdx.x & 31) == 0 && v) atomicAdd(counts + q, v);
  }
}

}  // namespace
}  // namespace chm

extern "C" int cudahm_twostate_run(double pi1, int32_t precision, int64_t n_chains, int64_t sweeps, uint64_t seed,
                                   int32_t device, int64_t* counts_host) {
  using namespace chm;
  if (!counts_host) return record_error(CUDAHM_EINVAL, "cudahm_twostate_run: counts_host is NULL");
  if (!(pi1 > 0.0 && pi1 < 1.0)) return record_error(CUDAHM_EINVAL, "cudahm_twostate_run: pi1 must lie in (0, 1)");
  if (precision != CUDAHM_FP64 && precision != CUDAHM_FP32)
    return record_error(CUDAHM_EINVAL, "cudahm_twostate_run: unknown precision");
  if (n_chains < 1 || n_chains > (1ll << 31) || sweeps < 1 || sweeps > (1ll << 32) - 2)
    return record_error(CUDAHM_EINVAL, "cudahm_twostate_run: n_chains in [1, 2^31] and sweeps in [1, 2^32 - 2]");
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev)
    return record_error(CUDAHM_EINVAL, "cudahm_twostate_run: device not present");
  if (cudaSetDevice(device) != cudaSuccess) return record_error(CUDAHM_ECUDA, "cudahm_twostate_run: cudaSetDevice");
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  double* tab = nullptr;
  unsigned long long* cnt = nullptr;
  cudaStream_t st = nullptr;
  int rc = CUDAHM_OK;
  if (cudaMalloc(&tab, sizeof(double) * kMathWords) != cudaSuccess ||
      cudaMalloc(&cnt, sizeof(unsigned long long) * 4) != cudaSuccess) {
    rc = record_error(CUDAHM_ENOMEM, "cudahm_twostate_run: device allocation failed");
  } else if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
    rc = record_error(CUDAHM_ECUDA, "cudahm_twostate_run: cannot create a stream");
  } else {
    const int block = 256;
    const long long want = (n_chains + block - 1) / block;
    const int grid = static_cast<int>(want < 8ll * sms ? want : 8ll * sms);
    const double lp0 = std::log(1.0 - pi1), lp1 = std::log(pi1);
    const uint32_t k0 = static_cast<uint32_t>(seed & 0xffffffffull), k1 = static_cast<uint32_t>(seed >> 32);
    unsigned long long h[4] = {0ull, 0ull, 0ull, 0ull};
    cudaMemsetAsync(cnt, 0, sizeof(unsigned long long) * 4, st);
    launch_math_table(tab, st);
    const size_t smem = sizeof(double) * kMathWords;
    if (precision == CUDAHM_FP32)
      twostate_kernel<true><<<grid, block, smem, st>>>(n_chains, sweeps, lp0, lp1, k0, k1, tab, cnt);
    else
      twostate_kernel<false><<<grid, block, smem, st>>>(n_chains, sweeps, lp0, lp1, k0, k1, tab, cnt);
    cudaMemcpyAsync(h, cnt, sizeof(h), cudaMemcpyDeviceToHost, st);
    const cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess || cudaGetLastError() != cudaSuccess) {
      rc = record_error(CUDAHM_ECUDA, "cudahm_twostate_run: kernel failed");
    } else {
      for (int q = 0; q < 4; ++q) counts_host[q] = static_cast<int64_t>(h[q]);
    }
  }
  if (st) cudaStreamDestroy(st);
  if (tab) cudaFree(tab);
  if (cnt) cudaFree(cnt);
  return rc;
}
