// Device building blocks of the sweep kernels (sm_103a).
//
//  - Philox4x32-10 counter-based generator (Salmon et al., SC'11) keyed by the run
//    seed; counter = (block j, stream s, member i, sweep k).
//  - Uniforms (2m+1) 2^-53 built from the bits (exact), Box-Muller normals.
//  - Xacc: a 192-bit two's-complement fixed-point accumulator with 2^-96 resolution.
//    Each addend is rounded toward zero to a multiple of 2^-96 and then added exactly,
//    so a sum is the same for every order and every launch shape.
//  - A grid barrier whose spin is bounded by %globaltimer: on expiry it records
//    CUDAHM_ETIMEOUT in the run's error word and every block leaves the kernel.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "cudahm.h"

namespace chm {

// ------------------------------------------------------------------ RNG -----
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return c;
}

// (2m+1) 2^-53 with m the top 52 bits of (wa:wb): 1 + m 2^-52 is assembled from the
// bits, then 1 - 2^-53 is subtracted; the difference is representable, hence exact.
__device__ __forceinline__ double uniform53(uint32_t wa, uint32_t wb) {
  const unsigned long long m = ((static_cast<unsigned long long>(wa) << 32) | wb) >> 12;
  const double v = __longlong_as_double(static_cast<long long>(0x3FF0000000000000ull | m));
  return v - 0x1.fffffffffffffp-1;
}

// --------------------------------------------------- integer comparisons ----
// Orderings of doubles decided on the integer pipe (the FP64 pipe is the sampler's bound).
// dkey maps a double's bits to a signed integer with the same order as the values (-0 sorts
// just below +0; NaN is never passed here).
__device__ __forceinline__ long long dkey(double x) {
  const long long b = __double_as_longlong(x);
  return b ^ ((b >> 63) & 0x7FFFFFFFFFFFFFFFll);
}
__device__ __forceinline__ bool dgt(double x, double y) { return dkey(x) > dkey(y); }
__device__ __forceinline__ bool dsign(double x) { return __double_as_longlong(x) < 0; }
__device__ __forceinline__ bool disnan(double x) {
  return (__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFll) > 0x7FF0000000000000ll;
}
// |x| >= 2^94 (infinities included)
__device__ __forceinline__ bool dhuge(double x) {
  return (__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFll) >= 0x45D0000000000000ll;
}

// ------------------------------------------------------------- Xacc ---------
struct Xacc {
  unsigned long long w0, w1, w2;  // little-endian limbs; value = (signed 192-bit) * 2^-96
};

__device__ __forceinline__ void xacc_zero(Xacc& a) { a.w0 = a.w1 = a.w2 = 0ull; }

__device__ __forceinline__ void xacc_add(Xacc& a, const Xacc& b) {
  asm("add.cc.u64 %0, %0, %3;\n\taddc.cc.u64 %1, %1, %4;\n\taddc.u64 %2, %2, %5;"
      : "+l"(a.w0), "+l"(a.w1), "+l"(a.w2)
      : "l"(b.w0), "l"(b.w1), "l"(b.w2));
}

// Flags counted next to the sum.
struct XFlags {
  unsigned int neg_inf;  // -inf addends (support violations)
  unsigned int nan;      // NaN addends
  unsigned int big;      // finite addends with |v| >= 2^94 (outside the fixed-point range)
};

// Add v (rounded toward zero to a multiple of 2^-96). Non-finite or huge values are
// counted in f instead of added.
__device__ __forceinline__ void xacc_add_double(Xacc& a, double v, XFlags& f) {
  const unsigned long long u = static_cast<unsigned long long>(__double_as_longlong(v));
  const int e = static_cast<int>((u >> 52) & 0x7ff);
  if (e == 0x7ff) {
    if (u & 0x000FFFFFFFFFFFFFull) f.nan++;
    else if (u >> 63) f.neg_inf++;
    else f.big++;
    return;
  }
  if (e >= 1023 + 94) { f.big++; return; }
  const int sh = e - 979;  // value * 2^96 = m * 2^(e - 1075 + 96)
  if (e == 0 || sh <= -53) return;  // below 2^-96 (or subnormal): rounds to zero
  const unsigned long long m = (u & 0x000FFFFFFFFFFFFFull) | 0x0010000000000000ull;
  Xacc t;
  if (sh < 0) {
    t.w0 = m >> (-sh); t.w1 = 0ull; t.w2 = 0ull;
  } else {
    const int q = sh >> 6, r = sh & 63;
    const unsigned long long lo = m << r;
    const unsigned long long hi = r ? (m >> (64 - r)) : 0ull;
    t.w0 = (q == 0) ? lo : 0ull;
    t.w1 = (q == 1) ? lo : ((q == 0) ? hi : 0ull);
    t.w2 = (q == 2) ? lo : ((q == 1) ? hi : 0ull);
  }
  if (u >> 63) {  // two's-complement negate
    t.w0 = ~t.w0; t.w1 = ~t.w1; t.w2 = ~t.w2;
    asm("add.cc.u64 %0, %0, 1;\n\taddc.cc.u64 %1, %1, 0;\n\taddc.u64 %2, %2, 0;"
        : "+l"(t.w0), "+l"(t.w1), "+l"(t.w2));
  }
  xacc_add(a, t);
}

// Add a binary32 value (rounded toward zero to a multiple of 2^-96); same flags.
__device__ __forceinline__ void xacc_add_float(Xacc& a, float v, XFlags& f) {
  const unsigned int u = __float_as_uint(v);
  const int e = static_cast<int>((u >> 23) & 0xff);
  if (e == 0xff) {
    if (u & 0x007FFFFFu) f.nan++;
    else if (u >> 31) f.neg_inf++;
    else f.big++;
    return;
  }
  if (e >= 127 + 94) { f.big++; return; }
  const int sh = e - 54;  // value * 2^96 = m * 2^(e - 150 + 96)
  if (e == 0 || sh <= -24) return;
  const unsigned long long m = static_cast<unsigned long long>((u & 0x007FFFFFu) | 0x00800000u);
  Xacc t;
  if (sh < 0) {
    t.w0 = m >> (-sh); t.w1 = 0ull; t.w2 = 0ull;
  } else {
    const int q = sh >> 6, r = sh & 63;
    const unsigned long long lo = m << r;
    const unsigned long long hi = r ? (m >> (64 - r)) : 0ull;
    t.w0 = (q == 0) ? lo : 0ull;
    t.w1 = (q == 1) ? lo : ((q == 0) ? hi : 0ull);
    t.w2 = (q == 2) ? lo : ((q == 1) ? hi : 0ull);
  }
  if (u >> 31) {
    t.w0 = ~t.w0; t.w1 = ~t.w1; t.w2 = ~t.w2;
    asm("add.cc.u64 %0, %0, 1;\n\taddc.cc.u64 %1, %1, 0;\n\taddc.u64 %2, %2, 0;"
        : "+l"(t.w0), "+l"(t.w1), "+l"(t.w2));
  }
  xacc_add(a, t);
}

// A binary32 addend v = m 2^(e - 150) (m the 24-bit significand, e the biased exponent field) with
// e in [102, 134], i.e. 2^-25 <= |v| < 2^8, is the integer m 2^(e - 102) < 2^56 times 2^-48. Such
// addends (nearly every theta' partial of a sweep) are summed exactly in one signed 64-bit word q
// (value q 2^-48) with a shift, a conditional negate and one 64-bit add, instead of the 192-bit
// add; the rest take xacc_add_float. The caller folds q into the Xacc (xacc_fold_q) after at most
// 127 additions, so q cannot overflow. xacc_add_float adds these addends without rounding too, so
// the total is the same to the last bit.
__device__ __forceinline__ void xacc_add_float_q(Xacc& a, long long& q, float v, XFlags& f) {
  const unsigned int u = __float_as_uint(v);
  const unsigned int sh = ((u >> 23) & 0xffu) - 102u;  // wraps for e < 102
  if (sh <= 32u) {
    const long long t =
        static_cast<long long>(static_cast<unsigned long long>((u & 0x007FFFFFu) | 0x00800000u) << sh);
    q += (u >> 31) ? -t : t;
  } else {
    xacc_add_float(a, v, f);
  }
}

// Adds q 2^-48 (as the 192-bit value q 2^48 times 2^-96, sign-extended) into a and clears q.
__device__ __forceinline__ void xacc_fold_q(Xacc& a, long long& q) {
  Xacc t;
  t.w0 = static_cast<unsigned long long>(q) << 48;
  t.w1 = static_cast<unsigned long long>(q >> 16);
  t.w2 = static_cast<unsigned long long>(q >> 63);
  xacc_add(a, t);
  q = 0;
}

// Round-to-nearest-even conversion of the fixed-point value to binary64.
__device__ __forceinline__ double xacc_to_double(Xacc a) {
  const bool neg = (a.w2 >> 63) != 0;
  if (neg) {
    a.w0 = ~a.w0; a.w1 = ~a.w1; a.w2 = ~a.w2;
    asm("add.cc.u64 %0, %0, 1;\n\taddc.cc.u64 %1, %1, 0;\n\taddc.u64 %2, %2, 0;"
        : "+l"(a.w0), "+l"(a.w1), "+l"(a.w2));
  }
  int hb;  // index of the highest set bit
  if (a.w2) hb = 128 + 63 - __clzll(static_cast<long long>(a.w2));
  else if (a.w1) hb = 64 + 63 - __clzll(static_cast<long long>(a.w1));
  else if (a.w0) hb = 63 - __clzll(static_cast<long long>(a.w0));
  else return 0.0;
  // top 64 bits starting at hb (left-aligned), and a sticky bit for everything below
  unsigned long long top, rest_nonzero;
  const int lo_bit = hb - 63;  // bit index of the LSB of 'top'
  if (lo_bit <= 0) {  // hb <= 63: the value sits in w0
    top = a.w0 << (-lo_bit);
    rest_nonzero = 0ull;
  } else {
    const int q = lo_bit >> 6, r = lo_bit & 63;
    const unsigned long long limb[4] = {a.w0, a.w1, a.w2, 0ull};
    top = r ? ((limb[q] >> r) | (limb[q + 1] << (64 - r))) : limb[q];
    unsigned long long below = 0ull;
    for (int i = 0; i < q; ++i) below |= limb[i];
    if (r) below |= (limb[q] << (64 - r));
    rest_nonzero = below;
  }
  // 53-bit mantissa, guard bit, sticky
  unsigned long long mant = top >> 11;
  const unsigned long long guard = (top >> 10) & 1ull;
  const unsigned long long sticky = ((top & 0x3FFull) != 0ull) | (rest_nonzero != 0ull);
  if (guard && (sticky || (mant & 1ull))) mant += 1ull;
  int exp2 = hb - 96 - 52;  // value = mant * 2^exp2, mant in [2^52, 2^53)
  if (mant >> 53) { mant >>= 1; exp2 += 1; }
  // assembled from its fields: exp2 lies in [-148, 44], so the value is a normal binary64
  const unsigned long long bits = (static_cast<unsigned long long>(exp2 + 1075) << 52) |
                                  (mant & 0x000FFFFFFFFFFFFFull) | (neg ? 0x8000000000000000ull : 0ull);
  return __longlong_as_double(static_cast<long long>(bits));
}

__device__ __forceinline__ Xacc xacc_shfl_xor(const Xacc& a, int lane_mask) {
  Xacc b;
  b.w0 = __shfl_xor_sync(0xffffffffu, a.w0, lane_mask);
  b.w1 = __shfl_xor_sync(0xffffffffu, a.w1, lane_mask);
  b.w2 = __shfl_xor_sync(0xffffffffu, a.w2, lane_mask);
  return b;
}

// ---------------------------------------------------------- barrier ----------
__device__ __forceinline__ long long globaltimer_ns() {
  long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned int ld_acquire_u32(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release_u32(unsigned int* p, unsigned int v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" : : "l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ int ld_volatile_i32(const int* p) {
  return *reinterpret_cast<const volatile int*>(p);
}

// A grid-wide barrier in two halves, so that a block can work between its arrival and the
// others': grid_arrive (all threads of the block; thread 0 publishes the block's writes and
// counts it in) and grid_wait (all threads; thread 0 waits, bounded, until barrier `index` has
// every block, or the first nb arrivals when nb > 0). grid_barrier below is the two back to back.
__device__ __forceinline__ void grid_arrive(unsigned int* count, bool skip_arrival) {
  __syncthreads();
  if (threadIdx.x == 0 && !skip_arrival) {
    __threadfence();
    atomicAdd(count, 1u);
  }
}
// Thread 0's bounded wait for grid barrier `index` (nb arrivals per barrier; 0: the grid): true
// once every block has arrived, false if the run failed meanwhile or the wait ran out (the
// run's error word then says why). Nothing else of the block waits.
__device__ __forceinline__ bool grid_poll(unsigned int* count, unsigned int index, int* err, long long limit_ns,
                                          unsigned int nb) {
  const unsigned int target = (index + 1u) * (nb ? nb : gridDim.x);
  const long long t0 = globaltimer_ns();
  bool ok = true;
  while (true) {
    if (ld_acquire_u32(count) >= target) break;
    if (ld_volatile_i32(err) != 0) { ok = false; break; }
    if (globaltimer_ns() - t0 > limit_ns) {
      atomicCAS(err, 0, CUDAHM_ETIMEOUT);
      ok = false;
      break;
    }
    __nanosleep(64);
  }
  if (ld_volatile_i32(err) != 0) ok = false;
  __threadfence();
  return ok;
}
__device__ __forceinline__ bool grid_wait(unsigned int* count, unsigned int index, int* err, long long limit_ns,
                                          unsigned int nb = 0u) {
  __shared__ int s_ok;
  if (threadIdx.x == 0) s_ok = grid_poll(count, index, err, limit_ns, nb) ? 1 : 0;
  __syncthreads();
  return s_ok != 0;
}

// Grid-wide barrier number `index` (0-based) of this launch. The counter starts at 0 for
// every launch. Returns false if the run has failed (timeout here or an error elsewhere);
// the caller then leaves the kernel. Must be called by all threads of the block.
__device__ __forceinline__ bool grid_barrier(unsigned int* count, unsigned int index, int* err, long long limit_ns,
                                             bool skip_arrival) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    if (!skip_arrival) {
      __threadfence();
      atomicAdd(count, 1u);
    }
    const unsigned int target = (index + 1u) * gridDim.x;
    const long long t0 = globaltimer_ns();
    while (true) {
      if (ld_acquire_u32(count) >= target) break;
      if (ld_volatile_i32(err) != 0) { ok = 0; break; }
      if (globaltimer_ns() - t0 > limit_ns) {
        atomicCAS(err, 0, CUDAHM_ETIMEOUT);
        ok = 0;
        break;
      }
      __nanosleep(64);
    }
    if (ld_volatile_i32(err) != 0) ok = 0;
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// ------------------------------------------------ bulk copies (TMA engine) --
// One-dimensional bulk copies global -> shared (cp.async.bulk), completed on an mbarrier that
// counts the bytes. Source and destination must be 16-byte aligned and the size a multiple of 16.
__device__ __forceinline__ unsigned int smem_addr(const void* p) {
  return static_cast<unsigned int>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned int count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" : : "r"(smem_addr(bar)), "r"(count) : "memory");
}
// the issuing thread's arrival, announcing the bytes the copies on this barrier will deliver
__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long* bar, unsigned int bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" : : "r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned int parity) {
  unsigned int done;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(done)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return done != 0u;
}
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, unsigned int bytes, unsigned long long* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
               :
               : "r"(smem_addr(dst)), "l"(src), "r"(bytes), "r"(smem_addr(bar))
               : "memory");
}
// orders this thread's earlier generic-proxy writes to global memory before later bulk copies
// (async proxy) that read them
__device__ __forceinline__ void fence_proxy_async_global() {
  asm volatile("fence.proxy.async.global;" : : : "memory");
}
// makes mbarrier initialisation visible to the async proxy
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.proxy.async.shared::cta;" : : : "memory");
}
// Waits (the calling thread) until the barrier's phase `parity` has completed, bounded by
// limit_ns of %globaltimer; on expiry records CUDAHM_ETIMEOUT and returns false.
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long* bar, unsigned int parity, int* err,
                                                  long long limit_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = globaltimer_ns();
  while (!mbar_try_wait(bar, parity)) {
    if (globaltimer_ns() - t0 > limit_ns) {
      atomicCAS(err, 0, CUDAHM_ETIMEOUT);
      return false;
    }
  }
  return true;
}

}  // namespace chm
