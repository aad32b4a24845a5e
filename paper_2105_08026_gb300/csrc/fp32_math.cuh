// Binary32 e^x and e^x - 1 for the FP32 bulk form's member log targets.
//
// The FP32 form's bar includes the sum over a million members of their log targets, so a
// rounding bias of the exponential adds up: CUDA's expf rounds with a mean error of about
// +0.07 ulp over the arguments these models use (measured), which moves the luminosity model's
// sum by ~8e-3 at N = 1e6. These two round without a common sign:
//  - x = k ln2 + r with |r| <= ln2/2 (Cody-Waite: ln 2 as a 15-bit head, so that k head is exact
//    and x - k head is exact by Sterbenz's lemma, and a binary32 tail kept as a separate term);
//  - e^r - 1 from its Taylor series r + r^2 (1/2! + r/3! + ... + r^7/9!) by Horner's rule in
//    binary32 FMAs (remainder below 2^-30 relative; no cancellation near r = 0);
//  - e^x = 2^k + 2^k (e^r - 1) and e^x - 1 = (2^k - 1) + 2^k (e^r - 1), each one FMA that rounds
//    once, to nearest (2^k from the exponent bits; 2^k - 1 is exact for |k| <= 24).
// Outside |x| <= 86 (and for NaN) they return CUDA's expf (minus 1). Tested within 1.25 ulp of the
// exact value and with a mean error below 0.01 ulp (tests/test_gpu_math.py).
#pragma once

namespace chm {

// e^r - 1 = r + r^2 q, q = 1/2! + r/3! + ... + r^(D-2)/D!, so that the rounding of q and of r^2
// enter scaled by |r q|: D = 9 for |r| <= ln2/2 (remainder below 2^-30 relative), D = 12 for
// |r| <= 0.7 (remainder below 2^-33)
__device__ __forceinline__ float em1_reduced(float r) {
  float q = 2.75573192239858907e-06f;             // 1/9!
  q = __fmaf_rn(q, r, 2.48015873015873016e-05f);  // 1/8!
  q = __fmaf_rn(q, r, 1.98412698412698413e-04f);  // 1/7!
  q = __fmaf_rn(q, r, 1.38888888888888889e-03f);  // 1/6!
  q = __fmaf_rn(q, r, 8.33333333333333333e-03f);  // 1/5!
  q = __fmaf_rn(q, r, 4.16666666666666667e-02f);  // 1/4!
  q = __fmaf_rn(q, r, 1.66666666666666667e-01f);  // 1/3!
  q = __fmaf_rn(q, r, 0.5f);
  return __fmaf_rn(__fmul_rn(r, r), q, r);
}
__device__ __forceinline__ float em1_wide(float r) {
  float q = 2.08767569878680990e-09f;             // 1/12!
  q = __fmaf_rn(q, r, 2.50521083854417188e-08f);  // 1/11!
  q = __fmaf_rn(q, r, 2.75573192239858907e-07f);  // 1/10!
  q = __fmaf_rn(q, r, 2.75573192239858907e-06f);  // 1/9!
  q = __fmaf_rn(q, r, 2.48015873015873016e-05f);  // 1/8!
  q = __fmaf_rn(q, r, 1.98412698412698413e-04f);  // 1/7!
  q = __fmaf_rn(q, r, 1.38888888888888889e-03f);  // 1/6!
  q = __fmaf_rn(q, r, 8.33333333333333333e-03f);  // 1/5!
  q = __fmaf_rn(q, r, 4.16666666666666667e-02f);  // 1/4!
  q = __fmaf_rn(q, r, 1.66666666666666667e-01f);  // 1/3!
  q = __fmaf_rn(q, r, 0.5f);
  return __fmaf_rn(__fmul_rn(r, r), q, r);
}

// x = k ln2 + r_hi + r_lo with r_hi = x - k head (exact) and r_lo = -k tail; sets s = 2^k
// (|x| <= 86, so |k| <= 124). Rounding r_hi + r_lo to one binary32 value would add a fixed
// offset for every x of a binade (the tail's fraction of the grid): a bias, so the tail stays apart.
// k = x log2(e) rounded to the nearest integer by adding and subtracting 1.5 2^23 (binary32
// addition rounds to an integer there), its bits read as the integer: no conversion instruction.
__device__ __forceinline__ float exp_reduce(float x, float& s, float& r_lo) {
  const float t = __fadd_rn(__fmul_rn(x, 1.44269504088896341f), 12582912.0f);
  const float k = __fsub_rn(t, 12582912.0f);
  r_lo = __fmul_rn(-k, 1.42860676533018704e-06f);
  s = __int_as_float((127 + (__float_as_int(t) - 0x4B400000)) << 23);
  return __fmaf_rn(-k, 0.693145751953125f, x);
}

// e^(r_hi + r_lo) - 1 = E + r_lo (1 + E), E = e^r_hi - 1 (the r_lo^2 term is below 2^-36)
__device__ __forceinline__ float em1_split(float r_hi, float r_lo) {
  const float e = em1_reduced(r_hi);
  return __fadd_rn(e, __fmaf_rn(r_lo, e, r_lo));
}

__device__ __forceinline__ float exp32(float x) {
  if (!(fabsf(x) <= 86.0f)) return expf(x);
  float s, r_lo;
  const float r_hi = exp_reduce(x, s, r_lo);
  return __fmaf_rn(s, em1_split(r_hi, r_lo), s);
}

__device__ __forceinline__ float expm1_32(float x) {
  if (fabsf(x) <= 0.7f) return em1_wide(x);
  if (!(fabsf(x) <= 86.0f)) return __fsub_rn(expf(x), 1.0f);
  float s, r_lo;
  const float r_hi = exp_reduce(x, s, r_lo);
  return __fmaf_rn(s, em1_split(r_hi, r_lo), __fsub_rn(s, 1.0f));
}

}  // namespace chm
