// Table-driven FP64 exp and log for the member step (Tang, "Table-driven implementation of
// the exponential function in IEEE floating-point arithmetic", ACM TOMS 15, 1989, and
// "... of the logarithm function", ACM TOMS 16, 1990). On this GPU the FP64 pipe is the
// bound of the sampler; these versions use about half of the FP64 instructions of the
// general-purpose library routines, and are within ~2 ulp.
//
// Table (doubles, built on the device once per handle by math_table_kernel):
//   [0, 64)     2^(j/64)
//   [64, 156)   ln F_j,  F_j = (j + 90)/128, j = 0..91
//   [156, 248)  1/F_j
//   [248, 377)  sin(pi j/64), j = 0..128
//   [377, 506)  cos(pi j/64)
#pragma once
#include <cuda_runtime.h>

namespace chm {

constexpr int kSinOff = 64 + 2 * 92;
constexpr int kCosOff = kSinOff + 129;
constexpr int kMathWords = kCosOff + 129;

static __global__ void math_table_kernel(double* t) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < 64) {
    t[i] = exp2(i / 64.0);
  } else if (i < 64 + 92) {
    const int j = i - 64;
    const double F = (j + 90) / 128.0;
    t[i] = log(F);
    t[i + 92] = 1.0 / F;
  } else if (i >= 256 && i < 256 + 129) {
    const int j = i - 256;
    double sn, cs;
    sincospi(j / 64.0, &sn, &cs);
    t[kSinOff + j] = sn;
    t[kCosOff + j] = cs;
  }
}

// exp(x): x = k ln2/64 + r with k = round(64 x/ln2) and |r| <= ln2/128 (two-constant
// reduction); e^x = 2^(k div 64) 2^((k mod 64)/64) (1 + expm1(r)), expm1 by its degree-5
// Taylor polynomial (remainder r^6/720 < 3.5e-17, a third of an ulp of 1 + expm1(r)). Outside
// (-700, 709), and for NaN and infinities, the library routine is used.
__device__ __forceinline__ double exp_tab(double x, const double* __restrict__ T) {
  // fast path for -700 < x < 709, tested on the bits: |x| < 700, or 0 <= x < 709
  const long long b = __double_as_longlong(x);
  const long long mag = b & 0x7FFFFFFFFFFFFFFFll;
  if (!(mag < 0x4085E00000000000ll || (b >= 0 && b < 0x4086280000000000ll))) return exp(x);
  const double magic = 0x1.8p52;
  const double km = fma(x, 0x1.71547652b82fep+6, magic);  // 64/ln2
  const int k = __double2loint(km);
  const double kd = km - magic;
  double r = fma(-kd, 0x1.62e42fefa4000p-7, x);   // ln2/64, high 40 bits
  r = fma(-kd, -0x1.8432a1b0e2634p-49, r);        // ln2/64, remainder
  double p = fma(r, 1.0 / 120.0, 1.0 / 24.0);
  p = fma(p, r, 1.0 / 6.0);
  p = fma(p, r, 0.5);
  p = fma(p, r, 1.0);
  p *= r;  // expm1(r)
  const double t = T[k & 63];
  const double res = fma(t, p, t);
  return __hiloint2double(__double2hiint(res) + ((k >> 6) << 20), __double2loint(res));
}

// ln(u) for a positive normal u: u = 2^e m with m in [sqrt(1/2), sqrt 2), F = nearest (j+90)/128,
// ln u = e ln2 + ln F + log1p((m - F)/F) with log1p by its degree-8 Taylor polynomial
// (|r| <= 1/181, remainder < 1e-21); m - F is exact.
__device__ __forceinline__ double log_tab(double u, const double* __restrict__ T) {
  long long b = __double_as_longlong(u);
  int e = static_cast<int>(b >> 52) - 1023;
  long long mb = (b & 0x000FFFFFFFFFFFFFll) | 0x3FF0000000000000ll;  // m in [1, 2)
  if (mb >= 0x3FF6A09E667F3BCDll) {                                    // m >= sqrt 2: use m/2
    mb -= 0x0010000000000000ll;
    e += 1;
  }
  const double m = __longlong_as_double(mb);
  const double magic = 0x1.8p52;
  const double jm = fma(m, 128.0, magic);
  const int j = __double2loint(jm) - 90;
  const double F = (jm - magic) * 0.0078125;
  const double r = (m - F) * T[64 + 92 + j];
  double p = fma(r, -0.125, 1.0 / 7.0);
  p = fma(p, r, -1.0 / 6.0);
  p = fma(p, r, 0.2);
  p = fma(p, r, -0.25);
  p = fma(p, r, 1.0 / 3.0);
  p = fma(p, r, -0.5);
  p *= r;
  p = fma(p, r, r);  // log1p(r)
  const double ed = static_cast<double>(e);
  const double hi = fma(ed, 0x1.62e42fefa4000p-1, T[64 + j]);  // e ln2 (high 40 bits, exact) + ln F
  return hi + fma(ed, -0x1.8432a1b0e2634p-43, p);
}

// sin(pi a), cos(pi a) for 0 <= a <= 2 (the Box-Muller angle 2 pi u): a = j/64 + r with
// j = round(64 a), |r| <= 1/128 (r exact), theta = pi r (|theta| <= 0.0246); sin theta by its
// degree-7 Taylor polynomial (remainder < 1e-20), cos theta by its degree-6 polynomial (remainder
// < 4e-18), then the angle-sum formulas with the tabulated sin(pi j/64), cos(pi j/64).
__device__ __forceinline__ void sincospi_tab(double a, const double* __restrict__ T, double* sn, double* cs) {
  const double magic = 0x1.8p52;
  const double jm = fma(a, 64.0, magic);
  const int j = __double2loint(jm);
  const double r = fma(jm - magic, -0.015625, a);          // exact
  const double th = fma(r, 0x1.921fb54442d18p+1, r * 0x1.1a62633145c07p-53);  // pi r, pi as hi + lo
  const double t2 = th * th;
  double ps = fma(t2, -1.0 / 5040.0, 1.0 / 120.0);
  ps = fma(ps, t2, -1.0 / 6.0);
  const double st = fma(th * t2, ps, th);                   // sin theta
  double pc = fma(t2, -1.0 / 720.0, 1.0 / 24.0);
  pc = fma(pc, t2, -0.5);
  const double ct = fma(t2, pc, 1.0);                       // cos theta
  const double sj = T[kSinOff + j], cj = T[kCosOff + j];
  *sn = fma(sj, ct, cj * st);
  *cs = fma(cj, ct, -sj * st);
}

// e^x - 1 for the theta step's constants (a dependent chain on one lane, so short matters more
// than throughput): for |x| <= 1/2 the Taylor series x (1 + x/2! + ... + x^15/16!) by Horner
// (remainder below 1e-18 relative), else the library routine.
__device__ __forceinline__ double expm1_theta(double x) {
  if (!(fabs(x) <= 0.5)) return expm1(x);
  constexpr double c[16] = {1.0,
                            1.0 / 2.0,
                            1.0 / 6.0,
                            1.0 / 24.0,
                            1.0 / 120.0,
                            1.0 / 720.0,
                            1.0 / 5040.0,
                            1.0 / 40320.0,
                            1.0 / 362880.0,
                            1.0 / 3628800.0,
                            1.0 / 39916800.0,
                            1.0 / 479001600.0,
                            1.0 / 6227020800.0,
                            1.0 / 87178291200.0,
                            1.0 / 1307674368000.0,
                            1.0 / 20922789888000.0};
  double q = c[15];
#pragma unroll
  for (int k = 14; k >= 0; --k) q = fma(q, x, c[k]);
  return q * x;
}

}  // namespace chm
