// Device code shared by the persistent kernels (sweep.cu: one population per launch;
// batch.cu: many populations per launch): models, the theta RAM update, the normal-CDF
// table, the selection-rule segments, block reductions and the theta proposal.
#pragma once
#include <cmath>
#include <cstdint>
#include <type_traits>

#include "device_common.cuh"
#include "fp32_math.cuh"
#include "fp64_math.cuh"
#include "internal.h"

namespace chm {

// ----------------------------------------------------------------- models ----
// Per-theta constants a0..a4 (computed once per theta by one thread).
struct ThetaC {
  double a0, a1, a2, a3, a4;
};

// binary32 theta constants for the FP32 bulk form; a location parameter is held as a sum of
// two floats (hi + lo) so that chi - location keeps full binary32 relative accuracy.
struct ThetaCf {
  float sc_hi, sc_lo, loc_hi, loc_lo, low_hi, low_lo;  // scale, location, lower bound (hi + lo)
};
// binary32 constants of one theta step (theta -> theta'), each as hi + lo: the FP32 form's
// d_i = log f(chi;theta') - log f(chi;theta) is formed from them directly (LF; unused by NN1)
struct ThetaDf {
  float dsc_hi, dsc_lo, c_hi, c_lo, em_hi, em_lo;
};
__device__ __forceinline__ void split_f(double v, float& hi, float& lo) {
  hi = static_cast<float>(v);
  lo = static_cast<float>(v - static_cast<double>(hi));
}
// chi - (hi + lo): the first subtraction is exact whenever chi is near hi
__device__ __forceinline__ float sub2(float chi, float hi, float lo) { return __fsub_rn(__fsub_rn(chi, hi), lo); }
// chi - (hi + lo) as an unevaluated sum r_hi + r_lo (Knuth's TwoSum for chi - hi). Latents
// lie on the binary32 grid, so the rounding error of chi - hi repeats from member to member;
// keeping it avoids a bias that would grow with N in sums over members.
__device__ __forceinline__ void sub2x(float chi, float hi, float lo, float& r_hi, float& r_lo) {
  const float s = __fsub_rn(chi, hi);
  const float a1 = __fadd_rn(s, hi);  // chi's share of s
  const float b1 = __fsub_rn(s, a1);  // -hi's share of s
  const float err = __fadd_rn(__fsub_rn(chi, a1), __fsub_rn(-hi, b1));
  r_hi = s;
  r_lo = __fsub_rn(err, lo);
}

// A binary32 value carried as an unevaluated sum hi + lo: lo holds terms below hi's rounding that
// have the same sign for every member (the rounding parts of a shared constant). Added into hi
// they would be lost, always the same way, and the sum over members would drift with N.
struct F2 {
  float hi, lo;
};

struct NN1 {
  // a0 = mu, a1 = 1/(2 tau^2)
  using TC = ThetaC;
  using TCf = ThetaCf;
  static constexpr int kD = 1;
  static constexpr bool kRule = false;  // no selection integral
  static constexpr bool kExp = false;
  // binary32 forms of the member terms (FP32 bulk precision): loc = mu, scale = 1/(2 tau^2)
  __device__ static ThetaCf consts32(const ThetaC& c) {
    ThetaCf f{};
    split_f(c.a0, f.loc_hi, f.loc_lo);
    split_f(c.a1, f.sc_hi, f.sc_lo);
    return f;
  }
  __device__ static bool support32(float, const ThetaCf&) { return true; }
  __device__ static float logf32(float chi, const ThetaCf& c) {
    float rh, rl;
    sub2x(chi, c.loc_hi, c.loc_lo, rh, rl);
    const float r2 = __fmaf_rn(rh, rh, __fmul_rn(__fmul_rn(2.0f, rh), rl));
    return -__fmaf_rn(c.sc_hi, r2, __fmul_rn(c.sc_lo, r2));  // the scale's rounding would bias every member alike
  }
  __device__ static F2 logf32p(float chi, const ThetaCf& c) { return F2{logf32(chi, c), 0.0f}; }
  // the member step's log f and what the theta' partial needs of the state: here log f itself
  __device__ static float logf32_e(float chi, const ThetaCf& c, float& carry) {
    carry = logf32(chi, c);
    return carry;
  }
  __device__ static ThetaDf dconsts32(const ThetaC&, const ThetaC&) { return ThetaDf{}; }
  __device__ static float dtheta32(float chi, float lf_cur, const ThetaCf&, const ThetaCf& cp, const ThetaDf&) {
    return __fsub_rn(logf32(chi, cp), lf_cur);
  }
  // member data d[0], d[1] = y_i as hi + lo, d[2] = 1/(2 sigma_i^2)
  static constexpr int kData32 = 3;
  __device__ static void data32(double y, double aux, const ModelConsts&, float* d) {
    split_f(y, d[0], d[1]);
    d[2] = static_cast<float>(0.5 * aux);
  }
  __device__ static float loglike32(float chi, const float* d) {
    const float r = __fadd_rn(__fsub_rn(d[0], chi), d[1]);
    return __fmul_rn(-d[2], __fmul_rn(r, r));
  }
  // per-theta constants; T is the exp/log table (the theta step runs these on its serial path)
  __device__ static ThetaC consts(const double* th, const ModelConsts&, const double* T) {
    ThetaC c;
    c.a0 = th[0];
    c.a1 = 0.5 * exp_tab(-2.0 * th[1], T);
    c.a2 = 0.0;
    c.a3 = 0.0;
    c.a4 = 0.0;
    return c;
  }
  __device__ static bool support(double, const ThetaC&) { return true; }
  __device__ static double logf(double chi, double, const ThetaC& c) {
    const double r = __dsub_rn(chi, c.a0);
    return __dmul_rn(-c.a1, __dmul_rn(r, r));
  }
  // y = y_i, aux = 1/sigma_i^2
  __device__ static double loglike(double chi, double, double y, double aux, const ModelConsts&) {
    const double r = __dsub_rn(y, chi);
    return __dmul_rn(__dmul_rn(-0.5, aux), __dmul_rn(r, r));
  }
  __device__ static double cterm(const double* th) { return -th[1]; }
  __device__ static double logprior(const double* th, const ModelConsts& mc, const double*) {
    return (th[1] >= mc.lo && th[1] <= mc.hi) ? 0.0 : -INFINITY;
  }
};

struct LF {
  // a0 = beta + 1, a1 = ln L*, a2 = 1/L*, a3 = ln L_low
  using TC = ThetaC;
  using TCf = ThetaCf;
  static constexpr int kD = 1;
  static constexpr bool kRule = true;  // selection integral with constant sigma_F
  static constexpr bool kExp = true;
  // binary32 forms: scale = beta + 1, loc = ln L*, low = ln L_low; log f = scale x - e^x, x = chi - ln L*
  __device__ static ThetaCf consts32(const ThetaC& c) {
    ThetaCf f{};
    split_f(c.a0, f.sc_hi, f.sc_lo);
    split_f(c.a1, f.loc_hi, f.loc_lo);
    split_f(c.a3, f.low_hi, f.low_lo);
    return f;
  }
  __device__ static bool support32(float chi, const ThetaCf& c) { return (chi - c.low_hi) > c.low_lo; }
  // log f = sc x - e^x with x = xh + xl and sc = sc_hi + sc_lo, as hi = sc_hi xh - e^xh (one
  // rounding) plus lo = sc_hi xl + sc_lo xh - e^xh xl (e^(xh + xl) to first order in xl): the
  // small terms share a sign across members (xl and sc_lo are the roundings of ln L* and beta + 1)
  // and would be rounded away in hi
  __device__ static F2 logf32p(float chi, const ThetaCf& c) {
    float xh, xl;
    sub2x(chi, c.loc_hi, c.loc_lo, xh, xl);
    const float e = exp32(xh);
    return F2{__fmaf_rn(c.sc_hi, xh, -e), __fmaf_rn(c.sc_hi, xl, __fmaf_rn(c.sc_lo, xh, -__fmul_rn(e, xl)))};
  }
  // the member step's log f (one binary32 value; the accept needs no more) and e^x, which the
  // theta' partial of the state needs
  __device__ static float logf32_e(float chi, const ThetaCf& c, float& carry) {
    float xh, xl;
    sub2x(chi, c.loc_hi, c.loc_lo, xh, xl);
    const float e = exp32(xh);
    carry = e;
    const float ex = __fmaf_rn(e, xl, e);  // e^(xh + xl) to first order in xl
    return __fmaf_rn(c.sc_hi, xh, __fmaf_rn(c.sc_hi, xl, __fmaf_rn(c.sc_lo, xh, -ex)));
  }
  // theta -> theta' constants in binary64, each rounded to hi + lo: dsc = beta' - beta,
  // c = (beta' + 1)(ln L*' - ln L*), em = e^(ln L* - ln L*') - 1
  __device__ static ThetaDf dconsts32(const ThetaC& t, const ThetaC& tp) {
    ThetaDf d{};
    const double dL = tp.a1 - t.a1;
    split_f(tp.a0 - t.a0, d.dsc_hi, d.dsc_lo);
    split_f(tp.a0 * dL, d.c_hi, d.c_lo);
    split_f(expm1_theta(-dL), d.em_hi, d.em_lo);
    return d;
  }
  // d_i = log f(chi;theta') - log f(chi;theta) = dsc x - c - e^x em with x = chi - ln L* (xh + xl)
  // and e = e^xh (e^x = e (1 + xl) to first order): the small terms (the lo parts, xl) are summed
  // first and enter the large ones inside single roundings, so none is rounded away alike for
  // every member; the difference of two O(1) log f values would lose ~1e-7 of each
  __device__ static float dtheta32(float chi, float e, const ThetaCf& c, const ThetaCf&, const ThetaDf& d) {
    float xh, xl;
    sub2x(chi, c.loc_hi, c.loc_lo, xh, xl);
    float b = __fmaf_rn(-e, __fmaf_rn(xl, d.em_hi, d.em_lo), -d.c_lo);
    b = __fmaf_rn(d.dsc_lo, xh, b);
    b = __fmaf_rn(d.dsc_hi, xl, b);
    return __fmaf_rn(d.dsc_hi, xh, __fmaf_rn(-e, d.em_hi, __fsub_rn(b, d.c_hi)));
  }
  // member data: d[0], d[1] = ln(Fhat_i/q_i) as hi + lo, d[2] = Fhat_i^2/(2 sigma_F^2) > 0, so
  // that log l_i = -d[2] expm1(chi - ln(Fhat_i/q_i))^2 keeps binary32 relative accuracy however
  // large Fhat_i/sigma_F is; a member with Fhat_i/sigma_F below 1e-3 (none is detected there)
  // holds d[0] = Fhat_i, d[1] = q_i and the marker d[2] = -1/(2 sigma_F^2) < 0, and evaluates
  // -(Fhat_i - e^chi q_i)^2/(2 sigma_F^2) directly. Three floats: 12 bytes per member-update.
  static constexpr int kData32 = 3;
  __device__ static void data32(double y, double aux, const ModelConsts& mc, float* d) {
    if (y > 0.0 && y * y * mc.inv2sig2 >= 5e-7) {
      split_f(log(y / aux), d[0], d[1]);
      d[2] = static_cast<float>(y * y * mc.inv2sig2);
    } else {
      d[0] = static_cast<float>(y);
      d[1] = static_cast<float>(aux);
      d[2] = static_cast<float>(-mc.inv2sig2);
    }
  }
  __device__ static float loglike32(float chi, const float* d) {
    if (!(d[2] < 0.0f)) {
      const float e = expm1_32(sub2(chi, d[0], d[1]));
      return __fmul_rn(-d[2], __fmul_rn(e, e));
    }
    const float r = __fmaf_rn(-exp32(chi), d[1], d[0]);
    return __fmul_rn(__fmul_rn(r, r), d[2]);
  }
  __device__ static ThetaC consts(const double* th, const ModelConsts&, const double* T) {
    ThetaC c;
    c.a0 = th[0] + 1.0;
    c.a1 = th[1];
    c.a2 = exp_tab(-th[1], T);
    c.a3 = th[2];
    c.a4 = 0.0;
    return c;
  }
  __device__ static bool support(double chi, const ThetaC& c) { return dgt(chi, c.a3); }
  __device__ static double logf(double chi, double echi, const ThetaC& c) {
    return __fma_rn(c.a0, __dsub_rn(chi, c.a1), -__dmul_rn(echi, c.a2));
  }
  // y = Fhat_i, aux = q_i = 1/(4 pi r_i^2)
  __device__ static double loglike(double, double echi, double y, double aux, const ModelConsts& mc) {
    const double r = __fma_rn(-echi, aux, y);
    return -__dmul_rn(__dmul_rn(r, r), mc.inv2sig2);
  }
  __device__ static double cterm(const double*) { return 0.0; }
  __device__ static double logprior(const double* th, const ModelConsts&, const double* T) {
    if (!(th[0] > -2.0 && th[0] < 0.0)) return -INFINITY;
    if (!(th[2] < th[1])) return -INFINITY;
    return -log_tab(1.0 + th[0] * th[0], T) + th[2];  // 1 + beta^2 in [1, 5): a normal argument
  }
};

// The paper's BB1 luminosity function (Sec. 5.1-5.2, App. B eq. lumPDF), chi = ln L, theta =
// (beta, ln l, ln u): log f = ln(1 - e^{-L/l}) + beta (chi - ln u) - L/u + chi (the normaliser
// C(beta,u,l)/u cancels against the normalised selection integral); member likelihood the normal
// density of Fhat_i with sd sigma(F), sigma(F)^2 = sigma0^2 + (alpha F)^2, F = e^chi q_i;
// prior -ln(1 + beta^2) + ln l on -2 < beta < 0, l < u. FP64 form only.
// a0 = beta, a1 = ln u, a2 = 1/u, a3 = 1/l, a4 = ln l
struct BB1 {
  using TC = ThetaC;
  using TCf = ThetaCf;
  static constexpr int kD = 1;
  static constexpr bool kExp = true;
  static constexpr bool kRule = true;  // selection integral with sigma(F) inside Phi
  __device__ static ThetaC consts(const double* th, const ModelConsts&, const double* T) {
    ThetaC c;
    c.a0 = th[0];
    c.a1 = th[2];
    c.a2 = exp_tab(-th[2], T);
    c.a3 = exp_tab(-th[1], T);
    c.a4 = th[1];
    return c;
  }
  __device__ static bool support(double, const ThetaC&) { return true; }
  // ln(1 - e^{-x}), x > 0 (Maechler's two branches)
  __device__ static double log1mexp(double x) {
    return (x <= 0.69314718055994530942) ? log(-expm1(-x)) : log1p(-exp(-x));
  }
  __device__ static double logf(double chi, double echi, const ThetaC& c) {
    const double lg = log1mexp(__dmul_rn(echi, c.a3));
    return __dadd_rn(__dadd_rn(lg, __fma_rn(c.a0, __dsub_rn(chi, c.a1), -__dmul_rn(echi, c.a2))), chi);
  }
  // y = Fhat_i, aux = q_i = 1/(4 pi r_i^2)
  __device__ static double loglike(double, double echi, double y, double aux, const ModelConsts& mc) {
    const double F = __dmul_rn(echi, aux);
    const double aF = __dmul_rn(mc.alpha, F);
    const double s2 = __fma_rn(aF, aF, mc.s0sq);
    const double r = __dsub_rn(y, F);
    return __dsub_rn(__dmul_rn(-0.5, log(s2)), __ddiv_rn(__dmul_rn(r, r), __dmul_rn(2.0, s2)));
  }
  __device__ static double cterm(const double*) { return 0.0; }
  __device__ static double logprior(const double* th, const ModelConsts&, const double* T) {
    if (!(th[0] > -2.0 && th[0] < 0.0)) return -INFINITY;
    if (!(th[1] < th[2])) return -INFINITY;
    return -log_tab(1.0 + th[0] * th[0], T) + th[1];
  }
  // no binary32 form; these keep the FP32 instantiations of generic code compiling
  static constexpr int kData32 = 1;
  __device__ static ThetaCf consts32(const ThetaC&) { return ThetaCf{}; }
  __device__ static bool support32(float, const ThetaCf&) { return true; }
  __device__ static float logf32(float, const ThetaCf&) { return 0.0f; }
  __device__ static F2 logf32p(float, const ThetaCf&) { return F2{0.0f, 0.0f}; }
  __device__ static float logf32_e(float, const ThetaCf&, float& carry) {
    carry = 0.0f;
    return 0.0f;
  }
  __device__ static ThetaDf dconsts32(const ThetaC&, const ThetaC&) { return ThetaDf{}; }
  __device__ static float dtheta32(float, float, const ThetaCf&, const ThetaCf&, const ThetaDf&) { return 0.0f; }
  __device__ static void data32(double, double, const ModelConsts&, float* d) { d[0] = 0.0f; }
  __device__ static float loglike32(float, const float*) { return 0.0f; }
};

// d = 3 normal population (Sec. 3 with C_pop unknown). theta = (mu[3], L11, L21, L22, L31, L32,
// L33) with L the lower Cholesky factor of C_pop, its diagonal entries stored as logs. The
// per-theta constants hold mu and the packed inverse factor Li = L^-1 (lower, row-major:
// li0 = Li00, li1 = Li10, li2 = Li11, li3 = Li20, li4 = Li21, li5 = Li22), so that
// log f = -|Li (chi - mu)|^2 / 2 needs no division per member. Member data are stored per
// component (structure of arrays): y_ij and aux_ij = 1/s_ij^2.
struct ThetaC3 {
  double mu[3];
  double li[6];
};
// binary32 form: every constant as hi + lo, since each one is shared by all members and its
// rounding would otherwise bias the sum over members
struct ThetaC3f {
  float mu_hi[3], mu_lo[3];
  float li_hi[6], li_lo[6];
};

// d = 3 normal population. kKnown = false: theta = (mu, L_C) with L_C lower-triangular and
// log-diagonal (p = 9). kKnown = true: the paper's normal-normal benchmark (Sec. 3), C_pop
// known, theta = mu (p = 3), the inverse factor of C_pop taken from the model constants.
template <bool kKnown>
struct MVN3T {
  using TC = ThetaC3;
  using TCf = ThetaC3f;
  static constexpr int kD = 3;
  static constexpr bool kRule = false;
  static constexpr bool kExp = false;
  __device__ static ThetaC3 consts(const double* th, const ModelConsts& mc, const double* T) {
    ThetaC3 c;
    c.mu[0] = th[0];
    c.mu[1] = th[1];
    c.mu[2] = th[2];
    if constexpr (kKnown) {
      for (int j = 0; j < 6; ++j) c.li[j] = mc.li3[j];
    } else {
      const double L00 = exp_tab(th[3], T), L10 = th[4], L11 = exp_tab(th[5], T), L20 = th[6], L21 = th[7],
                   L22 = exp_tab(th[8], T);
      c.li[0] = 1.0 / L00;
      c.li[2] = 1.0 / L11;
      c.li[5] = 1.0 / L22;
      c.li[1] = -(L10 * c.li[0]) * c.li[2];
      c.li[4] = -(L21 * c.li[2]) * c.li[5];
      c.li[3] = -(L20 * c.li[0] + L21 * c.li[1]) * c.li[5];
    }
    return c;
  }
  __device__ static double logf(const double* x, const ThetaC3& c) {
    const double r0 = __dsub_rn(x[0], c.mu[0]), r1 = __dsub_rn(x[1], c.mu[1]), r2 = __dsub_rn(x[2], c.mu[2]);
    const double z0 = __dmul_rn(c.li[0], r0);
    const double z1 = __fma_rn(c.li[1], r0, __dmul_rn(c.li[2], r1));
    const double z2 = __fma_rn(c.li[3], r0, __fma_rn(c.li[4], r1, __dmul_rn(c.li[5], r2)));
    return __dmul_rn(-0.5, __fma_rn(z0, z0, __fma_rn(z1, z1, __dmul_rn(z2, z2))));
  }
  // y[j], w[j] = 1/s_j^2
  __device__ static double loglike(const double* x, const double* y, const double* w) {
    const double e0 = __dsub_rn(y[0], x[0]), e1 = __dsub_rn(y[1], x[1]), e2 = __dsub_rn(y[2], x[2]);
    const double q = __fma_rn(__dmul_rn(w[0], e0), e0,
                              __fma_rn(__dmul_rn(w[1], e1), e1, __dmul_rn(__dmul_rn(w[2], e2), e2)));
    return __dmul_rn(-0.5, q);
  }
  __device__ static double cterm(const double* th) {
    if constexpr (kKnown) return 0.0;  // -ln det L_C is a constant when C_pop is known
    else return -((th[3] + th[5]) + th[8]);
  }
  // flat in mu (and, unknown C_pop, in the off-diagonal and log-diagonal entries); improper
  __device__ static double logprior(const double*, const ModelConsts&, const double*) { return 0.0; }

  __device__ static ThetaC3f consts32(const ThetaC3& c) {
    ThetaC3f f;
    for (int j = 0; j < 3; ++j) split_f(c.mu[j], f.mu_hi[j], f.mu_lo[j]);
    for (int j = 0; j < 6; ++j) split_f(c.li[j], f.li_hi[j], f.li_lo[j]);
    return f;
  }
  // -|Li (chi - mu)|^2/2 in binary32 with chi - mu and Li carried as hi + lo pairs: each z_j is
  // the sum of the hi products plus the first-order cross terms, rounded once per fma.
  __device__ static float logf32(const float* x, const ThetaC3f& c) {
    float rh[3], rl[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) sub2x(x[j], c.mu_hi[j], c.mu_lo[j], rh[j], rl[j]);
    const float* h = c.li_hi;
    const float* l = c.li_lo;
    const float e0 = __fmaf_rn(h[0], rl[0], __fmul_rn(l[0], rh[0]));
    const float z0 = __fmaf_rn(h[0], rh[0], e0);
    const float e1 = __fmaf_rn(h[1], rl[0], __fmaf_rn(l[1], rh[0], __fmaf_rn(h[2], rl[1], __fmul_rn(l[2], rh[1]))));
    const float z1 = __fmaf_rn(h[1], rh[0], __fmaf_rn(h[2], rh[1], e1));
    const float e2 = __fmaf_rn(h[3], rl[0], __fmaf_rn(l[3], rh[0], __fmaf_rn(h[4], rl[1],
                     __fmaf_rn(l[4], rh[1], __fmaf_rn(h[5], rl[2], __fmul_rn(l[5], rh[2]))))));
    const float z2 = __fmaf_rn(h[3], rh[0], __fmaf_rn(h[4], rh[1], __fmaf_rn(h[5], rh[2], e2)));
    return __fmul_rn(-0.5f, __fmaf_rn(z0, z0, __fmaf_rn(z1, z1, __fmul_rn(z2, z2))));
  }
  // member data: d[2j], d[2j+1] = y_ij as hi + lo, d[6 + j] = 1/(2 s_ij^2)
  static constexpr int kData32 = 9;
  __device__ static float loglike32(const float* x, const float* d) {
    const float e0 = __fadd_rn(__fsub_rn(d[0], x[0]), d[1]);
    const float e1 = __fadd_rn(__fsub_rn(d[2], x[1]), d[3]);
    const float e2 = __fadd_rn(__fsub_rn(d[4], x[2]), d[5]);
    const float q = __fmaf_rn(__fmul_rn(d[6], e0), e0,
                              __fmaf_rn(__fmul_rn(d[7], e1), e1, __fmul_rn(__fmul_rn(d[8], e2), e2)));
    return -q;
  }
};

using MVN3 = MVN3T<false>;
using NN3 = MVN3T<true>;

// RAM factor update for d = 3 (Sec. 2.2): S' S'^T = S (I + c U U^T/|U|^2) S^T
// = S S^T + sig w w^T with w = S U and sig = c/|U|^2, as a rank-one Cholesky modification
// of the packed lower factor S = (S00, S10, S11, S20, S21, S22). Column k: with a = S_kk,
// b = w_k and r = sqrt(a^2 + sig b^2), S'_kk = r, S'_ik = (a S_ik + sig b w_i)/r and the
// vector carried to the next column is w_i' = (a w_i - b S_ik)/r (i > k). The diagonal
// stays positive because 1 + c >= 1 - alpha_* > 0.
__device__ __forceinline__ void ram3_update(double (&S)[6], double w0, double w1, double w2, double sig) {
  {
    const double a = S[0], b = w0, sb = sig * b;
    const double t = fma(sb, b, a * a);
    const double ir = rsqrt(t);
    const double n1 = fma(a, S[1], sb * w1) * ir, v1 = fma(a, w1, -b * S[1]) * ir;
    const double n3 = fma(a, S[3], sb * w2) * ir, v2 = fma(a, w2, -b * S[3]) * ir;
    S[0] = t * ir;
    S[1] = n1;
    S[3] = n3;
    w1 = v1;
    w2 = v2;
  }
  {
    const double a = S[2], b = w1, sb = sig * b;
    const double t = fma(sb, b, a * a);
    const double ir = rsqrt(t);
    const double n4 = fma(a, S[4], sb * w2) * ir, v2 = fma(a, w2, -b * S[4]) * ir;
    S[2] = t * ir;
    S[4] = n4;
    w2 = v2;
  }
  S[5] = sqrt(fma(sig * w2, w2, S[5] * S[5]));
}

// ----------------------------------------------------- theta RAM update -------
// Lower-triangular L (p x p, row-major) with L' L'^T = L (I + c U U^T/|U|^2) L^T
// = L L^T + sig w w^T, c = eta (alpha - alpha_*), w = L U, sig = c/|U|^2: the rank-one Cholesky
// modification of ram3_update for any p. Column k: a = L_kk, b = w_k, t = a^2 + sig b^2,
// L'_kk = sqrt t, L'_ik = (a L_ik + sig b w_i)/sqrt t, w_i <- (a w_i - b L_ik)/sqrt t (i > k).
// t > 0 because 1 + c >= 1 - alpha_* > 0. This runs once per sweep on the theta step's serial
// path, so it is written with one reciprocal square root per column and no divisions there.
__device__ inline void ram_update_theta(int p, double* L, const double* U, double alpha, double astar, double eta) {
  const double c = eta * (alpha - astar);
  if (c == 0.0) return;
  double uu = 0.0;
  for (int j = 0; j < p; ++j) uu = fma(U[j], U[j], uu);
  const double sig = c / uu;
  double w[kMaxP];
  for (int a = 0; a < p; ++a) {
    double t = 0.0;
    for (int b = 0; b <= a; ++b) t = fma(L[a * p + b], U[b], t);
    w[a] = t;
  }
  for (int k = 0; k < p; ++k) {
    const double a = L[k * p + k], b = w[k], sb = sig * b;
    const double t = fma(sb, b, a * a);
    const double ir = rsqrt(t);
    L[k * p + k] = t * ir;
    const double air = a * ir, bir = b * ir, sbir = sb * ir;
    for (int i = k + 1; i < p; ++i) {
      const double lik = L[i * p + k];
      L[i * p + k] = fma(air, lik, sbir * w[i]);
      w[i] = fma(air, w[i], -bir * lik);
    }
  }
}

// ------------------------------------------------------- normal CDF Phi -------
// Phi(x) = erfc(-x/sqrt 2)/2 (Sec. 5.2, eq. key) by a table of local Taylor polynomials in the
// scaled variable v = 16 x: intervals centred at c_i = -8 + i/16 (i = 0..kPhiN-1, so v_i = 16 c_i
// is the integer i - 128), |x - c_i| <= 1/32, degree kPhiDeg = 8. With phi = Phi' and
// d^n Phi/dx^n = (-1)^(n-1) He_(n-1)(x) phi(x) (He = probabilists' Hermite polynomials), the
// Taylor coefficients are a_0 = Phi(c), a_n = (-1)^(n-1) He_(n-1)(c) phi(c)/n!; the table holds
// b_n = a_n/16^n, the coefficients of the series in u = v - v_i = 16 (x - c_i), |u| <= 1/2.
// a_0 is Phi(c) itself, taken as 1 - erfc(c/sqrt 2)/2 for c > 0, so values near 1 carry an
// absolute error of an ulp of 1. The remainder of the degree-8 series on |x - c| <= 1/32 is
// below 4e-18 (|He_8 phi| <= 42); the table is built once per handle on the device from CUDA's
// erfc and exp. Above x = 8.5 (v = 136), Phi rounds to 1 exactly; below x = -8 (Phi < 7e-16)
// erfc is called directly.
constexpr int kPhiN = 265;
constexpr int kPhiDeg = 8;
constexpr int kPhiWords = kPhiN * (kPhiDeg + 1);  // coefficient-major: coef[n * kPhiN + i]

// Phi(v/16): four FP64 operations to reach u, eight for the polynomial.
__device__ __forceinline__ double phi_table16(double v, const double* __restrict__ coef) {
  const long long b = __double_as_longlong(v);
  if (b > 0x4061000000000000ll) return 1.0;  // v > 136 (and +inf)
  if (static_cast<unsigned long long>(b) > 0xC060000000000000ull)  // v < -128 (and -inf)
    return 0.5 * erfc(-(v * 0.0625) * 0.70710678118654752440);
  const double magic = 6755399441055744.0;  // 1.5 * 2^52
  const double r = v + magic;               // round(v) sits in the low mantissa bits
  const int i = __double2loint(r) + 128;
  const double u = v - (r - magic);         // exact, |u| <= 1/2
  double q = coef[kPhiDeg * kPhiN + i];
#pragma unroll
  for (int n = kPhiDeg - 1; n >= 0; --n) q = fma(q, u, coef[n * kPhiN + i]);
  return q;
}
__device__ __forceinline__ double phi_table(double x, const double* __restrict__ coef) {
  return phi_table16(16.0 * x, coef);
}

// ------------------------------------------------------------ LF rule --------
// The 2-D rule is cut into segments of kSeg consecutive inner nodes of one outer node:
// segment g = s * nL + j covers outer node j and inner nodes [s kSeg, (s+1) kSeg). Block b
// of B takes segments b, b + B, b + 2B, ...: every block sees the whole range of L and of r,
// so blocks get the same mix of pairs that need erfc and pairs where Phi = 1 exactly.
constexpr int kSegShift = 7;
constexpr int kSeg = 1 << kSegShift;

__device__ __forceinline__ int lf_block_segments(const SweepArgs& a, int b, int B) {
  const int spr = (a.nr + kSeg - 1) >> kSegShift;
  const int G = a.nL * spr;
  return (b < G) ? (G - b + B - 1) / B : 0;
}

// Per-block segment table in shared memory, R slots: 16 L_j, G_j, the row's prefix term, the
// first active inner node kb and the exclusive offsets of the active pair counts (R + 1).
struct SegTab {
  double* L;
  double* G;
  double* pre;
  int* kb;
  int* off;
};
__host__ __device__ inline size_t segtab_bytes(int R) {
  return 3 * sizeof(double) * static_cast<size_t>(R) + sizeof(int) * (2 * static_cast<size_t>(R) + 1);
}
__device__ __forceinline__ SegTab segtab_carve(double* base, int R) {
  SegTab t;
  t.L = base;
  t.G = base + R;
  t.pre = base + 2 * R;
  t.kb = reinterpret_cast<int*>(base + 3 * R);
  t.off = t.kb + R;
  return t;
}

// Values of segment t (one thread; T is the exp/log table): L_j = e^t_j and G_j = (half-width)
// w_j g(e^t_j) e^t_j over the outer interval (LF: [ln L_low, ln L* + ln_upper] with the Schechter
// form; BB1: [ln l + ln_lower, ln u + ln_upper] with the BB1 form). Since x_jk (the argument of Phi)
// decreases along the inner nodes (r ascending), the pairs with x > 8.5, where Phi is exactly 1,
// are a prefix k < k*_j of the row; they contribute G_j CW[k*_j] with CW the prefix sums of the
// inner weights, added once per row (by its segment s = 0). Only k >= max(k*_j, s kSeg) is left to
// evaluate; the count goes to off[t] until the block scans it. LF keeps 16 L_j, so that
// v = 16 x_jk = fma(16 L_j, qs_k, -16 F_th/sigma_F) is one operation (qs_k = q_k/sigma_F); BB1 keeps
// L_j and evaluates x = (L_j q_k - F_th)/sigma(L_j q_k) per pair.
template <class M>
__device__ __forceinline__ void lf_segment_row(const ThetaC& tc, const SweepArgs& a, int b, int B, int t, int slot,
                                               const SegTab& tab, const double* __restrict__ T) {
  constexpr bool bb1 = std::is_same<M, BB1>::value;
  const double lo = bb1 ? tc.a4 + a.mc.ln_lower : tc.a3;
  const double hi = tc.a1 + a.mc.ln_upper;
  const double half = 0.5 * (hi - lo), mid = 0.5 * (hi + lo);
  const int g = b + t * B;
  const int j = g % a.nL;
  const int sseg = g / a.nL;
  const double tt = fma(half, __ldg(a.xL + j), mid);
  double Lrow, G, thr_d;
  if constexpr (bb1) {
    const double L = exp_tab(tt, T);
    const double lg = BB1::log1mexp(L * tc.a3);
    G = half * __ldg(a.wL + j) * exp_tab(lg + fma(tc.a0, tt - tc.a1, -L * tc.a2) + tt, T);
    Lrow = L;
    thr_d = a.mc.F_pre / L;  // q_k > F_pre/L_j  <=>  x_jk > 8.5
  } else {
    const double x = tt - tc.a1;
    const double L16 = 16.0 * exp_tab(tt, T);
    G = half * __ldg(a.wL + j) * exp_tab(fma(tc.a0, x, -exp_tab(x, T)), T);
    Lrow = L16;
    thr_d = (136.0 + 16.0 * a.mc.cth) / L16;  // qs_k > thr  <=>  v_jk > 136, up to rounding
  }
  // first k with qs_k <= thr (both sides of that boundary give Phi = 1 exactly); positive doubles
  // compared as integers
  const long long thr = __double_as_longlong(thr_d);
  int klo = 0, khi = a.nr;
  while (klo < khi) {
    const int km = (klo + khi) >> 1;
    if (__double_as_longlong(__ldg(a.qs + km)) > thr) klo = km + 1;
    else khi = km;
  }
  const int k0 = sseg << kSegShift;
  const int kend = min(k0 + kSeg, a.nr);
  const int kb = max(k0, klo);
  tab.L[slot] = Lrow;
  tab.G[slot] = G;
  tab.pre[slot] = (sseg == 0 && klo > 0) ? G * __ldg(a.cw + klo) : 0.0;
  tab.kb[slot] = kb;
  tab.off[slot] = max(0, kend - kb);
}

// Exclusive scan of the active counts (one warp); off[nseg] receives the total.
__device__ __forceinline__ void lf_segment_scan(int nseg, const SegTab& tab) {
  const int lane = threadIdx.x & 31;
  int carry = 0;
  for (int base = 0; base < nseg; base += 32) {
    const int t = base + lane;
    const int c = (t < nseg) ? tab.off[t] : 0;
    int v = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, v, o);
      if (lane >= o) v += y;
    }
    if (t < nseg) tab.off[t] = carry + v - c;
    carry += __shfl_sync(0xffffffffu, v, 31);
  }
  if (lane == 0) tab.off[nseg] = carry;
}

// All segment rows and the scan by the whole block (set-up paths).
template <class M>
__device__ __forceinline__ void lf_segment_rows(const ThetaC& tc, const SweepArgs& a, int b, int B, int nseg,
                                                const SegTab& tab, const double* __restrict__ T) {
  for (int t = threadIdx.x; t < nseg; t += blockDim.x) lf_segment_row<M>(tc, a, b, B, t, t, tab, T);
  __syncthreads();
  if (threadIdx.x < 32) lf_segment_scan(nseg, tab);
}

// The block's active pairs (all lanes busy) and its rows' prefix terms; each term
// G_j W_k Phi(x_jk) is added exactly.
template <class M>
__device__ __forceinline__ void lf_segment_pairs(const SweepArgs& a, int nseg, const SegTab& tab, const double* s_phi,
                                                 Xacc& xe, XFlags& fe) {
  constexpr bool bb1 = std::is_same<M, BB1>::value;
  const int total = tab.off[nseg];
  const double mcth16 = -16.0 * a.mc.cth;
  for (int q = threadIdx.x; q < total; q += blockDim.x) {
    int lo = 0, hi = nseg - 1;  // last segment with off <= q
    while (lo < hi) {
      const int m = (lo + hi + 1) >> 1;
      if (tab.off[m] <= q) lo = m;
      else hi = m - 1;
    }
    const int k = tab.kb[lo] + (q - tab.off[lo]);
    double v;
    if constexpr (bb1) {  // 16 (F - F_th)/sigma(F), F = L_j q_k
      const double F = tab.L[lo] * __ldg(a.qs + k);
      const double aF = a.mc.alpha * F;
      v = 16.0 * (F - a.mc.F_th) * rsqrt(fma(aF, aF, a.mc.s0sq));
    } else {
      v = fma(tab.L[lo], __ldg(a.qs + k), mcth16);
    }
    xacc_add_double(xe, tab.G[lo] * (__ldg(a.Wr + k) * phi_table16(v, s_phi)), fe);
  }
  for (int t = threadIdx.x; t < nseg; t += blockDim.x)
    if (tab.pre[t] != 0.0) xacc_add_double(xe, tab.pre[t], fe);
}

// ------------------------------------------------ tabulated inner sum -------
// The selection integral is etabar(theta) = sum_j G_j(theta) H(t_j) over the outer nodes t_j
// (ln L), with the inner sum H(u) = sum_k W_k Phi(x_k(e^u)) of the rule. H depends on L alone,
// not on theta, so it is tabulated once per handle (htab_build_kernel: each cell's Chebyshev
// interpolant of degree kHDeg through the rule's exact inner sums at the Chebyshev points; within
// a few ulp of H over the whole range), and a sweep evaluates n_L table lookups instead of
// n_L n_r normal CDFs. Below the table H is constant to rounding (every x_k equals its L = 0
// value), above it every pair has Phi = 1.
__device__ __forceinline__ double htab_eval(double u, const SweepArgs& a) {
  if (!(u < a.h_ub)) return a.h_hi;
  if (!(u > a.h_ua)) return a.h_lo;
  const double z = (u - a.h_ua) * (1.0 / kHDelta);
  const int ci = min(static_cast<int>(z), a.h_ncell - 1);
  const double sx = fma(2.0, z - static_cast<double>(ci), -1.0);
  const double* c = a.htab + ci * (kHDeg + 1);
  double b1 = 0.0, b2 = 0.0;  // Clenshaw
#pragma unroll
  for (int j = kHDeg; j >= 1; --j) {
    const double t = fma(2.0 * sx, b1, __ldg(c + j) - b2);
    b2 = b1;
    b1 = t;
  }
  return fma(sx, b1, __ldg(c) - b2);
}

// The outer node j's term G_j H(t_j) (LF: G_j = half w_j e^{(beta+1)(t - ln L*) - e^{t - ln L*}};
// BB1: half w_j (1 - e^{-L/l}) e^{beta (t - ln u) - L/u + t}), added exactly to xe.
template <class M>
__device__ __forceinline__ void etabar_node(const ThetaC& tc, const SweepArgs& a, int j, const double* __restrict__ T,
                                            Xacc& xe, XFlags& fe) {
  constexpr bool bb1 = std::is_same<M, BB1>::value;
  const double lo = bb1 ? tc.a4 + a.mc.ln_lower : tc.a3;
  const double hi = tc.a1 + a.mc.ln_upper;
  const double half = 0.5 * (hi - lo), mid = 0.5 * (hi + lo);
  const double tt = fma(half, __ldg(a.xL + j), mid);
  double G;
  if constexpr (bb1) {
    const double L = exp_tab(tt, T);
    const double lg = BB1::log1mexp(L * tc.a3);
    G = half * __ldg(a.wL + j) * exp_tab(lg + fma(tc.a0, tt - tc.a1, -L * tc.a2) + tt, T);
  } else {
    const double x = tt - tc.a1;
    G = half * __ldg(a.wL + j) * exp_tab(fma(tc.a0, x, -exp_tab(x, T)), T);
  }
  xacc_add_double(xe, G * htab_eval(tt, a), fe);
}

// The outer nodes of the selection rule spread over the threads of all B blocks (block b, thread
// t: j = rule_j0 + b + B t), each node's term etabar_node added exactly to xe. A shard of a split
// population covers its own range [rule_j0, rule_j1) (rule_j1 = 0: all n_L), so that every node
// is counted once over all shards.
template <class M>
__device__ __forceinline__ void etabar_terms(const ThetaC& tc, const SweepArgs& a, int b, int B,
                                             const double* __restrict__ T, Xacc& xe, XFlags& fe) {
  const int j1 = a.rule_j1 ? a.rule_j1 : a.nL;
  for (int j = a.rule_j0 + b + B * static_cast<int>(threadIdx.x); j < j1; j += B * static_cast<int>(blockDim.x))
    etabar_node<M>(tc, a, j, T, xe, fe);
}

// ------------------------------------------------------ member accept rule ---
// The member step's Metropolis accept (Sec. 2.2; strict, as ln u < Delta): alpha = min(1, e^Delta)
// (0 at Delta = -inf), accepted iff u < alpha. Binary64: every Delta with its sign bit clear
// accepts; otherwise u and alpha are both >= +0, so their bit patterns order as their values.
// Binary32 (bulk form): the same rule with the special-function unit's exponential.
// Below Delta = -700, alpha = e^Delta < 1e-304 is taken as 0: every accept uniform is at least
// 2^-53, so the decision is the same, and alpha - alpha_* rounds to -alpha_* either way, so the
// RAM update is too; this keeps the exponential on its table path (the library routine that
// exp_tab falls back to there is several times longer, and early in a chain, before the RAM
// factors adapt, most bright members propose that far out).
__device__ __forceinline__ bool mh_accept(double delta, double u, const double* s_math, double& alpha) {
  const bool dneg = dsign(delta);  // -inf and -0 included
  alpha = !dneg ? 1.0 : (dgt(delta, -700.0) ? exp_tab(delta, s_math) : 0.0);
  return !dneg || (__double_as_longlong(u) < __double_as_longlong(alpha));
}

__device__ __forceinline__ bool mh_accept32(float delta, float u, float& alpha) {
  alpha = (delta >= 0.0f) ? 1.0f : __expf(delta);  // the special-function unit's 2^x (a few ulp)
  return (delta >= 0.0f) || (u < alpha);
}

// Binary32 uniform in (0, 1) of the FP32 bulk form from one Philox word: (m + 1/2) 2^-23 with m the
// word's top 23 bits, assembled from the bits (1 + m 2^-23, then 1 - 2^-24 subtracted: exact by
// Sterbenz's lemma), with no integer-to-float conversion instruction.
__device__ __forceinline__ float uniform23(uint32_t w) {
  return __fsub_rn(__uint_as_float(0x3F800000u | (w >> 9)), 0x1.fffffep-1f);
}

// A standard normal pair of the FP32 bulk form by Box-Muller from two uniforms: radius
// sqrt(-2 ln u1) (ln by CUDA's logf: -2 ln u1 >= 2^-23 > 0 for every u1 uniform23 gives), angle
// 2 pi u2 taken as pi (2 u2 - 1) + pi, so that the special-function unit's sine and cosine see an
// argument in [-pi, pi) (absolute error ~2^-21); the square root from the reciprocal square
// root. The draws of the FP32 form are held to statistics, not to bit-parity with the oracle.
__device__ __forceinline__ void box_muller32(uint32_t wa, uint32_t wb, float& z_cos, float& z_sin) {
  const float t = __fmul_rn(-2.0f, logf(uniform23(wa)));
  const float rad = __fmul_rn(t, rsqrtf(t));
  float sn, cs;
  __sincosf(__fmul_rn(3.14159265358979323846f, __fsub_rn(__fmul_rn(2.0f, uniform23(wb)), 1.0f)), &sn, &cs);
  z_cos = -__fmul_rn(rad, cs);  // cos(a + pi) = -cos a, sin(a + pi) = -sin a
  z_sin = -__fmul_rn(rad, sn);
}

// ------------------------------------ FP32 bulk form: the d = 1 RAM factor ---
// The FP32 form keeps S in binary64 and steps members in binary32. The conversions between the
// two run on the integer pipe (GB300's FP64 pipe is the scarce unit), and the factor update
// S <- S sqrt(1 + c), c = eta (alpha - alpha_*) (Sec. 2.2, d = 1) costs one binary64 FMA:
// S + S d with the increment d = sqrt(1 + c) - 1 = c / (1 + sqrt(1 + c)) formed in binary32
// (no cancellation; alpha is a binary32 value, so c carries binary32 error anyway). The update
// is then exact to ~1e-7 |c| relative, and S itself never loses binary64 precision.

// binary64 -> binary32 rounded toward zero, on the integer pipe only (the proposal scale of a
// member; any positive scale gives a valid proposal): magnitudes beyond binary32's normal range
// clamp to its largest or smallest normal value.
__device__ __forceinline__ float f32_rz(double x) {
  const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(x));
  const int e = static_cast<int>((b >> 52) & 0x7ff) - 1023 + 127;
  const unsigned int sign = static_cast<unsigned int>(b >> 32) & 0x80000000u;
  const unsigned int body = (e >= 255) ? 0x7F7FFFFFu
                            : (e <= 0) ? 0x00800000u
                                       : (static_cast<unsigned int>(e) << 23) |
                                             static_cast<unsigned int>((b >> 29) & 0x7FFFFFull);
  return __uint_as_float(sign | body);
}

// binary32 -> binary64, exact, on the integer pipe only (every class: zeros, subnormals
// normalised by a leading-zero count, normal values, infinities and NaN)
__device__ __forceinline__ double f64_of(float v) {
  const unsigned int u = __float_as_uint(v);
  const unsigned int e = (u >> 23) & 0xffu, m = u & 0x7FFFFFu;
  const unsigned long long sign = static_cast<unsigned long long>(u >> 31) << 63;
  unsigned long long body;
  if (e == 0xffu) {
    body = (0x7FFull << 52) | (static_cast<unsigned long long>(m) << 29);
  } else if (e != 0u) {
    body = (static_cast<unsigned long long>(e + 896u) << 52) | (static_cast<unsigned long long>(m) << 29);
  } else if (m != 0u) {  // m 2^-149: shift the leading bit to position 23
    const unsigned int k = static_cast<unsigned int>(__clz(m)) - 8u;
    body = (static_cast<unsigned long long>(897u - k) << 52) |
           (static_cast<unsigned long long>((m << k) & 0x7FFFFFu) << 29);
  } else {
    body = 0ull;
  }
  return __longlong_as_double(static_cast<long long>(sign | body));
}

// One RAM step of a d = 1 factor in the FP32 form: S + S d, d = c / (1 + sqrt(1 + c)) (1 + c >= 0.6:
// the square root from the reciprocal square root, the quotient by the fast reciprocal; d keeps
// a few binary32 ulp, far below the step's own randomness).
__device__ __forceinline__ double ram1_f32(double S, float alpha, float eta, float astar) {
  const float c = __fmul_rn(eta, __fsub_rn(alpha, astar));
  const float x = __fadd_rn(1.0f, c);
  const float d = __fdividef(c, __fadd_rn(1.0f, __fmul_rn(x, rsqrtf(x))));
  return __fma_rn(S, f64_of(d), S);
}

// ------------------------------------------- running moments of the latents -
// a8 (optional): every latent component's mean and sum of squared deviations M2 over the kept
// sweeps, by Welford's (1962) recurrence: with x the m-th kept value,
//   mean_m = mean_{m-1} + (x - mean_{m-1}) (1/m),  M2_m = M2_{m-1} + (x - mean_{m-1})(x - mean_m)
// (the sample variance is M2/(m - 1)). The moments sit in two buffers of [mean[d][n], M2[d][n]]:
// a launch reads the committed one (ChainState::mom_sel) at its first kept sweep, writes the
// other, and commits that one at its successful end, so a failed launch leaves the committed
// moments as they were, like the latents it did not write back.

// Sweep s of a launch is kept when it lies past the burn-in and its post-burn index counts a
// multiple of thin (the theta-row rule).
__device__ __forceinline__ bool kept_sweep(long long s, long long burn_left, long long keep_phase, long long thin) {
  const long long post = s - burn_left;
  return post >= 0 && thin > 0 && ((keep_phase + post + 1) % thin) == 0;
}

struct MomStep {
  const double* rd;  // mean at rd[q], M2 at rd[q + dn]
  double* wr;
  size_t dn;         // d n
  double rn;         // 1/m
};

// The k-th kept sweep of a launch whose committed buffer is sel and holds m0 kept sweeps.
__device__ __forceinline__ MomStep mom_step(const SweepArgs& a, int d, int sel, long long m0, long long k) {
  const size_t dn = static_cast<size_t>(d) * static_cast<size_t>(a.n);
  MomStep m;
  m.dn = dn;
  m.wr = a.mom + static_cast<size_t>(1 - sel) * 2 * dn;
  m.rd = (k == 1) ? a.mom + static_cast<size_t>(sel) * 2 * dn : m.wr;
  m.rn = 1.0 / static_cast<double>(m0 + k);
  return m;
}

// Adds the kept value x of component entry q (j n + i).
__device__ __forceinline__ void mom_add(const MomStep& m, size_t q, double x) {
  const double mean = m.rd[q], m2 = m.rd[q + m.dn];
  const double dl = x - mean;
  const double mn = fma(dl, m.rn, mean);
  m.wr[q] = mn;
  m.wr[q + m.dn] = fma(dl, x - mn, m2);
}

// ------------------------------------------------- block reduce helpers ------
struct BlockRed {
  Xacc d[32];
  Xacc e[32];
  unsigned int f[32][4];
};

__device__ __forceinline__ void warp_reduce(Xacc& d, Xacc& e, unsigned int f[4]) {
#pragma unroll
  for (int m = 16; m >= 1; m >>= 1) {
    Xacc t = xacc_shfl_xor(d, m);
    xacc_add(d, t);
    t = xacc_shfl_xor(e, m);
    xacc_add(e, t);
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) f[q] = __reduce_add_sync(0xffffffffu, f[q]);
}

// Grid totals by fire-and-forget atomic adds (red.global.add.u64): a block's exact partial
// (192-bit two's complement) is split into six 32-bit limbs, each added to its own 64-bit
// counter. No counter can overflow (fewer than 2^32 blocks add values below 2^32), and carrying
// the counters back into 192 bits gives the exact sum modulo 2^192, the value the partials'
// sum in any order has.
__device__ __forceinline__ void acc_add_limbs(unsigned long long* acc, const Xacc& x) {
  const unsigned long long w[3] = {x.w0, x.w1, x.w2};
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    atomicAdd(acc + 2 * q, w[q] & 0xFFFFFFFFull);
    atomicAdd(acc + 2 * q + 1, w[q] >> 32);
  }
}

__device__ __forceinline__ void acc_to_xacc(const unsigned long long* acc, Xacc& x) {
  unsigned long long w[3] = {0ull, 0ull, 0ull}, c = 0ull;
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    const unsigned long long t = __ldcg(acc + k) + c;
    c = t >> 32;
    w[k >> 1] |= (t & 0xFFFFFFFFull) << (32 * (k & 1));
  }
  x.w0 = w[0];
  x.w1 = w[1];
  x.w2 = w[2];
}

// Sum of nb consecutive per-block partials (kPartWords words each, from base) by the whole
// block: every thread loads at most a few partials at once (the loads overlap instead of one
// warp walking the list), then warp and block reductions. Must be called by every thread of
// the block; the totals are valid in warp 0. Uses red; syncs the block once.
__device__ __forceinline__ void sum_partials(const unsigned long long* base, int nb, BlockRed& red, Xacc& D, Xacc& E,
                                             unsigned int f[4]) {
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  xacc_zero(D);
  xacc_zero(E);
  f[0] = f[1] = f[2] = f[3] = 0u;
  for (int b = tid; b < nb; b += blockDim.x) {
    const unsigned long long* src = base + static_cast<size_t>(b) * kPartWords;
    Xacc t, u;
    t.w0 = __ldcg(src + 0);
    t.w1 = __ldcg(src + 1);
    t.w2 = __ldcg(src + 2);
    u.w0 = __ldcg(src + 3);
    u.w1 = __ldcg(src + 4);
    u.w2 = __ldcg(src + 5);
    const unsigned long long f01 = __ldcg(src + 6), f23 = __ldcg(src + 7);
    xacc_add(D, t);
    xacc_add(E, u);
    f[0] += static_cast<unsigned int>(f01);
    f[1] += static_cast<unsigned int>(f01 >> 32);
    f[2] += static_cast<unsigned int>(f23);
    f[3] += static_cast<unsigned int>(f23 >> 32);
  }
  warp_reduce(D, E, f);
  if (lane == 0) {
    red.d[wid] = D;
    red.e[wid] = E;
    for (int q = 0; q < 4; ++q) red.f[wid][q] = f[q];
  }
  __syncthreads();
  if (wid == 0) {
    const int nw = blockDim.x >> 5;
    xacc_zero(D);
    xacc_zero(E);
    f[0] = f[1] = f[2] = f[3] = 0u;
    if (lane < nw) {
      D = red.d[lane];
      E = red.e[lane];
      for (int q = 0; q < 4; ++q) f[q] = red.f[lane][q];
    }
    warp_reduce(D, E, f);
  }
}

// ln x for the selection integral: the table routine for positive normal finite x (the value
// of every theta step), the library routine otherwise (0, subnormal, inf).
__device__ __forceinline__ double log_etabar(double x, const double* s_math) {
  const long long b = __double_as_longlong(x);
  return (b >= 0x0010000000000000ll && b < 0x7FF0000000000000ll) ? log_tab(x, s_math) : log(x);
}

// theta' of one sweep as block 0 publishes it for the other blocks of a launch (one proposal
// and one RAM update of S_theta per sweep for the whole grid instead of one per block).
struct ThetaPub {
  double thp[kMaxP];
  double lpri_new;
  ThetaC tcp;
  ThetaCf tcpf;
  ThetaDf tdf;  // FP32 form: constants of the step from the sweep's theta to this theta'
};
static_assert(sizeof(ThetaPub) <= sizeof(double) * kPubWords, "ThetaPub does not fit its buffer");

// Publication of theta' proposals by block 0 to the other blocks of the sweep kernel: slots of
// kPubWords doubles in a.pub (slot 0: the launch's first theta'; slot 1 + 2 (t & 1) + c: the
// proposal of the launch's sweep t for outcome c of the decision before it), released by the
// sequence word a.bar[1] = t + 1 once sweep t's slots are written. Parity slots suffice: block 0
// writes sweep t + 2's after barrier t, which every block passes only after reading sweep t's.
__device__ __forceinline__ ThetaPub* pub_slot(const SweepArgs& a, int slot) {
  return reinterpret_cast<ThetaPub*>(a.pub + static_cast<size_t>(slot) * kPubWords);
}
__device__ __forceinline__ void put_pub(ThetaPub* dst, const ThetaPub& v, int p) {
  for (int q = 0; q < p; ++q) __stcg(dst->thp + q, v.thp[q]);
  __stcg(&dst->lpri_new, v.lpri_new);
  __stcg(&dst->tcp.a0, v.tcp.a0);
  __stcg(&dst->tcp.a1, v.tcp.a1);
  __stcg(&dst->tcp.a2, v.tcp.a2);
  __stcg(&dst->tcp.a3, v.tcp.a3);
  __stcg(&dst->tcp.a4, v.tcp.a4);
  const float* f = &v.tcpf.sc_hi;
  float* g = &dst->tcpf.sc_hi;
  for (int q = 0; q < 6; ++q) __stcg(g + q, f[q]);
  const float* fd = &v.tdf.dsc_hi;
  float* gd = &dst->tdf.dsc_hi;
  for (int q = 0; q < 6; ++q) __stcg(gd + q, fd[q]);
}
__device__ __forceinline__ void get_pub(ThetaPub& v, const ThetaPub* src, int p) {
  for (int q = 0; q < p; ++q) v.thp[q] = __ldcg(src->thp + q);
  v.lpri_new = __ldcg(&src->lpri_new);
  v.tcp.a0 = __ldcg(&src->tcp.a0);
  v.tcp.a1 = __ldcg(&src->tcp.a1);
  v.tcp.a2 = __ldcg(&src->tcp.a2);
  v.tcp.a3 = __ldcg(&src->tcp.a3);
  v.tcp.a4 = __ldcg(&src->tcp.a4);
  const float* g = &src->tcpf.sc_hi;
  float* f = &v.tcpf.sc_hi;
  for (int q = 0; q < 6; ++q) f[q] = __ldcg(g + q);
  const float* gd = &src->tdf.dsc_hi;
  float* fd = &v.tdf.dsc_hi;
  for (int q = 0; q < 6; ++q) fd[q] = __ldcg(gd + q);
}
// Both proposals of a sweep, word by word over the 32 lanes of a warp (every lane calls):
// pub2_put writes them to slots base and base + 1 and releases seq (each lane fences its own
// stores before the warp meets; then lane 0 releases); pub2_get reads them after the release.
constexpr int kPubU32 = static_cast<int>(sizeof(ThetaPub) / 4);
static_assert(sizeof(ThetaPub) % 8 == 0, "ThetaPub is copied as 32-bit words");
__device__ __forceinline__ void pub2_put(const SweepArgs& a, int base, const ThetaPub* cand, unsigned int seq,
                                         int lane) {
  for (int w = lane; w < 2 * kPubU32; w += 32) {
    const int c = w / kPubU32, o = w - c * kPubU32;
    __stcg(reinterpret_cast<unsigned int*>(pub_slot(a, base + c)) + o,
           reinterpret_cast<const unsigned int*>(cand + c)[o]);
  }
  __threadfence();
  __syncwarp();
  if (lane == 0) st_release_u32(a.bar + 1, seq);
}
__device__ __forceinline__ void pub2_get(const SweepArgs& a, int base, ThetaPub* cand, int lane) {
  (void)ld_acquire_u32(a.bar + 1);  // this lane's loads are ordered after the release it saw
  for (int w = lane; w < 2 * kPubU32; w += 32) {
    const int c = w / kPubU32, o = w - c * kPubU32;
    reinterpret_cast<unsigned int*>(cand + c)[o] =
        __ldcg(reinterpret_cast<const unsigned int*>(pub_slot(a, base + c)) + o);
  }
}
// Block 0: release sequence number seq after writing its slots.
__device__ __forceinline__ void release_pub(const SweepArgs& a, unsigned int seq) {
  __threadfence();
  st_release_u32(a.bar + 1, seq);
}
// Other blocks: wait (bounded) until block 0 has released seq. Returns false if the run failed
// meanwhile or the wait ran out (the run's error word then says why).
__device__ __forceinline__ bool wait_pub(const SweepArgs& a, unsigned int seq) {
  const long long t0 = globaltimer_ns();
  while (ld_acquire_u32(a.bar + 1) < seq) {
    if (ld_volatile_i32(a.err) != 0) return false;
    if (globaltimer_ns() - t0 > a.timeout_ns) {
      atomicCAS(a.err, 0, CUDAHM_ETIMEOUT);
      return false;
    }
    __nanosleep(32);
  }
  return true;
}

template <class M>
__device__ __forceinline__ void propose_theta(const SweepArgs& a, long long s, int p, const double* theta, double* Sth,
                                              double* thp, double& lpri_new, typename M::TC& tcp,
                                              const double* T) {
  for (int q = 0; q < p; ++q) {
    double t = theta[q];
    for (int b = 0; b <= q; ++b) t = fma(Sth[q * p + b], __ldg(a.tab_U + s * p + b), t);
    thp[q] = t;
  }
  lpri_new = M::logprior(thp, a.mc, T);
  tcp = M::consts(thp, a.mc, T);
}

// One lane's part of the theta proposal theta' = theta + S_theta U (U: a row of the tables, staged
// in shared memory: a chain of global loads would dominate), so that
// three lanes share its serial chain: role 0 the log prior, role 1 theta' and the model
// constants (binary64 and binary32 pairs), role 2 (FP32 form) the constants of the step from
// tc_from to theta'. Each role forms theta' itself, with the operations of propose_theta (the
// same bits).
template <class M, bool F32>
__device__ __forceinline__ void propose_part(const SweepArgs& a, const double* U, int p, int role, const double* theta,
                                             const double* Sth, const typename M::TC& tc_from, ThetaPub& o,
                                             const double* T) {
  double thp[kMaxP];
  for (int q = 0; q < p; ++q) {
    double t = theta[q];
    for (int b = 0; b <= q; ++b) t = fma(Sth[q * p + b], U[b], t);
    thp[q] = t;
  }
  if (role == 0) {
    o.lpri_new = M::logprior(thp, a.mc, T);
  } else if (role == 1) {
    for (int q = 0; q < p; ++q) o.thp[q] = thp[q];
    o.tcp = M::consts(thp, a.mc, T);
    o.tcpf = M::consts32(o.tcp);
  } else {
    if constexpr (F32) o.tdf = M::dconsts32(tc_from, M::consts(thp, a.mc, T));
  }
}

// The theta step's log acceptance ratio (Sec. 2.2, with the selection term of Eq. 12 for LF and
// BB1) from a sweep's exact totals: D = sum_i [log f(chi_i; theta') - log f(chi_i; theta)], E =
// etabar(theta'), and the flag counts f (f[0]: some d_i is -inf or <= -2^94, which rejects;
// f[2]: some d_i >= 2^94, which accepts). log alpha = D + nn (c(theta') - c(theta)) + ln pi(theta')
// - ln pi(theta) - nn (ln etabar(theta') - ln etabar(theta)), nn the population's member count.
// Drec is D as binary64 (for the trace), eb_new and logeb_new the new selection integral.
template <class M>
__device__ __forceinline__ void theta_logalpha(const Xacc& D, const Xacc& E, const unsigned int f[4], bool prior_ok,
                                               double nn, const double* theta, const double* thp, double lpri,
                                               double lpri_new, double logeb, const double* T, double& logalpha,
                                               double& Drec, double& eb_new, double& logeb_new) {
  eb_new = 0.0;
  logeb_new = 0.0;
  if (!prior_ok) {
    logalpha = -INFINITY;
    Drec = 0.0;
  } else if (f[0] != 0u) {  // a member off the proposal's support (or d <= -2^94)
    logalpha = -INFINITY;
    Drec = -INFINITY;
  } else if (f[2] != 0u) {  // only huge positive differences remain
    logalpha = INFINITY;
    Drec = INFINITY;
  } else {
    Drec = xacc_to_double(D);
    logalpha = Drec + nn * (M::cterm(thp) - M::cterm(theta)) + lpri_new - lpri;
    if constexpr (M::kRule) {
      eb_new = xacc_to_double(E);
      logeb_new = log_etabar(eb_new, T);
      logalpha -= nn * (logeb_new - logeb);
    }
  }
}

}  // namespace chm
