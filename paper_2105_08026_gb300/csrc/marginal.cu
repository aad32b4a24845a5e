// Latent marginalisation by cubature: the theta-only chain (Sec. 6 proposes it for populations
// whose members have a low-dimensional latent). Each member's latent is integrated out,
//   log p_i(theta) = log int l_i(chi) f(chi;theta) dchi,
// by fixed Gauss-Legendre panels in chi (NN1: one 64-node panel on the integrand's mean
// +- 10 sd; LF: a 64-node panel over the likelihood window [max(ln L_low, ln(F_c/q_i)),
// ln(F_b/q_i)], F_b = Fhat_i + 10 sigma_F, F_c = max(Fhat_i - 10 sigma_F, Fhat_i/2), and, for a
// faint member (F_c = Fhat_i/2), a 32-node panel over [ln L_low, ln(F_c/q_i)] when that is not
// empty; BB1: the same with sigma(F), F_b - Fhat_i = 10 sigma(F_b), the lower end ln l +
// ln(lower/l) and a 128-node tail panel). The theta step is the
// member form's (Sec. 2.2, last paragraph) with D = sum_i [log p_i(theta') - log p_i(theta)]:
// one persistent cooperative launch per chunk of steps, each block integrating a contiguous
// range of members (and its share of the selection rule's outer nodes for LF), an exact
// fixed-point sum over blocks, one bounded grid barrier per step, and the identical decision
// in every block. log p_i at the current theta and at the proposal live in two device arrays
// whose roles swap on acceptance.
#include <cmath>
#include <cstdint>
#include <type_traits>

#include "cudahm.h"
#include "sweep_common.cuh"

namespace chm {

namespace {

// Member integral of the rule above at the theta constants tc. nd: the panels' nodes and
// weights on [-1, 1] (xp[64], wp[64], xt[32], wt[32]). The sum runs relative to the log
// integrand at a point near its peak (the integrand's mean for NN1, the likelihood peak
// clamped into the window for LF); every term is at most ~e^60 times that reference, so the
// scaled sum neither overflows nor loses the peak. Returns -inf when the window leaves the
// support.
template <class M>
__device__ double marg_logp(double y, double aux, const ThetaC& tc, const ModelConsts& mc, const double* T,
                            const double* nd) {
  const double* xp = nd;
  const double* wp = nd + kMargPeak;
  constexpr bool bb1 = std::is_same<M, BB1>::value;
  constexpr int nt = bb1 ? kMargTailBB1 : kMargTail;
  const double* xt = nd + 2 * kMargPeak + (bb1 ? 2 * kMargTail : 0);
  const double* wt = xt + nt;
  if constexpr (std::is_same<M, NN1>::value) {
    // aux = 1/sigma^2, tc.a1 = 1/(2 tau^2): precision of the Gaussian integrand aux + 2 a1
    const double prec = __dadd_rn(aux, __dmul_rn(2.0, tc.a1));
    const double mean = __ddiv_rn(__fma_rn(y, aux, __dmul_rn(__dmul_rn(2.0, tc.a1), tc.a0)), prec);
    const double h = __dmul_rn(kMargK, __dsqrt_rn(__drcp_rn(prec)));
    const double m0 = __dadd_rn(NN1::loglike(mean, 0.0, y, aux, mc), NN1::logf(mean, 0.0, tc));
    double s = 0.0;
#pragma unroll 4
    for (int j = 0; j < kMargPeak; ++j) {
      const double chi = __fma_rn(h, xp[j], mean);
      const double v = __dadd_rn(NN1::loglike(chi, 0.0, y, aux, mc), NN1::logf(chi, 0.0, tc));
      s = __fma_rn(wp[j], exp_tab(__dsub_rn(v, m0), T), s);
    }
    return __dadd_rn(m0, log_tab(__dmul_rn(h, s), T));
  } else {
    // LF, BB1: y = Fhat_i, aux = q_i; the lower end tc.a3 = ln L_low (LF), tc.a4 + ln(lower/l) (BB1)
    double Fb, Fc0;
    if constexpr (bb1) {
      const double den = 1.0 - kMargK * kMargK * mc.alpha * mc.alpha;
      const double ay = mc.alpha * y;
      Fb = (y + kMargK * sqrt(fma(ay, ay, den * mc.s0sq))) / den;
      Fc0 = y - kMargK * sqrt(fma(ay, ay, mc.s0sq));
    } else {
      Fb = __fma_rn(kMargK, mc.sigF, y);
      Fc0 = __fma_rn(-kMargK, mc.sigF, y);
    }
    const bool faint = Fc0 < __dmul_rn(0.5, y);
    const double Fc = faint ? __dmul_rn(0.5, y) : Fc0;
    const double chib = log_tab(__ddiv_rn(Fb, aux), T);
    const double chic = log_tab(__ddiv_rn(Fc, aux), T);
    const double lo = bb1 ? tc.a4 + mc.ln_lower : tc.a3;
    const double a2 = fmax(chic, lo);
    if (!(a2 < chib)) return -INFINITY;
    const double cref = fmin(fmax(log_tab(__ddiv_rn(y, aux), T), a2), chib);
    const double eref = exp_tab(cref, T);
    const double m0 = __dadd_rn(M::loglike(cref, eref, y, aux, mc), M::logf(cref, eref, tc));
    const double c2 = __dmul_rn(0.5, __dadd_rn(a2, chib)), h2 = __dmul_rn(0.5, __dsub_rn(chib, a2));
    double s2 = 0.0;
#pragma unroll 4
    for (int j = 0; j < kMargPeak; ++j) {
      const double chi = __fma_rn(h2, xp[j], c2);
      const double e = exp_tab(chi, T);
      const double v = __dadd_rn(M::loglike(chi, e, y, aux, mc), M::logf(chi, e, tc));
      s2 = __fma_rn(wp[j], exp_tab(__dsub_rn(v, m0), T), s2);
    }
    double s = __dmul_rn(h2, s2);
    if (faint && lo < chic) {
      const double c1 = __dmul_rn(0.5, __dadd_rn(lo, chic)), h1 = __dmul_rn(0.5, __dsub_rn(chic, lo));
      double s1 = 0.0;
#pragma unroll 4
      for (int j = 0; j < nt; ++j) {
        const double chi = __fma_rn(h1, xt[j], c1);
        const double e = exp_tab(chi, T);
        const double v = __dadd_rn(M::loglike(chi, e, y, aux, mc), M::logf(chi, e, tc));
        s1 = __fma_rn(wt[j], exp_tab(__dsub_rn(v, m0), T), s1);
      }
      s = __fma_rn(h1, s1, s);
    }
    return __dadd_rn(m0, log_tab(s, T));
  }
}

// FP32 bulk form of the LF member integral: the same panels, the log integrand at each node in
// binary32 relative to a reference point c_r (the likelihood peak chi* = ln(Fhat/q) clamped into
// the window), written so that nothing cancels: with u = chi - c_r, e1 = expm1(u),
// R = e^{c_r - chi*}, D0 = 1 - R, A = Fhat^2/(2 sigma_F^2) and E_r = e^{c_r - ln L*},
//   log l(chi) - log l(c_r) = A R e1 (2 D0 - R e1),
//   log f(chi) - log f(c_r) = (beta + 1) u - E_r e1.
// The window, c_r, the reference value and the panel geometry are binary64 (per member, a few
// operations: chi*, Fhat/q and the window ends are precomputed once, md32); the nodes' terms are
// binary32, summed with Kahan's compensation (a plain binary32 sum of the 96 terms biased log p_i
// by ~1e-8 in a host emulation), and log p_i = (binary64 reference) + log(sum) in binary64.
__device__ double marg_logp32_lf(long long i, long long n, const double* __restrict__ md, const ThetaC& tc,
                                 const double* T, const float* nd) {
  const double chis = __ldg(md + i), Lhat = __ldg(md + n + i), chib = __ldg(md + 2 * n + i),
               chic = __ldg(md + 3 * n + i), A = __ldg(md + 4 * n + i);
  const bool faint = __ldg(md + 5 * n + i) != 0.0;
  const double lo = tc.a3;
  const double a2 = fmax(chic, lo);
  if (!(a2 < chib)) return -INFINITY;
  const double cref = fmin(fmax(chis, a2), chib);
  double R = 1.0, D0 = 0.0, Eref, m0;
  if (cref == chis) {  // the usual case: the peak lies in the window
    Eref = Lhat * tc.a2;
    m0 = fma(tc.a0, chis - tc.a1, -Eref);
  } else {
    R = exp_tab(cref - chis, T);
    D0 = 1.0 - R;
    Eref = Lhat * R * tc.a2;
    m0 = fma(-A * D0, D0, fma(tc.a0, cref - tc.a1, -Eref));
  }
  const float ARf = static_cast<float>(A * R), Rf = static_cast<float>(R), twoD0 = static_cast<float>(2.0 * D0);
  const float b1 = static_cast<float>(tc.a0), Ef = static_cast<float>(Eref);
  const float* xp = nd;
  const float* wp = nd + kMargPeak;
  const float* xt = nd + 2 * kMargPeak;
  const float* wt = xt + kMargTail;
  const double c2 = 0.5 * (a2 + chib), h2 = 0.5 * (chib - a2);
  const float cf2 = static_cast<float>(c2 - cref), hf2 = static_cast<float>(h2);
  float s2 = 0.0f, k2 = 0.0f;
#pragma unroll 8
  for (int j = 0; j < kMargPeak; ++j) {
    const float u = fmaf(hf2, xp[j], cf2);
    const float e1 = expm1f(u);
    const float dv = fmaf(ARf * e1, fmaf(-Rf, e1, twoD0), fmaf(b1, u, -Ef * e1));
    const float y = __fsub_rn(__fmul_rn(wp[j], __expf(dv)), k2);
    const float t = __fadd_rn(s2, y);
    k2 = __fsub_rn(__fsub_rn(t, s2), y);
    s2 = t;
  }
  double s = h2 * static_cast<double>(s2);
  if (faint && lo < chic) {
    const double c1 = 0.5 * (lo + chic), h1 = 0.5 * (chic - lo);
    const float cf1 = static_cast<float>(c1 - cref), hf1 = static_cast<float>(h1);
    float s1 = 0.0f, k1 = 0.0f;
#pragma unroll 8
    for (int j = 0; j < kMargTail; ++j) {
      const float u = fmaf(hf1, xt[j], cf1);
      const float e1 = expm1f(u);
      const float dv = fmaf(ARf * e1, fmaf(-Rf, e1, twoD0), fmaf(b1, u, -Ef * e1));
      const float y = __fsub_rn(__fmul_rn(wt[j], __expf(dv)), k1);
      const float t = __fadd_rn(s1, y);
      k1 = __fsub_rn(__fsub_rn(t, s1), y);
      s1 = t;
    }
    s = fma(h1, static_cast<double>(s1), s);
  }
  return m0 + log_tab(s, T);
}

// nd: the nodes and weights in binary64, nd32 the same in binary32 (FP32 form)
template <class M, bool F32>
__device__ __forceinline__ double marg_member(const SweepArgs& a, long long i, const ThetaC& tc, const double* T,
                                              const double* nd, const float* nd32) {
  if constexpr (F32 && std::is_same<M, LF>::value) return marg_logp32_lf(i, a.n, a.marg_d32, tc, T, nd32);
  else return marg_logp<M>(__ldg(a.y + i), __ldg(a.aux + i), tc, a.mc, T, nd);
}

template <class M, bool F32>
__global__ void __launch_bounds__(256, 2) marg_kernel(const SweepArgs a) {
  extern __shared__ double s_dyn[];
  __shared__ double s_theta[kMaxP], s_thp[kMaxP], s_Sth[kMaxP * kMaxP];
  __shared__ ThetaC s_tc, s_tcp;
  __shared__ double s_etabar, s_logeb, s_lpri, s_lpri_new;
  __shared__ int s_stop, s_cur;
  __shared__ long long s_rows_written, s_tacc;
  __shared__ BlockRed s_red;

  const int tid = threadIdx.x;
  const int lane = tid & 31, wid = tid >> 5;
  const int p = a.p;
  constexpr bool is_lf = M::kRule;
  const unsigned int nb0 = static_cast<unsigned int>((a.n * blockIdx.x) / gridDim.x);
  const unsigned int nb1 = static_cast<unsigned int>((a.n * (blockIdx.x + 1)) / gridDim.x);
  const bool skip_me = (a.skip_cta == static_cast<int>(blockIdx.x));
  double* s_math = s_dyn;
  double* s_nodes = s_math + kMathWords;
  float* s_nodes32 = reinterpret_cast<float*>(s_nodes + kMargNodeWords);
  for (int q = tid; q < kMathWords; q += blockDim.x) s_math[q] = a.math_tab[q];
  for (int q = tid; q < kMargNodeWords; q += blockDim.x) {
    s_nodes[q] = a.marg_nodes[q];
    s_nodes32[q] = static_cast<float>(a.marg_nodes[q]);
  }
  __syncthreads();  // tables in place before thread 0 uses them

  if (tid == 0) {
    for (int q = 0; q < p; ++q) s_theta[q] = a.chain->theta[q];
    for (int q = 0; q < p * p; ++q) s_Sth[q] = a.chain->S_theta[q];
    s_etabar = a.chain->etabar;
    s_logeb = is_lf ? log_etabar(s_etabar, s_math) : 0.0;
    s_tc = M::consts(s_theta, a.mc, s_math);
    s_lpri = M::logprior(s_theta, a.mc, s_math);
    s_cur = a.chain->mcur;
    s_rows_written = 0;
    s_tacc = 0;
    s_stop = 0;
  }
  __syncthreads();

  for (long long s = 0; s < a.ns; ++s) {
    if (tid == 0) {
      double lp;
      ThetaC tcp;
      propose_theta<M>(a, s, p, s_theta, s_Sth, s_thp, lp, tcp, s_math);
      s_lpri_new = lp;
      s_tcp = tcp;
    }
    __syncthreads();
    const bool prior_ok = (s_lpri_new != -INFINITY);
    Xacc xd, xe;
    xacc_zero(xd);
    xacc_zero(xe);
    XFlags fd = {0u, 0u, 0u}, fe = {0u, 0u, 0u};
    unsigned int neg_big = 0, pos_big = 0;
    if (prior_ok) {
      const ThetaC tcp = s_tcp;
      const double* lpc = a.marg_lp + static_cast<long long>(s_cur) * a.n;
      double* lpn = a.marg_lp + static_cast<long long>(1 - s_cur) * a.n;
      for (unsigned int i = nb0 + tid; i < nb1; i += blockDim.x) {
        const double v = marg_member<M, F32>(a, i, tcp, s_math, s_nodes, s_nodes32);
        lpn[i] = v;
        const double dn = (v == -INFINITY) ? -INFINITY : v - lpc[i];
        if (disnan(dn)) fd.nan++;
        else if (dhuge(dn)) {
          if (dsign(dn)) neg_big++;  // no mass left on the proposal's support
          else pos_big++;
        } else {
          xacc_add_double(xd, dn, fd);
        }
      }
      if constexpr (is_lf) etabar_terms<M>(tcp, a, blockIdx.x, gridDim.x, s_math, xe, fe);
    }
    // block partial: f[0] d_i <= -2^94 (reject), f[1] NaN (error), f[2] d_i >= 2^94
    {
      unsigned int f[4] = {neg_big, fd.nan + fe.nan + fe.big, pos_big, 0u};
      warp_reduce(xd, xe, f);
      if (lane == 0) {
        s_red.d[wid] = xd;
        s_red.e[wid] = xe;
        for (int q = 0; q < 4; ++q) s_red.f[wid][q] = f[q];
      }
      __syncthreads();
      if (wid == 0) {
        const int nw = blockDim.x >> 5;
        Xacc bd, be;
        unsigned int bf[4] = {0u, 0u, 0u, 0u};
        xacc_zero(bd);
        xacc_zero(be);
        if (lane < nw) {
          bd = s_red.d[lane];
          be = s_red.e[lane];
          for (int q = 0; q < 4; ++q) bf[q] = s_red.f[lane][q];
        }
        warp_reduce(bd, be, bf);
        if (lane == 0) {  // into the grid totals of this step (exact limb sums, as in the sweep kernel)
          unsigned long long* acc = a.acc3 + (s % 3) * kAccWords;
          acc_add_limbs(acc, bd);
          acc_add_limbs(acc + 6, be);
          atomicAdd(acc + 12, (static_cast<unsigned long long>(bf[1]) << 32) | bf[0]);
          atomicAdd(acc + 13, (static_cast<unsigned long long>(bf[3]) << 32) | bf[2]);
          // step s + 1 reuses the buffer of step s - 2, which every block read before arriving
          // at barrier s - 1: block 0 clears it before it arrives here
          if (blockIdx.x == 0) {
            unsigned long long* nxt = a.acc3 + ((s + 1) % 3) * kAccWords;
            for (int q = 0; q < kAccWords; ++q) __stcg(nxt + q, 0ull);
          }
        }
      }
    }
    if (!grid_barrier(a.bar, static_cast<unsigned int>(s), a.err, a.timeout_ns, skip_me)) return;
    {
      Xacc D, E;
      unsigned int f[4];
      if (tid == 0) {
        const unsigned long long* acc = a.acc3 + (s % 3) * kAccWords;
        acc_to_xacc(acc, D);
        acc_to_xacc(acc + 6, E);
        const unsigned long long f01 = __ldcg(acc + 12), f23 = __ldcg(acc + 13);
        f[0] = static_cast<unsigned int>(f01);
        f[1] = static_cast<unsigned int>(f01 >> 32);
        f[2] = static_cast<unsigned int>(f23);
        f[3] = static_cast<unsigned int>(f23 >> 32);
        const long long sg = a.trace_off + s;
        if (f[1] != 0u) {
          atomicCAS(a.err, 0, CUDAHM_ENUMERIC);
          s_stop = 1;
        } else {
          double logalpha, Drec, eb_new = 0.0, logeb_new = 0.0;
          if (!prior_ok) {
            logalpha = -INFINITY;
            Drec = 0.0;
          } else if (f[0] != 0u) {
            logalpha = -INFINITY;
            Drec = -INFINITY;
          } else if (f[2] != 0u) {
            logalpha = INFINITY;
            Drec = INFINITY;
          } else {
            Drec = xacc_to_double(D);
            const double nn = static_cast<double>(a.n);
            logalpha = Drec + nn * (M::cterm(s_thp) - M::cterm(s_theta)) + s_lpri_new - s_lpri;
            if (is_lf) {
              eb_new = xacc_to_double(E);
              logeb_new = log_etabar(eb_new, s_math);
              logalpha -= nn * (logeb_new - s_logeb);
            }
          }
          const bool acc = __ldg(a.tab_lnu + s) < logalpha;
          if (blockIdx.x == 0 && sg < a.trace_T) {
            for (int q = 0; q < p; ++q) a.tr_thprop[sg * p + q] = s_thp[q];
            a.tr_D[sg] = Drec;
            a.tr_logalpha[sg] = logalpha;
            a.tr_ut[sg] = __ldg(a.tab_u + s);
            a.tr_tacc[sg] = acc ? 1 : 0;
            a.tr_eb[sg] = eb_new;
          }
          if (acc) {
            for (int q = 0; q < p; ++q) s_theta[q] = s_thp[q];
            s_tc = s_tcp;
            s_lpri = s_lpri_new;
            s_cur = 1 - s_cur;
            if (is_lf) {
              s_etabar = eb_new;
              s_logeb = logeb_new;
            }
            s_tacc++;
          }
          if (a.adapt_theta) {
            const double alpha = (logalpha >= 0.0) ? 1.0 : exp_tab(logalpha, s_math);
            ram_update_theta(p, s_Sth, a.tab_U + s * p, alpha, a.astar_theta, __ldg(a.tab_eta + s));
          }
          const long long post = s - a.burn_left;
          if (post >= 0 && a.thin > 0 && ((a.keep_phase + post + 1) % a.thin) == 0) {
            if (blockIdx.x == 0)
              for (int q = 0; q < p; ++q) a.rows[s_rows_written * p + q] = s_theta[q];
            s_rows_written++;
          }
        }
      }
    }
    __syncthreads();
    if (s_stop) return;
  }
  if (tid == 0 && blockIdx.x == 0) {
    for (int q = 0; q < p; ++q) a.chain->theta[q] = s_theta[q];
    for (int q = 0; q < p * p; ++q) a.chain->S_theta[q] = s_Sth[q];
    a.chain->etabar = s_etabar;
    a.chain->sweeps = a.k0 + a.ns;
    a.chain->theta_acc += s_tacc;
    a.chain->rows = s_rows_written;
    a.chain->mcur = s_cur;
  }
}

// log p_i(theta) of every member at theta (device, p doubles), into out[n].
template <class M, bool F32>
__global__ void marg_eval_kernel(long long n, const double* y, const double* aux, const double* theta,
                                 ModelConsts mc, const double* T, const double* nodes, const double* md32,
                                 double* out) {
  __shared__ double s_math[kMathWords];
  __shared__ double s_nodes[kMargNodeWords];
  __shared__ float s_nodes32[kMargNodeWords];
  __shared__ ThetaC s_tc;
  for (int q = threadIdx.x; q < kMathWords; q += blockDim.x) s_math[q] = T[q];
  for (int q = threadIdx.x; q < kMargNodeWords; q += blockDim.x) {
    s_nodes[q] = nodes[q];
    s_nodes32[q] = static_cast<float>(nodes[q]);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double th[kMaxP];
    for (int q = 0; q < 3; ++q) th[q] = (q < 2 || M::kRule) ? theta[q] : 0.0;
    s_tc = M::consts(th, mc, s_math);
  }
  __syncthreads();
  const long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if constexpr (F32 && std::is_same<M, LF>::value) out[i] = marg_logp32_lf(i, n, md32, s_tc, s_math, s_nodes32);
  else out[i] = marg_logp<M>(y[i], aux[i], s_tc, mc, s_math, s_nodes);
}

// Per-member window data of the FP32 LF form (theta-independent): ln(Fhat/q), Fhat/q, the window
// ends ln(F_b/q), ln(F_c/q) as the binary64 form computes them, Fhat^2/(2 sigma_F^2).
__global__ void marg_data32_kernel(long long n, const double* y, const double* aux, ModelConsts mc,
                                   const double* T, double* md) {
  __shared__ double s_math[kMathWords];
  for (int q = threadIdx.x; q < kMathWords; q += blockDim.x) s_math[q] = T[q];
  __syncthreads();
  const long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double F = y[i], q = aux[i];
  const double Fb = __fma_rn(kMargK, mc.sigF, F);
  const double Fc0 = __fma_rn(-kMargK, mc.sigF, F);
  const bool faint = Fc0 < __dmul_rn(0.5, F);
  const double Fc = faint ? __dmul_rn(0.5, F) : Fc0;
  md[i] = log_tab(__ddiv_rn(F, q), s_math);
  md[n + i] = F / q;
  md[2 * n + i] = log_tab(__ddiv_rn(Fb, q), s_math);
  md[3 * n + i] = log_tab(__ddiv_rn(Fc, q), s_math);
  md[4 * n + i] = F * F * mc.inv2sig2;
  md[5 * n + i] = faint ? 1.0 : 0.0;
}

size_t marg_smem() { return sizeof(double) * (kMathWords + kMargNodeWords) + sizeof(float) * kMargNodeWords; }

}  // namespace

size_t marg_smem_bytes(int, int) { return marg_smem(); }

static const void* marg_fn(int model, bool f32) {
  if (model == CUDAHM_LF)
    return f32 ? reinterpret_cast<const void*>(&marg_kernel<LF, true>) : reinterpret_cast<const void*>(&marg_kernel<LF, false>);
  if (model == CUDAHM_BB1) return reinterpret_cast<const void*>(&marg_kernel<BB1, false>);  // FP64 only
  return reinterpret_cast<const void*>(&marg_kernel<NN1, false>);  // NN1: binary64 in both forms
}

cudaError_t marg_occupancy(int model, bool f32, int block, int smem_bytes, int* blocks_per_sm) {
  const void* fn = marg_fn(model, f32);
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, fn, block, smem_bytes);
}

cudaError_t launch_marg(const SweepArgs& a, int grid, int block, cudaStream_t st) {
  const size_t smem = marg_smem_bytes(a.model, a.rows_smem);
  void* args[] = {const_cast<SweepArgs*>(&a)};
  const void* fn = marg_fn(a.model, a.f32 != 0);
  return cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(block), args, smem, st);
}

cudaError_t launch_marg_eval(int model, bool f32, long long n, const double* y, const double* aux,
                             const double* theta_dev, const ModelConsts& mc, const double* math_tab,
                             const double* nodes, const double* md32, double* out, cudaStream_t st) {
  const int blk = 256;
  const unsigned int grid = static_cast<unsigned int>((n + blk - 1) / blk);
  if (model == CUDAHM_LF && f32)
    marg_eval_kernel<LF, true><<<grid, blk, 0, st>>>(n, y, aux, theta_dev, mc, math_tab, nodes, md32, out);
  else if (model == CUDAHM_LF)
    marg_eval_kernel<LF, false><<<grid, blk, 0, st>>>(n, y, aux, theta_dev, mc, math_tab, nodes, md32, out);
  else if (model == CUDAHM_BB1)
    marg_eval_kernel<BB1, false><<<grid, blk, 0, st>>>(n, y, aux, theta_dev, mc, math_tab, nodes, md32, out);
  else if (model == CUDAHM_NN1)
    marg_eval_kernel<NN1, false><<<grid, blk, 0, st>>>(n, y, aux, theta_dev, mc, math_tab, nodes, md32, out);
  else
    return cudaErrorInvalidValue;
  return cudaGetLastError();
}

cudaError_t launch_marg_data32(long long n, const double* y, const double* aux, const ModelConsts& mc,
                               const double* math_tab, double* md32, cudaStream_t st) {
  const int blk = 256;
  marg_data32_kernel<<<static_cast<unsigned int>((n + blk - 1) / blk), blk, 0, st>>>(n, y, aux, mc, math_tab, md32);
  return cudaGetLastError();
}

// Nodes and weights of the panels on [-1, 1]: xp[64], wp[64], xt[32], wt[32], xb[128], wb[128].
cudaError_t launch_marg_nodes(double* nodes, cudaStream_t st) {
  cudaError_t e = launch_gauss_legendre(kMargPeak, nodes, nodes + kMargPeak, st);
  if (e != cudaSuccess) return e;
  double* t = nodes + 2 * kMargPeak;
  e = launch_gauss_legendre(kMargTail, t, t + kMargTail, st);
  if (e != cudaSuccess) return e;
  return launch_gauss_legendre(kMargTailBB1, t + 2 * kMargTail, t + 2 * kMargTail + kMargTailBB1, st);
}

}  // namespace chm
