/*
 * CUDAHM oracle: a plain, slow, single-threaded FP64 CPU implementation of the
 * Metropolis-within-Gibbs (MWG) sampler for single-plate hierarchical models of
 * arXiv:2105.08026 (Szalai-Gindl et al., "GPU-Accelerated Hierarchical Bayesian
 * Inference with Application to Modeling Cosmic Populations: CUDAHM").
 *
 * TEST INFRASTRUCTURE ONLY. This file is the reference the CUDA path is checked
 * against. Only the test suite, the smoke check and the benchmark's CPU-baseline
 * leg may load it. It shares no code, header, table or constant generator with
 * the CUDA library, and the CUDA library never calls it.
 *
 * Build: gcc -O2 -ffp-contract=off -fPIC -shared (no -ffast-math), so that every
 * floating-point operation is a separately rounded IEEE-754 binary64 operation.
 *
 * What it follows (paper sections / equations):
 *   - Joint density pi(theta) prod_i f(psi_i;theta) l_i(psi_i): Sec. 2.1, eq. (joint-2level).
 *   - MWG order: every member update given theta first (eq. psi_sampling), then the
 *     theta update given all members (eq. theta_sampling): Sec. 2.1.
 *   - Robust adaptive Metropolis (RAM) member update (Sec. 2.2, after Vihola 2012):
 *     Y = X + S U, U ~ N(0, I); accept with prob. min(1, pi(Y)/pi(X));
 *     S_n S_n^T = S_{n-1}(I + eta_n (alpha_n - alpha_*) U U^T/|U|^2) S_{n-1}^T,
 *     alpha_* = 0.4, eta_n = n^(-2/3), S_1 = I.
 *   - theta update: Metropolis-Hastings with the sum over members of
 *     log f(chi_i;theta') - log f(chi_i;theta) (Sec. 2.2, last paragraph).
 *   - Thinned latent point-process likelihood with the selection integral in the
 *     denominator of the effective density (Sec. 4.2, eqs. rho-mlike and epdf),
 *     detection efficiency eta(F) = Phi((F - F_th)/sigma) (Sec. 5.2, eq. key).
 *
 * Readings where the paper is silent (each is listed in the design notes):
 *   R1 RAM index: sweep k = 1, 2, ... uses eta = (k+1)^(-gamma) (S_1 given, first
 *      update produces S_2).
 *   R2 adaptation runs through burn-in and sampling alike.
 *   R3 theta proposal: RAM on theta with the same eta and its own target acceptance,
 *      each step's update applied one sweep late: the proposal of sweep k + 1 uses the
 *      factor updated with the steps up to k - 1 (S_{k+1} = RAM(S_k, U_{k-1}, alpha_{k-1},
 *      eta_{k-1})), so that it can be formed before sweep k's accept decision (the marginal
 *      form keeps the undelayed update); adapt_theta = 0 gives plain random-walk MH with
 *      fixed S_theta.
 *   R4 accept iff ln u < Delta (strict), alpha = exp(min(0, Delta)), alpha = 0 off support.
 *   R5 random numbers: Philox4x32-10 (Salmon et al., SC'11), key = (seed lo, seed hi),
 *      counter = (block j, stream s, object i, sweep k); uniform u = (2m+1) 2^-53 with
 *      m the top 52 bits of (w_a:w_b); Box-Muller pairs c = sqrt(-2 ln u_a) cos(2 pi u_b),
 *      s = sqrt(-2 ln u_a) sin(2 pi u_b) from the words (w0,w1), (w2,w3) of a block.
 *      Member draws (stream 0): the two normals of one Box-Muller pair serve two consecutive
 *      sweeps. For the odd sweep k_o = 2m-1 and the even sweep k_o + 1, component a of U
 *      comes from block (j = a, stream 0, member i, sweep k_o): its cosine for sweep k_o,
 *      its sine for sweep k_o + 1. The accept uniform of sweep k is the first uniform of
 *      block (d, 0, i, k). Theta draws (stream 1, index 0): block j gives normals 2j, 2j+1
 *      of sweep k; the accept uniform is the first uniform of block ceil(p/2).
 *   R6 luminosity model in chi = ln L (Schechter form truncated at L_low), the
 *      normaliser of f cancels against the normalised selection integral, so the
 *      theta step uses the unnormalised integrand (see lf_* below). The same holds for the
 *      paper's BB1 model with its flux-dependent measurement error (see bb1_* below).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_NN1 0
#define ORC_MVN3 1
#define ORC_LF 2
#define ORC_BB1 3
#define ORC_NN3 4

/* ------------------------------------------------------------------------- */
/* R5: Philox4x32-10 block cipher (Salmon, Moraes, Dror, Shaw, SC'11).         */
/* Each of the 10 rounds multiplies two 32-bit lanes by the published          */
/* multipliers, mixes the high halves with the other lanes and the round key,  */
/* and bumps the key by the published Weyl constants.                          */
/* ------------------------------------------------------------------------- */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)x0;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)x2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t y0 = hi1 ^ x1 ^ k0;
    uint32_t y1 = lo1;
    uint32_t y2 = hi0 ^ x3 ^ k1;
    uint32_t y3 = lo0;
    x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* R5: uniform on (0,1) from two words; exact: (2m+1) has at most 53 bits. */
double orc_uniform(uint32_t wa, uint32_t wb) {
  uint64_t x = ((uint64_t)wa << 32) | (uint64_t)wb;
  uint64_t m = x >> 12;
  return ((double)m + 0.5) * 0x1p-52;
}

static void block_words(uint64_t seed, uint32_t j, uint32_t s, uint32_t i, uint32_t k, uint32_t w[4]) {
  uint32_t ctr[4] = {j, s, i, k};
  uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
  orc_philox4x32_10(ctr, key, w);
}

/* R5: member draw of sweep k: d standard normals (shared Box-Muller pairs) and the accept uniform. */
void orc_draw_member(uint64_t seed, uint32_t i, uint32_t k, int d, double* z, double* u_accept) {
  const double two_pi = 6.283185307179586476925286766559;
  uint32_t k_odd = (k & 1u) ? k : k - 1u;
  for (int a = 0; a < d; ++a) {
    uint32_t w[4];
    block_words(seed, (uint32_t)a, 0u, i, k_odd, w);
    double ua = orc_uniform(w[0], w[1]);
    double ub = orc_uniform(w[2], w[3]);
    double rad = sqrt(-2.0 * log(ua));
    z[a] = (k & 1u) ? rad * cos(two_pi * ub) : rad * sin(two_pi * ub);
  }
  uint32_t w[4];
  block_words(seed, (uint32_t)d, 0u, i, k, w);
  *u_accept = orc_uniform(w[0], w[1]);
}

/* R5: theta draw: d standard normals and the accept uniform (stream s, index i, sweep k). */
void orc_draw(uint64_t seed, uint32_t s, uint32_t i, uint32_t k, int d, double* z, double* u_accept) {
  const double two_pi = 6.283185307179586476925286766559;
  int nblk = (d + 1) / 2;
  for (int j = 0; j < nblk; ++j) {
    uint32_t w[4];
    block_words(seed, (uint32_t)j, s, i, k, w);
    double ua = orc_uniform(w[0], w[1]);
    double ub = orc_uniform(w[2], w[3]);
    double rad = sqrt(-2.0 * log(ua));
    z[2 * j] = rad * cos(two_pi * ub);
    if (2 * j + 1 < d) z[2 * j + 1] = rad * sin(two_pi * ub);
  }
  uint32_t w[4];
  block_words(seed, (uint32_t)nblk, s, i, k, w);
  *u_accept = orc_uniform(w[0], w[1]);
}

/* ------------------------------------------------------------------------- */
/* Neumaier compensated summation (Neumaier 1974), used for every long sum.    */
/* ------------------------------------------------------------------------- */
typedef struct { double s, c; } ksum;
static void ks_add(ksum* a, double v) {
  double t = a->s + v;
  if (fabs(a->s) >= fabs(v)) a->c += (a->s - t) + v;
  else a->c += (v - t) + a->s;
  a->s = t;
}
static double ks_val(const ksum* a) { return a->s + a->c; }

double orc_neumaier_sum(const double* v, int64_t n) {
  ksum a = {0.0, 0.0};
  for (int64_t i = 0; i < n; ++i) ks_add(&a, v[i]);
  return ks_val(&a);
}

/* ------------------------------------------------------------------------- */
/* Dense helpers for the RAM factor update (row-major d x d).                   */
/* ------------------------------------------------------------------------- */
/* Cholesky factor of a symmetric positive-definite matrix (lower, row-major).
 * Returns 0 on success, -1 if a pivot is not positive. */
int orc_cholesky(int d, const double* A, double* Lout) {
  double L[81];
  memset(L, 0, sizeof(L));
  for (int j = 0; j < d; ++j) {
    double s = A[j * d + j];
    for (int k = 0; k < j; ++k) s -= L[j * d + k] * L[j * d + k];
    if (!(s > 0.0)) return -1;
    L[j * d + j] = sqrt(s);
    for (int i = j + 1; i < d; ++i) {
      double t = A[i * d + j];
      for (int k = 0; k < j; ++k) t -= L[i * d + k] * L[j * d + k];
      L[i * d + j] = t / L[j * d + j];
    }
  }
  memcpy(Lout, L, sizeof(double) * d * d);
  return 0;
}

/* RAM factor update, Sec. 2.2 step 3: form M = S (I + c U U^T/|U|^2) S^T with
 * c = eta (alpha - alpha_*), then S <- chol(M). Written exactly as stated: the
 * right-hand side is built explicitly, then factored. S is d x d lower, row-major. */
int orc_ram_update(int d, double* S, const double* U, double alpha, double alpha_star, double eta) {
  double c = eta * (alpha - alpha_star);
  double uu = 0.0;
  for (int j = 0; j < d; ++j) uu += U[j] * U[j];
  double inner[81], tmp[81], M[81];
  for (int a = 0; a < d; ++a)
    for (int b = 0; b < d; ++b)
      inner[a * d + b] = (a == b ? 1.0 : 0.0) + c * U[a] * U[b] / uu;
  for (int a = 0; a < d; ++a)
    for (int b = 0; b < d; ++b) {
      double t = 0.0;
      for (int k = 0; k < d; ++k) t += S[a * d + k] * inner[k * d + b];
      tmp[a * d + b] = t;
    }
  for (int a = 0; a < d; ++a)
    for (int b = 0; b < d; ++b) {
      double t = 0.0;
      for (int k = 0; k < d; ++k) t += tmp[a * d + k] * S[b * d + k];
      M[a * d + b] = t;
    }
  /* symmetrise against rounding before factoring */
  for (int a = 0; a < d; ++a)
    for (int b = 0; b < a; ++b) {
      double m = 0.5 * (M[a * d + b] + M[b * d + a]);
      M[a * d + b] = m; M[b * d + a] = m;
    }
  return orc_cholesky(d, M, S);
}

/* ------------------------------------------------------------------------- */
/* Gauss-Legendre nodes and weights on [-1,1]: Newton's method on P_n, with    */
/* P_n and P_n' from the three-term recurrence; w = 2/((1-x^2) P_n'(x)^2).     */
/* ------------------------------------------------------------------------- */
void orc_gauss_legendre(int n, double* x, double* w) {
  const double pi = 3.14159265358979323846264338328;
  for (int i = 0; i < (n + 1) / 2; ++i) {
    double z = cos(pi * (i + 0.75) / (n + 0.5));
    double dp = 0.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int m = 2; m <= n; ++m) {
        double p2 = ((2.0 * m - 1.0) * z * p1 - (m - 1.0) * p0) / m;
        p0 = p1; p1 = p2;
      }
      if (n == 1) { p0 = 1.0; p1 = z; }
      dp = n * (z * p1 - p0) / ((z - 1.0) * (z + 1.0));
      double dz = p1 / dp;
      z -= dz;
      if (fabs(dz) < 1e-17) break;
    }
    /* final derivative at the converged node */
    {
      double p0 = 1.0, p1 = z;
      for (int m = 2; m <= n; ++m) {
        double p2 = ((2.0 * m - 1.0) * z * p1 - (m - 1.0) * p0) / m;
        p0 = p1; p1 = p2;
      }
      if (n == 1) { p0 = 1.0; p1 = z; }
      dp = n * (z * p1 - p0);
    }
    /* w = 2/((1-z^2) P_n'(z)^2) with P_n'(z) = n (z P_n - P_{n-1})/(z^2 - 1); 1 - z^2 is
       formed as (1-z)(1+z) to avoid cancellation near the ends */
    double omz2 = (1.0 - z) * (1.0 + z);
    double wi = 2.0 * omz2 / (dp * dp);
    x[i] = -z; w[i] = wi;            /* ascending order */
    x[n - 1 - i] = z; w[n - 1 - i] = wi;
  }
  if (n % 2 == 1) x[n / 2] = 0.0;
}

/* ------------------------------------------------------------------------- */
/* Models. lp_i(chi;theta) = log l_i(chi) + log f_obj(chi;theta); c(theta) holds */
/* the theta-only part of log f, added N times in the theta step.               */
/* ------------------------------------------------------------------------- */

/* Normal-normal, d = 1 (Sec. 3 with one characteristic; theta = (mu, ln tau)).
 * data y_i, sigma_i. log l_i = -(y_i - chi)^2/(2 sigma_i^2). */
static double nn1_loglike(double chi, double y, double sig) {
  double r = y - chi;
  return -(r * r) / (2.0 * sig * sig);
}
static double nn1_logf_obj(double chi, const double* th) {
  double tau = exp(th[1]);
  double r = chi - th[0];
  return -(r * r) / (2.0 * tau * tau);
}
static double nn1_c(const double* th) { return -th[1]; }
/* flat in mu and ln tau; ln tau truncated to [lo, hi] to make the posterior proper */
static double nn1_logprior(const double* th, const double* consts) {
  if (!(th[1] >= consts[0] && th[1] <= consts[1])) return -INFINITY;
  return 0.0;
}

/* Luminosity function (Sec. 4-5), latent chi = ln L, Schechter-form population
 * truncated below at L_low, theta = (beta, ln L*, ln L_low).
 * g(L) = (L/L*)^beta exp(-L/L*)/L*; with the Jacobian e^chi of the ln L coordinate,
 * log f_obj = (beta+1)(chi - ln L*) - exp(chi - ln L*), support chi > ln L_low.
 * Member likelihood (Gaussian in flux, Sec. 5.2): log l_i = -(Fhat_i - e^chi q_i)^2/(2 sigma_F^2),
 * q_i = 1/(4 pi r_i^2) (inverse-square law, Sec. 4.1, eq. fluxPDF).
 * consts: [0] sigma_F, [1] F_th, [2] r_max, [3] n_L nodes, [4] n_r nodes, [5] ln(upper/L*). */
static double lf_q(double r) { return 1.0 / (4.0 * 3.14159265358979323846264338328 * r * r); }
static double lf_loglike(double chi, double fhat, double r, const double* consts) {
  double res = fhat - exp(chi) * lf_q(r);
  return -(res * res) / (2.0 * consts[0] * consts[0]);
}
static double lf_logf_obj(double chi, const double* th) {
  if (!(chi > th[2])) return -INFINITY;
  double x = chi - th[1];
  return (th[0] + 1.0) * x - exp(x);
}
/* Prior: truncated Cauchy in beta on (-2, 0) (Sec. 5.1), flat in ln L* (log-flat L*),
 * flat in L_low -> Jacobian L_low in ln L_low, and L_low < L*. */
static double lf_logprior(const double* th) {
  if (!(th[0] > -2.0 && th[0] < 0.0)) return -INFINITY;
  if (!(th[2] < th[1])) return -INFINITY;
  return -log(1.0 + th[0] * th[0]) + th[2];
}

/* Standard normal CDF, Phi(x) = erfc(-x/sqrt 2)/2 (Sec. 5.2, eq. key). */
static double phi_cdf(double x) { return 0.5 * erfc(-x * 0.70710678118654752440084436210); }

/* Selection integral with the unnormalised population (eq. epdf denominator, h(r) ~ r^2 on
 * [0, r_max] normalised, eta(F) = Phi((F - F_th)/sigma_F)):
 *   etabar(theta) = int_{L_low}^{inf} g(L) H(L) dL,
 *   H(L) = int_0^{r_max} (3 r^2/r_max^3) Phi((L q(r) - F_th)/sigma_F) dr.
 * Rule: Gauss-Legendre with n_L nodes in t = ln L on [ln L_low, ln L* + ln(upper/L*)]
 * (integrand g(e^t) e^t H(e^t)) and n_r nodes in r on [0, r_max]. */
typedef struct {
  int nL, nr;
  double *xL, *wL, *xr, *wr;
} gl_rule;

static void gl_rule_init(gl_rule* R, int nL, int nr) {
  R->nL = nL; R->nr = nr;
  R->xL = (double*)malloc(sizeof(double) * nL); R->wL = (double*)malloc(sizeof(double) * nL);
  R->xr = (double*)malloc(sizeof(double) * nr); R->wr = (double*)malloc(sizeof(double) * nr);
  orc_gauss_legendre(nL, R->xL, R->wL);
  orc_gauss_legendre(nr, R->xr, R->wr);
}
static void gl_rule_free(gl_rule* R) { free(R->xL); free(R->wL); free(R->xr); free(R->wr); }

static double lf_H(double L, const gl_rule* R, const double* consts) {
  double sigF = consts[0], Fth = consts[1], rmax = consts[2];
  ksum h = {0.0, 0.0};
  for (int k = 0; k < R->nr; ++k) {
    double r = 0.5 * rmax * (R->xr[k] + 1.0);
    double wk = 0.5 * rmax * R->wr[k] * 3.0 * r * r / (rmax * rmax * rmax);
    double F = L * lf_q(r);
    ks_add(&h, wk * phi_cdf((F - Fth) / sigF));
  }
  return ks_val(&h);
}

static double lf_etabar_rule(const double* th, const gl_rule* R, const double* consts) {
  double a = th[2], b = th[1] + consts[5];
  double half = 0.5 * (b - a), mid = 0.5 * (b + a);
  ksum s = {0.0, 0.0};
  for (int j = 0; j < R->nL; ++j) {
    double t = half * R->xL[j] + mid;
    double x = t - th[1];
    double gl = exp((th[0] + 1.0) * x - exp(x)); /* g(e^t) e^t */
    ks_add(&s, half * R->wL[j] * gl * lf_H(exp(t), R, consts));
  }
  return ks_val(&s);
}

double orc_lf_etabar(const double* th, const double* consts) {
  gl_rule R;
  gl_rule_init(&R, (int)consts[3], (int)consts[4]);
  double v = lf_etabar_rule(th, &R, consts);
  gl_rule_free(&R);
  return v;
}

/* The same rule built once, for a caller that evaluates etabar(theta) every sweep (the all-cores
 * timing driver): orc_lf_rule_etabar(R, th) equals orc_lf_etabar(th) bit for bit. */
void* orc_lf_rule_new(const double* consts) {
  gl_rule* R = (gl_rule*)malloc(sizeof(gl_rule));
  if (R) gl_rule_init(R, (int)consts[3], (int)consts[4]);
  return R;
}
double orc_lf_rule_etabar(void* R, const double* th, const double* consts) {
  return lf_etabar_rule(th, (gl_rule*)R, consts);
}
void orc_lf_rule_free(void* R) {
  if (!R) return;
  gl_rule_free((gl_rule*)R);
  free(R);
}

/* Detection efficiency eta(F) = Phi((F - F_th)/sigma_F) (Sec. 5.2, eq. key). */
double orc_lf_detection(double F, const double* consts) { return phi_cdf((F - consts[1]) / consts[0]); }

double orc_lf_H(double L, const double* consts) {
  gl_rule R;
  gl_rule_init(&R, (int)consts[3], (int)consts[4]);
  double v = lf_H(L, &R, consts);
  gl_rule_free(&R);
  return v;
}

/* ------------------------------------------------------------------------- */
/* BB1 luminosity function (Sec. 5.1, App. B eq. lumPDF), the paper's simulation model.    */
/* Latent chi = ln L, theta = (beta, ln l, ln u). Unnormalised population                 */
/*   g(L) = (1 - e^{-L/l}) (L/u)^beta e^{-L/u};                                          */
/* the normaliser C(beta,u,l)/u (App. B eq. normLumPDF) depends on theta only and cancels  */
/* against the normalised selection integral exactly as for the Schechter model (R6), so  */
/* the theta step uses g and the selection integral of g. With the Jacobian e^chi:         */
/*   log f_obj = ln(1 - e^{-L/l}) + beta (chi - ln u) - L/u + chi,  L = e^chi (all chi).   */
/* Measurement (Sec. 5.2, eq. sig-F): sigma(F)^2 = sigma0^2 + (alpha F)^2, and the member  */
/* likelihood is the sampling density of Fhat_i as a function of F (the g(n_obs;F) form):  */
/*   log l_i = -ln sigma(F) - (Fhat_i - F)^2/(2 sigma(F)^2),  F = e^chi q_i.               */
/* Detection (eq. Fth, eq. key): F_th = nu sigma0/sqrt(1 - alpha^2),                      */
/*   eta(F) = Phi((F - F_th)/sigma(F)).                                                    */
/* Prior (Sec. 5.1): truncated Cauchy in beta on (-2, 0), log-flat in u, flat in l with    */
/* l < u; in (beta, ln l, ln u): -ln(1 + beta^2) + ln l.                                   */
/* consts: [0] sigma0, [1] alpha, [2] nu, [3] r_max, [4] n_L, [5] n_r, [6] ln(upper/u),    */
/* [7] ln(lower/l) (the outer rule runs over t = ln L in [ln l + [7], ln u + [6]]).        */
/* ------------------------------------------------------------------------- */
double orc_bb1_threshold(double sigma0, double alpha, double nu) { return nu * sigma0 / sqrt(1.0 - alpha * alpha); }

static double bb1_sigma2(double F, const double* consts) {
  return consts[0] * consts[0] + (consts[1] * F) * (consts[1] * F);
}
/* ln(1 - e^{-x}) for x > 0 (Maechler's two branches: accurate for small and large x) */
static double log1mexp(double x) {
  return (x <= 0.69314718055994530942) ? log(-expm1(-x)) : log1p(-exp(-x));
}
static double bb1_logf_obj(double chi, const double* th) {
  double L = exp(chi);
  double lg = log1mexp(L / exp(th[1]));
  if (lg == -INFINITY) return -INFINITY;
  return lg + th[0] * (chi - th[2]) - L / exp(th[2]) + chi;
}
static double bb1_loglike(double chi, double fhat, double r, const double* consts) {
  double F = exp(chi) * lf_q(r);
  double s2 = bb1_sigma2(F, consts);
  double res = fhat - F;
  return -0.5 * log(s2) - (res * res) / (2.0 * s2);
}
static double bb1_logprior(const double* th) {
  if (!(th[0] > -2.0 && th[0] < 0.0)) return -INFINITY;
  if (!(th[1] < th[2])) return -INFINITY;
  return -log(1.0 + th[0] * th[0]) + th[1];
}
double orc_bb1_detection(double F, const double* consts) {
  double Fth = orc_bb1_threshold(consts[0], consts[1], consts[2]);
  return phi_cdf((F - Fth) / sqrt(bb1_sigma2(F, consts)));
}
static double bb1_H(double L, const gl_rule* R, const double* consts) {
  double rmax = consts[3];
  ksum h = {0.0, 0.0};
  for (int k = 0; k < R->nr; ++k) {
    double r = 0.5 * rmax * (R->xr[k] + 1.0);
    double wk = 0.5 * rmax * R->wr[k] * 3.0 * r * r / (rmax * rmax * rmax);
    ks_add(&h, wk * orc_bb1_detection(L * lf_q(r), consts));
  }
  return ks_val(&h);
}
/* etabar(theta) = int g(L) H(L) dL: n_L-node rule in t = ln L on [ln l + consts[7],
 * ln u + consts[6]] (integrand g(e^t) e^t H(e^t)) times the n_r-node rule of H in r. */
static double bb1_etabar_rule(const double* th, const gl_rule* R, const double* consts) {
  double a = th[1] + consts[7], b = th[2] + consts[6];
  double half = 0.5 * (b - a), mid = 0.5 * (b + a);
  ksum s = {0.0, 0.0};
  for (int j = 0; j < R->nL; ++j) {
    double t = half * R->xL[j] + mid;
    double L = exp(t);
    double gl = exp(log1mexp(L / exp(th[1])) + th[0] * (t - th[2]) - L / exp(th[2]) + t); /* g(e^t) e^t */
    ks_add(&s, half * R->wL[j] * gl * bb1_H(L, R, consts));
  }
  return ks_val(&s);
}
double orc_bb1_etabar(const double* th, const double* consts) {
  gl_rule R;
  gl_rule_init(&R, (int)consts[4], (int)consts[5]);
  double v = bb1_etabar_rule(th, &R, consts);
  gl_rule_free(&R);
  return v;
}
double orc_bb1_H(double L, const double* consts) {
  gl_rule R;
  gl_rule_init(&R, (int)consts[4], (int)consts[5]);
  double v = bb1_H(L, &R, consts);
  gl_rule_free(&R);
  return v;
}

/* Multivariate normal, d = 3 (Sec. 3 with C_pop unknown): theta = (mu[3], lower-triangular
 * Cholesky factor L_C of C_pop packed row-major (L11, L21, L22, L31, L32, L33) with the
 * diagonal entries stored as logs). log f_obj = -|L_C^{-1}(chi - mu)|^2/2,
 * c(theta) = -sum ln L_C,jj; data y_i[3], s_i[3]: log l_i = -sum (y_ij - chi_j)^2/(2 s_ij^2). */
static void mvn3_unpack(const double* th, double Lc[9]) {
  Lc[0] = exp(th[3]); Lc[1] = 0.0; Lc[2] = 0.0;
  Lc[3] = th[4]; Lc[4] = exp(th[5]); Lc[5] = 0.0;
  Lc[6] = th[6]; Lc[7] = th[7]; Lc[8] = exp(th[8]);
}
static double mvn3_logf_obj(const double* chi, const double* th) {
  double Lc[9];
  mvn3_unpack(th, Lc);
  double r[3] = {chi[0] - th[0], chi[1] - th[1], chi[2] - th[2]};
  double z0 = r[0] / Lc[0];
  double z1 = (r[1] - Lc[3] * z0) / Lc[4];
  double z2 = (r[2] - Lc[6] * z0 - Lc[7] * z1) / Lc[8];
  return -0.5 * (z0 * z0 + z1 * z1 + z2 * z2);
}
static double mvn3_c(const double* th) { return -(th[3] + th[5] + th[8]); }
static double mvn3_loglike(const double* chi, const double* y, const double* s) {
  double acc = 0.0;
  for (int j = 0; j < 3; ++j) {
    double r = y[j] - chi[j];
    acc += -(r * r) / (2.0 * s[j] * s[j]);
  }
  return acc;
}

/* Normal-normal benchmark, d = 3 (Sec. 3): C_pop known, theta = mu (flat prior). consts =
 * the lower triangle of C_pop packed row-major (C11, C21, C22, C31, C32, C33). log f_obj =
 * -(chi - mu)^T C_pop^{-1} (chi - mu)/2 through the Cholesky factor L of C_pop (L L^T = C_pop)
 * and a forward substitution; ln det C_pop is a constant, so c(theta) = 0. */
static void nn3_factor(const double* C, double Lc[9]) {
  double A[9] = {C[0], C[1], C[3], C[1], C[2], C[4], C[3], C[4], C[5]};
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b <= a; ++b) {
      double v = A[3 * a + b];
      for (int k = 0; k < b; ++k) v -= Lc[3 * a + k] * Lc[3 * b + k];
      Lc[3 * a + b] = (a == b) ? sqrt(v) : v / Lc[3 * b + b];
    }
  Lc[1] = Lc[2] = Lc[5] = 0.0;
}
static double nn3_logf_obj(const double* chi, const double* th, const double* C) {
  double Lc[9];
  nn3_factor(C, Lc);
  double r[3] = {chi[0] - th[0], chi[1] - th[1], chi[2] - th[2]};
  double z0 = r[0] / Lc[0];
  double z1 = (r[1] - Lc[3] * z0) / Lc[4];
  double z2 = (r[2] - Lc[6] * z0 - Lc[7] * z1) / Lc[8];
  return -0.5 * (z0 * z0 + z1 * z1 + z2 * z2);
}

/* ------------------------------------------------------------------------- */
/* Problem dispatch                                                            */
/* ------------------------------------------------------------------------- */
typedef struct {
  int model, d, p;
  int64_t n;
  const double* y;    /* NN1: y[n]; LF: Fhat[n]; MVN3, NN3: y[n*3] */
  const double* aux;  /* NN1: sigma[n]; LF: r[n]; MVN3, NN3: s[n*3] */
  const double* consts;
  gl_rule rule;       /* LF only */
} problem;

static double logf_obj(const problem* P, const double* chi, const double* th) {
  switch (P->model) {
    case ORC_NN1: return nn1_logf_obj(chi[0], th);
    case ORC_LF: return lf_logf_obj(chi[0], th);
    case ORC_BB1: return bb1_logf_obj(chi[0], th);
    case ORC_NN3: return nn3_logf_obj(chi, th, P->consts);
    default: return mvn3_logf_obj(chi, th);
  }
}
static double loglike(const problem* P, int64_t i, const double* chi) {
  switch (P->model) {
    case ORC_NN1: return nn1_loglike(chi[0], P->y[i], P->aux[i]);
    case ORC_LF: return lf_loglike(chi[0], P->y[i], P->aux[i], P->consts);
    case ORC_BB1: return bb1_loglike(chi[0], P->y[i], P->aux[i], P->consts);
    default: return mvn3_loglike(chi, P->y + 3 * i, P->aux + 3 * i);  /* MVN3, NN3 */
  }
}
/* member log target lp_i = log l_i + log f_obj; -inf off support */
static double member_lp(const problem* P, int64_t i, const double* chi, const double* th) {
  double f = logf_obj(P, chi, th);
  if (f == -INFINITY) return -INFINITY;
  return loglike(P, i, chi) + f;
}
static double c_theta(const problem* P, const double* th) {
  switch (P->model) {
    case ORC_NN1: return nn1_c(th);
    case ORC_LF: return 0.0;
    case ORC_BB1: return 0.0;
    case ORC_NN3: return 0.0;
    default: return mvn3_c(th);
  }
}
static double logprior(const problem* P, const double* th) {
  switch (P->model) {
    case ORC_NN1: return nn1_logprior(th, P->consts);
    case ORC_LF: return lf_logprior(th);
    case ORC_BB1: return bb1_logprior(th);
    default: return 0.0;
  }
}

/* log f_obj(chi;theta) alone (the population term of the member target), for the pins;
 * consts: the model constants (nullable unless the model reads them, as NN3 does). */
double orc_logf_obj(int model, int d, const double* chi, const double* theta, const double* consts) {
  problem P;
  memset(&P, 0, sizeof(P));
  P.model = model; P.d = d; P.consts = consts;
  return logf_obj(&P, chi, theta);
}

/* Per-object log target at the current state (the quantity compared in parity). */
void orc_member_logdens(int model, int d, int64_t n, const double* y, const double* aux, const double* consts,
                        const double* chi, const double* theta, double* lp_out) {
  problem P;
  P.model = model; P.d = d; P.p = 0; P.n = n; P.y = y; P.aux = aux; P.consts = consts;
  for (int64_t i = 0; i < n; ++i) lp_out[i] = member_lp(&P, i, chi + (int64_t)d * i, theta);
}

/* ------------------------------------------------------------------------- */
/* The MWG chain.                                                               */
/*   state: chi[n*d], S[n*d*d] (lower, row-major per object), theta[p],         */
/*   S_theta[p*p], *sweep (sweeps done so far), *etabar_cur (LF: etabar(theta), */
/*   0 = not yet computed).                                                     */
/*   outputs: theta_rows (kept sweeps), trace arrays (nullable).                */
/* ------------------------------------------------------------------------- */
typedef struct {
  double target_accept;        /* alpha_* for members (0.4, Sec. 2.2) */
  double adapt_exponent;       /* gamma in eta = n^-gamma (2/3, Sec. 2.2) */
  double theta_target_accept;  /* R3 */
  int32_t adapt_theta;         /* R3 */
  uint64_t seed;
} orc_params;

int orc_run(int model, int d, int p, int64_t n, const double* y, const double* aux, const double* consts,
            const double* params_vec, uint64_t seed,
            double* chi, double* S, double* theta, double* S_theta, int64_t* sweep, double* etabar_cur,
            int64_t n_burn, int64_t n_iter, int64_t thin, double* theta_rows, int64_t* rows_out,
            int64_t* member_accepts, int64_t* theta_accepts,
            /* optional lockstep trace, first trace_sweeps sweeps of this call: */
            int64_t trace_sweeps, double* tr_delta, double* tr_u, uint8_t* tr_acc,
            double* tr_theta_prop, double* tr_D, double* tr_logalpha, double* tr_utheta, uint8_t* tr_tacc,
            double* tr_etabar,
            /* theta RAM update pending from the previous sweep (R3), kept across calls:
               [U (p), alpha, eta]; eta = 0: none */
            double* theta_pend,
            /* optional running moments of the latents over the kept sweeps (n*d each, member-major,
               continued across calls; mom_n = kept sweeps so far); NULL mom_mean: off */
            double* mom_mean, double* mom_m2, int64_t* mom_n) {
  orc_params prm;
  prm.target_accept = params_vec[0];
  prm.adapt_exponent = params_vec[1];
  prm.theta_target_accept = params_vec[2];
  prm.adapt_theta = (int32_t)params_vec[3];
  prm.seed = seed;

  problem P;
  P.model = model; P.d = d; P.p = p; P.n = n; P.y = y; P.aux = aux; P.consts = consts;
  if (model == ORC_LF) gl_rule_init(&P.rule, (int)consts[3], (int)consts[4]);
  if (model == ORC_BB1) gl_rule_init(&P.rule, (int)consts[4], (int)consts[5]);
  const int has_rule = (model == ORC_LF || model == ORC_BB1);

  if (has_rule && *etabar_cur == 0.0)
    *etabar_cur = (model == ORC_LF) ? lf_etabar_rule(theta, &P.rule, consts) : bb1_etabar_rule(theta, &P.rule, consts);

  int64_t total = n_burn + n_iter;
  int64_t rows = 0;
  double U[9], Y[9], th_prop[9];
  int64_t macc = 0, tacc = 0;

  for (int64_t s = 0; s < total; ++s) {
    int64_t k = *sweep + 1; /* 1-based sweep index */
    double eta = pow((double)(k + 1), -prm.adapt_exponent); /* R1 */
    int tr = (s < trace_sweeps);

    /* (1) member updates given theta (eq. psi_sampling), any order; here i = 0..n-1 */
    for (int64_t i = 0; i < n; ++i) {
      double* x = chi + (int64_t)d * i;
      double* Si = S + (int64_t)d * d * i;
      double u;
      orc_draw_member(prm.seed, (uint32_t)i, (uint32_t)k, d, U, &u);
      for (int a = 0; a < d; ++a) {
        double t = x[a];
        for (int b = 0; b <= a; ++b) t += Si[a * d + b] * U[b];
        Y[a] = t;
      }
      double lpY = member_lp(&P, i, Y, theta);
      double lpX = member_lp(&P, i, x, theta);
      double delta = (lpY == -INFINITY) ? -INFINITY : lpY - lpX;
      int acc = log(u) < delta; /* R4 */
      double alpha = (delta >= 0.0) ? 1.0 : exp(delta);
      if (acc) { for (int a = 0; a < d; ++a) x[a] = Y[a]; ++macc; }
      orc_ram_update(d, Si, U, alpha, prm.target_accept, eta);
      if (tr) {
        tr_delta[s * n + i] = delta;
        tr_u[s * n + i] = u;
        tr_acc[s * n + i] = (uint8_t)acc;
      }
    }

    /* (2) theta update given all members (eq. theta_sampling) */
    {
      double ut;
      orc_draw(prm.seed, 1u, 0u, (uint32_t)k, p, U, &ut);
      for (int a = 0; a < p; ++a) {
        double t = theta[a];
        for (int b = 0; b <= a; ++b) t += S_theta[a * p + b] * U[b];
        th_prop[a] = t;
      }
      double lpri_new = logprior(&P, th_prop);
      double logalpha = -INFINITY, D = 0.0, eb_new = 0.0;
      if (lpri_new != -INFINITY) {
        ksum acc_sum = {0.0, 0.0};
        int off = 0;
        for (int64_t i = 0; i < n; ++i) {
          const double* x = chi + (int64_t)d * i;
          double fn = logf_obj(&P, x, th_prop);
          if (fn == -INFINITY) { off = 1; break; }
          ks_add(&acc_sum, fn - logf_obj(&P, x, theta));
        }
        if (!off) {
          D = ks_val(&acc_sum);
          logalpha = D + (double)n * (c_theta(&P, th_prop) - c_theta(&P, theta)) + lpri_new - logprior(&P, theta);
          if (has_rule) {
            eb_new = (model == ORC_LF) ? lf_etabar_rule(th_prop, &P.rule, consts)
                                       : bb1_etabar_rule(th_prop, &P.rule, consts);
            logalpha -= (double)n * (log(eb_new) - log(*etabar_cur));
          }
        } else {
          D = -INFINITY;
        }
      }
      int acc = log(ut) < logalpha; /* R4 */
      double alpha = (logalpha >= 0.0) ? 1.0 : exp(logalpha);
      if (tr) {
        for (int a = 0; a < p; ++a) tr_theta_prop[s * p + a] = th_prop[a];
        tr_D[s] = D; tr_logalpha[s] = logalpha; tr_utheta[s] = ut; tr_tacc[s] = (uint8_t)acc;
        tr_etabar[s] = eb_new;
      }
      if (acc) {
        for (int a = 0; a < p; ++a) theta[a] = th_prop[a];
        if (has_rule) *etabar_cur = eb_new;
        ++tacc;
      }
      if (prm.adapt_theta) { /* R3: apply the previous step's update, keep this one for the next sweep */
        if (theta_pend[p + 1] > 0.0)
          orc_ram_update(p, S_theta, theta_pend, theta_pend[p], prm.theta_target_accept, theta_pend[p + 1]);
        for (int a = 0; a < p; ++a) theta_pend[a] = U[a];
        theta_pend[p] = alpha;
        theta_pend[p + 1] = eta;
      }
    }

    /* (3) record kept sweeps: the theta row and, when asked, every latent component's running
       mean and sum of squared deviations by Welford's (1962) recurrence: with x the m-th kept
       value, mean_m = mean_{m-1} + (x - mean_{m-1})/m and
       M2_m = M2_{m-1} + (x - mean_{m-1})(x - mean_m) */
    int kept = s >= n_burn && thin > 0 && ((s - n_burn + 1) % thin) == 0;
    if (kept && theta_rows) {
      for (int a = 0; a < p; ++a) theta_rows[rows * p + a] = theta[a];
      ++rows;
    }
    if (kept && mom_mean) {
      const int64_t m = ++*mom_n;
      for (int64_t q = 0; q < n * d; ++q) {
        const double x = chi[q], dl = x - mom_mean[q];
        mom_mean[q] += dl / (double)m;
        mom_m2[q] += dl * (x - mom_mean[q]);
      }
    }
    *sweep = k;
  }
  if (rows_out) *rows_out = rows;
  if (member_accepts) *member_accepts += macc;
  if (theta_accepts) *theta_accepts += tacc;
  if (has_rule) gl_rule_free(&P.rule);
  return 0;
}

/* ------------------------------------------------------------------------- */
/* Test model of the member accept rule (Sec. 2.2: accept with probability     */
/* min(1, pi(Y)/pi(X)); R4: accept iff ln u < Delta). n independent chains on   */
/* the states {0, 1} with target (1 - pi1, pi1); every step proposes the other  */
/* state (symmetric flip), Delta = ln pi(other) - ln pi(current), u the accept  */
/* uniform of a d = 1 member of that sweep (orc_draw_member). Chain i starts in */
/* state i mod 2. counts[2 from + to] sums the transitions.                      */
/* ------------------------------------------------------------------------- */
void orc_twostate_run(double pi1, int64_t n, int64_t sweeps, uint64_t seed, int64_t* counts) {
  const double lp[2] = {log(1.0 - pi1), log(pi1)};
  for (int q = 0; q < 4; ++q) counts[q] = 0;
  for (int64_t i = 0; i < n; ++i) {
    int x = (int)(i & 1);
    for (int64_t k = 1; k <= sweeps; ++k) {
      double z, u;
      orc_draw_member(seed, (uint32_t)i, (uint32_t)k, 1, &z, &u);
      const double delta = lp[1 - x] - lp[x];
      const int y = (log(u) < delta) ? 1 - x : x;
      counts[2 * x + y]++;
      x = y;
    }
  }
}

/* ------------------------------------------------------------------------- */
/* Latent marginalisation by cubature (Sec. 6: for low-dimensional latents the  */
/* members can be integrated out by quadrature, leaving an MCMC over theta      */
/* alone). Reading R9 fixes the rule:                                           */
/*   log p_i(theta) = log int l_i(chi) f_obj(chi;theta) dchi                    */
/* by Gauss-Legendre panels in chi:                                             */
/*   NN1: one 64-node panel on m +- 10 s, with m, s the mean and standard       */
/*        deviation of the (Gaussian) integrand;                                */
/*   LF:  with F_b = Fhat + 10 sigma_F and F_c = max(Fhat - 10 sigma_F, Fhat/2), */
/*        a 64-node panel on [max(ln L_low, ln(F_c/q)), ln(F_b/q)] and, for a    */
/*        faint member (F_c = Fhat/2, whose likelihood keeps e^{-Fhat^2/2sigma^2} */
/*        of its peak down to F = 0), a 32-node panel on [ln L_low, ln(F_c/q)]   */
/*        when that is not empty (for the others the likelihood below F_c is     */
/*        below e^-50 of its peak); -inf when ln L_low >= ln(F_b/q).             */
/*   BB1: the same panels with the flux-dependent error sigma(F): F_b solves    */
/*        F_b - Fhat = 10 sigma(F_b) (alpha < 1/10), F_c = max(Fhat - 10         */
/*        sigma(Fhat), Fhat/2), the lower end ln l + ln(lower/l), the selection  */
/*        rule's own lower end (BB1 has no truncation), and a 128-node tail      */
/*        panel (it spans ~40 e-folds of L and the rise of 1 - e^{-L/l}).        */
/* The marginal posterior of theta is prod_i p_i(theta) e^{N c(theta)} pi(theta) */
/* (LF: divided by etabar(theta)^N, as in the member form).                     */
/* ------------------------------------------------------------------------- */
#define ORC_MARG_NPEAK 64
#define ORC_MARG_NTAIL 32
#define ORC_MARG_NTAIL_BB1 128
#define ORC_MARG_K 10.0

typedef struct {
  double xp[ORC_MARG_NPEAK], wp[ORC_MARG_NPEAK];
  double xt[ORC_MARG_NTAIL], wt[ORC_MARG_NTAIL];
  double xb[ORC_MARG_NTAIL_BB1], wb[ORC_MARG_NTAIL_BB1];
} marg_rule;

static void marg_rule_init(marg_rule* R) {
  orc_gauss_legendre(ORC_MARG_NPEAK, R->xp, R->wp);
  orc_gauss_legendre(ORC_MARG_NTAIL, R->xt, R->wt);
  orc_gauss_legendre(ORC_MARG_NTAIL_BB1, R->xb, R->wb);
}

/* log of sum_j w_j exp(v_j), by the largest v_j */
static double log_wsum(const double* v, const double* w, int m) {
  double vmax = -INFINITY;
  for (int j = 0; j < m; ++j)
    if (v[j] > vmax) vmax = v[j];
  if (vmax == -INFINITY) return -INFINITY;
  ksum s = {0.0, 0.0};
  for (int j = 0; j < m; ++j) ks_add(&s, w[j] * exp(v[j] - vmax));
  return vmax + log(ks_val(&s));
}

static double marg_logp_one(const problem* P, const marg_rule* R, int64_t i, const double* th) {
  double v[ORC_MARG_NPEAK + ORC_MARG_NTAIL_BB1], w[ORC_MARG_NPEAK + ORC_MARG_NTAIL_BB1];
  int m = 0;
  if (P->model == ORC_NN1) {
    double y = P->y[i], sig = P->aux[i], tau = exp(th[1]);
    double s2 = sig * sig, t2 = tau * tau;
    double mean = (y * t2 + th[0] * s2) / (s2 + t2);
    double sd = sig * tau / sqrt(s2 + t2);
    double a = mean - ORC_MARG_K * sd, b = mean + ORC_MARG_K * sd;
    for (int j = 0; j < ORC_MARG_NPEAK; ++j) {
      double chi = 0.5 * (a + b) + 0.5 * (b - a) * R->xp[j];
      v[m] = nn1_loglike(chi, y, sig) + nn1_logf_obj(chi, th);
      w[m] = 0.5 * (b - a) * R->wp[j];
      ++m;
    }
    return log_wsum(v, w, m);
  }
  /* LF and BB1 */
  const int bb1 = (P->model == ORC_BB1);
  double fhat = P->y[i], q = lf_q(P->aux[i]);
  double Fb, Fc, lo;
  if (bb1) {
    double s0 = P->consts[0], al = P->consts[1], K = ORC_MARG_K;
    double den = 1.0 - K * K * al * al;
    Fb = (fhat + K * sqrt(al * al * fhat * fhat + den * s0 * s0)) / den;
    Fc = fhat - K * sqrt(bb1_sigma2(fhat, P->consts));
    lo = th[1] + P->consts[7];
  } else {
    double sigF = P->consts[0];
    Fb = fhat + ORC_MARG_K * sigF;
    Fc = fhat - ORC_MARG_K * sigF;
    lo = th[2];
  }
  const int faint = (Fc < 0.5 * fhat);
  if (faint) Fc = 0.5 * fhat;
  double chib = log(Fb / q), chic = log(Fc / q);
  double a2 = (chic > lo) ? chic : lo;
  if (!(a2 < chib)) return -INFINITY;
  for (int j = 0; j < ORC_MARG_NPEAK; ++j) {
    double chi = 0.5 * (a2 + chib) + 0.5 * (chib - a2) * R->xp[j];
    v[m] = bb1 ? bb1_loglike(chi, fhat, P->aux[i], P->consts) + bb1_logf_obj(chi, th)
               : lf_loglike(chi, fhat, P->aux[i], P->consts) + lf_logf_obj(chi, th);
    w[m] = 0.5 * (chib - a2) * R->wp[j];
    ++m;
  }
  if (faint && lo < chic) {
    const int nt = bb1 ? ORC_MARG_NTAIL_BB1 : ORC_MARG_NTAIL;
    const double* xt = bb1 ? R->xb : R->xt;
    const double* wt = bb1 ? R->wb : R->wt;
    for (int j = 0; j < nt; ++j) {
      double chi = 0.5 * (lo + chic) + 0.5 * (chic - lo) * xt[j];
      v[m] = bb1 ? bb1_loglike(chi, fhat, P->aux[i], P->consts) + bb1_logf_obj(chi, th)
                 : lf_loglike(chi, fhat, P->aux[i], P->consts) + lf_logf_obj(chi, th);
      w[m] = 0.5 * (chic - lo) * wt[j];
      ++m;
    }
  }
  return log_wsum(v, w, m);
}

/* Per-member log p_i(theta) of the rule above (NN1: aux = sigma_i; LF, BB1: aux = r_i). */
void orc_marg_logp(int model, int64_t n, const double* y, const double* aux, const double* consts,
                   const double* theta, double* out) {
  problem P;
  memset(&P, 0, sizeof(P));
  P.model = model; P.d = 1; P.n = n; P.y = y; P.aux = aux; P.consts = consts;
  marg_rule R;
  marg_rule_init(&R);
  for (int64_t i = 0; i < n; ++i) out[i] = marg_logp_one(&P, &R, i, theta);
}

/* theta-only chain on the marginal posterior: the theta step of orc_run with
 * D = sum_i [log p_i(theta') - log p_i(theta)] in place of the sum over log f_obj;
 * the same theta draws (Philox stream 1), RAM on theta (R3) and index (R1).
 * lp[n]: log p_i at the current theta (updated on accept). Trace arrays nullable. */
int orc_marg_run(int model, int p, int64_t n, const double* y, const double* aux, const double* consts,
                 const double* params_vec, uint64_t seed, double* theta, double* S_theta, double* lp,
                 int64_t* sweep, double* etabar_cur, int64_t n_burn, int64_t n_iter, int64_t thin,
                 double* theta_rows, int64_t* rows_out, int64_t* theta_accepts, int64_t trace_sweeps,
                 double* tr_theta_prop, double* tr_D, double* tr_logalpha, double* tr_utheta, uint8_t* tr_tacc,
                 double* tr_etabar) {
  problem P;
  memset(&P, 0, sizeof(P));
  P.model = model; P.d = 1; P.p = p; P.n = n; P.y = y; P.aux = aux; P.consts = consts;
  const int has_rule = (model == ORC_LF || model == ORC_BB1);
  if (model == ORC_LF) gl_rule_init(&P.rule, (int)consts[3], (int)consts[4]);
  if (model == ORC_BB1) gl_rule_init(&P.rule, (int)consts[4], (int)consts[5]);
  if (has_rule && *etabar_cur == 0.0)
    *etabar_cur = (model == ORC_LF) ? lf_etabar_rule(theta, &P.rule, consts) : bb1_etabar_rule(theta, &P.rule, consts);
  marg_rule R;
  marg_rule_init(&R);
  double* lpn = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  const double adapt_exponent = params_vec[1], theta_target_accept = params_vec[2];
  const int adapt_theta = (int)params_vec[3];
  int64_t total = n_burn + n_iter, rows = 0, tacc = 0;
  double U[9], th_prop[9];
  for (int64_t s = 0; s < total; ++s) {
    int64_t k = *sweep + 1;
    double eta = pow((double)(k + 1), -adapt_exponent); /* R1 */
    double ut;
    orc_draw(seed, 1u, 0u, (uint32_t)k, p, U, &ut);
    for (int a = 0; a < p; ++a) {
      double t = theta[a];
      for (int b = 0; b <= a; ++b) t += S_theta[a * p + b] * U[b];
      th_prop[a] = t;
    }
    double lpri_new = logprior(&P, th_prop);
    double logalpha = -INFINITY, D = 0.0, eb_new = 0.0;
    if (lpri_new != -INFINITY) {
      ksum acc_sum = {0.0, 0.0};
      int off = 0;
      for (int64_t i = 0; i < n; ++i) {
        lpn[i] = marg_logp_one(&P, &R, i, th_prop);
        if (lpn[i] == -INFINITY) { off = 1; break; }
        ks_add(&acc_sum, lpn[i] - lp[i]);
      }
      if (!off) {
        D = ks_val(&acc_sum);
        logalpha = D + (double)n * (c_theta(&P, th_prop) - c_theta(&P, theta)) + lpri_new - logprior(&P, theta);
        if (has_rule) {
          eb_new = (model == ORC_LF) ? lf_etabar_rule(th_prop, &P.rule, consts)
                                     : bb1_etabar_rule(th_prop, &P.rule, consts);
          logalpha -= (double)n * (log(eb_new) - log(*etabar_cur));
        }
      } else {
        D = -INFINITY;
      }
    }
    int acc = log(ut) < logalpha; /* R4 */
    double alpha = (logalpha >= 0.0) ? 1.0 : exp(logalpha);
    if (s < trace_sweeps) {
      for (int a = 0; a < p; ++a) tr_theta_prop[s * p + a] = th_prop[a];
      tr_D[s] = D; tr_logalpha[s] = logalpha; tr_utheta[s] = ut; tr_tacc[s] = (uint8_t)acc;
      tr_etabar[s] = eb_new;
    }
    if (acc) {
      for (int a = 0; a < p; ++a) theta[a] = th_prop[a];
      for (int64_t i = 0; i < n; ++i) lp[i] = lpn[i];
      if (has_rule) *etabar_cur = eb_new;
      ++tacc;
    }
    if (adapt_theta) orc_ram_update(p, S_theta, U, alpha, theta_target_accept, eta);
    if (s >= n_burn && thin > 0 && ((s - n_burn + 1) % thin) == 0 && theta_rows) {
      for (int a = 0; a < p; ++a) theta_rows[rows * p + a] = theta[a];
      ++rows;
    }
    *sweep = k;
  }
  free(lpn);
  if (rows_out) *rows_out = rows;
  if (theta_accepts) *theta_accepts += tacc;
  if (has_rule) gl_rule_free(&P.rule);
  return 0;
}

/* ------------------------------------------------------------------------- */
/* One member pass of sweep k over the members [i0, i1) (the member half of the  */
/* MWG sweep, Sec. 2.1; the RAM step of Sec. 2.2 with eta = (k+1)^-gamma, R1),   */
/* for a driver that splits the members over ranks: updates chi and S of those   */
/* members in place and writes d_i = log f(chi_i;theta') - log f(chi_i;theta)   */
/* of the updated chi_i to d_out[i - i0] (-inf off the support of theta'; not    */
/* written when theta_prop is NULL). The draws are keyed by (seed, i, k), so a   */
/* split gives the same members' steps as one pass over all of them.             */
/* ------------------------------------------------------------------------- */
int orc_member_pass(int model, int d, int64_t n, const double* y, const double* aux, const double* consts,
                    const double* params_vec, uint64_t seed, int64_t k, int64_t i0, int64_t i1,
                    const double* theta, const double* theta_prop, double* chi, double* S, double* d_out,
                    int64_t* accepts) {
  problem P;
  memset(&P, 0, sizeof(P));
  P.model = model; P.d = d; P.n = n; P.y = y; P.aux = aux; P.consts = consts;
  const double target_accept = params_vec[0], adapt_exponent = params_vec[1];
  double eta = pow((double)(k + 1), -adapt_exponent); /* R1 */
  double U[9], Y[9];
  int64_t macc = 0;
  for (int64_t i = i0; i < i1; ++i) {
    double* x = chi + (int64_t)d * i;
    double* Si = S + (int64_t)d * d * i;
    double u;
    orc_draw_member(seed, (uint32_t)i, (uint32_t)k, d, U, &u);
    for (int a = 0; a < d; ++a) {
      double t = x[a];
      for (int b = 0; b <= a; ++b) t += Si[a * d + b] * U[b];
      Y[a] = t;
    }
    double lpY = member_lp(&P, i, Y, theta);
    double lpX = member_lp(&P, i, x, theta);
    double delta = (lpY == -INFINITY) ? -INFINITY : lpY - lpX;
    int acc = log(u) < delta; /* R4 */
    double alpha = (delta >= 0.0) ? 1.0 : exp(delta);
    if (acc) { for (int a = 0; a < d; ++a) x[a] = Y[a]; ++macc; }
    orc_ram_update(d, Si, U, alpha, target_accept, eta);
    if (theta_prop) {
      double fn = logf_obj(&P, x, theta_prop);
      d_out[i - i0] = (fn == -INFINITY) ? -INFINITY : fn - logf_obj(&P, x, theta);
    }
  }
  if (accepts) *accepts += macc;
  return 0;
}
