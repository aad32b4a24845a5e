/*
 * cudahm.h -- C ABI of the GB300 (sm_103a) Metropolis-within-Gibbs sampler for
 * single-plate hierarchical models (arXiv:2105.08026, "CUDAHM").
 *
 * One handle holds one population (N members, latent dimension d, population
 * parameters theta of dimension p) and one Markov chain over (theta, chi_1..chi_N).
 * Each sweep of cudahm_run is one Metropolis-within-Gibbs cycle (Sec. 2.1,
 * eqs. psi_sampling and theta_sampling):
 *   1. every member chi_i takes one robust adaptive Metropolis (RAM) step given
 *      theta (Sec. 2.2: Y = X + S U, accept with min(1, pi(Y)/pi(X)), then
 *      S S^T <- S (I + eta_n (alpha - alpha_*) U U^T/|U|^2) S^T);
 *   2. theta takes one Metropolis-Hastings step whose log ratio is the sum over
 *      members of log f(chi_i;theta') - log f(chi_i;theta) (Sec. 2.2), plus, for
 *      the luminosity model, -N (ln etabar(theta') - ln etabar(theta)) from the
 *      selection integral of the thinned point-process likelihood (Sec. 4.2,
 *      eqs. rho-mlike and epdf).
 * All of a sweep runs on the GPU in one persistent cooperative kernel; theta is
 * accepted or rejected on the device after a bounded grid barrier, with no host
 * round trip per sweep.
 *
 * Conventions
 *   - Every int-returning call returns CUDAHM_OK (0) or a negative CUDAHM_E* code;
 *     cudahm_last_error() then describes the failure (thread-local, never NULL).
 *   - Array arguments named *_host are host pointers; they are copied and stay
 *     owned by the caller. *_dev arguments are device pointers on the handle's
 *     device, also copied (the handle never keeps a caller's pointer).
 *   - Outputs go to caller-provided buffers whose required size is stated.
 *   - A handle is not thread-safe; distinct handles are independent.
 *   - All work is enqueued on the handle's stream; calls that return host data
 *     synchronise that stream.
 *   - A call that fails with EINVAL/ESTATE/EUNSUPPORTED leaves the chain unchanged.
 *     A run that fails with ETIMEOUT/ENUMERIC/ECUDA leaves the chain state as it
 *     was before that run (latents and theta are written back only on success).
 */
#ifndef CUDAHM_H
#define CUDAHM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CUDAHM_ABI_VERSION 1u

#define CUDAHM_OK 0
#define CUDAHM_EINVAL (-1)       /* bad argument or configuration */
#define CUDAHM_ENOMEM (-2)       /* device allocation failed */
#define CUDAHM_ECUDA (-3)        /* a CUDA runtime call failed */
#define CUDAHM_ETIMEOUT (-4)     /* a bounded device-side wait expired (grid barrier) */
#define CUDAHM_ENUMERIC (-5)     /* NaN in a log-density or a non-finite theta */
#define CUDAHM_ESTATE (-6)       /* call out of order (e.g. run before set_data) */
#define CUDAHM_EUNSUPPORTED (-7) /* valid request the library does not handle */

#define CUDAHM_MAX_P 9      /* largest theta dimension (d = 3 normal model) */
#define CUDAHM_MAX_CONSTS 8 /* model constants */

typedef struct cudahm* cudahm_t;

/* Models (fixed enum; each is a member density l_i, a population density f and a prior).
 *  NN1  normal-normal, d = 1, theta = (mu, ln tau), p = 2 (Sec. 3 with one characteristic):
 *       log l_i = -(y_i - chi)^2/(2 sigma_i^2), log f = -(chi - mu)^2/(2 tau^2) - ln tau;
 *       prior flat in mu and in ln tau on [consts[0], consts[1]].
 *  MVN3 normal population, d = 3 (Sec. 3 with C_pop unknown), theta = (mu[3], L11, L21, L22,
 *       L31, L32, L33), p = 9, with L the lower Cholesky factor of C_pop and its diagonal
 *       entries given as logs: log f = -|L^-1 (chi - mu)|^2/2 - sum_j ln L_jj,
 *       log l_i = -sum_j (y_ij - chi_j)^2/(2 s_ij^2); prior flat in every theta component.
 *       Member state always streams from device memory (batched kernel), per component.
 *  LF   thinned luminosity function (Sec. 4-5), d = 1, chi = ln L, theta = (beta, ln L*, ln L_low),
 *       p = 3: log f = (beta+1)(chi - ln L*) - e^(chi - ln L*) on chi > ln L_low,
 *       log l_i = -(Fhat_i - e^chi/(4 pi r_i^2))^2/(2 sigma_F^2), selection efficiency
 *       eta(F) = Phi((F - F_th)/sigma_F), distance density ~ r^2 on [0, r_max];
 *       prior -ln(1 + beta^2) + ln L_low on -2 < beta < 0, L_low < L*.
 *       consts = {sigma_F, F_th, r_max, n_L, n_r, ln(upper/L*)}: the selection integral
 *       uses an n_L-node Gauss-Legendre rule in ln L on [ln L_low, ln L* + consts[5]] times
 *       an n_r-node rule in r on [0, r_max] (n_L, n_r <= 4096).
 *  BB1  the paper's simulation model (Sec. 5.1-5.2, App. B), d = 1, chi = ln L,
 *       theta = (beta, ln l, ln u), p = 3, FP64 only:
 *       log f = ln(1 - e^(-L/l)) + beta (chi - ln u) - L/u + chi (all chi; BB1 form, its normaliser
 *       C(beta,u,l)/u cancels against the normalised selection integral),
 *       log l_i = -ln sigma(F) - (Fhat_i - F)^2/(2 sigma(F)^2), F = e^chi/(4 pi r_i^2),
 *       sigma(F)^2 = sigma0^2 + (alpha F)^2 (eq. sig-F), detection F_th = nu sigma0/sqrt(1 - alpha^2)
 *       (eq. Fth), eta(F) = Phi((F - F_th)/sigma(F)); prior -ln(1 + beta^2) + ln l on
 *       -2 < beta < 0, l < u. consts = {sigma0, alpha, nu, r_max, n_L, n_r, ln(upper/u),
 *       ln(lower/l)}: the outer rule runs over ln L in [ln l + consts[7], ln u + consts[6]].
 *  NN3  the paper's normal-normal benchmark (Sec. 3): d = 3, C_pop known, theta = mu, p = 3:
 *       log f = -|L^-1 (chi - mu)|^2/2 with L L^T = C_pop, log l_i as MVN3 (the benchmark's
 *       common measurement scales are s_ij = sigma_j for every i); prior flat in mu.
 *       consts = the packed lower triangle of C_pop {C11, C21, C22, C31, C32, C33}, which must
 *       be positive definite (else CUDAHM_EINVAL). Member state streams as for MVN3. */
typedef enum { CUDAHM_NN1 = 0, CUDAHM_MVN3 = 1, CUDAHM_LF = 2, CUDAHM_BB1 = 3, CUDAHM_NN3 = 4 } cudahm_model;

/* FP64: all arithmetic in binary64.
 * FP32 (bulk form): the member step (proposal, member log target, accept) and the theta
 * partials log f(chi;theta') - log f(chi;theta) run in binary32, with binary32 draws of their
 * own (Philox block (0, stream 2, member, odd sweep): a Box-Muller pair from 23-bit uniforms,
 * cosine for the odd sweep and sine for the next, accept uniforms from words 2 and 3); the
 * RAM factors S, the exact sum over members, the theta accept and its RAM update, and the
 * selection integral stay binary64 (a d = 1 factor is updated as S + S d, one binary64 FMA, with
 * the increment d = sqrt(1 + c) - 1 = c/(1 + sqrt(1 + c)) formed in binary32). Latents are
 * binary32 values (held as doubles in the API).
 * MVN3 in FP32 draws from Philox blocks (0, 2, member, odd sweep) and (1, 2, member, odd sweep):
 * pairs from words (0,1), (2,3) of the first and (0,1) of the second give U's three components,
 * words 2 and 3 of the second the odd and even sweep's accept uniforms; v = S U and the RAM
 * update of its 3 x 3 factor are binary64. */
typedef enum { CUDAHM_FP64 = 0, CUDAHM_FP32 = 1 } cudahm_precision;

typedef void* (*cudahm_alloc_fn)(size_t bytes, void* ctx);
typedef void (*cudahm_free_fn)(void* ptr, void* ctx);

typedef struct {
  uint32_t abi_version;          /* must be CUDAHM_ABI_VERSION */
  int32_t model;                 /* cudahm_model */
  int32_t precision;             /* cudahm_precision */
  int32_t d;                     /* latent dimension; must match the model */
  int64_t n;                     /* number of members N >= 1 */
  uint64_t seed;                 /* Philox4x32-10 key (low word, high word) */
  double target_accept;          /* alpha_* of the member RAM (Sec. 2.2: 0.4) */
  double adapt_exponent;         /* gamma of eta_n = n^-gamma (Sec. 2.2: 2/3) */
  double chi_init_scale;         /* S_1 = scale * I for every member (Sec. 2.2: 1) */
  double theta_target_accept;    /* alpha_* of the theta RAM (default 0.4) */
  int32_t adapt_theta;           /* 1: RAM on theta (member form: each step's update applied one
                                    sweep later, so that the next proposal can be formed during
                                    the sweep); 0: fixed random-walk MH */
  int32_t trace_sweeps;          /* >0: record a lockstep trace of the first trace_sweeps sweeps of each run */
  double theta_init[CUDAHM_MAX_P];       /* initial theta (first p entries) */
  double theta_prop_scale[CUDAHM_MAX_P]; /* S_theta,1 = diag(scale) */
  double model_consts[CUDAHM_MAX_CONSTS];
  int32_t device;                /* CUDA device ordinal */
  int32_t block_threads;         /* threads per block of the sweep kernel; 0 = default (256) */
  void* cuda_stream;             /* cudaStream_t to enqueue on; NULL = a stream the handle creates */
  cudahm_alloc_fn dev_alloc;     /* optional device allocator (e.g. a framework's caching allocator) */
  cudahm_free_fn dev_free;       /* must be given together with dev_alloc */
  void* alloc_ctx;               /* passed back to dev_alloc / dev_free */
  int64_t barrier_timeout_ns;    /* bound on every device-side wait; 0 = 2 s */
  int32_t debug_skip_barrier_cta;/* >= 0: that block never arrives at the grid barrier (tests the
                                    timeout path); -1 = off. Block 0 of a multi-block sweep launch
                                    holds no members and never arrives anyway (it proposes theta'
                                    and decides), so pick a block >= 1 there */
  int32_t marginal;              /* 1: integrate each member's latent out by cubature and run the
                                    chain on theta alone (NN1, LF, BB1; see cudahm_eval_marginal) */
  int32_t keep_chi_moments;      /* 1: keep every latent component's running mean and variance over
                                    the kept sweeps (see cudahm_get_chi_moments); member form only */
} cudahm_config;

typedef struct {
  int64_t sweeps;             /* sweeps done since create (or since the restored checkpoint) */
  int64_t member_accepts;     /* accepted member proposals since create */
  int64_t theta_accepts;      /* accepted theta proposals since create */
  int64_t rows;               /* theta rows held in the sample buffer */
  double last_run_ms;         /* device time of the last cudahm_run: CUDA events on its stream from
                                 before its first kernel to after the kept rows' copy to the host */
  double etabar;              /* LF: selection integral at the current theta; 0 otherwise */
  int32_t grid_blocks;        /* launch shape of the sweep kernel */
  int32_t block_threads;
  int32_t objects_per_thread;
  int32_t reserved;
} cudahm_stats;

/* Fill *cfg with the defaults above for the given model and N (seed 1, theta_init 0,
 * theta_prop_scale 0.01, NN1 prior on ln tau [-10, 10], LF rule 1024 x 1024 with
 * upper limit 60 L*). */
void cudahm_config_init(cudahm_config* cfg, int32_t model, int64_t n);

/* Create a handle: validates cfg, selects the device, allocates the device state and,
 * for LF, builds the quadrature tables on the device. *out is set only on success. */
int cudahm_create(const cudahm_config* cfg, cudahm_t* out);

/* Member data, N entries each (N*d for MVN3, member-major; copied):
 *   NN1: y = y_i, aux = sigma_i (> 0);   LF, BB1: y = Fhat_i, aux = r_i (> 0);
 *   MVN3: y = y_i[3], aux = s_i[3] (> 0, the measurement sd of each component).
 * Resets the latents to the default start (NN1, MVN3: chi_i = y_i; LF, BB1: chi_i = ln(4 pi r_i^2
 * max(Fhat_i, F_th)), for LF raised to ln L_low + 1e-6 if below), every S_i to
 * chi_init_scale * I, theta to theta_init, S_theta to diag(theta_prop_scale), and the
 * sweep counter and sample buffer to zero. */
int cudahm_set_data(cudahm_t h, const double* y_host, const double* aux_host, int64_t n);
int cudahm_set_data_device(cudahm_t h, const double* y_dev, const double* aux_dev, int64_t n);

/* Override the starting latents (N*d values, member-major; copied). Must follow set_data
 * and precede the first run. EINVAL if a value is off the model's support at theta. */
int cudahm_set_chi(cudahm_t h, const double* chi_host, int64_t n);

/* Run n_burn + n_iter sweeps, continuing the chain; keep theta after every thin-th sweep
 * of the n_iter (sweeps n_burn + thin, n_burn + 2 thin, ...). The sample buffer is replaced
 * by this run's rows. Blocking. run(a) then run(b) gives the same chain as run(a + b), and
 * the rows of the second call continue those of the first. Populations small enough keep
 * every member in registers for a whole launch; larger ones (beyond ~6e5 members) and every
 * MVN3 population stream member state from device memory through the batched kernel, with
 * the same chain. */
int cudahm_run(cudahm_t h, int64_t n_burn, int64_t n_iter, int64_t thin);

/* Copy up to cap_rows theta rows (row-major, p doubles each) of the last run. */
int cudahm_get_samples(cudahm_t h, double* theta_host, int64_t cap_rows, int64_t* rows_out);

/* Current latents (N*d doubles) and/or per-member RAM factors (N*d*d doubles, lower,
 * row-major per member); either pointer may be NULL. */
int cudahm_get_chi(cudahm_t h, double* chi_host, double* S_host);

/* Posterior summaries of the latents (Appendix A: the paper's samplers store every kept sample
 * in memory or stream it to a file; a handle created with keep_chi_moments = 1 keeps instead,
 * on the device, each member's running moments). Over the kept sweeps since
 * set_data (the sweeps whose theta row is recorded, across runs; a restored checkpoint brings
 * its own), mean_host receives each latent component's mean and var_host its sample variance
 * (divisor count - 1; 0 when count < 2), N*d doubles each, member-major; *count_out the number
 * of kept sweeps. Any pointer may be NULL. Computed by Welford's recurrence in binary64 (the
 * FP32 form adds its binary32 latents exactly); the cost is one read and one write of 2 d
 * doubles per member and kept sweep. A failed run leaves the moments of its completed launches,
 * like the latents. CUDAHM_ESTATE without keep_chi_moments. */
int cudahm_get_chi_moments(cudahm_t h, double* mean_host, double* var_host, int64_t* count_out);

/* Current theta (p doubles) and S_theta (p*p, lower, row-major); either may be NULL. */
int cudahm_get_theta(cudahm_t h, double* theta_host, double* S_theta_host);

int cudahm_get_stats(cudahm_t h, cudahm_stats* s);

/* Effective sample size of each column of a row-major sample matrix x_host (rows x cols,
 * host, e.g. the theta rows of cudahm_get_samples), written to ess_out (cols doubles, host).
 * The paper measures samplers by the time to an ESS of about 1000 in the population
 * parameters after burn-in (Sec. 3). Estimator: Geyer's initial monotone sequence on the
 * biased autocovariances (pair sums rho_2m + rho_2m+1 summed while positive, each capped by
 * the previous; tau = 2 sum - 1, at least 1/rows; ESS = rows/tau); rows < 4 or a constant
 * column give ESS = rows. Host computation, no handle or GPU needed. Returns CUDAHM_EINVAL for
 * NULL pointers or rows, cols < 1 and CUDAHM_ENUMERIC for a non-finite sample. */
int cudahm_ess(const double* x_host, int64_t rows, int32_t cols, double* ess_out);

/* Per-member log target lp_i = log l_i(chi_i) + log f(chi_i;theta) without the theta-only
 * term (-inf off support), at the current latents and the given theta (p doubles, host).
 * Writes N doubles to lp_host. Evaluated by a device kernel in the handle's precision. */
int cudahm_eval_logdens(cudahm_t h, const double* theta_host, double* lp_host);

/* Marginal form (Sec. 6: for low-dimensional latents the members can be integrated out by
 * quadrature, leaving a Markov chain over theta alone). For NN1, LF and BB1 handles, writes
 * lp_host[i] = log int l_i(chi) f(chi;theta) dchi (N doubles, host) at the given theta (p
 * doubles, host), with l_i and f as in the member form (no theta-only term). The rule is fixed:
 * NN1, a 64-node Gauss-Legendre panel on the integrand's mean +- 10 sd; LF, with
 * F_b = Fhat_i + 10 sigma_F and F_c = max(Fhat_i - 10 sigma_F, Fhat_i/2), a 64-node panel in chi
 * over [max(ln L_low, ln(F_c/q_i)), ln(F_b/q_i)] and, for a faint member (F_c = Fhat_i/2), a
 * 32-node panel over [ln L_low, ln(F_c/q_i)] when that is not empty; -inf when
 * ln L_low >= ln(F_b/q_i). BB1: the same with sigma(F), F_b solving F_b - Fhat_i = 10 sigma(F_b)
 * (alpha < 1/10, else CUDAHM_EUNSUPPORTED), F_c = max(Fhat_i - 10 sigma(Fhat_i), Fhat_i/2), the
 * lower end ln l + consts[7] and a 128-node tail panel. A handle created with marginal = 1
 * runs cudahm_run as a theta-only chain on prod_i p_i(theta) e^{N c(theta)} pi(theta) (LF:
 * divided by etabar(theta)^N): the member form's theta proposal, RAM adaptation, draws and
 * accept rule, with D = sum_i [log p_i(theta') - log p_i(theta)] summed exactly. Such a handle
 * has no latents (set_chi and get_chi give CUDAHM_EUNSUPPORTED), needs Fhat_i > 0 for LF
 * (CUDAHM_EINVAL at set_data) and runs alone (not in batch_run or the server). Other models:
 * CUDAHM_EUNSUPPORTED. FP32 handles (LF; BB1 has the FP64 form only): each node's log integrand, relative to a binary64
 * reference at the likelihood peak clamped into the window, and the panel sums are binary32
 * (log p_i within ~1e-6 of the binary64 rule); the window, the reference, log p_i, the exact
 * sum over members, the selection integral and the theta step stay binary64. NN1 has no
 * binary32 variant: its FP32 handles integrate in binary64. */
int cudahm_eval_marginal(cudahm_t h, const double* theta_host, double* lp_host);

/* Test model of the member accept rule (Sec. 2.2: accept with probability min(1, pi(Y)/pi(X))).
 * Runs n_chains independent chains on two states with target (1 - pi1, pi1) for `sweeps` steps;
 * every step proposes the other state and applies the member step's own device accept routine
 * with Delta = ln pi(other) - ln pi(current) and the member's own accept uniform of that sweep
 * (FP64: Philox block (1, stream 0, chain, sweep), the uniform of every d = 1 member; FP32: the
 * bulk form's binary32 uniform and expf). Chain i starts in state i mod 2. counts_host receives
 * 4 int64: the transitions 0->0, 0->1, 1->0, 1->1 summed over chains and sweeps. For such chains
 * P01 = min(1, pi1/pi0), P10 = min(1, pi0/pi1) and pi0 P01 = pi1 P10 (detailed balance). Needs
 * no handle; allocates and frees its own device buffers on `device`. EINVAL for pi1 outside
 * (0, 1), an unknown precision, n_chains outside [1, 2^31] or sweeps outside [1, 2^32 - 2]. */
int cudahm_twostate_run(double pi1, int32_t precision, int64_t n_chains, int64_t sweeps, uint64_t seed,
                        int32_t device, int64_t* counts_host);

/* LF and BB1: the selection integral etabar(theta) of the handle's rule at the given theta. */
int cudahm_eval_etabar(cudahm_t h, const double* theta_host, double* out);

/* LF and BB1: detection efficiency eta(F) = Phi((F - F_th)/sigma) (Sec. 5.2, eq. key; sigma_F for
 * LF, sigma(F) for BB1) for n fluxes, evaluated by the same device routine the selection integral
 * uses. */
int cudahm_eval_detection(cudahm_t h, const double* F_host, double* eta_host, int64_t n);

/* Lockstep trace of the first T = min(trace_sweeps, sweeps of the last run) sweeps of the
 * last run. Member arrays are [T][N] (sweep-major): delta = lp(Y) - lp(X) (-inf off support),
 * u = accept uniform, acc = 1 if accepted. Theta arrays: theta_prop [T][p], D [T] = sum of
 * log f(chi_i;theta') - log f(chi_i;theta) (-inf if a member is off the proposal's support,
 * 0 if theta' is off the prior), logalpha [T], utheta [T], tacc [T], etabar_prop [T]
 * (LF: etabar(theta'), else 0). Any pointer may be NULL. *t_out receives T. A marginal-form
 * handle records no member arrays (delta, u, acc are left untouched) and its D is
 * sum_i [log p_i(theta') - log p_i(theta)]. */
int cudahm_get_trace(cudahm_t h, double* delta, double* u, uint8_t* acc, double* theta_prop, double* D,
                     double* logalpha, double* utheta, uint8_t* tacc, double* etabar_prop, int64_t* t_out);

/* Serialise the whole chain state (latents, RAM factors, theta, S_theta, the pending theta RAM
 * update, counters and, with keep_chi_moments, the latents' moments) into buf. With buf == NULL
 * or cap too small, *used receives the required size and the call returns EINVAL (buf NULL:
 * OK). cudahm_restore loads such a buffer into a handle created with the same config and data;
 * the continued chain is bit-identical to an uninterrupted one. The buffer starts with a magic
 * word and a layout version; restore gives EINVAL for another version or configuration. */
int cudahm_checkpoint(cudahm_t h, void* buf, size_t cap, size_t* used);
int cudahm_restore(cudahm_t h, const void* buf, size_t size);

/* LF selection integral etabar(theta) that allocates no device memory. The paper has no
 * counterpart: this serves callers that cannot call cudaMalloc when they need the value
 * (a process that gives all device memory to its own pool up front and forbids later
 * allocations, a latency-critical loop that must not pay for the synchronisation an
 * allocation implies, a caller that is out of device memory). The tables and partial sums
 * live in one fixed array compiled into the library (about 113 KB on every GPU that loads
 * it, held until the process exits), which bounds the rule to
 * n_L, n_r <= CUDAHM_NOALLOC_MAX_NODES.
 *   theta_dev    3 doubles on the current device: (beta, ln L*, ln L_low)
 *   consts_host  6 doubles on the host: sigma_F, F_th, r_max, n_L, n_r, ln(upper/L*)
 *   etabar_dev   1 double on the current device: receives etabar(theta)
 *   cuda_stream  cudaStream_t to enqueue on (NULL = the default stream); the call returns
 *                once the work is enqueued; read the result after synchronising.
 * Returns EINVAL (with a message) for rule sizes above the limit or bad constants. The
 * value agrees with cudahm_eval_etabar's for the same theta and constants within 1e-13
 * relative: this call sums the rule pair by pair, a handle interpolates a table of the inner
 * sum over r. The first call on a
 * device looks up the array's device address (cudaGetSymbolAddress, once per device, with
 * that device current); make that first call before any stream capture. Every call on a
 * device shares the array and it keeps the last call's contents (nothing in it must start
 * at zero). A call rebuilds the rule tables (about a millisecond of kernels) only when n_L,
 * n_r, r_max or sigma_F differ from the previous call's on the device; otherwise it reads the
 * tables that call left, so when consecutive calls use different streams, let the earlier
 * one's work finish first. Calls that overlap on the GPU race on the array. */
#define CUDAHM_NOALLOC_MAX_NODES 1024
int cudahm_lf_etabar_noalloc(const double* theta_dev, const double* consts_host, double* etabar_dev,
                             void* cuda_stream);

/* Launch shape of a batched run. Zero fields are chosen automatically, and a tuned shape is
 * cached per (precision, number of populations, LF count, size class) for the process:
 *  - block size and grid: trial launches of 16 sweeps each at the start of the run (they are
 *    ordinary sweeps of it) over 128 and 256 threads x the largest grid the occupancy allows and
 *    half of it; the fastest device time per sweep wins;
 *  - then two launches of 32 sweeps whose per-population device times (like the trials')
 *    rebalance each population's share of the blocks (the first share comes from a cost model);
 *  - then launches of sweeps_per_launch sweeps: enough that the measured host cost of a launch
 *    (synchronisation, graph launch, the error words) is about 1% of its device time, 64..4096.
 * A population's chain does not depend on the launch shape (all sums are exact). */
typedef struct {
  int32_t block_threads;      /* 128 or 256; 0 = tune */
  int32_t sweeps_per_launch;  /* sweeps of each long launch (each launch ends with a grid-wide sync); 0 = tune */
  int32_t use_graph;          /* 1: replay the launch sequence from a captured CUDA graph */
  int32_t grid_blocks;        /* blocks of the launch (at most what the occupancy allows); 0 = tune;
                                 out: the blocks used */
} cudahm_tune;

/* Run n_burn + n_iter sweeps of k populations (handles created and loaded as usual, on one
 * device, one precision; a trace only for k = 1) in one persistent launch per chunk of sweeps.
 * Population q gets a block range sized by a cost model (members, selection-rule pairs),
 * refined twice from each population's measured device time; its blocks meet at a bounded
 * per-population barrier each sweep, so populations never wait for one another. Every
 * population's chain and samples are bit-identical to what cudahm_run gives for it alone.
 * Work goes to handle 0's stream; the call blocks. tune may be NULL; chosen (nullable)
 * receives the shape used. On failure every handle's chain stops where its last launch ended. */
int cudahm_batch_run(cudahm_t* handles, int32_t k, int64_t n_burn, int64_t n_iter, int64_t thin,
                     const cudahm_tune* tune, cudahm_tune* chosen);

/* Shards: one population split across devices (Sec. 6, populations larger than one device
 * holds). Each shard is a handle created with the population's config (same model, constants,
 * theta start, seed and precision) whose n members are the population's members
 * [member_offset, member_offset + n), loaded with set_data as usual. A sweep is
 *   1. cudahm_shard_pass on every shard: the member steps of its members (the draws of member i
 *      carry its population index member_offset + i, so they are the unsplit chain's), and the
 *      shard's part of the theta' sum D = sum_i [log f(chi_i;theta') - log f(chi_i;theta)] and of
 *      the selection integral at theta' (LF, BB1: outer nodes [n_L part/parts, n_L (part+1)/parts)),
 *      written as CUDAHM_SHARD_WORDS exchange words;
 *   2. the caller adds the words of all shards as unsigned 64-bit integers (an all-reduce with
 *      the sum operation, e.g. NCCL or gloo on int64/uint64 buffers; wrap-around never occurs);
 *   3. cudahm_shard_decide on every shard with the summed words: the theta decision (Sec. 2.2),
 *      taken identically on every shard.
 * The chain, the latents and the kept theta rows equal those of one handle holding the whole
 * population (cudahm_run), bit for bit: all sums are exact.
 * Exchange words (little-endian u64): [0..5] D, [6..11] the selection integral, each the 32-bit
 * limbs (low first) of a 192-bit two's-complement fixed-point number with 2^-96 resolution (each
 * addend rounded toward zero to a multiple of 2^-96); [12] count of d_i <= -2^94 or off the
 * support | NaN count << 32; [13] count of d_i >= 2^94 | member-step NaN count << 32; [14] the
 * shard's member count; [15] 1. decide checks that [14] sums to population_n and [15] to parts.
 * Work goes to the handle's stream (config cuda_stream), in call order, without host
 * synchronisation between begin and end; words_dev and total_dev are device buffers of 16
 * words, 8-byte aligned, which may be the same buffer (an in-place all-reduce between the two
 * calls). Not with the marginal form, a lockstep trace or latent moments (EUNSUPPORTED). */
#define CUDAHM_SHARD_WORDS 16

/* This handle is shard `part` of `parts` of a population of population_n members (< 2^32). */
int cudahm_shard_config(cudahm_t h, int64_t member_offset, int64_t population_n, int32_t part, int32_t parts);
/* Starts a sharded run of n_burn + n_iter sweeps (thin as in cudahm_run); synchronises. */
int cudahm_shard_begin(cudahm_t h, int64_t n_burn, int64_t n_iter, int64_t thin);
/* Enqueues the next sweep's pass; its exchange words go to words_dev (overwritten). */
int cudahm_shard_pass(cudahm_t h, uint64_t* words_dev);
/* Enqueues the decision of the sweep whose pass came last, from the summed words. */
int cudahm_shard_decide(cudahm_t h, const uint64_t* total_dev);
/* Synchronises and ends the run (after any number of pass/decide pairs); rows_out (nullable)
 * receives the kept rows, which cudahm_get_samples returns. ESTATE if the words of some sweep
 * did not come from every shard once (the chain stops before that sweep's decision), or if the
 * last pass was not decided (the run still ends; the latents are then one sweep past theta);
 * ENUMERIC, ETIMEOUT as for cudahm_run. Until the run ends, cudahm_run and cudahm_batch_run on
 * the handle fail with ESTATE, and other calls see the chain between sweeps. */
int cudahm_shard_end(cudahm_t h, int64_t* rows_out);

/* Serving: a request loop with continuous batching.
 * A server owns a worker thread and a stream on one device. Requests (a config, member data
 * and run lengths; the data are copied) queue in arrival order; the worker admits them while
 * fewer than max_active are on the device and their estimated device memory fits the budget,
 * creates their chain state, and advances every admitted request by sweeps_per_step sweeps
 * per batched launch, each at its own stage. A finished request's theta rows are copied out
 * and its memory released, which lets the next queued request in. A request's result is
 * bit-identical to running it alone with cudahm_run (batched chains do not depend on what
 * shares the launch). All requests of a server use its precision. */
typedef struct cudahm_server* cudahm_server_t;

int cudahm_server_create(size_t mem_budget_bytes, int32_t device, int32_t precision, int32_t max_active,
                         int32_t sweeps_per_step, cudahm_server_t* out);
/* ENOMEM if the request alone would exceed the budget; *ticket identifies it afterwards. */
int cudahm_server_submit(cudahm_server_t s, const cudahm_config* cfg, const double* y_host,
                         const double* aux_host, int64_t n_burn, int64_t n_iter, int64_t thin, uint64_t* ticket);
/* *done = 1 once the request has finished (successfully or not). */
int cudahm_server_poll(cudahm_server_t s, uint64_t ticket, int32_t* done);
/* Block until the request has finished; ETIMEOUT after timeout_ms (< 0: no limit). */
int cudahm_server_wait(cudahm_server_t s, uint64_t ticket, int64_t timeout_ms);
/* Copy up to cap_rows theta rows of a finished request and release it (the ticket becomes
 * unknown); latency_ms = completion time - submission time (host clock). Returns the
 * request's error if it failed. */
int cudahm_server_result(cudahm_server_t s, uint64_t ticket, double* theta_host, int64_t cap_rows,
                         int64_t* rows_out, double* latency_ms);
/* Completed requests, sum of members x sweeps over them, time spent in launches, queue and
 * active counts (any pointer may be NULL). */
int cudahm_server_stats(cudahm_server_t s, int64_t* completed, double* member_sweeps, double* busy_ms,
                        int64_t* queued, int64_t* active);
/* Stop the worker (after its current launch), release everything; NULL is ignored. */
int cudahm_server_destroy(cudahm_server_t s);

/* sizeof(cudahm_config) and sizeof(cudahm_stats) as compiled into the library, so that
 * bindings can check their struct layouts. */
size_t cudahm_sizeof_config(void);
size_t cudahm_sizeof_stats(void);

/* Message of the last failed call on this thread; never NULL. */
const char* cudahm_last_error(void);

/* Release the handle and its device memory; NULL is ignored. */
void cudahm_destroy(cudahm_t h);

#ifdef __cplusplus
}
#endif
#endif /* CUDAHM_H */
