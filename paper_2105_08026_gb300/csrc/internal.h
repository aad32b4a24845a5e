// Internal interface between the host runtime (runtime.cu) and the kernels (sweep.cu).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace chm {

constexpr int kMaxP = 9;
constexpr int kPartWords = 8;  // u64 words of one block's partial: D[3], E[3], flags[2]
// grid totals of the persistent kernels, added by every member block: D and E as six 32-bit
// limbs each (in u64 counters) in words 0-5 and 6-11, the flags as two packed u64 in 12-13; the
// sweep kernel's selection integral at the sweep's other possible theta' in 14-19 (E at the
// proposal made for a rejected theta in 6-11, for an accepted one in 14-19) and their flag
// counts in 20; three buffers, one per sweep mod 3
constexpr int kAccWords = 22;

// Chain state kept on the device between runs.
struct ChainState {
  double theta[kMaxP];
  double S_theta[kMaxP * kMaxP];
  double etabar;     // LF: selection integral at theta (0 = not computed)
  long long sweeps;  // sweeps done
  long long member_acc;
  long long theta_acc;
  long long rows;    // rows written by the last launch
  int mcur;          // marginal form: which of the two log p_i arrays holds the current theta's
  int mom_sel;       // running moments of the latents: which of the two buffers is committed
  long long mom_n;   // kept sweeps accumulated in the committed moments
  // member form: the theta RAM update of the last sweep, applied one sweep late (U, alpha, eta;
  // pend_eta = 0: none)
  double pend_U[kMaxP];
  double pend_alpha;
  double pend_eta;
};

// Model constants used inside kernels.
struct ModelConsts {
  double lo, hi;        // NN1: prior range of ln tau
  double inv2sig2;      // LF: 1/(2 sigma_F^2)
  double cth;           // LF: F_th / sigma_F
  double F_th;          // LF, BB1
  double ln_upper;      // LF: ln(upper/L*); BB1: ln(upper/u)
  double chi_init_scale;
  // BB1
  double s0sq;          // sigma0^2
  double alpha;         // slope of the flux-dependent error, sigma(F)^2 = sigma0^2 + (alpha F)^2
  double F_pre;         // flux above which Phi((F - F_th)/sigma(F)) > Phi(8.5) (rule prefix); inf if none
  double ln_lower;      // ln(lower/l)
  // NN3: inverse of the lower Cholesky factor of the known C_pop, packed (00, 10, 11, 20, 21, 22)
  double li3[6];
  double sigF;          // LF: sigma_F
  int marginal;         // 1: latents integrated out by cubature (theta-only chain)
};

struct SweepArgs {
  int model;
  int f32;  // 1: FP32 bulk member arithmetic
  int p;
  long long n;
  const double* y;    // NN1: y_i;  LF: Fhat_i
  const double* aux;  // NN1: 1/sigma_i^2;  LF: 1/(4 pi r_i^2)
  double* chi;
  double* S;
  ChainState* chain;
  unsigned long long* partials;  // streaming kernel: [2][grid][kPartWords] per-block partials
  unsigned long long* acc3;      // sweep kernel: [3][kAccWords] grid totals (zeroed before each launch)
  unsigned int* bar;
  int* err;
  const double* tab_U;    // [ns][p] theta-proposal normals
  const double* tab_u;    // [ns] theta accept uniforms
  const double* tab_lnu;  // [ns] their logarithms
  const double* tab_eta;  // [ns] adaptation weights (k+1)^-gamma
  long long k0;           // sweeps done before this launch
  long long ns;           // sweeps in this launch
  long long burn_left;    // sweeps of this launch still in burn-in
  long long thin;
  long long keep_phase;   // post-burn sweeps already done by earlier launches of this run
  double* rows;           // theta rows of this launch
  double astar, astar_theta;
  int adapt_theta;
  uint32_t key0, key1;
  ModelConsts mc;
  // LF selection rule
  const double* xL;
  const double* wL;
  const double* qs;  // q(r_k)/sigma_F
  const double* Wr;  // inner weights
  const double* phi_coef;  // Taylor table of the normal CDF
  const double* cw;        // prefix sums of the inner weights (n_r + 1)
  const double* math_tab;  // exp/log tables
  int nL, nr;
  int rows_smem;     // segment slots per block for the outer-node values
  int mpb;           // members of the largest block (shared-memory slots for y, aux)
  // trace (nullable)
  long long trace_T;
  long long trace_off;  // sweeps of this run traced by earlier launches
  double* tr_delta;
  double* tr_u;
  uint8_t* tr_acc;
  double* tr_thprop;
  double* tr_D;
  double* tr_logalpha;
  double* tr_ut;
  uint8_t* tr_tacc;
  double* tr_eb;
  long long timeout_ns;
  int skip_cta;
  double gamma;       // adaptation exponent (eta = n^-gamma)
  const float* d32;   // FP32 form: precomputed binary32 member data (kData32 x n32, member-minor)
  float* chi32;       // FP32 form, d = 1: the latents (binary32 state; chi is a binary64 copy for the API)
  float* even32;      // FP32 form, d = 1: the streaming kernel's cache of each member's next (even) sweep
                      // normal and accept uniform, written by the odd sweep before it (rows 0, 1), and of
                      // its log l_i at the current latent (row 2, luminosity model), [3][n32]
  long long n32;      // FP32 form, d = 1: row stride of d32 and padded length of chi32 and S (a multiple
                      // of kTilePad, so that bulk copies of aligned member tiles stay in bounds); else n
  double* pub;        // theta' proposals published by block 0 (kPubSlots slots of kPubWords doubles);
                      // its sequence word is bar[1]
  double* marg_lp;           // marginal form: log p_i at two thetas, [2][n]
  const double* marg_nodes;  // marginal form: panel nodes and weights (kMargNodeWords)
  const double* marg_d32;    // marginal form, FP32 bulk, LF: per-member window data, [kMarg32Words][n]
  double* spare3;            // d = 3, FP64: the sine halves of the odd sweep's Box-Muller pairs, [3][n]
  // running moments of the latents over the kept sweeps (nullptr: off): two buffers of
  // [mean[d][n], M2[d][n]], the committed one named by ChainState::mom_sel
  double* mom;
  // the rule's inner sum H(ln L) tabulated (h_ncell cells of kHDeg + 1 Chebyshev coefficients);
  // nullptr: evaluate the rule pair by pair
  const double* htab;
  double h_ua, h_ub;  // table range in ln L; H = h_lo below it, h_hi above it
  double h_lo, h_hi;
  int h_ncell;
  // shard of a population split across devices: the population index of member 0 (the member
  // word of every member draw is moff + i), the rule's outer nodes [rule_j0, rule_j1) this shard
  // adds (rule_j1 = 0: all n_L), and (non-null: the streaming kernel's shard pass) where the
  // pass writes the shard's exchange words
  unsigned int moff;
  int rule_j0, rule_j1;
  unsigned long long* shard_out;
};

constexpr int kPubWords = 32;  // doubles per publication slot of the sweep kernel
// slots: 0 the launch's first theta'; 1 + 2 (t & 1) + c the proposal of sweep t for outcome c of
// the decision before it
constexpr int kPubSlots = 5;

// Exchange words of one shard's sweep (cudahm_shard_pass): the theta' partial D and the
// selection-rule partial E as six 32-bit limbs each (in u64 words, so that the words of all
// shards add as integers), the flag counts packed two to a word, the shard's member count and 1
// (the number of shards that contributed).
constexpr int kShardWords = 16;

// FP32 form, d = 1: member arrays are padded to a multiple of kTilePad members, so that the
// streaming kernel's bulk copies of member tiles (starting at multiples of 4 members: 16-byte
// aligned for binary32 and binary64 arrays) stay in bounds.
constexpr long long kTilePad = 64;

// Tabulated inner sum of the selection rule: Chebyshev series of degree kHDeg on cells of
// width kHDelta in u = ln L.
constexpr int kHDeg = 12;
constexpr double kHDelta = 0.125;

// Cubature rule of the marginal form: Gauss-Legendre panels of kMargPeak and kMargTail nodes,
// the likelihood window +- kMargK standard deviations.
constexpr int kMargPeak = 64;
constexpr int kMargTail = 32;
constexpr int kMargTailBB1 = 128;
constexpr double kMargK = 10.0;
constexpr int kMargNodeWords = 2 * (kMargPeak + kMargTail + kMargTailBB1);
constexpr int kMarg32Words = 6;  // ln(Fhat/q), Fhat/q, ln(F_b/q), ln(F_c/q), Fhat^2/(2 sigma_F^2), faint (1/0)

// Progress of one population through a batched run (device memory, updated by the kernel).
struct BatchProg {
  long long total;   // sweeps of the run
  long long off;     // sweeps done
  long long n_burn;
  long long thin;
  long long rows;    // theta rows written
  long long t_ns;    // device time of the population's last launch (%globaltimer), for balancing
};

// Batched launches (batch.cu).
size_t batch_smem_bytes(bool f32, bool any_d1, int block);
// d1: every population has a one-dimensional latent (the lighter kernel variant)
cudaError_t batch_occupancy(bool f32, bool d1, int block, int smem_bytes, int* blocks_per_sm);
cudaError_t launch_batch(bool f32, bool d1, const SweepArgs* pops, BatchProg* progs, const int* b0s, const int* nbs,
                         int npop, int chunk, int seg_slots, int grid, int block, int smem_bytes, cudaStream_t st);
cudaError_t launch_batch_tables(const SweepArgs* pops, const BatchProg* progs, int npop, int chunk, cudaStream_t st);
// The theta decision of one sweep of a split population from the summed exchange words of all
// its shards (one block); parts: the number of shards, n_pop: the population's member count.
cudaError_t launch_shard_decide(int model, const SweepArgs* pop, BatchProg* prog, const unsigned long long* total,
                                long long n_pop, int parts, cudaStream_t st);
cudaError_t launch_data32(int model, long long n, long long n32, const double* y, const double* aux,
                          const ModelConsts& mc, float* d32, cudaStream_t st);
cudaError_t launch_chi_to32(long long n, long long n32, const double* chi, float* chi32, cudaStream_t st);
cudaError_t launch_chi_from32(long long n, const float* chi32, double* chi, cudaStream_t st);
int data32_words(int model);

// Marginal form (marginal.cu).
size_t marg_smem_bytes(int model, int rows_smem);
cudaError_t marg_occupancy(int model, bool f32, int block, int smem_bytes, int* blocks_per_sm);
cudaError_t launch_marg(const SweepArgs& a, int grid, int block, cudaStream_t st);
// f32: the FP32 bulk form (LF reads md32; NN1 has no binary32 variant and uses binary64)
cudaError_t launch_marg_eval(int model, bool f32, long long n, const double* y, const double* aux,
                             const double* theta_dev, const ModelConsts& mc, const double* math_tab,
                             const double* nodes, const double* md32, double* out, cudaStream_t st);
cudaError_t launch_marg_data32(long long n, const double* y, const double* aux, const ModelConsts& mc,
                               const double* math_tab, double* md32, cudaStream_t st);
cudaError_t launch_marg_nodes(double* nodes, cudaStream_t st);

// Records a failure for cudahm_last_error() (runtime.cu); returns code.
int record_error(int code, const char* msg);

// Kernel launch helpers (sweep.cu). Return cudaError_t of the launch.
cudaError_t launch_sweep(const SweepArgs& a, int K, int grid, int block, cudaStream_t st);
cudaError_t sweep_occupancy(int model, int K, bool f32, int block, int smem_bytes, int* blocks_per_sm);
size_t sweep_smem_bytes(int model, int mpb, int rows_smem);
cudaError_t launch_phi_table(double* coef, cudaStream_t st);
cudaError_t launch_prefix_weights(int nr, const double* Wr, double* cw, cudaStream_t st);
cudaError_t launch_math_table(double* t, cudaStream_t st);
int math_table_words();
int phi_table_words();
cudaError_t launch_detection(int model, long long n, const double* F, const ModelConsts& mc, double sigma_F,
                             const double* coef, double* out, cudaStream_t st);
cudaError_t sweep_set_smem(int model, int K, bool f32, int smem_bytes);
cudaError_t launch_prepare(int model, long long n, const double* y_raw, const double* aux_raw, double* y, double* aux,
                           double* chi, double* S, const ModelConsts& mc, const double* theta, int* bad,
                           int set_default_chi, cudaStream_t st);
cudaError_t launch_check_chi(int model, long long n, const double* chi, const double* theta, int* bad,
                             cudaStream_t st);
cudaError_t launch_gauss_legendre(int n, double* x, double* w, cudaStream_t st);
cudaError_t launch_lf_inner(int nr, const double* xr, const double* wr, double r_max, double sigma_F, double* qs,
                            double* Wr, cudaStream_t st);
cudaError_t launch_tables(int p, uint32_t key0, uint32_t key1, long long k0, long long ns, double gamma, double* U,
                          double* u, double* lnu, double* eta, unsigned int* bar, unsigned long long* acc, int nacc,
                          int* err, cudaStream_t st);
cudaError_t launch_eval_logdens(int model, bool f32, long long n, const double* y, const double* aux,
                                const double* chi, const double* theta_dev, const ModelConsts& mc,
                                const double* math_tab, double* out, cudaStream_t st);
cudaError_t launch_eval_etabar(const double* theta_dev, const SweepArgs& rule, unsigned long long* partials,
                               int grid, double* out, cudaStream_t st);
// Builds the H table of a handle's rule (LF, BB1): ncell cells from u = ua; coef receives
// ncell (kHDeg + 1) coefficients, then H(ua) and H(ub) (ub = ua + ncell kHDelta).
cudaError_t launch_htab_build(const SweepArgs& rule, double ua, int ncell, double* coef, cudaStream_t st);

}  // namespace chm
