// Host runtime behind the C ABI of include/cudahm.h: handle ownership, validation,
// device buffers, launch-shape selection, chunked persistent launches, checkpoints.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <cstdarg>
#include <cstdio>
#include <cstddef>
#include <cstring>
#include <string>
#include <vector>

#include "cudahm.h"
#include "internal.h"

using namespace chm;

namespace {

thread_local std::string g_last_error = "no error";

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return code;
}

#define CU(call)                                                                              \
  do {                                                                                        \
    cudaError_t e_ = (call);                                                                  \
    if (e_ != cudaSuccess) return fail(CUDAHM_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

int model_d(int m) { return (m == CUDAHM_MVN3 || m == CUDAHM_NN3) ? 3 : 1; }
// doubles of one member's RAM factor as stored on the device (d = 3: six packed rows)
int factor_words(int d) { return d == 3 ? 6 : 1; }

}  // namespace

int chm::record_error(int code, const char* msg) { return fail(code, "%s", msg); }

namespace {

int model_p(int m) {
  if (m == CUDAHM_NN1) return 2;
  return m == CUDAHM_MVN3 ? 9 : 3;
}

// Inverse of the lower Cholesky factor of the 3x3 covariance C given as its packed lower
// triangle (C00, C10, C11, C20, C21, C22), packed the same way; false unless C is positive
// definite.
bool chol3_inverse(const double* C, double* li) {
  for (int q = 0; q < 6; ++q)
    if (!std::isfinite(C[q])) return false;
  if (!(C[0] > 0.0)) return false;
  const double L00 = std::sqrt(C[0]), L10 = C[1] / L00, L20 = C[3] / L00;
  const double d1 = C[2] - L10 * L10;
  if (!(d1 > 0.0)) return false;
  const double L11 = std::sqrt(d1), L21 = (C[4] - L20 * L10) / L11;
  const double d2 = C[5] - L20 * L20 - L21 * L21;
  if (!(d2 > 0.0)) return false;
  const double L22 = std::sqrt(d2);
  li[0] = 1.0 / L00;
  li[2] = 1.0 / L11;
  li[5] = 1.0 / L22;
  li[1] = -(L10 * li[0]) * li[2];
  li[4] = -(L21 * li[2]) * li[5];
  li[3] = -(L20 * li[0] + L21 * li[1]) * li[5];
  return true;
}
// models with a selection integral, and the positions of their rule sizes in model_consts
bool has_rule(int m) { return m == CUDAHM_LF || m == CUDAHM_BB1; }
int rule_nL(const cudahm_config& c) { return static_cast<int>(c.model_consts[c.model == CUDAHM_BB1 ? 4 : 3]); }
int rule_nr(const cudahm_config& c) { return static_cast<int>(c.model_consts[c.model == CUDAHM_BB1 ? 5 : 4]); }

constexpr long long kChunk = 4096;  // sweeps per persistent launch
// checkpoint layout version: 2 = ChainState with the running-moment and pending theta-update
// fields; 3 = a header of 10 words with a hash of the chain's configuration
constexpr int64_t kCheckpointVersion = 3;
constexpr int kHeaderWords = 10;
constexpr int64_t kCheckpointMagic = 0x4d48414455434f4bll;

// model constants each model reads (the rest of model_consts is unused)
int consts_used(int m) {
  switch (m) {
    case CUDAHM_NN1: return 2;
    case CUDAHM_LF: return 6;
    case CUDAHM_BB1: return 8;
    case CUDAHM_NN3: return 6;
    default: return 0;
  }
}

// FNV-1a hash of everything a chain's continuation depends on besides its state: model, sizes,
// precision, form, seed, the RAM settings and the model constants (the rule sizes and limits
// among them). The start values (theta_init, its proposal scales, chi_init_scale) are not in it:
// a restored checkpoint replaces the state they set.
uint64_t config_hash(const cudahm_config& c) {
  uint64_t h = 1469598103934665603ull;
  auto mix = [&h](const void* p, size_t bytes) {
    const unsigned char* b = static_cast<const unsigned char*>(p);
    for (size_t q = 0; q < bytes; ++q) {
      h ^= b[q];
      h *= 1099511628211ull;
    }
  };
  const int32_t ints[7] = {c.model, c.precision, c.d, c.adapt_theta, c.marginal, c.keep_chi_moments, 0};
  mix(ints, sizeof(ints));
  mix(&c.n, sizeof(c.n));
  mix(&c.seed, sizeof(c.seed));
  mix(&c.target_accept, sizeof(double));
  mix(&c.adapt_exponent, sizeof(double));
  mix(&c.theta_target_accept, sizeof(double));
  mix(c.model_consts, sizeof(double) * consts_used(c.model));
  return h;
}

}  // namespace

struct cudahm {
  cudahm_config cfg{};
  int d = 1, p = 2;
  long long n = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int sms = 0;
  // launch shape
  int grid = 0, block = 256, K = 1, rows_smem = 1, mpb = 1;
  ModelConsts mc{};
  // device buffers
  std::vector<void*> allocs;
  double *y = nullptr, *aux = nullptr, *chi = nullptr, *S = nullptr;
  double *y_raw = nullptr, *aux_raw = nullptr;
  ChainState* chain = nullptr;
  unsigned long long* acc3 = nullptr;  // sweep kernel: grid totals, one buffer per sweep mod 3
  unsigned int* bar = nullptr;
  int* err = nullptr;
  int* bad = nullptr;
  double* theta_dev = nullptr;
  double* eval_out = nullptr;
  double *tab_U = nullptr, *tab_u = nullptr, *tab_lnu = nullptr, *tab_eta = nullptr;
  double* rows = nullptr;
  long long rows_cap = 0;
  long long factor_n = 0;  // doubles of the RAM factors on the device (n * factor_words(d))
  // trace
  long long trace_cap_T = 0;
  double *tr_delta = nullptr, *tr_u = nullptr, *tr_thprop = nullptr, *tr_D = nullptr, *tr_logalpha = nullptr,
         *tr_ut = nullptr, *tr_eb = nullptr;
  uint8_t *tr_acc = nullptr, *tr_tacc = nullptr;
  long long trace_T_last = 0;
  // LF rule
  double *xL = nullptr, *wL = nullptr, *xr = nullptr, *wr = nullptr, *qs = nullptr, *Wr = nullptr;
  double* phi_coef = nullptr;
  double* cw = nullptr;
  float* d32 = nullptr;
  // FP32 form, d = 1: the binary32 latent state (chi holds its binary64 copy for the API; it is
  // refreshed before every read and copied in after every write of chi) and the padded length
  float* chi32 = nullptr;
  float* even32 = nullptr;  // the streaming kernel's even-sweep draws and cached log l_i, [3][n32]
  long long n32 = 0;
  double* math_tab = nullptr;
  double* pub = nullptr;  // theta' published by block 0 of the sweep kernel
  unsigned long long* eb_partials = nullptr;
  int eb_grid = 0, eb_rows_smem = 1;
  // marginal form (latents integrated out by cubature)
  double* marg_lp = nullptr;     // [2][n] log p_i at the current theta and at the proposal
  double* marg_nodes = nullptr;  // panel nodes and weights
  double* marg_d32 = nullptr;    // FP32 form, LF: per-member window data
  double* spare3 = nullptr;      // d = 3, FP64: the odd sweep's Box-Muller sines, [3][n]
  double* mom = nullptr;         // running moments of the latents: two buffers of [mean[d][n], M2[d][n]]
  int mgrid = 0, mrows_smem = 1;
  bool marg_valid = false;       // marg_lp[mcur] holds log p_i at the chain's theta
  // the rule's inner sum H(ln L), tabulated (LF, BB1)
  double* htab = nullptr;
  double h_ua = 0.0, h_ub = 0.0, h_lo = 0.0, h_hi = 0.0;
  int h_ncell = 0;
  // host mirrors
  bool data_set = false;
  bool etabar_valid = false;
  long long sweeps = 0;
  long long rows_last = 0;
  double last_run_ms = 0.0;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  int* host_err = nullptr;  // pinned
  // pinned copy of the last run's kept theta rows, filled in the same synchronisation as the
  // run's error word (rows_host_n rows; capacity rows_host_cap)
  double* rows_host = nullptr;
  long long rows_host_cap = 0, rows_host_n = 0;
  // shard of a population split across devices (cudahm_shard_config): population index of
  // member 0, population size, this shard's part of the selection rule
  bool shard_set = false;
  long long shard_moff = 0, shard_npop = 0;
  int shard_part = 0, shard_parts = 1;
  // the sharded run in progress (cudahm_shard_begin .. cudahm_shard_end): the pass's arguments
  // and progress on the device, its launch shape, and the calls made so far
  bool shard_active = false;
  long long shard_total = 0, shard_passes = 0, shard_decides = 0;
  SweepArgs* sh_pop = nullptr;
  BatchProg* sh_prog = nullptr;
  int* sh_b0 = nullptr;
  int* sh_nb = nullptr;
  unsigned long long* sh_partials = nullptr;
  unsigned int* sh_bar = nullptr;
  unsigned long long* sh_out_last = nullptr;
  int sh_grid = 0, sh_block = 0, sh_smem = 0;

  void* dalloc(size_t bytes) {
    if (bytes == 0) bytes = 16;
    void* ptr = nullptr;
    if (cfg.dev_alloc) {
      ptr = cfg.dev_alloc(bytes, cfg.alloc_ctx);
    } else if (cudaMalloc(&ptr, bytes) != cudaSuccess) {
      ptr = nullptr;
    }
    if (ptr) allocs.push_back(ptr);
    return ptr;
  }
  void dfree(void* ptr) {
    if (!ptr) return;
    auto it = std::find(allocs.begin(), allocs.end(), ptr);
    if (it != allocs.end()) allocs.erase(it);
    if (cfg.dev_free) cfg.dev_free(ptr, cfg.alloc_ctx);
    else cudaFree(ptr);
  }
  ~cudahm() {
    if (stream) cudaStreamSynchronize(stream);
    for (void* ptr : allocs) {
      if (cfg.dev_free) cfg.dev_free(ptr, cfg.alloc_ctx);
      else cudaFree(ptr);
    }
    if (host_err) cudaFreeHost(host_err);
    if (rows_host) cudaFreeHost(rows_host);
    if (ev0) cudaEventDestroy(ev0);
    if (ev1) cudaEventDestroy(ev1);
    if (own_stream && stream) cudaStreamDestroy(stream);
  }
};

namespace {

template <class T>
int alloc_into(cudahm* h, T** out, size_t count) {
  *out = static_cast<T*>(h->dalloc(sizeof(T) * count));
  if (!*out) return fail(CUDAHM_ENOMEM, "device allocation of %zu bytes failed", sizeof(T) * count);
  return CUDAHM_OK;
}

#define TRY(x)                \
  do {                        \
    int r_ = (x);             \
    if (r_ != CUDAHM_OK) return r_; \
  } while (0)

int validate(const cudahm_config* c) {
  if (!c) return fail(CUDAHM_EINVAL, "config is NULL");
  if (c->abi_version != CUDAHM_ABI_VERSION)
    return fail(CUDAHM_EINVAL, "abi_version %u != %u", c->abi_version, CUDAHM_ABI_VERSION);
  if (c->model != CUDAHM_NN1 && c->model != CUDAHM_LF && c->model != CUDAHM_MVN3 && c->model != CUDAHM_BB1 &&
      c->model != CUDAHM_NN3)
    return fail(CUDAHM_EINVAL, "unknown model %d", c->model);
  if (c->precision != CUDAHM_FP64 && c->precision != CUDAHM_FP32)
    return fail(CUDAHM_EINVAL, "unknown precision %d", c->precision);
  if (c->d != model_d(c->model)) return fail(CUDAHM_EINVAL, "d = %d does not match the model", c->d);
  if (c->n < 1 || c->n > (1ll << 31)) return fail(CUDAHM_EINVAL, "n = %lld out of range [1, 2^31]", (long long)c->n);
  if (!(c->target_accept > 0.0 && c->target_accept < 1.0)) return fail(CUDAHM_EINVAL, "target_accept not in (0,1)");
  if (!(c->theta_target_accept > 0.0 && c->theta_target_accept < 1.0))
    return fail(CUDAHM_EINVAL, "theta_target_accept not in (0,1)");
  if (!(c->adapt_exponent > 0.5 && c->adapt_exponent <= 1.0))
    return fail(CUDAHM_EINVAL, "adapt_exponent must lie in (1/2, 1]");
  if (!(c->chi_init_scale > 0.0) || !std::isfinite(c->chi_init_scale))
    return fail(CUDAHM_EINVAL, "chi_init_scale must be positive");
  if ((c->dev_alloc == nullptr) != (c->dev_free == nullptr))
    return fail(CUDAHM_EINVAL, "dev_alloc and dev_free must be given together");
  if (c->block_threads != 0 && c->block_threads != 128 && c->block_threads != 256)
    return fail(CUDAHM_EINVAL, "block_threads must be 0, 128 or 256");
  if (c->trace_sweeps < 0) return fail(CUDAHM_EINVAL, "trace_sweeps < 0");
  const int p = model_p(c->model);
  for (int q = 0; q < p; ++q) {
    if (!std::isfinite(c->theta_init[q])) return fail(CUDAHM_EINVAL, "theta_init[%d] not finite", q);
    if (!(c->theta_prop_scale[q] >= 0.0) || !std::isfinite(c->theta_prop_scale[q]))
      return fail(CUDAHM_EINVAL, "theta_prop_scale[%d] must be >= 0", q);
  }
  if (c->adapt_theta) {
    for (int q = 0; q < p; ++q)
      if (!(c->theta_prop_scale[q] > 0.0))
        return fail(CUDAHM_EINVAL, "adapt_theta needs theta_prop_scale[%d] > 0", q);
  }
  const double* k = c->model_consts;
  if (c->model == CUDAHM_NN1) {
    if (!(k[0] < k[1])) return fail(CUDAHM_EINVAL, "NN1 prior range needs consts[0] < consts[1]");
    if (!(c->theta_init[1] >= k[0] && c->theta_init[1] <= k[1]))
      return fail(CUDAHM_EINVAL, "theta_init outside the NN1 prior");
  } else if (c->model == CUDAHM_LF) {
    if (!(k[0] > 0.0) || !(k[1] > 0.0) || !(k[2] > 0.0)) return fail(CUDAHM_EINVAL, "LF needs sigma_F, F_th, r_max > 0");
    const double nL = k[3], nr = k[4];
    if (!(nL >= 1 && nL <= 4096 && nL == std::floor(nL)) || !(nr >= 1 && nr <= 4096 && nr == std::floor(nr)))
      return fail(CUDAHM_EINVAL, "LF rule sizes must be integers in [1, 4096]");
    if (!(k[5] > 0.0)) return fail(CUDAHM_EINVAL, "LF upper limit ln(upper/L*) must be > 0");
    const double* t = c->theta_init;
    if (!(t[0] > -2.0 && t[0] < 0.0 && t[2] < t[1])) return fail(CUDAHM_EINVAL, "theta_init outside the LF prior");
  } else if (c->model == CUDAHM_BB1) {
    if (c->precision != CUDAHM_FP64) return fail(CUDAHM_EUNSUPPORTED, "BB1 has the FP64 form only");
    if (!(k[0] > 0.0) || !(k[1] >= 0.0 && k[1] < 1.0) || !(k[2] > 0.0) || !(k[3] > 0.0))
      return fail(CUDAHM_EINVAL, "BB1 needs sigma0 > 0, 0 <= alpha < 1, nu > 0, r_max > 0");
    const double nL = k[4], nr = k[5];
    if (!(nL >= 1 && nL <= 4096 && nL == std::floor(nL)) || !(nr >= 1 && nr <= 4096 && nr == std::floor(nr)))
      return fail(CUDAHM_EINVAL, "BB1 rule sizes must be integers in [1, 4096]");
    if (!(k[6] > 0.0) || !(k[7] < 0.0)) return fail(CUDAHM_EINVAL, "BB1 rule limits need ln(upper/u) > 0 > ln(lower/l)");
    const double* t = c->theta_init;
    if (!(t[0] > -2.0 && t[0] < 0.0 && t[1] < t[2])) return fail(CUDAHM_EINVAL, "theta_init outside the BB1 prior");
  } else if (c->model == CUDAHM_NN3) {
    double li[6];
    if (!chol3_inverse(k, li)) return fail(CUDAHM_EINVAL, "NN3 needs a positive definite C_pop in consts[0..5]");
  }
  if (c->marginal != 0 && c->marginal != 1) return fail(CUDAHM_EINVAL, "marginal must be 0 or 1");
  if (c->keep_chi_moments != 0 && c->keep_chi_moments != 1) return fail(CUDAHM_EINVAL, "keep_chi_moments must be 0 or 1");
  if (c->keep_chi_moments && c->marginal) return fail(CUDAHM_EINVAL, "the marginal form has no latents to keep moments of");
  if (c->marginal) {
    if (c->model != CUDAHM_NN1 && c->model != CUDAHM_LF && c->model != CUDAHM_BB1)
      return fail(CUDAHM_EUNSUPPORTED, "the marginal form integrates one-dimensional latents (NN1, LF, BB1)");
    if (c->model == CUDAHM_BB1 && !(k[1] * kMargK < 1.0))
      return fail(CUDAHM_EUNSUPPORTED, "the BB1 marginal window needs alpha < 1/10");
  }
  return CUDAHM_OK;
}

int choose_shape(cudahm* h) {
  const int block = h->cfg.block_threads ? h->cfg.block_threads : 256;
  h->block = block;
  const long long n = h->n;
  const int model = h->cfg.model;
  const bool lf = has_rule(model);
  const bool f32 = (h->cfg.precision == CUDAHM_FP32);
  // selection rule: segments of 128 inner nodes, G = n_L * ceil(n_r / 128), dealt round-robin
  const long long G = lf ? static_cast<long long>(rule_nL(h->cfg)) * ((static_cast<long long>(rule_nr(h->cfg)) + 127) / 128)
                         : 0;
  const int Ks[4] = {1, 2, 4, 8};
  // the d = 3 model always streams its member state through the batched kernel
  for (int ki = (model_d(model) == 3 ? 4 : 0); ki < 4 && h->grid == 0; ++ki) {
    const int K = Ks[ki];
    // the grid depends on the occupancy, which depends on the shared memory, which depends on
    // the grid: iterate from the register-limited occupancy down until it is consistent
    int bps = 0;
    CU(sweep_occupancy(model, K, f32, block, 0, &bps));
    for (; bps >= 1; --bps) {
      int grid = lf ? bps * h->sms
                    : static_cast<int>(std::min<long long>(static_cast<long long>(bps) * h->sms,
                                                           (n + block - 1) / block));
      const int mgrid = (grid > 1) ? grid - 1 : grid;  // block 0 holds no members
      const long long mpb = (n + mgrid - 1) / mgrid;           // members of the largest block
      if ((mpb + block - 1) / block > K) break;     // needs a larger K
      const int rows = lf ? static_cast<int>((G + grid - 1) / grid) : 1;
      const size_t smem = sweep_smem_bytes(model, static_cast<int>(mpb), rows);
      if (smem > 200 * 1024) break;
      int fit = 0;
      CU(sweep_occupancy(model, K, f32, block, static_cast<int>(smem), &fit));
      if (fit * h->sms >= grid) {
        CU(sweep_set_smem(model, K, f32, static_cast<int>(smem)));
        h->K = K;
        h->grid = grid;
        h->mpb = static_cast<int>(mpb);
        h->rows_smem = rows;
        break;
      }
    }
  }
  // Too many members to keep in registers: cudahm_run streams the state through the batched
  // kernel (a batch of one) instead; K = 0 marks that.
  if (h->grid == 0) h->K = 0;
  if (lf) {
    h->eb_grid = 4 * h->sms;
    h->eb_rows_smem = static_cast<int>((G + h->eb_grid - 1) / h->eb_grid);
  }
  return CUDAHM_OK;
}

// Launch shape of the marginal kernel: a cooperative grid of whole SMs (LF: the selection rule
// spreads over every block), at most one block per 256 members for NN1.
int choose_marg_shape(cudahm* h) {
  const int model = h->cfg.model;
  const bool lf = has_rule(model);
  const long long G = lf ? static_cast<long long>(rule_nL(h->cfg)) * ((static_cast<long long>(rule_nr(h->cfg)) + 127) / 128)
                         : 0;
  for (int bps = 2; bps >= 1 && h->mgrid == 0; --bps) {
    const int grid = lf ? bps * h->sms
                        : static_cast<int>(std::min<long long>(static_cast<long long>(bps) * h->sms, (h->n + 255) / 256));
    const int rows = lf ? static_cast<int>((G + grid - 1) / grid) : 1;
    const size_t smem = marg_smem_bytes(model, rows);
    if (smem > 200 * 1024) continue;
    int fit = 0;
    CU(marg_occupancy(model, h->cfg.precision == CUDAHM_FP32, 256, static_cast<int>(smem), &fit));
    if (fit * h->sms >= grid) {
      h->mgrid = grid;
      h->mrows_smem = rows;
    }
  }
  if (h->mgrid == 0) return fail(CUDAHM_EUNSUPPORTED, "no launch shape fits the marginal kernel");
  return CUDAHM_OK;
}

SweepArgs base_args(cudahm* h) {
  SweepArgs a{};
  a.model = h->cfg.model;
  a.f32 = (h->cfg.precision == CUDAHM_FP32) ? 1 : 0;
  a.p = h->p;
  a.n = h->n;
  a.y = h->y;
  a.aux = h->aux;
  a.chi = h->chi;
  a.S = h->S;
  a.chain = h->chain;
  a.partials = nullptr;  // per-block partials belong to the batched launch (BatchBufs)
  a.acc3 = h->acc3;
  a.bar = h->bar;
  a.err = h->err;
  a.astar = h->cfg.target_accept;
  a.astar_theta = h->cfg.theta_target_accept;
  a.adapt_theta = h->cfg.adapt_theta;
  a.key0 = static_cast<uint32_t>(h->cfg.seed & 0xffffffffull);
  a.key1 = static_cast<uint32_t>(h->cfg.seed >> 32);
  a.mc = h->mc;
  a.xL = h->xL;
  a.wL = h->wL;
  a.qs = h->qs;
  a.Wr = h->Wr;
  a.phi_coef = h->phi_coef;
  a.cw = h->cw;
  a.math_tab = h->math_tab;
  a.pub = h->pub;
  a.nL = has_rule(h->cfg.model) ? rule_nL(h->cfg) : 0;
  a.nr = has_rule(h->cfg.model) ? rule_nr(h->cfg) : 0;
  a.rows_smem = h->rows_smem;
  a.mpb = h->mpb;
  a.timeout_ns = h->cfg.barrier_timeout_ns > 0 ? h->cfg.barrier_timeout_ns : 2000000000ll;
  a.skip_cta = h->cfg.debug_skip_barrier_cta;
  a.gamma = h->cfg.adapt_exponent;
  a.d32 = h->d32;
  a.chi32 = h->chi32;
  a.even32 = h->even32;
  a.n32 = h->n32;
  a.tab_U = h->tab_U;
  a.tab_u = h->tab_u;
  a.tab_lnu = h->tab_lnu;
  a.tab_eta = h->tab_eta;
  a.marg_lp = h->marg_lp;
  a.marg_nodes = h->marg_nodes;
  a.marg_d32 = h->marg_d32;
  a.spare3 = h->spare3;
  a.mom = h->mom;
  a.htab = h->htab;
  a.h_ua = h->h_ua;
  a.h_ub = h->h_ub;
  a.h_lo = h->h_lo;
  a.h_hi = h->h_hi;
  a.h_ncell = h->h_ncell;
  return a;
}

// Tabulates the rule's inner sum H(u), u = ln L (LF, BB1), once per handle. Range: below
// ua = ln(2^-56 F_th/q_max) every x_k equals its value at L = 0 to rounding, so H is constant;
// above ub every pair has x >= 8.5 (Phi = 1; LF: L q_min >= F_th + 8.5 sigma_F, BB1:
// L q_min >= F_pre), or, for BB1 when x never reaches 8.5, x has reached its limit 1/alpha to
// rounding (L q_min >= 2^56 F_th).
// Set-up tables computed on the device once per process and then kept on the host: a handle
// that needs a table already computed (a Gauss-Legendre rule of the same size, the tabulated
// inner sum of the same selection rule) gets it by a host-to-device copy instead of the kernels
// (about half a millisecond per 1024-node rule, 0.4 ms per tabulated rule: a served request
// creates its handle on the request's path). The values are the ones the kernels gave, bit for
// bit. At most kTabCacheMax tables are kept (the cache starts over when full).
constexpr size_t kTabCacheMax = 256;
std::mutex g_tab_mu;
std::map<std::string, std::vector<double>> g_tab_cache;

std::string tab_key(const char* kind, int model, const double* v, int nv, long long extra) {
  std::string k(kind);
  k.append(reinterpret_cast<const char*>(&model), sizeof(model));
  k.append(reinterpret_cast<const char*>(&extra), sizeof(extra));
  k.append(reinterpret_cast<const char*>(v), sizeof(double) * static_cast<size_t>(nv));
  return k;
}
bool tab_get(const std::string& key, std::vector<double>& out) {
  std::lock_guard<std::mutex> lk(g_tab_mu);
  auto it = g_tab_cache.find(key);
  if (it == g_tab_cache.end()) return false;
  out = it->second;
  return true;
}
void tab_put(const std::string& key, std::vector<double> v) {
  std::lock_guard<std::mutex> lk(g_tab_mu);
  if (g_tab_cache.size() >= kTabCacheMax) g_tab_cache.clear();
  g_tab_cache[key] = std::move(v);
}

// n-node Gauss-Legendre rule on [-1, 1] into x, w (device)
int gl_rule(cudahm* h, int n, double* x, double* w) {
  const std::string key = tab_key("gl", 0, nullptr, 0, n);
  std::vector<double> v;
  if (tab_get(key, v)) {
    CU(cudaMemcpyAsync(x, v.data(), sizeof(double) * n, cudaMemcpyHostToDevice, h->stream));
    CU(cudaMemcpyAsync(w, v.data() + n, sizeof(double) * n, cudaMemcpyHostToDevice, h->stream));
    CU(cudaStreamSynchronize(h->stream));  // the host copy is not pinned
    return CUDAHM_OK;
  }
  CU(launch_gauss_legendre(n, x, w, h->stream));
  v.resize(2 * static_cast<size_t>(n));
  CU(cudaMemcpyAsync(v.data(), x, sizeof(double) * n, cudaMemcpyDeviceToHost, h->stream));
  CU(cudaMemcpyAsync(v.data() + n, w, sizeof(double) * n, cudaMemcpyDeviceToHost, h->stream));
  CU(cudaStreamSynchronize(h->stream));
  tab_put(key, std::move(v));
  return CUDAHM_OK;
}

int build_htab(cudahm* h) {
  // cached: [ua, ub, h_lo, h_hi, ncell, coefficients of every cell, the two end values]
  const std::string key = tab_key("htab", h->cfg.model, h->cfg.model_consts, consts_used(h->cfg.model), 0);
  {
    std::vector<double> v;
    if (tab_get(key, v)) {
      const int ncell = static_cast<int>(v[4]);
      const size_t words = static_cast<size_t>(ncell) * (kHDeg + 1) + 2;
      TRY(alloc_into(h, &h->htab, words));
      CU(cudaMemcpyAsync(h->htab, v.data() + 5, sizeof(double) * words, cudaMemcpyHostToDevice, h->stream));
      CU(cudaStreamSynchronize(h->stream));
      h->h_ua = v[0];
      h->h_ub = v[1];
      h->h_lo = v[2];
      h->h_hi = v[3];
      h->h_ncell = ncell;
      return CUDAHM_OK;
    }
  }
  const int nr = rule_nr(h->cfg);
  std::vector<double> qs(static_cast<size_t>(nr));
  CU(cudaMemcpyAsync(qs.data(), h->qs, sizeof(double) * nr, cudaMemcpyDeviceToHost, h->stream));
  CU(cudaStreamSynchronize(h->stream));
  double qmin = qs[0], qmax = qs[0];
  for (double v : qs) {
    qmin = std::min(qmin, v);
    qmax = std::max(qmax, v);
  }
  if (!(qmin > 0.0) || !std::isfinite(qmax)) return fail(CUDAHM_EINVAL, "rule distances give no positive flux factors");
  const bool bb1 = h->cfg.model == CUDAHM_BB1;
  double ua, ub;
  if (bb1) {
    const double Fth = h->mc.F_th;
    ua = std::log(std::ldexp(Fth, -56) / qmax);
    ub = std::isfinite(h->mc.F_pre) ? std::log(h->mc.F_pre / qmin) : std::log(std::ldexp(Fth, 56) / qmin);
  } else {  // qs = q/sigma_F, x = L qs - F_th/sigma_F
    ua = std::log(std::ldexp(h->mc.cth, -56) / qmax);
    ub = std::log((h->mc.cth + 8.5) / qmin);
  }
  ub += 1e-9;
  const int ncell = static_cast<int>(std::ceil((ub - ua) / kHDelta));
  if (ncell < 1 || ncell > (1 << 16)) return fail(CUDAHM_EINVAL, "selection rule range too wide to tabulate");
  TRY(alloc_into(h, &h->htab, static_cast<size_t>(ncell) * (kHDeg + 1) + 2));
  SweepArgs r = base_args(h);
  CU(launch_htab_build(r, ua, ncell, h->htab, h->stream));
  double ends[2];
  CU(cudaMemcpyAsync(ends, h->htab + static_cast<size_t>(ncell) * (kHDeg + 1), sizeof(ends), cudaMemcpyDeviceToHost,
                     h->stream));
  CU(cudaStreamSynchronize(h->stream));
  h->h_ua = ua;
  h->h_ub = ua + kHDelta * ncell;
  h->h_lo = ends[0];
  h->h_hi = ends[1];
  h->h_ncell = ncell;
  const size_t words = static_cast<size_t>(ncell) * (kHDeg + 1) + 2;
  std::vector<double> v(5 + words);
  v[0] = h->h_ua;
  v[1] = h->h_ub;
  v[2] = h->h_lo;
  v[3] = h->h_hi;
  v[4] = ncell;
  CU(cudaMemcpyAsync(v.data() + 5, h->htab, sizeof(double) * words, cudaMemcpyDeviceToHost, h->stream));
  CU(cudaStreamSynchronize(h->stream));
  tab_put(key, std::move(v));
  return CUDAHM_OK;
}

// Cost (FP64-pipe operations per sweep) of one population, for the batched allocation.
double pop_cost(const cudahm* h) {
  const bool f32 = h->cfg.precision == CUDAHM_FP32;
  double c = 3000.0 + static_cast<double>(h->n) * (h->d == 3 ? (f32 ? 80.0 : 260.0) : (f32 ? 20.0 : 120.0));
  if (has_rule(h->cfg.model)) c += 80.0 * rule_nL(h->cfg);  // one table lookup per outer node
  return c;
}

// Blocks per population proportional to cost (at least one each), total <= grid: the next
// block always goes to the population with the largest cost per block.
std::vector<int> allocate_blocks(const std::vector<double>& cost, const std::vector<int>& cap, int grid) {
  const int k = static_cast<int>(cost.size());
  std::vector<int> nb(k, 1);
  int used = k;
  while (used < grid) {
    int best = -1;
    double bw = -1.0;
    for (int q = 0; q < k; ++q) {
      if (nb[q] >= cap[q]) continue;
      const double w = cost[q] / nb[q];
      if (w > bw) {
        bw = w;
        best = q;
      }
    }
    if (best < 0) break;
    nb[best]++;
    used++;
  }
  return nb;
}

int reset_chain(cudahm* h) {
  ChainState cs{};
  for (int q = 0; q < h->p; ++q) cs.theta[q] = h->cfg.theta_init[q];
  for (int q = 0; q < h->p; ++q) cs.S_theta[q * h->p + q] = h->cfg.theta_prop_scale[q];
  CU(cudaMemcpyAsync(h->chain, &cs, sizeof(cs), cudaMemcpyHostToDevice, h->stream));
  if (h->mom) CU(cudaMemsetAsync(h->mom, 0, sizeof(double) * 4 * h->d * static_cast<size_t>(h->n), h->stream));
  CU(cudaStreamSynchronize(h->stream));
  h->sweeps = 0;
  h->rows_last = 0;
  h->rows_host_n = 0;
  h->etabar_valid = false;
  h->marg_valid = false;
  return CUDAHM_OK;
}

int read_err(cudahm* h, int* code) {
  CU(cudaMemcpyAsync(h->host_err, h->err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  CU(cudaStreamSynchronize(h->stream));
  *code = *h->host_err;
  return CUDAHM_OK;
}

// Lockstep trace buffers for the first T sweeps of a run.
int ensure_trace(cudahm* h, long long T) {
  if (T <= h->trace_cap_T) return CUDAHM_OK;
  for (void** q : {(void**)&h->tr_delta, (void**)&h->tr_u, (void**)&h->tr_acc, (void**)&h->tr_thprop, (void**)&h->tr_D,
                   (void**)&h->tr_logalpha, (void**)&h->tr_ut, (void**)&h->tr_tacc, (void**)&h->tr_eb}) {
    h->dfree(*q);
    *q = nullptr;
  }
  h->trace_cap_T = 0;
  const size_t tn = static_cast<size_t>(T) * (h->cfg.marginal ? 1 : h->n);  // no member trace when marginal
  TRY(alloc_into(h, &h->tr_delta, tn));
  TRY(alloc_into(h, &h->tr_u, tn));
  TRY(alloc_into(h, &h->tr_acc, tn));
  TRY(alloc_into(h, &h->tr_thprop, static_cast<size_t>(T) * h->p));
  TRY(alloc_into(h, &h->tr_D, T));
  TRY(alloc_into(h, &h->tr_logalpha, T));
  TRY(alloc_into(h, &h->tr_ut, T));
  TRY(alloc_into(h, &h->tr_tacc, T));
  TRY(alloc_into(h, &h->tr_eb, T));
  h->trace_cap_T = T;
  return CUDAHM_OK;
}

int compute_etabar_into(cudahm* h, const double* theta_dev, double* out_dev) {
  SweepArgs r = base_args(h);
  r.rows_smem = h->eb_rows_smem;
  CU(launch_eval_etabar(theta_dev, r, h->eb_partials, h->eb_grid, out_dev, h->stream));
  return CUDAHM_OK;
}

// FP32 form with d = 1: the binary32 latents are the state
bool has_chi32(const cudahm* h) { return h->chi32 != nullptr; }
// chi (binary64 copy) -> chi32 after chi was written
int chi_to_state(cudahm* h) {
  if (has_chi32(h)) CU(launch_chi_to32(h->n, h->n32, h->chi, h->chi32, h->stream));
  return CUDAHM_OK;
}
// chi32 -> chi before chi is read
int chi_from_state(cudahm* h) {
  if (has_chi32(h)) CU(launch_chi_from32(h->n, h->chi32, h->chi, h->stream));
  return CUDAHM_OK;
}

int prepare(cudahm* h, const double* y_dev_raw, const double* aux_dev_raw, int set_default) {
  CU(cudaMemsetAsync(h->bad, 0, sizeof(int), h->stream));
  CU(launch_prepare(h->cfg.model, h->n, y_dev_raw, aux_dev_raw, h->y, h->aux, h->chi, h->S, h->mc, h->cfg.theta_init,
                    h->bad, set_default, h->stream));
  int bad = 0;
  CU(cudaMemcpyAsync(h->host_err, h->bad, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  CU(cudaStreamSynchronize(h->stream));
  bad = *h->host_err;
  if (bad)
    return fail(CUDAHM_EINVAL, "%d members have non-finite data or a non-positive scale (or, marginal LF, flux)", bad);
  if (set_default) TRY(chi_to_state(h));
  if (h->cfg.precision == CUDAHM_FP32) {  // binary32 member data for the batched FP32 form
    if (!h->d32) TRY(alloc_into(h, &h->d32, static_cast<size_t>(data32_words(h->cfg.model)) * h->n32));
    CU(launch_data32(h->cfg.model, h->n, h->n32, h->y, h->aux, h->mc, h->d32, h->stream));
    if (h->cfg.marginal && h->cfg.model == CUDAHM_LF) {  // the FP32 marginal form's window data
      if (!h->marg_d32) TRY(alloc_into(h, &h->marg_d32, static_cast<size_t>(kMarg32Words) * h->n));
      CU(launch_marg_data32(h->n, h->y, h->aux, h->mc, h->math_tab, h->marg_d32, h->stream));
    }
  }
  TRY(reset_chain(h));
  h->data_set = true;
  return CUDAHM_OK;
}

}  // namespace

extern "C" {

void cudahm_config_init(cudahm_config* cfg, int32_t model, int64_t n) {
  if (!cfg) return;
  std::memset(cfg, 0, sizeof(*cfg));
  cfg->abi_version = CUDAHM_ABI_VERSION;
  cfg->model = model;
  cfg->precision = CUDAHM_FP64;
  cfg->d = model_d(model);
  cfg->n = n;
  cfg->seed = 1;
  cfg->target_accept = 0.4;
  cfg->adapt_exponent = 2.0 / 3.0;
  cfg->chi_init_scale = 1.0;
  cfg->theta_target_accept = 0.4;
  cfg->adapt_theta = 1;
  for (int q = 0; q < CUDAHM_MAX_P; ++q) cfg->theta_prop_scale[q] = 0.01;
  if (model == CUDAHM_NN1) {
    cfg->model_consts[0] = -10.0;
    cfg->model_consts[1] = 10.0;
  } else if (model == CUDAHM_LF) {
    cfg->model_consts[3] = 1024;
    cfg->model_consts[4] = 1024;
    cfg->model_consts[5] = std::log(60.0);
  } else if (model == CUDAHM_BB1) {
    cfg->model_consts[4] = 1024;
    cfg->model_consts[5] = 1024;
    cfg->model_consts[6] = std::log(60.0);
    cfg->model_consts[7] = -40.0;
  }
  cfg->device = 0;
  cfg->debug_skip_barrier_cta = -1;
}

const char* cudahm_last_error(void) { return g_last_error.c_str(); }

size_t cudahm_sizeof_config(void) { return sizeof(cudahm_config); }
size_t cudahm_sizeof_stats(void) { return sizeof(cudahm_stats); }

int cudahm_create(const cudahm_config* cfg, cudahm_t* out) {
  if (!out) return fail(CUDAHM_EINVAL, "out is NULL");
  TRY(validate(cfg));
  int ndev = 0;
  CU(cudaGetDeviceCount(&ndev));
  if (cfg->device < 0 || cfg->device >= ndev) return fail(CUDAHM_EINVAL, "device %d not present", cfg->device);
  CU(cudaSetDevice(cfg->device));
  int coop = 0;
  CU(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, cfg->device));
  if (!coop) return fail(CUDAHM_EUNSUPPORTED, "device has no cooperative launch");

  cudahm* h = new cudahm();
  h->cfg = *cfg;
  h->d = cfg->d;
  h->p = model_p(cfg->model);
  h->n = cfg->n;
  auto bail = [&](int code) {
    delete h;
    return code;
  };
  if (cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, cfg->device) != cudaSuccess)
    return bail(fail(CUDAHM_ECUDA, "cannot query SM count"));
  if (cfg->cuda_stream) {
    h->stream = static_cast<cudaStream_t>(cfg->cuda_stream);
  } else {
    if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess)
      return bail(fail(CUDAHM_ECUDA, "cannot create a stream"));
    h->own_stream = true;
  }
  if (cudaHostAlloc(reinterpret_cast<void**>(&h->host_err), sizeof(int) * 4, cudaHostAllocDefault) != cudaSuccess)
    return bail(fail(CUDAHM_ECUDA, "cannot allocate pinned host memory"));
  if (cudaEventCreate(&h->ev0) != cudaSuccess || cudaEventCreate(&h->ev1) != cudaSuccess)
    return bail(fail(CUDAHM_ECUDA, "cannot create events"));

  // model constants
  const double* k = cfg->model_consts;
  h->mc.chi_init_scale = cfg->chi_init_scale;
  h->mc.F_pre = INFINITY;
  if (cfg->model == CUDAHM_NN1) {
    h->mc.lo = k[0];
    h->mc.hi = k[1];
  } else if (cfg->model == CUDAHM_LF) {
    h->mc.sigF = k[0];
    h->mc.inv2sig2 = 1.0 / (2.0 * k[0] * k[0]);
    h->mc.cth = k[1] / k[0];
    h->mc.F_th = k[1];
    h->mc.ln_upper = k[5];
  } else if (cfg->model == CUDAHM_BB1) {
    const double s0 = k[0], al = k[1], nu = k[2];
    h->mc.s0sq = s0 * s0;
    h->mc.alpha = al;
    h->mc.F_th = nu * s0 / std::sqrt(1.0 - al * al);  // eq. Fth
    // F where (F - F_th)/sigma(F) = 8.5: (1 - 72.25 alpha^2) F^2 - 2 F_th F + F_th^2 - 72.25 sigma0^2 = 0
    const double A = 1.0 - 72.25 * al * al;
    if (A > 0.0) {
      const double Ft = h->mc.F_th;
      h->mc.F_pre = (Ft + std::sqrt(72.25 * (al * al * Ft * Ft + A * s0 * s0))) / A;
    }
    h->mc.ln_upper = k[6];
    h->mc.ln_lower = k[7];
  } else if (cfg->model == CUDAHM_NN3) {
    chol3_inverse(k, h->mc.li3);
  }
  h->mc.marginal = cfg->marginal;
  int rc = choose_shape(h);
  if (rc != CUDAHM_OK) return bail(rc);
  if (cfg->marginal && (rc = choose_marg_shape(h)) != CUDAHM_OK) return bail(rc);

  const long long n = h->n;
  const int p = h->p;
  h->factor_n = n * factor_words(h->d);
  // FP32 form, d = 1: member arrays padded to whole aligned tiles (bulk copies stay in bounds)
  const bool tiled = cfg->precision == CUDAHM_FP32 && h->d == 1 && !cfg->marginal;
  h->n32 = tiled ? (n + kTilePad - 1) / kTilePad * kTilePad : n;
  if ((rc = alloc_into(h, &h->y, n * h->d)) || (rc = alloc_into(h, &h->aux, n * h->d)) ||
      (rc = alloc_into(h, &h->chi, n * h->d)) ||
      (rc = alloc_into(h, &h->S, tiled ? h->n32 : h->factor_n)) ||
      (tiled && (rc = alloc_into(h, &h->chi32, h->n32))) ||
      (tiled && (rc = alloc_into(h, &h->even32, 3 * h->n32))) ||
      (rc = alloc_into(h, &h->chain, 1)) ||
      (rc = alloc_into(h, &h->acc3, 3ull * kAccWords)) ||
      (rc = alloc_into(h, &h->bar, 4)) ||
      (rc = alloc_into(h, &h->err, 4)) || (rc = alloc_into(h, &h->bad, 4)) ||
      (rc = alloc_into(h, &h->theta_dev, kMaxP)) || (rc = alloc_into(h, &h->eval_out, 4)) ||
      (rc = alloc_into(h, &h->tab_U, kChunk * p)) || (rc = alloc_into(h, &h->tab_u, kChunk)) ||
      (rc = alloc_into(h, &h->tab_lnu, kChunk)) ||
      (rc = alloc_into(h, &h->math_tab, static_cast<size_t>(math_table_words()))) ||
      (rc = alloc_into(h, &h->pub, static_cast<size_t>(kPubWords) * kPubSlots)) ||
      (rc = alloc_into(h, &h->tab_eta, kChunk)))
    return bail(rc);
  if (has_rule(cfg->model)) {
    const int nL = rule_nL(*cfg), nr = rule_nr(*cfg);
    const bool bb1 = cfg->model == CUDAHM_BB1;
    const double r_max = bb1 ? k[3] : k[2], sigma_F = bb1 ? 1.0 : k[0];  // BB1 keeps q_k itself
    if ((rc = alloc_into(h, &h->xL, nL)) || (rc = alloc_into(h, &h->wL, nL)) || (rc = alloc_into(h, &h->xr, nr)) ||
        (rc = alloc_into(h, &h->wr, nr)) || (rc = alloc_into(h, &h->qs, nr)) || (rc = alloc_into(h, &h->Wr, nr)) ||
        (rc = alloc_into(h, &h->eb_partials, 4ull * h->eb_grid)) ||
        (rc = alloc_into(h, &h->phi_coef, static_cast<size_t>(phi_table_words()))) ||
        (rc = alloc_into(h, &h->cw, static_cast<size_t>(nr) + 1)))
      return bail(rc);
    if (launch_phi_table(h->phi_coef, h->stream) != cudaSuccess)
      return bail(fail(CUDAHM_ECUDA, "normal-CDF table set-up failed: %s", cudaGetErrorString(cudaGetLastError())));
    if ((rc = gl_rule(h, nL, h->xL, h->wL)) != CUDAHM_OK || (rc = gl_rule(h, nr, h->xr, h->wr)) != CUDAHM_OK)
      return bail(rc);
    if (launch_lf_inner(nr, h->xr, h->wr, r_max, sigma_F, h->qs, h->Wr, h->stream) != cudaSuccess ||
        launch_prefix_weights(nr, h->Wr, h->cw, h->stream) != cudaSuccess)
      return bail(fail(CUDAHM_ECUDA, "quadrature set-up failed: %s", cudaGetErrorString(cudaGetLastError())));
    if ((rc = build_htab(h)) != CUDAHM_OK) return bail(rc);
  }
  if (launch_math_table(h->math_tab, h->stream) != cudaSuccess)
    return bail(fail(CUDAHM_ECUDA, "exp/log table set-up failed: %s", cudaGetErrorString(cudaGetLastError())));
  if (h->d == 3 && cfg->precision == CUDAHM_FP64 && (rc = alloc_into(h, &h->spare3, 3ull * n))) return bail(rc);
  if (cfg->keep_chi_moments && (rc = alloc_into(h, &h->mom, 4ull * h->d * n))) return bail(rc);
  if (cfg->model == CUDAHM_NN1 || cfg->model == CUDAHM_LF || cfg->model == CUDAHM_BB1) {  // the cubature rule
    if ((rc = alloc_into(h, &h->marg_nodes, kMargNodeWords))) return bail(rc);
    if (cfg->marginal && (rc = alloc_into(h, &h->marg_lp, 2ull * n))) return bail(rc);
    if (launch_marg_nodes(h->marg_nodes, h->stream) != cudaSuccess)
      return bail(fail(CUDAHM_ECUDA, "cubature set-up failed: %s", cudaGetErrorString(cudaGetLastError())));
  }
  if (cudaMemsetAsync(h->err, 0, sizeof(int), h->stream) != cudaSuccess ||
      cudaStreamSynchronize(h->stream) != cudaSuccess)
    return bail(fail(CUDAHM_ECUDA, "initialisation failed"));
  if ((rc = reset_chain(h)) != CUDAHM_OK) return bail(rc);
  *out = h;
  return CUDAHM_OK;
}

void cudahm_destroy(cudahm_t h) { delete h; }

static int set_data_impl(cudahm_t h, const double* y, const double* aux, int64_t n, cudaMemcpyKind kind) {
  if (!h) return fail(CUDAHM_EINVAL, "handle is NULL");
  if (!y || !aux) return fail(CUDAHM_EINVAL, "data pointers are NULL");
  if (n != h->n) return fail(CUDAHM_EINVAL, "n = %lld but the handle has %lld members", (long long)n, h->n);
  CU(cudaSetDevice(h->cfg.device));
  const size_t cnt = static_cast<size_t>(h->n) * h->d;
  if (!h->y_raw) {
    TRY(alloc_into(h, &h->y_raw, cnt));
    TRY(alloc_into(h, &h->aux_raw, cnt));
  }
  CU(cudaMemcpyAsync(h->y_raw, y, sizeof(double) * cnt, kind, h->stream));
  CU(cudaMemcpyAsync(h->aux_raw, aux, sizeof(double) * cnt, kind, h->stream));
  return prepare(h, h->y_raw, h->aux_raw, 1);
}

int cudahm_set_data(cudahm_t h, const double* y_host, const double* aux_host, int64_t n) {
  return set_data_impl(h, y_host, aux_host, n, cudaMemcpyHostToDevice);
}

int cudahm_set_data_device(cudahm_t h, const double* y_dev, const double* aux_dev, int64_t n) {
  return set_data_impl(h, y_dev, aux_dev, n, cudaMemcpyDeviceToDevice);
}

int cudahm_set_chi(cudahm_t h, const double* chi_host, int64_t n) {
  if (!h) return fail(CUDAHM_EINVAL, "handle is NULL");
  if (h->cfg.marginal) return fail(CUDAHM_EUNSUPPORTED, "the marginal form has no latents");
  if (!h->data_set) return fail(CUDAHM_ESTATE, "set_chi before set_data");
  if (h->sweeps != 0) return fail(CUDAHM_ESTATE, "set_chi after the chain has started");
  if (!chi_host || n != h->n) return fail(CUDAHM_EINVAL, "bad chi argument");
  CU(cudaSetDevice(h->cfg.device));
  const size_t cnt = static_cast<size_t>(h->n) * h->d;
  std::vector<double> soa;
  if (h->d > 1) {  // member-major in the API, per component on the device
    soa.resize(cnt);
    for (size_t i = 0; i < static_cast<size_t>(h->n); ++i)
      for (int j = 0; j < h->d; ++j) soa[j * h->n + i] = chi_host[i * h->d + j];
    chi_host = soa.data();
  }
  double* tmp = nullptr;
  TRY(alloc_into(h, &tmp, cnt));
  CU(cudaMemcpyAsync(tmp, chi_host, sizeof(double) * cnt, cudaMemcpyHostToDevice, h->stream));
  CU(cudaMemsetAsync(h->bad, 0, sizeof(int), h->stream));
  CU(launch_check_chi(h->cfg.model, static_cast<long long>(cnt), tmp, h->cfg.theta_init, h->bad, h->stream));
  CU(cudaMemcpyAsync(h->host_err, h->bad, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  CU(cudaStreamSynchronize(h->stream));
  if (*h->host_err) {
    h->dfree(tmp);
    return fail(CUDAHM_EINVAL, "%d latents are non-finite or off the support at theta", *h->host_err);
  }
  CU(cudaMemcpyAsync(h->chi, tmp, sizeof(double) * cnt, cudaMemcpyDeviceToDevice, h->stream));
  TRY(chi_to_state(h));
  CU(cudaStreamSynchronize(h->stream));
  h->dfree(tmp);
  return CUDAHM_OK;
}

int cudahm_run(cudahm_t h, int64_t n_burn, int64_t n_iter, int64_t thin) {
  if (!h) return fail(CUDAHM_EINVAL, "handle is NULL");
  if (!h->data_set) return fail(CUDAHM_ESTATE, "run before set_data");
  if (h->shard_active) return fail(CUDAHM_ESTATE, "a sharded run is in progress (cudahm_shard_end first)");
  if (h->K == 0 && !h->cfg.marginal) {  // streaming form: a batch of one population
    cudahm_t one[1] = {h};
    CU(cudaEventRecord(h->ev0, h->stream));
    const int rc = cudahm_batch_run(one, 1, n_burn, n_iter, thin, nullptr, nullptr);
    return rc;
  }
  if (n_burn < 0 || n_iter < 0) return fail(CUDAHM_EINVAL, "negative sweep counts");
  if (n_iter > 0 && thin < 1) return fail(CUDAHM_EINVAL, "thin must be >= 1");
  const long long total = n_burn + n_iter;
  if (h->sweeps + total >= (1ll << 32) - 2) return fail(CUDAHM_EINVAL, "sweep counter would exceed 2^32");
  CU(cudaSetDevice(h->cfg.device));
  const long long nrows = (n_iter > 0) ? n_iter / thin : 0;
  if (nrows > h->rows_cap) {
    h->dfree(h->rows);
    h->rows = nullptr;
    TRY(alloc_into(h, &h->rows, static_cast<size_t>(nrows) * h->p));
    h->rows_cap = nrows;
  }
  const long long T = std::min<long long>(h->cfg.trace_sweeps, total);
  TRY(ensure_trace(h, T));
  CU(cudaEventRecord(h->ev0, h->stream));
  if (has_rule(h->cfg.model) && !h->etabar_valid) {
    // selection integral at the current theta, once per chain (kept on the device afterwards)
    char* base = reinterpret_cast<char*>(h->chain);
    TRY(compute_etabar_into(h, reinterpret_cast<const double*>(base + offsetof(ChainState, theta)),
                            reinterpret_cast<double*>(base + offsetof(ChainState, etabar))));
    h->etabar_valid = true;
  }
  if (h->cfg.marginal && !h->marg_valid) {
    // log p_i at the current theta into array 0, once per chain
    char* base = reinterpret_cast<char*>(h->chain);
    CU(launch_marg_eval(h->cfg.model, h->cfg.precision == CUDAHM_FP32, h->n, h->y, h->aux,
                        reinterpret_cast<const double*>(base + offsetof(ChainState, theta)), h->mc, h->math_tab,
                        h->marg_nodes, h->marg_d32, h->marg_lp, h->stream));
    CU(cudaMemsetAsync(base + offsetof(ChainState, mcur), 0, sizeof(int), h->stream));
    h->marg_valid = true;
  }
  SweepArgs a = base_args(h);
  if (h->cfg.marginal) a.rows_smem = h->mrows_smem;
  a.thin = thin;
  a.keep_phase = 0;
  a.trace_T = T;
  a.tr_delta = h->tr_delta;
  a.tr_u = h->tr_u;
  a.tr_acc = h->tr_acc;
  a.tr_thprop = h->tr_thprop;
  a.tr_D = h->tr_D;
  a.tr_logalpha = h->tr_logalpha;
  a.tr_ut = h->tr_ut;
  a.tr_tacc = h->tr_tacc;
  a.tr_eb = h->tr_eb;
  a.tab_U = h->tab_U;
  a.tab_u = h->tab_u;
  a.tab_lnu = h->tab_lnu;
  a.tab_eta = h->tab_eta;
  long long off = 0, rows_done = 0;
  if (total == 0) CU(cudaMemsetAsync(h->err, 0, sizeof(int), h->stream));  // else cleared by the first chunk
  while (off < total) {
    const long long ns = std::min<long long>(kChunk, total - off);
    // theta tables of this chunk; also clears the barrier count and theta' sequence, the grid
    // totals, and (first chunk) the run's error word
    CU(launch_tables(h->p, a.key0, a.key1, h->sweeps, ns, h->cfg.adapt_exponent, h->tab_U, h->tab_u, h->tab_lnu,
                     h->tab_eta, h->bar, h->acc3, 3 * kAccWords, off == 0 ? h->err : nullptr, h->stream));
    a.k0 = h->sweeps;
    a.ns = ns;
    a.burn_left = n_burn - off;
    a.trace_off = off;
    a.rows = h->rows ? h->rows + rows_done * h->p : nullptr;
    if (h->cfg.marginal) CU(launch_marg(a, h->mgrid, 256, h->stream));
    else CU(launch_sweep(a, h->K, h->grid, h->block, h->stream));
    // rows kept in [off, off + ns): post-burn indices q with (q + 1) % thin == 0
    if (n_iter > 0) {
      const long long q0 = std::max<long long>(0, off - n_burn), q1 = off + ns - n_burn;
      if (q1 > q0) rows_done += q1 / thin - q0 / thin;
    }
    h->sweeps += ns;
    off += ns;
  }
  // the kept rows come back with the error word (one synchronisation for both), through a pinned
  // buffer that cudahm_get_samples reads; a run keeping more rows than it holds grows it (pinned
  // host memory, not device memory). The run's device time (ev0 .. ev1) includes that copy.
  h->rows_host_n = 0;
  if (rows_done > 0 && rows_done * h->p <= (1ll << 20)) {
    if (rows_done > h->rows_host_cap) {
      if (h->rows_host) cudaFreeHost(h->rows_host);
      h->rows_host = nullptr;
      h->rows_host_cap = 0;
      if (cudaHostAlloc(reinterpret_cast<void**>(&h->rows_host), sizeof(double) * rows_done * h->p,
                        cudaHostAllocDefault) == cudaSuccess)
        h->rows_host_cap = rows_done;
    }
    if (h->rows_host && rows_done <= h->rows_host_cap) {
      CU(cudaMemcpyAsync(h->rows_host, h->rows, sizeof(double) * rows_done * h->p, cudaMemcpyDeviceToHost,
                         h->stream));
      h->rows_host_n = rows_done;
    }
  }
  CU(cudaEventRecord(h->ev1, h->stream));
  int code = 0;
  TRY(read_err(h, &code));
  float ms = 0.f;
  CU(cudaEventElapsedTime(&ms, h->ev0, h->ev1));
  h->last_run_ms = ms;
  if (code != 0) {
    // device state was written back only by the launches that completed
    ChainState cs;
    CU(cudaMemcpy(&cs, h->chain, sizeof(cs), cudaMemcpyDeviceToHost));
    h->sweeps = cs.sweeps;
    h->rows_last = 0;
    h->rows_host_n = 0;
    if (code == CUDAHM_ETIMEOUT) return fail(code, "a grid barrier wait exceeded its bound; run stopped");
    if (code == CUDAHM_ENUMERIC) return fail(code, "NaN in a log-density; run stopped");
    return fail(code, "device error %d", code);
  }
  h->rows_last = rows_done;
  h->trace_T_last = T;
  return CUDAHM_OK;
}

int cudahm_get_samples(cudahm_t h, double* theta_host, int64_t cap_rows, int64_t* rows_out) {
  if (!h) return fail(CUDAHM_EINVAL, "handle is NULL");
  const long long r = std::min<long long>(cap_rows, h->rows_last);
  if (rows_out) *rows_out = h->rows_last;
  if (r > 0 && h->rows_host_n == h->rows_last) {  // already on the host
    if (!theta_host) return fail(CUDAHM_EINVAL, "theta_host is NULL");
    std::memcpy(theta_host, h->rows_host, sizeof(double) * r * h->p);
    return CUDAHM_OK;
  }
  if (r > 0) {
    if (!theta_host) return fail(CUDAHM_EINVAL, "theta_host is NULL");
    CU(cudaSetDevice(h->cfg.device));
    CU(cudaMemcpyAsync(theta_host, h->rows, sizeof(double) * r * h->p, cudaMemcpyDeviceToHost, h->stream));
    CU(cudaStreamSynchronize(h->stream));
  }
  return CUDAHM_OK;
}

int cudahm_get_chi(cudahm_t h, double* chi_host, double* S_host) {
  if (!h) return fail(CUDAHM_EINVAL, "handle is NULL");
  if (h->cfg.marginal) return fail(CUDAHM_EUNSUPPORTED, "the marginal form has no latents");
  CU(cudaSetDevice(h->cfg.device));
  if (h->d == 3) {  // per-component device arrays to member-major host arrays
    const size_t n = static_cast<size_t>(h->n);
    if (chi_host) {
      std::vector<double> t(3 * n);
      CU(cudaMemcpyAsync(t.data(), h->chi, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, h->stream));
      CU(cudaStreamSynchronize(h->stream));
      for (size_t i = 0; i < n; ++i)
        for (int j = 0; j < 3; ++j) chi_host[3 * i + j] = t[j * n + i];
    }
    if (S_host) {
      std::vector<double> t(6 * n);
      CU(cudaMemcpyAsync(t.data(), h->S, sizeof(double) * 6 * n, cudaMemcpyDeviceToHost, h->stream));
      CU(cudaStreamSynchronize(h->stream));
      const int at[6] = {0, 3, 4, 6, 7, 8};  // packed rows -> row-major 3 x 3 positions
      for (size_t i = 0; i < n; ++i) {
        double* m = S_host + 9 * i;
        for (int q = 0; q < 9; ++q) m[q] = 0.0;
        for (int q = 0; q < 6; ++q) m[at[q]] = t[q * n + i];
      }
    }
    return CUDAHM_OK;
  }
  if (chi_host) {
    TRY(chi_from_state(h));
    CU(cudaMemcpyAsync(chi_host, h->chi, sizeof(double) * h->n * h->d, cudaMemcpyDeviceToHost, h->stream));
  }
  if (S_host)
    CU(cudaMemcpyAsync(S_host, h->S, sizeof(double) * h->n * h->d * h->d, cudaMemcpyDeviceToHost, h->stream));
  CU(cudaStreamSynchronize(h->stream));
  return CUDAHM_OK;
}

int cudahm_get_chi_moments(cudahm_t h, double* mean_host, double* var_host, int64_t* count_out) {
  if (!h) return fail(CUDAHM_EINVAL, "handle is NULL");
  if (!h->mom) return fail(CUDAHM_ESTATE, "the handle was created without keep_chi_moments");
  CU(cudaSetDevice(h->cfg.device));
  ChainState cs;
  CU(cudaMemcpyAsync(&cs, h->chain, sizeof(cs), cudaMemcpyDeviceToHost, h->stream));
  CU(cudaStreamSynchronize(h->stream));
  if (count_out) *count_out = cs.mom_n;
  if (!mean_host && !var_host) return CUDAHM_OK;
  const size_t n = static_cast<size_t>(h->n), dn = n * h->d;
  std::vector<double> t(2 * dn);
  CU(cudaMemcpyAsync(t.data(), h->mom + static_cast<size_t>(cs.mom_sel) * 2 * dn, sizeof(double) * 2 * dn,
                     cudaMemcpyDeviceToHost, h->stream));
  CU(cudaStreamSynchronize(h->stream));
  const double m1 = static_cast<double>(cs.mom_n - 1);
  for (size_t i = 0; i < n; ++i)
    for (int j = 0; j < h->d; ++j) {  // per component on the device, member-major in the API
      const size_t q = j * n + i;
      if (mean_host) mean_host[i * h->d + j] = t[q];
      if (var_host) var_host[i * h->d + j] = cs.mom_n > 1 ? t[dn + q] / m1 : 0.0;
    }
  return CUDAHM_OK;
}

int cudahm_get_theta(cudahm_t h, double* theta_host, double* S_theta_host) {
  if (!h) return fail(CUDAHM_EINVAL, "handle is NULL");
  CU(cudaSetDevice(h->cfg.device));
  ChainState cs;
  CU(cudaMemcpyAsync(&cs, h->chain, sizeof(cs), cudaMemcpyDeviceToHost, h->stream));
  CU(cudaStreamSynchronize(h->stream));
  if (theta_host) std::memcpy(theta_host, cs.theta, sizeof(double) * h->p);
  if (S_theta_host) std::memcpy(S_theta_host, cs.S_theta, sizeof(double) * h->p * h->p);
  return CUDAHM_OK;
}

int cudahm_get_stats(cudahm_t h, cudahm_stats* s) {
  if (!h || !s) return fail(CUDAHM_EINVAL, "NULL argument");
  CU(cudaSetDevice(h->cfg.device));
  ChainState cs;
  CU(cudaMemcpyAsync(&cs, h->chain, sizeof(cs), cudaMemcpyDeviceToHost, h->stream));
  CU(cudaStreamSynchronize(h->stream));
  std::memset(s, 0, sizeof(*s));
  s->sweeps = cs.sweeps;
  s->member_accepts = cs.member_acc;
  s->theta_accepts = cs.theta_acc;
  s->rows = h->rows_last;
  s->last_run_ms = h->last_run_ms;
  s->etabar = cs.etabar;
  s->grid_blocks = h->cfg.marginal ? h->mgrid : h->grid;
  s->block_threads = h->cfg.marginal ? 256 : h->block;
  s->objects_per_thread = h->cfg.marginal ? 0 : h->K;
  return CUDAHM_OK;
}

int cudahm_eval_marginal(cudahm_t h, const double* theta_host, double* lp_host) {
  if (!h || !theta_host || !lp_host) return fail(CUDAHM_EINVAL, "NULL argument");
  if (h->cfg.model != CUDAHM_NN1 && h->cfg.model != CUDAHM_LF && h->cfg.model != CUDAHM_BB1)
    return fail(CUDAHM_EUNSUPPORTED, "the cubature rule integrates one-dimensional latents (NN1, LF, BB1)");
  if (h->cfg.model == CUDAHM_BB1 && !(h->mc.alpha * kMargK < 1.0))
    return fail(CUDAHM_EUNSUPPORTED, "the BB1 marginal window needs alpha < 1/10");
  if (!h->data_set) return fail(CUDAHM_ESTATE, "eval before set_data");
  CU(cudaSetDevice(h->cfg.device));
  double* out = nullptr;
  TRY(alloc_into(h, &out, h->n));
  CU(cudaMemcpyAsync(h->theta_dev, theta_host, sizeof(double) * h->p, cudaMemcpyHostToDevice, h->stream));
  const cudaError_t e = launch_marg_eval(h->cfg.model, h->cfg.precision == CUDAHM_FP32, h->n, h->y, h->aux,
                                         h->theta_dev, h->mc, h->math_tab, h->marg_nodes, h->marg_d32, out, h->stream);
  if (e != cudaSuccess) {
    h->dfree(out);
    return fail(CUDAHM_ECUDA, "marginal evaluation failed: %s", cudaGetErrorString(e));
  }
  CU(cudaMemcpyAsync(lp_host, out, sizeof(double) * h->n, cudaMemcpyDeviceToHost, h->stream));
  CU(cudaStreamSynchronize(h->stream));
  h->dfree(out);
  return CUDAHM_OK;
}

int cudahm_eval_logdens(cudahm_t h, const double* theta_host, double* lp_host) {
  if (!h || !theta_host || !lp_host) return fail(CUDAHM_EINVAL, "NULL argument");
  if (!h->data_set) return fail(CUDAHM_ESTATE, "eval before set_data");
  CU(cudaSetDevice(h->cfg.device));
  double* out = nullptr;
  TRY(alloc_into(h, &out, h->n));
  CU(cudaMemcpyAsync(h->theta_dev, theta_host, sizeof(double) * h->p, cudaMemcpyHostToDevice, h->stream));
  TRY(chi_from_state(h));
  CU(launch_eval_logdens(h->cfg.model, h->cfg.precision == CUDAHM_FP32, h->n, h->y, h->aux, h->chi, h->theta_dev,
                         h->mc, h->math_tab, out, h->stream));
  CU(cudaMemcpyAsync(lp_host, out, sizeof(double) * h->n, cudaMemcpyDeviceToHost, h->stream));
  CU(cudaStreamSynchronize(h->stream));
  h->dfree(out);
  return CUDAHM_OK;
}

int cudahm_eval_etabar(cudahm_t h, const double* theta_host, double* out) {
  if (!h || !theta_host || !out) return fail(CUDAHM_EINVAL, "NULL argument");
  if (!has_rule(h->cfg.model)) return fail(CUDAHM_EINVAL, "etabar exists only for the LF and BB1 models");
  CU(cudaSetDevice(h->cfg.device));
  CU(cudaMemcpyAsync(h->theta_dev, theta_host, sizeof(double) * h->p, cudaMemcpyHostToDevice, h->stream));
  TRY(compute_etabar_into(h, h->theta_dev, h->eval_out));
  CU(cudaMemcpyAsync(out, h->eval_out, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CU(cudaStreamSynchronize(h->stream));
  return CUDAHM_OK;
}

int cudahm_eval_detection(cudahm_t h, const double* F_host, double* eta_host, int64_t n) {
  if (!h || !F_host || !eta_host || n < 0) return fail(CUDAHM_EINVAL, "bad argument");
  if (!has_rule(h->cfg.model))
    return fail(CUDAHM_EINVAL, "detection efficiency exists only for the LF and BB1 models");
  if (n == 0) return CUDAHM_OK;
  CU(cudaSetDevice(h->cfg.device));
  double *F = nullptr, *out = nullptr;
  TRY(alloc_into(h, &F, n));
  int rc = alloc_into(h, &out, n);
  if (rc != CUDAHM_OK) {
    h->dfree(F);
    return rc;
  }
  cudaError_t e = cudaMemcpyAsync(F, F_host, sizeof(double) * n, cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess)
    e = launch_detection(h->cfg.model, n, F, h->mc, h->cfg.model_consts[0], h->phi_coef, out, h->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(eta_host, out, sizeof(double) * n, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  h->dfree(F);
  h->dfree(out);
  if (e != cudaSuccess) return fail(CUDAHM_ECUDA, "eval_detection: %s", cudaGetErrorString(e));
  return CUDAHM_OK;
}

int cudahm_get_trace(cudahm_t h, double* delta, double* u, uint8_t* acc, double* theta_prop, double* D,
                     double* logalpha, double* utheta, uint8_t* tacc, double* etabar_prop, int64_t* t_out) {
  if (!h) return fail(CUDAHM_EINVAL, "handle is NULL");
  const long long T = h->trace_T_last;
  if (t_out) *t_out = T;
  if (T == 0) return CUDAHM_OK;
  CU(cudaSetDevice(h->cfg.device));
  const size_t tn = static_cast<size_t>(T) * h->n;
  auto cp = [&](void* dst, const void* src, size_t bytes) -> cudaError_t {
    if (!dst) return cudaSuccess;
    return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, h->stream);
  };
  if (!h->cfg.marginal) {  // the marginal form has no member steps to record
    CU(cp(delta, h->tr_delta, sizeof(double) * tn));
    CU(cp(u, h->tr_u, sizeof(double) * tn));
    CU(cp(acc, h->tr_acc, tn));
  }
  CU(cp(theta_prop, h->tr_thprop, sizeof(double) * T * h->p));
  CU(cp(D, h->tr_D, sizeof(double) * T));
  CU(cp(logalpha, h->tr_logalpha, sizeof(double) * T));
  CU(cp(utheta, h->tr_ut, sizeof(double) * T));
  CU(cp(tacc, h->tr_tacc, T));
  CU(cp(etabar_prop, h->tr_eb, sizeof(double) * T));
  CU(cudaStreamSynchronize(h->stream));
  return CUDAHM_OK;
}

// Checkpoint layout: header (10 x int64: magic, layout version, model, n, d, p, seed, data set,
// configuration hash, 0), ChainState, then the latents and RAM factors as the device holds them
// (d = 1: chi[n], S[n]; d = 3: chi[3][n], S[6][n]), then the committed moments when kept.
int cudahm_checkpoint(cudahm_t h, void* buf, size_t cap, size_t* used) {
  if (!h || !used) return fail(CUDAHM_EINVAL, "NULL argument");
  const size_t nchi = static_cast<size_t>(h->n) * h->d, nS = static_cast<size_t>(h->factor_n);
  const size_t nmom = h->mom ? 2 * nchi : 0;  // the committed moments
  const size_t need = kHeaderWords * sizeof(int64_t) + sizeof(ChainState) + sizeof(double) * (nchi + nS + nmom);
  *used = need;
  if (!buf) return CUDAHM_OK;
  if (cap < need) return fail(CUDAHM_EINVAL, "checkpoint buffer too small: need %zu bytes", need);
  CU(cudaSetDevice(h->cfg.device));
  int64_t hdr[kHeaderWords] = {kCheckpointMagic, kCheckpointVersion, h->cfg.model, h->n, h->d, h->p,
                               static_cast<int64_t>(h->cfg.seed), h->data_set ? 1 : 0,
                               static_cast<int64_t>(config_hash(h->cfg)), 0};
  char* c = static_cast<char*>(buf);
  std::memcpy(c, hdr, sizeof(hdr));
  c += sizeof(hdr);
  CU(cudaMemcpyAsync(c, h->chain, sizeof(ChainState), cudaMemcpyDeviceToHost, h->stream));
  c += sizeof(ChainState);
  TRY(chi_from_state(h));
  CU(cudaMemcpyAsync(c, h->chi, sizeof(double) * nchi, cudaMemcpyDeviceToHost, h->stream));
  c += sizeof(double) * nchi;
  CU(cudaMemcpyAsync(c, h->S, sizeof(double) * nS, cudaMemcpyDeviceToHost, h->stream));
  CU(cudaStreamSynchronize(h->stream));
  if (nmom) {
    c += sizeof(double) * nS;
    ChainState cs;
    std::memcpy(&cs, static_cast<char*>(buf) + sizeof(hdr), sizeof(cs));
    CU(cudaMemcpyAsync(c, h->mom + static_cast<size_t>(cs.mom_sel) * nmom, sizeof(double) * nmom,
                       cudaMemcpyDeviceToHost, h->stream));
    CU(cudaStreamSynchronize(h->stream));
  }
  return CUDAHM_OK;
}

int cudahm_restore(cudahm_t h, const void* buf, size_t size) {
  if (!h || !buf) return fail(CUDAHM_EINVAL, "NULL argument");
  if (!h->data_set) return fail(CUDAHM_ESTATE, "restore needs set_data first");
  const size_t nchi = static_cast<size_t>(h->n) * h->d, nS = static_cast<size_t>(h->factor_n);
  const size_t nmom = h->mom ? 2 * nchi : 0;
  const size_t need = kHeaderWords * sizeof(int64_t) + sizeof(ChainState) + sizeof(double) * (nchi + nS + nmom);
  if (size < kHeaderWords * sizeof(int64_t)) return fail(CUDAHM_EINVAL, "checkpoint buffer too small");
  int64_t hdr[kHeaderWords];
  const char* c = static_cast<const char*>(buf);
  std::memcpy(hdr, c, sizeof(hdr));
  if (hdr[0] != kCheckpointMagic || hdr[1] != kCheckpointVersion)
    return fail(CUDAHM_EINVAL, "not a checkpoint of this layout version (%d)", static_cast<int>(kCheckpointVersion));
  if (hdr[2] != h->cfg.model || hdr[3] != h->n || hdr[4] != h->d || hdr[5] != h->p ||
      hdr[6] != static_cast<int64_t>(h->cfg.seed) || hdr[8] != static_cast<int64_t>(config_hash(h->cfg)))
    return fail(CUDAHM_EINVAL, "checkpoint does not match this handle's configuration");
  if (size < need) return fail(CUDAHM_EINVAL, "checkpoint buffer too small");
  c += sizeof(hdr);
  ChainState cs;
  std::memcpy(&cs, c, sizeof(cs));
  // the chain state indexes device buffers and sizes launches: check it before any copy
  bool ok = (cs.mom_sel == 0 || cs.mom_sel == 1) && (cs.mcur == 0 || cs.mcur == 1) && cs.sweeps >= 0 &&
            cs.sweeps < (1ll << 32) - 2 && cs.mom_n >= 0 && cs.mom_n <= cs.sweeps && cs.member_acc >= 0 &&
            cs.theta_acc >= 0 && cs.rows >= 0 && std::isfinite(cs.pend_alpha) && std::isfinite(cs.pend_eta) &&
            cs.pend_eta >= 0.0 && std::isfinite(cs.etabar) && cs.etabar >= 0.0;
  for (int q = 0; q < h->p && ok; ++q) ok = std::isfinite(cs.theta[q]) && std::isfinite(cs.pend_U[q]);
  for (int q = 0; q < h->p * h->p && ok; ++q) ok = std::isfinite(cs.S_theta[q]);
  if (!ok) return fail(CUDAHM_EINVAL, "checkpoint chain state is out of range");
  CU(cudaSetDevice(h->cfg.device));
  CU(cudaMemcpyAsync(h->chain, c, sizeof(ChainState), cudaMemcpyHostToDevice, h->stream));
  c += sizeof(ChainState);
  CU(cudaMemcpyAsync(h->chi, c, sizeof(double) * nchi, cudaMemcpyHostToDevice, h->stream));
  TRY(chi_to_state(h));
  c += sizeof(double) * nchi;
  CU(cudaMemcpyAsync(h->S, c, sizeof(double) * nS, cudaMemcpyHostToDevice, h->stream));
  if (nmom) {
    c += sizeof(double) * nS;
    CU(cudaMemcpyAsync(h->mom + static_cast<size_t>(cs.mom_sel) * nmom, c, sizeof(double) * nmom,
                       cudaMemcpyHostToDevice, h->stream));
  }
  CU(cudaStreamSynchronize(h->stream));
  h->sweeps = cs.sweeps;
  h->rows_last = 0;
  h->rows_host_n = 0;
  // etabar(theta) is recomputed by this handle's own rule before the next run (the same bits as
  // the stored value when the rule is the same, which the configuration hash checks)
  h->etabar_valid = false;
  h->marg_valid = false;  // log p_i is recomputed at the restored theta before the next run
  return CUDAHM_OK;
}

// ------------------------------------------------------------------ shards --
// A population split across devices (Sec. 6: larger N than one device holds): each shard is a
// handle holding a contiguous range of the population's members. Every shard draws the same
// theta' (same seed, same theta tables); its pass steps its members, whose draws carry their
// population index, and reduces its part of the theta' sum and of the selection rule into
// exchange words; the caller adds the words of all shards (an all-reduce of 16 integers); every
// shard then takes the same decision from the sum. The chain is the unsplit one, bit for bit.
int cudahm_shard_config(cudahm_t h, int64_t member_offset, int64_t population_n, int32_t part, int32_t parts) {
  if (!h) return fail(CUDAHM_EINVAL, "handle is NULL");
  if (h->shard_active) return fail(CUDAHM_ESTATE, "a sharded run is in progress");
  if (h->cfg.marginal) return fail(CUDAHM_EUNSUPPORTED, "the marginal form is not split into shards");
  if (h->cfg.trace_sweeps > 0 || h->cfg.keep_chi_moments)
    return fail(CUDAHM_EUNSUPPORTED, "a shard records neither a lockstep trace nor latent moments");
  if (parts < 1 || part < 0 || part >= parts) return fail(CUDAHM_EINVAL, "need 0 <= part < parts");
  if (member_offset < 0 || population_n < 1 || member_offset + h->n > population_n)
    return fail(CUDAHM_EINVAL, "members [offset, offset + n) must lie in [0, population_n)");
  if (population_n > 0xFFFFFFFFll) return fail(CUDAHM_EINVAL, "population_n must fit the 32-bit member word");
  h->shard_set = true;
  h->shard_moff = member_offset;
  h->shard_npop = population_n;
  h->shard_part = part;
  h->shard_parts = parts;
  return CUDAHM_OK;
}

int cudahm_shard_begin(cudahm_t h, int64_t n_burn, int64_t n_iter, int64_t thin) {
  if (!h) return fail(CUDAHM_EINVAL, "handle is NULL");
  if (!h->shard_set) return fail(CUDAHM_ESTATE, "cudahm_shard_config first");
  if (!h->data_set) return fail(CUDAHM_ESTATE, "shard run before set_data");
  if (h->shard_active) return fail(CUDAHM_ESTATE, "a sharded run is already in progress");
  if (n_burn < 0 || n_iter < 0 || n_burn + n_iter < 1) return fail(CUDAHM_EINVAL, "bad sweep counts");
  if (n_iter > 0 && thin < 1) return fail(CUDAHM_EINVAL, "thin must be >= 1");
  const long long total = n_burn + n_iter;
  if (h->sweeps + total >= (1ll << 32) - 2) return fail(CUDAHM_EINVAL, "sweep counter would exceed 2^32");
  CU(cudaSetDevice(h->cfg.device));
  cudaStream_t st = h->stream;
  const long long nrows = (n_iter > 0) ? n_iter / thin : 0;
  if (nrows > h->rows_cap) {
    h->dfree(h->rows);
    h->rows = nullptr;
    TRY(alloc_into(h, &h->rows, static_cast<size_t>(nrows) * h->p));
    h->rows_cap = nrows;
  }
  if (has_rule(h->cfg.model) && !h->etabar_valid) {  // the whole rule at theta, as an unsplit run
    char* base = reinterpret_cast<char*>(h->chain);
    TRY(compute_etabar_into(h, reinterpret_cast<const double*>(base + offsetof(ChainState, theta)),
                            reinterpret_cast<double*>(base + offsetof(ChainState, etabar))));
    h->etabar_valid = true;
  }
  if (!h->sh_pop) {
    TRY(alloc_into(h, &h->sh_pop, 1));
    TRY(alloc_into(h, &h->sh_prog, 1));
    TRY(alloc_into(h, &h->sh_b0, 1));
    TRY(alloc_into(h, &h->sh_nb, 1));
    TRY(alloc_into(h, &h->sh_bar, 1));
  }
  // launch shape: 128-thread blocks, as many as the occupancy allows and the members can use
  const bool f32 = h->cfg.precision == CUDAHM_FP32, d1 = h->d == 1;
  const int blk = 128;
  const int smem = static_cast<int>(batch_smem_bytes(f32, d1, blk));
  int bps = 0;
  CU(batch_occupancy(f32, d1, blk, smem, &bps));
  if (bps < 1) return fail(CUDAHM_EUNSUPPORTED, "the streaming kernel does not fit on this device");
  long long cap = (h->n + 31) / 32 + (has_rule(h->cfg.model) ? 8 : 0);
  const int grid = static_cast<int>(std::max<long long>(1, std::min<long long>(cap, static_cast<long long>(bps) * h->sms)));
  if (grid > h->sh_grid || !h->sh_partials) {
    h->dfree(h->sh_partials);
    h->sh_partials = nullptr;
    TRY(alloc_into(h, &h->sh_partials, static_cast<size_t>(2) * grid * kPartWords));
  }
  h->sh_grid = grid;
  h->sh_block = blk;
  h->sh_smem = smem;

  SweepArgs a = base_args(h);
  a.partials = h->sh_partials;
  a.bar = h->sh_bar;
  a.rows = h->rows;
  a.thin = thin;
  a.trace_T = 0;
  a.skip_cta = -1;
  a.moff = static_cast<unsigned int>(h->shard_moff);
  if (has_rule(h->cfg.model)) {
    const long long nL = rule_nL(h->cfg);
    a.rule_j0 = static_cast<int>(nL * h->shard_part / h->shard_parts);
    a.rule_j1 = static_cast<int>(nL * (h->shard_part + 1) / h->shard_parts);
    if (a.rule_j1 == 0) a.rule_j0 = a.rule_j1 = -1;  // no outer node (rule_j1 = 0 would mean all)
  }
  a.shard_out = nullptr;
  const BatchProg prog{total, 0, n_burn, thin, 0, 0};
  const int zero = 0;
  CU(cudaMemcpyAsync(h->sh_pop, &a, sizeof(a), cudaMemcpyHostToDevice, st));
  CU(cudaMemcpyAsync(h->sh_prog, &prog, sizeof(prog), cudaMemcpyHostToDevice, st));
  CU(cudaMemcpyAsync(h->sh_b0, &zero, sizeof(int), cudaMemcpyHostToDevice, st));
  CU(cudaMemcpyAsync(h->sh_nb, &grid, sizeof(int), cudaMemcpyHostToDevice, st));
  CU(cudaMemsetAsync(h->sh_bar, 0, sizeof(unsigned int), st));
  CU(cudaMemsetAsync(h->err, 0, sizeof(int), st));
  CU(launch_batch_tables(h->sh_pop, h->sh_prog, 1, 1, st));  // theta tables of the first sweep
  CU(cudaStreamSynchronize(st));
  h->sh_out_last = nullptr;
  h->shard_total = total;
  h->shard_passes = 0;
  h->shard_decides = 0;
  h->rows_last = 0;
  h->rows_host_n = 0;
  h->shard_active = true;
  return CUDAHM_OK;
}

int cudahm_shard_pass(cudahm_t h, uint64_t* words_dev) {
  if (!h || !words_dev) return fail(CUDAHM_EINVAL, "NULL argument");
  if (!h->shard_active) return fail(CUDAHM_ESTATE, "cudahm_shard_begin first");
  if (h->shard_passes != h->shard_decides) return fail(CUDAHM_ESTATE, "the previous pass has not been decided");
  if (h->shard_passes >= h->shard_total) return fail(CUDAHM_ESTATE, "every sweep of the run has been made");
  if (reinterpret_cast<uintptr_t>(words_dev) % 8 != 0) return fail(CUDAHM_EINVAL, "words_dev must be 8-byte aligned");
  cudaStream_t st = h->stream;
  unsigned long long* out = reinterpret_cast<unsigned long long*>(words_dev);
  if (out != h->sh_out_last) {  // the pass's arguments name the caller's buffer
    CU(cudaMemcpyAsync(reinterpret_cast<char*>(h->sh_pop) + offsetof(SweepArgs, shard_out), &out, sizeof(out),
                       cudaMemcpyHostToDevice, st));
    h->sh_out_last = out;
  }
  const bool f32 = h->cfg.precision == CUDAHM_FP32;
  CU(launch_batch(f32, h->d == 1, h->sh_pop, h->sh_prog, h->sh_b0, h->sh_nb, 1, 1, 128, h->sh_grid, h->sh_block,
                  h->sh_smem, st));
  h->shard_passes++;
  return CUDAHM_OK;
}

int cudahm_shard_decide(cudahm_t h, const uint64_t* total_dev) {
  if (!h || !total_dev) return fail(CUDAHM_EINVAL, "NULL argument");
  if (!h->shard_active) return fail(CUDAHM_ESTATE, "cudahm_shard_begin first");
  if (h->shard_decides + 1 != h->shard_passes) return fail(CUDAHM_ESTATE, "decide follows a pass");
  if (reinterpret_cast<uintptr_t>(total_dev) % 8 != 0) return fail(CUDAHM_EINVAL, "total_dev must be 8-byte aligned");
  CU(launch_shard_decide(h->cfg.model, h->sh_pop, h->sh_prog, reinterpret_cast<const unsigned long long*>(total_dev),
                         h->shard_npop, h->shard_parts, h->stream));
  h->shard_decides++;
  return CUDAHM_OK;
}

int cudahm_shard_end(cudahm_t h, int64_t* rows_out) {
  if (!h) return fail(CUDAHM_EINVAL, "handle is NULL");
  if (!h->shard_active) return fail(CUDAHM_ESTATE, "no sharded run in progress");
  h->shard_active = false;
  int code = 0;
  TRY(read_err(h, &code));
  BatchProg prog;
  ChainState cs;
  CU(cudaMemcpy(&prog, h->sh_prog, sizeof(prog), cudaMemcpyDeviceToHost));
  CU(cudaMemcpy(&cs, h->chain, sizeof(cs), cudaMemcpyDeviceToHost));
  h->sweeps = cs.sweeps;
  h->rows_host_n = 0;
  if (code != 0) {
    h->rows_last = 0;
    if (code == CUDAHM_ESTATE)
      return fail(code, "exchange words did not come from every shard of the population once; run stopped");
    if (code == CUDAHM_ETIMEOUT) return fail(code, "a bounded device-side wait expired; run stopped");
    if (code == CUDAHM_ENUMERIC) return fail(code, "NaN in a log-density; run stopped");
    return fail(code, "device error %d", code);
  }
  h->rows_last = prog.rows;
  if (rows_out) *rows_out = prog.rows;
  if (h->shard_passes != h->shard_decides)
    return fail(CUDAHM_ESTATE, "run ended after a pass without its decision: the latents are one sweep past theta");
  return CUDAHM_OK;
}

// ---------------------------------------------------------------- batched --
namespace {

struct TuneKey {
  int precision, k, nlf;
  long long nbucket;
  bool operator==(const TuneKey& o) const {
    return precision == o.precision && k == o.k && nlf == o.nlf && nbucket == o.nbucket;
  }
};
struct TuneEntry {
  TuneKey key;
  int block, chunk, grid;
};
std::vector<TuneEntry> g_tune_cache;  // decisions of the autotuner for this process

struct BatchBufs {
  cudahm* owner = nullptr;
  SweepArgs* pops = nullptr;
  BatchProg* progs = nullptr;
  int* b0s = nullptr;
  int* nbs = nullptr;
  unsigned long long* partials = nullptr;
  unsigned int* bars = nullptr;
  int* errs = nullptr;
  ~BatchBufs() {
    if (!owner) return;
    for (void* q : {(void*)pops, (void*)progs, (void*)b0s, (void*)nbs, (void*)partials, (void*)bars, (void*)errs})
      owner->dfree(q);
  }
};

}  // namespace

int cudahm_batch_run(cudahm_t* hs, int32_t k, int64_t n_burn, int64_t n_iter, int64_t thin, const cudahm_tune* tune,
                     cudahm_tune* chosen) {
  if (!hs || k < 1) return fail(CUDAHM_EINVAL, "need at least one handle");
  if (n_burn < 0 || n_iter < 0 || n_burn + n_iter < 1) return fail(CUDAHM_EINVAL, "bad sweep counts");
  if (n_iter > 0 && thin < 1) return fail(CUDAHM_EINVAL, "thin must be >= 1");
  cudahm* h0 = hs[0];
  if (!h0) return fail(CUDAHM_EINVAL, "handle 0 is NULL");
  for (int q = 0; q < k; ++q) {
    cudahm* h = hs[q];
    if (!h) return fail(CUDAHM_EINVAL, "handle %d is NULL", q);
    if (!h->data_set) return fail(CUDAHM_ESTATE, "handle %d has no data", q);
    if (h->shard_active) return fail(CUDAHM_ESTATE, "handle %d is in a sharded run", q);
    if (h->cfg.marginal) return fail(CUDAHM_EUNSUPPORTED, "handle %d uses the marginal form, which runs alone", q);
    if (h->cfg.device != h0->cfg.device) return fail(CUDAHM_EINVAL, "handles are on different devices");
    if (h->cfg.precision != h0->cfg.precision) return fail(CUDAHM_EINVAL, "handles mix precisions");
    if (h->cfg.trace_sweeps > 0 && k > 1)
      return fail(CUDAHM_EUNSUPPORTED, "only a batch of one population records a trace");
    for (int r = 0; r < q; ++r)
      if (hs[r] == h) return fail(CUDAHM_EINVAL, "handle %d appears twice", q);
    if (h->sweeps + n_burn + n_iter >= (1ll << 32) - 2) return fail(CUDAHM_EINVAL, "sweep counter would overflow");
  }
  const bool f32 = h0->cfg.precision == CUDAHM_FP32;
  bool d1 = true;  // one-dimensional latents only: the lighter kernel variant
  bool any1 = false;  // some one-dimensional population (FP32: member tiles in shared memory)
  for (int q = 0; q < k; ++q) {
    d1 = d1 && hs[q]->d == 1;
    any1 = any1 || hs[q]->d == 1;
  }
  CU(cudaSetDevice(h0->cfg.device));
  cudaStream_t st = h0->stream;
  for (int q = 0; q < k; ++q) CU(cudaStreamSynchronize(hs[q]->stream));
  const long long total = n_burn + n_iter;
  const long long nrows = (n_iter > 0) ? n_iter / thin : 0;

  // per-handle preparation: sample buffer, selection integral at the current theta
  for (int q = 0; q < k; ++q) {
    cudahm* h = hs[q];
    if (nrows > h->rows_cap) {
      h->dfree(h->rows);
      h->rows = nullptr;
      TRY(alloc_into(h, &h->rows, static_cast<size_t>(nrows) * h->p));
      h->rows_cap = nrows;
    }
    if (has_rule(h->cfg.model) && !h->etabar_valid) {
      char* base = reinterpret_cast<char*>(h->chain);
      TRY(compute_etabar_into(h, reinterpret_cast<const double*>(base + offsetof(ChainState, theta)),
                              reinterpret_cast<double*>(base + offsetof(ChainState, etabar))));
      h->etabar_valid = true;
    }
    TRY(ensure_trace(h, std::min<long long>(h->cfg.trace_sweeps, total)));
    CU(cudaStreamSynchronize(h->stream));
  }

  // launch shape: asked for, cached from an earlier tuned run of the same kind, or tuned here
  int nlf = 0;
  long long ntot = 0;
  for (int q = 0; q < k; ++q) {
    nlf += has_rule(hs[q]->cfg.model);
    ntot += hs[q]->n;
  }
  TuneKey key{h0->cfg.precision, k, nlf, static_cast<long long>(std::log2(static_cast<double>(ntot) + 1.0))};
  int block = tune && tune->block_threads ? tune->block_threads : 0;
  int chunk = tune && tune->sweeps_per_launch ? tune->sweeps_per_launch : 0;
  int grid_ask = tune && tune->grid_blocks ? tune->grid_blocks : 0;
  const bool use_graph = !tune || tune->use_graph != 0 || (tune->block_threads == 0 && tune->sweeps_per_launch == 0);
  if (block && block != 128 && block != 256) return fail(CUDAHM_EINVAL, "block_threads must be 128 or 256");
  if (chunk < 0 || chunk > kChunk) return fail(CUDAHM_EINVAL, "sweeps_per_launch must be in [1, %lld]", kChunk);
  if (grid_ask < 0) return fail(CUDAHM_EINVAL, "grid_blocks must be >= 0");
  bool cached = false;
  if (!block || !chunk || !grid_ask) {
    for (const TuneEntry& e : g_tune_cache)
      if (e.key == key) {
        if (!block) block = e.block;
        if (!chunk) chunk = e.chunk;
        if (!grid_ask) grid_ask = e.grid;
        cached = true;
      }
  }

  const int R = 128;  // segment slots per block
  int sms = h0->sms;

  BatchBufs bb;
  bb.owner = h0;
  const int max_grid = 4 * sms * 2;  // 128-thread blocks, up to 8 per SM
  TRY(alloc_into(h0, &bb.pops, k));
  TRY(alloc_into(h0, &bb.progs, k));
  TRY(alloc_into(h0, &bb.b0s, k));
  TRY(alloc_into(h0, &bb.nbs, k));
  TRY(alloc_into(h0, &bb.partials, 2ull * max_grid * kPartWords));
  TRY(alloc_into(h0, &bb.bars, k));
  TRY(alloc_into(h0, &bb.errs, k));

  std::vector<SweepArgs> pops(k);
  std::vector<BatchProg> progs(k);
  std::vector<double> cost(k);
  std::vector<int> cap(k);
  for (int q = 0; q < k; ++q) {
    cudahm* h = hs[q];
    SweepArgs a = base_args(h);
    a.partials = bb.partials;
    a.bar = bb.bars + q;
    a.err = bb.errs + q;
    a.rows = h->rows;
    a.thin = thin;
    a.trace_T = std::min<long long>(h->cfg.trace_sweeps, total);
    a.tr_delta = h->tr_delta;
    a.tr_u = h->tr_u;
    a.tr_acc = h->tr_acc;
    a.tr_thprop = h->tr_thprop;
    a.tr_D = h->tr_D;
    a.tr_logalpha = h->tr_logalpha;
    a.tr_ut = h->tr_ut;
    a.tr_tacc = h->tr_tacc;
    a.tr_eb = h->tr_eb;
    a.skip_cta = -1;
    pops[q] = a;
    progs[q] = BatchProg{total, 0, n_burn, thin, 0, 0};
    cost[q] = pop_cost(h);
    long long c = (h->n + 31) / 32;
    if (has_rule(h->cfg.model)) c += 8;  // the rule's outer nodes need no more than a few blocks
    cap[q] = static_cast<int>(std::min<long long>(c, max_grid));
  }
  CU(cudaMemcpyAsync(bb.pops, pops.data(), sizeof(SweepArgs) * k, cudaMemcpyHostToDevice, st));
  CU(cudaMemcpyAsync(bb.progs, progs.data(), sizeof(BatchProg) * k, cudaMemcpyHostToDevice, st));
  CU(cudaMemsetAsync(bb.errs, 0, sizeof(int) * k, st));

  // the largest grid the occupancy allows for a block size (128-thread blocks up to 8 per SM)
  auto grid_max = [&](int blk, int* out) -> int {
    int bps = 0;
    CU(batch_occupancy(f32, d1, blk, static_cast<int>(batch_smem_bytes(f32, any1, blk)), &bps));
    if (bps < 1) return fail(CUDAHM_EUNSUPPORTED, "batched kernel does not fit on this device");
    *out = std::min(bps * sms, blk == 128 ? max_grid : max_grid / 2);
    return CUDAHM_OK;
  };

  // The plan of launches. Autotuning (no shape asked for and none cached): trial launches of
  // kTrialSweeps sweeps, part of the run, over block sizes {128, 256} x grids {the occupancy's
  // maximum, half of it}; the fastest device time per sweep wins. Then (tuned or not) a few short
  // launches whose per-population device times rebalance the blocks, then long launches. Sweeps
  // per launch of the long launches (asked for, else cached, else tuned): enough that the measured
  // host cost of a launch (synchronisation, graph launch, reading the error words) stays near 1%
  // of its device time, at most 4096.
  struct Shape {
    int block, grid;
  };
  const int kTrialSweeps = 16, kBalanceSweeps = 32;
  std::vector<Shape> trials;
  const bool tuning = !cached && (!block || !grid_ask || !chunk);
  if (tuning) {
    for (int blk : {128, 256}) {
      if (block && blk != block) continue;
      int g = 0;
      TRY(grid_max(blk, &g));
      if (grid_ask) {
        trials.push_back({blk, std::min(grid_ask, g)});
      } else {
        trials.push_back({blk, g});
        if (g / 2 >= k) trials.push_back({blk, g / 2});
      }
    }
  }
  Shape best{block ? block : 128, 0};
  if (!tuning) {
    int g = 0;
    TRY(grid_max(best.block, &g));
    best.grid = grid_ask ? std::min(grid_ask, g) : g;
  }

  cudaGraphExec_t gexec = nullptr;
  int g_block = 0, g_chunk = 0, g_grid = 0;
  std::vector<int> nb;
  auto set_alloc = [&](int grid_) -> int {
    std::vector<int> b0(k);
    int acc = 0;
    for (int q = 0; q < k; ++q) {
      b0[q] = acc;
      acc += nb[q];
    }
    if (acc > grid_) return fail(CUDAHM_EUNSUPPORTED, "%d populations need more blocks than fit (%d)", k, grid_);
    CU(cudaMemcpyAsync(bb.b0s, b0.data(), sizeof(int) * k, cudaMemcpyHostToDevice, st));
    CU(cudaMemcpyAsync(bb.nbs, nb.data(), sizeof(int) * k, cudaMemcpyHostToDevice, st));
    CU(cudaStreamSynchronize(st));
    return CUDAHM_OK;
  };
  auto enqueue = [&](int blk, int ch, int grid_) -> cudaError_t {
    const int smem = static_cast<int>(batch_smem_bytes(f32, any1, blk));
    cudaError_t e = cudaMemsetAsync(bb.bars, 0, sizeof(unsigned int) * k, st);
    if (e == cudaSuccess) e = launch_batch_tables(bb.pops, bb.progs, k, ch, st);
    if (e == cudaSuccess) e = launch_batch(f32, d1, bb.pops, bb.progs, bb.b0s, bb.nbs, k, ch, R, grid_, blk, smem, st);
    return e;
  };

  long long done = 0;
  double best_ms = 1e300, host_ms_per_launch = 0.0;
  int host_samples = 0;
  bool graph_ok = use_graph;
  float run_ms_total = 0.f;
  cudaEvent_t ea, eb;
  CU(cudaEventCreate(&ea));
  CU(cudaEventCreate(&eb));
  auto cleanup_events = [&]() {
    cudaEventDestroy(ea);
    cudaEventDestroy(eb);
    if (gexec) cudaGraphExecDestroy(gexec);
  };
  int rc = CUDAHM_OK;
  size_t ti = 0;
  int balance_left = (k > 1) ? 2 : 0;
  while (done < total && rc == CUDAHM_OK) {
    const bool trial = ti < trials.size();
    const bool balance = !trial && balance_left > 0;
    const Shape sh = trial ? trials[ti] : best;
    const long long left = total - done;
    long long ns;
    if (trial) {
      ns = std::min<long long>(kTrialSweeps, left);
    } else if (balance) {
      ns = std::min<long long>(kBalanceSweeps, left);
    } else {
      if (!chunk) {  // the measured host cost of a launch against the device time of a sweep
        const double per = best_ms < 1e299 ? best_ms : 1.0;
        const double hms = host_samples ? host_ms_per_launch / host_samples : 0.05;
        chunk = static_cast<int>(std::min<double>(kChunk, std::max(64.0, std::ceil(100.0 * hms / per))));
      }
      ns = std::min<long long>(chunk, left);
    }
    if (nb.empty() || sh.grid != g_grid) {
      nb = allocate_blocks(cost, cap, sh.grid);
      if ((rc = set_alloc(sh.grid)) != CUDAHM_OK) break;
      if (gexec && sh.grid != g_grid) {
        cudaGraphExecDestroy(gexec);
        gexec = nullptr;
      }
    }
    const auto h0t = std::chrono::steady_clock::now();
    cudaError_t e = cudaSuccess;
    CU(cudaEventRecord(ea, st));
    if (graph_ok && !trial) {
      if (!gexec || g_block != sh.block || g_chunk != ns || g_grid != sh.grid) {
        if (gexec) cudaGraphExecDestroy(gexec);
        gexec = nullptr;
        cudaGraph_t graph = nullptr;
        e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
          const cudaError_t e2 = enqueue(sh.block, static_cast<int>(ns), sh.grid);
          e = cudaStreamEndCapture(st, &graph);
          if (e2 != cudaSuccess) e = e2;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&gexec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        if (e != cudaSuccess) {  // capture not available: plain launches from here on
          cudaGetLastError();
          if (gexec) cudaGraphExecDestroy(gexec);
          gexec = nullptr;
          graph_ok = false;
          e = enqueue(sh.block, static_cast<int>(ns), sh.grid);
        } else {
          g_block = sh.block;
          g_chunk = static_cast<int>(ns);
          e = cudaGraphLaunch(gexec, st);
        }
      } else {
        e = cudaGraphLaunch(gexec, st);
      }
    } else {
      e = enqueue(sh.block, static_cast<int>(ns), sh.grid);
    }
    g_grid = sh.grid;
    if (e != cudaSuccess) {
      rc = fail(CUDAHM_ECUDA, "batched launch failed: %s", cudaGetErrorString(e));
      break;
    }
    CU(cudaEventRecord(eb, st));
    CU(cudaEventSynchronize(eb));
    float ms = 0.f;
    CU(cudaEventElapsedTime(&ms, ea, eb));
    run_ms_total += ms;
    done += ns;
    // stop at the first failing population
    std::vector<int> errs(k);
    CU(cudaMemcpy(errs.data(), bb.errs, sizeof(int) * k, cudaMemcpyDeviceToHost));
    for (int q = 0; q < k && rc == CUDAHM_OK; ++q)
      if (errs[q] != 0) rc = fail(errs[q], "population %d failed with device error %d", q, errs[q]);
    if (rc != CUDAHM_OK) break;
    const double wall_ms =
        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - h0t).count();
    host_ms_per_launch += std::max(0.0, wall_ms - ms);
    ++host_samples;
    if (trial) {
      const double per = ms / static_cast<double>(ns);
      if (per < best_ms) {
        best_ms = per;
        best = sh;
      }
      ++ti;
    } else if (balance) {
      --balance_left;
      if (best_ms >= 1e299) best_ms = ms / static_cast<double>(ns);
    }
    // rebalance from the measured device time of each population (work ~ time x blocks), after
    // every trial and balancing launch
    if (k > 1 && done < total && (trial || balance)) {
      std::vector<BatchProg> pr(k);
      CU(cudaMemcpy(pr.data(), bb.progs, sizeof(BatchProg) * k, cudaMemcpyDeviceToHost));
      bool ok = true;
      for (int q = 0; q < k; ++q) ok = ok && pr[q].t_ns > 0;
      if (ok) {
        for (int q = 0; q < k; ++q) cost[q] = static_cast<double>(pr[q].t_ns) * nb[q];
        const int gnext = (ti < trials.size()) ? trials[ti].grid : best.grid;
        nb = allocate_blocks(cost, cap, gnext);
        if ((rc = set_alloc(gnext)) != CUDAHM_OK) break;
        g_grid = gnext;
        if (gexec) {
          cudaGraphExecDestroy(gexec);
          gexec = nullptr;
        }
      }
    }
  }
  if (rc == CUDAHM_OK && tuning) {
    g_tune_cache.push_back(TuneEntry{key, best.block, chunk ? chunk : static_cast<int>(kChunk), best.grid});
  }
  cleanup_events();
  if (rc != CUDAHM_OK) {
    for (int q = 0; q < k; ++q) {
      ChainState cs;
      if (cudaMemcpy(&cs, hs[q]->chain, sizeof(cs), cudaMemcpyDeviceToHost) == cudaSuccess) hs[q]->sweeps = cs.sweeps;
      hs[q]->rows_last = 0;
      hs[q]->rows_host_n = 0;
    }
    return rc;
  }
  CU(cudaStreamSynchronize(st));
  for (int q = 0; q < k; ++q) {
    cudahm* h = hs[q];
    h->sweeps += total;
    h->rows_last = nrows;
    h->rows_host_n = 0;  // the batched run leaves its rows on the device
    h->trace_T_last = std::min<long long>(h->cfg.trace_sweeps, total);
    h->last_run_ms = run_ms_total;
  }
  if (chosen) {
    chosen->block_threads = best.block;
    chosen->sweeps_per_launch = chunk ? chunk : static_cast<int>(std::min<long long>(total, kChunk));
    chosen->use_graph = graph_ok ? 1 : 0;
    chosen->grid_blocks = best.grid;
  }
  return CUDAHM_OK;
}

// ---------------------------------------------------------------- serving --
namespace {

// One chunk of sweeps for handles at their own stages (progs: host mirrors, updated).
int batch_step(const std::vector<cudahm*>& hs, std::vector<BatchProg>& progs, int chunk, int block, BatchBufs& bb,
               int max_grid, cudaStream_t st, bool f32) {
  const int k = static_cast<int>(hs.size());
  const int R = 128;
  bool d1 = true, any1 = false;
  for (const cudahm* h : hs) {
    d1 = d1 && h->d == 1;
    any1 = any1 || h->d == 1;
  }
  const int smem = static_cast<int>(batch_smem_bytes(f32, any1, block));
  int bps = 0;
  CU(batch_occupancy(f32, d1, block, smem, &bps));
  if (bps < 1) return fail(CUDAHM_EUNSUPPORTED, "batched kernel does not fit on this device");
  const int grid = std::min(bps * hs[0]->sms, block == 128 ? max_grid : max_grid / 2);
  std::vector<SweepArgs> pops(k);
  std::vector<double> cost(k);
  std::vector<int> cap(k);
  for (int q = 0; q < k; ++q) {
    cudahm* h = hs[q];
    SweepArgs a = base_args(h);
    a.partials = bb.partials;
    a.bar = bb.bars + q;
    a.err = bb.errs + q;
    a.rows = h->rows;
    a.thin = progs[q].thin;
    a.trace_T = 0;
    a.skip_cta = -1;
    pops[q] = a;
    cost[q] = pop_cost(h);
    long long c = (h->n + 31) / 32;
    if (has_rule(h->cfg.model)) c += 8;  // the rule's outer nodes need no more than a few blocks
    cap[q] = static_cast<int>(std::min<long long>(c, max_grid));
  }
  std::vector<int> nb = allocate_blocks(cost, cap, grid), b0(k);
  int acc = 0;
  for (int q = 0; q < k; ++q) {
    b0[q] = acc;
    acc += nb[q];
  }
  if (acc > grid) return fail(CUDAHM_EUNSUPPORTED, "%d populations need more blocks than fit (%d)", k, grid);
  CU(cudaMemcpyAsync(bb.pops, pops.data(), sizeof(SweepArgs) * k, cudaMemcpyHostToDevice, st));
  CU(cudaMemcpyAsync(bb.progs, progs.data(), sizeof(BatchProg) * k, cudaMemcpyHostToDevice, st));
  CU(cudaMemcpyAsync(bb.b0s, b0.data(), sizeof(int) * k, cudaMemcpyHostToDevice, st));
  CU(cudaMemcpyAsync(bb.nbs, nb.data(), sizeof(int) * k, cudaMemcpyHostToDevice, st));
  CU(cudaMemsetAsync(bb.errs, 0, sizeof(int) * k, st));
  CU(cudaMemsetAsync(bb.bars, 0, sizeof(unsigned int) * k, st));
  CU(launch_batch_tables(bb.pops, bb.progs, k, chunk, st));
  CU(launch_batch(f32, d1, bb.pops, bb.progs, bb.b0s, bb.nbs, k, chunk, R, grid, block, smem, st));
  CU(cudaMemcpyAsync(progs.data(), bb.progs, sizeof(BatchProg) * k, cudaMemcpyDeviceToHost, st));
  std::vector<int> errs(k);
  CU(cudaMemcpyAsync(errs.data(), bb.errs, sizeof(int) * k, cudaMemcpyDeviceToHost, st));
  CU(cudaStreamSynchronize(st));
  for (int q = 0; q < k; ++q)
    if (errs[q] != 0) return fail(errs[q], "population %d failed with device error %d", q, errs[q]);
  return CUDAHM_OK;
}

double now_ms() {
  using namespace std::chrono;
  return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

struct Request {
  uint64_t ticket = 0;
  cudahm_config cfg{};
  std::vector<double> y, aux;
  long long n_burn = 0, n_iter = 0, thin = 1;
  size_t bytes = 0;
  double t_submit = 0, t_admit = 0, t_done = 0;
  cudahm* h = nullptr;
  BatchProg prog{};
  std::vector<double> rows;
  int state = 0;  // 0 queued, 1 active, 2 done
  int err = 0;
  std::string msg;
};

size_t request_bytes(const cudahm_config& c, long long n_iter, long long thin) {
  const size_t n = static_cast<size_t>(c.n), d = c.d;
  const size_t p = model_p(c.model);
  size_t b = n * (4 * 8 + d * 8 + d * d * 8) + (c.precision == CUDAHM_FP32 ? n * 7 * 4 : 0);  // FP32: data, latent, draws
  b += static_cast<size_t>(n_iter / std::max<long long>(thin, 1)) * p * 8;
  b += static_cast<size_t>(kChunk) * (p + 3) * 8 + 64 * 1024;
  if (has_rule(c.model)) b += static_cast<size_t>(8 * 4096 + 2048 + 1024 * (kHDeg + 1)) * 8;  // rule, H table
  if (d == 3 && c.precision == CUDAHM_FP64) b += 3 * n * 8;  // Box-Muller spares
  if (c.keep_chi_moments) b += 4 * d * n * 8;
  b += static_cast<size_t>(kMargNodeWords) * 8;
  return b;
}

}  // namespace

struct cudahm_server {
  size_t budget = 0, in_use = 0;
  int device = 0, max_active = 0, chunk = 0, precision = 0, block = 128;
  cudaStream_t stream = nullptr;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<Request*> pending;
  std::vector<Request*> active;
  std::map<uint64_t, Request*> all;
  uint64_t next_ticket = 1;
  bool stop = false;
  std::thread worker;
  cudahm* owner = nullptr;  // buffer owner (a tiny handle that only provides the allocator)
  BatchBufs bb;
  int max_grid = 0;
  long long done_count = 0;
  double member_sweeps = 0.0;  // sum of n x sweeps over completed requests
  double busy_ms = 0.0;
};

namespace {

void serve_loop(cudahm_server* sv) {
  cudaSetDevice(sv->device);
  std::vector<Request*> admitted;
  while (true) {
    {
      std::unique_lock<std::mutex> lk(sv->mu);
      sv->cv.wait_for(lk, std::chrono::milliseconds(20),
                      [&] { return sv->stop || !sv->pending.empty() || !sv->active.empty(); });
      if (sv->stop) return;
      // continuous batching: admit in arrival order while a slot and the memory budget allow
      while (!sv->pending.empty() && static_cast<int>(sv->active.size() + admitted.size()) < sv->max_active &&
             sv->in_use + sv->pending.front()->bytes <= sv->budget) {
        Request* r = sv->pending.front();
        sv->pending.pop_front();
        sv->in_use += r->bytes;
        r->t_admit = now_ms();
        admitted.push_back(r);
      }
      if (sv->active.empty() && admitted.empty()) continue;
    }
    for (Request* r : admitted) {  // create and load outside the lock
      cudahm_t h = nullptr;
      r->cfg.cuda_stream = sv->stream;
      int rc = cudahm_create(&r->cfg, &h);
      if (rc == CUDAHM_OK) rc = cudahm_set_data(h, r->y.data(), r->aux.data(), r->cfg.n);
      if (rc == CUDAHM_OK && has_rule(r->cfg.model)) {
        char* base = reinterpret_cast<char*>(h->chain);
        rc = compute_etabar_into(h, reinterpret_cast<const double*>(base + offsetof(ChainState, theta)),
                                 reinterpret_cast<double*>(base + offsetof(ChainState, etabar)));
        h->etabar_valid = true;
      }
      const long long nrows = r->n_iter > 0 ? r->n_iter / r->thin : 0;
      if (rc == CUDAHM_OK && nrows > 0) {
        rc = alloc_into(h, &h->rows, static_cast<size_t>(nrows) * h->p);
        h->rows_cap = nrows;
      }
      std::lock_guard<std::mutex> lk(sv->mu);
      if (rc != CUDAHM_OK) {
        r->err = rc;
        r->msg = cudahm_last_error();
        r->state = 2;
        r->t_done = now_ms();
        sv->in_use -= r->bytes;
        if (h) cudahm_destroy(h);
        r->y.clear();
        r->aux.clear();
        sv->cv.notify_all();
        continue;
      }
      r->h = h;
      r->prog = BatchProg{r->n_burn + r->n_iter, 0, r->n_burn, r->thin, 0, 0};
      r->state = 1;
      r->y.clear();
      r->y.shrink_to_fit();
      r->aux.clear();
      r->aux.shrink_to_fit();
      sv->active.push_back(r);
    }
    admitted.clear();
    std::vector<cudahm*> hs;
    std::vector<BatchProg> progs;
    std::vector<Request*> act;
    {
      std::lock_guard<std::mutex> lk(sv->mu);
      act = sv->active;
    }
    if (act.empty()) continue;
    for (Request* r : act) {
      hs.push_back(r->h);
      progs.push_back(r->prog);
    }
    const double t0 = now_ms();
    const int rc = batch_step(hs, progs, sv->chunk, sv->block, sv->bb, sv->max_grid, sv->stream,
                              sv->precision == CUDAHM_FP32);
    const double t1 = now_ms();
    std::vector<Request*> finished;
    {
      std::lock_guard<std::mutex> lk(sv->mu);
      sv->busy_ms += t1 - t0;
      for (size_t q = 0; q < act.size(); ++q) {
        Request* r = act[q];
        if (rc != CUDAHM_OK) {
          r->err = rc;
          r->msg = cudahm_last_error();
        } else {
          r->prog = progs[q];
        }
        if (rc != CUDAHM_OK || r->prog.off >= r->prog.total) finished.push_back(r);
      }
      for (Request* r : finished) sv->active.erase(std::find(sv->active.begin(), sv->active.end(), r));
    }
    for (Request* r : finished) {  // collect results and release memory outside the lock
      if (r->err == 0 && r->prog.rows > 0) {
        r->rows.resize(static_cast<size_t>(r->prog.rows) * r->h->p);
        cudaMemcpy(r->rows.data(), r->h->rows, sizeof(double) * r->rows.size(), cudaMemcpyDeviceToHost);
      }
      const double ms = now_ms();
      cudahm_destroy(r->h);
      r->h = nullptr;
      std::lock_guard<std::mutex> lk(sv->mu);
      r->t_done = ms;
      r->state = 2;
      sv->in_use -= r->bytes;
      if (r->err == 0) {
        sv->done_count++;
        sv->member_sweeps += static_cast<double>(r->cfg.n) * static_cast<double>(r->prog.total);
      }
      sv->cv.notify_all();
    }
  }
}

}  // namespace

int cudahm_server_create(size_t mem_budget_bytes, int32_t device, int32_t precision, int32_t max_active,
                         int32_t sweeps_per_step, cudahm_server_t* out) {
  if (!out) return fail(CUDAHM_EINVAL, "out is NULL");
  if (precision != CUDAHM_FP64 && precision != CUDAHM_FP32) return fail(CUDAHM_EINVAL, "unknown precision");
  if (max_active < 1 || max_active > 4096) return fail(CUDAHM_EINVAL, "max_active must be in [1, 4096]");
  if (sweeps_per_step < 1 || sweeps_per_step > kChunk) return fail(CUDAHM_EINVAL, "bad sweeps_per_step");
  if (mem_budget_bytes == 0) return fail(CUDAHM_EINVAL, "memory budget is zero");
  int ndev = 0;
  CU(cudaGetDeviceCount(&ndev));
  if (device < 0 || device >= ndev) return fail(CUDAHM_EINVAL, "device %d not present", device);
  CU(cudaSetDevice(device));
  auto* sv = new cudahm_server();
  sv->budget = mem_budget_bytes;
  sv->device = device;
  sv->precision = precision;
  sv->max_active = max_active;
  sv->chunk = sweeps_per_step;
  if (cudaStreamCreateWithFlags(&sv->stream, cudaStreamNonBlocking) != cudaSuccess) {
    delete sv;
    return fail(CUDAHM_ECUDA, "cannot create the server stream");
  }
  // a one-member handle provides the allocator and device properties for the server's buffers
  cudahm_config oc;
  cudahm_config_init(&oc, CUDAHM_NN1, 1);
  oc.device = device;
  oc.adapt_theta = 0;
  oc.cuda_stream = sv->stream;
  int rc = cudahm_create(&oc, &sv->owner);
  if (rc == CUDAHM_OK) {
    sv->bb.owner = sv->owner;
    sv->max_grid = 8 * sv->owner->sms;
    if ((rc = alloc_into(sv->owner, &sv->bb.pops, max_active)) == CUDAHM_OK &&
        (rc = alloc_into(sv->owner, &sv->bb.progs, max_active)) == CUDAHM_OK &&
        (rc = alloc_into(sv->owner, &sv->bb.b0s, max_active)) == CUDAHM_OK &&
        (rc = alloc_into(sv->owner, &sv->bb.nbs, max_active)) == CUDAHM_OK &&
        (rc = alloc_into(sv->owner, &sv->bb.partials, 2ull * sv->max_grid * kPartWords)) == CUDAHM_OK &&
        (rc = alloc_into(sv->owner, &sv->bb.bars, max_active)) == CUDAHM_OK)
      rc = alloc_into(sv->owner, &sv->bb.errs, max_active);
  }
  if (rc != CUDAHM_OK) {
    sv->bb.owner = nullptr;
    if (sv->owner) cudahm_destroy(sv->owner);
    cudaStreamDestroy(sv->stream);
    delete sv;
    return rc;
  }
  sv->worker = std::thread(serve_loop, sv);
  *out = sv;
  return CUDAHM_OK;
}

int cudahm_server_submit(cudahm_server_t sv, const cudahm_config* cfg, const double* y_host, const double* aux_host,
                         int64_t n_burn, int64_t n_iter, int64_t thin, uint64_t* ticket) {
  if (!sv || !cfg || !y_host || !aux_host || !ticket) return fail(CUDAHM_EINVAL, "NULL argument");
  TRY(validate(cfg));
  if (cfg->precision != sv->precision) return fail(CUDAHM_EINVAL, "request precision differs from the server's");
  if (cfg->device != sv->device) return fail(CUDAHM_EINVAL, "request device differs from the server's");
  if (cfg->trace_sweeps > 0) return fail(CUDAHM_EUNSUPPORTED, "served requests do not record traces");
  if (cfg->marginal) return fail(CUDAHM_EUNSUPPORTED, "served requests use the member form");
  if (cfg->keep_chi_moments) return fail(CUDAHM_EUNSUPPORTED, "served requests return theta rows only");
  if (n_burn < 0 || n_iter < 0 || n_burn + n_iter < 1 || (n_iter > 0 && thin < 1))
    return fail(CUDAHM_EINVAL, "bad sweep counts");
  auto* r = new Request();
  r->cfg = *cfg;
  r->cfg.dev_alloc = nullptr;
  r->cfg.dev_free = nullptr;
  r->n_burn = n_burn;
  r->n_iter = n_iter;
  r->thin = n_iter > 0 ? thin : 1;
  r->bytes = request_bytes(*cfg, n_iter, r->thin);
  if (r->bytes > sv->budget) {
    const size_t need = r->bytes;
    delete r;
    return fail(CUDAHM_ENOMEM, "request needs about %zu bytes, more than the whole budget", need);
  }
  const size_t cnt = static_cast<size_t>(cfg->n) * cfg->d;
  r->y.assign(y_host, y_host + cnt);
  r->aux.assign(aux_host, aux_host + cnt);
  std::lock_guard<std::mutex> lk(sv->mu);
  r->ticket = sv->next_ticket++;
  r->t_submit = now_ms();
  sv->pending.push_back(r);
  sv->all[r->ticket] = r;
  *ticket = r->ticket;
  sv->cv.notify_all();
  return CUDAHM_OK;
}

int cudahm_server_poll(cudahm_server_t sv, uint64_t ticket, int32_t* done) {
  if (!sv || !done) return fail(CUDAHM_EINVAL, "NULL argument");
  std::lock_guard<std::mutex> lk(sv->mu);
  auto it = sv->all.find(ticket);
  if (it == sv->all.end()) return fail(CUDAHM_EINVAL, "unknown ticket %llu", (unsigned long long)ticket);
  *done = it->second->state == 2 ? 1 : 0;
  return CUDAHM_OK;
}

int cudahm_server_wait(cudahm_server_t sv, uint64_t ticket, int64_t timeout_ms) {
  if (!sv) return fail(CUDAHM_EINVAL, "NULL argument");
  std::unique_lock<std::mutex> lk(sv->mu);
  auto it = sv->all.find(ticket);
  if (it == sv->all.end()) return fail(CUDAHM_EINVAL, "unknown ticket %llu", (unsigned long long)ticket);
  Request* r = it->second;
  const bool ok = sv->cv.wait_for(lk, std::chrono::milliseconds(timeout_ms < 0 ? (1ll << 40) : timeout_ms),
                                  [&] { return r->state == 2; });
  if (!ok) return fail(CUDAHM_ETIMEOUT, "request %llu not done within %lld ms", (unsigned long long)ticket,
                       (long long)timeout_ms);
  return CUDAHM_OK;
}

int cudahm_server_result(cudahm_server_t sv, uint64_t ticket, double* theta_host, int64_t cap_rows,
                         int64_t* rows_out, double* latency_ms) {
  if (!sv) return fail(CUDAHM_EINVAL, "NULL argument");
  std::lock_guard<std::mutex> lk(sv->mu);
  auto it = sv->all.find(ticket);
  if (it == sv->all.end()) return fail(CUDAHM_EINVAL, "unknown ticket %llu", (unsigned long long)ticket);
  Request* r = it->second;
  if (r->state != 2) return fail(CUDAHM_ESTATE, "request %llu is not done", (unsigned long long)ticket);
  if (r->err != 0) {
    const int e = r->err;
    const std::string m = r->msg;
    sv->all.erase(it);
    delete r;
    return fail(e, "request failed: %s", m.c_str());
  }
  const int p = model_p(r->cfg.model);
  const long long rows = static_cast<long long>(r->rows.size()) / p;
  if (rows_out) *rows_out = rows;
  if (latency_ms) *latency_ms = r->t_done - r->t_submit;
  if (theta_host && cap_rows > 0)
    std::memcpy(theta_host, r->rows.data(), sizeof(double) * std::min<long long>(rows, cap_rows) * p);
  sv->all.erase(it);
  delete r;
  return CUDAHM_OK;
}

int cudahm_server_stats(cudahm_server_t sv, int64_t* completed, double* member_sweeps, double* busy_ms,
                        int64_t* queued, int64_t* active) {
  if (!sv) return fail(CUDAHM_EINVAL, "NULL argument");
  std::lock_guard<std::mutex> lk(sv->mu);
  if (completed) *completed = sv->done_count;
  if (member_sweeps) *member_sweeps = sv->member_sweeps;
  if (busy_ms) *busy_ms = sv->busy_ms;
  if (queued) *queued = static_cast<int64_t>(sv->pending.size());
  if (active) *active = static_cast<int64_t>(sv->active.size());
  return CUDAHM_OK;
}

int cudahm_server_destroy(cudahm_server_t sv) {
  if (!sv) return CUDAHM_OK;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->stop = true;
  }
  sv->cv.notify_all();
  if (sv->worker.joinable()) sv->worker.join();
  cudaSetDevice(sv->device);
  for (Request* r : sv->active)
    if (r->h) cudahm_destroy(r->h);
  for (auto& kv : sv->all) delete kv.second;
  // the batch buffers go back through their owner, then the owner itself
  for (void* q : {(void*)sv->bb.pops, (void*)sv->bb.progs, (void*)sv->bb.b0s, (void*)sv->bb.nbs,
                  (void*)sv->bb.partials, (void*)sv->bb.bars, (void*)sv->bb.errs})
    sv->owner->dfree(q);
  sv->bb.owner = nullptr;
  cudahm_destroy(sv->owner);
  cudaStreamDestroy(sv->stream);
  delete sv;
  return CUDAHM_OK;
}

}  // extern "C"
