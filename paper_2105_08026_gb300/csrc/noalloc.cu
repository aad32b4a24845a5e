// Selection integral etabar(theta) without any device allocation.
//
// Some programs cannot call cudaMalloc when they need this value: a serving process
// that hands all device memory to its own pool at start-up and forbids any later
// allocation, a latency-critical loop that must not pay for the device-wide
// synchronisation an allocation implies, or a caller that has simply run out of
// device memory. cudahm_lf_etabar_noalloc serves them: every table and partial sum
// it needs lives in one fixed array compiled into this library (g_noalloc_scratch
// below), so the call allocates nothing. The caller passes theta and receives the
// result in its own device memory.
//
// The array belongs to every GPU that loads the library and stays allocated until the
// process exits. All calls on a device share it and it keeps what the last call wrote;
// nothing in it needs to start at zero. A call rebuilds the rule tables unless the previous
// call on the device built them for the same n_L, n_r, r_max and sigma_F (then it only
// rewrites the partial sums it reads). Calls whose work overlaps on the GPU (two host
// threads, or two streams) race on the array and may return wrong values: serialise them,
// and when consecutive calls use different streams, let the earlier call's work finish
// first (a call that reuses the tables reads what the earlier one wrote).
#include <cuda_runtime.h>

#include <mutex>

#include "cudahm.h"
#include "internal.h"

namespace chm {
namespace {

constexpr int kNoallocMaxNodes = CUDAHM_NOALLOC_MAX_NODES;
constexpr int kNoallocMaxGrid = 1024;
constexpr int kPhiWordsMax = 265 * 9;  // normal-CDF Taylor table
constexpr int kMathWordsMax = 506;     // exp/log/sin/cos tables
// layout in doubles: xL, wL, xr, wr, qs, Wr (max nodes each), the Phi table, the exp/log table,
// the prefix sums of the inner weights (max nodes + 1), then the per-block partials (4 x u64
// per block)
constexpr size_t kScratchDoubles = 6 * static_cast<size_t>(kNoallocMaxNodes) + kPhiWordsMax + kMathWordsMax +
                                   (kNoallocMaxNodes + 1) + 4 * static_cast<size_t>(kNoallocMaxGrid);

static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_addr[kMaxDevices] = {nullptr};
// What the array's rule tables were last built for, per device: the Gauss-Legendre nodes and the
// inner-rule tables depend on (n_L, n_r, r_max, sigma_F) only; the normal-CDF and exp/log tables
// on nothing. A call with the same constants skips the rebuild (about a millisecond of kernels).
struct RuleTag {
  bool valid;
  int nL, nr;
  double rmax, sigF;
};
RuleTag g_tag[kMaxDevices] = {};

int noalloc_fail(int code, const char* msg) { return record_error(code, msg); }

}  // namespace
}  // namespace chm

using namespace chm;

extern "C" int cudahm_lf_etabar_noalloc(const double* theta_dev, const double* consts_host, double* etabar_dev,
                                        void* cuda_stream) {
  if (!theta_dev || !consts_host || !etabar_dev) return noalloc_fail(CUDAHM_EINVAL, "NULL argument");
  const double sigF = consts_host[0], Fth = consts_host[1], rmax = consts_host[2];
  const double nLd = consts_host[3], nrd = consts_host[4], ln_upper = consts_host[5];
  if (!(sigF > 0.0) || !(Fth > 0.0) || !(rmax > 0.0) || !(ln_upper > 0.0))
    return noalloc_fail(CUDAHM_EINVAL, "sigma_F, F_th, r_max and ln(upper/L*) must be positive");
  if (!(nLd >= 1.0 && nLd <= kNoallocMaxNodes && nLd == static_cast<double>(static_cast<int>(nLd))) ||
      !(nrd >= 1.0 && nrd <= kNoallocMaxNodes && nrd == static_cast<double>(static_cast<int>(nrd))))
    return noalloc_fail(CUDAHM_EINVAL,
                        "rule sizes n_L and n_r must be integers in [1, 1024] (the fixed scratch array's limit)");
  const int nL = static_cast<int>(nLd), nr = static_cast<int>(nrd);
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return noalloc_fail(CUDAHM_ECUDA, "cannot query the current device");
  double* base = nullptr;
  bool rebuild = true;
  {
    // once per device, with that device current: the device address of the fixed array
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
      void* p = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess || !p) return noalloc_fail(CUDAHM_ECUDA, "cudaGetSymbolAddress of the scratch array failed");
      g_addr[dev] = static_cast<double*>(p);
    }
    base = g_addr[dev];
    const RuleTag& t = g_tag[dev];
    rebuild = !(t.valid && t.nL == nL && t.nr == nr && t.rmax == rmax && t.sigF == sigF);
    g_tag[dev].valid = false;  // set again below once the rebuild is enqueued
  }
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return noalloc_fail(CUDAHM_ECUDA, "cannot query the SM count");
  const int grid = (4 * sms < kNoallocMaxGrid) ? 4 * sms : kNoallocMaxGrid;

  double* xL = base;
  double* wL = xL + kNoallocMaxNodes;
  double* xr = wL + kNoallocMaxNodes;
  double* wr = xr + kNoallocMaxNodes;
  double* qs = wr + kNoallocMaxNodes;
  double* Wr = qs + kNoallocMaxNodes;
  double* phi = Wr + kNoallocMaxNodes;
  double* mtab = phi + kPhiWordsMax;
  double* cw = mtab + kMathWordsMax;
  unsigned long long* partials = reinterpret_cast<unsigned long long*>(cw + kNoallocMaxNodes + 1);
  if (phi_table_words() > kPhiWordsMax) return noalloc_fail(CUDAHM_ECUDA, "normal-CDF table larger than its slot");
  if (math_table_words() > kMathWordsMax) return noalloc_fail(CUDAHM_ECUDA, "exp/log table larger than its slot");

  // the rule tables, rewritten on the caller's stream unless the last call built them for the
  // same constants
  cudaError_t e = cudaSuccess;
  if (rebuild) {
    e = launch_gauss_legendre(nL, xL, wL, st);
    if (e == cudaSuccess) e = launch_gauss_legendre(nr, xr, wr, st);
    if (e == cudaSuccess) e = launch_lf_inner(nr, xr, wr, rmax, sigF, qs, Wr, st);
    if (e == cudaSuccess) e = launch_phi_table(phi, st);
    if (e == cudaSuccess) e = launch_math_table(mtab, st);
    if (e == cudaSuccess) e = launch_prefix_weights(nr, Wr, cw, st);
    if (e != cudaSuccess) return noalloc_fail(CUDAHM_ECUDA, cudaGetErrorString(e));
  }

  SweepArgs rule{};
  rule.model = CUDAHM_LF;
  rule.p = 3;
  rule.nL = nL;
  rule.nr = nr;
  rule.xL = xL;
  rule.wL = wL;
  rule.qs = qs;
  rule.Wr = Wr;
  rule.phi_coef = phi;
  rule.math_tab = mtab;
  rule.cw = cw;
  rule.mc.cth = Fth / sigF;
  rule.mc.ln_upper = ln_upper;
  const long long G = static_cast<long long>(nL) * ((nr + 127) / 128);
  rule.rows_smem = static_cast<int>((G + grid - 1) / grid);
  e = launch_eval_etabar(theta_dev, rule, partials, grid, etabar_dev, st);
  if (e != cudaSuccess) return noalloc_fail(CUDAHM_ECUDA, cudaGetErrorString(e));
  {
    std::lock_guard<std::mutex> lk(g_mu);
    g_tag[dev] = RuleTag{true, nL, nr, rmax, sigF};
  }
  return CUDAHM_OK;
}

