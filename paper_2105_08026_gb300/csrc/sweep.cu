// Persistent Metropolis-within-Gibbs sweep kernel and its set-up kernels (FP64).
//
// One cooperative launch runs `ns` sweeps. Per sweep (Sec. 2.1, eqs. psi_sampling then
// theta_sampling; Sec. 2.2 for RAM):
//   a0  theta' = theta + S_theta U_theta           (block 0, one sweep ahead for both outcomes of
//                                                   the pending decision; normals from a table)
//   a1  every member: Y = chi + S z                 (Philox4x32-10 -> Box-Muller)
//   a2  accept iff u < exp(lp(Y) - lp(chi))         (lp = log l_i + log f(.;theta))
//   a3  RAM factor S <- S sqrt(1 + eta (alpha - alpha_*))   (d = 1 closed form of Sec. 2.2 step 3)
//   a4  d_i = log f(chi_i;theta') - log f(chi_i;theta) into an exact fixed-point sum
//   a6  LF: etabar(theta') outer terms of the 2-D rule into a second exact sum (Sec. 4.2, eq. epdf)
//   a5  block partials -> exact atomic adds into the grid totals -> bounded grid barrier
//   a7  every block takes the same theta accept decision; block 0 applies its S_theta RAM
//       update one sweep later
//   a8  block 0 records the kept theta row; optionally every member adds its latent to its
//       running moments (Welford)
// Each thread keeps its K members (latent, RAM factor, cached e^chi and log l) in
// registers for the whole launch; data are read once at launch start.
#include <cmath>
#include <cstdint>
#include <type_traits>

#include "sweep_common.cuh"

namespace chm {

__global__ void phi_table_kernel(double* coef) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= kPhiN) return;
  const double c = -8.0 + 0.0625 * i;
  const double dens = exp(-0.5 * (c * c)) * 0.39894228040143267794;  // phi(c)
  coef[i] = (c > 0.0) ? 1.0 - 0.5 * erfc(c * 0.70710678118654752440) : 0.5 * erfc(-c * 0.70710678118654752440);
  double hm1 = 0.0, h = 1.0;  // He_(n-2), He_(n-1) at c
  double fact = 1.0, scale = 1.0;
  for (int n = 1; n <= kPhiDeg; ++n) {
    fact *= n;
    scale *= 0.0625;  // 16^-n, exact
    coef[n * kPhiN + i] = ((n - 1) & 1 ? -h : h) * dens / fact * scale;  // (-1)^(n-1) He_(n-1)(c) phi(c)/(n! 16^n)
    const double hn = c * h - (n - 1) * hm1;  // He_n = c He_(n-1) - (n-1) He_(n-2)
    hm1 = h;
    h = hn;
  }
}

cudaError_t launch_phi_table(double* coef, cudaStream_t st) {
  phi_table_kernel<<<(kPhiN + 127) / 128, 128, 0, st>>>(coef);
  return cudaGetLastError();
}

int phi_table_words() { return kPhiWords; }

// Detection efficiency eta(F) = Phi((F - F_th)/sigma_F) for a list of fluxes.
// LF: sigma_F constant; BB1: sigma(F)^2 = sigma0^2 + (alpha F)^2, evaluated as in the rule's pairs.
__global__ void detection_kernel(int model, long long n, const double* F, ModelConsts mc, double sigma_F,
                                 const double* coef, double* out) {
  const long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (model == CUDAHM_BB1) {
    const double aF = mc.alpha * F[i];
    out[i] = phi_table16(16.0 * (F[i] - mc.F_th) * rsqrt(fma(aF, aF, mc.s0sq)), coef);
  } else {
    out[i] = phi_table((F[i] - mc.F_th) / sigma_F, coef);
  }
}

cudaError_t launch_detection(int model, long long n, const double* F, const ModelConsts& mc, double sigma_F,
                             const double* coef, double* out, cudaStream_t st) {
  const int blk = 256;
  detection_kernel<<<static_cast<unsigned int>((n + blk - 1) / blk), blk, 0, st>>>(model, n, F, mc, sigma_F, coef,
                                                                                   out);
  return cudaGetLastError();
}

// Prefix sums of the inner weights, CW[k] = sum_{k' < k} W_k' (k = 0..nr), each rounded once
// from an exact running sum.
__global__ void prefix_weights_kernel(int nr, const double* Wr, double* cw) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  Xacc acc;
  xacc_zero(acc);
  XFlags f = {0u, 0u, 0u};
  cw[0] = 0.0;
  for (int k = 0; k < nr; ++k) {
    xacc_add_double(acc, Wr[k], f);
    cw[k + 1] = xacc_to_double(acc);
  }
}

cudaError_t launch_prefix_weights(int nr, const double* Wr, double* cw, cudaStream_t st) {
  prefix_weights_kernel<<<1, 1, 0, st>>>(nr, Wr, cw);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- kernel -----
// Work that only the next theta proposal needs (the S_theta RAM update of the previous sweep,
// theta' = theta + S_theta U, its prior and constants, the rule's outer-node values at theta')
// runs on the last warp while every warp does its member steps; only the accept decision
// itself sits between the grid barrier and the next member phase.
// The RAM factor update of a member's previous step, S <- S sqrt(1 + eta (alpha - alpha_*))
// (Sec. 2.2, d = 1), with alpha kept in the member's slot of pu (binary64; binary32 in the upper
// half of the slot array in the FP32 form, which takes the one-FMA form ram1_f32 with eta and
// alpha_* rounded to binary32).
template <bool F32>
__device__ __forceinline__ double ram_pending(const SweepArgs& a, double S, double eta, const double* s_pu,
                                              unsigned int q) {
  if constexpr (F32) {
    return ram1_f32(S, reinterpret_cast<const float*>(s_pu)[a.mpb + q], __double2float_rn(eta),
                    __double2float_rn(a.astar));
  } else {
    return S * sqrt(fma(eta, s_pu[q] - a.astar, 1.0));
  }
}

// The theta-independent half of each member's step for sweep sa of this launch
// (k = k0 + sa + 1): the previous step's RAM factor update (sa > 0), the draws, the proposal
// Y = chi + S z and its log-likelihood (with e^Y), stored per member in shared memory (pY, peY,
// pll, pu). The kernel computes it while the previous sweep's grid barrier completes; the
// theta-dependent half (log f, the accept, alpha) follows the theta decision. Same operations
// as a whole step, so the same bits.
template <class M, int K, bool F32, class R>
__device__ __forceinline__ void sweep_part_a(const SweepArgs& a, long long sa, unsigned int nb0, unsigned int nb1,
                                             const R (&chi)[K], double (&S)[K], const double* s_math,
                                             const double* s_y, const double* s_aux, double* s_zs,
                                             const float* s_d32, double* s_pY, double* s_peY, double* s_pll,
                                             double* s_pu) {
  const uint32_t k = static_cast<uint32_t>(a.k0 + sa + 1);
  const bool odd = (k & 1u) != 0u;
  const double eta_prev = (sa > 0) ? __ldg(a.tab_eta + sa - 1) : 0.0;
#pragma unroll
  for (int m = 0; m < K; ++m) {
    const unsigned int i = nb0 + threadIdx.x + m * blockDim.x;
    if (i < nb1) {
      const unsigned int q = i - nb0;
      if (sa > 0) S[m] = ram_pending<F32>(a, S[m], eta_prev, s_pu, q);
      if constexpr (F32) {
        // Philox block (0, stream 2, member i, odd sweep k_o): a Box-Muller pair from 23-bit
        // uniforms of words 0 and 1 (cosine for k_o, sine for k_o + 1), the accept uniforms of
        // k_o (word 2) and k_o + 1 (word 3)
        float d[M::kData32];
#pragma unroll
        for (int c = 0; c < M::kData32; ++c) d[c] = s_d32[c * a.mpb + q];
        // the odd sweep keeps the pair's sine and the even sweep's uniform in shared memory (the
        // binary32 views of the spare-normal slots) for the next sweep; a launch that starts on an
        // even sweep recomputes them
        float* s_even = reinterpret_cast<float*>(s_zs);
        float z, u;
        if (odd || sa == 0) {
          const uint4 w = philox4x32_10(make_uint4(0u, 2u, static_cast<uint32_t>(i), odd ? k : k - 1u), a.key0,
                                        a.key1);
          float zc, zs;
          box_muller32(w.x, w.y, zc, zs);
          z = odd ? zc : zs;
          u = uniform23(odd ? w.z : w.w);
          if (odd) {
            s_even[q] = zs;
            s_even[a.mpb + q] = uniform23(w.w);
          }
        } else {
          z = s_even[q];
          u = s_even[a.mpb + q];
        }
        const float Y = fmaf(f32_rz(S[m]), z, chi[m]);
        // binary32 views of the slots (a conversion to binary64 and back would cost FP64 issue)
        reinterpret_cast<float*>(s_pY)[q] = Y;
        reinterpret_cast<float*>(s_pll)[q] = M::loglike32(Y, d);
        reinterpret_cast<float*>(s_pu)[q] = u;
      } else {
        // One Box-Muller pair serves the odd sweep (cosine) and the next even sweep (sine, kept
        // in shared memory; recomputed if a launch starts on an even sweep)
        double z;
        if (odd || sa == 0) {
          const uint4 w0 = philox4x32_10(make_uint4(0u, 0u, static_cast<uint32_t>(i), odd ? k : k - 1u), a.key0,
                                         a.key1);
          const double ua = uniform53(w0.x, w0.y), ub = uniform53(w0.z, w0.w);
          const double rad = sqrt(-2.0 * log_tab(ua, s_math));
          double sn, cs;
          sincospi_tab(2.0 * ub, s_math, &sn, &cs);
          z = odd ? rad * cs : rad * sn;
          if (odd) s_zs[q] = rad * sn;
        } else {
          z = s_zs[q];
        }
        const uint4 w1 = philox4x32_10(make_uint4(1u, 0u, static_cast<uint32_t>(i), k), a.key0, a.key1);
        const double Y = fma(S[m], z, chi[m]);
        const double eY = M::kExp ? exp_tab(Y, s_math) : 0.0;
        s_pY[q] = Y;
        s_peY[q] = eY;
        s_pll[q] = M::loglike(Y, eY, s_y[q], s_aux[q], a.mc);
        s_pu[q] = uniform53(w1.x, w1.y);
      }
    }
  }
}

template <class M, int K, bool F32>
__global__ void __launch_bounds__(256, 2) sweep_kernel(const SweepArgs a) {
  using R = typename std::conditional<F32, float, double>::type;  // member arithmetic
  // dynamic shared memory: [mpb] y, [mpb] aux of this block's members, then the rule segment
  // values [rows_smem] L_j, [rows_smem] G_j, [rows_smem] int first inner node
  extern __shared__ double s_dyn[];
  __shared__ double s_theta[kMaxP], s_thp[kMaxP], s_Sth[kMaxP * kMaxP];
  __shared__ ThetaC s_tc, s_tcp;
  __shared__ ThetaCf s_tcf, s_tcpf;
  __shared__ ThetaDf s_tdf;  // FP32 form: constants of this sweep's step theta -> theta'
  __shared__ double s_etabar, s_logeb, s_lpri, s_lpri_new;
  __shared__ int s_stop, s_fail, s_acc_prev;
  // the theta RAM update pending from the previous sweep (applied one sweep late): U (s_pend_idx
  // >= 0: row s_pend_idx of this launch's table, else s_pendU), alpha (from s_pend_lal when
  // s_pend_from_lal), eta (0: none)
  __shared__ double s_pendU[kMaxP], s_pend_alpha, s_pend_lal, s_pend_eta;
  __shared__ double s_Unext[kMaxP], s_Ucur[kMaxP];  // block 0: the table rows of the next and this sweep
  __shared__ long long s_pend_idx;
  __shared__ int s_pend_from_lal;
  // block 0: the next sweep's proposal for a rejected [0] and an accepted [1] theta'
  __shared__ ThetaPub s_cand[2];
  __shared__ long long s_rows_written, s_tacc, s_mom_n0;
  __shared__ int s_mom_sel;
  __shared__ BlockRed s_red;
  // this block's share of the selection integral at the sweep's two possible theta' (rejected,
  // accepted outcome of the decision before it), evaluated by the last warp while thread 0 takes
  // that decision, and their NaN / out-of-range counts
  __shared__ Xacc s_e[2];
  __shared__ unsigned int s_ef[2];

  const int tid = threadIdx.x;
  const int lane = tid & 31, wid = tid >> 5;
  const int ctrl_warp = (blockDim.x >> 5) - 1;  // the warp that runs the deferred theta work
  const int p = a.p;
  // members of this block: the contiguous range [nb0, nb1), equal sizes to within one.
  // Block 0 (which makes the grid's theta proposal on its serial path) holds no members, so that
  // its FP64 unit is not shared with member work; the other blocks split them.
  const unsigned int mb0 = (gridDim.x > 1) ? 1u : 0u;
  const unsigned int mgrid = gridDim.x - mb0, mblk = blockIdx.x - mb0;
  const bool leader_only = (mb0 == 1u && blockIdx.x == 0);
  // blocks that meet at the grid barrier and hold a partial: the member blocks (block 0, when it
  // holds no members, only proposes and decides: it waits at the barrier without arriving)
  const unsigned int nbar = gridDim.x - mb0;
  const unsigned int nb0 = leader_only ? 0u : static_cast<unsigned int>((a.n * mblk) / mgrid);
  const unsigned int nb1 = leader_only ? 0u : static_cast<unsigned int>((a.n * (mblk + 1)) / mgrid);
  const bool skip_me = (a.skip_cta == static_cast<int>(blockIdx.x));
  constexpr bool is_lf = M::kRule;  // the model has a selection integral (LF, BB1)
  double* s_math = s_dyn;                 // [kMathWords] exp/log tables
  double* s_y = s_dyn + kMathWords;
  double* s_aux = s_y + a.mpb;
  double* s_zs = s_y + 2 * a.mpb;  // spare (sine) normal of each member's Box-Muller pair
  // log f(chi_i;theta) of each member after its step (binary32 in the FP32 form), reused by the
  // theta' partial
  double* s_lf = s_y + 3 * a.mpb;
  float* s_lf32 = reinterpret_cast<float*>(s_lf);
  // the theta-independent half of each member's next step (sweep_part_a)
  double* s_pY = s_y + 4 * a.mpb;
  double* s_peY = s_y + 5 * a.mpb;
  double* s_pll = s_y + 6 * a.mpb;
  double* s_pu = s_y + 7 * a.mpb;
  if (!F32) {
    for (unsigned int q = tid; q < nb1 - nb0; q += blockDim.x) {
      s_y[q] = a.y[nb0 + q];
      s_aux[q] = a.aux[nb0 + q];
    }
  }
  for (int q = tid; q < kMathWords; q += blockDim.x) s_math[q] = a.math_tab[q];
  __syncthreads();  // tables in place before thread 0 uses them

  if (tid == 0) {
    for (int q = 0; q < p; ++q) s_theta[q] = a.chain->theta[q];
    for (int q = 0; q < p * p; ++q) s_Sth[q] = a.chain->S_theta[q];
    s_etabar = a.chain->etabar;
    s_logeb = is_lf ? log_etabar(s_etabar, s_math) : 0.0;
    s_tc = M::consts(s_theta, a.mc, s_math);
    s_lpri = M::logprior(s_theta, a.mc, s_math);
    s_rows_written = 0;
    s_tacc = 0;
    s_mom_n0 = a.chain->mom_n;
    s_mom_sel = a.chain->mom_sel;
    s_stop = 0;
    s_fail = 0;
    s_acc_prev = 0;
    for (int q = 0; q < p; ++q) s_pendU[q] = a.chain->pend_U[q];
    s_pend_alpha = a.chain->pend_alpha;
    s_pend_eta = a.adapt_theta ? a.chain->pend_eta : 0.0;
    s_pend_lal = 0.0;
    s_pend_idx = -1;
    s_pend_from_lal = 0;
    s_tcf = M::consts32(s_tc);
    // theta' of the first sweep: proposed by block 0 and fetched by the others
    ThetaPub& first = s_cand[0];
    if (blockIdx.x == 0) {
      propose_theta<M>(a, 0, p, s_theta, s_Sth, first.thp, first.lpri_new, first.tcp, s_math);
      first.tcpf = M::consts32(first.tcp);
      if (F32) first.tdf = M::dconsts32(s_tc, first.tcp);
      put_pub(pub_slot(a, 0), first, p);
      release_pub(a, 1u);
    } else if (wait_pub(a, 1u)) {
      get_pub(first, pub_slot(a, 0), p);
    } else {
      s_fail = 1;
    }
    for (int q = 0; q < p; ++q) s_thp[q] = first.thp[q];
    s_lpri_new = first.lpri_new;
    s_tcp = first.tcp;
    s_tcpf = first.tcpf;
    s_tdf = first.tdf;
  }
  __syncthreads();
  if (s_fail) return;

  // members of this thread: i = nb0 + tid + m blockDim (latent, RAM factor, e^chi, log l in registers)
  R chi[K], echi[K], ll[K];
  double S[K];
  // FP32 bulk form: the model's binary32 member data, M::kData32 arrays of mpb floats, in the
  // region that holds y, aux and the spare normals in the FP64 form (3 mpb doubles = 6 mpb floats)
  float* s_d32 = reinterpret_cast<float*>(s_y);
  if (F32) {  // the handle's prepared binary32 data (rows of stride n32), as the streaming kernel reads them
    for (unsigned int q = tid; q < nb1 - nb0; q += blockDim.x) {
#pragma unroll
      for (int c = 0; c < M::kData32; ++c) s_d32[c * a.mpb + q] = __ldg(a.d32 + c * a.n32 + nb0 + q);
    }
    __syncthreads();
  }
#pragma unroll
  for (int m = 0; m < K; ++m) {
    const unsigned int i = nb0 + tid + m * blockDim.x;
    if (i < nb1) {
      if constexpr (F32) chi[m] = a.chi32[i];  // the FP32 form's latent state is binary32
      else chi[m] = a.chi[i];
      S[m] = a.S[i];
      if constexpr (F32) {
        float d[M::kData32];
#pragma unroll
        for (int c = 0; c < M::kData32; ++c) d[c] = s_d32[c * a.mpb + (i - nb0)];
        echi[m] = 0.0f;
        ll[m] = M::loglike32(chi[m], d);
      } else {
        echi[m] = M::kExp ? exp_tab(chi[m], s_math) : 0.0;  // same routine as in the sweep
        ll[m] = M::loglike(chi[m], echi[m], a.y[i], a.aux[i], a.mc);
      }
    } else {
      chi[m] = echi[m] = ll[m] = R(0);
      S[m] = 0.0;
    }
  }
  unsigned int member_acc = 0;
  const long long mom_n0 = s_mom_n0;
  const int mom_sel = s_mom_sel;
  long long mom_k = 0;  // kept sweeps of this launch
  __syncthreads();
  if (a.ns > 0)
    sweep_part_a<M, K, F32>(a, 0, nb0, nb1, chi, S, s_math, s_y, s_aux, s_zs, s_d32, s_pY, s_peY, s_pll, s_pu);

  // The last warp's share of the selection rule (LF, BB1) at the two possible theta' of a sweep:
  // this block's outer nodes j = rule_j0 + mblk + mgrid k, for both proposals, one (node,
  // proposal) pair per lane, reduced over the warp into s_e (the first sweep of a launch has one
  // theta', as the first).
  auto rule_terms = [&](const ThetaPub* cand, int ncand) {
    Xacc xe0, xe1;
    xacc_zero(xe0);
    xacc_zero(xe1);
    XFlags fe0 = {0u, 0u, 0u}, fe1 = {0u, 0u, 0u};
    const int j1 = a.rule_j1 ? a.rule_j1 : a.nL;
    const int nk = (j1 - a.rule_j0 - static_cast<int>(mblk) + static_cast<int>(mgrid) - 1) / static_cast<int>(mgrid);
    for (int idx = lane; idx < ncand * nk; idx += 32) {
      const int c = idx % ncand, k = idx / ncand;
      const int j = a.rule_j0 + static_cast<int>(mblk) + static_cast<int>(mgrid) * k;
      if (j < j1 && cand[c].lpri_new != -INFINITY) {
        // one code path for both proposals (lanes of a warp on different paths would run one
        // after the other): the term into a temporary, then added to its proposal's sum
        Xacc t;
        xacc_zero(t);
        XFlags ft = {0u, 0u, 0u};
        etabar_node<M>(cand[c].tcp, a, j, s_math, t, ft);
        Xacc z;
        xacc_zero(z);
        xacc_add(xe0, c == 0 ? t : z);
        xacc_add(xe1, c == 0 ? z : t);
        fe0.nan += (c == 0) ? ft.nan + ft.big : 0u;
        fe1.nan += (c == 0) ? 0u : ft.nan + ft.big;
      }
    }
    unsigned int f[4] = {fe0.nan, fe1.nan, 0u, 0u};
    warp_reduce(xe0, xe1, f);
    if (lane == 0) {
      s_e[0] = xe0;
      s_e[1] = xe1;
      s_ef[0] = f[0];
      s_ef[1] = f[1];
    }
  };
  // FP32 form: the rule's share is evaluated a decision ahead (during the decision before the
  // sweep, by one warp, whose FP64 unit is idle then: off the path from the decision to the
  // partial sums); on two blocks per SM the second block's warp sits on another SM sub-partition.
  // FP64 form: with the partial sums (the decision window's FP64 units are shared there).
  constexpr bool kRuleAhead = F32 && is_lf;
  const int rule_warp = ctrl_warp - ((gridDim.x >= 2 && blockIdx.x >= gridDim.x / 2) ? 1 : 0);
  if (kRuleAhead && wid == rule_warp && !leader_only) rule_terms(s_cand, 1);  // theta' of the first sweep

  for (long long s = 0; s < a.ns; ++s) {
    // theta' of this sweep (s > 0): the proposal prepared for the outcome of the last decision
    if (s > 0 && tid == 0) {
      const ThetaPub& c = s_cand[s_acc_prev];
      for (int q = 0; q < p; ++q) s_thp[q] = c.thp[q];
      s_lpri_new = c.lpri_new;
      s_tcp = c.tcp;
      s_tcpf = c.tcpf;
      s_tdf = c.tdf;
    }
    // block 0, from the start of the sweep (while the member blocks work): the theta step's
    // serial part, off the path between the decision and the next proposal. The RAM update of
    // S_theta pending from the previous decision (each step's update is applied one sweep late),
    // then the next sweep's proposal theta + S_theta U for both outcomes of this sweep's decision
    // (theta rejected, theta' accepted), each split into three tasks (propose_part) on lane 0 of
    // six different warps (lanes of one warp would run divergent tasks one after another), and
    // released to the other blocks, which fetch them before this sweep's decision.
    if (blockIdx.x == 0) {
      // the table rows it reads, staged in shared memory first (one load per lane)
      if (tid < p) {
        if (s + 1 < a.ns) s_Unext[tid] = __ldg(a.tab_U + (s + 1) * p + tid);
        s_Ucur[tid] = __ldg(a.tab_U + s * p + tid);
        if (s_pend_idx >= 0) s_pendU[tid] = __ldg(a.tab_U + s_pend_idx * p + tid);
      }
      __syncthreads();  // this sweep's theta' and the rows are in place
      if (wid == ctrl_warp && lane == 0 && s_pend_eta > 0.0) {
        const double lal = s_pend_lal;
        const double alpha = s_pend_from_lal ? ((lal >= 0.0) ? 1.0 : exp_tab(lal, s_math)) : s_pend_alpha;
        ram_update_theta(p, s_Sth, s_pendU, alpha, a.astar_theta, s_pend_eta);
        s_pend_eta = 0.0;
      }
      __syncthreads();
      if (s + 1 < a.ns) {
        // task t: outcome c = t & 1, part 2 - (t >> 1) (the longest first); on 8 warps tasks 4, 5
        // go to warps 6, 7, so that each SM sub-partition's FP64 unit runs at most one long task
        const int nw = blockDim.x >> 5;
        for (int t = 0; t < 6; ++t) {
          const int w = (nw == 8) ? (t < 4 ? t : t + 2) : (t % nw);
          if (wid == w && lane == 0) {
            const int c = t & 1;
            propose_part<M, F32>(a, s_Unext, p, 2 - (t >> 1), c ? s_thp : s_theta, s_Sth, c ? s_tcp : s_tc,
                                 s_cand[c], s_math);
          }
        }
        __syncthreads();
        if (gridDim.x > 1 && wid == ctrl_warp)
          pub2_put(a, 1 + 2 * static_cast<int>((s + 1) & 1), s_cand, static_cast<unsigned int>(s + 2), lane);
      }
    }
    const ThetaC tc = s_tc;
    const bool trace = (a.trace_off + s) < a.trace_T;
    unsigned int member_nan = 0;

    if constexpr (F32) {
      // a1-a3 in binary32 (FP32 bulk form), the theta-dependent half (the draws, Y and its
      // likelihood come from sweep_part_a). The RAM factor S stays binary64.
      const ThetaCf tf = s_tcf;
#pragma unroll
      for (int m = 0; m < K; ++m) {
        const unsigned int i = nb0 + tid + m * blockDim.x;
        if (i < nb1) {
          const float Y = reinterpret_cast<const float*>(s_pY)[i - nb0];
          const float u = reinterpret_cast<const float*>(s_pu)[i - nb0];
          float delta, llY = 0.0f, lfY = 0.0f, cY = 0.0f, cX;
          const float lfX = M::logf32_e(chi[m], tf, cX);
          if (!M::support32(Y, tf)) {
            delta = -INFINITY;
          } else {
            llY = reinterpret_cast<const float*>(s_pll)[i - nb0];
            lfY = M::logf32_e(Y, tf, cY);
            delta = (llY + lfY) - (ll[m] + lfX);
          }
          float alpha;
          const bool acc = mh_accept32(delta, u, alpha);
          if (delta != delta) member_nan++;
          if (acc) {
            chi[m] = Y;
            ll[m] = llY;
            member_acc++;
          }
          s_lf32[i - nb0] = acc ? cY : cX;  // what the theta' partial needs of the new state
          reinterpret_cast<float*>(s_pu)[a.mpb + (i - nb0)] = alpha;  // RAM update in the next half-step
          if (trace) {
            const long long o = (a.trace_off + s) * a.n + static_cast<long long>(i);
            a.tr_delta[o] = delta;
            a.tr_u[o] = u;
            a.tr_acc[o] = acc ? 1 : 0;
          }
        }
      }
    } else {
      // a1-a3: member RAM steps under theta, the theta-dependent half (the draws, Y, e^Y and
      // log l(Y) come from sweep_part_a).
  #pragma unroll
      for (int m = 0; m < K; ++m) {
        const unsigned int i = nb0 + tid + m * blockDim.x;
        if (i < nb1) {
          const double Y = s_pY[i - nb0];
          const double u = s_pu[i - nb0];
          double delta, eY = 0.0, llY = 0.0, lfY = 0.0;
          const double lfX = M::logf(chi[m], echi[m], tc);
          if (!M::support(Y, tc)) {
            delta = -INFINITY;
          } else {
            eY = s_peY[i - nb0];
            llY = s_pll[i - nb0];
            lfY = M::logf(Y, eY, tc);
            delta = (llY + lfY) - (ll[m] + lfX);
          }
          double alpha;
          const bool acc = mh_accept(delta, u, s_math, alpha);  // NaN is counted below
          if (disnan(delta)) member_nan++;
          if (acc) {
            chi[m] = Y;
            echi[m] = eY;
            ll[m] = llY;
            member_acc++;
          }
          s_lf[i - nb0] = acc ? lfY : lfX;
          s_pu[i - nb0] = alpha;  // RAM update in the next half-step (u has been read)
          if (trace) {
            const long long o = (a.trace_off + s) * a.n + static_cast<long long>(i);
            a.tr_delta[o] = delta;
            a.tr_u[o] = u;
            a.tr_acc[o] = acc ? 1 : 0;
          }
        }
      }
    }
    __syncthreads();  // theta' is ready

    // a4: theta' partial; a6: selection integral at theta'
    const ThetaC tcp = s_tcp;
    const bool prior_ok = (s_lpri_new != -INFINITY);
    Xacc xd, xe;
    xacc_zero(xd);
    xacc_zero(xe);
    XFlags fd = {0u, 0u, 0u}, fe = {0u, 0u, 0u};
    unsigned int neg_big = 0, pos_big = 0;
    if (prior_ok && F32) {
      const ThetaCf tpf = s_tcpf, tf = s_tcf;
      const ThetaDf tdf = s_tdf;
      long long xq = 0;  // K <= 8 addends: one fold after the loop
#pragma unroll
      for (int m = 0; m < K; ++m) {
        const unsigned int i = nb0 + tid + m * blockDim.x;
        if (i < nb1) {
          const float c = static_cast<float>(chi[m]);
          const float dn = M::support32(c, tpf) ? M::dtheta32(c, s_lf32[i - nb0], tf, tpf, tdf) : -INFINITY;
          if (dn != dn) fd.nan++;
          else if (fabsf(dn) >= 0x1p94f) {
            if (dn < 0.0f) neg_big++;
            else pos_big++;
          } else {
            xacc_add_float_q(xd, xq, dn, fd);
          }
        }
      }
      xacc_fold_q(xd, xq);
    }
    if (prior_ok && !F32) {
#pragma unroll
      for (int m = 0; m < K; ++m) {
        const unsigned int i = nb0 + tid + m * blockDim.x;
        if (i < nb1) {
          const double dn = M::support(static_cast<double>(chi[m]), tcp)
                                ? M::logf(static_cast<double>(chi[m]), static_cast<double>(echi[m]), tcp) -
                                      s_lf[i - nb0]
                                : -INFINITY;
          if (disnan(dn)) fd.nan++;
          else if (dhuge(dn)) {
            if (dsign(dn)) neg_big++;  // off the support of theta' (-inf) or hopeless
            else pos_big++;            // outside the fixed-point range (+inf included)
          } else {
            xacc_add_double(xd, dn, fd);
          }
        }
      }
    }

    if constexpr (is_lf && !kRuleAhead)
      if (prior_ok && !leader_only) etabar_terms<M>(tcp, a, mblk, mgrid, s_math, xe, fe);

    // a5: block partial
    {
      // f[0]: d_i <= -2^94 (reject), f[1]: NaN anywhere (error), f[2]: d_i >= 2^94, f[3]: member NaN
      unsigned int f[4] = {neg_big, fd.nan + fe.nan + fe.big + member_nan, pos_big, member_nan};
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
        if (lane == 0 && !leader_only) {  // into the grid totals of this sweep
          unsigned long long* acc = a.acc3 + (s % 3) * kAccWords;
          acc_add_limbs(acc, bd);
          atomicAdd(acc + 12, (static_cast<unsigned long long>(bf[1]) << 32) | bf[0]);
          atomicAdd(acc + 13, (static_cast<unsigned long long>(bf[3]) << 32) | bf[2]);
          if constexpr (kRuleAhead) {  // the rule's share, evaluated during the previous decision
            acc_add_limbs(acc + 6, s_e[0]);
            acc_add_limbs(acc + 14, s_e[1]);
            atomicAdd(acc + 20, (static_cast<unsigned long long>(s_ef[1]) << 32) | s_ef[0]);
          } else if constexpr (is_lf) {
            acc_add_limbs(acc + 6, be);
          }
        }
        // the totals of sweep s + 1 reuse the buffer of sweep s - 2, which every block has read
        // (the member blocks before arriving at barrier s - 1, block 0 before publishing the
        // theta' they fetched first): the first member block clears it before it arrives here
        if (lane == 0 && blockIdx.x == mb0) {
          unsigned long long* nxt = a.acc3 + ((s + 1) % 3) * kAccWords;
          for (int q = 0; q < kAccWords; ++q) __stcg(nxt + q, 0ull);
        }
      }
    }
    // a7: every block reads the grid totals and takes the same decision (thread 0)
    auto decide = [&]() {
      const double lnut = __ldg(a.tab_lnu + s), eta_s = __ldg(a.tab_eta + s);  // loads issued first
      Xacc D, E;
      unsigned int f[4];
      const unsigned long long* acc = a.acc3 + (s % 3) * kAccWords;
      // the rule's total at this sweep's theta' (evaluated ahead: the proposal for the last outcome)
      const int ec = kRuleAhead ? s_acc_prev : 0;
      acc_to_xacc(acc, D);
      acc_to_xacc(acc + (ec ? 14 : 6), E);
      const unsigned long long f01 = __ldcg(acc + 12), f23 = __ldcg(acc + 13);
      f[0] = static_cast<unsigned int>(f01);
      f[1] = static_cast<unsigned int>(f01 >> 32);
      if (kRuleAhead) f[1] += static_cast<unsigned int>(__ldcg(acc + 20) >> (ec ? 32 : 0));
      f[2] = static_cast<unsigned int>(f23);
      f[3] = static_cast<unsigned int>(f23 >> 32);
      const long long sg = a.trace_off + s;  // sweep index within this run
      if (f[1] != 0u) {
        atomicCAS(a.err, 0, CUDAHM_ENUMERIC);
        s_stop = 1;
      } else {
        double logalpha, Drec, eb_new, logeb_new;
        theta_logalpha<M>(D, E, f, prior_ok, static_cast<double>(a.n), s_theta, s_thp, s_lpri, s_lpri_new, s_logeb,
                          s_math, logalpha, Drec, eb_new, logeb_new);
        const bool acc = lnut < logalpha;
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
          s_tcf = s_tcpf;
          s_lpri = s_lpri_new;
          if (is_lf) {
            s_etabar = eb_new;
            s_logeb = logeb_new;
          }
          s_tacc++;
        }
        if (a.adapt_theta) {  // this step's RAM update, applied during the next sweep
          s_pend_lal = logalpha;
          s_pend_from_lal = 1;
          s_pend_idx = s;
          s_pend_eta = eta_s;
          // block 0 applies it at once (the proposal of the next sweep, prepared before this
          // decision, used S_theta without it; the one after uses it): off its path to the next
          // proposals. The last sweep of a launch keeps it pending for the next launch.
          if (blockIdx.x == 0 && s + 1 < a.ns) {
            ram_update_theta(p, s_Sth, s_Ucur, (logalpha >= 0.0) ? 1.0 : exp_tab(logalpha, s_math), a.astar_theta,
                             eta_s);
            s_pend_eta = 0.0;
          }
        }
        // a8: record kept sweeps
        const long long post = s - a.burn_left;
        if (post >= 0 && a.thin > 0 && ((a.keep_phase + post + 1) % a.thin) == 0) {
          if (blockIdx.x == 0)
            for (int q = 0; q < p; ++q) a.rows[s_rows_written * p + q] = s_theta[q];
          s_rows_written++;
        }
        s_acc_prev = acc ? 1 : 0;
      }
    };
    // arrive, prepare the next sweep's theta-independent half while the other blocks arrive, wait
    grid_arrive(a.bar, skip_me || leader_only);
    // a8 (optional): this sweep's latents into the running moments
    if (a.mom != nullptr && kept_sweep(s, a.burn_left, a.keep_phase, a.thin)) {
      const MomStep ms = mom_step(a, 1, mom_sel, mom_n0, ++mom_k);
#pragma unroll
      for (int m = 0; m < K; ++m) {
        const unsigned int i = nb0 + tid + m * blockDim.x;
        if (i < nb1) mom_add(ms, i, F32 ? f64_of(static_cast<float>(chi[m])) : static_cast<double>(chi[m]));
      }
    }
    if (s + 1 < a.ns)
      sweep_part_a<M, K, F32>(a, s + 1, nb0, nb1, chi, S, s_math, s_y, s_aux, s_zs, s_d32, s_pY, s_peY, s_pll,
                              s_pu);
    // the other blocks fetch both proposals of the next sweep while the barrier completes (block
    // 0 released them early in this sweep; a failed wait sets the error word, which the barrier
    // wait sees)
    if (blockIdx.x != 0 && s + 1 < a.ns && wid == ctrl_warp) {
      const bool ok = (lane == 0) ? wait_pub(a, static_cast<unsigned int>(s + 2)) : false;
      if (__shfl_sync(0xffffffffu, ok ? 1 : 0, 0)) pub2_get(a, 1 + 2 * static_cast<int>((s + 1) & 1), s_cand, lane);
    }
    if (!grid_wait(a.bar, static_cast<unsigned int>(s), a.err, a.timeout_ns, nbar)) return;
    if (tid == 0) decide();
    // while thread 0 decides: the rule's share at both possible theta' of the next sweep
    if (kRuleAhead && wid == rule_warp && !leader_only && s + 1 < a.ns) rule_terms(s_cand, 2);
    __syncthreads();
    if (s_stop) return;
  }

  // write back (only reached when every sweep succeeded), with the last step's RAM update
  const double eta_last = (a.ns > 0) ? __ldg(a.tab_eta + a.ns - 1) : 0.0;
#pragma unroll
  for (int m = 0; m < K; ++m) {
    const unsigned int i = nb0 + tid + m * blockDim.x;
    if (i < nb1) {
      if constexpr (F32) a.chi32[i] = chi[m];
      else a.chi[i] = chi[m];
      a.S[i] = (a.ns > 0) ? ram_pending<F32>(a, S[m], eta_last, s_pu, i - nb0) : S[m];
    }
  }
  __shared__ unsigned int s_macc;
  if (tid == 0) s_macc = 0;
  __syncthreads();
  atomicAdd(&s_macc, member_acc);
  __syncthreads();
  if (tid == 0) {
    atomicAdd(reinterpret_cast<unsigned long long*>(&a.chain->member_acc), static_cast<unsigned long long>(s_macc));
    if (blockIdx.x == 0) {
      // the last step's RAM update stays pending for the next launch
      const double lal = s_pend_lal;
      for (int q = 0; q < p; ++q)
        a.chain->pend_U[q] = (s_pend_idx >= 0) ? __ldg(a.tab_U + s_pend_idx * p + q) : s_pendU[q];
      a.chain->pend_alpha = s_pend_from_lal ? ((lal >= 0.0) ? 1.0 : exp_tab(lal, s_math)) : s_pend_alpha;
      a.chain->pend_eta = s_pend_eta;
      for (int q = 0; q < p; ++q) a.chain->theta[q] = s_theta[q];
      for (int q = 0; q < p * p; ++q) a.chain->S_theta[q] = s_Sth[q];
      a.chain->etabar = s_etabar;
      a.chain->sweeps = a.k0 + a.ns;
      a.chain->theta_acc += s_tacc;
      a.chain->rows = s_rows_written;
      if (mom_k > 0) {  // commit the moments this launch wrote
        a.chain->mom_n = mom_n0 + mom_k;
        a.chain->mom_sel = 1 - mom_sel;
      }
    }
  }
}

template <class M, bool F32>
static const void* kernel_for_p(int K) {
  switch (K) {
    case 1: return reinterpret_cast<const void*>(&sweep_kernel<M, 1, F32>);
    case 2: return reinterpret_cast<const void*>(&sweep_kernel<M, 2, F32>);
    case 4: return reinterpret_cast<const void*>(&sweep_kernel<M, 4, F32>);
    case 8: return reinterpret_cast<const void*>(&sweep_kernel<M, 8, F32>);
    default: return nullptr;
  }
}

template <class M>
static const void* kernel_for(int K, bool f32) {
  if constexpr (std::is_same<M, BB1>::value) {  // FP64 form only
    return f32 ? nullptr : kernel_for_p<M, false>(K);
  } else {
    return f32 ? kernel_for_p<M, true>(K) : kernel_for_p<M, false>(K);
  }
}

size_t sweep_smem_bytes(int, int mpb, int) {
  return sizeof(double) * kMathWords + 8 * sizeof(double) * static_cast<size_t>(mpb);
}

cudaError_t launch_math_table(double* t, cudaStream_t st) {
  math_table_kernel<<<4, 128, 0, st>>>(t);
  return cudaGetLastError();
}

int math_table_words() { return kMathWords; }

template <class M>
static cudaError_t launch_model(const SweepArgs& a, int K, int grid, int block, cudaStream_t st) {
  void* args[] = {const_cast<SweepArgs*>(&a)};
  const size_t smem = sweep_smem_bytes(a.model, a.mpb, a.rows_smem);
  const void* fn = kernel_for<M>(K, a.f32 != 0);
  if (!fn) return cudaErrorInvalidValue;
  return cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(block), args, smem, st);
}

cudaError_t launch_sweep(const SweepArgs& a, int K, int grid, int block, cudaStream_t st) {
  if (a.model == CUDAHM_NN1) return launch_model<NN1>(a, K, grid, block, st);
  if (a.model == CUDAHM_LF) return launch_model<LF>(a, K, grid, block, st);
  if (a.model == CUDAHM_BB1) return launch_model<BB1>(a, K, grid, block, st);
  return cudaErrorInvalidValue;
}

static const void* sweep_fn(int model, int K, bool f32) {
  if (model == CUDAHM_NN1) return kernel_for<NN1>(K, f32);
  if (model == CUDAHM_LF) return kernel_for<LF>(K, f32);
  if (model == CUDAHM_BB1) return kernel_for<BB1>(K, f32);
  return nullptr;
}

cudaError_t sweep_set_smem(int model, int K, bool f32, int smem_bytes) {
  const void* fn = sweep_fn(model, K, f32);
  if (!fn) return cudaErrorInvalidValue;
  return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes);
}

cudaError_t sweep_occupancy(int model, int K, bool f32, int block, int smem_bytes, int* blocks_per_sm) {
  const void* fn = sweep_fn(model, K, f32);
  if (!fn) return cudaErrorInvalidValue;
  if (smem_bytes > 48 * 1024) {
    const cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes);
    if (e != cudaSuccess) return e;
  }
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, fn, block, smem_bytes);
}

// --------------------------------------------------------- set-up kernels ----
// Derived per-member data, validation and (optionally) the default start.
__global__ void prepare_kernel(int model, long long n, const double* y_raw, const double* aux_raw, double* y,
                               double* aux, double* chi, double* S, ModelConsts mc, double th0, double th1,
                               double th2, int* bad, int set_default_chi) {
  const long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double yr = y_raw[i], ar = aux_raw[i];
  bool ok = isfinite(yr) && isfinite(ar) && ar > 0.0;
  if (model == CUDAHM_NN1) {
    y[i] = yr;
    aux[i] = 1.0 / (ar * ar);
    if (set_default_chi) chi[i] = yr;
  } else {
    y[i] = yr;
    aux[i] = 1.0 / (4.0 * 3.14159265358979323846 * ar * ar);
    ok = ok && aux[i] > 0.0 && isfinite(aux[i]);
    if (mc.marginal) ok = ok && yr > 0.0;  // the cubature window sits at Fhat_i > 0
    if (set_default_chi) {
      double c = log(4.0 * 3.14159265358979323846 * ar * ar * fmax(yr, mc.F_th));
      if (model == CUDAHM_LF) {  // raised into the support chi > ln L_low
        const double floor_c = th2 + 1e-6;
        c = (c > th2) ? c : floor_c;
      }
      chi[i] = c;
    }
  }
  if (set_default_chi) S[i] = mc.chi_init_scale;
  if (!ok) atomicAdd(bad, 1);
}

// d = 3 model: member-major inputs y_raw[3 i + j], s = aux_raw[3 i + j] to per-component arrays
// y[j n + i], aux[j n + i] = 1/s^2; default start chi_i = y_i and S_i = scale I (six packed rows).
__global__ void prepare3_kernel(long long n, const double* y_raw, const double* aux_raw, double* y, double* aux,
                                double* chi, double* S, double scale, int* bad, int set_default_chi) {
  const long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  bool ok = true;
  for (int j = 0; j < 3; ++j) {
    const double yr = y_raw[3 * i + j], sr = aux_raw[3 * i + j];
    const double w = 1.0 / (sr * sr);
    ok = ok && isfinite(yr) && isfinite(sr) && sr > 0.0 && isfinite(w) && w > 0.0;
    y[j * n + i] = yr;
    aux[j * n + i] = w;
    if (set_default_chi) chi[j * n + i] = yr;
  }
  if (set_default_chi)
    for (int q = 0; q < 6; ++q) S[q * n + i] = (q == 0 || q == 2 || q == 5) ? scale : 0.0;
  if (!ok) atomicAdd(bad, 1);
}

cudaError_t launch_prepare(int model, long long n, const double* y_raw, const double* aux_raw, double* y, double* aux,
                           double* chi, double* S, const ModelConsts& mc, const double* theta, int* bad,
                           int set_default_chi, cudaStream_t st) {
  const int blk = 256;
  const long long grid = (n + blk - 1) / blk;
  if (model == CUDAHM_MVN3 || model == CUDAHM_NN3) {
    prepare3_kernel<<<static_cast<unsigned int>(grid), blk, 0, st>>>(n, y_raw, aux_raw, y, aux, chi, S,
                                                                      mc.chi_init_scale, bad, set_default_chi);
    return cudaGetLastError();
  }
  prepare_kernel<<<static_cast<unsigned int>(grid), blk, 0, st>>>(model, n, y_raw, aux_raw, y, aux, chi, S, mc,
                                                                  theta[0], theta[1], theta[2], bad,
                                                                  set_default_chi);
  return cudaGetLastError();
}

// Latents must lie in the support at theta (LF: chi > ln L_low) and be finite (n values; the
// d = 3 model passes all 3 N components).
__global__ void check_chi_kernel(int model, long long n, const double* chi, double lnlow, int* bad) {
  const long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double c = chi[i];
  bool ok = isfinite(c);
  if (model == CUDAHM_LF) ok = ok && (c > lnlow);
  if (!ok) atomicAdd(bad, 1);
}

cudaError_t launch_check_chi(int model, long long n, const double* chi, const double* theta, int* bad,
                             cudaStream_t st) {
  const int blk = 256;
  const long long grid = (n + blk - 1) / blk;
  check_chi_kernel<<<static_cast<unsigned int>(grid), blk, 0, st>>>(model, n, chi,
                                                                     model == CUDAHM_LF ? theta[2] : 0.0, bad);
  return cudaGetLastError();
}

// Gauss-Legendre rule on [-1, 1], one thread per node: Newton's method on P_n from the
// asymptotic first guess x ~ (1 - 1/(8n^2) + 1/(8n^3)) cos(pi (4i+3)/(4n+2)), with P_n and
// P_{n-1} by the three-term recurrence; w = 2 (1 - x^2)/(n P_{n-1}(x))^2 (which equals
// 2/((1 - x^2) P_n'(x)^2) at a root). Nodes ascend.
__global__ void gauss_legendre_kernel(int n, double* x, double* w) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (n + 1) / 2) return;
  const double pi = 3.14159265358979323846;
  const double nd = static_cast<double>(n);
  double z = (1.0 - 1.0 / (8.0 * nd * nd) + 1.0 / (8.0 * nd * nd * nd)) * cos(pi * (4.0 * i + 3.0) / (4.0 * nd + 2.0));
  double pn = 0.0, pm = 0.0;
  for (int it = 0; it < 12; ++it) {
    double p0 = 1.0, p1 = z;
    for (int m = 2; m <= n; ++m) {
      const double p2 = ((2.0 * m - 1.0) * z * p1 - (m - 1.0) * p0) / m;
      p0 = p1;
      p1 = p2;
    }
    if (n == 1) p0 = 1.0;
    pn = p1;
    pm = p0;
    const double omz2 = (1.0 - z) * (1.0 + z);
    const double dp = nd * (pm - z * pn) / omz2;  // P_n'
    const double dz = pn / dp;
    z -= dz;
    if (fabs(dz) <= 1e-17) break;
  }
  {
    double p0 = 1.0, p1 = z;
    for (int m = 2; m <= n; ++m) {
      const double p2 = ((2.0 * m - 1.0) * z * p1 - (m - 1.0) * p0) / m;
      p0 = p1;
      p1 = p2;
    }
    if (n == 1) p0 = 1.0;
    pm = p0;
  }
  const double omz2 = (1.0 - z) * (1.0 + z);
  const double wi = (n == 1) ? 2.0 : 2.0 * omz2 / ((nd * pm) * (nd * pm));
  x[n - 1 - i] = z;
  x[i] = -z;
  w[i] = wi;
  w[n - 1 - i] = wi;
  if ((n & 1) && i == n / 2) x[i] = 0.0;
}

cudaError_t launch_gauss_legendre(int n, double* x, double* w, cudaStream_t st) {
  const int half = (n + 1) / 2;
  gauss_legendre_kernel<<<(half + 127) / 128, 128, 0, st>>>(n, x, w);
  return cudaGetLastError();
}

// Inner-rule tables: r_k = r_max (x_k + 1)/2, qs_k = 1/(4 pi r_k^2 sigma_F),
// W_k = (r_max/2) w_k 3 r_k^2/r_max^3 (distance density ~ r^2 on [0, r_max], normalised).
__global__ void lf_inner_kernel(int nr, const double* xr, const double* wr, double rmax, double sigF, double* qs,
                                double* Wr) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nr) return;
  const double r = 0.5 * rmax * (xr[k] + 1.0);
  qs[k] = 1.0 / (4.0 * 3.14159265358979323846 * r * r) / sigF;
  Wr[k] = 0.5 * rmax * wr[k] * 3.0 * r * r / (rmax * rmax * rmax);
}

cudaError_t launch_lf_inner(int nr, const double* xr, const double* wr, double r_max, double sigma_F, double* qs,
                            double* Wr, cudaStream_t st) {
  lf_inner_kernel<<<(nr + 127) / 128, 128, 0, st>>>(nr, xr, wr, r_max, sigma_F, qs, Wr);
  return cudaGetLastError();
}

// Per-sweep theta tables: p normals (Philox stream 1, member index 0, sweep k; block j gives
// normals 2j, 2j+1), the accept uniform (first uniform of block ceil(p/2)), eta = (k+1)^-gamma.
// One thread per (sweep, task): task j < ceil(p/2) the normal pair of block j, the next task the
// uniform and its logarithm, the last eta, so that a row's serial FP64 chain is one of these
// (the longest, pow) rather than all of them one after another.
// Thread 0 also resets what the next persistent launch counts from: the grid barrier and theta'
// sequence words, the grid totals of its first sweeps, and (when given) the run's error word.
__global__ void tables_kernel(int p, uint32_t key0, uint32_t key1, long long k0, long long ns, double gamma,
                              double* U, double* u, double* lnu, double* eta, unsigned int* bar,
                              unsigned long long* acc, int nacc, int* err) {
  const long long t = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t == 0) {
    bar[0] = 0u;
    bar[1] = 0u;
    for (int q = 0; q < nacc; ++q) acc[q] = 0ull;
    if (err) *err = 0;
  }
  const int nblk = (p + 1) / 2, ntask = nblk + 2;
  const long long s = t / ntask;
  const int j = static_cast<int>(t - s * ntask);
  if (s >= ns) return;
  const uint32_t k = static_cast<uint32_t>(k0 + s + 1);
  if (j < nblk) {
    const uint4 w = philox4x32_10(make_uint4(static_cast<uint32_t>(j), 1u, 0u, k), key0, key1);
    const double ua = uniform53(w.x, w.y), ub = uniform53(w.z, w.w);
    const double rad = sqrt(-2.0 * log(ua));
    double sn, cs;
    sincospi(2.0 * ub, &sn, &cs);
    U[s * p + 2 * j] = rad * cs;
    if (2 * j + 1 < p) U[s * p + 2 * j + 1] = rad * sn;
  } else if (j == nblk) {
    const uint4 w = philox4x32_10(make_uint4(static_cast<uint32_t>(nblk), 1u, 0u, k), key0, key1);
    const double us = uniform53(w.x, w.y);
    u[s] = us;
    lnu[s] = log(us);
  } else {
    eta[s] = pow(static_cast<double>(k) + 1.0, -gamma);
  }
}

cudaError_t launch_tables(int p, uint32_t key0, uint32_t key1, long long k0, long long ns, double gamma, double* U,
                          double* u, double* lnu, double* eta, unsigned int* bar, unsigned long long* acc, int nacc,
                          int* err, cudaStream_t st) {
  const int blk = 128;
  const long long nthr = ns > 0 ? ns * ((p + 1) / 2 + 2) : 1;
  tables_kernel<<<static_cast<unsigned int>((nthr + blk - 1) / blk), blk, 0, st>>>(p, key0, key1, k0, ns, gamma, U,
                                                                                   u, lnu, eta, bar, acc, nacc, err);
  return cudaGetLastError();
}

// Per-member log target at theta (read from device memory), in the handle's precision: the
// FP32 form evaluates exactly the binary32 expressions its member step uses.
template <class M, bool F32>
__global__ void eval_logdens_kernel(long long n, const double* y, const double* aux, const double* chi,
                                    const double* theta, ModelConsts mc, const double* T, double* out) {
  const long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double th[kMaxP];
  for (int q = 0; q < 3; ++q) th[q] = theta[q];
  const ThetaC tc = M::consts(th, mc, T);
  if (F32) {
    const ThetaCf tf = M::consts32(tc);
    const float c = static_cast<float>(chi[i]);
    if (!M::support32(c, tf)) {
      out[i] = -INFINITY;
      return;
    }
    float d[M::kData32];
    M::data32(y[i], aux[i], mc, d);
    const F2 lf = M::logf32p(c, tf);
    out[i] = static_cast<double>(M::loglike32(c, d)) + (static_cast<double>(lf.hi) + static_cast<double>(lf.lo));
    return;
  }
  const double c = chi[i];
  if (!M::support(c, tc)) {
    out[i] = -INFINITY;
    return;
  }
  const double e = M::kExp ? exp(c) : 0.0;
  out[i] = M::loglike(c, e, y[i], aux[i], mc) + M::logf(c, e, tc);
}

// d = 3 models: the same binary64 or binary32 expressions as their member step (per-component arrays).
template <class M, bool F32>
__global__ void eval_logdens3_kernel(long long n, const double* y, const double* aux, const double* chi,
                                     const double* theta, ModelConsts mc, const double* T, double* out) {
  const long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double th[kMaxP];
  for (int q = 0; q < 9; ++q) th[q] = (q < 3 || !std::is_same<M, NN3>::value) ? theta[q] : 0.0;
  const ThetaC3 tc = M::consts(th, mc, T);
  if constexpr (F32) {
    const ThetaC3f tf = M::consts32(tc);
    float x[3], d[M::kData32];
    for (int j = 0; j < 3; ++j) {
      x[j] = static_cast<float>(chi[j * n + i]);
      split_f(y[j * n + i], d[2 * j], d[2 * j + 1]);
      d[6 + j] = static_cast<float>(0.5 * aux[j * n + i]);
    }
    out[i] = static_cast<double>(M::loglike32(x, d)) + static_cast<double>(M::logf32(x, tf));
  } else {
    double x[3], yy[3], w[3];
    for (int j = 0; j < 3; ++j) {
      x[j] = chi[j * n + i];
      yy[j] = y[j * n + i];
      w[j] = aux[j * n + i];
    }
    out[i] = M::loglike(x, yy, w) + M::logf(x, tc);
  }
}

cudaError_t launch_eval_logdens(int model, bool f32, long long n, const double* y, const double* aux,
                                const double* chi, const double* theta_dev, const ModelConsts& mc,
                                const double* math_tab, double* out, cudaStream_t st) {
  const int blk = 256;
  const unsigned int grid = static_cast<unsigned int>((n + blk - 1) / blk);
  if (model == CUDAHM_MVN3) {
    if (f32) eval_logdens3_kernel<MVN3, true><<<grid, blk, 0, st>>>(n, y, aux, chi, theta_dev, mc, math_tab, out);
    else eval_logdens3_kernel<MVN3, false><<<grid, blk, 0, st>>>(n, y, aux, chi, theta_dev, mc, math_tab, out);
  } else if (model == CUDAHM_NN3) {
    if (f32) eval_logdens3_kernel<NN3, true><<<grid, blk, 0, st>>>(n, y, aux, chi, theta_dev, mc, math_tab, out);
    else eval_logdens3_kernel<NN3, false><<<grid, blk, 0, st>>>(n, y, aux, chi, theta_dev, mc, math_tab, out);
  } else if (model == CUDAHM_NN1) {
    if (f32) eval_logdens_kernel<NN1, true><<<grid, blk, 0, st>>>(n, y, aux, chi, theta_dev, mc, math_tab, out);
    else eval_logdens_kernel<NN1, false><<<grid, blk, 0, st>>>(n, y, aux, chi, theta_dev, mc, math_tab, out);
  } else if (model == CUDAHM_LF) {
    if (f32) eval_logdens_kernel<LF, true><<<grid, blk, 0, st>>>(n, y, aux, chi, theta_dev, mc, math_tab, out);
    else eval_logdens_kernel<LF, false><<<grid, blk, 0, st>>>(n, y, aux, chi, theta_dev, mc, math_tab, out);
  } else if (model == CUDAHM_BB1 && !f32) {
    eval_logdens_kernel<BB1, false><<<grid, blk, 0, st>>>(n, y, aux, chi, theta_dev, mc, math_tab, out);
  } else {
    return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// Stand-alone selection integral. With the handle's H table: the same outer-node terms and
// exact sum as the sweep kernels, so the value is bit-identical to the one they compute for the
// same theta. Without a table (the allocation-free entry point): the rule pair by pair.
template <class M>
__global__ void etabar_partial_kernel(const double* theta, const SweepArgs a, unsigned long long* partials) {
  extern __shared__ double s_rows[];
  __shared__ ThetaC s_tc;
  __shared__ BlockRed s_red;
  if (threadIdx.x == 0) {
    double th[kMaxP];
    for (int q = 0; q < 3; ++q) th[q] = theta[q];
    s_tc = M::consts(th, a.mc, a.math_tab);
  }
  __syncthreads();
  Xacc xd, xe;
  xacc_zero(xd);
  xacc_zero(xe);
  XFlags fe = {0u, 0u, 0u};
  if (a.htab) {
    etabar_terms<M>(s_tc, a, blockIdx.x, gridDim.x, a.math_tab, xe, fe);
  } else {
    const int nseg = lf_block_segments(a, blockIdx.x, gridDim.x);
    double* s_phi = s_rows;
    const SegTab tab = segtab_carve(s_rows + kPhiWords, a.rows_smem);
    for (int q = threadIdx.x; q < kPhiWords; q += blockDim.x) s_phi[q] = a.phi_coef[q];
    lf_segment_rows<M>(s_tc, a, blockIdx.x, gridDim.x, nseg, tab, a.math_tab);
    __syncthreads();
    lf_segment_pairs<M>(a, nseg, tab, s_phi, xe, fe);
  }
  unsigned int f[4] = {0u, fe.nan, fe.big, 0u};
  warp_reduce(xd, xe, f);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
    s_red.e[wid] = xe;
    s_red.f[wid][1] = f[1];
  }
  __syncthreads();
  if (wid == 0) {
    Xacc be, bd;
    xacc_zero(be);
    xacc_zero(bd);
    unsigned int bf[4] = {0u, 0u, 0u, 0u};
    if (lane < static_cast<int>(blockDim.x >> 5)) {
      be = s_red.e[lane];
      bf[1] = s_red.f[lane][1];
    }
    warp_reduce(bd, be, bf);
    if (lane == 0) {
      unsigned long long* dst = partials + blockIdx.x * 4;
      dst[0] = be.w0;
      dst[1] = be.w1;
      dst[2] = be.w2;
      dst[3] = bf[1];
    }
  }
}

// H table of the rule (see htab_eval): block c < ncell evaluates the inner sum
// H(u) = sum_k W_k Phi(x_k(e^u)) exactly (fixed-point sum of the rounded terms, the normal CDF
// from the device table) at the kHDeg + 1 Chebyshev points of cell c, [ua + c kHDelta,
// ua + (c + 1) kHDelta], and stores the interpolant's Chebyshev coefficients (discrete cosine
// transform of the values); block ncell stores H(ua) and H(ua + ncell kHDelta).
template <class M>
__global__ void htab_build_kernel(const SweepArgs a, double ua, int ncell, double* coef) {
  constexpr bool bb1 = std::is_same<M, BB1>::value;
  __shared__ double s_phi[kPhiWords];
  __shared__ double s_H[kHDeg + 1];
  __shared__ BlockRed s_red;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  for (int q = tid; q < kPhiWords; q += blockDim.x) s_phi[q] = a.phi_coef[q];
  __syncthreads();
  const int c = blockIdx.x;
  const int npts = (c < ncell) ? kHDeg + 1 : 2;
  for (int m = 0; m < npts; ++m) {
    const double u = (c < ncell) ? ua + kHDelta * (c + 0.5 * (cospi((m + 0.5) / (kHDeg + 1)) + 1.0))
                                 : ua + (m == 0 ? 0.0 : kHDelta * ncell);
    const double L = exp(u);
    Xacc acc, zero;
    xacc_zero(acc);
    xacc_zero(zero);
    XFlags f = {0u, 0u, 0u};
    for (int k = tid; k < a.nr; k += blockDim.x) {
      double v;
      if constexpr (bb1) {
        const double F = L * __ldg(a.qs + k);
        const double aF = a.mc.alpha * F;
        v = 16.0 * (F - a.mc.F_th) * rsqrt(fma(aF, aF, a.mc.s0sq));
      } else {
        v = fma(16.0 * L, __ldg(a.qs + k), -16.0 * a.mc.cth);
      }
      xacc_add_double(acc, __ldg(a.Wr + k) * phi_table16(v, s_phi), f);
    }
    unsigned int fl[4] = {0u, 0u, 0u, 0u};
    warp_reduce(acc, zero, fl);
    if (lane == 0) s_red.d[wid] = acc;
    __syncthreads();
    if (wid == 0) {
      Xacc t, z2;
      xacc_zero(t);
      xacc_zero(z2);
      unsigned int g[4] = {0u, 0u, 0u, 0u};
      if (lane < static_cast<int>(blockDim.x >> 5)) t = s_red.d[lane];
      warp_reduce(t, z2, g);
      if (lane == 0) s_H[m] = xacc_to_double(t);
    }
    __syncthreads();
  }
  if (c < ncell) {
    if (tid <= kHDeg) {
      double sum = 0.0;
      for (int m = 0; m <= kHDeg; ++m) sum = fma(s_H[m], cospi(tid * (m + 0.5) / (kHDeg + 1)), sum);
      sum *= 2.0 / (kHDeg + 1);
      coef[c * (kHDeg + 1) + tid] = (tid == 0) ? 0.5 * sum : sum;
    }
  } else if (tid < 2) {
    coef[ncell * (kHDeg + 1) + tid] = s_H[tid];
  }
}

__global__ void etabar_final_kernel(const unsigned long long* partials, int nblocks, double* out) {
  Xacc E, D;
  xacc_zero(E);
  xacc_zero(D);
  unsigned int f[4] = {0u, 0u, 0u, 0u};
  for (int b = threadIdx.x; b < nblocks; b += 32) {
    Xacc t;
    t.w0 = partials[b * 4 + 0];
    t.w1 = partials[b * 4 + 1];
    t.w2 = partials[b * 4 + 2];
    xacc_add(E, t);
    f[1] += static_cast<unsigned int>(partials[b * 4 + 3]);
  }
  warp_reduce(D, E, f);
  if (threadIdx.x == 0) *out = (f[1] != 0u) ? NAN : xacc_to_double(E);
}

cudaError_t launch_htab_build(const SweepArgs& rule, double ua, int ncell, double* coef, cudaStream_t st) {
  if (rule.model == CUDAHM_BB1) htab_build_kernel<BB1><<<ncell + 1, 256, 0, st>>>(rule, ua, ncell, coef);
  else htab_build_kernel<LF><<<ncell + 1, 256, 0, st>>>(rule, ua, ncell, coef);
  return cudaGetLastError();
}

cudaError_t launch_eval_etabar(const double* theta_dev, const SweepArgs& rule, unsigned long long* partials,
                               int grid, double* out, cudaStream_t st) {
  const size_t smem = rule.htab ? 0 : sizeof(double) * kPhiWords + segtab_bytes(rule.rows_smem);
  if (rule.model == CUDAHM_BB1) etabar_partial_kernel<BB1><<<grid, 256, smem, st>>>(theta_dev, rule, partials);
  else etabar_partial_kernel<LF><<<grid, 256, smem, st>>>(theta_dev, rule, partials);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  etabar_final_kernel<<<1, 32, 0, st>>>(partials, grid, out);
  return cudaGetLastError();
}

}  // namespace chm
