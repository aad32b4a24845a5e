// Many populations in one persistent cooperative launch (batched form).
//
// Population p owns the contiguous block range [b0_p, b0_p + nb_p), sized by the host from
// a cost model (members, the selection rule's pairs, fixed per-sweep work). Its blocks split
// its members into equal contiguous ranges and deal its rule segments round-robin, exactly
// as the single-population kernel does over the whole grid, and meet at a bounded
// per-population barrier each sweep; populations never wait for each other. Member state
// streams from device memory each sweep (latent, RAM factor; the cached e^chi and log l_i are
// recomputed with the same routines), so a population's chain is bit-identical to the one
// the single-population kernel produces for it: every sum is exact and every per-member
// value is the same function of the same inputs.
//
// Launches are chunk-invariant: each population's progress through the current run lives
// in device memory, so one captured CUDA graph (theta tables, barrier reset, this kernel)
// is replayed for every chunk of sweeps.
#include <cuda_runtime.h>

#include <type_traits>

#include "sweep_common.cuh"

namespace chm {

namespace {

// members per staged tile, per lane of a warp (two stages of them per warp)
constexpr unsigned int kTileFactor = 2u;
constexpr int kMaxBlockWarps = 8;  // blocks of at most 256 threads

// The luminosity model's log l_i (an e^x - 1 in binary32, ~25 instructions) is kept from one
// sweep of a launch to the next in row 2 of a.even32 (4 bytes read and 4 written per member-update)
// instead of being recomputed from the latent: the same routine on the same latent and data, so
// the same bits. The first sweep of a launch computes it (the row may hold another chain's or
// run's values). The normal-normal model's log l_i costs four operations and is recomputed.
template <class M>
constexpr bool kCacheLL = std::is_same<M, LF>::value;

// byte offset of the member-tile stages in the dynamic shared memory (after the exp/log tables)
__host__ __device__ constexpr unsigned int tile_offset_bytes() {
  return (static_cast<unsigned int>(sizeof(double)) * kMathWords + 127u) & ~127u;
}

__device__ __forceinline__ int find_pop(const int* b0s, int npop, int b) {
  int lo = 0, hi = npop - 1;  // last population whose first block is <= b
  while (lo < hi) {
    const int m = (lo + hi + 1) >> 1;
    if (b0s[m] <= b) lo = m;
    else hi = m - 1;
  }
  return lo;
}

// Per-population barrier: counter `count` reaches (index + 1) * nb.
__device__ __forceinline__ bool pop_barrier(unsigned int* count, unsigned int index, unsigned int nb, int* err,
                                            long long limit_ns) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    __threadfence();
    atomicAdd(count, 1u);
    const unsigned int target = (index + 1u) * nb;
    const long long t0 = globaltimer_ns();
    while (true) {
      if (ld_acquire_u32(count) >= target) break;
      if (ld_volatile_i32(err) != 0) { ok = 0; break; }
      if (globaltimer_ns() - t0 > limit_ns) {
        atomicCAS(err, 0, CUDAHM_ETIMEOUT);
        ok = 0;
        break;
      }
      __nanosleep(64);
    }
    if (ld_volatile_i32(err) != 0) ok = 0;
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// One member's sweep: RAM step under theta, then its theta' partial (FP64 form).
template <class M>
__device__ __forceinline__ void member_f64(const SweepArgs& a, unsigned int i, uint32_t k, double eta,
                                           const ThetaC& tc, const ThetaC& tcp, bool prior_ok, const double* s_math,
                                           Xacc& xd, XFlags& fd, unsigned int& neg_big, unsigned int& pos_big,
                                           unsigned int& nan_cnt, unsigned int& acc_cnt, long long tro,
                                           bool keep, const MomStep& ms) {
  double chi = a.chi[i], S = a.S[i];
  const double yv = a.y[i], av = a.aux[i];
  double echi = M::kExp ? exp_tab(chi, s_math) : 0.0;
  double ll = M::loglike(chi, echi, yv, av, a.mc);
  const bool odd = (k & 1u) != 0u;
  const uint4 w0 = philox4x32_10(make_uint4(0u, 0u, a.moff + i, odd ? k : k - 1u), a.key0, a.key1);
  const double ua = uniform53(w0.x, w0.y), ub = uniform53(w0.z, w0.w);
  const double rad = sqrt(-2.0 * log_tab(ua, s_math));
  double sn, cs;
  sincospi_tab(2.0 * ub, s_math, &sn, &cs);
  const double z = odd ? rad * cs : rad * sn;
  const uint4 w1 = philox4x32_10(make_uint4(1u, 0u, a.moff + i, k), a.key0, a.key1);
  const double u = uniform53(w1.x, w1.y);
  const double Y = fma(S, z, chi);
  double delta, eY = 0.0, llY = 0.0, lfY = 0.0;
  const double lfX = M::logf(chi, echi, tc);
  if (!M::support(Y, tc)) {
    delta = -INFINITY;
  } else {
    eY = M::kExp ? exp_tab(Y, s_math) : 0.0;
    llY = M::loglike(Y, eY, yv, av, a.mc);
    lfY = M::logf(Y, eY, tc);
    delta = (llY + lfY) - (ll + lfX);
  }
  double alpha;
  const bool acc = mh_accept(delta, u, s_math, alpha);
  if (disnan(delta)) nan_cnt++;
  const double lf_cur = acc ? lfY : lfX;
  if (acc) {
    chi = Y;
    echi = eY;
    acc_cnt++;
  }
  S *= sqrt(fma(eta, alpha - a.astar, 1.0));
  a.chi[i] = chi;
  a.S[i] = S;
  if (keep) mom_add(ms, i, chi);
  if (tro >= 0) {
    a.tr_delta[tro + i] = delta;
    a.tr_u[tro + i] = u;
    a.tr_acc[tro + i] = acc ? 1 : 0;
  }
  if (prior_ok) {
    const double dn = M::support(chi, tcp) ? M::logf(chi, echi, tcp) - lf_cur : -INFINITY;
    if (disnan(dn)) fd.nan++;
    else if (dhuge(dn)) {
      if (dsign(dn)) neg_big++;
      else pos_big++;
    } else {
      xacc_add_double(xd, dn, fd);
    }
  }
}

// One member's sweep in the FP32 bulk form, d = 1, from its staged tile slot: the latent (binary32
// state), the RAM factor (binary64) and the binary32 data. The same operations as the
// register-resident kernel's two half-steps, so the same bits. Writes the new latent and factor.
template <class M>
__device__ __forceinline__ void member1_f32(const SweepArgs& a, unsigned int i, float chi, double S, const float* d,
                                            float ll, float z, float u, float eta_f, float astar_f,
                                            const ThetaCf& tf, const ThetaCf& tpf, const ThetaDf& tdf,
                                            bool prior_ok, Xacc& xd, long long& xq, XFlags& fd,
                                            unsigned int& neg_big, unsigned int& pos_big, unsigned int& nan_cnt,
                                            unsigned int& acc_cnt, long long tro, bool keep, const MomStep& ms) {
  const float Y = fmaf(f32_rz(S), z, chi);
  float delta, llY = 0.0f, lfY = 0.0f, cY = 0.0f, cX;
  const float lfX = M::logf32_e(chi, tf, cX);
  if (!M::support32(Y, tf)) {
    delta = -INFINITY;
  } else {
    llY = M::loglike32(Y, d);
    lfY = M::logf32_e(Y, tf, cY);
    delta = (llY + lfY) - (ll + lfX);
  }
  float alpha;
  const bool acc = mh_accept32(delta, u, alpha);
  if (delta != delta) nan_cnt++;
  const float carry = acc ? cY : cX;
  if (acc) {
    chi = Y;
    acc_cnt++;
  }
  S = ram1_f32(S, alpha, eta_f, astar_f);
  a.chi32[i] = chi;
  a.S[i] = S;
  if constexpr (kCacheLL<M>) a.even32[2 * a.n32 + i] = acc ? llY : ll;  // log l at the new latent
  if (keep) mom_add(ms, i, f64_of(chi));
  if (tro >= 0) {
    a.tr_delta[tro + i] = static_cast<double>(delta);
    a.tr_u[tro + i] = static_cast<double>(u);
    a.tr_acc[tro + i] = acc ? 1 : 0;
  }
  if (prior_ok) {
    const float dn = M::support32(chi, tpf) ? M::dtheta32(chi, carry, tf, tpf, tdf) : -INFINITY;
    if (dn != dn) fd.nan++;
    else if (fabsf(dn) >= 0x1p94f) {
      if (dn < 0.0f) neg_big++;
      else pos_big++;
    } else {
      xacc_add_float_q(xd, xq, dn, fd);
    }
  }
}

// Member tiles of the FP32 form, d = 1, in the streaming kernel, staged per warp. The block's
// members [nb0, nb1) lie in the aligned range [a0, a1): nb0 rounded down and nb1 rounded up to a
// multiple of 4 (the arrays are padded to n32 members). Warp w takes the stretch
// [a0 + w C, a0 + (w + 1) C) of it (C a multiple of 4, clipped to a1) in tiles of
// T = kTileFactor x 32 members. Lane 0 brings each tile's latents, RAM factors and binary32 data
// (on even sweeps also the two cached draws, from the second sweep of a launch also the cached
// log l_i) into one of the warp's two shared-memory stages by bulk copies (the TMA engine) while
// the warp steps the members of its other stage. A warp waits only for its own tiles, so the
// warps of a block do not wait for one another during the member phase. Every copy starts on a
// 16-byte boundary and moves a multiple of 16 bytes. The few members of a neighbouring block
// that the first or last aligned tile covers are read but never used or written.
struct TileRing {
  char* buf;                // this warp's two stages of T tile_member_bytes<M>() bytes
  unsigned long long* bar;  // this warp's mbarriers, one per stage
  unsigned int T;           // members per tile
  unsigned int count;       // tiles this warp consumed so far: stage count & 1, phase parity (count >> 1) & 1
  bool prefetched;          // the warp's first tile of a sweep (counter `count`) is in flight
};

// the calling warp's stretch [w0, w1) of the block's aligned range [a0, a1)
__device__ __forceinline__ void warp_stretch(unsigned int a0, unsigned int a1, unsigned int& w0, unsigned int& w1) {
  const unsigned int nw = blockDim.x >> 5, w = threadIdx.x >> 5;
  const unsigned int C = ((a1 - a0 + nw - 1u) / nw + 3u) & ~3u;
  w0 = min(a0 + w * C, a1);
  w1 = min(w0 + C, a1);
}

// the block's aligned range [a0, a1) of its members [nb0, nb1), nb1 > nb0
__device__ __forceinline__ void tile_range(const SweepArgs& a, unsigned int nb0, unsigned int nb1, unsigned int& a0,
                                           unsigned int& a1) {
  a0 = nb0 & ~3u;
  const unsigned long long a1l = (static_cast<unsigned long long>(nb1) + 3ull) & ~3ull;
  a1 = static_cast<unsigned int>(a1l < static_cast<unsigned long long>(a.n32) ? a1l : a.n32);
}

// the theta' partials of at most this many tiles (kTileFactor addends per lane each) share one
// 64-bit word before it is folded into the lane's exact sum (xacc_add_float_q: at most 127)
constexpr unsigned int kFoldTiles = 64u / kTileFactor;
static_assert(kTileFactor >= 1u && kTileFactor <= 64u, "fold interval");

// bytes of one member in a stage: latent, RAM factor, data, the even sweep's two draws and the
// cached log l_i (models with kCacheLL)
template <class M>
__host__ __device__ constexpr unsigned int tile_member_bytes() {
  return 12u + 4u * M::kData32 + 8u + (kCacheLL<M> ? 4u : 0u);
}

// Issues the tile of len members from b into stage cnt & 1; `even`: also the two draws the odd
// sweep before stored for each member (a.even32), which an even sweep reads instead of drawing;
// `llc`: also the cached log l_i (row 2 of a.even32, written by the sweep before in this launch).
template <class M>
__device__ __forceinline__ void tile_issue(const SweepArgs& a, const TileRing& r, unsigned int b, unsigned int len,
                                           unsigned int cnt, bool even, bool llc) {
  constexpr int K32 = M::kData32;
  constexpr unsigned int mb = tile_member_bytes<M>();
  const bool ll = kCacheLL<M> && llc;
  char* st = r.buf + static_cast<size_t>(cnt & 1u) * r.T * mb;
  unsigned long long* bar = r.bar + (cnt & 1u);
  mbar_arrive_expect_tx(bar, len * (12u + 4u * K32 + (even ? 8u : 0u) + (ll ? 4u : 0u)));
  bulk_copy_g2s(st, a.chi32 + b, len * 4u, bar);
  bulk_copy_g2s(st + 4u * r.T, a.S + b, len * 8u, bar);
#pragma unroll
  for (int c = 0; c < K32; ++c) bulk_copy_g2s(st + (12u + 4u * c) * r.T, a.d32 + c * a.n32 + b, len * 4u, bar);
  if (even) {
    bulk_copy_g2s(st + (12u + 4u * K32) * r.T, a.even32 + b, len * 4u, bar);
    bulk_copy_g2s(st + (16u + 4u * K32) * r.T, a.even32 + a.n32 + b, len * 4u, bar);
  }
  if (ll) bulk_copy_g2s(st + (20u + 4u * K32) * r.T, a.even32 + 2 * a.n32 + b, len * 4u, bar);
}

// The block's member phase of one sweep (FP32 form, d = 1). Returns false if a stage wait
// timed out (the run's error word is set; copies in flight have been waited for).
// The draws of an odd sweep k (Philox block (0, stream 2, member word, k)) give that sweep's
// normal (the Box-Muller cosine) and uniform (word 2) and the next sweep's (the sine, word 3).
// `cached`: an even sweep whose odd predecessor ran in this launch, so its two draws are in the
// stage (written to a.even32 by that sweep) instead of being drawn again; the first sweep of a
// launch always draws (a.even32 may hold another chain's or run's values). `llc`: not the first
// sweep of the launch, so the cached log l_i is in the stage (kCacheLL models).
template <class M>
__device__ __forceinline__ bool members1_f32_tiled(const SweepArgs& a, TileRing& r, unsigned int nb0,
                                                   unsigned int nb1, uint32_t k, bool cached, bool llc,
                                                   float eta_f,
                                                   float astar_f, const ThetaCf& tf, const ThetaCf& tpf,
                                                   const ThetaDf& tdf, bool prior_ok, Xacc& xd,
                                                   XFlags& fd, unsigned int& neg_big, unsigned int& pos_big,
                                                   unsigned int& nan_cnt, unsigned int& acc_cnt, long long tro,
                                                   bool keep, const MomStep& ms) {
  constexpr int K32 = M::kData32;
  constexpr unsigned int mb = tile_member_bytes<M>();
  if (nb1 <= nb0) return true;
  const bool odd = (k & 1u) != 0u;
  const unsigned int lane = threadIdx.x & 31u;
  unsigned int a0, a1, w0, w1;
  tile_range(a, nb0, nb1, a0, a1);
  warp_stretch(a0, a1, w0, w1);
  const unsigned int ntiles = (w1 - w0 + r.T - 1u) / r.T;
  if (ntiles > 0u && !r.prefetched && lane == 0u) tile_issue<M>(a, r, w0, min(r.T, w1 - w0), r.count, cached, llc);
  r.prefetched = false;
  bool ok = true;  // this lane's stage waits all completed
  long long xq = 0;
  for (unsigned int t = 0; t < ntiles; ++t) {
    const unsigned int cnt = r.count;
    const unsigned int b = w0 + t * r.T, len = min(r.T, w1 - b);
    if (t + 1u < ntiles && lane == 0u) tile_issue<M>(a, r, b + r.T, min(r.T, w1 - b - r.T), cnt + 1u, cached, llc);
    if (ok) ok = mbar_wait_bounded(r.bar + (cnt & 1u), (cnt >> 1) & 1u, a.err, a.timeout_ns);
    if (!ok) {  // the run has failed: skip the members, keep the warp's stages in step
      __syncwarp();
      r.count = cnt + 1u;
      continue;
    }
    const char* st = r.buf + static_cast<size_t>(cnt & 1u) * r.T * mb;
    const float* s_chi = reinterpret_cast<const float*>(st);
    const double* s_S = reinterpret_cast<const double*>(st + 4u * r.T);
    const float* s_d = reinterpret_cast<const float*>(st + 12u * r.T);
    const float* s_ev = reinterpret_cast<const float*>(st + (12u + 4u * K32) * r.T);
    const float* s_ll = reinterpret_cast<const float*>(st + (20u + 4u * K32) * r.T);
    for (unsigned int m = lane; m < len; m += 32u) {
      const unsigned int i = b + m;
      if (i < nb0 || i >= nb1) continue;
      float d[K32];
#pragma unroll
      for (int c = 0; c < K32; ++c) d[c] = s_d[c * r.T + m];
      float z, u;
      if (cached) {
        z = s_ev[m];
        u = s_ev[r.T + m];
      } else {
        const uint4 w = philox4x32_10(make_uint4(0u, 2u, a.moff + i, odd ? k : k - 1u), a.key0, a.key1);
        float zc, zs;
        box_muller32(w.x, w.y, zc, zs);
        z = odd ? zc : zs;
        u = uniform23(odd ? w.z : w.w);
        if (odd) {  // the next sweep's two draws
          a.even32[i] = zs;
          a.even32[a.n32 + i] = uniform23(w.w);
        }
      }
      const float chi = s_chi[m];
      const float ll = (kCacheLL<M> && llc) ? s_ll[m] : M::loglike32(chi, d);
      member1_f32<M>(a, i, chi, s_S[m], d, ll, z, u, eta_f, astar_f, tf, tpf, tdf, prior_ok, xd, xq, fd, neg_big,
                     pos_big, nan_cnt, acc_cnt, tro, keep, ms);
    }
    if ((t + 1u) % kFoldTiles == 0u) xacc_fold_q(xd, xq);
    __syncwarp();  // the stage is free for the warp's tile after next
    r.count = cnt + 1u;
  }
  xacc_fold_q(xd, xq);
  // this thread's writes of the sweep before any later bulk copy reads them (within the sweep the
  // copies read only other members: the warps' stretches are disjoint, and the few members of a
  // neighbouring block that an aligned tile covers are never used)
  fence_proxy_async_global();
  if (__syncthreads_or(ok ? 0 : 1)) {
    // a stage wait timed out: leave no copy in flight into this block's shared memory (every
    // lane waits, bounded again, for the last phase issued on each of its warp's stages)
    for (unsigned int c = r.count - min(r.count, 2u); c < r.count; ++c)
      mbar_wait_bounded(r.bar + (c & 1u), (c >> 1) & 1u, a.err, a.timeout_ns);
    __syncthreads();
    return false;
  }
  return true;
}

// Issues the warp's first tile of the next sweep (lane 0), after every write of this sweep;
// `cached` as for members1_f32_tiled, for the next sweep (which has the cached log l_i).
template <class M>
__device__ __forceinline__ void tile_prefetch_first(const SweepArgs& a, TileRing& r, unsigned int nb0,
                                                    unsigned int nb1, bool cached) {
  if (nb1 <= nb0) return;
  unsigned int a0, a1, w0, w1;
  tile_range(a, nb0, nb1, a0, a1);
  warp_stretch(a0, a1, w0, w1);
  if (w1 <= w0) return;
  if ((threadIdx.x & 31u) == 0u) tile_issue<M>(a, r, w0, min(r.T, w1 - w0), r.count, cached, true);
  r.prefetched = true;
}

// One member's sweep for the d = 3 model (FP64 form). State and data are stored per component
// (structure of arrays, component j of member i at j n + i; the RAM factor as six packed rows).
// Draws as the oracle defines them: component c of U from the Box-Muller pair of Philox block
// (c, stream 0, i, odd sweep) (cosine for the odd sweep, sine for the next), the accept
// uniform from block (3, 0, i, k). The odd sweep keeps the three sines in a.spare3 for the next
// sweep; a launch that starts on an even sweep (first) recomputes them.
template <class M>
__device__ __forceinline__ void member3_f64(const SweepArgs& a, unsigned int i, uint32_t k, double eta,
                                            const ThetaC3& tc, const ThetaC3& tcp, bool prior_ok,
                                            const double* s_math, Xacc& xd, XFlags& fd, unsigned int& neg_big,
                                            unsigned int& pos_big, unsigned int& nan_cnt, unsigned int& acc_cnt,
                                            long long tro, bool first, bool keep, const MomStep& ms) {
  const size_t n = static_cast<size_t>(a.n);
  double x[3], y[3], w[3], S[6];
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    x[j] = a.chi[j * n + i];
    y[j] = __ldg(a.y + j * n + i);
    w[j] = __ldg(a.aux + j * n + i);
  }
#pragma unroll
  for (int q = 0; q < 6; ++q) S[q] = a.S[q * n + i];
  const bool odd = (k & 1u) != 0u;
  const uint32_t ko = odd ? k : k - 1u;
  double z[3];
  if (odd || first) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const uint4 b = philox4x32_10(make_uint4(static_cast<uint32_t>(c), 0u, a.moff + i, ko), a.key0, a.key1);
      const double ua = uniform53(b.x, b.y), ub = uniform53(b.z, b.w);
      const double rad = sqrt(-2.0 * log_tab(ua, s_math));
      double sn, cs;
      sincospi_tab(2.0 * ub, s_math, &sn, &cs);
      z[c] = odd ? rad * cs : rad * sn;
      if (odd) a.spare3[c * n + i] = rad * sn;
    }
  } else {
#pragma unroll
    for (int c = 0; c < 3; ++c) z[c] = a.spare3[c * n + i];
  }
  const uint4 bu = philox4x32_10(make_uint4(3u, 0u, a.moff + i, k), a.key0, a.key1);
  const double u = uniform53(bu.x, bu.y);
  // v = S z (lower triangular), proposal Y = chi + v
  const double v0 = S[0] * z[0];
  const double v1 = fma(S[1], z[0], S[2] * z[1]);
  const double v2 = fma(S[3], z[0], fma(S[4], z[1], S[5] * z[2]));
  const double Y[3] = {x[0] + v0, x[1] + v1, x[2] + v2};
  const double lfX = M::logf(x, tc), lfY = M::logf(Y, tc);
  const double delta = (M::loglike(Y, y, w) + lfY) - (M::loglike(x, y, w) + lfX);
  double alpha;
  const bool acc = mh_accept(delta, u, s_math, alpha);
  if (disnan(delta)) nan_cnt++;
  double lf_cur = lfX;
  if (acc) {
#pragma unroll
    for (int j = 0; j < 3; ++j) x[j] = Y[j];
    lf_cur = lfY;
    acc_cnt++;
  }
  const double zz = fma(z[0], z[0], fma(z[1], z[1], z[2] * z[2]));
  ram3_update(S, v0, v1, v2, (eta * (alpha - a.astar)) / zz);
#pragma unroll
  for (int j = 0; j < 3; ++j) a.chi[j * n + i] = x[j];
#pragma unroll
  for (int q = 0; q < 6; ++q) a.S[q * n + i] = S[q];
  if (keep)
#pragma unroll
    for (int j = 0; j < 3; ++j) mom_add(ms, j * n + i, x[j]);
  if (tro >= 0) {
    a.tr_delta[tro + i] = delta;
    a.tr_u[tro + i] = u;
    a.tr_acc[tro + i] = acc ? 1 : 0;
  }
  if (prior_ok) {
    const double dn = M::logf(x, tcp) - lf_cur;
    if (disnan(dn)) fd.nan++;
    else if (dhuge(dn)) {
      if (dsign(dn)) neg_big++;
      else pos_big++;
    } else {
      xacc_add_double(xd, dn, fd);
    }
  }
}

// Standard normal of sweep k from one Box-Muller pair of binary32 uniforms
__device__ __forceinline__ float bm23(uint32_t wa, uint32_t wb, bool odd) {
  float zc, zs;
  box_muller32(wa, wb, zc, zs);
  return odd ? zc : zs;
}

// One member's sweep for the d = 3 model in the FP32 bulk form: binary32 draws (Philox blocks
// (0, stream 2, i, odd sweep) and (1, 2, i, odd sweep): Box-Muller pairs from words (0,1), (2,3)
// of the first and (0,1) of the second give components 0, 1, 2, cosine for the odd sweep and
// sine for the next; words 2 and 3 of the second are the odd and even sweep's accept uniforms),
// binary32 member log targets, binary64 v = S z and RAM factor update.
template <class M>
__device__ __forceinline__ void member3_f32(const SweepArgs& a, unsigned int i, uint32_t k, double eta,
                                            const ThetaC3f& tf, const ThetaC3f& tpf, bool prior_ok, Xacc& xd,
                                            XFlags& fd, unsigned int& neg_big, unsigned int& pos_big,
                                            unsigned int& nan_cnt, unsigned int& acc_cnt, long long tro,
                                            bool keep, const MomStep& ms) {
  const size_t n = static_cast<size_t>(a.n);
  float x[3], d[M::kData32];
  double S[6];
#pragma unroll
  for (int j = 0; j < 3; ++j) x[j] = static_cast<float>(a.chi[j * n + i]);
#pragma unroll
  for (int c = 0; c < M::kData32; ++c) d[c] = __ldg(a.d32 + c * n + i);
#pragma unroll
  for (int q = 0; q < 6; ++q) S[q] = a.S[q * n + i];
  const bool odd = (k & 1u) != 0u;
  const uint32_t ko = odd ? k : k - 1u;
  const uint4 b0 = philox4x32_10(make_uint4(0u, 2u, a.moff + i, ko), a.key0, a.key1);
  const uint4 b1 = philox4x32_10(make_uint4(1u, 2u, a.moff + i, ko), a.key0, a.key1);
  const float z0 = bm23(b0.x, b0.y, odd), z1 = bm23(b0.z, b0.w, odd), z2 = bm23(b1.x, b1.y, odd);
  const float u = uniform23(odd ? b1.z : b1.w);
  const double zd0 = z0, zd1 = z1, zd2 = z2;
  const double v0 = S[0] * zd0;
  const double v1 = fma(S[1], zd0, S[2] * zd1);
  const double v2 = fma(S[3], zd0, fma(S[4], zd1, S[5] * zd2));
  const float Y[3] = {__fadd_rn(x[0], static_cast<float>(v0)), __fadd_rn(x[1], static_cast<float>(v1)),
                      __fadd_rn(x[2], static_cast<float>(v2))};
  const float lfX = M::logf32(x, tf), lfY = M::logf32(Y, tf);
  const float delta = __fsub_rn(__fadd_rn(M::loglike32(Y, d), lfY), __fadd_rn(M::loglike32(x, d), lfX));
  float alpha;
  const bool acc = mh_accept32(delta, u, alpha);
  if (delta != delta) nan_cnt++;
  float lf_cur = lfX;
  if (acc) {
#pragma unroll
    for (int j = 0; j < 3; ++j) x[j] = Y[j];
    lf_cur = lfY;
    acc_cnt++;
  }
  const double zz = fma(zd0, zd0, fma(zd1, zd1, zd2 * zd2));
  ram3_update(S, v0, v1, v2, (eta * (static_cast<double>(alpha) - a.astar)) / zz);
#pragma unroll
  for (int j = 0; j < 3; ++j) a.chi[j * n + i] = static_cast<double>(x[j]);
#pragma unroll
  for (int q = 0; q < 6; ++q) a.S[q * n + i] = S[q];
  if (keep)
#pragma unroll
    for (int j = 0; j < 3; ++j) mom_add(ms, j * n + i, static_cast<double>(x[j]));
  if (tro >= 0) {
    a.tr_delta[tro + i] = static_cast<double>(delta);
    a.tr_u[tro + i] = static_cast<double>(u);
    a.tr_acc[tro + i] = acc ? 1 : 0;
  }
  if (prior_ok) {
    const float dn = __fsub_rn(M::logf32(x, tpf), lf_cur);
    if (dn != dn) fd.nan++;
    else if (fabsf(dn) >= 0x1p94f) {
      if (dn < 0.0f) neg_big++;
      else pos_big++;
    } else {
      xacc_add_float(xd, dn, fd);
    }
  }
}

// Shard pass: the block's partial of the sweep is in its slot; the last block of the population
// to finish (an atomic count of finished blocks on the population's barrier word, which it resets)
// sums all nb partials and writes the shard's exchange words: D and E as six 32-bit limbs each,
// the flag counts, the shard's member count and 1. Called by every thread of the block.
__device__ void shard_export(const SweepArgs& a, const unsigned long long* base, int nb, BlockRed& red) {
  __shared__ int s_last;
  __syncthreads();  // the block's partial is written (warp 0, lane 0)
  if (threadIdx.x == 0) {
    __threadfence();
    s_last = (atomicAdd(a.bar, 1u) == static_cast<unsigned int>(nb) - 1u) ? 1 : 0;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();  // every other block's partial is visible
  Xacc D, E;
  unsigned int f[4];
  sum_partials(base, nb, red, D, E, f);
  if (threadIdx.x == 0) {
    unsigned long long* o = a.shard_out;
    const unsigned long long d[3] = {D.w0, D.w1, D.w2}, e[3] = {E.w0, E.w1, E.w2};
    for (int q = 0; q < 3; ++q) {
      o[2 * q] = d[q] & 0xFFFFFFFFull;
      o[2 * q + 1] = d[q] >> 32;
      o[6 + 2 * q] = e[q] & 0xFFFFFFFFull;
      o[6 + 2 * q + 1] = e[q] >> 32;
    }
    o[12] = (static_cast<unsigned long long>(f[1]) << 32) | f[0];
    o[13] = (static_cast<unsigned long long>(f[3]) << 32) | f[2];
    o[14] = static_cast<unsigned long long>(a.n);
    o[15] = 1ull;
    *a.bar = 0u;  // for the next pass
  }
}

template <class M, bool F32>
__device__ void run_population(const SweepArgs& a, BatchProg* prog, int b0, int lb, int nb, int chunk, int R,
                               double* s_dyn, double* s_theta, double* s_thp, double* s_Sth, BlockRed& s_red) {
  using TC = typename M::TC;
  using TCf = typename M::TCf;
  __shared__ TC s_tc, s_tcp;
  __shared__ TCf s_tcf, s_tcpf;
  __shared__ ThetaDf s_tdf;  // FP32 form, d = 1: constants of this sweep's step theta -> theta'
  __shared__ double s_etabar, s_logeb, s_lpri, s_lpri_new;
  __shared__ double s_pendU[kMaxP], s_pend_alpha, s_pend_eta;
  __shared__ int s_stop;
  __shared__ long long s_rows_written, s_tacc, s_k0, s_off, s_ns, s_mom_n0;
  __shared__ int s_mom_sel;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int p = a.p;
  constexpr bool is_lf = M::kRule;  // the model has a selection integral (LF, BB1)
  double* s_math = s_dyn;
  const long long t_start = globaltimer_ns();
  for (int q = tid; q < kMathWords; q += blockDim.x) s_math[q] = a.math_tab[q];
  __syncthreads();  // tables in place before thread 0 uses them
  if (tid == 0) {
    s_k0 = a.chain->sweeps;
    s_off = prog->off;
    const long long left = prog->total - prog->off;
    s_ns = left < chunk ? left : chunk;
    for (int q = 0; q < p; ++q) s_theta[q] = a.chain->theta[q];
    for (int q = 0; q < p * p; ++q) s_Sth[q] = a.chain->S_theta[q];
    s_etabar = a.chain->etabar;
    s_logeb = is_lf ? log_etabar(s_etabar, s_math) : 0.0;
    s_tc = M::consts(s_theta, a.mc, s_math);
    s_tcf = M::consts32(s_tc);
    s_lpri = M::logprior(s_theta, a.mc, s_math);
    s_rows_written = 0;
    s_tacc = 0;
    s_mom_n0 = a.chain->mom_n;
    s_mom_sel = a.chain->mom_sel;
    for (int q = 0; q < p; ++q) s_pendU[q] = a.chain->pend_U[q];
    s_pend_alpha = a.chain->pend_alpha;
    s_pend_eta = a.chain->pend_eta;
    s_stop = 0;
  }
  __syncthreads();
  const long long ns = s_ns, k0 = s_k0, off = s_off;
  const long long mom_n0 = s_mom_n0, thin = prog->thin;
  const int mom_sel = s_mom_sel;
  long long mom_k = 0;  // kept sweeps of this launch
  const long long burn_left = prog->n_burn - off;
  double* rows = a.rows ? a.rows + prog->rows * p : nullptr;
  const unsigned int nb0 = static_cast<unsigned int>((a.n * lb) / nb);
  const unsigned int nb1 = static_cast<unsigned int>((a.n * (lb + 1)) / nb);
  unsigned int member_acc = 0;
  // FP32 form, d = 1: member tiles staged in shared memory by bulk copies (after the tables)
  constexpr bool kTiled = F32 && M::kD == 1;
  __shared__ __align__(8) unsigned long long s_tbar[2 * kMaxBlockWarps];  // two per warp
  TileRing ring{};
  if constexpr (kTiled) {
    const size_t base = reinterpret_cast<size_t>(reinterpret_cast<char*>(s_dyn) + tile_offset_bytes());
    ring.T = kTileFactor * 32u;
    // this warp's two stages (16-byte copies need 16-byte alignment: the base is 128-aligned and
    // a stage is a multiple of 128 bytes)
    ring.buf = reinterpret_cast<char*>((base + 127u) & ~static_cast<size_t>(127u)) +
               static_cast<size_t>(wid) * 2u * ring.T * tile_member_bytes<M>();
    ring.bar = s_tbar + 2 * wid;
    ring.count = 0u;
    ring.prefetched = false;
    if (tid == 0) {
      for (int q = 0; q < 2 * (static_cast<int>(blockDim.x) >> 5); ++q) mbar_init(&s_tbar[q], 1u);
      fence_mbar_init();
    }
    __syncthreads();
  }
  const float astar_f = __double2float_rn(a.astar);

  for (long long s = 0; s < ns; ++s) {
    const uint32_t k = static_cast<uint32_t>(k0 + s + 1);
    const double eta = __ldg(a.tab_eta + s);
    // theta' = theta + S_theta U (the table of this launch's sweeps starts at index 0)
    if (tid == 0) {
      double lp;
      TC tcp;
      propose_theta<M>(a, s, p, s_theta, s_Sth, s_thp, lp, tcp, s_math);
      s_lpri_new = lp;
      s_tcp = tcp;
      s_tcpf = M::consts32(tcp);
      if constexpr (F32 && M::kD == 1) s_tdf = M::dconsts32(s_tc, tcp);
    }
    __syncthreads();
    const bool prior_ok = (s_lpri_new != -INFINITY);
    Xacc xd, xe;
    xacc_zero(xd);
    xacc_zero(xe);
    XFlags fd = {0u, 0u, 0u}, fe = {0u, 0u, 0u};
    unsigned int neg_big = 0, pos_big = 0, member_nan = 0;
    const long long sg = off + s;  // sweep index within this run
    const long long tro = (sg < a.trace_T) ? sg * a.n : -1;
    // a8 (optional): the kept sweep's latents go into the running moments
    const bool keep = (a.mom != nullptr) && kept_sweep(s, burn_left, 0, thin);
    MomStep ms{};
    if (keep) ms = mom_step(a, M::kD, mom_sel, mom_n0, ++mom_k);
    if constexpr (M::kD == 3) {
      if constexpr (F32) {
        for (unsigned int i = nb0 + tid; i < nb1; i += blockDim.x)
          member3_f32<M>(a, i, k, eta, s_tcf, s_tcpf, prior_ok, xd, fd, neg_big, pos_big, member_nan, member_acc,
                         tro, keep, ms);
      } else {
        for (unsigned int i = nb0 + tid; i < nb1; i += blockDim.x)
          member3_f64<M>(a, i, k, eta, s_tc, s_tcp, prior_ok, s_math, xd, fd, neg_big, pos_big, member_nan,
                         member_acc, tro, s == 0, keep, ms);
      }
    } else if constexpr (F32) {
      const TCf tf = s_tcf, tpf = s_tcpf;
      const ThetaDf tdf = s_tdf;
      const bool cached = (k & 1u) == 0u && s > 0;  // the odd sweep before ran in this launch
      if (!members1_f32_tiled<M>(a, ring, nb0, nb1, k, cached, s > 0, __double2float_rn(eta), astar_f, tf, tpf, tdf,
                                 prior_ok, xd, fd, neg_big, pos_big, member_nan, member_acc, tro, keep, ms))
        return;  // a stage wait timed out: the run's error word is set, the population stops
    } else {
      const TC tc = s_tc, tcp = s_tcp;
      for (unsigned int i = nb0 + tid; i < nb1; i += blockDim.x)
        member_f64<M>(a, i, k, eta, tc, tcp, prior_ok, s_math, xd, fd, neg_big, pos_big, member_nan, member_acc,
                      tro, keep, ms);
    }
    // a6: this block's share of the selection rule's outer nodes at theta'
    if constexpr (M::kRule)
      if (prior_ok) etabar_terms<M>(s_tcp, a, lb, nb, s_math, xe, fe);
    {
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
        if (lane == 0) {
          unsigned long long* dst = a.partials + ((s & 1) * gridDim.x + b0 + lb) * kPartWords;
          __stcg(dst + 0, bd.w0);
          __stcg(dst + 1, bd.w1);
          __stcg(dst + 2, bd.w2);
          __stcg(dst + 3, be.w0);
          __stcg(dst + 4, be.w1);
          __stcg(dst + 5, be.w2);
          __stcg(dst + 6, (static_cast<unsigned long long>(bf[1]) << 32) | bf[0]);
          __stcg(dst + 7, (static_cast<unsigned long long>(bf[3]) << 32) | bf[2]);
        }
      }
    }
    if (a.shard_out != nullptr) {  // shard pass: the decision waits for the words of every shard
      shard_export(a, a.partials + static_cast<size_t>(b0) * kPartWords, nb, s_red);
      break;
    }
    if (!pop_barrier(a.bar, static_cast<unsigned int>(s), static_cast<unsigned int>(nb), a.err, a.timeout_ns))
      return;
    {
      Xacc D, E;
      unsigned int f[4];
      sum_partials(a.partials + ((s & 1) * gridDim.x + b0) * kPartWords, nb, s_red, D, E, f);
      if (tid == 0) {
        if (f[1] != 0u) {
          atomicCAS(a.err, 0, CUDAHM_ENUMERIC);
          s_stop = 1;
        } else {
          double logalpha, Drec, eb_new, logeb_new;
          theta_logalpha<M>(D, E, f, prior_ok, static_cast<double>(a.n), s_theta, s_thp, s_lpri, s_lpri_new, s_logeb,
                            s_math, logalpha, Drec, eb_new, logeb_new);
          const bool acc = __ldg(a.tab_lnu + s) < logalpha;
          if (lb == 0 && sg < a.trace_T) {
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
          if (a.adapt_theta) {  // the previous step's RAM update; this step's waits one sweep
            if (s_pend_eta > 0.0) ram_update_theta(p, s_Sth, s_pendU, s_pend_alpha, a.astar_theta, s_pend_eta);
            s_pend_alpha = (logalpha >= 0.0) ? 1.0 : exp_tab(logalpha, s_math);
            for (int q = 0; q < p; ++q) s_pendU[q] = __ldg(a.tab_U + s * p + q);
            s_pend_eta = eta;
          }
          const long long post = s - burn_left;
          if (post >= 0 && prog->thin > 0 && ((post + 1) % prog->thin) == 0) {
            if (lb == 0 && rows)
              for (int q = 0; q < p; ++q) rows[s_rows_written * p + q] = s_theta[q];
            s_rows_written++;
          }
        }
      }
    }
    __syncthreads();
    if (s_stop) return;
    if constexpr (kTiled)
      if (s + 1 < ns) tile_prefetch_first<M>(a, ring, nb0, nb1, ((k + 1u) & 1u) == 0u);  // overlaps the next proposal
  }
  __shared__ unsigned int s_macc;
  if (tid == 0) s_macc = 0;
  __syncthreads();
  atomicAdd(&s_macc, member_acc);
  __syncthreads();
  if (tid == 0) {
    atomicAdd(reinterpret_cast<unsigned long long*>(&a.chain->member_acc), static_cast<unsigned long long>(s_macc));
    if (lb == 0 && a.shard_out == nullptr) {  // (a shard's theta side moves in shard_decide_kernel)
      for (int q = 0; q < p; ++q) a.chain->theta[q] = s_theta[q];
      for (int q = 0; q < p * p; ++q) a.chain->S_theta[q] = s_Sth[q];
      for (int q = 0; q < p; ++q) a.chain->pend_U[q] = s_pendU[q];
      a.chain->pend_alpha = s_pend_alpha;
      a.chain->pend_eta = s_pend_eta;
      a.chain->etabar = s_etabar;
      a.chain->sweeps = k0 + ns;
      a.chain->theta_acc += s_tacc;
      prog->off = off + ns;
      prog->rows += s_rows_written;
      if (mom_k > 0) {  // commit the moments this launch wrote
        a.chain->mom_n = mom_n0 + mom_k;
        a.chain->mom_sel = 1 - mom_sel;
      }
      prog->t_ns = globaltimer_ns() - t_start;
    }
  }
}

// kD1: a batch of one-dimensional latents only (NN1, LF, BB1). Without the d = 3 member code the
// kernel needs far fewer registers, so more warps per SM hide the latency of the streamed state.
template <bool F32, bool kD1>
__global__ void __launch_bounds__(256, (kD1 && F32) ? 4 : 2) batch_kernel(const SweepArgs* __restrict__ pops,
                                                       BatchProg* __restrict__ progs, const int* __restrict__ b0s,
                                                       const int* __restrict__ nbs, int npop, int chunk, int R) {
  extern __shared__ double s_dyn[];
  __shared__ double s_theta[kMaxP], s_thp[kMaxP], s_Sth[kMaxP * kMaxP];
  __shared__ BlockRed s_red;
  __shared__ SweepArgs s_args;
  __shared__ int s_pop;
  if (threadIdx.x == 0) s_pop = find_pop(b0s, npop, blockIdx.x);
  __syncthreads();
  const int pop = s_pop;
  // the population's arguments, copied word by word into shared memory
  {
    const int words = static_cast<int>(sizeof(SweepArgs) / sizeof(int));
    const int* src = reinterpret_cast<const int*>(pops + pop);
    int* dst = reinterpret_cast<int*>(&s_args);
    for (int q = threadIdx.x; q < words; q += blockDim.x) dst[q] = src[q];
  }
  __syncthreads();
  const int b0 = b0s[pop], lb = blockIdx.x - b0, nb = nbs[pop];
  BatchProg* prog = progs + pop;
  if (lb >= nb || prog->off >= prog->total) return;  // spare block, or the population has finished
  if (s_args.shard_out != nullptr) {  // a shard pass after a failed decision does nothing
    __shared__ int s_failed;
    if (threadIdx.x == 0) s_failed = ld_volatile_i32(s_args.err);
    __syncthreads();
    if (s_failed) return;
  }
  if (s_args.model == CUDAHM_NN1)
    run_population<NN1, F32>(s_args, prog, b0, lb, nb, chunk, R, s_dyn, s_theta, s_thp, s_Sth, s_red);
  else if (s_args.model == CUDAHM_LF)
    run_population<LF, F32>(s_args, prog, b0, lb, nb, chunk, R, s_dyn, s_theta, s_thp, s_Sth, s_red);
  else if (s_args.model == CUDAHM_BB1) {
    if constexpr (!F32)  // FP64 form only
      run_population<BB1, false>(s_args, prog, b0, lb, nb, chunk, R, s_dyn, s_theta, s_thp, s_Sth, s_red);
  } else if constexpr (!kD1) {
    if (s_args.model == CUDAHM_NN3)
      run_population<NN3, F32>(s_args, prog, b0, lb, nb, chunk, R, s_dyn, s_theta, s_thp, s_Sth, s_red);
    else
      run_population<MVN3, F32>(s_args, prog, b0, lb, nb, chunk, R, s_dyn, s_theta, s_thp, s_Sth, s_red);
  }
}

const void* batch_fn(bool f32, bool d1) {
  if (f32) return d1 ? reinterpret_cast<const void*>(&batch_kernel<true, true>)
                     : reinterpret_cast<const void*>(&batch_kernel<true, false>);
  return d1 ? reinterpret_cast<const void*>(&batch_kernel<false, true>)
            : reinterpret_cast<const void*>(&batch_kernel<false, false>);
}

// binary32 member data of the FP32 form (kData32 rows of stride n32 >= n, member-minor; the
// padding members hold zeros)
template <class M>
__global__ void data32_kernel(long long n, long long n32, const double* y, const double* aux, ModelConsts mc,
                              float* d32) {
  const long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n32) return;
  float d[M::kData32];
  if (i < n) M::data32(y[i], aux[i], mc, d);
  else
    for (int c = 0; c < M::kData32; ++c) d[c] = 0.0f;
#pragma unroll
  for (int c = 0; c < M::kData32; ++c) d32[c * n32 + i] = d[c];
}

// binary32 member data of the d = 3 model: y_ij as hi + lo, 1/(2 s_ij^2) (inputs stored per component)
__global__ void data32_mvn3_kernel(long long n, const double* y, const double* aux, float* d32) {
  const long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int j = 0; j < 3; ++j) {
    float hi, lo;
    split_f(y[j * n + i], hi, lo);
    d32[(2 * j) * n + i] = hi;
    d32[(2 * j + 1) * n + i] = lo;
    d32[(6 + j) * n + i] = static_cast<float>(0.5 * aux[j * n + i]);
  }
}

// The theta draws of sweep k into slot s of a population's tables: p normals (Philox stream 1,
// member word 0, sweep k; block j gives normals 2j, 2j+1), the accept uniform (first uniform of
// block ceil(p/2)) and its logarithm, and eta = (k+1)^-gamma.
__device__ void theta_draws(const SweepArgs& a, uint32_t k, long long s) {
  const int p = a.p;
  const int nblk = (p + 1) / 2;
  double* U = const_cast<double*>(a.tab_U);
  for (int j = 0; j < nblk; ++j) {
    const uint4 w = philox4x32_10(make_uint4(static_cast<uint32_t>(j), 1u, 0u, k), a.key0, a.key1);
    const double ua = uniform53(w.x, w.y), ub = uniform53(w.z, w.w);
    const double rad = sqrt(-2.0 * log(ua));
    double sn, cs;
    sincospi(2.0 * ub, &sn, &cs);
    U[s * p + 2 * j] = rad * cs;
    if (2 * j + 1 < p) U[s * p + 2 * j + 1] = rad * sn;
  }
  const uint4 w = philox4x32_10(make_uint4(static_cast<uint32_t>(nblk), 1u, 0u, k), a.key0, a.key1);
  const double u = uniform53(w.x, w.y);
  const_cast<double*>(a.tab_u)[s] = u;
  const_cast<double*>(a.tab_lnu)[s] = log(u);
  const_cast<double*>(a.tab_eta)[s] = pow(static_cast<double>(k) + 1.0, -a.gamma);
}

// Theta tables of every population for the next chunk: sweep k0 + 1 + s, s < ns.
__global__ void batch_tables_kernel(const SweepArgs* __restrict__ pops, const BatchProg* __restrict__ progs, int npop,
                                    int chunk) {
  const int pop = blockIdx.y;
  if (pop >= npop) return;
  const SweepArgs& a = pops[pop];
  const BatchProg& pr = progs[pop];
  const long long left = pr.total - pr.off;
  const long long ns = left < chunk ? left : chunk;
  const long long s = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (s >= ns) return;
  theta_draws(a, static_cast<uint32_t>(a.chain->sweeps + s + 1), s);
}

// The theta step of one sweep of a split population (thread 0 of shard_decide_kernel), after
// every shard's pass: theta' from the same tables and S_theta as the passes used, log alpha from
// the summed exchange words (total, kShardWords words) with the population's member count n_pop,
// the decision, the RAM update of S_theta pending from the previous sweep and this sweep's (as
// run_population takes them), and the kept row. Every
// shard runs it on the same words and chain state, so every shard takes the same decision. The
// words must come from all `parts` shards with n_pop members in all; otherwise, or after a NaN,
// the run's error word is set and the chain stays as it was.
template <class M>
__device__ void shard_decide_one(const SweepArgs& a, BatchProg* __restrict__ prog,
                                 const unsigned long long* __restrict__ total, long long n_pop, int parts,
                                 const double* s_math) {
  using TC = typename M::TC;
  const int p = a.p;
  ChainState& ch = *a.chain;
  double theta[kMaxP], thp[kMaxP], Sth[kMaxP * kMaxP];
  for (int q = 0; q < p; ++q) theta[q] = ch.theta[q];
  for (int q = 0; q < p * p; ++q) Sth[q] = ch.S_theta[q];
  const double lpri = M::logprior(theta, a.mc, s_math);
  const double logeb = M::kRule ? log_etabar(ch.etabar, s_math) : 0.0;
  double lpri_new;
  TC tcp;
  propose_theta<M>(a, 0, p, theta, Sth, thp, lpri_new, tcp, s_math);
  const bool prior_ok = (lpri_new != -INFINITY);
  if (total[14] != static_cast<unsigned long long>(n_pop) || total[15] != static_cast<unsigned long long>(parts)) {
    atomicCAS(a.err, 0, CUDAHM_ESTATE);  // words missing, doubled, or from another split
    return;
  }
  Xacc D, E;
  acc_to_xacc(total, D);
  acc_to_xacc(total + 6, E);
  const unsigned int f[4] = {static_cast<unsigned int>(total[12]), static_cast<unsigned int>(total[12] >> 32),
                             static_cast<unsigned int>(total[13]), static_cast<unsigned int>(total[13] >> 32)};
  if (f[1] != 0u) {
    atomicCAS(a.err, 0, CUDAHM_ENUMERIC);
    return;
  }
  double logalpha, Drec, eb_new, logeb_new;
  theta_logalpha<M>(D, E, f, prior_ok, static_cast<double>(n_pop), theta, thp, lpri, lpri_new, logeb, s_math,
                    logalpha, Drec, eb_new, logeb_new);
  const bool acc = __ldg(a.tab_lnu) < logalpha;
  if (acc) {
    for (int q = 0; q < p; ++q) ch.theta[q] = thp[q];
    if (M::kRule) ch.etabar = eb_new;
    ch.theta_acc += 1;
  }
  if (a.adapt_theta) {  // the previous step's RAM update; this step's waits one sweep
    if (ch.pend_eta > 0.0) {
      ram_update_theta(p, Sth, ch.pend_U, ch.pend_alpha, a.astar_theta, ch.pend_eta);
      for (int q = 0; q < p * p; ++q) ch.S_theta[q] = Sth[q];
    }
    ch.pend_alpha = (logalpha >= 0.0) ? 1.0 : exp_tab(logalpha, s_math);
    for (int q = 0; q < p; ++q) ch.pend_U[q] = __ldg(a.tab_U + q);
    ch.pend_eta = __ldg(a.tab_eta);
  }
  const long long post = prog->off - prog->n_burn;
  if (post >= 0 && prog->thin > 0 && ((post + 1) % prog->thin) == 0) {
    if (a.rows)
      for (int q = 0; q < p; ++q) a.rows[prog->rows * p + q] = acc ? thp[q] : theta[q];
    prog->rows += 1;
  }
  ch.sweeps += 1;
  prog->off += 1;
}

// One block of two warps: thread 0 takes the decision (shard_decide_one) while warp 1 draws the
// next sweep's theta tables into slot 1 (they do not depend on the decision), which thread 0
// then moves to slot 0, where the next pass and decision read them.
template <class M>
__global__ void shard_decide_kernel(const SweepArgs* __restrict__ pop, BatchProg* __restrict__ prog,
                                    const unsigned long long* __restrict__ total, long long n_pop, int parts) {
  __shared__ double s_math[kMathWords];
  __shared__ long long s_off, s_total, s_k;
  __shared__ int s_run;
  const SweepArgs& a = *pop;
  if (threadIdx.x == 0) {
    s_off = prog->off;
    s_total = prog->total;
    s_k = a.chain->sweeps;
    s_run = (ld_volatile_i32(a.err) == 0 && s_off < s_total) ? 1 : 0;
  }
  for (int q = threadIdx.x; q < kMathWords; q += blockDim.x) s_math[q] = a.math_tab[q];
  __syncthreads();
  if (!s_run) return;
  const bool next = s_off + 1 < s_total;
  if (threadIdx.x == 32 && next) theta_draws(a, static_cast<uint32_t>(s_k + 2), 1);
  if (threadIdx.x == 0) shard_decide_one<M>(a, prog, total, n_pop, parts, s_math);
  __syncthreads();
  if (threadIdx.x == 0 && next) {
    const int p = a.p;
    double* U = const_cast<double*>(a.tab_U);
    for (int q = 0; q < p; ++q) U[q] = U[p + q];
    const_cast<double*>(a.tab_u)[0] = a.tab_u[1];
    const_cast<double*>(a.tab_lnu)[0] = a.tab_lnu[1];
    const_cast<double*>(a.tab_eta)[0] = a.tab_eta[1];
  }
}

}  // namespace

int data32_words(int model) {
  if (model == CUDAHM_LF) return LF::kData32;
  if (model == CUDAHM_MVN3 || model == CUDAHM_NN3) return MVN3::kData32;
  return NN1::kData32;
}

cudaError_t launch_data32(int model, long long n, long long n32, const double* y, const double* aux,
                          const ModelConsts& mc, float* d32, cudaStream_t st) {
  const int blk = 256;
  const unsigned int grid = static_cast<unsigned int>((n32 + blk - 1) / blk);
  if (model == CUDAHM_LF) data32_kernel<LF><<<grid, blk, 0, st>>>(n, n32, y, aux, mc, d32);
  else if (model == CUDAHM_MVN3 || model == CUDAHM_NN3) data32_mvn3_kernel<<<grid, blk, 0, st>>>(n, y, aux, d32);
  else data32_kernel<NN1><<<grid, blk, 0, st>>>(n, n32, y, aux, mc, d32);
  return cudaGetLastError();
}

// FP32 form, d = 1: binary32 latents into the state array (and zeros in its padding), and back
__global__ void chi_to32_kernel(long long n, long long n32, const double* chi, float* chi32) {
  const long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < n32) chi32[i] = (i < n) ? static_cast<float>(chi[i]) : 0.0f;
}
__global__ void chi_from32_kernel(long long n, const float* chi32, double* chi) {
  const long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < n) chi[i] = static_cast<double>(chi32[i]);
}

cudaError_t launch_chi_to32(long long n, long long n32, const double* chi, float* chi32, cudaStream_t st) {
  chi_to32_kernel<<<static_cast<unsigned int>((n32 + 255) / 256), 256, 0, st>>>(n, n32, chi, chi32);
  return cudaGetLastError();
}
cudaError_t launch_chi_from32(long long n, const float* chi32, double* chi, cudaStream_t st) {
  chi_from32_kernel<<<static_cast<unsigned int>((n + 255) / 256), 256, 0, st>>>(n, chi32, chi);
  return cudaGetLastError();
}

// Dynamic shared memory of the batched kernel: the exp/log tables, and when the FP32 form has
// one-dimensional populations (they stream member tiles) two stages of kTileFactor x block members of
// 4 + 8 + 4 kData32 bytes, plus slack to align them to 128 bytes.
size_t batch_smem_bytes(bool f32, bool any_d1, int block) {
  size_t b = sizeof(double) * kMathWords;
  if (f32 && any_d1) {
    static_assert(LF::kData32 == NN1::kData32, "one tile layout for the one-dimensional models");
    const size_t per = tile_member_bytes<LF>();
    b = tile_offset_bytes() + 128u + 2u * (kTileFactor * static_cast<size_t>(block)) * per;
  }
  return b;
}

cudaError_t batch_occupancy(bool f32, bool d1, int block, int smem_bytes, int* blocks_per_sm) {
  const void* fn = batch_fn(f32, d1);
  if (smem_bytes > 48 * 1024) {
    const cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes);
    if (e != cudaSuccess) return e;
  }
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, fn, block, smem_bytes);
}

cudaError_t launch_batch(bool f32, bool d1, const SweepArgs* pops, BatchProg* progs, const int* b0s, const int* nbs,
                         int npop, int chunk, int seg_slots, int grid, int block, int smem_bytes, cudaStream_t st) {
  void* args[] = {const_cast<SweepArgs**>(&pops), &progs, const_cast<int**>(&b0s), const_cast<int**>(&nbs), &npop,
                  &chunk, &seg_slots};
  const void* fn = batch_fn(f32, d1);
  return cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(block), args, smem_bytes, st);
}

cudaError_t launch_shard_decide(int model, const SweepArgs* pop, BatchProg* prog, const unsigned long long* total,
                                long long n_pop, int parts, cudaStream_t st) {
  switch (model) {
    case CUDAHM_NN1: shard_decide_kernel<NN1><<<1, 64, 0, st>>>(pop, prog, total, n_pop, parts); break;
    case CUDAHM_LF: shard_decide_kernel<LF><<<1, 64, 0, st>>>(pop, prog, total, n_pop, parts); break;
    case CUDAHM_BB1: shard_decide_kernel<BB1><<<1, 64, 0, st>>>(pop, prog, total, n_pop, parts); break;
    case CUDAHM_NN3: shard_decide_kernel<NN3><<<1, 64, 0, st>>>(pop, prog, total, n_pop, parts); break;
    case CUDAHM_MVN3: shard_decide_kernel<MVN3><<<1, 64, 0, st>>>(pop, prog, total, n_pop, parts); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_batch_tables(const SweepArgs* pops, const BatchProg* progs, int npop, int chunk, cudaStream_t st) {
  dim3 grid((chunk + 127) / 128, npop);
  batch_tables_kernel<<<grid, 128, 0, st>>>(pops, progs, npop, chunk);
  return cudaGetLastError();
}

}  // namespace chm
