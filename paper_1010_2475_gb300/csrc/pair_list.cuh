// Interaction-list form of the all-pairs kernel (FP32 records, far field on).
//
// The direct form (pair_launch.cuh) stages 32-source tiles for a CTA that
// holds several target groups and decides near or far per (warp, tile):
// warps whose targets see a tile as far wait at the CTA barrier while the
// others evaluate it.  Here the pairs are sorted by kind before any is
// evaluated, so that every warp of a CTA does the same work:
//  1. near lists (near_list_kernel): for each target group tg (32
//     consecutive sorted targets, one warp), the source groups whose box
//     comes within x_far(M) of tg's box, each with the 32-bit mask of its
//     sources that lie within x_far(M) of tg's box;
//  2. near pairs (near_pair_kernel): one CTA per (target group, list
//     segment).  Its W warps serve the same 32 targets and take the
//     segment's near sources in turn: in round r warp w evaluates the
//     (r W + w)-th near source, then the CTA meets at one barrier, so all
//     warps run the same code in step.  Each warp brings its sources into
//     shared-memory slots of its own by 1-D bulk copies (cp.async.bulk,
//     completion on an mbarrier per slot) issued NST rounds ahead.  Each
//     warp keeps (hi, lo) sums of its own in shared memory; they are added
//     across the warps in FP64 at the end;
//  3. far field (far_pair_kernel): one warp per (target group, range of
//     source groups), no CTA barrier: far tiles through their expansion
//     about the tile centre when far enough (tile_takes_m2p), else source by
//     source with the point-vortex multipoles, and the sources of near tiles
//     that lie beyond x_far(M) of the target box, also one by one.  Writes
//     the edge columns (beta1 <= 1) of its own partial block: the far field
//     is harmonic and has no Laplacian columns.
// The criteria (tile_is_far, point_is_far, tile_takes_m2p) and the per-pair
// arithmetic (PairNear, FarSums) are those of the direct form, so the result
// differs from it only in the order of the sums.
#pragma once

#include "pair_launch.cuh"

namespace mmvm {

// ------------------------------------------------------------------ PTX helpers
__device__ __forceinline__ unsigned smem_addr(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
               : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// Arrive once on bar and expect `bytes` of transaction (the bulk copy's).
__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}
// 1-D bulk copy global -> shared; dst, src 16-byte aligned, bytes a multiple
// of 16; completes `bytes` of transaction on bar.
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, unsigned bytes,
                                              unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}" : "=r"(ok) : "r"(smem_addr(bar)), "r"(parity) : "memory");
  return ok != 0;
}
// Bounded wait for the phase of the given parity to complete: false if it
// did not complete within the limit (each try_wait itself suspends for a
// while, so the limit is seconds of waiting).
constexpr int kWaitLimit = 1 << 22;
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long* bar, unsigned parity) {
  for (int i = 0; i < kWaitLimit; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

// ------------------------------------------------------------------ boxes
__device__ __forceinline__ float box_dist2(const float4 a, const float4 b) {
  const float dx = fmaxf(0.f, fmaxf(a.x - b.y, b.x - a.y));
  const float dy = fmaxf(0.f, fmaxf(a.z - b.w, b.z - a.w));
  return dx * dx + dy * dy;
}
// tile_takes_m2p for a target box tb and a source group's (centre, radius) c.
__device__ __forceinline__ bool takes_m2p(const float4 tb, const float4 c) {
  const float dx = fmaxf(0.f, fmaxf(tb.x - c.x, c.x - tb.y));
  const float dy = fmaxf(0.f, fmaxf(tb.z - c.y, c.y - tb.w));
  return c.z * c.z <= kM2PTheta2 * (dx * dx + dy * dy);
}

// ------------------------------------------------------------------ 1. near lists
// ent[tg * G + e] = (source group, near mask), e < cnt[tg], in increasing
// source-group order; only groups with a non-empty mask are listed.  One warp
// per target group; groups of kGroup sorted records, the last one partial.
template <int M>
__global__ void near_list_kernel(const float* __restrict__ rec, int n, int G,
                                 const float* __restrict__ gdata, int2* __restrict__ ent,
                                 int* __restrict__ cnt) {
  constexpr int R = rec_len<float>(M), GL = gdata_len(M);
  const int lane = threadIdx.x & 31;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int tg = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; tg < G; tg += nwarps) {
    const float4 tb = *reinterpret_cast<const float4*>(gdata + (size_t)tg * GL);
    int c = 0;
    for (int gb = 0; gb < G; gb += 32) {
      const int g = gb + lane;
      bool nearg = false;
      if (g < G) {
        const float4 sb = *reinterpret_cast<const float4*>(gdata + (size_t)g * GL);
        nearg = box_dist2(tb, sb) < x_far(M);
      }
      unsigned bal = __ballot_sync(0xffffffffu, nearg);
      while (bal) {
        const int gg = gb + __ffs(bal) - 1;
        bal &= bal - 1;
        const int s = gg * kGroup + lane;
        bool ns = false;
        if (s < n) {
          const float* r = rec + (size_t)s * R;
          ns = !point_is_far<M>(tb, r[0], r[1]);
        }
        const unsigned m = __ballot_sync(0xffffffffu, ns);
        if (m) {
          if (lane == 0) ent[(size_t)tg * G + c] = make_int2(gg, (int)m);
          ++c;
        }
      }
    }
    if (lane == 0) cnt[tg] = c;
  }
}

// ------------------------------------------------------------------ 2. near pairs
template <int M, int LO, int HI, int PART, int W, int NST>
struct NearListSmem {
  static constexpr int R = rec_len<float>(M);
  static constexpr int NS = PartCols<LO, HI, PART>::NS;
  // per warp: NST slots of one source record each, NST mbarriers
  static constexpr size_t slot_off = 0;
  static constexpr size_t acc_off = slot_off + (size_t)W * NST * R * 4;
  static constexpr size_t ent_off = acc_off + (size_t)2 * W * NS * 32 * 4;
  // list entries per window: 256, or 128 where the (hi, lo) sums leave too
  // little shared memory for the window's source list
  static constexpr size_t win_bytes(int win) {
    return ((ent_off + (size_t)win * 8 + (win + 1) * 4 + (size_t)win * 64 + 7) / 8 * 8) +
           (size_t)W * NST * 8;
  }
  static constexpr int WIN = win_bytes(256) <= 232448 ? 256 : 128;
  static constexpr size_t pref_off = ent_off + (size_t)WIN * 8;
  // the window's near sources in order, (entry << 5) | lane of the source
  static constexpr size_t src_off = pref_off + (WIN + 1) * 4;
  static constexpr size_t bar_off = (src_off + (size_t)WIN * 32 * 2 + 7) / 8 * 8;
  static constexpr size_t bytes = bar_off + (size_t)W * NST * 8;
  static_assert(WIN * 32 <= 65536, "source entries are 16-bit");
  static_assert((R * 4) % 16 == 0, "a record must be a whole number of 16-byte chunks");
};

// Rounds between flushes of a warp's FP32 register sums into its (hi, lo)
// pair: one source per round, so 32 sources per flush as in the direct form.
constexpr int kNearFlush = 32;

// One CTA: the near pairs of target group blockIdx.x against list segment
// blockIdx.y of C (the entries [y cnt / C, (y+1) cnt / C) of its list); writes
// this part's columns of partial block blockIdx.y ([NB][n] FP64).
//
// The segment is taken in windows of WIN list entries: warp 0 forms the
// exclusive prefix sums of the entries' near counts, the CTA lists the
// window's near sources in order (16-bit entry and lane), then round k gives
// warp w the (k W + w)-th near source of the window.  Each warp brings its own
// sources into NST record slots of its own, one bulk copy per source issued
// by its lane 0 NST rounds ahead (completion on the slot's mbarrier), so a
// warp only ever waits for copies it issued itself.  SYNC > 0: a CTA barrier
// after every SYNC rounds keeps the warps on the same code (shared
// instruction fetch); SYNC = 0 lets them drift apart within a window (their
// stalls then overlap less).  err (set to 1) reports a copy that did not
// complete within the wait limit.
template <int M, int LO, int HI, int PART, int W, int MINB, int NST, int SYNC>
__global__ void __launch_bounds__(W * 32, MINB)
    near_pair_kernel(const float* __restrict__ rec, int n, int G, const int2* __restrict__ ent,
                     const int* __restrict__ cnt, int C, double* __restrict__ partial,
                     unsigned long long* __restrict__ counts, int* __restrict__ err) {
  using PN = PairNear<M, float, LO, HI, PART>;
  using PC = PartCols<LO, HI, PART>;
  using L = NearListSmem<M, LO, HI, PART, W, NST>;
  constexpr int R = L::R, NS = PC::NS, NBL = PN::NBL, NB = n_beta(M), WIN = L::WIN;
  extern __shared__ __align__(16) unsigned char smem_list[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float* slots = reinterpret_cast<float*>(smem_list + L::slot_off) + (size_t)warp * NST * R;
  float* acc_hi = reinterpret_cast<float*>(smem_list + L::acc_off);
  float* acc_lo = acc_hi + W * NS * 32;
  int2* ent_s = reinterpret_cast<int2*>(smem_list + L::ent_off);
  int* pref_s = reinterpret_cast<int*>(smem_list + L::pref_off);
  unsigned short* src_s = reinterpret_cast<unsigned short*>(smem_list + L::src_off);
  unsigned long long* bar =
      reinterpret_cast<unsigned long long*>(smem_list + L::bar_off) + (size_t)warp * NST;

  const int tg = blockIdx.x;
  const int j = tg * kGroup + lane;
  const int ne = cnt[tg];
  const int e0 = (int)((long long)blockIdx.y * ne / C);
  const int e1 = (int)((long long)(blockIdx.y + 1) * ne / C);
  const int2* tent = ent + (size_t)tg * G;

  float tz1 = 3e15f, tz2 = 3e15f, tl1 = 0.f, tl2 = 0.f;
  if (j < n) {
    const float* r = rec + (size_t)j * R;
    tz1 = r[0];
    tz2 = r[1];
    tl1 = r[2];
    tl2 = r[3];
  }
  float acc[NBL];
#pragma unroll
  for (int b = 0; b < NBL; ++b) acc[b] = 0.f;
  float* my_hi = acc_hi + warp * NS * 32;
  float* my_lo = acc_lo + warp * NS * 32;
  for (int i = lane; i < NS * 32; i += 32) {
    my_hi[i] = 0.f;
    my_lo[i] = 0.f;
  }
  if (lane == 0) {
    for (int s = 0; s < NST; ++s) mbar_init(bar + s, 1);
    fence_mbar_init();
  }
  __syncthreads();

  unsigned n_near = 0;
  bool timeout = false;
  int since_flush = 0;
  int tbase = 0;  // sources this warp took in earlier windows (slot t % NST, phase t / NST)
  for (int wb = e0; wb < e1; wb += WIN) {
    const int nw = min(e1 - wb, WIN);
    // the window's entries and the exclusive prefix sum of their near counts
    // (warp 0: each lane scans WIN/32 consecutive entries; past nw they count 0)
    if (warp == 0) {
      constexpr int PER = WIN / 32;
      int cnts[PER];
      int loc = 0;
#pragma unroll
      for (int i = 0; i < PER; ++i) {
        const int e = lane * PER + i;
        int c = 0;
        if (e < nw) {
          const int2 en = tent[wb + e];
          ent_s[e] = en;
          c = __popc((unsigned)en.y);
        }
        cnts[i] = c;
        loc += c;
      }
      int incl = loc;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
      }
      int run = incl - loc;
#pragma unroll
      for (int i = 0; i < PER; ++i) {
        pref_s[lane * PER + i] = run;
        run += cnts[i];
      }
      if (lane == 31) pref_s[WIN] = incl;
    }
    __syncthreads();
    // every thread lists the near sources of one entry at the entry's offset
    for (int e = threadIdx.x; e < nw; e += W * 32) {
      unsigned m = (unsigned)ent_s[e].y;
      int q = pref_s[e];
      while (m) {
        src_s[q++] = (unsigned short)((e << 5) | (__ffs(m) - 1));
        m &= m - 1;
      }
    }
    __syncthreads();
    const int Lw = pref_s[WIN];
    const int mine = Lw > warp ? (Lw - 1 - warp) / W + 1 : 0;  // this warp's sources
    // lane 0: bulk copy of the k-th source of this warp into slot (tbase + k) % NST
    auto issue = [&](int k) {
      const unsigned sv = src_s[warp + k * W];
      const int ls = (int)(sv & 31u);
      const int2 en = ent_s[sv >> 5];
      const int t = tbase + k;
      unsigned long long* b = bar + t % NST;
      mbar_arrive_expect_tx(b, (unsigned)(R * 4));
      bulk_copy_g2s(slots + (size_t)(t % NST) * R, rec + ((size_t)en.x * kGroup + ls) * R,
                    (unsigned)(R * 4), b);
    };
    if (lane == 0)
      for (int k = 0; k < min(NST, mine); ++k) issue(k);
    for (int k = 0; k * W < Lw; ++k) {
      const int p = warp + k * W;
      if (p < Lw) {
        const unsigned sv = src_s[p];
        const int ls = (int)(sv & 31u);
        const int2 en = ent_s[sv >> 5];
        const int t = tbase + k;
        if (!mbar_wait_bounded(bar + t % NST, (unsigned)((t / NST) & 1))) timeout = true;
        near_source<M, float, LO, HI, PART>(slots + (size_t)(t % NST) * R, en.x * kGroup + ls,
                                            j, tz1, tz2, tl1, tl2, acc);
        if (j < n) ++n_near;
      }
      if (++since_flush == kNearFlush) {
        flush_sums<LO, HI, PART, 32>(acc, my_hi, my_lo, lane);
        since_flush = 0;
      }
      if constexpr (SYNC > 0) {
        if (k % SYNC == SYNC - 1) __syncthreads();  // CTA-uniform: the warps stay in step
      }
      __syncwarp();  // every lane has read this round's slot before it is refilled
      if (lane == 0 && k + NST < mine) {
        fence_proxy_async_smem();
        issue(k + NST);
      }
    }
    tbase += mine;
    __syncthreads();  // the next window overwrites ent_s / pref_s
  }
  flush_sums<LO, HI, PART, 32>(acc, my_hi, my_lo, lane);
  if (timeout) {
    // a copy may still be in flight: wait (bounded) for this warp's last
    // NST copies before the CTA's shared memory is released
    if (lane == 0) {
      for (int t = max(0, tbase - NST); t < tbase; ++t)
        mbar_wait_bounded(bar + t % NST, (unsigned)((t / NST) & 1));
      atomicExch(err, 1);
    }
  }
  if (LO == 1 && PART != 2 && counts != nullptr) {
    const unsigned wn = __reduce_add_sync(0xffffffffu, n_near);
    if (lane == 0 && wn) atomicAdd(counts, (unsigned long long)wn);
  }
  __syncthreads();  // every warp's (hi, lo) sums are in shared memory
  // (hi, lo) sums of the W warps -> FP64, this part's columns of block y:
  // column c (slot q) is summed by warp q mod W, one target per lane (the
  // column of each slot is a compile-time constant).  The W pairs are added
  // in FP32 with the rounding of every hi addition carried into lo, and only
  // the final pair is widened: FP64 arithmetic is a small fraction of the
  // FP32 rate here, and the CTA's tail runs alone on its SM.
  double* out = partial + (size_t)blockIdx.y * NB * n + (size_t)PN::B0 * n;
  const int jj = tg * kGroup + lane;
  static_for<0, NBL>([&](auto cc) {
    constexpr int c = decltype(cc)::value;
    if constexpr (PC::in(c)) {
      constexpr int q = PC::slot(c);
      if (warp == q % W) {
        float h = 0.f, l = 0.f;
#pragma unroll
        for (int w = 0; w < W; ++w) {
          const float v = acc_hi[(w * NS + q) * 32 + lane];
          const float sum = h + v;
          const float bp = sum - h;
          l += ((h - (sum - bp)) + (v - bp)) + acc_lo[(w * NS + q) * 32 + lane];
          h = sum;
        }
        if (jj < n) out[(size_t)c * n + jj] = (double)h + (double)l;
      }
    }
  });
}

// ------------------------------------------------------------------ 3. far field
// Edge column e = 2 (|beta| - 1) + beta1 of the far partial blocks
// ([S][2 BMAX][n] FP64): beta = (beta1, |beta| - beta1), beta1 in {0, 1}.
__host__ __device__ constexpr int n_edge(int M) { return 2 * bmax_of(M); }

constexpr int kFarWarps = 4;  // warps (target groups) per CTA of the far kernel
constexpr int kFarFlush = 8;  // tile expansions summed in FP32 between flushes

__device__ __forceinline__ void two_sum_into(float& hi, float& lo, float v) {
  const float s = hi + v;
  const float bp = s - hi;
  lo += (hi - (s - bp)) + (v - bp);
  hi = s;
}

// One warp: target group tg against source groups [g0, g1).
template <int M>
__global__ void __launch_bounds__(kFarWarps * 32)
    far_pair_kernel(const float* __restrict__ rec, int n, int G, const float* __restrict__ gdata,
                    int S, double* __restrict__ fpart, unsigned long long* __restrict__ counts) {
  constexpr int R = rec_len<float>(M), K = n_moments(M), HDR = Rec<float>::HDR;
  constexpr int GL = gdata_len(M), NA = m2p_terms(M), BM = bmax_of(M), NE = n_edge(M);
  constexpr int NF = 2 * (M + 1);  // floats of a source's multipoles A'_n
  const int lane = threadIdx.x & 31;
  const int tg = blockIdx.x * kFarWarps + (threadIdx.x >> 5);
  if (tg >= G) return;  // the whole warp (no CTA barrier in this kernel)
  const int g0 = (int)((long long)blockIdx.y * G / S);
  const int g1 = (int)((long long)(blockIdx.y + 1) * G / S);
  const int j = tg * kGroup + lane;
  float tz1 = 3e15f, tz2 = 3e15f, tl1 = 0.f, tl2 = 0.f;
  if (j < n) {
    const float* r = rec + (size_t)j * R;
    tz1 = r[0];
    tz2 = r[1];
    tl1 = r[2];
    tl2 = r[3];
  }
  const float4 tb = *reinterpret_cast<const float4*>(gdata + (size_t)tg * GL);
  float yhr[BM], yhi[BM], ylr[BM], yli[BM], tyr[BM], tyi[BM];
#pragma unroll
  for (int b = 0; b < BM; ++b) {
    yhr[b] = yhi[b] = ylr[b] = yli[b] = tyr[b] = tyi[b] = 0.f;
  }
  auto flush = [&]() {
#pragma unroll
    for (int b = 0; b < BM; ++b) {
      two_sum_into(yhr[b], ylr[b], tyr[b]);
      two_sum_into(yhi[b], yli[b], tyi[b]);
      tyr[b] = 0.f;
      tyi[b] = 0.f;
    }
  };
  unsigned n_far = 0, n_m2p = 0, n_m2p_pairs = 0;
  int pending = 0;  // tile expansions in ty since the last flush
  for (int g = g0; g < g1; ++g) {
    const float* gd = gdata + (size_t)g * GL;
    const float4 sb = *reinterpret_cast<const float4*>(gd);
    const int nsrc = min(kGroup, n - g * kGroup);
    const bool far_tile = box_dist2(tb, sb) >= x_far(M);
    if (far_tile && takes_m2p(tb, *reinterpret_cast<const float4*>(gd + 4))) {
      // the tile through its expansion about its centre
      const float cx = gd[4], cy = gd[5];
      const float d1 = tz1 - cx, d2 = tz2 - cy;
      const float b1 = d1 + tl1, b2 = d2 + tl2;
      const float v1 = b1 - d1, v2 = b2 - d2;
      const float l1 = (d1 - (b1 - v1)) + (tl1 - v1);
      const float l2 = (d2 - (b2 - v2)) + (tl2 - v2);
      FarSums<NA, float, 1, BM>::run(b1, b2, l1, l2, gd + 8, tyr, tyi);
      if (j < n) {
        n_m2p += 1;
        n_m2p_pairs += nsrc;
      }
      if (++pending == kFarFlush) {
        flush();
        pending = 0;
      }
      continue;
    }
    // source by source: every source of a far tile, or the sources of a near
    // tile that lie beyond x_far(M) of the whole target box
    const int s = g * kGroup + lane;
    float z[4] = {0.f, 0.f, 0.f, 0.f}, af[NF];
#pragma unroll
    for (int q = 0; q < NF; ++q) af[q] = 0.f;
    bool mine = false;
    if (lane < nsrc) {
      const float* r = rec + (size_t)s * R;
      const float4 zz = *reinterpret_cast<const float4*>(r);
      z[0] = zz.x;
      z[1] = zz.y;
      z[2] = zz.z;
      z[3] = zz.w;
      mine = far_tile || point_is_far<M>(tb, zz.x, zz.y);
      if (mine) {
#pragma unroll
        for (int q = 0; q < NF; ++q) af[q] = r[HDR + K + q];
      }
    }
    unsigned fm = __ballot_sync(0xffffffffu, mine);
    if (!fm) continue;
    if (j < n) n_far += __popc(fm);
    while (fm) {
      const int src = __ffs(fm) - 1;
      fm &= fm - 1;
      float a[NF];
#pragma unroll
      for (int q = 0; q < NF; ++q) a[q] = __shfl_sync(0xffffffffu, af[q], src);
      const float sz1 = __shfl_sync(0xffffffffu, z[0], src);
      const float sz2 = __shfl_sync(0xffffffffu, z[1], src);
      const float sl1 = __shfl_sync(0xffffffffu, z[2], src);
      const float sl2 = __shfl_sync(0xffffffffu, z[3], src);
      const float d1 = tz1 - sz1, e1 = tl1 - sl1;
      const float d2 = tz2 - sz2, e2 = tl2 - sl2;
      const float b1 = d1 + e1, b2 = d2 + e2;
      const float v1 = b1 - d1, v2 = b2 - d2;
      const float l1 = (d1 - (b1 - v1)) + (e1 - v1);
      const float l2 = (d2 - (b2 - v2)) + (e2 - v2);
      FarSums<M + 1, float, 1, BM>::run(b1, b2, l1, l2, a, tyr, tyi);
    }
    flush();
    pending = 0;
  }
  flush();
  if (counts != nullptr) {
    const unsigned wf = __reduce_add_sync(0xffffffffu, n_far);
    const unsigned we = __reduce_add_sync(0xffffffffu, n_m2p);
    const unsigned wp = __reduce_add_sync(0xffffffffu, n_m2p_pairs);
    if (lane == 0) {
      if (wf) atomicAdd(counts + 1, (unsigned long long)wf);
      if (we) atomicAdd(counts + 2, (unsigned long long)we);
      if (wp) atomicAdd(counts + 3, (unsigned long long)wp);
    }
  }
  if (j < n) {
    // Psi[beta] += -Re((-i)^{beta1 + |beta|} Y[|beta|]) / (2 pi) (see fold_far), in FP64
    constexpr double s2pi = 1.0 / (2.0 * 3.14159265358979323846);
    double* o = fpart + (size_t)blockIdx.y * NE * n + j;
#pragma unroll
    for (int nb = 1; nb <= BM; ++nb) {
      const double yr = (double)yhr[nb - 1] + (double)ylr[nb - 1];
      const double yi = (double)yhi[nb - 1] + (double)yli[nb - 1];
#pragma unroll
      for (int bb1 = 0; bb1 < 2; ++bb1) {
        const int r = (bb1 + nb) & 3;
        const double v = r == 0 ? -yr : r == 1 ? -yi : r == 2 ? yr : yi;
        o[(size_t)(2 * (nb - 1) + bb1) * n] = s2pi * v;
      }
    }
  }
}

// ------------------------------------------------------------------ 4. tree far field
// A binary tree over the Morton order of the groups: level 0 is the groups
// themselves (gdata), node i of level L >= 1 holds the groups of nodes 2i and
// 2i+1 of level L-1, i.e. the consecutive groups [i 2^L, (i+1) 2^L).  A node
// record has the group-record layout (gdata_len): the union of the children's
// boxes, the box centre c, a radius bounding |source - c| over its sources
// (max over the children of |c_child - c| + radius_child), the number of
// its sources (float, in the slot that groups leave 0), and its expansion
// about c, obtained from the children's expansions by the exact shift
//   B_j(c) = sum_{k <= j} B^child_{j-k}(c_child) Delta^k / k!,
//   Delta = c_child - c
// (the multipoles of a source at distance delta from c_child sit at delta +
// Delta from c; truncation at j < m2p_terms(M) drops nothing the child had).
// A node whose box is beyond x_far(M) of a target group's box and whose
// radius is at most 0.1 of the distance from that box to its centre is
// summed through its expansion for every target of the group, as a group
// is (tile_takes_m2p), so the error bound of the tile expansions holds for
// every node; the traversal replaces the per-group expansions of far groups
// by as few node expansions as the criterion allows.

// Node i of a level from its children in the level below (nchild records;
// counts of level-0 children: min(kGroup, n - kGroup g)).
template <int M>
__global__ void tree_level_kernel(const float* __restrict__ child, int nchild, int child_is_group,
                                  int n, float* __restrict__ node, int nnode) {
  constexpr int GL = gdata_len(M), NA = m2p_terms(M);
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nnode) return;
  const int c0 = 2 * i, c1 = min(2 * i + 1, nchild - 1);
  const float* a = child + (size_t)c0 * GL;
  const float* b = child + (size_t)c1 * GL;
  float4 box = *reinterpret_cast<const float4*>(a);
  if (c1 != c0) {
    const float4 bb = *reinterpret_cast<const float4*>(b);
    box = make_float4(fminf(box.x, bb.x), fmaxf(box.y, bb.y), fminf(box.z, bb.z),
                      fmaxf(box.w, bb.w));
  }
  const float cx = 0.5f * (box.x + box.y), cy = 0.5f * (box.z + box.w);
  float br[NA], bi[NA];
#pragma unroll
  for (int j = 0; j < NA; ++j) {
    br[j] = 0.f;
    bi[j] = 0.f;
  }
  float rad = 0.f, count = 0.f;
  for (int c = c0; c <= c1; ++c) {
    const float* r = child + (size_t)c * GL;
    const float dx = r[4] - cx, dy = r[5] - cy;
    rad = fmaxf(rad, sqrtf(dx * dx + dy * dy) + r[6]);
    count += child_is_group ? (float)min(kGroup, n - kGroup * c) : r[7];
    // B_j += sum_k B^child_{j-k} Delta^k / k!
    float er = 1.f, ei = 0.f;  // Delta^k / k!
#pragma unroll
    for (int k = 0; k < NA; ++k) {
      if (k > 0) {
        const float tr = (er * dx - ei * dy) * (1.f / k);
        ei = (er * dy + ei * dx) * (1.f / k);
        er = tr;
      }
#pragma unroll
      for (int j = k; j < NA; ++j) {
        const float cr = r[8 + 2 * (j - k)], ci = r[9 + 2 * (j - k)];
        br[j] = fmaf(cr, er, fmaf(-ci, ei, br[j]));
        bi[j] = fmaf(cr, ei, fmaf(ci, er, bi[j]));
      }
    }
  }
  float* o = node + (size_t)i * GL;
  *reinterpret_cast<float4*>(o) = box;
  *reinterpret_cast<float4*>(o + 4) = make_float4(cx, cy, rad, count);
#pragma unroll
  for (int j = 0; j < NA; ++j) {
    o[8 + 2 * j] = br[j];
    o[9 + 2 * j] = bi[j];
  }
}

// Node id on the walk's stack: level << kTreeShift | index (levels <= 25 for
// n <= 2^30, indices < 2^25).  A depth-first walk holds at most one pending
// sibling per level, so the stack never exceeds levels + 2 <= 27 entries.
constexpr int kTreeShift = 26;
constexpr int kTreeStack = 32;

// One warp: target group tg against the subtree rooted at node blockIdx.y of
// level Lc (the far-field partial block blockIdx.y); S = nodes of level Lc.
template <int M>
__global__ void __launch_bounds__(kFarWarps * 32)
    far_tree_kernel(const float* __restrict__ rec, int n, int G, const float* __restrict__ gdata,
                    const float* __restrict__ tree, int Lc, double* __restrict__ fpart,
                    unsigned long long* __restrict__ counts) {
  constexpr int R = rec_len<float>(M), K = n_moments(M), HDR = Rec<float>::HDR;
  constexpr int GL = gdata_len(M), NA = m2p_terms(M), BM = bmax_of(M), NE = n_edge(M);
  constexpr int NF = 2 * (M + 1);
  __shared__ int stack_s[kFarWarps][kTreeStack];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int tg = blockIdx.x * kFarWarps + wib;
  if (tg >= G) return;  // the whole warp (no CTA barrier in this kernel)
  int* stack = stack_s[wib];
  const int j = tg * kGroup + lane;
  float tz1 = 3e15f, tz2 = 3e15f, tl1 = 0.f, tl2 = 0.f;
  if (j < n) {
    const float* r = rec + (size_t)j * R;
    tz1 = r[0];
    tz2 = r[1];
    tl1 = r[2];
    tl2 = r[3];
  }
  const float4 tb = *reinterpret_cast<const float4*>(gdata + (size_t)tg * GL);
  float yhr[BM], yhi[BM], ylr[BM], yli[BM], tyr[BM], tyi[BM];
#pragma unroll
  for (int b = 0; b < BM; ++b) {
    yhr[b] = yhi[b] = ylr[b] = yli[b] = tyr[b] = tyi[b] = 0.f;
  }
  auto flush = [&]() {
#pragma unroll
    for (int b = 0; b < BM; ++b) {
      two_sum_into(yhr[b], ylr[b], tyr[b]);
      two_sum_into(yhi[b], yli[b], tyi[b]);
      tyr[b] = 0.f;
      tyi[b] = 0.f;
    }
  };
  auto node_rec = [&](int L, int i) -> const float* {
    return L == 0 ? gdata + (size_t)i * GL : tree + (size_t)(tree_level_offset(G, L) + i) * GL;
  };
  unsigned n_far = 0, n_m2p = 0, n_m2p_pairs = 0;
  int pending = 0;
  int sp = 0;
  if (lane == 0) stack[0] = (Lc << kTreeShift) | blockIdx.y;
  sp = 1;
  __syncwarp();
  while (sp > 0) {
    const int top = stack[--sp];
    __syncwarp();
    const int L = top >> kTreeShift, i = top & ((1 << kTreeShift) - 1);
    const float* nd = node_rec(L, i);
    const float4 box = *reinterpret_cast<const float4*>(nd);
    const float4 cen = *reinterpret_cast<const float4*>(nd + 4);
    const bool far_box = box_dist2(tb, box) >= x_far(M);
    if (far_box && takes_m2p(tb, cen)) {
      // the node (or group) through its expansion about its centre
      const float d1 = tz1 - cen.x, d2 = tz2 - cen.y;
      const float b1 = d1 + tl1, b2 = d2 + tl2;
      const float v1 = b1 - d1, v2 = b2 - d2;
      const float l1 = (d1 - (b1 - v1)) + (tl1 - v1);
      const float l2 = (d2 - (b2 - v2)) + (tl2 - v2);
      FarSums<NA, float, 1, BM>::run(b1, b2, l1, l2, nd + 8, tyr, tyi);
      if (j < n) {
        n_m2p += 1;
        n_m2p_pairs += L == 0 ? min(kGroup, n - kGroup * i) : (unsigned)cen.w;
      }
      if (++pending == kFarFlush) {
        flush();
        pending = 0;
      }
      continue;
    }
    if (L > 0) {  // open the node: children 2i (taken first) and 2i+1 (if any)
      const bool two = 2 * i + 1 < tree_level_nodes(G, L - 1);
      if (lane == 0) {
        if (two) stack[sp] = ((L - 1) << kTreeShift) | (2 * i + 1);
        stack[sp + (two ? 1 : 0)] = ((L - 1) << kTreeShift) | (2 * i);
      }
      sp += two ? 2 : 1;
      __syncwarp();
      continue;
    }
    // a group not summed through its expansion: source by source, every
    // source of a far group or the sources of a near group that lie beyond
    // x_far(M) of the whole target box
    const int g = i;
    const int nsrc = min(kGroup, n - g * kGroup);
    const int s = g * kGroup + lane;
    float z[4] = {0.f, 0.f, 0.f, 0.f}, af[NF];
#pragma unroll
    for (int q = 0; q < NF; ++q) af[q] = 0.f;
    bool mine = false;
    if (lane < nsrc) {
      const float* r = rec + (size_t)s * R;
      const float4 zz = *reinterpret_cast<const float4*>(r);
      z[0] = zz.x;
      z[1] = zz.y;
      z[2] = zz.z;
      z[3] = zz.w;
      mine = far_box || point_is_far<M>(tb, zz.x, zz.y);
      if (mine) {
#pragma unroll
        for (int q = 0; q < NF; ++q) af[q] = r[HDR + K + q];
      }
    }
    unsigned fm = __ballot_sync(0xffffffffu, mine);
    if (!fm) continue;
    if (j < n) n_far += __popc(fm);
    while (fm) {
      const int src = __ffs(fm) - 1;
      fm &= fm - 1;
      float a[NF];
#pragma unroll
      for (int q = 0; q < NF; ++q) a[q] = __shfl_sync(0xffffffffu, af[q], src);
      const float sz1 = __shfl_sync(0xffffffffu, z[0], src);
      const float sz2 = __shfl_sync(0xffffffffu, z[1], src);
      const float sl1 = __shfl_sync(0xffffffffu, z[2], src);
      const float sl2 = __shfl_sync(0xffffffffu, z[3], src);
      const float d1 = tz1 - sz1, e1 = tl1 - sl1;
      const float d2 = tz2 - sz2, e2 = tl2 - sl2;
      const float b1 = d1 + e1, b2 = d2 + e2;
      const float v1 = b1 - d1, v2 = b2 - d2;
      const float l1 = (d1 - (b1 - v1)) + (e1 - v1);
      const float l2 = (d2 - (b2 - v2)) + (e2 - v2);
      FarSums<M + 1, float, 1, BM>::run(b1, b2, l1, l2, a, tyr, tyi);
    }
    flush();
    pending = 0;
  }
  flush();
  if (counts != nullptr) {
    const unsigned wf = __reduce_add_sync(0xffffffffu, n_far);
    const unsigned we = __reduce_add_sync(0xffffffffu, n_m2p);
    const unsigned wp = __reduce_add_sync(0xffffffffu, n_m2p_pairs);
    if (lane == 0) {
      if (wf) atomicAdd(counts + 1, (unsigned long long)wf);
      if (we) atomicAdd(counts + 2, (unsigned long long)we);
      if (wp) atomicAdd(counts + 3, (unsigned long long)wp);
    }
  }
  if (j < n) {
    constexpr double s2pi = 1.0 / (2.0 * 3.14159265358979323846);
    double* o = fpart + (size_t)blockIdx.y * NE * n + j;
#pragma unroll
    for (int nb = 1; nb <= BM; ++nb) {
      const double yr = (double)yhr[nb - 1] + (double)ylr[nb - 1];
      const double yi = (double)yhi[nb - 1] + (double)yli[nb - 1];
#pragma unroll
      for (int bb1 = 0; bb1 < 2; ++bb1) {
        const int r = (bb1 + nb) & 3;
        const double v = r == 0 ? -yr : r == 1 ? -yi : r == 2 ? yr : yi;
        o[(size_t)(2 * (nb - 1) + bb1) * n] = s2pi * v;
      }
    }
  }
}

template <int M, int LO, int HI, int PART, int W, int NST>
constexpr size_t near_list_smem_bytes() {
  return NearListSmem<M, LO, HI, PART, W, NST>::bytes;
}

}  // namespace mmvm
