// Launch wrapper of the all-pairs kernel: one thread per target, source
// records staged through shared memory in tiles of S = kGroup, FP32 partial
// sums carried across tiles as (hi, lo) float pairs (TwoSum), and the
// per-(source chunk, target) result written as FP64.
//
// One kernel computes one slice of the outputs: the orders
// LO <= |beta| <= HI, and of those all columns (PART 0), the edge columns
// beta1 <= 1 only (PART 1: the jet and the far field), or the Laplacian
// columns only (PART 2: Hermite functions, near sources only).  A variant
// launches its slices one after another.  Order slices keep the fully
// unrolled per-pair code short and need only the jet orders LO .. HI + M;
// column parts let the two halves of the work run with fewer registers
// each.  Parameters of a variant or slice, chosen per order by the
// autotuner:
//   TPC   targets per CTA (a multiple of 32, so each warp is one group);
//   MINB  CTAs per SM the register budget must allow;
//   SYNC  > 0: a CTA barrier after every SYNC sources, which keeps the warps
//         of a CTA on nearby code so they share instruction-cache lines.
// FP32 runs two passes over the chunk's source tiles, deciding near or far
// per (warp, tile) from the bounding boxes (x_far(M)):
//   pass 1  far tiles: through the tile's expansion about its centre when it
//           is far enough, else source by source with the point-vortex
//           multipoles; a source-by-source tile that another warp of the CTA
//           needs as near is left to pass 2;
//   pass 2  tiles some warp needs as near: near sources through the full jet
//           (PairNear), sources beyond x_far of the warp's whole box and the
//           tiles pass 1 left through the point-vortex multipoles.
// The near and far paths never hold registers at the same time, and every
// barrier is one instruction executed by the whole CTA.
#pragma once

#include "common.cuh"
#include "pair_kernel.cuh"

namespace mmvm {

// One near-field source.  acc points at the register array of the slice;
// every index used is a compile-time constant after inlining.
template <int M, typename T, int LO, int HI, int PART>
__device__ __forceinline__ void near_source(const T* r, int src, int j, T tz1, T tz2, T tl1,
                                            T tl2, T* acc) {
  using PN = PairNear<M, T, LO, HI, PART>;
  constexpr int K = n_moments(M);
  constexpr int HDR = Rec<T>::HDR;
  T (&accr)[PN::NBL] = *reinterpret_cast<T(*)[PN::NBL]>(acc);
  T a[K];
#pragma unroll
  for (int m = 0; m < K; ++m) a[m] = r[HDR + m];
  T b1, b2, l1 = T(0), l2 = T(0);
  if constexpr (std::is_same<T, float>::value) {
    // b = (hi difference) + (lo difference) as an exact (hi, lo) pair
    const T d1 = tz1 - r[0], e1 = tl1 - r[2];
    const T d2 = tz2 - r[1], e2 = tl2 - r[3];
    b1 = d1 + e1;
    b2 = d2 + e2;
    const T v1 = b1 - d1, v2 = b2 - d2;
    l1 = (d1 - (b1 - v1)) + (e1 - v1);
    l2 = (d2 - (b2 - v2)) + (e2 - v2);
  } else {
    b1 = tz1 - r[0];
    b2 = tz2 - r[1];
  }
  T wm = T(1);
  if (src == j) {  // self pair: excluded here, added exactly by the finish
    b1 = T(1e15);
    b2 = T(0);
    l1 = T(0);
    l2 = T(0);
    wm = T(0);
  }
  PN::run(b1, b2, l1, l2, wm, a, accr);
}

// Fold one FP32 register sum into this thread's shared-memory (hi, lo) pair.
__device__ __forceinline__ void flush_one(float& v, float* acc_hi, float* acc_lo, int idx) {
  const float hi = acc_hi[idx];
  const float sum = hi + v;
  const float bp = sum - hi;
  const float err = (hi - (sum - bp)) + (v - bp);
  acc_hi[idx] = sum;
  acc_lo[idx] += err;
  v = 0.f;
}

// beta1 of correlation column col (col = bcol(b1, b2)).
__host__ __device__ constexpr int col_beta1(int col) {
  int k = 1;
  while (tri(k + 1) - 1 <= col) ++k;
  return k - (col + 1 - tri(k));
}

// The columns of slice [LO, HI] that part PART accumulates (see SliceSpec),
// numbered from the slice's first column, and their compact shared-memory
// slots: column c of the slice sits at slot(c).
template <int LO, int HI, int PART>
struct PartCols {
  static constexpr int B0 = tri(LO) - 1;
  static constexpr int NBL = tri(HI + 1) - 1 - B0;
  __host__ __device__ static constexpr bool in(int c) {
    return PART == 0 || ((col_beta1(c + B0) <= 1) == (PART == 1));
  }
  __host__ __device__ static constexpr int slot(int c) {
    int s = 0;
    for (int i = 0; i < c; ++i) s += in(i) ? 1 : 0;
    return s;
  }
  static constexpr int NS = slot(NBL);  // slots in use
};

// Fold this part's FP32 register sums into this thread's shared-memory
// (hi, lo) pairs.
template <int LO, int HI, int PART, int TPC>
__device__ __forceinline__ void flush_sums(float* acc, float* acc_hi, float* acc_lo, int slot) {
  using PC = PartCols<LO, HI, PART>;
  static_for<0, PC::NBL>([&](auto cc) {
    constexpr int c = decltype(cc)::value;
    if constexpr (PC::in(c)) flush_one(acc[c], acc_hi, acc_lo, PC::slot(c) * TPC + slot);
  });
}

// The same for the edge columns (beta1 in {0, 1}) only: the far field writes
// nothing else.
template <int M, int LO, int HI, int PART, int TPC>
__device__ __forceinline__ void flush_edge_sums(float* acc, float* acc_hi, float* acc_lo,
                                                int slot) {
  using PC = PartCols<LO, HI, PART>;
  static_assert(PART != 2, "the Laplacian part has no edge columns");
  static_for<LO, HI + 1>([&](auto nbc) {
    constexpr int nb = decltype(nbc)::value;
    constexpr int c0 = bcol(0, nb) - PC::B0, c1 = bcol(1, nb - 1) - PC::B0;
    flush_one(acc[c0], acc_hi, acc_lo, PC::slot(c0) * TPC + slot);
    flush_one(acc[c1], acc_hi, acc_lo, PC::slot(c1) * TPC + slot);
  });
}

// One far-field source (FP32): multipole sums of the tile in yr/yi.
template <int M, int LO, int HI>
__device__ __forceinline__ void far_source(const float* r, float tz1, float tz2, float tl1,
                                           float tl2, float (&yr)[HI - LO + 1],
                                           float (&yi)[HI - LO + 1]) {
  constexpr int K = n_moments(M);
  constexpr int HDR = Rec<float>::HDR;
  const float d1 = tz1 - r[0], e1 = tl1 - r[2];
  const float d2 = tz2 - r[1], e2 = tl2 - r[3];
  const float b1 = d1 + e1, b2 = d2 + e2;
  const float v1 = b1 - d1, v2 = b2 - d2;
  const float l1 = (d1 - (b1 - v1)) + (e1 - v1);
  const float l2 = (d2 - (b2 - v2)) + (e2 - v2);
  PairFar<M, float, LO, HI>::run(b1, b2, l1, l2, r + HDR + K, yr, yi);
}

// Group record g (see gdata_len in common.cuh).
template <int M>
__device__ __forceinline__ const float* group_rec(const float* __restrict__ gdata, int g) {
  return gdata + (size_t)g * gdata_len(M);
}

// Does this warp's target group see source group sg only beyond x_far(M)?
template <int M>
__device__ __forceinline__ bool tile_is_far(const float* __restrict__ gdata, int tgroup, int sg) {
  const float4 sb = *reinterpret_cast<const float4*>(group_rec<M>(gdata, sg));
  const float4 tb = *reinterpret_cast<const float4*>(group_rec<M>(gdata, tgroup));
  const float dx = fmaxf(0.f, fmaxf(tb.x - sb.y, sb.x - tb.y));
  const float dy = fmaxf(0.f, fmaxf(tb.z - sb.w, sb.z - tb.w));
  return dx * dx + dy * dy >= x_far(M);
}

// Is the source centre (z1, z2) (hi parts) beyond x_far(M) of every target
// in the box tb = (min1, max1, min2, max2)?
template <int M>
__device__ __forceinline__ bool point_is_far(const float4 tb, float z1, float z2) {
  const float dx = fmaxf(0.f, fmaxf(tb.x - z1, z1 - tb.y));
  const float dy = fmaxf(0.f, fmaxf(tb.z - z2, z2 - tb.w));
  return dx * dx + dy * dy >= x_far(M);
}

// May source group sg be summed through its expansion about its centre for
// every target of group tgroup (radius <= theta x distance from the target
// box to the centre)?
template <int M>
__device__ __forceinline__ bool tile_takes_m2p(const float* __restrict__ gdata, int tgroup,
                                               int sg) {
  const float4 c = *reinterpret_cast<const float4*>(group_rec<M>(gdata, sg) + 4);
  const float4 tb = *reinterpret_cast<const float4*>(group_rec<M>(gdata, tgroup));
  const float dx = fmaxf(0.f, fmaxf(tb.x - c.x, c.x - tb.y));
  const float dy = fmaxf(0.f, fmaxf(tb.z - c.y, c.y - tb.w));
  return c.z * c.z <= kM2PTheta2 * (dx * dx + dy * dy);
}

// The far group sg summed through its expansion about its centre for this
// thread's target (centre zeta as hi parts tz, lo parts tl; warp-uniform, no
// barrier), folded into the edge columns of the thread's (hi, lo) sums.
template <int M, int LO, int HI, int PART, int TPC>
__device__ __forceinline__ void m2p_tile(const float* __restrict__ gdata, int sg, float tz1,
                                         float tz2, float tl1, float tl2, float* acc_hi,
                                         float* acc_lo, int slot) {
  constexpr int NA = m2p_terms(M);
  constexpr int NY = HI - LO + 1;
  constexpr int NBL = PairNear<M, float, LO, HI>::NBL;
  const float* g = group_rec<M>(gdata, sg);
  const float cx = g[4], cy = g[5];
  // w = target - centre = (hi - centre) + lo, as an exact (hi, lo) pair
  const float d1 = tz1 - cx, d2 = tz2 - cy;
  const float b1 = d1 + tl1, b2 = d2 + tl2;
  const float v1 = b1 - d1, v2 = b2 - d2;
  const float l1 = (d1 - (b1 - v1)) + (tl1 - v1);
  const float l2 = (d2 - (b2 - v2)) + (tl2 - v2);
  float yr[NY], yi[NY];
#pragma unroll
  for (int b = 0; b < NY; ++b) {
    yr[b] = 0.f;
    yi[b] = 0.f;
  }
  FarSums<NA, float, LO, HI>::run(b1, b2, l1, l2, g + 8, yr, yi);
  float tmp[NBL];
#pragma unroll
  for (int b = 0; b < NBL; ++b) tmp[b] = 0.f;
  fold_far<M, float, LO, HI>(yr, yi, tmp);
  flush_edge_sums<M, LO, HI, PART, TPC>(tmp, acc_hi, acc_lo, slot);
}

// The work of one CTA: targets tile0 .. tile0 + TPC - 1 (those below n) of
// one instance against its sources c0 .. c1 - 1.  rec holds the instance's n
// records (indices are local to it); gdata: one record per group of kGroup
// consecutive records (box of the hi parts, centre, radius, expansion about
// the centre; see gdata_len), null disables the far-field path (FP64
// always).  A far tile is summed through its expansion when it is far enough
// for it (tile_takes_m2p), else source by source with the point-vortex jet.
// out: this chunk's block [NB][n] of the partial sums (coalesced FP64
// stores); only the slice's columns are written.  counts (nullable):
// cumulative (near pairs, far pairs source by source, tile expansions
// evaluated, pairs they cover), added by the slice with LO = 1 that is not
// the Laplacian part.  Called by every thread of the CTA; begins by writing
// only its own shared-memory slots and reuses the tile only after a
// barrier, so a persistent CTA may call it for one item after another.
template <int M, typename T, int LO, int HI, int PART, int TPC, int SYNC>
__device__ __forceinline__ void pair_tile_work(const T* __restrict__ rec, int n, int tile0, int c0,
                                               int c1, int S, const float* __restrict__ gdata,
                                               double* __restrict__ out,
                                               unsigned long long* __restrict__ counts,
                                               unsigned char* smem_raw) {
  using PN = PairNear<M, T, LO, HI, PART>;
  using PC = PartCols<LO, HI, PART>;
  constexpr int R = rec_len<T>(M);
  constexpr int NBL = PN::NBL;
  constexpr int NY = HI - LO + 1;
  constexpr bool f32 = std::is_same<T, float>::value;
  T* tile = reinterpret_cast<T*>(smem_raw);
  float* acc_hi = reinterpret_cast<float*>(tile + (size_t)S * R);
  float* acc_lo = acc_hi + PC::NS * TPC;
  const int warp = threadIdx.x >> 5;
  const int slot = threadIdx.x;
  const int j = tile0 + slot;
  T tz1, tz2, tl1 = T(0), tl2 = T(0);
  if (j < n) {
    const T* r = rec + (size_t)j * R;
    tz1 = r[0];
    tz2 = r[1];
    if constexpr (f32) {
      tl1 = r[2];
      tl2 = r[3];
    }
  } else {
    tz1 = T(3e15);
    tz2 = T(3e15);
  }
  T acc[NBL];
#pragma unroll
  for (int b = 0; b < NBL; ++b) acc[b] = T(0);
  if constexpr (f32) {
    for (int i = threadIdx.x; i < 2 * PC::NS * TPC; i += blockDim.x) acc_hi[i] = 0.f;
  }
  // far tiles: skipped by every part; summed (pass 1) by parts 0 and 1 (the
  // Laplacian columns of a far tile are zero)
  const bool use_far = f32 && gdata != nullptr;
  // this thread's target: pairs on each path, tile expansions evaluated
  unsigned n_near = 0, n_far = 0, n_m2p = 0, n_m2p_pairs = 0;
  // did this warp accumulate anything? (warp-uniform; a warp that did not
  // stores zeros without touching its sums: FP64 arithmetic is scarce)
  bool work = false;
  // this warp's 32 targets form one group; a warp wholly past n does no work
  // (but still takes part in every barrier)
  const int wfirst = tile0 + warp * 32;
  const bool warp_valid = wfirst < n;
  const int tgroup = wfirst / kGroup;
  auto load_tile = [&](int t0, int cnt) {
    // cooperative 16-byte copy of cnt records into the tile
    const int nvec = cnt * R * (int)sizeof(T) / 16;
    const int4* src = reinterpret_cast<const int4*>(rec + (size_t)t0 * R);
    int4* dst = reinterpret_cast<int4*>(tile);
    for (int i = threadIdx.x; i < nvec; i += blockDim.x) dst[i] = __ldg(src + i);
  };
  if constexpr (f32 && PART != 2) {
    if (use_far) {
      // pass 1: far tiles (tiles start at multiples of kGroup: chunk_len is a
      // multiple of S = kGroup)
#pragma unroll 1
      for (int t0 = c0; t0 < c1; t0 += S) {
        const int cnt = min(S, c1 - t0);
        const int sg = t0 / kGroup;
        const bool far_tile = warp_valid && tile_is_far<M>(gdata, tgroup, sg);
        const bool m2p = far_tile && tile_takes_m2p<M>(gdata, tgroup, sg);
        // a tile some warp of the CTA needs as near is left to pass 2, where
        // this warp sums it (expansion or source by source) while the others
        // do near work
        const bool anynear = __syncthreads_or(warp_valid && !far_tile);
        const bool far = far_tile && !m2p && !anynear;
        if (m2p && !anynear) {  // left to pass 2 when the CTA loads the tile anyway
          work = true;
          m2p_tile<M, LO, HI, PART, TPC>(gdata, sg, tz1, tz2, tl1, tl2, acc_hi, acc_lo, slot);
          if (j < n) {
            n_m2p += 1;
            n_m2p_pairs += cnt;
          }
        }
        if (far && j < n) n_far += cnt;
        if (__syncthreads_or(far)) {
          load_tile(t0, cnt);
          __syncthreads();
          float yr[NY], yi[NY];  // multipole sums of this tile
#pragma unroll
          for (int b = 0; b < NY; ++b) {
            yr[b] = 0.f;
            yi[b] = 0.f;
          }
#pragma unroll 1
          for (int s = 0; s < cnt; ++s) {
            if (far)
              far_source<M, LO, HI>(reinterpret_cast<const float*>(tile) + s * R, tz1, tz2, tl1,
                                    tl2, yr, yi);
            if constexpr (SYNC > 0) {
              if (s % SYNC == SYNC - 1 || s == cnt - 1) __syncthreads();  // CTA-uniform
            }
          }
          if (far) {
            work = true;
            float tmp[NBL];
#pragma unroll
            for (int b = 0; b < NBL; ++b) tmp[b] = 0.f;
            fold_far<M, float, LO, HI>(yr, yi, tmp);
            flush_edge_sums<M, LO, HI, PART, TPC>(tmp, acc_hi, acc_lo, slot);
          }
        }
      }
    }
  }
  // pass 2: near tiles (every tile when the far field is off).  Within a near
  // tile, a source beyond x_far(M) of the warp's whole target box takes the
  // point-vortex path (warp-uniform): parts 0 and 1 add its edge columns,
  // part 2 has nothing to add.
  float4 tbox = make_float4(0.f, 0.f, 0.f, 0.f);
  if constexpr (f32) {
    if (use_far && warp_valid) tbox = *reinterpret_cast<const float4*>(group_rec<M>(gdata, tgroup));
  }
#pragma unroll 1
  for (int t0 = c0; t0 < c1; t0 += S) {
    const int cnt = min(S, c1 - t0);
    bool near = warp_valid;
    // far for this warp and left by pass 1: summed here through the group's
    // expansion (m2p2) or source by source (sbs) while the near warps work
    bool sbs = false, m2p2 = false;
    if constexpr (f32) {
      if (use_far && warp_valid) {
        near = !tile_is_far<M>(gdata, tgroup, t0 / kGroup);
        if constexpr (PART != 2) {
          if (!near) {
            m2p2 = tile_takes_m2p<M>(gdata, tgroup, t0 / kGroup);
            sbs = !m2p2;
          }
        }
      }
    }
    if (__syncthreads_or(near)) {
      load_tile(t0, cnt);
      __syncthreads();
      if constexpr (f32 && PART != 2) {
        if (m2p2) {
          work = true;
          m2p_tile<M, LO, HI, PART, TPC>(gdata, t0 / kGroup, tz1, tz2, tl1, tl2, acc_hi, acc_lo,
                                         slot);
          if (j < n) {
            n_m2p += 1;
            n_m2p_pairs += cnt;
          }
        }
      }
#pragma unroll 1
      for (int s = 0; s < cnt; ++s) {
        if (near || sbs) {
          const T* rs = tile + s * R;
          bool sfar = sbs;  // every source of a far tile is far from the warp's box
          if constexpr (f32) {
            if (use_far && near) sfar = point_is_far<M>(tbox, rs[0], rs[1]);
          }
          if (!sfar) {
            near_source<M, T, LO, HI, PART>(rs, t0 + s, j, tz1, tz2, tl1, tl2, acc);
          } else if constexpr (f32 && PART != 2) {
            float yr[NY], yi[NY];
#pragma unroll
            for (int b = 0; b < NY; ++b) {
              yr[b] = 0.f;
              yi[b] = 0.f;
            }
            far_source<M, LO, HI>(reinterpret_cast<const float*>(rs), tz1, tz2, tl1, tl2, yr,
                                  yi);
            fold_far<M, float, LO, HI>(yr, yi, reinterpret_cast<float*>(acc));
          }
          if (j < n) {
            if (sfar)
              ++n_far;
            else
              ++n_near;
          }
        }
        if constexpr (SYNC > 0) {
          if (s % SYNC == SYNC - 1 || s == cnt - 1) __syncthreads();  // CTA-uniform
        }
      }
      if constexpr (f32) {
        if (near || sbs) flush_sums<LO, HI, PART, TPC>(acc, acc_hi, acc_lo, slot);
      }
      work = work || near || sbs;
    }
  }
  if (LO == 1 && PART != 2 && counts != nullptr) {
    const unsigned wn = __reduce_add_sync(0xffffffffu, n_near);
    const unsigned wf = __reduce_add_sync(0xffffffffu, n_far);
    const unsigned we = __reduce_add_sync(0xffffffffu, n_m2p);
    const unsigned wp = __reduce_add_sync(0xffffffffu, n_m2p_pairs);
    if ((threadIdx.x & 31) == 0) {
      if (wn) atomicAdd(counts, (unsigned long long)wn);
      if (wf) atomicAdd(counts + 1, (unsigned long long)wf);
      if (we) atomicAdd(counts + 2, (unsigned long long)we);
      if (wp) atomicAdd(counts + 3, (unsigned long long)wp);
    }
  }
  if (j < n) {
    double* o = out + (size_t)PN::B0 * n + j;
    static_for<0, NBL>([&](auto bc) {
      constexpr int b = decltype(bc)::value;
      if constexpr (PC::in(b)) {
        double v = 0.0;
        if constexpr (f32) {
          constexpr int q = PC::slot(b) * TPC;
          if (work) v = (double)acc_hi[q + slot] + (double)acc_lo[q + slot];
        } else {
          v = acc[b];
        }
        o[(size_t)b * n] = v;
      }
    });
  }
}

// One context: grid (target tiles, source chunks) over n records.
// Layout of `partial`: [chunk][beta column][target] FP64.
template <int M, typename T, int LO, int HI, int PART, int TPC, int MINB, int SYNC>
__global__ void __launch_bounds__(TPC, MINB)
    pair_kernel(const T* __restrict__ rec, int n, int chunk_len, int S,
                const float* __restrict__ gdata, double* __restrict__ partial,
                unsigned long long* __restrict__ counts) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int NB = n_beta(M);
  const int c0 = blockIdx.y * chunk_len;
  const int c1 = min(n, c0 + chunk_len);
  pair_tile_work<M, T, LO, HI, PART, TPC, SYNC>(rec, n, blockIdx.x * TPC, c0, c1, S, gdata,
                                          partial + (size_t)blockIdx.y * NB * n, counts,
                                          smem_raw);
}

// Many independent instances of one order in one persistent launch: every
// CTA takes work items (instance, target tile, source chunk) from a shared
// counter until none is left.  Items are listed by the host, costliest first.
// The counter must be zero at launch (the caller clears it).  gdata (null: no
// far field) holds the group records of the whole batch (instances start on
// group boundaries).
template <int M, typename T, int LO, int HI, int PART, int TPC, int MINB, int SYNC>
__global__ void __launch_bounds__(TPC, MINB)
    pair_batch_kernel(const T* __restrict__ rec, const BatchInst* __restrict__ inst,
                      const int4* __restrict__ items, const int* __restrict__ n_items,
                      int* __restrict__ counter, int S, const float* __restrict__ gdata,
                      double* __restrict__ partial) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int item_s;
  constexpr int NB = n_beta(M);
  constexpr int R = rec_len<T>(M);
  const int total = *n_items;
#pragma unroll 1
  for (;;) {
    if (threadIdx.x == 0) item_s = atomicAdd(counter, 1);
    __syncthreads();
    const int it = item_s;
    __syncthreads();  // every thread has read item_s before it is overwritten
    if (it >= total) break;
    const int4 w = items[it];  // (instance, first target, chunk, -)
    const BatchInst ip = inst[w.x];
    const int c0 = w.z * ip.chunk_len;
    const int c1 = min(ip.n, c0 + ip.chunk_len);
    pair_tile_work<M, T, LO, HI, PART, TPC, SYNC>(rec + (size_t)ip.slot0 * R, ip.n, w.y, c0, c1, S,
                                            gdata ? group_rec<M>(gdata, ip.slot0 / kGroup)
                                                  : nullptr,
                                            partial + ip.part_off + (size_t)w.z * NB * ip.n,
                                            nullptr, smem_raw);
  }
}

template <int M, typename T, int LO, int HI, int PART, int TPC>
size_t pair_smem_bytes(int S) {  // shared memory of one CTA
  size_t b = (size_t)S * rec_len<T>(M) * sizeof(T);
  if (std::is_same<T, float>::value)
    b += 2 * (size_t)PartCols<LO, HI, PART>::NS * TPC * sizeof(float);
  return b;
}

}  // namespace mmvm
