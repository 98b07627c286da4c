// Launch wrapper of the all-pairs kernel: one thread per (target, output
// slice), source records staged through shared memory in tiles of S, FP32
// partial sums carried across tiles as (hi, lo) float pairs (TwoSum), and the
// per-(source chunk, target) result written as FP64.
#pragma once

#include "common.cuh"
#include "pair_kernel.cuh"

namespace mmvm {

struct PairLaunch {
  int targets_per_cta;  // TPC
  int tile;             // S sources per shared-memory tile
  int chunks;           // source chunks (grid.y)
};

// Layout of `partial`: [chunk][beta column][target] FP64 (coalesced writes).
// acc points at a register array of at least NBL entries; every index used
// below is a compile-time constant after inlining, so it stays in registers.

// Accumulate `cnt` staged sources into this slice's registers, then (FP32)
// fold the tile's sums into the shared-memory (hi, lo) pairs.
template <int M, typename T, int G, int g, int TPC>
__device__ __forceinline__ void pair_tile(const T* tile, int cnt, int t0, int j, T tz1, T tz2,
                                          T tl1, T tl2, T* acc, float* acc_hi, float* acc_lo,
                                          int slot) {
  using PN = PairNear<M, T, G, g>;
  constexpr int K = n_moments(M);
  constexpr int NBL = PN::NBL;
  constexpr int R = rec_len<T>(M);
  constexpr int HDR = Rec<T>::HDR;
  constexpr bool f32 = std::is_same<T, float>::value;
  T (&accr)[NBL] = *reinterpret_cast<T(*)[NBL]>(acc);
#pragma unroll 1
  for (int s = 0; s < cnt; ++s) {
    const T* r = tile + s * R;
    T a[K];
#pragma unroll
    for (int m = 0; m < K; ++m) a[m] = r[HDR + m];
    T b1, b2, l1 = T(0), l2 = T(0);
    if constexpr (f32) {
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
    if (t0 + s == j) {  // self pair: excluded here, added exactly by the finish
      b1 = T(1e15);
      b2 = T(0);
      l1 = T(0);
      l2 = T(0);
      wm = T(0);
    }
    PN::run(b1, b2, l1, l2, wm, a, accr);
  }
  if constexpr (f32) {
#pragma unroll
    for (int b = 0; b < NBL; ++b) {
      const int idx = (PN::B0 + b) * TPC + slot;
      const float hi = acc_hi[idx];
      const float sum = hi + accr[b];
      const float bp = sum - hi;
      const float err = (hi - (sum - bp)) + (accr[b] - bp);
      acc_hi[idx] = sum;
      acc_lo[idx] += err;
      accr[b] = 0.f;
    }
  }
}

// Warp-uniform dispatch to output slice gg (forced inline, no lambda).
template <int M, typename T, int G, int TPC, int gg>
__device__ __forceinline__ void pair_tile_dispatch(int g, const T* tile, int cnt, int t0, int j,
                                                   T tz1, T tz2, T tl1, T tl2, T* acc,
                                                   float* acc_hi, float* acc_lo, int slot) {
  if (g == gg) {
    pair_tile<M, T, G, gg, TPC>(tile, cnt, t0, j, tz1, tz2, tl1, tl2, acc, acc_hi, acc_lo, slot);
  } else if constexpr (gg + 1 < G) {
    pair_tile_dispatch<M, T, G, TPC, gg + 1>(g, tile, cnt, t0, j, tz1, tz2, tl1, tl2, acc,
                                             acc_hi, acc_lo, slot);
  }
}

template <int M, typename T, int G, int TPC, int gg>
__device__ __forceinline__ void pair_store_dispatch(int g, int n, int j, const T* acc,
                                                    const float* acc_hi, const float* acc_lo,
                                                    int slot, double* __restrict__ out) {
  using PN = PairNear<M, T, G, gg>;
  if (g == gg) {
#pragma unroll
    for (int b = 0; b < PN::NBL; ++b) {
      double v;
      if constexpr (std::is_same<T, float>::value) {
        const int idx = (PN::B0 + b) * TPC + slot;
        v = (double)acc_hi[idx] + (double)acc_lo[idx];
      } else {
        v = acc[b];
      }
      out[(size_t)(PN::B0 + b) * n + j] = v;
    }
  } else if constexpr (gg + 1 < G) {
    pair_store_dispatch<M, T, G, TPC, gg + 1>(g, n, j, acc, acc_hi, acc_lo, slot, out);
  }
}

template <int M, typename T, int G, int TPC>
__global__ void __launch_bounds__(TPC * G) pair_kernel(const T* __restrict__ rec, int n,
                                                       int chunk_len, int S,
                                                       double* __restrict__ partial) {
  constexpr int R = rec_len<T>(M);
  constexpr int NB = n_beta(M);
  constexpr int NBLMAX = (NB + G - 1) / G;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* tile = reinterpret_cast<T*>(smem_raw);
  float* acc_hi = reinterpret_cast<float*>(tile + (size_t)S * R);
  float* acc_lo = acc_hi + NB * TPC;
  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const int g = warp % G;
  const int slot = (warp / G) * 32 + lane;
  const int j = blockIdx.x * TPC + slot;
  const int c0 = blockIdx.y * chunk_len;
  const int c1 = min(n, c0 + chunk_len);
  T tz1, tz2, tl1 = T(0), tl2 = T(0);
  if (j < n) {
    const T* r = rec + (size_t)j * R;
    tz1 = r[0];
    tz2 = r[1];
    if constexpr (std::is_same<T, float>::value) {
      tl1 = r[2];
      tl2 = r[3];
    }
  } else {
    tz1 = T(3e15);
    tz2 = T(3e15);
  }
  T acc[NBLMAX];
#pragma unroll
  for (int b = 0; b < NBLMAX; ++b) acc[b] = T(0);
  if constexpr (std::is_same<T, float>::value) {
    for (int i = threadIdx.x; i < 2 * NB * TPC; i += blockDim.x) acc_hi[i] = 0.f;
  }
#pragma unroll 1
  for (int t0 = c0; t0 < c1; t0 += S) {
    const int cnt = min(S, c1 - t0);
    __syncthreads();
    {
      // cooperative 16-byte copy of cnt records into the tile
      const int nvec = cnt * R * (int)sizeof(T) / 16;
      const int4* src = reinterpret_cast<const int4*>(rec + (size_t)t0 * R);
      int4* dst = reinterpret_cast<int4*>(tile);
      for (int i = threadIdx.x; i < nvec; i += blockDim.x) dst[i] = __ldg(src + i);
    }
    __syncthreads();
    pair_tile_dispatch<M, T, G, TPC, 0>(g, tile, cnt, t0, j, tz1, tz2, tl1, tl2, acc, acc_hi,
                                        acc_lo, slot);
  }
  if (j < n) {
    pair_store_dispatch<M, T, G, TPC, 0>(g, n, j, acc, acc_hi, acc_lo, slot,
                                         partial + (size_t)blockIdx.y * NB * n);
  }
}

template <int M, typename T, int G, int TPC>
size_t pair_smem_bytes(int S) {
  size_t b = (size_t)S * rec_len<T>(M) * sizeof(T);
  if (std::is_same<T, float>::value) b += 2 * (size_t)n_beta(M) * TPC * sizeof(float);
  return b;
}

template <int M, typename T, int G, int TPC>
cudaError_t launch_pair_t(const T* rec, int n, int chunks, int S, double* partial,
                          cudaStream_t st) {
  const int chunk_len = (n + chunks - 1) / chunks;
  const size_t smem = pair_smem_bytes<M, T, G, TPC>(S);
  auto kern = pair_kernel<M, T, G, TPC>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid((n + TPC - 1) / TPC, chunks);
  kern<<<grid, TPC * G, smem, st>>>(rec, n, chunk_len, S, partial);
  return cudaGetLastError();
}

}  // namespace mmvm
