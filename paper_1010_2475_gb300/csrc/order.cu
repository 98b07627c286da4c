// Spatial ordering of the particles for the all-pairs kernel: consecutive
// positions are close in space, so the 32-particle groups (source tiles and
// target warps) have small bounding boxes and the far-field test of the pair
// kernel can take the point-vortex jet for whole tiles.  Morton (Z-order)
// keys of the centres quantised to 16 bits per axis over the bounding box,
// sorted with a stable radix sort (ties keep the index order), so the order
// is deterministic.
#include <cub/device/device_radix_sort.cuh>

#include <algorithm>

#include "common.cuh"
#include "particle_kernels.h"

namespace mmvm {

namespace {

__device__ __forceinline__ unsigned spread16(unsigned v) {
  v &= 0xffffu;
  v = (v | (v << 8)) & 0x00ff00ffu;
  v = (v | (v << 4)) & 0x0f0f0f0fu;
  v = (v | (v << 2)) & 0x33333333u;
  v = (v | (v << 1)) & 0x55555555u;
  return v;
}

// One block: bounding box of all centres -> box[0..3] = (min1, min2, max1, max2).
__global__ void bbox_kernel(int n, const double* __restrict__ x, double* __restrict__ box) {
  __shared__ double red[4][32];
  double lo1 = 1e300, lo2 = 1e300, hi1 = -1e300, hi2 = -1e300;
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    const double a = x[2 * j], b = x[2 * j + 1];
    lo1 = fmin(lo1, a);
    hi1 = fmax(hi1, a);
    lo2 = fmin(lo2, b);
    hi2 = fmax(hi2, b);
  }
  for (int o = 16; o > 0; o >>= 1) {
    lo1 = fmin(lo1, __shfl_xor_sync(0xffffffffu, lo1, o));
    hi1 = fmax(hi1, __shfl_xor_sync(0xffffffffu, hi1, o));
    lo2 = fmin(lo2, __shfl_xor_sync(0xffffffffu, lo2, o));
    hi2 = fmax(hi2, __shfl_xor_sync(0xffffffffu, hi2, o));
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) {
    red[0][w] = lo1;
    red[1][w] = lo2;
    red[2][w] = hi1;
    red[3][w] = hi2;
  }
  __syncthreads();
  if (w == 0) {
    const int nw = blockDim.x >> 5;
    lo1 = l < nw ? red[0][l] : 1e300;
    lo2 = l < nw ? red[1][l] : 1e300;
    hi1 = l < nw ? red[2][l] : -1e300;
    hi2 = l < nw ? red[3][l] : -1e300;
    for (int o = 16; o > 0; o >>= 1) {
      lo1 = fmin(lo1, __shfl_xor_sync(0xffffffffu, lo1, o));
      hi1 = fmax(hi1, __shfl_xor_sync(0xffffffffu, hi1, o));
      lo2 = fmin(lo2, __shfl_xor_sync(0xffffffffu, lo2, o));
      hi2 = fmax(hi2, __shfl_xor_sync(0xffffffffu, hi2, o));
    }
    if (l == 0) {
      box[0] = lo1;
      box[1] = lo2;
      box[2] = hi1;
      box[3] = hi2;
    }
  }
}

__global__ void morton_kernel(int n, const double* __restrict__ x, const double* __restrict__ box,
                              unsigned* __restrict__ keys, int* __restrict__ idx) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const double s1 = fmax(box[2] - box[0], 1e-300), s2 = fmax(box[3] - box[1], 1e-300);
  const double q1 = fmin(fmax((x[2 * j] - box[0]) / s1, 0.0), 1.0) * 65535.0;
  const double q2 = fmin(fmax((x[2 * j + 1] - box[1]) / s2, 0.0), 1.0) * 65535.0;
  keys[j] = spread16((unsigned)q1) | (spread16((unsigned)q2) << 1);
  idx[j] = j;
}

// scratch layout: [box 4 doubles][keys_in n][keys_out n][idx_in n][cub temp]
size_t cub_bytes(int n) {
  size_t b = 0;
  cub::DeviceRadixSort::SortPairs(nullptr, b, (const unsigned*)nullptr, (unsigned*)nullptr,
                                  (const int*)nullptr, (int*)nullptr, n);
  return b;
}

// Batches: one block per instance -> bounding box of its step-start centres,
// ibox[i] = (min1, min2, max1, max2).
__global__ void bbox_batch_kernel(const BatchInst* __restrict__ inst, const int* __restrict__ n_inst,
                                  double4* __restrict__ ibox) {
  __shared__ double red[4][32];
  const int total = *n_inst;
  for (int i = blockIdx.x; i < total; i += gridDim.x) {
    const BatchInst& I = inst[i];
    double lo1 = 1e300, lo2 = 1e300, hi1 = -1e300, hi2 = -1e300;
    for (int j = threadIdx.x; j < I.n; j += blockDim.x) {
      const double a = I.state[2 * j], b = I.state[2 * j + 1];
      lo1 = fmin(lo1, a);
      hi1 = fmax(hi1, a);
      lo2 = fmin(lo2, b);
      hi2 = fmax(hi2, b);
    }
    for (int o = 16; o > 0; o >>= 1) {
      lo1 = fmin(lo1, __shfl_xor_sync(0xffffffffu, lo1, o));
      hi1 = fmax(hi1, __shfl_xor_sync(0xffffffffu, hi1, o));
      lo2 = fmin(lo2, __shfl_xor_sync(0xffffffffu, lo2, o));
      hi2 = fmax(hi2, __shfl_xor_sync(0xffffffffu, hi2, o));
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) {
      red[0][w] = lo1;
      red[1][w] = lo2;
      red[2][w] = hi1;
      red[3][w] = hi2;
    }
    __syncthreads();
    if (w == 0) {
      const int nw = blockDim.x >> 5;
      lo1 = l < nw ? red[0][l] : 1e300;
      lo2 = l < nw ? red[1][l] : 1e300;
      hi1 = l < nw ? red[2][l] : -1e300;
      hi2 = l < nw ? red[3][l] : -1e300;
      for (int o = 16; o > 0; o >>= 1) {
        lo1 = fmin(lo1, __shfl_xor_sync(0xffffffffu, lo1, o));
        hi1 = fmax(hi1, __shfl_xor_sync(0xffffffffu, hi1, o));
        lo2 = fmin(lo2, __shfl_xor_sync(0xffffffffu, lo2, o));
        hi2 = fmax(hi2, __shfl_xor_sync(0xffffffffu, hi2, o));
      }
      if (l == 0) ibox[i] = make_double4(lo1, lo2, hi1, hi2);
    }
    __syncthreads();  // red is reused by the next instance
  }
}

// Key of slot p: (instance << 32) | Morton code in the instance's own box;
// padding slots of an instance sort after its particles, slots past the
// batch after everything.
__global__ void morton_batch_kernel(int slot_cap, const int* __restrict__ n_slots,
                                    const BatchInst* __restrict__ inst,
                                    const int* __restrict__ slot_inst,
                                    const double4* __restrict__ ibox,
                                    unsigned long long* __restrict__ keys, int* __restrict__ idx) {
  const int total = *n_slots;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < slot_cap; p += gridDim.x * blockDim.x) {
    unsigned long long key = ~0ull;
    if (p < total) {
      const int i = slot_inst[p / kGroup];
      const BatchInst& I = inst[i];
      const int j = p - I.slot0;
      unsigned code = 0xffffffffu;
      if (j < I.n) {
        const double4 b = ibox[i];
        const double s1 = fmax(b.z - b.x, 1e-300), s2 = fmax(b.w - b.y, 1e-300);
        const double q1 = fmin(fmax((I.state[2 * j] - b.x) / s1, 0.0), 1.0) * 65535.0;
        const double q2 = fmin(fmax((I.state[2 * j + 1] - b.y) / s2, 0.0), 1.0) * 65535.0;
        code = spread16((unsigned)q1) | (spread16((unsigned)q2) << 1);
      }
      key = ((unsigned long long)i << 32) | code;
    }
    keys[p] = key;
    idx[p] = p;
  }
}

// Sorted slot p of instance i holds its particle perm_local[p] (local index).
__global__ void perm_batch_kernel(const int* __restrict__ n_slots, const BatchInst* __restrict__ inst,
                                  const int* __restrict__ slot_inst, const int* __restrict__ sorted,
                                  int* __restrict__ perm_local) {
  const int total = *n_slots;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < total; p += gridDim.x * blockDim.x) {
    const BatchInst& I = inst[slot_inst[p / kGroup]];
    perm_local[p] = (p - I.slot0 < I.n) ? sorted[p] - I.slot0 : 0;
  }
}

size_t cub_bytes64(int n) {
  size_t b = 0;
  cub::DeviceRadixSort::SortPairs(nullptr, b, (const unsigned long long*)nullptr,
                                  (unsigned long long*)nullptr, (const int*)nullptr, (int*)nullptr,
                                  n);
  return b;
}

}  // namespace

size_t batch_order_temp_bytes(int slot_cap) { return cub_bytes64(slot_cap) + 256; }

cudaError_t launch_batch_order(int slot_cap, const int* n_slots, const BatchInst* inst,
                               const int* n_inst, int inst_cap, const int* slot_inst, void* ibox,
                               unsigned long long* kin, unsigned long long* kout, int* iin,
                               int* iout, void* temp, size_t temp_bytes, int* perm_local,
                               cudaStream_t st) {
  size_t cb = cub_bytes64(slot_cap);
  if (cb > temp_bytes) return cudaErrorInvalidValue;
  bbox_batch_kernel<<<std::max(1, std::min(inst_cap, 1024)), 256, 0, st>>>(
      inst, n_inst, static_cast<double4*>(ibox));
  const int blocks = std::max(1, std::min((slot_cap + 255) / 256, 4096));
  morton_batch_kernel<<<blocks, 256, 0, st>>>(slot_cap, n_slots, inst, slot_inst,
                                              static_cast<const double4*>(ibox), kin, iin);
  cudaError_t e = cub::DeviceRadixSort::SortPairs(temp, cb, kin, kout, iin, iout, slot_cap, 0, 64,
                                                  st);
  if (e != cudaSuccess) return e;
  perm_batch_kernel<<<blocks, 256, 0, st>>>(n_slots, inst, slot_inst, iout, perm_local);
  return cudaGetLastError();
}

size_t spatial_order_temp_bytes(int n) {
  return 64 + (size_t)3 * ((size_t)n * 4 + 256) + cub_bytes(n) + 256;
}

cudaError_t launch_spatial_order(int n, const double* x, void* temp, size_t temp_bytes,
                                 int* perm, cudaStream_t st) {
  auto align = [](size_t v) { return (v + 255) & ~(size_t)255; };
  char* base = static_cast<char*>(temp);
  double* box = reinterpret_cast<double*>(base);
  size_t off = 64;
  unsigned* kin = reinterpret_cast<unsigned*>(base + off);
  off = align(off + (size_t)n * 4);
  unsigned* kout = reinterpret_cast<unsigned*>(base + off);
  off = align(off + (size_t)n * 4);
  int* iin = reinterpret_cast<int*>(base + off);
  off = align(off + (size_t)n * 4);
  size_t cb = cub_bytes(n);
  if (off + cb > temp_bytes) return cudaErrorInvalidValue;
  bbox_kernel<<<1, 1024, 0, st>>>(n, x, box);
  morton_kernel<<<(n + 255) / 256, 256, 0, st>>>(n, x, box, kin, iin);
  return cub::DeviceRadixSort::SortPairs(base + off, cb, kin, kout, iin, perm, n, 0, 32, st);
}

}  // namespace mmvm
