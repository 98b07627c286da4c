// Dispatch from (order, precision, variant) to the compiled slice kernels.
#include <algorithm>

#include "pair_registry.h"
#include "common.cuh"

namespace mmvm {

SliceEntry pair_slice_m0_p0_v0_s0();
SliceEntry pair_slice_m0_p1_v0_s0();
SliceEntry pair_slice_m1_p0_v0_s0();
SliceEntry pair_slice_m1_p1_v0_s0();
SliceEntry pair_slice_m2_p0_v0_s0();
SliceEntry pair_slice_m2_p1_v0_s0();
SliceEntry pair_slice_m3_p0_v0_s0();
SliceEntry pair_slice_m3_p1_v0_s0();
SliceEntry pair_slice_m4_p0_v0_s0();
SliceEntry pair_slice_m4_p0_v0_s1();
SliceEntry pair_slice_m4_p1_v0_s0();
SliceEntry pair_slice_m4_p1_v1_s0();
SliceEntry pair_slice_m4_p1_v2_s0();
SliceEntry pair_slice_m4_p1_v2_s1();
SliceEntry pair_slice_m5_p0_v0_s0();
SliceEntry pair_slice_m5_p0_v0_s1();
SliceEntry pair_slice_m5_p1_v0_s0();
SliceEntry pair_slice_m5_p1_v1_s0();
SliceEntry pair_slice_m5_p1_v1_s1();
SliceEntry pair_slice_m5_p1_v2_s0();
SliceEntry pair_slice_m5_p1_v2_s1();
SliceEntry pair_slice_m6_p0_v0_s0();
SliceEntry pair_slice_m6_p0_v0_s1();
SliceEntry pair_slice_m6_p0_v0_s2();
SliceEntry pair_slice_m6_p1_v0_s0();
SliceEntry pair_slice_m6_p1_v1_s0();
SliceEntry pair_slice_m6_p1_v1_s1();
SliceEntry pair_slice_m6_p1_v2_s0();
SliceEntry pair_slice_m6_p1_v2_s1();
SliceEntry pair_slice_m6_p1_v2_s2();
SliceEntry pair_slice_m6_p1_v3_s0();
SliceEntry pair_slice_m6_p1_v3_s1();
SliceEntry pair_slice_m7_p0_v0_s0();
SliceEntry pair_slice_m7_p0_v0_s1();
SliceEntry pair_slice_m7_p0_v0_s2();
SliceEntry pair_slice_m7_p0_v0_s3();
SliceEntry pair_slice_m7_p1_v0_s0();
SliceEntry pair_slice_m7_p1_v0_s1();
SliceEntry pair_slice_m7_p1_v1_s0();
SliceEntry pair_slice_m7_p1_v1_s1();
SliceEntry pair_slice_m7_p1_v1_s2();
SliceEntry pair_slice_m8_p0_v0_s0();
SliceEntry pair_slice_m8_p0_v0_s1();
SliceEntry pair_slice_m8_p0_v0_s2();
SliceEntry pair_slice_m8_p0_v0_s3();
SliceEntry pair_slice_m8_p1_v0_s0();
SliceEntry pair_slice_m8_p1_v0_s1();
SliceEntry pair_slice_m8_p1_v0_s2();
SliceEntry pair_slice_m8_p1_v1_s0();
SliceEntry pair_slice_m8_p1_v1_s1();
SliceEntry pair_slice_m8_p1_v1_s2();
SliceEntry pair_slice_m8_p1_v1_s3();
SliceEntry pair_slice_m8_p1_v2_s0();
SliceEntry pair_slice_m8_p1_v2_s1();
SliceEntry pair_slice_m8_p1_v2_s2();
SliceEntry pair_slice_m8_p1_v2_s3();

int pair_variant_count(int M, int precision) {
  if (M < 0 || M > 8 || (precision != 0 && precision != 1)) return 0;
  return n_variants(M, precision);
}

PairEntry pair_entry(int M, int precision, int v) {
  PairEntry e;
  if (v < 0 || v >= pair_variant_count(M, precision)) return e;
  const VariantSpec sp = variant_spec(M, precision, v);
  switch ((M * 2 + precision) * kMaxVariants + v) {
    case 0: e.slices[0] = pair_slice_m0_p0_v0_s0(); break;
    case 4: e.slices[0] = pair_slice_m0_p1_v0_s0(); break;
    case 8: e.slices[0] = pair_slice_m1_p0_v0_s0(); break;
    case 12: e.slices[0] = pair_slice_m1_p1_v0_s0(); break;
    case 16: e.slices[0] = pair_slice_m2_p0_v0_s0(); break;
    case 20: e.slices[0] = pair_slice_m2_p1_v0_s0(); break;
    case 24: e.slices[0] = pair_slice_m3_p0_v0_s0(); break;
    case 28: e.slices[0] = pair_slice_m3_p1_v0_s0(); break;
    case 32: e.slices[0] = pair_slice_m4_p0_v0_s0(); e.slices[1] = pair_slice_m4_p0_v0_s1(); break;
    case 36: e.slices[0] = pair_slice_m4_p1_v0_s0(); break;
    case 37: e.slices[0] = pair_slice_m4_p1_v1_s0(); break;
    case 38: e.slices[0] = pair_slice_m4_p1_v2_s0(); e.slices[1] = pair_slice_m4_p1_v2_s1(); break;
    case 40: e.slices[0] = pair_slice_m5_p0_v0_s0(); e.slices[1] = pair_slice_m5_p0_v0_s1(); break;
    case 44: e.slices[0] = pair_slice_m5_p1_v0_s0(); break;
    case 45: e.slices[0] = pair_slice_m5_p1_v1_s0(); e.slices[1] = pair_slice_m5_p1_v1_s1(); break;
    case 46: e.slices[0] = pair_slice_m5_p1_v2_s0(); e.slices[1] = pair_slice_m5_p1_v2_s1(); break;
    case 48: e.slices[0] = pair_slice_m6_p0_v0_s0(); e.slices[1] = pair_slice_m6_p0_v0_s1(); e.slices[2] = pair_slice_m6_p0_v0_s2(); break;
    case 52: e.slices[0] = pair_slice_m6_p1_v0_s0(); break;
    case 53: e.slices[0] = pair_slice_m6_p1_v1_s0(); e.slices[1] = pair_slice_m6_p1_v1_s1(); break;
    case 54: e.slices[0] = pair_slice_m6_p1_v2_s0(); e.slices[1] = pair_slice_m6_p1_v2_s1(); e.slices[2] = pair_slice_m6_p1_v2_s2(); break;
    case 55: e.slices[0] = pair_slice_m6_p1_v3_s0(); e.slices[1] = pair_slice_m6_p1_v3_s1(); break;
    case 56: e.slices[0] = pair_slice_m7_p0_v0_s0(); e.slices[1] = pair_slice_m7_p0_v0_s1(); e.slices[2] = pair_slice_m7_p0_v0_s2(); e.slices[3] = pair_slice_m7_p0_v0_s3(); break;
    case 60: e.slices[0] = pair_slice_m7_p1_v0_s0(); e.slices[1] = pair_slice_m7_p1_v0_s1(); break;
    case 61: e.slices[0] = pair_slice_m7_p1_v1_s0(); e.slices[1] = pair_slice_m7_p1_v1_s1(); e.slices[2] = pair_slice_m7_p1_v1_s2(); break;
    case 64: e.slices[0] = pair_slice_m8_p0_v0_s0(); e.slices[1] = pair_slice_m8_p0_v0_s1(); e.slices[2] = pair_slice_m8_p0_v0_s2(); e.slices[3] = pair_slice_m8_p0_v0_s3(); break;
    case 68: e.slices[0] = pair_slice_m8_p1_v0_s0(); e.slices[1] = pair_slice_m8_p1_v0_s1(); e.slices[2] = pair_slice_m8_p1_v0_s2(); break;
    case 69: e.slices[0] = pair_slice_m8_p1_v1_s0(); e.slices[1] = pair_slice_m8_p1_v1_s1(); e.slices[2] = pair_slice_m8_p1_v1_s2(); e.slices[3] = pair_slice_m8_p1_v1_s3(); break;
    case 70: e.slices[0] = pair_slice_m8_p1_v2_s0(); e.slices[1] = pair_slice_m8_p1_v2_s1(); e.slices[2] = pair_slice_m8_p1_v2_s2(); e.slices[3] = pair_slice_m8_p1_v2_s3(); break;
    default: return e;
  }
  e.M = M;
  e.precision = precision;
  e.variant = v;
  e.tpc = sp.TPC;
  e.minb = sp.MINB;
  e.sync = sp.SYNC;
  e.nslices = sp.nslices;
  e.rec_len = precision == 1 ? rec_len<float>(M) : rec_len<double>(M);
  e.elem_bytes = precision == 1 ? 4 : 8;
  return e;
}

cudaError_t pair_prepare(const PairEntry& e, int S) {
  for (int s = 0; s < e.nslices; ++s) {
    cudaError_t r = e.slices[s].prepare(S);
    if (r != cudaSuccess) return r;
  }
  return cudaSuccess;
}

int pair_occupancy(const PairEntry& e, int S) {
  int best = 1 << 30;
  for (int s = 0; s < e.nslices; ++s) {
    int b = 0;
    if (e.slices[s].occupancy(S, &b) != cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
    best = std::min(best, b);
  }
  return e.nslices ? best : 0;
}

cudaError_t pair_launch(const PairEntry& e, const void* rec, int n, int chunks, int S,
                        const void* gbox, double* partial, int grid_y_limit, cudaStream_t st,
                        unsigned long long* counts) {
  // chunks start on group boundaries so every source tile is one group
  const int chunk_len = round_up((n + chunks - 1) / chunks, S);
  const int gy = (grid_y_limit > 0 && chunks > grid_y_limit) ? grid_y_limit : chunks;
  for (int s = 0; s < e.nslices; ++s) {
    cudaError_t r = e.slices[s].launch(rec, n, chunk_len, gy, S, gbox, partial, counts, st);
    if (r != cudaSuccess) return r;
  }
  return cudaSuccess;
}

int pair_batch_occupancy(const PairEntry& e, int S) {
  int best = 1 << 30;
  for (int s = 0; s < e.nslices; ++s) {
    int b = 0;
    if (e.slices[s].occupancy_batch(S, &b) != cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
    best = std::min(best, b);
  }
  return e.nslices ? best : 0;
}

cudaError_t pair_launch_batch(const PairEntry& e, const void* rec, const BatchInst* inst,
                              const int4* items, const int* n_items, int* counters, int grid,
                              int S, const void* gbox, double* partial, cudaStream_t st) {
  for (int s = 0; s < e.nslices; ++s) {
    cudaError_t r = e.slices[s].launch_batch(rec, inst, items, n_items, counters + s, grid, S,
                                             gbox, partial, st);
    if (r != cudaSuccess) return r;
  }
  return cudaSuccess;
}

}  // namespace mmvm
