// Registry of compiled all-pairs kernel variants, one per (order, precision).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

namespace mmvm {

struct PairEntry {
  int M = -1;
  int precision = 0;      // 0: FP64, 1: FP32
  int tpc = 0;            // targets per CTA
  int g = 1;              // threads (output slices) per target
  int rec_len = 0;        // record length in elements
  int elem_bytes = 0;     // sizeof(T)
  size_t (*smem)(int S) = nullptr;
  cudaError_t (*prepare)(int S) = nullptr;   // set the dynamic shared-memory limit
  cudaError_t (*launch)(const void* rec, int n, int chunks, int S, double* partial,
                        cudaStream_t st) = nullptr;
  cudaError_t (*occupancy)(int S, int* blocks_per_sm) = nullptr;
};

// nullptr-like entry (M == -1) if the variant is not compiled.
PairEntry pair_entry(int M, int precision);

}  // namespace mmvm
