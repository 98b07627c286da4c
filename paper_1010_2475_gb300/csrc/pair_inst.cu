// One compiled variant of the all-pairs kernel.  Built once per (order,
// precision) with -DMMVM_INST_M=<order> -DMMVM_INST_PREC=<0|1> so the
// variants compile in parallel.
#include "pair_launch.cuh"
#include "pair_registry.h"

#ifndef MMVM_INST_M
#error "MMVM_INST_M must be defined"
#endif
#ifndef MMVM_INST_PREC
#error "MMVM_INST_PREC must be defined"
#endif

namespace mmvm {

namespace {
constexpr int kM = MMVM_INST_M;
using T = std::conditional_t<MMVM_INST_PREC == 1, float, double>;
// Output slices per target (G) and targets per CTA: chosen so the per-thread
// accumulators and one jet order fit in registers without spilling.
constexpr int kG = (MMVM_INST_PREC == 1) ? (kM <= 6 ? 1 : 2)
                                         : (kM <= 3 ? 1 : (kM <= 6 ? 2 : 4));
constexpr int kTPC = (MMVM_INST_PREC == 1) ? (kG == 1 ? 128 : 64) : 32;

size_t smem_fn(int S) { return pair_smem_bytes<kM, T, kG, kTPC>(S); }
cudaError_t prepare_fn(int S) {
  return cudaFuncSetAttribute(pair_kernel<kM, T, kG, kTPC>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_fn(S));
}
cudaError_t launch_fn(const void* rec, int n, int chunks, int S, double* partial,
                      cudaStream_t st) {
  const int chunk_len = (n + chunks - 1) / chunks;
  dim3 grid((n + kTPC - 1) / kTPC, chunks);
  pair_kernel<kM, T, kG, kTPC><<<grid, kTPC * kG, smem_fn(S), st>>>(
      static_cast<const T*>(rec), n, chunk_len, S, partial);
  return cudaGetLastError();
}
cudaError_t occ_fn(int S, int* blocks) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, pair_kernel<kM, T, kG, kTPC>,
                                                       kTPC * kG, smem_fn(S));
}
}  // namespace

#define MMVM_CAT3(a, b, c) a##b##c
#define MMVM_ENTRY_NAME(m, p) MMVM_CAT3(pair_entry_m, m, _p##p)
#define MMVM_ENTRY(m, p) MMVM_ENTRY_NAME(m, p)

PairEntry MMVM_ENTRY(MMVM_INST_M, MMVM_INST_PREC)() {
  PairEntry e;
  e.M = kM;
  e.precision = MMVM_INST_PREC;
  e.tpc = kTPC;
  e.g = kG;
  e.rec_len = rec_len<T>(kM);
  e.elem_bytes = (int)sizeof(T);
  e.smem = smem_fn;
  e.prepare = prepare_fn;
  e.launch = launch_fn;
  e.occupancy = occ_fn;
  return e;
}

}  // namespace mmvm
