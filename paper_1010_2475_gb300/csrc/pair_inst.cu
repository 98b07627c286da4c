// One order slice of one variant of the all-pairs kernel.  Built once per
// (order, precision, variant, slice) with -DMMVM_INST_M, -DMMVM_INST_PREC,
// -DMMVM_INST_V and -DMMVM_INST_S so the kernels compile in parallel.
#include "pair_launch.cuh"
#include "pair_registry.h"
#include "pair_variants.h"

#if !defined(MMVM_INST_M) || !defined(MMVM_INST_PREC) || !defined(MMVM_INST_V) || \
    !defined(MMVM_INST_S)
#error "MMVM_INST_M, MMVM_INST_PREC, MMVM_INST_V and MMVM_INST_S must be defined"
#endif

namespace mmvm {

namespace {
constexpr int kM = MMVM_INST_M;
using T = std::conditional_t<MMVM_INST_PREC == 1, float, double>;
constexpr VariantSpec kSpec = variant_spec(kM, MMVM_INST_PREC, MMVM_INST_V);
static_assert(MMVM_INST_S < kSpec.nslices, "slice index out of range");
constexpr int kLO = kSpec.s[MMVM_INST_S].lo;
constexpr int kHI = kSpec.s[MMVM_INST_S].hi;
constexpr int kPART = kSpec.s[MMVM_INST_S].part;
constexpr int kTPC = kSpec.s[MMVM_INST_S].tpc ? kSpec.s[MMVM_INST_S].tpc : kSpec.TPC;
constexpr int kMINB = kSpec.s[MMVM_INST_S].minb ? kSpec.s[MMVM_INST_S].minb : kSpec.MINB;
constexpr int kSYNC = kSpec.SYNC;
static_assert(kTPC % 32 == 0, "targets per CTA must be whole warps");
#define MMVM_KERNEL pair_kernel<kM, T, kLO, kHI, kPART, kTPC, kMINB, kSYNC>
#define MMVM_BATCH_KERNEL pair_batch_kernel<kM, T, kLO, kHI, kPART, kTPC, kMINB, kSYNC>

size_t smem_fn(int S) { return pair_smem_bytes<kM, T, kLO, kHI, kPART, kTPC>(S); }
cudaError_t prepare_fn(int S) {
  cudaError_t e = cudaFuncSetAttribute(MMVM_KERNEL, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem_fn(S));
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(MMVM_BATCH_KERNEL, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)smem_fn(S));
}
cudaError_t launch_batch_fn(const void* rec, const BatchInst* inst, const int4* items,
                            const int* n_items, int* counter, int grid, int S, const void* gbox,
                            double* partial, cudaStream_t st) {
  MMVM_BATCH_KERNEL<<<grid, kTPC, smem_fn(S), st>>>(static_cast<const T*>(rec), inst, items,
                                                    n_items, counter, S,
                                                    static_cast<const float*>(gbox), partial);
  return cudaGetLastError();
}
cudaError_t occ_batch_fn(int S, int* blocks) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, MMVM_BATCH_KERNEL, kTPC,
                                                       smem_fn(S));
}
cudaError_t launch_fn(const void* rec, int n, int chunk_len, int gy, int S, const void* gbox,
                      double* partial, unsigned long long* counts, cudaStream_t st) {
  dim3 grid((n + kTPC - 1) / kTPC, gy);
  MMVM_KERNEL<<<grid, kTPC, smem_fn(S), st>>>(static_cast<const T*>(rec), n, chunk_len, S,
                                              static_cast<const float*>(gbox), partial, counts);
  return cudaGetLastError();
}
cudaError_t occ_fn(int S, int* blocks) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, MMVM_KERNEL, kTPC, smem_fn(S));
}
}  // namespace

#define MMVM_CAT5(a, b, c, d, e) a##b##c##d##e
#define MMVM_SLICE_NAME(m, p, v, s) MMVM_CAT5(pair_slice_m, m, _p##p, _v##v, _s##s)
#define MMVM_SLICE(m, p, v, s) MMVM_SLICE_NAME(m, p, v, s)

SliceEntry MMVM_SLICE(MMVM_INST_M, MMVM_INST_PREC, MMVM_INST_V, MMVM_INST_S)() {
  SliceEntry e;
  e.lo = kLO;
  e.hi = kHI;
  e.tpc = kTPC;
  e.smem = smem_fn;
  e.prepare = prepare_fn;
  e.launch = launch_fn;
  e.occupancy = occ_fn;
  e.launch_batch = launch_batch_fn;
  e.occupancy_batch = occ_batch_fn;
  return e;
}

}  // namespace mmvm
