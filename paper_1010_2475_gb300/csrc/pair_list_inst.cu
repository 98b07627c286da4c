// One near-pair kernel of one interaction-list variant (pair_list.cuh,
// pair_list_variants.h), built with -DMMVM_INST_M, -DMMVM_INST_V and
// -DMMVM_INST_S so the kernels compile in parallel; with -DMMVM_INST_FAR
// instead of -DMMVM_INST_V / -DMMVM_INST_S, the list build and the far
// kernel of order MMVM_INST_M.
#include "pair_list.cuh"
#include "pair_registry.h"

#if !defined(MMVM_INST_M)
#error "MMVM_INST_M must be defined"
#endif

namespace mmvm {

#if defined(MMVM_INST_FAR)

namespace {
constexpr int kM = MMVM_INST_M;
cudaError_t build_fn(const float* rec, int n, int G, const float* gdata, int2* ent, int* cnt,
                     cudaStream_t st) {
  const int blocks = (G + 7) / 8;  // 8 warps (target groups) per block
  near_list_kernel<kM><<<blocks, 256, 0, st>>>(rec, n, G, gdata, ent, cnt);
  return cudaGetLastError();
}
cudaError_t far_fn(const float* rec, int n, int G, const float* gdata, int S, double* fpart,
                   unsigned long long* counts, cudaStream_t st) {
  dim3 grid((G + kFarWarps - 1) / kFarWarps, S);
  far_pair_kernel<kM><<<grid, kFarWarps * 32, 0, st>>>(rec, n, G, gdata, S, fpart, counts);
  return cudaGetLastError();
}
cudaError_t far_occ_fn(int* blocks) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, far_pair_kernel<kM>,
                                                       kFarWarps * 32, 0);
}
cudaError_t tree_build_fn(const float* gdata, int n, int G, float* tree, cudaStream_t st) {
  const int top = tree_levels(G);
  for (int L = 1; L <= top; ++L) {
    const float* child = L == 1 ? gdata : tree + (size_t)tree_level_offset(G, L - 1) * gdata_len(kM);
    const int nchild = tree_level_nodes(G, L - 1), nnode = tree_level_nodes(G, L);
    tree_level_kernel<kM><<<(nnode + 127) / 128, 128, 0, st>>>(
        child, nchild, L == 1 ? 1 : 0, n, tree + (size_t)tree_level_offset(G, L) * gdata_len(kM),
        nnode);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}
cudaError_t far_tree_fn(const float* rec, int n, int G, const float* gdata, const float* tree,
                        int Lc, double* fpart, unsigned long long* counts, cudaStream_t st) {
  dim3 grid((G + kFarWarps - 1) / kFarWarps, tree_level_nodes(G, Lc));
  far_tree_kernel<kM><<<grid, kFarWarps * 32, 0, st>>>(rec, n, G, gdata, tree, Lc, fpart, counts);
  return cudaGetLastError();
}
}  // namespace

#define MMVM_CAT2(a, b) a##b
#define MMVM_FAR_NAME(m) MMVM_CAT2(list_far_m, m)
#define MMVM_FAR(m) MMVM_FAR_NAME(m)

ListFarEntry MMVM_FAR(MMVM_INST_M)() {
  ListFarEntry e;
  e.build = build_fn;
  e.far = far_fn;
  e.far_occupancy = far_occ_fn;
  e.tree_build = tree_build_fn;
  e.far_tree = far_tree_fn;
  e.n_edge = n_edge(kM);
  return e;
}

#else

#if !defined(MMVM_INST_V) || !defined(MMVM_INST_S)
#error "MMVM_INST_V and MMVM_INST_S must be defined"
#endif

namespace {
constexpr int kM = MMVM_INST_M;
constexpr ListVariantSpec kSpec = list_variant_spec(kM, MMVM_INST_V);
static_assert(MMVM_INST_S < kSpec.nslices, "slice index out of range");
constexpr ListSliceSpec kS = kSpec.s[MMVM_INST_S];
constexpr size_t kSmem = near_list_smem_bytes<kM, kS.lo, kS.hi, kS.part, kS.w, kS.nst>();
static_assert(kSmem <= 232448, "near-pair kernel needs more shared memory than a CTA has");
#define MMVM_NEAR_KERNEL near_pair_kernel<kM, kS.lo, kS.hi, kS.part, kS.w, kS.minb, kS.nst, kS.sync>

cudaError_t prepare_fn() {
  return cudaFuncSetAttribute(MMVM_NEAR_KERNEL, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)kSmem);
}
cudaError_t launch_fn(const float* rec, int n, int G, const int2* ent, const int* cnt, int C,
                      double* partial, unsigned long long* counts, int* err, cudaStream_t st) {
  dim3 grid(G, C);
  MMVM_NEAR_KERNEL<<<grid, kS.w * 32, kSmem, st>>>(rec, n, G, ent, cnt, C, partial, counts, err);
  return cudaGetLastError();
}
cudaError_t occ_fn(int* blocks) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, MMVM_NEAR_KERNEL, kS.w * 32,
                                                       kSmem);
}
}  // namespace

#define MMVM_CAT4(a, b, c, d) a##b##c##d
#define MMVM_LSLICE_NAME(m, v, s) MMVM_CAT4(list_slice_m, m, _v##v, _s##s)
#define MMVM_LSLICE(m, v, s) MMVM_LSLICE_NAME(m, v, s)

ListSliceEntry MMVM_LSLICE(MMVM_INST_M, MMVM_INST_V, MMVM_INST_S)() {
  ListSliceEntry e;
  e.lo = kS.lo;
  e.hi = kS.hi;
  e.part = kS.part;
  e.warps = kS.w;
  e.prepare = prepare_fn;
  e.launch = launch_fn;
  e.occupancy = occ_fn;
  return e;
}

#endif

}  // namespace mmvm
