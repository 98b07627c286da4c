// Dispatch from (order, precision, variant) to the compiled slice kernels.
#include <algorithm>

#include "pair_registry.h"
#include "common.cuh"

namespace mmvm {

// the slice entry points of every compiled variant, and fill_slices()
#include "pair_registry_table.inc"
// the near-kernel and far-kernel entry points of the list form, and fill_list()
#include "pair_list_table.inc"

int pair_variant_count(int M, int precision) {
  if (M < 0 || M > 8 || (precision != 0 && precision != 1)) return 0;
  return n_variants(M, precision);
}

PairEntry pair_entry(int M, int precision, int v) {
  PairEntry e;
  if (v < 0 || v >= pair_variant_count(M, precision)) return e;
  const VariantSpec sp = variant_spec(M, precision, v);
  if (!fill_slices((M * 2 + precision) * kMaxVariants + v, e)) return e;
  e.M = M;
  e.precision = precision;
  e.variant = v;
  e.tpc = sp.TPC;
  e.minb = sp.MINB;
  e.sync = sp.SYNC;
  e.nslices = sp.nslices;
  for (int k = 0; k < e.nslices; ++k)
    if (e.slices[k].tpc != e.tpc) e.uniform_tpc = false;
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

int list_variant_count(int M) {
  if (M < 0 || M > 8) return 0;
  return n_list_variants(M);
}

ListEntry list_entry(int M, int v) {
  ListEntry e;
  if (v < 0 || v >= list_variant_count(M)) return e;
  if (!fill_list(M * kMaxListVariants + v, e)) return e;
  e.M = M;
  e.variant = v;
  e.nslices = list_variant_spec(M, v).nslices;
  return e;
}

cudaError_t list_prepare(const ListEntry& e) {
  for (int s = 0; s < e.nslices; ++s) {
    cudaError_t r = e.slices[s].prepare();
    if (r != cudaSuccess) return r;
  }
  return cudaSuccess;
}

int list_occupancy(const ListEntry& e) {
  int best = 1 << 30;
  for (int s = 0; s < e.nslices; ++s) {
    int b = 0;
    if (e.slices[s].occupancy(&b) != cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
    best = std::min(best, b);
  }
  return e.nslices ? best : 0;
}

long long tree_nodes(int G) { return tree_level_offset(G, tree_levels(G) + 1); }

int tree_chunk_level(int G, int blocks, int* nodes) {
  int L = 0;
  while (tree_level_nodes(G, L) > std::max(blocks, 1)) ++L;
  *nodes = tree_level_nodes(G, L);
  return L;
}

cudaError_t list_launch(const ListEntry& e, const float* rec, int n, const float* gdata,
                        int2* ent, int* cnt, int C, double* partial, int S, double* fpart,
                        float* tree, int Lc, unsigned long long* counts, int* err,
                        cudaStream_t st, cudaEvent_t* marks) {
  const int G = (n + kGroup - 1) / kGroup;
  cudaError_t r = e.far.build(rec, n, G, gdata, ent, cnt, st);
  if (tree && r == cudaSuccess) r = e.far.tree_build(gdata, n, G, tree, st);
  if (marks && r == cudaSuccess) r = cudaEventRecord(marks[0], st);
  if (r == cudaSuccess)
    r = tree ? e.far.far_tree(rec, n, G, gdata, tree, Lc, fpart, counts, st)
             : e.far.far(rec, n, G, gdata, S, fpart, counts, st);
  if (marks && r == cudaSuccess) r = cudaEventRecord(marks[1], st);
  for (int s = 0; s < e.nslices && r == cudaSuccess; ++s) {
    r = e.slices[s].launch(rec, n, G, ent, cnt, C, partial, counts, err, st);
    if (marks && r == cudaSuccess) r = cudaEventRecord(marks[2 + s], st);
  }
  return r;
}

}  // namespace mmvm
