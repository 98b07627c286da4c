// Registry of compiled all-pairs kernel variants, per (order, precision).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

#include "common.cuh"
#include "pair_list_variants.h"
#include "pair_variants.h"

namespace mmvm {

// One order slice of a variant (one kernel).
struct SliceEntry {
  int lo = 0, hi = 0;
  int tpc = 0;  // targets per CTA of this slice's kernel
  size_t (*smem)(int S) = nullptr;
  cudaError_t (*prepare)(int S) = nullptr;  // set the dynamic shared-memory limit
  cudaError_t (*launch)(const void* rec, int n, int chunk_len, int gy, int S, const void* gbox,
                        double* partial, unsigned long long* counts, cudaStream_t st) = nullptr;
  cudaError_t (*occupancy)(int S, int* blocks_per_sm) = nullptr;
  // persistent batched form (pair_batch_kernel): `grid` CTAs
  cudaError_t (*launch_batch)(const void* rec, const BatchInst* inst, const int4* items,
                              const int* n_items, int* counter, int grid, int S, const void* gbox,
                              double* partial, cudaStream_t st) = nullptr;
  cudaError_t (*occupancy_batch)(int S, int* blocks_per_sm) = nullptr;
};

struct PairEntry {
  int M = -1;               // -1: no such variant
  int precision = 0;        // 0: FP64, 1: FP32
  int variant = 0;
  int tpc = 0;              // targets per CTA
  int minb = 1;             // CTAs per SM the register budget allows
  int sync = 0;             // barrier after every source
  bool uniform_tpc = true;  // every slice runs tpc targets per CTA (servable)
  int nslices = 0;
  SliceEntry slices[kMaxSlices];
  int rec_len = 0;          // record length in elements
  int elem_bytes = 0;       // sizeof(T)
};

// Number of compiled variants of (M, precision); 0 if none.
int pair_variant_count(int M, int precision);
// Variant v (an entry with M == -1 if it does not exist).
PairEntry pair_entry(int M, int precision, int v);
// Set the shared-memory limit of every slice kernel.
cudaError_t pair_prepare(const PairEntry& e, int S);
// CTAs per SM of the slice kernels (the smallest), 0 on error.
int pair_occupancy(const PairEntry& e, int S);
// Launch every slice.  gbox: float4 per group of kGroup records (null: every
// pair takes the full jet); S must equal kGroup.  Sources are split into
// `chunks` chunks of a multiple of S; `partial` holds min(chunks, grid_y_limit)
// chunks (grid_y_limit > 0 launches only the first grid_y_limit chunks, used
// when timing variants; 0 launches all of them).  counts (nullable) receives
// the cumulative (near, far) pair counts.
cudaError_t pair_launch(const PairEntry& e, const void* rec, int n, int chunks, int S,
                        const void* gbox, double* partial, int grid_y_limit, cudaStream_t st,
                        unsigned long long* counts = nullptr);
// CTAs per SM of the batched slice kernels (the smallest), 0 on error.
int pair_batch_occupancy(const PairEntry& e, int S);
// Launch every slice of the batched form, `grid` persistent CTAs each;
// counters[s] (zero at launch) hands out the items to slice s; gbox (null:
// no far field) holds the batch's group boxes.
cudaError_t pair_launch_batch(const PairEntry& e, const void* rec, const BatchInst* inst,
                              const int4* items, const int* n_items, int* counters, int grid,
                              int S, const void* gbox, double* partial, cudaStream_t st);

// ---------------------------------------------------------------- list form
// Interaction-list form (pair_list.cuh): one near-pair kernel per slice.
struct ListSliceEntry {
  int lo = 0, hi = 0, part = 0;
  int warps = 0;  // warps per CTA (all on one target group)
  cudaError_t (*prepare)() = nullptr;  // set the dynamic shared-memory limit
  // grid (G target groups, C list segments); partial: C blocks [NB][n]
  cudaError_t (*launch)(const float* rec, int n, int G, const int2* ent, const int* cnt, int C,
                        double* partial, unsigned long long* counts, int* err,
                        cudaStream_t st) = nullptr;
  cudaError_t (*occupancy)(int* blocks_per_sm) = nullptr;
};
// The list build and the far kernel of one order.
struct ListFarEntry {
  cudaError_t (*build)(const float* rec, int n, int G, const float* gdata, int2* ent, int* cnt,
                       cudaStream_t st) = nullptr;
  // grid (target groups / 4, S source ranges); fpart: S blocks [n_edge][n]
  cudaError_t (*far)(const float* rec, int n, int G, const float* gdata, int S, double* fpart,
                     unsigned long long* counts, cudaStream_t st) = nullptr;
  cudaError_t (*far_occupancy)(int* blocks_per_sm) = nullptr;
  // the tree over the groups (node storage: tree_nodes(G) records of
  // gdata_len(M) floats) and the far kernel walking it from the nodes of
  // level Lc (one far block per node of that level)
  cudaError_t (*tree_build)(const float* gdata, int n, int G, float* tree,
                            cudaStream_t st) = nullptr;
  cudaError_t (*far_tree)(const float* rec, int n, int G, const float* gdata, const float* tree,
                          int Lc, double* fpart, unsigned long long* counts,
                          cudaStream_t st) = nullptr;
  int n_edge = 0;  // edge columns of a far block (2 BMAX)
};
struct ListEntry {
  int M = -1;  // -1: no such variant
  int variant = 0;
  int nslices = 0;
  ListSliceEntry slices[kMaxListSlices];
  ListFarEntry far;
};

// Number of compiled list variants of order M (FP32 only).
int list_variant_count(int M);
ListEntry list_entry(int M, int v);
cudaError_t list_prepare(const ListEntry& e);
// CTAs per SM of the near kernels (the smallest), 0 on error.
int list_occupancy(const ListEntry& e);
// The whole list form of one right-hand side: list build, far field, near
// kernels (C list segments into partial).  ent: G x G entries, cnt: G counts
// (G = groups of kGroup records).  Far field: tree == nullptr: the flat far
// kernel over S source ranges; else the tree (tree_nodes(G) node records)
// built and walked from the nodes of level Lc (tree_level_nodes(G, Lc) far
// blocks; S is ignored).
// marks (nullable, 2 + nslices events): recorded after the list build and
// tree, after the far kernel and after each near kernel (per-kernel timing).
cudaError_t list_launch(const ListEntry& e, const float* rec, int n, const float* gdata,
                        int2* ent, int* cnt, int C, double* partial, int S, double* fpart,
                        float* tree, int Lc, unsigned long long* counts, int* err,
                        cudaStream_t st, cudaEvent_t* marks = nullptr);
// Node records of levels >= 1 of the tree over G groups.
long long tree_nodes(int G);
// Level whose node count is closest to (not above) `blocks`, and its count.
int tree_chunk_level(int G, int blocks, int* nodes);

}  // namespace mmvm
