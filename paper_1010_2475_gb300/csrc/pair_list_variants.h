// Compiled variants of the interaction-list form of the all-pairs kernel
// (pair_list.cuh; FP32 records with the far field), per order M.  A variant
// lists its near-pair kernels, one per (order range, column part), each with
// W warps per CTA (all on one target group), MINB CTAs per SM the register
// budget must allow and NST shared-memory stages of source groups.  The far
// kernel and the list build are the same for every variant of an order.
// A part-2 kernel keeps 2 W x (its Laplacian columns) x 32 floats of (hi, lo)
// sums in shared memory, which is why the wide orders split part 2 in two
// order ranges.
#pragma once

namespace mmvm {

struct ListSliceSpec {
  int lo = 0, hi = 0;
  int part = 0;  // 0: all columns, 1: edge columns (beta1 <= 1), 2: Laplacian columns
  int w = 0;     // warps per CTA
  int minb = 1;  // CTAs per SM
  int nst = 4;   // record slots per warp (copies issued this many sources ahead)
  int sync = 1;  // CTA barrier every `sync` rounds (0: only between list windows)
};

constexpr int kMaxListVariants = 16;
constexpr int kMaxListSlices = 3;

struct ListVariantSpec {
  int nslices;
  ListSliceSpec s[kMaxListSlices];
};

constexpr int n_list_variants(int M) { return M <= 3 ? 2 : (M == 6 ? 8 : 2); }

constexpr ListVariantSpec list_variant_spec(int M, int v) {
  switch (M) {
    case 0: return v == 0 ? ListVariantSpec{1, {{1, 1, 0, 12, 1, 4}}}
                          : ListVariantSpec{1, {{1, 1, 0, 8, 2, 4}}};
    case 1: return v == 0 ? ListVariantSpec{1, {{1, 2, 0, 12, 1, 4}}}
                          : ListVariantSpec{1, {{1, 2, 0, 8, 2, 4}}};
    case 2: return v == 0 ? ListVariantSpec{1, {{1, 4, 0, 12, 1, 4}}}
                          : ListVariantSpec{1, {{1, 4, 0, 8, 2, 4}}};
    case 3: return v == 0 ? ListVariantSpec{1, {{1, 6, 0, 12, 1, 4}}}
                          : ListVariantSpec{2, {{1, 6, 1, 12, 1, 4}, {1, 6, 2, 12, 1, 4}}};
    case 4: return v == 0 ? ListVariantSpec{2, {{1, 8, 1, 16, 1, 4}, {1, 8, 2, 16, 1, 4}}}
                          : ListVariantSpec{2, {{1, 8, 1, 12, 1, 4}, {1, 8, 2, 12, 1, 4}}};
    case 5: return v == 0 ? ListVariantSpec{2, {{1, 10, 1, 12, 1, 4}, {1, 10, 2, 12, 1, 4}}}
                          : ListVariantSpec{2, {{1, 10, 1, 16, 1, 4}, {1, 10, 2, 16, 1, 4}}};
    case 6:
      return v == 0 ? ListVariantSpec{2, {{1, 12, 1, 12, 1, 4}, {1, 12, 2, 12, 1, 4}}}
           : v == 1 ? ListVariantSpec{2, {{1, 12, 1, 12, 1, 4}, {1, 12, 2, 8, 1, 4}}}
           : v == 2 ? ListVariantSpec{2, {{1, 12, 1, 8, 1, 4}, {1, 12, 2, 8, 1, 4}}}
           : v == 3 ? ListVariantSpec{1, {{1, 12, 0, 8, 1, 4}}}
           : v == 4 ? ListVariantSpec{2, {{1, 12, 1, 12, 1, 4, 0}, {1, 12, 2, 12, 1, 4, 0}}}
           : v == 5 ? ListVariantSpec{2, {{1, 12, 1, 12, 1, 4, 4}, {1, 12, 2, 12, 1, 4, 4}}}
           : v == 6 ? ListVariantSpec{1, {{1, 12, 0, 8, 1, 4, 0}}}
                    : ListVariantSpec{1, {{1, 12, 0, 8, 1, 4, 4}}};
    case 7:
      return v == 0 ? ListVariantSpec{3, {{1, 14, 1, 12, 1, 4}, {1, 10, 2, 12, 1, 4},
                                          {11, 14, 2, 12, 1, 4}}}
                    : ListVariantSpec{3, {{1, 14, 1, 8, 1, 4}, {1, 10, 2, 8, 1, 4},
                                          {11, 14, 2, 8, 1, 4}}};
    default:
      return v == 0 ? ListVariantSpec{3, {{1, 16, 1, 12, 1, 4}, {1, 12, 2, 12, 1, 4},
                                          {13, 16, 2, 12, 1, 4}}}
                    : ListVariantSpec{3, {{1, 16, 1, 8, 1, 4}, {1, 12, 2, 8, 1, 4},
                                          {13, 16, 2, 8, 1, 4}}};
  }
}

}  // namespace mmvm
