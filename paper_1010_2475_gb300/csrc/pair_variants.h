// Compiled variants of the all-pairs kernel per (order M, precision).  A
// variant is a list of order slices [lo, hi] of the outputs (one kernel each,
// launched in turn) plus the CTA shape: TPC targets per CTA, MINB CTAs per SM
// the register budget must allow, SYNC > 0 a CTA barrier after every SYNC
// sources (keeps the warps on nearby code for the instruction cache).  The
// autotuner times the variants on the first state of each size and keeps the
// fastest.  FP32 keeps 2 x (outputs of the slice) x TPC floats of (hi, lo)
// sums in shared memory, which bounds TPC for wide slices.
#pragma once

namespace mmvm {

// part: which columns of the orders lo..hi the kernel accumulates.  A slice
// may run its own CTA shape (tpc targets per CTA, minb CTAs per SM); such a
// variant serves contexts only (the server hands out work items of the
// variant's TPC targets).
// 0: all of them; 1: the edge columns beta1 <= 1 (the jet, and the far
// field); 2: the Laplacian columns beta1 >= 2 (Hermite functions only, near
// tiles only).  A variant that splits a range lists it once per part.
struct SliceSpec {
  int lo = 0, hi = 0;
  int part = 0;
  int tpc = 0, minb = 0;  // CTA shape of this slice (0: the variant's)
};

constexpr int kMaxVariants = 12;
constexpr int kMaxSlices = 4;

struct VariantSpec {
  int nslices;
  SliceSpec s[kMaxSlices];
  int TPC, MINB, SYNC;
};

constexpr int n_variants(int M, int prec) {
  if (prec == 0) return 1;
  return M <= 3 ? 1 : (M == 7 ? 5 : (M == 6 ? 12 : (M == 8 ? 6 : 8)));
}

constexpr VariantSpec variant_spec(int M, int prec, int v) {
  if (prec == 0) {  // FP64: narrow slices keep the FP64 accumulators in registers
    switch (M) {
      case 0: return {1, {{1, 1}}, 64, 1, 0};
      case 1: return {1, {{1, 2}}, 64, 1, 0};
      case 2: return {1, {{1, 4}}, 64, 1, 0};
      case 3: return {1, {{1, 6}}, 64, 1, 0};
      case 4: return {2, {{1, 5}, {6, 8}}, 64, 1, 0};
      case 5: return {2, {{1, 6}, {7, 10}}, 64, 1, 0};
      case 6: return {3, {{1, 7}, {8, 10}, {11, 12}}, 64, 1, 0};
      case 7: return {4, {{1, 7}, {8, 10}, {11, 12}, {13, 14}}, 64, 1, 0};
      default: return {4, {{1, 8}, {9, 11}, {12, 14}, {15, 16}}, 64, 1, 0};
    }
  }
  switch (M) {
    case 0: return {1, {{1, 1}}, 128, 3, 0};
    case 1: return {1, {{1, 2}}, 128, 3, 0};
    case 2: return {1, {{1, 4}}, 128, 3, 0};
    case 3: return {1, {{1, 6}}, 128, 3, 0};
    case 4:
      return v == 0 ? VariantSpec{1, {{1, 8}}, 128, 3, 0}
           : v == 1 ? VariantSpec{1, {{1, 8}}, 256, 1, 1}
           : v == 2 ? VariantSpec{2, {{1, 5}, {6, 8}}, 128, 2, 1}
           : v == 3 ? VariantSpec{1, {{1, 8}}, 256, 1, 4}
           : v == 4 ? VariantSpec{1, {{1, 8}}, 64, 6, 2}
           : v == 5 ? VariantSpec{1, {{1, 8}}, 128, 3, 2}
           : v == 6 ? VariantSpec{2, {{1, 8, 1}, {1, 8, 2}}, 128, 4, 1}
                    : VariantSpec{2, {{1, 8, 1}, {1, 8, 2}}, 128, 5, 1};
    case 5:
      return v == 0 ? VariantSpec{1, {{1, 10}}, 256, 1, 1}
           : v == 1 ? VariantSpec{2, {{1, 7}, {8, 10}}, 128, 2, 1}
           : v == 2 ? VariantSpec{2, {{1, 7}, {8, 10}}, 256, 1, 1}
           : v == 3 ? VariantSpec{1, {{1, 10}}, 256, 1, 4}
           : v == 4 ? VariantSpec{1, {{1, 10}}, 64, 4, 2}
           : v == 5 ? VariantSpec{1, {{1, 10}}, 128, 2, 2}
           : v == 6 ? VariantSpec{2, {{1, 10, 1}, {1, 10, 2}}, 128, 3, 1}
                    : VariantSpec{2, {{1, 10, 1}, {1, 10, 2}}, 128, 4, 1};
    case 6:
      return v == 0 ? VariantSpec{1, {{1, 12}}, 256, 1, 1}
           : v == 1 ? VariantSpec{2, {{1, 8}, {9, 12}}, 128, 2, 1}
           : v == 2 ? VariantSpec{3, {{1, 6}, {7, 9}, {10, 12}}, 128, 2, 1}
           : v == 3 ? VariantSpec{2, {{1, 8}, {9, 12}}, 256, 1, 1}
           : v == 4 ? VariantSpec{1, {{1, 12}}, 256, 1, 4}
           : v == 5 ? VariantSpec{1, {{1, 12}}, 256, 1, 2}
           : v == 6 ? VariantSpec{1, {{1, 12}}, 64, 4, 2}
           : v == 7 ? VariantSpec{1, {{1, 12}}, 128, 2, 2}
           : v == 8 ? VariantSpec{2, {{1, 12, 1}, {1, 12, 2}}, 128, 3, 1}
           : v == 9 ? VariantSpec{2, {{1, 12, 1}, {1, 12, 2}}, 128, 4, 1}
           : v == 10 ? VariantSpec{2, {{1, 12, 1}, {1, 12, 2}}, 384, 1, 1}
                     : VariantSpec{2, {{1, 12, 1}, {1, 12, 2, 128, 3}}, 384, 1, 1};
    case 7:
      return v == 0 ? VariantSpec{2, {{1, 8}, {9, 14}}, 128, 2, 1}
           : v == 1 ? VariantSpec{3, {{1, 7}, {8, 11}, {12, 14}}, 128, 2, 1}
           : v == 2 ? VariantSpec{2, {{1, 8}, {9, 14}}, 128, 2, 4}
           : v == 3 ? VariantSpec{3, {{1, 14, 1}, {1, 10, 2}, {11, 14, 2}}, 128, 3, 1}
                    : VariantSpec{2, {{1, 14, 1}, {1, 14, 2}}, 128, 2, 1};
    default:
      return v == 0 ? VariantSpec{3, {{1, 8}, {9, 12}, {13, 16}}, 128, 2, 1}
           : v == 1 ? VariantSpec{4, {{1, 8}, {9, 11}, {12, 14}, {15, 16}}, 128, 2, 1}
           : v == 2 ? VariantSpec{4, {{1, 8}, {9, 11}, {12, 14}, {15, 16}}, 256, 1, 1}
           : v == 3 ? VariantSpec{3, {{1, 8}, {9, 12}, {13, 16}}, 128, 2, 4}
           : v == 4 ? VariantSpec{3, {{1, 16, 1}, {1, 12, 2}, {13, 16, 2}}, 128, 3, 1}
                    : VariantSpec{3, {{1, 16, 1}, {1, 12, 2}, {13, 16, 2}}, 128, 2, 1};
  }
}

}  // namespace mmvm
