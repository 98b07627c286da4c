// Dispatch from (order, precision) to the compiled pair-kernel variants.
#include "pair_registry.h"

namespace mmvm {

#define MMVM_DECL(m)              \
  PairEntry pair_entry_m##m##_p0(); \
  PairEntry pair_entry_m##m##_p1();
MMVM_DECL(0)
MMVM_DECL(1)
MMVM_DECL(2)
MMVM_DECL(3)
MMVM_DECL(4)
MMVM_DECL(5)
MMVM_DECL(6)
MMVM_DECL(7)
MMVM_DECL(8)
#undef MMVM_DECL

PairEntry pair_entry(int M, int precision) {
  const bool f32 = precision == 1;
  switch (M) {
#define MMVM_CASE(m) \
  case m:            \
    return f32 ? pair_entry_m##m##_p1() : pair_entry_m##m##_p0();
    MMVM_CASE(0)
    MMVM_CASE(1)
    MMVM_CASE(2)
    MMVM_CASE(3)
    MMVM_CASE(4)
    MMVM_CASE(5)
    MMVM_CASE(6)
    MMVM_CASE(7)
    MMVM_CASE(8)
#undef MMVM_CASE
    default:
      return PairEntry{};
  }
}

}  // namespace mmvm
