// One limb width of libhk: instantiates every kernel and launcher for
// M = HK_M (n = 32 M limbs per number).
#include "ops.cuh"
#include "ops_tail.cuh"

#ifndef HK_M
#error "compile with -DHK_M=<limbs per lane>"
#endif

#define HK_CAT2(a, b) a##b
#define HK_CAT(a, b) HK_CAT2(a, b)

namespace hk {
const OpsTable* HK_CAT(ops_m, HK_M)() {
  static const OpsTable t = Ops<HK_M>::table();
  return &t;
}
}  // namespace hk
