// Launchers of the stages after the factorisation (placeholders until the
// kernels of those stages are in place).
#pragma once
#include "ops.cuh"

namespace hk {
template <int M>
hk_status Ops<M>::inv_block(Ctx& c) { return set_error(c, HK_ERR_UNSUPPORTED, "inv_block not built"); }
template <int M>
hk_status Ops<M>::lambda(Ctx& c, int) { return set_error(c, HK_ERR_UNSUPPORTED, "lambda1 not built"); }
template <int M>
hk_status Ops<M>::grad(Ctx& c, int32_t*, int32_t*, uint32_t*, double*) {
  return set_error(c, HK_ERR_UNSUPPORTED, "lambda1_grad not built");
}
}  // namespace hk
