// Moments mu_j = Gamma((j+1)/beta)/beta for beta = 1/m (Sec. 2, eq. "moments").
//
// For beta = 1/m the moments are the integers mu_j = m * (m(j+1) - 1)!, so one
// warp keeps the exact running product G_j = mu_j in shared memory
// (G_0 = m!, G_{j+1} = G_j * m(j+1) * (m(j+1)+1) * ... * (m(j+2)-1)) and emits
// each mu_j truncated once to n limbs.  Lane l owns the limbs
// [l*C, (l+1)*C) of G (C = cap/32).
#pragma once
#include "common.cuh"

namespace hk {

__device__ __forceinline__ void big_mul_small(uint32_t* G, int C, uint32_t f, int* err) {
  const int lane = threadIdx.x & 31;
  uint32_t* g = G + lane * C;
  uint32_t carry = 0;
  for (int i = 0; i < C; ++i) {
    const uint64_t t = (uint64_t)g[i] * f + carry;
    g[i] = (uint32_t)t;
    carry = (uint32_t)(t >> 32);
  }
  // carries cross lane boundaries; a word-size carry can ripple further
  for (int it = 0; it < 40; ++it) {
    uint32_t cin = __shfl_up_sync(0xffffffffu, carry, 1);
    if (lane == 0) cin = 0;
    if (lane == 31 && carry && it == 0) atomicOr(err, 8);
    if (!__any_sync(0xffffffffu, cin != 0)) break;
    carry = 0;
    for (int i = 0; i < C && cin; ++i) {
      const uint64_t t = (uint64_t)g[i] + cin;
      g[i] = (uint32_t)t;
      cin = (uint32_t)(t >> 32);
    }
    carry = cin;
    if (lane == 31 && carry) atomicOr(err, 8);
  }
  __syncwarp();
}

// mu: 2N-1 numbers of n limbs.  smem: cap words (cap a multiple of 32).
__global__ void k_moments_exact(int m, int N, int n, int cap, MPVec mu, int* err) {
  extern __shared__ uint32_t G[];
  const int lane = threadIdx.x & 31;
  const int C = cap / 32;
  for (int i = lane; i < cap; i += 32) G[i] = 0;
  __syncwarp();
  if (lane == 0) G[0] = 1;
  __syncwarp();
  for (int f = 2; f <= m; ++f) big_mul_small(G, C, (uint32_t)f, err);
  for (int j = 0; j < 2 * N - 1; ++j) {
    // top non-zero limb of G
    int top = -1;
    for (int i = C - 1; i >= 0; --i)
      if (G[lane * C + i]) { top = lane * C + i; break; }
    for (int off = 16; off; off >>= 1) top = max(top, __shfl_xor_sync(0xffffffffu, top, off));
    const int lowest = top - n + 1;
    uint32_t* out = mu.mant + (int64_t)j * n;
    for (int k = lane; k < n; k += 32) {
      const int i = lowest + k;
      out[k] = (i >= 0) ? G[i] : 0u;
    }
    if (lane == 0) {
      mu.sgn[j] = 0;
      mu.exp[j] = lowest;
    }
    __syncwarp();
    if (j < 2 * N - 2)
      for (int64_t f = (int64_t)m * (j + 1); f < (int64_t)m * (j + 2); ++f) big_mul_small(G, C, (uint32_t)f, err);
  }
}

}  // namespace hk
