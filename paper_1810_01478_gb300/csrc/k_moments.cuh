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

// Moments for a rational beta = a/b (gcd 1) from supplied constants
// C_r = Gamma(r/a), r = 1..a-1 (Sec. 2, eq. "moments"): with
// b(j+1) = q a + r (0 <= r < a) the functional equation Gamma(x+1) = x Gamma(x)
// gives mu_j = (b/a) Gamma(q + r/a) = b C_r prod_{i<q} (r + i a) / a^(q+1), and
// mu_j = b (q-1)! / a when r = 0.  One warp per moment forms the integer
// G = 2^64 b M_r prod (...) exactly (M_r: C_r's mantissa; C_r = M_r 2^(32 e_r)),
// divides it by a^(q+1) (or a) in word-sized chunks -- floor(floor(x/u)/v) =
// floor(x/(uv)) keeps the quotient exact -- and keeps the top n limbs, i.e.
// the exact value truncated once.  The division passes run as a wavefront
// over the lanes (lane l works on pass t - (31 - l) at time t).
// smem: cap words per warp (cap a multiple of 32).
__global__ void k_moments_gamma(int a, int b, int N, int n, int cap, int nc, const int32_t* __restrict__ cexp,
                                const uint32_t* __restrict__ clim, MPVec mu, int* err) {
  extern __shared__ uint32_t sm_g[];
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  uint32_t* G = sm_g + (size_t)wib * cap;
  const int C = cap / 32;
  // a^k < 2^32: the largest chunk of the divisor
  int kmax = 0;
  uint64_t ak = 1;
  while (ak * (uint64_t)a < (1ull << 32)) {
    ak *= (uint64_t)a;
    ++kmax;
  }
  const int nw = gridDim.x * (blockDim.x >> 5);
  for (int j = blockIdx.x * (blockDim.x >> 5) + wib; j < 2 * N - 1; j += nw) {
    const int64_t bj = (int64_t)b * (j + 1);
    const int64_t q = bj / a, r = bj % a;
    for (int i = lane; i < cap; i += 32) G[i] = 0;
    __syncwarp();
    if (r == 0) {
      if (lane == 0) G[2] = (uint32_t)b;
    } else {
      const uint32_t* m = clim + (size_t)(r - 1) * nc;
      for (int i = lane; i < nc; i += 32) G[2 + i] = m[i];
    }
    __syncwarp();
    if (r != 0) big_mul_small(G, C, (uint32_t)b, err);
    // the factors, several per pass while their product fits a word
    const int64_t f0 = (r == 0) ? 2 : 0;  // (q-1)! = prod_{2 <= i < q} i; else i in [0, q)
    uint64_t acc = 1;
    for (int64_t i = f0; i < q; ++i) {
      const uint64_t f = (r == 0) ? (uint64_t)i : (uint64_t)(r + i * a);
      if (acc * f >= (1ull << 32)) {
        big_mul_small(G, C, (uint32_t)acc, err);
        acc = 1;
      }
      acc *= f;
    }
    if (acc > 1) big_mul_small(G, C, (uint32_t)acc, err);
    // G /= a^e (e = q + 1, or 1 when r = 0), in passes of a^kmax (the last smaller)
    const int64_t e = (r == 0) ? 1 : q + 1;
    const int64_t passes = (e + kmax - 1) / kmax;
    uint32_t* g = G + lane * C;
    uint32_t rem_out = 0;
    for (int64_t t = 0; t < passes + 31; ++t) {
      const uint32_t from_above = __shfl_down_sync(0xffffffffu, rem_out, 1);
      const int64_t p = t - (31 - lane);
      if (p >= 0 && p < passes) {
        const int64_t kk = (p == passes - 1) ? e - (passes - 1) * kmax : kmax;
        uint64_t d = 1;
        for (int64_t u = 0; u < kk; ++u) d *= (uint64_t)a;
        uint64_t rem = (lane == 31) ? 0 : from_above;
        for (int i = C - 1; i >= 0; --i) {
          const uint64_t cur = (rem << 32) | g[i];
          g[i] = (uint32_t)(cur / d);
          rem = cur % d;
        }
        rem_out = (uint32_t)rem;
      }
      __syncwarp();
    }
    // top non-zero limb and the n limbs below it
    int top = -1;
    for (int i = C - 1; i >= 0; --i)
      if (g[i]) { top = lane * C + i; break; }
    for (int off = 16; off; off >>= 1) top = max(top, __shfl_xor_sync(0xffffffffu, top, off));
    const int lowest = top - n + 1;
    uint32_t* out = mu.mant + (int64_t)j * n;
    for (int k = lane; k < n; k += 32) {
      const int i = lowest + k;
      out[k] = (i >= 0) ? G[i] : 0u;
    }
    if (lane == 0) {
      mu.sgn[j] = 0;
      mu.exp[j] = lowest - 2 + (r == 0 ? 0 : cexp[r - 1]);
      if (r != 0 && lowest < 0) atomicOr(err, 8);  // fewer than n limbs: the caller's constant is too short
    }
    __syncwarp();
  }
}

}  // namespace hk
