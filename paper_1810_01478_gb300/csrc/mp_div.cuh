// Warp-cooperative reciprocal and exactly truncated quotient.
//
// Algorithm 1 (Sec. 4.3) divides the pivot column by the pivot,
// B_i[j] = A_i[j] / A_i[i], and the paper stresses that these divisions are
// expensive, so they are done once per column entry rather than inside the
// trailing update.  Here every pivot d gets one Newton reciprocal
// R = floor(2^(64n-1) / D') (D' = D's mantissa shifted so its top bit is set),
// and each quotient is then one product A*R plus one product Q*D for an exact
// remainder check, which yields floor(A * 2^(32t) / D) exactly.
#pragma once
#include "mp_warp.cuh"

namespace hk {

// ---------------------------------------------------------------------------
// raw integer helpers on 2n-limb values held as (lo, hi) chunk pairs
// ---------------------------------------------------------------------------
// r = x - y (mod 2^(64n)); returns 1 when x < y.
template <int M>
__device__ __forceinline__ bool dsub(const uint32_t (&xlo)[M], const uint32_t (&xhi)[M],
                                     const uint32_t (&ylo)[M], const uint32_t (&yhi)[M],
                                     uint32_t (&rlo)[M], uint32_t (&rhi)[M]) {
  const int lane = lane_id();
  const bool g0 = chunk_sub<M>(rlo, xlo, ylo) != 0;
  const bool g1 = chunk_sub<M>(rhi, xhi, yhi) != 0;
  const bool p0 = !g0 && chunk_is_zero<M>(rlo);
  const bool p1 = !g1 && chunk_is_zero<M>(rhi);
  const uint64_t G = (uint64_t)__ballot_sync(FULL, g0) | ((uint64_t)__ballot_sync(FULL, g1) << 32);
  const uint64_t P = (uint64_t)__ballot_sync(FULL, p0) | ((uint64_t)__ballot_sync(FULL, p1) << 32);
  const u128 A = (u128)(G | P);
  const u128 B = (A + (u128)G) ^ A ^ (u128)G;
  if ((B >> lane) & 1) chunk_dec<M>(rlo);
  if ((B >> (32 + lane)) & 1) chunk_dec<M>(rhi);
  return (B >> 64) & 1;
}

// r += v for an n-limb value (one chunk per lane); returns the carry out of the top.
template <int M>
__device__ __forceinline__ bool nadd(uint32_t (&r)[M], const uint32_t (&v)[M]) {
  const int lane = lane_id();
  uint32_t s[M];
  const bool g = chunk_add<M>(s, r, v) != 0;
  const bool p = !g && chunk_is_ones<M>(s);
  const uint64_t G = __ballot_sync(FULL, g), P = __ballot_sync(FULL, p);
  const uint64_t A = G | P;
  const uint64_t C = (A + G) ^ A ^ G;
#pragma unroll
  for (int k = 0; k < M; ++k) r[k] = s[k];
  if ((C >> lane) & 1) chunk_add_word<M>(r, 1u);
  return (C >> 32) & 1;
}

// r += 1 for an n-limb value; returns the carry out of the top.
template <int M>
__device__ __forceinline__ bool ninc(uint32_t (&r)[M]) {
  const int lane = lane_id();
  const unsigned ones = __ballot_sync(FULL, chunk_is_ones<M>(r));
  // +1 enters chunk 0 and ripples through the run of all-ones chunks above it
  const int t = (~ones == 0u) ? 32 : __ffs(~ones) - 1;
  if (lane <= t) chunk_add_word<M>(r, 1u);
  return t == 32;
}

// -1 / 0 / +1 comparing two n-limb values (one chunk per lane)
template <int M>
__device__ __forceinline__ int ncmp(const uint32_t (&a)[M], const uint32_t (&b)[M]) {
  int c = 0;
#pragma unroll
  for (int k = 0; k < M; ++k)
    if (a[k] != b[k]) c = a[k] > b[k] ? 1 : -1;
  const unsigned d = __ballot_sync(FULL, c != 0);
  if (!d) return 0;
  return __shfl_sync(FULL, c, 31 - __clz(d));
}

// compare a 2n-limb value (lo, hi) with an n-limb value b (limbs [0, n))
template <int M>
__device__ __forceinline__ int dcmp_n(const uint32_t (&lo)[M], const uint32_t (&hi)[M], const uint32_t (&b)[M]) {
  if (__any_sync(FULL, !chunk_is_zero<M>(hi))) return 1;
  return ncmp<M>(lo, b);
}

// Read an n-limb window [w, w+n) of a 2n-limb value staged in smem at sp[0..2n]
// (sp[2n] == 0), shifted right by b bits (0 <= b < 32).
template <int M>
__device__ __forceinline__ void read_shifted(const uint32_t* sp, int w, int b, uint32_t (&v)[M]) {
  const int base = w + lane_id() * M;
#pragma unroll
  for (int k = 0; k < M; ++k) {
    const uint32_t l = sp[base + k];
    const uint32_t h = sp[base + k + 1];
    v[k] = b ? __funnelshift_r(l, h, b) : l;
  }
}

// ---------------------------------------------------------------------------
// reciprocal
// ---------------------------------------------------------------------------
// Given D (n-limb mantissa, top limb non-zero; lane chunk in d), returns
// sh = leading zero bits of D's top limb and R = min(floor(2^(64n-1)/D'),
// 2^(32n)-1), D' = D << sh.  ys: n words of this warp's smem (R lives there
// between products); sp: 2n+1 words of scratch.  Sets *err on a bound overrun.
// Products of the full-width steps: `wide(w)` says whether steps at width w
// take them from the policy (set_r: R is in ys; mul_d: D' R; mul_r: x R);
// the default forms every product with warp_mul.
struct RecipSchoolbook {
  __device__ bool wide(int) const { return false; }
  template <int M>
  __device__ void set_r(const uint32_t*) {}
  template <int M>
  __device__ void mul_d(const uint32_t (&)[M], uint32_t (&)[M], uint32_t (&)[M]) {}
  template <int M>
  __device__ void mul_r(const uint32_t (&)[M], uint32_t (&)[M], uint32_t (&)[M]) {}
};

template <int M, class P>
__device__ void warp_recip_p(const uint32_t (&d)[M], uint32_t* ys, uint32_t* sp, uint32_t (&R)[M], int& sh,
                             int* err, P& prod);

template <int M>
__device__ void warp_recip(const uint32_t (&d)[M], uint32_t* ys, uint32_t* sp, uint32_t (&R)[M], int& sh,
                           int* err) {
  RecipSchoolbook pol;
  warp_recip_p<M>(d, ys, sp, R, sh, err, pol);
}

template <int M, class P>
__device__ void warp_recip_p(const uint32_t (&d)[M], uint32_t* ys, uint32_t* sp, uint32_t (&R)[M], int& sh,
                             int* err, P& prod) {
  constexpr int n = 32 * M;
  const int lane = lane_id();
  // D' = D << sh
  uint32_t dp[M];
  {
    const uint32_t dtop = __shfl_sync(FULL, d[M - 1], 31);
    sh = __clz(dtop);
#pragma unroll
    for (int k = 0; k < M; ++k) sp[lane * M + k] = d[k];
    __syncwarp();
#pragma unroll
    for (int k = 0; k < M; ++k) {
      const int i = lane * M + k;
      const uint32_t cur = d[k];
      const uint32_t below = i > 0 ? sp[i - 1] : 0u;
      dp[k] = sh ? __funnelshift_l(below, cur, sh) : cur;
    }
    __syncwarp();
  }
  // initial approximation from the top 64 bits, from below:
  // R0_top = floor(2^126 / (D_hi + 1)) (exact integer division, about 61
  // correct bits) and R0 = R0_top * 2^(32n-63)
  {
    const uint32_t h1 = __shfl_sync(FULL, dp[M - 1], 31);
    uint32_t h0b;
    if constexpr (M >= 2) h0b = __shfl_sync(FULL, dp[M - 2], 31);
    else h0b = __shfl_sync(FULL, dp[0], 30);
    const uint64_t Dhi = ((uint64_t)h1 << 32) | h0b;
    const uint64_t r0 = (uint64_t)(((u128)1 << 126) / ((u128)Dhi + 1)) << 1;  // R0_top * 2
#pragma unroll
    for (int k = 0; k < M; ++k) {
      const int i = lane * M + k;
      R[k] = (i == n - 1) ? (uint32_t)(r0 >> 32) : (i == n - 2) ? (uint32_t)r0 : 0u;
    }
  }
  // constant C = 2^(64n-1) as (lo, hi) chunks
  uint32_t clo[M], chi[M];
#pragma unroll
  for (int k = 0; k < M; ++k) {
    clo[k] = 0;
    chi[k] = (lane == 31 && k == M - 1) ? 0x80000000u : 0u;
  }
  // Newton from below: R += floor(R * floor(E / 2^(32n)) / 2^(32n-1)), E = C - D'R >= 0.
  // The precision doubles per step, so R is kept truncated to its top w limbs
  // (w = 4, 8, 16, ... limbs; truncation keeps R below the true value) and the
  // two products skip R's zero limbs (warp_mul skips all-zero blocks of y).
  // `bits` is a lower bound on R's correct bits: 60 from the start above,
  // doubling per step while below the truncation width (32 w - 8); with 60
  // the schedule w = 4, 8, ..., 512 reaches 32n - 8 bits at w = n = 768 in a
  // single full-width step.
  int w = 2, bits = 60;
#pragma unroll 1
  for (int it = 0; it < 48; ++it) {
    w = min(n, 2 * w);
#pragma unroll
    for (int k = 0; k < M; ++k) ys[lane * M + k] = R[k];
    __syncwarp();
    uint32_t plo[M], phi[M], elo[M], ehi[M];
    const bool wide = prod.wide(w);
    if (wide) {
      prod.template set_r<M>(ys);
      prod.template mul_d<M>(dp, plo, phi);
    } else {
      warp_mul<M>(dp, ys, sp, plo, phi);
    }
    dsub<M>(clo, chi, plo, phi, elo, ehi);  // E >= 0 while R <= floor(C/D')
    uint32_t qlo[M], qhi[M];
    if (wide) prod.template mul_r<M>(ehi, qlo, qhi);
    else warp_mul<M>(ehi, ys, sp, qlo, qhi);  // (E >> 32n) * R
    // corr = floor(Q / 2^(32n-1)) = (Q >> (32n)) * 2 + top bit of Q's limb n-1
    uint32_t corr[M];
    {
      const uint32_t carry_in = __shfl_up_sync(FULL, qhi[M - 1], 1);
      const uint32_t lo_top = __shfl_sync(FULL, qlo[M - 1], 31);
#pragma unroll
      for (int k = M - 1; k >= 0; --k) {
        const uint32_t below = k > 0 ? qhi[k - 1] : (lane > 0 ? carry_in : lo_top);
        corr[k] = __funnelshift_l(below, qhi[k], 1);
      }
    }
    __syncwarp();
    const bool done = (w == n) && !__any_sync(FULL, !chunk_is_zero<M>(corr));
    if (done) break;
    if (nadd<M>(R, corr)) {
#pragma unroll
      for (int k = 0; k < M; ++k) R[k] = 0xffffffffu;
      break;
    }
    bits = min(2 * bits, 32 * w - 8);
    if (w < n) {  // keep the top w limbs
#pragma unroll
      for (int k = 0; k < M; ++k)
        if (lane * M + k < n - w) R[k] = 0;
    }
    // the exact correction below removes the last few units
    if (w == n && bits >= 32 * n - 8) break;
    if (it == 47 && lane == 0) atomicOr(err, ERR_LOOP);
  }
  // exact correction: while C - D'R >= D': R += 1
#pragma unroll 1
  for (int it = 0; it < 16; ++it) {
#pragma unroll
    for (int k = 0; k < M; ++k) ys[lane * M + k] = R[k];
    __syncwarp();
    uint32_t plo[M], phi[M], elo[M], ehi[M];
    if (prod.wide(n)) {
      prod.template set_r<M>(ys);
      prod.template mul_d<M>(dp, plo, phi);
    } else {
      warp_mul<M>(dp, ys, sp, plo, phi);
    }
    const bool negative = dsub<M>(clo, chi, plo, phi, elo, ehi);
    __syncwarp();
    if (negative) {  // cannot happen when R stays below the true value
      if (lane == 0) atomicOr(err, ERR_LOOP);
      break;
    }
    if (dcmp_n<M>(elo, ehi, dp) < 0) break;
    const bool all_ones = __all_sync(FULL, chunk_is_ones<M>(R));
    if (all_ones) break;  // D' = 2^(32n-1): the true value 2^(32n) is clamped
    ninc<M>(R);
    if (it == 15 && lane == 0) atomicOr(err, ERR_LOOP);
  }
  __syncwarp();
}

template <int M>
__device__ void quot_fix(const uint32_t (&a)[M], const uint32_t (&d)[M], int t, const uint32_t (&qlo)[M],
                         const uint32_t (&qhi)[M], uint32_t* sp, uint32_t (&q)[M], int* err);

// ---------------------------------------------------------------------------
// exactly truncated quotient
// ---------------------------------------------------------------------------
// q = trunc_n(a / d).  a: lane chunk of A (non-zero), d: lane chunk of D,
// R/sh from warp_recip for D, stored in ys (n words).  sp: 2n+2 words scratch.
// Returns Q's chunk in q and the limb shift t (q = floor(A 2^(32t) / D)).
template <int M>
__device__ void warp_quot(const uint32_t (&a)[M], const uint32_t (&d)[M], const uint32_t* ys_R, int sh,
                          uint32_t* ys_tmp, uint32_t* sp, uint32_t (&q)[M], int& t, int* err) {
  constexpr int n = 32 * M;
  const int lane = lane_id();
  t = (ncmp<M>(a, d) >= 0) ? n - 1 : n;
  uint32_t plo[M], phi[M];
  warp_mul<M>(a, ys_R, sp, plo, phi);
  // Q~ = floor(A*R / 2^shift), shift = 64n - 1 - 32t - sh
  const int shift = 64 * n - 1 - 32 * t - sh;
#pragma unroll
  for (int k = 0; k < M; ++k) {
    sp[lane * M + k] = plo[k];
    sp[n + lane * M + k] = phi[k];
  }
  if (lane == 0) sp[2 * n] = 0;
  __syncwarp();
  read_shifted<M>(sp, shift >> 5, shift & 31, q);
  __syncwarp();
  // Rem = A*2^(32t) - Q~ D  (>= 0 because Q~ <= Q)
#pragma unroll
  for (int k = 0; k < M; ++k) ys_tmp[lane * M + k] = d[k];
  __syncwarp();
  uint32_t qlo[M], qhi[M];
  warp_mul<M>(q, ys_tmp, sp, qlo, qhi);
  quot_fix<M>(a, d, t, qlo, qhi, sp, q, err);
}

// The end of an exact quotient: given Q~ (q) and the product Q~ D as (qlo,
// qhi), forms Rem = A 2^(32t) - Q~ D and steps Q~ up while Rem >= D.
// sp: 2n words of scratch.
template <int M>
__device__ void quot_fix(const uint32_t (&a)[M], const uint32_t (&d)[M], int t, const uint32_t (&qlo)[M],
                         const uint32_t (&qhi)[M], uint32_t* sp, uint32_t (&q)[M], int* err) {
  constexpr int n = 32 * M;
  const int lane = lane_id();
  // A * 2^(32t) as (lo, hi): stage A at limb offset t
#pragma unroll
  for (int k = 0; k < M; ++k) {
    sp[lane * M + k] = 0;
    sp[n + lane * M + k] = 0;
  }
  __syncwarp();
#pragma unroll
  for (int k = 0; k < M; ++k) sp[t + lane * M + k] = a[k];
  __syncwarp();
  uint32_t xlo[M], xhi[M];
#pragma unroll
  for (int k = 0; k < M; ++k) {
    xlo[k] = sp[lane * M + k];
    xhi[k] = sp[n + lane * M + k];
  }
  __syncwarp();
  uint32_t rlo[M], rhi[M];
  if (dsub<M>(xlo, xhi, qlo, qhi, rlo, rhi)) {
    if (lane == 0) atomicOr(err, ERR_LOOP);
  }
  // while Rem >= D: Rem -= D, Q~ += 1
  uint32_t zero[M];
#pragma unroll
  for (int k = 0; k < M; ++k) zero[k] = 0;
#pragma unroll 1
  for (int it = 0; it < 8; ++it) {
    if (dcmp_n<M>(rlo, rhi, d) < 0) break;
    uint32_t nlo[M], nhi[M];
    dsub<M>(rlo, rhi, d, zero, nlo, nhi);
#pragma unroll
    for (int k = 0; k < M; ++k) { rlo[k] = nlo[k]; rhi[k] = nhi[k]; }
    ninc<M>(q);
    if (it == 7 && lane == 0) atomicOr(err, ERR_LOOP);
  }
}

}  // namespace hk
