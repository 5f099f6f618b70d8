// Warp-cooperative radix-2^32 multiprecision arithmetic for sm_103a.
//
// Number format (Sec. 4.1's "compute exactly, then truncate", carried from the
// paper's fixed point to a floating format): a value is
//     (-1)^sgn * M * 2^(32*exp),   M = sum_k mant[k] 2^(32k),  k < n,
// with the top limb mant[n-1] != 0, or M == 0 (then sgn == exp == 0).  Every
// operation returns its exact result with the magnitude truncated toward zero
// to n limbs.
//
// Work split: one warp owns one number; lane l holds the M = n/32 consecutive
// limbs [l*M, l*M + M) ("chunk l").  Double-width values (products) use two
// chunks per lane (chunks l and l+32) and the combine frame uses three
// (chunks l, l+32, l+64), i.e. 3n limbs.
#pragma once
#include <cstdint>

#include "common.cuh"

namespace hk {

constexpr unsigned FULL = 0xffffffffu;
typedef unsigned __int128 u128;


__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }

// ---------------------------------------------------------------------------
// chunk primitives (M limbs in registers, little endian)
// ---------------------------------------------------------------------------
template <int M>
__device__ __forceinline__ uint32_t chunk_add(uint32_t (&r)[M], const uint32_t (&a)[M],
                                              const uint32_t (&b)[M]) {
  uint32_t c;
  asm volatile("add.cc.u32 %0, %1, %2;" : "=r"(r[0]) : "r"(a[0]), "r"(b[0]));
#pragma unroll
  for (int k = 1; k < M; ++k)
    asm volatile("addc.cc.u32 %0, %1, %2;" : "=r"(r[k]) : "r"(a[k]), "r"(b[k]));
  asm volatile("addc.u32 %0, 0, 0;" : "=r"(c));
  return c;
}

template <int M>
__device__ __forceinline__ uint32_t chunk_sub(uint32_t (&r)[M], const uint32_t (&a)[M],
                                              const uint32_t (&b)[M]) {
  uint32_t c;
  asm volatile("sub.cc.u32 %0, %1, %2;" : "=r"(r[0]) : "r"(a[0]), "r"(b[0]));
#pragma unroll
  for (int k = 1; k < M; ++k)
    asm volatile("subc.cc.u32 %0, %1, %2;" : "=r"(r[k]) : "r"(a[k]), "r"(b[k]));
  asm volatile("subc.u32 %0, 0, 0;" : "=r"(c));
  return c & 1u;
}

// r += v (v a single word); returns the carry out
template <int M>
__device__ __forceinline__ uint32_t chunk_add_word(uint32_t (&r)[M], uint32_t v) {
  uint32_t c;
  asm volatile("add.cc.u32 %0, %0, %1;" : "+r"(r[0]) : "r"(v));
#pragma unroll
  for (int k = 1; k < M; ++k) asm volatile("addc.cc.u32 %0, %0, 0;" : "+r"(r[k]));
  asm volatile("addc.u32 %0, 0, 0;" : "=r"(c));
  return c;
}

template <int M>
__device__ __forceinline__ void chunk_dec(uint32_t (&r)[M]) {
  asm volatile("sub.cc.u32 %0, %0, 1;" : "+r"(r[0]));
#pragma unroll
  for (int k = 1; k < M; ++k) asm volatile("subc.cc.u32 %0, %0, 0;" : "+r"(r[k]));
}

template <int M>
__device__ __forceinline__ bool chunk_is_zero(const uint32_t (&r)[M]) {
  uint32_t o = 0;
#pragma unroll
  for (int k = 0; k < M; ++k) o |= r[k];
  return o == 0;
}

template <int M>
__device__ __forceinline__ bool chunk_is_ones(const uint32_t (&r)[M]) {
  uint32_t o = 0xffffffffu;
#pragma unroll
  for (int k = 0; k < M; ++k) o &= r[k];
  return o == 0xffffffffu;
}

// index of the highest non-zero limb of the chunk, or -1
template <int M>
__device__ __forceinline__ int chunk_top(const uint32_t (&r)[M]) {
  int t = -1;
#pragma unroll
  for (int k = 0; k < M; ++k)
    if (r[k]) t = k;
  return t;
}

__device__ __forceinline__ int top_bit128(u128 v) {  // v != 0
  uint64_t hi = (uint64_t)(v >> 64), lo = (uint64_t)v;
  return hi ? 127 - __clzll((long long)hi) : 63 - __clzll((long long)lo);
}

__device__ __forceinline__ u128 ballot3(bool b0, bool b1, bool b2) {
  u128 r = (u128)__ballot_sync(FULL, b0);
  r |= (u128)__ballot_sync(FULL, b1) << 32;
  r |= (u128)__ballot_sync(FULL, b2) << 64;
  return r;
}

// ---------------------------------------------------------------------------
// global <-> register chunk moves
// ---------------------------------------------------------------------------
template <int M>
__device__ __forceinline__ void load_chunk(const uint32_t* __restrict__ src, uint32_t (&v)[M]) {
  const uint32_t* p = src + lane_id() * M;
  if constexpr (M % 4 == 0) {
#pragma unroll
    for (int k = 0; k < M; k += 4) {
      uint4 t = *reinterpret_cast<const uint4*>(p + k);
      v[k] = t.x; v[k + 1] = t.y; v[k + 2] = t.z; v[k + 3] = t.w;
    }
  } else if constexpr (M % 2 == 0) {
#pragma unroll
    for (int k = 0; k < M; k += 2) {
      uint2 t = *reinterpret_cast<const uint2*>(p + k);
      v[k] = t.x; v[k + 1] = t.y;
    }
  } else {
#pragma unroll
    for (int k = 0; k < M; ++k) v[k] = p[k];
  }
}

template <int M>
__device__ __forceinline__ void store_chunk(uint32_t* __restrict__ dst, const uint32_t (&v)[M]) {
  uint32_t* p = dst + lane_id() * M;
  if constexpr (M % 4 == 0) {
#pragma unroll
    for (int k = 0; k < M; k += 4)
      *reinterpret_cast<uint4*>(p + k) = make_uint4(v[k], v[k + 1], v[k + 2], v[k + 3]);
  } else if constexpr (M % 2 == 0) {
#pragma unroll
    for (int k = 0; k < M; k += 2) *reinterpret_cast<uint2*>(p + k) = make_uint2(v[k], v[k + 1]);
  } else {
#pragma unroll
    for (int k = 0; k < M; ++k) p[k] = v[k];
  }
}

// Index policies for a warp's staging areas in shared memory.  IxPlain puts
// word i at i.  IxPad leaves one spare word after every 32 (word i at
// i + i/32).  Lane l's chunk starts at word l M, so under IxPlain the lanes
// of one access fall into only 32/gcd(M, 32) banks (4 at M = 24, 2 at
// M = 16); under IxPad at most two lanes share a bank for M <= 32.
struct IxPlain {
  __host__ __device__ static constexpr int at(int i) { return i; }
  __host__ __device__ static constexpr int words(int w) { return w; }
};
struct IxPad {
  __host__ __device__ static constexpr int at(int i) { return i + (i >> 5); }
  __host__ __device__ static constexpr int words(int w) { return w + (w + 31) / 32; }
};

// smem copy of a whole n-limb mantissa by the warp (n = 32 M)
template <int M, class IX = IxPlain>
__device__ __forceinline__ void copy_to_smem(uint32_t* dst, const uint32_t* __restrict__ src) {
  uint32_t v[M];
  load_chunk<M>(src, v);
#pragma unroll
  for (int k = 0; k < M; ++k) dst[IX::at(lane_id() * M + k)] = v[k];
}

// ---------------------------------------------------------------------------
// exact product: operand scanning with a systolic cross-lane reduction
// ---------------------------------------------------------------------------
// acc[0..M] += x[0..M-1] * y.  Requires acc[M] == 0 on entry; the bound
// acc < 2^(32M) and x*y <= (2^(32M)-1)(2^32-1) keeps the sum below 2^(32(M+1)).
template <int M>
__device__ __forceinline__ void mac_row(uint32_t (&acc)[M + 1], const uint32_t (&x)[M], uint32_t y) {
  asm volatile("mad.lo.cc.u32 %0, %1, %2, %0;" : "+r"(acc[0]) : "r"(x[0]), "r"(y));
#pragma unroll
  for (int k = 1; k < M; ++k)
    asm volatile("madc.lo.cc.u32 %0, %1, %2, %0;" : "+r"(acc[k]) : "r"(x[k]), "r"(y));
  asm volatile("addc.u32 %0, %0, 0;" : "+r"(acc[M]));
  if constexpr (M == 1) {
    asm volatile("mad.hi.u32 %0, %1, %2, %0;" : "+r"(acc[1]) : "r"(x[0]), "r"(y));
  } else {
    asm volatile("mad.hi.cc.u32 %0, %1, %2, %0;" : "+r"(acc[1]) : "r"(x[0]), "r"(y));
#pragma unroll
    for (int k = 1; k < M - 1; ++k)
      asm volatile("madc.hi.cc.u32 %0, %1, %2, %0;" : "+r"(acc[k + 1]) : "r"(x[k]), "r"(y));
    asm volatile("madc.hi.u32 %0, %1, %2, %0;" : "+r"(acc[M]) : "r"(x[M - 1]), "r"(y));
  }
}

// P = X * Y exactly (2n limbs).  x: this lane's chunk of X; ys: Y's n limbs in
// shared memory (read as broadcasts).  On return lane l holds product limbs
// [lM, lM+M) in lo and [n + lM, n + lM + M) in hi, fully carry-resolved.
//
// Lane l forms Z_l = X_l * Y (X_l = its chunk) one y-limb at a time, keeping
// an (M+1)-word window; after each block of M y-limbs the lane has finished M
// words of Z_l, which belong to product chunk l+q (q = block index).  Those
// words are added into a travelling buffer that moves one lane down per
// block, so the buffer for chunk c collects the contributions of lanes
// c, c-1, ... in turn and is complete when it reaches lane 0 (c < 32) or after
// the last block (c >= 32).  Carry words ride along and are resolved at the end.
//
// lo_stage: n + 32 words of this warp's shared memory; the finished low
// chunks (and their carry words) are parked there during the loop instead of
// in registers, which keeps the loop's register footprint at about 4M words.
template <int M>
__device__ __forceinline__ void warp_mul(const uint32_t (&x)[M], const uint32_t* ys, uint32_t* lo_stage,
                                         uint32_t (&lo)[M], uint32_t (&hi)[M]) {
  constexpr int n = 32 * M;
  const int lane = lane_id();
  uint32_t acc[M + 1];
  uint32_t buf[M];
  uint32_t bufc = 0, loc = 0, hic = 0;
#pragma unroll
  for (int k = 0; k <= M; ++k) acc[k] = 0;
#pragma unroll
  for (int k = 0; k < M; ++k) buf[k] = 0;

#pragma unroll 1
  for (int q = 0; q < 32; ++q) {
    uint32_t out[M];
    const uint32_t* yq = ys + q * M;
    uint32_t any = 0;
#pragma unroll
    for (int jj = 0; jj < M; ++jj) any |= yq[jj];
    if (any) {
#pragma unroll
      for (int jj = 0; jj < M; ++jj) {
        const uint32_t y = yq[jj];
        mac_row<M>(acc, x, y);
        out[jj] = acc[0];
#pragma unroll
        for (int k = 0; k < M; ++k) acc[k] = acc[k + 1];
        acc[M] = 0;
      }
    } else {
      // an all-zero block of y adds nothing: the window only moves on by M words
#pragma unroll
      for (int jj = 0; jj < M; ++jj) out[jj] = acc[jj];
      acc[0] = acc[M];
#pragma unroll
      for (int k = 1; k <= M; ++k) acc[k] = 0;
    }
    // buf += out
    asm volatile("add.cc.u32 %0, %0, %1;" : "+r"(buf[0]) : "r"(out[0]));
#pragma unroll
    for (int k = 1; k < M; ++k) asm volatile("addc.cc.u32 %0, %0, %1;" : "+r"(buf[k]) : "r"(out[k]));
    asm volatile("addc.u32 %0, %0, 0;" : "+r"(bufc));
    // lane 0 now holds the finished chunk q: park it in shared memory
    if (lane == 0) {
#pragma unroll
      for (int k = 0; k < M; ++k) lo_stage[q * M + k] = buf[k];
      lo_stage[n + q] = bufc;
    }
    // move every buffer one lane down; lane 31 starts a fresh chunk
#pragma unroll
    for (int k = 0; k < M; ++k) {
      buf[k] = __shfl_down_sync(FULL, buf[k], 1);
      if (lane == 31) buf[k] = 0;
    }
    bufc = __shfl_down_sync(FULL, bufc, 1);
    if (lane == 31) bufc = 0;
  }
  __syncwarp();
#pragma unroll
  for (int k = 0; k < M; ++k) lo[k] = lo_stage[lane * M + k];
  loc = lo_stage[n + lane];
  __syncwarp();
  // lane l: buf = chunk l+32 from lanes l+1..31, acc[0..M) = top of Z_l (chunk l+32)
  {
    uint32_t top[M];
#pragma unroll
    for (int k = 0; k < M; ++k) top[k] = acc[k];
    hic = bufc + chunk_add<M>(hi, buf, top);
  }
  // resolve carry words: chunk c's carry goes to chunk c+1
#pragma unroll 1
  for (int it = 0; it < 70; ++it) {
    uint32_t cin_lo = __shfl_up_sync(FULL, loc, 1);
    uint32_t cin_hi = __shfl_up_sync(FULL, hic, 1);
    const uint32_t c31 = __shfl_sync(FULL, loc, 31);
    if (lane == 0) { cin_lo = 0; cin_hi = c31; }
    if (!__any_sync(FULL, (cin_lo | cin_hi) != 0)) break;
    loc = chunk_add_word<M>(lo, cin_lo);
    hic = chunk_add_word<M>(hi, cin_hi);
  }
}

// ---------------------------------------------------------------------------
// the combine frame: R = (+-)|X| (+-) |Y| with both magnitudes staged in smem
// ---------------------------------------------------------------------------
// A staged magnitude occupies frame limbs [off, off + len); p == nullptr means
// a single 1 at frame limb `off` (a sticky stand-in for an operand that lies
// entirely below the other's last limb; see combine()).
struct Staged {
  const uint32_t* p;
  int off, len;
};

template <int M, class IX = IxPlain>
__device__ __forceinline__ void frame_chunk(const Staged& s, int c, uint32_t (&v)[M]) {
#pragma unroll
  for (int k = 0; k < M; ++k) {
    const int i = c * M + k - s.off;
    if (s.p) v[k] = (i >= 0 && i < s.len) ? s.p[IX::at(i)] : 0u;
    else v[k] = (i == 0) ? 1u : 0u;
  }
}

struct Result {
  int sgn, exp;
  bool zero;
  // a short product's truncation is not determined (nothing was written to
  // out; the caller recomputes the entry with the whole product)
  bool amb = false;
};

// trunc_n( sX*|X| + sY*|Y| ), sX/sY in {0:+, 1:-}, frame limb 0 having weight
// 2^(32*base).  fr: per-warp smem of >= 3n+2 words (it may alias the staging
// areas: every read of X and Y happens before the first write).  The lane's
// chunk of the result mantissa is returned in out.
//
// Exactness: the whole of both operands fits the 3n-limb frame, except when
// one lies entirely below the other by at least two limbs; the caller then
// stages a single 1 two limbs below the larger one.  Any value strictly
// between 0 and the larger operand's last-limb weight gives the same
// truncated result (the larger one is a multiple of that weight, and the
// result's own last limb is at most one limb lower), so the stand-in is exact.
//
// Short products (CUT, chk >= 0): Y holds P~, a product without its terms
// below some position, and the exact sum differs from the frame's by less
// than the weight of frame limb chk.  The truncation of the exact sum is the
// frame's when the frame limbs from chk up to the result's last limb hold
// one limb that is not 0 and one that is not all ones: then the remainder
// below the result's last limb is at least that weight and at most the last
// limb's weight minus it, so no perturbation smaller than chk's weight can
// carry or borrow across the last limb or change the leading limb.
// Otherwise (also for a zero frame) the result is flagged amb and not formed.
template <int M, class IX = IxPlain, bool CUT = false>
__device__ __forceinline__ Result combine(const Staged& X, int sX, const Staged& Y, int sY, int base,
                                          uint32_t* fr, uint32_t (&out)[M], int chk = -1) {
  constexpr int n = 32 * M;
  const int lane = lane_id();
  uint32_t r[3][M];
  uint32_t top = 0;
  int rs = sX;
  if (sX == sY) {
    bool g[3], p[3];
#pragma unroll
    for (int grp = 0; grp < 3; ++grp) {
      uint32_t xv[M], yv[M];
      frame_chunk<M, IX>(X, grp * 32 + lane, xv);
      frame_chunk<M, IX>(Y, grp * 32 + lane, yv);
      g[grp] = chunk_add<M>(r[grp], xv, yv) != 0;
      p[grp] = !g[grp] && chunk_is_ones<M>(r[grp]);
    }
    const u128 G = ballot3(g[0], g[1], g[2]);
    const u128 P = ballot3(p[0], p[1], p[2]);
    const u128 A = G | P;
    const u128 C = (A + G) ^ A ^ G;  // carry into chunk c is bit c
#pragma unroll
    for (int grp = 0; grp < 3; ++grp)
      if ((C >> (grp * 32 + lane)) & 1) chunk_add_word<M>(r[grp], 1u);
    top = (uint32_t)(C >> 96) & 1u;
  } else {
    bool g[3], p[3];
#pragma unroll
    for (int grp = 0; grp < 3; ++grp) {
      uint32_t xv[M], yv[M];
      frame_chunk<M, IX>(X, grp * 32 + lane, xv);
      frame_chunk<M, IX>(Y, grp * 32 + lane, yv);
      g[grp] = chunk_sub<M>(r[grp], xv, yv) != 0;
      p[grp] = !g[grp] && chunk_is_zero<M>(r[grp]);
    }
    const u128 G = ballot3(g[0], g[1], g[2]);
    const u128 P = ballot3(p[0], p[1], p[2]);
    const u128 A = G | P;
    const u128 B = (A + G) ^ A ^ G;  // borrow into chunk c is bit c
#pragma unroll
    for (int grp = 0; grp < 3; ++grp)
      if ((B >> (grp * 32 + lane)) & 1) chunk_dec<M>(r[grp]);
    if ((B >> 96) & 1) {
      // |X| < |Y|: negate the 3n-limb two's complement value
      bool ones[3];
#pragma unroll
      for (int grp = 0; grp < 3; ++grp) {
#pragma unroll
        for (int k = 0; k < M; ++k) r[grp][k] = ~r[grp][k];
        ones[grp] = chunk_is_ones<M>(r[grp]);
      }
      const u128 O = ballot3(ones[0], ones[1], ones[2]);
      // +1 enters chunk 0 and ripples through every all-ones chunk above it
      const u128 notO = ~O;
      // count trailing ones of O (number of chunks the +1 ripples through)
      int tz;
      {
        const uint64_t lo64 = (uint64_t)notO, hi64 = (uint64_t)(notO >> 64);
        tz = lo64 ? __ffsll((long long)lo64) - 1 : (hi64 ? 64 + __ffsll((long long)hi64) - 1 : 128);
      }
#pragma unroll
      for (int grp = 0; grp < 3; ++grp)
        if (grp * 32 + lane <= tz) chunk_add_word<M>(r[grp], 1u);
      rs = sY;
    }
  }
  // normalise: highest non-zero limb T of the frame (limb 3n is `top`)
  const u128 NZ = ballot3(!chunk_is_zero<M>(r[0]), !chunk_is_zero<M>(r[1]), !chunk_is_zero<M>(r[2]));
  Result res;
  int T;
  if (top) {
    T = 3 * n;
  } else if (NZ == 0) {
#pragma unroll
    for (int k = 0; k < M; ++k) out[k] = 0;
    res.sgn = 0; res.exp = 0; res.zero = true;
    if (CUT && chk >= 0) res.amb = true;
    return res;
  } else {
    const int h = top_bit128(NZ);
    const int grp = h >> 5, src = h & 31;
    int kk = -1;
    if (grp == 0) kk = chunk_top<M>(r[0]);
    else if (grp == 1) kk = chunk_top<M>(r[1]);
    else kk = chunk_top<M>(r[2]);
    kk = __shfl_sync(FULL, kk, src);
    T = h * M + kk;
  }
  if constexpr (CUT) {
    if (chk >= 0) {
      const int last = T - n + 1;
      bool nz = false, nf = false;
#pragma unroll
      for (int grp = 0; grp < 3; ++grp)
#pragma unroll
        for (int k = 0; k < M; ++k) {
          const int f = (grp * 32 + lane) * M + k;
          if (f >= chk && f < last) {
            nz |= r[grp][k] != 0u;
            nf |= r[grp][k] != 0xFFFFFFFFu;
          }
        }
      if (!__any_sync(FULL, nz) || !__any_sync(FULL, nf)) {
        res.sgn = 0; res.exp = 0; res.zero = false;
        res.amb = true;
        return res;
      }
    }
  }
  __syncwarp();
#pragma unroll
  for (int grp = 0; grp < 3; ++grp)
#pragma unroll
    for (int k = 0; k < M; ++k) fr[IX::at((grp * 32 + lane) * M + k)] = r[grp][k];
  if (lane == 0) fr[IX::at(3 * n)] = top;
  __syncwarp();
  const int lowest = T - n + 1;
#pragma unroll
  for (int k = 0; k < M; ++k) {
    const int i = lowest + lane * M + k;
    out[k] = (i >= 0) ? fr[IX::at(i)] : 0u;
  }
  __syncwarp();
  res.sgn = rs;
  res.exp = base + lowest;
  res.zero = false;
  return res;
}

// combine() on a frame of one chunk of MC limbs per lane (32 MC limbs,
// n = 32 M < 32 MC), for operands that both lie inside it, with the
// short-product test on when chk >= 1 (see combine()) and off for chk < 0
// (an exact frame, such as combine()'s stand-in for an operand wholly below
// the other).  The carry or borrow between the lanes' chunks is resolved
// with one 32-bit ballot per kind and a 64-bit prefix sum whose bit 32 is
// the carry out of the frame.
template <int MC, int M, class IX>
__device__ __forceinline__ Result combine_narrow(const Staged& X, int sX, const Staged& Y, int sY, int base,
                                                 uint32_t* fr, uint32_t (&out)[M], int chk) {
  constexpr int n = 32 * M, W = 32 * MC;
  static_assert(MC > M, "the frame must be wider than a result");
  const int lane = lane_id();
  uint32_t r[MC];
  uint32_t top = 0;
  int rs = sX;
  {
    // r = X's chunk, then Y's elements added or subtracted one by one along
    // the carry chain (Y's chunk is never held whole)
    frame_chunk<MC, IX>(X, lane, r);
    auto yel = [&](int k) -> uint32_t {
      const int i = lane * MC + k - Y.off;
      if (Y.p) return (i >= 0 && i < Y.len) ? Y.p[IX::at(i)] : 0u;
      return i == 0 ? 1u : 0u;
    };
    uint32_t cy;
    if (sX == sY) {
      asm volatile("add.cc.u32 %0, %0, %1;" : "+r"(r[0]) : "r"(yel(0)));
#pragma unroll
      for (int k = 1; k < MC; ++k) asm volatile("addc.cc.u32 %0, %0, %1;" : "+r"(r[k]) : "r"(yel(k)));
      asm volatile("addc.u32 %0, 0, 0;" : "=r"(cy));
    } else {
      asm volatile("sub.cc.u32 %0, %0, %1;" : "+r"(r[0]) : "r"(yel(0)));
#pragma unroll
      for (int k = 1; k < MC; ++k) asm volatile("subc.cc.u32 %0, %0, %1;" : "+r"(r[k]) : "r"(yel(k)));
      asm volatile("subc.u32 %0, 0, 0;" : "=r"(cy));
      cy &= 1u;
    }
    if (sX == sY) {
      const bool g = cy != 0;
      const bool p = !g && chunk_is_ones<MC>(r);
      const uint64_t G = __ballot_sync(FULL, g), A = G | __ballot_sync(FULL, p);
      const uint64_t C = (A + G) ^ A ^ G;  // carry into chunk l is bit l, out of the frame bit 32
      if ((C >> lane) & 1) chunk_add_word<MC>(r, 1u);
      top = (uint32_t)(C >> 32) & 1u;
    } else {
      const bool g = cy != 0;
      const bool p = !g && chunk_is_zero<MC>(r);
      const uint64_t G = __ballot_sync(FULL, g), A = G | __ballot_sync(FULL, p);
      const uint64_t B = (A + G) ^ A ^ G;  // borrow into chunk l is bit l
      if ((B >> lane) & 1) chunk_dec<MC>(r);
      if ((B >> 32) & 1) {
        // |X| < |Y|: negate the frame's two's complement value
#pragma unroll
        for (int k = 0; k < MC; ++k) r[k] = ~r[k];
        const uint32_t O = __ballot_sync(FULL, chunk_is_ones<MC>(r));
        const uint32_t notO = ~O;  // +1 enters chunk 0 and ripples through the all-ones chunks
        const int tz = notO ? __ffs((int)notO) - 1 : 32;
        if (lane <= tz) chunk_add_word<MC>(r, 1u);
        rs = sY;
      }
    }
  }
  const uint32_t NZ = __ballot_sync(FULL, !chunk_is_zero<MC>(r));
  Result res;
  int T;
  if (top) {
    T = W;
  } else if (NZ == 0) {
#pragma unroll
    for (int k = 0; k < M; ++k) out[k] = 0;
    res.sgn = 0; res.exp = 0; res.zero = true;
    res.amb = chk >= 0;  // a zero short difference says nothing about the exact one
    return res;
  } else {
    const int h = 31 - __clz((int)NZ);
    const int kk = __shfl_sync(FULL, chunk_top<MC>(r), h);
    T = h * MC + kk;
  }
  if (chk >= 0) {
    const int last = T - n + 1;
    bool nz = false, nf = false;
#pragma unroll
    for (int k = 0; k < MC; ++k) {
      const int f = lane * MC + k;
      if (f >= chk && f < last) {
        nz |= r[k] != 0u;
        nf |= r[k] != 0xFFFFFFFFu;
      }
    }
    if (!__any_sync(FULL, nz) || !__any_sync(FULL, nf)) {
      res.sgn = 0; res.exp = 0; res.zero = false;
      res.amb = true;
      return res;
    }
  }
  __syncwarp();
#pragma unroll
  for (int k = 0; k < MC; ++k) fr[IX::at(lane * MC + k)] = r[k];
  if (lane == 0) fr[IX::at(W)] = top;
  __syncwarp();
  const int lowest = T - n + 1;  // >= chk + 1 once the test has passed, >= 0 for an exact frame
#pragma unroll
  for (int k = 0; k < M; ++k) out[k] = fr[IX::at(lowest + lane * M + k)];
  __syncwarp();
  res.sgn = rs;
  res.exp = base + lowest;
  res.zero = false;
  return res;
}

// ---------------------------------------------------------------------------
// per-warp shared-memory layout for the fused operation
// ---------------------------------------------------------------------------
//   ys : n      words   (the broadcast operand Y)
//   sa : n + 2  words   (staging of the addend; combine frame starts here)
//   sp : 2n     words   (staging of the product)
// combine() writes its 3n+2 word frame over sa..sp.
template <int M>
struct WarpSmem {
  static constexpr int n = 32 * M;
  static constexpr int words = 4 * n + 2;
  uint32_t* ys;
  uint32_t* sa;
  uint32_t* sp;
  __device__ explicit WarpSmem(uint32_t* base) : ys(base), sa(base + n), sp(base + 2 * n + 2) {}
};

// The same areas under IxPad (no ys): sa at logical word n, sp at 2n + 32,
// both multiples of 32, so that sa[IxPad::at(i)] and sp[IxPad::at(i)] are
// the logical words n + i and 2n + 32 + i of the padded region, and the
// combine frame (3n + 1 words from sa) stays inside it.
template <int M>
struct WarpSmemPad {
  static constexpr int n = 32 * M;
  static constexpr int words = IxPad::words(4 * n + 32);
  uint32_t* sa;
  uint32_t* sp;
  __device__ explicit WarpSmemPad(uint32_t* base) : sa(base + IxPad::at(n)), sp(base + IxPad::at(2 * n + 32)) {}
};

// Stage the product (lo/hi chunks) into sp.
template <int M, class IX = IxPlain>
__device__ __forceinline__ void stage_product(uint32_t* sp, const uint32_t (&lo)[M], const uint32_t (&hi)[M]) {
  constexpr int n = 32 * M;
  const int lane = lane_id();
#pragma unroll
  for (int k = 0; k < M; ++k) {
    sp[IX::at(lane * M + k)] = lo[k];
    sp[IX::at(n + lane * M + k)] = hi[k];
  }
}

// Top limb index of the 2n-limb product held in (lo, hi); -1 if zero.
template <int M>
__device__ __forceinline__ int product_top(const uint32_t (&lo)[M], const uint32_t (&hi)[M]) {
  const unsigned bh = __ballot_sync(FULL, !chunk_is_zero<M>(hi));
  const unsigned bl = __ballot_sync(FULL, !chunk_is_zero<M>(lo));
  if (bh) {
    const int src = 31 - __clz(bh);
    const int kk = __shfl_sync(FULL, chunk_top<M>(hi), src);
    return 32 * M + src * M + kk;
  }
  if (bl) {
    const int src = 31 - __clz(bl);
    const int kk = __shfl_sync(FULL, chunk_top<M>(lo), src);
    return src * M + kk;
  }
  return -1;
}

// trunc_n(a - P) where P = (product in sp, 2n limbs, exponent ep, sign sp_sgn)
// and a = (sa staged n limbs, sign sa_sgn, exponent ea, a_zero).  Chooses the
// frame placement described at combine().  CUT, lc >= 0: sp holds a short
// product whose difference from the exact one is below the weight of its
// limb lc (see combine); lc is carried to the frame where P's limbs are used.
template <int M, class IX = IxPlain, bool CUT = false, class SMEM>
__device__ __forceinline__ Result sub_product(const SMEM& sm, int sa_sgn, int ea, bool a_zero,
                                              int sp_sgn, int ep, bool p_zero, uint32_t (&out)[M], int lc = -1) {
  constexpr int n = 32 * M;
  const int neg_p = sp_sgn ^ 1;  // a - P = a + (-P)
  if (p_zero) {
    // result is a itself (already normalised)
#pragma unroll
    for (int k = 0; k < M; ++k) out[k] = sm.sa[IX::at(lane_id() * M + k)];
    __syncwarp();
    Result r;
    r.zero = a_zero;
    r.sgn = a_zero ? 0 : sa_sgn;
    r.exp = a_zero ? 0 : ea;
    return r;
  }
  Staged X, Y;
  int base;
  int chk = -1;  // frame limb of P's limb lc; P's value is not used in the stand-in case
  if (a_zero) {
    X = Staged{sm.sa, 0, 0};
    Y = Staged{sm.sp, 0, 2 * n};
    base = ep;
    if (lc >= 0) chk = lc;
  } else {
    const long long delta = (long long)ea - (long long)ep;
    if (delta > 2 * n) {          // P entirely below a by >= 1 limb of a's frame
      X = Staged{sm.sa, 2, n};
      Y = Staged{nullptr, 0, 1};
      base = ea - 2;
    } else if (delta < -n) {      // a entirely below P (the stand-in for a is below P's limb 0 too)
      X = Staged{nullptr, 0, 1};
      Y = Staged{sm.sp, 2, 2 * n};
      base = ep - 2;
      if (lc >= 0) chk = lc + 2;
    } else {
      const int o = delta < 0 ? (int)delta : 0;
      X = Staged{sm.sa, (int)delta - o, n};
      Y = Staged{sm.sp, -o, 2 * n};
      base = ep + o;
      if (lc >= 0) chk = lc - o;
    }
  }
  return combine<M, IX, CUT>(X, sa_sgn, Y, neg_p, base, sm.sa, out, chk);
}

}  // namespace hk
