// Exact limb products through a number-theoretic transform (NTT) modulo three
// 30-bit primes, for the wide formats where schoolbook products dominate.
//
// The limbs of X and Y (32 bits each) are read as polynomial coefficients;
// their product's coefficients c_t = sum_{s+u=t} x_s y_u are below
// n 2^64 <= 2^74, far below p1 p2 p3 ~ 2^90, so the cyclic convolution of
// length L >= 2n computed modulo each prime and recombined by the Chinese
// remainder theorem (Garner's form) gives every c_t exactly, and the exact
// product is sum_t c_t 2^(32 t).  Every prime is below 2^30 and has the form
// k 3 2^11 + 1, so lengths 2^a and 3 2^a (a <= 11) have roots of unity.
//
// Length: the least L = 2^a or L = 3 K (K = 2^a) with L >= 2n; 3 K saves a
// quarter of the work and memory when 2n is 3 2^a (1536 at n = 768, 768 at
// n = 384).  With gcd(3, K) = 1 the index map t -> (t mod 3, t mod K) turns
// the cyclic convolution of length 3 K into a two-dimensional one of size
// 3 x K (Good-Thomas), whose transform is three length-K transforms (rows)
// and K three-point transforms (columns), with no twiddles between them.
// Row r of the 3 x K array is held at positions r K .. r K + K - 1.
//
// Layout: rows are kept in bit-reversed order (forward: decimation in
// frequency, natural -> bit-reversed; inverse: decimation in time,
// bit-reversed -> natural), so pointwise products need no reordering.
// Twiddle factors w^k (k < LMAX/2, w a primitive LMAX-th root) and their
// inverses live in a device table with Shoup companions floor(w 2^32 / p).
//
// Speed: butterflies are lazy (values kept in [0, 2p) or [0, 4p), which fit
// 32 bits because p < 2^30; reductions happen once at the ends), three stages
// run per pass on eight elements held in registers, and shared memory is
// padded by one word per 32 so that short-stride passes avoid bank conflicts.
#pragma once
#include "mp_warp.cuh"

namespace hk {

constexpr int NTT_Q = 3;
constexpr int NTT_LMAX = 2048;  // power-of-two length limit: n <= 1024 limbs

struct NttConst {
  uint32_t p[NTT_Q], pinv[NTT_Q];  // primes, -p^{-1} mod 2^32 (Montgomery)
  uint32_t rl[NTT_Q], rls[NTT_Q];  // 2^32 / L mod p and its Shoup companion
  uint32_t w3[NTT_Q], w3s[NTT_Q];  // a primitive cube root of unity mod p (+ Shoup)
  uint32_t w3i[NTT_Q], w3is[NTT_Q];  // its inverse (+ Shoup)
  uint32_t i12, i12s, i13, i13s, i23, i23s;  // p1^{-1} mod p2, p1^{-1} mod p3, p2^{-1} mod p3 (+ Shoup)
  uint64_t p12;                    // p1 p2
  const uint2* twf;                // [q][k]: (w^k, Shoup), k < LMAX/2
  const uint2* twi;                // [q][k]: (w^-k, Shoup)
  int L, logL;                     // transform length and log2 of its row length
};

__device__ __forceinline__ uint32_t mod_add(uint32_t a, uint32_t b, uint32_t p) {
  const uint32_t s = a + b;  // a, b < p < 2^30: no overflow
  return s >= p ? s - p : s;
}
__device__ __forceinline__ uint32_t mod_sub(uint32_t a, uint32_t b, uint32_t p) { return a >= b ? a - b : a + p - b; }

// x w mod p, lazily in [0, 2p), for a constant w < p with ws = floor(w 2^32 / p), any x < 2^32
__device__ __forceinline__ uint32_t mul_shoup_lazy(uint32_t x, uint32_t w, uint32_t ws, uint32_t p) {
  return x * w - __umulhi(x, ws) * p;
}
__device__ __forceinline__ uint32_t mul_shoup(uint32_t x, uint32_t w, uint32_t ws, uint32_t p) {
  const uint32_t r = mul_shoup_lazy(x, w, ws, p);
  return r >= p ? r - p : r;
}

// a b 2^-32 mod p (Montgomery), lazily in [0, 2p); a, b < p
__device__ __forceinline__ uint32_t mont_mul_lazy(uint32_t a, uint32_t b, uint32_t p, uint32_t pinv) {
  const uint32_t lo = a * b, hi = __umulhi(a, b);
  const uint32_t m = lo * pinv;
  return hi + __umulhi(m, p) + (lo != 0u ? 1u : 0u);  // (a b + m p) / 2^32
}

// a[q] for a runtime q without spilling the constant struct to local memory
__device__ __forceinline__ uint32_t sel3(const uint32_t (&a)[NTT_Q], int q) {
  return q == 0 ? a[0] : (q == 1 ? a[1] : a[2]);
}

// 16-byte read-only load that does not allocate in L1: the transforms stream
// through once per product and would otherwise evict the twiddle table
__device__ __forceinline__ uint4 ld_stream(const uint4* ptr) {
  uint4 v;
  asm("ld.global.nc.L1::no_allocate.v4.u32 {%0, %1, %2, %3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "l"(ptr));
  return v;
}

// [0, 4p) -> [0, p)
__device__ __forceinline__ uint32_t reduce4(uint32_t x, uint32_t p) {
  x = x >= 2 * p ? x - 2 * p : x;
  return x >= p ? x - p : x;
}

// padded shared-memory index of transform element i (one word of padding per 32)
__device__ __forceinline__ int npad(int i) { return i + (i >> 5); }
__host__ __device__ constexpr int ntt_stride(int L) { return L + L / 32; }

// Transform shape for n limbs: L = rows 2^logk, rows in {1, 3}, the least
// such L >= 2n (ties go to the power of two).
__host__ __device__ constexpr int ntt_log2_ceil(int x) {
  int l = 0;
  while ((1 << l) < x) ++l;
  return l;
}
__host__ __device__ constexpr int ntt_rows(int n) {
  return (3 << ntt_log2_ceil((2 * n + 2) / 3)) < (1 << ntt_log2_ceil(2 * n)) ? 3 : 1;
}
__host__ __device__ constexpr int ntt_logk(int n) {
  return ntt_rows(n) == 3 ? ntt_log2_ceil((2 * n + 2) / 3) : ntt_log2_ceil(2 * n);
}
__host__ __device__ constexpr int ntt_len(int n) { return ntt_rows(n) << ntt_logk(n); }

// position of coefficient t (< L) in the rows x K array
template <int n>
__device__ __forceinline__ int ntt_pos(int t) {
  constexpr int K = 1 << ntt_logk(n);
  if constexpr (ntt_rows(n) == 1) return t;
  else return (t % 3) * K + (t & (K - 1));
}

// One pass of S stages on groups of R = 2^S elements i = hi 2^(s+S) + m 2^s + lo,
// everything but lo and hi known at compile time.  The twiddle of the
// butterfly (m, m + 2^t) at stage h = 2^(s+t) is w_{2h}^j with
// j = (m mod 2^t) 2^s + lo, i.e. table entry j LMAX/(2h) =
// (m mod 2^t) (LMAX/2^(t+1)) + lo (LMAX/2^(s+t+1)).
constexpr int NTT_LOG_HALF = 10;  // log2(NTT_LMAX / 2)

// Which groups the 32 lanes take together.  Group g of a pass has its low s
// bits in lo and the rest in hi; lanes take g's bits [0, A) and [B, B + 5 - A)
// and the iteration counter j the others.  A = B = 5 is the plain g = lane +
// 32 j.  For the short strides 0 < s < 5 that order puts lanes 2^s words
// apart and up to four of them in one bank; taking two of the lane bits from
// hi's upper bits instead spreads the 32 lanes over all 32 banks of the
// padded layout (A = s - 2, B = s, where the length allows).
template <int LOGL, int S, int s>
struct LaneMap {
  static constexpr bool plain = s == 0 || s >= 5 || (1 << (LOGL - S)) < 32;
  static constexpr int A = plain ? 5 : (s >= 2 ? s - 2 : 0);
  static constexpr int B0 = LOGL - S - 5 + A;
  static constexpr int B = plain ? 5 : (s < B0 ? (s < A ? A : s) : (B0 < A ? A : B0));
  __device__ __forceinline__ static int group(int lane, int j) {
    if constexpr (A == 5 && B == 5) {
      return lane + 32 * j;
    } else {
      return (lane & ((1 << A) - 1)) | ((j & ((1 << (B - A)) - 1)) << A) | ((lane >> A) << B) |
             ((j >> (B - A)) << (B + 5 - A));
    }
  }
};

template <int S, int s>
__device__ __forceinline__ int pass_index(int base, int m) {
  if constexpr (s >= 5) return npad(base) + m * ((1 << s) + (1 << (s - 5)));
  else return npad(base + (m << s));
}

// forward (decimation in frequency, stages s+S-1 .. s): [0, 2p) -> [0, 2p)
template <int LOGL, int S, int s>
__device__ __forceinline__ void dif_pass(uint32_t* buf, const uint2* __restrict__ tw, uint32_t p) {
  constexpr int R = 1 << S, groups = (1 << LOGL) >> S;
  const uint32_t p2 = 2 * p;
  using LM = LaneMap<LOGL, S, s>;
  const int lane = lane_id();
  for (int g0 = lane; g0 < groups; g0 += 32) {
    const int g = LM::plain ? g0 : LM::group(lane, g0 >> 5);
    const int lo = g & ((1 << s) - 1);
    const int base = ((g >> s) << (s + S)) + lo;
    uint32_t x[R];
#pragma unroll
    for (int m = 0; m < R; ++m) x[m] = buf[pass_index<S, s>(base, m)];
#pragma unroll
    for (int t = S - 1; t >= 0; --t) {
      const uint2* twt = tw + (lo << (NTT_LOG_HALF - s - t));
#pragma unroll
      for (int b = 0; b < (1 << t); ++b) {
        const uint2 w = __ldg(twt + b * (1 << (NTT_LOG_HALF - t)));
#pragma unroll
        for (int hgh = 0; hgh < R; hgh += (2 << t)) {
          const int m = hgh + b;
          const uint32_t u = x[m], v = x[m + (1 << t)];
          const uint32_t sm = u + v;
          x[m] = sm >= p2 ? sm - p2 : sm;
          x[m + (1 << t)] = mul_shoup_lazy(u - v + p2, w.x, w.y, p);
        }
      }
    }
#pragma unroll
    for (int m = 0; m < R; ++m) buf[pass_index<S, s>(base, m)] = x[m];
  }
}

// inverse (decimation in time, stages s .. s+S-1): [0, 4p) -> [0, 4p)
template <int LOGL, int S, int s>
__device__ __forceinline__ void dit_pass(uint32_t* buf, const uint2* __restrict__ tw, uint32_t p) {
  constexpr int R = 1 << S, groups = (1 << LOGL) >> S;
  const uint32_t p2 = 2 * p;
  using LM = LaneMap<LOGL, S, s>;
  const int lane = lane_id();
  for (int g0 = lane; g0 < groups; g0 += 32) {
    const int g = LM::plain ? g0 : LM::group(lane, g0 >> 5);
    const int lo = g & ((1 << s) - 1);
    const int base = ((g >> s) << (s + S)) + lo;
    uint32_t x[R];
#pragma unroll
    for (int m = 0; m < R; ++m) x[m] = buf[pass_index<S, s>(base, m)];
#pragma unroll
    for (int t = 0; t < S; ++t) {
      const uint2* twt = tw + (lo << (NTT_LOG_HALF - s - t));
#pragma unroll
      for (int b = 0; b < (1 << t); ++b) {
        const uint2 w = __ldg(twt + b * (1 << (NTT_LOG_HALF - t)));
#pragma unroll
        for (int hgh = 0; hgh < R; hgh += (2 << t)) {
          const int m = hgh + b;
          uint32_t X = x[m];
          X = X >= p2 ? X - p2 : X;
          const uint32_t T = mul_shoup_lazy(x[m + (1 << t)], w.x, w.y, p);
          x[m] = X + T;
          x[m + (1 << t)] = X - T + p2;
        }
      }
    }
#pragma unroll
    for (int m = 0; m < R; ++m) buf[pass_index<S, s>(base, m)] = x[m];
  }
}

template <int LOGL, int TOP>
__device__ __forceinline__ void dif_passes(uint32_t* buf, const uint2* tw, uint32_t p) {
  if constexpr (TOP > 0) {
    constexpr int S = TOP >= 3 ? 3 : TOP;
    dif_pass<LOGL, S, TOP - S>(buf, tw, p);
    __syncwarp();
    dif_passes<LOGL, TOP - S>(buf, tw, p);
  }
}

template <int LOGL, int s>
__device__ __forceinline__ void dit_passes(uint32_t* buf, const uint2* tw, uint32_t p) {
  if constexpr (s < LOGL) {
    constexpr int S = LOGL - s >= 3 ? 3 : LOGL - s;
    dit_pass<LOGL, S, s>(buf, tw, p);
    __syncwarp();
    dit_passes<LOGL, s + S>(buf, tw, p);
  }
}

// Three-point transforms of the K columns (a, b, c) = rows 0, 1, 2 at
// position j, with w a primitive cube root of unity (w^2 = -1 - w):
//   X0 = a + b + c,  X1 = (a - c) + w (b - c),  X2 = (a - b) - w (b - c).
// Inputs in [0, 2p), outputs in [0, 2p).
template <int K>
__device__ __forceinline__ void warp_dft3(uint32_t* buf, uint32_t w, uint32_t ws, uint32_t p) {
  constexpr int st = ntt_stride(K);
  const uint32_t p2 = 2 * p;
  for (int j = lane_id(); j < K; j += 32) {
    const int i = npad(j);
    uint32_t a = buf[i], b = buf[st + i], c = buf[2 * st + i];
    a = a >= p ? a - p : a;
    b = b >= p ? b - p : b;
    c = c >= p ? c - p : c;
    const uint32_t m = mul_shoup_lazy(b - c + p, w, ws, p);  // [0, 2p)
    uint32_t x0 = a + b + c;                                 // [0, 3p)
    uint32_t x1 = a - c + p + m;                             // [0, 4p)
    uint32_t x2 = a - b + 3 * p - m;                         // (0, 4p)
    x0 = x0 >= p2 ? x0 - p2 : x0;
    x1 = x1 >= p2 ? x1 - p2 : x1;
    x2 = x2 >= p2 ? x2 - p2 : x2;
    buf[i] = x0;
    buf[st + i] = x1;
    buf[2 * st + i] = x2;
  }
}

// Forward transform of the padded buf (rows x 2^LOGK) modulo prime q, in
// place ([0, 2p) in and out): rows first, then columns.
template <int LOGK, int ROWS>
__device__ __forceinline__ void warp_ntt_fwd(uint32_t* buf, const NttConst& nc, int q) {
  const uint32_t p = sel3(nc.p, q);
#pragma unroll 1
  for (int r = 0; r < ROWS; ++r) {
    dif_passes<LOGK, LOGK>(buf + r * ntt_stride(1 << LOGK), nc.twf + q * (NTT_LMAX / 2), p);
    __syncwarp();
  }
  if constexpr (ROWS == 3) {
    warp_dft3<1 << LOGK>(buf, sel3(nc.w3, q), sel3(nc.w3s, q), p);
    __syncwarp();
  }
}

// Inverse transform of the padded buf modulo prime q, in place, without the
// 1/L factor (folded into the stored transforms): columns first, then rows;
// [0, 2p) in, [0, 4p) out.
template <int LOGK, int ROWS>
__device__ __forceinline__ void warp_ntt_inv(uint32_t* buf, const NttConst& nc, int q) {
  const uint32_t p = sel3(nc.p, q);
  if constexpr (ROWS == 3) {
    warp_dft3<1 << LOGK>(buf, sel3(nc.w3i, q), sel3(nc.w3is, q), p);
    __syncwarp();
  }
#pragma unroll 1
  for (int r = 0; r < ROWS; ++r) {
    dit_passes<LOGK, 0>(buf + r * ntt_stride(1 << LOGK), nc.twi + q * (NTT_LMAX / 2), p);
    __syncwarp();
  }
}

// Transform of one n-limb mantissa (global) for all three primes into
// out[q * L .. q * L + L) (reduced, unpadded).  buf: ntt_stride(L) words of
// shared memory.  scaled: multiply by 2^32 / L so that a Montgomery product
// with the other operand's transform yields F(X) F(Y) / L.
template <int M>
__device__ __forceinline__ void warp_ntt_number(const uint32_t* __restrict__ mant, uint32_t* buf,
                                                uint32_t* __restrict__ out, const NttConst& nc, bool scaled) {
  constexpr int n = 32 * M, L = ntt_len(n);
  const int lane = lane_id();
  // the mantissa once, coalesced, into registers (limb lane + 32 t)
  uint32_t mv[M];
#pragma unroll
  for (int t = 0; t < M; ++t) mv[t] = mant[lane + 32 * t];
#pragma unroll 1
  for (int q = 0; q < NTT_Q; ++q) {
    const uint32_t p = sel3(nc.p, q), rl = sel3(nc.rl, q), rls = sel3(nc.rls, q);
#pragma unroll
    for (int t = 0; t < L / 32; ++t) {
      const int k = lane + 32 * t;
      uint32_t v = t < M ? mv[t < M ? t : 0] : 0u;
      v = v >= 2 * p ? v - 2 * p : v;  // 2^32 < 4p: now in [0, 2p)
      buf[npad(ntt_pos<n>(k))] = v >= 2 * p ? v - 2 * p : v;
    }
    __syncwarp();
    warp_ntt_fwd<ntt_logk(n), ntt_rows(n)>(buf, nc, q);
    uint32_t* o = out + (size_t)q * L;
    for (int k = lane; k < L; k += 32) {
      uint32_t v = buf[npad(k)];
      v = v >= p ? v - p : v;
      o[k] = scaled ? mul_shoup(v, rl, rls, p) : v;
    }
    __syncwarp();
  }
}

// c_t (< 2^90) from its residues (each < p) by Garner's mixed radix:
// c = r1 + p1 y2 + p1 p2 y3 (p1 > p2 > p3 and p1 < 2 p3)
__device__ __forceinline__ void crt3(uint32_t r1, uint32_t r2, uint32_t r3, const NttConst& nc, uint32_t& w0,
                                     uint32_t& w1, uint32_t& w2) {
  const uint32_t p1 = nc.p[0], p2 = nc.p[1], p3 = nc.p[2];
  const uint32_t r1m2 = r1 >= p2 ? r1 - p2 : r1;
  const uint32_t y2 = mul_shoup(mod_sub(r2, r1m2, p2), nc.i12, nc.i12s, p2);
  const uint32_t r1m3 = r1 >= p3 ? r1 - p3 : r1;
  const uint32_t t = mul_shoup(mod_sub(r3, r1m3, p3), nc.i13, nc.i13s, p3);
  const uint32_t y2m3 = y2 >= p3 ? y2 - p3 : y2;
  const uint32_t y3 = mul_shoup(mod_sub(t, y2m3, p3), nc.i23, nc.i23s, p3);
  const u128 v = (u128)nc.p12 * y3 + ((uint64_t)p1 * y2 + r1);
  w0 = (uint32_t)v;
  w1 = (uint32_t)(v >> 32);
  w2 = (uint32_t)(v >> 64);
}

// Garner's recombination in place: at every position of the three prime
// buffers the residues of one c_t (each in [0, 4p)) become the three 32-bit
// words of c_t.  A loop over positions, so its code stays small.
template <int n>
__device__ __forceinline__ void crt_in_place(uint32_t* res, const NttConst& nc) {
  constexpr int L = ntt_len(n), st = ntt_stride(L);
  const uint32_t p1 = nc.p[0], p2 = nc.p[1], p3 = nc.p[2];
#pragma unroll 1
  for (int k = lane_id(); k < L; k += 32) {
    const int i = npad(k);
    uint32_t w0, w1, w2;
    crt3(reduce4(res[i], p1), reduce4(res[st + i], p2), reduce4(res[2 * st + i], p3), nc, w0, w1, w2);
    res[i] = w0;
    res[st + i] = w1;
    res[2 * st + i] = w2;
  }
}

// Product limbs of one chunk [k0, k0 + M) from the words of crt_in_place:
// limb k = w0(c_k) + w1(c_{k-1}) + w2(c_{k-2}) + carry; returns the carry
// out (<= 3).  The window words of c_{k0-2}, c_{k0-1} are re-read here, so
// only carries cross chunks.
template <int M>
__device__ __forceinline__ uint32_t crt_chunk(const uint32_t* W, int k0, uint32_t (&out)[M]) {
  constexpr int n = 32 * M;
  constexpr int st = ntt_stride(ntt_len(n));
  constexpr int K = 1 << ntt_logk(n);
  const int r0 = ntt_rows(n) == 3 ? k0 % 3 : 0;
  // position of coefficient k0 + d (d >= -2 at compile time), c = 0 below 0
  auto at = [&](int d) -> int {
    if constexpr (ntt_rows(n) == 1) {
      return npad(k0 + d);
    } else {
      int r = r0 + ((d % 3) + 3) % 3;
      r = r >= 3 ? r - 3 : r;
      return npad(r * K + ((k0 + d) & (K - 1)));
    }
  };
  uint32_t a1 = 0, a2 = 0, b2 = 0;  // w1(c_{k-1}), w2(c_{k-1}), w2(c_{k-2})
  if (k0 >= 2) b2 = W[2 * st + at(-2)];
  if (k0 >= 1) {
    const int q = at(-1);
    a1 = W[st + q];
    a2 = W[2 * st + q];
  }
  uint64_t carry = 0;
#pragma unroll
  for (int kk = 0; kk < M; ++kk) {
    const int q = at(kk);
    const uint32_t w0 = W[q], w1 = W[st + q], w2 = W[2 * st + q];
    const uint64_t s = (uint64_t)w0 + a1 + b2 + carry;
    out[kk] = (uint32_t)s;
    carry = s >> 32;
    b2 = a2;
    a1 = w1;
    a2 = w2;
  }
  return (uint32_t)carry;
}

// Exact product P = X * Y from their stored transforms (fx: unscaled, fy:
// scaled by 2^32/L), in the lo/hi chunk layout of warp_mul.  nb:
// 3 ntt_stride(L) words of this warp's shared memory.
// X_RO / Y_RO: fx / fy is global memory that is read-only for the whole
// kernel; otherwise (written by this warp earlier, or shared memory) it is
// read through the generic path.
template <int M, bool X_RO = true, bool Y_RO = true>
__device__ __forceinline__ void warp_mul_ntt(const uint32_t* __restrict__ fx, const uint32_t* __restrict__ fy,
                                             uint32_t* nb, const NttConst& nc, uint32_t (&lo)[M],
                                             uint32_t (&hi)[M]) {
  constexpr int n = 32 * M;
  const int lane = lane_id();
  constexpr int L = ntt_len(n), st = ntt_stride(L);
#pragma unroll 1
  for (int q = 0; q < NTT_Q; ++q) {
    const uint32_t p = sel3(nc.p, q), pinv = sel3(nc.pinv, q);
    const uint4* a4 = reinterpret_cast<const uint4*>(fx + (size_t)q * L);
    const uint4* b4 = reinterpret_cast<const uint4*>(fy + (size_t)q * L);
    uint32_t* o = nb + q * st;
    // a trip count known at compile time and the loop unrolled, so that all
    // of a lane's loads of this prime are in flight together (one L2 round
    // trip per prime instead of one per iteration)
#pragma unroll
    for (int it = 0; it < (L / 4 + 31) / 32; ++it) {
      const int k = lane + 32 * it;
      if ((L / 4) % 32 != 0 && k >= L / 4) break;
      const uint4 a = X_RO ? ld_stream(a4 + k) : a4[k], b = Y_RO ? ld_stream(b4 + k) : b4[k];
      const int i = npad(4 * k);  // the four words share one padding block
      o[i] = mont_mul_lazy(a.x, b.x, p, pinv);
      o[i + 1] = mont_mul_lazy(a.y, b.y, p, pinv);
      o[i + 2] = mont_mul_lazy(a.z, b.z, p, pinv);
      o[i + 3] = mont_mul_lazy(a.w, b.w, p, pinv);
    }
    __syncwarp();
    warp_ntt_inv<ntt_logk(n), ntt_rows(n)>(o, nc, q);
  }
  crt_in_place<n>(nb, nc);
  __syncwarp();
  uint32_t loc = crt_chunk<M>(nb, lane * M, lo);
  uint32_t hic = crt_chunk<M>(nb, n + lane * M, hi);
  __syncwarp();
  for (int it = 0; it < 70; ++it) {
    uint32_t cin_lo = __shfl_up_sync(FULL, loc, 1);
    uint32_t cin_hi = __shfl_up_sync(FULL, hic, 1);
    const uint32_t c31 = __shfl_sync(FULL, loc, 31);
    if (lane == 0) {
      cin_lo = 0;
      cin_hi = c31;
    }
    if (!__any_sync(FULL, (cin_lo | cin_hi) != 0)) break;
    loc = chunk_add_word<M>(lo, cin_lo);
    hic = chunk_add_word<M>(hi, cin_hi);
  }
}

}  // namespace hk
