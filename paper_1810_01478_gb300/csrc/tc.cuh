// Exact limb products on the 5th-generation tensor cores (tcgen05, kind::f16
// with bf16 operands and fp32 accumulators in tensor memory), for the
// trailing update of Algorithm 1 (Sec. 4.3) and the elementwise fused batch.
//
// Why this is exact.  A magnitude m < 2^(32n) is recoded into D balanced
// 7-bit digits, m = sum_k d_k 2^(7k) with d_k in [-64, 63] (a carry
// recode: raw digit t + carry >= 64 becomes t + carry - 128 and carries one).
// Every digit is an integer bf16 represents exactly.  The product U B has
// coefficients v_q = sum_k B_k U_(q-k), at most D terms of magnitude at most
// 64 * 64, so |v_q| <= D 2^12 < 2^24 (D = floor(32n/7) + 2 <= 3512 at 768
// limbs): every partial sum an fp32 accumulator holds is an integer it
// represents exactly, whatever the order of the additions.  The limbs of the
// product are then sum_q v_q 2^(7q), formed with 64-bit integer arithmetic.
//
// The contraction.  For one column c of a step (U = U_c fixed) and 128 rows
// r (the scaled B_i[r]), C[r][q] = sum_k B_r(k) U(q - k) is a GEMM: the A
// operand is the rows' digit matrix (128 x K, loaded by the bulk-copy engine
// from a kgroup-major copy in global memory), the B operand is the Toeplitz
// matrix of U.  A shared-memory descriptor cannot step backwards, so the
// position axis of a 256-position tile is reversed (column n <-> position
// Q0 - n) which turns the Toeplitz matrix into a Hankel one, and a Hankel
// matrix of 8 x 8 core matrices has core (a, b) depending on a + b only: one
// stored core per 8 positions, addressed with leading and stride byte offsets
// both 128.  The stored cores of U_c (about 66 KB at 768 limbs) serve every
// tile and K-step of the column.
//
// Short products.  The result keeps n limbs below its leading one, so the
// product's low positions matter only through the carry they send up.  A
// launch forms the positions from Q up (Q = QCUT, a multiple of 32, about
// D - 16 limbs' worth of positions below the middle): the omitted terms
// sum to less than 2^(7Q + 18) in absolute value (below 2^24 at each
// position, as above, and the positions' weights 2^(7q) form a geometric
// series of ratio 2^-7), and combine() takes the truncation
// of the formed difference only where that bound cannot change it (a limb
// between the bound and the result's last limb that is neither 0 nor all
// ones).  Rows it cannot decide are not written; their items go on a list
// that a second launch of the same kernel re-runs with Q = 0 (the whole
// product), forming only those rows.  Every result is therefore the
// truncation of the exact a - x y, as on every other product path.
//
// Schedule.  Tiles t (256 positions each) run in staggered pairs on two
// 256-column fp32 accumulators: the pair's K-blocks (64 digits, one bulk-copy
// stage) are loaded once and used by both tiles where their bands overlap,
// and one accumulator is drained (tcgen05.ld) while the other finishes.
//
// Warp roles of the persistent kernel (320 threads, one CTA per SM):
//   warp 0      producer: streams the A-operand stages with cp.async.bulk
//               and builds the Hankel cores of each item's U_c from its
//               digits (brought in by a bulk copy during the item before)
//   warp 1      tensor-memory owner and MMA issuer (one thread)
//   warps 2..9  two sets of four that take the block's items in turn; a
//               warp drains its 32 TMEM lanes (one row per thread:
//               accumulator -> integer coefficients -> product limbs, into
//               a global buffer), then forms trunc(a - P) for those 32 rows
//               one row at a time with the whole warp, the same
//               single-rounding combine as every other product path.  While
//               one set combines, the other drains the next item.
// Every wait is bounded; a wait that gives up raises ERR_TIMEOUT, and the
// kernel still drains its copies and MMAs and frees its tensor memory.
#pragma once
#include <cuda_bf16.h>

#include "k_ldlt.cuh"

namespace hk {

constexpr int tc_fdiv(int a, int b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }

template <int M>
struct TcShape {
  static constexpr int n = 32 * M;
  static constexpr int D = (32 * n) / 7 + 2;                // digits per number (data + one carry digit + 1)
  static constexpr int ND = (D + 63) / 64 * 64;              // digit slots: whole 64-digit K-blocks
  static constexpr int T = (2 * D - 1 + 255) / 256;           // 256-position tiles of a product
  static constexpr int PL = 56 * T;                           // limbs emitted per product (7 per 32 positions)
  static constexpr int XMIN = 8 * tc_fdiv(-D - 318, 8) + 1;   // Hankel core arguments x = XMIN + 8h
  static constexpr int XMAX = 304;
  static constexpr int NHC = (XMAX - XMIN) / 8 + 1;           // stored cores
  static constexpr int Z0 = 320;                              // staging: digit y of U at su[y + Z0]
  static constexpr int ZN = (Z0 - XMIN + 1 + 7) / 8 * 8 + 8;  // (8 more: the core build reads whole words)
  static constexpr int PD = ((D + 31) / 32 + 7) / 8 * 8;      // digits per lane of the recode
  // first position of a short product: its limb 7 QCUT / 32 lies GUARD + 2
  // limbs below the middle limb n of the 2n-limb product (the guard absorbs
  // cancellation in a - x y and leaves room for the determinacy test)
  static constexpr int GUARD = 16;
  static constexpr int QCUT = 32 * ((n - GUARD - 2) / 7);
  static constexpr int tiles(int q) { return (2 * D - 1 - q + 255) / 256; }
  static_assert((long long)D * 4096 < (1ll << 24), "digit sums must stay exact in fp32");
  static_assert(2 * n <= PL, "emitted limbs must cover the product");
  static_assert(32 * PD >= ND, "recode lanes must cover every digit slot");
  static_assert(Z0 - XMAX - 14 >= 0, "staging must cover the lowest Hankel index");
  static_assert(QCUT > 0 && 7 * QCUT / 32 + 2 + GUARD <= n, "the cut must leave the guard below the middle");
  static_assert(7 * QCUT + 18 <= 32 * n, "a short product stays below 2^(64 n)");
  static_assert(tiles(QCUT) <= T, "a short product's limbs fit the row");
};

#include "../../include/hk.h"  // HK_TC_MIN_ROWS

constexpr int TC_STAGES = 4;
constexpr int TC_STAGE_BYTES = 8 * 128 * 16;  // 64 digits x 128 rows of bf16, 8 kgroups of 2 KB
constexpr int TC_THREADS = 320;
constexpr int TC_ROWS = 128;
// tcgen05 instruction descriptor, kind::f16: fp32 D, bf16 A and B, both K-major, N = 256, M = 128
constexpr uint32_t TC_IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((256u >> 3) << 17) | ((128u >> 4) << 24);
constexpr long long TC_WAIT_CYCLES = 4000000000ll;  // about two seconds of SM clock

// ---------------------------------------------------------------------------
// PTX wrappers
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait for the phase of `parity`.  Gives up when *abort is set by
// another role, or after TC_WAIT_CYCLES; then it records its call site
// (1..15) in *abort unless another wait gave up first.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort, int site = 15) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (abort && *abort) return false;
    if (clock64() - t0 > TC_WAIT_CYCLES) {
      if (abort) atomicCAS(const_cast<int*>(abort), 0, site);
      return false;
    }
  }
  return true;
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void fence_barrier_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)), "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                       uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
// the barrier completes one arrival once every tcgen05 operation this thread issued before has completed
__device__ __forceinline__ void tc_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
// 32 consecutive accumulator columns of this warp's 32 lanes: thread i gets
// lane (base lane + i).  The load and its wait are one asm statement, so no
// use of the registers can be scheduled before the data has arrived.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
        "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
        "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
        "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
      : "r"(taddr)
      : "memory");
}

// Shared-memory matrix descriptor, no swizzling: start address, leading
// (K-direction) and stride (M/N-direction) byte offsets between 8 x 16-byte
// core matrices, and the fixed version bits 46..48 = 0b001.
// Two 32-column loads (columns at taddr0 and taddr1) and one wait.
__device__ __forceinline__ void tmem_ld32x2(uint32_t taddr0, uint32_t taddr1, uint32_t (&v)[32], uint32_t (&w)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%64];\n\t"
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%32, %33, %34, %35, %36, %37, %38, %39, %40, %41, %42, %43, %44, %45, %46, %47, "
      "%48, %49, %50, %51, %52, %53, %54, %55, %56, %57, %58, %59, %60, %61, %62, %63}, [%65];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
        "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
        "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
        "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31]),
        "=r"(w[0]), "=r"(w[1]), "=r"(w[2]), "=r"(w[3]), "=r"(w[4]), "=r"(w[5]), "=r"(w[6]), "=r"(w[7]),
        "=r"(w[8]), "=r"(w[9]), "=r"(w[10]), "=r"(w[11]), "=r"(w[12]), "=r"(w[13]), "=r"(w[14]), "=r"(w[15]),
        "=r"(w[16]), "=r"(w[17]), "=r"(w[18]), "=r"(w[19]), "=r"(w[20]), "=r"(w[21]), "=r"(w[22]), "=r"(w[23]),
        "=r"(w[24]), "=r"(w[25]), "=r"(w[26]), "=r"(w[27]), "=r"(w[28]), "=r"(w[29]), "=r"(w[30]), "=r"(w[31])
      : "r"(taddr0), "r"(taddr1)
      : "memory");
}

// acc += sum_u v[31 - u] 2^(7u) for the 32 positions of one group (v holds
// the group's accumulator columns in reversed order), emitting its 7 limbs;
// acc keeps the signed carry into the next limb.  Coefficients are added in
// pairs: |v_u + 128 v_(u+1)| < 129 * 2^24 < 2^31 fits 32 bits, which halves
// the 64-bit additions; a pair spans at most one limb boundary (its
// successor starts 14 bits higher), so at most one limb is emitted after it.
// The 64-bit additions are multiply-adds (acc += w * 2^s, s = 7u mod 32 <= 30
// for even u), which run on the FMA pipe and leave the integer ALU, the
// drain's busiest pipe, to the shifts of the limb emission.
__device__ __forceinline__ void tc_group_limbs(const uint32_t (&v)[32], long long& acc, uint32_t* lim) {
#pragma unroll
  for (int u = 0; u < 32; u += 2) {
    int w;
    asm("mad.lo.s32 %0, %1, 128, %2;"
        : "=r"(w)
        : "r"(__float2int_rn(__uint_as_float(v[30 - u]))), "r"(__float2int_rn(__uint_as_float(v[31 - u]))));
    asm("mad.wide.s32 %0, %1, %2, %0;" : "+l"(acc) : "r"(w), "r"(1 << ((7 * u) & 31)));
    if (((7 * (u + 2)) >> 5) != ((7 * u) >> 5)) {
      lim[(7 * u) >> 5] = (uint32_t)acc;
      acc >>= 32;
    }
  }
}

__device__ __forceinline__ uint64_t tc_sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo & 0x3FFFFu) >> 4) << 16) |
         ((uint64_t)((sbo & 0x3FFFFu) >> 4) << 32) | (1ull << 46);
}

// K-blocks (64 digits) of the tile of positions [qt, qt + 256): [lo, hi]
template <int M>
__device__ __forceinline__ void tc_band(int qt, int& lo, int& hi) {
  constexpr int D = TcShape<M>::D;
  lo = max(0, qt - D + 1) >> 6;
  hi = min(D - 1, qt + 255) >> 6;
}

// The MMAs of K-block kb (ring stage s) for the tile at qt into the accumulator at
// column d_tmem: the 16-digit sub-blocks that meet the tile's band.  first:
// no MMA of the tile issued yet (the first one overwrites the accumulator).
// Returns the new `first`.
//
// The descriptors are formed by addition: the start-address field is the
// low 14 bits (byte address / 16), so the A descriptor of stage s, sub-block
// s4 is adesc0 + 1024 s + 256 s4, and the Hankel descriptor of digit k0 is
// bdesc0 + (k0 - q_hi - XMIN) (core (k0 - q_hi - XMIN) / 8, 128 bytes each),
// which is >= 0 for every sub-block inside the band.  A K-block wholly inside
// the band (all but the band's edges) needs no per-sub-block test: this
// keeps the single issuing thread to a few instructions per MMA.
template <int M>
__device__ __forceinline__ bool tc_issue_kblock(uint32_t d_tmem, uint64_t adesc0, uint64_t bdesc0, int s, int kb,
                                                int qt, bool first) {
  using S = TcShape<M>;
  const int q_lo = qt - S::D + 1, q_hi = qt + 255;  // the tile's digit band
  const uint64_t ad = adesc0 + (uint64_t)(1024 * s);
  const int k00 = 64 * kb;
  const uint64_t bd = bdesc0 + (uint64_t)(int64_t)(k00 - q_hi - S::XMIN);
  if (k00 >= q_lo && k00 + 63 <= q_hi) {
    tc_mma(d_tmem, ad, bd, TC_IDESC, first ? 0u : 1u);
    tc_mma(d_tmem, ad + 256, bd + 16, TC_IDESC, 1u);
    tc_mma(d_tmem, ad + 512, bd + 32, TC_IDESC, 1u);
    tc_mma(d_tmem, ad + 768, bd + 48, TC_IDESC, 1u);
    return false;
  }
#pragma unroll
  for (int s4 = 0; s4 < 4; ++s4) {
    const int k0 = k00 + 16 * s4;
    if (k0 > q_hi || k0 + 15 < q_lo) continue;
    tc_mma(d_tmem, ad + 256 * s4, bd + 16 * s4, TC_IDESC, first ? 0u : 1u);
    first = false;
  }
  return first;
}

// ---------------------------------------------------------------------------
// balanced 7-bit digits of `count` numbers (one warp each), as bf16 bit patterns
//   layout 0: out[row * ND + k]                       (U columns: row = column c)
//   layout 1: out[((k / 8) * pitch + row) * 8 + k % 8] (B rows, kgroup-major)
// number t is mant + (first + t) n, written to row row0 + t
// ---------------------------------------------------------------------------
template <int M>
__device__ __forceinline__ uint32_t tc_raw_digit(const uint32_t* __restrict__ m, int k) {
  constexpr int n = 32 * M;
  const int bit = 7 * k, w = bit >> 5, b = bit & 31;
  uint32_t lo = w < n ? m[w] >> b : 0u;
  if (b > 25 && w + 1 < n) lo |= m[w + 1] << (32 - b);
  return lo & 127u;
}

template <int M>
__global__ void k_tc_digits(const uint32_t* __restrict__ mant, int64_t first, int count, int row0,
                            uint16_t* __restrict__ out, int layout, int pitch) {
  using S = TcShape<M>;
  constexpr int n = S::n;
  const int lane = lane_id();
  const int nw = gridDim.x * (blockDim.x >> 5);
  for (int t = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); t < count; t += nw) {
    const uint32_t* m = mant + (first + t) * (int64_t)n;
    const int k0 = lane * S::PD, k1 = min(k0 + S::PD, S::D);
    // carry out of this lane's digits with carry in 0 and with carry in 1
    uint32_t c0 = 0, c1 = 1;
    for (int k = k0; k < k1; ++k) {
      const uint32_t tk = tc_raw_digit<M>(m, k);
      c0 = (tk + c0) >= 64u;
      c1 = (tk + c1) >= 64u;
    }
    const uint32_t G = __ballot_sync(FULL, c0 != 0);
    const uint32_t P = __ballot_sync(FULL, c1 != 0 && c0 == 0);
    const uint32_t A = G | P;
    const uint32_t C = (A + G) ^ A ^ G;  // bit l: carry into lane l
    uint32_t c = (C >> lane) & 1u;
    const int row = row0 + t;
    for (int g = k0; g < k0 + S::PD && g < S::ND; g += 8) {
      uint32_t w[4];
#pragma unroll
      for (int e = 0; e < 8; e += 2) {
        uint32_t h[2];
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          const int k = g + e + q;
          int d = 0;
          if (k < S::D) {
            const uint32_t s = tc_raw_digit<M>(m, k) + c;
            c = s >= 64u;
            d = (int)s - (c ? 128 : 0);
          }
          h[q] = (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn((float)d));
        }
        w[e >> 1] = h[0] | (h[1] << 16);
      }
      uint4* dst = layout == 0 ? reinterpret_cast<uint4*>(out + (int64_t)row * S::ND + g)
                               : reinterpret_cast<uint4*>(out + ((int64_t)(g >> 3) * pitch + row) * 8);
      *dst = make_uint4(w[0], w[1], w[2], w[3]);
    }
  }
}

// The warp's lanes bring `words` words at p into L2 (one 128-byte line each).
__device__ __forceinline__ void prefetch_l2(const uint32_t* p, int words) {
  for (int l = lane_id(); 32 * l < words; l += 32) asm volatile("prefetch.global.L2 [%0];" ::"l"(p + 32 * l));
}

// ---------------------------------------------------------------------------
// work items: one U column and up to 128 consecutive rows of digit matrix B
// ---------------------------------------------------------------------------
// The operands of one fused update trunc(a - x y) of an item.
struct TcFused {
  const uint32_t* amant;
  int asgn, aexp;
  int sx, ex;
  bool xz;
  int sy, ey;
  bool yz;
  MPVec out;
  int64_t opos;
};

// Step i of Algorithm 1: column cc (c = i + 1 + cc) of the trailing triangle
// (m = N - 1 - i rows and columns) holds rows cc..m-1 (column 0 from row 1:
// the entry (i+1, i+1) is updated first, by the look-ahead launch).  Its rows
// split into 128-row tiles kt; items run from the highest kt down, columns
// ascending, so the short items come last.
template <int M>
struct TcTrail {
  MPVec A, U;
  int N, i;
  __device__ int m() const { return N - 1 - i; }
  __device__ int cols(int kt) const { return (m() - 1 > 128 * kt) ? m() - 128 * kt : 0; }
  __device__ int items() const {
    int s = 0;
    for (int kt = 0; cols(kt) > 0; ++kt) s += cols(kt);
    return s;
  }
  // ucol: the U row (global column c); row0, nrows: rows of the digit matrix (global r)
  __device__ void item(int idx, int& ucol, int& row0, int& nrows) const {
    int kt = 0;
    while (cols(kt + 1) > 0) ++kt;
    for (; kt > 0 && idx >= cols(kt); --kt) idx -= cols(kt);
    const int cc = idx;
    const int rs = cc == 0 ? 1 : cc;
    const int r0 = rs + 128 * kt;
    ucol = i + 1 + cc;
    row0 = i + 1 + r0;
    nrows = min(128, m() - r0);
  }
  __device__ const uint32_t* addend(int ucol, int r) const { return A.mant + tri_pos(N, r, ucol) * (32 * M); }
  __device__ void operands(int ucol, int r, TcFused& f) const {
    constexpr int n = 32 * M;
    const int c = ucol;
    const int64_t apos = tri_pos(N, r, c), bpos = tri_pos(N, r, i);
    f.amant = A.mant + apos * n;
    f.asgn = A.sgn[apos];
    f.aexp = A.exp[apos];
    f.sx = U.sgn[c];
    f.ex = U.exp[c];
    f.xz = U.mant[(int64_t)c * n + n - 1] == 0u;
    f.sy = A.sgn[bpos];
    f.ey = A.exp[bpos];
    f.yz = A.mant[bpos * n + n - 1] == 0u;
    f.out = A;
    f.opos = apos;
  }
  static constexpr bool kRedo = false;
  __device__ uint32_t take_rows(int, int) const { return 0xFFFFFFFFu; }
};

// Step i of Algorithm 1 together with step i of Algorithm 4 (Sec. 4.4):
// X[j][c] = trunc(X[j][c] - L[j][i] X[i][c]) for j > i, c < min(k, i), with
// the same digit rows L[j][i] as the trailing update and X[i][c] as the U
// operand (its digits in U row N + c).  The Algorithm 4 items (column c, 128
// rows of X from i + 1) come first, then the trailing items.
template <int M>
struct TcStep {
  TcTrail<M> tr;
  MPVec X;
  int k;
  __device__ int cols() const { return min(k, tr.i); }
  __device__ int tiles4() const { return (tr.m() + 127) / 128; }
  __device__ int items() const { return cols() * tiles4() + tr.items(); }
  __device__ void item(int idx, int& ucol, int& row0, int& nrows) const {
    const int n4 = cols() * tiles4();
    if (idx >= n4) {
      tr.item(idx - n4, ucol, row0, nrows);
      return;
    }
    const int c = idx % cols(), kt = idx / cols();
    ucol = tr.N + c;
    row0 = tr.i + 1 + 128 * kt;
    nrows = min(128, tr.m() - 128 * kt);
  }
  __device__ const uint32_t* addend(int ucol, int r) const {
    if (ucol < tr.N) return tr.addend(ucol, r);
    return X.mant + ((int64_t)r * k + (ucol - tr.N)) * (32 * M);
  }
  __device__ void operands(int ucol, int r, TcFused& f) const {
    if (ucol < tr.N) {
      tr.operands(ucol, r, f);
      return;
    }
    constexpr int n = 32 * M;
    const int c = ucol - tr.N;
    const int64_t apos = (int64_t)r * k + c, xpos = (int64_t)tr.i * k + c, bpos = tri_pos(tr.N, r, tr.i);
    f.amant = X.mant + apos * n;
    f.asgn = X.sgn[apos];
    f.aexp = X.exp[apos];
    f.sx = X.sgn[xpos];
    f.ex = X.exp[xpos];
    f.xz = X.mant[xpos * n + n - 1] == 0u;
    f.sy = tr.A.sgn[bpos];
    f.ey = tr.A.exp[bpos];
    f.yz = tr.A.mant[bpos * n + n - 1] == 0u;
    f.out = X;
    f.opos = apos;
  }
  static constexpr bool kRedo = false;
  __device__ uint32_t take_rows(int, int) const { return 0xFFFFFFFFu; }
};

// Algorithm 4's copies X[j][i] = -L[j][i] (j > i) of a step i < k, one warp per row.
template <int M>
__global__ void k_alg4_copy(MPVec A, MPVec X, int N, int k, int i) {
  constexpr int n = 32 * M;
  const int nw = gridDim.x * (blockDim.x >> 5);
  for (int j = i + 1 + blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); j < N; j += nw) {
    const int64_t fpos = tri_pos(N, j, i);
    uint32_t v[M];
    load_chunk<M>(A.mant + fpos * n, v);
    const bool zero = __shfl_sync(FULL, v[M - 1], 31) == 0u;
    Result r{zero ? 0 : (A.sgn[fpos] ^ 1), A.exp[fpos], zero};
    store_result<M>(X, (int64_t)j * k + i, r, v);
  }
}

// Elementwise out[e] = trunc(a[e] - x[e] y[e]): item e is U row e with the single digit row e.
template <int M>
struct TcBatch {
  MPVec a, x, y, out;
  int count;
  __device__ int items() const { return count; }
  __device__ void item(int idx, int& ucol, int& row0, int& nrows) const {
    ucol = idx;
    row0 = idx;
    nrows = 1;
  }
  __device__ const uint32_t* addend(int, int r) const { return a.mant + (int64_t)r * (32 * M); }
  __device__ void operands(int ucol, int r, TcFused& f) const {
    constexpr int n = 32 * M;
    const int64_t e = r;
    f.amant = a.mant + e * n;
    f.asgn = a.sgn[e];
    f.aexp = a.exp[e];
    f.sx = x.sgn[e];
    f.ex = x.exp[e];
    f.xz = x.mant[e * n + n - 1] == 0u;
    f.sy = y.sgn[e];
    f.ey = y.exp[e];
    f.yz = y.mant[e * n + n - 1] == 0u;
    f.out = out;
    f.opos = e;
  }
  static constexpr bool kRedo = false;
  __device__ uint32_t take_rows(int, int) const { return 0xFFFFFFFFu; }
};

// Where a launch's short products start, and where it lists the rows it
// could not decide (q > 0 only).
struct TcCut {
  int q;            // first product position formed: a multiple of 32, 0 for the whole product
  int* list;        // items with undecided rows
  int* count;       // entries of list (zero before the launch)
  int* listed;      // per item: 1 once it is in list
  uint32_t* mask;   // per item, 4 words: undecided rows (bit j of word w: row 32 w + j)
  int* total;       // re-run launch: running count of the items it re-ran (profiling)
};

// The re-run of the listed items with whole products: only the rows in the
// item's mask are formed (the others were written by the first launch, in
// place).  Reading a mask resets it, and the listed flag, for the next step.
template <class Base>
struct TcRedo {
  Base base;
  const int* list;
  const int* count;
  int* listed;
  uint32_t* mask;
  static constexpr bool kRedo = true;
  __device__ int items() const { return *count; }
  __device__ void item(int idx, int& ucol, int& row0, int& nrows) const { base.item(list[idx], ucol, row0, nrows); }
  __device__ const uint32_t* addend(int ucol, int r) const { return base.addend(ucol, r); }
  __device__ void operands(int ucol, int r, TcFused& f) const { base.operands(ucol, r, f); }
  // rows of warp q (its 32 TMEM lanes) to form; called once by the whole warp
  __device__ uint32_t take_rows(int idx, int q) const {
    const int id = list[idx];
    const uint32_t m = *reinterpret_cast<volatile uint32_t*>(mask + (size_t)id * 4 + q);
    __syncwarp();
    if (lane_id() == 0) {
      mask[(size_t)id * 4 + q] = 0u;
      if (q == 0) listed[id] = 0;
    }
    return m;
  }
};

// A warp's combine area under IxPad: the addend at logical word 0 and the
// product at logical word n + 32 (both multiples of 32, so that
// sa[IxPad::at(i)] is logical word i and sp[IxPad::at(i)] logical word
// n + 32 + i); the combine frame (3n + 1 words from sa) overlaps the product,
// which combine() reads before its first write.
template <int M>
struct TcComb {
  uint32_t* sa;
  uint32_t* sp;
  __device__ explicit TcComb(uint32_t* base) : sa(base), sp(base + IxPad::at(32 * M + 32)) {}
};

// ---------------------------------------------------------------------------
// shared-memory plan of the product kernel
// ---------------------------------------------------------------------------
template <int M>
struct TcSmem {
  using S = TcShape<M>;
  static constexpr size_t hc = 0;                                            // NHC x 128 B Hankel cores
  static constexpr size_t su = hc + (size_t)S::NHC * 128;                    // ZN bf16: staged U digits
  static constexpr size_t ring = (su + (size_t)S::ZN * 2 + 1023) / 1024 * 1024;  // TC_STAGES x 16 KB
  static constexpr size_t comb = ring + (size_t)TC_STAGES * TC_STAGE_BYTES;  // 8 combine areas
  static constexpr size_t comb_words = (size_t)IxPad::words(3 * S::n + 32);
  static constexpr size_t bars = comb + 8 * comb_words * 4;
  // full, empty (TC_STAGES each); acc_full, acc_empty, hc_full, hc_empty, turn (2 slots each); fin
  static constexpr int NBARS = 2 * TC_STAGES + 5 * 2 + 1;
  static constexpr size_t misc = bars + NBARS * 8;
  static constexpr size_t bytes = misc + 16;
};

// ---------------------------------------------------------------------------
// the product kernel
// ---------------------------------------------------------------------------
// DB: kgroup-major digit matrix, `pitch` rows per kgroup (rows beyond the
// valid ones are zero); DU: U digits, ND per row; P: per block 2 x 128 rows x
// PL limbs of products (a row holds the product's limbs from 7 q / 32 up).
template <int M, class Items>
__global__ void __launch_bounds__(TC_THREADS, 1)
    k_tc_fused(Items items, TcCut cut, const uint16_t* __restrict__ DB, int pitch, const uint16_t* __restrict__ DU,
               uint32_t* __restrict__ P, int* err) {
  using S = TcShape<M>;
  using SM = TcSmem<M>;
  constexpr int n = S::n;
  extern __shared__ __align__(1024) uint8_t tc_smem[];
  if (*err & (ERR_NOT_PD | ERR_TIMEOUT)) return;
  const int n_items = items.items();
  if (cut.total && blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(cut.total, n_items);
  if ((int)blockIdx.x >= n_items) return;  // the re-run launch has a fixed grid
  const int Q = cut.q;                     // tiles start at positions Q + 256 t
  const int TT = S::tiles(Q);
  const int L0 = 7 * Q / 32;               // first limb formed
  const int warp = threadIdx.x >> 5, lane = lane_id();
  uint8_t* hc = tc_smem + SM::hc;
  uint16_t* su = reinterpret_cast<uint16_t*>(tc_smem + SM::su);
  uint8_t* ring = tc_smem + SM::ring;
  uint64_t* bar = reinterpret_cast<uint64_t*>(tc_smem + SM::bars);
  uint64_t* full = bar;                        // [TC_STAGES] stage loaded
  uint64_t* empty = bar + TC_STAGES;           // [TC_STAGES] stage consumed by its MMAs
  uint64_t* acc_full = bar + 2 * TC_STAGES;    // [2] accumulator holds a finished tile
  uint64_t* acc_empty = acc_full + 2;          // [2] accumulator drained
  uint64_t* hc_full = acc_empty + 2;           // Hankel cores of the item built
  uint64_t* su_full = hc_full + 1;             // the next item's U digits copied into su
  uint64_t* hc_empty = hc_full + 2;            // [1] MMAs of the item done ([0] used)
  uint64_t* turn = hc_empty + 2;               // [2] set s has drained every tile of its item (turn[s])
  uint64_t* fin = turn + 2;                    // every MMA of the kernel done
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(tc_smem + SM::misc);
  volatile int* abort = reinterpret_cast<volatile int*>(tc_smem + SM::misc + 4);

  if (threadIdx.x == 0) {
    for (int s = 0; s < TC_STAGES; ++s) {
      mbar_init(full + s, 1);
      mbar_init(empty + s, 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(acc_full + b, 1);
      mbar_init(acc_empty + b, 4);
    }
    mbar_init(hc_full, 1);
    mbar_init(hc_empty, 1);
    mbar_init(su_full, 1);
    mbar_init(turn, 4);
    mbar_init(turn + 1, 4);
    mbar_init(fin, 1);
    *abort = 0;
    fence_barrier_init();
  }
  if (warp == 1) {
    tmem_alloc(tmem_slot, 512);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    // ------------------------------------------------------------ producer
    // Per item: the A-operand stages in the pairs' order, the first
    // TC_STAGES of them issued before the item's Hankel cores are built (the
    // ring is free once the previous item's MMAs have consumed it), and the
    // next item's U digits brought into su by a bulk copy as soon as the
    // cores are built, so that neither the copies nor the staging wait on
    // the build.
    int L = 0;  // stages issued
    int k = 0;
    int su_uses = 0;        // bulk copies into su waited for
    bool su_pending = false;
    bool ok = true;
    // su outside [Z0, Z0 + ND) stays zero: the digits of U past its ends
    for (int z = lane * 8; z < S::ZN; z += 256)
      if (z < S::Z0 || z >= S::Z0 + S::ND) *reinterpret_cast<uint4*>(su + z) = make_uint4(0u, 0u, 0u, 0u);
    __syncwarp();
    auto copy_u = [&](int item) {
      int ucol, row0, nrows;
      items.item(item, ucol, row0, nrows);
      if (lane == 0) {
        mbar_expect_tx(su_full, S::ND * 2);
        bulk_g2s(su + S::Z0, DU + (int64_t)ucol * S::ND, S::ND * 2, su_full);
      }
      su_pending = true;
    };
    // the cores of item k (x = XMIN + 8h, row i of core h = U(-x - i - j), j < 8),
    // then the copy of the next item's digits
    auto build = [&](int it) -> bool {
      if (k > 0 && !mbar_wait(hc_empty, (k - 1) & 1, abort, 1)) return false;
      if (!mbar_wait(su_full, su_uses & 1, abort, 10)) return false;
      ++su_uses;
      su_pending = false;
      const uint32_t* su32 = reinterpret_cast<const uint32_t*>(su);
#pragma unroll 4
      for (int row = lane; row < S::NHC * 8; row += 32) {
        // the row is su[p + 7], su[p + 6], ..., su[p] with p = Z0 - XMIN - row - 7:
        // five aligned words from p rounded down, and a byte permutation
        // that takes the right halves in reverse order
        const int p = S::Z0 - S::XMIN - row - 7;
        const uint32_t* v = su32 + (p >> 1);
        const uint32_t v0 = v[0], v1 = v[1], v2 = v[2], v3 = v[3], v4 = v[4];
        const uint32_t sel = (p & 1) ? 0x3254u : 0x1032u;
        *reinterpret_cast<uint4*>(hc + (size_t)row * 16) =
            make_uint4(__byte_perm(v3, v4, sel), __byte_perm(v2, v3, sel), __byte_perm(v1, v2, sel),
                       __byte_perm(v0, v1, sel));
      }
      fence_proxy_async();
      __syncwarp();
      if (lane == 0) mbar_arrive(hc_full);
      if (it + (int)gridDim.x < n_items) copy_u(it + gridDim.x);
      return true;
    };
    if (ok) copy_u(blockIdx.x);
    for (int it = blockIdx.x; it < n_items && ok; it += gridDim.x, ++k) {
      int ucol, row0, nrows;
      items.item(it, ucol, row0, nrows);
      int issued = 0;
      bool built = false;
      for (int j = 0; 2 * j < TT && ok; ++j) {
        int lo_a, hi_a, lo_b = 1, hi_b = 0;
        tc_band<M>(Q + 512 * j, lo_a, hi_a);
        if (2 * j + 1 < TT) tc_band<M>(Q + 512 * j + 256, lo_b, hi_b);
        const int hi = max(hi_a, hi_b);
        for (int kb = lo_a; kb <= hi; ++kb, ++L, ++issued) {
          if (issued == TC_STAGES && !built) {
            if (!build(it)) {
              ok = false;
              break;
            }
            built = true;
          }
          const int s = L % TC_STAGES;
          if (!mbar_wait(empty + s, ((L / TC_STAGES) & 1) ^ 1, abort, 2)) {
            ok = false;
            break;
          }
          if (lane == 0) {
            mbar_expect_tx(full + s, TC_STAGE_BYTES);
            uint8_t* dst = ring + (size_t)s * TC_STAGE_BYTES;
#pragma unroll 1
            for (int g = 0; g < 8; ++g)
              bulk_g2s(dst + g * 2048, DB + ((int64_t)(kb * 8 + g) * pitch + row0) * 8, 2048, full + s);
          }
          __syncwarp();
        }
      }
      if (ok && !built && !build(it)) ok = false;
    }
    // copies that may still be in flight: wait for them before leaving
    if (su_pending) mbar_wait(su_full, su_uses & 1, nullptr);
    if (*abort) {
      for (int q = max(0, L - TC_STAGES); q < L; ++q) mbar_wait(full + q % TC_STAGES, (q / TC_STAGES) & 1, nullptr);
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      int s = 0, phase = 0, k = 0;   // ring stage and its phase
      int u0 = 0, u1 = 0;            // uses of accumulators 0 and 1
      bool ok = true;
      const uint64_t adesc0 = tc_sdesc(smem_u32(ring), 2048, 128);  // stage 0, sub-block 0
      const uint64_t bdesc0 = tc_sdesc(smem_u32(hc), 128, 128);      // Hankel core 0 (x = XMIN)
      for (int it = blockIdx.x; it < n_items && ok; it += gridDim.x, ++k) {
        if (!mbar_wait(hc_full, k & 1, abort, 3)) break;
        tc_fence_after();
        for (int j = 0; 2 * j < TT && ok; ++j) {
          int lo0, hi0, lo1 = 1, hi1 = 0;
          tc_band<M>(Q + 512 * j, lo0, hi0);
          if (2 * j + 1 < TT) tc_band<M>(Q + 512 * j + 256, lo1, hi1);
          bool f0 = true, f1 = true;
          const int hi_all = max(hi0, hi1);
          for (int kb = lo0; kb <= hi_all; ++kb) {
            if (!mbar_wait(full + s, phase, abort, 4)) {
              ok = false;
              break;
            }
            tc_fence_after();
            if (kb <= hi0) {
              if (f0) {
                if (!mbar_wait(acc_empty, (u0 & 1) ^ 1, abort, 5)) {
                  ok = false;
                  break;
                }
                tc_fence_after();
              }
              f0 = tc_issue_kblock<M>(tmem, adesc0, bdesc0, s, kb, Q + 512 * j, f0);
              if (kb == hi0) {
                tc_commit(acc_full);
                ++u0;
              }
            }
            if (kb >= lo1 && kb <= hi1) {
              if (f1) {
                if (!mbar_wait(acc_empty + 1, (u1 & 1) ^ 1, abort, 6)) {
                  ok = false;
                  break;
                }
                tc_fence_after();
              }
              f1 = tc_issue_kblock<M>(tmem + 256u, adesc0, bdesc0, s, kb, Q + 512 * j + 256, f1);
              if (kb == hi1) {
                tc_commit(acc_full + 1);
                ++u1;
              }
            }
            tc_commit(empty + s);
            if (++s == TC_STAGES) {
              s = 0;
              phase ^= 1;
            }
          }
        }
        tc_commit(hc_empty);
      }
      tc_commit(fin);
      mbar_wait(fin, 0, nullptr);
    }
    __syncwarp();
  } else {
    // ------------------------------------------------------------ drain + combine
    const int set = (warp - 2) >> 2;  // items k = set (mod 2)
    const int q = warp & 3;           // this warp's TMEM lanes 32q .. 32q + 31
    const int mrow = 32 * q + lane;
    const int C0 = (TT + 1) / 2, C1 = TT / 2;  // tiles per item in accumulators 0 and 1
    uint32_t* nb = reinterpret_cast<uint32_t*>(tc_smem + SM::comb) + (size_t)(warp - 2) * SM::comb_words;
    uint32_t* pset = P + (size_t)(blockIdx.x * 2 + set) * TC_ROWS * S::PL;
    bool ok = true;
    for (int k = set, it = blockIdx.x + set * gridDim.x; it < n_items && ok; k += 2, it += 2 * gridDim.x) {
      // The sets drain in item order: a parity wait only tells the current
      // phase from the one before, so set s may wait on the accumulators for
      // item k only once the other set has drained item k - 1.  Each set
      // signals on its own barrier (turn[s], completion j after its j-th item)
      // and waits on the other's: one shared barrier would let a warp that
      // had already arrived wait on the next phase while its set-mates had
      // not completed the current one, and so pass early.
      if (k > 0 && !mbar_wait(turn + (set ^ 1), ((k - 1) >> 1) & 1, abort, 7)) break;
      int u0 = k * C0, u1 = k * C1;  // uses of accumulators 0 and 1 before this item
      uint32_t* prow = pset + (size_t)mrow * S::PL;
      long long acc = 0;  // signed carry into the next limb
      for (int t = 0; t < TT; ++t) {
        const int b = t & 1;
        if (!mbar_wait(acc_full + b, (b ? u1 : u0) & 1, abort, 8 + b)) {
          ok = false;
          break;
        }
        tc_fence_after();
        uint32_t lim[56];
        // Two independent chains: the tile's low half (groups 0..3, limbs
        // 0..27, starting from the carry of the previous tile) and its high
        // half (groups 4..7, limbs 28..55, from zero); the low half's carry
        // is then added into the high half.  Positions Q + 256t + 32g + u
        // are columns 255 - 32g - u; the tile's limbs are L0 + 56t + w.
        long long acc_hi = 0;
        const uint32_t tcol = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(b * 256);
#pragma unroll
        for (int g = 0; g < 4; ++g) {
          uint32_t va[32], vb[32];
          tmem_ld32x2(tcol + (uint32_t)(224 - 32 * g), tcol + (uint32_t)(96 - 32 * g), va, vb);
          tc_group_limbs(va, acc, lim + 7 * g);
          tc_group_limbs(vb, acc_hi, lim + 28 + 7 * g);
        }
#pragma unroll
        for (int w = 28; w < 56; ++w) {
          const long long x = (long long)lim[w] + acc;
          lim[w] = (uint32_t)x;
          acc = x >> 32;
        }
        acc += acc_hi;
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(acc_empty + b);
        if (b) ++u1;
        else ++u0;
#pragma unroll
        for (int w = 0; w < 14; ++w)
          reinterpret_cast<uint4*>(prow + 56 * t)[w] = make_uint4(lim[4 * w], lim[4 * w + 1], lim[4 * w + 2], lim[4 * w + 3]);
        // the product (short or whole) is in [0, 2^(64 n)): the limbs past
        // 2n and the last carry are zero
        uint32_t stray = (t == TT - 1) ? (uint32_t)(acc != 0) : 0u;
        if (L0 + 56 * t + 55 >= 2 * n) {  // only the last tiles reach limb 2n
#pragma unroll
          for (int w = 0; w < 56; ++w)
            if (L0 + 56 * t + w >= 2 * n) stray |= lim[w];
        }
        if (stray) atomicOr(err, ERR_LOOP);
      }
      if (!ok) break;
      __syncwarp();  // this warp's product rows are written
      if (lane == 0) mbar_arrive(turn + set);
      // trunc(a - P) for this warp's rows, one row at a time with the whole warp
      int ucol, row0, nrows;
      items.item(it, ucol, row0, nrows);
      const uint32_t rows = items.take_rows(it, q);
      uint32_t undecided = 0;
      // the next row's addend and product limbs are brought into L2 while
      // this one is formed: one row's loads are otherwise all latency
      if (rows & 1u) {
        prefetch_l2(items.addend(ucol, row0 + 32 * q), n);
        prefetch_l2(pset + (size_t)(32 * q) * S::PL, 2 * n - L0);
      }
      for (int j = 0; j < 32 && 32 * q + j < nrows; ++j) {
        if (!((rows >> j) & 1u)) continue;
        const int mm = 32 * q + j;
        if (j + 1 < 32 && 32 * q + j + 1 < nrows && ((rows >> (j + 1)) & 1u)) {
          prefetch_l2(items.addend(ucol, row0 + mm + 1), n);
          prefetch_l2(pset + (size_t)(mm + 1) * S::PL, 2 * n - L0);
        }
        TcFused f;
        items.operands(ucol, row0 + mm, f);
        const uint32_t* pr = pset + (size_t)mm * S::PL;
        TcComb<M> sm(nb);
        const bool p_zero = f.xz || f.yz;
        // every load of the row in flight at once, then the stores to shared memory
        uint32_t av[M], pv[2 * M];
        load_chunk<M>(f.amant, av);
        if (!p_zero) {
#pragma unroll
          for (int w = 0; w < 2 * M; ++w) {
            const int l = 32 * w + lane - L0;  // limbs below L0 are zero in a short product
            pv[w] = l >= 0 ? __ldcg(pr + l) : 0u;
          }
#pragma unroll
          for (int w = 0; w < 2 * M; ++w) sm.sp[IxPad::at(32 * w + lane)] = pv[w];
        }
#pragma unroll
        for (int w = 0; w < M; ++w) sm.sa[IxPad::at(lane * M + w)] = av[w];
        __syncwarp();
        const bool a_zero = sm.sa[IxPad::at(n - 1)] == 0u;
        uint32_t o[M];
        // A short product's difference on a frame of n + 32 limbs whose top
        // is just above the higher of the two leading limbs: frame limb 0 is
        // the product's limb F0 = max(n - 32, d - 32), d = ea - ep (the
        // addend's limb 0 in the product's limbs).  Limbs of either operand
        // below F0 are left out like the omitted terms: all three together
        // are below 2^(32 F0 + 1) + 2^(32 L0 + 18), under frame limb
        // max(L0 - F0, 0) + 2.  A product wholly below the addend (d > 2n)
        // goes through the exact stand-in of sub_product instead.
        // A product wholly below the addend (d > 2n) changes the truncated
        // result only through its sign (combine()'s stand-in: a single 1
        // two limbs below the addend's last limb gives the same result), on
        // the same frame with the test off.  The re-run launch forms whole
        // products and takes the general frame (sub_product).
        const long long d = (long long)f.aexp - (long long)(f.ex + f.ey);
        Result res;
        if constexpr (!Items::kRedo) {
          if (p_zero) {  // the result is a itself
#pragma unroll
            for (int w = 0; w < M; ++w) o[w] = sm.sa[IxPad::at(lane * M + w)];
            __syncwarp();
            res.zero = a_zero;
            res.sgn = a_zero ? 0 : f.asgn;
            res.exp = a_zero ? 0 : f.aexp;
          } else if (d <= 2 * n) {
            const int F0 = (int)max((long long)n - 32, (a_zero ? (long long)n : d) - 32);
            const bool a_out = a_zero || d - F0 < -(long long)n;  // the addend wholly below the frame
            res = combine_narrow<M + 1, M, IxPad>(Staged{sm.sa, a_out ? 0 : (int)(d - F0), a_out ? 0 : n},
                                                  f.asgn, Staged{sm.sp, -F0, 2 * n}, f.sx ^ f.sy ^ 1,
                                                  f.ex + f.ey + F0, sm.sa, o, max(L0 - F0, 0) + 2);
          } else {
            res = combine_narrow<M + 1, M, IxPad>(Staged{sm.sa, 32, n}, f.asgn, Staged{nullptr, 30, 1},
                                                  f.sx ^ f.sy ^ 1, f.aexp - 32, sm.sa, o, -1);
          }
        } else {
          res = sub_product<M, IxPad>(sm, f.asgn, f.aexp, a_zero, f.sx ^ f.sy, f.ex + f.ey, p_zero, o);
        }
        if (res.amb) undecided |= 1u << j;
        else store_result<M>(f.out, f.opos, res, o);
        __syncwarp();
      }
      if (undecided && lane == 0) {
        cut.mask[(size_t)it * 4 + q] = undecided;
        if (atomicExch(cut.listed + it, 1) == 0) cut.list[atomicAdd(cut.count, 1)] = it;
      }
    }
  }

  __syncthreads();
  if (threadIdx.x == 0 && *abort) atomicOr(err, ERR_TIMEOUT | ((*abort & 15) << 8));
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, 512);
  }
}

}  // namespace hk
