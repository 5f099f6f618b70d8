// Kernels of the factorisation: elementwise primitives, Hankel assembly,
// pivot reciprocal, column scale (B_i) and the trailing rank-1 update
// (Algorithm 1, Sec. 4.3).
#pragma once
#include "common.cuh"
#include "mp_div.cuh"
#include "ntt.cuh"

namespace hk {

template <int M>
__device__ __forceinline__ void load_hdr(const MPVec& v, int64_t i, int& s, int& e) {
  s = v.sgn[i];
  e = v.exp[i];
}

template <int M>
__device__ __forceinline__ void store_result(const MPVec& v, int64_t i, const Result& r, const uint32_t (&out)[M]) {
  constexpr int n = 32 * M;
  store_chunk<M>(v.mant + i * n, out);
  if (lane_id() == 0) {
    v.sgn[i] = r.sgn;
    v.exp[i] = r.exp;
  }
}

// One fused operation out = trunc_n(a - x*y) for a warp; x in registers (xc),
// y staged in sm.ys, a staged in sm.sa.
template <int M>
__device__ __forceinline__ Result fused_staged(const WarpSmem<M>& sm, const uint32_t (&xc)[M], int sx, int ex,
                                               int sy, int ey, int sa_sgn, int ea, uint32_t (&out)[M]) {
  constexpr int n = 32 * M;
  const bool x_zero = __shfl_sync(FULL, xc[M - 1], 31) == 0u;
  const bool y_zero = sm.ys[n - 1] == 0u;
  const bool a_zero = sm.sa[n - 1] == 0u;
  const bool p_zero = x_zero || y_zero;
  if (!p_zero) {
    uint32_t lo[M], hi[M];
    warp_mul<M>(xc, sm.ys, sm.sp, lo, hi);
    stage_product<M>(sm.sp, lo, hi);
    __syncwarp();
  }
  return sub_product<M>(sm, sa_sgn, ea, a_zero, sx ^ sy, ex + ey, p_zero, out);
}

// ---------------------------------------------------------------------------
// elementwise primitives (used by the format tests and exported as-is)
// ---------------------------------------------------------------------------
template <int M>
__global__ void k_fused_batch(MPVec a, MPVec x, MPVec y, MPVec out, int64_t count) {
  constexpr int n = 32 * M;
  extern __shared__ uint32_t smem[];
  const int wib = threadIdx.x >> 5;
  WarpSmem<M> sm(smem + wib * WarpSmem<M>::words);
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t e = (int64_t)blockIdx.x * (blockDim.x >> 5) + wib; e < count; e += nw) {
    copy_to_smem<M>(sm.ys, y.mant + e * n);
    copy_to_smem<M>(sm.sa, a.mant + e * n);
    uint32_t xc[M];
    load_chunk<M>(x.mant + e * n, xc);
    __syncwarp();
    uint32_t o[M];
    const Result r = fused_staged<M>(sm, xc, x.sgn[e], x.exp[e], y.sgn[e], y.exp[e], a.sgn[e], a.exp[e], o);
    store_result<M>(out, e, r, o);
    __syncwarp();
  }
}

// out = trunc_n(a / d), each warp forming its own reciprocal (test primitive).
template <int M>
__global__ void k_div_batch(MPVec a, MPVec d, MPVec out, int64_t count, int* err) {
  constexpr int n = 32 * M;
  extern __shared__ uint32_t smem[];
  const int wib = threadIdx.x >> 5;
  uint32_t* ys = smem + wib * (4 * n + 4);
  uint32_t* yt = ys + n;
  uint32_t* sp = yt + n;
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t e = (int64_t)blockIdx.x * (blockDim.x >> 5) + wib; e < count; e += nw) {
    uint32_t dc[M], ac[M], R[M], q[M];
    load_chunk<M>(d.mant + e * n, dc);
    load_chunk<M>(a.mant + e * n, ac);
    const bool d_zero = __shfl_sync(FULL, dc[M - 1], 31) == 0u;
    const bool a_zero = __shfl_sync(FULL, ac[M - 1], 31) == 0u;
    if (d_zero || a_zero) {
      if (d_zero && lane_id() == 0) atomicOr(err, ERR_ARG);
#pragma unroll
      for (int k = 0; k < M; ++k) q[k] = 0;
      Result r{0, 0, true};
      store_result<M>(out, e, r, q);
      continue;
    }
    int sh, t;
    warp_recip<M>(dc, ys, sp, R, sh, err);
#pragma unroll
    for (int k = 0; k < M; ++k) ys[lane_id() * M + k] = R[k];
    __syncwarp();
    warp_quot<M>(ac, dc, ys, sh, yt, sp, q, t, err);
    Result r;
    r.zero = false;
    r.sgn = a.sgn[e] ^ d.sgn[e];
    r.exp = a.exp[e] - d.exp[e] - t;
    store_result<M>(out, e, r, q);
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------
// Hankel assembly: A[r][c] = mu_{r+c} (packed lower triangle)
// ---------------------------------------------------------------------------
template <int M>
__global__ void k_assemble(MPVec mu, MPVec A, int N) {
  constexpr int n = 32 * M;
  const int64_t total = (int64_t)N * (N + 1) / 2;
  const int64_t q4 = n / 4;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < total * q4; g += stride) {
    const int64_t pos = g / q4, w = g % q4;
    // column of pos: largest c with tri_pos(N, c, c) <= pos
    int64_t c = trail_col(N, pos);
    const int64_t r = c + (pos - trail_off(N, c));
    const int64_t s = r + c;
    reinterpret_cast<uint4*>(A.mant + pos * n)[w] = reinterpret_cast<const uint4*>(mu.mant + s * n)[w];
    if (w == 0) {
      A.sgn[pos] = mu.sgn[s];
      A.exp[pos] = mu.exp[s];
    }
  }
}

// ---------------------------------------------------------------------------
// pivot reciprocal (one warp): R_i for d_i = A[i][i]
// ---------------------------------------------------------------------------
// Products of the reciprocal's full-width steps through transforms held in
// shared memory: fd = F(D') (formed once), fr = F(R) (scaled), fx = F(x).
template <int M>
struct RecipNtt {
  NttConst nc;
  uint32_t *fd, *fr, *fx, *nb, *stage;
  bool have_d;
  __device__ bool wide(int w) const { return w == 32 * M; }
  template <int MM>
  __device__ void set_r(const uint32_t* ys) {
    warp_ntt_number<M>(ys, nb, fr, nc, true);
    __syncwarp();
  }
  __device__ void transform(const uint32_t (&x)[M], uint32_t* out) {
#pragma unroll
    for (int k = 0; k < M; ++k) stage[lane_id() * M + k] = x[k];
    __syncwarp();
    warp_ntt_number<M>(stage, nb, out, nc, false);
    __syncwarp();
  }
  template <int MM>
  __device__ void mul_d(const uint32_t (&dp)[M], uint32_t (&lo)[M], uint32_t (&hi)[M]) {
    if (!have_d) {
      transform(dp, fd);
      have_d = true;
    }
    warp_mul_ntt<M, false, false>(fd, fr, nb, nc, lo, hi);
    __syncwarp();
  }
  template <int MM>
  __device__ void mul_r(const uint32_t (&x)[M], uint32_t (&lo)[M], uint32_t (&hi)[M]) {
    transform(x, fx);
    warp_mul_ntt<M, false, false>(fx, fr, nb, nc, lo, hi);
    __syncwarp();
  }
};

// shared-memory words of k_recip_pivot: ys, sp (schoolbook), and with NTT
// products a staging area, three transforms and the product's work area
template <int M>
__host__ __device__ constexpr size_t recip_pivot_words(bool ntt) {
  return ntt ? (size_t)4 * (32 * M) + 4 + 3 * (size_t)NTT_Q * ntt_len(32 * M) + (size_t)NTT_Q * ntt_stride(ntt_len(32 * M))
             : (size_t)3 * (32 * M) + 4;
}

// rec: n limbs of R, then (sh) in rec_meta[0].  use_ntt: the full-width
// steps take NTT products (shared memory of recip_pivot_words(true)).
template <int M>
__global__ void k_recip_pivot(MPVec A, int N, int i, uint32_t* rec, int* rec_meta, int* err, NttConst nc,
                              int use_ntt) {
  constexpr int n = 32 * M;
  extern __shared__ uint32_t smem[];
  uint32_t* ys = smem;
  uint32_t* sp = smem + n;
  const int64_t pos = tri_pos(N, i, i);
  uint32_t dc[M], R[M];
  load_chunk<M>(A.mant + pos * n, dc);
  const bool zero = __shfl_sync(FULL, dc[M - 1], 31) == 0u;
  if (zero || A.sgn[pos] != 0) {
    if (lane_id() == 0) atomicOr(err, ERR_NOT_PD);
    return;
  }
  int sh;
  if (use_ntt) {
    constexpr int L = ntt_len(n);
    uint32_t* stage = smem + 3 * n + 4;
    uint32_t* fd = stage + n;
    RecipNtt<M> pol{nc, fd, fd + NTT_Q * L, fd + 2 * NTT_Q * L, fd + 3 * NTT_Q * L, stage, false};
    warp_recip_p<M>(dc, ys, sp, R, sh, err, pol);
  } else {
    warp_recip<M>(dc, ys, sp, R, sh, err);
  }
  store_chunk<M>(rec, R);
  if (lane_id() == 0) rec_meta[0] = sh;
}

// ---------------------------------------------------------------------------
// column scale of step i: U[r] = A[r][i];  A[r][i] = B_i[r] = trunc(A[r][i] / d_i)
// ---------------------------------------------------------------------------
template <int M>
__global__ void k_scale(MPVec A, MPVec U, int N, int i, const uint32_t* rec, const int* rec_meta, int* err) {
  constexpr int n = 32 * M;
  extern __shared__ uint32_t smem[];
  const int wib = threadIdx.x >> 5;
  uint32_t* ys = smem + wib * (4 * n + 4);
  uint32_t* yt = ys + n;
  uint32_t* sp = yt + n;
  if (*err & ERR_NOT_PD) return;
  const int64_t dpos = tri_pos(N, i, i);
  uint32_t dc[M], R[M];
  load_chunk<M>(A.mant + dpos * n, dc);
  load_chunk<M>(rec, R);
  const int sh = rec_meta[0];
  const int ed = A.exp[dpos];
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t r = i + 1 + (int64_t)blockIdx.x * (blockDim.x >> 5) + wib; r < N; r += nw) {
    const int64_t pos = tri_pos(N, r, i);
    uint32_t ac[M], q[M];
    load_chunk<M>(A.mant + pos * n, ac);
    const int sa = A.sgn[pos], ea = A.exp[pos];
    store_chunk<M>(U.mant + r * n, ac);
    if (lane_id() == 0) {
      U.sgn[r] = sa;
      U.exp[r] = ea;
    }
    const bool a_zero = __shfl_sync(FULL, ac[M - 1], 31) == 0u;
    Result res;
    if (a_zero) {
#pragma unroll
      for (int k = 0; k < M; ++k) q[k] = 0;
      res = Result{0, 0, true};
    } else {
#pragma unroll
      for (int k = 0; k < M; ++k) ys[lane_id() * M + k] = R[k];
      __syncwarp();
      int t;
      warp_quot<M>(ac, dc, ys, sh, yt, sp, q, t, err);
      res = Result{sa, ea - ed - t, false};
    }
    store_result<M>(A, pos, res, q);
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------
// trailing update of step i (Algorithm 1 inner loops, Sec. 4.3):
//   A[r][c] = trunc(A[r][c] - U[c] * B_i[r]),  i < c <= r < N
// U[c] = A[c][i] before scaling (saved by k_scale), B_i[r] = A[r][i] after.
// One warp per entry; entries enumerated column by column so consecutive
// warps share U[c].
// ---------------------------------------------------------------------------
#ifndef HK_TRAIL_MIN_BLOCKS
#define HK_TRAIL_MIN_BLOCKS 3  // resident blocks of 4 warps per SM the register budget is sized for
#endif
template <int M>
__global__ void __launch_bounds__(128, HK_TRAIL_MIN_BLOCKS) k_trailing(MPVec A, MPVec U, int N, int i, int64_t t0, int64_t t1,
                                                   const int* err) {
  constexpr int n = 32 * M;
  extern __shared__ uint32_t smem[];
  const int wib = threadIdx.x >> 5;
  WarpSmem<M> sm(smem + wib * WarpSmem<M>::words);
  if (*err & ERR_NOT_PD) return;
  const int64_t m = N - 1 - i;
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t t = t0 + (int64_t)blockIdx.x * (blockDim.x >> 5) + wib; t < t1; t += nw) {
    const int64_t cc = trail_col(m, t);
    const int64_t c = i + 1 + cc;
    const int64_t r = c + (t - trail_off(m, cc));
    const int64_t apos = tri_pos(N, r, c);
    const int64_t bpos = tri_pos(N, r, i);
    copy_to_smem<M>(sm.ys, A.mant + bpos * n);
    copy_to_smem<M>(sm.sa, A.mant + apos * n);
    uint32_t xc[M];
    load_chunk<M>(U.mant + c * n, xc);
    __syncwarp();
    uint32_t o[M];
    const Result res = fused_staged<M>(sm, xc, U.sgn[c], U.exp[c], A.sgn[bpos], A.exp[bpos], A.sgn[apos],
                                       A.exp[apos], o);
    store_result<M>(A, apos, res, o);
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------
// NTT variants: products through the stored transforms (ntt.cuh)
// ---------------------------------------------------------------------------
// Transforms of count consecutive numbers src[first + t] into out[t * 3L ..].
template <int M>
__global__ void k_ntt_fwd(MPVec src, int64_t first, int count, uint32_t* __restrict__ out, NttConst nc, int scaled) {
  constexpr int n = 32 * M;
  extern __shared__ uint32_t smem[];
  const int wib = threadIdx.x >> 5;
  uint32_t* buf = smem + wib * ntt_stride(nc.L);
  const int nw = gridDim.x * (blockDim.x >> 5);
  for (int t = blockIdx.x * (blockDim.x >> 5) + wib; t < count; t += nw)
    warp_ntt_number<M>(src.mant + (first + t) * n, buf, out + (size_t)t * NTT_Q * nc.L, nc, scaled != 0);
}

// trunc(a - x*y) with the product from stored transforms fx (unscaled) and fy
// (scaled); nb: this warp's 3 ntt_stride(L) words of shared memory (reused for the combine).
// stage_a(sa) writes the addend's n limbs into sa under IxPad.  X_RO: fx is
// read-only for the kernel (see warp_mul_ntt).
template <int M, class StageA, bool X_RO = true>
__device__ __forceinline__ Result fused_ntt_core(uint32_t* nb, const NttConst& nc, const uint32_t* fx, bool x_zero,
                                                 int sx, int ex, const uint32_t* fy, bool y_zero, int sy, int ey,
                                                 StageA stage_a, int sa_sgn, int ea, uint32_t (&out)[M]) {
  constexpr int n = 32 * M;
  static_assert(WarpSmemPad<M>::words <= NTT_Q * ntt_stride(ntt_len(n)), "combine frame exceeds the NTT buffer");
  const bool p_zero = x_zero || y_zero;
  uint32_t lo[M], hi[M];
  if (!p_zero) {
    warp_mul_ntt<M, X_RO>(fx, fy, nb, nc, lo, hi);
    __syncwarp();  // every lane has read the residues before the region is reused
  }
  WarpSmemPad<M> sm(nb);
  if (!p_zero) stage_product<M, IxPad>(sm.sp, lo, hi);
  stage_a(sm.sa);
  __syncwarp();
  const bool a_zero = sm.sa[IxPad::at(n - 1)] == 0u;
  return sub_product<M, IxPad>(sm, sa_sgn, ea, a_zero, sx ^ sy, ex + ey, p_zero, out);
}

// the addend from global memory
template <int M>
__device__ __forceinline__ Result fused_ntt(uint32_t* nb, const NttConst& nc, const uint32_t* fx, bool x_zero, int sx,
                                            int ex, const uint32_t* fy, bool y_zero, int sy, int ey,
                                            const uint32_t* amant, int sa_sgn, int ea, uint32_t (&out)[M]) {
  return fused_ntt_core<M>(nb, nc, fx, x_zero, sx, ex, fy, y_zero, sy, ey,
                           [&](uint32_t* sa) { copy_to_smem<M, IxPad>(sa, amant); }, sa_sgn, ea, out);
}

// Blocks of HK_NTT_TRAIL_WARPS warps, two resident per SM: at 768 limbs a warp
// needs 19 KB of shared memory, so 2 x 6 warps fill the SM's 228 KB.
#ifndef HK_NTT_TRAIL_WARPS
#define HK_NTT_TRAIL_WARPS 6
#endif

// Column scale of step i with NTT products: U[r] = A[r][i] and
// A[r][i] = B_i[r] = trunc(A[r][i] / d_i), the same exact quotient as k_scale
// (warp_quot), with its two products A R and Q~ D from transforms.
// FU[r - i - 1] = F(A[r][i]) (unscaled; the trailing update reuses it),
// FRD = F(R) then F(D) (scaled), FQ[r - i - 1]: scratch for F(Q~) (the slot
// that F(B_i[r]) takes afterwards).
// Blocks of HK_SCALE_WARPS warps, two per SM: the exact quotient's
// correction holds several n-limb chunks at once, and the 255 registers a
// thread gets at that size keep it out of local memory.
#ifndef HK_SCALE_WARPS
#define HK_SCALE_WARPS 4
#endif
template <int M>
__global__ void __launch_bounds__(32 * HK_SCALE_WARPS, 2)
    k_scale_ntt(MPVec A, MPVec U, int N, int i, const uint32_t* __restrict__ FU, const uint32_t* __restrict__ FRD,
                uint32_t* FQ, const int* rec_meta, NttConst nc, int* err) {
  constexpr int n = 32 * M;
  extern __shared__ uint32_t smem[];
  const int wib = threadIdx.x >> 5;
  uint32_t* nb = smem + (size_t)wib * NTT_Q * ntt_stride(nc.L);
  uint32_t* qs = nb + ntt_stride(nc.L) + 32;  // Q~ staged for its transform (nb[0, stride) is the work area)
  if (*err & ERR_NOT_PD) return;
  const size_t per = (size_t)NTT_Q * nc.L;
  const int lane = lane_id();
  const int64_t dpos = tri_pos(N, i, i);
  uint32_t dc[M];
  load_chunk<M>(A.mant + dpos * n, dc);
  const int sh = rec_meta[0];
  const int ed = A.exp[dpos];
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t r = i + 1 + (int64_t)blockIdx.x * (blockDim.x >> 5) + wib; r < N; r += nw) {
    const int64_t pos = tri_pos(N, r, i);
    uint32_t ac[M], q[M];
    load_chunk<M>(A.mant + pos * n, ac);
    const int sa = A.sgn[pos], ea = A.exp[pos];
    store_chunk<M>(U.mant + r * n, ac);
    if (lane == 0) {
      U.sgn[r] = sa;
      U.exp[r] = ea;
    }
    const bool a_zero = __shfl_sync(FULL, ac[M - 1], 31) == 0u;
    Result res;
    if (a_zero) {
#pragma unroll
      for (int k = 0; k < M; ++k) q[k] = 0;
      res = Result{0, 0, true};
    } else {
      const int t = (ncmp<M>(ac, dc) >= 0) ? n - 1 : n;
      // Q~ = floor(A R / 2^shift), shift = 64n - 1 - 32t - sh
      uint32_t plo[M], phi[M];
      warp_mul_ntt<M>(FU + (size_t)(r - i - 1) * per, FRD, nb, nc, plo, phi);
      __syncwarp();
      const int shift = 64 * n - 1 - 32 * t - sh;
#pragma unroll
      for (int k = 0; k < M; ++k) {
        nb[lane * M + k] = plo[k];
        nb[n + lane * M + k] = phi[k];
      }
      if (lane == 0) nb[2 * n] = 0;
      __syncwarp();
      read_shifted<M>(nb, shift >> 5, shift & 31, q);
      __syncwarp();
      // Q~ D through F(Q~) (written and read back by this warp)
#pragma unroll
      for (int k = 0; k < M; ++k) qs[lane * M + k] = q[k];
      __syncwarp();
      uint32_t* fq = FQ + (size_t)(r - i - 1) * per;
      warp_ntt_number<M>(qs, nb, fq, nc, false);
      __syncwarp();
      uint32_t qlo[M], qhi[M];
      warp_mul_ntt<M, false>(fq, FRD + per, nb, nc, qlo, qhi);
      __syncwarp();
      quot_fix<M>(ac, dc, t, qlo, qhi, nb, q, err);
      res = Result{sa, ea - ed - t, false};
    }
    store_result<M>(A, pos, res, q);
    __syncwarp();
  }
}

// Transforms (scaled) of the pivot's reciprocal R (n raw limbs) and of the
// pivot D = A[dpos]: warp 0 and warp 1 of one block.
template <int M>
__global__ void k_ntt_pivot(const uint32_t* __restrict__ rec, MPVec A, int64_t dpos, uint32_t* __restrict__ FRD,
                            NttConst nc) {
  constexpr int n = 32 * M;
  extern __shared__ uint32_t smem[];
  const int wib = threadIdx.x >> 5;
  if (wib > 1) return;
  uint32_t* buf = smem + wib * ntt_stride(nc.L);
  warp_ntt_number<M>(wib == 0 ? rec : A.mant + dpos * n, buf, FRD + (size_t)wib * NTT_Q * nc.L, nc, true);
}

// The trailing update of step i with NTT products.  FU[c - i - 1], FB[r - i - 1]
// hold the transforms of U[c] (unscaled) and B_i[r] (scaled) for this step.
// Blocks of HK_NTT_TRAIL_WARPS warps (see k_scale_ntt above).
template <int M>
__global__ void __launch_bounds__(32 * HK_NTT_TRAIL_WARPS, 2) k_trailing_ntt(MPVec A, MPVec U, const uint32_t* __restrict__ FU,
                                                      const uint32_t* __restrict__ FB, int N, int i, int64_t t0,
                                                      int64_t t1, NttConst nc, const int* err) {
  constexpr int n = 32 * M;
  extern __shared__ uint32_t smem[];
  const int wib = threadIdx.x >> 5;
  uint32_t* nb = smem + (size_t)wib * NTT_Q * ntt_stride(nc.L);
  if (*err & ERR_NOT_PD) return;
  const int64_t m = N - 1 - i;
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t t = t0 + (int64_t)blockIdx.x * (blockDim.x >> 5) + wib; t < t1; t += nw) {
    const int64_t cc = trail_col(m, t);
    const int64_t c = i + 1 + cc;
    const int64_t r = c + (t - trail_off(m, cc));
    const int64_t apos = tri_pos(N, r, c);
    const int64_t bpos = tri_pos(N, r, i);
    const bool x_zero = U.mant[c * n + n - 1] == 0u;
    const bool y_zero = A.mant[bpos * n + n - 1] == 0u;
    uint32_t o[M];
    const Result res = fused_ntt<M>(nb, nc, FU + (size_t)cc * NTT_Q * nc.L, x_zero, U.sgn[c], U.exp[c],
                                    FB + (size_t)(r - i - 1) * NTT_Q * nc.L, y_zero, A.sgn[bpos], A.exp[bpos],
                                    A.mant + apos * n, A.sgn[apos], A.exp[apos], o);
    store_result<M>(A, apos, res, o);
    __syncwarp();
  }
}

// Elementwise trunc(a - x*y) with NTT products (FX, FY: transforms of x, y).
template <int M>
__global__ void k_fused_batch_ntt(MPVec a, MPVec x, MPVec y, const uint32_t* __restrict__ FX,
                                  const uint32_t* __restrict__ FY, MPVec out, int64_t count, NttConst nc) {
  constexpr int n = 32 * M;
  extern __shared__ uint32_t smem[];
  const int wib = threadIdx.x >> 5;
  uint32_t* nb = smem + (size_t)wib * NTT_Q * ntt_stride(nc.L);
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t e = (int64_t)blockIdx.x * (blockDim.x >> 5) + wib; e < count; e += nw) {
    uint32_t o[M];
    const Result res = fused_ntt<M>(nb, nc, FX + (size_t)e * NTT_Q * nc.L, x.mant[e * n + n - 1] == 0u, x.sgn[e],
                                    x.exp[e], FY + (size_t)e * NTT_Q * nc.L, y.mant[e * n + n - 1] == 0u, y.sgn[e],
                                    y.exp[e], a.mant + e * n, a.sgn[e], a.exp[e], o);
    store_result<M>(out, e, res, o);
    __syncwarp();
  }
}

}  // namespace hk
