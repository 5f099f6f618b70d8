// Kernels after the factorisation: Algorithm 4 (first k columns of L^{-1}),
// the k x k block of H^{-1}, the block eigenvalues and the gradient.  They are
// built from a few warp-per-number kernels:
//   k_chain     acc <- acc -/+ x*y along affine index maps (dot products,
//               matrix products, sums), one rounding per step
//   k_recip_tab Newton reciprocals of a list of divisors
//   k_quot      exactly truncated quotients a/d using those reciprocals
// plus per-step kernels for Algorithm 4 and the back substitution.
#pragma once
#include <climits>

#include "k_ldlt.cuh"

namespace hk {

// One chain: out = init (or 0) followed by len steps acc = trunc(acc -/+ x[x0 + q sx] * y[y0 + q sy]).
struct ChainTask {
  int64_t out, init, x0, y0;
  int32_t sx, sy, len, flags;
};
enum ChainFlags : int32_t {
  CH_ZERO_INIT = 1,   // start from 0 instead of INIT[init]
  CH_ADD = 2,         // acc + x*y instead of acc - x*y
  CH_NEG_OUT = 4,     // store -acc
  CH_NEG_INIT = 8,    // start from -INIT[init]
};

// Quotient task: out = trunc(a[ia] / d[id]) with reciprocal slot rid.
struct QuotTask {
  int64_t out, ia, id, rid;
  int32_t neg, pad;
};

// The warp runs one fused step with the accumulator staged in sm.sa
// (header in registers); x read from global into registers, y into sm.ys.
template <int M>
__device__ __forceinline__ void chain_step(const WarpSmem<M>& sm, int& as, int& ae, const MPVec& X, int64_t ix,
                                           const MPVec& Y, int64_t iy, bool add) {
  constexpr int n = 32 * M;
  uint32_t xc[M], out[M];
  load_chunk<M>(X.mant + ix * n, xc);
  copy_to_smem<M>(sm.ys, Y.mant + iy * n);
  const int sx = X.sgn[ix], ex = X.exp[ix];
  const int sy = Y.sgn[iy] ^ (add ? 1 : 0), ey = Y.exp[iy];
  __syncwarp();
  const Result r = fused_staged<M>(sm, xc, sx, ex, sy, ey, as, ae, out);
  // fused_staged leaves the warp synchronised; put the result back as the accumulator
#pragma unroll
  for (int k = 0; k < M; ++k) sm.sa[lane_id() * M + k] = out[k];
  __syncwarp();
  as = r.sgn;
  ae = r.exp;
}

template <int M>
__global__ void __launch_bounds__(128) k_chain(const ChainTask* __restrict__ tasks, int ntasks, MPVec X, MPVec Y,
                                               MPVec INIT, MPVec OUT) {
  constexpr int n = 32 * M;
  extern __shared__ uint32_t smem[];
  const int wib = threadIdx.x >> 5;
  WarpSmem<M> sm(smem + wib * WarpSmem<M>::words);
  const int nw = gridDim.x * (blockDim.x >> 5);
  for (int t = blockIdx.x * (blockDim.x >> 5) + wib; t < ntasks; t += nw) {
    const ChainTask tk = tasks[t];
    int as = 0, ae = 0;
    if (tk.flags & CH_ZERO_INIT) {
#pragma unroll
      for (int k = 0; k < M; ++k) sm.sa[lane_id() * M + k] = 0;
    } else {
      copy_to_smem<M>(sm.sa, INIT.mant + tk.init * n);
      as = INIT.sgn[tk.init] ^ ((tk.flags & CH_NEG_INIT) ? 1 : 0);
      ae = INIT.exp[tk.init];
      if (sm.sa[n - 1] == 0u) as = 0;  // a zero init stays canonical
    }
    __syncwarp();
    if (sm.sa[n - 1] == 0u) { as = 0; ae = 0; }
    for (int q = 0; q < tk.len; ++q)
      chain_step<M>(sm, as, ae, X, tk.x0 + (int64_t)q * tk.sx, Y, tk.y0 + (int64_t)q * tk.sy, (tk.flags & CH_ADD) != 0);
    uint32_t out[M];
#pragma unroll
    for (int k = 0; k < M; ++k) out[k] = sm.sa[lane_id() * M + k];
    const bool zero = __shfl_sync(FULL, out[M - 1], 31) == 0u;
    Result r{zero ? 0 : (as ^ ((tk.flags & CH_NEG_OUT) ? 1 : 0)), zero ? 0 : ae, zero};
    store_result<M>(OUT, tk.out, r, out);
    __syncwarp();
  }
}

// k_chain with NTT products: FX[i], FY[i] hold the transforms of X[i]
// (unscaled) and Y[i] (scaled); the accumulator stays in registers.  Same
// exact products and the same combine as k_chain, so the same results.
template <int M>
__global__ void __launch_bounds__(32 * HK_NTT_TRAIL_WARPS, 2)
    k_chain_ntt(const ChainTask* __restrict__ tasks, int ntasks, MPVec X, MPVec Y, const uint32_t* __restrict__ FX,
                const uint32_t* __restrict__ FY, MPVec INIT, MPVec OUT, NttConst nc) {
  constexpr int n = 32 * M;
  extern __shared__ uint32_t smem[];
  const int wib = threadIdx.x >> 5;
  uint32_t* nb = smem + (size_t)wib * NTT_Q * ntt_stride(nc.L);
  const size_t per = (size_t)NTT_Q * nc.L;
  const int nw = gridDim.x * (blockDim.x >> 5);
  for (int t = blockIdx.x * (blockDim.x >> 5) + wib; t < ntasks; t += nw) {
    const ChainTask tk = tasks[t];
    uint32_t acc[M];
    int as = 0, ae = 0;
    if (tk.flags & CH_ZERO_INIT) {
#pragma unroll
      for (int k = 0; k < M; ++k) acc[k] = 0;
    } else {
      load_chunk<M>(INIT.mant + tk.init * n, acc);
      as = INIT.sgn[tk.init] ^ ((tk.flags & CH_NEG_INIT) ? 1 : 0);
      ae = INIT.exp[tk.init];
    }
    if (__shfl_sync(FULL, acc[M - 1], 31) == 0u) { as = 0; ae = 0; }
    const int flip = (tk.flags & CH_ADD) ? 1 : 0;
    for (int q = 0; q < tk.len; ++q) {
      const int64_t ix = tk.x0 + (int64_t)q * tk.sx, iy = tk.y0 + (int64_t)q * tk.sy;
      uint32_t o[M];
      const Result r = fused_ntt_core<M>(
          nb, nc, FX + (size_t)ix * per, X.mant[ix * n + n - 1] == 0u, X.sgn[ix], X.exp[ix], FY + (size_t)iy * per,
          Y.mant[iy * n + n - 1] == 0u, Y.sgn[iy] ^ flip, Y.exp[iy],
          [&](uint32_t* sa) {
#pragma unroll
            for (int k = 0; k < M; ++k) sa[IxPad::at(lane_id() * M + k)] = acc[k];
          },
          as, ae, o);
#pragma unroll
      for (int k = 0; k < M; ++k) acc[k] = o[k];
      as = r.sgn;
      ae = r.exp;
      __syncwarp();
    }
    const bool zero = __shfl_sync(FULL, acc[M - 1], 31) == 0u;
    Result r{zero ? 0 : (as ^ ((tk.flags & CH_NEG_OUT) ? 1 : 0)), zero ? 0 : ae, zero};
    store_result<M>(OUT, tk.out, r, acc);
    __syncwarp();
  }
}

// Reciprocals of D[idx[i]] (or D[first + i] when idx == nullptr) into Rtab[i].
template <int M>
__global__ void k_recip_tab(MPVec D, const int64_t* __restrict__ idx, int64_t first, int count,
                            uint32_t* __restrict__ Rtab, int* __restrict__ shtab, int* err) {
  constexpr int n = 32 * M;
  extern __shared__ uint32_t smem[];
  const int wib = threadIdx.x >> 5;
  uint32_t* ys = smem + wib * (3 * n + 4);
  uint32_t* sp = ys + n;
  const int nw = gridDim.x * (blockDim.x >> 5);
  for (int i = blockIdx.x * (blockDim.x >> 5) + wib; i < count; i += nw) {
    const int64_t j = idx ? idx[i] : first + i;
    uint32_t dc[M], R[M];
    load_chunk<M>(D.mant + j * n, dc);
    const bool zero = __shfl_sync(FULL, dc[M - 1], 31) == 0u;
    if (zero) {
      if (lane_id() == 0) atomicOr(err, ERR_ARG);
      continue;
    }
    int sh;
    warp_recip<M>(dc, ys, sp, R, sh, err);
    store_chunk<M>(Rtab + (int64_t)i * n, R);
    if (lane_id() == 0) shtab[i] = sh;
    __syncwarp();
  }
}

template <int M>
__global__ void k_quot(const QuotTask* __restrict__ tasks, int ntasks, MPVec A, MPVec D,
                       const uint32_t* __restrict__ Rtab, const int* __restrict__ shtab, MPVec OUT, int* err) {
  constexpr int n = 32 * M;
  extern __shared__ uint32_t smem[];
  const int wib = threadIdx.x >> 5;
  uint32_t* ys = smem + wib * (4 * n + 4);
  uint32_t* yt = ys + n;
  uint32_t* sp = yt + n;
  const int nw = gridDim.x * (blockDim.x >> 5);
  for (int t = blockIdx.x * (blockDim.x >> 5) + wib; t < ntasks; t += nw) {
    const QuotTask tk = tasks[t];
    uint32_t ac[M], dc[M], q[M];
    load_chunk<M>(A.mant + tk.ia * n, ac);
    load_chunk<M>(D.mant + tk.id * n, dc);
    const bool a_zero = __shfl_sync(FULL, ac[M - 1], 31) == 0u;
    Result r;
    if (a_zero) {
#pragma unroll
      for (int k = 0; k < M; ++k) q[k] = 0;
      r = Result{0, 0, true};
    } else {
      copy_to_smem<M>(ys, Rtab + tk.rid * n);
      __syncwarp();
      int t_shift;
      warp_quot<M>(ac, dc, ys, shtab[tk.rid], yt, sp, q, t_shift, err);
      r = Result{A.sgn[tk.ia] ^ D.sgn[tk.id] ^ tk.neg, A.exp[tk.ia] - D.exp[tk.id] - t_shift, false};
    }
    store_result<M>(OUT, tk.out, r, q);
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------
// Algorithm 4 (Sec. 4.4), step i, on X (row major N x k):
//   for j > i:  f = L[j][i];  if i < k: X[j][i] = -f;
//               X[j][c] = trunc(X[j][c] - f * X[i][c])   for c < min(k, i)
// One warp per (j, c) update; the negated copies are done by the same warps.
// ---------------------------------------------------------------------------
template <int M>
__global__ void __launch_bounds__(128) k_alg4_step(MPVec A, MPVec X, int N, int k, int i) {
  constexpr int n = 32 * M;
  extern __shared__ uint32_t smem[];
  const int wib = threadIdx.x >> 5;
  WarpSmem<M> sm(smem + wib * WarpSmem<M>::words);
  const int cols = min(k, i);
  const int64_t rows = N - 1 - i;
  const int64_t total = rows * (cols + (i < k ? 1 : 0));
  const int per_row = cols + (i < k ? 1 : 0);
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t t = (int64_t)blockIdx.x * (blockDim.x >> 5) + wib; t < total; t += nw) {
    const int64_t j = i + 1 + t / per_row;
    const int c = (int)(t % per_row);
    const int64_t fpos = tri_pos(N, j, i);
    if (c == cols) {  // X[j][i] = -L[j][i]
      uint32_t v[M];
      load_chunk<M>(A.mant + fpos * n, v);
      const bool zero = __shfl_sync(FULL, v[M - 1], 31) == 0u;
      Result r{zero ? 0 : (A.sgn[fpos] ^ 1), A.exp[fpos], zero};
      store_result<M>(X, j * k + i, r, v);
      continue;
    }
    const int64_t apos = j * k + c, ypos = (int64_t)i * k + c;
    copy_to_smem<M>(sm.ys, X.mant + ypos * n);
    copy_to_smem<M>(sm.sa, X.mant + apos * n);
    uint32_t xc[M], o[M];
    load_chunk<M>(A.mant + fpos * n, xc);
    __syncwarp();
    const Result r = fused_staged<M>(sm, xc, A.sgn[fpos], A.exp[fpos], X.sgn[ypos], X.exp[ypos], X.sgn[apos],
                                     X.exp[apos], o);
    store_result<M>(X, apos, r, o);
    __syncwarp();
  }
}

// Algorithm 4 step i with NTT products: FL[j - i - 1] = transform of L[j][i]
// (unscaled), FXr[c] = transform of X[i][c] (scaled).
template <int M>
__global__ void __launch_bounds__(32 * HK_NTT_TRAIL_WARPS, 2) k_alg4_ntt(MPVec A, MPVec X, const uint32_t* __restrict__ FL,
                                                  const uint32_t* __restrict__ FXr, int N, int k, int i, NttConst nc) {
  constexpr int n = 32 * M;
  extern __shared__ uint32_t smem[];
  const int wib = threadIdx.x >> 5;
  uint32_t* nb = smem + (size_t)wib * NTT_Q * ntt_stride(nc.L);
  const int cols = min(k, i);
  const int per_row = cols + (i < k ? 1 : 0);
  const int64_t total = (int64_t)(N - 1 - i) * per_row;
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t t = (int64_t)blockIdx.x * (blockDim.x >> 5) + wib; t < total; t += nw) {
    const int64_t j = i + 1 + t / per_row;
    const int c = (int)(t % per_row);
    const int64_t fpos = tri_pos(N, j, i);
    if (c == cols) {  // X[j][i] = -L[j][i]
      uint32_t v[M];
      load_chunk<M>(A.mant + fpos * n, v);
      const bool zero = __shfl_sync(FULL, v[M - 1], 31) == 0u;
      Result r{zero ? 0 : (A.sgn[fpos] ^ 1), A.exp[fpos], zero};
      store_result<M>(X, j * k + i, r, v);
      continue;
    }
    const int64_t apos = j * k + c, ypos = (int64_t)i * k + c;
    uint32_t o[M];
    const Result r = fused_ntt<M>(nb, nc, FL + (size_t)(j - i - 1) * NTT_Q * nc.L, A.mant[fpos * n + n - 1] == 0u,
                                  A.sgn[fpos], A.exp[fpos], FXr + (size_t)c * NTT_Q * nc.L,
                                  X.mant[ypos * n + n - 1] == 0u, X.sgn[ypos], X.exp[ypos], X.mant + apos * n,
                                  X.sgn[apos], X.exp[apos], o);
    store_result<M>(X, apos, r, o);
    __syncwarp();
  }
}

// X[r][c] = 1 if r == c (c < k), else 0, for the rows r <= c that Algorithm 4 never writes.
template <int M>
__global__ void k_x_init(MPVec X, int N, int k) {
  constexpr int n = 32 * M;
  const int64_t total = (int64_t)N * k * n;
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < total; g += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = g / n;
    const int w = (int)(g % n);
    const int64_t r = e / k, c = e % k;
    const bool one = (r == c);
    X.mant[g] = (one && w == n - 1) ? 1u : 0u;
    if (w == 0) {
      X.sgn[e] = 0;
      X.exp[e] = one ? -(n - 1) : 0;
    }
  }
}

// Back substitution step j of L^T w = y (column form): y[i] -= L[j][i] * y[j] for i < j.
// y[j] is final once every later column has been applied.
template <int M>
__global__ void __launch_bounds__(128) k_backsub_step(MPVec A, MPVec Yv, int N, int j) {
  constexpr int n = 32 * M;
  extern __shared__ uint32_t smem[];
  const int wib = threadIdx.x >> 5;
  WarpSmem<M> sm(smem + wib * WarpSmem<M>::words);
  const int nw = gridDim.x * (blockDim.x >> 5);
  for (int i = blockIdx.x * (blockDim.x >> 5) + wib; i < j; i += nw) {
    const int64_t lpos = tri_pos(N, j, i);
    copy_to_smem<M>(sm.ys, Yv.mant + (int64_t)j * n);
    copy_to_smem<M>(sm.sa, Yv.mant + (int64_t)i * n);
    uint32_t xc[M], o[M];
    load_chunk<M>(A.mant + lpos * n, xc);
    __syncwarp();
    const Result r = fused_staged<M>(sm, xc, A.sgn[lpos], A.exp[lpos], Yv.sgn[j], Yv.exp[j], Yv.sgn[i], Yv.exp[i], o);
    store_result<M>(Yv, i, r, o);
    __syncwarp();
  }
}

// The same step with NTT products: FY = transform of y[j] (scaled); each
// warp transforms its L[j][i] into its slot of FX (scratch, read back by the
// same warp).
template <int M>
__global__ void __launch_bounds__(32 * HK_NTT_TRAIL_WARPS, 2)
    k_backsub_ntt(MPVec A, MPVec Yv, int N, int j, const uint32_t* __restrict__ FY, uint32_t* FX, NttConst nc) {
  constexpr int n = 32 * M;
  extern __shared__ uint32_t smem[];
  const int wib = threadIdx.x >> 5;
  uint32_t* nb = smem + (size_t)wib * NTT_Q * ntt_stride(nc.L);
  const size_t per = (size_t)NTT_Q * nc.L;
  const int gw = blockIdx.x * (blockDim.x >> 5) + wib;
  uint32_t* fx = FX + (size_t)gw * per;
  const int nw = gridDim.x * (blockDim.x >> 5);
  const bool y_zero = Yv.mant[(int64_t)j * n + n - 1] == 0u;
  for (int i = gw; i < j; i += nw) {
    const int64_t lpos = tri_pos(N, j, i);
    const bool x_zero = A.mant[lpos * n + n - 1] == 0u;
    if (!x_zero && !y_zero) {
      warp_ntt_number<M>(A.mant + lpos * n, nb, fx, nc, false);
      __syncwarp();
    }
    uint32_t o[M];
    const uint32_t* am = Yv.mant + (int64_t)i * n;
    auto stage = [&](uint32_t* sa) { copy_to_smem<M, IxPad>(sa, am); };
    const Result r = fused_ntt_core<M, decltype(stage), false>(nb, nc, fx, x_zero, A.sgn[lpos], A.exp[lpos], FY,
                                                                y_zero, Yv.sgn[j], Yv.exp[j], stage, Yv.sgn[i],
                                                                Yv.exp[i], o);
    store_result<M>(Yv, i, r, o);
    __syncwarp();
  }
}

// Small exact constants: out[i] = trunc(num[i] / den[i]) for 64-bit integers
// (num may be 0), formed by long division (one lane per number).
template <int M>
__global__ void k_small_ratio(const int64_t* __restrict__ num, const int64_t* __restrict__ den, int count,
                              MPVec OUT) {
  constexpr int n = 32 * M;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  int64_t a = num[i], b = den[i];
  int s = 0;
  if (a < 0) { a = -a; s ^= 1; }
  if (b < 0) { b = -b; s ^= 1; }
  uint32_t* o = OUT.mant + (int64_t)i * n;
  if (a == 0) {
    for (int k = 0; k < n; ++k) o[k] = 0;
    OUT.sgn[i] = 0;
    OUT.exp[i] = 0;
    return;
  }
  // integer part q = a / b (< 2^64), remainder r; then fractional limbs
  const uint64_t ua = (uint64_t)a, ub = (uint64_t)b;
  uint64_t q = ua / ub, r = ua % ub;
  // limbs of the value in radix 2^32, from the top: integer part first
  int ilimbs = q >> 32 ? 2 : (q ? 1 : 0);
  int lead_zero_frac = 0;
  // when q == 0, skip fractional limbs that are zero
  uint32_t buf_first[2] = {(uint32_t)(q >> 32), (uint32_t)q};
  int pos = n - 1;
  int exp_top;  // limb exponent of the top limb
  if (ilimbs == 2) {
    o[pos--] = buf_first[0];
    o[pos--] = buf_first[1];
    exp_top = 1;
  } else if (ilimbs == 1) {
    o[pos--] = buf_first[1];
    exp_top = 0;
  } else {
    exp_top = -1;
    for (;;) {
      const unsigned __int128 t = (unsigned __int128)r << 32;
      const uint64_t d = (uint64_t)(t / ub);
      r = (uint64_t)(t % ub);
      if (d) { o[pos--] = (uint32_t)d; break; }
      --exp_top;
      ++lead_zero_frac;
    }
  }
  while (pos >= 0) {
    const unsigned __int128 t = (unsigned __int128)r << 32;
    o[pos--] = (uint32_t)(t / ub);
    r = (uint64_t)(t % ub);
  }
  OUT.sgn[i] = s;
  OUT.exp[i] = exp_top - (n - 1);
}

// Index (by an approximate magnitude: limb exponent, then top limb) of the
// largest |T[j][j]|, j < kk, written to out[0].  One warp.
static __global__ void k_argmax_diag(MPVec T, int k, int kk, int n, int* out) {
  const int lane = threadIdx.x & 31;
  long long best_key = LLONG_MIN;
  int best = 0;
  for (int j = lane; j < kk; j += 32) {
    const int64_t p = (int64_t)j * k + j;
    const uint32_t top = T.mant[p * n + n - 1];
    const long long key = top ? (long long)T.exp[p] * 4294967296LL + (long long)top : LLONG_MIN + 1;
    if (key > best_key) { best_key = key; best = j; }
  }
  for (int off = 16; off; off >>= 1) {
    const long long ok = __shfl_xor_sync(0xffffffffu, best_key, off);
    const int oj = __shfl_xor_sync(0xffffffffu, best, off);
    if (ok > best_key || (ok == best_key && oj < best)) { best_key = ok; best = oj; }
  }
  if (lane == 0) out[0] = best;
}

// flag[0] = 1 when |D[id]| <= 2^(-32 tol) |V[iv]| (top-limb indices differ by
// at least tol) or D[id] == 0.  One thread.
static __global__ void k_rel_small(MPVec D, int64_t id, MPVec V, int64_t iv, int n, int tol, int* flag) {
  if (threadIdx.x || blockIdx.x) return;
  const bool dz = D.mant[id * n + n - 1] == 0u;
  const bool vz = V.mant[iv * n + n - 1] == 0u;
  flag[0] = (dz || (!vz && (int64_t)V.exp[iv] - (int64_t)D.exp[id] >= tol)) ? 1 : 0;
}

}  // namespace hk
