// Batched factorisation: Algorithm 1 (Sec. 4.3) for several independent
// instances of one width in ONE persistent launch (the batched form of the
// sweeps over beta and N, Sec. 5 and 6).
//
// Each instance's factorisation is a chain of phases:
//   phase 0          the reciprocal of d_0                       (1 item)
//   phase 1 + 2i     column scale of step i, rows i+1 .. N-1     (m = N-1-i items)
//   phase 2 + 2i     trailing update of step i                   (m(m+1)/2 items)
//                    item 0 is the entry (i+1, i+1) = d_{i+1}; the warp that
//                    forms it goes on to the reciprocal of d_{i+1} (the
//                    look-ahead of Alg. 2 inside the update); then, for an
//                    instance planned with a block size k, step i of
//                    Algorithm 4 (Sec. 4.4) on X = L^-1[:, :k]: it needs
//                    only column i of L (final after the scale) and row i
//                    of X (final after step i - 1), so it shares the phase
//   phase 2N - 1     finished
// Every item of a phase depends only on phases before it, so any warp may
// take any item of an instance's current phase.  Warps claim items with an
// atomic ticket per phase and count them done with a second counter; the
// warp that completes a phase publishes the next one (release store, read
// back with acquire loads).  No warp ever waits for a particular other warp:
// a warp without an item scans the instances again after a short sleep, so
// the launch needs no co-residency guarantee.  That idle wait is bounded: if
// no phase of any instance advances for `limit_ns` the launch records
// ERR_TIMEOUT in every unfinished instance and returns.
//
// Data written during the launch (the factor, U, the reciprocal) is read
// with L2-only loads (ld.global.cg), after an acquire load of the phase.
// Products are schoolbook at every width this form serves (up to 8192
// bits, where the step-by-step launches take NTT products instead); every
// product is exact and every entry goes through the same truncated
// operations in the same step order, so the factor is bit-identical.
#pragma once
#include "batch_sched.h"
#include "k_ldlt.cuh"

namespace hk {

// One instance of the batch (device copy, written once before the launch).
struct BatchInst {
  MPVec A;           // packed factor, assembled H_N on entry
  MPVec U;           // N numbers: the pivot column before scaling
  uint32_t* rec;     // n limbs: reciprocal of the current pivot
  int* rec_meta;     // [0]: its shift
  int* err;          // the instance's error word (ErrBits)
  int* state;        // [0] phase, [1 .. 2N-1] tickets, [2N .. 4N-2] done counts
  MPVec X;           // N x k, row major: Algorithm 4's X, first k columns of
                     // the identity on entry (k = 0: no Algorithm 4)
  int N;
  int k;
};

// Launch-wide control words.
struct BatchCtl {
  int finished;  // instances whose last phase is done
  int progress;  // phases completed so far (all instances)
  int abort;     // set by a warp whose idle wait ran out
  int pad;
};

#ifndef HK_BATCH_WARPS
#define HK_BATCH_WARPS 4
#endif


// shared-memory words per warp: the largest of the reciprocal (3n + 4), the
// exact quotient (4n + 4) and the fused update (WarpSmem, 4n + 2)
template <int M>
__host__ __device__ constexpr size_t batch_warp_words() {
  return (size_t)4 * (32 * M) + 4;
}

__device__ __forceinline__ int ld_acquire_gpu(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_gpu(int* p, int v) {
  asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ int ld_relaxed_gpu(const int* p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// lane chunk of an n-limb number through L2 (never a stale L1 line)
template <int M>
__device__ __forceinline__ void load_chunk_l2(const uint32_t* src, uint32_t (&v)[M]) {
  const uint32_t* p = src + lane_id() * M;
  if constexpr (M % 4 == 0) {
#pragma unroll
    for (int k = 0; k < M; k += 4) {
      const uint4 t = __ldcg(reinterpret_cast<const uint4*>(p + k));
      v[k] = t.x; v[k + 1] = t.y; v[k + 2] = t.z; v[k + 3] = t.w;
    }
  } else if constexpr (M % 2 == 0) {
#pragma unroll
    for (int k = 0; k < M; k += 2) {
      const uint2 t = __ldcg(reinterpret_cast<const uint2*>(p + k));
      v[k] = t.x; v[k + 1] = t.y;
    }
  } else {
#pragma unroll
    for (int k = 0; k < M; ++k) v[k] = __ldcg(p + k);
  }
}

template <int M>
__device__ __forceinline__ void stage_l2(uint32_t* dst, const uint32_t* src) {
  uint32_t v[M];
  load_chunk_l2<M>(src, v);
#pragma unroll
  for (int k = 0; k < M; ++k) dst[lane_id() * M + k] = v[k];
}

__device__ __forceinline__ int64_t batch_items(const BatchInst& b, int ph) { return batch_phase_items(b.N, b.k, ph); }

// Reciprocal of a pivot held in registers (dc, sign sgn): R and its shift
// into the instance's buffers; a pivot <= 0 sets ERR_NOT_PD instead.
template <int M>
__device__ void batch_recip(const BatchInst& b, const uint32_t (&dc)[M], int sgn, uint32_t* w) {
  const bool zero = __shfl_sync(FULL, dc[M - 1], 31) == 0u;
  if (zero || sgn != 0) {
    if (lane_id() == 0) atomicOr(b.err, ERR_NOT_PD);
    return;
  }
  uint32_t R[M];
  int sh;
  warp_recip<M>(dc, w, w + 32 * M, R, sh, b.err);
  store_chunk<M>(b.rec, R);
  if (lane_id() == 0) b.rec_meta[0] = sh;
}

// Column scale of step i, row r: U[r] = A[r][i], A[r][i] = trunc(A[r][i] / d_i).
template <int M>
__device__ void batch_scale(const BatchInst& b, int i, int64_t r, uint32_t* w) {
  constexpr int n = 32 * M;
  const int N = b.N;
  uint32_t* ys = w;
  uint32_t* yt = w + n;
  uint32_t* sp = w + 2 * n;
  const int64_t dpos = tri_pos(N, i, i);
  const int64_t pos = tri_pos(N, r, i);
  uint32_t dc[M], ac[M], q[M];
  load_chunk_l2<M>(b.A.mant + dpos * n, dc);
  load_chunk_l2<M>(b.A.mant + pos * n, ac);
  const int ed = __ldcg(b.A.exp + dpos);
  const int sa = __ldcg(b.A.sgn + pos), ea = __ldcg(b.A.exp + pos);
  store_chunk<M>(b.U.mant + r * n, ac);
  if (lane_id() == 0) {
    b.U.sgn[r] = sa;
    b.U.exp[r] = ea;
  }
  const bool a_zero = __shfl_sync(FULL, ac[M - 1], 31) == 0u;
  Result res;
  if (a_zero) {
#pragma unroll
    for (int k = 0; k < M; ++k) q[k] = 0;
    res = Result{0, 0, true};
  } else {
    stage_l2<M>(ys, b.rec);
    const int sh = __ldcg(b.rec_meta);
    __syncwarp();
    int t;
    warp_quot<M>(ac, dc, ys, sh, yt, sp, q, t, b.err);
    res = Result{sa, ea - ed - t, false};
  }
  store_result<M>(b.A, pos, res, q);
}

// Trailing update of step i, entry t of the packed trailing triangle:
// A[r][c] = trunc(A[r][c] - U[c] B_i[r]); entry 0 (= d_{i+1}) also takes the
// reciprocal of the next pivot.
// Algorithm 4, step i, update u of the step (row j = i + 1 + u / per_row,
// column c = u % per_row):  X[j][i] = -L[j][i] when c = i < k, else
// X[j][c] = trunc(X[j][c] - L[j][i] X[i][c]).
template <int M>
__device__ void batch_alg4(const BatchInst& b, int i, int64_t u, uint32_t* w) {
  constexpr int n = 32 * M;
  const int N = b.N, k = b.k;
  const int cols = i < k ? i : k;
  int64_t j;
  int c;
  batch_alg4_item(k, i, u, j, c);
  const int64_t fpos = tri_pos(N, j, i);
  if (c == cols) {
    uint32_t v[M];
    load_chunk_l2<M>(b.A.mant + fpos * n, v);
    const bool zero = __shfl_sync(FULL, v[M - 1], 31) == 0u;
    const Result r{zero ? 0 : (__ldcg(b.A.sgn + fpos) ^ 1), __ldcg(b.A.exp + fpos), zero};
    store_result<M>(b.X, j * k + i, r, v);
    return;
  }
  const int64_t apos = j * k + c, ypos = (int64_t)i * k + c;
  WarpSmem<M> sm(w);
  stage_l2<M>(sm.ys, b.X.mant + ypos * n);
  stage_l2<M>(sm.sa, b.X.mant + apos * n);
  uint32_t xc[M], o[M];
  load_chunk_l2<M>(b.A.mant + fpos * n, xc);
  const int sl = __ldcg(b.A.sgn + fpos), el = __ldcg(b.A.exp + fpos);
  const int sy = __ldcg(b.X.sgn + ypos), ey = __ldcg(b.X.exp + ypos);
  const int sa = __ldcg(b.X.sgn + apos), ea = __ldcg(b.X.exp + apos);
  __syncwarp();
  const Result r = fused_staged<M>(sm, xc, sl, el, sy, ey, sa, ea, o);
  store_result<M>(b.X, apos, r, o);
}

template <int M>
__device__ void batch_trailing(const BatchInst& b, int i, int64_t t, uint32_t* w) {
  constexpr int n = 32 * M;
  const int N = b.N;
  const int64_t m = N - 1 - i;
  const int64_t cc = trail_col(m, t);
  const int64_t c = i + 1 + cc;
  const int64_t r = c + (t - trail_off(m, cc));
  const int64_t apos = tri_pos(N, r, c);
  const int64_t bpos = tri_pos(N, r, i);
  WarpSmem<M> sm(w);
  stage_l2<M>(sm.ys, b.A.mant + bpos * n);
  stage_l2<M>(sm.sa, b.A.mant + apos * n);
  uint32_t xc[M];
  load_chunk_l2<M>(b.U.mant + c * n, xc);
  const int su = __ldcg(b.U.sgn + c), eu = __ldcg(b.U.exp + c);
  const int sb = __ldcg(b.A.sgn + bpos), eb = __ldcg(b.A.exp + bpos);
  const int sa = __ldcg(b.A.sgn + apos), ea = __ldcg(b.A.exp + apos);
  __syncwarp();
  uint32_t o[M];
  const Result res = fused_staged<M>(sm, xc, su, eu, sb, eb, sa, ea, o);
  store_result<M>(b.A, apos, res, o);
  __syncwarp();
  if (t == 0) batch_recip<M>(b, o, res.sgn, w);
}

__device__ __forceinline__ int atom_add_acq_rel_gpu(int* p, int v) {
  int old;
  asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
  return old;
}

// Lane 0: claim a chunk of instance jj's current phase, if it has one left.
__device__ __forceinline__ bool batch_claim(const BatchInst& b, int chunk, bool precheck, int& ph, int64_t& first,
                                            int64_t& last) {
  const int q = ld_acquire_gpu(b.state);
  if (q >= 2 * b.N - 1) return false;
  const int64_t cnt = batch_items(b, q);
  const int64_t chunks = batch_chunks(cnt, chunk);
  int* tick = b.state + 1 + q;
  if (precheck && ld_relaxed_gpu(tick) >= chunks) return false;  // all claimed: take no ticket
  const int64_t t = atomicAdd(tick, 1);
  if (t >= chunks) return false;
  ph = q;
  batch_chunk_range(cnt, chunk, t, first, last);
  return true;
}

template <int M>
__global__ void __launch_bounds__(32 * HK_BATCH_WARPS)
    k_ldlt_batch(const BatchInst* __restrict__ inst, int count, BatchCtl* ctl, long long limit_ns, int chunk) {
  extern __shared__ uint32_t smem[];
  const int wib = threadIdx.x >> 5;
  const int lane = lane_id();
  uint32_t* w = smem + (size_t)wib * batch_warp_words<M>();
  const int gw = blockIdx.x * (blockDim.x >> 5) + wib;
  int cur = gw % count;     // the instance this warp looks at first
  bool worked = false;      // the last pass took a chunk of instance cur
  int scanned = -1;         // progress count before this warp's last scan that found nothing
  int seen = -1;            // progress count at the start of the current idle spell
  uint64_t idle_since = 0;
  unsigned nap = 64;        // idle sleep (ns), doubled up to 2 us while nothing changes
  while (true) {
    // lane 0 claims a chunk: first from the instance it just worked on, else
    // from the first instance (from cur on) whose phase has one left.  A scan
    // that finds none need not be repeated until some phase advances (the
    // progress count changes).
    int j = -1, ph = 0, stop = 0;
    int64_t first = 0, last = 0;
    if (lane == 0) {
      if (worked && batch_claim(inst[cur], chunk, false, ph, first, last)) {
        j = cur;
      } else if (ld_relaxed_gpu(&ctl->abort) != 0) {
        stop = 1;
      } else {
        const int p = ld_acquire_gpu(&ctl->progress);
        if (p != scanned) {
          for (int probe = 0; probe < count && j < 0; ++probe) {
            const int jj = cur + probe < count ? cur + probe : cur + probe - count;
            if (batch_claim(inst[jj], chunk, true, ph, first, last)) j = jj;
          }
          if (j < 0) scanned = p;
        }
        if (j < 0) {
          if (ld_acquire_gpu(&ctl->finished) >= count) {
            stop = 1;
          } else {
            const uint64_t now = global_ns();
            if (p != seen) {
              seen = p;
              idle_since = now;
            } else if (now - idle_since > (uint64_t)limit_ns) {
              // no phase advanced anywhere for the whole limit: give up
              if (atomicExch(&ctl->abort, 1) == 0)
                for (int jj = 0; jj < count; ++jj)
                  if (ld_relaxed_gpu(inst[jj].state) < 2 * inst[jj].N - 1) atomicOr(inst[jj].err, ERR_TIMEOUT);
              stop = 1;
            }
          }
        }
      }
    }
    if (__shfl_sync(FULL, stop, 0)) break;
    j = __shfl_sync(FULL, j, 0);
    worked = j >= 0;
    if (j < 0) {
      __nanosleep(nap);
      nap = nap < 2048 ? 2 * nap : 2048;
      continue;
    }
    nap = 64;
    seen = -1;
    cur = j;
    ph = __shfl_sync(FULL, ph, 0);
    first = __shfl_sync(FULL, first, 0);
    last = __shfl_sync(FULL, last, 0);
    const BatchInst& b = inst[j];
    (void)ld_acquire_gpu(b.state);  // every lane: what the earlier phases wrote is visible
    for (int64_t item = first; item < last; ++item) {
      if (ph == 0) {
        uint32_t dc[M];
        load_chunk_l2<M>(b.A.mant, dc);
        batch_recip<M>(b, dc, __ldcg(b.A.sgn), w);
      } else if (ph & 1) {
        const int i = (ph - 1) >> 1;
        batch_scale<M>(b, i, i + 1 + item, w);
      } else {
        const int i = (ph - 2) >> 1;
        const int64_t m = b.N - 1 - i, T = m * (m + 1) / 2;
        if (item < T)
          batch_trailing<M>(b, i, item, w);
        else
          batch_alg4<M>(b, i, item - T, w);
      }
      __syncwarp();
    }
    // release: the warp's writes (ordered before lane 0's by the warp
    // barrier), then one count for the chunk
    if (lane == 0) {
      const int64_t cnt = batch_items(b, ph);
      int* done = b.state + 2 * b.N + ph;
      const int k = (int)(last - first);
      if (atom_add_acq_rel_gpu(done, k) + k == cnt) {
        const int fin = 2 * b.N - 1;
        int np = ph + 1;
        if (np < fin && (ld_relaxed_gpu(b.err) & ERR_NOT_PD)) np = fin;  // a pivot <= 0 ends the instance
        st_release_gpu(b.state, np);
        if (np == fin) atomicAdd(&ctl->finished, 1);
        __threadfence();
        atomicAdd(&ctl->progress, 1);  // after the phase: a warp that sees the count sees the phase
      }
    }
    __syncwarp();
  }
}

}  // namespace hk
