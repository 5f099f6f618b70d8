// Index arithmetic of the batched factorisation's phases and claims
// (k_batch.cuh): plain functions that the kernel and a host test share.
//
// Phases of one instance of size N (block size k, 0 = no Algorithm 4):
//   0          the reciprocal of d_0                                   1 item
//   1 + 2i     column scale of step i                                  m = N-1-i items
//   2 + 2i     trailing update of step i, then Algorithm 4's step i    m(m+1)/2 + m * per_row(k, i)
//   2N - 1     finished
// Items of a phase are claimed in chunks: chunk 0 is item 0 alone (in a
// trailing phase it carries the next pivot's reciprocal, the step's
// critical path), chunk t >= 1 holds items 1 + (t-1) G .. t G (the last
// one fewer), with G growing with the phase up to `chunk` so that large
// phases pay one claim per G updates while small ones keep every warp busy.
#pragma once
#include <cstdint>

#ifdef __CUDACC__
#define HK_SCHED_FN __host__ __device__ __forceinline__
#else
#define HK_SCHED_FN inline
#endif

namespace hk {

// Algorithm 4's updates in step i, per row j > i: the columns c < min(k, i)
// and, while i < k, the new entry X[j][i] = -L[j][i]
HK_SCHED_FN int batch_alg4_per_row(int k, int i) { return k <= 0 ? 0 : (i < k ? i + 1 : k); }

// Algorithm 4's update u of step i: row j and column c (c == i: the new
// entry X[j][i] = -L[j][i]; c < min(k, i): X[j][c] -= L[j][i] X[i][c])
HK_SCHED_FN void batch_alg4_item(int k, int i, int64_t u, int64_t& j, int& c) {
  const int per_row = batch_alg4_per_row(k, i);
  j = i + 1 + u / per_row;
  c = (int)(u % per_row);
}

HK_SCHED_FN int64_t batch_phase_items(int N, int k, int ph) {
  if (ph == 0) return 1;
  const int i = (ph - 1) >> 1;
  const int64_t m = N - 1 - i;
  return (ph & 1) ? m : m * (m + 1) / 2 + m * batch_alg4_per_row(k, i);
}

HK_SCHED_FN int64_t batch_group(int64_t cnt, int chunk) {
  const int64_t g = cnt >= 4096 ? chunk : cnt >= 1024 ? (chunk + 1) / 2 : cnt >= 256 ? (chunk + 3) / 4 : 1;
  return g < 1 ? 1 : g;
}

HK_SCHED_FN int64_t batch_chunks(int64_t cnt, int chunk) {
  const int64_t g = batch_group(cnt, chunk);
  return cnt <= 1 ? cnt : 1 + (cnt - 1 + g - 1) / g;
}

// items [first, last) of chunk t (0 <= t < batch_chunks(cnt, chunk))
HK_SCHED_FN void batch_chunk_range(int64_t cnt, int chunk, int64_t t, int64_t& first, int64_t& last) {
  const int64_t g = batch_group(cnt, chunk);
  first = t == 0 ? 0 : 1 + (t - 1) * g;
  last = t == 0 ? 1 : (first + g < cnt ? first + g : cnt);
}

}  // namespace hk
