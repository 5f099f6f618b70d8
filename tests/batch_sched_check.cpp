// Host check of the batched factorisation's index arithmetic
// (paper_1810_01478_gb300/csrc/batch_sched.h, and the trailing triangle's
// enumeration in common.cuh): every phase's items are claimed exactly once,
// the phases hold exactly the operations of Algorithm 1 (Sec. 4.3) and
// Algorithm 4 (Sec. 4.4), and each item decodes to a distinct entry.
// Prints "ok" or the first failure; exit status 0 only on "ok".
#include <cmath>
#include <cstdio>
#include <cstdint>
#include <set>
#include <utility>
#include <vector>

#include "batch_sched.h"
#include "common.cuh"

using namespace hk;

static int fail(const char* what, long long a, long long b, long long c) {
  std::printf("FAIL %s (%lld, %lld, %lld)\n", what, a, b, c);
  return 1;
}

int main() {
  const int chunks_tried[] = {1, 2, 3, 4, 8, 16};
  for (int N = 1; N <= 48; ++N) {
    const int ks[] = {0, 1, 2, 5, N < 16 ? N : 16, N < 64 ? N : 64};
    for (int k : ks) {
      if (k > N) continue;
      // operations Algorithm 1 and Algorithm 4 perform, counted by their loops
      long long quot = 0, trail = 0, a4 = 0;
      for (int i = 0; i < N; ++i)
        for (int r = i + 1; r < N; ++r) {
          ++quot;
          for (int c = i + 1; c <= r; ++c) ++trail;
          for (int c = 0; c < k; ++c)
            if (c <= i) ++a4;  // c < i: an update; c == i: the new entry -L[r][i]
        }
      for (int chunk : chunks_tried) {
        long long total = 0;
        for (int ph = 0; ph < 2 * N - 1; ++ph) {
          const int64_t cnt = batch_phase_items(N, k, ph);
          if (cnt < 1) return fail("empty phase", N, k, ph);
          total += cnt;
          // the chunks tile [0, cnt): chunk 0 is item 0 alone, none larger than chunk
          const int64_t nch = batch_chunks(cnt, chunk);
          int64_t next = 0;
          for (int64_t t = 0; t < nch; ++t) {
            int64_t first, last;
            batch_chunk_range(cnt, chunk, t, first, last);
            if (first != next || last <= first || last > cnt) return fail("chunk range", N, ph, t);
            if (t == 0 && last != 1) return fail("chunk 0 is not item 0 alone", N, ph, last);
            if (last - first > (chunk > 1 ? chunk : 1)) return fail("chunk too large", N, ph, last - first);
            next = last;
          }
          if (next != cnt) return fail("chunks do not cover the phase", N, ph, next);
          if (chunk != 1 || !(ph >= 2 && ph % 2 == 0)) continue;
          // trailing phase of step i: the items decode to distinct entries
          const int i = (ph - 2) / 2;
          const int64_t m = N - 1 - i, T = m * (m + 1) / 2;
          std::set<std::pair<int64_t, int64_t>> seen;
          for (int64_t t = 0; t < T; ++t) {
            const int64_t cc = trail_col(m, t);
            const int64_t c = i + 1 + cc, r = c + (t - trail_off(m, cc));
            if (c <= i || r < c || r >= N || !seen.insert({r, c}).second) return fail("trailing item", N, i, t);
            if (t == 0 && (r != i + 1 || c != i + 1)) return fail("item 0 is not d_{i+1}", N, i, r);
          }
          std::set<std::pair<int64_t, int>> xs;
          for (int64_t u = 0; u < cnt - T; ++u) {
            int64_t j;
            int c;
            batch_alg4_item(k, i, u, j, c);
            if (j <= i || j >= N || c < 0 || c > i || c >= k || !xs.insert({j, c}).second)
              return fail("Algorithm 4 item", N, i, u);
          }
        }
        // phase 0 is the first reciprocal; the later ones ride on trailing items 0
        if (total != 1 + quot + trail + a4) return fail("phase totals", N, k, total);
      }
    }
  }
  // the trailing triangle's enumeration at large sizes (floating-point inversion)
  const int64_t ms[] = {1000, 65535, 1048575};
  for (int64_t m : ms) {
    const int64_t T = m * (m + 1) / 2;
    for (int64_t s = 0; s < 200000; ++s) {
      const int64_t t = (s * 2654435761LL) % T;
      const int64_t cc = trail_col(m, t);
      if (cc < 0 || cc >= m || trail_off(m, cc) > t || (cc + 1 < m && trail_off(m, cc + 1) <= t))
        return fail("trail_col", m, t, cc);
    }
    if (trail_col(m, T - 1) != m - 1 || trail_col(m, 0) != 0) return fail("trail_col ends", m, 0, 0);
  }
  // claims of a large phase
  const int64_t big = 50000000;
  for (int chunk : chunks_tried) {
    int64_t first, last;
    batch_chunk_range(big, chunk, batch_chunks(big, chunk) - 1, first, last);
    if (last != big) return fail("last chunk of a large phase", chunk, first, last);
  }
  std::printf("ok\n");
  return 0;
}
