// CPU oracle of Algorithm 1 (the LDL^T of the Hankel moment matrix,
// arXiv 1810.01478 Sec. 4.3) in C++ with OpenMP, following the paper's own
// parallel loop (Sec. 4.3.3): the trailing update as one flattened loop over
// the trailing triangle, run from the last index down to the first, with
// OpenMP dynamic scheduling and chunk = max(5, iterations / (200 threads)).
//
// TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
// CPU-baseline legs of bench.py run this program; nothing in the library
// links or calls it.  It shares no code with the CUDA path.
//
// Number format (the same definition the Python oracle oracle/mpfloat.py
// and the library use, implemented independently): a value is
//   (-1)^sign * M * 2^(32 exp),  M = sum_k m[k] 2^(32 k), k < n,
// with m[n-1] != 0, or M = 0 with sign = exp = 0.  Every operation forms its
// exact result and truncates the magnitude toward zero to n limbs (Sec. 4.1's
// "compute exactly, then truncate").
//
// Modes (all sizes in bits must be multiples of 32):
//   hk_oracle factor <m> <N> <bits> <file>
//       LDL^T of H_N for beta = 1/m (mu_j = m (m(j+1)-1)!); writes the packed
//       factor, column by column (D_c, then L[r][c] for r > c), each entry
//       as int32 sign, int32 exp, n uint32 limbs, little endian.
//   hk_oracle time <m> <N> <bits> <cols>
//       step 0 of Algorithm 1 on H_N: the column scale, then the trailing
//       updates of columns 1..cols (all N-1 of them when cols = 0); prints
//       one JSON line with the seconds of each part, the operation counts
//       and the OpenMP thread count.
//   hk_oracle prims <n>
//       reads lines "F a x y" (trunc(a - x y)) or "Q a d" (trunc(a / d)),
//       each number as "sign exp limb0 limb1 ... limb(n-1)" in hex, and
//       prints each result in the same form.
#include <omp.h>

#include <chrono>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <stdexcept>
#include <string>
#include <vector>

namespace {

typedef uint32_t u32;
typedef uint64_t u64;

// A number of the format: sign, exponent and a pointer to its n limbs.
struct Num {
  int32_t sign;
  int32_t exp;
  u32* m;
};

bool is_zero(const u32* m, int n) { return m[n - 1] == 0; }

// ---------------------------------------------------------------------------
// magnitudes (little-endian limb vectors)
// ---------------------------------------------------------------------------
// p[0 .. nx+ny) = x * y (schoolbook)
void mag_mul(const u32* x, int nx, const u32* y, int ny, u32* p) {
  std::memset(p, 0, sizeof(u32) * (nx + ny));
  for (int i = 0; i < nx; ++i) {
    u64 carry = 0;
    const u64 xi = x[i];
    for (int j = 0; j < ny; ++j) {
      const u64 t = xi * y[j] + p[i + j] + carry;
      p[i + j] = (u32)t;
      carry = t >> 32;
    }
    p[i + ny] = (u32)carry;
  }
}

// compare a and b (both len limbs): -1, 0, 1
int mag_cmp(const u32* a, const u32* b, int len) {
  for (int i = len - 1; i >= 0; --i)
    if (a[i] != b[i]) return a[i] < b[i] ? -1 : 1;
  return 0;
}

// Truncate the exact value (-1)^sign * V * 2^(32 e), V = v[0 .. len), to n
// limbs: the top n limbs of V from its highest non-zero limb down (limbs
// below v[0] count as zero).
void round_to(int sign, const u32* v, int len, int64_t e, int n, Num& out) {
  int top = len - 1;
  while (top >= 0 && v[top] == 0) --top;
  if (top < 0) {
    out.sign = 0;
    out.exp = 0;
    std::memset(out.m, 0, sizeof(u32) * n);
    return;
  }
  const int low = top - n + 1;  // index of the kept lowest limb (may be < 0)
  for (int k = 0; k < n; ++k) {
    const int i = low + k;
    out.m[k] = (i >= 0) ? v[i] : 0u;
  }
  const int64_t ex = e + low;
  if (ex < INT32_MIN || ex > INT32_MAX) throw std::runtime_error("exponent out of range");
  out.sign = sign;
  out.exp = (int32_t)ex;
}

// per-thread work areas of the primitives
struct Scratch {
  std::vector<u32> p, X, Y, R, U, V, Q;
};

// ---------------------------------------------------------------------------
// the two primitives of Algorithm 1
// ---------------------------------------------------------------------------
// out = trunc_n(a - x y), the product exact (one rounding).  The exact
// difference is formed in a frame that starts at the lower of the two
// exponents and holds both operands whole.  out may alias a.
void fused(const Num& a, const Num& x, const Num& y, int n, Num& out, Scratch& w) {
  const bool pz = is_zero(x.m, n) || is_zero(y.m, n);
  const bool az = is_zero(a.m, n);
  if (pz) {
    // a itself (already in the format)
    out.sign = a.sign;
    out.exp = a.exp;
    if (out.m != a.m) std::memcpy(out.m, a.m, sizeof(u32) * n);
    return;
  }
  const int psign = x.sign ^ y.sign;
  const int64_t pe = (int64_t)x.exp + y.exp;
  w.p.resize(2 * n);
  mag_mul(x.m, n, y.m, n, w.p.data());
  if (az) {
    round_to(psign ^ 1, w.p.data(), 2 * n, pe, n, out);
    return;
  }
  const int64_t e = a.exp < pe ? (int64_t)a.exp : pe;
  const int64_t oa = a.exp - e, op = pe - e;  // limb offsets in the frame
  const int64_t len64 = std::max<int64_t>(oa + n, op + 2 * n) + 1;
  if (len64 > (1 << 24)) throw std::runtime_error("exponent gap too large for the frame");
  const int len = (int)len64;
  w.X.assign(len, 0u);
  w.Y.assign(len, 0u);
  w.R.assign(len, 0u);
  for (int k = 0; k < n; ++k) w.X[oa + k] = a.m[k];
  for (int k = 0; k < 2 * n; ++k) w.Y[op + k] = w.p[k];
  // a - P = (-1)^a.sign |a| - (-1)^psign |P|
  int rsign;
  if (a.sign != psign) {
    // opposite signs: the magnitudes add, the sign is a's
    u64 c = 0;
    for (int k = 0; k < len; ++k) {
      const u64 t = (u64)w.X[k] + w.Y[k] + c;
      w.R[k] = (u32)t;
      c = t >> 32;
    }
    rsign = a.sign;
  } else {
    // same signs: |a| - |P| with a's sign if |a| >= |P|, else the flipped sign
    const bool a_ge = mag_cmp(w.X.data(), w.Y.data(), len) >= 0;
    const u32* big = a_ge ? w.X.data() : w.Y.data();
    const u32* small = a_ge ? w.Y.data() : w.X.data();
    u64 b = 0;
    for (int k = 0; k < len; ++k) {
      const u64 sub = (u64)small[k] + b;
      const u64 cur = big[k];
      w.R[k] = (u32)(cur - sub);
      b = cur < sub ? 1u : 0u;
    }
    rsign = a_ge ? a.sign : (a.sign ^ 1);
  }
  round_to(rsign, w.R.data(), len, e, n, out);
}

// Q[0 .. lu-nv+1) = floor(U / V) by long division in base 2^32 (Knuth,
// TAOCP vol. 2, 4.3.1, Algorithm D): U has lu limbs, V has nv >= 2 limbs
// with V[nv-1] != 0.  Each quotient limb is estimated from the top two limbs
// of the remainder and the top limb of the divisor (both normalised so that
// the divisor's top bit is set), corrected with the divisor's second limb,
// and fixed by one add-back when the multiply-subtract goes negative.
void mag_divide(const u32* U, int lu, const u32* V, int nv, u32* Q, Scratch& w) {
  const int sh = __builtin_clz(V[nv - 1]);
  w.V.assign(nv, 0u);
  w.U.assign(lu + 1, 0u);
  for (int i = nv - 1; i > 0; --i) w.V[i] = (V[i] << sh) | (sh ? (u32)((u64)V[i - 1] >> (32 - sh)) : 0u);
  w.V[0] = V[0] << sh;
  w.U[lu] = sh ? (u32)((u64)U[lu - 1] >> (32 - sh)) : 0u;
  for (int i = lu - 1; i > 0; --i) w.U[i] = (U[i] << sh) | (sh ? (u32)((u64)U[i - 1] >> (32 - sh)) : 0u);
  w.U[0] = U[0] << sh;
  const u64 B = (u64)1 << 32;
  const u64 v1 = w.V[nv - 1], v2 = w.V[nv - 2];
  for (int j = lu - nv; j >= 0; --j) {
    const u64 num = ((u64)w.U[j + nv] << 32) | w.U[j + nv - 1];
    u64 qhat = num / v1, rhat = num % v1;
    while (qhat >= B || qhat * v2 > ((rhat << 32) | w.U[j + nv - 2])) {
      --qhat;
      rhat += v1;
      if (rhat >= B) break;
    }
    // U[j .. j+nv] -= qhat V
    u64 carry = 0, borrow = 0;
    for (int i = 0; i < nv; ++i) {
      const u64 p = qhat * w.V[i] + carry;
      carry = p >> 32;
      const u64 sub = (p & 0xFFFFFFFFu) + borrow;
      const u64 cur = w.U[i + j];
      w.U[i + j] = (u32)(cur - sub);
      borrow = cur < sub ? 1u : 0u;
    }
    const u64 sub = carry + borrow;
    const u64 cur = w.U[j + nv];
    w.U[j + nv] = (u32)(cur - sub);
    if (cur < sub) {
      // qhat was one too large: add V back
      --qhat;
      u64 c = 0;
      for (int i = 0; i < nv; ++i) {
        const u64 t = (u64)w.U[i + j] + w.V[i] + c;
        w.U[i + j] = (u32)t;
        c = t >> 32;
      }
      w.U[j + nv] = (u32)((u64)w.U[j + nv] + c);
    }
    Q[j] = (u32)qhat;
  }
}

// out = trunc_n(a / d), the exact quotient with its magnitude floored to n
// limbs (Algorithm 1's B_i[j] = A_i[j] / A_i[i]).  With |a| = A, |d| = D (n
// limbs each): floor(A 2^(32 n) / D) has n limbs when A < D; when A >= D the
// numerator A 2^(32 (n-1)) gives the n-limb quotient and the exponent grows
// by one.
void divide(const Num& a, const Num& d, int n, Num& out, Scratch& w) {
  if (is_zero(d.m, n)) throw std::runtime_error("division by a zero pivot");
  if (is_zero(a.m, n)) {
    out.sign = 0;
    out.exp = 0;
    std::memset(out.m, 0, sizeof(u32) * n);
    return;
  }
  const bool ge = mag_cmp(a.m, d.m, n) >= 0;
  const int lu = ge ? 2 * n - 1 : 2 * n;  // A shifted up by n-1 or n limbs
  std::vector<u32> num(lu, 0u);
  for (int k = 0; k < n; ++k) num[lu - n + k] = a.m[k];
  w.Q.assign(lu - n + 1, 0u);
  mag_divide(num.data(), lu, d.m, n, w.Q.data(), w);
  for (int k = n; k < lu - n + 1; ++k)
    if (w.Q[k]) throw std::runtime_error("quotient longer than n limbs");
  std::memcpy(out.m, w.Q.data(), sizeof(u32) * n);
  out.sign = a.sign ^ d.sign;
  const int64_t ex = (int64_t)a.exp - d.exp - n + (ge ? 1 : 0);
  out.exp = (int32_t)ex;
}

}  // namespace

namespace {

// ---------------------------------------------------------------------------
// moments and the packed matrix
// ---------------------------------------------------------------------------
// The packed lower triangle of H_N, column major (column c holds rows c..N-1
// from offset c N - c (c - 1) / 2): the factor's layout on output too.
struct Tri {
  int N = 0, n = 0;
  std::vector<int32_t> sign, exp;
  std::vector<u32> mant;
  int64_t pos(int r, int c) const { return (int64_t)c * N - (int64_t)c * (c - 1) / 2 + (r - c); }
  Num at(int r, int c) {
    const int64_t p = pos(r, c);
    return Num{sign[p], exp[p], mant.data() + p * n};
  }
  void store(int r, int c, const Num& v) {
    const int64_t p = pos(r, c);
    sign[p] = v.sign;
    exp[p] = v.exp;
    if (v.m != mant.data() + p * n) std::memcpy(mant.data() + p * n, v.m, sizeof(u32) * n);
  }
};

// mu_j = m (m (j + 1) - 1)!, j = 0 .. 2N-2 (beta = 1/m, Sec. 2), each exact
// integer truncated to n limbs.
void moments(int m, int N, int n, std::vector<int32_t>& sg, std::vector<int32_t>& ex, std::vector<u32>& mt) {
  const int J = 2 * N - 1;
  sg.assign(J, 0);
  ex.assign(J, 0);
  mt.assign((size_t)J * n, 0u);
  std::vector<u32> f(1, 1u);  // K! for K = 0, 1, ...
  int K = 0;
  auto mul_small = [](std::vector<u32>& v, u32 s) {
    u64 c = 0;
    for (auto& w : v) {
      const u64 t = (u64)w * s + c;
      w = (u32)t;
      c = t >> 32;
    }
    if (c) v.push_back((u32)c);
  };
  for (int j = 0; j < J; ++j) {
    const int target = m * (j + 1) - 1;
    while (K < target) mul_small(f, (u32)(++K));
    std::vector<u32> mu = f;
    mul_small(mu, (u32)m);
    Num out{0, 0, mt.data() + (size_t)j * n};
    round_to(0, mu.data(), (int)mu.size(), 0, n, out);
    sg[j] = out.sign;
    ex[j] = out.exp;
  }
}

void assemble(Tri& A, int N, int n, const std::vector<int32_t>& sg, const std::vector<int32_t>& ex,
              const std::vector<u32>& mt) {
  A.N = N;
  A.n = n;
  const int64_t tri = (int64_t)N * (N + 1) / 2;
  A.sign.assign(tri, 0);
  A.exp.assign(tri, 0);
  A.mant.assign(tri * n, 0u);
  for (int c = 0; c < N; ++c)
    for (int r = c; r < N; ++r) {
      const int64_t p = A.pos(r, c);
      A.sign[p] = sg[r + c];
      A.exp[p] = ex[r + c];
      std::memcpy(A.mant.data() + p * n, mt.data() + (size_t)(r + c) * n, sizeof(u32) * n);
    }
}

// Column cc of the trailing triangle of size m (column cc holds m - cc
// entries) that contains flattened index t, t in [0, m (m + 1) / 2).
int64_t col_of(int64_t m, int64_t t) {
  auto off = [m](int64_t cc) { return cc * m - cc * (cc - 1) / 2; };
  const double b = 2.0 * (double)m + 1.0;
  int64_t cc = (int64_t)((b - std::sqrt(b * b - 8.0 * (double)t)) / 2.0);
  if (cc < 0) cc = 0;
  if (cc > m - 1) cc = m - 1;
  while (cc > 0 && off(cc) > t) --cc;
  while (cc < m - 1 && off(cc + 1) <= t) ++cc;
  return cc;
}

struct StepTimes {
  double scale_s = 0, update_s = 0;
  int64_t quotients = 0, updates = 0;
};

// Step i of Algorithm 1 (Sec. 4.3, 0-based): B_i[r] = A[r][i] / A[i][i] for
// r > i, then A[r][c] = A[r][c] - A[c][i] B_i[r] for i < c <= r (the column
// index supplies the unscaled entry, the row index the scaled one), then
// column i of L is B_i.  The update runs over the columns i+1 .. i+cols of
// the trailing triangle only (every column when cols <= 0).
//
// The update is the paper's single flattened loop (Sec. 4.3.3): one index
// over the whole trailing triangle, OpenMP dynamic scheduling with
// chunk = max(5, iterations / (200 threads)), from the last index down to
// the first.
bool step(Tri& A, int i, int cols, StepTimes& st) {
  const int N = A.N, n = A.n;
  Num d = A.at(i, i);
  if (is_zero(d.m, n) || d.sign) return false;  // a non-positive pivot
  const int m = N - 1 - i;
  std::vector<int32_t> us(N), ue(N), bs(N), be(N);
  std::vector<u32> um((size_t)N * n), bm((size_t)N * n);
  auto t0 = std::chrono::steady_clock::now();
#pragma omp parallel
  {
    Scratch w;
#pragma omp for schedule(dynamic)
    for (int r = i + 1; r < N; ++r) {
      Num a = A.at(r, i);
      us[r] = a.sign;
      ue[r] = a.exp;
      std::memcpy(um.data() + (size_t)r * n, a.m, sizeof(u32) * n);
      Num b{0, 0, bm.data() + (size_t)r * n};
      divide(a, d, n, b, w);
      bs[r] = b.sign;
      be[r] = b.exp;
    }
  }
  auto t1 = std::chrono::steady_clock::now();
  const int ncols = (cols <= 0 || cols > m) ? m : cols;
  // flattened entries of the first ncols columns of the trailing triangle
  const int64_t iters = (int64_t)ncols * m - (int64_t)ncols * (ncols - 1) / 2;
  const int threads = omp_get_max_threads();
  const int64_t chunk = std::max<int64_t>(5, iters / (200 * (int64_t)threads));
#pragma omp parallel
  {
    Scratch w;
#pragma omp for schedule(dynamic, chunk)
    for (int64_t t = iters - 1; t >= 0; --t) {
      const int64_t cc = col_of(m, t);
      const int64_t rr = t - (cc * m - cc * (cc - 1) / 2);  // 0 .. m - cc - 1
      const int c = i + 1 + (int)cc, r = c + (int)rr;
      Num a = A.at(r, c);
      const Num u{us[c], ue[c], um.data() + (size_t)c * n};
      const Num b{bs[r], be[r], bm.data() + (size_t)r * n};
      fused(a, u, b, n, a, w);
      A.store(r, c, a);
    }
  }
  auto t2 = std::chrono::steady_clock::now();
  for (int r = i + 1; r < N; ++r) A.store(r, i, Num{bs[r], be[r], bm.data() + (size_t)r * n});
  st.scale_s += std::chrono::duration<double>(t1 - t0).count();
  st.update_s += std::chrono::duration<double>(t2 - t1).count();
  st.quotients += m;
  st.updates += iters;
  return true;
}

// ---------------------------------------------------------------------------
// text I/O of the prims mode
// ---------------------------------------------------------------------------
bool read_num(FILE* f, int n, int32_t& sg, int32_t& ex, std::vector<u32>& m) {
  long long s, e;
  if (std::fscanf(f, "%llx %llx", &s, &e) != 2) return false;
  sg = (int32_t)s;
  ex = (int32_t)(uint32_t)e;
  m.assign(n, 0u);
  for (int k = 0; k < n; ++k) {
    unsigned long v;
    if (std::fscanf(f, "%lx", &v) != 1) return false;
    m[k] = (u32)v;
  }
  return true;
}

void print_num(const Num& v, int n) {
  std::printf("%x %x", (unsigned)v.sign, (unsigned)(uint32_t)v.exp);
  for (int k = 0; k < n; ++k) std::printf(" %x", (unsigned)v.m[k]);
  std::printf("\n");
}

}  // namespace

int main(int argc, char** argv) {
  if (argc < 2) {
    std::fprintf(stderr, "usage: hk_oracle factor|time|prims ...\n");
    return 2;
  }
  const std::string mode = argv[1];
  try {
    if (mode == "prims" && argc == 3) {
      const int n = std::atoi(argv[2]);
      Scratch w;
      char op[4];
      while (std::fscanf(stdin, "%3s", op) == 1) {
        int32_t s[3], e[3];
        std::vector<u32> m[3];
        const int cnt = op[0] == 'F' ? 3 : 2;
        for (int k = 0; k < cnt; ++k)
          if (!read_num(stdin, n, s[k], e[k], m[k])) throw std::runtime_error("bad operand");
        std::vector<u32> om(n, 0u);
        Num out{0, 0, om.data()};
        Num a{s[0], e[0], m[0].data()}, x{s[1], e[1], m[1].data()};
        if (cnt == 3) {
          Num y{s[2], e[2], m[2].data()};
          fused(a, x, y, n, out, w);
        } else {
          divide(a, x, n, out, w);
        }
        print_num(out, n);
      }
      return 0;
    }
    if ((mode == "factor" || mode == "time") && argc == 6) {
      const int m = std::atoi(argv[2]), N = std::atoi(argv[3]), bits = std::atoi(argv[4]);
      if (m < 1 || N < 1 || bits < 64 || bits % 32) throw std::runtime_error("bad sizes");
      const int n = bits / 32;
      std::vector<int32_t> sg, ex;
      std::vector<u32> mt;
      moments(m, N, n, sg, ex, mt);
      Tri A;
      assemble(A, N, n, sg, ex, mt);
      StepTimes st;
      if (mode == "time") {
        const int cols = std::atoi(argv[5]);
        if (!step(A, 0, cols, st)) throw std::runtime_error("non-positive pivot");
        std::printf(
            "{\"threads\": %d, \"N\": %d, \"bits\": %d, \"scale_seconds\": %.6f, \"quotients\": %lld, "
            "\"update_seconds\": %.6f, \"updates\": %lld}\n",
            omp_get_max_threads(), N, bits, st.scale_s, (long long)st.quotients, st.update_s,
            (long long)st.updates);
        return 0;
      }
      for (int i = 0; i < N; ++i)
        if (!step(A, i, 0, st)) throw std::runtime_error("non-positive pivot at step " + std::to_string(i));
      FILE* f = std::fopen(argv[5], "wb");
      if (!f) throw std::runtime_error("cannot open the output file");
      for (int c = 0; c < N; ++c)
        for (int r = c; r < N; ++r) {
          const int64_t p = A.pos(r, c);
          std::fwrite(&A.sign[p], 4, 1, f);
          std::fwrite(&A.exp[p], 4, 1, f);
          std::fwrite(A.mant.data() + p * n, 4, n, f);
        }
      std::fclose(f);
      return 0;
    }
  } catch (const std::exception& e) {
    std::fprintf(stderr, "hk_oracle: %s\n", e.what());
    return 1;
  }
  std::fprintf(stderr, "hk_oracle: bad arguments\n");
  return 2;
}
