// Device-side containers and index maps shared by the kernels.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace hk {

// Device error flags, OR-ed into one int per context.
enum ErrBits : int {
  ERR_NOT_PD = 1,        // a pivot d_i <= 0 (Sec. 4.3 footnote: H is positive definite)
  ERR_LOOP = 2,          // a correction loop exceeded its bound (should never happen)
  ERR_PRECISION = 4,     // the working precision was too low for the requested result
  ERR_ARG = 8,
  ERR_TIMEOUT = 16,      // a bounded device wait gave up (the kernel returned without finishing);
                         // bits 8..11 then name the wait (a kernel's own numbering of its call sites)
};


// An array of multiprecision numbers in structure-of-arrays layout:
// sgn[i] in {0, 1}, exp[i] the limb exponent, mant[i*n .. i*n+n) the limbs
// (little endian, top limb non-zero unless the number is zero).
struct MPVec {
  int32_t* sgn;
  int32_t* exp;
  uint32_t* mant;
};

// Packed lower triangle, column major: column c holds rows c..N-1.
__host__ __device__ __forceinline__ int64_t tri_pos(int64_t N, int64_t r, int64_t c) {
  return c * N - c * (c - 1) / 2 + (r - c);
}

// Packed strictly-lower part of the trailing block of step i: column cc (0..m-1)
// holds m - cc entries.  Offset of column cc:
__host__ __device__ __forceinline__ int64_t trail_off(int64_t m, int64_t cc) {
  return cc * m - cc * (cc - 1) / 2;
}

// Inverse of trail_off: column of linear index t (0 <= t < m(m+1)/2).
__host__ __device__ __forceinline__ int64_t trail_col(int64_t m, int64_t t) {
  const double b = 2.0 * (double)m + 1.0;
  int64_t cc = (int64_t)((b - sqrt(b * b - 8.0 * (double)t)) * 0.5);
  if (cc < 0) cc = 0;
  if (cc > m - 1) cc = m - 1;
  while (cc > 0 && trail_off(m, cc) > t) --cc;
  while (cc < m - 1 && trail_off(m, cc + 1) <= t) ++cc;
  return cc;
}

}  // namespace hk
