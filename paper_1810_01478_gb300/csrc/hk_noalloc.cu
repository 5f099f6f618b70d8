// hk_ldlt_noalloc: the LDL^T factorisation for callers that must not allocate
// device memory.
//
// hk_ldlt needs scratch besides its input (the moments) and its output (the
// factor): the unscaled pivot column U (N numbers), the pivot's reciprocal
// (n limbs) and an error word.  It gets them from cudaMalloc.  Some callers
// cannot let a library allocate: a process whose device memory is owned by
// one allocator (a framework's caching allocator or a fixed serving budget,
// where a foreign cudaMalloc can fail or fragment the pool), or code that runs
// where a plain cudaMalloc is not allowed.  This entry point instead takes its
// scratch from one fixed array in device memory, declared below, so a call
// makes no allocation at all; the caller still passes the moments and the
// factor buffer.

#include "ctx.h"
#include "widths.h"

namespace {

// Scratch of hk_ldlt_noalloc: HK_NOALLOC_SCRATCH_WORDS 32-bit words (4 MiB).
// Every GPU that loads libhk holds this array until the process exits.  All
// calls share it, so calls whose work overlaps on the GPU (two streams, or two
// host threads) race on it and must be serialised by the caller.
constexpr size_t kScratchWords = HK_NOALLOC_SCRATCH_WORDS;
static __device__ __align__(256) uint32_t hk_noalloc_scratch[kScratchWords];

// Host code cannot use the array's name as a device address: the address is
// looked up on every call (with the caller's device current), so nothing
// goes stale when a device is reset and the module reloaded.
hk_status scratch_for_current_device(uint32_t** out) {
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, hk_noalloc_scratch) != cudaSuccess || !p) return HK_ERR_CUDA;
  *out = static_cast<uint32_t*>(p);
  return HK_OK;
}

}  // namespace

extern "C" hk_status hk_ldlt_noalloc(int bits, int N, const int32_t* mu_sign, const int32_t* mu_exp,
                                     const uint32_t* mu_limbs, int32_t* f_sign, int32_t* f_exp, uint32_t* f_limbs,
                                     void* cuda_stream) {
  using namespace hk;
  if (bits <= 0 || bits % 1024 != 0 || N < 1) return HK_ERR_ARG;
  const int n = bits / 32;
  // layout inside the scratch: U mantissas | U signs | U exps | rec (16-byte aligned) | meta | error word
  const size_t u_words = (size_t)N * n + 2 * (size_t)N;
  const size_t rec_off = (u_words + 3) / 4 * 4;
  const size_t need = rec_off + (size_t)n + 32;
  if (need > kScratchWords) return HK_ERR_ARG;  // N (bits/32 + 2) + bits/32 + 35 words must fit
  const OpsTable* ops = ops_for(bits / 1024);
  if (!ops) return HK_ERR_ARG;
  if (!mu_sign || !mu_exp || !mu_limbs || !f_sign || !f_exp || !f_limbs) return HK_ERR_ARG;
  uint32_t* base = nullptr;
  hk_status st = scratch_for_current_device(&base);
  if (st != HK_OK) return st;
  int dev = 0;
  cudaGetDevice(&dev);
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  MPVec U{reinterpret_cast<int32_t*>(base + (size_t)N * n), reinterpret_cast<int32_t*>(base + (size_t)N * n + N),
          base};
  uint32_t* rec = base + rec_off;
  int* rec_meta = reinterpret_cast<int*>(rec + n);
  int* err = rec_meta + 16;
  // the error word keeps the previous call's value: clear it
  if (cudaMemsetAsync(err, 0, sizeof(int), s) != cudaSuccess) return HK_ERR_CUDA;
  const MPVec mu{const_cast<int32_t*>(mu_sign), const_cast<int32_t*>(mu_exp), const_cast<uint32_t*>(mu_limbs)};
  const MPVec A{f_sign, f_exp, f_limbs};
  if (ops->ldlt_raw(mu, A, U, rec, rec_meta, err, N, s, dev) != cudaSuccess) return HK_ERR_CUDA;
  int flags = 0;
  if (cudaMemcpyAsync(&flags, err, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return HK_ERR_CUDA;
  // the same status for the same device flags as every other entry point
  return status_of_flags(flags, nullptr);
}
