// The C ABI of libhk (declared in include/hk.h): context management, call-order
// enforcement, host <-> device transfers and dispatch to the per-width launchers.
#include <algorithm>
#include <atomic>
#include <mutex>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <functional>
#include <map>
#include <new>
#include <thread>

#include "ctx.h"
#include "k_moments.cuh"
#include "widths.h"

namespace hk {

#define HK_DECL(m) const OpsTable* ops_m##m();
HK_FOR_EACH_M(HK_DECL)
#undef HK_DECL

const OpsTable* ops_for(int M) {
#define HK_CASE(m) \
  if (M == m) return ops_m##m();
  HK_FOR_EACH_M(HK_CASE)
#undef HK_CASE
  return nullptr;
}

// ---------------------------------------------------------------------------
// product algorithm and NTT tables
// ---------------------------------------------------------------------------
static std::atomic<int> g_product_alg(HK_PRODUCT_AUTO);

int product_algorithm() { return g_product_alg.load(); }

bool use_ntt(int M) {
  const int a = product_algorithm();
  if (a == HK_PRODUCT_NTT) return 32 * M * 2 <= NTT_LMAX;
  if (a == HK_PRODUCT_SCHOOLBOOK) return false;
  return M >= HK_NTT_AUTO_MIN_M && 32 * M * 2 <= NTT_LMAX;
}

bool use_tc(int M) {
  const int a = product_algorithm();
  if (M < HK_TC_MIN_M || !use_ntt(M)) return false;
  return a == HK_PRODUCT_TENSOR || (a == HK_PRODUCT_AUTO && M >= HK_TC_AUTO_MIN_M);
}

namespace {
// the three largest primes k 3 2^11 + 1 below 2^30 (p1 > p2 > p3, p1 < 2 p3)
// with primitive roots 23, 5, 10
constexpr uint32_t kPrimes[NTT_Q] = {1073707009u, 1073682433u, 1073651713u};
constexpr uint32_t kGen[NTT_Q] = {23u, 5u, 10u};

uint32_t pow_mod(uint64_t b, uint64_t e, uint32_t p) {
  uint64_t r = 1;
  b %= p;
  while (e) {
    if (e & 1) r = r * b % p;
    b = b * b % p;
    e >>= 1;
  }
  return (uint32_t)r;
}
uint32_t shoup(uint32_t w, uint32_t p) { return (uint32_t)(((uint64_t)w << 32) / p); }
uint32_t inv_mod(uint32_t a, uint32_t p) { return pow_mod(a, p - 2, p); }

struct NttTables {
  uint2* twf = nullptr;
  uint2* twi = nullptr;
};
std::mutex g_ntt_mu;
NttTables g_ntt[64];
}  // namespace

NttConst ntt_const(int n) {
  int dev = 0;
  cudaGetDevice(&dev);
  NttConst nc{};
  {
    std::lock_guard<std::mutex> lock(g_ntt_mu);
    NttTables& t = g_ntt[dev & 63];
    if (!t.twf) {
      std::vector<uint2> f((size_t)NTT_Q * NTT_LMAX / 2), iv((size_t)NTT_Q * NTT_LMAX / 2);
      for (int q = 0; q < NTT_Q; ++q) {
        const uint32_t p = kPrimes[q];
        const uint32_t w = pow_mod(kGen[q], (p - 1) / NTT_LMAX, p), wi = inv_mod(w, p);
        uint64_t a = 1, b = 1;
        for (int k = 0; k < NTT_LMAX / 2; ++k) {
          f[(size_t)q * NTT_LMAX / 2 + k] = make_uint2((uint32_t)a, shoup((uint32_t)a, p));
          iv[(size_t)q * NTT_LMAX / 2 + k] = make_uint2((uint32_t)b, shoup((uint32_t)b, p));
          a = a * w % p;
          b = b * wi % p;
        }
      }
      const size_t bytes = f.size() * sizeof(uint2);
      if (cudaMalloc(&t.twf, bytes) == cudaSuccess && cudaMalloc(&t.twi, bytes) == cudaSuccess) {
        cudaMemcpy(t.twf, f.data(), bytes, cudaMemcpyHostToDevice);
        cudaMemcpy(t.twi, iv.data(), bytes, cudaMemcpyHostToDevice);
      }
    }
    nc.twf = t.twf;
    nc.twi = t.twi;
  }
  const int L = ntt_len(n);
  nc.L = L;
  nc.logL = ntt_logk(n);
  for (int q = 0; q < NTT_Q; ++q) {
    const uint32_t p = kPrimes[q];
    nc.p[q] = p;
    nc.w3[q] = pow_mod(kGen[q], (p - 1) / 3, p);
    nc.w3s[q] = shoup(nc.w3[q], p);
    nc.w3i[q] = inv_mod(nc.w3[q], p);
    nc.w3is[q] = shoup(nc.w3i[q], p);
    uint32_t x = p;  // Newton: x = p^{-1} mod 2^32
    for (int it = 0; it < 5; ++it) x *= 2u - p * x;
    nc.pinv[q] = 0u - x;
    const uint32_t r = (uint32_t)((((uint64_t)1) << 32) % p);
    nc.rl[q] = (uint32_t)((uint64_t)r * inv_mod((uint32_t)L, p) % p);
    nc.rls[q] = shoup(nc.rl[q], p);
  }
  nc.i12 = inv_mod(kPrimes[0] % kPrimes[1], kPrimes[1]);
  nc.i12s = shoup(nc.i12, kPrimes[1]);
  nc.i13 = inv_mod(kPrimes[0], kPrimes[2]);
  nc.i13s = shoup(nc.i13, kPrimes[2]);
  nc.i23 = inv_mod(kPrimes[1], kPrimes[2]);
  nc.i23s = shoup(nc.i23, kPrimes[2]);
  nc.p12 = (uint64_t)kPrimes[0] * kPrimes[1];
  return nc;
}

cudaError_t dev_alloc(DevVec& v, int64_t count, int n) {
  v.count = count;
  v.n = n;
  cudaError_t e;
  const int64_t c = count > 0 ? count : 1;
  if ((e = cudaMalloc(&v.sgn, c * 4)) != cudaSuccess) return e;
  if ((e = cudaMalloc(&v.exp, c * 4)) != cudaSuccess) return e;
  if ((e = cudaMalloc(&v.mant, c * (int64_t)n * 4)) != cudaSuccess) return e;
  return cudaSuccess;
}

void dev_free(DevVec& v) {
  if (v.sgn) cudaFree(v.sgn);
  if (v.exp) cudaFree(v.exp);
  if (v.mant) cudaFree(v.mant);
  v = DevVec{};
}

hk_status set_error(Ctx& c, hk_status s, const std::string& msg) {
  if (c.sticky == HK_OK) {
    c.sticky = s;
    c.err = msg;
  }
  return s;
}

hk_status check_cuda(Ctx& c, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return HK_OK;
  const hk_status s = (e == cudaErrorMemoryAllocation) ? HK_ERR_NOMEM : HK_ERR_CUDA;
  return set_error(c, s, std::string(what) + ": " + cudaGetErrorString(e));
}

DevVec* pool_get(Ctx& c, const std::string& name, int64_t count) {
  DevVec& v = c.pool[name];
  if (v.count >= count && v.n == c.n && v.mant) return &v;
  if (v.mant) cudaStreamSynchronize(c.stream);  // earlier kernels may still read it
  if (v.mant && v.mant == c.one_mant) c.one_mant = nullptr;
  dev_free(v);
  if (dev_alloc(v, count, c.n) != cudaSuccess) {
    set_error(c, HK_ERR_NOMEM, "allocating scratch " + name);
    dev_free(v);
    return nullptr;
  }
  return &v;
}

hk_status upload_tasks(Ctx& c, const void* host, size_t bytes) {
  if (bytes > c.tasks_cap) {
    if (c.d_tasks) {
      cudaStreamSynchronize(c.stream);
      cudaFree(c.d_tasks);
      c.d_tasks = nullptr;
    }
    size_t cap = 1 << 16;
    while (cap < bytes) cap <<= 1;
    hk_status st = check_cuda(c, cudaMalloc(&c.d_tasks, cap), "allocating task buffer");
    if (st != HK_OK) return st;
    c.tasks_cap = cap;
  }
  // pageable source: the call returns once the bytes are staged, so the host
  // vector may be released; the device copy is ordered before later kernels
  return check_cuda(c, cudaMemcpyAsync(c.d_tasks, host, bytes, cudaMemcpyHostToDevice, c.stream), "task upload");
}

size_t prof_mark(Ctx& c) {
  if (c.ev_used == c.events.size()) {
    cudaEvent_t e;
    cudaEventCreate(&e);
    c.events.push_back(e);
  }
  cudaEventRecord(c.events[c.ev_used], c.stream);
  return c.ev_used++;
}

hk_status status_of_flags(int flags, const char** msg) {
  const char* m = "";
  hk_status st = HK_OK;
  // a kernel that gave up a wait left its results unfinished, so whatever
  // later kernels flagged may follow from that: report it first
  if (flags & ERR_TIMEOUT) {
    st = HK_ERR_TIMEOUT;
    m = "a bounded device wait gave up";
  } else if (flags & ERR_NOT_PD) {
    st = HK_ERR_NOT_PD;
    m = "a pivot d_i <= 0: raise the working precision";
  } else if (flags & ERR_PRECISION) {
    st = HK_ERR_PRECISION;
    m = "working precision too low";
  } else if (flags & ERR_LOOP) {
    st = HK_ERR_CUDA;
    m = "internal correction loop exceeded its bound";
  } else if (flags & ERR_ARG) {
    st = HK_ERR_ARG;
    m = "invalid device operand (zero divisor or capacity)";
  }
  if (msg) *msg = m;
  return st;
}

hk_status read_device_flags(Ctx& c) {
  hk_status st = check_cuda(c, cudaStreamSynchronize(c.stream), "synchronising");
  if (st != HK_OK) return st;
  int flags = 0;
  st = check_cuda(c, cudaMemcpy(&flags, c.d_err, sizeof(int), cudaMemcpyDeviceToHost), "reading device flags");
  if (st != HK_OK) return st;
  const char* msg = nullptr;
  st = status_of_flags(flags, &msg);
  if (st == HK_ERR_TIMEOUT && (flags >> 8)) return set_error(c, st, std::string(msg) + " (wait site " +
                                                                        std::to_string((flags >> 8) & 15) + ")");
  return st == HK_OK ? HK_OK : set_error(c, st, msg);
}

}  // namespace hk

using namespace hk;

struct hk_ctx {
  Ctx c;
};

static bool valid_bits(int bits) { return bits > 0 && bits % 1024 == 0 && ops_for(bits / 1024) != nullptr; }

static hk_status enter(hk_ctx* h) {
  if (!h) return HK_ERR_ARG;
  if (h->c.sticky != HK_OK) return h->c.sticky;
  return check_cuda(h->c, cudaSetDevice(h->c.device), "cudaSetDevice");
}

// Loss estimate of the factorisation: max(0, max_i ceil(log2(mu_{2i}/d_i)))
// over the pivots d_i = A[i][i].  Each pivot is what is left of its diagonal
// moment after the eliminations (Sec. 4.3), so the ratio counts the leading
// bits that cancelled.  One thread per pivot, into *out (cleared before);
// non-positive pivots are left to the ERR_NOT_PD flag.
__global__ void k_loss_estimate(MPVec MU, MPVec A, int N, int n, int* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const int64_t pd = tri_pos(N, i, i);
  const uint32_t* d = A.mant + pd * n;
  const uint32_t* m = MU.mant + (int64_t)(2 * i) * n;
  if (A.sgn[pd] || d[n - 1] == 0u || m[n - 1] == 0u) return;
  // the top two limbs give log2 of each to far better than a bit
  const double td = (double)d[n - 1] + (double)d[n - 2] * 0x1p-32;
  const double tm = (double)m[n - 1] + (double)m[n - 2] * 0x1p-32;
  const double l = 32.0 * ((double)MU.exp[2 * i] - (double)A.exp[pd]) + log2(tm) - log2(td);
  const int v = (int)ceil(fmin(l, 1.0e9));  // imported moments may carry any exponents
  if (v > 0) atomicMax(out, v);
}

// Throughput of the integer multiply pipe, in operations per SM clock: one
// block of kPeakThreads per SM (its dynamic shared memory keeps a second
// block off the SM), kPeakChains independent chains per thread, the block's
// clock64 span.  KIND 0: mad.lo.u32 (x = x x + c; an affine step would let
// the compiler merge unrolled steps into one); KIND 1: the lazy Shoup
// modular multiplication of the transforms (x w - hi(x w') p).
constexpr int kPeakThreads = 1024, kPeakChains = 8, kPeakIters = 1 << 14;
constexpr int kPeakSmem = 160 * 1024;

template <int KIND>
__global__ void __launch_bounds__(1024, 1) k_alu_peak(int iters, uint32_t seed, long long* span, uint32_t* sink) {
  uint32_t x[kPeakChains];
#pragma unroll
  for (int j = 0; j < kPeakChains; ++j) x[j] = seed + threadIdx.x * kPeakChains + j;
  const uint32_t p = 1073707009u, w = 0x2A3B4C5Du % 1073707009u;
  const uint32_t ws = (uint32_t)(((uint64_t)w << 32) / p);
  __syncthreads();
  const long long t0 = clock64();
#pragma unroll 4
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int j = 0; j < kPeakChains; ++j) {
      if constexpr (KIND == 0) x[j] = x[j] * x[j] + (0x7F4A7C15u + j);  // not affine: no folding of steps
      else x[j] = mul_shoup_lazy(x[j], w, ws, p);
    }
  }
  __syncthreads();
  const long long t1 = clock64();
  uint32_t acc = 0;
#pragma unroll
  for (int j = 0; j < kPeakChains; ++j) acc ^= x[j];
  if (acc == 0x5A5A5A5Au) sink[threadIdx.x & 15] = acc;  // keeps the chains live
  if (threadIdx.x == 0) span[blockIdx.x] = t1 - t0;
}

extern "C" {

int hk_supported_bits(int* out, int cap) {
  int cnt = 0;
#define HK_LIST(m)                      \
  if (out && cnt < cap) out[cnt] = 1024 * m; \
  ++cnt;
  HK_FOR_EACH_M(HK_LIST)
#undef HK_LIST
  return cnt;
}

hk_status hk_create(int device, void* cuda_stream, hk_ctx** out) {
  if (!out) return HK_ERR_ARG;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return HK_ERR_CUDA;
  hk_ctx* h = new (std::nothrow) hk_ctx();
  if (!h) return HK_ERR_NOMEM;
  h->c.device = device;
  h->c.stream = static_cast<cudaStream_t>(cuda_stream);
  if (cudaSetDevice(device) != cudaSuccess || cudaMalloc(&h->c.d_err, 64) != cudaSuccess ||
      cudaMemsetAsync(h->c.d_err, 0, 64, h->c.stream) != cudaSuccess) {
    if (h->c.d_err) cudaFree(h->c.d_err);
    delete h;
    return HK_ERR_CUDA;
  }
  *out = h;
  return HK_OK;
}

void hk_destroy(hk_ctx* h) {
  if (!h) return;
  cudaSetDevice(h->c.device);
  cudaStreamSynchronize(h->c.stream);
  Ctx& c = h->c;
  dev_free(c.mu);
  dev_free(c.A);
  dev_free(c.U);
  dev_free(c.X);
  dev_free(c.S);
  dev_free(c.evec);
  dev_free(c.psi);
  dev_free(c.scratch);
  for (auto& kv : c.pool) dev_free(kv.second);
  if (c.d_tasks) cudaFree(c.d_tasks);
  for (cudaEvent_t e : c.events) cudaEventDestroy(e);
  if (c.ev_diag) cudaEventDestroy(c.ev_diag);
  if (c.ev_recip) cudaEventDestroy(c.ev_recip);
  if (c.aux) cudaStreamDestroy(c.aux);
  for (cudaEvent_t e : c.ev_col) cudaEventDestroy(e);
  for (cudaEvent_t e : {c.ev_fork, c.ev_join, c.ev_ldlt_start, c.ev_a4})
    if (e) cudaEventDestroy(e);
  if (c.ms) cudaStreamDestroy(c.ms);
  if (c.a4) cudaStreamDestroy(c.a4);
  if (c.rec) cudaFree(c.rec);
  if (c.ntt_buf) cudaFree(c.ntt_buf);
  if (c.ntt_buf2) cudaFree(c.ntt_buf2);
  if (c.tc_db) cudaFree(c.tc_db);
  if (c.tc_du) cudaFree(c.tc_du);
  if (c.tc_p) cudaFree(c.tc_p);
  if (c.tc_redo) cudaFree(c.tc_redo);
  if (c.d_err) cudaFree(c.d_err);
  delete h;
}

const char* hk_last_error(const hk_ctx* h) { return h ? h->c.err.c_str() : "null context"; }

static hk_status begin_moments(hk_ctx* h, int N, int bits) {
  Ctx& c = h->c;
  if (N < 1 || N > (1 << 20)) return set_error(c, HK_ERR_ARG, "N out of range");
  if (!valid_bits(bits)) return set_error(c, HK_ERR_UNSUPPORTED, "bits must be 1024*M for a compiled M");
  c.N = N;
  c.bits = bits;
  c.n = bits / 32;
  c.M = bits / 1024;
  c.k = 0;
  c.stage = ST_NONE;
  if (c.mu.count != 2 * N - 1 || c.mu.n != c.n) {
    dev_free(c.mu);
    hk_status st = check_cuda(c, dev_alloc(c.mu, 2 * N - 1, c.n), "allocating moments");
    if (st != HK_OK) return st;
  }
  return check_cuda(c, cudaMemsetAsync(c.d_err, 0, 64, c.stream), "clearing flags");
}

hk_status hk_moments(hk_ctx* h, int64_t beta_num, int64_t beta_den, int N, int bits) {
  hk_status st = enter(h);
  if (st != HK_OK) return st;
  Ctx& c = h->c;
  if (beta_num <= 0 || beta_den <= 0) return set_error(c, HK_ERR_ARG, "beta must be positive");
  if (beta_den % beta_num != 0)
    return set_error(c, HK_ERR_UNSUPPORTED, "device moments need beta = 1/m; use hk_set_moments");
  const int64_t m = beta_den / beta_num;
  if (m > 64) return set_error(c, HK_ERR_UNSUPPORTED, "beta = 1/m with m > 64");
  if ((st = begin_moments(h, N, bits)) != HK_OK) return st;
  // limbs of G_{2N-2} = m * (m(2N-1) - 1)!
  const double top = (double)m * (2.0 * N - 1.0);
  const double bits_needed = (std::lgamma(top) + std::log((double)m)) / std::log(2.0) + 96.0;
  int64_t cap = ((int64_t)(bits_needed / 32.0) + 2 + 31) / 32 * 32;
  if (cap < 64) cap = 64;
  constexpr int kMomentsSmemCap = 200 * 1024;
  if (cap * 4 > kMomentsSmemCap) return set_error(c, HK_ERR_UNSUPPORTED, "moments too long for the exact kernel");
  // the attribute is process-wide: always set the same (maximal) cap, so that
  // contexts working concurrently never lower it under each other's launches
  if ((st = check_cuda(c, cudaFuncSetAttribute(k_moments_exact, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               kMomentsSmemCap),
                       "smem attribute")) != HK_OK)
    return st;
  const size_t pe0 = c.prof ? prof_mark(c) : 0;
  k_moments_exact<<<1, 32, cap * 4, c.stream>>>((int)m, N, c.n, (int)cap, c.mu.view(), c.d_err);
  count_launch(c);
  if (c.prof) c.stage_ev.push_back({0, {pe0, prof_mark(c)}});
  if ((st = check_cuda(c, cudaGetLastError(), "launching the moments")) != HK_OK) return st;
  c.beta_num = beta_num;
  c.beta_den = beta_den;
  c.stage = ST_MOMENTS;
  c.psi_count = -1;
  return HK_OK;
}

hk_status hk_moments_gamma(hk_ctx* h, int64_t beta_num, int64_t beta_den, int N, int bits, int nc,
                           const int32_t* c_exp, const uint32_t* c_limbs) {
  hk_status st = enter(h);
  if (st != HK_OK) return st;
  Ctx& c = h->c;
  if (beta_num <= 0 || beta_den <= 0) return set_error(c, HK_ERR_ARG, "beta must be positive");
  int64_t x = beta_num, y = beta_den;
  while (y) {
    const int64_t t = x % y;
    x = y;
    y = t;
  }
  const int64_t a = beta_num / x, b = beta_den / x;
  if (a == 1) return hk_moments(h, beta_num, beta_den, N, bits);
  if (a > 64) return set_error(c, HK_ERR_UNSUPPORTED, "beta = a/b with a > 64");
  if (nc < 1 || nc > 4096 || !c_exp || !c_limbs) return set_error(c, HK_ERR_ARG, "need a-1 constants of nc limbs");
  if (N < 1 || b * (2 * (int64_t)N - 1) >= (1ll << 31)) return set_error(c, HK_ERR_ARG, "b (2N-1) too large");
  for (int64_t r = 1; r < a; ++r)
    if (c_limbs[(r - 1) * nc + nc - 1] == 0u) return set_error(c, HK_ERR_ARG, "constants must be normalised");
  if ((st = begin_moments(h, N, bits)) != HK_OK) return st;
  // bits of G for the largest moment: 2^64 b M_r prod_{i<q} (r + i a), q = b(2N-1)/a
  const double q = (double)b * (2.0 * N - 1.0) / (double)a;
  const double gbits = 64.0 + std::log2((double)b) + 32.0 * nc + q * std::log2((double)a) +
                       (std::lgamma(q + 2.0)) / std::log(2.0) + 64.0;
  const int64_t cap = ((int64_t)(gbits / 32.0) + 2 + 31) / 32 * 32;
  constexpr int kWarps = 8;
  if (cap * 4 * kWarps > 200 * 1024) return set_error(c, HK_ERR_UNSUPPORTED, "moments too long for the kernel");
  int32_t* d_exp = nullptr;
  uint32_t* d_lim = nullptr;
  if ((st = check_cuda(c, cudaMallocAsync(&d_exp, (size_t)(a - 1) * 4, c.stream), "constants")) ||
      (st = check_cuda(c, cudaMallocAsync(&d_lim, (size_t)(a - 1) * nc * 4, c.stream), "constants")) ||
      (st = check_cuda(c, cudaMemcpyAsync(d_exp, c_exp, (size_t)(a - 1) * 4, cudaMemcpyHostToDevice, c.stream),
                       "constants H2D")) ||
      (st = check_cuda(c, cudaMemcpyAsync(d_lim, c_limbs, (size_t)(a - 1) * nc * 4, cudaMemcpyHostToDevice,
                                          c.stream), "constants H2D")) ||
      (st = check_cuda(c, cudaStreamSynchronize(c.stream), "constants H2D")))
    return st;
  if ((st = check_cuda(c, cudaFuncSetAttribute(k_moments_gamma, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               200 * 1024), "smem attribute")) != HK_OK)
    return st;
  const size_t pe0 = c.prof ? prof_mark(c) : 0;
  const int blocks = (2 * N - 1 + kWarps - 1) / kWarps;
  k_moments_gamma<<<blocks, 32 * kWarps, (size_t)cap * 4 * kWarps, c.stream>>>((int)a, (int)b, N, c.n, (int)cap,
                                                                               nc, d_exp, d_lim, c.mu.view(),
                                                                               c.d_err);
  count_launch(c);
  if (c.prof) c.stage_ev.push_back({0, {pe0, prof_mark(c)}});
  cudaFreeAsync(d_exp, c.stream);
  cudaFreeAsync(d_lim, c.stream);
  if ((st = check_cuda(c, cudaGetLastError(), "launching the moments")) != HK_OK) return st;
  c.beta_num = beta_num;
  c.beta_den = beta_den;
  c.stage = ST_MOMENTS;
  c.psi_count = -1;
  return HK_OK;
}

hk_status hk_set_psi_constants(hk_ctx* h, int count, int nc, const int32_t* sign, const int32_t* exp,
                               const uint32_t* limbs) {
  hk_status st = enter(h);
  if (st != HK_OK) return st;
  Ctx& c = h->c;
  if (c.stage < ST_MOMENTS) return set_error(c, HK_ERR_ORDER, "hk_set_psi_constants before the moments");
  if (count < 0 || count > 63 || nc < 1 || nc > 4096 || (count && (!sign || !exp || !limbs)))
    return set_error(c, HK_ERR_ARG, "psi constants: count in 0..63, nc >= 1, host arrays");
  const int n = c.n;
  // each constant truncated (or zero-extended) to the working width
  std::vector<int32_t> s(count), e(count);
  std::vector<uint32_t> m((size_t)count * n, 0u);
  for (int r = 0; r < count; ++r) {
    const uint32_t* src = limbs + (size_t)r * nc;
    if (src[nc - 1] == 0u) {
      for (int i = 0; i < nc; ++i)
        if (src[i]) return set_error(c, HK_ERR_ARG, "psi constants must be normalised");
      s[r] = 0;
      e[r] = 0;
      continue;
    }
    s[r] = sign[r] ? 1 : 0;
    e[r] = exp[r] + (nc - n);
    for (int i = 0; i < n; ++i) {
      const int j = nc - n + i;
      m[(size_t)r * n + i] = j >= 0 ? src[j] : 0u;
    }
  }
  if (c.psi.count != count || c.psi.n != n) {
    dev_free(c.psi);
    if (count && (st = check_cuda(c, dev_alloc(c.psi, count, n), "allocating psi")) != HK_OK) return st;
  }
  if (count &&
      ((st = check_cuda(c, cudaMemcpy(c.psi.sgn, s.data(), (size_t)count * 4, cudaMemcpyHostToDevice), "H2D")) ||
       (st = check_cuda(c, cudaMemcpy(c.psi.exp, e.data(), (size_t)count * 4, cudaMemcpyHostToDevice), "H2D")) ||
       (st = check_cuda(c, cudaMemcpy(c.psi.mant, m.data(), m.size() * 4, cudaMemcpyHostToDevice), "H2D"))))
    return st;
  c.psi_count = count;
  return HK_OK;
}

hk_status hk_set_moments(hk_ctx* h, int N, int bits, const int32_t* sign, const int32_t* exp,
                         const uint32_t* limbs, int64_t beta_num, int64_t beta_den) {
  hk_status st = enter(h);
  if (st != HK_OK) return st;
  Ctx& c = h->c;
  if (!sign || !exp || !limbs) return set_error(c, HK_ERR_ARG, "null host array");
  if ((st = begin_moments(h, N, bits)) != HK_OK) return st;
  const int64_t cnt = 2 * (int64_t)N - 1;
  if ((st = check_cuda(c, cudaMemcpyAsync(c.mu.sgn, sign, cnt * 4, cudaMemcpyHostToDevice, c.stream), "H2D")) ||
      (st = check_cuda(c, cudaMemcpyAsync(c.mu.exp, exp, cnt * 4, cudaMemcpyHostToDevice, c.stream), "H2D")) ||
      (st = check_cuda(c, cudaMemcpyAsync(c.mu.mant, limbs, cnt * c.n * 4, cudaMemcpyHostToDevice, c.stream),
                       "H2D")))
    return st;
  // the copies read pageable host memory: finish them before returning
  if ((st = check_cuda(c, cudaStreamSynchronize(c.stream), "H2D sync")) != HK_OK) return st;
  c.beta_num = beta_num;
  c.beta_den = beta_den;
  c.stage = ST_MOMENTS;
  c.psi_count = -1;
  return HK_OK;
}

// The rule on the loss estimate: the bits precision doubling shows lost stay
// below 2 loss + 32 (beta = 1/4 ... 1), so a result keeps 133 bits (1e-40)
// and 64 to spare when bits >= 2 loss + 32 + 197.
static int min_bits_for(int loss) { return (int)std::min<int64_t>(2 * (int64_t)loss + 229, 2000000000); }

static hk_status read_loss(Ctx& c, int& loss) {
  hk_status st = check_cuda(c, cudaStreamSynchronize(c.stream), "synchronising");
  if (st != HK_OK) return st;
  return check_cuda(c, cudaMemcpy(&loss, c.d_err + 1, sizeof(int), cudaMemcpyDeviceToHost), "reading the loss");
}

hk_status hk_ldlt(hk_ctx* h) {
  hk_status st = enter(h);
  if (st != HK_OK) return st;
  Ctx& c = h->c;
  if (c.stage < ST_MOMENTS) return set_error(c, HK_ERR_ORDER, "hk_ldlt before the moments");
  if (c.plan_k > c.N) return set_error(c, HK_ERR_ARG, "the planned k exceeds N");
  c.alg4_k = 0;
  c.alg4_done = 0;
  const size_t pe0 = c.prof ? prof_mark(c) : 0;
  st = ops_for(c.M)->ldlt(c);
  if (st == HK_OK && (st = check_cuda(c, cudaMemsetAsync(c.d_err + 1, 0, sizeof(int), c.stream), "clearing")) == HK_OK) {
    k_loss_estimate<<<(c.N + 127) / 128, 128, 0, c.stream>>>(c.mu.view(), c.A.view(), c.N, c.n, c.d_err + 1);
    count_launch(c);
    st = check_cuda(c, cudaGetLastError(), "k_loss_estimate");
  }
  if (c.prof) c.stage_ev.push_back({1, {pe0, prof_mark(c)}});
  if (st == HK_OK) c.stage = ST_LDLT;
  return st;
}

// Launch shape of the batched factorisation (blocks per SM, items per claim
// in the largest phases), per width and bucket of the largest N: what
// hk_tune_batch measured fastest, else a default.
namespace {
struct BatchShape {
  int blocks, chunk;
};
std::mutex g_tune_mu;
std::map<std::pair<int, int>, BatchShape> g_tune;
// untuned: the tuner's picks on one GB300 (8 blocks per SM at 2048 bits, 6
// at 4096, 4 at 8192; 8 items per claim)
BatchShape batch_default(int M) { return BatchShape{M <= 2 ? 8 : M <= 6 ? 6 : 4, 8}; }
int n_bucket(int N) {
  int b = 0;
  while (b < 8 && (128 << b) < N) ++b;
  return b;  // N <= 128, <= 256, ... , > 16384
}
BatchShape batch_shape(int M, int max_n) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  auto it = g_tune.find({M, n_bucket(max_n)});
  return it == g_tune.end() ? batch_default(M) : it->second;
}
}  // namespace

static hk_status ldlt_batch_shaped(hk_ctx* const* hs, int count, double idle_limit_s, const BatchShape* force);

hk_status hk_ldlt_batch(hk_ctx* const* hs, int count, double idle_limit_s) {
  return ldlt_batch_shaped(hs, count, idle_limit_s, nullptr);
}

static hk_status ldlt_batch_shaped(hk_ctx* const* hs, int count, double idle_limit_s, const BatchShape* force) {
  if (!hs || count < 1) return HK_ERR_ARG;
  std::vector<Ctx*> cs(count);
  for (int q = 0; q < count; ++q) {
    hk_status st = enter(hs[q]);
    if (st != HK_OK) return st;
    Ctx& c = hs[q]->c;
    if (c.stage < ST_MOMENTS) return set_error(c, HK_ERR_ORDER, "hk_ldlt_batch before the moments");
    if (c.plan_k > c.N) return set_error(c, HK_ERR_ARG, "the planned k exceeds N");
    // the launch's per-phase claim and done counters are 32-bit
    if (c.N > HK_BATCH_MAX_N) return set_error(c, HK_ERR_ARG, "hk_ldlt_batch serves N up to HK_BATCH_MAX_N");
    if (q > 0 && (c.device != cs[0]->device || c.M != cs[0]->M))
      return set_error(c, HK_ERR_ARG, "hk_ldlt_batch: every context must have the first one's device and width");
    for (int p = 0; p < q; ++p)
      if (cs[p] == &c) return set_error(c, HK_ERR_ARG, "hk_ldlt_batch: a context appears twice");
    cs[q] = &c;
  }
  if ((cs[0]->M > HK_BATCH_MAX_M))
    return set_error(*cs[0], HK_ERR_UNSUPPORTED, "hk_ldlt_batch serves widths up to 8192 bits");
  if (cudaSetDevice(cs[0]->device) != cudaSuccess) return HK_ERR_CUDA;
  const long long limit_ns =
      idle_limit_s < 0 ? 2000000000LL : (long long)std::min(idle_limit_s * 1e9, 3.6e12);
  for (Ctx* c : cs) {
    c->alg4_k = 0;
    c->alg4_done = 0;
  }
  int max_n = 0;
  for (Ctx* c : cs) max_n = std::max(max_n, c->N);
  const BatchShape shape = force ? *force : batch_shape(cs[0]->M, max_n);
  hk_status st = ops_for(cs[0]->M)->ldlt_batch(cs.data(), count, limit_ns, shape.blocks, shape.chunk);
  for (Ctx* cp : cs) {
    Ctx& c = *cp;
    if (st != HK_OK) break;
    if ((st = check_cuda(c, cudaMemsetAsync(c.d_err + 1, 0, sizeof(int), c.stream), "clearing")) != HK_OK) break;
    k_loss_estimate<<<(c.N + 127) / 128, 128, 0, c.stream>>>(c.mu.view(), c.A.view(), c.N, c.n, c.d_err + 1);
    count_launch(c);
    if ((st = check_cuda(c, cudaGetLastError(), "k_loss_estimate")) != HK_OK) break;
    c.stage = ST_LDLT;
    // Algorithm 4 ran inside the launch for the planned k: hk_inv_block(k)
    // goes straight to the block
    if (c.plan_k > 0 && c.N > 1) {
      c.alg4_k = c.plan_k;
      c.alg4_done = c.N - 1;
    }
  }
  return st;
}

hk_status hk_tune_batch(int device, int bits, int N, int count, int32_t* blocks_per_sm, int32_t* chunk,
                        double* seconds) {
  if (!valid_bits(bits) || N < 1 || N > 16384 || count < 1 || count > 256) return HK_ERR_ARG;
  const int M = bits / 1024;
  if (M > HK_BATCH_MAX_M) return HK_ERR_UNSUPPORTED;
  if (cudaSetDevice(device) != cudaSuccess) return HK_ERR_CUDA;
  const int most = ops_for(M)->batch_max_blocks();
  if (most < 1) return HK_ERR_CUDA;
  // the instances: beta = 1/m, m = 1, 2, 3, 4 in turn, all of size N
  std::vector<hk_ctx*> hs(count, nullptr);
  std::vector<cudaStream_t> ss(count, nullptr);
  hk_status st = HK_OK;
  for (int q = 0; q < count && st == HK_OK; ++q) {
    if (cudaStreamCreateWithFlags(&ss[q], cudaStreamNonBlocking) != cudaSuccess) {
      st = HK_ERR_CUDA;
      break;
    }
    st = hk_create(device, ss[q], &hs[q]);
    if (st == HK_OK) st = hk_moments(hs[q], 1, 1 + q % 4, N, bits);
  }
  BatchShape best{0, 0};
  double best_s = 0;
  for (int b : {1, 2, 3, 4, 6, 8, 12, 16}) {
    if (st != HK_OK || b > most) break;
    for (int g : {1, 4, 8, 16}) {
      const BatchShape sh{b, g};
      double t = 0;
      for (int rep = 0; rep < 2 && st == HK_OK; ++rep) {  // the faster of two runs
        if (cudaDeviceSynchronize() != cudaSuccess) {
          st = HK_ERR_CUDA;
          break;
        }
        const auto t0 = std::chrono::steady_clock::now();
        st = ldlt_batch_shaped(hs.data(), count, -1.0, &sh);
        if (st == HK_OK && cudaStreamSynchronize(ss[0]) != cudaSuccess) st = HK_ERR_CUDA;
        const double dt = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        t = rep == 0 ? dt : std::min(t, dt);
      }
      if (st == HK_OK) {
        int flags = 0;  // a run that did not finish (timeout, pivot <= 0) does not count
        for (hk_ctx* h : hs)
          if (st == HK_OK && (st = read_device_flags(h->c)) != HK_OK) flags = 1;
        if (flags) break;
      }
      if (st == HK_OK && (best.blocks == 0 || t < best_s)) {
        best = sh;
        best_s = t;
      }
    }
  }
  for (int q = 0; q < count; ++q) {
    if (hs[q]) hk_destroy(hs[q]);
    if (ss[q]) cudaStreamDestroy(ss[q]);
  }
  if (st != HK_OK) return st;
  if (best.blocks < 1) return HK_ERR_CUDA;  // no shape could be timed
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune[{M, n_bucket(N)}] = best;
  }
  if (blocks_per_sm) *blocks_per_sm = best.blocks;
  if (chunk) *chunk = best.chunk;
  if (seconds) *seconds = best_s;
  return HK_OK;
}

hk_status hk_alu_peak(int device, int kind, double* per_clk_per_sm) {
  if (kind < 0 || kind > 1 || !per_clk_per_sm) return HK_ERR_ARG;
  if (cudaSetDevice(device) != cudaSuccess) return HK_ERR_CUDA;
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || sms < 1)
    return HK_ERR_CUDA;
  auto kern = kind == 0 ? k_alu_peak<0> : k_alu_peak<1>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kPeakSmem) != cudaSuccess)
    return HK_ERR_CUDA;
  long long* span = nullptr;
  uint32_t* sink = nullptr;
  if (cudaMalloc(&span, sizeof(long long) * sms) != cudaSuccess) return HK_ERR_NOMEM;
  if (cudaMalloc(&sink, 64) != cudaSuccess) {
    cudaFree(span);
    return HK_ERR_NOMEM;
  }
  std::vector<long long> h(sms);
  cudaError_t e = cudaSuccess;
  for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {  // the first launch warms up
    kern<<<sms, kPeakThreads, kPeakSmem>>>(kPeakIters, 0x2545F491u + rep, span, sink);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
  }
  if (e == cudaSuccess) e = cudaMemcpy(h.data(), span, sizeof(long long) * sms, cudaMemcpyDeviceToHost);
  cudaFree(span);
  cudaFree(sink);
  if (e != cudaSuccess) return HK_ERR_CUDA;
  std::sort(h.begin(), h.end());
  const double med = (double)h[sms / 2];
  if (med <= 0) return HK_ERR_CUDA;
  *per_clk_per_sm = (double)kPeakThreads * kPeakChains * (double)kPeakIters / med;
  return HK_OK;
}

hk_status hk_precision_loss(hk_ctx* h, int32_t* loss_bits, int32_t* min_bits) {
  hk_status st = enter(h);
  if (st != HK_OK) return st;
  Ctx& c = h->c;
  if (c.stage < ST_LDLT) return set_error(c, HK_ERR_ORDER, "hk_precision_loss before hk_ldlt");
  int loss = 0;
  if ((st = read_loss(c, loss)) != HK_OK) return st;
  if (loss_bits) *loss_bits = loss;
  if (min_bits) *min_bits = min_bits_for(loss);
  return HK_OK;
}

hk_status hk_plan_block(hk_ctx* h, int k) {
  hk_status st = enter(h);
  if (st != HK_OK) return st;
  Ctx& c = h->c;
  if (k < 0 || k > 64) return set_error(c, HK_ERR_ARG, "the planned k must be in 0..64");
  c.plan_k = k;
  return HK_OK;
}

hk_status hk_inv_block(hk_ctx* h, int k) {
  hk_status st = enter(h);
  if (st != HK_OK) return st;
  Ctx& c = h->c;
  if (c.stage < ST_LDLT) return set_error(c, HK_ERR_ORDER, "hk_inv_block before hk_ldlt");
  if (k < 1 || k > c.N || k > 64) return set_error(c, HK_ERR_ARG, "k must be in 1..min(N, 64)");
  c.k = k;
  const size_t pe0 = c.prof ? prof_mark(c) : 0;
  st = ops_for(c.M)->inv_block(c);
  if (c.prof) c.stage_ev.push_back({2, {pe0, prof_mark(c)}});
  if (st == HK_OK) c.stage = ST_INVBLOCK;
  return st;
}

hk_status hk_lambda1(hk_ctx* h, int n_eig, int32_t* sign, int32_t* exp, uint32_t* limbs, double* lambda_f64,
                     double* trunc_err_f64) {
  hk_status st = enter(h);
  if (st != HK_OK) return st;
  Ctx& c = h->c;
  if (c.stage < ST_INVBLOCK) return set_error(c, HK_ERR_ORDER, "hk_lambda1 before hk_inv_block");
  if (n_eig < 1 || n_eig > 3 || n_eig > c.k) return set_error(c, HK_ERR_ARG, "n_eig must be in 1..min(3, k)");
  const size_t pe0 = c.prof ? prof_mark(c) : 0;
  if ((st = ops_for(c.M)->lambda(c, n_eig)) != HK_OK) return st;
  if (c.prof) c.stage_ev.push_back({3, {pe0, prof_mark(c)}});
  if ((st = read_device_flags(c)) != HK_OK) return st;
  int loss = 0;
  if ((st = read_loss(c, loss)) != HK_OK) return st;
  if (32 * c.n < min_bits_for(loss)) {
    char msg[192];
    std::snprintf(msg, sizeof(msg),
                  "estimated loss of %d bits leaves fewer than 133 + 64 of the %d: use at least %d bits", loss,
                  32 * c.n, min_bits_for(loss));
    return set_error(c, HK_ERR_PRECISION, msg);
  }
  for (int m = 0; m < n_eig; ++m) {
    if (sign) sign[m] = c.lam_sgn[m];
    if (exp) exp[m] = c.lam_exp[m];
    if (limbs) std::memcpy(limbs + (size_t)m * c.n, c.lam_mant.data() + (size_t)m * c.n, (size_t)c.n * 4);
    if (lambda_f64) lambda_f64[m] = c.lam_f64[m];
    if (trunc_err_f64) trunc_err_f64[m] = c.trunc_f64[m];
  }
  c.stage = ST_LAMBDA;
  return HK_OK;
}

hk_status hk_lambda1_grad(hk_ctx* h, int32_t* sign, int32_t* exp, uint32_t* limbs, double* f64) {
  hk_status st = enter(h);
  if (st != HK_OK) return st;
  Ctx& c = h->c;
  if (c.stage < ST_LAMBDA) return set_error(c, HK_ERR_ORDER, "hk_lambda1_grad before hk_lambda1");
  if (c.beta_den <= 0 || c.beta_num <= 0) return set_error(c, HK_ERR_UNSUPPORTED, "the gradient needs beta");
  {
    int64_t x = c.beta_num, y = c.beta_den;
    while (y) {
      const int64_t t = x % y;
      x = y;
      y = t;
    }
    const int64_t a = c.beta_num / x;
    if (a > 1 && c.psi_count != a - 1)
      return set_error(c, HK_ERR_UNSUPPORTED, "beta = a/b needs psi(r/a), r = 1..a-1 (hk_set_psi_constants)");
  }
  const size_t pe0 = c.prof ? prof_mark(c) : 0;
  if ((st = ops_for(c.M)->grad(c, sign, exp, limbs, f64)) != HK_OK) return st;
  if (c.prof) c.stage_ev.push_back({4, {pe0, prof_mark(c)}});
  return read_device_flags(c);
}

hk_status hk_export(hk_ctx* h, int what, int64_t first, int64_t count, int32_t* sign, int32_t* exp,
                    uint32_t* limbs) {
  hk_status st = enter(h);
  if (st != HK_OK) return st;
  Ctx& c = h->c;
  const DevVec* v = nullptr;
  int64_t base = 0, total = 0;
  switch (what) {
    case HK_MU: if (c.stage >= ST_MOMENTS) { v = &c.mu; total = 2 * (int64_t)c.N - 1; } break;
    case HK_FACTOR: if (c.stage >= ST_LDLT) { v = &c.A; total = (int64_t)c.N * (c.N + 1) / 2; } break;
    case HK_D:
      if (c.stage >= ST_LDLT) { v = &c.A; total = c.N; }
      break;
    case HK_X: if (c.stage >= ST_INVBLOCK) { v = &c.X; total = (int64_t)c.N * c.k; } break;
    case HK_S: if (c.stage >= ST_INVBLOCK) { v = &c.S; total = (int64_t)c.k * c.k; } break;
    case HK_EVEC: if (c.stage >= ST_LAMBDA) { v = &c.evec; total = c.k; } break;
    default: return set_error(c, HK_ERR_ARG, "unknown export");
  }
  if (!v) return set_error(c, HK_ERR_ORDER, "export of a stage not yet computed");
  if (first < 0 || count < 0 || first + count > total) return set_error(c, HK_ERR_ARG, "export range");
  if ((st = read_device_flags(c)) != HK_OK) return st;
  auto copy = [&](int64_t dst, int64_t src, int64_t cnt) -> hk_status {
    hk_status s2 = HK_OK;
    if (sign && (s2 = check_cuda(c, cudaMemcpy(sign + dst, v->sgn + src, cnt * 4, cudaMemcpyDeviceToHost), "D2H")))
      return s2;
    if (exp && (s2 = check_cuda(c, cudaMemcpy(exp + dst, v->exp + src, cnt * 4, cudaMemcpyDeviceToHost), "D2H")))
      return s2;
    if (limbs && (s2 = check_cuda(c, cudaMemcpy(limbs + dst * c.n, v->mant + src * c.n, cnt * c.n * 4,
                                                cudaMemcpyDeviceToHost), "D2H")))
      return s2;
    return HK_OK;
  };
  if (what == HK_D) {  // the pivots sit on the diagonal of the packed factor
    for (int64_t i = 0; i < count; ++i)
      if ((st = copy(i, tri_pos(c.N, first + i, first + i), 1)) != HK_OK) return st;
    return HK_OK;
  }
  return count ? copy(0, base + first, count) : HK_OK;
}

hk_status hk_set_product_algorithm(int algorithm) {
  if (algorithm < HK_PRODUCT_AUTO || algorithm > HK_PRODUCT_TENSOR) return HK_ERR_ARG;
  g_product_alg.store(algorithm);
  return HK_OK;
}

hk_status hk_set_profiling(hk_ctx* h, int on) {
  hk_status st = enter(h);
  if (st != HK_OK) return st;
  Ctx& c = h->c;
  if ((st = check_cuda(c, cudaStreamSynchronize(c.stream), "synchronising")) != HK_OK) return st;
  c.prof = on != 0;
  c.ev_used = 0;
  c.trail_ev.clear();
  c.scale_ev.clear();
  c.stage_ev.clear();
  c.trail_macs = 0.0;
  c.tc_ev.clear();
  c.tc_mmas = 0.0;
  if (c.tc_redo && (st = check_cuda(c, cudaMemset(c.tc_redo + 1, 0, sizeof(int)), "clearing")) != HK_OK) return st;
  c.launches = 0;
  return HK_OK;
}

hk_status hk_get_profile(hk_ctx* h, double* out, int cap) {
  hk_status st = enter(h);
  if (st != HK_OK) return st;
  Ctx& c = h->c;
  if (!out || cap < HK_PROFILE_FIELDS) return set_error(c, HK_ERR_ARG, "profile buffer too small");
  if ((st = check_cuda(c, cudaStreamSynchronize(c.stream), "synchronising")) != HK_OK) return st;
  for (int i = 0; i < HK_PROFILE_FIELDS; ++i) out[i] = 0.0;
  out[0] = (double)c.launches;
  double tms = 0.0;
  for (auto& p : c.trail_ev) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, c.events[p.first], c.events[p.second]);
    tms += ms;
  }
  out[1] = tms;
  out[2] = (double)c.trail_ev.size();
  out[3] = c.trail_macs;
  for (auto& p : c.stage_ev) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, c.events[p.second.first], c.events[p.second.second]);
    out[4 + p.first] += ms;
  }
  for (auto& p : c.scale_ev) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, c.events[p.first], c.events[p.second]);
    out[9] += ms;
  }
  for (auto& p : c.tc_ev) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, c.events[p.first], c.events[p.second]);
    out[10] += ms;
  }
  int redo = 0;
  if (c.tc_redo && (st = check_cuda(c, cudaMemcpy(&redo, c.tc_redo + 1, sizeof(int), cudaMemcpyDeviceToHost),
                                    "reading the re-run count")) != HK_OK)
    return st;
  out[11] = (double)c.tc_ev.size();
  out[12] = c.tc_mmas + redo * c.tc_mmas_whole;
  out[13] = (double)redo;
  return HK_OK;
}

// hk_batch_run in three parts per instance: its stream, context and
// moments; its factorisation (alone, or in one launch with the instances of
// its width when that width is a batched one); its block and eigenvalues.
struct BatchJob {
  hk_ctx* h = nullptr;
  cudaStream_t s = nullptr;
  std::chrono::steady_clock::time_point t0;
};

static hk_status setup_instance(int device, hk_instance& in, BatchJob& j) {
  j.t0 = std::chrono::steady_clock::now();
  if (cudaSetDevice(device) != cudaSuccess || cudaStreamCreateWithFlags(&j.s, cudaStreamNonBlocking) != cudaSuccess)
    return HK_ERR_CUDA;
  hk_status st = hk_create(device, j.s, &j.h);
  if (st == HK_OK) {
    if (in.mu_sign && in.mu_exp && in.mu_limbs)
      st = hk_set_moments(j.h, in.N, in.bits, in.mu_sign, in.mu_exp, in.mu_limbs, in.beta_num, in.beta_den);
    else if (in.gamma_exp && in.gamma_limbs && in.gamma_nc > 0)
      st = hk_moments_gamma(j.h, in.beta_num, in.beta_den, in.N, in.bits, in.gamma_nc, in.gamma_exp, in.gamma_limbs);
    else
      st = hk_moments(j.h, in.beta_num, in.beta_den, in.N, in.bits);
  }
  if (st == HK_OK) st = hk_plan_block(j.h, in.k);
  return st;
}

static void finish_instance(int device, hk_instance& in, BatchJob& j, hk_status st) {
  cudaSetDevice(device);
  if (st == HK_OK) st = hk_inv_block(j.h, in.k);
  if (st == HK_OK)
    st = hk_lambda1(j.h, in.n_eig, in.lambda_sign, in.lambda_exp, in.lambda_limbs, in.lambda_f64, in.trunc_err_f64);
  in.message[0] = 0;
  if (st != HK_OK) {
    std::snprintf(in.message, sizeof(in.message), "%s", j.h ? hk_last_error(j.h) : "context creation failed");
    if (!in.message[0]) std::snprintf(in.message, sizeof(in.message), "status %d", (int)st);
  }
  if (j.h) hk_destroy(j.h);
  if (j.s) cudaStreamDestroy(j.s);
  in.status = st;
  in.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - j.t0).count();
}

hk_status hk_batch_run(int device, hk_instance* inst, int count, int max_concurrent) {
  if (!inst || count < 0) return HK_ERR_ARG;
  for (int i = 0; i < count; ++i) {
    hk_instance& in = inst[i];
    if (in.N < 1 || in.k < 1 || in.k > in.N || in.n_eig < 1 || in.n_eig > 3 || in.n_eig > in.k || !valid_bits(in.bits))
      return HK_ERR_ARG;
    in.status = HK_OK;
  }
  const int workers = (max_concurrent <= 0 || max_concurrent > count) ? count : max_concurrent;
  // fn(0 .. items-1) on up to `workers` host threads
  auto parallel = [&](int items, const std::function<void(int)>& fn) {
    std::atomic<int> next(0);
    std::vector<std::thread> pool;
    for (int w = 0; w < std::min(workers, items); ++w)
      pool.emplace_back([&]() {
        for (int q = next++; q < items; q = next++) fn(q);
      });
    for (auto& t : pool) t.join();
  };
  // waves of at most `workers` instances, so that no more contexts than that
  // hold device memory at once
  for (int w0 = 0; w0 < count; w0 += workers) {
    const int wn = std::min(workers, count - w0);
    std::vector<BatchJob> jobs(wn);
    std::vector<hk_status> st(wn, HK_OK);
    parallel(wn, [&](int q) { st[q] = setup_instance(device, inst[w0 + q], jobs[q]); });
    // factorisations: the instances of one batched width (two or more) in one
    // launch; every other instance on its own
    std::vector<std::vector<int>> tasks;
    std::map<int, std::vector<int>> by_bits;
    for (int q = 0; q < wn; ++q) {
      if (st[q] != HK_OK) continue;
      if (inst[w0 + q].bits / 1024 <= HK_BATCH_MAX_M)
        by_bits[inst[w0 + q].bits].push_back(q);
      else
        tasks.push_back({q});
    }
    for (auto& g : by_bits) {
      if (g.second.size() >= 2)
        tasks.push_back(g.second);
      else
        tasks.push_back({g.second[0]});
    }
    parallel((int)tasks.size(), [&](int t) {
      const std::vector<int>& v = tasks[t];
      cudaSetDevice(device);
      if (v.size() == 1) {
        st[v[0]] = hk_ldlt(jobs[v[0]].h);
        return;
      }
      std::vector<hk_ctx*> hs;
      for (int q : v) hs.push_back(jobs[q].h);
      const hk_status r = hk_ldlt_batch(hs.data(), (int)hs.size(), -1.0);
      for (int q : v) st[q] = r;
    });
    parallel(wn, [&](int q) { finish_instance(device, inst[w0 + q], jobs[q], st[q]); });
  }
  for (int i = 0; i < count; ++i)
    if (inst[i].status != HK_OK) return (hk_status)inst[i].status;
  return HK_OK;
}

static MPVec cvec(const int32_t* s, const int32_t* e, const uint32_t* m) {
  return MPVec{const_cast<int32_t*>(s), const_cast<int32_t*>(e), const_cast<uint32_t*>(m)};
}

hk_status hk_fused_batch(int bits, int64_t count, const int32_t* a_sign, const int32_t* a_exp,
                         const uint32_t* a_limbs, const int32_t* x_sign, const int32_t* x_exp,
                         const uint32_t* x_limbs, const int32_t* y_sign, const int32_t* y_exp,
                         const uint32_t* y_limbs, int32_t* out_sign, int32_t* out_exp, uint32_t* out_limbs,
                         void* cuda_stream) {
  if (!valid_bits(bits) || count < 0) return HK_ERR_ARG;
  if (count == 0) return HK_OK;
  if (!a_sign || !a_exp || !a_limbs || !x_sign || !x_exp || !x_limbs || !y_sign || !y_exp || !y_limbs ||
      !out_sign || !out_exp || !out_limbs)
    return HK_ERR_ARG;
  int flags = 0;
  const cudaError_t e = ops_for(bits / 1024)->fused_batch(
      cvec(a_sign, a_exp, a_limbs), cvec(x_sign, x_exp, x_limbs), cvec(y_sign, y_exp, y_limbs),
      MPVec{out_sign, out_exp, out_limbs}, count, static_cast<cudaStream_t>(cuda_stream), &flags);
  if (e != cudaSuccess) return HK_ERR_CUDA;
  return status_of_flags(flags, nullptr);
}

hk_status hk_div_batch(int bits, int64_t count, const int32_t* a_sign, const int32_t* a_exp,
                       const uint32_t* a_limbs, const int32_t* d_sign, const int32_t* d_exp,
                       const uint32_t* d_limbs, int32_t* out_sign, int32_t* out_exp, uint32_t* out_limbs,
                       void* cuda_stream) {
  if (!valid_bits(bits) || count < 0) return HK_ERR_ARG;
  if (count == 0) return HK_OK;
  if (!a_sign || !a_exp || !a_limbs || !d_sign || !d_exp || !d_limbs || !out_sign || !out_exp || !out_limbs)
    return HK_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  int* flag = nullptr;
  if (cudaMallocAsync(&flag, sizeof(int), s) != cudaSuccess) return HK_ERR_NOMEM;
  cudaMemsetAsync(flag, 0, sizeof(int), s);
  cudaError_t e = ops_for(bits / 1024)->div_batch(cvec(a_sign, a_exp, a_limbs), cvec(d_sign, d_exp, d_limbs),
                                                   MPVec{out_sign, out_exp, out_limbs}, count, flag, s);
  int host_flag = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&host_flag, flag, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFreeAsync(flag, s);
  if (e != cudaSuccess) return HK_ERR_CUDA;
  return host_flag ? HK_ERR_ARG : HK_OK;
}

}  // extern "C"
