// Host-side context of libhk (one factorisation problem on one device).
#pragma once
#include <cuda_runtime.h>
#include <cstdint>
#include <map>
#include <string>
#include <vector>

#include "../../include/hk.h"
#include "common.cuh"
#include "ntt.cuh"

namespace hk {

// A device array of `count` numbers of n limbs each (owned).
struct DevVec {
  int64_t count = 0;
  int n = 0;
  int32_t* sgn = nullptr;
  int32_t* exp = nullptr;
  uint32_t* mant = nullptr;
  MPVec view() const { return MPVec{sgn, exp, mant}; }
  MPVec at(int64_t i) const { return MPVec{sgn + i, exp + i, mant + i * n}; }
};

cudaError_t dev_alloc(DevVec& v, int64_t count, int n);
void dev_free(DevVec& v);

enum Stage { ST_NONE = 0, ST_MOMENTS = 1, ST_LDLT = 2, ST_INVBLOCK = 3, ST_LAMBDA = 4 };

struct Ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  std::string err;
  hk_status sticky = HK_OK;
  int stage = ST_NONE;
  int N = 0, bits = 0, n = 0, M = 0, k = 0;
  int64_t beta_num = 0, beta_den = 0;
  int* d_err = nullptr;       // device error flags (ErrBits)
  DevVec mu, A, U, X, S, evec, scratch;
  DevVec psi;                 // psi(r/a), r = 1..a-1, for the gradient at beta = a/b (hk_set_psi_constants)
  int psi_count = -1;
  uint32_t* rec = nullptr;    // pivot reciprocal scratch (n limbs)
  int* rec_meta = nullptr;
  // look-ahead: the next pivot's reciprocal runs on `aux` while the main
  // stream finishes the current trailing update (Alg. 2's look-ahead, Sec. 4.3.1)
  cudaStream_t aux = nullptr;
  cudaEvent_t ev_diag = nullptr, ev_recip = nullptr;
  // transforms of the current step's U and B columns (NTT products)
  uint32_t* ntt_buf = nullptr;
  size_t ntt_cap = 0;  // words
  // Algorithm 4 beside the factorisation (NTT widths): the LDL^T runs on the
  // high-priority stream `ms` (forked from and joined back to the caller's
  // stream), marks each finished column i with ev_col[i], and hk_inv_block
  // runs Algorithm 4's step i on the low-priority stream `a4` once column i
  // is marked, with its own transform buffer ntt_buf2.
  cudaStream_t ms = nullptr, a4 = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_ldlt_start = nullptr, ev_a4 = nullptr;
  std::vector<cudaEvent_t> ev_col;
  bool cols_marked = false;
  uint32_t* ntt_buf2 = nullptr;
  size_t ntt_cap2 = 0;  // words
  // tensor-core products of the trailing update (tc.cuh): digit matrix of the
  // step's B column (kgroup-major, N + 128 rows), digits of its U column, and
  // the product buffers of the persistent kernel's blocks
  uint16_t* tc_db = nullptr;
  uint16_t* tc_du = nullptr;
  uint32_t* tc_p = nullptr;
  size_t tc_db_cap = 0, tc_du_cap = 0, tc_p_cap = 0;  // elements
  // undecided rows of the short-product launches: count, running total of
  // re-run items, then per-item records (Ops::tc_redo_ints)
  int* tc_redo = nullptr;
  // hk_plan_block: the k whose Algorithm 4 steps the factorisation runs on
  // the tensor cores, and after hk_ldlt the steps it ran (X holds their result)
  int plan_k = 0;
  int alg4_k = 0, alg4_done = 0;
  size_t tc_redo_ints = 0;
  double tc_mmas = 0.0;  // tcgen05.mma instructions of the profiled trailing launches (first launches)
  double tc_mmas_whole = 0.0;  // ... of one item of a re-run launch (whole product)
  std::vector<std::pair<size_t, size_t>> tc_ev;  // events around every tensor-core trailing launch
  // named scratch arrays of the later stages (grown on demand, freed in hk_destroy)
  std::map<std::string, DevVec> pool;
  const uint32_t* one_mant = nullptr;  // pool "one" holds 1 while its mant is this (cleared on reallocation)
  int one_n = 0;
  void* d_tasks = nullptr;    // task descriptors of the current launch
  size_t tasks_cap = 0;
  // profiling (hk_set_profiling): CUDA events around every trailing-update
  // launch and every stage, and a count of kernel launches
  bool prof = false;
  int64_t launches = 0;
  std::vector<cudaEvent_t> events;
  size_t ev_used = 0;
  std::vector<std::pair<size_t, size_t>> trail_ev;
  std::vector<std::pair<size_t, size_t>> scale_ev;  // column scale + transforms of each step
  double trail_macs = 0.0;
  std::vector<std::pair<int, std::pair<size_t, size_t>>> stage_ev;  // (stage id, events)
  // eigen results (host copies, filled by the lambda stage)
  int n_eig = 0;
  std::vector<int32_t> lam_sgn, lam_exp;
  std::vector<uint32_t> lam_mant;
  std::vector<double> lam_f64, trunc_f64;
};

hk_status set_error(Ctx& c, hk_status s, const std::string& msg);
hk_status check_cuda(Ctx& c, cudaError_t e, const char* what);
hk_status read_device_flags(Ctx& c);  // synchronises
// The status (and a message) that a device flags word (ErrBits) maps to;
// every entry point that reads the flags reports them through this.
hk_status status_of_flags(int flags, const char** msg);

// Per-width operations, one instantiation per limb count M (= n/32).
struct OpsTable {
  int M;
  hk_status (*ldlt)(Ctx&);
  hk_status (*inv_block)(Ctx&);
  hk_status (*lambda)(Ctx&, int n_eig);
  hk_status (*grad)(Ctx&, int32_t* sgn, int32_t* exp, uint32_t* mant, double* f64);
  // flags: host, the device flags (ErrBits) of paths that read them back, else 0
  cudaError_t (*fused_batch)(MPVec a, MPVec x, MPVec y, MPVec out, int64_t count, cudaStream_t s, int* flags);
  cudaError_t (*div_batch)(MPVec a, MPVec d, MPVec out, int64_t count, int* err, cudaStream_t s);
  // Algorithm 1 on caller-provided buffers (no allocation): see hk_ldlt_noalloc
  cudaError_t (*ldlt_raw)(MPVec mu, MPVec A, MPVec U, uint32_t* rec, int* rec_meta, int* err, int N,
                          cudaStream_t s, int device);
  // Algorithm 1 for several contexts of this width in one launch: see hk_ldlt_batch
  hk_status (*ldlt_batch)(Ctx* const* cs, int count, long long limit_ns, int blocks_per_sm, int chunk);
  int (*batch_max_blocks)();
};

const OpsTable* ops_for(int M);

// next profiling event recorded on the context's stream (prof must be on)
size_t prof_mark(Ctx& c);
// count one kernel launch
inline void count_launch(Ctx& c, int64_t k = 1) { c.launches += k; }

// Product algorithm of the wide kernels (hk_set_product_algorithm).
int product_algorithm();
bool use_ntt(int M);
// Tensor-core products (tcgen05) for the trailing update at this width.
bool use_tc(int M);
// NTT constants for n limbs on the current device (tables built on first use).
NttConst ntt_const(int n);

// pool array `name` with at least `count` numbers of c.n limbs
DevVec* pool_get(Ctx& c, const std::string& name, int64_t count);
// device copy of a host byte range into the task buffer (stream ordered)
hk_status upload_tasks(Ctx& c, const void* host, size_t bytes);

}  // namespace hk
