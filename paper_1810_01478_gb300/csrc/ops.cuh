// Host launchers for one limb width M (n = 32 M limbs).  Compiled once per
// supported width by inst.cu with -DHK_M=<M>.
#pragma once
#include <algorithm>
#include <cstdio>

#include "ctx.h"
#include "k_ldlt.cuh"

namespace hk {

template <typename K>
static cudaError_t allow_smem(K kernel, size_t bytes) {
  // prefer the largest shared-memory carveout so that shared memory does not
  // cap the number of resident blocks below what registers allow
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  if (e != cudaSuccess || bytes <= 48 * 1024) return e;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

static int sm_count(int device) {
  int v = 0;
  cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, device);
  return v > 0 ? v : 1;
}

template <int M>
struct Ops {
  static constexpr int n = 32 * M;
  static constexpr int WARPS = 4;  // warps per block of the warp-per-number kernels
  static constexpr size_t fused_smem = (size_t)WARPS * WarpSmem<M>::words * 4;
  static constexpr size_t div_smem = (size_t)WARPS * (4 * n + 4) * 4;
  static constexpr size_t recip_smem = (size_t)(3 * n + 4) * 4;

  // resident blocks of a kernel on the whole device
  template <typename K>
  static int resident_blocks(K kernel, int threads, size_t smem, int device) {
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem);
    return std::max(1, per_sm) * sm_count(device);
  }

  static cudaError_t fused_batch(MPVec a, MPVec x, MPVec y, MPVec out, int64_t count, cudaStream_t s) {
    cudaError_t e = allow_smem(k_fused_batch<M>, fused_smem);
    if (e != cudaSuccess) return e;
    if (count <= 0) return cudaSuccess;
    int dev = 0;
    cudaGetDevice(&dev);
    const int64_t want = (count + WARPS - 1) / WARPS;
    const int grid = (int)std::min<int64_t>(want, resident_blocks(k_fused_batch<M>, 32 * WARPS, fused_smem, dev));
    k_fused_batch<M><<<grid, 32 * WARPS, fused_smem, s>>>(a, x, y, out, count);
    return cudaGetLastError();
  }

  static cudaError_t div_batch(MPVec a, MPVec d, MPVec out, int64_t count, int* err, cudaStream_t s) {
    cudaError_t e = allow_smem(k_div_batch<M>, div_smem);
    if (e != cudaSuccess) return e;
    if (count <= 0) return cudaSuccess;
    int dev = 0;
    cudaGetDevice(&dev);
    const int64_t want = (count + WARPS - 1) / WARPS;
    const int grid = (int)std::min<int64_t>(want, resident_blocks(k_div_batch<M>, 32 * WARPS, div_smem, dev));
    k_div_batch<M><<<grid, 32 * WARPS, div_smem, s>>>(a, d, out, count, err);
    return cudaGetLastError();
  }

  // a2-a4: assemble H_N and run Algorithm 1 (Sec. 4.3) step by step.
  static hk_status ldlt(Ctx& c) {
    const int N = c.N;
    const int64_t tri = (int64_t)N * (N + 1) / 2;
    hk_status st;
    if (c.A.count != tri || c.A.n != n) {
      dev_free(c.A);
      if ((st = check_cuda(c, dev_alloc(c.A, tri, n), "allocating the factor")) != HK_OK) return st;
    }
    if (c.U.count != N || c.U.n != n) {
      dev_free(c.U);
      if ((st = check_cuda(c, dev_alloc(c.U, N, n), "allocating the pivot column")) != HK_OK) return st;
    }
    if (!c.rec) {
      if ((st = check_cuda(c, cudaMalloc(&c.rec, (size_t)n * 4 + 64), "allocating the reciprocal")) != HK_OK)
        return st;
      c.rec_meta = reinterpret_cast<int*>(c.rec + n);
    }
    if ((st = check_cuda(c, allow_smem(k_trailing<M>, fused_smem), "smem attribute")) != HK_OK) return st;
    if ((st = check_cuda(c, allow_smem(k_scale<M>, div_smem), "smem attribute")) != HK_OK) return st;
    if ((st = check_cuda(c, allow_smem(k_recip_pivot<M>, recip_smem), "smem attribute")) != HK_OK) return st;
    const int trail_res = resident_blocks(k_trailing<M>, 32 * WARPS, fused_smem, c.device);
    const int scale_res = resident_blocks(k_scale<M>, 32 * WARPS, div_smem, c.device);
    cudaStream_t s = c.stream;
    if (!c.aux) {
      if ((st = check_cuda(c, cudaStreamCreateWithFlags(&c.aux, cudaStreamNonBlocking), "aux stream")) ||
          (st = check_cuda(c, cudaEventCreateWithFlags(&c.ev_diag, cudaEventDisableTiming), "event")) ||
          (st = check_cuda(c, cudaEventCreateWithFlags(&c.ev_recip, cudaEventDisableTiming), "event")))
        return st;
    }
    {
      const int64_t work = tri * (n / 4);
      const int grid = (int)std::min<int64_t>((work + 255) / 256, 8 * sm_count(c.device) * 8);
      k_assemble<M><<<grid, 256, 0, s>>>(c.mu.view(), c.A.view(), N);
      count_launch(c);
    }
    // reciprocal of d_0 on the auxiliary stream
    cudaEventRecord(c.ev_diag, s);
    cudaStreamWaitEvent(c.aux, c.ev_diag, 0);
    k_recip_pivot<M><<<1, 32, recip_smem, c.aux>>>(c.A.view(), N, 0, c.rec, c.rec_meta, c.d_err);
    cudaEventRecord(c.ev_recip, c.aux);
    count_launch(c);
    for (int i = 0; i < N - 1; ++i) {
      const int64_t rows = N - 1 - i;
      const int64_t T = rows * (rows + 1) / 2;
      cudaStreamWaitEvent(s, c.ev_recip, 0);  // R_i is ready
      const int gs = (int)std::min<int64_t>((rows + WARPS - 1) / WARPS, scale_res);
      k_scale<M><<<gs, 32 * WARPS, div_smem, s>>>(c.A.view(), c.U.view(), N, i, c.rec, c.rec_meta, c.d_err);
      // look-ahead: update d_{i+1} = A[i+1][i+1] first (entry t = 0 of the trailing triangle) ...
      const size_t e0 = c.prof ? prof_mark(c) : 0;
      k_trailing<M><<<1, 32 * WARPS, fused_smem, s>>>(c.A.view(), c.U.view(), N, i, 0, 1, c.d_err);
      if (c.prof) {
        c.trail_ev.push_back({e0, prof_mark(c)});
        c.trail_macs += (double)n * n;
      }
      // ... start its reciprocal on the auxiliary stream ...
      cudaEventRecord(c.ev_diag, s);
      cudaStreamWaitEvent(c.aux, c.ev_diag, 0);
      k_recip_pivot<M><<<1, 32, recip_smem, c.aux>>>(c.A.view(), N, i + 1, c.rec, c.rec_meta, c.d_err);
      cudaEventRecord(c.ev_recip, c.aux);
      // ... while the main stream updates the rest of the trailing triangle
      if (T > 1) {
        const int gt = (int)std::min<int64_t>((T - 1 + WARPS - 1) / WARPS, trail_res);
        const size_t e1 = c.prof ? prof_mark(c) : 0;
        k_trailing<M><<<gt, 32 * WARPS, fused_smem, s>>>(c.A.view(), c.U.view(), N, i, 1, T, c.d_err);
        if (c.prof) {
          c.trail_ev.push_back({e1, prof_mark(c)});
          c.trail_macs += (double)(T - 1) * n * n;  // n^2 limb products per fused operation
        }
      }
      count_launch(c, T > 1 ? 4 : 3);
    }
    cudaStreamWaitEvent(s, c.ev_recip, 0);  // the last pivot's check belongs to this call
    return check_cuda(c, cudaGetLastError(), "launching the factorisation");
  }

  // The same launch sequence as ldlt() on buffers the caller provides
  // (hk_ldlt_noalloc): mu (2N-1), A (packed factor), U (N), rec (n limbs),
  // rec_meta and err (device ints).  Launches only; allocates nothing.
  static cudaError_t ldlt_raw(MPVec mu, MPVec A, MPVec U, uint32_t* rec, int* rec_meta, int* err, int N,
                              cudaStream_t s, int device) {
    cudaError_t e;
    if ((e = allow_smem(k_trailing<M>, fused_smem)) != cudaSuccess) return e;
    if ((e = allow_smem(k_scale<M>, div_smem)) != cudaSuccess) return e;
    if ((e = allow_smem(k_recip_pivot<M>, recip_smem)) != cudaSuccess) return e;
    const int trail_res = resident_blocks(k_trailing<M>, 32 * WARPS, fused_smem, device);
    const int scale_res = resident_blocks(k_scale<M>, 32 * WARPS, div_smem, device);
    const int64_t tri = (int64_t)N * (N + 1) / 2;
    {
      const int64_t work = tri * (n / 4);
      const int grid = (int)std::min<int64_t>((work + 255) / 256, 8 * sm_count(device) * 8);
      k_assemble<M><<<grid, 256, 0, s>>>(mu, A, N);
    }
    for (int i = 0; i < N; ++i) {
      k_recip_pivot<M><<<1, 32, recip_smem, s>>>(A, N, i, rec, rec_meta, err);
      if (i == N - 1) break;
      const int64_t rows = N - 1 - i;
      const int gs = (int)std::min<int64_t>((rows + WARPS - 1) / WARPS, scale_res);
      k_scale<M><<<gs, 32 * WARPS, div_smem, s>>>(A, U, N, i, rec, rec_meta, err);
      const int64_t T = rows * (rows + 1) / 2;
      const int gt = (int)std::min<int64_t>((T + WARPS - 1) / WARPS, trail_res);
      k_trailing<M><<<gt, 32 * WARPS, fused_smem, s>>>(A, U, N, i, 0, T, err);
    }
    return cudaGetLastError();
  }

  static hk_status inv_block(Ctx& c);
  static hk_status lambda(Ctx& c, int n_eig);
  static hk_status grad(Ctx& c, int32_t* sgn, int32_t* exp, uint32_t* mant, double* f64);

  static OpsTable table() {
    return OpsTable{M,           &Ops::ldlt,        &Ops::inv_block, &Ops::lambda, &Ops::grad,
                    &Ops::fused_batch, &Ops::div_batch, &Ops::ldlt_raw};
  }
};

}  // namespace hk
