// Host launchers for one limb width M (n = 32 M limbs).  Compiled once per
// supported width by inst.cu with -DHK_M=<M>.
#pragma once
#include <algorithm>
#include <cstdio>

#include "ctx.h"
#include "k_batch.cuh"
#include "k_ldlt.cuh"
#include "k_tail.cuh"
#include "tc.cuh"

namespace hk {

// dynamic shared memory of `bytes` per block, and a carveout that leaves the
// rest of the SM's 228 KB to L1 once `blocks` blocks fit
template <typename K>
static cudaError_t allow_smem_blocks(K kernel, size_t bytes, int blocks) {
  const size_t total = 233472;  // 228 KB
  int pct = (int)((blocks * (bytes + 1024) * 100 + total - 1) / total);
  pct = pct < 1 ? 1 : (pct > 100 ? 100 : pct);
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, pct);
  if (e != cudaSuccess || bytes <= 48 * 1024) return e;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

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
  static constexpr int NTW = HK_NTT_TRAIL_WARPS;  // warps per block of k_trailing_ntt
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

  // ------------------------------------------------------------------ tensor cores
  static constexpr bool kTc = M >= HK_TC_MIN_M;
  static constexpr size_t tc_smem = TcSmem<M>::bytes;

  // items of step i (TcTrail::items on the host)
  static int tc_trail_items(int N, int i) {
    const int m = N - 1 - i;
    int s = 0;
    for (int kt = 0; m - 1 > 128 * kt; ++kt) s += m - 128 * kt;
    return s;
  }
  // tcgen05.mma instructions of one 128-row item forming the positions from
  // q up (the same walk as the MMA warp)
  static double tc_mmas_per_item(int q) {
    using S = TcShape<M>;
    double c = 0;
    for (int t = 0; t < S::tiles(q); ++t) {
      const int qt = q + 256 * t;
      const int lo = std::max(0, qt - S::D + 1) >> 6, hi = std::min(S::D - 1, qt + 255) >> 6;
      for (int kb = lo; kb <= hi; ++kb)
        for (int s4 = 0; s4 < 4; ++s4) {
          const int k0 = 64 * kb + 16 * s4;
          if (!(k0 > qt + 255 || k0 + 15 < qt - S::D + 1)) c += 1;
        }
    }
    return c;
  }
  static int tc_grid(int device) { return std::max(1, sm_count(device) - 1); }
  static size_t tc_p_words(int grid) { return (size_t)grid * 2 * TC_ROWS * TcShape<M>::PL; }
  // the undecided-row records of up to cap items: count, total, 2 spare,
  // listed[cap], list[cap], mask[4 cap] (ints; zero when allocated)
  static size_t tc_redo_ints(size_t cap) { return 4 + 6 * cap; }
  static TcCut tc_cut(int* redo, size_t cap) {
    return TcCut{TcShape<M>::QCUT, redo + 4 + cap, redo, redo + 4, reinterpret_cast<uint32_t*>(redo + 4 + 2 * cap),
                 nullptr};
  }

  // A short-product launch over the items, then the re-run of the items it
  // listed with whole products (a fixed grid whose blocks read the count on
  // the device and leave at once when there is nothing to re-run).
  template <class Items>
  static cudaError_t tc_launch(const Items& it, int n_items, int* redo, size_t redo_cap, const uint16_t* DB,
                               int pitch, const uint16_t* DU, uint32_t* P, int grid, int* err, cudaStream_t s) {
    if constexpr (kTc) {
      using R = TcRedo<Items>;
      cudaError_t e = cudaFuncSetAttribute(k_tc_fused<M, Items>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)tc_smem);
      if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_tc_fused<M, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc_smem);
      if (e != cudaSuccess) return e;
      if (n_items <= 0 || grid <= 0) return cudaSuccess;
      if ((size_t)n_items > redo_cap) return cudaErrorInvalidValue;
      const TcCut cut = tc_cut(redo, redo_cap);
      if ((e = cudaMemsetAsync(cut.count, 0, sizeof(int), s)) != cudaSuccess) return e;
      k_tc_fused<M, Items><<<std::min(grid, n_items), TC_THREADS, tc_smem, s>>>(it, cut, DB, pitch, DU, P, err);
      TcCut whole = cut;
      whole.q = 0;
      whole.total = redo + 1;
      k_tc_fused<M, R><<<grid, TC_THREADS, tc_smem, s>>>(R{it, cut.list, cut.count, cut.listed, cut.mask}, whole, DB,
                                                         pitch, DU, P, err);
      return cudaGetLastError();
    } else {
      return cudaErrorNotSupported;
    }
  }

  // digits of count numbers mant[(first + t) n] into rows row0 + t of DU (layout 0) or DB (layout 1)
  static void tc_digits(const uint32_t* mant, int64_t first, int count, int row0, uint16_t* out, int layout,
                        int pitch, int device, cudaStream_t s) {
    if constexpr (kTc) {
      if (count <= 0) return;
      const int g = (int)std::min<int64_t>((count + WARPS - 1) / WARPS, 4 * sm_count(device));
      k_tc_digits<M><<<g, 32 * WARPS, 0, s>>>(mant, first, count, row0, out, layout, pitch);
    }
  }

  static cudaError_t fused_batch(MPVec a, MPVec x, MPVec y, MPVec out, int64_t count, cudaStream_t s, int* flags) {
    if (flags) *flags = 0;
    if (count <= 0) return cudaSuccess;
    int dev = 0;
    cudaGetDevice(&dev);
    if (kTc && use_tc(M) && count < (1 << 30)) {
      // x[e] is the U column of item e, y[e] its single digit row; every launch
      // is checked for device flags (a stray limb or a wait that gave up)
      using S = TcShape<M>;
      const int cnt = (int)count, pitch = cnt + TC_ROWS, grid = tc_grid(dev);
      const size_t db = (size_t)S::ND * pitch, du = (size_t)S::ND * cnt, pw = tc_p_words(grid);
      const size_t ri = tc_redo_ints((size_t)cnt);
      uint8_t* buf = nullptr;
      cudaError_t e = cudaMallocAsync(&buf, (db + du) * 2 + pw * 4 + 16 + ri * 4, s);
      if (e != cudaSuccess) return e;
      uint16_t* DB = reinterpret_cast<uint16_t*>(buf);
      uint16_t* DU = DB + db;
      uint32_t* P = reinterpret_cast<uint32_t*>(DU + du);
      int* flag = reinterpret_cast<int*>(P + pw);
      int* redo = flag + 4;
      cudaMemsetAsync(DB, 0, db * 2, s);
      cudaMemsetAsync(flag, 0, 16 + ri * 4, s);
      tc_digits(x.mant, 0, cnt, 0, DU, 0, 0, dev, s);
      tc_digits(y.mant, 0, cnt, 0, DB, 1, pitch, dev, s);
      e = tc_launch(TcBatch<M>{a, x, y, out, cnt}, cnt, redo, (size_t)cnt, DB, pitch, DU, P, grid, flag, s);
      int host_flag = 0;
      if (e == cudaSuccess) e = cudaMemcpyAsync(&host_flag, flag, sizeof(int), cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      cudaFreeAsync(buf, s);
      if (flags) *flags = host_flag;
      return e;
    }
    if (use_ntt(M)) {
      const NttConst nc = ntt_const(n);
      const size_t per = (size_t)NTT_Q * nc.L;
      uint32_t* F = nullptr;
      cudaError_t e = cudaMallocAsync(&F, 2 * per * count * sizeof(uint32_t), s);
      if (e != cudaSuccess) return e;
      const size_t fsm = (size_t)WARPS * ntt_stride(nc.L) * 4, tsm = (size_t)WARPS * NTT_Q * ntt_stride(nc.L) * 4;
      if ((e = allow_smem(k_ntt_fwd<M>, fsm)) != cudaSuccess) return e;
      if ((e = allow_smem_blocks(k_fused_batch_ntt<M>, tsm, 2)) != cudaSuccess) return e;
      const int g = (int)std::min<int64_t>((count + WARPS - 1) / WARPS, 4 * sm_count(dev));
      k_ntt_fwd<M><<<g, 32 * WARPS, fsm, s>>>(x, 0, (int)count, F, nc, 0);
      k_ntt_fwd<M><<<g, 32 * WARPS, fsm, s>>>(y, 0, (int)count, F + per * count, nc, 1);
      k_fused_batch_ntt<M><<<g, 32 * WARPS, tsm, s>>>(a, x, y, F, F + per * count, out, count, nc);
      e = cudaGetLastError();
      cudaFreeAsync(F, s);
      return e;
    }
    cudaError_t e = allow_smem(k_fused_batch<M>, fused_smem);
    if (e != cudaSuccess) return e;
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

  // a2-a4: assemble H_N and run Algorithm 1 (Sec. 4.3) step by step.  At
  // NTT widths the factorisation runs on the high-priority stream c.ms,
  // forked from and joined back to the caller's stream, and marks every
  // finished column for Algorithm 4 (see Ctx).
  static hk_status ldlt(Ctx& c) {
    c.cols_marked = false;
    if (!use_ntt(M)) return ldlt_body(c);
    hk_status st;
    if (!c.ms) {
      int least = 0, greatest = 0;
      cudaDeviceGetStreamPriorityRange(&least, &greatest);
      if ((st = check_cuda(c, cudaStreamCreateWithPriority(&c.ms, cudaStreamNonBlocking, greatest), "stream")) ||
          (st = check_cuda(c, cudaStreamCreateWithPriority(&c.a4, cudaStreamNonBlocking, least), "stream")))
        return st;
      for (cudaEvent_t* e : {&c.ev_fork, &c.ev_join, &c.ev_ldlt_start, &c.ev_a4})
        if ((st = check_cuda(c, cudaEventCreateWithFlags(e, cudaEventDisableTiming), "event")) != HK_OK) return st;
    }
    while ((int)c.ev_col.size() < c.N) {
      cudaEvent_t e;
      if ((st = check_cuda(c, cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "event")) != HK_OK) return st;
      c.ev_col.push_back(e);
    }
    const size_t need2 = (size_t)NTT_Q * ntt_len(n) * ((size_t)c.N + 64);
    if (c.ntt_cap2 < need2) {
      if (c.ntt_buf2) {
        cudaStreamSynchronize(c.stream);
        cudaFree(c.ntt_buf2);
        c.ntt_buf2 = nullptr;
        c.ntt_cap2 = 0;
      }
      if ((st = check_cuda(c, cudaMalloc(&c.ntt_buf2, need2 * 4), "allocating the transforms")) != HK_OK) return st;
      c.ntt_cap2 = need2;
    }
    cudaStream_t user = c.stream;
    cudaEventRecord(c.ev_fork, user);
    cudaEventRecord(c.ev_ldlt_start, user);
    cudaStreamWaitEvent(c.ms, c.ev_fork, 0);
    c.stream = c.ms;
    st = ldlt_body(c);
    c.stream = user;
    cudaEventRecord(c.ev_join, c.ms);
    cudaStreamWaitEvent(user, c.ev_join, 0);
    if (st == HK_OK) c.cols_marked = true;
    return st;
  }

  static hk_status ldlt_body(Ctx& c) {
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
    // NTT products: transforms of U and B_i once per step, reused by every update
    const bool ntt = use_ntt(M);
    NttConst nc{};
    size_t per = 0, ntt_smem = 0, fwd_smem = 0, scale_smem = 0;
    int ntt_res = 0, fwd_res = 0, scale_ntt_res = 0;
    if (ntt) {
      nc = ntt_const(n);
      per = (size_t)NTT_Q * nc.L;
      const size_t need = 2 * per * (size_t)N + 2 * per;  // FU, FB, then F(R), F(D) of the current pivot
      if (c.ntt_cap < need) {
        if (c.ntt_buf) {
          cudaStreamSynchronize(c.stream);
          cudaFree(c.ntt_buf);
          c.ntt_buf = nullptr;
          c.ntt_cap = 0;
        }
        if ((st = check_cuda(c, cudaMalloc(&c.ntt_buf, need * 4), "allocating the transforms")) != HK_OK) return st;
        c.ntt_cap = need;
      }
      ntt_smem = (size_t)NTW * NTT_Q * ntt_stride(nc.L) * 4;
      scale_smem = (size_t)HK_SCALE_WARPS * NTT_Q * ntt_stride(nc.L) * 4;
      fwd_smem = (size_t)WARPS * ntt_stride(nc.L) * 4;
      if ((st = check_cuda(c, allow_smem(k_trailing_ntt<M>, ntt_smem), "smem attribute")) ||
          (st = check_cuda(c, allow_smem(k_ntt_fwd<M>, fwd_smem), "smem attribute")))
        return st;
      // as many blocks as registers allow, the rest of the SM's memory to L1
      int per_sm = 0;
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_trailing_ntt<M>, 32 * NTW, ntt_smem);
      if ((st = check_cuda(c, allow_smem_blocks(k_trailing_ntt<M>, ntt_smem, std::max(per_sm, 1)), "smem attribute")))
        return st;
      ntt_res = resident_blocks(k_trailing_ntt<M>, 32 * NTW, ntt_smem, c.device);
      fwd_res = resident_blocks(k_ntt_fwd<M>, 32 * WARPS, fwd_smem, c.device);
      if ((st = check_cuda(c, allow_smem(k_scale_ntt<M>, scale_smem), "smem attribute")) != HK_OK) return st;
      scale_ntt_res = resident_blocks(k_scale_ntt<M>, 32 * HK_SCALE_WARPS, scale_smem, c.device);
    }
    // tensor-core products: digit matrices and the blocks' product buffers
    const bool tc = ntt && kTc && use_tc(M);
    const int tc_g = tc_grid(c.device);
    const int tc_pitch = N + TC_ROWS;
    if (tc) {
      using S = TcShape<M>;
      auto grow = [&](auto*& p, size_t& cap, size_t need, size_t elem) -> hk_status {
        if (cap >= need) return HK_OK;
        if (p) {
          cudaStreamSynchronize(c.stream);
          cudaFree(p);
          p = nullptr;
          cap = 0;
        }
        hk_status r = check_cuda(c, cudaMalloc((void**)&p, need * elem), "allocating the tensor-core buffers");
        if (r == HK_OK) cap = need;
        return r;
      };
      int* const redo_before = c.tc_redo;
      // U rows: the trailing update's columns, then k rows of X for Algorithm 4
      const size_t max_items = (size_t)tc_trail_items(N, 0) + 64 * (size_t)((N + 127) / 128);
      if ((st = grow(c.tc_db, c.tc_db_cap, (size_t)S::ND * tc_pitch, 2)) ||
          (st = grow(c.tc_du, c.tc_du_cap, (size_t)S::ND * (N + 64), 2)) ||
          (st = grow(c.tc_p, c.tc_p_cap, tc_p_words(tc_g), 4)) ||
          (st = grow(c.tc_redo, c.tc_redo_ints, tc_redo_ints(max_items), 4)))
        return st;
      // rows past N stay zero: they fill the last 128-row tile of a column;
      // the undecided-row records start clear (the running total only when
      // the records are new)
      const size_t keep = c.tc_redo == redo_before ? 4 : 0;
      if ((st = check_cuda(c, cudaMemsetAsync(c.tc_db, 0, (size_t)S::ND * tc_pitch * 2, c.stream), "clearing")) ||
          (st = check_cuda(c, cudaMemsetAsync(c.tc_redo + keep, 0, (c.tc_redo_ints - keep) * 4, c.stream),
                           "clearing")))
        return st;
      c.tc_mmas_whole = tc_mmas_per_item(0);
    }
    // Algorithm 4 for the planned k inside the tensor-core steps: X starts as
    // the first k columns of the identity (hk_plan_block)
    const int pk = tc ? c.plan_k : 0;
    if (pk > 0) {
      if (c.X.count != (int64_t)N * pk || c.X.n != n) {
        dev_free(c.X);
        if ((st = check_cuda(c, dev_alloc(c.X, (int64_t)N * pk, n), "allocating X")) != HK_OK) return st;
      }
      const int64_t work = (int64_t)N * pk * n;
      k_x_init<M><<<(int)std::min<int64_t>((work + 255) / 256, 4096), 256, 0, c.stream>>>(c.X.view(), N, pk);
      count_launch(c);
    }
    int alg4_steps = 0;
    uint32_t* FU = c.ntt_buf;
    uint32_t* FB = c.ntt_buf ? c.ntt_buf + per * (size_t)N : nullptr;
    uint32_t* FRD = c.ntt_buf ? c.ntt_buf + 2 * per * (size_t)N : nullptr;
    // the reciprocal of pivot i and, for NTT quotients, the transforms of R and d_i
    const size_t rp_smem = recip_pivot_words<M>(ntt) * 4;
    if ((st = check_cuda(c, allow_smem(k_recip_pivot<M>, rp_smem), "smem attribute")) != HK_OK) return st;
    auto pivot = [&](int i) {
      k_recip_pivot<M><<<1, 32, rp_smem, c.aux>>>(c.A.view(), N, i, c.rec, c.rec_meta, c.d_err, nc, ntt ? 1 : 0);
      if (ntt) {
        k_ntt_pivot<M><<<1, 64, 2 * ntt_stride(nc.L) * 4, c.aux>>>(c.rec, c.A.view(), tri_pos(N, i, i), FRD, nc);
        count_launch(c);
      }
      cudaEventRecord(c.ev_recip, c.aux);
    };
    // The launch that runs beside the next pivot's reciprocal (t0 > 0) leaves
    // one block slot free: with every SM's registers taken by trailing blocks
    // the reciprocal's warp could not start until the update had finished.
    auto trailing = [&](int i, int64_t t0, int64_t t1) {
      const int64_t cnt = t1 - t0;
      if (ntt) {
        const int cap = (t0 > 0 && ntt_res > 1) ? ntt_res - 1 : ntt_res;
        const int g = (int)std::min<int64_t>((cnt + NTW - 1) / NTW, cap);
        k_trailing_ntt<M><<<g, 32 * NTW, ntt_smem, c.stream>>>(c.A.view(), c.U.view(), FU, FB, N, i, t0, t1, nc,
                                                                   c.d_err);
      } else {
        const int cap = (t0 > 0 && trail_res > 1) ? trail_res - 1 : trail_res;
        const int g = (int)std::min<int64_t>((cnt + WARPS - 1) / WARPS, cap);
        k_trailing<M><<<g, 32 * WARPS, fused_smem, c.stream>>>(c.A.view(), c.U.view(), N, i, t0, t1, c.d_err);
      }
    };
    cudaStream_t s = c.stream;
    if (!c.aux) {
      int least = 0, greatest = 0;
      cudaDeviceGetStreamPriorityRange(&least, &greatest);
      if ((st = check_cuda(c, cudaStreamCreateWithPriority(&c.aux, cudaStreamNonBlocking, greatest), "aux stream")) ||
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
    pivot(0);
    count_launch(c);
    for (int i = 0; i < N - 1; ++i) {
      const int64_t rows = N - 1 - i;
      const int64_t T = rows * (rows + 1) / 2;
      cudaStreamWaitEvent(s, c.ev_recip, 0);  // R_i is ready
      const int gs = (int)std::min<int64_t>((rows + WARPS - 1) / WARPS, scale_res);
      const size_t es = c.prof ? prof_mark(c) : 0;
      if (ntt) {
        // F(U[r]) = F(A[r][i]) before the scale; the quotients A R and Q~ D
        // through transforms; then F(B_i[r]) for the update
        const int g = (int)std::min<int64_t>((rows + WARPS - 1) / WARPS, fwd_res);
        k_ntt_fwd<M><<<g, 32 * WARPS, fwd_smem, s>>>(c.A.view(), tri_pos(N, i + 1, i), (int)rows, FU, nc, 0);
        const int gq = (int)std::min<int64_t>((rows + HK_SCALE_WARPS - 1) / HK_SCALE_WARPS, scale_ntt_res);
        k_scale_ntt<M><<<gq, 32 * HK_SCALE_WARPS, scale_smem, s>>>(c.A.view(), c.U.view(), N, i, FU, FRD, FB, c.rec_meta, nc,
                                                       c.d_err);
        // with tensor-core products only the look-ahead entry (i+1, i+1) needs F(B_i)
        const bool tc_step = tc && rows >= HK_TC_MIN_ROWS;
        const int fb_rows = tc_step ? 1 : (int)rows;
        k_ntt_fwd<M><<<std::min(g, fb_rows), 32 * WARPS, fwd_smem, s>>>(c.A.view(), tri_pos(N, i + 1, i), fb_rows,
                                                                         FB, nc, 1);
        count_launch(c, 2);
        if (tc_step) {
          tc_digits(c.U.mant, i + 1, (int)rows, i + 1, c.tc_du, 0, 0, c.device, s);
          tc_digits(c.A.mant, tri_pos(N, i + 1, i), (int)rows, i + 1, c.tc_db, 1, tc_pitch, c.device, s);
          count_launch(c, 2);
          if (pk > 0) {
            // Algorithm 4, step i: the copies X[j][i] = -L[j][i] (i < k), and
            // the digits of row i of X (final since step i - 1) as U rows N + c
            if (i < pk) {
              k_alg4_copy<M><<<(int)std::min<int64_t>((rows + 3) / 4, 4 * sm_count(c.device)), 128, 0, s>>>(
                  c.A.view(), c.X.view(), N, pk, i);
              count_launch(c);
            }
            const int cols = std::min(pk, i);
            if (cols > 0) {
              tc_digits(c.X.mant, (int64_t)i * pk, cols, N, c.tc_du, 0, 0, c.device, s);
              count_launch(c);
            }
            alg4_steps = i + 1;
          }
        }
        if (i < (int)c.ev_col.size()) cudaEventRecord(c.ev_col[i], s);  // column i of L is final
      } else {
        k_scale<M><<<gs, 32 * WARPS, div_smem, s>>>(c.A.view(), c.U.view(), N, i, c.rec, c.rec_meta, c.d_err);
      }
      if (c.prof) c.scale_ev.push_back({es, prof_mark(c)});
      // look-ahead: update d_{i+1} = A[i+1][i+1] first (entry t = 0 of the trailing triangle) ...
      const size_t e0 = c.prof ? prof_mark(c) : 0;
      trailing(i, 0, 1);
      if (c.prof) {
        c.trail_ev.push_back({e0, prof_mark(c)});
        c.trail_macs += (double)n * n;
      }
      // ... start its reciprocal on the auxiliary stream ...
      cudaEventRecord(c.ev_diag, s);
      cudaStreamWaitEvent(c.aux, c.ev_diag, 0);
      pivot(i + 1);
      // ... while the main stream updates the rest of the trailing triangle
      if (T > 1) {
        const size_t e1 = c.prof ? prof_mark(c) : 0;
        const bool tc_step = tc && rows >= HK_TC_MIN_ROWS;
        if (tc_step) {
          const size_t cap = (c.tc_redo_ints - 4) / 6;
          const TcTrail<M> tr{c.A.view(), c.U.view(), N, i};
          int items = tc_trail_items(N, i);
          cudaError_t e;
          if (pk > 0) {
            items += std::min(pk, i) * (int)((rows + 127) / 128);
            e = tc_launch(TcStep<M>{tr, c.X.view(), pk}, items, c.tc_redo, cap, c.tc_db, tc_pitch, c.tc_du, c.tc_p,
                          tc_g, c.d_err, s);
          } else {
            e = tc_launch(tr, items, c.tc_redo, cap, c.tc_db, tc_pitch, c.tc_du, c.tc_p, tc_g, c.d_err, s);
          }
          if ((st = check_cuda(c, e, "launching the tensor-core update")) != HK_OK) return st;
          count_launch(c);  // the re-run launch
          if (c.prof) {
            c.tc_mmas += items * tc_mmas_per_item(TcShape<M>::QCUT);
            c.tc_ev.push_back({e1, prof_mark(c)});
          }
        } else {
          trailing(i, 1, T);
        }
        if (c.prof) {
          c.trail_ev.push_back({e1, prof_mark(c)});
          c.trail_macs += (double)(T - 1) * n * n;  // n^2 limb products per fused operation
        }
      }
      count_launch(c, T > 1 ? 4 : 3);
    }
    cudaStreamWaitEvent(s, c.ev_recip, 0);  // the last pivot's check belongs to this call
    if (alg4_steps > 0) {
      c.alg4_k = pk;
      c.alg4_done = alg4_steps;
    }
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
      k_recip_pivot<M><<<1, 32, recip_smem, s>>>(A, N, i, rec, rec_meta, err, NttConst{}, 0);
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

  // Blocks per SM the batched launch can hold (0 above the batched widths).
  static int batch_max_blocks() {
    if constexpr (M > HK_BATCH_MAX_M) {
      return 0;
    } else {
      constexpr size_t bsmem = (size_t)HK_BATCH_WARPS * batch_warp_words<M>() * 4;
      if (allow_smem(k_ldlt_batch<M>, bsmem) != cudaSuccess) return 0;
      int per_sm = 0;
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_ldlt_batch<M>, 32 * HK_BATCH_WARPS, bsmem);
      return per_sm;
    }
  }

  // a9: Algorithm 1 for several contexts of this width in one persistent
  // launch (k_ldlt_batch).  Each context's moments are ready on its own
  // stream; the launch runs on the first context's stream after the others'
  // assemblies, and every context's stream waits for it.  limit_ns bounds
  // the launch's idle wait (ERR_TIMEOUT in the unfinished instances).
  static hk_status ldlt_batch(Ctx* const* cs, int count, long long limit_ns, int blocks_per_sm, int chunk) {
    if (count < 1) return HK_OK;
    Ctx& c0 = *cs[0];
    hk_status st;
    if constexpr (M > HK_BATCH_MAX_M) {
      return set_error(c0, HK_ERR_UNSUPPORTED, "the batched factorisation serves widths up to 8192 bits");
    } else {
      constexpr size_t bsmem = (size_t)HK_BATCH_WARPS * batch_warp_words<M>() * 4;
      if ((st = check_cuda(c0, allow_smem(k_ldlt_batch<M>, bsmem), "smem attribute")) != HK_OK) return st;
      std::vector<BatchInst> hb(count);
      size_t state_words = 0;
      for (int q = 0; q < count; ++q) state_words += 4 * (size_t)cs[q]->N;
      // device block: instances | control | per-instance phase, tickets, done counts
      const size_t inst_bytes = ((size_t)count * sizeof(BatchInst) + 15) / 16 * 16;
      const size_t bytes = inst_bytes + sizeof(BatchCtl) + state_words * 4;
      char* blk = nullptr;
      if ((st = check_cuda(c0, cudaMallocAsync((void**)&blk, bytes, c0.stream), "allocating the batch state")) != HK_OK)
        return st;
      int* state = reinterpret_cast<int*>(blk + inst_bytes + sizeof(BatchCtl));
      size_t off = 0;
      std::vector<cudaEvent_t> evs;
      auto event = [&](cudaStream_t on) -> cudaError_t {
        cudaEvent_t e;
        cudaError_t r = cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
        if (r == cudaSuccess) r = cudaEventRecord(e, on);
        if (r == cudaSuccess) evs.push_back(e);
        return r;
      };
      for (int q = 0; q < count && st == HK_OK; ++q) {
        Ctx& c = *cs[q];
        c.cols_marked = false;
        const int N = c.N;
        const int64_t tri = (int64_t)N * (N + 1) / 2;
        if (c.A.count != tri || c.A.n != n) {
          dev_free(c.A);
          if ((st = check_cuda(c, dev_alloc(c.A, tri, n), "allocating the factor")) != HK_OK) break;
        }
        if (c.U.count != N || c.U.n != n) {
          dev_free(c.U);
          if ((st = check_cuda(c, dev_alloc(c.U, N, n), "allocating the pivot column")) != HK_OK) break;
        }
        if (!c.rec) {
          if ((st = check_cuda(c, cudaMalloc(&c.rec, (size_t)n * 4 + 64), "allocating the reciprocal")) != HK_OK) break;
          c.rec_meta = reinterpret_cast<int*>(c.rec + n);
        }
        const int64_t work = tri * (n / 4);
        const int grid = (int)std::min<int64_t>((work + 255) / 256, 8 * sm_count(c.device) * 8);
        k_assemble<M><<<grid, 256, 0, c.stream>>>(c.mu.view(), c.A.view(), N);
        count_launch(c);
        // a planned block size (hk_plan_block): Algorithm 4 runs inside the
        // launch, X starts as the first k columns of the identity
        const int pk = c.plan_k;
        if (pk > 0) {
          if (c.X.count != (int64_t)N * pk || c.X.n != n) {
            dev_free(c.X);
            if ((st = check_cuda(c, dev_alloc(c.X, (int64_t)N * pk, n), "allocating X")) != HK_OK) break;
          }
          const int64_t xw = (int64_t)N * pk * n;
          k_x_init<M><<<(int)std::min<int64_t>((xw + 255) / 256, 4096), 256, 0, c.stream>>>(c.X.view(), N, pk);
          count_launch(c);
        }
        if (q > 0) {
          if ((st = check_cuda(c, event(c.stream), "event")) != HK_OK) break;
          cudaStreamWaitEvent(c0.stream, evs.back(), 0);
        }
        hb[q] = BatchInst{c.A.view(), c.U.view(), c.rec, c.rec_meta, c.d_err, state + off,
                          pk > 0 ? c.X.view() : MPVec{}, N, pk};
        off += 4 * (size_t)N;
      }
      cudaStream_t s = c0.stream;
      if (st == HK_OK) {
        // pageable source: the copy has read it when the call returns
        st = check_cuda(c0, cudaMemcpyAsync(blk, hb.data(), (size_t)count * sizeof(BatchInst), cudaMemcpyHostToDevice, s),
                        "copying the batch");
      }
      if (st == HK_OK)
        st = check_cuda(c0, cudaMemsetAsync(blk + inst_bytes, 0, sizeof(BatchCtl) + state_words * 4, s), "clearing");
      if (st == HK_OK) {
        // blocks_per_sm blocks on every SM (at most what fits)
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_ldlt_batch<M>, 32 * HK_BATCH_WARPS, bsmem);
        const int grid = std::max(1, std::min(per_sm, blocks_per_sm)) * sm_count(c0.device);
        k_ldlt_batch<M><<<grid, 32 * HK_BATCH_WARPS, bsmem, s>>>(reinterpret_cast<const BatchInst*>(blk), count,
                                                                 reinterpret_cast<BatchCtl*>(blk + inst_bytes), limit_ns,
                                                                 std::max(1, chunk));
        count_launch(c0);
        st = check_cuda(c0, cudaGetLastError(), "k_ldlt_batch");
      }
      if (st == HK_OK && (st = check_cuda(c0, event(s), "event")) == HK_OK)
        for (int q = 1; q < count; ++q) cudaStreamWaitEvent(cs[q]->stream, evs.back(), 0);
      cudaFreeAsync(blk, s);
      for (cudaEvent_t e : evs) cudaEventDestroy(e);  // released once their work is done
      return st;
    }
  }

  static hk_status inv_block(Ctx& c);
  static hk_status lambda(Ctx& c, int n_eig);
  static hk_status grad(Ctx& c, int32_t* sgn, int32_t* exp, uint32_t* mant, double* f64);

  static OpsTable table() {
    return OpsTable{M,           &Ops::ldlt,        &Ops::inv_block, &Ops::lambda, &Ops::grad,
                    &Ops::fused_batch, &Ops::div_batch, &Ops::ldlt_raw, &Ops::ldlt_batch,
                    &Ops::batch_max_blocks};
  }
};

}  // namespace hk
