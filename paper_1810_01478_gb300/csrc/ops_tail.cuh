// Launchers of the stages after the factorisation:
//   inv_block  Algorithm 4 (Sec. 4.4) and S = (H^{-1})[0:k,0:k] (Sec. 4.5)
//   lambda     largest eigenvalues of S, lambda = 1/nu (Secs. 4.2, 4.5)
//   grad       d lambda_1 / d beta (first-order perturbation of nu_1)
#pragma once
#include <cmath>
#include <cstring>

#include "euler_gamma.inc"
#include "k_tail.cuh"
#include "ops.cuh"

namespace hk {

// a dot product sum_q x[x0 + q sx] * y[y0 + q sy] (q < len), negated if neg
struct Dot {
  int64_t out, x0, y0;
  int32_t sx, sy, len;
  bool neg;
};

static double to_double(int32_t s, int32_t e, const uint32_t* m, int n) {
  if (m[n - 1] == 0) return 0.0;
  // the top limb may hold a single bit: three limbs give >= 65 significant bits
  const double v = ((double)m[n - 1] * 4294967296.0 + (double)m[n - 2]) * 4294967296.0 + (double)m[n - 3];
  const double r = std::ldexp(v, 32 * (e + n - 3));
  return s ? -r : r;
}


template <int M>
struct Tail {
  static constexpr int n = 32 * M;
  static constexpr int W = Ops<M>::WARPS;
  static constexpr int SEG = 8;  // chain length of one partial sum (latency of a dot product ~ SEG + its reduction)

  static hk_status chains(Ctx& c, const std::vector<ChainTask>& t, MPVec X, MPVec Y, MPVec INIT, MPVec OUT) {
    if (t.empty()) return HK_OK;
    hk_status st = upload_tasks(c, t.data(), t.size() * sizeof(ChainTask));
    if (st != HK_OK) return st;
    const size_t smem = Ops<M>::fused_smem;
    if ((st = check_cuda(c, allow_smem(k_chain<M>, smem), "smem attribute")) != HK_OK) return st;
    const int res = Ops<M>::resident_blocks(k_chain<M>, 32 * W, smem, c.device);
    const int grid = (int)std::min<int64_t>(((int64_t)t.size() + W - 1) / W, res);
    k_chain<M><<<grid, 32 * W, smem, c.stream>>>(static_cast<const ChainTask*>(c.d_tasks), (int)t.size(), X, Y,
                                                   INIT, OUT);
    count_launch(c);
    return check_cuda(c, cudaGetLastError(), "k_chain");
  }

  // chains with NTT products: transforms of X[0, nx) and Y[0, ny) first
  // (scratch from the stream-ordered pool), then k_chain_ntt.  Same results
  // as chains().
  static hk_status chains_ntt(Ctx& c, const std::vector<ChainTask>& t, MPVec X, int64_t nx, MPVec Y, int64_t ny,
                              MPVec INIT, MPVec OUT) {
    if (t.empty()) return HK_OK;
    hk_status st = upload_tasks(c, t.data(), t.size() * sizeof(ChainTask));
    if (st != HK_OK) return st;
    const NttConst nc = ntt_const(n);
    const size_t per = (size_t)NTT_Q * nc.L;
    constexpr int NTW = Ops<M>::NTW;
    const size_t fsm = (size_t)W * ntt_stride(nc.L) * 4, tsm = (size_t)NTW * NTT_Q * ntt_stride(nc.L) * 4;
    if ((st = check_cuda(c, allow_smem(k_ntt_fwd<M>, fsm), "smem attribute")) ||
        (st = check_cuda(c, allow_smem(k_chain_ntt<M>, tsm), "smem attribute")))
      return st;
    uint32_t* F = nullptr;
    if ((st = check_cuda(c, cudaMallocAsync(&F, (size_t)(nx + ny) * per * 4, c.stream), "chain transforms")) != HK_OK)
      return st;
    const int fres = Ops<M>::resident_blocks(k_ntt_fwd<M>, 32 * W, fsm, c.device);
    k_ntt_fwd<M><<<(int)std::min<int64_t>((nx + W - 1) / W, fres), 32 * W, fsm, c.stream>>>(X, 0, (int)nx, F, nc, 0);
    k_ntt_fwd<M><<<(int)std::min<int64_t>((ny + W - 1) / W, fres), 32 * W, fsm, c.stream>>>(Y, 0, (int)ny,
                                                                                         F + nx * per, nc, 1);
    const int res = Ops<M>::resident_blocks(k_chain_ntt<M>, 32 * NTW, tsm, c.device);
    const int grid = (int)std::min<int64_t>(((int64_t)t.size() + NTW - 1) / NTW, res);
    k_chain_ntt<M><<<grid, 32 * NTW, tsm, c.stream>>>(static_cast<const ChainTask*>(c.d_tasks), (int)t.size(), X, Y,
                                                        F, F + nx * per, INIT, OUT, nc);
    count_launch(c, 3);
    const cudaError_t e = cudaGetLastError();
    cudaFreeAsync(F, c.stream);
    return check_cuda(c, e, "k_chain_ntt");
  }

  static hk_status quots(Ctx& c, const std::vector<QuotTask>& t, MPVec A, MPVec D, const DevVec& R, MPVec OUT) {
    if (t.empty()) return HK_OK;
    hk_status st = upload_tasks(c, t.data(), t.size() * sizeof(QuotTask));
    if (st != HK_OK) return st;
    const size_t smem = Ops<M>::div_smem;
    if ((st = check_cuda(c, allow_smem(k_quot<M>, smem), "smem attribute")) != HK_OK) return st;
    const int res = Ops<M>::resident_blocks(k_quot<M>, 32 * W, smem, c.device);
    const int grid = (int)std::min<int64_t>(((int64_t)t.size() + W - 1) / W, res);
    k_quot<M><<<grid, 32 * W, smem, c.stream>>>(static_cast<const QuotTask*>(c.d_tasks), (int)t.size(), A, D,
                                                  R.mant, R.sgn, OUT, c.d_err);
    count_launch(c);
    return check_cuda(c, cudaGetLastError(), "k_quot");
  }

  // reciprocals of D[idx[i]] into slots [0, idx.size()) of R (mant = table, sgn = shifts)
  static hk_status recips(Ctx& c, MPVec D, const std::vector<int64_t>& idx, const DevVec& R) {
    if (idx.empty()) return HK_OK;
    hk_status st = upload_tasks(c, idx.data(), idx.size() * sizeof(int64_t));
    if (st != HK_OK) return st;
    const size_t smem = (size_t)W * (3 * n + 4) * 4;
    if ((st = check_cuda(c, allow_smem(k_recip_tab<M>, smem), "smem attribute")) != HK_OK) return st;
    const int res = Ops<M>::resident_blocks(k_recip_tab<M>, 32 * W, smem, c.device);
    const int grid = (int)std::min<int64_t>(((int64_t)idx.size() + W - 1) / W, res);
    k_recip_tab<M><<<grid, 32 * W, smem, c.stream>>>(D, static_cast<const int64_t*>(c.d_tasks), 0, (int)idx.size(),
                                                       R.mant, R.sgn, c.d_err);
    count_launch(c);
    return check_cuda(c, cudaGetLastError(), "k_recip_tab");
  }

  // out[i] = trunc(num[i] / den[i]) for small integers
  static hk_status small(Ctx& c, const std::vector<int64_t>& num, const std::vector<int64_t>& den, MPVec OUT) {
    if (num.empty()) return HK_OK;
    std::vector<int64_t> both(num);
    both.insert(both.end(), den.begin(), den.end());
    hk_status st = upload_tasks(c, both.data(), both.size() * sizeof(int64_t));
    if (st != HK_OK) return st;
    const int cnt = (int)num.size();
    const int64_t* d = static_cast<const int64_t*>(c.d_tasks);
    k_small_ratio<M><<<(cnt + 127) / 128, 128, 0, c.stream>>>(d, d + cnt, cnt, OUT);
    count_launch(c);
    return check_cuda(c, cudaGetLastError(), "k_small_ratio");
  }

  // the constant 1 (pool "one"), formed once per allocation
  static DevVec* one(Ctx& c) {
    DevVec* v = pool_get(c, "one", 1);
    if (!v) return nullptr;
    if (c.one_mant == v->mant && c.one_n == n) return v;
    if (small(c, {1}, {1}, v->view()) != HK_OK) return nullptr;
    c.one_mant = v->mant;
    c.one_n = n;
    return v;
  }

  // dot products, split into chains of SEG terms whose partial sums are added
  // by a second level of chains (recursively).
  // nx, ny > 0: X and Y hold nx and ny numbers and the products go through
  // transforms of them (NTT widths; worth it when every number is used often).
  static hk_status dots(Ctx& c, const std::vector<Dot>& d, MPVec X, MPVec Y, MPVec OUT, int level = 0,
                        int64_t nx = 0, int64_t ny = 0) {
    if (d.empty()) return HK_OK;
    const bool ntt = nx > 0 && ny > 0 && use_ntt(M);
    int maxlen = 0;
    for (const Dot& e : d) maxlen = std::max(maxlen, e.len);
    if (maxlen <= SEG) {
      std::vector<ChainTask> t;
      t.reserve(d.size());
      for (const Dot& e : d)
        t.push_back(ChainTask{e.out, 0, e.x0, e.y0, e.sx, e.sy, e.len,
                              CH_ZERO_INIT | CH_ADD | (e.neg ? CH_NEG_OUT : 0)});
      return ntt ? chains_ntt(c, t, X, nx, Y, ny, X, OUT) : chains(c, t, X, Y, X, OUT);
    }
    int64_t total = 0;
    for (const Dot& e : d) total += (e.len + SEG - 1) / SEG;
    DevVec* P = pool_get(c, "partial" + std::to_string(level), total);
    DevVec* ONE = one(c);
    if (!P || !ONE) return c.sticky;
    std::vector<ChainTask> t;
    std::vector<Dot> up;
    t.reserve(total);
    int64_t base = 0;
    for (const Dot& e : d) {
      const int segs = (e.len + SEG - 1) / SEG;
      for (int g = 0; g < segs; ++g) {
        const int q0 = g * SEG, len = std::min(SEG, e.len - q0);
        t.push_back(ChainTask{base + g, 0, e.x0 + (int64_t)q0 * e.sx, e.y0 + (int64_t)q0 * e.sy, e.sx, e.sy, len,
                              CH_ZERO_INIT | CH_ADD});
      }
      up.push_back(Dot{e.out, base, 0, 1, 0, segs, e.neg});  // P[base + q] * 1
      base += segs;
    }
    hk_status st = ntt ? chains_ntt(c, t, X, nx, Y, ny, X, P->view()) : chains(c, t, X, Y, X, P->view());
    if (st != HK_OK) return st;
    // the constant 1 as the y operand: the schoolbook product skips its zero blocks
    return dots(c, up, P->view(), ONE->view(), OUT, level + 1);
  }

  // ------------------------------------------------------------------------
  // a5, a6
  // ------------------------------------------------------------------------
  static hk_status inv_block(Ctx& c) {
    const int N = c.N, k = c.k;
    hk_status st;
    if (c.X.count != (int64_t)N * k || c.X.n != n) {
      dev_free(c.X);
      if ((st = check_cuda(c, dev_alloc(c.X, (int64_t)N * k, n), "allocating X")) != HK_OK) return st;
    }
    if (c.S.count != (int64_t)k * k || c.S.n != n) {
      dev_free(c.S);
      if ((st = check_cuda(c, dev_alloc(c.S, (int64_t)k * k, n), "allocating S")) != HK_OK) return st;
    }
    const bool ntt = use_ntt(M) && c.ntt_buf && c.ntt_cap >= 2 * (size_t)NTT_Q * ntt_len(n) * N;
    // steps 0 .. alg4_done - 1 already ran inside the factorisation's
    // tensor-core launches for this k (hk_plan_block): X holds their result
    const int i0 = (c.alg4_done > 0 && c.alg4_k == k && c.X.count == (int64_t)N * k && c.X.n == n) ? c.alg4_done : 0;
    // Algorithm 4 beside the factorisation: on the low-priority stream a4,
    // step i after column i of L is marked (the LDL^T queued just before)
    const bool beside = ntt && c.cols_marked && c.a4 && c.ntt_buf2 &&
                        c.ntt_cap2 >= (size_t)NTT_Q * ntt_len(n) * ((size_t)N + k) && (int)c.ev_col.size() >= N;
    c.cols_marked = false;
    cudaStream_t xs = beside ? c.a4 : c.stream;
    if (beside) cudaStreamWaitEvent(xs, c.ev_ldlt_start, 0);
    if (i0 == 0) {
      const int64_t work = (int64_t)N * k * n;
      const int grid = (int)std::min<int64_t>((work + 255) / 256, 4096);
      k_x_init<M><<<grid, 256, 0, xs>>>(c.X.view(), N, k);
      count_launch(c);
    }
    if (ntt) {
      // Algorithm 4 with NTT products: per step, the transforms of the pivot
      // column L[i+1..N)[i] (unscaled) and of the finished row X[i][0..cols) (scaled)
      const NttConst nc = ntt_const(n);
      const size_t per = (size_t)NTT_Q * nc.L;
      uint32_t* FL = beside ? c.ntt_buf2 : c.ntt_buf;
      uint32_t* FXr = FL + per * N;
      constexpr int NTW = Ops<M>::NTW;
      const size_t tsm = (size_t)NTW * NTT_Q * ntt_stride(nc.L) * 4, fsm = (size_t)W * ntt_stride(nc.L) * 4;
      if ((st = check_cuda(c, allow_smem(k_alg4_ntt<M>, tsm), "smem attribute")) ||
          (st = check_cuda(c, allow_smem(k_ntt_fwd<M>, fsm), "smem attribute")))
        return st;
      const int res = Ops<M>::resident_blocks(k_alg4_ntt<M>, 32 * NTW, tsm, c.device);
      const int fres = Ops<M>::resident_blocks(k_ntt_fwd<M>, 32 * W, fsm, c.device);
      for (int i = i0; i < N - 1; ++i) {
        const int cols = std::min(k, i);
        const int64_t per_row = cols + (i < k ? 1 : 0);
        const int64_t rows = N - 1 - i;
        const int64_t total = rows * per_row;
        if (beside) cudaStreamWaitEvent(xs, c.ev_col[i], 0);
        if (cols > 0) {
          const int g1 = (int)std::min<int64_t>((rows + W - 1) / W, fres);
          k_ntt_fwd<M><<<g1, 32 * W, fsm, xs>>>(c.A.view(), tri_pos(N, i + 1, i), (int)rows, FL, nc, 0);
          const int g2 = (int)std::min<int64_t>((cols + W - 1) / W, fres);
          k_ntt_fwd<M><<<g2, 32 * W, fsm, xs>>>(c.X.view(), (int64_t)i * k, cols, FXr, nc, 1);
          count_launch(c, 2);
        }
        // beside the factorisation: one update per warp, so that blocks are
        // short and free their SM quickly for the higher-priority stream
        const int grid = (int)std::min<int64_t>((total + NTW - 1) / NTW, beside ? (1 << 20) : res);
        k_alg4_ntt<M><<<grid, 32 * NTW, tsm, xs>>>(c.A.view(), c.X.view(), FL, FXr, N, k, i, nc);
        count_launch(c);
      }
      if (beside) {
        cudaEventRecord(c.ev_a4, xs);
        cudaStreamWaitEvent(c.stream, c.ev_a4, 0);
      }
    } else {
      const size_t smem = Ops<M>::fused_smem;
      if ((st = check_cuda(c, allow_smem(k_alg4_step<M>, smem), "smem attribute")) != HK_OK) return st;
      const int res = Ops<M>::resident_blocks(k_alg4_step<M>, 32 * W, smem, c.device);
      // Algorithm 4: N-1 steps in increasing pivot order
      for (int i = i0; i < N - 1; ++i) {
        const int64_t per_row = std::min(k, i) + (i < k ? 1 : 0);
        const int64_t total = (int64_t)(N - 1 - i) * per_row;
        if (total == 0) continue;
        const int grid = (int)std::min<int64_t>((total + W - 1) / W, res);
        k_alg4_step<M><<<grid, 32 * W, smem, c.stream>>>(c.A.view(), c.X.view(), N, k, i);
        count_launch(c);
      }
    }
    c.alg4_done = 0;  // X now holds every step: a later call starts again from the identity
    if ((st = check_cuda(c, cudaGetLastError(), "Algorithm 4")) != HK_OK) return st;
    // reciprocals of the pivots (kept for the gradient), then Y[l][b] = X[l][b] / D_l
    DevVec* Rd = pool_get(c, "recip_d", N);
    DevVec* Yq = pool_get(c, "xq", (int64_t)N * k);
    if (!Rd || !Yq) return c.sticky;
    std::vector<int64_t> diag(N);
    for (int l = 0; l < N; ++l) diag[l] = tri_pos(N, l, l);
    if ((st = recips(c, c.A.view(), diag, *Rd)) != HK_OK) return st;
    std::vector<QuotTask> qt;
    for (int l = 0; l < N; ++l)
      for (int b = 0; b <= std::min(l, k - 1); ++b)
        qt.push_back(QuotTask{(int64_t)l * k + b, (int64_t)l * k + b, diag[l], l, 0, 0});
    if ((st = quots(c, qt, c.X.view(), c.A.view(), *Rd, Yq->view())) != HK_OK) return st;
    // S_ab = sum_{l >= b} X[l][a] * Y[l][b]  (a <= b), then the mirror image
    std::vector<Dot> dd;
    for (int a = 0; a < k; ++a)
      for (int b = a; b < k; ++b)
        dd.push_back(Dot{(int64_t)a * k + b, (int64_t)b * k + a, (int64_t)b * k + b, k, k, N - b, false});
    if ((st = dots(c, dd, c.X.view(), Yq->view(), c.S.view(), 0, (int64_t)N * k, (int64_t)N * k)) != HK_OK)
      return st;
    std::vector<ChainTask> mirror;
    for (int a = 0; a < k; ++a)
      for (int b = a + 1; b < k; ++b)
        mirror.push_back(ChainTask{(int64_t)b * k + a, (int64_t)a * k + b, 0, 0, 0, 0, 0, 0});
    return chains(c, mirror, c.S.view(), c.S.view(), c.S.view(), c.S.view());
  }

  // ------------------------------------------------------------------------
  // a7: largest eigenvalue of the leading kk x kk block of the k x k matrix Sm
  // ------------------------------------------------------------------------
  // T = Sm^(2^s) by repeated squaring (T -> nu_1^(2^s) u u^T), v = the column
  // of T with the largest diagonal entry, nu = v^T Sm v / v^T v (Rayleigh
  // quotient, error ~ (nu_2/nu_1)^(2^(s+1))).  After s0 squarings it keeps
  // squaring until two successive quotients agree to `tol` limbs (at most 40
  // squarings).  Writes v (kk numbers) into V and nu, v^T v into scal[slot],
  // scal[slot + 1].
  static hk_status rayleigh(Ctx& c, MPVec Sm, MPVec T, int k, int kk, MPVec V, DevVec& scal, int slot) {
    DevVec* Wv = pool_get(c, "w", k);
    DevVec* Rs = pool_get(c, "recip_s", 4);
    DevVec* tmp = pool_get(c, "eig_tmp", 2);
    if (!Wv || !Rs || !tmp) return c.sticky;
    hk_status st;
    int* d_j = c.d_err + 4;
    k_argmax_diag<<<1, 32, 0, c.stream>>>(T, k, kk, n, d_j);
    count_launch(c);
    int j = 0;
    if ((st = check_cuda(c, cudaMemcpyAsync(&j, d_j, sizeof(int), cudaMemcpyDeviceToHost, c.stream), "argmax")) ||
        (st = check_cuda(c, cudaStreamSynchronize(c.stream), "argmax sync")))
      return st;
    std::vector<ChainTask> col;
    for (int a = 0; a < kk; ++a) col.push_back(ChainTask{a, (int64_t)a * k + j, 0, 0, 0, 0, 0, 0});
    if ((st = chains(c, col, T, T, T, V)) != HK_OK) return st;
    std::vector<Dot> sv;
    for (int a = 0; a < kk; ++a) sv.push_back(Dot{a, (int64_t)a * k, 0, 1, 1, kk, false});
    if ((st = dots(c, sv, Sm, V, Wv->view())) != HK_OK) return st;
    if ((st = dots(c, {Dot{0, 0, 0, 1, 1, kk, false}}, V, Wv->view(), tmp->view())) != HK_OK) return st;
    if ((st = dots(c, {Dot{1, 0, 0, 1, 1, kk, false}}, V, V, tmp->view())) != HK_OK) return st;
    if ((st = recips(c, tmp->view(), {1}, *Rs)) != HK_OK) return st;
    if ((st = quots(c, {QuotTask{slot, 0, 1, 0, 0, 0}}, tmp->view(), tmp->view(), *Rs, scal.view())) != HK_OK)
      return st;
    return chains(c, {ChainTask{slot + 1, 1, 0, 0, 0, 0, 0, 0}}, tmp->view(), tmp->view(), tmp->view(), scal.view());
  }

  static hk_status eig_top(Ctx& c, MPVec Sm, int k, int kk, int s0, int tol, MPVec V, DevVec& scal, int slot) {
    DevVec* T0 = pool_get(c, "T0", (int64_t)k * k);
    DevVec* T1 = pool_get(c, "T1", (int64_t)k * k);
    DevVec* ONE = one(c);
    if (!T0 || !T1 || !ONE) return c.sticky;
    hk_status st;
    std::vector<ChainTask> cp;
    for (int a = 0; a < kk; ++a)
      for (int b = 0; b < kk; ++b)
        cp.push_back(ChainTask{(int64_t)a * k + b, (int64_t)a * k + b, 0, 0, 0, 0, 0, 0});
    if ((st = chains(c, cp, Sm, Sm, Sm, T0->view())) != HK_OK) return st;
    std::vector<Dot> sq;
    for (int a = 0; a < kk; ++a)
      for (int b = 0; b < kk; ++b) sq.push_back(Dot{(int64_t)a * k + b, (int64_t)a * k, b, 1, k, kk, false});
    const int64_t kk2 = (int64_t)k * k;
    for (int it = 0; it < s0; ++it) {
      if ((st = dots(c, sq, T0->view(), T0->view(), T1->view(), 0, kk2, kk2)) != HK_OK) return st;
      std::swap(*T0, *T1);
    }
    if ((st = rayleigh(c, Sm, T0->view(), k, kk, V, scal, slot)) != HK_OK) return st;
    // keep squaring until the quotient is stable: nu' - nu small against nu
    const int pslot = slot + 8;  // scal[pslot], scal[pslot + 1]: the next quotient
    int* flag = c.d_err + 8;
    for (int it = s0; it < 40; ++it) {
      if ((st = dots(c, sq, T0->view(), T0->view(), T1->view(), 0, kk2, kk2)) != HK_OK) return st;
      std::swap(*T0, *T1);
      if ((st = rayleigh(c, Sm, T0->view(), k, kk, V, scal, pslot)) != HK_OK) return st;
      // scal[pslot + 2] = nu' - 1 * nu
      if ((st = chains(c, {ChainTask{pslot + 2, pslot, slot, 0, 0, 0, 1, 0}}, scal.view(), ONE->view(),
                       scal.view(), scal.view())) != HK_OK)
        return st;
      k_rel_small<<<1, 32, 0, c.stream>>>(scal.view(), pslot + 2, scal.view(), pslot, n, tol, flag);
      count_launch(c);
      int close = 0;
      if ((st = check_cuda(c, cudaMemcpyAsync(&close, flag, sizeof(int), cudaMemcpyDeviceToHost, c.stream), "flag")) ||
          (st = check_cuda(c, cudaStreamSynchronize(c.stream), "flag sync")))
        return st;
      // adopt the newer quotient either way
      if ((st = chains(c, {ChainTask{slot, pslot, 0, 0, 0, 0, 0, 0}, ChainTask{slot + 1, pslot + 1, 0, 0, 0, 0, 0, 0}},
                       scal.view(), scal.view(), scal.view(), scal.view())) != HK_OK)
        return st;
      if (close) return HK_OK;
    }
    return set_error(c, HK_ERR_PRECISION, "block eigenvalue did not converge in 40 squarings");
  }

  // Sm <- Sm - (nu / v^T v) v v^T on the leading kk block (removes nu from the spectrum)
  static hk_status deflate(Ctx& c, MPVec Sm, int k, int kk, MPVec V, DevVec& scal, int slot) {
    DevVec* Rs = pool_get(c, "recip_s", 4);
    DevVec* cv = pool_get(c, "cv", k);
    DevVec* cf = pool_get(c, "cf", 1);
    if (!Rs || !cv || !cf) return c.sticky;
    hk_status st;
    if ((st = recips(c, scal.view(), {(int64_t)slot + 1}, *Rs)) != HK_OK) return st;
    if ((st = quots(c, {QuotTask{0, slot, slot + 1, 0, 0, 0}}, scal.view(), scal.view(), *Rs, cf->view())) != HK_OK)
      return st;
    std::vector<Dot> cvd;
    for (int a = 0; a < kk; ++a) cvd.push_back(Dot{a, 0, a, 0, 0, 1, false});
    if ((st = dots(c, cvd, cf->view(), V, cv->view())) != HK_OK) return st;
    std::vector<ChainTask> t;
    for (int a = 0; a < kk; ++a)
      for (int b = 0; b < kk; ++b)
        t.push_back(ChainTask{(int64_t)a * k + b, (int64_t)a * k + b, a, b, 0, 0, 1, 0});
    return chains(c, t, cv->view(), V, Sm, Sm);
  }

  static int squarings_for(int bits_target) {
    // (nu_2/nu_1)^(2^(s+1)) < 2^-bits_target when nu_2/nu_1 <= 1/2; eig_top
    // squares further if the quotient has not settled
    int s = 1;
    while ((1 << (s + 1)) < bits_target) ++s;
    return s;
  }

  // Eigenvalues of a symmetric kk x kk matrix (row stride kk) by cyclic
  // Jacobi rotations, in double precision; descending.  Empty on failure.
  static std::vector<double> jacobi_eigenvalues(std::vector<double> a, int kk) {
    for (int sweep = 0; sweep < 60; ++sweep) {
      double off = 0, tot = 0;
      for (int i = 0; i < kk; ++i)
        for (int j = 0; j < kk; ++j) {
          tot += a[i * kk + j] * a[i * kk + j];
          if (i != j) off += a[i * kk + j] * a[i * kk + j];
        }
      if (!std::isfinite(tot)) return {};
      if (off <= 1e-60 * tot) break;
      for (int p = 0; p < kk; ++p)
        for (int q = p + 1; q < kk; ++q) {
          const double apq = a[p * kk + q];
          if (apq == 0.0) continue;
          const double th = (a[q * kk + q] - a[p * kk + p]) / (2 * apq);
          const double t = (th >= 0 ? 1.0 : -1.0) / (std::fabs(th) + std::sqrt(th * th + 1));
          const double cs = 1 / std::sqrt(t * t + 1), sn = t * cs;
          for (int r = 0; r < kk; ++r) {  // columns p, q
            const double x = a[r * kk + p], y = a[r * kk + q];
            a[r * kk + p] = cs * x - sn * y;
            a[r * kk + q] = sn * x + cs * y;
          }
          for (int r = 0; r < kk; ++r) {  // rows p, q
            const double x = a[p * kk + r], y = a[q * kk + r];
            a[p * kk + r] = cs * x - sn * y;
            a[q * kk + r] = sn * x + cs * y;
          }
        }
    }
    std::vector<double> ev(kk);
    for (int i = 0; i < kk; ++i) ev[i] = a[i * kk + i];
    std::sort(ev.begin(), ev.end(), [](double x, double y) { return x > y; });
    return ev;
  }

  // Squarings before eig_top first tests convergence, per eigenvalue m < ne
  // of the leading kk block: after s squarings the quotient's error is about
  // (nu_{m+1}/nu_m)^(2^(s+1)), so a double-precision estimate of the block's
  // spectrum gives the least s that reaches bits_target.  It only moves the
  // first test: eig_top squares on until two successive quotients agree, so
  // an estimate that is off costs time, not accuracy.  Never more than the
  // rule that assumes a ratio of 1/2 (squarings_for), which is also taken
  // when the estimate fails or the ratio is not below 1/2.
  static std::vector<int> squarings_est(Ctx& c, int kk, int ne, int bits_target) {
    const int k = c.k;
    std::vector<int> s(ne, squarings_for(bits_target));
    const size_t kk2 = (size_t)k * k;
    std::vector<int32_t> sg(kk2), ex(kk2);
    std::vector<uint32_t> top(3 * kk2);
    if (cudaMemcpyAsync(sg.data(), c.S.sgn, kk2 * 4, cudaMemcpyDeviceToHost, c.stream) != cudaSuccess ||
        cudaMemcpyAsync(ex.data(), c.S.exp, kk2 * 4, cudaMemcpyDeviceToHost, c.stream) != cudaSuccess ||
        cudaMemcpy2DAsync(top.data(), 12, c.S.mant + (n - 3), (size_t)n * 4, 12, kk2, cudaMemcpyDeviceToHost,
                          c.stream) != cudaSuccess ||
        cudaStreamSynchronize(c.stream) != cudaSuccess) {
      cudaGetLastError();
      return s;
    }
    int emax = INT_MIN;
    for (int a = 0; a < kk; ++a)
      for (int b = 0; b < kk; ++b)
        if (top[3 * ((size_t)a * k + b) + 2]) emax = std::max(emax, ex[(size_t)a * k + b]);
    if (emax == INT_MIN) return s;
    std::vector<double> m2((size_t)kk * kk);
    for (int a = 0; a < kk; ++a)
      for (int b = 0; b < kk; ++b) {
        const size_t e = (size_t)a * k + b;
        const double v = ((double)top[3 * e + 2] * 4294967296.0 + (double)top[3 * e + 1]) * 4294967296.0 +
                         (double)top[3 * e];
        const double x = std::ldexp(v, 32 * (ex[e] - emax) - 64);  // scaled by 2^(-32 (emax + n - 1))
        m2[(size_t)a * kk + b] = sg[e] ? -x : x;
      }
    const std::vector<double> ev = jacobi_eigenvalues(m2, kk);
    if ((int)ev.size() != kk) return s;
    for (int m = 0; m < ne; ++m) {
      if (!(ev[m] > 0)) break;
      const double r = m + 1 < kk ? std::max(ev[m + 1], 0.0) / ev[m] : 0.0;
      if (!(r < 0.5)) continue;
      const double need = r > 0 ? (double)bits_target / -std::log2(r) : 1.0;
      int sm = 1;
      while ((double)(1 << (sm + 1)) < need && sm < s[m]) ++sm;
      s[m] = std::min(s[m], sm);
    }
    return s;
  }

  // eigenvalues of the leading kk block: lam[m] = 1/nu_m (m < ne) into LAM[m]
  static hk_status block_lambdas(Ctx& c, int kk, int ne, const std::vector<int>& s, int tol, MPVec LAM,
                                 bool keep_vector) {
    const int k = c.k;
    DevVec* Sw = pool_get(c, "Sw", (int64_t)k * k);
    DevVec* V = pool_get(c, "v", k);
    DevVec* scal = pool_get(c, "scal", 16);
    DevVec* Rs = pool_get(c, "recip_s", 4);
    DevVec* ONE = one(c);
    if (!Sw || !V || !scal || !Rs || !ONE) return c.sticky;
    hk_status st;
    std::vector<ChainTask> cp;
    for (int64_t e = 0; e < (int64_t)k * k; ++e) cp.push_back(ChainTask{e, e, 0, 0, 0, 0, 0, 0});
    if ((st = chains(c, cp, c.S.view(), c.S.view(), c.S.view(), Sw->view())) != HK_OK) return st;
    for (int m = 0; m < ne; ++m) {
      if ((st = eig_top(c, Sw->view(), k, kk, s[m], tol, V->view(), *scal, 2 * m)) != HK_OK) return st;
      if (m == 0 && keep_vector) {
        DevVec* E1 = pool_get(c, "eig1", 2);  // nu_1, v^T v
        if (!E1) return c.sticky;
        if (c.evec.count != k || c.evec.n != n) {
          dev_free(c.evec);
          if ((st = check_cuda(c, dev_alloc(c.evec, k, n), "allocating evec")) != HK_OK) return st;
        }
        std::vector<ChainTask> cv;
        for (int a = 0; a < k; ++a) cv.push_back(ChainTask{a, a, 0, 0, 0, 0, 0, a < kk ? 0 : CH_ZERO_INIT});
        if ((st = chains(c, cv, V->view(), V->view(), V->view(), c.evec.view())) != HK_OK) return st;
        if ((st = chains(c, {ChainTask{0, 0, 0, 0, 0, 0, 0, 0}, ChainTask{1, 1, 0, 0, 0, 0, 0, 0}}, scal->view(),
                         scal->view(), scal->view(), E1->view())) != HK_OK)
          return st;
      }
      if (m + 1 < ne && (st = deflate(c, Sw->view(), k, kk, V->view(), *scal, 2 * m)) != HK_OK) return st;
    }
    // lambda_m = 1 / nu_m
    std::vector<int64_t> nus;
    for (int m = 0; m < ne; ++m) nus.push_back(2 * m);
    if ((st = recips(c, scal->view(), nus, *Rs)) != HK_OK) return st;
    std::vector<QuotTask> q;
    for (int m = 0; m < ne; ++m) q.push_back(QuotTask{m, 0, 2 * m, m, 0, 0});
    return quots(c, q, ONE->view(), scal->view(), *Rs, LAM);
  }

  static hk_status lambda(Ctx& c, int n_eig) {
    const int k = c.k;
    hk_status st;
    DevVec* LAM = pool_get(c, "lam", 3);
    DevVec* LAM1 = pool_get(c, "lam_km1", 3);
    DevVec* DIF = pool_get(c, "lam_diff", 3);
    if (!LAM || !LAM1 || !DIF) return c.sticky;
    // lambda to the working precision (agreement to n - 3 limbs) ...
    if ((st = block_lambdas(c, k, n_eig, squarings_est(c, k, n_eig, 32 * n + 64), n - 3, LAM->view(), true)) !=
        HK_OK)
      return st;
    const int ne1 = std::min(n_eig, k - 1);
    if (ne1 > 0) {
      // the (k-1) x (k-1) estimate only feeds a double-precision difference
      // ... the (k-1) estimate only to ~640 bits (it feeds a double-precision difference)
      if ((st = block_lambdas(c, k - 1, ne1, squarings_est(c, k - 1, ne1, 640), std::min(n - 3, 20), LAM1->view(),
                              false)) != HK_OK)
        return st;
      DevVec* ONE = one(c);
      if (!ONE) return c.sticky;
      std::vector<ChainTask> t;
      for (int m = 0; m < ne1; ++m) t.push_back(ChainTask{m, m, m, 0, 0, 0, 1, 0});
      // lam(k) - lam(k-1) * 1
      if ((st = chains(c, t, LAM1->view(), ONE->view(), LAM->view(), DIF->view())) != HK_OK) return st;
    }
    if ((st = read_device_flags(c)) != HK_OK) return st;
    c.n_eig = n_eig;
    c.lam_sgn.assign(n_eig, 0);
    c.lam_exp.assign(n_eig, 0);
    c.lam_mant.assign((size_t)n_eig * n, 0);
    c.lam_f64.assign(n_eig, 0.0);
    c.trunc_f64.assign(n_eig, NAN);
    std::vector<int32_t> ds(3), de(3);
    std::vector<uint32_t> dm(3 * n);
    if ((st = check_cuda(c, cudaMemcpy(c.lam_sgn.data(), LAM->sgn, n_eig * 4, cudaMemcpyDeviceToHost), "D2H")) ||
        (st = check_cuda(c, cudaMemcpy(c.lam_exp.data(), LAM->exp, n_eig * 4, cudaMemcpyDeviceToHost), "D2H")) ||
        (st = check_cuda(c, cudaMemcpy(c.lam_mant.data(), LAM->mant, (size_t)n_eig * n * 4, cudaMemcpyDeviceToHost),
                         "D2H")))
      return st;
    for (int m = 0; m < n_eig; ++m)
      c.lam_f64[m] = to_double(c.lam_sgn[m], c.lam_exp[m], c.lam_mant.data() + (size_t)m * n, n);
    if (ne1 > 0) {
      if ((st = check_cuda(c, cudaMemcpy(ds.data(), DIF->sgn, ne1 * 4, cudaMemcpyDeviceToHost), "D2H")) ||
          (st = check_cuda(c, cudaMemcpy(de.data(), DIF->exp, ne1 * 4, cudaMemcpyDeviceToHost), "D2H")) ||
          (st = check_cuda(c, cudaMemcpy(dm.data(), DIF->mant, (size_t)ne1 * n * 4, cudaMemcpyDeviceToHost), "D2H")))
        return st;
      for (int m = 0; m < ne1; ++m) c.trunc_f64[m] = to_double(ds[m], de[m], dm.data() + (size_t)m * n, n);
    }
    return HK_OK;
  }

  // ------------------------------------------------------------------------
  // a8: d lambda_1 / d beta = (w^T Hdot w) / (nu_1^2 v^T v),
  //     w = L^{-T} D^{-1} X v,  Hdot_ij = mudot_{i+j},
  //     mudot_s = -m mu_s (1 + m(s+1) (H_{m(s+1)-1} - gamma))   for beta = 1/m
  // ------------------------------------------------------------------------
  // mudot_s = d mu_s / d beta = -(b/a) mu_s (1 + x psi(x)), x = b(s+1)/a, for beta = a/b
  // (a > 1) into Z[s].  psi(v/a) for v = 1..b(2N-1) is a prefix sum within each
  // residue class mod a: the seeds psi(r/a) (r < a, c.psi) and psi(1) = -gamma
  // at v = a, then psi(v/a) = psi((v-a)/a) + a/(v-a) (psi(x+1) = psi(x) + 1/x),
  // summed by a Hillis-Steele scan with strides a, 2a, 4a, ...
  static hk_status mudot_rational(Ctx& c, int64_t a, int64_t b, DevVec* H0, DevVec* H1, DevVec* hq, DevVec* kint,
                                  DevVec* cst, DevVec* Z, DevVec* ONE) {
    const int N = c.N;
    const int64_t V = b * (2 * N - 1);
    hk_status st;
    // constants b/a and gamma
    if ((st = small(c, {b}, {a}, cst->view())) != HK_OK) return st;
    {
      std::vector<uint32_t> g(n);
      for (int i = 0; i < n; ++i) g[i] = hk_euler_gamma[HK_GAMMA_LIMBS - n + i];
      const int32_t gs = 0, ge = -n;
      if ((st = check_cuda(c, cudaMemcpyAsync(cst->sgn + 1, &gs, 4, cudaMemcpyHostToDevice, c.stream), "H2D")) ||
          (st = check_cuda(c, cudaMemcpyAsync(cst->exp + 1, &ge, 4, cudaMemcpyHostToDevice, c.stream), "H2D")) ||
          (st = check_cuda(c, cudaMemcpyAsync(cst->mant + n, g.data(), (size_t)n * 4, cudaMemcpyHostToDevice,
                                              c.stream), "H2D")) ||
          (st = check_cuda(c, cudaStreamSynchronize(c.stream), "H2D sync")))
        return st;
    }
    // terms: a/(v-a) for v > a, 0 elsewhere; then the seeds at v = 1..a
    {
      std::vector<int64_t> num(V + 1), den(V + 1);
      for (int64_t v = 0; v <= V; ++v) {
        num[v] = v > a ? a : 0;
        den[v] = v > a ? v - a : 1;
      }
      if ((st = small(c, num, den, H0->view())) != HK_OK) return st;
      // (only the v <= V that exist: beta > 2N - 1 leaves some seeds unused)
      std::vector<ChainTask> seeds;
      for (int64_t r = 1; r < a && r <= V; ++r) seeds.push_back(ChainTask{r, r - 1, 0, 0, 0, 0, 0, 0});
      if ((st = chains(c, seeds, ONE->view(), ONE->view(), c.psi.view(), H0->view())) != HK_OK) return st;
      if (a <= V && (st = chains(c, {ChainTask{a, 1, 0, 0, 0, 0, 0, CH_NEG_INIT}}, ONE->view(), ONE->view(),
                                 cst->view(), H0->view())) != HK_OK)
        return st;
    }
    for (int64_t d = a; d <= V; d <<= 1) {
      std::vector<ChainTask> t;
      t.reserve(V + 1);
      for (int64_t i = 0; i <= V; ++i)
        t.push_back(i >= d ? ChainTask{i, i, i - d, 0, 0, 0, 1, CH_ADD} : ChainTask{i, i, 0, 0, 0, 0, 0, 0});
      if ((st = chains(c, t, H0->view(), ONE->view(), H0->view(), H1->view())) != HK_OK) return st;
      std::swap(*H0, *H1);
    }
    // h_s = psi(x_s); q_s = 1 + x_s h_s; p_s = mu_s q_s; mudot_s = -(b/a) p_s
    std::vector<int64_t> kn, kd;
    for (int s = 0; s <= 2 * N - 2; ++s) {
      kn.push_back(b * (s + 1));
      kd.push_back(a);
    }
    if ((st = small(c, kn, kd, kint->view())) != HK_OK) return st;
    std::vector<ChainTask> t1, t2, t3, t4;
    for (int s = 0; s <= 2 * N - 2; ++s) {
      t1.push_back(ChainTask{s, b * (s + 1), 0, 0, 0, 0, 0, 0});          // psi(x_s)
      t2.push_back(ChainTask{s, 0, s, s, 0, 0, 1, CH_ADD});                // 1 + x_s h_s
      t3.push_back(ChainTask{s, 0, s, s, 0, 0, 1, CH_ZERO_INIT | CH_ADD}); // mu_s q_s
      t4.push_back(ChainTask{s, 0, 0, s, 0, 0, 1, CH_ZERO_INIT});          // -(b/a) p_s
    }
    if ((st = chains(c, t1, ONE->view(), ONE->view(), H0->view(), hq->view())) != HK_OK) return st;
    if ((st = chains(c, t2, kint->view(), hq->view(), ONE->view(), Z->view())) != HK_OK) return st;
    if ((st = chains(c, t3, c.mu.view(), Z->view(), Z->view(), hq->view())) != HK_OK) return st;
    return chains(c, t4, cst->view(), hq->view(), hq->view(), Z->view());
  }

  static hk_status grad(Ctx& c, int32_t* osgn, int32_t* oexp, uint32_t* omant, double* of64) {
    const int N = c.N, k = c.k;
    // beta = a/b in lowest terms; a = 1 is beta = 1/m (m = b)
    int64_t ga = c.beta_num, gb = c.beta_den;
    while (gb) {
      const int64_t t = ga % gb;
      ga = gb;
      gb = t;
    }
    const int64_t a = c.beta_num / ga, b = c.beta_den / ga;
    const int64_t m = b;
    hk_status st;
    DevVec* Rd = pool_get(c, "recip_d", N);
    DevVec* E1 = pool_get(c, "eig1", 2);
    DevVec* z = pool_get(c, "gz", 2 * N - 1);  // z = X v (N), later q_s and mudot_s (2N-1)
    DevVec* y = pool_get(c, "gy", N);
    DevVec* cs = pool_get(c, "gc", 2 * N - 1);
    // scan length: H_t for t <= m(2N-1) - 1 (a = 1), or psi(v/a) for v <= b(2N-1)
    const int64_t tmax = (a == 1) ? m * (2 * N - 1) - 1 : b * (2 * N - 1);
    DevVec* H0 = pool_get(c, "gh0", tmax + 1);
    DevVec* H1 = pool_get(c, "gh1", tmax + 1);
    DevVec* hq = pool_get(c, "ghq", 2 * N - 1);
    DevVec* kint = pool_get(c, "gk", 2 * N - 1);
    DevVec* cst = pool_get(c, "gconst", 4);  // 0: m, 1: gamma
    DevVec* res = pool_get(c, "gres", 4);
    DevVec* Rs = pool_get(c, "recip_s", 4);
    DevVec* ONE = one(c);
    if (!Rd || !E1 || !z || !y || !cs || !H0 || !H1 || !hq || !kint || !cst || !res || !Rs || !ONE) return c.sticky;
    // z = X v, y = D^{-1} z
    std::vector<Dot> zd;
    for (int l = 0; l < N; ++l) zd.push_back(Dot{l, (int64_t)l * k, 0, 1, 1, std::min(l + 1, k), false});
    if ((st = dots(c, zd, c.X.view(), c.evec.view(), z->view())) != HK_OK) return st;
    std::vector<QuotTask> qt;
    for (int l = 0; l < N; ++l) qt.push_back(QuotTask{l, l, tri_pos(N, l, l), l, 0, 0});
    if ((st = quots(c, qt, z->view(), c.A.view(), *Rd, y->view())) != HK_OK) return st;
    // w = L^{-T} y by column back substitution
    if (use_ntt(M)) {
      // NTT products: per step the transform of y[j] (scaled), and each warp
      // transforms its L[j][i] into its own scratch slot
      const NttConst nc = ntt_const(n);
      const size_t per = (size_t)NTT_Q * nc.L;
      constexpr int NTW = Ops<M>::NTW;
      const size_t fsm = (size_t)W * ntt_stride(nc.L) * 4, tsm = (size_t)NTW * NTT_Q * ntt_stride(nc.L) * 4;
      if ((st = check_cuda(c, allow_smem(k_ntt_fwd<M>, fsm), "smem attribute")) ||
          (st = check_cuda(c, allow_smem(k_backsub_ntt<M>, tsm), "smem attribute")))
        return st;
      const int resb = Ops<M>::resident_blocks(k_backsub_ntt<M>, 32 * NTW, tsm, c.device);
      uint32_t* F = nullptr;
      if ((st = check_cuda(c, cudaMallocAsync(&F, ((size_t)resb * NTW + 1) * per * 4, c.stream), "transforms")) !=
          HK_OK)
        return st;
      for (int j = N - 1; j >= 1; --j) {
        k_ntt_fwd<M><<<1, 32, fsm, c.stream>>>(y->view(), j, 1, F, nc, 1);
        const int grid = std::min((j + NTW - 1) / NTW, resb);
        k_backsub_ntt<M><<<grid, 32 * NTW, tsm, c.stream>>>(c.A.view(), y->view(), N, j, F, F + per, nc);
        count_launch(c, 2);
      }
      const cudaError_t e = cudaGetLastError();
      cudaFreeAsync(F, c.stream);
      if ((st = check_cuda(c, e, "back substitution")) != HK_OK) return st;
    } else {
      const size_t smem = Ops<M>::fused_smem;
      if ((st = check_cuda(c, allow_smem(k_backsub_step<M>, smem), "smem attribute")) != HK_OK) return st;
      const int resb = Ops<M>::resident_blocks(k_backsub_step<M>, 32 * W, smem, c.device);
      for (int j = N - 1; j >= 1; --j) {
        const int grid = std::min((j + W - 1) / W, resb);
        k_backsub_step<M><<<grid, 32 * W, smem, c.stream>>>(c.A.view(), y->view(), N, j);
        count_launch(c);
      }
      if ((st = check_cuda(c, cudaGetLastError(), "back substitution")) != HK_OK) return st;
    }
    // c_s = sum_{i+j=s} w_i w_j
    std::vector<Dot> cd;
    for (int s = 0; s <= 2 * N - 2; ++s) {
      const int lo = std::max(0, s - N + 1), hi = std::min(s, N - 1);
      cd.push_back(Dot{s, lo, s - lo, 1, -1, hi - lo + 1, false});
    }
    if ((st = dots(c, cd, y->view(), y->view(), cs->view(), 0, N, N)) != HK_OK) return st;
    if (a == 1) {
      // harmonic numbers H_t = sum_{j<=t} 1/j (Hillis-Steele scan of the reciprocals)
      {
        std::vector<int64_t> num(tmax + 1, 1), den(tmax + 1);
        num[0] = 0;
        for (int64_t j = 0; j <= tmax; ++j) den[j] = j ? j : 1;
        if ((st = small(c, num, den, H0->view())) != HK_OK) return st;
        for (int64_t d = 1; d <= tmax; d <<= 1) {
          std::vector<ChainTask> t;
          t.reserve(tmax + 1);
          for (int64_t i = 0; i <= tmax; ++i)
            t.push_back(i >= d ? ChainTask{i, i, i - d, 0, 0, 0, 1, CH_ADD} : ChainTask{i, i, 0, 0, 0, 0, 0, 0});
          if ((st = chains(c, t, H0->view(), ONE->view(), H0->view(), H1->view())) != HK_OK) return st;
          std::swap(*H0, *H1);
        }
      }
      // constants m and gamma
      if ((st = small(c, {m}, {1}, cst->view())) != HK_OK) return st;
      {
        std::vector<uint32_t> g(n);
        for (int i = 0; i < n; ++i) g[i] = hk_euler_gamma[HK_GAMMA_LIMBS - n + i];
        const int32_t gs = 0, ge = -n;
        if ((st = check_cuda(c, cudaMemcpyAsync(cst->sgn + 1, &gs, 4, cudaMemcpyHostToDevice, c.stream), "H2D")) ||
            (st = check_cuda(c, cudaMemcpyAsync(cst->exp + 1, &ge, 4, cudaMemcpyHostToDevice, c.stream), "H2D")) ||
            (st = check_cuda(c, cudaMemcpyAsync(cst->mant + n, g.data(), (size_t)n * 4, cudaMemcpyHostToDevice,
                                                c.stream), "H2D")) ||
            (st = check_cuda(c, cudaStreamSynchronize(c.stream), "H2D sync")))
          return st;
      }
      // h_s = H_{m(s+1)-1} - gamma ; q_s = 1 + m(s+1) h_s ; p_s = mu_s q_s ; mudot_s = -m p_s
      std::vector<int64_t> kn, kd;
      for (int s = 0; s <= 2 * N - 2; ++s) { kn.push_back(m * (s + 1)); kd.push_back(1); }
      if ((st = small(c, kn, kd, kint->view())) != HK_OK) return st;
      std::vector<ChainTask> t1, t2, t3, t4;
      for (int s = 0; s <= 2 * N - 2; ++s) {
        t1.push_back(ChainTask{s, m * (s + 1) - 1, 1, 0, 0, 0, 1, 0});             // H - gamma*1
        t2.push_back(ChainTask{s, 0, s, s, 0, 0, 1, CH_ADD});                      // 1 + kint*h
        t3.push_back(ChainTask{s, 0, s, s, 0, 0, 1, CH_ZERO_INIT | CH_ADD});       // mu*q
        t4.push_back(ChainTask{s, 0, 0, s, 0, 0, 1, CH_ZERO_INIT});                // -m*p
      }
      if ((st = chains(c, t1, cst->view(), ONE->view(), H0->view(), hq->view())) != HK_OK) return st;
      if ((st = chains(c, t2, kint->view(), hq->view(), ONE->view(), z->view())) != HK_OK) return st;
      if ((st = chains(c, t3, c.mu.view(), z->view(), z->view(), hq->view())) != HK_OK) return st;
      if ((st = chains(c, t4, cst->view(), hq->view(), hq->view(), z->view())) != HK_OK) return st;
    } else if ((st = mudot_rational(c, a, b, H0, H1, hq, kint, cst, z, ONE)) != HK_OK) {
      return st;
    }
    // g = sum_s mudot_s c_s ; t = nu^2 (v^T v) ; result = g / t
    if ((st = dots(c, {Dot{0, 0, 0, 1, 1, 2 * N - 1, false}}, z->view(), cs->view(), res->view())) != HK_OK)
      return st;
    if ((st = chains(c, {ChainTask{1, 0, 0, 0, 0, 0, 1, CH_ZERO_INIT | CH_ADD}}, E1->view(), E1->view(), E1->view(),
                     res->view())) != HK_OK)
      return st;
    if ((st = chains(c, {ChainTask{2, 0, 1, 1, 0, 0, 1, CH_ZERO_INIT | CH_ADD}}, res->view(), E1->view(),
                     res->view(), res->view())) != HK_OK)
      return st;
    if ((st = recips(c, res->view(), {2}, *Rs)) != HK_OK) return st;
    if ((st = quots(c, {QuotTask{3, 0, 2, 0, 0, 0}}, res->view(), res->view(), *Rs, res->view())) != HK_OK)
      return st;
    if ((st = read_device_flags(c)) != HK_OK) return st;
    int32_t s_ = 0, e_ = 0;
    std::vector<uint32_t> mm(n);
    if ((st = check_cuda(c, cudaMemcpy(&s_, res->sgn + 3, 4, cudaMemcpyDeviceToHost), "D2H")) ||
        (st = check_cuda(c, cudaMemcpy(&e_, res->exp + 3, 4, cudaMemcpyDeviceToHost), "D2H")) ||
        (st = check_cuda(c, cudaMemcpy(mm.data(), res->mant + 3 * (int64_t)n, (size_t)n * 4, cudaMemcpyDeviceToHost),
                         "D2H")))
      return st;
    if (osgn) *osgn = s_;
    if (oexp) *oexp = e_;
    if (omant) std::memcpy(omant, mm.data(), (size_t)n * 4);
    if (of64) *of64 = to_double(s_, e_, mm.data(), n);
    return HK_OK;
  }
};

template <int M>
hk_status Ops<M>::inv_block(Ctx& c) { return Tail<M>::inv_block(c); }
template <int M>
hk_status Ops<M>::lambda(Ctx& c, int n_eig) { return Tail<M>::lambda(c, n_eig); }
template <int M>
hk_status Ops<M>::grad(Ctx& c, int32_t* s, int32_t* e, uint32_t* m, double* f) { return Tail<M>::grad(c, s, e, m, f); }

}  // namespace hk
