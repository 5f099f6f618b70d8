/*
 * hk.h -- C ABI of libhk: the smallest eigenvalue of the Hankel moment matrix
 * H_N = (mu_{i+j}), mu_j = Gamma((j+1)/beta)/beta, by extreme-precision LDL^T
 * (arXiv 1810.01478, Secs. 2 and 4), on one GB300 GPU (sm_103a).
 *
 * Number format.  Every multiprecision value is a radix-2^32 float with n
 * limbs (n = bits/32):  value = (-1)^sign * (sum_k limb[k] 2^(32k)) * 2^(32*exp),
 * limbs little endian, the top limb (k = n-1) non-zero, or all limbs zero for
 * the value 0 (then sign = exp = 0).  Every operation of the path forms its
 * exact result and truncates the magnitude toward zero to n limbs (the
 * "compute exactly, then truncate" rule of Sec. 4.1 applied to a floating
 * format).  `bits` must be a multiple of 1024 with 32 <= n <= 1024 among the
 * compiled widths (hk_supported_bits).
 *
 * Arrays of numbers cross the boundary as three parallel arrays
 * (structure of arrays): int32 sign[count], int32 exp[count] and
 * uint32 limbs[count * n] (number i occupies limbs[i*n .. i*n+n)).
 *
 * Ownership.  A context owns all device memory it allocates (cudaMalloc) and
 * frees it in hk_destroy.  Host buffers are owned by the caller; the library
 * reads or writes them only during the call.  Device buffers passed to the
 * elementwise primitives are owned by the caller.
 *
 * Streams.  Every call is ordered on the cudaStream_t given to hk_create
 * (borrowed, never destroyed).  hk_lambda1, hk_lambda1_grad, hk_export and
 * hk_precision_loss synchronise that stream; hk_set_moments and
 * hk_set_psi_constants wait for their host-to-device copies; the other
 * calls only enqueue work.  Internally the
 * LDL^T at NTT widths runs on high-priority streams of the context, forked
 * from and joined back to that stream, and hk_inv_block runs Algorithm 4 on a
 * low-priority stream beside the still-running factorisation (each step
 * after its column of L is final) before joining back: results are as if
 * everything ran on the caller's stream.
 *
 * Errors.  Calls return hk_status; nothing aborts, traps or throws.  The
 * context keeps the first error (sticky) and hk_last_error describes it.
 * Device-side failures (a non-positive pivot, an exhausted correction loop)
 * are raised as flags in device memory and reported by the next
 * synchronising call.
 */
#ifndef HK_H
#define HK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define HK_API __attribute__((visibility("default")))
#else
#define HK_API
#endif

typedef struct hk_ctx hk_ctx;

typedef enum hk_status {
  HK_OK = 0,
  HK_ERR_ARG = 1,          /* invalid argument (size, width, pointer)            */
  HK_ERR_NOMEM = 2,        /* device allocation failed                           */
  HK_ERR_CUDA = 3,         /* a CUDA runtime call failed                         */
  HK_ERR_ORDER = 4,        /* call out of order (moments -> ldlt -> inv_block ->
                              lambda1 -> lambda1_grad)                           */
  HK_ERR_NOT_PD = 5,       /* a pivot d_i <= 0: the truncated matrix is not
                              positive definite at this precision (Sec. 4.3,
                              footnote: exact H_N needs no pivoting)            */
  HK_ERR_PRECISION = 6,    /* working precision too low for the result asked   */
  HK_ERR_TIMEOUT = 7,      /* a bounded device wait gave up                      */
  HK_ERR_UNSUPPORTED = 8   /* beta or width not supported by this build          */
} hk_status;

/* what hk_export reads */
typedef enum hk_what {
  HK_MU = 0,      /* moments mu_0..mu_{2N-2}                                     */
  HK_FACTOR = 1,  /* packed lower triangle, column major: column c holds rows
                     c..N-1 at offset c*N - c(c-1)/2; diagonal = D, below = L   */
  HK_D = 2,       /* pivots D_0..D_{N-1}                                         */
  HK_X = 3,       /* first k columns of L^{-1}, row major N x k                   */
  HK_S = 4,       /* k x k top-left block of H_N^{-1}, row major                   */
  HK_EVEC = 5     /* eigenvector of S for its largest eigenvalue (k entries)      */
} hk_what;

/* Widths compiled into this library: writes up to cap entries of bits values
 * into out and returns how many there are. */
HK_API int hk_supported_bits(int* out, int cap);

/* Create a context on CUDA device `device`, ordering work on `cuda_stream`
 * (a cudaStream_t, borrowed; NULL = legacy default stream). */
HK_API hk_status hk_create(int device, void* cuda_stream, hk_ctx** out);
HK_API void hk_destroy(hk_ctx* ctx);
/* Human-readable description of the context's first error ("" if none). */
HK_API const char* hk_last_error(const hk_ctx* ctx);

/* a1. Moments mu_j = Gamma((j+1)/beta)/beta, j = 0..2N-2, truncated to `bits`
 * (Sec. 2, eq. "moments").  beta = beta_num/beta_den, an exact rational.  This
 * build computes them on the device for beta = 1/m (m >= 1 an integer), where
 * they are the integers m * (m(j+1)-1)!  (beta = 1/2: 2 (2j+1)!; beta = 1: j!),
 * formed exactly and truncated once.  Any other beta returns
 * HK_ERR_UNSUPPORTED: use hk_moments_gamma (constants Gamma(r/a) supplied)
 * or import the moments with hk_set_moments. */
HK_API hk_status hk_moments(hk_ctx* ctx, int64_t beta_num, int64_t beta_den, int N, int bits);

/* a1 for a rational beta = beta_num/beta_den = a/b (lowest terms, a <= 64)
 * from supplied constants C_r = Gamma(r/a), r = 1..a-1 (Sec. 2, eq.
 * "moments"): with b(j+1) = q a + r, 0 <= r < a, the functional equation
 * Gamma(x+1) = x Gamma(x) gives mu_j = b C_r prod_{i<q} (r + i a) / a^(q+1),
 * and mu_j = b (q-1)! / a when r = 0.  Each mu_j is that exact product of the
 * given constant (a binary number) with a rational, truncated once to `bits`.
 *   nc:      limbs per constant
 *   c_exp:   host, a-1 limb exponents (C_r = M_r 2^(32 c_exp[r-1]))
 *   c_limbs: host, (a-1) x nc limbs, M_r little endian, top limb non-zero
 * The constants should carry at least bits + 128 correct bits (the result is
 * the exact truncation of the product with the constants as given; a moment
 * with fewer than bits/32 limbs of constant-derived value sets HK_ERR_ARG at
 * the next synchronising call).  a = 1 (beta = 1/m) needs no constants and
 * behaves as hk_moments.  b (2N-1) < 2^31.  The constants are copied before
 * the call returns. */
HK_API hk_status hk_moments_gamma(hk_ctx* ctx, int64_t beta_num, int64_t beta_den, int N, int bits, int nc,
                                  const int32_t* c_exp, const uint32_t* c_limbs);

/* a1'. Import 2N-1 moments (host arrays, number layout above) for any weight;
 * beta_num/beta_den is recorded for hk_lambda1_grad (0/0 = unknown). */
HK_API hk_status hk_set_moments(hk_ctx* ctx, int N, int bits, const int32_t* sign, const int32_t* exp,
                                const uint32_t* limbs, int64_t beta_num, int64_t beta_den);

/* a2-a4. LDL^T of H_N in place by Algorithm 1 (Sec. 4.3): for each column i,
 * B_i[r] = trunc(A[r][i] / A[i][i]) (exactly truncated quotient), then
 * A[r][c] = trunc(A[r][c] - A[c][i] * B_i[r]) for i < c <= r, one rounding per
 * update.  No pivoting.  Enqueues only; a non-positive pivot is reported as
 * HK_ERR_NOT_PD by the next synchronising call. */
HK_API hk_status hk_ldlt(hk_ctx* ctx);

/* Declares the k of the hk_inv_block that follows the next hk_ldlt (0: no
 * plan; the setting stays until changed).  With a plan, at widths and steps
 * where the trailing update runs on the tensor cores (HK_TC_MIN_ROWS), the
 * factorisation also runs those steps of Algorithm 4 (Sec. 4.4) inside the
 * same launches: row i of X is final once step i - 1 has run, and step i's
 * updates X[j][c] = trunc(X[j][c] - L[j][i] X[i][c]) use the digits of
 * column i of L that the trailing update already holds.  hk_inv_block with the
 * same k then runs only the remaining steps.  Every update is the same
 * truncated operation, in the same order for each entry, so X and S are bit
 * for bit those of the unplanned call.  hk_ldlt_batch runs every step of
 * Algorithm 4 for a planned context inside its launch.  0 <= k <= 64; a k
 * above N is HK_ERR_ARG at hk_ldlt or hk_ldlt_batch.  Enqueues nothing. */
HK_API hk_status hk_plan_block(hk_ctx* ctx, int k);

/* a5-a6. X = first k columns of L^{-1} by Algorithm 4 (Sec. 4.4; row
 * elimination, updates in increasing pivot order, one rounding each), then
 * S = (H_N^{-1})[0:k, 0:k], S_ab = sum_l X[l][a] X[l][b] / D_l (Sec. 4.4 eq.
 * "index", Sec. 4.5), each term and partial sum truncated to the working
 * precision.  1 <= k <= min(N, 64). */
HK_API hk_status hk_inv_block(hk_ctx* ctx, int k);

/* a7. The n_eig (1..3) largest eigenvalues nu_m of S and lambda_m = 1/nu_m
 * (Sec. 4.2), with the truncation estimate lambda_m(k) - lambda_m(k-1) from the
 * leading (k-1) x (k-1) block (Sec. 4.5, Table 2).  Outputs (host, any may be
 * NULL): lambda in the number layout (n_eig numbers), lambda_f64[n_eig],
 * trunc_err_f64[n_eig] (NaN when k == 1).  Synchronises.  Returns
 * HK_ERR_PRECISION (nothing written) when the working precision is below the
 * min_bits of hk_precision_loss. */
HK_API hk_status hk_lambda1(hk_ctx* ctx, int n_eig, int32_t* sign, int32_t* exp, uint32_t* limbs,
                            double* lambda_f64, double* trunc_err_f64);

/* Measured throughput of the integer multiply pipe that the exact products
 * run on, for the rooflines: operations per SM clock from a microbenchmark
 * (one 1024-thread block per SM, 8 independent chains per thread, the
 * block's own clock count, median over SMs).  kind 0: 32-bit multiply-add
 * (mad.lo.u32, x = x x + c); kind 1: the lazy Shoup modular multiplication the transforms
 * use (x w - hi(x w') p).  Runs two launches of a few ms on `device`'s
 * default stream and synchronises the device. */
HK_API hk_status hk_alu_peak(int device, int kind, double* per_clk_per_sm);

/* Precision check of the factorisation (Sec. 4.3 leaves the working
 * precision to the user; Sec. 4.1 confirms it by doubling).  loss_bits =
 * max(0, max_i ceil(log2(mu_{2i} / d_i))): the leading bits that cancelled in
 * the pivots, formed on the device right after hk_ldlt.  min_bits =
 * 2 loss + 32 + 197: the bits precision doubling shows lost stay below
 * 2 loss + 32 (beta = 1/4 ... 1), and 197 = 133 bits for 1e-40 plus 64 to
 * spare.  After hk_ldlt; outputs (host) may be NULL; synchronises. */
HK_API hk_status hk_precision_loss(hk_ctx* ctx, int32_t* loss_bits, int32_t* min_bits);

/* a8. d lambda_1 / d beta of the block estimate lambda_1 = 1/nu_1:
 * (w^T Hdot w)/nu_1^2 with w = L^{-T} D^{-1} X u (u the unit eigenvector) and
 * Hdot_ij = d mu_{i+j}/d beta = -(mu/beta)(1 + x psi(x)), x = (i+j+1)/beta.
 * For beta = 1/m, psi(x) = H_{x-1} - gamma (x an integer); for beta = a/b
 * (a > 1) psi(x) follows from psi(x + 1) = psi(x) + 1/x and the constants
 * psi(r/a), r = 1..a-1, given beforehand with hk_set_psi_constants (else
 * HK_ERR_UNSUPPORTED).  Outputs (host, may be NULL): one number, and its
 * double.  Synchronises. */
HK_API hk_status hk_lambda1_grad(hk_ctx* ctx, int32_t* sign, int32_t* exp, uint32_t* limbs, double* f64);

/* The constants psi(r/a) (digamma), r = 1..a-1, for hk_lambda1_grad at
 * beta = a/b: `count` numbers of nc limbs each (host, number layout above,
 * copied before the call returns), truncated or zero-extended to the working
 * width.  After the moments; count = a - 1. */
HK_API hk_status hk_set_psi_constants(hk_ctx* ctx, int count, int nc, const int32_t* sign, const int32_t* exp,
                                      const uint32_t* limbs);

/* Copy count numbers starting at index first of `what` to host arrays.
 * Synchronises. */
HK_API hk_status hk_export(hk_ctx* ctx, int what, int64_t first, int64_t count, int32_t* sign, int32_t* exp,
                           uint32_t* limbs);

/* Profiling (the paper reports per-phase wall times, Table 2; here CUDA
 * events on the context's stream).  hk_set_profiling(ctx, 1) clears and
 * enables the counters; hk_get_profile synchronises and writes
 * HK_PROFILE_FIELDS doubles:
 *   [0] kernel launches since enabling
 *   [1] total device time of the trailing-update kernels (Algorithm 1), ms
 *   [2] number of trailing-update launches
 *   [3] algorithmic limb products of those launches (n^2 per fused update)
 *   [4] moments ms, [5] LDL^T ms, [6] Algorithm 4 + block ms,
 *   [7] eigenvalues ms, [8] gradient ms,
 *   [9] column scale (B_i) and its transforms within the LDL^T, ms
 *   [10] device time of the trailing-update launches with tensor-core
 *        products (included in [1]), ms; [11] their number; [12] the
 *        tcgen05.mma instructions they issued (M = 128, N = 256, K = 16 each)
 *   [13] 128-row items whose short products left a row undecided, re-run
 *        with whole products (their instructions are included in [12]) */
#define HK_PROFILE_FIELDS 14
HK_API hk_status hk_set_profiling(hk_ctx* ctx, int on);
HK_API hk_status hk_get_profile(hk_ctx* ctx, double* out, int cap);

/* Exact limb products of the factorisation and of hk_fused_batch, chosen
 * process-wide: HK_PRODUCT_SCHOOLBOOK (n^2 32x32-bit limb products, warp
 * operand scanning), HK_PRODUCT_NTT (number-theoretic transforms of length
 * 2^a or 3 2^a modulo three primes k 3 2^11 + 1 below 2^30 and Chinese
 * remaindering; the transforms of a step's pivot column are computed once and
 * reused by every update, n <= 1024 limbs), HK_PRODUCT_TENSOR (from
 * HK_TC_MIN_M * 1024 bits: the trailing update's products as bf16 GEMMs on
 * the tensor cores, balanced 7-bit digits whose convolution sums stay below
 * 2^24 and so are exact in fp32; the other products of the path use the
 * NTT), or HK_PRODUCT_AUTO (the NTT from HK_NTT_AUTO_MIN_M * 1024 bits up,
 * the tensor cores from HK_TC_AUTO_MIN_M * 1024 bits up).  All give the same
 * exact product, so results are identical bit for bit; this only changes
 * speed.  The paper's GMP multiplies likewise switch algorithm by size. */
#define HK_PRODUCT_AUTO 0
#define HK_PRODUCT_SCHOOLBOOK 1
#define HK_PRODUCT_NTT 2
#define HK_PRODUCT_TENSOR 3
#define HK_NTT_AUTO_MIN_M 8
#define HK_TC_MIN_M 8
/* widest width of hk_ldlt_batch: 1024 * HK_BATCH_MAX_M bits; largest N */
#define HK_BATCH_MAX_M 8
#define HK_BATCH_MAX_N 32768
#define HK_TC_AUTO_MIN_M 12
/* With tensor-core products, steps of Algorithm 1 whose trailing triangle has
 * fewer rows than this keep NTT products (too few 128-row work items to fill
 * the GPU), and so does each step's look-ahead entry (i+1, i+1). */
#define HK_TC_MIN_ROWS 256
HK_API hk_status hk_set_product_algorithm(int algorithm);

/* Elementwise primitives on caller-owned DEVICE arrays of `count` numbers of
 * width `bits`, ordered on cuda_stream (no synchronisation, except that
 * hk_div_batch and hk_fused_batch with HK_PRODUCT_TENSOR read their device
 * flags back and synchronise):
 *   hk_fused_batch: out[i] = trunc(a[i] - x[i]*y[i])  (the update of Alg. 1/4)
 *   hk_div_batch:   out[i] = trunc(a[i] / d[i])      (d[i] != 0)
 * `out` may not alias the inputs. */
HK_API hk_status hk_fused_batch(int bits, int64_t count, const int32_t* a_sign, const int32_t* a_exp,
                                const uint32_t* a_limbs, const int32_t* x_sign, const int32_t* x_exp,
                                const uint32_t* x_limbs, const int32_t* y_sign, const int32_t* y_exp,
                                const uint32_t* y_limbs, int32_t* out_sign, int32_t* out_exp,
                                uint32_t* out_limbs, void* cuda_stream);
HK_API hk_status hk_div_batch(int bits, int64_t count, const int32_t* a_sign, const int32_t* a_exp,
                              const uint32_t* a_limbs, const int32_t* d_sign, const int32_t* d_exp,
                              const uint32_t* d_limbs, int32_t* out_sign, int32_t* out_exp, uint32_t* out_limbs,
                              void* cuda_stream);

/* a9. Batched form: `count` independent instances (uneven beta, N, k, bits)
 * solved concurrently on one device, each on its own stream and context,
 * in waves of up to `max_concurrent` instances (0 = all in one wave), each
 * wave driven by as many host threads.  Per instance: moments on the device
 * when mu_* are NULL (beta = 1/m), else imported from the host arrays; then
 * the factorisation: the wave's instances of one width up to
 * HK_BATCH_MAX_M * 1024 bits, when there are two or more, share one
 * persistent launch (hk_ldlt_batch), every other instance runs hk_ldlt;
 * then hk_inv_block(k) and hk_lambda1(n_eig).  Results and the instance's
 * own status are written into its struct; the call returns HK_OK when every
 * instance succeeded, else the first failing instance's status. */
typedef struct hk_instance {
  int64_t beta_num, beta_den;
  int32_t N, k, bits, n_eig;
  const int32_t* mu_sign;       /* host, 2N-1 moments, or NULL */
  const int32_t* mu_exp;
  const uint32_t* mu_limbs;
  const int32_t* gamma_exp;     /* host, constants of hk_moments_gamma (a-1 of */
  const uint32_t* gamma_limbs;  /* gamma_nc limbs), used when mu_* are NULL and */
                                /* beta is not 1/m; else NULL */
  int32_t* lambda_sign;         /* host outputs, n_eig numbers, or NULL */
  int32_t* lambda_exp;
  uint32_t* lambda_limbs;
  double lambda_f64[3];
  double trunc_err_f64[3];
  double seconds;               /* wall time of this instance */
  int32_t status;
  int32_t gamma_nc;
  char message[128];            /* hk_last_error of a failed instance ("" if none) */
} hk_instance;
HK_API hk_status hk_batch_run(int device, hk_instance* inst, int count, int max_concurrent);

/* a9. Algorithm 1 (Sec. 4.3) for `count` contexts in ONE persistent launch.
 * Every context must be on one device, at one width of at most
 * HK_BATCH_MAX_M * 1024 bits (else HK_ERR_ARG / HK_ERR_UNSUPPORTED), with
 * its moments set (else HK_ERR_ORDER), N <= HK_BATCH_MAX_N and a planned k
 * <= N (else HK_ERR_ARG), and appear once.  Each instance's
 * factorisation is a chain of phases (the pivot's reciprocal, the column
 * scale, the trailing update of each step); the launch's warps take work
 * items from whichever instance has some, so small instances share the
 * device without a launch per step.  A context planned with a block size
 * k (hk_plan_block) also gets Algorithm 4's X = L^-1[:, :k] inside the
 * launch (step i's updates share step i's trailing phase), so its
 * hk_inv_block(k) goes straight to the block.  Afterwards every context is
 * where hk_ldlt leaves it, with a bit-identical factor and X (schoolbook
 * products).
 * Ordering: the launch runs on the first context's stream after every
 * context's stream reaches this call; every context's stream then waits
 * for it.  The contexts must not be used from other threads meanwhile.
 * idle_limit_s bounds how long the launch waits while no phase of any
 * instance advances (negative: 2 s); when it runs out the launch returns
 * and every unfinished instance reports HK_ERR_TIMEOUT at its next
 * synchronising call (the device stays usable; the context keeps that
 * error like any other, so a new context repeats the work).
 * A pivot <= 0 ends that instance only (HK_ERR_NOT_PD as for hk_ldlt). */
HK_API hk_status hk_ldlt_batch(hk_ctx* const* ctx, int count, double idle_limit_s);

/* a9. Autotuner of hk_ldlt_batch's launch shape.  Times one batch of `count`
 * instances (beta = 1/m, m = 1, 2, 3, 4 in turn, each of size N, at `bits`)
 * under each candidate shape (blocks per SM in {1, 2, 3, 4, 6, 8, 12, 16} up to
 * what fits, items per claim in the largest phases in {1, 4, 8, 16}; the
 * faster of two runs each) and keeps the fastest for this width and N's
 * bucket (N <= 128, <= 256, ... doubling), where every later hk_ldlt_batch
 * whose largest N falls in that bucket uses it (process-wide; untuned
 * buckets take 8 items and 8, 6 or 4 blocks per SM up to 2048, 6144 and
 * 8192 bits).  Outputs (host, may be NULL):
 * the chosen shape and its seconds.  Synchronises the device.  Errors:
 * HK_ERR_ARG (N outside 1..16384, count outside 1..256, bits not
 * compiled), HK_ERR_UNSUPPORTED (bits above the batched widths), or the
 * status of a run that failed (e.g. HK_ERR_NOT_PD when bits is too low for
 * N); nothing is stored then. */
HK_API hk_status hk_tune_batch(int device, int bits, int N, int count, int32_t* blocks_per_sm, int32_t* chunk,
                               double* seconds);

/* Allocation-free LDL^T (no counterpart in the paper: an interface for
 * callers that cannot allow a library to allocate device memory, e.g. a
 * process whose device memory belongs to one allocator or to a fixed budget).
 * Runs the same Algorithm 1 as hk_ldlt, with the same results, but takes
 * every byte of scratch (the pivot column, the pivot reciprocal, an error
 * word) from one fixed 4 MiB array in device memory that the library declares;
 * it calls no cudaMalloc/cudaFree and allocates nothing else.
 *   mu_*:  DEVICE arrays of the 2N-1 moments (layout above), read only
 *   f_*:   DEVICE arrays of N(N+1)/2 numbers, the packed factor as HK_FACTOR
 *          describes it (caller-allocated), written
 *   limit: N * (bits/32 + 2) + bits/32 + 35 <= HK_NOALLOC_SCRATCH_WORDS,
 *          else HK_ERR_ARG (e.g. N <= 1024 at bits <= 24576)
 * Each call looks the array's address up on the current device.  No call
 * may run on a capturing stream: each one reads the device error word back
 * and synchronises cuda_stream (below).  Every call shares the array,
 * so calls that overlap on the GPU race: the caller serialises them.  Each
 * call reads the device error word back and synchronises cuda_stream before
 * it returns, and reports device flags with the same status codes as
 * hk_ldlt's next synchronising call (HK_ERR_NOT_PD for a non-positive pivot).
 * Products are schoolbook (n^2 limb products) at every width, so at the NTT
 * widths (from HK_NTT_AUTO_MIN_M * 1024 bits) it is slower than hk_ldlt. */
#define HK_NOALLOC_SCRATCH_WORDS (1u << 20)
HK_API hk_status hk_ldlt_noalloc(int bits, int N, const int32_t* mu_sign, const int32_t* mu_exp,
                                 const uint32_t* mu_limbs, int32_t* f_sign, int32_t* f_exp, uint32_t* f_limbs,
                                 void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* HK_H */
