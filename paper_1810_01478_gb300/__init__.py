"""Python binding of libhk (include/hk.h): argument marshalling only.

Every step of the path runs in the CUDA library; this module loads
``_build/libhk.so`` (built by ``build.build()``), forwards calls with the same
names as the C ABI, and converts the (sign, exp, limbs) layout to and from
numpy arrays.  There is no CPU fallback: if the library is missing the first
call raises.

Number layout: value = (-1)^sign * (sum_k limbs[k] 2^(32k)) * 2^(32*exp), n limbs
little endian with a non-zero top limb, or all zero for 0.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libhk.so")

HK_OK, HK_ERR_ARG, HK_ERR_NOMEM, HK_ERR_CUDA, HK_ERR_ORDER = 0, 1, 2, 3, 4
HK_ERR_NOT_PD, HK_ERR_PRECISION, HK_ERR_TIMEOUT, HK_ERR_UNSUPPORTED = 5, 6, 7, 8
HK_MU, HK_FACTOR, HK_D, HK_X, HK_S, HK_EVEC = 0, 1, 2, 3, 4, 5

STATUS_NAMES = {0: "HK_OK", 1: "HK_ERR_ARG", 2: "HK_ERR_NOMEM", 3: "HK_ERR_CUDA", 4: "HK_ERR_ORDER",
                5: "HK_ERR_NOT_PD", 6: "HK_ERR_PRECISION", 7: "HK_ERR_TIMEOUT", 8: "HK_ERR_UNSUPPORTED"}

# every entry point declared in include/hk.h
EXPORTS = ["hk_supported_bits", "hk_create", "hk_destroy", "hk_last_error", "hk_moments", "hk_set_moments",
           "hk_ldlt", "hk_plan_block", "hk_inv_block", "hk_lambda1", "hk_lambda1_grad", "hk_export", "hk_fused_batch",
           "hk_div_batch", "hk_set_profiling", "hk_get_profile", "hk_ldlt_noalloc", "hk_batch_run",
           "hk_ldlt_batch", "hk_tune_batch",
           "hk_set_product_algorithm", "hk_moments_gamma", "hk_set_psi_constants", "hk_precision_loss", "hk_alu_peak"]
HK_PRODUCT_AUTO, HK_PRODUCT_SCHOOLBOOK, HK_PRODUCT_NTT, HK_PRODUCT_TENSOR = 0, 1, 2, 3
HK_NTT_AUTO_MIN_M = 8  # include/hk.h: AUTO uses NTT products from 32 * 8 limbs (8192 bits)
HK_TC_MIN_M = 8        # include/hk.h: tensor-core products exist from 8192 bits
HK_TC_AUTO_MIN_M = 12  # include/hk.h: AUTO uses them from 12288 bits
HK_TC_MIN_ROWS = 256   # include/hk.h: steps with fewer trailing rows keep NTT products


class Instance(ctypes.Structure):
    """hk_instance of include/hk.h (one problem of hk_batch_run)."""
    _fields_ = [("beta_num", ctypes.c_int64), ("beta_den", ctypes.c_int64), ("N", ctypes.c_int32),
                ("k", ctypes.c_int32), ("bits", ctypes.c_int32), ("n_eig", ctypes.c_int32),
                ("mu_sign", ctypes.c_void_p), ("mu_exp", ctypes.c_void_p), ("mu_limbs", ctypes.c_void_p),
                ("gamma_exp", ctypes.c_void_p), ("gamma_limbs", ctypes.c_void_p),
                ("lambda_sign", ctypes.c_void_p), ("lambda_exp", ctypes.c_void_p), ("lambda_limbs", ctypes.c_void_p),
                ("lambda_f64", ctypes.c_double * 3), ("trunc_err_f64", ctypes.c_double * 3),
                ("seconds", ctypes.c_double), ("status", ctypes.c_int32), ("gamma_nc", ctypes.c_int32),
                ("message", ctypes.c_char * 128)]
PROFILE_FIELDS = 14


class HKError(RuntimeError):
    def __init__(self, status, msg=""):
        self.status = status
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")


_lib = None
_P = ctypes.c_void_p
_I32P = ctypes.POINTER(ctypes.c_int32)
_U32P = ctypes.POINTER(ctypes.c_uint32)
_F64P = ctypes.POINTER(ctypes.c_double)


def load(path=LIB_PATH):
    """Load libhk.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libhk.so not found at {path}: call paper_1810_01478_gb300.build.build() first")
    L = ctypes.CDLL(path)
    L.hk_supported_bits.argtypes = [_I32P, ctypes.c_int]
    L.hk_supported_bits.restype = ctypes.c_int
    L.hk_create.argtypes = [ctypes.c_int, _P, ctypes.POINTER(_P)]
    L.hk_destroy.argtypes = [_P]
    L.hk_destroy.restype = None
    L.hk_last_error.argtypes = [_P]
    L.hk_last_error.restype = ctypes.c_char_p
    L.hk_moments.argtypes = [_P, ctypes.c_int64, ctypes.c_int64, ctypes.c_int, ctypes.c_int]
    L.hk_set_moments.argtypes = [_P, ctypes.c_int, ctypes.c_int, _I32P, _I32P, _U32P, ctypes.c_int64,
                                 ctypes.c_int64]
    L.hk_moments_gamma.argtypes = [_P, ctypes.c_int64, ctypes.c_int64, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                   _I32P, _U32P]
    L.hk_set_psi_constants.argtypes = [_P, ctypes.c_int, ctypes.c_int, _I32P, _I32P, _U32P]
    L.hk_precision_loss.argtypes = [_P, _I32P, _I32P]
    L.hk_alu_peak.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]
    L.hk_ldlt.argtypes = [_P]
    L.hk_inv_block.argtypes = [_P, ctypes.c_int]
    L.hk_plan_block.argtypes = [_P, ctypes.c_int]
    L.hk_lambda1.argtypes = [_P, ctypes.c_int, _I32P, _I32P, _U32P, _F64P, _F64P]
    L.hk_lambda1_grad.argtypes = [_P, _I32P, _I32P, _U32P, _F64P]
    L.hk_export.argtypes = [_P, ctypes.c_int, ctypes.c_int64, ctypes.c_int64, _I32P, _I32P, _U32P]
    L.hk_fused_batch.argtypes = [ctypes.c_int, ctypes.c_int64] + [_P] * 12 + [_P]
    L.hk_div_batch.argtypes = [ctypes.c_int, ctypes.c_int64] + [_P] * 9 + [_P]
    L.hk_set_profiling.argtypes = [_P, ctypes.c_int]
    L.hk_set_product_algorithm.argtypes = [ctypes.c_int]
    L.hk_batch_run.argtypes = [ctypes.c_int, ctypes.POINTER(Instance), ctypes.c_int, ctypes.c_int]
    L.hk_ldlt_noalloc.argtypes = [ctypes.c_int, ctypes.c_int] + [_P] * 6 + [_P]
    L.hk_ldlt_batch.argtypes = [ctypes.POINTER(_P), ctypes.c_int, ctypes.c_double]
    L.hk_tune_batch.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _I32P, _I32P, _F64P]
    L.hk_get_profile.argtypes = [_P, _F64P, ctypes.c_int]
    for name in ("hk_set_product_algorithm", "hk_batch_run", "hk_ldlt_noalloc", "hk_ldlt_batch", "hk_tune_batch", "hk_set_profiling", "hk_get_profile", "hk_create", "hk_moments", "hk_set_moments", "hk_ldlt", "hk_inv_block", "hk_lambda1",
                 "hk_plan_block", "hk_lambda1_grad", "hk_export", "hk_fused_batch", "hk_div_batch", "hk_moments_gamma", "hk_set_psi_constants", "hk_precision_loss", "hk_alu_peak"):
        getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def _ptr(a, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def _check(st, ctx=None, what=""):
    if st != HK_OK:
        msg = load().hk_last_error(ctx).decode() if ctx else what
        raise HKError(st, msg or what)


def hk_supported_bits():
    L = load()
    cnt = L.hk_supported_bits(None, 0)
    out = np.zeros(cnt, np.int32)
    L.hk_supported_bits(_ptr(out, ctypes.c_int32), cnt)
    return [int(v) for v in out]


def hk_create(device=0, stream=None):
    """stream: a cudaStream_t as an int (e.g. torch.cuda.current_stream().cuda_stream) or None."""
    L = load()
    h = _P()
    _check(L.hk_create(device, _P(stream or 0), ctypes.byref(h)), what="hk_create")
    return h


def hk_destroy(ctx):
    load().hk_destroy(ctx)


def hk_last_error(ctx):
    return load().hk_last_error(ctx).decode()


def hk_moments(ctx, beta_num, beta_den, N, bits):
    _check(load().hk_moments(ctx, beta_num, beta_den, N, bits), ctx)


def hk_moments_gamma(ctx, beta_num, beta_den, N, bits, c_exp, c_limbs):
    """Moments for beta = a/b from constants Gamma(r/a), r = 1..a-1:
    c_exp (a-1 int32 limb exponents), c_limbs ((a-1) x nc uint32)."""
    c_exp = np.ascontiguousarray(c_exp, dtype=np.int32)
    c_limbs = np.ascontiguousarray(c_limbs, dtype=np.uint32)
    nc = c_limbs.shape[1] if c_limbs.ndim == 2 and c_limbs.shape[0] else 1
    _check(load().hk_moments_gamma(ctx, beta_num, beta_den, N, bits, nc, _ptr(c_exp, ctypes.c_int32),
                                   _ptr(c_limbs, ctypes.c_uint32)), ctx)


def hk_alu_peak(device, kind):
    """Measured operations per SM clock of the integer multiply pipe:
    kind 0 = mad.lo.u32, kind 1 = lazy Shoup modular multiplication."""
    v = ctypes.c_double(0.0)
    _check(load().hk_alu_peak(device, kind, ctypes.byref(v)), None, "hk_alu_peak")
    return v.value


def hk_precision_loss(ctx):
    """(loss_bits, min_bits) of the factorisation (after hk_ldlt)."""
    loss = np.zeros(1, np.int32)
    mb = np.zeros(1, np.int32)
    _check(load().hk_precision_loss(ctx, _ptr(loss, ctypes.c_int32), _ptr(mb, ctypes.c_int32)), ctx)
    return int(loss[0]), int(mb[0])


def hk_set_psi_constants(ctx, sign, exp, limbs):
    """psi(r/a), r = 1..a-1, for hk_lambda1_grad at beta = a/b: sign, exp
    (int32 per constant) and limbs (count x nc uint32)."""
    sign = np.ascontiguousarray(sign, dtype=np.int32)
    exp = np.ascontiguousarray(exp, dtype=np.int32)
    limbs = np.ascontiguousarray(limbs, dtype=np.uint32)
    count = len(sign)
    nc = limbs.shape[1] if count else 1
    _check(load().hk_set_psi_constants(ctx, count, nc, _ptr(sign, ctypes.c_int32), _ptr(exp, ctypes.c_int32),
                                       _ptr(limbs, ctypes.c_uint32)), ctx)


def hk_set_moments(ctx, N, bits, sign, exp, limbs, beta_num=0, beta_den=0):
    sign = np.ascontiguousarray(sign, np.int32)
    exp = np.ascontiguousarray(exp, np.int32)
    limbs = np.ascontiguousarray(limbs, np.uint32)
    n = bits // 32
    if sign.size != 2 * N - 1 or exp.size != 2 * N - 1 or limbs.size != (2 * N - 1) * n:
        raise ValueError("hk_set_moments needs 2N-1 numbers of bits/32 limbs")
    _check(load().hk_set_moments(ctx, N, bits, _ptr(sign, ctypes.c_int32), _ptr(exp, ctypes.c_int32),
                                 _ptr(limbs, ctypes.c_uint32), beta_num, beta_den), ctx)


def hk_ldlt(ctx):
    _check(load().hk_ldlt(ctx), ctx)


def hk_plan_block(ctx, k):
    """Declare the k of the coming hk_inv_block (see include/hk.h)."""
    _check(load().hk_plan_block(ctx, k), ctx)


def hk_inv_block(ctx, k):
    _check(load().hk_inv_block(ctx, k), ctx)


def hk_lambda1(ctx, n_eig, n):
    """Returns (sign[n_eig], exp[n_eig], limbs[n_eig, n], lambda_f64[n_eig], trunc_err_f64[n_eig])."""
    s = np.zeros(n_eig, np.int32)
    e = np.zeros(n_eig, np.int32)
    m = np.zeros((n_eig, n), np.uint32)
    f = np.zeros(n_eig, np.float64)
    t = np.zeros(n_eig, np.float64)
    _check(load().hk_lambda1(ctx, n_eig, _ptr(s, ctypes.c_int32), _ptr(e, ctypes.c_int32),
                             _ptr(m, ctypes.c_uint32), _ptr(f, ctypes.c_double), _ptr(t, ctypes.c_double)), ctx)
    return s, e, m, f, t


def hk_lambda1_grad(ctx, n):
    s = np.zeros(1, np.int32)
    e = np.zeros(1, np.int32)
    m = np.zeros((1, n), np.uint32)
    f = np.zeros(1, np.float64)
    _check(load().hk_lambda1_grad(ctx, _ptr(s, ctypes.c_int32), _ptr(e, ctypes.c_int32),
                                  _ptr(m, ctypes.c_uint32), _ptr(f, ctypes.c_double)), ctx)
    return s, e, m, f


def hk_export(ctx, what, first, count, n):
    s = np.zeros(count, np.int32)
    e = np.zeros(count, np.int32)
    m = np.zeros((count, n), np.uint32)
    _check(load().hk_export(ctx, what, first, count, _ptr(s, ctypes.c_int32), _ptr(e, ctypes.c_int32),
                            _ptr(m, ctypes.c_uint32)), ctx)
    return s, e, m


def hk_fused_batch(bits, count, a, x, y, out, stream=None):
    """a, x, y, out: (sign_ptr, exp_ptr, limbs_ptr) device addresses (ints)."""
    args = [_P(p) for t in (a, x, y, out) for p in t]
    _check(load().hk_fused_batch(bits, count, *args, _P(stream or 0)), what="hk_fused_batch")


def hk_div_batch(bits, count, a, d, out, stream=None):
    args = [_P(p) for t in (a, d, out) for p in t]
    _check(load().hk_div_batch(bits, count, *args, _P(stream or 0)), what="hk_div_batch")


def hk_set_product_algorithm(algorithm):
    """HK_PRODUCT_AUTO / _SCHOOLBOOK / _NTT / _TENSOR (process-wide)."""
    _check(load().hk_set_product_algorithm(algorithm), what="hk_set_product_algorithm")


def hk_set_profiling(ctx, on=True):
    _check(load().hk_set_profiling(ctx, 1 if on else 0), ctx)


def hk_get_profile(ctx):
    """dict of the counters described in include/hk.h (hk_get_profile)."""
    out = np.zeros(PROFILE_FIELDS, np.float64)
    _check(load().hk_get_profile(ctx, _ptr(out, ctypes.c_double), PROFILE_FIELDS), ctx)
    keys = ["launches", "trailing_ms", "trailing_launches", "trailing_limb_macs", "moments_ms", "ldlt_ms",
            "invblock_ms", "eig_ms", "grad_ms", "scale_ms", "tc_ms", "tc_launches", "tc_mmas",
            "tc_redo_items"]
    return dict(zip(keys, out.tolist()))


def hk_ldlt_noalloc(bits, N, mu, factor, stream=None):
    """LDL^T into a caller-allocated factor without any device allocation.

    mu: (sign_ptr, exp_ptr, limbs_ptr) device addresses of the 2N-1 moments;
    factor: the same for N(N+1)/2 numbers (written).  For callers that cannot
    let the library allocate device memory; see include/hk.h for the scratch
    limit and the rule that overlapping calls race."""
    args = [_P(p) for t in (mu, factor) for p in t]
    _check(load().hk_ldlt_noalloc(bits, N, *args, _P(stream or 0)), what="hk_ldlt_noalloc")


def hk_ldlt_batch(ctxs, idle_limit_s=-1.0):
    """Algorithm 1 for several contexts (one device and width, moments set)
    in one persistent launch; see include/hk.h.  idle_limit_s < 0: 2 s."""
    arr = (_P * len(ctxs))(*[c.value if isinstance(c, _P) else c for c in ctxs])
    _check(load().hk_ldlt_batch(arr, len(ctxs), float(idle_limit_s)), ctxs[0] if ctxs else None,
           what="hk_ldlt_batch")


def hk_tune_batch(device, bits, N, count):
    """Time hk_ldlt_batch's launch shapes on `count` instances of size N at
    `bits` and keep the fastest for that width and N bucket (include/hk.h).
    Returns (blocks_per_sm, items_per_claim, seconds)."""
    b = np.zeros(1, np.int32)
    g = np.zeros(1, np.int32)
    t = np.zeros(1, np.float64)
    _check(load().hk_tune_batch(device, bits, N, count, _ptr(b, ctypes.c_int32), _ptr(g, ctypes.c_int32),
                                _ptr(t, ctypes.c_double)), what="hk_tune_batch")
    return int(b[0]), int(g[0]), float(t[0])


def hk_batch_run(device, problems, max_concurrent=0):
    """Solve several instances concurrently.  problems: list of dicts with
    beta (num, den), N, k, bits, n_eig and optionally mu = (sign, exp, limbs)
    (imported moments) or gamma = (exp, limbs) (the constants of
    hk_moments_gamma).  Returns a list of dicts (status, lambda_f64,
    trunc_err_f64, lambda = (sign, exp, limbs), seconds) in the same order."""
    arr = (Instance * len(problems))()
    keep, lams = [], []
    for i, p in enumerate(problems):
        it = arr[i]
        it.beta_num, it.beta_den = p["beta"]
        it.N, it.k, it.bits, it.n_eig = p["N"], p["k"], p["bits"], p.get("n_eig", 1)
        n = p["bits"] // 32
        if p.get("mu") is not None:
            s, e, m = (np.ascontiguousarray(p["mu"][0], np.int32), np.ascontiguousarray(p["mu"][1], np.int32),
                       np.ascontiguousarray(p["mu"][2], np.uint32))
            keep += [s, e, m]
            it.mu_sign, it.mu_exp, it.mu_limbs = s.ctypes.data, e.ctypes.data, m.ctypes.data
        if p.get("gamma") is not None:
            ge = np.ascontiguousarray(p["gamma"][0], np.int32)
            gl = np.ascontiguousarray(p["gamma"][1], np.uint32)
            keep += [ge, gl]
            it.gamma_exp, it.gamma_limbs, it.gamma_nc = ge.ctypes.data, gl.ctypes.data, gl.shape[1]
        ls = np.zeros(it.n_eig, np.int32)
        le = np.zeros(it.n_eig, np.int32)
        lm = np.zeros((it.n_eig, n), np.uint32)
        lams.append((ls, le, lm))
        it.lambda_sign, it.lambda_exp, it.lambda_limbs = ls.ctypes.data, le.ctypes.data, lm.ctypes.data
    st = load().hk_batch_run(device, arr, len(problems), max_concurrent)
    out = []
    for i in range(len(problems)):
        it = arr[i]
        out.append({"status": it.status, "message": it.message.decode(errors="replace"),
                    "lambda_f64": list(it.lambda_f64)[:it.n_eig],
                    "trunc_err_f64": list(it.trunc_err_f64)[:it.n_eig], "seconds": it.seconds, "lambda": lams[i]})
    return st, out


# --- layout helpers (host-side marshalling) ---------------------------------

def limbs_to_int(row):
    v = 0
    for i, w in enumerate(np.asarray(row, np.uint64).tolist()):
        v |= int(w) << (32 * i)
    return v


def int_to_limbs(v, n):
    return np.array([(v >> (32 * i)) & 0xFFFFFFFF for i in range(n)], np.uint32)


def int_to_layout(v, n):
    """An exact integer truncated into the number layout (sign, exp, limbs)."""
    if v == 0:
        return 0, 0, np.zeros(n, np.uint32)
    s = 1 if v < 0 else 0
    a = -v if v < 0 else v
    L = (a.bit_length() + 31) // 32
    e = L - n
    a = a >> (32 * e) if e >= 0 else a << (32 * -e)
    return s, e, int_to_limbs(a, n)


class Hankel:
    """The whole path on one device: moments -> LDL^T -> block -> lambda (-> gradient)."""

    def __init__(self, device=0, stream=None):
        self.ctx = hk_create(device, stream)
        self.n = None

    def close(self):
        if self.ctx is not None:
            hk_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def moments(self, beta_num, beta_den, N, bits):
        self.n = bits // 32
        hk_moments(self.ctx, beta_num, beta_den, N, bits)

    def moments_gamma(self, beta_num, beta_den, N, bits, c_exp, c_limbs):
        self.n = bits // 32
        hk_moments_gamma(self.ctx, beta_num, beta_den, N, bits, c_exp, c_limbs)

    def precision_loss(self):
        return hk_precision_loss(self.ctx)

    def set_psi_constants(self, sign, exp, limbs):
        hk_set_psi_constants(self.ctx, sign, exp, limbs)

    def set_moments(self, N, bits, sign, exp, limbs, beta_num=0, beta_den=0):
        self.n = bits // 32
        hk_set_moments(self.ctx, N, bits, sign, exp, limbs, beta_num, beta_den)

    def ldlt(self, k=None):
        """LDL^T; with k, Algorithm 4 for that k runs inside the tensor-core
        steps (hk_plan_block) and inv_block(k) finishes it."""
        if k is not None:
            hk_plan_block(self.ctx, k)
        hk_ldlt(self.ctx)

    def inv_block(self, k):
        hk_inv_block(self.ctx, k)

    def lambda1(self, n_eig=1):
        return hk_lambda1(self.ctx, n_eig, self.n)

    def lambda1_grad(self):
        return hk_lambda1_grad(self.ctx, self.n)

    def export(self, what, first, count):
        return hk_export(self.ctx, what, first, count, self.n)


# ---------------------------------------------------------------------------
# differentiable front end
# ---------------------------------------------------------------------------
def _exact_beta(beta, max_den=1000):
    """beta (a float, a 0-dim tensor or a Fraction) as an exact a/b with b <= max_den."""
    from fractions import Fraction
    v = Fraction(beta) if isinstance(beta, Fraction) else Fraction(float(beta))
    r = v.limit_denominator(max_den)
    if abs(float(r) - float(v)) > 2.0 ** -50 * abs(float(v)):
        raise ValueError("beta must be a rational a/b with b <= %d" % max_den)
    return r


_LAMBDA1_FN = None


def _torch_function():
    global _LAMBDA1_FN
    if _LAMBDA1_FN is not None:
        return _LAMBDA1_FN
    import torch

    class Lambda1(torch.autograd.Function):
        """lambda_1 of the k x k block of H_N^-1 as a float64 tensor of beta.

        forward runs moments -> LDL^T -> Algorithm 4 -> block -> lambda_1 in
        libhk at `bits` bits and also forms d lambda_1 / d beta (the adjoint
        of hk_lambda1_grad, first-order perturbation of the block's top
        eigenvalue); backward multiplies it by the incoming gradient.  beta
        = 1/m needs nothing else (moments exact on the device); beta = a/b
        with a > 1 needs `constants` = {"gamma": (exp, limbs) of Gamma(r/a),
        "psi": (sign, exp, limbs) of psi(r/a)}, r = 1..a-1 (the inputs of
        hk_moments_gamma and hk_set_psi_constants).  The multiprecision
        values stay available through Hankel."""

        @staticmethod
        def forward(ctx, beta, N, k, bits, device=0, constants=None):
            b = _exact_beta(beta.item() if hasattr(beta, "item") else beta)
            if b.numerator > 1 and (not constants or "gamma" not in constants or "psi" not in constants):
                raise ValueError("beta = a/b with a > 1 needs constants={'gamma': ..., 'psi': ...}")
            with Hankel(device) as h:
                if b.numerator == 1:
                    h.moments(b.numerator, b.denominator, N, bits)
                else:
                    h.moments_gamma(b.numerator, b.denominator, N, bits, *constants["gamma"])
                h.ldlt()
                h.inv_block(k)
                lam = h.lambda1(1)
                if b.numerator > 1:
                    h.set_psi_constants(*constants["psi"])
                g = h.lambda1_grad()
            ctx.save_for_backward(torch.tensor(float(g[3][0]), dtype=torch.float64))
            return torch.tensor(float(lam[3][0]), dtype=torch.float64)

        @staticmethod
        def backward(ctx, grad_out):
            (g,) = ctx.saved_tensors
            return grad_out * g.to(grad_out.device), None, None, None, None, None

    _LAMBDA1_FN = Lambda1
    return Lambda1


def lambda1(beta, N, k, bits, device=0, constants=None):
    """Differentiable lambda_1(beta) (torch.autograd); see Lambda1 above."""
    return _torch_function().apply(beta, N, k, bits, device, constants)
