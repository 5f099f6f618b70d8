"""CPU oracle for the extreme-precision Hankel LDL^T -> lambda_1 path.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
link anything in this package: only ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.
It shares no code with the CUDA library (``paper_1810_01478_gb300/csrc``).

What it computes, in the paper's order and notation (arXiv 1810.01478):

* moments mu_j = Gamma((j+1)/beta)/beta              (Sec. 2, eq. "moments")
* H_N = (mu_{i+j})                                    (Sec. 2, eq. "matrix")
* LDL^T by the right-looking loop of Algorithm 1      (Sec. 4.3)
* the first k columns of L^{-1} by Algorithm 4        (Sec. 4.4)
* (H_N^{-1})_{ab} = sum_l X_la X_lb / D_ll            (Sec. 4.4, eq. "index"; Sec. 4.5)
* eigenvalues of that k x k block, lambda = 1/nu      (Sec. 4.2, Sec. 4.5)
* d lambda_1 / d beta (first-order perturbation of the block eigenvalue)

Number format (shared *definition* with the GPU path, independent code):
a value is ``(m, e)`` meaning m * 2**(32*e) with m a Python int,
2**(32(n-1)) <= |m| < 2**(32 n) (top 32-bit limb non-zero) or m == 0 (then
e == 0).  Every primitive returns the exact result truncated toward zero to
n limbs (``mpfloat.rnd``).  This is the paper's "truncate" rule of Sec. 4.1
carried over from fixed point to a radix-2^32 floating format.

Module map:
  mpfloat   the format and its primitives (rnd, fused a-x*y, div, add, mul)
  moments   mu_j for beta = 1/m (exact integers) and rational beta (mpmath)
  ldlt      Algorithm 1, plus the entry-subset form used for sampled parity
  invblock  Algorithm 4 and the k x k block of H^{-1}
  eigen     eigenvalues of the block (mpmath.eigsy), lambda, truncation error
  grad      analytic d lambda_1/d beta and the central finite difference
  exact     exact-rational (Fraction) LDL^T / inverse for small N and the
            beta = 1 closed forms; used only to pin the truncating oracle
"""
