"""Writes euler_gamma.inc: Euler's constant gamma truncated to GAMMA_LIMBS
32-bit limbs below the radix point (floor(gamma * 2^(32*GAMMA_LIMBS))).

The gradient of lambda_1 needs psi(x) = H_{x-1} - gamma at integer x (the
digamma function of the moments' Gamma((j+1)/beta), beta = 1/m).  gamma is
computed here with the Brent-McMillan formula (Brent & McMillan, Math. Comp.
34 (1980), algorithm B1) in Python fixed-point integers:
    gamma = U/V,  U = sum A_k, V = sum B_k,
    B_0 = 1, A_0 = -log(a), B_k = B_{k-1} a^2/k^2, A_k = (A_{k-1} a^2/k + B_k)/k,
with a = 2^13 (error ~ exp(-4a)), and log 2 = sum_k 1/(k 2^k).
Run: python gen_euler_gamma.py  (writes the .inc beside it).
"""
import os

GAMMA_LIMBS = 1040          # 33280 bits: covers every compiled width (<= 1024 limbs)
GUARD = 256


def log2_fixed(bits):
    one = 1 << bits
    s, k, p = 0, 1, one >> 1
    while p:
        s += p // k
        k += 1
        p >>= 1
    return s


def tdiv(x, y):
    """Integer division truncating toward zero (so negative terms reach 0)."""
    return -((-x) // y) if x < 0 else x // y


def euler_gamma_fixed(bits):
    w = bits + GUARD
    one = 1 << w
    e = 13
    a = 1 << e
    loga = e * log2_fixed(w)
    A = -loga
    B = one
    U, V = A, B
    a2 = a * a
    k = 1
    while True:
        B = B * a2 // (k * k)
        A = tdiv(tdiv(A * a2, k) + B, k)
        if B == 0 and A == 0:
            break
        U += A
        V += B
        k += 1
    g = (U << w) // V
    return g >> GUARD


def main():
    bits = 32 * GAMMA_LIMBS
    g = euler_gamma_fixed(bits)
    limbs = [(g >> (32 * i)) & 0xFFFFFFFF for i in range(GAMMA_LIMBS)]
    here = os.path.dirname(os.path.abspath(__file__))
    with open(os.path.join(here, "euler_gamma.inc"), "w") as f:
        f.write("// generated by gen_euler_gamma.py: floor(gamma * 2^(32*%d)), little-endian limbs\n" % GAMMA_LIMBS)
        f.write("#define HK_GAMMA_LIMBS %d\n" % GAMMA_LIMBS)
        f.write("static const uint32_t hk_euler_gamma[HK_GAMMA_LIMBS] = {\n")
        for i in range(0, GAMMA_LIMBS, 8):
            f.write("  " + ", ".join("0x%08xu" % v for v in limbs[i:i + 8]) + ",\n")
        f.write("};\n")


if __name__ == "__main__":
    main()
