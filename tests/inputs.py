"""Seeded synthetic inputs shared by the oracle tests and the GPU parity tests.

Holds none of the method's arithmetic: it only draws operands in the number
layout (sign, limb exponent, n-limb mantissa with a non-zero top limb) and
exact integer moment sequences.  Expected values always come from ``oracle``.

Recipes
* ``fused_operands``: triples (a, x, y) for a - x*y.  Mantissas are uniform
  random n-limb integers, or "structured" ones (all-ones limbs, a single set
  bit, trailing zero limbs).  Exponents are chosen so that the product and a
  overlap closely (the common case of the factorisation, including near-total
  cancellation where a is the product's leading limbs), or sit far apart
  (gaps of up to 4n limbs either way), or one operand is zero.
* ``digit_extreme_mant``: the mantissa whose 7-bit groups are 64, 63, 63, ...
  (top limb made non-zero): its balanced 7-bit digits are all -64, the
  largest digit magnitudes a tensor-core product meets.
* ``measure_moments``: mu_j = sum_m w_m t_m^j for a random discrete positive
  measure (integer weights w_m, distinct integer nodes t_m >= 1): the Hankel
  matrix of such moments is exactly positive definite while N <= #atoms.
"""
import random

MASK = 0xFFFFFFFF


def rand_mant(rng, n, kind="uniform"):
    if kind == "uniform":
        m = rng.getrandbits(32 * n)
        return m | (rng.randint(1, MASK) << (32 * (n - 1)))
    if kind == "ones":
        return (1 << (32 * n)) - 1
    if kind == "pow2":
        return 1 << (32 * (n - 1) + rng.randint(0, 31))
    if kind == "sparse":  # trailing zero limbs
        keep = rng.randint(1, n)
        m = rng.getrandbits(32 * keep) | (1 << (32 * keep - 1))
        return m << (32 * (n - keep))
    if kind == "topones":  # top limbs all ones, rest random
        t = rng.randint(1, n)
        m = rng.getrandbits(32 * n)
        return m | (((1 << (32 * t)) - 1) << (32 * (n - t)))
    raise ValueError(kind)


def digit_extreme_mant(n):
    m = 64 | sum(63 << (7 * k) for k in range(1, (32 * n) // 7 + 1))
    m &= (1 << (32 * n)) - 1
    return m | (1 << (32 * n - 1))


def rand_num(rng, n, e_lo=-8, e_hi=8, kinds=("uniform",)):
    m = rand_mant(rng, n, rng.choice(kinds))
    return (-m if rng.random() < 0.5 else m, rng.randint(e_lo, e_hi))


KINDS = ("uniform", "uniform", "uniform", "ones", "pow2", "sparse", "topones")


def fused_operands(rng, n, count):
    out = []
    for t in range(count):
        x = rand_num(rng, n, kinds=KINDS)
        y = rand_num(rng, n, kinds=KINDS)
        pm, pe = x[0] * y[0], x[1] + y[1]
        mode = t % 6
        if mode == 0:     # a near the product's magnitude
            a = rand_num(rng, n, kinds=KINDS)
            plimbs = (abs(pm).bit_length() + 31) // 32
            a = (a[0], pe + plimbs - n + rng.randint(-2, 2))
        elif mode == 1:   # a = leading limbs of the product (deep cancellation)
            p = abs(pm)
            plimbs = (p.bit_length() + 31) // 32
            m = p >> (32 * (plimbs - n))
            m ^= rng.choice([0, 0, 1, rng.getrandbits(16)])
            m |= 1 << (32 * n - 1) if m.bit_length() <= 32 * (n - 1) else 0
            sgn = 1 if (pm > 0) else -1
            a = (sgn * m, pe + plimbs - n)
        elif mode == 2:   # far apart either way
            a = rand_num(rng, n, kinds=KINDS)
            a = (a[0], pe + rng.choice([-1, 1]) * rng.randint(n, 4 * n + 3))
        elif mode == 3:   # zero operands
            a = rand_num(rng, n, kinds=KINDS)
            which = rng.randint(0, 2)
            if which == 0:
                a = (0, 0)
            elif which == 1:
                x = (0, 0)
            else:
                y = (0, 0)
        else:             # anything in a moderate window
            a = rand_num(rng, n, e_lo=pe - 3 * n, e_hi=pe + 3 * n, kinds=KINDS)
        out.append((a, x, y))
    return out


def measure_moments(seed, N, atoms=None, w_bits=20, t_max=None):
    """Exact integer moments mu_0..mu_{2N-2} of a random positive measure."""
    rng = random.Random(seed)
    atoms = atoms or N + 2
    t_max = t_max or 8 * atoms
    nodes = rng.sample(range(1, t_max + 1), atoms)
    weights = [rng.randint(1, 1 << w_bits) for _ in range(atoms)]
    return [sum(w * t ** j for w, t in zip(weights, nodes)) for j in range(2 * N - 1)]


def near_degenerate_moments(d):
    """mu_0..mu_4 of the measure with weights 10^6, 2 10^6, 12 10^6 + d,
    2 10^6, 10^6 at the nodes -2, -1, 0, 1, 2.  For N = 3 its Hankel matrix
    has eigenvalues 12 10^6 (twice) and 42 10^6 when d = 0 (the odd moments
    vanish, so e_2 is an eigenvector with eigenvalue mu_2, and
    (mu_0 - mu_2)(mu_4 - mu_2) = mu_2^2 puts mu_2 in the spectrum of the outer
    2 x 2 block too); d > 0 splits the pair (d = 1: relative gap 7e-8;
    d = 24: 1.6e-6)."""
    nodes = (-2, -1, 0, 1, 2)
    weights = (10 ** 6, 2 * 10 ** 6, 12 * 10 ** 6 + d, 2 * 10 ** 6, 10 ** 6)
    return [sum(w * t ** j for w, t in zip(weights, nodes)) for j in range(5)]
