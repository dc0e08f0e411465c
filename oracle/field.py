"""Prime-field operations of the modular arithmetic layer (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

* ``mul``      modmul: a * b mod p (the result Algorithm 2 reaches, canonical)
* ``mont_mul`` the Montgomery product a * b * D^-m mod p, D = 2^32 (Algorithm 2
               with its final comparison read as c >= q)
* ``inv``      modinv, x^(p-2) mod p by Fermat's little theorem (Section 2.2);
               the guard 0^-1 := 0 is this library's convention
* ``batch_inverse``  Montgomery's trick (Section 2.2.1): compress (running
               products), one inversion, decompress (walk back), following the
               paper's three steps; zero elements are skipped and map to 0.

Parity pins (``tests/test_oracle_field.py``): Fermat a^(p-1) = 1, comparison
with Python's built-in ``pow(x, -1, p)`` (extended Euclid, a different
algorithm), brute force over tiny primes, the Montgomery identity against an
explicit long-hand limb loop of Algorithm 2 on tiny limb sizes.
"""


def mul(p, a, b):
    return a * b % p


def add(p, a, b):
    return (a + b) % p


def sub(p, a, b):
    return (a - b) % p


def mont_mul(p, a, b, limbs):
    """Montgomery product with R = 2^(32*limbs)."""
    R = 1 << (32 * limbs)
    return a * b * pow(R, -1, p) % p


def inv(p, x):
    x %= p
    if x == 0:
        return 0
    return pow(x, p - 2, p)


def batch_inverse(p, xs):
    """Montgomery's trick over a list: returns [x^-1 mod p] (0 -> 0)."""
    n = len(xs)
    out = [0] * n
    # compress: prefix[i] = product of the non-zero inputs before i
    prefix = [1] * n
    acc = 1
    for i, x in enumerate(xs):
        prefix[i] = acc
        if x % p:
            acc = acc * x % p
    # inverse step: one modinv of the total product
    acc_inv = inv(p, acc)
    # decompress: walk back, peeling one factor at a time
    for i in range(n - 1, -1, -1):
        x = xs[i] % p
        if x == 0:
            continue
        out[i] = acc_inv * prefix[i] % p
        acc_inv = acc_inv * x % p
    return out
