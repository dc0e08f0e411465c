"""Pins for the oracle's field layer (Section 2.2, Algorithm 2, Section 2.2.1)."""
import random

import pytest

from oracle import curves, field

MODS = [c.p for c in curves.BY_ID.values()] + [c.n for c in curves.BY_ID.values()]


@pytest.mark.parametrize("p", MODS, ids=lambda p: hex(p)[:10])
def test_inverse_fermat_vs_euclid(p):
    rng = random.Random(p & 0xFFFFF)
    vals = [1, 2, p - 1, p - 2, (1 << 255) % p] + [rng.randrange(1, p) for _ in range(50)]
    for x in vals:
        i = field.inv(p, x)
        assert i == pow(x, -1, p)  # extended Euclid, a different algorithm
        assert x * i % p == 1
        assert pow(x, p - 1, p) == 1
    assert field.inv(p, 0) == 0


def test_batch_inverse_matches_elementwise():
    rng = random.Random(3)
    for p in MODS + [101, 65537]:
        xs = [rng.randrange(p) for _ in range(37)] + [0, 1, p - 1, 0]
        got = field.batch_inverse(p, xs)
        assert got == [pow(x, -1, p) if x % p else 0 for x in xs]
    assert field.batch_inverse(101, []) == []


def _mont_longhand(p, a, b, m):
    """Algorithm 2 written out on 32-bit limbs: full product, then m rows of
    M_i = C_i * q_inv mod D, C += M_i * q * D^i, then one conditional subtract."""
    D = 1 << 32
    qinv = (-pow(p, -1, D)) % D
    A = [(a >> (32 * i)) % D for i in range(m)]
    B = [(b >> (32 * i)) % D for i in range(m)]
    Cl = [0] * (2 * m + 1)
    for i in range(m):
        carry = 0
        for j in range(m):
            t = Cl[i + j] + A[j] * B[i] + carry
            Cl[i + j], carry = t % D, t // D
        Cl[i + m] += carry
    for i in range(m):
        Mi = Cl[i] * qinv % D
        carry = 0
        for j in range(m):
            t = Cl[i + j] + Mi * ((p >> (32 * j)) % D) + carry
            Cl[i + j], carry = t % D, t // D
        k = i + m
        while carry:
            t = Cl[k] + carry
            Cl[k], carry = t % D, t // D
            k += 1
    c = sum(Cl[m + i] << (32 * i) for i in range(m + 1))
    return c - p if c >= p else c


@pytest.mark.parametrize("p", MODS + [101, 2**61 - 1], ids=lambda p: hex(p)[:10])
def test_montgomery_definition(p):
    m = (p.bit_length() + 31) // 32
    rng = random.Random(p % 997)
    R = 1 << (32 * m)
    for _ in range(40):
        a, b = rng.randrange(p), rng.randrange(p)
        c = field.mont_mul(p, a, b, m)
        assert c == _mont_longhand(p, a, b, m)
        assert c * R % p == a * b % p
        assert 0 <= c < p
    # mont(a, R^2 mod p) = a R mod p, mont(aR, 1) = a
    a = rng.randrange(p)
    assert field.mont_mul(p, a, R * R % p, m) == a * R % p
    assert field.mont_mul(p, a * R % p, 1, m) == a


def test_small_field_bruteforce():
    for p in (11, 13, 101):
        for a in range(p):
            for b in range(p):
                assert field.mul(p, a, b) == (a * b) % p
                assert field.add(p, a, b) == (a + b) % p
                assert field.sub(p, a, b) == (a - b) % p
            if a:
                assert [x for x in range(1, p) if a * x % p == 1] == [field.inv(p, a)]
