"""Pins for the oracle's curve constants (not the GPU path).

Each constant is checked against something other than its own transcription:
primality, the closed-form BN / BLS12 parameterisations, OpenSSL's explicit
curve parameters and key derivation, and the group order (n * G = O).
"""
import re
import shutil
import subprocess

import pytest
import sympy

from oracle import curves, ec

ALL = list(curves.BY_ID.values())


@pytest.mark.parametrize("C", ALL, ids=lambda c: c.name)
def test_moduli_prime(C):
    assert sympy.isprime(C.p)
    assert sympy.isprime(C.n)


@pytest.mark.parametrize("C", ALL, ids=lambda c: c.name)
def test_generator_on_curve_and_order(C):
    assert ec.on_curve(C, C.G)
    assert ec.mul(C, C.n, C.G) is None
    assert ec.mul(C, C.n - 1, C.G) == ec.neg(C, C.G)
    # Hasse: |#E - (p + 1)| <= 2 sqrt(p) with #E = h n
    t = C.p + 1 - C.h * C.n
    assert t * t <= 4 * C.p


def test_bit_lengths():
    assert [c.p.bit_length() for c in ALL] == [256, 256, 254, 381, 256]
    assert [c.n.bit_length() for c in ALL] == [256, 256, 254, 255, 256]
    assert [c.limbs for c in ALL] == [8, 8, 8, 12, 8]


def test_special_forms():
    # secp256k1 and P-256 primes in the forms the standards give them
    assert curves.SECP256K1.p == 2**256 - 2**32 - 2**9 - 2**8 - 2**7 - 2**6 - 2**4 - 1
    assert curves.P256.p == 0xFFFFFFFF00000001000000000000000000000000FFFFFFFFFFFFFFFFFFFFFFFF
    # q_inv = -p^-1 mod 2^32 equals 1 for P-256 (Section 2.2 notes this for SCA-256)
    assert (-pow(curves.P256.p, -1, 2**32)) % 2**32 == 1


def test_bn_bls_closed_forms():
    u = curves.BN_U
    bn = curves.BN254
    assert bn.p == 36 * u**4 + 36 * u**3 + 24 * u**2 + 6 * u + 1
    assert bn.n == bn.p + 1 - (6 * u**2 + 1)  # trace t = 6u^2 + 1
    x = curves.BLS_X
    bls = curves.BLS12_381
    assert bls.n == x**4 - x**2 + 1
    assert 3 * (bls.p - x) == (x - 1) ** 2 * bls.n
    assert bls.h * bls.n == bls.p + 1 - (x + 1)  # #E(F_p) = p + 1 - t, t = x + 1
    # G1 of BLS12-381 lies in the order-r subgroup, not merely on the curve
    assert ec.mul(bls, bls.n, bls.G) is None


def _openssl_params(name):
    out = subprocess.run(
        ["openssl", "ecparam", "-name", name, "-param_enc", "explicit", "-text", "-noout"],
        capture_output=True, text=True, check=True,
    ).stdout
    fields = {}
    key = None
    for line in out.splitlines():
        m = re.match(r"^(\w[\w ()]*):\s*(.*)$", line)
        if m:
            key = m.group(1).strip()
            fields[key] = m.group(2).strip()
        elif key:
            fields[key] += line.strip()
    def num(s):
        s = s.split("(")[0].replace(":", "").strip()
        return int(s, 16)
    gen = fields["Generator (uncompressed)"].replace(":", "")
    gen = bytes.fromhex(gen)
    return {
        "p": num(fields["Prime"]), "a": num(fields["A"]), "b": num(fields["B"]),
        "gx": int.from_bytes(gen[1:33], "big"), "gy": int.from_bytes(gen[33:65], "big"),
        "n": num(fields["Order"]),
    }


@pytest.mark.skipif(shutil.which("openssl") is None, reason="openssl binary not available")
@pytest.mark.parametrize("C,name", [(curves.SECP256K1, "secp256k1"), (curves.P256, "prime256v1"),
                                    (curves.SM2, "SM2")])
def test_against_openssl_explicit_params(C, name):
    o = _openssl_params(name)
    assert (o["p"], o["a"], o["b"], o["gx"], o["gy"], o["n"]) == (C.p, C.a, C.b, C.gx, C.gy, C.n)


@pytest.mark.parametrize("C,cname", [(curves.SECP256K1, "SECP256K1"), (curves.P256, "SECP256R1")])
def test_openssl_key_derivation_matches_group_law(C, cname):
    """d * G from OpenSSL equals the oracle's double-and-add for several d."""
    crypto_ec = pytest.importorskip("cryptography.hazmat.primitives.asymmetric.ec")
    curve = getattr(crypto_ec, cname)()
    for d in [1, 2, 3, 0xDEADBEEF, C.n - 1, C.n // 3, 2**200 + 12345]:
        pub = crypto_ec.derive_private_key(d, curve).public_key().public_numbers()
        assert ec.mul(C, d, C.G) == (pub.x, pub.y), d


def test_sm2_prime_form():
    """The SM2 prime is the SCA-256 modulus the paper quotes (Section 4.2)."""
    assert curves.SM2.p == 2**256 - 2**224 - 2**96 + 2**64 - 1
    assert curves.SM2.a == curves.SM2.p - 3
