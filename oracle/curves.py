"""Curve parameters for the oracle (test infrastructure only).

All four curves are short Weierstrass curves y^2 = x^3 + a x + b over F_p
(Eqn 1, Section 2.1).  The paper evaluates only SM2 and prints no constants for
the curves used here except the NIST P-256 prime (in a comment of Section 2.2);
the values below are the published standard parameters, each derived or pinned
by ``tests/test_oracle_curves.py``:

* secp256k1 (SEC 2): p = 2^256 - 2^32 - 977, a = 0, b = 7.
* P-256 (FIPS 186-4 / SEC 2 secp256r1): p = 2^256 - 2^224 + 2^192 + 2^96 - 1, a = -3.
  Both pinned against OpenSSL's explicit parameters and its key derivation.
* BN254 G1: p and r from the BN polynomial in u = 0x44E992B44A6909F1,
  p = 36u^4 + 36u^3 + 24u^2 + 6u + 1, r = 36u^4 + 36u^3 + 18u^2 + 6u + 1,
  b = 3, generator (1, 2).
* BLS12-381 G1: x = -0xd201000000010000, r = x^4 - x^2 + 1,
  p = (x - 1)^2 r / 3 + x, b = 4, the standard G1 generator.
  Pinned by primality, on-curve and r*G = O.

``n`` is the prime order of the generator (for the two pairing curves it is the
scalar-field modulus r).  ``h`` is the cofactor of the full group.
"""
from dataclasses import dataclass


@dataclass(frozen=True)
class Curve:
    name: str
    p: int
    a: int
    b: int
    gx: int
    gy: int
    n: int
    h: int

    @property
    def limbs(self):
        """32-bit limbs needed for a base-field element."""
        return (self.p.bit_length() + 31) // 32

    @property
    def G(self):
        return (self.gx, self.gy)


SECP256K1 = Curve(
    name="secp256k1",
    p=2**256 - 2**32 - 977,
    a=0,
    b=7,
    gx=0x79BE667EF9DCBBAC55A06295CE870B07029BFCDB2DCE28D959F2815B16F81798,
    gy=0x483ADA7726A3C4655DA4FBFC0E1108A8FD17B448A68554199C47D08FFB10D4B8,
    n=0xFFFFFFFFFFFFFFFFFFFFFFFFFFFFFFFEBAAEDCE6AF48A03BBFD25E8CD0364141,
    h=1,
)

_P256_P = 2**256 - 2**224 + 2**192 + 2**96 - 1
P256 = Curve(
    name="P-256",
    p=_P256_P,
    a=_P256_P - 3,
    b=0x5AC635D8AA3A93E7B3EBBD55769886BC651D06B0CC53B0F63BCE3C3E27D2604B,
    gx=0x6B17D1F2E12C4247F8BCE6E563A440F277037D812DEB33A0F4A13945D898C296,
    gy=0x4FE342E2FE1A7F9B8EE7EB4A7C0F9E162BCE33576B315ECECBB6406837BF51F5,
    n=0xFFFFFFFF00000000FFFFFFFFFFFFFFFFBCE6FAADA7179E84F3B9CAC2FC632551,
    h=1,
)

BN_U = 0x44E992B44A6909F1
_BN_P = 36 * BN_U**4 + 36 * BN_U**3 + 24 * BN_U**2 + 6 * BN_U + 1
_BN_R = 36 * BN_U**4 + 36 * BN_U**3 + 18 * BN_U**2 + 6 * BN_U + 1
BN254 = Curve(name="BN254", p=_BN_P, a=0, b=3, gx=1, gy=2, n=_BN_R, h=1)

BLS_X = -0xD201000000010000
_BLS_R = BLS_X**4 - BLS_X**2 + 1
_BLS_P = (BLS_X - 1) ** 2 * _BLS_R // 3 + BLS_X
BLS12_381 = Curve(
    name="BLS12-381",
    p=_BLS_P,
    a=0,
    b=4,
    gx=0x17F1D3A73197D7942695638C4FA9AC0FC3688C4F9774B905A14E3A3F171BAC586C55E83FF97A1AEFFB3AF00ADB22C6BB,
    gy=0x08B3F481E3AAA0F1A09E30ED741D8AE4FCF5E095D5D00AF600DB18CB2C04B3EDD03CC744A2888AE40CAA232946C5E7E1,
    n=_BLS_R,
    h=(BLS_X - 1) ** 2 // 3,
)

_SM2_P = 2**256 - 2**224 - 2**96 + 2**64 - 1
SM2 = Curve(
    name="SM2",
    p=_SM2_P,
    a=_SM2_P - 3,
    b=0x28E9FA9E9D9F5E344D5A9E4BCF6509A7F39789F515AB8F92DDBCBD414D940E93,
    gx=0x32C4AE2C1F1981195F9904466A39C9948FE30BBFF2660BE1715A4589334C74C7,
    gy=0xBC3736A2F4F6779C59BDCEE36B692153D0A9877CC62A474002DF32E52139F0A0,
    n=0xFFFFFFFEFFFFFFFFFFFFFFFFFFFFFFFF7203DF6B21C6052B53BBF40939D54123,
    h=1,
)

# Curve identifiers shared with the C-ABI enumeration (argument values only).
BY_ID = {0: SECP256K1, 1: P256, 2: BN254, 3: BLS12_381, 4: SM2}
BY_NAME = {c.name: c for c in BY_ID.values()}
