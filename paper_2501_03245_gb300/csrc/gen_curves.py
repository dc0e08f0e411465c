#!/usr/bin/env python3
"""Writes curves_gen.cuh: compile-time constants of the four curves for the CUDA
library (moduli, Montgomery constants R mod q, R^2 mod q, -q^-1 mod 2^32, q-2,
curve coefficients in Montgomery form, generators).

Run from this directory: ``python gen_curves.py`` (the output is committed).
The parameters are the published standard ones: SEC 2 (secp256k1,
secp256r1 = NIST P-256), the BN254 polynomial in u = 0x44E992B44A6909F1 with
b = 3 and generator (1, 2), and BLS12-381 (x = -0xd201000000010000, b = 4, the
standard G1 generator), and the SM2 recommended curve of GB/T 32918.5.
"""
import os

CURVES = [
    # name, field prime p, a, b, Gx, Gy, group order n
    ("Secp256k1",
     0xFFFFFFFFFFFFFFFFFFFFFFFFFFFFFFFFFFFFFFFFFFFFFFFFFFFFFFFEFFFFFC2F, 0, 7,
     0x79BE667EF9DCBBAC55A06295CE870B07029BFCDB2DCE28D959F2815B16F81798,
     0x483ADA7726A3C4655DA4FBFC0E1108A8FD17B448A68554199C47D08FFB10D4B8,
     0xFFFFFFFFFFFFFFFFFFFFFFFFFFFFFFFEBAAEDCE6AF48A03BBFD25E8CD0364141),
    ("P256",
     0xFFFFFFFF00000001000000000000000000000000FFFFFFFFFFFFFFFFFFFFFFFF, -3,
     0x5AC635D8AA3A93E7B3EBBD55769886BC651D06B0CC53B0F63BCE3C3E27D2604B,
     0x6B17D1F2E12C4247F8BCE6E563A440F277037D812DEB33A0F4A13945D898C296,
     0x4FE342E2FE1A7F9B8EE7EB4A7C0F9E162BCE33576B315ECECBB6406837BF51F5,
     0xFFFFFFFF00000000FFFFFFFFFFFFFFFFBCE6FAADA7179E84F3B9CAC2FC632551),
    ("BN254",
     0x30644E72E131A029B85045B68181585D97816A916871CA8D3C208C16D87CFD47, 0, 3, 1, 2,
     0x30644E72E131A029B85045B68181585D2833E84879B9709143E1F593F0000001),
    ("BLS12_381",
     0x1A0111EA397FE69A4B1BA7B6434BACD764774B84F38512BF6730D2A0F6B0F6241EABFFFEB153FFFFB9FEFFFFFFFFAAAB,
     0, 4,
     0x17F1D3A73197D7942695638C4FA9AC0FC3688C4F9774B905A14E3A3F171BAC586C55E83FF97A1AEFFB3AF00ADB22C6BB,
     0x08B3F481E3AAA0F1A09E30ED741D8AE4FCF5E095D5D00AF600DB18CB2C04B3EDD03CC744A2888AE40CAA232946C5E7E1,
     0x73EDA753299D7D483339D80809A1D80553BDA402FFFE5BFEFFFFFFFF00000001),
    ("SM2",
     0xFFFFFFFEFFFFFFFFFFFFFFFFFFFFFFFFFFFFFFFF00000000FFFFFFFFFFFFFFFF, -3,
     0x28E9FA9E9D9F5E344D5A9E4BCF6509A7F39789F515AB8F92DDBCBD414D940E93,
     0x32C4AE2C1F1981195F9904466A39C9948FE30BBFF2660BE1715A4589334C74C7,
     0xBC3736A2F4F6779C59BDCEE36B692153D0A9877CC62A474002DF32E52139F0A0,
     0xFFFFFFFEFFFFFFFFFFFFFFFFFFFFFFFF7203DF6B21C6052B53BBF40939D54123),
]


# Moduli that also get a second traits class with a reduction of their own
# (fp.cuh, mont_mul): FORM 1 is the NIST P-256 prime 2^256 - 2^224 + 2^192 +
# 2^96 - 1, whose -q^-1 mod 2^32 is 1 and whose limbs are 0, 1 and 2^32 - 1
# only; FORM 2 is the secp256k1 prime 2^256 - 2^32 - 977.  The main traits
# classes are FORM 0 (the generic Montgomery reduction).
SPECIAL = {
    0xFFFFFFFF00000001000000000000000000000000FFFFFFFFFFFFFFFFFFFFFFFF: ("P256FpSpecial", 1),
    (1 << 256) - (1 << 32) - 977: ("Secp256k1FpSpecial", 2),
}


def limbs(v, n):
    return [(v >> (32 * i)) & 0xFFFFFFFF for i in range(n)]


def arr(name, v, n):
    """A constexpr limb accessor: name(i) is limb i (0 outside the range)."""
    cases = " ".join(f"case {i}: return 0x{x:08x}u;" for i, x in enumerate(limbs(v, n)))
    return (f"  ECC_DEV static constexpr uint32_t {name}(int i) {{\n"
            f"    switch (i) {{ {cases} default: return 0u; }}\n  }}\n")


def field(name, q):
    n = (q.bit_length() + 31) // 32
    n += n % 2  # even limb count for the even/odd carry chains
    R = 1 << (32 * n)
    qinv = (-pow(q, -1, 1 << 32)) % (1 << 32)
    s = f"struct {name} {{\n"
    s += f"  static constexpr int N = {n};\n"
    s += f"  static constexpr int BITS = {q.bit_length()};\n"
    s += f"  static constexpr uint32_t QINV = 0x{qinv:08x}u;\n"
    s += "  static constexpr int FORM = 0;\n"
    s += f"  static constexpr uint64_t QINV62 = 0x{pow(q, -1, 1 << 62):016x}ull;  // q^-1 mod 2^62\n"
    s += "  ECC_DEV static constexpr uint32_t qinv() { return QINV; }\n"
    s += "  ECC_DEV static constexpr uint64_t qinv62() { return QINV62; }\n"
    s += arr("p", q, n) + arr("r2", R * R % q, n) + arr("one", R % q, n) + arr("pm2", q - 2, n)
    s += arr("r3", R * R * R % q, n)
    s += "};\n\n"
    if q in SPECIAL:
        sname, form = SPECIAL[q]
        s += f"struct {sname} : {name} {{\n  static constexpr int FORM = {form};\n}};\n\n"
    return s, n, R


def main():
    out = ["// Generated by gen_curves.py; do not edit.\n#pragma once\n#include <cstdint>\n",
           "#ifndef ECC_DEV\n#define ECC_DEV __device__ __forceinline__\n#endif\n\n",
           "namespace ecc {\n\n"]
    for name, p, a, b, gx, gy, n in CURVES:
        fs, N, R = field(f"{name}Fp", p)
        ns, NN, RN = field(f"{name}Fn", n)
        out.append(fs)
        out.append(ns)
        a %= p
        s = f"struct {name} {{\n"
        s += f"  using Fp = {name}Fp;\n  using Fn = {name}Fn;\n"
        s += f"  static constexpr bool A_ZERO = {'true' if a == 0 else 'false'};\n"
        s += arr("a", a * R % p, N) + arr("b", b * R % p, N)
        s += arr("gx", gx, N) + arr("gy", gy, N)
        s += arr("n", n, 8)
        s += f"  static constexpr int SCALAR_BITS = {n.bit_length()};\n"
        s += "};\n\n"
        out.append(s)
    out.append("}  // namespace ecc\n")
    here = os.path.dirname(os.path.abspath(__file__))
    with open(os.path.join(here, "curves_gen.cuh"), "w") as f:
        f.write("".join(out))


if __name__ == "__main__":
    main()
