// Generated by gen_curves.py; do not edit.
#pragma once
#include <cstdint>
#ifndef ECC_DEV
#define ECC_DEV __device__ __forceinline__
#endif

namespace ecc {

struct Secp256k1Fp {
  static constexpr int N = 8;
  static constexpr int BITS = 256;
  static constexpr uint32_t QINV = 0xd2253531u;
  static constexpr int FORM = 0;
  static constexpr uint64_t QINV62 = 0x27c7f6e22ddacacfull;  // q^-1 mod 2^62
  ECC_DEV static constexpr uint32_t qinv() { return QINV; }
  ECC_DEV static constexpr uint64_t qinv62() { return QINV62; }
  ECC_DEV static constexpr uint32_t p(int i) {
    switch (i) { case 0: return 0xfffffc2fu; case 1: return 0xfffffffeu; case 2: return 0xffffffffu; case 3: return 0xffffffffu; case 4: return 0xffffffffu; case 5: return 0xffffffffu; case 6: return 0xffffffffu; case 7: return 0xffffffffu; default: return 0u; }
  }
  ECC_DEV static constexpr uint32_t r2(int i) {
    switch (i) { case 0: return 0x000e90a1u; case 1: return 0x000007a2u; case 2: return 0x00000001u; case 3: return 0x00000000u; case 4: return 0x00000000u; case 5: return 0x00000000u; case 6: return 0x00000000u; case 7: return 0x00000000u; default: return 0u; }
  }
  ECC_DEV static constexpr uint32_t one(int i) {
    switch (i) { case 0: return 0x000003d1u; case 1: return 0x00000001u; case 2: return 0x00000000u; case 3: return 0x00000000u; case 4: return 0x00000000u; case 5: return 0x00000000u; case 6: return 0x00000000u; case 7: return 0x00000000u; default: return 0u; }
  }
  ECC_DEV static constexpr uint32_t pm2(int i) {
    switch (i) { case 0: return 0xfffffc2du; case 1: return 0xfffffffeu; case 2: return 0xffffffffu; case 3: return 0xffffffffu; case 4: return 0xffffffffu; case 5: return 0xffffffffu; case 6: return 0xffffffffu; case 7: return 0xffffffffu; default: return 0u; }
  }
  ECC_DEV static constexpr uint32_t r3(int i) {
    switch (i) { case 0: return 0x3795f671u; case 1: return 0x002bb1e3u; case 2: return 0x00000b73u; case 3: return 0x00000001u; case 4: return 0x00000000u; case 5: return 0x00000000u; case 6: return 0x00000000u; case 7: return 0x00000000u; default: return 0u; }
  }
};

struct Secp256k1FpSpecial : Secp256k1Fp {
  static constexpr int FORM = 2;
};

struct Secp256k1Fn {
  static constexpr int N = 8;
  static constexpr int BITS = 256;
  static constexpr uint32_t QINV = 0x5588b13fu;
  static constexpr int FORM = 0;
  static constexpr uint64_t QINV62 = 0x34f20099aa774ec1ull;  // q^-1 mod 2^62
  ECC_DEV static constexpr uint32_t qinv() { return QINV; }
  ECC_DEV static constexpr uint64_t qinv62() { return QINV62; }
  ECC_DEV static constexpr uint32_t p(int i) {
    switch (i) { case 0: return 0xd0364141u; case 1: return 0xbfd25e8cu; case 2: return 0xaf48a03bu; case 3: return 0xbaaedce6u; case 4: return 0xfffffffeu; case 5: return 0xffffffffu; case 6: return 0xffffffffu; case 7: return 0xffffffffu; default: return 0u; }
  }
  ECC_DEV static constexpr uint32_t r2(int i) {
    switch (i) { case 0: return 0x67d7d140u; case 1: return 0x896cf214u; case 2: return 0x0e7cf878u; case 3: return 0x741496c2u; case 4: return 0x5bcd07c6u; case 5: return 0xe697f5e4u; case 6: return 0x81c69bc5u; case 7: return 0x9d671cd5u; default: return 0u; }
  }
  ECC_DEV static constexpr uint32_t one(int i) {
    switch (i) { case 0: return 0x2fc9bebfu; case 1: return 0x402da173u; case 2: return 0x50b75fc4u; case 3: return 0x45512319u; case 4: return 0x00000001u; case 5: return 0x00000000u; case 6: return 0x00000000u; case 7: return 0x00000000u; default: return 0u; }
  }
  ECC_DEV static constexpr uint32_t pm2(int i) {
    switch (i) { case 0: return 0xd036413fu; case 1: return 0xbfd25e8cu; case 2: return 0xaf48a03bu; case 3: return 0xbaaedce6u; case 4: return 0xfffffffeu; case 5: return 0xffffffffu; case 6: return 0xffffffffu; case 7: return 0xffffffffu; default: return 0u; }
  }
  ECC_DEV static constexpr uint32_t r3(int i) {
    switch (i) { case 0: return 0xe9ff41edu; case 1: return 0x7bc0cfe0u; case 2: return 0x44d4322cu; case 3: return 0x00176484u; case 4: return 0xf1d0b2dau; case 5: return 0xb1b31347u; case 6: return 0x18ef116du; case 7: return 0x555d800cu; default: return 0u; }
  }
};

struct Secp256k1 {
  using Fp = Secp256k1Fp;
  using Fn = Secp256k1Fn;
  static constexpr bool A_ZERO = true;
  ECC_DEV static constexpr uint32_t a(int i) {
    switch (i) { case 0: return 0x00000000u; case 1: return 0x00000000u; case 2: return 0x00000000u; case 3: return 0x00000000u; case 4: return 0x00000000u; case 5: return 0x00000000u; case 6: return 0x00000000u; case 7: return 0x00000000u; default: return 0u; }
  }
  ECC_DEV static constexpr uint32_t b(int i) {
    switch (i) { case 0: return 0x00001ab7u; case 1: return 0x00000007u; case 2: return 0x00000000u; case 3: return 0x00000000u; case 4: return 0x00000000u; case 5: return 0x00000000u; case 6: return 0x00000000u; case 7: return 0x00000000u; default: return 0u; }
  }
  ECC_DEV static constexpr uint32_t gx(int i) {
    switch (i) { case 0: return 0x16f81798u; case 1: return 0x59f2815bu; case 2: return 0x2dce28d9u; case 3: return 0x029bfcdbu; case 4: return 0xce870b07u; case 5: return 0x55a06295u; case 6: return 0xf9dcbbacu; case 7: return 0x79be667eu; default: return 0u; }
  }
  ECC_DEV static constexpr uint32_t gy(int i) {
    switch (i) { case 0: return 0xfb10d4b8u; case 1: return 0x9c47d08fu; case 2: return 0xa6855419u; case 3: return 0xfd17b448u; case 4: return 0x0e1108a8u; case 5: return 0x5da4fbfcu; case 6: return 0x26a3c465u; case 7: return 0x483ada77u; default: return 0u; }
  }
  ECC_DEV static constexpr uint32_t n(int i) {
    switch (i) { case 0: return 0xd0364141u; case 1: return 0xbfd25e8cu; case 2: return 0xaf48a03bu; case 3: return 0xbaaedce6u; case 4: return 0xfffffffeu; case 5: return 0xffffffffu; case 6: return 0xffffffffu; case 7: return 0xffffffffu; default: return 0u; }
  }
  static constexpr int SCALAR_BITS = 256;
};

struct P256Fp {
  static constexpr int N = 8;
  static constexpr int BITS = 256;
  static constexpr uint32_t QINV = 0x00000001u;
  static constexpr int FORM = 0;
  static constexpr uint64_t QINV62 = 0x3fffffffffffffffull;  // q^-1 mod 2^62
  ECC_DEV static constexpr uint32_t qinv() { return QINV; }
  ECC_DEV static constexpr uint64_t qinv62() { return QINV62; }
  ECC_DEV static constexpr uint32_t p(int i) {
    switch (i) { case 0: return 0xffffffffu; case 1: return 0xffffffffu; case 2: return 0xffffffffu; case 3: return 0x00000000u; case 4: return 0x00000000u; case 5: return 0x00000000u; case 6: return 0x00000001u; case 7: return 0xffffffffu; default: return 0u; }
  }
  ECC_DEV static constexpr uint32_t r2(int i) {
    switch (i) { case 0: return 0x00000003u; case 1: return 0x00000000u; case 2: return 0xffffffffu; case 3: return 0xfffffffbu; case 4: return 0xfffffffeu; case 5: return 0xffffffffu; case 6: return 0xfffffffdu; case 7: return 0x00000004u; default: return 0u; }
  }
  ECC_DEV static constexpr uint32_t one(int i) {
    switch (i) { case 0: return 0x00000001u; case 1: return 0x00000000u; case 2: return 0x00000000u; case 3: return 0xffffffffu; case 4: return 0xffffffffu; case 5: return 0xffffffffu; case 6: return 0xfffffffeu; case 7: return 0x00000000u; default: return 0u; }
  }
  ECC_DEV static constexpr uint32_t pm2(int i) {
    switch (i) { case 0: return 0xfffffffdu; case 1: return 0xffffffffu; case 2: return 0xffffffffu; case 3: return 0x00000000u; case 4: return 0x00000000u; case 5: return 0x00000000u; case 6: return 0x00000001u; case 7: return 0xffffffffu; default: return 0u; }
  }
  ECC_DEV static constexpr uint32_t r3(int i) {
    switch (i) { case 0: return 0x0000000au; case 1: return 0xfffffffdu; case 2: return 0xfffffff7u; case 3: return 0xffffffedu; case 4: return 0xfffffffcu; case 5: return 0x00000005u; case 6: return 0x00000001u; case 7: return 0x00000018u; default: return 0u; }
  }
};

struct P256FpSpecial : P256Fp {
  static constexpr int FORM = 1;
};

struct P256Fn {
  static constexpr int N = 8;
  static constexpr int BITS = 256;
  static constexpr uint32_t QINV = 0xee00bc4fu;
  static constexpr int FORM = 0;
  static constexpr uint64_t QINV62 = 0x332e375511ff43b1ull;  // q^-1 mod 2^62
  ECC_DEV static constexpr uint32_t qinv() { return QINV; }
  ECC_DEV static constexpr uint64_t qinv62() { return QINV62; }
  ECC_DEV static constexpr uint32_t p(int i) {
    switch (i) { case 0: return 0xfc632551u; case 1: return 0xf3b9cac2u; case 2: return 0xa7179e84u; case 3: return 0xbce6faadu; case 4: return 0xffffffffu; case 5: return 0xffffffffu; case 6: return 0x00000000u; case 7: return 0xffffffffu; default: return 0u; }
  }
  ECC_DEV static constexpr uint32_t r2(int i) {
    switch (i) { case 0: return 0xbe79eea2u; case 1: return 0x83244c95u; case 2: return 0x49bd6fa6u; case 3: return 0x4699799cu; case 4: return 0x2b6bec59u; case 5: return 0x2845b239u; case 6: return 0xf3d95620u; case 7: return 0x66e12d94u; default: return 0u; }
  }
  ECC_DEV static constexpr uint32_t one(int i) {
    switch (i) { case 0: return 0x039cdaafu; case 1: return 0x0c46353du; case 2: return 0x58e8617bu; case 3: return 0x43190552u; case 4: return 0x00000000u; case 5: return 0x00000000u; case 6: return 0xffffffffu; case 7: return 0x00000000u; default: return 0u; }
  }
  ECC_DEV static constexpr uint32_t pm2(int i) {
    switch (i) { case 0: return 0xfc63254fu; case 1: return 0xf3b9cac2u; case 2: return 0xa7179e84u; case 3: return 0xbce6faadu; case 4: return 0xffffffffu; case 5: return 0xffffffffu; case 6: return 0x00000000u; case 7: return 0xffffffffu; default: return 0u; }
  }
  ECC_DEV static constexpr uint32_t r3(int i) {
    switch (i) { case 0: return 0x0b65a624u; case 1: return 0xac8ebec9u; case 2: return 0x0c0555c9u; case 3: return 0x111f28aeu; case 4: return 0x6ba5e93fu; case 5: return 0x2543b924u; case 6: return 0x6407be65u; case 7: return 0x503a54e7u; default: return 0u; }
  }
};

struct P256 {
  using Fp = P256Fp;
  using Fn = P256Fn;
  static constexpr bool A_ZERO = false;
  ECC_DEV static constexpr uint32_t a(int i) {
    switch (i) { case 0: return 0xfffffffcu; case 1: return 0xffffffffu; case 2: return 0xffffffffu; case 3: return 0x00000003u; case 4: return 0x00000000u; case 5: return 0x00000000u; case 6: return 0x00000004u; case 7: return 0xfffffffcu; default: return 0u; }
  }
  ECC_DEV static constexpr uint32_t b(int i) {
    switch (i) { case 0: return 0x29c4bddfu; case 1: return 0xd89cdf62u; case 2: return 0x78843090u; case 3: return 0xacf005cdu; case 4: return 0xf7212ed6u; case 5: return 0xe5a220abu; case 6: return 0x04874834u; case 7: return 0xdc30061du; default: return 0u; }
  }
  ECC_DEV static constexpr uint32_t gx(int i) {
    switch (i) { case 0: return 0xd898c296u; case 1: return 0xf4a13945u; case 2: return 0x2deb33a0u; case 3: return 0x77037d81u; case 4: return 0x63a440f2u; case 5: return 0xf8bce6e5u; case 6: return 0xe12c4247u; case 7: return 0x6b17d1f2u; default: return 0u; }
  }
  ECC_DEV static constexpr uint32_t gy(int i) {
    switch (i) { case 0: return 0x37bf51f5u; case 1: return 0xcbb64068u; case 2: return 0x6b315eceu; case 3: return 0x2bce3357u; case 4: return 0x7c0f9e16u; case 5: return 0x8ee7eb4au; case 6: return 0xfe1a7f9bu; case 7: return 0x4fe342e2u; default: return 0u; }
  }
  ECC_DEV static constexpr uint32_t n(int i) {
    switch (i) { case 0: return 0xfc632551u; case 1: return 0xf3b9cac2u; case 2: return 0xa7179e84u; case 3: return 0xbce6faadu; case 4: return 0xffffffffu; case 5: return 0xffffffffu; case 6: return 0x00000000u; case 7: return 0xffffffffu; default: return 0u; }
  }
  static constexpr int SCALAR_BITS = 256;
};

struct BN254Fp {
  static constexpr int N = 8;
  static constexpr int BITS = 254;
  static constexpr uint32_t QINV = 0xe4866389u;
  static constexpr int FORM = 0;
  static constexpr uint64_t QINV62 = 0x382df87d1b799c77ull;  // q^-1 mod 2^62
  ECC_DEV static constexpr uint32_t qinv() { return QINV; }
  ECC_DEV static constexpr uint64_t qinv62() { return QINV62; }
  ECC_DEV static constexpr uint32_t p(int i) {
    switch (i) { case 0: return 0xd87cfd47u; case 1: return 0x3c208c16u; case 2: return 0x6871ca8du; case 3: return 0x97816a91u; case 4: return 0x8181585du; case 5: return 0xb85045b6u; case 6: return 0xe131a029u; case 7: return 0x30644e72u; default: return 0u; }
  }
  ECC_DEV static constexpr uint32_t r2(int i) {
    switch (i) { case 0: return 0x538afa89u; case 1: return 0xf32cfc5bu; case 2: return 0xd44501fbu; case 3: return 0xb5e71911u; case 4: return 0x0a417ff6u; case 5: return 0x47ab1effu; case 6: return 0xcab8351fu; case 7: return 0x06d89f71u; default: return 0u; }
  }
  ECC_DEV static constexpr uint32_t one(int i) {
    switch (i) { case 0: return 0xc58f0d9du; case 1: return 0xd35d438du; case 2: return 0xf5c70b3du; case 3: return 0x0a78eb28u; case 4: return 0x7879462cu; case 5: return 0x666ea36fu; case 6: return 0x9a07df2fu; case 7: return 0x0e0a77c1u; default: return 0u; }
  }
  ECC_DEV static constexpr uint32_t pm2(int i) {
    switch (i) { case 0: return 0xd87cfd45u; case 1: return 0x3c208c16u; case 2: return 0x6871ca8du; case 3: return 0x97816a91u; case 4: return 0x8181585du; case 5: return 0xb85045b6u; case 6: return 0xe131a029u; case 7: return 0x30644e72u; default: return 0u; }
  }
  ECC_DEV static constexpr uint32_t r3(int i) {
    switch (i) { case 0: return 0xda1530dfu; case 1: return 0xb1cd6dafu; case 2: return 0xa7283db6u; case 3: return 0x62f210e6u; case 4: return 0x0ada0afbu; case 5: return 0xef7f0b0cu; case 6: return 0x2d592544u; case 7: return 0x20fd6e90u; default: return 0u; }
  }
};

struct BN254Fn {
  static constexpr int N = 8;
  static constexpr int BITS = 254;
  static constexpr uint32_t QINV = 0xefffffffu;
  static constexpr int FORM = 0;
  static constexpr uint64_t QINV62 = 0x3d1e0a6c10000001ull;  // q^-1 mod 2^62
  ECC_DEV static constexpr uint32_t qinv() { return QINV; }
  ECC_DEV static constexpr uint64_t qinv62() { return QINV62; }
  ECC_DEV static constexpr uint32_t p(int i) {
    switch (i) { case 0: return 0xf0000001u; case 1: return 0x43e1f593u; case 2: return 0x79b97091u; case 3: return 0x2833e848u; case 4: return 0x8181585du; case 5: return 0xb85045b6u; case 6: return 0xe131a029u; case 7: return 0x30644e72u; default: return 0u; }
  }
  ECC_DEV static constexpr uint32_t r2(int i) {
    switch (i) { case 0: return 0xae216da7u; case 1: return 0x1bb8e645u; case 2: return 0xe35c59e3u; case 3: return 0x53fe3ab1u; case 4: return 0x53bb8085u; case 5: return 0x8c49833du; case 6: return 0x7f4e44a5u; case 7: return 0x0216d0b1u; default: return 0u; }
  }
  ECC_DEV static constexpr uint32_t one(int i) {
    switch (i) { case 0: return 0x4ffffffbu; case 1: return 0xac96341cu; case 2: return 0x9f60cd29u; case 3: return 0x36fc7695u; case 4: return 0x7879462eu; case 5: return 0x666ea36fu; case 6: return 0x9a07df2fu; case 7: return 0x0e0a77c1u; default: return 0u; }
  }
  ECC_DEV static constexpr uint32_t pm2(int i) {
    switch (i) { case 0: return 0xefffffffu; case 1: return 0x43e1f593u; case 2: return 0x79b97091u; case 3: return 0x2833e848u; case 4: return 0x8181585du; case 5: return 0xb85045b6u; case 6: return 0xe131a029u; case 7: return 0x30644e72u; default: return 0u; }
  }
  ECC_DEV static constexpr uint32_t r3(int i) {
    switch (i) { case 0: return 0xb4bf0040u; case 1: return 0x5e94d8e1u; case 2: return 0x1cfbb6b8u; case 3: return 0x2a489cbeu; case 4: return 0xa19fcfedu; case 5: return 0x893cc664u; case 6: return 0x7fcc657cu; case 7: return 0x0cf8594bu; default: return 0u; }
  }
};

struct BN254 {
  using Fp = BN254Fp;
  using Fn = BN254Fn;
  static constexpr bool A_ZERO = true;
  ECC_DEV static constexpr uint32_t a(int i) {
    switch (i) { case 0: return 0x00000000u; case 1: return 0x00000000u; case 2: return 0x00000000u; case 3: return 0x00000000u; case 4: return 0x00000000u; case 5: return 0x00000000u; case 6: return 0x00000000u; case 7: return 0x00000000u; default: return 0u; }
  }
  ECC_DEV static constexpr uint32_t b(int i) {
    switch (i) { case 0: return 0x50ad28d7u; case 1: return 0x7a17caa9u; case 2: return 0xe15521b9u; case 3: return 0x1f6ac17au; case 4: return 0x696bd284u; case 5: return 0x334bea4eu; case 6: return 0xce179d8eu; case 7: return 0x2a1f6744u; default: return 0u; }
  }
  ECC_DEV static constexpr uint32_t gx(int i) {
    switch (i) { case 0: return 0x00000001u; case 1: return 0x00000000u; case 2: return 0x00000000u; case 3: return 0x00000000u; case 4: return 0x00000000u; case 5: return 0x00000000u; case 6: return 0x00000000u; case 7: return 0x00000000u; default: return 0u; }
  }
  ECC_DEV static constexpr uint32_t gy(int i) {
    switch (i) { case 0: return 0x00000002u; case 1: return 0x00000000u; case 2: return 0x00000000u; case 3: return 0x00000000u; case 4: return 0x00000000u; case 5: return 0x00000000u; case 6: return 0x00000000u; case 7: return 0x00000000u; default: return 0u; }
  }
  ECC_DEV static constexpr uint32_t n(int i) {
    switch (i) { case 0: return 0xf0000001u; case 1: return 0x43e1f593u; case 2: return 0x79b97091u; case 3: return 0x2833e848u; case 4: return 0x8181585du; case 5: return 0xb85045b6u; case 6: return 0xe131a029u; case 7: return 0x30644e72u; default: return 0u; }
  }
  static constexpr int SCALAR_BITS = 254;
};

struct BLS12_381Fp {
  static constexpr int N = 12;
  static constexpr int BITS = 381;
  static constexpr uint32_t QINV = 0xfffcfffdu;
  static constexpr int FORM = 0;
  static constexpr uint64_t QINV62 = 0x360c000300030003ull;  // q^-1 mod 2^62
  ECC_DEV static constexpr uint32_t qinv() { return QINV; }
  ECC_DEV static constexpr uint64_t qinv62() { return QINV62; }
  ECC_DEV static constexpr uint32_t p(int i) {
    switch (i) { case 0: return 0xffffaaabu; case 1: return 0xb9feffffu; case 2: return 0xb153ffffu; case 3: return 0x1eabfffeu; case 4: return 0xf6b0f624u; case 5: return 0x6730d2a0u; case 6: return 0xf38512bfu; case 7: return 0x64774b84u; case 8: return 0x434bacd7u; case 9: return 0x4b1ba7b6u; case 10: return 0x397fe69au; case 11: return 0x1a0111eau; default: return 0u; }
  }
  ECC_DEV static constexpr uint32_t r2(int i) {
    switch (i) { case 0: return 0x1c341746u; case 1: return 0xf4df1f34u; case 2: return 0x09d104f1u; case 3: return 0x0a76e6a6u; case 4: return 0x4c95b6d5u; case 5: return 0x8de5476cu; case 6: return 0x939d83c0u; case 7: return 0x67eb88a9u; case 8: return 0xb519952du; case 9: return 0x9a793e85u; case 10: return 0x92cae3aau; case 11: return 0x11988fe5u; default: return 0u; }
  }
  ECC_DEV static constexpr uint32_t one(int i) {
    switch (i) { case 0: return 0x0002fffdu; case 1: return 0x76090000u; case 2: return 0xc40c0002u; case 3: return 0xebf4000bu; case 4: return 0x53c758bau; case 5: return 0x5f489857u; case 6: return 0x70525745u; case 7: return 0x77ce5853u; case 8: return 0xa256ec6du; case 9: return 0x5c071a97u; case 10: return 0xfa80e493u; case 11: return 0x15f65ec3u; default: return 0u; }
  }
  ECC_DEV static constexpr uint32_t pm2(int i) {
    switch (i) { case 0: return 0xffffaaa9u; case 1: return 0xb9feffffu; case 2: return 0xb153ffffu; case 3: return 0x1eabfffeu; case 4: return 0xf6b0f624u; case 5: return 0x6730d2a0u; case 6: return 0xf38512bfu; case 7: return 0x64774b84u; case 8: return 0x434bacd7u; case 9: return 0x4b1ba7b6u; case 10: return 0x397fe69au; case 11: return 0x1a0111eau; default: return 0u; }
  }
  ECC_DEV static constexpr uint32_t r3(int i) {
    switch (i) { case 0: return 0xd94ca1e0u; case 1: return 0xed48ac6bu; case 2: return 0x03a7adf8u; case 3: return 0x315f831eu; case 4: return 0x615e29ddu; case 5: return 0x9a53352au; case 6: return 0x921e1761u; case 7: return 0x34c04e5eu; case 8: return 0x65724728u; case 9: return 0x2512d435u; case 10: return 0x91755d4du; case 11: return 0x0aa63460u; default: return 0u; }
  }
};

struct BLS12_381Fn {
  static constexpr int N = 8;
  static constexpr int BITS = 255;
  static constexpr uint32_t QINV = 0xffffffffu;
  static constexpr int FORM = 0;
  static constexpr uint64_t QINV62 = 0x0000000100000001ull;  // q^-1 mod 2^62
  ECC_DEV static constexpr uint32_t qinv() { return QINV; }
  ECC_DEV static constexpr uint64_t qinv62() { return QINV62; }
  ECC_DEV static constexpr uint32_t p(int i) {
    switch (i) { case 0: return 0x00000001u; case 1: return 0xffffffffu; case 2: return 0xfffe5bfeu; case 3: return 0x53bda402u; case 4: return 0x09a1d805u; case 5: return 0x3339d808u; case 6: return 0x299d7d48u; case 7: return 0x73eda753u; default: return 0u; }
  }
  ECC_DEV static constexpr uint32_t r2(int i) {
    switch (i) { case 0: return 0xf3f29c6du; case 1: return 0xc999e990u; case 2: return 0x87925c23u; case 3: return 0x2b6cedcbu; case 4: return 0x7254398fu; case 5: return 0x05d31496u; case 6: return 0x9f59ff11u; case 7: return 0x0748d9d9u; default: return 0u; }
  }
  ECC_DEV static constexpr uint32_t one(int i) {
    switch (i) { case 0: return 0xfffffffeu; case 1: return 0x00000001u; case 2: return 0x00034802u; case 3: return 0x5884b7fau; case 4: return 0xecbc4ff5u; case 5: return 0x998c4fefu; case 6: return 0xacc5056fu; case 7: return 0x1824b159u; default: return 0u; }
  }
  ECC_DEV static constexpr uint32_t pm2(int i) {
    switch (i) { case 0: return 0xffffffffu; case 1: return 0xfffffffeu; case 2: return 0xfffe5bfeu; case 3: return 0x53bda402u; case 4: return 0x09a1d805u; case 5: return 0x3339d808u; case 6: return 0x299d7d48u; case 7: return 0x73eda753u; default: return 0u; }
  }
  ECC_DEV static constexpr uint32_t r3(int i) {
    switch (i) { case 0: return 0x439b73afu; case 1: return 0xc62c1807u; case 2: return 0x8cf06990u; case 3: return 0x1b3e0d18u; case 4: return 0xc7b5f418u; case 5: return 0x73d13c71u; case 6: return 0xc8db33e9u; case 7: return 0x6e2a5bb9u; default: return 0u; }
  }
};

struct BLS12_381 {
  using Fp = BLS12_381Fp;
  using Fn = BLS12_381Fn;
  static constexpr bool A_ZERO = true;
  ECC_DEV static constexpr uint32_t a(int i) {
    switch (i) { case 0: return 0x00000000u; case 1: return 0x00000000u; case 2: return 0x00000000u; case 3: return 0x00000000u; case 4: return 0x00000000u; case 5: return 0x00000000u; case 6: return 0x00000000u; case 7: return 0x00000000u; case 8: return 0x00000000u; case 9: return 0x00000000u; case 10: return 0x00000000u; case 11: return 0x00000000u; default: return 0u; }
  }
  ECC_DEV static constexpr uint32_t b(int i) {
    switch (i) { case 0: return 0x000cfff3u; case 1: return 0xaa270000u; case 2: return 0xfc34000au; case 3: return 0x53cc0032u; case 4: return 0x6b0a807fu; case 5: return 0x478fe97au; case 6: return 0xe6ba24d7u; case 7: return 0xb1d37ebeu; case 8: return 0xbf78ab2fu; case 9: return 0x8ec9733bu; case 10: return 0x3d83de7eu; case 11: return 0x09d64551u; default: return 0u; }
  }
  ECC_DEV static constexpr uint32_t gx(int i) {
    switch (i) { case 0: return 0xdb22c6bbu; case 1: return 0xfb3af00au; case 2: return 0xf97a1aefu; case 3: return 0x6c55e83fu; case 4: return 0x171bac58u; case 5: return 0xa14e3a3fu; case 6: return 0x9774b905u; case 7: return 0xc3688c4fu; case 8: return 0x4fa9ac0fu; case 9: return 0x2695638cu; case 10: return 0x3197d794u; case 11: return 0x17f1d3a7u; default: return 0u; }
  }
  ECC_DEV static constexpr uint32_t gy(int i) {
    switch (i) { case 0: return 0x46c5e7e1u; case 1: return 0x0caa2329u; case 2: return 0xa2888ae4u; case 3: return 0xd03cc744u; case 4: return 0x2c04b3edu; case 5: return 0x00db18cbu; case 6: return 0xd5d00af6u; case 7: return 0xfcf5e095u; case 8: return 0x741d8ae4u; case 9: return 0xa09e30edu; case 10: return 0xe3aaa0f1u; case 11: return 0x08b3f481u; default: return 0u; }
  }
  ECC_DEV static constexpr uint32_t n(int i) {
    switch (i) { case 0: return 0x00000001u; case 1: return 0xffffffffu; case 2: return 0xfffe5bfeu; case 3: return 0x53bda402u; case 4: return 0x09a1d805u; case 5: return 0x3339d808u; case 6: return 0x299d7d48u; case 7: return 0x73eda753u; default: return 0u; }
  }
  static constexpr int SCALAR_BITS = 255;
};

struct SM2Fp {
  static constexpr int N = 8;
  static constexpr int BITS = 256;
  static constexpr uint32_t QINV = 0x00000001u;
  static constexpr int FORM = 0;
  static constexpr uint64_t QINV62 = 0x3fffffffffffffffull;  // q^-1 mod 2^62
  ECC_DEV static constexpr uint32_t qinv() { return QINV; }
  ECC_DEV static constexpr uint64_t qinv62() { return QINV62; }
  ECC_DEV static constexpr uint32_t p(int i) {
    switch (i) { case 0: return 0xffffffffu; case 1: return 0xffffffffu; case 2: return 0x00000000u; case 3: return 0xffffffffu; case 4: return 0xffffffffu; case 5: return 0xffffffffu; case 6: return 0xffffffffu; case 7: return 0xfffffffeu; default: return 0u; }
  }
  ECC_DEV static constexpr uint32_t r2(int i) {
    switch (i) { case 0: return 0x00000003u; case 1: return 0x00000002u; case 2: return 0xffffffffu; case 3: return 0x00000002u; case 4: return 0x00000001u; case 5: return 0x00000001u; case 6: return 0x00000002u; case 7: return 0x00000004u; default: return 0u; }
  }
  ECC_DEV static constexpr uint32_t one(int i) {
    switch (i) { case 0: return 0x00000001u; case 1: return 0x00000000u; case 2: return 0xffffffffu; case 3: return 0x00000000u; case 4: return 0x00000000u; case 5: return 0x00000000u; case 6: return 0x00000000u; case 7: return 0x00000001u; default: return 0u; }
  }
  ECC_DEV static constexpr uint32_t pm2(int i) {
    switch (i) { case 0: return 0xfffffffdu; case 1: return 0xffffffffu; case 2: return 0x00000000u; case 3: return 0xffffffffu; case 4: return 0xffffffffu; case 5: return 0xffffffffu; case 6: return 0xffffffffu; case 7: return 0xfffffffeu; default: return 0u; }
  }
  ECC_DEV static constexpr uint32_t r3(int i) {
    switch (i) { case 0: return 0x00000016u; case 1: return 0x00000012u; case 2: return 0xfffffff8u; case 3: return 0x0000000eu; case 4: return 0x0000000cu; case 5: return 0x0000000au; case 6: return 0x00000009u; case 7: return 0x0000001bu; default: return 0u; }
  }
};

struct SM2Fn {
  static constexpr int N = 8;
  static constexpr int BITS = 256;
  static constexpr uint32_t QINV = 0x72350975u;
  static constexpr int FORM = 0;
  static constexpr uint64_t QINV62 = 0x0d8061778dcaf68bull;  // q^-1 mod 2^62
  ECC_DEV static constexpr uint32_t qinv() { return QINV; }
  ECC_DEV static constexpr uint64_t qinv62() { return QINV62; }
  ECC_DEV static constexpr uint32_t p(int i) {
    switch (i) { case 0: return 0x39d54123u; case 1: return 0x53bbf409u; case 2: return 0x21c6052bu; case 3: return 0x7203df6bu; case 4: return 0xffffffffu; case 5: return 0xffffffffu; case 6: return 0xffffffffu; case 7: return 0xfffffffeu; default: return 0u; }
  }
  ECC_DEV static constexpr uint32_t r2(int i) {
    switch (i) { case 0: return 0x7c114f20u; case 1: return 0x901192afu; case 2: return 0xde6fa2fau; case 3: return 0x3464504au; case 4: return 0x3affe0d4u; case 5: return 0x620fc84cu; case 6: return 0xa22b3d3bu; case 7: return 0x1eb5e412u; default: return 0u; }
  }
  ECC_DEV static constexpr uint32_t one(int i) {
    switch (i) { case 0: return 0xc62abeddu; case 1: return 0xac440bf6u; case 2: return 0xde39fad4u; case 3: return 0x8dfc2094u; case 4: return 0x00000000u; case 5: return 0x00000000u; case 6: return 0x00000000u; case 7: return 0x00000001u; default: return 0u; }
  }
  ECC_DEV static constexpr uint32_t pm2(int i) {
    switch (i) { case 0: return 0x39d54121u; case 1: return 0x53bbf409u; case 2: return 0x21c6052bu; case 3: return 0x7203df6bu; case 4: return 0xffffffffu; case 5: return 0xffffffffu; case 6: return 0xffffffffu; case 7: return 0xfffffffeu; default: return 0u; }
  }
  ECC_DEV static constexpr uint32_t r3(int i) {
    switch (i) { case 0: return 0x0eaa0b85u; case 1: return 0x6ff874c7u; case 2: return 0xaabe8d32u; case 3: return 0x87d0c315u; case 4: return 0x97185afcu; case 5: return 0x4c4fbbb3u; case 6: return 0xd574ea14u; case 7: return 0xc813249cu; default: return 0u; }
  }
};

struct SM2 {
  using Fp = SM2Fp;
  using Fn = SM2Fn;
  static constexpr bool A_ZERO = false;
  ECC_DEV static constexpr uint32_t a(int i) {
    switch (i) { case 0: return 0xfffffffcu; case 1: return 0xffffffffu; case 2: return 0x00000003u; case 3: return 0xfffffffcu; case 4: return 0xffffffffu; case 5: return 0xffffffffu; case 6: return 0xffffffffu; case 7: return 0xfffffffbu; default: return 0u; }
  }
  ECC_DEV static constexpr uint32_t b(int i) {
    switch (i) { case 0: return 0x2bc0dd42u; case 1: return 0x90d23063u; case 2: return 0xe9b537abu; case 3: return 0x71cf379au; case 4: return 0x5ea51c3cu; case 5: return 0x52798150u; case 6: return 0xba20e2c8u; case 7: return 0x240fe188u; default: return 0u; }
  }
  ECC_DEV static constexpr uint32_t gx(int i) {
    switch (i) { case 0: return 0x334c74c7u; case 1: return 0x715a4589u; case 2: return 0xf2660be1u; case 3: return 0x8fe30bbfu; case 4: return 0x6a39c994u; case 5: return 0x5f990446u; case 6: return 0x1f198119u; case 7: return 0x32c4ae2cu; default: return 0u; }
  }
  ECC_DEV static constexpr uint32_t gy(int i) {
    switch (i) { case 0: return 0x2139f0a0u; case 1: return 0x02df32e5u; case 2: return 0xc62a4740u; case 3: return 0xd0a9877cu; case 4: return 0x6b692153u; case 5: return 0x59bdcee3u; case 6: return 0xf4f6779cu; case 7: return 0xbc3736a2u; default: return 0u; }
  }
  ECC_DEV static constexpr uint32_t n(int i) {
    switch (i) { case 0: return 0x39d54123u; case 1: return 0x53bbf409u; case 2: return 0x21c6052bu; case 3: return 0x7203df6bu; case 4: return 0xffffffffu; case 5: return 0xffffffffu; case 6: return 0xffffffffu; case 7: return 0xfffffffeu; default: return 0u; }
  }
  static constexpr int SCALAR_BITS = 256;
};

}  // namespace ecc
