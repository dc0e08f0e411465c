// Prime-field arithmetic on 32-bit limbs (modular arithmetic layer, Section 4).
//
// Elements are N little-endian 32-bit limbs (N even: 8 for 254/256-bit fields,
// 12 for the 381-bit field) held in registers, in Montgomery form a*R mod q with
// R = 2^(32N), canonical in [0, q).  A field is a traits class F with
//   N, qinv() = -q^-1 mod 2^32, qinv62() = q^-1 mod 2^62, FORM (0 generic,
//   1 the P-256 prime, 2 the secp256k1 prime), p(i),
//   r2(i) = R^2 mod q, one(i) = R mod q, pm2(i) = q - 2.
//
// mont_mul is Montgomery multiplication (Algorithm 2) with the operand-scanning
// order interleaved row by row.  Each row A*b_i is split into an "even" chain
// (a_j b_i, j even) and an "odd" chain (a_j b_i, j odd), the mad_n carry chains
// of Section 4.1: within one chain the 64-bit products sit on disjoint word
// pairs, so one chain of alternating mad.lo / mad.hi links covers the row with a
// single carry.  The running value is kept as T = c + 2^32 d with c collecting
// the even chains and d the odd chains; the reduction row u*q (u = T_0 * QINV)
// is split the same way.  Dividing T by 2^32 then only renames registers
// (d becomes the new c, the upper words of c the new d) plus one add for word 0,
// whose carry enters the next odd chain as its carry-in -- so the count is
// 2N^2 + N multiply-adds (136 IMAD.WIDE-class for N = 8), as Section 4.1
// derives, and only ~4N extra adds.  The final value is < 2q and is brought
// into [0, q) with one conditional subtraction.
#pragma once
#include <cstdint>

#include "inv.cuh"
#include "ptx.cuh"

namespace ecc {

template <class F>
struct Fe {
  uint32_t v[F::N];
};

template <class F>
ECC_DEV void fe_copy(uint32_t* r, const uint32_t* a) {
#pragma unroll
  for (int i = 0; i < F::N; ++i) r[i] = a[i];
}

template <class F>
ECC_DEV void fe_set_one(uint32_t* r) {
#pragma unroll
  for (int i = 0; i < F::N; ++i) r[i] = F::one(i);
}

template <class F>
ECC_DEV void fe_set_zero(uint32_t* r) {
#pragma unroll
  for (int i = 0; i < F::N; ++i) r[i] = 0;
}

template <class F>
ECC_DEV bool fe_is_zero(const uint32_t* a) {
  uint32_t acc = 0;
#pragma unroll
  for (int i = 0; i < F::N; ++i) acc |= a[i];
  return acc == 0;
}

template <class F>
ECC_DEV bool fe_eq(const uint32_t* a, const uint32_t* b) {
  uint32_t acc = 0;
#pragma unroll
  for (int i = 0; i < F::N; ++i) acc |= a[i] ^ b[i];
  return acc == 0;
}

template <class F>
ECC_DEV bool fe_is_one(const uint32_t* a) {
  uint32_t acc = 0;
#pragma unroll
  for (int i = 0; i < F::N; ++i) acc |= a[i] ^ F::one(i);
  return acc == 0;
}

// r = cond ? a : b
template <class F>
ECC_DEV void fe_select(uint32_t* r, bool cond, const uint32_t* a, const uint32_t* b) {
#pragma unroll
  for (int i = 0; i < F::N; ++i) r[i] = cond ? a[i] : b[i];
}

// a < q as plain integers (used to validate canonical inputs)
template <class F>
ECC_DEV bool fe_lt_modulus(const uint32_t* a) {
  uint32_t t = ptx::sub_cc(a[0], F::p(0));
#pragma unroll
  for (int i = 1; i < F::N; ++i) t = ptx::subc_cc(a[i], F::p(i));
  uint32_t borrow = ptx::subc(0, 0);
  (void)t;
  return borrow != 0;
}

// r = a + b mod q
template <class F>
ECC_DEV void fe_add(uint32_t* r, const uint32_t* a, const uint32_t* b) {
  constexpr int N = F::N;
  uint32_t t[N], s[N];
  t[0] = ptx::add_cc(a[0], b[0]);
#pragma unroll
  for (int i = 1; i < N; ++i) t[i] = ptx::addc_cc(a[i], b[i]);
  uint32_t top = ptx::addc(0, 0);
  s[0] = ptx::sub_cc(t[0], F::p(0));
#pragma unroll
  for (int i = 1; i < N; ++i) s[i] = ptx::subc_cc(t[i], F::p(i));
  top = ptx::subc(top, 0);  // 0xffffffff iff a + b < q
#pragma unroll
  for (int i = 0; i < N; ++i) r[i] = top ? t[i] : s[i];
}

// r = a - b mod q
template <class F>
ECC_DEV void fe_sub(uint32_t* r, const uint32_t* a, const uint32_t* b) {
  constexpr int N = F::N;
  uint32_t t[N];
  t[0] = ptx::sub_cc(a[0], b[0]);
#pragma unroll
  for (int i = 1; i < N; ++i) t[i] = ptx::subc_cc(a[i], b[i]);
  uint32_t mask = ptx::subc(0, 0);  // 0xffffffff iff a < b
  r[0] = ptx::add_cc(t[0], F::p(0) & mask);
#pragma unroll
  for (int i = 1; i < N - 1; ++i) r[i] = ptx::addc_cc(t[i], F::p(i) & mask);
  r[N - 1] = ptx::addc(t[N - 1], F::p(N - 1) & mask);
}

template <class F>
ECC_DEV void fe_neg(uint32_t* r, const uint32_t* a) {
  uint32_t z[F::N];
  fe_set_zero<F>(z);
  fe_sub<F>(r, z, a);
}

// Reduction row of mont_mul for q = 2^256 - 2^224 + 2^192 + 2^96 - 1 (NIST
// P-256), the special-form reduction of Section 4.2 done our way: -q^-1 mod
// 2^32 is 1, so u = T_0, and every limb of q is 0, 1 or 2^32 - 1, so
// u q_j needs no multiplication: u (2^32 - 1) = hu 2^32 + nu with nu = -u mod
// 2^32 and hu = u - [u != 0].  The even chain adds u (q_0 + q_2 2^64 + q_6 2^192)
// to c (q_4 = 0): word 0 becomes u + nu, which is 0 with carry [u != 0], and
// that carry plus hu makes u at word 1.  The odd chain adds
// u (q_1 + q_7 2^192) to d (q_3 = q_5 = 0).  Both chains are additions: the
// row costs no multiply-adds instead of 2N + 2.
ECC_DEV void p256_reduce_row(uint32_t* c, uint32_t* d) {
  const uint32_t u = c[0];
  const uint32_t nu = 0u - u;
  const uint32_t hu = u - (u != 0u ? 1u : 0u);
  c[1] = ptx::add_cc(c[1], u);
  c[2] = ptx::addc_cc(c[2], nu);
  c[3] = ptx::addc_cc(c[3], hu);
  c[4] = ptx::addc_cc(c[4], 0);
  c[5] = ptx::addc_cc(c[5], 0);
  c[6] = ptx::addc_cc(c[6], u);
  c[7] = ptx::addc_cc(c[7], 0);
  c[8] = ptx::addc(c[8], 0);
  d[0] = ptx::add_cc(d[0], nu);
  d[1] = ptx::addc_cc(d[1], hu);
  d[2] = ptx::addc_cc(d[2], 0);
  d[3] = ptx::addc_cc(d[3], 0);
  d[4] = ptx::addc_cc(d[4], 0);
  d[5] = ptx::addc_cc(d[5], 0);
  d[6] = ptx::addc_cc(d[6], nu);
  d[7] = ptx::addc_cc(d[7], hu);
  d[8] = ptx::addc(d[8], 0);
}

// Reduction row of mont_mul for q = 2^256 - 2^32 - 977 (secp256k1), the
// special-form idea of Section 4.2 applied to this prime: u q = u 2^256 -
// u (2^32 + 977), so the row needs one 32 x 32 -> 64 product (977 u) instead
// of N.  -q^-1 mod 2^32 is not 1 for this prime, so u = T_0 QINV stays a
// multiplication.  Word 0 of T + u q is exactly 0 with no carry (u makes
// T_0 = 977 u mod 2^32), and the words above it receive
// A = u 2^224 - (u + floor(977 u / 2^32)) in the frame of d (d[k] is word
// k + 1): A is a non-negative 256-bit value (0 when u = 0), added with one
// carry chain whose carry lands in d's top word.
ECC_DEV void secp256k1_reduce_row(uint32_t* c, uint32_t* d, uint32_t qinv) {
  const uint32_t u = c[0] * qinv;
  const uint32_t s1 = ptx::add_cc(__umulhi(u, 977u), u);
  const uint32_t s2 = ptx::addc(0, 0);
  uint32_t A[8];
  A[0] = ptx::sub_cc(0, s1);
  A[1] = ptx::subc_cc(0, s2);
#pragma unroll
  for (int k = 2; k < 7; ++k) A[k] = ptx::subc_cc(0, 0);
  A[7] = ptx::subc(u, 0);
  d[0] = ptx::add_cc(d[0], A[0]);
#pragma unroll
  for (int k = 1; k < 8; ++k) d[k] = ptx::addc_cc(d[k], A[k]);
  d[8] = ptx::addc(d[8], 0);
}

// Montgomery product r = a * b * R^-1 mod q (r may alias a or b).
template <class F>
ECC_DEV void mont_mul(uint32_t* r, const uint32_t* a, const uint32_t* b) {
  constexpr int N = F::N;
  static_assert(N % 2 == 0, "even limb count");
  uint32_t c[N + 1], d[N + 1];
#pragma unroll
  for (int i = 0; i < N + 1; ++i) {
    c[i] = 0;
    d[i] = 0;
  }
#pragma unroll
  for (int i = 0; i < N; ++i) {
    const uint32_t bi = b[i];
    if (i == 0) {
      // odd chain: d[j-1], d[j] += a_j * b_0 for odd j
      d[0] = ptx::mad_lo_cc(a[1], bi, d[0]);
      d[1] = ptx::madc_hi_cc(a[1], bi, d[1]);
    } else {
      // T /= 2^32: new c = (d0 + c1, d1, .., dN), new d = (c2, .., cN, 0, 0);
      // the carry of d0 + c1 (word 1) is the carry-in of the odd chain.
      uint32_t nc0 = ptx::add_cc(d[0], c[1]);
#pragma unroll
      for (int k = 0; k < N - 1; ++k) {
        uint32_t t = d[k + 1];
        d[k] = c[k + 2];
        c[k + 1] = t;
      }
      c[N] = d[N];
      c[0] = nc0;
      d[N - 1] = 0;
      d[N] = 0;
      d[0] = ptx::madc_lo_cc(a[1], bi, d[0]);
      d[1] = ptx::madc_hi_cc(a[1], bi, d[1]);
    }
#pragma unroll
    for (int j = 3; j < N; j += 2) {
      d[j - 1] = ptx::madc_lo_cc(a[j], bi, d[j - 1]);
      d[j] = ptx::madc_hi_cc(a[j], bi, d[j]);
    }
    d[N] = ptx::addc(d[N], 0);
    // even chain: c[j], c[j+1] += a_j * b_i for even j
    c[0] = ptx::mad_lo_cc(a[0], bi, c[0]);
    c[1] = ptx::madc_hi_cc(a[0], bi, c[1]);
#pragma unroll
    for (int j = 2; j < N; j += 2) {
      c[j] = ptx::madc_lo_cc(a[j], bi, c[j]);
      c[j + 1] = ptx::madc_hi_cc(a[j], bi, c[j + 1]);
    }
    c[N] = ptx::addc(c[N], 0);
    if constexpr (F::FORM == 1) {
      p256_reduce_row(c, d);
      continue;
    }
    if constexpr (F::FORM == 2) {
      secp256k1_reduce_row(c, d, F::qinv());
      continue;
    }
    // reduction row: u = T_0 * QINV, T += u * q (even and odd chains)
    const uint32_t u = c[0] * F::qinv();
    c[0] = ptx::mad_lo_cc(u, F::p(0), c[0]);
    c[1] = ptx::madc_hi_cc(u, F::p(0), c[1]);
#pragma unroll
    for (int j = 2; j < N; j += 2) {
      c[j] = ptx::madc_lo_cc(u, F::p(j), c[j]);
      c[j + 1] = ptx::madc_hi_cc(u, F::p(j), c[j + 1]);
    }
    c[N] = ptx::addc(c[N], 0);
    d[0] = ptx::mad_lo_cc(u, F::p(1), d[0]);
    d[1] = ptx::madc_hi_cc(u, F::p(1), d[1]);
#pragma unroll
    for (int j = 3; j < N; j += 2) {
      d[j - 1] = ptx::madc_lo_cc(u, F::p(j), d[j - 1]);
      d[j] = ptx::madc_hi_cc(u, F::p(j), d[j]);
    }
    d[N] = ptx::addc(d[N], 0);
  }
  // last division by 2^32 and merge: t = d + (c >> 32 bits), t < 2q
  uint32_t t[N + 1];
  t[0] = ptx::add_cc(d[0], c[1]);
#pragma unroll
  for (int k = 1; k < N; ++k) t[k] = ptx::addc_cc(d[k], c[k + 1]);
  t[N] = ptx::addc(d[N], 0);
  uint32_t s[N];
  s[0] = ptx::sub_cc(t[0], F::p(0));
#pragma unroll
  for (int k = 1; k < N; ++k) s[k] = ptx::subc_cc(t[k], F::p(k));
  const uint32_t top = ptx::subc(t[N], 0);  // 0xffffffff iff t < q
#pragma unroll
  for (int k = 0; k < N; ++k) r[k] = top == 0xffffffffu ? t[k] : s[k];
}

template <class F>
ECC_DEV void mont_sqr(uint32_t* r, const uint32_t* a) {
  mont_mul<F>(r, a, a);
}

// canonical integer -> Montgomery form (a * R^2 * R^-1 = a R)
template <class F>
ECC_DEV void to_mont(uint32_t* r, const uint32_t* a) {
  uint32_t r2[F::N];
#pragma unroll
  for (int i = 0; i < F::N; ++i) r2[i] = F::r2(i);
  mont_mul<F>(r, a, r2);
}

// Montgomery form -> canonical integer
template <class F>
ECC_DEV void from_mont(uint32_t* r, const uint32_t* a) {
  uint32_t one[F::N];
#pragma unroll
  for (int i = 0; i < F::N; ++i) one[i] = i == 0 ? 1u : 0u;
  mont_mul<F>(r, a, one);
}

// r = a^(q-2) = a^-1 (Fermat, Section 2.2); a = 0 gives 0.  Fixed 4-bit
// windows over the exponent, most significant first.  Used by one thread per
// batch (the "apply" step of the gather-apply-scatter batch inversion).
template <class F>
__device__ __noinline__ void fe_inv_fermat(uint32_t* r, const uint32_t* a) {
  constexpr int N = F::N;
  uint32_t tab[16][N];
  fe_set_one<F>(tab[0]);
  fe_copy<F>(tab[1], a);
  for (int k = 2; k < 16; ++k) mont_mul<F>(tab[k], tab[k - 1], a);
  uint32_t acc[N];
  fe_set_one<F>(acc);
  for (int w = 8 * N - 1; w >= 0; --w) {
    const uint32_t digit = (F::pm2(w >> 3) >> (4 * (w & 7))) & 15u;
    for (int s = 0; s < 4; ++s) mont_sqr<F>(acc, acc);
    uint32_t t[N];
#pragma unroll
    for (int i = 0; i < N; ++i) t[i] = tab[digit][i];
    mont_mul<F>(acc, acc, t);
  }
  fe_copy<F>(r, acc);
}

// r = a^-1 in Montgomery form (a = x R -> r = x^-1 R), a = 0 gives 0, by the
// divstep inversion of inv.cuh on 30-bit limbs with branch-free single
// divsteps: (x R)^-1 is computed on the integer, then one Montgomery product
// with R^3 mod q restores the form.  Out of line: it runs on one thread per
// batch, where its latency is the serial step of every batched round (GB300,
// one thread, 256-bit field: 22.8 us, against 27.7 us with batched variable-
// time divsteps on 30-bit limbs and 32.6 us on 62-bit limbs).
template <class F, bool FLAT = true>
__device__ __noinline__ void fe_inv_mont(uint32_t* r, const uint32_t* a) {
  constexpr int N = F::N;
  constexpr int L = (32 * N + 2 + 29) / 30;
  uint32_t q[N], x[N], r3[N];
#pragma unroll
  for (int i = 0; i < N; ++i) {
    q[i] = F::p(i);
    r3[i] = F::r3(i);
  }
  inv_divsteps30<L, FLAT>(x, a, q, N, (uint32_t)F::qinv62() & (uint32_t)kM30);
  mont_mul<F>(r, x, r3);
}

// The same with the 62-bit-limb divsteps (64 x 64 -> 128-bit products), kept
// for the inversion probe.
template <class F>
__device__ __noinline__ void fe_inv_mont62(uint32_t* r, const uint32_t* a) {
  constexpr int N = F::N;
  constexpr int L = (32 * N + 2 + 61) / 62;
  uint32_t q[N], x[N], r3[N];
#pragma unroll
  for (int i = 0; i < N; ++i) {
    q[i] = F::p(i);
    r3[i] = F::r3(i);
  }
  inv_divsteps<L>(x, a, q, N, F::qinv62());
  mont_mul<F>(r, x, r3);
}

}  // namespace ecc
