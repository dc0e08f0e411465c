// Single modular inversion by Bernstein-Yang divsteps ("safegcd", Bernstein and
// Yang, "Fast constant-time gcd computation and modular inversion", TCHES 2019),
// variable-time form: the inputs of a batch inversion are public here.
//
// The paper discusses Fermat (x^(q-2)) versus extended-Euclid inversion and
// notes the latter is ~3x faster but branchy (Section 2.2); in the GAS batch
// inversion only one thread per batch runs it (Section 3.2), so branches cost
// nothing, while its short dependent chain shortens the serial "apply" step that
// the whole CTA waits for.
//
// State: f, g, d, e as signed integers in L limbs of 62 bits (least significant
// first, every limb but the top in [0, 2^62), top limb signed).  Start f = q,
// g = x, d = 0, e = 1, with the invariant f = d x, g = e x (mod q).  Each
// outer step runs 62 divsteps on the low 64 bits of (f, g) and records them as
// a 2x2 integer matrix T with 2^62 (f', g') = T (f, g); then (f, g) <- T (f, g)
// / 2^62 exactly and (d, e) <- T (d, e) / 2^62 mod q (adding the multiple of q
// that makes the division exact).  When g = 0, f = +-1 and x^-1 = +-d.
#pragma once
#include <cstdint>

#ifndef ECC_DEV
#define ECC_DEV __device__ __forceinline__
#endif

namespace ecc {

constexpr int64_t kM62 = (int64_t)(((uint64_t)1 << 62) - 1);

struct Trans {
  int64_t u, v, q, r;
};

ECC_DEV int ctz64(uint64_t x) {
#ifdef __CUDA_ARCH__
  return __ffsll((long long)x) - 1;
#else
  return __builtin_ctzll(x);
#endif
}

// 62 divsteps on the low bits of f and g (f odd).  delta is carried across calls.
// A run of k divsteps with g even (g <- g/2, delta <- delta + 1) is applied at
// once by counting trailing zeros.  With g odd and delta > 0 the divstep swaps
// and goes alone.  With g odd and delta <= 0, the next k <= 1 - delta divsteps
// cannot swap: each adds f when g is odd and halves, so together they add w f
// with w = -g / f mod 2^k (the unique multiple that clears k low bits) and
// halve k times; the addition is done here (k <= 6, f^-1 mod 64 by one Newton
// step from f, which is its own inverse mod 8) and the halvings by the next
// trailing-zero count.
ECC_DEV Trans divsteps62(int64_t& delta, uint64_t f, uint64_t g) {
  int64_t u = 1, v = 0, q = 0, r = 1;
  int left = 62;
  for (;;) {
    // the bit at position `left` keeps the count finite when g's low bits are 0
    int z = ctz64(g | ((uint64_t)1 << left));
    g >>= z;
    u <<= z;
    v <<= z;
    delta += z;
    left -= z;
    if (left == 0) break;
    if (delta > 0) {  // g odd: one swapping divstep
      delta = 1 - delta;
      const uint64_t nf = g;
      g = (g - f) >> 1;
      f = nf;
      const int64_t nu = 2 * q, nv = 2 * r;
      q = q - u;
      r = r - v;
      u = nu;
      v = nv;
      if (--left == 0) break;
    } else {  // g odd, delta <= 0: k non-swapping divsteps at once
      int k = 1 - delta < (int64_t)left ? (int)(1 - delta) : left;
      if (k > 6) k = 6;
      const uint32_t fl = (uint32_t)f;
      const uint32_t finv = fl * (2u - fl * fl);  // f^-1 mod 64
      const uint64_t w = (0u - (uint32_t)g * finv) & ((1u << k) - 1u);
      g += w * f;
      q += (int64_t)w * u;
      r += (int64_t)w * v;
    }
  }
  return Trans{u, v, q, r};
}

// (f, g) <- T (f, g) / 2^62 (exact)
template <int L>
ECC_DEV void update_fg(int64_t* f, int64_t* g, const Trans& t) {
  __int128 cf = (__int128)t.u * f[0] + (__int128)t.v * g[0];
  __int128 cg = (__int128)t.q * f[0] + (__int128)t.r * g[0];
  cf >>= 62;
  cg >>= 62;
#pragma unroll
  for (int i = 1; i < L; ++i) {
    cf += (__int128)t.u * f[i] + (__int128)t.v * g[i];
    cg += (__int128)t.q * f[i] + (__int128)t.r * g[i];
    f[i - 1] = (int64_t)cf & kM62;
    g[i - 1] = (int64_t)cg & kM62;
    cf >>= 62;
    cg >>= 62;
  }
  f[L - 1] = (int64_t)cf;
  g[L - 1] = (int64_t)cg;
}

template <int L>
ECC_DEV bool s62_is_zero(const int64_t* a) {
  int64_t acc = 0;
#pragma unroll
  for (int i = 0; i < L; ++i) acc |= a[i];
  return acc == 0;
}

// a += k q (k in {-1, +1}), keeping limbs normalised
template <int L>
ECC_DEV void s62_add_mul(int64_t* a, const int64_t* q, int64_t k) {
  int64_t c = 0;
#pragma unroll
  for (int i = 0; i < L - 1; ++i) {
    c += a[i] + k * q[i];
    a[i] = c & kM62;
    c >>= 62;
  }
  a[L - 1] += c + k * q[L - 1];
}

// a >= q for a >= 0 (normalised limbs)
template <int L>
ECC_DEV bool s62_ge(const int64_t* a, const int64_t* q) {
#pragma unroll
  for (int i = L - 1; i >= 0; --i) {
    if (a[i] != q[i]) return a[i] > q[i];
  }
  return true;
}

// bring a from (-3q, 3q) into [0, q)
template <int L>
ECC_DEV void s62_normalise(int64_t* a, const int64_t* q) {
  while (a[L - 1] < 0) s62_add_mul<L>(a, q, 1);
  while (s62_ge<L>(a, q)) s62_add_mul<L>(a, q, -1);
}

// (d, e) <- T (d, e) / 2^62 mod q, results in [0, q); qinv62 = q^-1 mod 2^62
template <int L>
ECC_DEV void update_de(int64_t* d, int64_t* e, const Trans& t, const int64_t* q, uint64_t qinv62) {
  // multiples of q that make the low 62 bits vanish
  const uint64_t ld = (uint64_t)(t.u * d[0] + t.v * e[0]);
  const uint64_t le = (uint64_t)(t.q * d[0] + t.r * e[0]);
  const int64_t md = (int64_t)((0 - ld * qinv62) & (uint64_t)kM62);
  const int64_t me = (int64_t)((0 - le * qinv62) & (uint64_t)kM62);
  __int128 cd = (__int128)t.u * d[0] + (__int128)t.v * e[0] + (__int128)md * q[0];
  __int128 ce = (__int128)t.q * d[0] + (__int128)t.r * e[0] + (__int128)me * q[0];
  cd >>= 62;
  ce >>= 62;
#pragma unroll
  for (int i = 1; i < L; ++i) {
    cd += (__int128)t.u * d[i] + (__int128)t.v * e[i] + (__int128)md * q[i];
    ce += (__int128)t.q * d[i] + (__int128)t.r * e[i] + (__int128)me * q[i];
    d[i - 1] = (int64_t)cd & kM62;
    e[i - 1] = (int64_t)ce & kM62;
    cd >>= 62;
    ce >>= 62;
  }
  d[L - 1] = (int64_t)cd;
  e[L - 1] = (int64_t)ce;
  s62_normalise<L>(d, q);
  s62_normalise<L>(e, q);
}

// 32-bit limbs (n words) -> signed62 limbs
template <int L>
ECC_DEV void to_s62(int64_t* out, const uint32_t* a, int n) {
#pragma unroll
  for (int i = 0; i < L; ++i) {
    // bits [62 i, 62 i + 62)
    const int bit = 62 * i;
    uint64_t v = 0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const int w = bit / 32 + k;
      if (w < n) {
        const int sh = 32 * w - bit;
        if (sh >= 0) {
          if (sh < 64) v |= (uint64_t)a[w] << sh;
        } else {
          v |= (uint64_t)a[w] >> (-sh);
        }
      }
    }
    out[i] = (int64_t)(v & (uint64_t)kM62);
  }
}

// signed62 limbs of a value in [0, 2^(32 n)) -> 32-bit limbs
template <int L>
ECC_DEV void from_s62(uint32_t* out, const int64_t* a, int n) {
  for (int w = 0; w < n; ++w) {
    const int bit = 32 * w;
    const int i = bit / 62, sh = bit % 62;
    uint64_t v = (uint64_t)a[i] >> sh;
    if (sh > 30 && i + 1 < L) v |= (uint64_t)a[i + 1] << (62 - sh);
    out[w] = (uint32_t)v;
  }
}

// x^-1 mod q for canonical x (0 gives 0).  q: n 32-bit limbs, odd;
// L = limbs of 62 bits with 62 L > bits(q) + 2.
template <int L>
ECC_DEV void inv_divsteps(uint32_t* out, const uint32_t* x, const uint32_t* q32, int n,
                          uint64_t qinv62) {
  int64_t f[L], g[L], d[L], e[L], q[L];
  to_s62<L>(q, q32, n);
  to_s62<L>(f, q32, n);
  to_s62<L>(g, x, n);
  if (s62_is_zero<L>(g)) {
    for (int w = 0; w < n; ++w) out[w] = 0;
    return;
  }
#pragma unroll
  for (int i = 0; i < L; ++i) {
    d[i] = 0;
    e[i] = i == 0 ? 1 : 0;
  }
  int64_t delta = 1;
  for (int it = 0; it < 64; ++it) {  // 62 * 64 divsteps bound any 1024-bit modulus
    const Trans t = divsteps62(delta, (uint64_t)f[0] | ((uint64_t)f[1] << 62),
                               (uint64_t)g[0] | ((uint64_t)g[1] << 62));
    update_fg<L>(f, g, t);
    update_de<L>(d, e, t, q, qinv62);
    if (s62_is_zero<L>(g)) break;
  }
  // f = +-1
  if (f[L - 1] < 0) {
    int64_t z[L];
#pragma unroll
    for (int i = 0; i < L; ++i) z[i] = 0;
    // d <- -d mod q = q - d (d in [0, q))
    if (!s62_is_zero<L>(d)) {
      s62_add_mul<L>(z, q, 1);
      int64_t c = 0;
#pragma unroll
      for (int i = 0; i < L - 1; ++i) {
        c += z[i] - d[i];
        d[i] = c & kM62;
        c >>= 62;
      }
      d[L - 1] = z[L - 1] - d[L - 1] + c;
    }
  }
  from_s62<L>(out, d, n);
}

}  // namespace ecc
