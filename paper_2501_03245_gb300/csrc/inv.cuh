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
    u = (int64_t)((uint64_t)u << z);  // u 2^z (two's complement shift)
    v = (int64_t)((uint64_t)v << z);
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
  // low 62 bits of T (d, e) (products taken mod 2^64)
  const uint64_t ld = (uint64_t)t.u * (uint64_t)d[0] + (uint64_t)t.v * (uint64_t)e[0];
  const uint64_t le = (uint64_t)t.q * (uint64_t)d[0] + (uint64_t)t.r * (uint64_t)e[0];
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

// ---------------------------------------------------------------------------
// The same method on 30-bit limbs with batches of 30 divsteps.  The transition
// matrix entries are below 2^30 in magnitude, so every product in the updates
// is one signed 32 x 32 -> 64-bit multiply-add (the 62-bit form needs 64 x 64
// -> 128-bit products, which a GPU builds from several 32-bit ones), and the
// divsteps run on 32-bit words.  Twice as many (cheaper) outer steps.

constexpr int32_t kM30 = (1 << 30) - 1;

struct Trans30 {
  int32_t u, v, q, r;
};

ECC_DEV int ctz32(uint32_t x) {
#ifdef __CUDA_ARCH__
  return __ffs((int)x) - 1;
#else
  return __builtin_ctz(x);
#endif
}

// 30 divsteps on the low 32 bits of f and g (f odd), as divsteps62 above:
// 2^30 (f', g') = T (f, g).  Runs of non-swapping steps add w f with w =
// -g / f mod 2^k (k <= 8; f^-1 mod 256 by two Newton steps from f, its own
// inverse mod 8).
ECC_DEV Trans30 divsteps30(int32_t& delta, uint32_t f, uint32_t g) {
  int32_t u = 1, v = 0, q = 0, r = 1;
  int left = 30;
  for (;;) {
    const int z = ctz32(g | (1u << left));
    g >>= z;
    u = (int32_t)((uint32_t)u << z);  // u 2^z (two's complement shift)
    v = (int32_t)((uint32_t)v << z);
    delta += z;
    left -= z;
    if (left == 0) break;
    if (delta > 0) {
      delta = 1 - delta;
      const uint32_t nf = g;
      g = (g - f) >> 1;
      f = nf;
      const int32_t nu = 2 * q, nv = 2 * r;
      q -= u;
      r -= v;
      u = nu;
      v = nv;
      if (--left == 0) break;
    } else {
      int k = 1 - delta < left ? 1 - delta : left;
      if (k > 8) k = 8;
      uint32_t finv = f * (2u - f * f);  // mod 2^6
      finv *= 2u - f * finv;             // mod 2^12
      const uint32_t w = (0u - g * finv) & ((1u << k) - 1u);
      g += w * f;
      q += (int32_t)w * u;
      r += (int32_t)w * v;
    }
  }
  return Trans30{u, v, q, r};
}

// The same 30 divsteps one at a time without branches (selects only): the
// GPU runs this thread's dependent chain without branch resolution.
ECC_DEV Trans30 divsteps30_flat(int32_t& delta, uint32_t f, uint32_t g) {
  int32_t u = 1, v = 0, q = 0, r = 1;
  // unrolled by 6: five trips of a short body keep the code small (it shares
  // the instruction cache with the kernel's rounds)
#pragma unroll 6
  for (int i = 0; i < 30; ++i) {
    const bool sw = (delta > 0) & ((g & 1u) != 0u);
    // swapping step: (delta, f, g, T) <- (-delta, g, -f, rows exchanged, new
    // second row negated); then g <- (g + (g odd) f) / 2 for both kinds
    const int32_t d1 = sw ? -delta : delta;
    const uint32_t f1 = sw ? g : f;
    const uint32_t g1 = sw ? 0u - f : g;
    const int32_t u1 = sw ? q : u, v1 = sw ? r : v;
    const int32_t q1 = sw ? -u : q, r1 = sw ? -v : r;
    const bool odd = (g1 & 1u) != 0u;
    g = (g1 + (odd ? f1 : 0u)) >> 1;
    q = q1 + (odd ? u1 : 0);
    r = r1 + (odd ? v1 : 0);
    f = f1;
    u = u1 * 2;
    v = v1 * 2;
    delta = d1 + 1;
  }
  return Trans30{u, v, q, r};
}

ECC_DEV int64_t mul32w(int32_t a, int32_t b) { return (int64_t)a * (int64_t)b; }

// (f, g) <- T (f, g) / 2^30 (exact)
template <int L>
ECC_DEV void update_fg30(int32_t* f, int32_t* g, const Trans30& t) {
  int64_t cf = mul32w(t.u, f[0]) + mul32w(t.v, g[0]);
  int64_t cg = mul32w(t.q, f[0]) + mul32w(t.r, g[0]);
  cf >>= 30;
  cg >>= 30;
#pragma unroll
  for (int i = 1; i < L; ++i) {
    cf += mul32w(t.u, f[i]) + mul32w(t.v, g[i]);
    cg += mul32w(t.q, f[i]) + mul32w(t.r, g[i]);
    f[i - 1] = (int32_t)cf & kM30;
    g[i - 1] = (int32_t)cg & kM30;
    cf >>= 30;
    cg >>= 30;
  }
  f[L - 1] = (int32_t)cf;
  g[L - 1] = (int32_t)cg;
}

template <int L>
ECC_DEV bool s30_is_zero(const int32_t* a) {
  int32_t acc = 0;
#pragma unroll
  for (int i = 0; i < L; ++i) acc |= a[i];
  return acc == 0;
}

// a += k q (k in {-1, +1}), keeping limbs normalised
template <int L>
ECC_DEV void s30_add_mul(int32_t* a, const int32_t* q, int32_t k) {
  int32_t c = 0;
#pragma unroll
  for (int i = 0; i < L - 1; ++i) {
    c += a[i] + k * q[i];
    a[i] = c & kM30;
    c >>= 30;
  }
  a[L - 1] += c + k * q[L - 1];
}

template <int L>
ECC_DEV bool s30_ge(const int32_t* a, const int32_t* q) {
#pragma unroll
  for (int i = L - 1; i >= 0; --i) {
    if (a[i] != q[i]) return a[i] > q[i];
  }
  return true;
}

// bring a from (-3q, 3q) into [0, q)
template <int L>
ECC_DEV void s30_normalise(int32_t* a, const int32_t* q) {
  while (a[L - 1] < 0) s30_add_mul<L>(a, q, 1);
  while (s30_ge<L>(a, q)) s30_add_mul<L>(a, q, -1);
}

// (d, e) <- T (d, e) / 2^30 mod q for d, e in (-2q, q), results in (-2q, q);
// qinv30 = q^-1 mod 2^30.  A negative input is first raised by q, folded into
// the multiple of q that is added anyway: with d, e in (-q, q) and |u| + |v|,
// |q| + |r| <= 2^30, T (d, e) + m q with m in [0, 2^30) lies in
// (-2^31 q, 2^30 q), so the exact quotient lies in (-2q, q) and no
// normalisation is needed until the end.
template <int L>
ECC_DEV void update_de30(int32_t* d, int32_t* e, const Trans30& t, const int32_t* q, uint32_t qinv30) {
  const int32_t sd = d[L - 1] >> 31, se = e[L - 1] >> 31;  // -1 when negative
  int32_t md = (t.u & sd) + (t.v & se);
  int32_t me = (t.q & sd) + (t.r & se);
  int64_t cd = mul32w(t.u, d[0]) + mul32w(t.v, e[0]);
  int64_t ce = mul32w(t.q, d[0]) + mul32w(t.r, e[0]);
  // subtract from m what makes the low 30 bits of T (d, e) + m q vanish
  md -= (int32_t)((qinv30 * (uint32_t)cd + (uint32_t)md) & (uint32_t)kM30);
  me -= (int32_t)((qinv30 * (uint32_t)ce + (uint32_t)me) & (uint32_t)kM30);
  cd += mul32w(md, q[0]);
  ce += mul32w(me, q[0]);
  cd >>= 30;
  ce >>= 30;
#pragma unroll
  for (int i = 1; i < L; ++i) {
    cd += mul32w(t.u, d[i]) + mul32w(t.v, e[i]) + mul32w(md, q[i]);
    ce += mul32w(t.q, d[i]) + mul32w(t.r, e[i]) + mul32w(me, q[i]);
    d[i - 1] = (int32_t)cd & kM30;
    e[i - 1] = (int32_t)ce & kM30;
    cd >>= 30;
    ce >>= 30;
  }
  d[L - 1] = (int32_t)cd;
  e[L - 1] = (int32_t)ce;
}

// 32-bit limbs (n words) -> 30-bit limbs
template <int L>
ECC_DEV void to_s30(int32_t* out, const uint32_t* a, int n) {
#pragma unroll
  for (int i = 0; i < L; ++i) {
    const int bit = 30 * i, w = bit >> 5, sh = bit & 31;
    uint64_t v = w < n ? (uint64_t)a[w] >> sh : 0u;
    if (w + 1 < n) v |= (uint64_t)a[w + 1] << (32 - sh);
    out[i] = (int32_t)(v & (uint64_t)kM30);
  }
}

// 30-bit limbs of a value in [0, 2^(32 n)) -> 32-bit limbs
template <int L>
ECC_DEV void from_s30(uint32_t* out, const int32_t* a, int n) {
  for (int w = 0; w < n; ++w) {
    const int bit = 32 * w, i = bit / 30, sh = bit % 30;
    uint64_t v = (uint64_t)(uint32_t)a[i] >> sh;
    if (i + 1 < L) v |= (uint64_t)(uint32_t)a[i + 1] << (30 - sh);
    if (i + 2 < L) v |= (uint64_t)(uint32_t)a[i + 2] << (60 - sh);
    out[w] = (uint32_t)v;
  }
}

// x^-1 mod q for canonical x (0 gives 0).  q: n 32-bit limbs, odd;
// L = limbs of 30 bits with 30 L > bits(q) + 2; qinv30 = q^-1 mod 2^30.
template <int L, bool FLAT = false>
ECC_DEV void inv_divsteps30(uint32_t* out, const uint32_t* x, const uint32_t* q32, int n, uint32_t qinv30) {
  int32_t f[L], g[L], d[L], e[L], q[L];
  to_s30<L>(q, q32, n);
  to_s30<L>(f, q32, n);
  to_s30<L>(g, x, n);
  if (s30_is_zero<L>(g)) {
    for (int w = 0; w < n; ++w) out[w] = 0;
    return;
  }
#pragma unroll
  for (int i = 0; i < L; ++i) {
    d[i] = 0;
    e[i] = i == 0 ? 1 : 0;
  }
  int32_t delta = 1;
  for (int it = 0; it < 128; ++it) {  // 30 * 128 divsteps bound any 1024-bit modulus
    const uint32_t fl = (uint32_t)f[0] | ((uint32_t)f[1] << 30), gl = (uint32_t)g[0] | ((uint32_t)g[1] << 30);
    const Trans30 t = FLAT ? divsteps30_flat(delta, fl, gl) : divsteps30(delta, fl, gl);
    update_fg30<L>(f, g, t);
    update_de30<L>(d, e, t, q, qinv30);
    if (s30_is_zero<L>(g)) break;
  }
  // f = +-1: x^-1 = f d, d in (-2q, q); q - d lies in (0, 3q)
  if (f[L - 1] < 0) {
    int32_t c = 0;
#pragma unroll
    for (int i = 0; i < L - 1; ++i) {
      c += q[i] - d[i];
      d[i] = c & kM30;
      c >>= 30;
    }
    d[L - 1] = q[L - 1] - d[L - 1] + c;
  }
  s30_normalise<L>(d, q);
  from_s30<L>(out, d, n);
}

}  // namespace ecc
