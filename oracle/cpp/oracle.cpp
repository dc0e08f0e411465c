// Plain C++ big-integer oracle: ECDSA sign/verify, scalar multiplication and
// naive multi-scalar multiplication on short Weierstrass curves (Eqn 1).
//
// TEST INFRASTRUCTURE ONLY.  Used by the tests (through ctypes) and as the
// timed CPU baseline.  It shares no code with the GPU library: its arithmetic is
// a different algorithm on purpose --
//   * field elements are plain integers (never Montgomery form);
//   * products are schoolbook on 32-bit limbs, reduced by Barrett reduction
//     (Handbook of Applied Cryptography, Algorithm 14.42);
//   * inversion is Fermat's little theorem x^(p-2) (Section 2.2);
//   * points are in Jacobian coordinates x = X/Z^2, y = Y/Z^3 (Section 2.1.2,
//     Table 1), with Z = 0 for the point at infinity;
//   * scalar multiplication is most-significant-bit-first double-and-add (the
//     mirror image of Algorithm 1);
//   * MSM is the definition: the sum of the k_i * P_i.
// ECDSA follows SEC 1 / FIPS 186-4 (the paper states verification is one FPMUL
// plus one UPMUL, Section 5.2).  Work items are spread over std::thread workers.
//
// Byte conventions at this interface: ECDSA integers are 32-byte big-endian,
// public keys 64 bytes (x || y); MSM points and scalars are little-endian
// 32-bit limbs, points (x, y) with m limbs per coordinate, (0, 0) for O.

#include <atomic>
#include <cstdint>
#include <cstring>
#include <thread>
#include <vector>

namespace {

constexpr int MAXL = 12;          // limbs of the largest field (381-bit)
constexpr int WIDE = 2 * MAXL + 4;

struct Field {
  int m = 0;                 // limbs of the modulus
  uint32_t p[MAXL] = {0};
  uint32_t mu[MAXL + 2] = {0};  // floor(2^(64 m) / p), m + 1 limbs (+ slack)
};

// ----------------------------------------------------------------- limbs

int cmp_n(const uint32_t* a, const uint32_t* b, int n) {
  for (int i = n - 1; i >= 0; --i) {
    if (a[i] != b[i]) return a[i] < b[i] ? -1 : 1;
  }
  return 0;
}

uint32_t add_n(uint32_t* r, const uint32_t* a, const uint32_t* b, int n) {
  uint64_t c = 0;
  for (int i = 0; i < n; ++i) {
    c += (uint64_t)a[i] + b[i];
    r[i] = (uint32_t)c;
    c >>= 32;
  }
  return (uint32_t)c;
}

uint32_t sub_n(uint32_t* r, const uint32_t* a, const uint32_t* b, int n) {
  int64_t br = 0;
  for (int i = 0; i < n; ++i) {
    int64_t d = (int64_t)a[i] - b[i] + br;
    r[i] = (uint32_t)d;
    br = d < 0 ? -1 : 0;
  }
  return br ? 1u : 0u;
}

// r[0 .. na+nb) = a * b (schoolbook)
void mul_nn(uint32_t* r, const uint32_t* a, int na, const uint32_t* b, int nb) {
  for (int i = 0; i < na + nb; ++i) r[i] = 0;
  for (int i = 0; i < na; ++i) {
    uint64_t c = 0;
    for (int j = 0; j < nb; ++j) {
      c += (uint64_t)a[i] * b[j] + r[i + j];
      r[i + j] = (uint32_t)c;
      c >>= 32;
    }
    r[i + nb] = (uint32_t)c;
  }
}

bool is_zero(const uint32_t* a, int n) {
  for (int i = 0; i < n; ++i)
    if (a[i]) return false;
  return true;
}

int bitlen_n(const uint32_t* a, int n) {
  for (int i = n - 1; i >= 0; --i)
    if (a[i]) return 32 * i + 32 - __builtin_clz(a[i]);
  return 0;
}

bool bit_n(const uint32_t* a, int i) { return (a[i >> 5] >> (i & 31)) & 1u; }

// ----------------------------------------------------------------- field

void field_init(Field& F, const uint32_t* p, int m) {
  F.m = m;
  for (int i = 0; i < MAXL; ++i) F.p[i] = i < m ? p[i] : 0;
  // mu = floor(2^(64 m) / p) by restoring long division, one bit at a time.
  uint32_t rem[MAXL + 2] = {0};
  uint32_t q[2 * MAXL + 2] = {0};
  uint32_t pp[MAXL + 2] = {0};
  for (int i = 0; i < m; ++i) pp[i] = p[i];
  const int nbits = 64 * m + 1;  // dividend 2^(64 m) has 64 m + 1 bits
  for (int bit = nbits - 1; bit >= 0; --bit) {
    // rem = 2 rem + (bit of dividend)
    uint32_t carry = (bit == 64 * m) ? 1u : 0u;
    for (int i = 0; i < m + 2; ++i) {
      uint32_t nc = rem[i] >> 31;
      rem[i] = (rem[i] << 1) | carry;
      carry = nc;
    }
    if (cmp_n(rem, pp, m + 2) >= 0) {
      sub_n(rem, rem, pp, m + 2);
      q[bit >> 5] |= 1u << (bit & 31);
    }
  }
  for (int i = 0; i < m + 2; ++i) F.mu[i] = q[i];
}

// r = x mod p for x < 2^(64 m) (x has 2m limbs): Barrett reduction.
void field_reduce(const Field& F, uint32_t* r, const uint32_t* x) {
  const int k = F.m;
  uint32_t q2[WIDE + 4];
  // q1 = floor(x / b^(k-1)): k + 1 limbs; q2 = q1 * mu (mu has k + 1 limbs)
  mul_nn(q2, x + (k - 1), k + 1, F.mu, k + 1);
  // q3 = floor(q2 / b^(k+1)): k + 1 limbs
  const uint32_t* q3 = q2 + (k + 1);
  // r1 = x mod b^(k+1); r2 = (q3 * p) mod b^(k+1)
  uint32_t t[WIDE + 4];
  mul_nn(t, q3, k + 1, F.p, k);
  uint32_t rr[MAXL + 2];
  sub_n(rr, x, t, k + 1);  // modulo b^(k+1): a borrow wraps, as the algorithm wants
  uint32_t pp[MAXL + 2] = {0};
  for (int i = 0; i < k; ++i) pp[i] = F.p[i];
  while (cmp_n(rr, pp, k + 1) >= 0) sub_n(rr, rr, pp, k + 1);
  for (int i = 0; i < k; ++i) r[i] = rr[i];
}

struct Fe {
  uint32_t v[MAXL];
};

void fe_set(const Field& F, Fe& r, const uint32_t* a) {
  for (int i = 0; i < MAXL; ++i) r.v[i] = i < F.m ? a[i] : 0;
}

void fe_zero(Fe& r) { std::memset(r.v, 0, sizeof r.v); }

void fe_small(const Field& F, Fe& r, uint32_t s) {
  fe_zero(r);
  r.v[0] = s;
  (void)F;
}

bool fe_is_zero(const Field& F, const Fe& a) { return is_zero(a.v, F.m); }
bool fe_eq(const Field& F, const Fe& a, const Fe& b) { return cmp_n(a.v, b.v, F.m) == 0; }

Fe fe_mul(const Field& F, const Fe& a, const Fe& b) {
  uint32_t t[WIDE];
  std::memset(t, 0, sizeof t);
  mul_nn(t, a.v, F.m, b.v, F.m);
  Fe r;
  fe_zero(r);
  field_reduce(F, r.v, t);
  return r;
}

Fe fe_add(const Field& F, const Fe& a, const Fe& b) {
  Fe r;
  fe_zero(r);
  uint32_t c = add_n(r.v, a.v, b.v, F.m);
  if (c || cmp_n(r.v, F.p, F.m) >= 0) sub_n(r.v, r.v, F.p, F.m);
  return r;
}

Fe fe_sub(const Field& F, const Fe& a, const Fe& b) {
  Fe r;
  fe_zero(r);
  if (sub_n(r.v, a.v, b.v, F.m)) add_n(r.v, r.v, F.p, F.m);
  return r;
}

// x^e mod p, e given as limbs (square-and-multiply, MSB first)
Fe fe_pow(const Field& F, const Fe& x, const uint32_t* e, int elimbs) {
  Fe r;
  fe_small(F, r, 1);
  for (int i = bitlen_n(e, elimbs) - 1; i >= 0; --i) {
    r = fe_mul(F, r, r);
    if (bit_n(e, i)) r = fe_mul(F, r, x);
  }
  return r;
}

// Fermat inversion x^(p-2); 0 maps to 0.
Fe fe_inv(const Field& F, const Fe& x) {
  uint32_t e[MAXL];
  uint32_t two[MAXL] = {2};
  sub_n(e, F.p, two, F.m);
  return fe_pow(F, x, e, F.m);
}

// Reduce an arbitrary m-limb value (possibly >= p) into [0, p).
Fe fe_from_any(const Field& F, const uint32_t* a, int alimbs) {
  uint32_t t[WIDE];
  std::memset(t, 0, sizeof t);
  for (int i = 0; i < alimbs; ++i) t[i] = a[i];
  Fe r;
  fe_zero(r);
  field_reduce(F, r.v, t);
  return r;
}

// ----------------------------------------------------------------- curve

struct CurveDef {
  Field fp, fn;
  Fe a, b, gx, gy;
};

struct Jac {
  Fe X, Y, Z;  // Z = 0 encodes O
};

Jac jac_inf(const Field& F) {
  Jac r;
  fe_small(F, r.X, 1);
  fe_small(F, r.Y, 1);
  fe_zero(r.Z);
  return r;
}

bool jac_is_inf(const Field& F, const Jac& P) { return fe_is_zero(F, P.Z); }

Jac jac_from_affine(const Field& F, const Fe& x, const Fe& y) {
  Jac r;
  r.X = x;
  r.Y = y;
  fe_small(F, r.Z, 1);
  return r;
}

// Doubling for general a: M = 3 X^2 + a Z^4, S = 4 X Y^2,
// X3 = M^2 - 2 S, Y3 = M (S - X3) - 8 Y^4, Z3 = 2 Y Z.
Jac jac_dbl(const CurveDef& C, const Jac& P) {
  const Field& F = C.fp;
  if (jac_is_inf(F, P) || fe_is_zero(F, P.Y)) return jac_inf(F);
  Fe XX = fe_mul(F, P.X, P.X);
  Fe YY = fe_mul(F, P.Y, P.Y);
  Fe YYYY = fe_mul(F, YY, YY);
  Fe ZZ = fe_mul(F, P.Z, P.Z);
  Fe S = fe_mul(F, P.X, YY);
  S = fe_add(F, S, S);
  S = fe_add(F, S, S);
  Fe M = fe_add(F, fe_add(F, XX, XX), XX);
  M = fe_add(F, M, fe_mul(F, C.a, fe_mul(F, ZZ, ZZ)));
  Jac R;
  R.X = fe_sub(F, fe_mul(F, M, M), fe_add(F, S, S));
  Fe Y8 = fe_add(F, YYYY, YYYY);
  Y8 = fe_add(F, Y8, Y8);
  Y8 = fe_add(F, Y8, Y8);
  R.Y = fe_sub(F, fe_mul(F, M, fe_sub(F, S, R.X)), Y8);
  Fe YZ = fe_mul(F, P.Y, P.Z);
  R.Z = fe_add(F, YZ, YZ);
  return R;
}

// General addition: U1 = X1 Z2^2, U2 = X2 Z1^2, S1 = Y1 Z2^3, S2 = Y2 Z1^3,
// H = U2 - U1, r = S2 - S1, X3 = r^2 - H^3 - 2 U1 H^2,
// Y3 = r (U1 H^2 - X3) - S1 H^3, Z3 = Z1 Z2 H.
Jac jac_add(const CurveDef& C, const Jac& P, const Jac& Q) {
  const Field& F = C.fp;
  if (jac_is_inf(F, P)) return Q;
  if (jac_is_inf(F, Q)) return P;
  Fe Z1Z1 = fe_mul(F, P.Z, P.Z);
  Fe Z2Z2 = fe_mul(F, Q.Z, Q.Z);
  Fe U1 = fe_mul(F, P.X, Z2Z2);
  Fe U2 = fe_mul(F, Q.X, Z1Z1);
  Fe S1 = fe_mul(F, P.Y, fe_mul(F, Q.Z, Z2Z2));
  Fe S2 = fe_mul(F, Q.Y, fe_mul(F, P.Z, Z1Z1));
  Fe H = fe_sub(F, U2, U1);
  Fe r = fe_sub(F, S2, S1);
  if (fe_is_zero(F, H)) {
    if (fe_is_zero(F, r)) return jac_dbl(C, P);
    return jac_inf(F);
  }
  Fe HH = fe_mul(F, H, H);
  Fe HHH = fe_mul(F, H, HH);
  Fe V = fe_mul(F, U1, HH);
  Jac R;
  R.X = fe_sub(F, fe_sub(F, fe_mul(F, r, r), HHH), fe_add(F, V, V));
  R.Y = fe_sub(F, fe_mul(F, r, fe_sub(F, V, R.X)), fe_mul(F, S1, HHH));
  R.Z = fe_mul(F, fe_mul(F, P.Z, Q.Z), H);
  return R;
}

void jac_to_affine(const CurveDef& C, const Jac& P, Fe& x, Fe& y, bool& inf) {
  const Field& F = C.fp;
  if (jac_is_inf(F, P)) {
    inf = true;
    fe_zero(x);
    fe_zero(y);
    return;
  }
  inf = false;
  Fe zi = fe_inv(F, P.Z);
  Fe zi2 = fe_mul(F, zi, zi);
  x = fe_mul(F, P.X, zi2);
  y = fe_mul(F, P.Y, fe_mul(F, zi2, zi));
}

// k * P, most-significant bit first; k is klimbs little-endian limbs.
Jac jac_mul(const CurveDef& C, const uint32_t* k, int klimbs, const Jac& P) {
  Jac R = jac_inf(C.fp);
  for (int i = bitlen_n(k, klimbs) - 1; i >= 0; --i) {
    R = jac_dbl(C, R);
    if (bit_n(k, i)) R = jac_add(C, R, P);
  }
  return R;
}

bool affine_on_curve(const CurveDef& C, const Fe& x, const Fe& y) {
  const Field& F = C.fp;
  Fe lhs = fe_mul(F, y, y);
  Fe rhs = fe_add(F, fe_add(F, fe_mul(F, fe_mul(F, x, x), x), fe_mul(F, C.a, x)), C.b);
  return fe_eq(F, lhs, rhs);
}

// ----------------------------------------------------------------- constants

int hexval(char c) {
  if (c >= '0' && c <= '9') return c - '0';
  if (c >= 'a' && c <= 'f') return c - 'a' + 10;
  if (c >= 'A' && c <= 'F') return c - 'A' + 10;
  return -1;
}

void parse_hex(uint32_t* out, int limbs, const char* s) {
  for (int i = 0; i < limbs; ++i) out[i] = 0;
  int len = (int)std::strlen(s);
  int nib = 0;
  for (int i = len - 1; i >= 0; --i) {
    int v = hexval(s[i]);
    if (v < 0) continue;
    out[nib >> 3] |= (uint32_t)v << (4 * (nib & 7));
    ++nib;
  }
}

struct CurveHex {
  int m;
  const char *p, *a, *b, *gx, *gy, *n;
};

// Standard parameters (SEC 2 for secp256k1 and secp256r1 = P-256; BN254 G1 from
// u = 0x44E992B44A6909F1; BLS12-381 G1 from x = -0xd201000000010000; the SM2
// recommended curve of GB/T 32918.5).
const CurveHex kCurves[5] = {
    {8, "fffffffffffffffffffffffffffffffffffffffffffffffffffffffefffffc2f", "0", "7",
     "79be667ef9dcbbac55a06295ce870b07029bfcdb2dce28d959f2815b16f81798",
     "483ada7726a3c4655da4fbfc0e1108a8fd17b448a68554199c47d08ffb10d4b8",
     "fffffffffffffffffffffffffffffffebaaedce6af48a03bbfd25e8cd0364141"},
    {8, "ffffffff00000001000000000000000000000000ffffffffffffffffffffffff",
     "ffffffff00000001000000000000000000000000fffffffffffffffffffffffc",
     "5ac635d8aa3a93e7b3ebbd55769886bc651d06b0cc53b0f63bce3c3e27d2604b",
     "6b17d1f2e12c4247f8bce6e563a440f277037d812deb33a0f4a13945d898c296",
     "4fe342e2fe1a7f9b8ee7eb4a7c0f9e162bce33576b315ececbb6406837bf51f5",
     "ffffffff00000000ffffffffffffffffbce6faada7179e84f3b9cac2fc632551"},
    {8, "30644e72e131a029b85045b68181585d97816a916871ca8d3c208c16d87cfd47", "0", "3", "1", "2",
     "30644e72e131a029b85045b68181585d2833e84879b9709143e1f593f0000001"},
    {12,
     "1a0111ea397fe69a4b1ba7b6434bacd764774b84f38512bf6730d2a0f6b0f6241eabfffeb153ffffb9feffffffffaaab",
     "0", "4",
     "17f1d3a73197d7942695638c4fa9ac0fc3688c4f9774b905a14e3a3f171bac586c55e83ff97a1aeffb3af00adb22c6bb",
     "08b3f481e3aaa0f1a09e30ed741d8ae4fcf5e095d5d00af600db18cb2c04b3edd03cc744a2888ae40caa232946c5e7e1",
     "73eda753299d7d483339d80809a1d80553bda402fffe5bfeffffffff00000001"},
    {8, "fffffffeffffffffffffffffffffffffffffffff00000000ffffffffffffffff",
     "fffffffeffffffffffffffffffffffffffffffff00000000fffffffffffffffc",
     "28e9fa9e9d9f5e344d5a9e4bcf6509a7f39789f515ab8f92ddbcbd414d940e93",
     "32c4ae2c1f1981195f9904466a39c9948fe30bbff2660be1715a4589334c74c7",
     "bc3736a2f4f6779c59bdcee36b692153d0a9877cc62a474002df32e52139f0a0",
     "fffffffeffffffffffffffffffffffff7203df6b21c6052b53bbf40939d54123"},
};

CurveDef g_curves[5];
std::atomic<bool> g_ready{false};

void init_curves() {
  if (g_ready.load()) return;
  static std::atomic_flag busy = ATOMIC_FLAG_INIT;
  while (busy.test_and_set()) {
  }
  if (!g_ready.load()) {
    for (int c = 0; c < 5; ++c) {
      const CurveHex& h = kCurves[c];
      uint32_t t[MAXL];
      parse_hex(t, h.m, h.p);
      field_init(g_curves[c].fp, t, h.m);
      parse_hex(t, 8, h.n);
      field_init(g_curves[c].fn, t, 8);
      parse_hex(t, h.m, h.a);
      fe_set(g_curves[c].fp, g_curves[c].a, t);
      parse_hex(t, h.m, h.b);
      fe_set(g_curves[c].fp, g_curves[c].b, t);
      parse_hex(t, h.m, h.gx);
      fe_set(g_curves[c].fp, g_curves[c].gx, t);
      parse_hex(t, h.m, h.gy);
      fe_set(g_curves[c].fp, g_curves[c].gy, t);
    }
    g_ready.store(true);
  }
  busy.clear();
}

// ----------------------------------------------------------------- bytes

void be32_to_limbs(uint32_t* out, const uint8_t* be) {  // 32 bytes -> 8 limbs
  for (int i = 0; i < 8; ++i) {
    const uint8_t* q = be + 32 - 4 * (i + 1);
    out[i] = ((uint32_t)q[0] << 24) | ((uint32_t)q[1] << 16) | ((uint32_t)q[2] << 8) | q[3];
  }
}

void limbs_to_be32(uint8_t* be, const uint32_t* v) {
  for (int i = 0; i < 8; ++i) {
    uint8_t* q = be + 32 - 4 * (i + 1);
    q[0] = (uint8_t)(v[i] >> 24);
    q[1] = (uint8_t)(v[i] >> 16);
    q[2] = (uint8_t)(v[i] >> 8);
    q[3] = (uint8_t)v[i];
  }
}

template <class Fn>
void parallel_for(size_t n, int threads, Fn fn) {
  if (threads <= 1 || n < 2) {
    for (size_t i = 0; i < n; ++i) fn(i, 0);
    return;
  }
  if ((size_t)threads > n) threads = (int)n;
  std::atomic<size_t> next{0};
  std::vector<std::thread> pool;
  for (int t = 0; t < threads; ++t) {
    pool.emplace_back([&, t] {
      for (;;) {
        size_t i = next.fetch_add(1);
        if (i >= n) break;
        fn(i, t);
      }
    });
  }
  for (auto& th : pool) th.join();
}

bool verify_one(const CurveDef& C, const uint8_t* h, const uint8_t* rb, const uint8_t* sb,
                const uint8_t* pub) {
  const Field& Fn = C.fn;
  const Field& Fp = C.fp;
  uint32_t e[8], r[8], s[8], qx[8], qy[8];
  be32_to_limbs(e, h);
  be32_to_limbs(r, rb);
  be32_to_limbs(s, sb);
  be32_to_limbs(qx, pub);
  be32_to_limbs(qy, pub + 32);
  // 1. r, s in [1, n-1]
  if (is_zero(r, 8) || is_zero(s, 8)) return false;
  if (cmp_n(r, Fn.p, 8) >= 0 || cmp_n(s, Fn.p, 8) >= 0) return false;
  // 2. Q on the curve, coordinates canonical, Q != O
  if (cmp_n(qx, Fp.p, 8) >= 0 || cmp_n(qy, Fp.p, 8) >= 0) return false;
  Fe X, Y;
  fe_set(Fp, X, qx);
  fe_set(Fp, Y, qy);
  if (fe_is_zero(Fp, X) && fe_is_zero(Fp, Y)) return false;
  if (!affine_on_curve(C, X, Y)) return false;
  // 3-4. w = s^-1, u1 = e w, u2 = r w (mod n)
  Fe S, Rn, E;
  fe_set(Fn, S, s);
  fe_set(Fn, Rn, r);
  E = fe_from_any(Fn, e, 8);
  Fe w = fe_inv(Fn, S);
  Fe u1 = fe_mul(Fn, E, w);
  Fe u2 = fe_mul(Fn, Rn, w);
  // 5. R = u1 G + u2 Q
  Jac G = jac_from_affine(Fp, C.gx, C.gy);
  Jac Q = jac_from_affine(Fp, X, Y);
  Jac R = jac_add(C, jac_mul(C, u1.v, 8, G), jac_mul(C, u2.v, 8, Q));
  Fe rx, ry;
  bool inf;
  jac_to_affine(C, R, rx, ry, inf);
  if (inf) return false;
  // 6. x_R mod n == r
  Fe xr = fe_from_any(Fn, rx.v, 8);
  return cmp_n(xr.v, r, 8) == 0;
}

}  // namespace

extern "C" {

// Returns 0 on success, -1 on a bad curve id.
int orc_verify(int curve, size_t n, const uint8_t* hash, const uint8_t* r, const uint8_t* s,
               const uint8_t* pub, uint8_t* ok, int threads) {
  if (curve != 0 && curve != 1 && curve != 4) return -1;
  init_curves();
  const CurveDef& C = g_curves[curve];
  parallel_for(n, threads, [&](size_t i, int) {
    ok[i] = verify_one(C, hash + 32 * i, r + 32 * i, s + 32 * i, pub + 64 * i) ? 1 : 0;
  });
  return 0;
}

// Signs with given private keys d, hashes e and nonces k (32-byte big-endian).
// Writes r, s (32 bytes each) and the public key d*G (64 bytes).  An item whose
// nonce gives r = 0 or s = 0 gets r = s = 0 (the caller redraws).
int orc_sign(int curve, size_t n, const uint8_t* d, const uint8_t* e, const uint8_t* k,
             uint8_t* r_out, uint8_t* s_out, uint8_t* pub_out, int threads) {
  if (curve != 0 && curve != 1 && curve != 4) return -1;
  init_curves();
  const CurveDef& C = g_curves[curve];
  parallel_for(n, threads, [&](size_t i, int) {
    const Field& Fn = C.fn;
    uint32_t dl[8], el[8], kl[8];
    be32_to_limbs(dl, d + 32 * i);
    be32_to_limbs(el, e + 32 * i);
    be32_to_limbs(kl, k + 32 * i);
    Jac G = jac_from_affine(C.fp, C.gx, C.gy);
    Fe px, py, rx, ry;
    bool inf;
    jac_to_affine(C, jac_mul(C, dl, 8, G), px, py, inf);
    limbs_to_be32(pub_out + 64 * i, px.v);
    limbs_to_be32(pub_out + 64 * i + 32, py.v);
    jac_to_affine(C, jac_mul(C, kl, 8, G), rx, ry, inf);
    Fe r = fe_from_any(Fn, rx.v, 8);
    Fe K = fe_from_any(Fn, kl, 8);
    Fe D = fe_from_any(Fn, dl, 8);
    Fe E = fe_from_any(Fn, el, 8);
    Fe s = fe_mul(Fn, fe_inv(Fn, K), fe_add(Fn, E, fe_mul(Fn, r, D)));
    if (fe_is_zero(Fn, r) || fe_is_zero(Fn, s)) {
      fe_zero(r);
      fe_zero(s);
    }
    limbs_to_be32(r_out + 32 * i, r.v);
    limbs_to_be32(s_out + 32 * i, s.v);
  });
  return 0;
}

// out_i = k_i * P_i (affine, (0,0) for O).  Scalars: 8 limbs; points: 2m limbs.
int orc_scalar_mul(int curve, size_t n, const uint32_t* k, const uint32_t* pts, uint32_t* out,
                   int threads) {
  if (curve < 0 || curve > 4) return -1;
  init_curves();
  const CurveDef& C = g_curves[curve];
  const int m = C.fp.m;
  parallel_for(n, threads, [&](size_t i, int) {
    Fe x, y;
    fe_set(C.fp, x, pts + 2 * m * i);
    fe_set(C.fp, y, pts + 2 * m * i + m);
    Jac P = (fe_is_zero(C.fp, x) && fe_is_zero(C.fp, y)) ? jac_inf(C.fp)
                                                          : jac_from_affine(C.fp, x, y);
    Fe rx, ry;
    bool inf;
    jac_to_affine(C, jac_mul(C, k + 8 * i, 8, P), rx, ry, inf);
    for (int j = 0; j < m; ++j) {
      out[2 * m * i + j] = rx.v[j];
      out[2 * m * i + m + j] = ry.v[j];
    }
  });
  return 0;
}

// out = sum_i k_i * P_i (affine, (0,0) for O).
int orc_msm(int curve, size_t n, const uint32_t* pts, const uint32_t* k, uint32_t* out,
            int threads) {
  if (curve < 0 || curve > 4) return -1;
  init_curves();
  const CurveDef& C = g_curves[curve];
  const int m = C.fp.m;
  if (threads < 1) threads = 1;
  std::vector<Jac> partial(threads, jac_inf(C.fp));
  parallel_for(n, threads, [&](size_t i, int t) {
    Fe x, y;
    fe_set(C.fp, x, pts + 2 * m * i);
    fe_set(C.fp, y, pts + 2 * m * i + m);
    if (fe_is_zero(C.fp, x) && fe_is_zero(C.fp, y)) return;
    Jac P = jac_from_affine(C.fp, x, y);
    partial[t] = jac_add(C, partial[t], jac_mul(C, k + 8 * i, 8, P));
  });
  Jac acc = jac_inf(C.fp);
  for (auto& J : partial) acc = jac_add(C, acc, J);
  Fe rx, ry;
  bool inf;
  jac_to_affine(C, acc, rx, ry, inf);
  for (int j = 0; j < m; ++j) {
    out[j] = rx.v[j];
    out[m + j] = ry.v[j];
  }
  return 0;
}

// Field helpers for pinning the bigint layer against Python integers:
// which = 0 for the base field p, 1 for the group order n.
int orc_fe_mul(int curve, int which, size_t n, const uint32_t* a, const uint32_t* b,
               uint32_t* out) {
  if (curve < 0 || curve > 4) return -1;
  init_curves();
  const Field& F = which ? g_curves[curve].fn : g_curves[curve].fp;
  for (size_t i = 0; i < n; ++i) {
    Fe x, y;
    fe_set(F, x, a + F.m * i);
    fe_set(F, y, b + F.m * i);
    Fe r = fe_mul(F, x, y);
    for (int j = 0; j < F.m; ++j) out[F.m * i + j] = r.v[j];
  }
  return 0;
}

int orc_fe_inv(int curve, int which, size_t n, const uint32_t* a, uint32_t* out) {
  if (curve < 0 || curve > 4) return -1;
  init_curves();
  const Field& F = which ? g_curves[curve].fn : g_curves[curve].fp;
  for (size_t i = 0; i < n; ++i) {
    Fe x;
    fe_set(F, x, a + F.m * i);
    Fe r = fe_inv(F, x);
    for (int j = 0; j < F.m; ++j) out[F.m * i + j] = r.v[j];
  }
  return 0;
}

int orc_limbs(int curve) {
  if (curve < 0 || curve > 4) return -1;
  return kCurves[curve].m;
}

}  // extern "C"
