// Batched ECDSA verification (the ECC algorithm layer over the EC operators).
//
// Verification of (e, r, s, Q) computes R = u1 G + u2 Q with w = s^-1 mod n,
// u1 = e w, u2 = r w, and accepts iff R != O and x_R mod n == r.  The paper
// states verification as one fixed-point multiplication (u1 G) plus one
// unknown-point multiplication (u2 Q) (Section 5.2); both are run here as
// batched affine operations sharing one inversion per round (Section 3.1):
//
//   * u1 G: fixed-base comb over a precomputed table TG[j][v] = v 2^(8j) G
//     (8-bit windows, 32 table additions, no doublings; Section 2.1.1 on FPMUL);
//   * u2 Q: signed kQW-bit fixed windows, most significant first, with a
//     per-item table {Q, 2Q, ..., 2^(kQW-1) Q} built in batched rounds of at most
//     four additions; (kQDigits - 1) x kQW doublings and kQDigits additions.
//     Every lane follows the same schedule (digit 0 is a no-op addition of O),
//     so warps never diverge on the scalar.  A wider window trades table
//     rounds and memory for fewer main-loop rounds, each of which costs one
//     CTA-wide inversion.
//   * the 32 G-table additions ride in the last 32 addition rounds, so their
//     denominators share those rounds' chains (the fusion idea of Section 3.4).
//
// Each CTA owns a contiguous slice of the batch for the whole verification:
// every round is compress -> per-CTA inversion -> DCWPA over the same slice, so
// the kernel runs all rounds in one launch with no grid-wide synchronisation.
#pragma once
#include "ops.cuh"

namespace ecc {

template <class C>
struct VerifyArgs {
  using Fp = typename C::Fp;
  using Fn = typename C::Fn;
  size_t n;
  const uint32_t* hash;  // n x 32 bytes big-endian (read as 8 words)
  const uint32_t* r;
  const uint32_t* s;
  const uint32_t* pub;   // n x 64 bytes (x || y) big-endian
  uint8_t* ok;
  SoA<Fn> S, E, Rn;      // s, e mod n, r in Montgomery form (mod n)
  PtSoA<Fp> TQ;          // per-item table, element (k - 1) * n + i holds k Q_i, k <= kQTable
  PtSoA<Fp> AQ, AG;      // accumulators of u2 Q and u1 G
  SoA<Fp> M;             // running products of the compress step
  int8_t* D2;            // signed kQW-bit digits of u2: D2[w * n + i], w < kQDigits
  uint8_t* U1B;          // bytes of u1: U1B[j * n + i], j = 0..31
  uint8_t* status;       // 1 = well-formed input
  PtSoA<Fp> TG;          // fixed-base table, entry j * 256 + v
  size_t per_cta;
};

// Signed radix-2^kQW digits of a 256-bit scalar: ceil(256 / kQW) digits, plus
// one when the top digit's bits (256 mod kQW, or kQW) can reach 2^(kQW-1) - 1
// and so carry out.
constexpr int kQW = 5;
constexpr int kQTable = 1 << (kQW - 1);
constexpr int kQTopBits = 256 - kQW * ((256 - 1) / kQW);
constexpr int kQDigits = (256 + kQW - 1) / kQW + ((1 << kQTopBits) - 1 + 1 >= (1 << (kQW - 1)) ? 1 : 0);
static_assert(kQDigits >= 32, "the G additions ride in 32 addition rounds");

ECC_DEV uint32_t bswap32(uint32_t x) { return __byte_perm(x, 0, 0x0123); }

// 8 little-endian limbs from 32 big-endian bytes (word-aligned)
ECC_DEV void load_be256(uint32_t* out, const uint32_t* src) {
#pragma unroll
  for (int k = 0; k < 8; ++k) out[k] = bswap32(src[7 - k]);
}

// a < b for 8-limb integers
ECC_DEV bool lt256(const uint32_t* a, const uint32_t* b) {
  uint32_t t = ptx::sub_cc(a[0], b[0]);
#pragma unroll
  for (int k = 1; k < 8; ++k) t = ptx::subc_cc(a[k], b[k]);
  (void)t;
  return ptx::subc(0, 0) != 0;
}

ECC_DEV bool is_zero256(const uint32_t* a) {
  uint32_t acc = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) acc |= a[k];
  return acc == 0;
}

ECC_DEV void sub256(uint32_t* r, const uint32_t* a, const uint32_t* b) {
  r[0] = ptx::sub_cc(a[0], b[0]);
#pragma unroll
  for (int k = 1; k < 7; ++k) r[k] = ptx::subc_cc(a[k], b[k]);
  r[7] = ptx::subc(a[7], b[7]);
}

template <class C>
ECC_DEV bool on_curve_mont(const uint32_t* x, const uint32_t* y) {
  using F = typename C::Fp;
  constexpr int N = F::N;
  uint32_t l[N], rr[N], t[N];
  mont_sqr<F>(l, y);
  mont_sqr<F>(rr, x);
  mont_mul<F>(rr, rr, x);
  if (!C::A_ZERO) {
    uint32_t a[N];
    curve_a<C>(a);
    mont_mul<F>(t, a, x);
    fe_add<F>(rr, rr, t);
  }
#pragma unroll
  for (int k = 0; k < N; ++k) t[k] = C::b(k);
  fe_add<F>(rr, rr, t);
  return fe_eq<F>(l, rr);
}

// Parse, range-check and convert one slice of the batch (SEC 1 steps 1-3).
template <class C, int BLOCK>
__device__ void verify_prep(const VerifyArgs<C>& a, size_t begin, size_t end) {
  using Fp = typename C::Fp;
  using Fn = typename C::Fn;
  for (size_t i = begin + threadIdx.x; i < end; i += BLOCK) {
    uint32_t e[8], r[8], s[8], qx[8], qy[8], nn[8], pp[8];
    load_be256(e, a.hash + 8 * i);
    load_be256(r, a.r + 8 * i);
    load_be256(s, a.s + 8 * i);
    load_be256(qx, a.pub + 16 * i);
    load_be256(qy, a.pub + 16 * i + 8);
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      nn[k] = C::n(k);
      pp[k] = Fp::p(k);
    }
    bool valid = !is_zero256(r) && !is_zero256(s) && lt256(r, nn) && lt256(s, nn);
    valid = valid && lt256(qx, pp) && lt256(qy, pp) && !(is_zero256(qx) && is_zero256(qy));
    uint32_t xm[8], ym[8];
    to_mont<Fp>(xm, qx);
    to_mont<Fp>(ym, qy);
    valid = valid && on_curve_mont<C>(xm, ym);
    if (!lt256(e, nn)) sub256(e, e, nn);  // e < 2^256 < 2n
    if (!valid) {
      // keep the arithmetic well-defined; the result is discarded
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        r[k] = k == 0 ? 1u : 0u;
        s[k] = r[k];
        qx[k] = C::gx(k);
        qy[k] = C::gy(k);
      }
      to_mont<Fp>(xm, qx);
      to_mont<Fp>(ym, qy);
    }
    uint32_t t[8];
    to_mont<Fn>(t, s);
    a.S.store(i, t);
    to_mont<Fn>(t, e);
    a.E.store(i, t);
    to_mont<Fn>(t, r);
    a.Rn.store(i, t);
    a.TQ.store(i, xm, ym);
    uint32_t z[8];
    fe_set_zero<Fp>(z);
    a.AQ.store(i, z, z);
    a.AG.store(i, z, z);
    a.status[i] = valid ? 1 : 0;
  }
}

// w = s^-1 (batched over n), u1 = e w, u2 = r w; digits of u2, bytes of u1.
template <class C>
struct ScalarRound {
  using Fn = typename C::Fn;
  static constexpr int OPS = 1;
  const VerifyArgs<C>* a;
  ECC_DEV void den_c(size_t i, int, uint32_t* d) { a->S.load(i, d); }
  ECC_DEV void den_d(size_t i, int, uint32_t* d) { a->S.load(i, d); }
  ECC_DEV void finish(size_t i, const uint32_t (*inv)[Fn::N]) {
    const size_t n = a->n;
    uint32_t t[8], u[8];
    a->E.load(i, t);
    mont_mul<Fn>(u, t, inv[0]);
    from_mont<Fn>(u, u);
#pragma unroll
    for (int j = 0; j < 32; ++j) a->U1B[j * n + i] = (uint8_t)(u[j >> 2] >> (8 * (j & 3)));
    a->Rn.load(i, t);
    mont_mul<Fn>(u, t, inv[0]);
    from_mont<Fn>(u, u);
    int carry = 0;
#pragma unroll
    for (int w = 0; w < kQDigits; ++w) {
      // bits [kQW w, kQW w + kQW) of u (zero above bit 255)
      const int pos = kQW * w, word = pos >> 5, sh = pos & 31;
      uint64_t bits = word < 8 ? u[word] : 0u;
      if (word + 1 < 8) bits |= (uint64_t)u[word + 1] << 32;
      const int v = (int)((bits >> sh) & (uint64_t)(kQTable * 2 - 1)) + carry;
      carry = v >= kQTable ? 1 : 0;
      a->D2[w * n + i] = (int8_t)(v - 2 * kQTable * carry);
    }
  }
};

// Per-item table {Q, ..., kQTable Q}: a round makes OPS consecutive multiples
// k = K0 .. K0 + OPS - 1 as B Q + (k - B) Q with B the largest power of two
// below K0 (2Q = Q + Q by the doubling branch of the addition): 2Q; 3Q, 4Q;
// 5Q..8Q; 9Q..12Q, 13Q..16Q; ...
template <class C, int K0, int OPS_>
struct TableRound {
  using F = typename C::Fp;
  static constexpr int N = F::N;
  static constexpr int OPS = OPS_;
  static constexpr int B = K0 <= 2 ? 1 : (K0 <= 4 ? 2 : (K0 <= 8 ? 4 : (K0 <= 16 ? 8 : 16)));
  const VerifyArgs<C>* a;
  int kind[OPS];
  ECC_DEV static void op(int j, int& dst, int& s1, int& s2) {
    // multiples k of Q are stored at table index k - 1
    dst = K0 + j;
    s1 = B;
    s2 = K0 + j - B;
  }
  ECC_DEV void operands(size_t i, int j, uint32_t* xp, uint32_t* yp, uint32_t* xt, uint32_t* yt) {
    int dst, s1, s2;
    op(j, dst, s1, s2);
    a->TQ.load((s1 - 1) * a->n + i, xp, yp);
    a->TQ.load((s2 - 1) * a->n + i, xt, yt);
  }
  ECC_DEV void den_c(size_t i, int j, uint32_t* d) {
    uint32_t xp[N], yp[N], xt[N], yt[N];
    operands(i, j, xp, yp, xt, yt);
    kind[j] = add_den<C>(d, xp, yp, xt, yt);
  }
  ECC_DEV void den_d(size_t i, int j, uint32_t* d) { den_c(i, j, d); }
  ECC_DEV void finish(size_t i, const uint32_t (*inv)[N]) {
#pragma unroll
    for (int j = 0; j < OPS; ++j) {
      uint32_t xp[N], yp[N], xt[N], yt[N], xr[N], yr[N];
      operands(i, j, xp, yp, xt, yt);
      add_finish<C>(xr, yr, kind[j], inv[j], xp, yp, xt, yt);
      int dst, s1, s2;
      op(j, dst, s1, s2);
      a->TQ.store((dst - 1) * a->n + i, xr, yr);
    }
  }
};

// AQ = 2 AQ
template <class C>
struct DblRound {
  using F = typename C::Fp;
  static constexpr int N = F::N;
  static constexpr int OPS = 1;
  const VerifyArgs<C>* a;
  bool live;
  ECC_DEV void den_c(size_t i, int, uint32_t* d) {
    uint32_t y[N];
    a->AQ.y.load(i, y);
    live = dbl_den<C>(d, y);
  }
  ECC_DEV void den_d(size_t i, int j, uint32_t* d) { den_c(i, j, d); }
  ECC_DEV void finish(size_t i, const uint32_t (*inv)[N]) {
    uint32_t x[N], y[N];
    a->AQ.load(i, x, y);
    dbl_finish<C>(x, y, live, inv[0], x, y);
    a->AQ.store(i, x, y);
  }
};

// AQ += d_w * Q (signed digit, table lookup) and, when GADD, AG += TG[jg][byte]
template <class C, bool GADD>
struct AddRound {
  using F = typename C::Fp;
  static constexpr int N = F::N;
  static constexpr int OPS = GADD ? 2 : 1;
  const VerifyArgs<C>* a;
  int w, jg;
  int kind[OPS];
  ECC_DEV void operands(size_t i, int j, uint32_t* xp, uint32_t* yp, uint32_t* xt, uint32_t* yt) {
    const size_t n = a->n;
    if (j == 0) {
      a->AQ.load(i, xp, yp);
      const int d = a->D2[w * n + i];
      if (d == 0) {
        fe_set_zero<F>(xt);
        fe_set_zero<F>(yt);
      } else {
        const int m = d < 0 ? -d : d;
        a->TQ.load((m - 1) * n + i, xt, yt);
        if (d < 0) fe_neg<F>(yt, yt);
      }
    } else {
      a->AG.load(i, xp, yp);
      const int v = a->U1B[jg * n + i];
      if (v == 0) {
        fe_set_zero<F>(xt);
        fe_set_zero<F>(yt);
      } else {
        a->TG.load(jg * 256 + v, xt, yt);
      }
    }
  }
  ECC_DEV void den_c(size_t i, int j, uint32_t* d) {
    uint32_t xp[N], yp[N], xt[N], yt[N];
    operands(i, j, xp, yp, xt, yt);
    kind[j] = add_den<C>(d, xp, yp, xt, yt);
  }
  ECC_DEV void den_d(size_t i, int j, uint32_t* d) { den_c(i, j, d); }
  ECC_DEV void finish(size_t i, const uint32_t (*inv)[N]) {
#pragma unroll
    for (int j = 0; j < OPS; ++j) {
      uint32_t xp[N], yp[N], xt[N], yt[N], xr[N], yr[N];
      operands(i, j, xp, yp, xt, yt);
      add_finish<C>(xr, yr, kind[j], inv[j], xp, yp, xt, yt);
      if (j == 0) {
        a->AQ.store(i, xr, yr);
      } else {
        a->AG.store(i, xr, yr);
      }
    }
  }
};

// R = AG + AQ; ok = well-formed && R != O && x_R mod n == r (SEC 1 steps 5-6)
template <class C>
struct FinalRound {
  using F = typename C::Fp;
  using Fn = typename C::Fn;
  static constexpr int N = F::N;
  static constexpr int OPS = 1;
  const VerifyArgs<C>* a;
  int kind;
  ECC_DEV void den_c(size_t i, int, uint32_t* d) {
    uint32_t xp[N], yp[N], xt[N], yt[N];
    a->AG.load(i, xp, yp);
    a->AQ.load(i, xt, yt);
    kind = add_den<C>(d, xp, yp, xt, yt);
  }
  ECC_DEV void den_d(size_t i, int j, uint32_t* d) { den_c(i, j, d); }
  ECC_DEV void finish(size_t i, const uint32_t (*inv)[N]) {
    uint32_t xp[N], yp[N], xt[N], yt[N], xr[N], yr[N];
    a->AG.load(i, xp, yp);
    a->AQ.load(i, xt, yt);
    add_finish<C>(xr, yr, kind, inv[0], xp, yp, xt, yt);
    const bool inf = pt_is_inf<F>(xr, yr);
    from_mont<F>(xr, xr);
    uint32_t nn[8], r[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) nn[k] = C::n(k);
    if (!lt256(xr, nn)) sub256(xr, xr, nn);  // x_R < p < 2n
    a->Rn.load(i, r);
    from_mont<Fn>(r, r);
    uint32_t diff = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) diff |= xr[k] ^ r[k];
    a->ok[i] = (a->status[i] && !inf && diff == 0) ? 1 : 0;
  }
};

// CL > 1: launched in clusters of CL CTAs that share each round's inversion
// (cta_invert); every CTA runs the same rounds, as that requires.
template <class C, int BLOCK, int CL = 1>
__global__ void __launch_bounds__(BLOCK, kGasResidentThreads / BLOCK) k_verify(VerifyArgs<C> a) {
  using Fp = typename C::Fp;
  using Fn = typename C::Fn;
  static_assert(Fp::N == 8 && Fn::N == 8, "256-bit curves");
  auto& sm = gas_smem<Fp::N, BLOCK>();
  const size_t begin = blockIdx.x * a.per_cta;
  size_t end = begin + a.per_cta < a.n ? begin + a.per_cta : a.n;
  if (end < begin) end = begin;

  verify_prep<C, BLOCK>(a, begin, end);
  {
    ScalarRound<C> rd{&a};
    batch_round<Fn, BLOCK, CL>(rd, begin, end, SoA<Fn>{a.M.vec, a.M.stride}, sm);
  }
  {
    TableRound<C, 2, 1> r1{&a};
    batch_round<Fp, BLOCK, CL>(r1, begin, end, a.M, sm);
    TableRound<C, 3, 2> r2{&a};
    batch_round<Fp, BLOCK, CL>(r2, begin, end, a.M, sm);
    TableRound<C, 5, 4> r3{&a};
    batch_round<Fp, BLOCK, CL>(r3, begin, end, a.M, sm);
    if (kQTable >= 16) {
      TableRound<C, 9, 4> r4{&a};
      batch_round<Fp, BLOCK, CL>(r4, begin, end, a.M, sm);
      TableRound<C, 13, 4> r5{&a};
      batch_round<Fp, BLOCK, CL>(r5, begin, end, a.M, sm);
    }
    if (kQTable >= 32) {
      TableRound<C, 17, 4> r6{&a};
      batch_round<Fp, BLOCK, CL>(r6, begin, end, a.M, sm);
      TableRound<C, 21, 4> r7{&a};
      batch_round<Fp, BLOCK, CL>(r7, begin, end, a.M, sm);
      TableRound<C, 25, 4> r8{&a};
      batch_round<Fp, BLOCK, CL>(r8, begin, end, a.M, sm);
      TableRound<C, 29, 4> r9{&a};
      batch_round<Fp, BLOCK, CL>(r9, begin, end, a.M, sm);
    }
  }
  for (int w = kQDigits - 1; w >= 0; --w) {
    if (w < kQDigits - 1) {
      for (int k = 0; k < kQW; ++k) {
        DblRound<C> rd{&a};
        batch_round<Fp, BLOCK, CL>(rd, begin, end, a.M, sm);
      }
    }
    if (w < 32) {  // G-table window jg = w rides along
      AddRound<C, true> rd{&a, w, w};
      batch_round<Fp, BLOCK, CL>(rd, begin, end, a.M, sm);
    } else {
      AddRound<C, false> rd{&a, w, 0};
      batch_round<Fp, BLOCK, CL>(rd, begin, end, a.M, sm);
    }
  }
  FinalRound<C> rf{&a};
  batch_round<Fp, BLOCK, CL>(rf, begin, end, a.M, sm);
}

}  // namespace ecc
