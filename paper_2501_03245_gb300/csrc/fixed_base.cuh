// Batched fixed-point multiplication (FPMUL, Section 2.1.1 / Table 5) and
// batched ECDSA signing (Section 5.2: one modinv plus one FPMUL).
//
// FPMUL k G uses the precomputed table TG[j][v] = v 2^(8j) G: with k written in
// bytes k_j, k G = sum_j TG[j][k_j], i.e. 32 batched affine additions and no
// doublings (the table removes the PDBL of Algorithm 1).  Each CTA owns a slice
// of the batch for all rounds, as in the verification kernel.
#pragma once
#include "verify.cuh"

namespace ecc {

template <class C>
struct FixedArgs {
  using Fp = typename C::Fp;
  using Fn = typename C::Fn;
  size_t n;
  int mode;                 // 0: FPMUL (scalars as LE limbs), 1: ECDSA sign
  const uint32_t* k;        // mode 0: n x 8 LE limbs; mode 1: n x 32 BE bytes (nonce)
  const uint32_t* d;        // mode 1: private keys, 32 BE bytes
  const uint32_t* e;        // mode 1: hashes, 32 BE bytes
  uint32_t* out_pt;         // mode 0: n x 2N LE limbs (affine, (0,0) = O)
  uint32_t* out_r;          // mode 1: n x 32 BE bytes
  uint32_t* out_s;          // mode 1: n x 32 BE bytes
  uint32_t* out_pub;        // mode 1: n x 64 BE bytes
  uint8_t* KB;              // bytes of the nonce / scalar: KB[j * n + i]
  uint8_t* DB;              // bytes of the private key (mode 1)
  PtSoA<Fp> AK, AD;         // accumulators k G and d G
  SoA<Fp> M;
  SoA<Fn> KN, EN, DN;       // mode 1: k, e, d in Montgomery form mod n
  uint8_t* status;
  PtSoA<Fp> TG;
  size_t per_cta;
};

ECC_DEV void store_be256(uint32_t* dst, const uint32_t* v) {
#pragma unroll
  for (int k = 0; k < 8; ++k) dst[7 - k] = bswap32(v[k]);
}

template <class C, int NOPS>
struct CombRound {
  using F = typename C::Fp;
  static constexpr int N = F::N;
  static constexpr int OPS = NOPS;
  const FixedArgs<C>* a;
  int jg;
  int kind[OPS];
  ECC_DEV void operands(size_t i, int j, uint32_t* xp, uint32_t* yp, uint32_t* xt, uint32_t* yt) {
    const PtSoA<F>& acc = j == 0 ? a->AK : a->AD;
    const uint8_t* bytes = j == 0 ? a->KB : a->DB;
    acc.load(i, xp, yp);
    const int v = bytes[jg * a->n + i];
    if (v == 0) {
      fe_set_zero<F>(xt);
      fe_set_zero<F>(yt);
    } else {
      a->TG.load(jg * 256 + v, xt, yt);
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
      (j == 0 ? a->AK : a->AD).store(i, xr, yr);
    }
  }
};

// s = k^-1 (e + r d) mod n with r = x(kG) mod n; public key d G.
template <class C>
struct SignRound {
  using Fp = typename C::Fp;
  using Fn = typename C::Fn;
  static constexpr int OPS = 1;
  const FixedArgs<C>* a;
  ECC_DEV void den_c(size_t i, int, uint32_t* d) { a->KN.load(i, d); }
  ECC_DEV void den_d(size_t i, int, uint32_t* d) { a->KN.load(i, d); }
  ECC_DEV void finish(size_t i, const uint32_t (*inv)[Fn::N]) {
    uint32_t x[8], y[8], r[8], t[8], s[8], nn[8];
    a->AK.load(i, x, y);
    from_mont<Fp>(x, x);
#pragma unroll
    for (int k = 0; k < 8; ++k) nn[k] = C::n(k);
    if (!lt256(x, nn)) sub256(x, x, nn);  // x < p < 2n
    fe_copy<Fn>(r, x);
    to_mont<Fn>(t, r);
    uint32_t dm[8], em[8];
    a->DN.load(i, dm);
    a->EN.load(i, em);
    mont_mul<Fn>(t, t, dm);
    fe_add<Fn>(t, t, em);
    mont_mul<Fn>(s, t, inv[0]);
    from_mont<Fn>(s, s);
    const bool good = a->status[i] && !is_zero256(r) && !is_zero256(s);
    if (!good) {
      fe_set_zero<Fn>(r);
      fe_set_zero<Fn>(s);
    }
    store_be256(a->out_r + 8 * i, r);
    store_be256(a->out_s + 8 * i, s);
    a->AD.load(i, x, y);
    from_mont<Fp>(x, x);
    from_mont<Fp>(y, y);
    store_be256(a->out_pub + 16 * i, x);
    store_be256(a->out_pub + 16 * i + 8, y);
  }
};

template <class C, int BLOCK>
__device__ void fixed_prep(const FixedArgs<C>& a, size_t begin, size_t end) {
  using Fp = typename C::Fp;
  using Fn = typename C::Fn;
  for (size_t i = begin + threadIdx.x; i < end; i += BLOCK) {
    uint32_t k[8];
    uint32_t z[Fp::N];
    fe_set_zero<Fp>(z);
    a.AK.store(i, z, z);
    if (a.mode == 0) {
#pragma unroll
      for (int q = 0; q < 8; ++q) k[q] = a.k[8 * i + q];
    } else {
      uint32_t d[8], e[8], nn[8];
      load_be256(k, a.k + 8 * i);
      load_be256(d, a.d + 8 * i);
      load_be256(e, a.e + 8 * i);
#pragma unroll
      for (int q = 0; q < 8; ++q) nn[q] = C::n(q);
      const bool valid = !is_zero256(k) && !is_zero256(d) && lt256(k, nn) && lt256(d, nn);
      if (!valid) {
#pragma unroll
        for (int q = 0; q < 8; ++q) k[q] = d[q] = q == 0 ? 1u : 0u;
      }
      if (!lt256(e, nn)) sub256(e, e, nn);
      uint32_t t[8];
      to_mont<Fn>(t, k);
      a.KN.store(i, t);
      to_mont<Fn>(t, d);
      a.DN.store(i, t);
      to_mont<Fn>(t, e);
      a.EN.store(i, t);
#pragma unroll
      for (int j = 0; j < 32; ++j) a.DB[j * a.n + i] = (uint8_t)(d[j >> 2] >> (8 * (j & 3)));
      a.AD.store(i, z, z);
      a.status[i] = valid ? 1 : 0;
    }
#pragma unroll
    for (int j = 0; j < 32; ++j) a.KB[j * a.n + i] = (uint8_t)(k[j >> 2] >> (8 * (j & 3)));
  }
}

template <class C, int BLOCK>
__global__ void __launch_bounds__(BLOCK, kGasResidentThreads / BLOCK) k_fixed_base(FixedArgs<C> a) {
  using Fp = typename C::Fp;
  using Fn = typename C::Fn;
  constexpr int N = Fp::N;
  auto& sm = gas_smem<N, BLOCK>();
  const size_t begin = blockIdx.x * a.per_cta;
  size_t end = begin + a.per_cta < a.n ? begin + a.per_cta : a.n;
  if (end < begin) end = begin;
  fixed_prep<C, BLOCK>(a, begin, end);
  if (a.mode == 0) {
    for (int j = 0; j < 32; ++j) {
      CombRound<C, 1> rd{&a, j};
      batch_round<Fp, BLOCK>(rd, begin, end, a.M, sm);
    }
    for (size_t i = begin + threadIdx.x; i < end; i += BLOCK) {
      uint32_t x[N], y[N];
      a.AK.load(i, x, y);
      from_mont<Fp>(x, x);
      from_mont<Fp>(y, y);
#pragma unroll
      for (int q = 0; q < N; ++q) {
        a.out_pt[2 * N * i + q] = x[q];
        a.out_pt[2 * N * i + N + q] = y[q];
      }
    }
  } else {
    if constexpr (N == 8) {
      for (int j = 0; j < 32; ++j) {
        CombRound<C, 2> rd{&a, j};
        batch_round<Fp, BLOCK>(rd, begin, end, a.M, sm);
      }
      SignRound<C> rs{&a};
      batch_round<Fn, BLOCK>(rs, begin, end, SoA<Fn>{a.M.vec, a.M.stride}, sm);
    }
  }
}

}  // namespace ecc
