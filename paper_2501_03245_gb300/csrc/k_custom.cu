// Batched affine PADD / PDBL (Section 3.3, Eqn 2-3) on a curve whose
// parameters are supplied at run time: y^2 = x^3 + a x + b over F_p for any
// odd prime 5 <= p < 2^256, in 8-limb Montgomery form (R = 2^256).
//
// The field constants (R mod p, R^2 and R^3 mod p, -p^-1 mod 2^32 and
// p^-1 mod 2^62) are derived on the host, passed by value as a kernel
// parameter, and copied into shared memory by every CTA before any arithmetic.
// The traits classes below read them from there, so one compiled copy of the
// field layer, the per-CTA gather-apply-scatter inversion and the batched
// PADD / PDBL rounds serves every such curve, and calls on different streams
// with different curves do not interfere.  The compiled curves keep their
// constants in the instruction stream (curves_gen.cuh); this path exists for
// curves the library was not built with, tiny test curves among them.
#include <cstring>

#include "internal.h"
#include "ops.cuh"

namespace ecc {

// The CTA's copy of the curve constants (static shared memory: the GAS scratch
// of the batched round is dynamic shared memory and follows it).
__shared__ CustomConsts g_custom;

struct CustomFp {
  static constexpr int N = 8;
  static constexpr int FORM = 0;
  ECC_DEV static uint32_t qinv() { return g_custom.qinv; }
  ECC_DEV static uint64_t qinv62() { return g_custom.qinv62; }
  ECC_DEV static uint32_t p(int i) { return g_custom.p[i]; }
  ECC_DEV static uint32_t r2(int i) { return g_custom.r2[i]; }
  ECC_DEV static uint32_t one(int i) { return g_custom.one[i]; }
  ECC_DEV static uint32_t pm2(int i) { return g_custom.pm2[i]; }
  ECC_DEV static uint32_t r3(int i) { return g_custom.r3[i]; }
};

struct CustomCurve {
  using Fp = CustomFp;
  static constexpr bool A_ZERO = false;  // a is read at run time (a = 0 adds zero)
  ECC_DEV static uint32_t a(int i) { return g_custom.a[i]; }
};

namespace {

// Every thread copies part of the constants; the barrier publishes them.
ECC_DEV void custom_enter(const CustomConsts& cc) {
  const uint32_t* src = reinterpret_cast<const uint32_t*>(&cc);
  uint32_t* dst = reinterpret_cast<uint32_t*>(&g_custom);
  for (unsigned i = threadIdx.x; i < sizeof(CustomConsts) / 4; i += blockDim.x) dst[i] = src[i];
  __syncthreads();
}

__global__ void k_custom_in(CustomConsts cc, const uint32_t* __restrict__ aos, size_t n,
                            size_t row_stride, size_t col, SoA<CustomFp> out) {
  custom_enter(cc);
  const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint32_t v[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) v[k] = aos[i * row_stride + col + k];
  to_mont<CustomFp>(v, v);
  out.store(i, v);
}

__global__ void k_custom_out(CustomConsts cc, SoA<CustomFp> in, size_t n, uint32_t* __restrict__ aos,
                             size_t row_stride, size_t col) {
  custom_enter(cc);
  const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint32_t v[8];
  in.load(i, v);
  from_mont<CustomFp>(v, v);
#pragma unroll
  for (int k = 0; k < 8; ++k) aos[i * row_stride + col + k] = v[k];
}

__global__ void k_custom_fill(PointOp* ops, size_t n, uint32_t dst0, uint32_t b0) {
  const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  ops[i] = PointOp{dst0 + (uint32_t)i, (uint32_t)i, b0 + (uint32_t)i};
}

// One batched round of independent point operations (the body of k_point_ops).
template <int BLOCK>
__global__ void __launch_bounds__(BLOCK, kGasResidentThreads / BLOCK)
    k_custom_point_ops(CustomConsts cc, PtSoA<CustomFp> pool, const PointOp* ops, size_t n_ops,
                       SoA<CustomFp> M, size_t per_cta) {
  custom_enter(cc);
  auto& sm = gas_smem<8, BLOCK>();
  const size_t begin = blockIdx.x * per_cta;
  size_t end = begin + per_cta < n_ops ? begin + per_cta : n_ops;
  if (end < begin) end = begin;
  OpRound<CustomCurve> rd{pool, ops};
  batch_round<CustomFp, BLOCK>(rd, begin, end, M, sm);
}

// ---------------------------------------------------------------- host side
// 8-limb little-endian arithmetic for deriving the constants.
using L8 = uint32_t[8];

bool ge(const uint32_t* x, uint32_t top, const uint32_t* p) {
  if (top) return true;
  for (int i = 7; i >= 0; --i) {
    if (x[i] != p[i]) return x[i] > p[i];
  }
  return true;
}

void sub_in_place(uint32_t* x, const uint32_t* p) {
  uint64_t borrow = 0;
  for (int i = 0; i < 8; ++i) {
    const uint64_t d = (uint64_t)x[i] - p[i] - borrow;
    x[i] = (uint32_t)d;
    borrow = (d >> 63) & 1;
  }
}

// x <- 2 x mod p (x < p)
void dbl_mod(uint32_t* x, const uint32_t* p) {
  uint32_t carry = 0;
  for (int i = 0; i < 8; ++i) {
    const uint32_t nx = (x[i] << 1) | carry;
    carry = x[i] >> 31;
    x[i] = nx;
  }
  if (ge(x, carry, p)) sub_in_place(x, p);
}

// x <- x 2^k mod p (x < p)
void shift_mod(uint32_t* x, int k, const uint32_t* p) {
  for (int i = 0; i < k; ++i) dbl_mod(x, p);
}

}  // namespace

int custom_consts(const uint32_t* p, const uint32_t* a, CustomConsts* cc) {
  if ((p[0] & 1u) == 0) return 1;                                  // even
  bool small = true;
  for (int i = 1; i < 8; ++i) small &= p[i] == 0;
  if (small && p[0] < 5) return 2;                                 // p < 5
  bool a_ok = false;                                               // a < p
  for (int i = 7; i >= 0; --i) {
    if (a[i] != p[i]) {
      a_ok = a[i] < p[i];
      break;
    }
  }
  if (!a_ok) return 3;
  std::memset(cc, 0, sizeof *cc);
  std::memcpy(cc->p, p, 32);
  // -p^-1 mod 2^32 and p^-1 mod 2^62 by Newton's iteration x <- x (2 - p x)
  uint32_t x32 = p[0];                                             // p^-1 mod 8
  for (int i = 0; i < 4; ++i) x32 *= 2u - p[0] * x32;
  cc->qinv = 0u - x32;
  const uint64_t p64 = (uint64_t)p[0] | ((uint64_t)p[1] << 32);
  uint64_t x64 = p64;
  for (int i = 0; i < 5; ++i) x64 *= 2u - p64 * x64;
  cc->qinv62 = x64 & (((uint64_t)1 << 62) - 1);
  // R^k mod p = 1 shifted 256 k times; a R mod p
  uint32_t t[8] = {1, 0, 0, 0, 0, 0, 0, 0};
  shift_mod(t, 256, p);
  std::memcpy(cc->one, t, 32);
  shift_mod(t, 256, p);
  std::memcpy(cc->r2, t, 32);
  shift_mod(t, 256, p);
  std::memcpy(cc->r3, t, 32);
  std::memcpy(t, a, 32);
  shift_mod(t, 256, p);
  std::memcpy(cc->a, t, 32);
  std::memcpy(t, p, 32);
  const uint32_t two[8] = {2, 0, 0, 0, 0, 0, 0, 0};
  sub_in_place(t, two);
  std::memcpy(cc->pm2, t, 32);
  return 0;
}

cudaError_t launch_point_add_custom(const CustomConsts& cc, size_t n, const uint32_t* p,
                                    const uint32_t* q, uint32_t* out, int dbl, cudaStream_t st) {
  using F = CustomFp;
  constexpr int B = kBlock;
  const size_t slots = dbl ? 2 * n : 3 * n;
  Scratch ws;
  const size_t soa = soa_bytes<F>(slots);
  cudaError_t e = ws.alloc(2 * soa + soa_bytes<F>(n) + n * sizeof(PointOp) + 64, st);
  if (e != cudaSuccess) return e;
  uint4* base = ws.as<uint4>();
  PtSoA<F> pool{SoA<F>{base, slots}, SoA<F>{base + soa / 16, slots}};
  SoA<F> M{base + 2 * soa / 16, n};
  PointOp* ops = reinterpret_cast<PointOp*>(base + (2 * soa + soa_bytes<F>(n)) / 16);
  const unsigned cb = (unsigned)((n + 255) / 256);
  k_custom_in<<<cb, 256, 0, st>>>(cc, p, n, 16, 0, pool.x);
  k_custom_in<<<cb, 256, 0, st>>>(cc, p, n, 16, 8, pool.y);
  if (!dbl) {
    k_custom_in<<<cb, 256, 0, st>>>(cc, q, n, 16, 0, pool.x.at(n));
    k_custom_in<<<cb, 256, 0, st>>>(cc, q, n, 16, 8, pool.y.at(n));
    k_custom_fill<<<cb, 256, 0, st>>>(ops, n, (uint32_t)(2 * n), (uint32_t)n);
  } else {
    k_custom_fill<<<cb, 256, 0, st>>>(ops, n, (uint32_t)n, 0);
  }
  size_t ctas = (size_t)device_sm_count() * kGasCtasPerSm;
  size_t per = (n + ctas - 1) / ctas;
  if (per < B) per = B;
  ctas = (n + per - 1) / per;
  const size_t smem = sizeof(GasSmem<8, B>);
  e = cudaFuncSetAttribute(k_custom_point_ops<B>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_custom_point_ops<B><<<(unsigned)ctas, B, smem, st>>>(cc, pool, ops, n, M, per);
  const size_t o = dbl ? n : 2 * n;
  k_custom_out<<<cb, 256, 0, st>>>(cc, pool.x.at(o), n, out, 16, 0);
  k_custom_out<<<cb, 256, 0, st>>>(cc, pool.y.at(o), n, out, 16, 8);
  return cudaGetLastError();
}

}  // namespace ecc
