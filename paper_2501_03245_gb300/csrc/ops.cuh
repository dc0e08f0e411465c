// Generic batched kernels: layout conversion between the caller's row-major
// canonical limbs and the device SoA Montgomery layout, field-operation unit
// kernels, batch inversion (Montgomery's trick with GAS, Section 3.2) and a
// batched point-operation kernel (PADD / PDBL, Section 3.3) driven by an op list.
#pragma once
#include <cstddef>
#include <cstdint>

#include "ec.cuh"

namespace ecc {

constexpr int kBlock = kGasThreads;

// ---------------------------------------------------------------- conversion

// row-major canonical limbs (n x N) -> SoA, optionally into Montgomery form
template <class F>
__global__ void k_fe_in(const uint32_t* __restrict__ aos, size_t n, size_t row_stride,
                        size_t col, SoA<F> out, int mont) {
  size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint32_t v[F::N];
#pragma unroll
  for (int k = 0; k < F::N; ++k) v[k] = aos[i * row_stride + col + k];
  if (mont) to_mont<F>(v, v);
  out.store(i, v);
}

template <class F>
__global__ void k_fe_out(SoA<F> in, size_t n, uint32_t* __restrict__ aos, size_t row_stride,
                         size_t col, int mont) {
  size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint32_t v[F::N];
  in.load(i, v);
  if (mont) from_mont<F>(v, v);
#pragma unroll
  for (int k = 0; k < F::N; ++k) aos[i * row_stride + col + k] = v[k];
}

// ---------------------------------------------------------------- unit ops

// out_i = a_i * b_i mod q on canonical row-major limbs (a2: Montgomery
// multiplication, Algorithm 2, with conversions in and out).
template <class F>
__global__ void k_fe_mul(const uint32_t* __restrict__ a, const uint32_t* __restrict__ b,
                         uint32_t* __restrict__ out, size_t n) {
  size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint32_t x[F::N], y[F::N], z[F::N];
#pragma unroll
  for (int k = 0; k < F::N; ++k) {
    x[k] = a[i * F::N + k];
    y[k] = b[i * F::N + k];
  }
  to_mont<F>(x, x);
  to_mont<F>(y, y);
  mont_mul<F>(z, x, y);
  from_mont<F>(z, z);
#pragma unroll
  for (int k = 0; k < F::N; ++k) out[i * F::N + k] = z[k];
}

// out_i = a_i + b_i or a_i - b_i mod q (a3)
template <class F>
__global__ void k_fe_addsub(const uint32_t* __restrict__ a, const uint32_t* __restrict__ b,
                            uint32_t* __restrict__ out, size_t n, int subtract) {
  size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint32_t x[F::N], y[F::N], z[F::N];
#pragma unroll
  for (int k = 0; k < F::N; ++k) {
    x[k] = a[i * F::N + k];
    y[k] = b[i * F::N + k];
  }
  if (subtract) {
    fe_sub<F>(z, x, y);
  } else {
    fe_add<F>(z, x, y);
  }
#pragma unroll
  for (int k = 0; k < F::N; ++k) out[i * F::N + k] = z[k];
}

// single inversion per element (a4: Fermat), canonical in/out, 0 -> 0
template <class F>
__global__ void k_fe_inv_single(const uint32_t* __restrict__ a, uint32_t* __restrict__ out,
                                size_t n) {
  size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint32_t x[F::N];
#pragma unroll
  for (int k = 0; k < F::N; ++k) x[k] = a[i * F::N + k];
  to_mont<F>(x, x);
  fe_inv_fermat<F>(x, x);
  from_mont<F>(x, x);
#pragma unroll
  for (int k = 0; k < F::N; ++k) out[i * F::N + k] = x[k];
}

// ---------------------------------------------------------------- batch inverse

template <class F>
struct InvRound {
  static constexpr int OPS = 1;
  SoA<F> in, out;
  uint32_t x[F::N];
  bool nz;
  ECC_DEV void den_c(size_t i, int, uint32_t* d) {
    in.load(i, x);
    nz = !fe_is_zero<F>(x);
    fe_copy<F>(d, x);
    if (!nz) fe_set_one<F>(d);
  }
  ECC_DEV void den_d(size_t i, int j, uint32_t* d) { den_c(i, j, d); }
  ECC_DEV void finish(size_t i, const uint32_t (*inv)[F::N]) {
    uint32_t r[F::N];
    fe_copy<F>(r, inv[0]);
    if (!nz) fe_set_zero<F>(r);
    out.store(i, r);
  }
};

// a5: out = in^-1 elementwise (Montgomery form, 0 -> 0); each CTA inverts the
// contiguous slice [blockIdx.x * per_cta, ...) with one modular inversion.
template <class F, int BLOCK>
__global__ void __launch_bounds__(BLOCK, kGasResidentThreads / BLOCK) k_batch_inverse(SoA<F> in, SoA<F> out, SoA<F> M,
                                                         size_t n, size_t per_cta) {
  auto& sm = gas_smem<F::N, BLOCK>();
  const size_t begin = blockIdx.x * per_cta;
  const size_t end = begin + per_cta < n ? begin + per_cta : n;
  InvRound<F> rd{in, out};
  batch_round<F, BLOCK>(rd, begin, end < begin ? begin : end, M, sm);
}

// ---------------------------------------------------------------- point ops

struct PointOp {
  uint32_t dst, a, b;  // pool[dst] = pool[a] + pool[b]  (a == b: doubling)
};

template <class C>
struct OpRound {
  using F = typename C::Fp;
  static constexpr int N = F::N;
  static constexpr int OPS = 1;
  PtSoA<F> pool;
  const PointOp* ops;
  uint32_t xp[N], yp[N], xt[N], yt[N];
  int kind;
  ECC_DEV void den_c(size_t i, int, uint32_t* d) {
    const PointOp op = ops[i];
    pool.load(op.a, xp, yp);
    pool.load(op.b, xt, yt);
    kind = add_den<C>(d, xp, yp, xt, yt);
  }
  ECC_DEV void den_d(size_t i, int j, uint32_t* d) { den_c(i, j, d); }
  ECC_DEV void finish(size_t i, const uint32_t (*inv)[N]) {
    uint32_t xr[N], yr[N];
    add_finish<C>(xr, yr, kind, inv[0], xp, yp, xt, yt);
    pool.store(ops[i].dst, xr, yr);
  }
};

// a6/a7: one batched round of independent point operations.  No op of a launch
// may read a slot that another op of the same launch writes.
template <class C, int BLOCK>
__global__ void __launch_bounds__(BLOCK, kGasResidentThreads / BLOCK) k_point_ops(PtSoA<typename C::Fp> pool,
                                                     const PointOp* ops, size_t n_ops,
                                                     SoA<typename C::Fp> M, size_t per_cta) {
  auto& sm = gas_smem<C::Fp::N, BLOCK>();
  const size_t begin = blockIdx.x * per_cta;
  size_t end = begin + per_cta < n_ops ? begin + per_cta : n_ops;
  if (end < begin) end = begin;
  OpRound<C> rd{pool, ops};
  batch_round<typename C::Fp, BLOCK>(rd, begin, end, M, sm);
}

}  // namespace ecc
