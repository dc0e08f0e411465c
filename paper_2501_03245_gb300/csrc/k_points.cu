// EC-operator launchers: batched affine PADD / PDBL on caller arrays, and the
// per-device fixed-base table v 2^(8j) G (FPMUL precomputation, Section 2.1.1).
#include <mutex>
#include <vector>

#include "internal.h"
#include "ops.cuh"

namespace ecc {

namespace {

__global__ void k_fill_ops(PointOp* ops, size_t n, uint32_t dst0, uint32_t a0, uint32_t b0,
                           uint32_t b_step) {
  size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  ops[i] = PointOp{dst0 + (uint32_t)i, a0 + (uint32_t)i, b0 + (uint32_t)(i * b_step)};
}

template <class C>
__global__ void k_set_generator(PtSoA<typename C::Fp> pool, uint32_t slot) {
  using F = typename C::Fp;
  uint32_t x[F::N], y[F::N];
#pragma unroll
  for (int k = 0; k < F::N; ++k) {
    x[k] = C::gx(k);
    y[k] = C::gy(k);
  }
  to_mont<F>(x, x);
  to_mont<F>(y, y);
  pool.store(slot, x, y);
}

// Runs ops[0 .. n_ops) as one batched round on `pool`.
template <class C>
cudaError_t run_ops(PtSoA<typename C::Fp> pool, const PointOp* ops, size_t n_ops,
                    SoA<typename C::Fp> M, cudaStream_t st) {
  constexpr int B = kBlock;
  using F = typename C::Fp;
  if (n_ops == 0) return cudaSuccess;
  size_t ctas = (size_t)device_sm_count() * kGasCtasPerSm;
  size_t per = (n_ops + ctas - 1) / ctas;
  if (per < B) per = B;
  ctas = (n_ops + per - 1) / per;
  const size_t smem = sizeof(GasSmem<F::N, B>);
  cudaError_t e = cudaFuncSetAttribute(k_point_ops<C, B>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_point_ops<C, B><<<(unsigned)ctas, B, smem, st>>>(pool, ops, n_ops, M, per);
  return cudaGetLastError();
}

template <class C>
cudaError_t point_add(size_t n, const uint32_t* p, const uint32_t* q, uint32_t* out, int dbl,
                      cudaStream_t st) {
  using F = typename C::Fp;
  constexpr int N = F::N;
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
  k_fe_in<F><<<cb, 256, 0, st>>>(p, n, 2 * N, 0, pool.x, 1);
  k_fe_in<F><<<cb, 256, 0, st>>>(p, n, 2 * N, N, pool.y, 1);
  if (!dbl) {
    k_fe_in<F><<<cb, 256, 0, st>>>(q, n, 2 * N, 0, pool.x.at(n), 1);
    k_fe_in<F><<<cb, 256, 0, st>>>(q, n, 2 * N, N, pool.y.at(n), 1);
    k_fill_ops<<<cb, 256, 0, st>>>(ops, n, (uint32_t)(2 * n), 0, (uint32_t)n, 1);
  } else {
    k_fill_ops<<<cb, 256, 0, st>>>(ops, n, (uint32_t)n, 0, 0, 1);
  }
  e = run_ops<C>(pool, ops, n, M, st);
  if (e != cudaSuccess) return e;
  const size_t o = dbl ? n : 2 * n;
  k_fe_out<F><<<cb, 256, 0, st>>>(pool.x.at(o), n, out, 2 * N, 0, 1);
  k_fe_out<F><<<cb, 256, 0, st>>>(pool.y.at(o), n, out, 2 * N, N, 1);
  return cudaGetLastError();
}

// --------------------------------------------------------------- G table

constexpr size_t kTabEntries = 32 * 256;

template <class C>
cudaError_t build_gtable(uint4** out, cudaStream_t st) {
  using F = typename C::Fp;
  const size_t soa = soa_bytes<F>(kTabEntries);
  uint4* tab = nullptr;
  cudaError_t e = cudaMalloc(&tab, 2 * soa);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(tab, 0, 2 * soa, st);
  if (e != cudaSuccess) return e;
  PtSoA<F> pool{SoA<F>{tab, kTabEntries}, SoA<F>{tab + soa / 16, kTabEntries}};
  // op list: the power-of-two chain (one op per launch), then 7 fill rounds
  std::vector<PointOp> ops;
  std::vector<std::pair<size_t, size_t>> launches;  // (offset, count)
  for (uint32_t j = 0; j < 32; ++j) {
    for (uint32_t k = 1; k < 8; ++k) {
      launches.push_back({ops.size(), 1});
      ops.push_back(PointOp{j * 256 + (1u << k), j * 256 + (1u << (k - 1)), j * 256 + (1u << (k - 1))});
    }
    if (j < 31) {
      launches.push_back({ops.size(), 1});
      ops.push_back(PointOp{(j + 1) * 256 + 1, j * 256 + 128, j * 256 + 128});
    }
  }
  for (uint32_t k = 1; k < 8; ++k) {
    size_t off = ops.size();
    for (uint32_t j = 0; j < 32; ++j)
      for (uint32_t u = 1; u < (1u << k); ++u)
        ops.push_back(PointOp{j * 256 + (1u << k) + u, j * 256 + (1u << k), j * 256 + u});
    launches.push_back({off, ops.size() - off});
  }
  Scratch ws_ops, ws_m;
  e = ws_ops.alloc(ops.size() * sizeof(PointOp), st);
  if (e != cudaSuccess) return e;
  e = ws_m.alloc(soa_bytes<F>(kTabEntries), st);
  if (e != cudaSuccess) return e;
  PointOp* dops = ws_ops.as<PointOp>();
  SoA<F> M{ws_m.as<uint4>(), kTabEntries};
  e = cudaMemcpyAsync(dops, ops.data(), ops.size() * sizeof(PointOp), cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return e;
  k_set_generator<C><<<1, 1, 0, st>>>(pool, 1);
  for (auto& l : launches) {
    e = run_ops<C>(pool, dops + l.first, l.second, M, st);
    if (e != cudaSuccess) return e;
  }
  e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return e;
  *out = tab;
  return cudaSuccess;
}

std::mutex g_tab_mu;
uint4* g_tabs[64][5] = {};

}  // namespace

cudaError_t gtable(int curve, const uint4** table, cudaStream_t st) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64 || curve < 0 || curve > 4) return cudaErrorInvalidValue;
  std::lock_guard<std::mutex> lock(g_tab_mu);
  if (!g_tabs[dev][curve]) {
    uint4* t = nullptr;
    switch (curve) {
      case 0: e = build_gtable<Secp256k1>(&t, st); break;
      case 1: e = build_gtable<P256>(&t, st); break;
      case 2: e = build_gtable<BN254>(&t, st); break;
      case 3: e = build_gtable<BLS12_381>(&t, st); break;
      case 4: e = build_gtable<SM2>(&t, st); break;
    }
    if (e != cudaSuccess) return e;
    g_tabs[dev][curve] = t;
  }
  *table = g_tabs[dev][curve];
  return cudaSuccess;
}

namespace {

// y^2 = x^3 + a x + b in Montgomery form, canonical coordinates; (0, 0) is O.
template <class C>
__global__ void k_validate(const uint32_t* __restrict__ p, size_t n, uint8_t* __restrict__ ok) {
  using F = typename C::Fp;
  constexpr int N = F::N;
  const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint32_t x[N], y[N];
#pragma unroll
  for (int k = 0; k < N; ++k) {
    x[k] = p[2 * N * i + k];
    y[k] = p[2 * N * i + N + k];
  }
  if (pt_is_inf<F>(x, y)) {
    ok[i] = 1;
    return;
  }
  if (!fe_lt_modulus<F>(x) || !fe_lt_modulus<F>(y)) {
    ok[i] = 0;
    return;
  }
  to_mont<F>(x, x);
  to_mont<F>(y, y);
  uint32_t lhs[N], rhs[N], t[N];
  mont_sqr<F>(lhs, y);
  mont_sqr<F>(t, x);
  if (!C::A_ZERO) {
    uint32_t a[N];
    curve_a<C>(a);
    fe_add<F>(t, t, a);
  }
  mont_mul<F>(rhs, t, x);
#pragma unroll
  for (int k = 0; k < N; ++k) t[k] = C::b(k);
  fe_add<F>(rhs, rhs, t);
  ok[i] = fe_eq<F>(lhs, rhs) ? 1 : 0;
}

}  // namespace

cudaError_t launch_validate_points(int curve, size_t n, const uint32_t* p, uint8_t* ok, cudaStream_t st) {
  const unsigned b = (unsigned)((n + 255) / 256);
  switch (curve) {
    case 0: k_validate<Secp256k1><<<b, 256, 0, st>>>(p, n, ok); break;
    case 1: k_validate<P256><<<b, 256, 0, st>>>(p, n, ok); break;
    case 2: k_validate<BN254><<<b, 256, 0, st>>>(p, n, ok); break;
    case 3: k_validate<BLS12_381><<<b, 256, 0, st>>>(p, n, ok); break;
    case 4: k_validate<SM2><<<b, 256, 0, st>>>(p, n, ok); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_point_add(int curve, size_t n, const uint32_t* p, const uint32_t* q,
                             uint32_t* out, int dbl, cudaStream_t st) {
  switch (curve) {
    case 0: return point_add<Secp256k1>(n, p, q, out, dbl, st);
    case 1: return point_add<P256>(n, p, q, out, dbl, st);
    case 2: return point_add<BN254>(n, p, q, out, dbl, st);
    case 3: return point_add<BLS12_381>(n, p, q, out, dbl, st);
    case 4: return point_add<SM2>(n, p, q, out, dbl, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace ecc
