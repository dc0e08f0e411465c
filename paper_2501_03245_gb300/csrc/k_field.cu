// Field-layer kernels and launchers: modmul / modadd / modinv unit operations,
// batch inversion, and the integer multiply-add issue-rate probes.
#include <mutex>

#include "internal.h"
#include "ops.cuh"

namespace ecc {

// Fixed device scratch of the allocation-free batch inversion: the input,
// output and prefix-product arrays of up to kNoAllocMaxElems elements of the
// widest field (12 limbs).  Every GPU that loads the library holds it
// (3 x 65536 x 48 B = 9 MiB) until the process exits.
static __device__ __align__(256) uint32_t g_noalloc_scratch[3 * kNoAllocMaxElems * 12];

namespace {

std::mutex g_noalloc_mu;
void* g_noalloc_addr[64] = {};

// Device address of the scratch array on the current device.  In host code the
// array's name is only a host-side stand-in, so the address is looked up once per
// device with that device current.
cudaError_t noalloc_scratch(void** ptr) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_noalloc_addr[dev] = p;
  }
  *ptr = g_noalloc_addr[dev];
  return cudaSuccess;
}

template <class F>
cudaError_t fe_ops(int op, size_t n, const uint32_t* a, const uint32_t* b, uint32_t* out,
                   cudaStream_t st) {
  const int threads = 256;
  const unsigned blocks = (unsigned)((n + threads - 1) / threads);
  switch (op) {
    case 0: k_fe_mul<F><<<blocks, threads, 0, st>>>(a, b, out, n); break;
    case 1: k_fe_addsub<F><<<blocks, threads, 0, st>>>(a, b, out, n, 0); break;
    case 2: k_fe_addsub<F><<<blocks, threads, 0, st>>>(a, b, out, n, 1); break;
    case 3: k_fe_inv_single<F><<<blocks, threads, 0, st>>>(a, out, n); break;
  }
  return cudaGetLastError();
}

template <class F>
cudaError_t fe_inv_batch(size_t n, const uint32_t* a, uint32_t* out, cudaStream_t st) {
  constexpr int B = kBlock;
  Scratch ws;
  const size_t soa = soa_bytes<F>(n);
  cudaError_t e = ws.alloc(3 * soa, st);
  if (e != cudaSuccess) return e;
  SoA<F> in{ws.as<uint4>(), n}, res{ws.as<uint4>() + soa / 16, n}, M{ws.as<uint4>() + 2 * soa / 16, n};
  const unsigned cb = (unsigned)((n + 255) / 256);
  k_fe_in<F><<<cb, 256, 0, st>>>(a, n, F::N, 0, in, 1);
  // one CTA per (SM x 2) slice, at least a full thread row per CTA
  size_t ctas = (size_t)device_sm_count() * kGasCtasPerSm;
  size_t per = (n + ctas - 1) / ctas;
  if (per < B) per = B;
  ctas = (n + per - 1) / per;
  const size_t smem = sizeof(GasSmem<F::N, B>);
  e = cudaFuncSetAttribute(k_batch_inverse<F, B>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem);
  if (e != cudaSuccess) return e;
  k_batch_inverse<F, B><<<(unsigned)ctas, B, smem, st>>>(in, res, M, n, per);
  k_fe_out<F><<<cb, 256, 0, st>>>(res, n, out, F::N, 0, 1);
  return cudaGetLastError();
}

template <class F>
__global__ void k_bench_modmul(int iters, uint32_t* sink) {
  constexpr int N = F::N;
  uint32_t x[4][N], y[4][N];
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
#pragma unroll
  for (int c = 0; c < 4; ++c)
#pragma unroll
    for (int k = 0; k < N; ++k) {
      x[c][k] = (t * 2654435761u + c * 40503u + k) & (k == N - 1 ? 0x0fffffffu : 0xffffffffu);
      y[c][k] = F::one(k) ^ (c + k);
    }
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < 4; ++c) mont_mul<F>(x[c], x[c], y[c]);
  }
  uint32_t acc = 0;
#pragma unroll
  for (int c = 0; c < 4; ++c)
#pragma unroll
    for (int k = 0; k < N; ++k) acc ^= x[c][k];
  sink[t] = acc;
}

// Batch inversion into caller-free scratch: the same three kernels as
// fe_inv_batch, with the in / out / prefix arrays carved from the file-scope
// device array below instead of a stream-ordered allocation.
template <class F>
cudaError_t fe_inv_batch_noalloc(void* scratch, size_t n, const uint32_t* a, uint32_t* out,
                                 cudaStream_t st) {
  constexpr int B = kBlock;
  const size_t soa = soa_bytes<F>(n);
  uint4* base = static_cast<uint4*>(scratch);
  SoA<F> in{base, n}, res{base + soa / 16, n}, M{base + 2 * soa / 16, n};
  const unsigned cb = (unsigned)((n + 255) / 256);
  k_fe_in<F><<<cb, 256, 0, st>>>(a, n, F::N, 0, in, 1);
  size_t ctas = (size_t)device_sm_count() * kGasCtasPerSm;
  size_t per = (n + ctas - 1) / ctas;
  if (per < B) per = B;
  ctas = (n + per - 1) / per;
  const size_t smem = sizeof(GasSmem<F::N, B>);
  cudaError_t e = cudaFuncSetAttribute(k_batch_inverse<F, B>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_batch_inverse<F, B><<<(unsigned)ctas, B, smem, st>>>(in, res, M, n, per);
  k_fe_out<F><<<cb, 256, 0, st>>>(res, n, out, F::N, 0, 1);
  return cudaGetLastError();
}

// a chain of `iters` dependent inversions per thread: method 0 Fermat, 1 divsteps
template <class F>
__global__ void k_bench_inv(int method, int iters, uint32_t* sink) {
  constexpr int N = F::N;
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t x[N];
#pragma unroll
  for (int k = 0; k < N; ++k) x[k] = F::one(k) ^ (t * 2654435761u + k);
  x[N - 1] &= 0x0fffffffu;
  for (int it = 0; it < iters; ++it) {
    if (method == 0) {
      fe_inv_fermat<F>(x, x);
    } else if (method == 1) {
      fe_inv_mont<F>(x, x);
    } else if (method == 2) {
      fe_inv_mont62<F>(x, x);
    } else {
      fe_inv_mont<F, false>(x, x);
    }
    x[0] ^= 1u;  // never a fixed point
  }
  uint32_t acc = 0;
#pragma unroll
  for (int k = 0; k < N; ++k) acc ^= x[k];
  sink[t] = acc;
}

// 8 independent carry chains of mad.lo.cc / madc.hi pairs per iteration
__global__ void k_bench_imad(int iters, uint32_t* sink) {
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t lo[8], hi[8], a[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    lo[c] = t + c;
    hi[c] = t ^ (c * 977u);
    a[c] = 0x9E3779B9u + 2u * c + 1u;
  }
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const uint32_t x = lo[c];
      lo[c] = ptx::mad_lo_cc(a[c], x, lo[c]);
      hi[c] = ptx::madc_hi(a[c], x, hi[c]);
    }
  }
  uint32_t acc = 0;
#pragma unroll
  for (int c = 0; c < 8; ++c) acc ^= lo[c] ^ hi[c];
  sink[t] = acc;
}

}  // namespace

int field_limbs(int curve, int field) {
  if (field == 1) return 8;
  return curve == 3 ? 12 : 8;
}

#define ECC_FIELD_DISPATCH(curve, field, CALL)          \
  switch ((curve) * 2 + (field)) {                      \
    case 0: { using F = Secp256k1FpSpecial; return CALL; } \
    case 1: { using F = Secp256k1Fn; return CALL; }     \
    case 2: { using F = P256FpSpecial; return CALL; }   \
    case 3: { using F = P256Fn; return CALL; }          \
    case 4: { using F = BN254Fp; return CALL; }         \
    case 5: { using F = BN254Fn; return CALL; }         \
    case 6: { using F = BLS12_381Fp; return CALL; }     \
    case 7: { using F = BLS12_381Fn; return CALL; }     \
    case 8: { using F = SM2Fp; return CALL; }           \
    case 9: { using F = SM2Fn; return CALL; }           \
  }                                                     \
  return cudaErrorInvalidValue;

cudaError_t launch_fe_mul(int curve, int field, size_t n, const uint32_t* a, const uint32_t* b,
                          uint32_t* out, cudaStream_t st) {
  ECC_FIELD_DISPATCH(curve, field, (fe_ops<F>(0, n, a, b, out, st)))
}

cudaError_t launch_fe_addsub(int curve, int field, size_t n, const uint32_t* a,
                             const uint32_t* b, uint32_t* out, int subtract, cudaStream_t st) {
  ECC_FIELD_DISPATCH(curve, field, (fe_ops<F>(subtract ? 2 : 1, n, a, b, out, st)))
}

cudaError_t launch_fe_inv(int curve, int field, size_t n, const uint32_t* a, uint32_t* out,
                          cudaStream_t st) {
  ECC_FIELD_DISPATCH(curve, field, (fe_ops<F>(3, n, a, nullptr, out, st)))
}

cudaError_t launch_fe_inv_batch(int curve, int field, size_t n, const uint32_t* a, uint32_t* out,
                                cudaStream_t st) {
  ECC_FIELD_DISPATCH(curve, field, (fe_inv_batch<F>(n, a, out, st)))
}

cudaError_t launch_fe_inv_batch_noalloc(int curve, int field, size_t n, const uint32_t* a,
                                        uint32_t* out, cudaStream_t st) {
  void* scratch = nullptr;
  cudaError_t e = noalloc_scratch(&scratch);
  if (e != cudaSuccess) return e;
  ECC_FIELD_DISPATCH(curve, field, (fe_inv_batch_noalloc<F>(scratch, n, a, out, st)))
}

cudaError_t launch_bench_imad(size_t threads, int iters, uint32_t* sink, cudaStream_t st) {
  k_bench_imad<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(iters, sink);
  return cudaGetLastError();
}

cudaError_t launch_bench_inv(int curve, int method, size_t threads, int iters, uint32_t* sink,
                             cudaStream_t st) {
  const unsigned t = (unsigned)(threads < 128 ? threads : 128);
  const unsigned b = (unsigned)((threads + t - 1) / t);
  switch (curve) {
    case 0: k_bench_inv<Secp256k1Fp><<<b, t, 0, st>>>(method, iters, sink); break;
    case 1: k_bench_inv<P256Fp><<<b, t, 0, st>>>(method, iters, sink); break;
    case 2: k_bench_inv<BN254Fp><<<b, t, 0, st>>>(method, iters, sink); break;
    case 3: k_bench_inv<BLS12_381Fp><<<b, t, 0, st>>>(method, iters, sink); break;
    case 4: k_bench_inv<SM2Fp><<<b, t, 0, st>>>(method, iters, sink); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_bench_modmul(int curve, int reduction, size_t threads, int iters,
                                uint32_t* sink, cudaStream_t st) {
  const unsigned b = (unsigned)((threads + 255) / 256);
  if (reduction == 1) {
    if (curve == 1) {
      k_bench_modmul<P256FpSpecial><<<b, 256, 0, st>>>(iters, sink);
    } else if (curve == 0) {
      k_bench_modmul<Secp256k1FpSpecial><<<b, 256, 0, st>>>(iters, sink);
    } else {
      return cudaErrorNotSupported;
    }
    return cudaGetLastError();
  }
  switch (curve) {
    case 0: k_bench_modmul<Secp256k1Fp><<<b, 256, 0, st>>>(iters, sink); break;
    case 1: k_bench_modmul<P256Fp><<<b, 256, 0, st>>>(iters, sink); break;
    case 2: k_bench_modmul<BN254Fp><<<b, 256, 0, st>>>(iters, sink); break;
    case 3: k_bench_modmul<BLS12_381Fp><<<b, 256, 0, st>>>(iters, sink); break;
    case 4: k_bench_modmul<SM2Fp><<<b, 256, 0, st>>>(iters, sink); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace ecc
