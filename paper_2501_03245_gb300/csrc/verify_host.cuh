// Host launcher of the batched ECDSA verification kernel, included by one
// translation unit per (curve, variant) so the library builds in parallel.
#pragma once
#include "internal.h"
#include "verify.cuh"

namespace ecc {

namespace verify_detail {

constexpr int kVerifyBlock = kGasThreads;

template <class C, int CL>
cudaError_t verify(size_t n, const uint8_t* hash, const uint8_t* r, const uint8_t* s,
                   const uint8_t* pub, uint8_t* ok, cudaStream_t st, int curve) {
  using Fp = typename C::Fp;
  using Fn = typename C::Fn;
  constexpr int B = kVerifyBlock;
  const uint4* tg = nullptr;
  cudaError_t e = gtable(curve, &tg, st);
  if (e != cudaSuccess) return e;
  // workspace: S, E, Rn (Fn) | TQ x,y (kQTable n each) | AQ, AG | M | D2 | U1B | status
  const size_t fe = soa_bytes<Fp>(n);
  const size_t bytes = 3 * fe + 2 * kQTable * fe + 4 * fe + fe + (kQDigits + 32 + 1) * n + 256;
  Scratch ws;
  e = ws.alloc(bytes, st);
  if (e != cudaSuccess) return e;
  uint4* v = ws.as<uint4>();
  const size_t q = fe / 16;  // uint4 per SoA array of n elements
  VerifyArgs<C> a;
  a.n = n;
  a.hash = reinterpret_cast<const uint32_t*>(hash);
  a.r = reinterpret_cast<const uint32_t*>(r);
  a.s = reinterpret_cast<const uint32_t*>(s);
  a.pub = reinterpret_cast<const uint32_t*>(pub);
  a.ok = ok;
  a.S = SoA<Fn>{v + 0 * q, n};
  a.E = SoA<Fn>{v + 1 * q, n};
  a.Rn = SoA<Fn>{v + 2 * q, n};
  const size_t T = kQTable;
  a.TQ = PtSoA<Fp>{SoA<Fp>{v + 3 * q, T * n}, SoA<Fp>{v + (3 + T) * q, T * n}};
  a.AQ = PtSoA<Fp>{SoA<Fp>{v + (3 + 2 * T) * q, n}, SoA<Fp>{v + (4 + 2 * T) * q, n}};
  a.AG = PtSoA<Fp>{SoA<Fp>{v + (5 + 2 * T) * q, n}, SoA<Fp>{v + (6 + 2 * T) * q, n}};
  a.M = SoA<Fp>{v + (7 + 2 * T) * q, n};
  uint8_t* tail = reinterpret_cast<uint8_t*>(v + (8 + 2 * T) * q);
  a.D2 = reinterpret_cast<int8_t*>(tail);
  a.U1B = tail + kQDigits * n;
  a.status = tail + (kQDigits + 32) * n;
  const size_t te = 32 * 256;
  a.TG = PtSoA<Fp>{SoA<Fp>{const_cast<uint4*>(tg), te}, SoA<Fp>{const_cast<uint4*>(tg) + soa_bytes<Fp>(te) / 16, te}};
  size_t ctas = (size_t)device_sm_count() * kGasCtasPerSm;
  size_t per = (n + ctas - 1) / ctas;
  if (per < 32) per = 32;
  ctas = (n + per - 1) / per;
  a.per_cta = per;
  const size_t smem = sizeof(GasSmem<Fp::N, B>);
  e = cudaFuncSetAttribute(k_verify<C, B, CL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if constexpr (CL > 1) {
    // clusters of CL CTAs sharing each round's inversion (a grid of whole
    // clusters; a CTA past the batch runs the rounds on an empty slice)
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)((ctas + CL - 1) / CL * CL));
    cfg.blockDim = dim3(B);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CL;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_verify<C, B, CL>, a);
  } else {
    k_verify<C, B><<<(unsigned)ctas, B, smem, st>>>(a);
    return cudaGetLastError();
  }
}

}  // namespace verify_detail

}  // namespace ecc
