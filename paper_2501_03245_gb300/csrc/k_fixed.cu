// Launchers of batched FPMUL (k G) and batched ECDSA signing.
#include "fixed_base.cuh"
#include "internal.h"

namespace ecc {

namespace {

constexpr int kFixedBlock = kGasThreads;

template <class C>
cudaError_t fixed_base(int curve, int mode, size_t n, const uint32_t* k, const uint32_t* d,
                       const uint32_t* e, uint32_t* out_pt, uint32_t* out_r, uint32_t* out_s,
                       uint32_t* out_pub, cudaStream_t st) {
  using Fp = typename C::Fp;
  using Fn = typename C::Fn;
  constexpr int B = kFixedBlock;
  const uint4* tg = nullptr;
  cudaError_t err = gtable(curve, &tg, st);
  if (err != cudaSuccess) return err;
  const size_t fp = soa_bytes<Fp>(n), fn = soa_bytes<Fn>(n);
  const size_t bytes = 5 * fp + 3 * fn + 65 * n + 256;
  Scratch ws;
  err = ws.alloc(bytes, st);
  if (err != cudaSuccess) return err;
  uint4* v = ws.as<uint4>();
  const size_t q = fp / 16, qn = fn / 16;
  FixedArgs<C> a{};
  a.n = n;
  a.mode = mode;
  a.k = k;
  a.d = d;
  a.e = e;
  a.out_pt = out_pt;
  a.out_r = out_r;
  a.out_s = out_s;
  a.out_pub = out_pub;
  a.AK = PtSoA<Fp>{SoA<Fp>{v, n}, SoA<Fp>{v + q, n}};
  a.AD = PtSoA<Fp>{SoA<Fp>{v + 2 * q, n}, SoA<Fp>{v + 3 * q, n}};
  a.M = SoA<Fp>{v + 4 * q, n};
  uint4* vn = v + 5 * q;
  a.KN = SoA<Fn>{vn, n};
  a.EN = SoA<Fn>{vn + qn, n};
  a.DN = SoA<Fn>{vn + 2 * qn, n};
  uint8_t* tail = reinterpret_cast<uint8_t*>(vn + 3 * qn);
  a.KB = tail;
  a.DB = tail + 32 * n;
  a.status = tail + 64 * n;
  const size_t te = 32 * 256;
  a.TG = PtSoA<Fp>{SoA<Fp>{const_cast<uint4*>(tg), te},
                   SoA<Fp>{const_cast<uint4*>(tg) + soa_bytes<Fp>(te) / 16, te}};
  size_t ctas = (size_t)device_sm_count() * kGasCtasPerSm;
  size_t per = (n + ctas - 1) / ctas;
  if (per < 32) per = 32;
  ctas = (n + per - 1) / per;
  a.per_cta = per;
  const size_t smem = sizeof(GasSmem<Fp::N, B>);
  err = cudaFuncSetAttribute(k_fixed_base<C, B>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  k_fixed_base<C, B><<<(unsigned)ctas, B, smem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_fixed_base_mul(int curve, size_t n, const uint32_t* k, uint32_t* out,
                                  cudaStream_t st) {
  switch (curve) {
    case 0: return fixed_base<Secp256k1>(0, 0, n, k, nullptr, nullptr, out, nullptr, nullptr, nullptr, st);
    case 1: return fixed_base<P256>(1, 0, n, k, nullptr, nullptr, out, nullptr, nullptr, nullptr, st);
    case 2: return fixed_base<BN254>(2, 0, n, k, nullptr, nullptr, out, nullptr, nullptr, nullptr, st);
    case 3: return fixed_base<BLS12_381>(3, 0, n, k, nullptr, nullptr, out, nullptr, nullptr, nullptr, st);
    case 4: return fixed_base<SM2>(4, 0, n, k, nullptr, nullptr, out, nullptr, nullptr, nullptr, st);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_sign(int curve, size_t n, const uint8_t* d, const uint8_t* e, const uint8_t* k,
                        uint8_t* r, uint8_t* s, uint8_t* pub, cudaStream_t st) {
  auto w = [](const uint8_t* p) { return reinterpret_cast<const uint32_t*>(p); };
  auto o = [](uint8_t* p) { return reinterpret_cast<uint32_t*>(p); };
  switch (curve) {
    case 0: return fixed_base<Secp256k1>(0, 1, n, w(k), w(d), w(e), nullptr, o(r), o(s), o(pub), st);
    case 1: return fixed_base<P256>(1, 1, n, w(k), w(d), w(e), nullptr, o(r), o(s), o(pub), st);
    case 4: return fixed_base<SM2>(4, 1, n, w(k), w(d), w(e), nullptr, o(r), o(s), o(pub), st);
  }
  return cudaErrorNotSupported;
}

}  // namespace ecc
