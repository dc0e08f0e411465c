// Dispatch of the batched ECDSA verification (secp256k1, P-256, SM2); the
// kernels are instantiated in k_verify_<curve>[_c2].cu (per-CTA inversion, or
// one inversion shared by the two CTAs of a cluster).
#include <atomic>

#include "internal.h"

namespace ecc {

#define ECC_VERIFY_DECL(name)                                                                  \
  cudaError_t verify_##name(size_t n, const uint8_t* hash, const uint8_t* r, const uint8_t* s, \
                            const uint8_t* pub, uint8_t* ok, cudaStream_t st);
ECC_VERIFY_DECL(secp256k1)
ECC_VERIFY_DECL(secp256k1_c2)
ECC_VERIFY_DECL(p256)
ECC_VERIFY_DECL(p256_c2)
ECC_VERIFY_DECL(sm2)
ECC_VERIFY_DECL(sm2_c2)
#undef ECC_VERIFY_DECL

namespace {
// CTAs per cluster sharing a round's inversion (2: measured 2.8% faster than
// 1 on the 2^20 P-256 batch; 4 was 54% slower and is not built)
std::atomic<int> g_gas_cluster{2};
}  // namespace

void set_gas_cluster(int ctas) { g_gas_cluster.store(ctas); }

cudaError_t launch_verify(int curve, size_t n, const uint8_t* hash, const uint8_t* r,
                          const uint8_t* s, const uint8_t* pub, uint8_t* ok, cudaStream_t st) {
  const bool pair = g_gas_cluster.load() == 2;
  switch (curve) {
    case 0: return pair ? verify_secp256k1_c2(n, hash, r, s, pub, ok, st) : verify_secp256k1(n, hash, r, s, pub, ok, st);
    case 1: return pair ? verify_p256_c2(n, hash, r, s, pub, ok, st) : verify_p256(n, hash, r, s, pub, ok, st);
    case 4: return pair ? verify_sm2_c2(n, hash, r, s, pub, ok, st) : verify_sm2(n, hash, r, s, pub, ok, st);
  }
  return cudaErrorNotSupported;
}

}  // namespace ecc
