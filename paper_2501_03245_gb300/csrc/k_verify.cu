// Dispatch of the batched ECDSA verification (secp256k1, P-256, SM2); the
// kernels are instantiated in k_verify_<curve>*.cu.
#include <atomic>

#include "internal.h"

namespace ecc {

#define ECC_VERIFY_DECL(name)                                                                  \
  cudaError_t verify_##name(size_t n, const uint8_t* hash, const uint8_t* r, const uint8_t* s, \
                            const uint8_t* pub, uint8_t* ok, cudaStream_t st);
ECC_VERIFY_DECL(secp256k1)
ECC_VERIFY_DECL(p256)
ECC_VERIFY_DECL(p256_c2)
ECC_VERIFY_DECL(p256_c4)
ECC_VERIFY_DECL(sm2)
#undef ECC_VERIFY_DECL

namespace {
std::atomic<int> g_gas_cluster{1};
}  // namespace

void set_gas_cluster(int ctas) { g_gas_cluster.store(ctas); }

cudaError_t launch_verify(int curve, size_t n, const uint8_t* hash, const uint8_t* r,
                          const uint8_t* s, const uint8_t* pub, uint8_t* ok, cudaStream_t st) {
  switch (curve) {
    case 0: return verify_secp256k1(n, hash, r, s, pub, ok, st);
    case 1:
      switch (g_gas_cluster.load()) {
        case 2: return verify_p256_c2(n, hash, r, s, pub, ok, st);
        case 4: return verify_p256_c4(n, hash, r, s, pub, ok, st);
        default: return verify_p256(n, hash, r, s, pub, ok, st);
      }
    case 4: return verify_sm2(n, hash, r, s, pub, ok, st);
  }
  return cudaErrorNotSupported;
}

}  // namespace ecc
