// Batched ECDSA verification kernel instantiated for one curve and cluster
// size (a translation unit per instantiation so the library builds in parallel).
#include "verify_host.cuh"

namespace ecc {

cudaError_t verify_sm2_c2(size_t n, const uint8_t* hash, const uint8_t* r, const uint8_t* s,
                           const uint8_t* pub, uint8_t* ok, cudaStream_t st) {
  return verify_detail::verify<SM2, 2>(n, hash, r, s, pub, ok, st, 4);
}

}  // namespace ecc
