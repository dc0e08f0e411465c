// MSM instantiation for BN254 (one translation unit per curve so the library
// builds in parallel).
#include "msm_host.cuh"

namespace ecc {

cudaError_t points_to_mont_bls12_381(const uint32_t* in, uint64_t n, uint32_t* out,
                                     cudaStream_t st);

cudaError_t msm_points_bn254(uint32_t num, const uint64_t* offsets, const uint32_t* points,
                             const uint32_t* scalars, uint32_t* out, cudaStream_t st) {
  return msm_detail::msm_points<BN254>(2, num, offsets, points, scalars, out, st);
}

cudaError_t msm_bases_bn254(void* bases, uint32_t num_vectors, const uint64_t* sizes,
                            const uint32_t* scalars,
                            uint32_t* out, cudaStream_t st) {
  return msm_detail::msm_bases_t<BN254>(static_cast<msm_detail::Bases*>(bases), num_vectors, sizes, scalars,
                                     out, st);
}

cudaError_t points_to_mont(int curve, const uint32_t* in, uint64_t n, uint32_t* out,
                           cudaStream_t st) {
  const unsigned b = (unsigned)((n + 255) / 256);
  if (curve == 2) {
    k_points_to_mont<BN254><<<b, 256, 0, st>>>(in, n, nullptr, out);
    return cudaGetLastError();
  }
  return points_to_mont_bls12_381(in, n, out, st);
}

cudaError_t msm_points_dev_bn254(uint32_t num, uint64_t cap, const uint64_t* offsets, int c,
                                const uint32_t* points, const uint32_t* scalars, uint32_t* out,
                                cudaStream_t st) {
  return msm_detail::msm_points_dev<BN254>(2, num, cap, offsets, c, points, scalars, out, st);
}

cudaError_t msm_bases_dev_bn254(void* bases, uint32_t num, uint64_t cap, const uint64_t* sizes, int c,
                               const uint32_t* scalars, uint32_t* out, cudaStream_t st) {
  return msm_detail::msm_bases_dev_t<BN254>(static_cast<msm_detail::Bases*>(bases), num, cap, sizes, c,
                                            scalars, out, st);
}

cudaError_t bases_precompute_bn254(void* bases, int c, cudaStream_t st) {
  return msm_detail::precompute_t<BN254>(static_cast<msm_detail::Bases*>(bases), c, st);
}

}  // namespace ecc
