// Small host tables passed to the device as kernel parameters instead of a
// host-to-device copy: kernel parameters are captured by value when the launch
// sequence is recorded in a CUDA graph, so a replay never reads host memory that
// the call has already released.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>

namespace ecc {

constexpr uint32_t kUploadWords = 4000;  // 16 KB of parameters per launch

struct UploadChunk {
  uint32_t w[kUploadWords];
};

static __global__ void k_upload(uint32_t* dst, UploadChunk c, uint32_t nwords) {
  for (uint32_t i = threadIdx.x; i < nwords; i += blockDim.x) dst[i] = c.w[i];
}

// dst (device) <- src (host), bytes a multiple of 4
inline cudaError_t upload_words(void* dst, const void* src, size_t bytes, cudaStream_t st) {
  const uint32_t* s = static_cast<const uint32_t*>(src);
  uint32_t* d = static_cast<uint32_t*>(dst);
  const size_t words = bytes / 4;
  for (size_t off = 0; off < words; off += kUploadWords) {
    UploadChunk c;
    const uint32_t n = (uint32_t)(words - off < kUploadWords ? words - off : kUploadWords);
    std::memcpy(c.w, s + off, n * 4);
    k_upload<<<1, 256, 0, st>>>(d + off, c, n);
  }
  return cudaGetLastError();
}

}  // namespace ecc
