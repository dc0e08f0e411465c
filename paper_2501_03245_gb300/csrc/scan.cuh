// Exclusive prefix sum of 32-bit counts (reduce, scan of block totals,
// per-block scan), used by the counting sort of the MSM bucket ids.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "internal.h"

namespace ecc {

constexpr int kScanThreads = 512;
constexpr int kScanPerThread = 4;
constexpr int kScanTile = kScanThreads * kScanPerThread;

__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t* total) {
  __shared__ uint32_t warp_sums[kScanThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, d);
    if (lane >= d) x += y;
  }
  if (lane == 31) warp_sums[warp] = x;
  __syncthreads();
  if (warp == 0) {
    uint32_t s = lane < kScanThreads / 32 ? warp_sums[lane] : 0;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, s, d);
      if (lane >= d) s += y;
    }
    if (lane < kScanThreads / 32) warp_sums[lane] = s;
  }
  __syncthreads();
  const uint32_t before = warp > 0 ? warp_sums[warp - 1] : 0;
  *total = warp_sums[kScanThreads / 32 - 1];
  __syncthreads();
  return before + x - v;
}

static __global__ void k_scan_reduce(const uint32_t* __restrict__ in, uint64_t n, uint32_t* __restrict__ sums) {
  const uint64_t base = (uint64_t)blockIdx.x * kScanTile + threadIdx.x * kScanPerThread;
  uint32_t s = 0;
#pragma unroll
  for (int k = 0; k < kScanPerThread; ++k)
    if (base + k < n) s += in[base + k];
  uint32_t total;
  block_excl_scan(s, &total);
  if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

static __global__ void k_scan_apply(const uint32_t* __restrict__ in, uint64_t n,
                             const uint32_t* __restrict__ block_off, uint32_t* __restrict__ out) {
  const uint64_t base = (uint64_t)blockIdx.x * kScanTile + threadIdx.x * kScanPerThread;
  uint32_t v[kScanPerThread], s = 0;
#pragma unroll
  for (int k = 0; k < kScanPerThread; ++k) {
    v[k] = base + k < n ? in[base + k] : 0;
    s += v[k];
  }
  uint32_t total;
  uint32_t run = block_excl_scan(s, &total) + (block_off ? block_off[blockIdx.x] : 0);
#pragma unroll
  for (int k = 0; k < kScanPerThread; ++k) {
    if (base + k < n) out[base + k] = run;
    run += v[k];
  }
  // the thread holding element n - 1 writes the grand total to out[n] (n >= 1)
  if (base <= n - 1 && n - 1 < base + kScanPerThread) out[n] = run;
}

// out[0..n) = exclusive prefix sums of in, out[n] = total.  out may not alias in.
inline cudaError_t exclusive_scan(const uint32_t* in, uint64_t n, uint32_t* out, cudaStream_t st) {
  if (n == 0) return cudaMemsetAsync(out, 0, sizeof(uint32_t), st);
  const uint64_t blocks = (n + kScanTile - 1) / kScanTile;
  if (blocks == 1) {
    k_scan_apply<<<1, kScanThreads, 0, st>>>(in, n, nullptr, out);
    return cudaGetLastError();
  }
  Scratch ws;
  cudaError_t e = ws.alloc((2 * blocks + 1) * sizeof(uint32_t), st);
  if (e != cudaSuccess) return e;
  uint32_t* sums = ws.as<uint32_t>();
  uint32_t* offs = sums + blocks;
  k_scan_reduce<<<(unsigned)blocks, kScanThreads, 0, st>>>(in, n, sums);
  e = exclusive_scan(sums, blocks, offs, st);
  if (e != cudaSuccess) return e;
  k_scan_apply<<<(unsigned)blocks, kScanThreads, 0, st>>>(in, n, offs, out);
  return cudaGetLastError();
}

}  // namespace ecc
