// MSM entry points shared by all curves: window-width table (cost model and
// autotuner overrides), resident bases, and dispatch to the per-curve
// translation units (k_msm_bn254.cu, k_msm_bls12_381.cu).
#include <algorithm>
#include <atomic>
#include <map>
#include <mutex>

#include "msm_host.cuh"

namespace ecc {

cudaError_t msm_points_bn254(uint32_t num, const uint64_t* offsets, const uint32_t* points,
                             const uint32_t* scalars, uint32_t* out, cudaStream_t st);
cudaError_t msm_points_bls12_381(uint32_t num, const uint64_t* offsets, const uint32_t* points,
                                 const uint32_t* scalars, uint32_t* out, cudaStream_t st);
cudaError_t msm_bases_bn254(void* bases, uint32_t num_vectors, const uint64_t* sizes,
                            const uint32_t* scalars,
                            uint32_t* out, cudaStream_t st);
cudaError_t msm_bases_bls12_381(void* bases, uint32_t num_vectors, const uint64_t* sizes,
                                const uint32_t* scalars,
                                uint32_t* out, cudaStream_t st);
cudaError_t points_to_mont(int curve, const uint32_t* in, uint64_t n, uint32_t* out,
                           cudaStream_t st);
cudaError_t bases_precompute_bn254(void* bases, int c, cudaStream_t st);
cudaError_t msm_points_dev_bn254(uint32_t num, uint64_t cap, const uint64_t* offsets, int c,
                                 const uint32_t* points, const uint32_t* scalars, uint32_t* out,
                                 cudaStream_t st);
cudaError_t msm_points_dev_bls12_381(uint32_t num, uint64_t cap, const uint64_t* offsets, int c,
                                     const uint32_t* points, const uint32_t* scalars, uint32_t* out,
                                     cudaStream_t st);
cudaError_t msm_bases_dev_bn254(void* bases, uint32_t num, uint64_t cap, const uint64_t* sizes, int c,
                                const uint32_t* scalars, uint32_t* out, cudaStream_t st);
cudaError_t msm_bases_dev_bls12_381(void* bases, uint32_t num, uint64_t cap, const uint64_t* sizes, int c,
                                    const uint32_t* scalars, uint32_t* out, cudaStream_t st);
cudaError_t bases_precompute_bls12_381(void* bases, int c, cudaStream_t st);

namespace {

std::mutex g_win_mu;
std::map<std::pair<int, int>, int> g_window_table;  // (curve, floor(log2 n)) -> c
std::map<std::pair<int, int>, int> g_chunk_table;   // (curve, floor(log2 n)) -> red_log

// Cost model: one batched addition (6 modmul) per (point, window) digit plus the
// bucket reduction, about two and a half batched additions per bucket (the walk's
// A and S events and the fold's share).
int model_window(int curve, uint64_t n) {
  int best = 4;
  double best_cost = 1e300;
  for (int c = 4; c <= 20; ++c) {
    const double W = msm_detail::windows_for(curve, c);
    const double cost = (double)n * W * 6.0 + W * (double)(1u << (c - 1)) * 15.0;
    if (cost < best_cost) {
      best_cost = cost;
      best = c;
    }
  }
  return best;
}

int ilog2(uint64_t n) {
  int l = 0;
  while ((n >> 1) > 0) {
    n >>= 1;
    ++l;
  }
  return l;
}

}  // namespace

int msm_window(int curve, uint64_t n) {
  if (n < 2) n = 2;
  {
    std::lock_guard<std::mutex> lock(g_win_mu);
    auto it = g_window_table.find({curve, ilog2(n)});
    if (it != g_window_table.end()) return it->second;
  }
  return model_window(curve, n);
}

void msm_set_window(int curve, int log2n, int c) {
  std::lock_guard<std::mutex> lock(g_win_mu);
  if (c <= 0) {
    g_window_table.erase({curve, log2n});
  } else {
    g_window_table[{curve, log2n}] = c;
  }
}

namespace {

std::atomic<bool> g_phase_on{false};

// One set of boundary events per host thread (and device), created on first use.
struct PhaseClock {
  int dev = -1;
  cudaEvent_t ev[kMsmPhases + 1] = {};
  bool marked[kMsmPhases + 1] = {};
  ~PhaseClock() {
    for (auto& e : ev)
      if (e) cudaEventDestroy(e);
  }
};
thread_local PhaseClock t_clock;

}  // namespace

void set_phase_timing(bool on) { g_phase_on.store(on); }

void phase_mark(int i, cudaStream_t st) {
  if (!g_phase_on.load() || i < 0 || i > kMsmPhases) return;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
    cudaGetLastError();
    return;
  }
  int dev = 0;
  cudaGetDevice(&dev);
  PhaseClock& pc = t_clock;
  if (pc.dev != dev) {
    for (auto& e : pc.ev) {
      if (e) cudaEventDestroy(e);
      e = nullptr;
    }
    pc.dev = dev;
  }
  if (!pc.ev[i] && cudaEventCreate(&pc.ev[i]) != cudaSuccess) {
    cudaGetLastError();
    return;
  }
  if (i == 0)
    for (auto& m : pc.marked) m = false;
  pc.marked[i] = cudaEventRecord(pc.ev[i], st) == cudaSuccess;
}

bool phase_times(float* ms) {
  PhaseClock& pc = t_clock;
  for (int i = 0; i <= kMsmPhases; ++i)
    if (!pc.marked[i]) return false;
  if (cudaEventSynchronize(pc.ev[kMsmPhases]) != cudaSuccess) return false;
  for (int i = 0; i < kMsmPhases; ++i)
    if (cudaEventElapsedTime(&ms[i], pc.ev[i], pc.ev[i + 1]) != cudaSuccess) return false;
  return true;
}

int msm_reduce_log(int curve, uint64_t n) {
  if (n < 2) n = 2;
  std::lock_guard<std::mutex> lock(g_win_mu);
  auto it = g_chunk_table.find({curve, ilog2(n)});
  return it != g_chunk_table.end() ? it->second : kRedLog1Default;
}

void msm_set_reduce_log(int curve, int log2n, int v) {
  std::lock_guard<std::mutex> lock(g_win_mu);
  if (v <= 0) {
    g_chunk_table.erase({curve, log2n});
  } else {
    g_chunk_table[{curve, log2n}] = v;
  }
}

cudaError_t launch_msm_dev(int curve, uint32_t num, uint64_t cap, const uint64_t* offsets, int c,
                           const uint32_t* points, const uint32_t* scalars, uint32_t* out,
                           cudaStream_t st) {
  if (c <= 0) c = msm_window(curve, num ? std::max<uint64_t>(cap / num, 2) : 2);
  switch (curve) {
    case 2: return msm_points_dev_bn254(num, cap, offsets, c, points, scalars, out, st);
    case 3: return msm_points_dev_bls12_381(num, cap, offsets, c, points, scalars, out, st);
  }
  return cudaErrorNotSupported;
}

cudaError_t launch_msm_bases_dev(void* handle, uint32_t num, uint64_t cap, const uint64_t* sizes, int c,
                                 const uint32_t* scalars, uint32_t* out, cudaStream_t st) {
  const int curve = bases_curve(handle);
  if (c <= 0) c = msm_window(curve, num ? std::max<uint64_t>(cap / num, 2) : 2);
  switch (curve) {
    case 2: return msm_bases_dev_bn254(handle, num, cap, sizes, c, scalars, out, st);
    case 3: return msm_bases_dev_bls12_381(handle, num, cap, sizes, c, scalars, out, st);
  }
  return cudaErrorNotSupported;
}

cudaError_t launch_msm(int curve, uint32_t num, const uint64_t* offsets, const uint32_t* points,
                       const uint32_t* scalars, uint32_t* out, cudaStream_t st) {
  switch (curve) {
    case 2: return msm_points_bn254(num, offsets, points, scalars, out, st);
    case 3: return msm_points_bls12_381(num, offsets, points, scalars, out, st);
  }
  return cudaErrorNotSupported;
}

cudaError_t bases_create(int curve, uint64_t n, const uint32_t* points, void** handle,
                         cudaStream_t st) {
  if (curve != 2 && curve != 3) return cudaErrorNotSupported;
  const int N = curve == 3 ? 12 : 8;
  uint32_t* m = nullptr;
  cudaError_t e = cudaMalloc(&m, std::max<uint64_t>(n, 1) * 2 * N * 4);
  if (e != cudaSuccess) return e;
  if (n) e = points_to_mont(curve, points, n, m, st);
  if (e != cudaSuccess) {
    cudaFree(m);
    return e;
  }
  *handle = new msm_detail::Bases{curve, n, m};
  return cudaSuccess;
}

int bases_curve(void* handle) { return static_cast<msm_detail::Bases*>(handle)->curve; }
uint64_t bases_count(void* handle) { return static_cast<msm_detail::Bases*>(handle)->n; }

cudaError_t bases_destroy(void* handle) {
  auto* b = static_cast<msm_detail::Bases*>(handle);
  cudaError_t e = cudaFree(b->mont);
  if (b->pre) {
    const cudaError_t e2 = cudaFree(b->pre);
    if (e == cudaSuccess) e = e2;
  }
  delete b;
  return e;
}

int bases_window(void* handle) { return static_cast<msm_detail::Bases*>(handle)->pre_c; }

void msm_counts(int curve, uint64_t num, const uint64_t* sizes, uint64_t size_all, int pre_c,
                uint64_t* digits, uint64_t* buckets) {
  uint64_t d = 0, b = 0;
  for (uint64_t i = 0; i < num; ++i) {
    const uint64_t n = sizes ? sizes[i] : size_all;
    const int c = pre_c > 0 ? pre_c : msm_window(curve, n);
    const uint64_t W = (uint64_t)msm_detail::windows_for(curve, c);
    d += W * n;
    b += (pre_c > 0 ? 1 : W) << (c - 1);
  }
  *digits = d;
  *buckets = b;
}

cudaError_t bases_precompute(void* handle, int c, cudaStream_t st) {
  switch (bases_curve(handle)) {
    case 2: return bases_precompute_bn254(handle, c, st);
    case 3: return bases_precompute_bls12_381(handle, c, st);
  }
  return cudaErrorNotSupported;
}

cudaError_t launch_msm_bases(void* handle, uint32_t num_vectors, const uint64_t* sizes,
                             const uint32_t* scalars,
                             uint32_t* out, cudaStream_t st) {
  switch (bases_curve(handle)) {
    case 2: return msm_bases_bn254(handle, num_vectors, sizes, scalars, out, st);
    case 3: return msm_bases_bls12_381(handle, num_vectors, sizes, scalars, out, st);
  }
  return cudaErrorNotSupported;
}

}  // namespace ecc
