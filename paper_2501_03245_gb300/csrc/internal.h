// Host-side interface between the C ABI (abi.cu) and the kernel translation
// units.  All pointers are device pointers; all launches are asynchronous on
// `st` and report launch errors through the returned cudaError_t.
#pragma once
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <string>

namespace ecc {

// Stream-ordered device scratch, released at scope exit (cudaFreeAsync on the
// same stream, so later work on the stream may still be using it safely), or
// through the caller's allocator hook when one is installed.
struct Scratch {
  void* ptr = nullptr;
  cudaStream_t st = nullptr;
  size_t bytes = 0;
  bool hooked = false;
  Scratch() = default;
  Scratch(const Scratch&) = delete;
  Scratch& operator=(const Scratch&) = delete;
  ~Scratch() { release(); }
  void release();
  cudaError_t alloc(size_t b, cudaStream_t s);
  template <class T>
  T* as() const {
    return reinterpret_cast<T*>(ptr);
  }
};

int device_sm_count();
std::string cuda_msg(cudaError_t e);

// field layer: curve 0..3, field 0 = base, 1 = scalar
cudaError_t launch_fe_mul(int curve, int field, size_t n, const uint32_t* a, const uint32_t* b,
                          uint32_t* out, cudaStream_t st);
cudaError_t launch_fe_addsub(int curve, int field, size_t n, const uint32_t* a,
                             const uint32_t* b, uint32_t* out, int subtract, cudaStream_t st);
cudaError_t launch_fe_inv(int curve, int field, size_t n, const uint32_t* a, uint32_t* out,
                          cudaStream_t st);
cudaError_t launch_fe_inv_batch(int curve, int field, size_t n, const uint32_t* a, uint32_t* out,
                                cudaStream_t st);
int field_limbs(int curve, int field);
// Allocation-free batch inversion: scratch is a fixed device array sized for
// kNoAllocMaxElems elements; a, out must be device memory.
constexpr size_t kNoAllocMaxElems = (size_t)1 << 16;
cudaError_t launch_fe_inv_batch_noalloc(int curve, int field, size_t n, const uint32_t* a,
                                        uint32_t* out, cudaStream_t st);

// EC operators
cudaError_t launch_point_add(int curve, size_t n, const uint32_t* p, const uint32_t* q,
                             uint32_t* out, int dbl, cudaStream_t st);
// Curve supplied at run time (k_custom.cu): the 8-limb Montgomery constants of
// an odd prime p < 2^256 and the curve's a in Montgomery form.
struct CustomConsts {
  uint32_t p[8], r2[8], one[8], pm2[8], r3[8], a[8];
  uint32_t qinv, pad;
  uint64_t qinv62;
};
// 0 on success; 1 p even, 2 p < 5, 3 a >= p.
int custom_consts(const uint32_t* p, const uint32_t* a, CustomConsts* cc);
cudaError_t launch_point_add_custom(const CustomConsts& cc, size_t n, const uint32_t* p,
                                    const uint32_t* q, uint32_t* out, int dbl, cudaStream_t st);
// ok[i] = 1 when point i is O ((0, 0)) or canonical and on the curve (Eqn 1)
cudaError_t launch_validate_points(int curve, size_t n, const uint32_t* p, uint8_t* ok, cudaStream_t st);
// Fixed-base table of a curve on the current device (built on first use,
// synchronously on `st`): 32 x 256 entries, entry j*256+v = v 2^(8j) G, SoA
// Montgomery (x block then y block).
cudaError_t gtable(int curve, const uint4** table, cudaStream_t st);

// ECDSA verification in clusters of `ctas` (1 or 2) CTAs sharing each round's
// inversion
void set_gas_cluster(int ctas);

// FPMUL k_i G (scalars n x 8 LE limbs; out n x 2N LE limbs)
cudaError_t launch_fixed_base_mul(int curve, size_t n, const uint32_t* k, uint32_t* out,
                                  cudaStream_t st);

// ECDSA
cudaError_t launch_sign(int curve, size_t n, const uint8_t* d, const uint8_t* e, const uint8_t* k,
                        uint8_t* r, uint8_t* s, uint8_t* pub, cudaStream_t st);
cudaError_t launch_verify(int curve, size_t n, const uint8_t* hash, const uint8_t* r,
                          const uint8_t* s, const uint8_t* pub, uint8_t* ok, cudaStream_t st);

// MSM: `num` instances, instance i = points / scalars rows
// [offsets[i] - offsets[0], offsets[i+1] - offsets[0]) (host offsets); out: num x 2N limbs
int msm_window(int curve, uint64_t n);
void msm_set_window(int curve, int log2n, int c);
// log2 of the buckets per first-level reduction chunk for an n-point MSM, and
// the autotuner's override for the size class log2n (0 restores the default)
int msm_reduce_log(int curve, uint64_t n);
void msm_set_reduce_log(int curve, int log2n, int v);
constexpr int kMsmReduceLogMax = 10;
cudaError_t launch_msm(int curve, uint32_t num, const uint64_t* offsets, const uint32_t* points,
                       const uint32_t* scalars, uint32_t* out, cudaStream_t st);
cudaError_t bases_create(int curve, uint64_t n, const uint32_t* points, void** handle,
                         cudaStream_t st);
cudaError_t bases_destroy(void* handle);
cudaError_t bases_precompute(void* handle, int c, cudaStream_t st);
int bases_window(void* handle);
// (point, window) digits and buckets of a batch of num MSMs (sizes, or
// size_all each when sizes is null) at the window widths the planner picks;
// the sort and reduction index both with 32-bit words.
void msm_counts(int curve, uint64_t num, const uint64_t* sizes, uint64_t size_all, int pre_c,
                uint64_t* digits, uint64_t* buckets);
constexpr uint64_t kMsmMaxDigits = 1ull << 31;
int bases_curve(void* handle);
uint64_t bases_count(void* handle);
cudaError_t launch_msm_bases(void* handle, uint32_t num_vectors, const uint64_t* sizes,
                             const uint32_t* scalars,
                             uint32_t* out, cudaStream_t st);

// MSM phase timers (diagnostics): with timing on, phase_mark(i, st) records
// boundary event i (0 .. kMsmPhases) of the calling thread's current MSM call
// on st; nothing is recorded while st is being captured into a graph.
constexpr int kMsmPhases = 5;  // sort, accumulation, fold, reduction, combination
void set_phase_timing(bool on);
void phase_mark(int i, cudaStream_t st);
// Device milliseconds of each phase of the thread's last timed call (waits for
// it); returns false if no complete timed call exists.
bool phase_times(float* ms);

// Device status word of the current device (library-owned, zero when no
// device-side error is pending): kernels that detect an error record its
// negative ECC_E* code with atomicCAS(word, 0, code).
int* status_word();

// Ragged MSMs whose instance sizes are in device memory (capacity cap rows,
// one window width c for every instance; 0 picks the library's width for the
// mean size cap / num).
cudaError_t launch_msm_dev(int curve, uint32_t num, uint64_t cap, const uint64_t* offsets, int c,
                           const uint32_t* points, const uint32_t* scalars, uint32_t* out,
                           cudaStream_t st);
cudaError_t launch_msm_bases_dev(void* handle, uint32_t num, uint64_t cap, const uint64_t* sizes, int c,
                                 const uint32_t* scalars, uint32_t* out, cudaStream_t st);

// benchmarks
cudaError_t launch_bench_imad(size_t threads, int iters, uint32_t* sink, cudaStream_t st);
cudaError_t launch_bench_modmul(int curve, int reduction, size_t threads, int iters, uint32_t* sink,
                                cudaStream_t st);
cudaError_t launch_bench_inv(int curve, int method, size_t threads, int iters, uint32_t* sink,
                             cudaStream_t st);

}  // namespace ecc
