// C ABI (include/gecc.h): argument checks, host-memory staging, error strings.
#include <cstdarg>
#include <cstdio>
#include <algorithm>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/gecc.h"
#include "internal.h"

namespace ecc {

namespace {

thread_local char g_err[512] = "";

int fail(int code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof g_err, fmt, ap);
  va_end(ap);
  return code;
}

int ok() {
  g_err[0] = 0;
  return ECC_OK;
}

int cuda_fail(cudaError_t e, const char* where) {
  if (e == cudaErrorMemoryAllocation) return fail(ECC_ENOMEM, "%s: %s", where, cudaGetErrorString(e));
  return fail(ECC_ECUDA, "%s: %s", where, cudaGetErrorString(e));
}

bool host_memory(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return true;
  }
  return at.type == cudaMemoryTypeHost || at.type == cudaMemoryTypeUnregistered;
}

bool aligned4(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 3u) == 0; }

// Device view of a caller array: the array itself when it is device memory,
// otherwise a stream-ordered device copy (inputs copied in; outputs copied back
// by flush()).
struct Arg {
  const void* user;
  void* dev = nullptr;
  size_t bytes;
  bool staged = false;
  Scratch buf;
  Arg(const void* p, size_t b) : user(p), bytes(b) {}
  cudaError_t in(cudaStream_t st) {
    if (!host_memory(user)) {
      dev = const_cast<void*>(user);
      return cudaSuccess;
    }
    staged = true;
    cudaError_t e = buf.alloc(bytes, st);
    if (e != cudaSuccess) return e;
    dev = buf.ptr;
    return cudaMemcpyAsync(dev, user, bytes, cudaMemcpyHostToDevice, st);
  }
  cudaError_t out(cudaStream_t st) {
    if (!host_memory(user)) {
      dev = const_cast<void*>(user);
      return cudaSuccess;
    }
    staged = true;
    cudaError_t e = buf.alloc(bytes, st);
    dev = buf.ptr;
    return e;
  }
  cudaError_t flush(cudaStream_t st) {
    if (!staged) return cudaSuccess;
    return cudaMemcpyAsync(const_cast<void*>(user), dev, bytes, cudaMemcpyDeviceToHost, st);
  }
};

bool valid_curve(int c) { return c >= 0 && c <= 4; }

// Runs `body` with device views of the inputs/outputs; synchronises when any
// of them was staged from host memory.
template <class Body>
int with_args(const char* name, cudaStream_t st, std::vector<Arg*> ins, std::vector<Arg*> outs,
              Body body) {
  for (Arg* a : ins) {
    cudaError_t e = a->in(st);
    if (e != cudaSuccess) return cuda_fail(e, name);
  }
  for (Arg* a : outs) {
    cudaError_t e = a->out(st);
    if (e != cudaSuccess) return cuda_fail(e, name);
  }
  cudaError_t e = body();
  if (e != cudaSuccess) return cuda_fail(e, name);
  bool staged = false;
  for (Arg* a : ins) staged |= a->staged;
  for (Arg* a : outs) {
    staged |= a->staged;
    e = a->flush(st);
    if (e != cudaSuccess) return cuda_fail(e, name);
  }
  if (staged) {
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, name);
  }
  return ok();
}

}  // namespace

namespace {

// Caller-installed workspace allocator (ecc_set_allocator); null: stream-ordered
// cudaMallocAsync / cudaFreeAsync.
std::mutex g_alloc_mu;
ecc_alloc_fn g_alloc = nullptr;
ecc_free_fn g_free = nullptr;
void* g_alloc_ctx = nullptr;

// Device status word (one per device that loads the library).
__device__ int g_status;
std::mutex g_status_mu;
int* g_status_ptr[64] = {};

}  // namespace

int* status_word() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> lock(g_status_mu);
  if (!g_status_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_status) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    g_status_ptr[dev] = static_cast<int*>(p);
  }
  return g_status_ptr[dev];
}

void Scratch::release() {
  if (!ptr) return;
  if (hooked) {
    ecc_free_fn f;
    void* ctx;
    {
      std::lock_guard<std::mutex> lock(g_alloc_mu);
      f = g_free;
      ctx = g_alloc_ctx;
    }
    if (f) f(ptr, st, ctx);
  } else {
    cudaFreeAsync(ptr, st);
  }
  ptr = nullptr;
}

cudaError_t Scratch::alloc(size_t b, cudaStream_t s) {
  release();
  st = s;
  bytes = b;
  if (b == 0) b = 16;
  {
    ecc_alloc_fn f;
    void* ctx;
    {
      std::lock_guard<std::mutex> lock(g_alloc_mu);
      f = g_alloc;
      ctx = g_alloc_ctx;
    }
    if (f) {
      hooked = true;
      ptr = f(b, s, ctx);
      return ptr ? cudaSuccess : cudaErrorMemoryAllocation;
    }
  }
  hooked = false;
  static bool pool_set = false;
  if (!pool_set) {
    // keep freed stream-ordered memory cached in the pool between calls
    int dev = 0;
    cudaMemPool_t pool;
    if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
      uint64_t thr = UINT64_MAX;
      cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    pool_set = true;
  }
  return cudaMallocAsync(&ptr, b, s);
}

int device_sm_count() {
  static int cache[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return 1;
  if (!cache[dev]) {
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    cache[dev] = v > 0 ? v : 1;
  }
  return cache[dev];
}

std::string cuda_msg(cudaError_t e) { return cudaGetErrorString(e); }

}  // namespace ecc

using namespace ecc;

extern "C" {

const char* ecc_last_error(void) { return g_err; }

const char* ecc_version(void) { return "gecc-gb300 0.1"; }

int ecc_limbs(ecc_curve_t curve) {
  if (!valid_curve(curve)) return fail(ECC_EINVAL, "ecc_limbs: unknown curve %d", (int)curve);
  return field_limbs(curve, 0);
}

static int fp_binary(const char* name, int op, ecc_curve_t curve, int field, size_t n,
                     const uint32_t* a, const uint32_t* b, uint32_t* out, void* stream) {
  if (!valid_curve(curve)) return fail(ECC_EINVAL, "%s: unknown curve %d", name, (int)curve);
  if (field != 0 && field != 1) return fail(ECC_EINVAL, "%s: field must be 0 or 1", name);
  if (n == 0) return ok();
  if (!a || !out || (op < 3 && !b)) return fail(ECC_EINVAL, "%s: NULL pointer", name);
  if (!aligned4(a) || !aligned4(out) || (b && !aligned4(b)))
    return fail(ECC_EINVAL, "%s: pointers must be 4-byte aligned", name);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t bytes = n * field_limbs(curve, field) * 4;
  Arg A(a, bytes), B(b ? b : a, bytes), O(out, bytes);
  std::vector<Arg*> ins{&A};
  if (op < 3) ins.push_back(&B);
  return with_args(name, st, ins, {&O}, [&]() {
    const uint32_t* da = static_cast<const uint32_t*>(A.dev);
    const uint32_t* db = static_cast<const uint32_t*>(B.dev);
    uint32_t* dout = static_cast<uint32_t*>(O.dev);
    switch (op) {
      case 0: return launch_fe_mul(curve, field, n, da, db, dout, st);
      case 1: return launch_fe_addsub(curve, field, n, da, db, dout, 0, st);
      case 2: return launch_fe_addsub(curve, field, n, da, db, dout, 1, st);
      case 3: return launch_fe_inv(curve, field, n, da, dout, st);
      default: return launch_fe_inv_batch(curve, field, n, da, dout, st);
    }
  });
}

int ecc_fp_mul(ecc_curve_t curve, int field, size_t n, const uint32_t* a, const uint32_t* b,
               uint32_t* out, void* stream) {
  return fp_binary("ecc_fp_mul", 0, curve, field, n, a, b, out, stream);
}

int ecc_fp_add(ecc_curve_t curve, int field, size_t n, const uint32_t* a, const uint32_t* b,
               uint32_t* out, void* stream) {
  return fp_binary("ecc_fp_add", 1, curve, field, n, a, b, out, stream);
}

int ecc_fp_sub(ecc_curve_t curve, int field, size_t n, const uint32_t* a, const uint32_t* b,
               uint32_t* out, void* stream) {
  return fp_binary("ecc_fp_sub", 2, curve, field, n, a, b, out, stream);
}

int ecc_fp_inv(ecc_curve_t curve, int field, size_t n, const uint32_t* a, uint32_t* out,
               void* stream) {
  return fp_binary("ecc_fp_inv", 3, curve, field, n, a, nullptr, out, stream);
}

int ecc_fp_inv_batch(ecc_curve_t curve, int field, size_t n, const uint32_t* a, uint32_t* out,
                     void* stream) {
  return fp_binary("ecc_fp_inv_batch", 4, curve, field, n, a, nullptr, out, stream);
}

static int point_op(const char* name, ecc_curve_t curve, size_t n, const uint32_t* p,
                    const uint32_t* q, uint32_t* out, int dbl, void* stream) {
  if (!valid_curve(curve)) return fail(ECC_EINVAL, "%s: unknown curve %d", name, (int)curve);
  if (n == 0) return ok();
  if (!p || !out || (!dbl && !q)) return fail(ECC_EINVAL, "%s: NULL pointer", name);
  if (!aligned4(p) || !aligned4(out) || (q && !aligned4(q)))
    return fail(ECC_EINVAL, "%s: pointers must be 4-byte aligned", name);
  if (n > (size_t)1 << 30) return fail(ECC_EINVAL, "%s: n > 2^30", name);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t bytes = n * 2 * field_limbs(curve, 0) * 4;
  Arg P(p, bytes), Q(q ? q : p, bytes), O(out, bytes);
  std::vector<Arg*> ins{&P};
  if (!dbl) ins.push_back(&Q);
  return with_args(name, st, ins, {&O}, [&]() {
    return launch_point_add(curve, n, static_cast<const uint32_t*>(P.dev),
                            static_cast<const uint32_t*>(Q.dev), static_cast<uint32_t*>(O.dev),
                            dbl, st);
  });
}

int ecc_point_add_batch(ecc_curve_t curve, size_t n, const uint32_t* p, const uint32_t* q,
                        uint32_t* out, void* stream) {
  return point_op("ecc_point_add_batch", curve, n, p, q, out, 0, stream);
}

int ecc_point_dbl_batch(ecc_curve_t curve, size_t n, const uint32_t* p, uint32_t* out,
                        void* stream) {
  return point_op("ecc_point_dbl_batch", curve, n, p, nullptr, out, 1, stream);
}

int ecc_point_op_custom(const uint32_t* prime, const uint32_t* a, size_t n, const uint32_t* p,
                        const uint32_t* q, uint32_t* out, int dbl, void* stream) {
  const char* name = "ecc_point_op_custom";
  if (!prime || !a) return fail(ECC_EINVAL, "%s: NULL curve parameter", name);
  if (!host_memory(prime) || !host_memory(a))
    return fail(ECC_EINVAL, "%s: prime and a must be host memory", name);
  CustomConsts cc;
  switch (custom_consts(prime, a, &cc)) {
    case 0: break;
    case 1: return fail(ECC_EINVAL, "%s: the prime must be odd", name);
    case 2: return fail(ECC_EINVAL, "%s: the prime must be at least 5", name);
    default: return fail(ECC_EINVAL, "%s: a must be below the prime", name);
  }
  if (n == 0) return ok();
  if (!p || !out || (!dbl && !q)) return fail(ECC_EINVAL, "%s: NULL pointer", name);
  if (!aligned4(p) || !aligned4(out) || (q && !aligned4(q)))
    return fail(ECC_EINVAL, "%s: pointers must be 4-byte aligned", name);
  if (n > (size_t)1 << 30) return fail(ECC_EINVAL, "%s: n > 2^30", name);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t bytes = n * 16 * 4;
  Arg P(p, bytes), Q(q ? q : p, bytes), O(out, bytes);
  std::vector<Arg*> ins{&P};
  if (!dbl) ins.push_back(&Q);
  return with_args(name, st, ins, {&O}, [&]() {
    return launch_point_add_custom(cc, n, static_cast<const uint32_t*>(P.dev),
                                   static_cast<const uint32_t*>(Q.dev), static_cast<uint32_t*>(O.dev),
                                   dbl, st);
  });
}

int ecc_verify_batch(ecc_curve_t curve, size_t n, const uint8_t* hash, const uint8_t* r,
                     const uint8_t* s, const uint8_t* pubkey, uint8_t* ok_out, void* stream) {
  const char* name = "ecc_verify_batch";
  if (!valid_curve(curve)) return fail(ECC_EINVAL, "%s: unknown curve %d", name, (int)curve);
  if (curve != ECC_SECP256K1 && curve != ECC_P256 && curve != ECC_SM2)
    return fail(ECC_EUNSUPPORTED, "%s: ECDSA is offered on secp256k1, P-256 and SM2", name);
  if (n == 0) return ok();
  if (!hash || !r || !s || !pubkey || !ok_out) return fail(ECC_EINVAL, "%s: NULL pointer", name);
  if (!aligned4(hash) || !aligned4(r) || !aligned4(s) || !aligned4(pubkey))
    return fail(ECC_EINVAL, "%s: input pointers must be 4-byte aligned", name);
  if (n > (size_t)1 << 26) return fail(ECC_EINVAL, "%s: n > 2^26", name);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Arg H(hash, 32 * n), R(r, 32 * n), S(s, 32 * n), Q(pubkey, 64 * n), O(ok_out, n);
  return with_args(name, st, {&H, &R, &S, &Q}, {&O}, [&]() {
    return launch_verify(curve, n, static_cast<const uint8_t*>(H.dev),
                         static_cast<const uint8_t*>(R.dev), static_cast<const uint8_t*>(S.dev),
                         static_cast<const uint8_t*>(Q.dev), static_cast<uint8_t*>(O.dev), st);
  });
}

int ecc_fixed_base_mul(ecc_curve_t curve, size_t n, const uint32_t* k, uint32_t* out,
                       void* stream) {
  const char* name = "ecc_fixed_base_mul";
  if (!valid_curve(curve)) return fail(ECC_EINVAL, "%s: unknown curve %d", name, (int)curve);
  if (n == 0) return ok();
  if (!k || !out) return fail(ECC_EINVAL, "%s: NULL pointer", name);
  if (!aligned4(k) || !aligned4(out)) return fail(ECC_EINVAL, "%s: pointers must be 4-byte aligned", name);
  if (n > (size_t)1 << 27) return fail(ECC_EINVAL, "%s: n > 2^27", name);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Arg K(k, 32 * n), O(out, n * 8 * field_limbs(curve, 0));
  return with_args(name, st, {&K}, {&O}, [&]() {
    return launch_fixed_base_mul(curve, n, static_cast<const uint32_t*>(K.dev),
                                 static_cast<uint32_t*>(O.dev), st);
  });
}

int ecc_sign_batch(ecc_curve_t curve, size_t n, const uint8_t* d, const uint8_t* e,
                   const uint8_t* k, uint8_t* r_out, uint8_t* s_out, uint8_t* pub_out,
                   void* stream) {
  const char* name = "ecc_sign_batch";
  if (!valid_curve(curve)) return fail(ECC_EINVAL, "%s: unknown curve %d", name, (int)curve);
  if (curve != ECC_SECP256K1 && curve != ECC_P256 && curve != ECC_SM2)
    return fail(ECC_EUNSUPPORTED, "%s: ECDSA is offered on secp256k1, P-256 and SM2", name);
  if (n == 0) return ok();
  if (!d || !e || !k || !r_out || !s_out || !pub_out) return fail(ECC_EINVAL, "%s: NULL pointer", name);
  if (!aligned4(d) || !aligned4(e) || !aligned4(k) || !aligned4(r_out) || !aligned4(s_out) ||
      !aligned4(pub_out))
    return fail(ECC_EINVAL, "%s: pointers must be 4-byte aligned", name);
  if (n > (size_t)1 << 26) return fail(ECC_EINVAL, "%s: n > 2^26", name);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Arg D(d, 32 * n), E(e, 32 * n), K(k, 32 * n), R(r_out, 32 * n), S(s_out, 32 * n), P(pub_out, 64 * n);
  return with_args(name, st, {&D, &E, &K}, {&R, &S, &P}, [&]() {
    return launch_sign(curve, n, static_cast<const uint8_t*>(D.dev), static_cast<const uint8_t*>(E.dev),
                       static_cast<const uint8_t*>(K.dev), static_cast<uint8_t*>(R.dev),
                       static_cast<uint8_t*>(S.dev), static_cast<uint8_t*>(P.dev), st);
  });
}

int ecc_msm_ragged(ecc_curve_t curve, size_t num, const uint64_t* offsets, const uint32_t* points,
                   const uint32_t* scalars, uint32_t* out, void* stream) {
  const char* name = "ecc_msm_ragged";
  if (!valid_curve(curve)) return fail(ECC_EINVAL, "%s: unknown curve %d", name, (int)curve);
  if (curve != ECC_BN254 && curve != ECC_BLS12_381)
    return fail(ECC_EUNSUPPORTED, "%s: MSM is offered on BN254 and BLS12-381", name);
  if (num == 0) return ok();
  if (!offsets || !out) return fail(ECC_EINVAL, "%s: NULL pointer", name);
  if (num > (1u << 20)) return fail(ECC_EINVAL, "%s: num > 2^20", name);
  if (!host_memory(offsets)) return fail(ECC_EINVAL, "%s: offsets must be host memory", name);
  for (size_t i = 0; i < num; ++i)
    if (offsets[i + 1] < offsets[i]) return fail(ECC_EINVAL, "%s: offsets must not decrease", name);
  const uint64_t rows = offsets[num] - offsets[0];
  if (rows > (1ull << 28)) return fail(ECC_EINVAL, "%s: more than 2^28 points", name);
  if (rows && (!points || !scalars)) return fail(ECC_EINVAL, "%s: NULL pointer", name);
  if ((points && !aligned4(points)) || (scalars && !aligned4(scalars)) || !aligned4(out))
    return fail(ECC_EINVAL, "%s: pointers must be 4-byte aligned", name);
  {
    std::vector<uint64_t> sz(num);
    for (size_t i = 0; i < num; ++i) sz[i] = offsets[i + 1] - offsets[i];
    uint64_t digits = 0, buckets = 0;
    msm_counts(curve, num, sz.data(), 0, 0, &digits, &buckets);
    if (digits >= kMsmMaxDigits || buckets >= kMsmMaxDigits)
      return fail(ECC_EINVAL, "%s: the batch needs 2^31 or more (point, window) digits or buckets; "
                  "split it", name);
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int L = field_limbs(curve, 0);
  const uint32_t* pb = points ? points + offsets[0] * 2 * L : points;
  const uint32_t* sb = scalars ? scalars + offsets[0] * 8 : scalars;
  std::vector<uint64_t> rel(num + 1);
  for (size_t i = 0; i <= num; ++i) rel[i] = offsets[i] - offsets[0];
  Arg P(pb ? pb : out, std::max<uint64_t>(rows, 1) * 2 * L * 4);
  Arg S(sb ? sb : out, std::max<uint64_t>(rows, 1) * 32);
  Arg O(out, num * 2 * L * 4);
  std::vector<Arg*> ins;
  if (rows) {
    ins.push_back(&P);
    ins.push_back(&S);
  }
  return with_args(name, st, ins, {&O}, [&]() {
    return launch_msm(curve, (uint32_t)num, rel.data(), static_cast<const uint32_t*>(P.dev),
                      static_cast<const uint32_t*>(S.dev), static_cast<uint32_t*>(O.dev), st);
  });
}

int ecc_msm(ecc_curve_t curve, size_t n, const uint32_t* points, const uint32_t* scalars,
            uint32_t* out, void* stream) {
  uint64_t off[2] = {0, n};
  int rc = ecc_msm_ragged(curve, 1, off, points, scalars, out, stream);
  if (rc != ECC_OK) {
    std::string m = g_err;
    size_t k = m.find("ecc_msm_ragged");
    if (k != std::string::npos) m.replace(k, 14, "ecc_msm");
    fail(rc, "%s", m.c_str());
  }
  return rc;
}

static bool msm_dev_sizes_ok(int curve, size_t num, size_t max_points, int c, int pre_c) {
  const int w = pre_c > 0 ? pre_c : (c > 0 ? c : msm_window(curve, num ? std::max<size_t>(max_points / num, 2) : 2));
  const uint64_t W = (uint64_t)((curve == ECC_BN254 ? 254 : 255) + 1 + w - 1) / w;
  const uint64_t rows = pre_c > 0 ? 1 : W;
  return (uint64_t)max_points * W < kMsmMaxDigits && (uint64_t)num * (rows << (w - 1)) < kMsmMaxDigits;
}

int ecc_msm_ragged_dev(ecc_curve_t curve, size_t num, size_t max_points, const uint64_t* offsets,
                       const uint32_t* points, const uint32_t* scalars, uint32_t* out, int c,
                       void* stream) {
  const char* name = "ecc_msm_ragged_dev";
  if (!valid_curve(curve)) return fail(ECC_EINVAL, "%s: unknown curve %d", name, (int)curve);
  if (curve != ECC_BN254 && curve != ECC_BLS12_381)
    return fail(ECC_EUNSUPPORTED, "%s: MSM is offered on BN254 and BLS12-381", name);
  if (num == 0) return ok();
  if (!offsets || !points || !scalars || !out) return fail(ECC_EINVAL, "%s: NULL pointer", name);
  if (num > (1u << 20)) return fail(ECC_EINVAL, "%s: num > 2^20", name);
  if (max_points == 0 || max_points > (1ull << 28))
    return fail(ECC_EINVAL, "%s: max_points must be in 1..2^28", name);
  if (c != 0 && (c < 2 || c > 20)) return fail(ECC_EINVAL, "%s: c must be 0 or 2..20", name);
  if (!aligned4(points) || !aligned4(scalars) || !aligned4(out) || (reinterpret_cast<uintptr_t>(offsets) & 7))
    return fail(ECC_EINVAL, "%s: pointers must be aligned (offsets to 8 bytes, the rest to 4)", name);
  if (host_memory(offsets) || host_memory(points) || host_memory(scalars) || host_memory(out))
    return fail(ECC_EINVAL, "%s: every array must be device memory", name);
  if (!msm_dev_sizes_ok(curve, num, max_points, c, 0))
    return fail(ECC_EINVAL, "%s: the capacity needs 2^31 or more (point, window) digits or buckets", name);
  cudaError_t e = launch_msm_dev(curve, (uint32_t)num, max_points, offsets, c, points, scalars, out,
                                 static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, name);
  return ok();
}

int ecc_msm_bases_ragged_dev(void* handle, size_t num, size_t max_points, const uint64_t* sizes,
                             const uint32_t* scalars, uint32_t* out, void* stream) {
  const char* name = "ecc_msm_bases_ragged_dev";
  if (!handle) return fail(ECC_EINVAL, "%s: NULL handle", name);
  if (num == 0) return ok();
  if (!sizes || !scalars || !out) return fail(ECC_EINVAL, "%s: NULL pointer", name);
  if (num > (1u << 20)) return fail(ECC_EINVAL, "%s: num > 2^20", name);
  if (max_points == 0 || max_points > (1ull << 28))
    return fail(ECC_EINVAL, "%s: max_points must be in 1..2^28", name);
  if (!aligned4(scalars) || !aligned4(out) || (reinterpret_cast<uintptr_t>(sizes) & 7))
    return fail(ECC_EINVAL, "%s: pointers must be aligned (sizes to 8 bytes, the rest to 4)", name);
  if (host_memory(sizes) || host_memory(scalars) || host_memory(out))
    return fail(ECC_EINVAL, "%s: every array must be device memory", name);
  if (!msm_dev_sizes_ok(bases_curve(handle), num, max_points, 0, bases_window(handle)))
    return fail(ECC_EINVAL, "%s: the capacity needs 2^31 or more (point, window) digits or buckets", name);
  cudaError_t e = launch_msm_bases_dev(handle, (uint32_t)num, max_points, sizes, 0, scalars, out,
                                       static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, name);
  return ok();
}

int ecc_sync_status(void* stream) {
  cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "ecc_sync_status");
  int* w = status_word();
  if (!w) return fail(ECC_ECUDA, "ecc_sync_status: no status word on this device");
  int v = 0;
  e = cudaMemcpy(&v, w, sizeof v, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && v != 0) {
    const int zero = 0;
    e = cudaMemcpy(w, &zero, sizeof zero, cudaMemcpyHostToDevice);
  }
  if (e != cudaSuccess) return cuda_fail(e, "ecc_sync_status");
  if (v == 0) return ok();
  return fail(v, "ecc_sync_status: a kernel reported error %d (%s)", v,
              v == ECC_EINVAL ? "refused device-resident sizes" : v == ECC_ETIMEOUT ? "a bounded wait gave up"
                                                                    : "device error");
}

int ecc_set_allocator(ecc_alloc_fn alloc, ecc_free_fn release, void* ctx) {
  if ((alloc == nullptr) != (release == nullptr))
    return fail(ECC_EINVAL, "ecc_set_allocator: give both functions or neither");
  std::lock_guard<std::mutex> lock(g_alloc_mu);
  g_alloc = alloc;
  g_free = release;
  g_alloc_ctx = ctx;
  return ok();
}

int ecc_validate_points(ecc_curve_t curve, size_t n, const uint32_t* points, uint8_t* ok_out,
                        void* stream) {
  const char* name = "ecc_validate_points";
  if (!valid_curve(curve)) return fail(ECC_EINVAL, "%s: unknown curve %d", name, (int)curve);
  if (n == 0) return ok();
  if (!points || !ok_out) return fail(ECC_EINVAL, "%s: NULL pointer", name);
  if (!aligned4(points)) return fail(ECC_EINVAL, "%s: points must be 4-byte aligned", name);
  if (n > (size_t)1 << 30) return fail(ECC_EINVAL, "%s: n > 2^30", name);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Arg P(points, n * 2 * field_limbs(curve, 0) * 4), O(ok_out, n);
  return with_args(name, st, {&P}, {&O}, [&]() {
    return launch_validate_points(curve, n, static_cast<const uint32_t*>(P.dev),
                                  static_cast<uint8_t*>(O.dev), st);
  });
}

int ecc_bases_create(ecc_curve_t curve, size_t n, const uint32_t* points, void** handle,
                     void* stream) {
  const char* name = "ecc_bases_create";
  if (!valid_curve(curve)) return fail(ECC_EINVAL, "%s: unknown curve %d", name, (int)curve);
  if (curve != ECC_BN254 && curve != ECC_BLS12_381)
    return fail(ECC_EUNSUPPORTED, "%s: MSM is offered on BN254 and BLS12-381", name);
  if (!handle || (n && !points)) return fail(ECC_EINVAL, "%s: NULL pointer", name);
  if (points && !aligned4(points)) return fail(ECC_EINVAL, "%s: pointers must be 4-byte aligned", name);
  if (n > (1ull << 28)) return fail(ECC_EINVAL, "%s: n > 2^28", name);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int L = field_limbs(curve, 0);
  Arg P(points ? points : (const uint32_t*)handle, std::max<size_t>(n, 1) * 2 * L * 4);
  std::vector<Arg*> ins;
  if (n) ins.push_back(&P);
  return with_args(name, st, ins, {}, [&]() {
    return bases_create(curve, n, static_cast<const uint32_t*>(P.dev), handle, st);
  });
}

int ecc_msm_bases(void* handle, size_t num_vectors, const uint32_t* scalars, uint32_t* out,
                  void* stream) {
  const char* name = "ecc_msm_bases";
  if (!handle) return fail(ECC_EINVAL, "%s: NULL handle", name);
  if (num_vectors == 0) return ok();
  if (!scalars || !out) return fail(ECC_EINVAL, "%s: NULL pointer", name);
  if (!aligned4(scalars) || !aligned4(out)) return fail(ECC_EINVAL, "%s: pointers must be 4-byte aligned", name);
  if (num_vectors > 4096) return fail(ECC_EINVAL, "%s: num_vectors > 4096", name);
  const int curve = bases_curve(handle);
  const uint64_t n = bases_count(handle);
  uint64_t digits = 0, buckets = 0;
  msm_counts(curve, num_vectors, nullptr, n, bases_window(handle), &digits, &buckets);
  if (digits >= kMsmMaxDigits || buckets >= kMsmMaxDigits)
    return fail(ECC_EINVAL, "%s: the call needs 2^31 or more (point, window) digits or buckets; "
                "use fewer vectors per call", name);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int L = field_limbs(curve, 0);
  Arg S(scalars, std::max<uint64_t>(n, 1) * num_vectors * 32), O(out, num_vectors * 2 * L * 4);
  return with_args(name, st, {&S}, {&O}, [&]() {
    return launch_msm_bases(handle, (uint32_t)num_vectors, nullptr, static_cast<const uint32_t*>(S.dev),
                            static_cast<uint32_t*>(O.dev), st);
  });
}

int ecc_msm_bases_ragged(void* handle, size_t num, const uint64_t* sizes, const uint32_t* scalars,
                         uint32_t* out, void* stream) {
  const char* name = "ecc_msm_bases_ragged";
  if (!handle) return fail(ECC_EINVAL, "%s: NULL handle", name);
  if (num == 0) return ok();
  if (!sizes || !out) return fail(ECC_EINVAL, "%s: NULL pointer", name);
  if (!host_memory(sizes)) return fail(ECC_EINVAL, "%s: sizes must be host memory", name);
  if (num > (1u << 20)) return fail(ECC_EINVAL, "%s: num > 2^20", name);
  const uint64_t n = bases_count(handle);
  uint64_t rows = 0;
  for (size_t i = 0; i < num; ++i) {
    if (sizes[i] > n) return fail(ECC_EINVAL, "%s: sizes[%zu] exceeds the %llu resident bases", name, i,
                                  (unsigned long long)n);
    rows += sizes[i];
  }
  if (rows && !scalars) return fail(ECC_EINVAL, "%s: NULL pointer", name);
  if ((scalars && !aligned4(scalars)) || !aligned4(out))
    return fail(ECC_EINVAL, "%s: pointers must be 4-byte aligned", name);
  {
    uint64_t digits = 0, buckets = 0;
    msm_counts(bases_curve(handle), num, sizes, 0, bases_window(handle), &digits, &buckets);
    if (digits >= kMsmMaxDigits || buckets >= kMsmMaxDigits)
      return fail(ECC_EINVAL, "%s: the call needs 2^31 or more (point, window) digits or buckets; "
                  "split it", name);
  }
  const int curve = bases_curve(handle);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int L = field_limbs(curve, 0);
  Arg S(scalars ? scalars : out, std::max<uint64_t>(rows, 1) * 32), O(out, num * 2 * L * 4);
  std::vector<Arg*> ins;
  if (rows) ins.push_back(&S);
  return with_args(name, st, ins, {&O}, [&]() {
    return launch_msm_bases(handle, (uint32_t)num, sizes, static_cast<const uint32_t*>(S.dev),
                            static_cast<uint32_t*>(O.dev), st);
  });
}

int ecc_bases_precompute(void* handle, int c, void* stream) {
  const char* name = "ecc_bases_precompute";
  if (!handle) return fail(ECC_EINVAL, "%s: NULL handle", name);
  if (c < 2 || c > 24) return fail(ECC_EINVAL, "%s: window width %d outside 2..24", name, c);
  cudaError_t e = bases_precompute(handle, c, static_cast<cudaStream_t>(stream));
  if (e == cudaErrorInvalidValue)
    return fail(ECC_EINVAL, "%s: windows x bases must stay below 2^31 points", name);
  if (e == cudaErrorMemoryAllocation) return fail(ECC_ENOMEM, "%s: out of device memory", name);
  if (e != cudaSuccess) return cuda_fail(e, name);
  return ok();
}

int ecc_bases_window(void* handle) {
  if (!handle) return fail(ECC_EINVAL, "ecc_bases_window: NULL handle");
  return bases_window(handle);
}

int ecc_bases_destroy(void* handle) {
  if (!handle) return fail(ECC_EINVAL, "ecc_bases_destroy: NULL handle");
  cudaError_t e = bases_destroy(handle);
  if (e != cudaSuccess) return cuda_fail(e, "ecc_bases_destroy");
  return ok();
}

int ecc_msm_window(ecc_curve_t curve, size_t n) {
  if (!valid_curve(curve)) return fail(ECC_EINVAL, "ecc_msm_window: unknown curve %d", (int)curve);
  return msm_window(curve, n);
}

int ecc_msm_set_window(ecc_curve_t curve, int log2_n, int c) {
  if (!valid_curve(curve)) return fail(ECC_EINVAL, "ecc_msm_set_window: unknown curve %d", (int)curve);
  if (log2_n < 0 || log2_n > 40 || c < 0 || c > 20 || c == 1)
    return fail(ECC_EINVAL, "ecc_msm_set_window: need 0 <= log2_n <= 40 and c = 0 or 2..20");
  msm_set_window(curve, log2_n, c);
  return ok();
}

int ecc_msm_reduce_chunk(ecc_curve_t curve, size_t n) {
  if (!valid_curve(curve)) return fail(ECC_EINVAL, "ecc_msm_reduce_chunk: unknown curve %d", (int)curve);
  return msm_reduce_log(curve, n);
}

int ecc_msm_set_reduce_chunk(ecc_curve_t curve, int log2_n, int log2_chunk) {
  if (!valid_curve(curve))
    return fail(ECC_EINVAL, "ecc_msm_set_reduce_chunk: unknown curve %d", (int)curve);
  if (log2_n < 0 || log2_n > 40 || log2_chunk < 0 || log2_chunk > kMsmReduceLogMax)
    return fail(ECC_EINVAL, "ecc_msm_set_reduce_chunk: need 0 <= log2_n <= 40 and 0 <= log2_chunk <= %d",
                kMsmReduceLogMax);
  msm_set_reduce_log(curve, log2_n, log2_chunk);
  return ok();
}

int ecc_set_gas_cluster(int ctas) {
  if (ctas != 1 && ctas != 2) return fail(ECC_EINVAL, "ecc_set_gas_cluster: ctas must be 1 or 2");
  set_gas_cluster(ctas);
  return ok();
}

int ecc_set_phase_timing(int on) {
  set_phase_timing(on != 0);
  return ok();
}

int ecc_msm_phase_times(float* ms_out, int max_phases) {
  if (!ms_out || max_phases < 1) return fail(ECC_EINVAL, "ecc_msm_phase_times: bad argument");
  float ms[kMsmPhases];
  if (!phase_times(ms))
    return fail(ECC_EINVAL, "ecc_msm_phase_times: no complete timed MSM call on this thread");
  const int k = max_phases < kMsmPhases ? max_phases : kMsmPhases;
  for (int i = 0; i < k; ++i) ms_out[i] = ms[i];
  return k;
}

int ecc_bench_imad(size_t threads, int iters, uint32_t* sink, void* stream) {
  if (threads == 0 || iters < 0 || !sink) return fail(ECC_EINVAL, "ecc_bench_imad: bad argument");
  cudaError_t e = launch_bench_imad(threads, iters, sink, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "ecc_bench_imad");
  return ok();
}

int ecc_bench_modmul(ecc_curve_t curve, int reduction, size_t threads, int iters, uint32_t* sink,
                     void* stream) {
  if (!valid_curve(curve)) return fail(ECC_EINVAL, "ecc_bench_modmul: unknown curve");
  if (threads == 0 || iters < 0 || !sink || reduction < 0 || reduction > 1)
    return fail(ECC_EINVAL, "ecc_bench_modmul: bad argument");
  if (reduction == 1 && curve != ECC_P256 && curve != ECC_SECP256K1)
    return fail(ECC_EUNSUPPORTED, "ecc_bench_modmul: the special-form reduction is offered for the "
                "P-256 and secp256k1 primes");
  cudaError_t e = launch_bench_modmul(curve, reduction, threads, iters, sink,
                                      static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "ecc_bench_modmul");
  return ok();
}

int ecc_fp_inv_batch_noalloc(ecc_curve_t curve, int field, size_t n, const uint32_t* a,
                             uint32_t* out, void* stream) {
  const char* name = "ecc_fp_inv_batch_noalloc";
  if (!valid_curve(curve)) return fail(ECC_EINVAL, "%s: unknown curve %d", name, (int)curve);
  if (field != 0 && field != 1) return fail(ECC_EINVAL, "%s: field must be 0 or 1", name);
  if (n == 0) return ok();
  if (n > kNoAllocMaxElems)
    return fail(ECC_EINVAL, "%s: n = %zu exceeds the fixed scratch capacity of %zu elements", name, n,
                kNoAllocMaxElems);
  if (!a || !out) return fail(ECC_EINVAL, "%s: NULL pointer", name);
  if (!aligned4(a) || !aligned4(out)) return fail(ECC_EINVAL, "%s: pointers must be 4-byte aligned", name);
  if (host_memory(a) || host_memory(out))
    return fail(ECC_EINVAL, "%s: a and out must be device memory (staging host buffers would allocate)",
                name);
  cudaError_t e = launch_fe_inv_batch_noalloc(curve, field, n, a, out, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, name);
  return ok();
}

int ecc_bench_inv(ecc_curve_t curve, int method, size_t threads, int iters, uint32_t* sink,
                  void* stream) {
  if (!valid_curve(curve)) return fail(ECC_EINVAL, "ecc_bench_inv: unknown curve");
  if (method < 0 || method > 3 || threads == 0 || iters < 0 || !sink)
    return fail(ECC_EINVAL, "ecc_bench_inv: bad argument");
  cudaError_t e = launch_bench_inv(curve, method, threads, iters, sink, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "ecc_bench_inv");
  return ok();
}

}  // extern "C"
