/*
 * gecc.h -- C ABI of the GB300 batched elliptic-curve library.
 *
 * The library implements the data-parallel hot path of gECC (arXiv 2501.03245):
 * Montgomery multiplication on 32-bit limbs (Section 4.1, Algorithm 2), batch
 * inversion by Montgomery's trick with per-CTA gather-apply-scatter (Sections
 * 2.2.1 and 3.2), batched affine point addition / doubling (Section 3.3,
 * Eqn 2-3), and on top of them ECDSA verification (Section 5.2: one fixed-point
 * plus one unknown-point multiplication) and Pippenger multi-scalar
 * multiplication.
 *
 * Conventions shared by every entry point
 *   - Return value: ECC_OK (0) or a negative ECC_E* code; the matching message
 *     is available from ecc_last_error() (thread-local, valid until the next
 *     call on the same thread).  Argument errors are reported synchronously;
 *     CUDA launch errors too.  Kernels run asynchronously on `stream` (a
 *     cudaStream_t; NULL = the legacy default stream).
 *   - n = 0 returns ECC_OK and does no work.
 *   - Memory: unless an entry point says otherwise, every array is caller-owned
 *     and may be device memory (results are ready when `stream` reaches the
 *     end of the call) or host memory (pageable or pinned; the call then
 *     stages through device memory and returns after the results are written
 *     back, i.e. it is synchronous).  The library owns only its internal
 *     workspace (stream-ordered allocations released at the end of each call)
 *     and the per-device fixed-base tables (built on first use of a curve and
 *     kept until process exit).  The first call that needs a curve's table
 *     builds it synchronously; do that call before any stream capture.
 *   - Field elements: little-endian 32-bit limbs, canonical (< modulus).  A
 *     base-field element of BN254 / secp256k1 / P-256 has 8 limbs, of
 *     BLS12-381 12 limbs (ecc_limbs()).  Scalars are always 8 limbs.
 *   - Affine points: x limbs then y limbs (2 * ecc_limbs() words per point);
 *     the point at infinity O is written (0, 0), which is on none of the
 *     supported curves (b != 0).
 *   - Pointers must be 4-byte aligned.
 */
#ifndef GECC_H
#define GECC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  ECC_SECP256K1 = 0,    /* SEC 2 secp256k1: a = 0, b = 7 */
  ECC_P256 = 1,         /* NIST P-256 (secp256r1): a = -3 */
  ECC_BN254 = 2,        /* BN254 G1: a = 0, b = 3 */
  ECC_BLS12_381 = 3,    /* BLS12-381 G1: a = 0, b = 4, 381-bit base field */
  ECC_SM2 = 4           /* SM2 recommended curve (GB/T 32918.5, the paper's curve): a = -3 */
} ecc_curve_t;

enum {
  ECC_OK = 0,
  ECC_EINVAL = -1,       /* bad argument (curve, NULL pointer, alignment, size) */
  ECC_EUNSUPPORTED = -2, /* operation not offered for this curve */
  ECC_ENOMEM = -3,       /* device workspace allocation failed */
  ECC_ECUDA = -4,        /* CUDA runtime error (message has the CUDA string) */
  ECC_ETIMEOUT = -5      /* a bounded device wait gave up */
};

/* Which field an ecc_fp_* call works in. */
enum { ECC_FIELD_BASE = 0, ECC_FIELD_SCALAR = 1 };

/* Thread-local message for the last non-OK return ("" if none). */
const char* ecc_last_error(void);

/* Library version string. */
const char* ecc_version(void);

/* Limbs of a base-field element (8 or 12), or ECC_EINVAL. */
int ecc_limbs(ecc_curve_t curve);

/* ---------------------------------------------------------------- field layer
 * out[i] = a[i] * b[i] mod q (Algorithm 2, Section 2.2: Montgomery
 * multiplication; inputs are converted into Montgomery form and back).
 * field: ECC_FIELD_BASE (q = p) or ECC_FIELD_SCALAR (q = group order n).
 * a, b, out: n rows of L limbs (L = ecc_limbs() for the base field, 8 for the
 * scalar field); inputs must be canonical.  On the P-256 and secp256k1 base
 * fields these unit operations reduce with the special form of the prime
 * (Section 4.2); the results are the same integers. */
int ecc_fp_mul(ecc_curve_t curve, int field, size_t n, const uint32_t* a, const uint32_t* b,
               uint32_t* out, void* stream);

/* out[i] = a[i] + b[i] mod q, and a[i] - b[i] mod q (Section 2.2 modadd). */
int ecc_fp_add(ecc_curve_t curve, int field, size_t n, const uint32_t* a, const uint32_t* b,
               uint32_t* out, void* stream);
int ecc_fp_sub(ecc_curve_t curve, int field, size_t n, const uint32_t* a, const uint32_t* b,
               uint32_t* out, void* stream);

/* out[i] = a[i]^-1 mod q, one Fermat inversion a^(q-2) per element
 * (Section 2.2 modinv); a[i] = 0 gives 0. */
int ecc_fp_inv(ecc_curve_t curve, int field, size_t n, const uint32_t* a, uint32_t* out,
               void* stream);

/* out[i] = a[i]^-1 mod q for the whole array by Montgomery's trick
 * (Section 2.2.1) with the gather-apply-scatter workflow of Section 3.2: one
 * modular inversion per CTA.  Zero elements give 0 and do not disturb the
 * others. */
int ecc_fp_inv_batch(ecc_curve_t curve, int field, size_t n, const uint32_t* a, uint32_t* out,
                     void* stream);

/* Allocation-free variant of ecc_fp_inv_batch (this entry point has no
 * counterpart in the paper).  It is for callers that may not allocate device
 * memory during a call: a service that fixes its memory budget at start-up and
 * forbids later allocation, a latency-critical loop that cannot afford the
 * device-wide synchronisation cudaMalloc implies, or a host library without an
 * allocator of its own.  It calls no cudaMalloc, cudaFree or allocating library
 * routine: its scratch is a fixed device array inside the library, sized for
 * n <= 65536 elements of any field (9 MiB, held by every GPU that loads the
 * library until the process exits); larger n returns ECC_EINVAL.
 *   - a, out: DEVICE memory only (host buffers would need a staging
 *     allocation: ECC_EINVAL); same layout and results as ecc_fp_inv_batch.
 *   - The first call on a device looks up the scratch array's device address
 *     (cudaGetSymbolAddress) with that device current; make that first call
 *     before any stream capture.
 *   - All calls share the one scratch array: calls that overlap on the GPU
 *     (different streams, or several host threads) race and corrupt each
 *     other's results; serialise them, e.g. on one stream.  No part of the
 *     scratch needs clearing between calls: every word is written before it is
 *     read. */
int ecc_fp_inv_batch_noalloc(ecc_curve_t curve, int field, size_t n, const uint32_t* a,
                             uint32_t* out, void* stream);

/* ---------------------------------------------------------------- EC operators
 * out[i] = p[i] + q[i] (batched affine PADD, Section 3.3, Eqn 2-3; PDBL when
 * p[i] = q[i]; O and p[i] = -q[i] follow the group law).  Points must be on the
 * curve (not checked). */
int ecc_point_add_batch(ecc_curve_t curve, size_t n, const uint32_t* p, const uint32_t* q,
                        uint32_t* out, void* stream);

/* out[i] = 2 p[i] (batched affine PDBL, Section 2.1.1). */
int ecc_point_dbl_batch(ecc_curve_t curve, size_t n, const uint32_t* p, uint32_t* out,
                        void* stream);

/* Batched affine PADD / PDBL (Section 3.3, Eqn 2-3) on a curve given at run
 * time: y^2 = x^3 + a x + b over F_p, for an odd prime 5 <= p < 2^256 (the
 * library's own curves have their constants compiled in; this entry point
 * serves any other curve, tiny test curves included).
 * prime, a: 8 little-endian limbs each, HOST memory, a < prime.  Primality of
 * the prime is the caller's promise (not checked; a composite modulus gives
 * meaningless results, but no fault).  b enters no formula, but must be nonzero
 * mod p so that (0, 0), the encoding of O, is not a point of the curve.
 * p, q, out: n points of 16 limbs (x then y, 8 canonical limbs each).
 * dbl = 0: out[i] = p[i] + q[i]; dbl != 0: out[i] = 2 p[i] (q unused, may be
 * NULL).  Points must be on the curve (not checked).  Errors: ECC_EINVAL for an
 * even prime, a prime below 5, a >= prime, NULL or misaligned pointers,
 * n > 2^30. */
int ecc_point_op_custom(const uint32_t* prime, const uint32_t* a, size_t n, const uint32_t* p,
                        const uint32_t* q, uint32_t* out, int dbl, void* stream);

/* ---------------------------------------------------------------- ECDSA
 * Batched ECDSA verification (Section 5.2; SEC 1 section 4.1.4).
 * curve: ECC_SECP256K1, ECC_P256 or ECC_SM2 (others: ECC_EUNSUPPORTED).
 * hash, r, s: n x 32 bytes, big-endian integers (the hash is used as e without
 * truncation: both group orders are 256-bit).
 * pubkey: n x 64 bytes, x || y big-endian, uncompressed, no 0x04 prefix.
 * ok_out: n bytes, 1 = valid signature, 0 = invalid.  Malformed input
 * (r or s outside [1, n-1], Q off the curve or not canonical, Q = (0, 0)) gives
 * 0, not an error. */
int ecc_verify_batch(ecc_curve_t curve, size_t n, const uint8_t* hash, const uint8_t* r,
                     const uint8_t* s, const uint8_t* pubkey, uint8_t* ok_out, void* stream);

/* ---------------------------------------------------------------- FPMUL
 * out[i] = k[i] * G (fixed-point multiplication, Section 2.1.1 and Table 5:
 * the generator's table v 2^(8j) G removes every PDBL; 32 batched affine
 * additions per scalar).  k: n x 8 limbs (any 256-bit integer); out: n affine
 * points ((0, 0) when k[i] * G = O). */
int ecc_fixed_base_mul(ecc_curve_t curve, size_t n, const uint32_t* k, uint32_t* out,
                       void* stream);

/* Batched ECDSA signing (Section 5.2: one modinv plus one FPMUL; SEC 1 section
 * 4.1.3 with the nonce supplied by the caller): r = x(k G) mod n,
 * s = k^-1 (e + r d) mod n, and the public key d G.
 * curve: ECC_SECP256K1, ECC_P256 or ECC_SM2.  d, e, k: n x 32 bytes big-endian;
 * r_out, s_out: n x 32 bytes; pub_out: n x 64 bytes (x || y).  An item with d
 * or k outside [1, n-1], or whose nonce gives r = 0 or s = 0, gets r = s = 0. */
int ecc_sign_batch(ecc_curve_t curve, size_t n, const uint8_t* d, const uint8_t* e,
                   const uint8_t* k, uint8_t* r_out, uint8_t* s_out, uint8_t* pub_out,
                   void* stream);

/* ---------------------------------------------------------------- MSM
 * Multi-scalar multiplication out = sum_i k_i P_i (Pippenger's bucket method
 * with batched affine bucket accumulation; the paper's batch inversion and
 * PADD, Sections 3.2-3.3).  Curves: ECC_BN254 and ECC_BLS12_381 (others give
 * ECC_EUNSUPPORTED).  Points: n affine points (canonical, (0, 0) = O,
 * assumed in the prime-order subgroup); scalars: n x 8 limbs, any 256-bit value
 * (reduced mod the group order r).  out: one affine point (2 * ecc_limbs()
 * limbs), (0, 0) when the sum is O.  The window width follows the size class
 * (ecc_msm_window).  Sizes: at most 2^28 points per call, and fewer than 2^31
 * (point, window) digits and 2^31 buckets over all instances of one call (the
 * sort and the reduction index with 32-bit words), else ECC_EINVAL. */
int ecc_msm(ecc_curve_t curve, size_t n, const uint32_t* points, const uint32_t* scalars,
            uint32_t* out, void* stream);

/* `num` independent MSMs in one launch sequence (one digit / sort /
 * accumulation pass over all of them, per-instance window widths).
 * offsets: HOST array of num + 1 row indices; instance i uses rows
 * [offsets[i], offsets[i+1]) of points and scalars; empty instances give O.
 * out: num points.  No host synchronisation inside: with device buffers the
 * call can be captured in a CUDA graph and replayed. */
int ecc_msm_ragged(ecc_curve_t curve, size_t num, const uint64_t* offsets, const uint32_t* points,
                   const uint32_t* scalars, uint32_t* out, void* stream);

/* Ragged MSMs whose instance boundaries live in DEVICE memory, so that one
 * captured CUDA graph can serve a new mix of sizes on every replay (the sizes
 * are read on the device; nothing about the launch sequence depends on them).
 * offsets: DEVICE array of num + 1 row indices with offsets[0] = 0; instance i
 * uses rows [offsets[i], offsets[i+1]) of points and scalars (DEVICE arrays of
 * at least max_points rows); out: num points (DEVICE).  max_points is the
 * capacity fixed when the call is made or recorded: every workspace is sized
 * for max_points rows in num instances.  Every instance uses one window width
 * c (2..20; 0 picks the library's width for max_points / num points), so the
 * bucket layout needs no sizes.  Offsets that decrease, do not start at 0 or
 * end above max_points are refused on the device: every output is then O and
 * the status word holds ECC_EINVAL (see ecc_sync_status).  The call is
 * asynchronous; it allocates stream-ordered workspace like ecc_msm_ragged. */
int ecc_msm_ragged_dev(ecc_curve_t curve, size_t num, size_t max_points, const uint64_t* offsets,
                       const uint32_t* points, const uint32_t* scalars, uint32_t* out, int c,
                       void* stream);

/* Resident bases: convert n points once into the library's device layout
 * (owned by the handle until ecc_bases_destroy), then run MSMs of many scalar
 * vectors against them.  ecc_msm_bases: scalars = num_vectors x n x 8 limbs,
 * out = num_vectors points; all vectors run through the same launches. */
int ecc_bases_create(ecc_curve_t curve, size_t n, const uint32_t* points, void** handle,
                     void* stream);
int ecc_msm_bases(void* handle, size_t num_vectors, const uint32_t* scalars, uint32_t* out,
                  void* stream);
int ecc_bases_destroy(void* handle);

/* Window multiples for reused bases (the paper's memory-for-time trade for
 * reused bases): stores 2^(c w) P_i for every window w of width c (W =
 * ceil((bits(r) + 1) / c) windows, W x n points, 64 or 96 bytes each, owned by
 * the handle and replacing an earlier table).  Afterwards every ecc_msm_bases /
 * ecc_msm_bases_ragged call on the handle uses window width c and one shared set
 * of 2^(c-1) buckets for all windows: no per-window reduction, no window
 * combination.  c in 2..24, W x n < 2^31, else ECC_EINVAL; ECC_ENOMEM when the
 * table does not fit.  Synchronous (returns after the table is built on
 * `stream`); no call on the handle may be in flight on another stream.
 * ecc_bases_window returns the handle's c, 0 when it has no table. */
int ecc_bases_precompute(void* handle, int c, void* stream);
int ecc_bases_window(void* handle);

/* Ragged MSMs over resident bases (the serving form): instance i is
 * sum_j k_ij P_j over the first sizes[i] resident bases; its sizes[i] scalar
 * rows follow those of instance i - 1 in `scalars`.  sizes: HOST array of num
 * counts, each <= the handle's base count.  out: num points.  No host
 * synchronisation inside (graph-capturable with device buffers). */
int ecc_msm_bases_ragged(void* handle, size_t num, const uint64_t* sizes, const uint32_t* scalars,
                         uint32_t* out, void* stream);

/* The serving form of ecc_msm_ragged_dev: instance i is sum_j k_ij P_j over
 * the first sizes[i] resident bases, its sizes[i] scalar rows following those
 * of instance i - 1.  sizes: DEVICE array of num counts, each at most the
 * handle's base count, at most max_points in all; scalars, out: DEVICE.  One
 * window width for every instance: the handle's window-multiple width, or the
 * library's width for max_points / num points.  Refused sizes give O outputs
 * and ECC_EINVAL in the status word. */
int ecc_msm_bases_ragged_dev(void* handle, size_t num, size_t max_points, const uint64_t* sizes,
                             const uint32_t* scalars, uint32_t* out, void* stream);

/* Device-side errors.  Kernels that find an error they can only see on the
 * device (device-resident sizes out of range; a bounded wait that gave up)
 * record its ECC_E* code in a status word of the current device (the first
 * error wins).  ecc_sync_status synchronises `stream`, returns the recorded
 * code (ECC_OK if none) with a message in ecc_last_error(), and clears it.
 * The word is per device, not per stream or per call: it reports errors of
 * any work on the device since the last ecc_sync_status. */
int ecc_sync_status(void* stream);

/* Caller-provided workspace allocator.  Every internal workspace of the
 * library (the per-call scratch of every entry point) is then taken from
 * alloc(bytes, stream, ctx) and returned with release(ptr, stream, ctx), both
 * called on the calling host thread with the call's stream; the memory must be
 * usable by work on that stream until release (stream-ordered semantics, e.g.
 * a framework's caching allocator).  alloc returning NULL makes the call fail
 * with ECC_ENOMEM.  Both NULL restores the default (cudaMallocAsync /
 * cudaFreeAsync).  Not used by ecc_fp_inv_batch_noalloc, nor for the
 * library-lifetime tables (fixed-base tables, resident bases). */
typedef void* (*ecc_alloc_fn)(size_t bytes, void* stream, void* ctx);
typedef void (*ecc_free_fn)(void* ptr, void* stream, void* ctx);
int ecc_set_allocator(ecc_alloc_fn alloc, ecc_free_fn release, void* ctx);

/* ok_out[i] = 1 when point i is O (written (0, 0)) or has canonical
 * coordinates that satisfy y^2 = x^3 + a x + b (Eqn 1), else 0.  Membership
 * of the prime-order subgroup is not checked (BN254 G1 has cofactor 1;
 * BLS12-381 G1 does not).  points as for ecc_msm; ok_out: n bytes. */
int ecc_validate_points(ecc_curve_t curve, size_t n, const uint32_t* points, uint8_t* ok_out,
                        void* stream);

/* Window width used for an n-point MSM, and the autotuner's override for the
 * size class floor(log2 n) (c = 0 restores the cost-model default). */
int ecc_msm_window(ecc_curve_t curve, size_t n);
int ecc_msm_set_window(ecc_curve_t curve, int log2_n, int c);

/* Bucket layout of the reduction (the autotuner's second knob): the bucket rows
 * of an n-point MSM are cut into first-level chunks of 2^k consecutive buckets,
 * each walked by running sums in k-dependent batched affine rounds (2^k + 1
 * addition rounds and k doubling rounds, one CTA-wide inversion each) before
 * the short Jacobian levels combine the chunks.  Smaller chunks mean fewer
 * rounds and more chunks.  ecc_msm_reduce_chunk returns k for an n-point MSM
 * (default 5, capped at c - 1); ecc_msm_set_reduce_chunk overrides it for the
 * size class floor(log2 n) (log2_chunk 1..10; 0 restores the default).  Results
 * do not depend on k. */
int ecc_msm_reduce_chunk(ecc_curve_t curve, size_t n);
int ecc_msm_set_reduce_chunk(ecc_curve_t curve, int log2_n, int log2_chunk);

/* Gather-apply-scatter across a thread-block cluster for ECDSA verification
 * (the memory-management idea of Section 3.3 taken to a cluster): with ctas =
 * 2 (the default), ecc_verify_batch runs in clusters of two CTAs that share
 * each round's single inversion through distributed shared memory (the second
 * CTA's product goes to the first, which inverts both products by Montgomery's
 * trick and sends the second its inverse back); ctas = 1 gives every CTA its
 * own inversion.  Process-wide setting; results are identical either way;
 * other values give ECC_EINVAL. */
int ecc_set_gas_cluster(int ctas);

/* MSM phase timers (diagnostics).  With timing on, every MSM entry point
 * records CUDA events on its stream at the boundaries of its five phases:
 * 0 counting sort by bucket id (histogram, scans, scatter), 1 batched affine
 * bucket accumulation, 2 fold of each bucket's partial sums, 3 bucket
 * reduction (the affine first level and the Jacobian upper levels), 4 window
 * combination.  Nothing is recorded while the stream is being captured.
 * ecc_msm_phase_times waits for the calling thread's last timed MSM call and
 * writes the device milliseconds of up to max_phases phases to ms_out (host);
 * returns the number written, or ECC_EINVAL if this thread has no complete
 * timed call.  Timing costs a few event records per call; off by default. */
int ecc_set_phase_timing(int on);
int ecc_msm_phase_times(float* ms_out, int max_phases);

/* ---------------------------------------------------------------- benchmarks
 * Integer multiply-add issue-rate probe (the microbenchmark method of
 * Section 4.1, Table 2): each of `threads` threads runs `iters` iterations of
 * `chains` independent mad.lo/madc.hi (IMAD.WIDE-class) carry chains.  Writes a
 * data-dependent checksum per thread to sink (device, threads words) so the
 * work cannot be elided.  Time it with CUDA events around the call. */
int ecc_bench_imad(size_t threads, int iters, uint32_t* sink, void* stream);

/* Montgomery multiplications in registers: each thread runs `iters` rounds of
 * 4 independent mont_mul chains of the curve's base field.  reduction 0 = the
 * generic Montgomery reduction (Algorithm 2, as in every fused kernel);
 * 1 = the special-form reduction of Section 4.2 (P-256: u = T_0 and u q by
 * additions; secp256k1: u q = u 2^256 - u (2^32 + 977), one product per row;
 * ECC_EUNSUPPORTED on the other curves; the ecc_fp_* unit operations on these
 * two base fields use it).
 * sink as above. */
int ecc_bench_modmul(ecc_curve_t curve, int reduction, size_t threads, int iters, uint32_t* sink,
                     void* stream);

/* Inversion latency probe: each thread runs a chain of `iters` dependent
 * inversions in the curve's base field, method 0 = Fermat (Section 2.2),
 * 1 = the GAS apply step's (branch-free single divsteps on 30-bit limbs),
 * 2 = batched variable-time divsteps on 62-bit limbs, 3 = the same on 30-bit
 * limbs.  With threads = 1 the kernel time / iters is the latency of one
 * inversion on one thread. */
int ecc_bench_inv(ecc_curve_t curve, int method, size_t threads, int iters, uint32_t* sink,
                  void* stream);

#ifdef __cplusplus
}
#endif
#endif /* GECC_H */
