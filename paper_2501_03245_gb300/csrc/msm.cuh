// Pippenger multi-scalar multiplication on top of the batched affine PADD.
//
// The paper's text has no MSM section; the method is the standard bucket
// method built from the paper's primitives:
//   1. digits: scalar k_i (reduced mod r) in signed c-bit windows
//      d_w in [-2^(c-1) + 1, 2^(c-1)], W = ceil((bits(r) + 1) / c) windows;
//   2. counting (one-digit radix) sort of the (bucket id, point) pairs by bucket
//      id: histogram with atomics, exclusive scan, scatter with atomic cursors;
//   3. bucket accumulation with batched affine additions (Section 3.3): the
//      sorted array is cut into chunks of CH consecutive entries and each chunk
//      keeps one running sum; round j adds entry j of every chunk to its running
//      sum, all chunks of a CTA sharing one inversion per round (Montgomery's
//      trick with GAS, Section 3.2).  A chunk entry that starts a new bucket
//      flushes the running sum as a partial bucket sum and restarts it (a copy,
//      no inversion needed).  CH rounds finish the whole array in one launch;
//   4. bucket reduction sum_k k B_k per window by chunked running sums and
//   5. window combination sum_w 2^(c w) S_w, both in Jacobian coordinates
//      (long dependent chains with little parallelism, where a batch inversion
//      per step would be pure latency).
// Several independent MSM instances (different sizes, windows and bases) run
// through the same launches: every instance owns a disjoint range of bucket ids.
#pragma once
#include "jac.cuh"

namespace ecc {

constexpr int kAccChunk = 32;       // entries per running-sum chunk (rounds of step 3)
constexpr uint32_t kNoKey = 0xffffffffu;

struct MsmInst {
  uint32_t n;            // points of the instance
  uint32_t c;            // window bits
  uint32_t W;            // windows
  uint32_t bucket_base;  // first global bucket id
  uint64_t point_off;    // first point in the global bases array
  uint64_t scalar_off;   // first scalar in the global scalar array
};

// ------------------------------------------------------------------ digits

// k mod r for a 256-bit k (at most a few subtractions: r > 2^253)
template <class C>
ECC_DEV void scalar_mod_r(uint32_t* k) {
  uint32_t rr[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) rr[q] = C::n(q);
  for (int it = 0; it < 8; ++it) {
    uint32_t t[8];
    t[0] = ptx::sub_cc(k[0], rr[0]);
#pragma unroll
    for (int q = 1; q < 8; ++q) t[q] = ptx::subc_cc(k[q], rr[q]);
    const uint32_t borrow = ptx::subc(0, 0);
    if (borrow) break;
#pragma unroll
    for (int q = 0; q < 8; ++q) k[q] = t[q];
  }
}

// bits [pos, pos + c) of k (c <= 24)
ECC_DEV uint32_t scalar_bits(const uint32_t* k, int pos, int c) {
  const int w = pos >> 5, s = pos & 31;
  if (w >= 8) return 0;
  uint64_t v = k[w];
  if (w + 1 < 8) v |= (uint64_t)k[w + 1] << 32;
  return (uint32_t)(v >> s) & ((1u << c) - 1u);
}

// Calls fn(w, d) for every window with signed digit d != 0.
template <class Fn>
ECC_DEV void for_each_digit(const uint32_t* k, int c, int W, Fn fn) {
  uint32_t carry = 0;
  const uint32_t half = 1u << (c - 1);
  for (int w = 0; w < W; ++w) {
    uint32_t v = scalar_bits(k, w * c, c) + carry;
    int d;
    if (v > half) {
      d = (int)v - (int)(1u << c);
      carry = 1;
    } else {
      d = (int)v;
      carry = 0;
    }
    if (d != 0) fn(w, d);
  }
}

ECC_DEV int find_inst(const MsmInst* inst, int num, uint64_t g) {
  int lo = 0, hi = num - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (inst[mid].scalar_off <= g) lo = mid; else hi = mid - 1;
  }
  return lo;
}

template <class C>
__global__ void k_msm_count(const MsmInst* inst, int num, const uint32_t* __restrict__ scalars,
                            uint64_t total, uint32_t* __restrict__ count) {
  const uint64_t g = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (g >= total) return;
  const MsmInst in = inst[find_inst(inst, num, g)];
  uint32_t k[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) k[q] = scalars[8 * g + q];
  scalar_mod_r<C>(k);
  const uint32_t half = 1u << (in.c - 1);
  for_each_digit(k, in.c, in.W, [&](int w, int d) {
    const uint32_t b = in.bucket_base + w * half + (uint32_t)(d < 0 ? -d : d) - 1;
    atomicAdd(count + b, 1u);
  });
}

// Entries are written chunk-transposed: entry p goes to [p % CH][p / CH].
template <class C>
__global__ void k_msm_scatter(const MsmInst* inst, int num, const uint32_t* __restrict__ scalars,
                              uint64_t total, uint32_t* __restrict__ cursor, uint32_t* __restrict__ keys,
                              uint32_t* __restrict__ vals, uint64_t n_chunks) {
  const uint64_t g = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (g >= total) return;
  const MsmInst in = inst[find_inst(inst, num, g)];
  uint32_t k[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) k[q] = scalars[8 * g + q];
  scalar_mod_r<C>(k);
  const uint32_t half = 1u << (in.c - 1);
  const uint32_t pidx = (uint32_t)(in.point_off + (g - in.scalar_off));
  for_each_digit(k, in.c, in.W, [&](int w, int d) {
    const uint32_t b = in.bucket_base + w * half + (uint32_t)(d < 0 ? -d : d) - 1;
    const uint32_t p = atomicAdd(cursor + b, 1u);
    const uint64_t slot = (uint64_t)(p % kAccChunk) * n_chunks + p / kAccChunk;
    keys[slot] = b;
    vals[slot] = pidx | (d < 0 ? 0x80000000u : 0u);
  });
}

// Partial-sum slots per bucket: one per chunk the bucket's entries touch.
static __global__ void k_msm_npart(const uint32_t* __restrict__ off, uint32_t n_buckets,
                            uint32_t* __restrict__ npart) {
  const uint32_t b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= n_buckets) return;
  const uint32_t lo = off[b], hi = off[b + 1];
  npart[b] = hi > lo ? (hi - 1) / kAccChunk - lo / kAccChunk + 1 : 0;
}

// ------------------------------------------------------------------ accumulation

template <class C>
struct AccArgs {
  using F = typename C::Fp;
  const uint32_t* keys;   // [CH][n_chunks]
  const uint32_t* vals;
  const uint32_t* off;    // bucket offsets (exclusive scan), off[n_buckets] = entries
  const uint32_t* poff;   // partial-slot offsets per bucket
  uint32_t n_buckets;
  uint64_t n_chunks;
  const uint32_t* bases;  // AoS Montgomery affine points, 2N words each
  PtSoA<F> S;             // running sum per chunk
  PtSoA<F> partial;       // partial bucket sums
  SoA<F> M;
  uint64_t per_cta;
};

template <class C>
ECC_DEV void load_base(const AccArgs<C>& a, uint32_t v, uint32_t* x, uint32_t* y) {
  using F = typename C::Fp;
  constexpr int N = F::N;
  const uint4* p = reinterpret_cast<const uint4*>(a.bases + (uint64_t)(v & 0x7fffffffu) * 2 * N);
#pragma unroll
  for (int g = 0; g < N / 4; ++g) {
    const uint4 t = p[g];
    x[4 * g] = t.x; x[4 * g + 1] = t.y; x[4 * g + 2] = t.z; x[4 * g + 3] = t.w;
  }
#pragma unroll
  for (int g = 0; g < N / 4; ++g) {
    const uint4 t = p[N / 4 + g];
    y[4 * g] = t.x; y[4 * g + 1] = t.y; y[4 * g + 2] = t.z; y[4 * g + 3] = t.w;
  }
  if (v & 0x80000000u) fe_neg<F>(y, y);
}

template <class C>
ECC_DEV uint64_t partial_slot(const AccArgs<C>& a, uint32_t b, uint64_t chunk) {
  return a.poff[b] + (chunk - a.off[b] / kAccChunk);
}

template <class C>
struct AccRound {
  using F = typename C::Fp;
  static constexpr int N = F::N;
  static constexpr int OPS = 1;
  const AccArgs<C>* a;
  int j;
  uint32_t entries;
  int kind;
  bool start, live;
  ECC_DEV void classify(size_t c, uint32_t& key, uint32_t& val, uint32_t& prev) {
    const uint64_t p = (uint64_t)c * kAccChunk + j;
    live = p < entries;
    key = live ? a->keys[(uint64_t)j * a->n_chunks + c] : kNoKey;
    val = live ? a->vals[(uint64_t)j * a->n_chunks + c] : 0u;
    prev = (live && j > 0) ? a->keys[(uint64_t)(j - 1) * a->n_chunks + c] : kNoKey;
    start = live && (j == 0 || key != prev);
  }
  ECC_DEV void den_c(size_t c, int, uint32_t* d) {
    uint32_t key, val, prev;
    classify(c, key, val, prev);
    if (!live || start) {
      fe_set_one<F>(d);
      kind = ADD_RET_T;
      return;
    }
    uint32_t xs[N], ys[N], xp[N], yp[N];
    a->S.load(c, xs, ys);
    load_base<C>(*a, val, xp, yp);
    kind = add_den<C>(d, xs, ys, xp, yp);
  }
  ECC_DEV void den_d(size_t c, int k, uint32_t* d) { den_c(c, k, d); }
  ECC_DEV void finish(size_t c, const uint32_t (*inv)[N]) {
    if (!live) return;
    uint32_t key, val, prev;
    classify(c, key, val, prev);
    uint32_t xs[N], ys[N], xp[N], yp[N];
    load_base<C>(*a, val, xp, yp);
    if (start) {
      if (j > 0) {
        a->S.load(c, xs, ys);
        a->partial.store(partial_slot(*a, prev, c), xs, ys);
      }
      a->S.store(c, xp, yp);
    } else {
      a->S.load(c, xs, ys);
      add_finish<C>(xs, ys, kind, inv[0], xs, ys, xp, yp);
      a->S.store(c, xs, ys);
    }
  }
};

template <class C, int BLOCK>
__global__ void __launch_bounds__(BLOCK, kGasResidentThreads / BLOCK) k_msm_accumulate(AccArgs<C> a) {
  using F = typename C::Fp;
  constexpr int N = F::N;
  auto& sm = gas_smem<N, BLOCK>();
  const uint32_t entries = a.off[a.n_buckets];
  const uint64_t used = (entries + kAccChunk - 1) / kAccChunk;
  const uint64_t begin = blockIdx.x * a.per_cta;
  uint64_t end = begin + a.per_cta;
  if (end > used) end = used;
  if (end < begin) end = begin;
  for (int j = 0; j < kAccChunk; ++j) {
    AccRound<C> rd{&a, j, entries};
    batch_round<F, BLOCK>(rd, begin, end, a.M, sm);
  }
  // flush the last running sum of every chunk
  for (uint64_t c = begin + threadIdx.x; c < end; c += BLOCK) {
    const uint64_t last = c * kAccChunk + kAccChunk - 1 < entries ? c * kAccChunk + kAccChunk - 1
                                                                  : entries - 1;
    const int jl = (int)(last - c * kAccChunk);
    const uint32_t key = a.keys[(uint64_t)jl * a.n_chunks + c];
    uint32_t xs[N], ys[N];
    a.S.load(c, xs, ys);
    a.partial.store(partial_slot(a, key, c), xs, ys);
  }
}

// ------------------------------------------------------------------ reduction

// Weighted chunk sums.  Elements e = lo .. hi of one window carry (R_e, S_e)
// with R the plain sum and S the sum weighted from the element's own first
// bucket; span is the bucket count of one element.  The chunk returns
// R = sum R_e and S = sum S_e + span * sum_e (e - lo) R_e, so that the window
// sum is sum over chunks of S + (first bucket - 1) R.
template <class C>
struct ReduceArgs {
  using F = typename C::Fp;
  const MsmInst* inst;     // instances of this group (same c and W)
  const uint32_t* inst_ids;
  uint32_t n_inst;
  uint32_t W;
  uint32_t elems;          // elements per window at this level
  uint32_t chunk;          // elements per output chunk
  uint32_t log_span;       // span = 2^log_span buckets per element
  // level 1 reads buckets from the partial sums
  const uint32_t* poff;
  PtSoA<F> partial;
  // other levels read (R, S) pairs written by the previous level
  const Jac<F>* in_R;
  const Jac<F>* in_S;
  Jac<F>* out_R;
  Jac<F>* out_S;
};

template <class C>
ECC_DEV void bucket_sum(const ReduceArgs<C>& a, uint32_t b, Jac<typename C::Fp>& B) {
  using F = typename C::Fp;
  constexpr int N = F::N;
  jac_set_inf<C>(B);
  const uint32_t lo = a.poff[b], hi = a.poff[b + 1];
  for (uint32_t s = lo; s < hi; ++s) {
    uint32_t x[N], y[N];
    a.partial.load(s, x, y);
    jac_add_mixed<C>(B, B, x, y);
  }
}

template <class C>
__global__ void k_msm_reduce(ReduceArgs<C> a, int level1) {
  using F = typename C::Fp;
  const uint32_t chunks = (a.elems + a.chunk - 1) / a.chunk;
  const uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (t >= (uint64_t)a.n_inst * a.W * chunks) return;
  const uint32_t u = (uint32_t)(t % chunks);
  const uint32_t w = (uint32_t)((t / chunks) % a.W);
  const uint32_t ii = (uint32_t)(t / chunks / a.W);
  const MsmInst in = a.inst[a.inst_ids[ii]];
  const uint32_t lo = u * a.chunk;
  const uint32_t hi = lo + a.chunk < a.elems ? lo + a.chunk : a.elems;  // exclusive
  const uint64_t win = (uint64_t)ii * a.W + w;                           // window row
  Jac<F> Rr, U, Ssum, E;
  jac_set_inf<C>(Rr);
  jac_set_inf<C>(U);
  jac_set_inf<C>(Ssum);
  for (uint32_t e = hi; e-- > lo;) {
    Jac<F> Se;
    if (level1) {
      bucket_sum<C>(a, in.bucket_base + w * (1u << (in.c - 1)) + e, E);
      Se = E;
    } else {
      E = a.in_R[win * a.elems + e];
      Se = a.in_S[win * a.elems + e];
    }
    jac_add<C>(Ssum, Ssum, Se);
    if (e > lo) {
      jac_add<C>(Rr, Rr, E);
      jac_add<C>(U, U, Rr);
    } else {
      jac_add<C>(Rr, Rr, E);
    }
  }
  for (uint32_t s = 0; s < a.log_span; ++s) jac_dbl<C>(U, U);
  jac_add<C>(Ssum, Ssum, U);
  a.out_R[win * chunks + u] = Rr;
  a.out_S[win * chunks + u] = Ssum;
}

// result_i = sum_w 2^(c w) S_w (Horner), converted to canonical affine limbs.
template <class C>
__global__ void k_msm_combine(const MsmInst* inst, const uint32_t* inst_ids, uint32_t n_inst,
                              uint32_t W, const Jac<typename C::Fp>* S, uint32_t* out_all) {
  using F = typename C::Fp;
  constexpr int N = F::N;
  const uint32_t ii = blockIdx.x * blockDim.x + threadIdx.x;
  if (ii >= n_inst) return;
  const uint32_t id = inst_ids[ii];
  const uint32_t c = inst[id].c;
  Jac<F> acc = S[(uint64_t)ii * W + (W - 1)];
  for (int w = (int)W - 2; w >= 0; --w) {
    for (uint32_t s = 0; s < c; ++s) jac_dbl<C>(acc, acc);
    jac_add<C>(acc, acc, S[(uint64_t)ii * W + w]);
  }
  uint32_t x[N], y[N];
  jac_to_affine<C>(x, y, acc);
  from_mont<F>(x, x);
  from_mont<F>(y, y);
  uint32_t* o = out_all + (uint64_t)id * 2 * N;
#pragma unroll
  for (int q = 0; q < N; ++q) {
    o[q] = x[q];
    o[N + q] = y[q];
  }
}

// canonical AoS points -> Montgomery AoS points (gather layout of the bases)
template <class C>
__global__ void k_points_to_mont(const uint32_t* __restrict__ in, uint64_t n, uint32_t* __restrict__ out) {
  using F = typename C::Fp;
  constexpr int N = F::N;
  const uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint32_t x[N], y[N];
#pragma unroll
  for (int q = 0; q < N; ++q) {
    x[q] = in[2 * N * i + q];
    y[q] = in[2 * N * i + N + q];
  }
  to_mont<F>(x, x);
  to_mont<F>(y, y);
#pragma unroll
  for (int q = 0; q < N; ++q) {
    out[2 * N * i + q] = x[q];
    out[2 * N * i + N + q] = y[q];
  }
}

}  // namespace ecc
