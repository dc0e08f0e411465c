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
//   4. bucket reduction sum_k k B_k per window by chunked running sums: the
//      first level (many independent chunks) as batched affine additions, the
//      short upper levels in Jacobian coordinates;
//   5. window combination sum_w 2^(c w) S_w in Jacobian coordinates (one long
//      dependent chain per instance, where a batch inversion per step would be
//      pure latency).
// Several independent MSM instances (different sizes, windows and bases) run
// through the same launches: every instance owns a disjoint range of bucket ids.
#pragma once
#include "jac.cuh"

namespace ecc {

constexpr int kAccChunk = 32;       // entries per running-sum chunk (rounds of step 3)

struct MsmInst {
  uint32_t n;            // points of the instance
  uint32_t c;            // window bits
  uint32_t W;            // windows (digits per scalar)
  uint32_t bucket_base;  // first global bucket id
  uint64_t point_off;    // first point in the global bases array
  uint64_t scalar_off;   // first scalar in the global scalar array
  // Bases with precomputed window multiples: window w of point i is the point
  // 2^(c w) P_i at index w * pre_stride + i, all windows share one set of
  // buckets (Wr = 1) and need no combination.  pre_stride = 0: Wr = W rows of
  // buckets, one per window.
  uint64_t pre_stride;
  uint32_t Wr;           // bucket rows (windows reduced separately)
  uint32_t red_log;      // log2 of the buckets per first-level reduction chunk
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

// A ragged batch whose instance sizes live in device memory: the scalar rows
// of all instances (rows [0, total)) and whether the sizes were refused.
struct MsmDevHdr {
  uint64_t total;
  uint32_t failed;
  uint32_t pad;
};

// Rows of the batch: the host's count, or the device header's when present.
ECC_DEV uint64_t batch_rows(uint64_t host_total, const MsmDevHdr* hdr) {
  return hdr ? hdr->total : host_total;
}

// Instance table of a ragged batch whose sizes are in device memory.  Every
// instance has the window width, bucket rows and reduction chunk of `proto`, so
// instance i's buckets start at i Wr 2^(c-1) and nothing else about the launch
// sequence depends on the sizes.  rows: sizes[num] (resident bases, scalar rows
// back to back, each size at most n_bases) or offsets[num + 1] (offsets[0] = 0,
// point and scalar rows of instance i from offsets[i]).  Sizes that break these
// rules or a total above `cap` leave an empty batch (total 0, failed = 1: every
// output is O) and record ECC_EINVAL (-1) in the status word.  One CTA.
static __global__ void k_msm_inst_dev(const uint64_t* __restrict__ rows, uint32_t num, int sizes_mode,
                               uint64_t n_bases, uint64_t cap, MsmInst proto, MsmInst* __restrict__ inst,
                               MsmDevHdr* hdr, int* status) {
  __shared__ uint64_t warp_sum[32];
  __shared__ uint64_t carry;
  __shared__ int bad;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (threadIdx.x == 0) {
    carry = 0;
    bad = !sizes_mode && rows[0] != 0;
  }
  __syncthreads();
  const uint64_t per_bucket_row = (uint64_t)proto.Wr << (proto.c - 1);
  for (uint32_t base = 0; base < num; base += blockDim.x) {
    const uint32_t i = base + threadIdx.x;
    uint64_t n = 0, off = 0;
    if (i < num) {
      if (sizes_mode) {
        n = rows[i];
        if (n > n_bases) bad = 1;
      } else {
        off = rows[i];
        const uint64_t hi = rows[i + 1];
        if (hi < off) bad = 1;
        n = hi >= off ? hi - off : 0;
      }
    }
    // block-wide exclusive prefix of n (scalar rows before instance i)
    uint64_t x = n;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint64_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) warp_sum[warp] = x;
    __syncthreads();
    if (warp == 0) {
      uint64_t w = lane < nw ? warp_sum[lane] : 0;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint64_t y = __shfl_up_sync(0xffffffffu, w, o);
        if (lane >= o) w += y;
      }
      if (lane < nw) warp_sum[lane] = w;
    }
    __syncthreads();
    const uint64_t before = carry + (warp > 0 ? warp_sum[warp - 1] : 0) + x - n;
    if (i < num) {
      MsmInst m = proto;
      m.n = (uint32_t)n;
      m.bucket_base = (uint32_t)(i * per_bucket_row);
      m.scalar_off = sizes_mode ? before : off;
      m.point_off = sizes_mode ? 0 : off;
      inst[i] = m;
    }
    __syncthreads();
    if (threadIdx.x == 0) carry += warp_sum[nw - 1];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const uint64_t total = sizes_mode ? carry : rows[num];
    const bool fail = bad || total > cap;
    hdr->total = fail ? 0 : total;
    hdr->failed = fail ? 1u : 0u;
    if (fail) atomicCAS(status, 0, -1);
  }
}

// Histogram of the bucket ids (fire-and-forget atomic increments).
template <class C>
__global__ void k_msm_count(const MsmInst* inst, int num, const uint32_t* __restrict__ scalars,
                            uint64_t total, const MsmDevHdr* hdr, uint32_t* __restrict__ count) {
  const uint64_t g = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (g >= batch_rows(total, hdr)) return;
  const MsmInst in = inst[find_inst(inst, num, g)];
  uint32_t k[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) k[q] = scalars[8 * g + q];
  scalar_mod_r<C>(k);
  const uint32_t half = 1u << (in.c - 1);
  const uint32_t row = in.pre_stride ? 0u : half;
  for_each_digit(k, in.c, in.W, [&](int w, int d) {
    const uint32_t b = in.bucket_base + w * row + (uint32_t)(d < 0 ? -d : d) - 1;
    atomicAdd(count + b, 1u);
  });
}

// Entries are written chunk-transposed: entry p goes to [p % CH][p / CH].  Only
// the point index is stored; the bucket of position p follows from the offsets.
// The bucket of each chunk's first entry is recorded in cur (the accumulation's
// per-chunk bucket cursor starts there).
template <class C>
__global__ void k_msm_scatter(const MsmInst* inst, int num, const uint32_t* __restrict__ scalars,
                              uint64_t total, const MsmDevHdr* hdr, uint32_t* __restrict__ cursor,
                              uint32_t* __restrict__ vals, uint64_t n_chunks,
                              uint32_t* __restrict__ cur) {
  const uint64_t g = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (g >= batch_rows(total, hdr)) return;
  const MsmInst in = inst[find_inst(inst, num, g)];
  uint32_t k[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) k[q] = scalars[8 * g + q];
  scalar_mod_r<C>(k);
  const uint32_t half = 1u << (in.c - 1);
  const uint32_t row = in.pre_stride ? 0u : half;
  const uint64_t pidx = in.point_off + (g - in.scalar_off);
  for_each_digit(k, in.c, in.W, [&](int w, int d) {
    const uint32_t b = in.bucket_base + w * row + (uint32_t)(d < 0 ? -d : d) - 1;
    const uint32_t p = atomicAdd(cursor + b, 1u);
    const uint32_t idx = (uint32_t)(pidx + (uint64_t)w * in.pre_stride);  // < 2^31 (host check)
    vals[(uint64_t)(p % kAccChunk) * n_chunks + p / kAccChunk] = idx | (d < 0 ? 0x80000000u : 0u);
    if (p % kAccChunk == 0) cur[p / kAccChunk] = b;
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
  const uint32_t* vals;   // sorted (point index | sign bit), [CH][n_chunks]
  const uint32_t* off;    // bucket offsets (exclusive scan), off[n_buckets] = entries
  const uint32_t* poff;   // partial-slot offsets per bucket
  uint32_t n_buckets;
  uint64_t n_chunks;
  const uint32_t* bases;  // AoS Montgomery affine points, 2N words each
  uint32_t* cur;          // bucket of the chunk's current entry
  PtSoA<F> S;             // running sum per chunk
  PtSoA<F> partial;       // partial bucket sums
  SoA<F> M;               // GAS prefix products
};

template <class C>
ECC_DEV const uint4* base_ptr(const AccArgs<C>& a, uint32_t v) {
  return reinterpret_cast<const uint4*>(a.bases + (uint64_t)(v & 0x7fffffffu) * 2 * C::Fp::N);
}

// x of the base a digit names (the sign only touches y)
template <class C>
ECC_DEV void load_base_x(const AccArgs<C>& a, uint32_t v, uint32_t* x) {
  constexpr int N = C::Fp::N;
  const uint4* p = base_ptr(a, v);
#pragma unroll
  for (int g = 0; g < N / 4; ++g) {
    const uint4 t = p[g];
    x[4 * g] = t.x; x[4 * g + 1] = t.y; x[4 * g + 2] = t.z; x[4 * g + 3] = t.w;
  }
}

// y of the base a digit names, negated for a negative digit
template <class C>
ECC_DEV void load_base_y(const AccArgs<C>& a, uint32_t v, uint32_t* y) {
  using F = typename C::Fp;
  constexpr int N = F::N;
  const uint4* p = base_ptr(a, v);
#pragma unroll
  for (int g = 0; g < N / 4; ++g) {
    const uint4 t = p[N / 4 + g];
    y[4 * g] = t.x; y[4 * g + 1] = t.y; y[4 * g + 2] = t.z; y[4 * g + 3] = t.w;
  }
  if (v & 0x80000000u) fe_neg<F>(y, y);
}

template <class C>
ECC_DEV void load_base(const AccArgs<C>& a, uint32_t v, uint32_t* x, uint32_t* y) {
  load_base_x<C>(a, v, x);
  load_base_y<C>(a, v, y);
}

template <class C>
ECC_DEV uint64_t partial_slot(const AccArgs<C>& a, uint32_t b, uint64_t chunk) {
  return a.poff[b] + (chunk - a.off[b] / kAccChunk);
}

// The bucket holding sorted position p: the last b in [lo, n) with off[b] <= p
// (requires off[lo] <= p < off[n]).
ECC_DEV uint32_t bucket_of(const uint32_t* off, uint32_t lo, uint32_t n, uint32_t p) {
  uint32_t hi = n;
  while (hi - lo > 1) {
    const uint32_t mid = lo + ((hi - lo) >> 1);
    if (off[mid] <= p) lo = mid; else hi = mid;
  }
  return lo;
}

// Entry j of chunk c: whether it exists, its bucket, and whether it starts a
// new running sum.  pb = the chunk's bucket before this entry (for j = 0 the
// bucket of the entry itself, recorded by the scatter); off1 = off[pb + 1],
// the end of that bucket (unused for j = 0).
struct AccCls {
  bool live, start;
  uint32_t bucket, prev;
};

template <class C>
ECC_DEV AccCls acc_classify(const AccArgs<C>& a, uint64_t c, int j, uint32_t entries, uint32_t pb,
                            uint32_t off1) {
  AccCls k{false, false, pb, pb};
  const uint32_t p = (uint32_t)(c * kAccChunk + j);
  if (p >= entries) return k;
  k.live = true;
  if (j == 0 || p >= off1) k.start = true;
  if (j == 0 || p < off1) return k;
  k.bucket = pb + 1;  // usually the next bucket; skip empty ones otherwise
  if (a.off[k.bucket + 1] <= p) k.bucket = bucket_of(a.off, k.bucket + 1, a.n_buckets, p);
  return k;
}

// ---- One round with every operand staged in shared memory (cp.async).
// Entry j of every chunk is added to the chunk's running sum S (or starts a
// new one at a bucket boundary).  Each thread owns 5 G 16-byte vectors of
// shared memory (G = N / 4 vectors per field element; layout [vector][thread],
// so a warp's copies of one vector are 512 contiguous bytes).  They are the
// thread's own column of the GAS tree, which is dead outside cta_invert: the
// staging costs no shared memory of its own.  While a thread computes on its
// item k, the copies of item k+1's operands and the first-level loads of item
// k+2 (its sorted entry and its chunk's bucket cursor, into registers) are in
// flight, and so is item k+1's bucket end off[pb + 1], so the gathers behind
// the sorted entries do not stall the arithmetic.  Compress stages only x of S
// and of the base (the compress step of Section 3.3); y is read, directly, only
// when an operand may be O (x = 0) or the two x agree (doubling or P = -T),
// which random inputs almost never hit.  DCWPA stages S, the base and the prefix
// product.  With 8 limbs it holds all of them in registers from the top of the
// item, so the next item's copies start at once; with 12 limbs (no registers to
// spare) it computes the item's two DCWPA products from the staged values first,
// then loads the finish operands and only then starts the next item's copies.
// No denominator array exists for either width.
template <int N, int BLOCK>
struct Stage {
  static constexpr int G = N / 4;
  // vector bases: S.x, S.y, base.x, base.y, prefix product
  static constexpr int SX = 0, SY = G, BX = 2 * G, BY = 3 * G, PRE = 4 * G;
  uint4* v;  // [5 G][BLOCK]
  ECC_DEV uint4* at(int k) const { return v + k * BLOCK + threadIdx.x; }
  ECC_DEV void get(int k0, uint32_t* r) const {
#pragma unroll
    for (int g = 0; g < G; ++g) {
      const uint4 p = *at(k0 + g);
      r[4 * g] = p.x;
      r[4 * g + 1] = p.y;
      r[4 * g + 2] = p.z;
      r[4 * g + 3] = p.w;
    }
  }
};

// Issues the copies of chunk c's operands (entry v): x of S and of the base,
// and with `full` also y of both and the prefix product.  The base is touched
// only for an existing entry (v is meaningful only then).
template <class C, int BLOCK>
ECC_DEV void acc_stage(const Stage<C::Fp::N, BLOCK>& sg, const AccArgs<C>& a, uint64_t c, uint32_t v,
                       bool live, bool full) {
  using S = Stage<C::Fp::N, BLOCK>;
#pragma unroll
  for (int g = 0; g < S::G; ++g) ptx::cp_async16(sg.at(S::SX + g), a.S.x.vec + g * a.S.x.stride + c);
  if (full) {
#pragma unroll
    for (int g = 0; g < S::G; ++g) {
      ptx::cp_async16(sg.at(S::SY + g), a.S.y.vec + g * a.S.y.stride + c);
      ptx::cp_async16(sg.at(S::PRE + g), a.M.vec + g * a.M.stride + c);
    }
  }
  if (live) {
    const uint4* p = base_ptr(a, v);
#pragma unroll
    for (int g = 0; g < S::G; ++g) ptx::cp_async16(sg.at(S::BX + g), p + g);
    if (full) {
#pragma unroll
      for (int g = 0; g < S::G; ++g) ptx::cp_async16(sg.at(S::BY + g), p + S::G + g);
    }
  }
  ptx::cp_async_commit();
}

template <class C, int BLOCK>
__device__ void acc_round_staged(const AccArgs<C>& a, int j, uint32_t entries, uint64_t begin,
                                 uint64_t end, GasSmem<C::Fp::N, BLOCK>& sm) {
  using F = typename C::Fp;
  constexpr int N = F::N;
  using S = Stage<N, BLOCK>;
  constexpr bool kEarly = N <= 8;
  static_assert(sizeof(sm.tree) >= 5 * S::G * BLOCK * sizeof(uint4), "staging fits the GAS tree");
  const S sg{&sm.tree[0][0][0]};
  const uint64_t i0 = begin + threadIdx.x;
  const uint64_t row = (uint64_t)j * a.n_chunks;
  auto is_live = [&](uint64_t c) { return (uint32_t)(c * kAccChunk + j) < entries; };
  // pipeline registers: item k (v0, pb0, o0), item k+1 (v1, pb1), item k+2 (v2, pb2)
  uint32_t v0 = 0, pb0 = 0, o0 = 0, v1 = 0, pb1 = 0;
  // ---- compress, ascending
  uint32_t run[N];
  fe_set_one<F>(run);
  if (i0 < end) {
    v0 = a.vals[row + i0];
    pb0 = a.cur[i0];
    acc_stage<C, BLOCK>(sg, a, i0, v0, is_live(i0), false);
    if (j > 0) o0 = a.off[pb0 + 1];
    if (i0 + BLOCK < end) {
      v1 = a.vals[row + i0 + BLOCK];
      pb1 = a.cur[i0 + BLOCK];
    }
  }
  for (uint64_t c = i0; c < end; c += BLOCK) {
    ptx::cp_async_wait_all();
    uint32_t x1[N], x2[N];
    sg.get(S::SX, x1);
    sg.get(S::BX, x2);
    const uint64_t cn = c + BLOCK;
    uint32_t o1 = 0, v2 = 0, pb2 = 0;
    if (cn < end) {
      acc_stage<C, BLOCK>(sg, a, cn, v1, is_live(cn), false);
      if (j > 0) o1 = a.off[pb1 + 1];
      if (cn + BLOCK < end) {
        v2 = a.vals[row + cn + BLOCK];
        pb2 = a.cur[cn + BLOCK];
      }
    }
    a.M.store(c, run);
    const AccCls k = acc_classify(a, c, j, entries, pb0, o0);
    uint32_t d[N];
    if (!k.live || k.start) {
      fe_set_one<F>(d);
    } else if (fe_is_zero<F>(x1) || fe_is_zero<F>(x2) || fe_eq<F>(x1, x2)) {
      uint32_t y1[N], y2[N];
      a.S.y.load(c, y1);
      load_base_y<C>(a, v0, y2);
      add_den<C>(d, x1, y1, x2, y2);
    } else {
      fe_sub<F>(d, x2, x1);
    }
    mont_mul<F>(run, run, d);
    v0 = v1; pb0 = pb1; o0 = o1;
    v1 = v2; pb1 = pb2;
  }
  // ---- inverse of the CTA's product (GAS, Section 3.2); the staging area is
  // the tree inside, so every copy of this thread has landed (waited above)
  uint32_t inv[N];
  cta_invert<F, BLOCK>(inv, run, sm);
  if (i0 >= end) return;
  // ---- DCWPA, descending
  const uint64_t last = i0 + ((end - 1 - i0) / BLOCK) * BLOCK;
  v0 = a.vals[row + last];
  pb0 = a.cur[last];
  acc_stage<C, BLOCK>(sg, a, last, v0, is_live(last), true);
  o0 = j > 0 ? a.off[pb0 + 1] : 0u;
  if (last >= i0 + BLOCK) {
    v1 = a.vals[row + last - BLOCK];
    pb1 = a.cur[last - BLOCK];
  }
  for (uint64_t c = last;; c -= BLOCK) {
    ptx::cp_async_wait_all();
    const bool more = c >= i0 + BLOCK;
    uint32_t o1 = 0, v2 = 0, pb2 = 0;
    // next item's copies and bucket end, first-level loads of the one after
    auto ahead = [&]() {
      if (!more) return;
      const uint64_t cn = c - BLOCK;
      acc_stage<C, BLOCK>(sg, a, cn, v1, is_live(cn), true);
      if (j > 0) o1 = a.off[pb1 + 1];
      if (cn >= i0 + BLOCK) {
        v2 = a.vals[row + cn - BLOCK];
        pb2 = a.cur[cn - BLOCK];
      }
    };
    const AccCls k = acc_classify(a, c, j, entries, pb0, o0);
    const bool neg = (v0 & 0x80000000u) != 0;
    uint32_t xs[N], ys[N], xp[N], yp[N], d[N], mine[N];
    int kind = ADD_RET_T;
    if constexpr (kEarly) {
      uint32_t pre[N];
      sg.get(S::SX, xs);
      sg.get(S::SY, ys);
      sg.get(S::BX, xp);
      sg.get(S::BY, yp);
      sg.get(S::PRE, pre);
      ahead();
      if (neg) fe_neg<F>(yp, yp);
      if (!k.live || k.start) {
        fe_set_one<F>(d);
      } else {
        kind = add_den<C>(d, xs, ys, xp, yp);
      }
      mont_mul<F>(mine, inv, pre);
      mont_mul<F>(inv, inv, d);
    } else {
      if (!k.live || k.start) {
        fe_set_one<F>(d);
      } else {
        sg.get(S::SX, xs);
        sg.get(S::BX, xp);
        if (fe_is_zero<F>(xs) || fe_is_zero<F>(xp) || fe_eq<F>(xs, xp)) {
          sg.get(S::SY, ys);
          sg.get(S::BY, yp);
          if (neg) fe_neg<F>(yp, yp);
          kind = add_den<C>(d, xs, ys, xp, yp);
        } else {
          kind = ADD_REGULAR;
          fe_sub<F>(d, xp, xs);
        }
      }
      {
        uint32_t pre[N];
        sg.get(S::PRE, pre);
        mont_mul<F>(mine, inv, pre);
      }
      mont_mul<F>(inv, inv, d);
      sg.get(S::SX, xs);
      sg.get(S::SY, ys);
      sg.get(S::BX, xp);
      sg.get(S::BY, yp);
      ahead();
      if (neg) fe_neg<F>(yp, yp);
    }
    if (k.live) {
      if (k.start) {
        if (j > 0) {
          a.partial.store(partial_slot(a, k.prev, c), xs, ys);
          a.cur[c] = k.bucket;
        }
        a.S.store(c, xp, yp);
      } else {
        add_finish<C>(xs, ys, kind, mine, xs, ys, xp, yp);
        a.S.store(c, xs, ys);
      }
    }
    if (!more) break;
    v0 = v1; pb0 = pb1; o0 = o1;
    v1 = v2; pb1 = pb2;
  }
}

template <class C, int BLOCK>
__global__ void __launch_bounds__(BLOCK, kGasResidentThreads / BLOCK) k_msm_accumulate(AccArgs<C> a) {
  using F = typename C::Fp;
  constexpr int N = F::N;
  auto& sm = gas_smem<N, BLOCK>();
  const uint32_t entries = a.off[a.n_buckets];
  const uint64_t used = (entries + kAccChunk - 1) / kAccChunk;
  // equal shares of the chunks actually used (at least 32 per CTA)
  uint64_t per = (used + gridDim.x - 1) / gridDim.x;
  if (per < 32) per = 32;
  const uint64_t begin = blockIdx.x * per;
  uint64_t end = begin + per;
  if (end > used) end = used;
  if (end < begin) end = begin;
  for (int j = 0; j < kAccChunk; ++j) acc_round_staged<C, BLOCK>(a, j, entries, begin, end, sm);
  // flush the last running sum of every chunk
  for (uint64_t c = begin + threadIdx.x; c < end; c += BLOCK) {
    uint32_t xs[N], ys[N];
    a.S.load(c, xs, ys);
    a.partial.store(partial_slot(a, a.cur[c], c), xs, ys);
  }
}

// ------------------------------------------------------------------ reduction
//
// Window sum sum_b b E_b (E_b the bucket sums, b = 1 .. 2^(c-1)) in levels.
// Level 1 cuts each window row into chunks of K = 2^red_log consecutive buckets;
// chunk u (buckets lo .. hi-1, 0-based) yields the plain sum R_u and the sum
// S_u = sum_e (e - lo + 1) E_e weighted from the chunk's own first bucket, so
// the window sum is sum_u (S_u + u (K R_u)).  Every later level takes
// elements (R~_e, S~_e) whose target is sum_e (S~_e + e R~_e) and cuts them
// into chunks of kRedChunkN: chunk v yields R_v = sum R~_e and
// S_v = sum_e (S~_e + (e - lo) R~_e), and hands (kRedChunkN R_v, S_v) on, until
// one element per row is left: its S is the window sum.  The multiples of R are
// taken by the producing level (log2 of the chunk size doublings per output).
//
// Before level 1 the partial sums of every bucket are folded into one (a
// batched affine pairwise tree, ceil(log2 k) rounds for k partials; CTAs take
// equal shares of the partial slots, so a bucket holding many entries costs
// rounds only in the CTA that owns it).  Level 1 then has 2^(c-1) / K
// independent chunks per window row (2^red_log buckets each, a per-instance
// layout parameter the autotuner picks) and runs as batched affine additions
// (Section 3.3) with one inversion per CTA per round (Section 3.2): the running
// sums R and S of every chunk walk the chunk's buckets downwards, adding the
// bucket sum to R ("A" event) and then R to S ("S" event).  An S event uses
// the R of before the next bucket's A event, so the two share a round and a
// chunk of k buckets takes k + 1 rounds.  The short upper levels run in
// Jacobian coordinates, one thread per chunk.

constexpr int kRedLog1Default = 5;      // log2 buckets per first-level chunk, by default
constexpr int kRedLog1Max = 10;
constexpr uint32_t kRedChunkN = 4;       // elements per chunk on the later levels
constexpr int kRedLogN = 2;

// First-level items (chunks) in group-major order: the items of one instance
// are [t0, t0 + W * chunks), window row w first, then chunk u.
struct RedRange {
  uint64_t t0;
  uint32_t inst;
  uint32_t chunks;  // chunks per window row
};

// ---- fold: the partial sums of every bucket into its first partial slot
template <class C>
struct FoldArgs {
  using F = typename C::Fp;
  const uint32_t* poff;         // partial-slot offsets per bucket (n_buckets + 1)
  uint32_t n_buckets;
  PtSoA<F> partial;
  SoA<F> M;                     // GAS prefix products, one per slot
  uint32_t* ops;                // per-round list of additions, one word per slot
};

// first b in [0, n] with poff[b] >= x
ECC_DEV uint32_t lower_bound_u32(const uint32_t* v, uint32_t n, uint64_t x) {
  uint32_t lo = 0, hi = n;
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    if (v[mid] < x) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// Round with stride h: slot l of a bucket with k partials adds slot l + h for
// every l that is a multiple of 2h with l + h < k (fold_round_staged below).

// Exclusive prefix sum of v over the CTA (warp shuffles, then the warp
// totals); total gets the CTA sum.  wsum: BLOCK / 32 shared words.
template <int BLOCK>
ECC_DEV uint32_t cta_exclusive_sum(uint32_t v, uint32_t* wsum, uint32_t& total) {
  constexpr int NW = BLOCK / 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wsum[warp] = x;
  __syncthreads();
  if (warp == 0) {
    uint32_t w = lane < NW ? wsum[lane] : 0u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < NW) wsum[lane] = w;
  }
  __syncthreads();
  const uint32_t before = warp > 0 ? wsum[warp - 1] : 0u;
  total = wsum[NW - 1];
  __syncthreads();  // wsum is reused
  return before + x - v;
}

// One fold round over the listed additions (slot s += slot s + h) with the
// operands staged in shared memory: the two partial sums and the prefix
// product of each addition (5 G 16-byte vectors, G = N / 4), the thread's own
// column of the GAS tree (dead outside cta_invert).  The slot list is read two
// additions ahead and the copies run one addition ahead.  With 8 limbs DCWPA
// holds every operand in registers from the top of an addition, so the next
// copies start at once; with 12 limbs it forms the two DCWPA products first
// and starts the next copies once the finish operands are in registers.
template <class C, int BLOCK>
__device__ void fold_round_staged(const FoldArgs<C>& a, uint32_t h, uint64_t s0, uint32_t n_ops,
                                  GasSmem<C::Fp::N, BLOCK>& sm) {
  using F = typename C::Fp;
  constexpr int N = F::N;
  constexpr int G = N / 4;
  constexpr int X0 = 0, Y0 = G, X1 = 2 * G, Y1 = 3 * G, PRE = 4 * G;
  constexpr bool kEarly = N <= 8;
  static_assert(sizeof(sm.tree) >= 5 * G * BLOCK * sizeof(uint4), "staging fits the GAS tree");
  uint4* const base = &sm.tree[0][0][0] + threadIdx.x;
  auto at = [&](int k) { return base + k * BLOCK; };
  auto get = [&](int k0, uint32_t* r) {
#pragma unroll
    for (int g = 0; g < G; ++g) {
      const uint4 q = *at(k0 + g);
      r[4 * g] = q.x;
      r[4 * g + 1] = q.y;
      r[4 * g + 2] = q.z;
      r[4 * g + 3] = q.w;
    }
  };
  auto stage = [&](uint32_t sl, bool full) {
#pragma unroll
    for (int g = 0; g < G; ++g) {
      ptx::cp_async16(at(X0 + g), a.partial.x.vec + g * a.partial.x.stride + sl);
      ptx::cp_async16(at(Y0 + g), a.partial.y.vec + g * a.partial.y.stride + sl);
      ptx::cp_async16(at(X1 + g), a.partial.x.vec + g * a.partial.x.stride + sl + h);
      ptx::cp_async16(at(Y1 + g), a.partial.y.vec + g * a.partial.y.stride + sl + h);
      if (full) ptx::cp_async16(at(PRE + g), a.M.vec + g * a.M.stride + sl);
    }
    ptx::cp_async_commit();
  };
  const uint32_t t = threadIdx.x;
  // ---- compress, ascending
  uint32_t run[N];
  fe_set_one<F>(run);
  uint32_t sA = 0, sB = 0;
  if (t < n_ops) {
    sA = a.ops[s0 + t];
    stage(sA, false);
    if (t + BLOCK < n_ops) sB = a.ops[s0 + t + BLOCK];
  }
  for (uint32_t e = t; e < n_ops; e += BLOCK) {
    ptx::cp_async_wait_all();
    uint32_t x0[N], y0[N], x1[N], y1[N], d[N];
    get(X0, x0);
    get(Y0, y0);
    get(X1, x1);
    get(Y1, y1);
    uint32_t sC = 0;
    if (e + BLOCK < n_ops) {
      stage(sB, false);
      if (e + 2 * BLOCK < n_ops) sC = a.ops[s0 + e + 2 * BLOCK];
    }
    a.M.store(sA, run);
    add_den<C>(d, x0, y0, x1, y1);
    mont_mul<F>(run, run, d);
    sA = sB;
    sB = sC;
  }
  // ---- inverse of the CTA's product (GAS, Section 3.2)
  uint32_t inv[N];
  cta_invert<F, BLOCK>(inv, run, sm);
  if (t >= n_ops) return;
  // ---- DCWPA, descending
  const uint32_t last = t + ((n_ops - 1 - t) / BLOCK) * BLOCK;
  sA = a.ops[s0 + last];
  stage(sA, true);
  sB = last >= t + BLOCK ? a.ops[s0 + last - BLOCK] : 0u;
  for (uint32_t e = last;; e -= BLOCK) {
    ptx::cp_async_wait_all();
    const bool more = e >= t + BLOCK;
    uint32_t sC = 0;
    auto ahead = [&]() {
      if (!more) return;
      stage(sB, true);
      if (e >= t + 2 * BLOCK) sC = a.ops[s0 + e - 2 * BLOCK];
    };
    uint32_t x0[N], y0[N], x1[N], y1[N], d[N], mine[N];
    int kind;
    if constexpr (kEarly) {
      uint32_t pre[N];
      get(X0, x0);
      get(Y0, y0);
      get(X1, x1);
      get(Y1, y1);
      get(PRE, pre);
      ahead();
      kind = add_den<C>(d, x0, y0, x1, y1);
      mont_mul<F>(mine, inv, pre);
    } else {
      get(X0, x0);
      get(X1, x1);
      if (fe_is_zero<F>(x0) || fe_is_zero<F>(x1) || fe_eq<F>(x0, x1)) {
        get(Y0, y0);
        get(Y1, y1);
        kind = add_den<C>(d, x0, y0, x1, y1);
      } else {
        kind = ADD_REGULAR;
        fe_sub<F>(d, x1, x0);
      }
      {
        uint32_t pre[N];
        get(PRE, pre);
        mont_mul<F>(mine, inv, pre);
      }
      get(Y0, y0);
      get(Y1, y1);
      ahead();
    }
    mont_mul<F>(inv, inv, d);
    add_finish<C>(x0, y0, kind, mine, x0, y0, x1, y1);
    a.partial.store(sA, x0, y0);
    if (!more) break;
    sA = sB;
    sB = sC;
  }
}

// Each round first lists the CTA's pair additions (slot of the left operand)
// in ops[s0 ..), then runs the batched additions over that list, so the work
// of a bucket with many partial sums (the top window often puts most entries
// into a few buckets) is shared by the whole CTA and lanes never idle on
// inactive slots.
template <class C, int BLOCK>
__global__ void __launch_bounds__(BLOCK, kGasResidentThreads / BLOCK) k_msm_fold(FoldArgs<C> a) {
  using F = typename C::Fp;
  constexpr int N = F::N;
  auto& sm = gas_smem<N, BLOCK>();
  __shared__ uint32_t wsum[BLOCK / 32];
  const uint64_t total_slots = a.poff[a.n_buckets];
  if (total_slots == 0) return;  // uniform over the grid
  // this CTA owns the buckets whose first slot lies in its equal share
  const uint64_t share = (total_slots + gridDim.x - 1) / gridDim.x;
  const uint32_t b0 = lower_bound_u32(a.poff, a.n_buckets, blockIdx.x * share);
  const uint32_t b1 = blockIdx.x + 1 == gridDim.x
                          ? a.n_buckets
                          : lower_bound_u32(a.poff, a.n_buckets, (blockIdx.x + 1) * share);
  const uint64_t s0 = a.poff[b0];
  uint32_t kmax = 0;
  for (uint32_t b = b0 + threadIdx.x; b < b1; b += BLOCK) {
    const uint32_t k = a.poff[b + 1] - a.poff[b];
    kmax = k > kmax ? k : kmax;
  }
  // ceil(log2 kmax) rounds; each halves the partials of every bucket
  for (uint32_t h = 1; __syncthreads_or(h < kmax); h *= 2) {
    // list the round's additions: l = 0, 2h, 4h, .. with l + h < k
    uint32_t cnt = 0;
    for (uint32_t b = b0 + threadIdx.x; b < b1; b += BLOCK) {
      const uint32_t k = a.poff[b + 1] - a.poff[b];
      if (k > h) cnt += (k - h - 1) / (2 * h) + 1;
    }
    uint32_t n_ops;
    uint32_t pos = cta_exclusive_sum<BLOCK>(cnt, wsum, n_ops);
    for (uint32_t b = b0 + threadIdx.x; b < b1; b += BLOCK) {
      const uint32_t p = a.poff[b];
      const uint32_t k = a.poff[b + 1] - p;
      for (uint32_t l = 0; l + h < k; l += 2 * h) a.ops[s0 + pos++] = p + l;
    }
    __syncthreads();  // the list is complete
    fold_round_staged<C, BLOCK>(a, h, s0, n_ops, sm);
  }
}

template <class C>
struct AffRedArgs {
  using F = typename C::Fp;
  const MsmInst* inst;
  const RedRange* ranges;
  uint32_t n_ranges;
  uint64_t items;
  const uint32_t* poff;   // partial-slot offsets per bucket (n_buckets + 1 entries)
  PtSoA<F> partial;       // partial bucket sums (affine)
  PtSoA<F> R, S;          // running sums per item (affine)
  SoA<F> M;               // GAS prefix products per item
  uint32_t* cur_e;        // 1 + the bucket the next event belongs to
  uint32_t* cur_a;        // whether that bucket's A event is done
  uint32_t* lo_b;         // first bucket of the item
  uint32_t* rlog;         // log2 of the item's chunk size (its instance's red_log)
  Jac<F>* out_R;          // 2^rlog R per item (Jacobian, Z = 1 or O)
  Jac<F>* out_S;
  uint64_t per_cta;
};

ECC_DEV uint32_t find_range(const RedRange* r, uint32_t num, uint64_t t) {
  uint32_t lo = 0, hi = num - 1;
  while (lo < hi) {
    const uint32_t mid = (lo + hi + 1) >> 1;
    if (r[mid].t0 <= t) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// The events of this round for an item at (ep, ad): ep = 1 + the current
// bucket, ad = whether its A event is done.  An S event (S += R) and/or an A
// event (R += bucket sum, held in the bucket's first partial slot after the
// fold); (ep2, ad2) is the position after them.
struct RedStep {
  bool opS, opA;
  uint32_t slot, ep2, ad2;
};

ECC_DEV RedStep red_step(const uint32_t* poff, uint32_t ep, uint32_t ad, uint32_t lo) {
  RedStep r{false, false, 0u, ep, ad};
  if (ep == lo) return r;                          // every event done
  if (!ad) {
    r.ad2 = 1;
    if (poff[ep] > poff[ep - 1]) {                 // bucket ep-1 is not empty
      r.opA = true;
      r.slot = poff[ep - 1];
      return r;
    }
  }
  r.opS = true;                                    // bucket ep-1 is complete
  r.ep2 = ep - 1;
  r.ad2 = 0;
  if (r.ep2 != lo) {
    r.ad2 = 1;
    if (poff[r.ep2] > poff[r.ep2 - 1]) {
      r.opA = true;
      r.slot = poff[r.ep2 - 1];
    }
  }
  return r;
}

template <class C>
struct AffRedRound {
  using F = typename C::Fp;
  static constexpr int N = F::N;
  static constexpr int OPS = 2;  // op 0: S += R, op 1: R += partial
  const AffRedArgs<C>* a;
  RedStep st;
  int kind_s, kind_a;
  bool more;
  ECC_DEV void den_c(size_t i, int j, uint32_t* d) {
    if (j == 0) {
      st = red_step(a->poff, a->cur_e[i], a->cur_a[i], a->lo_b[i]);
      if (!st.opS) {
        fe_set_one<F>(d);
        kind_s = ADD_RET_T;
        return;
      }
      uint32_t xs[N], ys[N], xr[N], yr[N];
      a->S.load(i, xs, ys);
      a->R.load(i, xr, yr);
      kind_s = add_den<C>(d, xs, ys, xr, yr);
    } else {
      if (!st.opA) {
        fe_set_one<F>(d);
        kind_a = ADD_RET_T;
        return;
      }
      uint32_t xr[N], yr[N], xp[N], yp[N];
      a->R.load(i, xr, yr);
      a->partial.load(st.slot, xp, yp);
      kind_a = add_den<C>(d, xr, yr, xp, yp);
    }
  }
  ECC_DEV void den_d(size_t i, int j, uint32_t* d) { den_c(i, j, d); }
  ECC_DEV void finish(size_t i, const uint32_t (*inv)[N]) {
    if (!st.opS && !st.opA) return;
    uint32_t xr[N], yr[N];
    a->R.load(i, xr, yr);
    if (st.opS) {
      uint32_t xs[N], ys[N];
      a->S.load(i, xs, ys);
      add_finish<C>(xs, ys, kind_s, inv[0], xs, ys, xr, yr);
      a->S.store(i, xs, ys);
    }
    if (st.opA) {
      uint32_t xp[N], yp[N];
      a->partial.load(st.slot, xp, yp);
      add_finish<C>(xr, yr, kind_a, inv[1], xr, yr, xp, yp);
      a->R.store(i, xr, yr);
    }
    a->cur_e[i] = st.ep2;
    a->cur_a[i] = st.ad2;
    more |= st.ep2 != a->lo_b[i];
  }
};

// ---- 8-limb fields: the walk's rounds with their operands staged in shared
// memory.  Each thread owns two sets (a double buffer) of 6 G 16-byte vectors
// holding S, R and the bucket's partial sum P (x and y of each, G = N / 4
// vectors per element, layout [vector][thread]): one set holds the current
// item's operands while the cp.async copies of the next item's land in the
// other.  The thread's own column of the GAS tree (dead outside cta_invert)
// provides 5 G of the vectors; the rest follows the GasSmem block.  The
// item's cursor words are loaded two items ahead, its bucket offsets (the
// event step) one item ahead together with the copies, and DCWPA's prefix
// product one item ahead into registers.
template <int N, int BLOCK>
struct RedStage {
  static constexpr int G = N / 4;
  static constexpr int SX = 0, SY = G, RX = 2 * G, RY = 3 * G, PX = 4 * G, PY = 5 * G;
  static constexpr int SET = 6 * G;
  static constexpr int TREE = 5 * G;
  static constexpr int EXTRA = 2 * SET - TREE;
  uint4* tree;
  uint4* extra;
  ECC_DEV uint4* at(int set, int k) const {
    const int s = set * SET + k;
    return (s < TREE ? tree + s * BLOCK : extra + (s - TREE) * BLOCK) + threadIdx.x;
  }
  ECC_DEV void get(int set, int k0, uint32_t* r) const {
#pragma unroll
    for (int g = 0; g < G; ++g) {
      const uint4 p = *at(set, k0 + g);
      r[4 * g] = p.x;
      r[4 * g + 1] = p.y;
      r[4 * g + 2] = p.z;
      r[4 * g + 3] = p.w;
    }
  }
};

template <int N, int BLOCK>
constexpr size_t red_smem_bytes() {
  return sizeof(GasSmem<N, BLOCK>) + (size_t)RedStage<N, BLOCK>::EXTRA * BLOCK * sizeof(uint4);
}

// Copies item t's S and R, and the partial sum its A event adds.
template <class C, int BLOCK>
ECC_DEV void red_stage(const RedStage<C::Fp::N, BLOCK>& sg, int set, const AffRedArgs<C>& a,
                       uint64_t t, const RedStep& st) {
  using S = RedStage<C::Fp::N, BLOCK>;
#pragma unroll
  for (int g = 0; g < S::G; ++g) {
    ptx::cp_async16(sg.at(set, S::SX + g), a.S.x.vec + g * a.S.x.stride + t);
    ptx::cp_async16(sg.at(set, S::SY + g), a.S.y.vec + g * a.S.y.stride + t);
    ptx::cp_async16(sg.at(set, S::RX + g), a.R.x.vec + g * a.R.x.stride + t);
    ptx::cp_async16(sg.at(set, S::RY + g), a.R.y.vec + g * a.R.y.stride + t);
  }
  if (st.opA) {
#pragma unroll
    for (int g = 0; g < S::G; ++g) {
      ptx::cp_async16(sg.at(set, S::PX + g), a.partial.x.vec + g * a.partial.x.stride + st.slot);
      ptx::cp_async16(sg.at(set, S::PY + g), a.partial.y.vec + g * a.partial.y.stride + st.slot);
    }
  }
  ptx::cp_async_commit();
}

// One round of the walk over the items [begin, end) of this CTA; returns
// whether any of this thread's items has events left.
template <class C, int BLOCK>
__device__ bool red_round_staged(const AffRedArgs<C>& a, uint64_t begin, uint64_t end,
                                 GasSmem<C::Fp::N, BLOCK>& sm, uint4* extra) {
  using F = typename C::Fp;
  constexpr int N = F::N;
  using S = RedStage<N, BLOCK>;
  const S sg{&sm.tree[0][0][0], extra};
  const uint64_t i0 = begin + threadIdx.x;
  bool more = false;
  // cursor words of item t: (ep, ad, lo)
  uint32_t e1 = 0, a1 = 0, l1 = 0;
  auto cursor = [&](uint64_t t, uint32_t& e, uint32_t& d, uint32_t& l) {
    e = a.cur_e[t];
    d = a.cur_a[t];
    l = a.lo_b[t];
  };
  // ---- compress, ascending
  uint32_t run[N];
  fe_set_one<F>(run);
  RedStep st0{};
  if (i0 < end) {
    uint32_t e0, d0, l0;
    cursor(i0, e0, d0, l0);
    st0 = red_step(a.poff, e0, d0, l0);
    red_stage<C, BLOCK>(sg, 0, a, i0, st0);
    if (i0 + BLOCK < end) cursor(i0 + BLOCK, e1, a1, l1);
  }
  int set = 0;
  for (uint64_t t = i0; t < end; t += BLOCK, set ^= 1) {
    RedStep st1{};
    const bool next = t + BLOCK < end;
    if (next) {
      st1 = red_step(a.poff, e1, a1, l1);
      red_stage<C, BLOCK>(sg, set ^ 1, a, t + BLOCK, st1);
      if (t + 2 * BLOCK < end) cursor(t + 2 * BLOCK, e1, a1, l1);
      ptx::cp_async_wait_prior();
    } else {
      ptx::cp_async_wait_all();
    }
    a.M.store(t, run);
    uint32_t d[N];
    if (st0.opS) {
      uint32_t xs[N], ys[N], xr[N], yr[N];
      sg.get(set, S::SX, xs);
      sg.get(set, S::SY, ys);
      sg.get(set, S::RX, xr);
      sg.get(set, S::RY, yr);
      add_den<C>(d, xs, ys, xr, yr);
      mont_mul<F>(run, run, d);
    }
    if (st0.opA) {
      uint32_t xr[N], yr[N], xp[N], yp[N];
      sg.get(set, S::RX, xr);
      sg.get(set, S::RY, yr);
      sg.get(set, S::PX, xp);
      sg.get(set, S::PY, yp);
      add_den<C>(d, xr, yr, xp, yp);
      mont_mul<F>(run, run, d);
    }
    st0 = st1;
  }
  // ---- inverse of the CTA's product (GAS, Section 3.2); every copy of this
  // thread has landed (waited above), so its tree column is free
  uint32_t inv[N];
  cta_invert<F, BLOCK>(inv, run, sm);
  if (i0 >= end) return false;
  // ---- DCWPA, descending
  const uint64_t last = i0 + ((end - 1 - i0) / BLOCK) * BLOCK;
  uint32_t e0, d0, lo0;
  cursor(last, e0, d0, lo0);
  st0 = red_step(a.poff, e0, d0, lo0);
  red_stage<C, BLOCK>(sg, 0, a, last, st0);
  uint32_t pre0[N];
  a.M.load(last, pre0);
  if (last >= i0 + BLOCK) cursor(last - BLOCK, e1, a1, l1);
  set = 0;
  for (uint64_t t = last;; t -= BLOCK, set ^= 1) {
    const bool next = t >= i0 + BLOCK;
    RedStep st1{};
    uint32_t pre1n[N], lo1 = 0;
    if (next) {
      st1 = red_step(a.poff, e1, a1, l1);
      lo1 = l1;
      red_stage<C, BLOCK>(sg, set ^ 1, a, t - BLOCK, st1);
      a.M.load(t - BLOCK, pre1n);
      if (t >= i0 + 2 * BLOCK) cursor(t - 2 * BLOCK, e1, a1, l1);
      ptx::cp_async_wait_prior();
    } else {
      ptx::cp_async_wait_all();
    }
    // the item's two denominators again (recompute), then its two inverses
    uint32_t dS[N], dA[N];
    int kind_s = ADD_RET_T, kind_a = ADD_RET_T;
    fe_set_one<F>(dS);
    fe_set_one<F>(dA);
    if (st0.opS) {
      uint32_t xs[N], ys[N], xr[N], yr[N];
      sg.get(set, S::SX, xs);
      sg.get(set, S::SY, ys);
      sg.get(set, S::RX, xr);
      sg.get(set, S::RY, yr);
      kind_s = add_den<C>(dS, xs, ys, xr, yr);
    }
    if (st0.opA) {
      uint32_t xr[N], yr[N], xp[N], yp[N];
      sg.get(set, S::RX, xr);
      sg.get(set, S::RY, yr);
      sg.get(set, S::PX, xp);
      sg.get(set, S::PY, yp);
      kind_a = add_den<C>(dA, xr, yr, xp, yp);
    }
    uint32_t invS[N], invA[N];
    {
      uint32_t pre1[N];
      mont_mul<F>(pre1, pre0, dS);
      mont_mul<F>(invA, inv, pre1);
    }
    mont_mul<F>(inv, inv, dA);
    mont_mul<F>(invS, inv, pre0);
    mont_mul<F>(inv, inv, dS);
    if (st0.opS || st0.opA) {
      uint32_t xr[N], yr[N];
      sg.get(set, S::RX, xr);
      sg.get(set, S::RY, yr);
      if (st0.opS) {  // S += R, with R of before this round's A event
        uint32_t xs[N], ys[N];
        sg.get(set, S::SX, xs);
        sg.get(set, S::SY, ys);
        add_finish<C>(xs, ys, kind_s, invS, xs, ys, xr, yr);
        a.S.store(t, xs, ys);
      }
      if (st0.opA) {  // R += the bucket's sum
        uint32_t xp[N], yp[N];
        sg.get(set, S::PX, xp);
        sg.get(set, S::PY, yp);
        add_finish<C>(xr, yr, kind_a, invA, xr, yr, xp, yp);
        a.R.store(t, xr, yr);
      }
      a.cur_e[t] = st0.ep2;
      a.cur_a[t] = st0.ad2;
      more |= st0.ep2 != lo0;
    }
    if (!next) break;
    st0 = st1;
    lo0 = lo1;
    fe_copy<F>(pre0, pre1n);
  }
  return more;
}

// R <- 2 R for every item whose chunk needs more than k doublings (batched PDBL)
template <class C>
struct AffDblRound {
  using F = typename C::Fp;
  static constexpr int N = F::N;
  static constexpr int OPS = 1;
  const AffRedArgs<C>* a;
  uint32_t k;
  bool live, skip;
  ECC_DEV void den_c(size_t i, int, uint32_t* d) {
    skip = a->rlog[i] <= k;
    if (skip) {
      fe_set_one<F>(d);
      return;
    }
    uint32_t x[N], y[N];
    a->R.load(i, x, y);
    live = dbl_den<C>(d, y);
  }
  ECC_DEV void den_d(size_t i, int j, uint32_t* d) { den_c(i, j, d); }
  ECC_DEV void finish(size_t i, const uint32_t (*inv)[N]) {
    if (skip) return;
    uint32_t x[N], y[N];
    a->R.load(i, x, y);
    dbl_finish<C>(x, y, live, inv[0], x, y);
    a->R.store(i, x, y);
  }
};

template <class C, int BLOCK>
__global__ void __launch_bounds__(BLOCK, kGasResidentThreads / BLOCK)
    k_msm_reduce_affine(AffRedArgs<C> a) {
  using F = typename C::Fp;
  constexpr int N = F::N;
  auto& sm = gas_smem<N, BLOCK>();
  const uint64_t begin = blockIdx.x * a.per_cta;
  uint64_t end = begin + a.per_cta;
  if (end > a.items) end = a.items;
  if (end < begin) end = begin;
  // start every item at the top of its chunk with R = S = O
  bool more = false;
  for (uint64_t t = begin + threadIdx.x; t < end; t += BLOCK) {
    const RedRange rg = a.ranges[find_range(a.ranges, a.n_ranges, t)];
    const MsmInst in = a.inst[rg.inst];
    const uint32_t B = 1u << (in.c - 1);
    const uint64_t local = t - rg.t0;
    const uint32_t w = (uint32_t)(local / rg.chunks), u = (uint32_t)(local % rg.chunks);
    const uint32_t K = 1u << in.red_log;
    const uint32_t lo = in.bucket_base + w * B + u * K;
    const uint32_t hi = lo + (B - u * K < K ? B - u * K : K);
    a.lo_b[t] = lo;
    a.rlog[t] = in.red_log;
    a.cur_e[t] = hi;
    a.cur_a[t] = 0;
    uint32_t z[N];
    fe_set_zero<F>(z);
    a.R.store(t, z, z);
    a.S.store(t, z, z);
    more = true;
  }
  // one bounded loop: each round completes at least one event of every live
  // item, and an item has at most 2^(rlog + 1) events
  while (__syncthreads_or(more)) {
    if constexpr (N == 8) {
      extern __shared__ __align__(16) unsigned char ecc_dyn_smem[];
      uint4* extra = reinterpret_cast<uint4*>(ecc_dyn_smem + sizeof(GasSmem<N, BLOCK>));
      more = red_round_staged<C, BLOCK>(a, begin, end, sm, extra);
    } else {
      AffRedRound<C> rd{&a};
      rd.more = false;
      batch_round<F, BLOCK>(rd, begin, end, a.M, sm);
      more = rd.more;
    }
  }
  // R <- 2^rlog R: as many doubling rounds as the CTA's largest chunk needs
  for (uint32_t k = 0; k < (uint32_t)kRedLog1Max; ++k) {
    bool want = false;
    for (uint64_t t = begin + threadIdx.x; t < end; t += BLOCK) want |= a.rlog[t] > k;
    if (!__syncthreads_or(want)) break;
    AffDblRound<C> rd{&a, k};
    batch_round<F, BLOCK>(rd, begin, end, a.M, sm);
  }
  for (uint64_t t = begin + threadIdx.x; t < end; t += BLOCK) {
    uint32_t x[N], y[N];
    Jac<F> P;
    a.R.load(t, x, y);
    jac_from_affine<C>(P, x, y);
    a.out_R[t] = P;
    a.S.load(t, x, y);
    jac_from_affine<C>(P, x, y);
    a.out_S[t] = P;
  }
}

// One later level for every window row of a set of groups.  Segment k covers
// threads [t0, t0 + rows * chunks); its input rows have `elems` elements at
// JR/JS + in_off, its outputs go to + out_off.
struct LevelSeg {
  uint64_t t0;
  uint64_t rows;
  uint32_t elems;
  uint32_t chunks;
  uint64_t in_off;
  uint64_t out_off;
};

ECC_DEV uint32_t find_seg(const LevelSeg* s, uint32_t num, uint64_t t) {
  uint32_t lo = 0, hi = num - 1;
  while (lo < hi) {
    const uint32_t mid = (lo + hi + 1) >> 1;
    if (s[mid].t0 <= t) lo = mid; else hi = mid - 1;
  }
  return lo;
}

template <class C>
__global__ void k_msm_reduce_level(const LevelSeg* segs, uint32_t n_segs, uint64_t threads,
                                   Jac<typename C::Fp>* JR, Jac<typename C::Fp>* JS) {
  using F = typename C::Fp;
  const uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (t >= threads) return;
  const LevelSeg sg = segs[find_seg(segs, n_segs, t)];
  const uint64_t local = t - sg.t0;
  const uint64_t row = local / sg.chunks;
  const uint32_t v = (uint32_t)(local % sg.chunks);
  const uint32_t lo = v * kRedChunkN;
  const uint32_t hi = lo + kRedChunkN < sg.elems ? lo + kRedChunkN : sg.elems;  // exclusive
  const Jac<F>* inR = JR + sg.in_off + row * sg.elems;
  const Jac<F>* inS = JS + sg.in_off + row * sg.elems;
  Jac<F> Rr, U, Ssum, E;
  jac_set_inf<C>(Rr);
  jac_set_inf<C>(U);
  jac_set_inf<C>(Ssum);
  for (uint32_t e = hi; e-- > lo;) {
    E = inS[e];
    jac_add<C>(Ssum, Ssum, E);
    E = inR[e];
    jac_add<C>(Rr, Rr, E);
    if (e > lo) jac_add<C>(U, U, Rr);
  }
  jac_add<C>(Ssum, Ssum, U);
  if (sg.chunks > 1) {
    for (int k = 0; k < kRedLogN; ++k) jac_dbl<C>(Rr, Rr);
  }
  JR[sg.out_off + row * sg.chunks + v] = Rr;
  JS[sg.out_off + row * sg.chunks + v] = Ssum;
}

// result_i = sum_w 2^(c w) S_w (Horner), converted to canonical affine limbs;
// instance i's window sums are S[fin[i] + w].  Thread t takes instance
// order[t]: the host lists the instances grouped by window width, so the lanes
// of a warp run chains of one length (a warp executes the longest chain among
// its lanes).
template <class C>
__global__ void k_msm_combine(const MsmInst* inst, const uint64_t* fin, const uint32_t* order,
                              uint32_t num, const Jac<typename C::Fp>* S, const MsmDevHdr* hdr,
                              uint32_t* out_all) {
  using F = typename C::Fp;
  constexpr int N = F::N;
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= num) return;
  const uint32_t id = order[t];
  if (hdr && hdr->failed) {  // refused sizes: O, written (0, 0)
    for (int q = 0; q < 2 * N; ++q) out_all[(uint64_t)id * 2 * N + q] = 0;
    return;
  }
  const uint32_t c = inst[id].c, W = inst[id].Wr;
  const Jac<F>* Sw = S + fin[id];
  Jac<F> acc = Sw[W - 1];
  for (int w = (int)W - 2; w >= 0; --w) {
    for (uint32_t s = 0; s < c; ++s) jac_dbl_inl<C>(acc, acc);
    jac_add_inl<C>(acc, acc, Sw[w]);
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
__global__ void k_points_to_mont(const uint32_t* __restrict__ in, uint64_t n, const MsmDevHdr* hdr,
                                 uint32_t* __restrict__ out) {
  using F = typename C::Fp;
  constexpr int N = F::N;
  const uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (i >= batch_rows(n, hdr)) return;
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

// ------------------------------------------------------------------ window multiples
// For bases reused across calls: window w of base i becomes 2^(c w) P_i
// (window-major AoS, Montgomery form), so one set of buckets serves every
// window.  Window w is window w-1 doubled c times: c batched PDBL rounds per
// window, every item an independent base.
template <class C>
struct ShiftArgs {
  using F = typename C::Fp;
  uint32_t* pre;     // W windows of n points, 2N words each; window 0 filled in
  uint64_t n;
  uint32_t W, c;
  SoA<F> M;
  uint64_t per_cta;
};

template <class C>
ECC_DEV void aos_load(const uint32_t* base, uint64_t i, uint32_t* x, uint32_t* y) {
  constexpr int N = C::Fp::N;
  const uint4* p = reinterpret_cast<const uint4*>(base + i * 2 * N);
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
}

template <class C>
ECC_DEV void aos_store(uint32_t* base, uint64_t i, const uint32_t* x, const uint32_t* y) {
  constexpr int N = C::Fp::N;
  uint4* p = reinterpret_cast<uint4*>(base + i * 2 * N);
#pragma unroll
  for (int g = 0; g < N / 4; ++g) p[g] = make_uint4(x[4 * g], x[4 * g + 1], x[4 * g + 2], x[4 * g + 3]);
#pragma unroll
  for (int g = 0; g < N / 4; ++g)
    p[N / 4 + g] = make_uint4(y[4 * g], y[4 * g + 1], y[4 * g + 2], y[4 * g + 3]);
}

template <class C>
struct ShiftRound {
  using F = typename C::Fp;
  static constexpr int N = F::N;
  static constexpr int OPS = 1;
  const uint32_t* src;
  uint32_t* dst;
  bool live;
  ECC_DEV void den_c(size_t i, int, uint32_t* d) {
    uint32_t x[N], y[N];
    aos_load<C>(src, i, x, y);
    live = dbl_den<C>(d, y);
  }
  ECC_DEV void den_d(size_t i, int j, uint32_t* d) { den_c(i, j, d); }
  ECC_DEV void finish(size_t i, const uint32_t (*inv)[N]) {
    uint32_t x[N], y[N];
    aos_load<C>(src, i, x, y);
    dbl_finish<C>(x, y, live, inv[0], x, y);
    aos_store<C>(dst, i, x, y);
  }
};

template <class C, int BLOCK>
__global__ void __launch_bounds__(BLOCK, kGasResidentThreads / BLOCK) k_bases_shift(ShiftArgs<C> a) {
  using F = typename C::Fp;
  constexpr int N = F::N;
  auto& sm = gas_smem<N, BLOCK>();
  const uint64_t begin = blockIdx.x * a.per_cta;
  uint64_t end = begin + a.per_cta;
  if (end > a.n) end = a.n;
  if (end < begin) end = begin;
  for (uint32_t w = 1; w < a.W; ++w) {
    uint32_t* dst = a.pre + (uint64_t)w * a.n * 2 * N;
    for (uint32_t r = 0; r < a.c; ++r) {
      ShiftRound<C> rd{r == 0 ? dst - a.n * 2 * N : dst, dst};
      batch_round<F, BLOCK>(rd, begin, end, a.M, sm);
    }
  }
}

}  // namespace ecc
