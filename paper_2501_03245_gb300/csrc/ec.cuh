// EC operator layer (Section 3): limb-interleaved SoA storage, the per-CTA
// gather-apply-scatter batch inversion (Section 3.2), and batched affine
// PADD / PDBL rounds with the compress / inverse / DCWPA structure (Section 3.3).
#pragma once
#include <cstddef>
#include <cstdint>

#include <cooperative_groups.h>

#include "curves_gen.cuh"
#include "fp.cuh"

namespace ecc {

// --------------------------------------------------------------------------
// Column-major ("limb-interleaved") storage of n field elements (Section 3.3,
// cache-efficient data layout): limbs 4g..4g+3 of element i form one 16-byte
// vector at vec[g * stride + i], so a warp reading element i = base + lane of
// one limb group issues 32 consecutive 16-byte loads.
template <class F>
struct SoA {
  static constexpr int G = F::N / 4;
  uint4* vec;
  size_t stride;

  ECC_DEV void load(size_t i, uint32_t* r) const {
#pragma unroll
    for (int g = 0; g < G; ++g) {
      uint4 v = vec[g * stride + i];
      r[4 * g + 0] = v.x;
      r[4 * g + 1] = v.y;
      r[4 * g + 2] = v.z;
      r[4 * g + 3] = v.w;
    }
  }
  ECC_DEV void store(size_t i, const uint32_t* r) const {
#pragma unroll
    for (int g = 0; g < G; ++g) {
      vec[g * stride + i] = make_uint4(r[4 * g + 0], r[4 * g + 1], r[4 * g + 2], r[4 * g + 3]);
    }
  }
  __host__ __device__ __forceinline__ SoA at(size_t offset) const { return SoA{vec + offset, stride}; }
};

template <class F>
struct PtSoA {
  SoA<F> x, y;
  ECC_DEV void load(size_t i, uint32_t* px, uint32_t* py) const {
    x.load(i, px);
    y.load(i, py);
  }
  ECC_DEV void store(size_t i, const uint32_t* px, const uint32_t* py) const {
    x.store(i, px);
    y.store(i, py);
  }
};

// Bytes of SoA storage for n elements of field F.
template <class F>
constexpr size_t soa_bytes(size_t n) {
  return n * F::N * 4;
}

// --------------------------------------------------------------------------
// Curve helpers.  Points are affine (x, y) in Montgomery form; the point at
// infinity O is stored as (0, 0), which lies on none of the supported curves
// (b != 0).
template <class C>
ECC_DEV void curve_a(uint32_t* r) {
#pragma unroll
  for (int i = 0; i < C::Fp::N; ++i) r[i] = C::a(i);
}

template <class F>
ECC_DEV bool pt_is_inf(const uint32_t* x, const uint32_t* y) {
  uint32_t acc = 0;
#pragma unroll
  for (int i = 0; i < F::N; ++i) acc |= x[i] | y[i];
  return acc == 0;
}

// 3 x^2 + a (numerator of the PDBL slope, Section 2.1.1)
template <class C>
ECC_DEV void dbl_numerator(uint32_t* num, const uint32_t* x) {
  using F = typename C::Fp;
  uint32_t t[F::N];
  mont_sqr<F>(t, x);
  fe_add<F>(num, t, t);
  fe_add<F>(num, num, t);
  if (!C::A_ZERO) {
    uint32_t a[F::N];
    curve_a<C>(a);
    fe_add<F>(num, num, a);
  }
}

// Classification of P + T for the batched formulas.
enum AddKind : int { ADD_REGULAR = 0, ADD_DOUBLE = 1, ADD_RET_T = 2, ADD_RET_P = 3, ADD_RET_INF = 4 };

// Denominator of lambda for P + T (Eqn 2, or PDBL when P = T), or 1 when the
// result needs no slope (an operand is O, or P = -T).
template <class C>
ECC_DEV int add_kind(const uint32_t* xp, const uint32_t* yp, const uint32_t* xt, const uint32_t* yt) {
  using F = typename C::Fp;
  if (pt_is_inf<F>(xp, yp)) return ADD_RET_T;
  if (pt_is_inf<F>(xt, yt)) return ADD_RET_P;
  if (!fe_eq<F>(xp, xt)) return ADD_REGULAR;
  if (fe_eq<F>(yp, yt) && !fe_is_zero<F>(yp)) return ADD_DOUBLE;
  return ADD_RET_INF;
}

template <class C>
ECC_DEV int add_den(uint32_t* den, const uint32_t* xp, const uint32_t* yp, const uint32_t* xt,
                    const uint32_t* yt) {
  using F = typename C::Fp;
  const int kind = add_kind<C>(xp, yp, xt, yt);
  if (kind == ADD_REGULAR) {
    fe_sub<F>(den, xt, xp);
  } else if (kind == ADD_DOUBLE) {
    fe_add<F>(den, yp, yp);
  } else {
    fe_set_one<F>(den);
  }
  return kind;
}

// Completes R = P + T given kind and inv = 1 / den (Eqn 2-3; PDBL slope for
// ADD_DOUBLE).  R may alias P or T.
template <class C>
ECC_DEV void add_finish(uint32_t* xr, uint32_t* yr, int kind, const uint32_t* inv,
                        const uint32_t* xp, const uint32_t* yp, const uint32_t* xt,
                        const uint32_t* yt) {
  using F = typename C::Fp;
  constexpr int N = F::N;
  if (kind == ADD_REGULAR || kind == ADD_DOUBLE) {
    uint32_t num[N], lam[N], x3[N], t[N];
    if (kind == ADD_REGULAR) {
      fe_sub<F>(num, yt, yp);
    } else {
      dbl_numerator<C>(num, xp);
    }
    mont_mul<F>(lam, num, inv);
    mont_sqr<F>(x3, lam);
    fe_sub<F>(x3, x3, xp);
    fe_sub<F>(x3, x3, xt);
    fe_sub<F>(t, xp, x3);
    mont_mul<F>(t, lam, t);
    fe_sub<F>(yr, t, yp);
    fe_copy<F>(xr, x3);
  } else if (kind == ADD_RET_T) {
    fe_copy<F>(xr, xt);
    fe_copy<F>(yr, yt);
  } else if (kind == ADD_RET_P) {
    fe_copy<F>(xr, xp);
    fe_copy<F>(yr, yp);
  } else {
    fe_set_zero<F>(xr);
    fe_set_zero<F>(yr);
  }
}

// PDBL denominator 2y, or 1 when the result is O (P = O or y = 0).
template <class C>
ECC_DEV bool dbl_den(uint32_t* den, const uint32_t* y) {
  using F = typename C::Fp;
  const bool live = !fe_is_zero<F>(y);
  if (live) {
    fe_add<F>(den, y, y);
  } else {
    fe_set_one<F>(den);
  }
  return live;
}

template <class C>
ECC_DEV void dbl_finish(uint32_t* xr, uint32_t* yr, bool live, const uint32_t* inv,
                        const uint32_t* x, const uint32_t* y) {
  using F = typename C::Fp;
  constexpr int N = F::N;
  if (live) {
    uint32_t num[N], lam[N], x3[N], t[N];
    dbl_numerator<C>(num, x);
    mont_mul<F>(lam, num, inv);
    mont_sqr<F>(x3, lam);
    fe_sub<F>(x3, x3, x);
    fe_sub<F>(x3, x3, x);
    fe_sub<F>(t, x, x3);
    mont_mul<F>(t, lam, t);
    fe_sub<F>(yr, t, y);
    fe_copy<F>(xr, x3);
  } else {
    fe_set_zero<F>(xr);
    fe_set_zero<F>(yr);
  }
}

// --------------------------------------------------------------------------
// Per-CTA gather-apply-scatter inversion (Section 3.2).  Every thread brings
// the product of its own chain; every thread gets back the inverse of its own
// product.  Gather: a butterfly product tree inside each warp (shuffles), then
// the warp totals in shared memory; apply: one thread inverts the CTA total
// (divstep inversion, the shortest serial chain available to one thread);
// scatter: the tree walked back down (each level peels the partner subtree).
// One batch-inversion group per CTA of kGasThreads threads; kGasCtasPerSm such
// CTAs are resident per SM (128 registers per thread), so while one CTA waits
// for its group's inversion the other keeps the SM's multiply-add pipe busy.
// (Measured on GB300: 2 x 256 threads beats 4 x 128, whose halved groups pay
// twice the inversions per item.)
constexpr int kGasThreads = 256;
constexpr int kGasCtasPerSm = 2;
constexpr int kGasResidentThreads = kGasThreads * kGasCtasPerSm;

template <int N, int BLOCK>
struct GasSmem {
  static constexpr int NW = BLOCK / 32;
  // subtree products per level as 16-byte vectors, thread-fastest (a warp's
  // stores of one vector are 512 contiguous bytes); every thread touches only
  // its own column [.][.][threadIdx.x], which is what lets a kernel reuse the
  // area as per-thread staging outside cta_invert
  uint4 tree[5][N / 4][BLOCK];
  uint32_t warp_tot[NW][N];
  uint32_t warp_inv[NW][N];
  uint32_t pair_in[4][N];  // cluster inversion: the other CTAs' totals (in CTA 0)
  uint32_t pair_out[N];    // and the inverse CTA 0 sends back
};

// The GAS scratch lives in dynamic shared memory (it exceeds the 48 KB static
// limit for 12-limb fields); launches pass sizeof(GasSmem<N, BLOCK>).
template <int N, int BLOCK>
ECC_DEV GasSmem<N, BLOCK>& gas_smem() {
  extern __shared__ __align__(16) unsigned char ecc_dyn_smem[];
  return *reinterpret_cast<GasSmem<N, BLOCK>*>(ecc_dyn_smem);
}

template <class F>
ECC_DEV void fe_shfl_xor(uint32_t* r, const uint32_t* a, int mask) {
#pragma unroll
  for (int i = 0; i < F::N; ++i) r[i] = __shfl_xor_sync(0xffffffffu, a[i], mask);
}

// CL > 1: the kernel runs in clusters of CL (2 or 4) CTAs that share one
// inversion per round (every CTA of a cluster must call this the same number
// of times).
template <class F, int BLOCK, int CL = 1>
__device__ void cta_invert(uint32_t* out, const uint32_t* in, GasSmem<F::N, BLOCK>& sm) {
  static_assert(CL == 1 || CL == 2 || CL == 4, "clusters of 1, 2 or 4 CTAs");
  constexpr int N = F::N;
  constexpr int NW = BLOCK / 32;
  const int tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  uint32_t v[N], t[N];
  fe_copy<F>(v, in);
#pragma unroll
  for (int l = 0; l < 5; ++l) {
#pragma unroll
    for (int g = 0; g < N / 4; ++g)
      sm.tree[l][g][tid] = make_uint4(v[4 * g], v[4 * g + 1], v[4 * g + 2], v[4 * g + 3]);
    fe_shfl_xor<F>(t, v, 1 << l);
    mont_mul<F>(v, v, t);
  }
  if (lane == 0) {
#pragma unroll
    for (int i = 0; i < N; ++i) sm.warp_tot[warp][i] = v[i];
  }
  __syncthreads();
  // the same butterfly over the warp totals in warp 0 (lanes >= NW carry 1),
  // so the serial part is log2(NW) products up, one inversion, log2(NW) down
  constexpr int LW = NW <= 1 ? 0 : (NW <= 2 ? 1 : (NW <= 4 ? 2 : (NW <= 8 ? 3 : (NW <= 16 ? 4 : 5))));
  uint32_t w[N], keep[LW > 0 ? LW : 1][N];
  if (warp == 0) {
    if (lane < NW) {
#pragma unroll
      for (int i = 0; i < N; ++i) w[i] = sm.warp_tot[lane][i];
    } else {
      fe_set_one<F>(w);
    }
#pragma unroll
    for (int l = 0; l < LW; ++l) {
      fe_copy<F>(keep[l], w);
      fe_shfl_xor<F>(t, w, 1 << l);
      mont_mul<F>(w, w, t);
    }
  }
  if constexpr (CL > 1) {
    // one inversion for the CL CTAs of a cluster: every other CTA's total goes
    // to the first through distributed shared memory; the first inverts the
    // product (Montgomery's trick over the CL totals) and sends each CTA its
    // own inverse back.  Two cluster barriers, passed by every thread of all
    // CL CTAs.
    namespace cg = cooperative_groups;
    cg::cluster_group cl = cg::this_cluster();
    const unsigned rank = cl.block_rank();
    if (warp == 0 && lane == 0 && rank != 0) {
      uint32_t* dst = cl.map_shared_rank(&sm.pair_in[rank][0], 0);
#pragma unroll
      for (int i = 0; i < N; ++i) dst[i] = w[i];
    }
    cl.sync();
    if (warp == 0 && lane == 0 && rank == 0) {
      // prefix products p_k = t_0 .. t_k of the CL totals, one inversion of
      // p_(CL-1), then walk back: t_k^-1 = acc p_(k-1), acc <- acc t_k
      uint32_t pre[CL][N], acc[N], tk[N];
      fe_copy<F>(pre[0], w);
#pragma unroll
      for (int k = 1; k < CL; ++k) {
#pragma unroll
        for (int i = 0; i < N; ++i) tk[i] = sm.pair_in[k][i];
        mont_mul<F>(pre[k], pre[k - 1], tk);
      }
      fe_inv_mont<F>(acc, pre[CL - 1]);
#pragma unroll
      for (int k = CL - 1; k >= 1; --k) {
        uint32_t mine[N];
        mont_mul<F>(mine, acc, pre[k - 1]);
        uint32_t* dst = cl.map_shared_rank(&sm.pair_out[0], k);
#pragma unroll
        for (int i = 0; i < N; ++i) dst[i] = mine[i];
#pragma unroll
        for (int i = 0; i < N; ++i) tk[i] = sm.pair_in[k][i];
        mont_mul<F>(acc, acc, tk);
      }
      fe_copy<F>(w, acc);
    }
    cl.sync();
    if (warp == 0 && lane == 0 && rank != 0) {
#pragma unroll
      for (int i = 0; i < N; ++i) w[i] = sm.pair_out[i];
    }
  } else {
    if (warp == 0 && lane == 0) fe_inv_mont<F>(w, w);
  }
  if (warp == 0) {
#pragma unroll
    for (int i = 0; i < N; ++i) w[i] = __shfl_sync(0xffffffffu, w[i], 0);
#pragma unroll
    for (int l = LW - 1; l >= 0; --l) {
      fe_shfl_xor<F>(t, keep[l], 1 << l);
      mont_mul<F>(w, w, t);
    }
    if (lane < NW) {
#pragma unroll
      for (int i = 0; i < N; ++i) sm.warp_inv[lane][i] = w[i];
    }
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < N; ++i) v[i] = sm.warp_inv[warp][i];
#pragma unroll
  for (int l = 4; l >= 0; --l) {
    uint32_t s[N];
#pragma unroll
    for (int g = 0; g < N / 4; ++g) {
      const uint4 q = sm.tree[l][g][tid];
      s[4 * g] = q.x;
      s[4 * g + 1] = q.y;
      s[4 * g + 2] = q.z;
      s[4 * g + 3] = q.w;
    }
    fe_shfl_xor<F>(t, s, 1 << l);
    mont_mul<F>(v, v, t);
  }
  fe_copy<F>(out, v);
  __syncthreads();  // shared storage is reused by the next round
}

// --------------------------------------------------------------------------
// One batched round over the items [begin, end) owned by this CTA (Montgomery's
// trick with the DCWPA step, Section 3.3).  R provides
//   OPS                       denominators per item,
//   den_c(i, j, d)            denominator j of item i, loading only what it needs
//                             (compress step: e.g. only x for PADD),
//   den_d(i, j, d)            the same value in the DCWPA step, where R may keep
//                             the loaded operands for finish,
//   finish(i, inv)            complete item i given inv[j] = 1 / den_j.
// Compress stores only the running product before each item in M (the
// intermediate array of Section 3.3); DCWPA recomputes the item's denominators
// and, for OPS > 1, the partial products inside the item (find-then-recompute,
// Section 3.4) instead of storing them.
template <class F, int BLOCK, int CL = 1, class R>
__device__ void batch_round(R& rd, size_t begin, size_t end, const SoA<F>& M,
                            GasSmem<F::N, BLOCK>& sm) {
  constexpr int N = F::N;
  constexpr int OPS = R::OPS;
  uint32_t run[N];
  fe_set_one<F>(run);
  const size_t i0 = begin + threadIdx.x;
  for (size_t i = i0; i < end; i += BLOCK) {
    M.store(i, run);
#pragma unroll
    for (int j = 0; j < OPS; ++j) {
      uint32_t d[N];
      rd.den_c(i, j, d);
      mont_mul<F>(run, run, d);
    }
  }
  uint32_t inv[N];
  cta_invert<F, BLOCK, CL>(inv, run, sm);
  if (i0 < end) {
    const size_t last = i0 + ((end - 1 - i0) / BLOCK) * BLOCK;
    for (size_t i = last + BLOCK; i > i0;) {
      i -= BLOCK;
      uint32_t pre[OPS][N], dd[OPS][N], invs[OPS][N];
      M.load(i, pre[0]);
#pragma unroll
      for (int j = 0; j < OPS; ++j) {
        rd.den_d(i, j, dd[j]);
        if (j + 1 < OPS) mont_mul<F>(pre[j + 1], pre[j], dd[j]);
      }
#pragma unroll
      for (int j = OPS - 1; j >= 0; --j) {
        mont_mul<F>(invs[j], inv, pre[j]);
        mont_mul<F>(inv, inv, dd[j]);
      }
      rd.finish(i, invs);
    }
  }
}

}  // namespace ecc
