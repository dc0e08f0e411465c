// Host side of the Pippenger MSM (included once per curve): planning (window
// width per instance, bucket id ranges), workspace layout and the launch
// sequence.  Every launch is stream-ordered and the call performs no host
// synchronisation, so a whole ragged batch can be captured once in a CUDA graph
// and replayed.
#pragma once
#include <algorithm>
#include <map>
#include <vector>

#include "internal.h"
#include "msm.cuh"
#include "scan.cuh"
#include "upload.cuh"

namespace ecc {

namespace msm_detail {

constexpr int kAccBlock = kGasThreads;
constexpr uint32_t kReduceChunk = 32;

inline int scalar_bits(int curve) {
  switch (curve) {
    case 0: return Secp256k1::SCALAR_BITS;
    case 1: return P256::SCALAR_BITS;
    case 2: return BN254::SCALAR_BITS;
    default: return BLS12_381::SCALAR_BITS;
  }
}

inline int windows_for(int curve, int c) { return (scalar_bits(curve) + 1 + c - 1) / c; }

struct Layout {
  std::vector<MsmInst> inst;
  uint64_t buckets = 0, entries_max = 0, n_chunks = 0, total_points = 0;
};

template <class C>
cudaError_t run_set(int curve, const Layout& L, const uint32_t* bases_mont, const uint32_t* scalars,
                    uint32_t* out, cudaStream_t st) {
  using F = typename C::Fp;
  constexpr int N = F::N;
  const int num = (int)L.inst.size();
  const uint64_t B = L.buckets, NC = std::max<uint64_t>(L.n_chunks, 1);
  const uint64_t n_part = B + NC;
  // ---- workspace
  auto up = [](uint64_t b) { return (b + 255) / 256 * 256; };
  const uint64_t sz_inst = up(num * sizeof(MsmInst));
  const uint64_t sz_b1 = up((B + 1) * 4);
  const uint64_t sz_kv = up(kAccChunk * NC * 4);
  const uint64_t sz_S = soa_bytes<F>(NC), sz_P = soa_bytes<F>(n_part);
  const uint64_t bytes = sz_inst + 5 * sz_b1 + 2 * sz_kv + 3 * sz_S + 2 * sz_P + 256;
  Scratch ws;
  cudaError_t e = ws.alloc(bytes, st);
  if (e != cudaSuccess) return e;
  char* p = ws.as<char>();
  auto take = [&](uint64_t b) { char* r = p; p += b; return r; };
  MsmInst* d_inst = reinterpret_cast<MsmInst*>(take(sz_inst));
  uint32_t* count = reinterpret_cast<uint32_t*>(take(sz_b1));
  uint32_t* off = reinterpret_cast<uint32_t*>(take(sz_b1));
  uint32_t* cursor = reinterpret_cast<uint32_t*>(take(sz_b1));
  uint32_t* npart = reinterpret_cast<uint32_t*>(take(sz_b1));
  uint32_t* poff = reinterpret_cast<uint32_t*>(take(sz_b1));
  uint32_t* keys = reinterpret_cast<uint32_t*>(take(sz_kv));
  uint32_t* vals = reinterpret_cast<uint32_t*>(take(sz_kv));
  uint4* sbuf = reinterpret_cast<uint4*>(take(3 * sz_S));
  uint4* pbuf = reinterpret_cast<uint4*>(take(2 * sz_P));
  e = upload_words(d_inst, L.inst.data(), num * sizeof(MsmInst), st);
  if (e != cudaSuccess) return e;
  // ---- 1-2: digits, counting sort by bucket id
  e = cudaMemsetAsync(count, 0, (B + 1) * 4, st);
  if (e != cudaSuccess) return e;
  const unsigned pb = (unsigned)((L.total_points + 255) / 256);
  if (L.total_points) k_msm_count<C><<<pb, 256, 0, st>>>(d_inst, num, scalars, L.total_points, count);
  e = exclusive_scan(count, B, off, st);
  if (e != cudaSuccess) return e;
  e = cudaMemcpyAsync(cursor, off, B * 4, cudaMemcpyDeviceToDevice, st);
  if (e != cudaSuccess) return e;
  if (B) k_msm_npart<<<(unsigned)((B + 255) / 256), 256, 0, st>>>(off, (uint32_t)B, npart);
  e = exclusive_scan(npart, B, poff, st);
  if (e != cudaSuccess) return e;
  if (L.total_points)
    k_msm_scatter<C><<<pb, 256, 0, st>>>(d_inst, num, scalars, L.total_points, cursor, keys, vals, NC);
  // ---- 3: bucket accumulation (batched affine, one launch)
  AccArgs<C> a;
  a.keys = keys;
  a.vals = vals;
  a.off = off;
  a.poff = poff;
  a.n_buckets = (uint32_t)B;
  a.n_chunks = NC;
  a.bases = bases_mont;
  a.S = PtSoA<F>{SoA<F>{sbuf, NC}, SoA<F>{sbuf + sz_S / 16, NC}};
  a.M = SoA<F>{sbuf + 2 * sz_S / 16, NC};
  a.partial = PtSoA<F>{SoA<F>{pbuf, n_part}, SoA<F>{pbuf + sz_P / 16, n_part}};
  uint64_t ctas = (uint64_t)device_sm_count() * kGasCtasPerSm;
  uint64_t per = (NC + ctas - 1) / ctas;
  if (per < 32) per = 32;
  ctas = (NC + per - 1) / per;
  a.per_cta = per;
  const size_t smem = sizeof(GasSmem<N, kAccBlock>);
  e = cudaFuncSetAttribute(k_msm_accumulate<C, kAccBlock>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_msm_accumulate<C, kAccBlock><<<(unsigned)ctas, kAccBlock, smem, st>>>(a);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // ---- 4-5: per window width: reduction levels, then the window combination
  std::map<uint32_t, std::vector<uint32_t>> groups;
  for (int i = 0; i < num; ++i) groups[L.inst[i].c].push_back((uint32_t)i);
  for (auto& g : groups) {
    const uint32_t c = g.first;
    const std::vector<uint32_t>& ids = g.second;
    const uint32_t W = L.inst[ids[0]].W;
    const uint32_t n_inst = (uint32_t)ids.size();
    Scratch rs;
    // level sizes
    std::vector<uint32_t> elems{1u << (c - 1)};
    while (elems.back() > 1) elems.push_back((elems.back() + kReduceChunk - 1) / kReduceChunk);
    uint64_t jac_elems = 0;
    for (size_t l = 1; l < elems.size(); ++l) jac_elems += 2ull * n_inst * W * elems[l];
    e = rs.alloc(up(n_inst * 4) + jac_elems * sizeof(Jac<F>) + 256, st);
    if (e != cudaSuccess) return e;
    char* q = rs.as<char>();
    uint32_t* d_ids = reinterpret_cast<uint32_t*>(q);
    q += up(n_inst * 4);
    e = upload_words(d_ids, ids.data(), n_inst * 4, st);
    if (e != cudaSuccess) return e;
    const Jac<F>* in_R = nullptr;
    const Jac<F>* in_S = nullptr;
    uint32_t log_span = 0;
    for (size_t l = 1; l < elems.size(); ++l) {
      Jac<F>* oR = reinterpret_cast<Jac<F>*>(q);
      q += (uint64_t)n_inst * W * elems[l] * sizeof(Jac<F>);
      Jac<F>* oS = reinterpret_cast<Jac<F>*>(q);
      q += (uint64_t)n_inst * W * elems[l] * sizeof(Jac<F>);
      ReduceArgs<C> r;
      r.inst = d_inst;
      r.inst_ids = d_ids;
      r.n_inst = n_inst;
      r.W = W;
      r.elems = elems[l - 1];
      r.chunk = kReduceChunk;
      r.log_span = log_span;
      r.poff = poff;
      r.partial = a.partial;
      r.in_R = in_R;
      r.in_S = in_S;
      r.out_R = oR;
      r.out_S = oS;
      const uint64_t threads = (uint64_t)n_inst * W * elems[l];
      k_msm_reduce<C><<<(unsigned)((threads + 63) / 64), 64, 0, st>>>(r, l == 1 ? 1 : 0);
      e = cudaGetLastError();
      if (e != cudaSuccess) return e;
      in_R = oR;
      in_S = oS;
      log_span += 5;  // kReduceChunk = 2^5 elements per chunk
    }
    if (elems.size() == 1) return cudaErrorInvalidValue;  // c >= 2 always gives a level
    k_msm_combine<C><<<(n_inst + 63) / 64, 64, 0, st>>>(d_inst, d_ids, n_inst, W, in_S, out);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

inline Layout plan(int curve, uint32_t num, const uint64_t* sizes, const uint64_t* point_off,
            const uint64_t* scalar_off, const int* cs) {
  Layout L;
  L.inst.resize(num);
  for (uint32_t i = 0; i < num; ++i) {
    MsmInst& m = L.inst[i];
    m.n = (uint32_t)sizes[i];
    m.c = (uint32_t)(cs && cs[i] > 0 ? cs[i] : msm_window(curve, sizes[i]));
    m.W = (uint32_t)windows_for(curve, (int)m.c);
    m.bucket_base = (uint32_t)L.buckets;
    m.point_off = point_off[i];
    m.scalar_off = scalar_off[i];
    L.buckets += (uint64_t)m.W << (m.c - 1);
    L.entries_max += (uint64_t)m.W * m.n;
    L.total_points += m.n;
  }
  L.n_chunks = (L.entries_max + kAccChunk - 1) / kAccChunk;
  return L;
}

template <class C>
cudaError_t msm_points(int curve, uint32_t num, const uint64_t* offsets, const uint32_t* points,
                       const uint32_t* scalars, uint32_t* out, cudaStream_t st) {
  using F = typename C::Fp;
  const uint64_t total = offsets[num] - offsets[0];
  std::vector<uint64_t> sizes(num), poff(num), soff(num);
  for (uint32_t i = 0; i < num; ++i) {
    sizes[i] = offsets[i + 1] - offsets[i];
    poff[i] = offsets[i] - offsets[0];
    soff[i] = poff[i];
  }
  Layout L = plan(curve, num, sizes.data(), poff.data(), soff.data(), nullptr);
  Scratch bases;
  cudaError_t e = bases.alloc(std::max<uint64_t>(total, 1) * 2 * F::N * 4, st);
  if (e != cudaSuccess) return e;
  if (total) {
    k_points_to_mont<C><<<(unsigned)((total + 255) / 256), 256, 0, st>>>(
        points + offsets[0] * 2 * F::N, total, bases.as<uint32_t>());
  }
  return run_set<C>(curve, L, bases.as<uint32_t>(), scalars + offsets[0] * 8, out, st);
}


struct Bases {
  int curve;
  uint64_t n;
  uint32_t* mont;  // AoS Montgomery affine, owned
};

template <class C>
cudaError_t msm_bases_t(Bases* bs, uint32_t num_vectors, const uint64_t* vec_sizes,
                        const uint32_t* scalars, uint32_t* out, cudaStream_t st) {
  // instance v uses bases [0, size_v) and the scalar rows that follow the
  // previous instances' (all n bases each when vec_sizes is null)
  std::vector<uint64_t> sizes(num_vectors, bs->n), poff(num_vectors, 0), soff(num_vectors);
  uint64_t acc = 0;
  for (uint32_t v = 0; v < num_vectors; ++v) {
    if (vec_sizes) sizes[v] = vec_sizes[v];
    soff[v] = acc;
    acc += sizes[v];
  }
  Layout L = plan(bs->curve, num_vectors, sizes.data(), poff.data(), soff.data(), nullptr);
  return run_set<C>(bs->curve, L, bs->mont, scalars, out, st);
}

}  // namespace msm_detail
}  // namespace ecc
