// Host side of the Pippenger MSM (included once per curve): planning (window
// width per instance, bucket id ranges), workspace layout and the launch
// sequence.  Every launch is stream-ordered and the call performs no host
// synchronisation, so a whole ragged batch can be captured once in a CUDA graph
// and replayed.
#pragma once
#include <algorithm>
#include <map>
#include <tuple>
#include <vector>

#include "internal.h"
#include "msm.cuh"
#include "scan.cuh"
#include "upload.cuh"

namespace ecc {

namespace msm_detail {

constexpr int kAccBlock = kGasThreads;
static_assert(kRedLog1Max == kMsmReduceLogMax, "one bound for the first-level reduction chunk");

inline int scalar_bits(int curve) {
  switch (curve) {
    case 0: return Secp256k1::SCALAR_BITS;
    case 1: return P256::SCALAR_BITS;
    case 2: return BN254::SCALAR_BITS;
    case 4: return SM2::SCALAR_BITS;
    default: return BLS12_381::SCALAR_BITS;
  }
}

inline int windows_for(int curve, int c) { return (scalar_bits(curve) + 1 + c - 1) / c; }

struct Layout {
  std::vector<MsmInst> inst;
  uint64_t buckets = 0, entries_max = 0, n_chunks = 0, total_points = 0;
};

// Instance sizes held in device memory (capture-time capacity): rows are
// sizes[num] (sizes_mode, resident bases) or offsets[num + 1]; every instance
// has the layout of L.inst[0], and L's totals are the capacity.
struct DevRows {
  const uint64_t* rows;
  int sizes_mode;
  uint64_t n_bases;
  uint64_t cap;
};

// raw_points (optional): canonical caller points to convert into the gather
// layout first (rows [0, total) of the batch); otherwise bases_mont is used.
template <class C>
cudaError_t run_set(int curve, const Layout& L, const uint32_t* bases_mont, const uint32_t* scalars,
                    uint32_t* out, cudaStream_t st, const DevRows* dev = nullptr,
                    const uint32_t* raw_points = nullptr) {
  using F = typename C::Fp;
  constexpr int N = F::N;
  const int num = (int)L.inst.size();
  const uint64_t B = L.buckets, NC = std::max<uint64_t>(L.n_chunks, 1);
  const uint64_t n_part = B + NC;
  // ---- workspace
  auto up = [](uint64_t b) { return (b + 255) / 256 * 256; };
  const uint64_t sz_inst = up(num * sizeof(MsmInst));
  const uint64_t sz_b1 = up((B + 1) * 4);
  const uint64_t sz_kv = up(kAccChunk * NC * 4), sz_cur = up(NC * 4);
  const uint64_t sz_S = soa_bytes<F>(NC), sz_P = soa_bytes<F>(n_part);
  const uint64_t sz_ops = up(n_part * 4);
  // per chunk: running sum (x, y) and prefix product
  constexpr uint64_t kChunkArrays = 3;
  const uint64_t sz_hdr = up(sizeof(MsmDevHdr));
  const uint64_t sz_pts = raw_points ? up(std::max<uint64_t>(L.total_points, 1) * 2 * N * 4) : 0;
  const uint64_t bytes = sz_inst + sz_hdr + sz_pts + 5 * sz_b1 + sz_kv + sz_cur + kChunkArrays * sz_S +
                         3 * sz_P + sz_ops + 256;
  Scratch ws;
  cudaError_t e = ws.alloc(bytes, st);
  if (e != cudaSuccess) return e;
  char* p = ws.as<char>();
  auto take = [&](uint64_t b) { char* r = p; p += b; return r; };
  MsmInst* d_inst = reinterpret_cast<MsmInst*>(take(sz_inst));
  MsmDevHdr* hdr = dev ? reinterpret_cast<MsmDevHdr*>(take(sz_hdr)) : nullptr;
  uint32_t* pts_mont = raw_points ? reinterpret_cast<uint32_t*>(take(sz_pts)) : nullptr;
  uint32_t* count = reinterpret_cast<uint32_t*>(take(sz_b1));
  uint32_t* off = reinterpret_cast<uint32_t*>(take(sz_b1));
  uint32_t* cursor = reinterpret_cast<uint32_t*>(take(sz_b1));
  uint32_t* npart = reinterpret_cast<uint32_t*>(take(sz_b1));
  uint32_t* poff = reinterpret_cast<uint32_t*>(take(sz_b1));
  uint32_t* vals = reinterpret_cast<uint32_t*>(take(sz_kv));
  uint32_t* cur = reinterpret_cast<uint32_t*>(take(sz_cur));
  uint4* sbuf = reinterpret_cast<uint4*>(take(kChunkArrays * sz_S));
  uint4* pbuf = reinterpret_cast<uint4*>(take(3 * sz_P));
  uint32_t* fold_ops = reinterpret_cast<uint32_t*>(take(sz_ops));
  if (dev) {
    k_msm_inst_dev<<<1, 1024, 0, st>>>(dev->rows, (uint32_t)num, dev->sizes_mode, dev->n_bases, dev->cap,
                                       L.inst[0], d_inst, hdr, status_word());
    e = cudaGetLastError();
  } else {
    e = upload_words(d_inst, L.inst.data(), num * sizeof(MsmInst), st);
  }
  if (e != cudaSuccess) return e;
  if (raw_points && L.total_points) {
    k_points_to_mont<C><<<(unsigned)((L.total_points + 255) / 256), 256, 0, st>>>(raw_points, L.total_points,
                                                                                 hdr, pts_mont);
    bases_mont = pts_mont;
  }
  phase_mark(0, st);
  // ---- 1-2: digits, counting sort by bucket id
  e = cudaMemsetAsync(count, 0, (B + 1) * 4, st);
  if (e != cudaSuccess) return e;
  const unsigned pb = (unsigned)((L.total_points + 255) / 256);
  if (L.total_points)
    k_msm_count<C><<<pb, 256, 0, st>>>(d_inst, num, scalars, L.total_points, hdr, count);
  e = exclusive_scan(count, B, off, st);
  if (e != cudaSuccess) return e;
  e = cudaMemcpyAsync(cursor, off, B * 4, cudaMemcpyDeviceToDevice, st);
  if (e != cudaSuccess) return e;
  if (B) k_msm_npart<<<(unsigned)((B + 255) / 256), 256, 0, st>>>(off, (uint32_t)B, npart);
  e = exclusive_scan(npart, B, poff, st);
  if (e != cudaSuccess) return e;
  if (L.total_points)
    k_msm_scatter<C><<<pb, 256, 0, st>>>(d_inst, num, scalars, L.total_points, hdr, cursor, vals, NC,
                                          cur);
  phase_mark(1, st);
  // ---- 3: bucket accumulation (batched affine, one launch)
  AccArgs<C> a;
  a.vals = vals;
  a.cur = cur;
  a.off = off;
  a.poff = poff;
  a.n_buckets = (uint32_t)B;
  a.n_chunks = NC;
  a.bases = bases_mont;
  a.S = PtSoA<F>{SoA<F>{sbuf, NC}, SoA<F>{sbuf + sz_S / 16, NC}};
  a.M = SoA<F>{sbuf + 2 * sz_S / 16, NC};
  a.partial = PtSoA<F>{SoA<F>{pbuf, n_part}, SoA<F>{pbuf + sz_P / 16, n_part}};
  // persistent CTAs; each takes an equal share of the chunks the sort filled
  uint64_t ctas = (uint64_t)device_sm_count() * kGasCtasPerSm;
  ctas = std::max<uint64_t>(1, std::min<uint64_t>(ctas, (NC + 31) / 32));
  const size_t smem = sizeof(GasSmem<N, kAccBlock>);
  e = cudaFuncSetAttribute(k_msm_accumulate<C, kAccBlock>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_msm_accumulate<C, kAccBlock><<<(unsigned)ctas, kAccBlock, smem, st>>>(a);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  phase_mark(2, st);
  // ---- fold the partial sums of every bucket into its first slot
  if (B) {
    FoldArgs<C> f;
    f.poff = poff;
    f.n_buckets = (uint32_t)B;
    f.partial = a.partial;
    f.M = SoA<F>{pbuf + 2 * sz_P / 16, n_part};
    f.ops = fold_ops;
    e = cudaFuncSetAttribute(k_msm_fold<C, kAccBlock>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_msm_fold<C, kAccBlock><<<(unsigned)(device_sm_count() * kGasCtasPerSm), kAccBlock, smem, st>>>(f);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  phase_mark(3, st);
  // ---- 4: bucket reduction.  Instances are grouped by window width (same
  // level structure); the items of every level are laid out group-major so a
  // level of all groups is one launch.
  // groups by (window width, bucket rows per instance, first-level chunk)
  std::map<std::tuple<uint32_t, uint32_t, uint32_t>, std::vector<uint32_t>> groups;
  for (int i = 0; i < num; ++i)
    groups[{L.inst[i].c, L.inst[i].Wr, L.inst[i].red_log}].push_back((uint32_t)i);
  std::vector<std::vector<uint32_t>> elems;  // per group: elements per row, by level
  std::vector<uint64_t> rows;
  for (auto& g : groups) {
    std::vector<uint32_t> el{1u << (std::get<0>(g.first) - 1)};
    const uint32_t K = 1u << std::get<2>(g.first);
    el.push_back((el[0] + K - 1) / K);
    while (el.back() > 1) el.push_back((el.back() + kRedChunkN - 1) / kRedChunkN);
    elems.push_back(el);
    rows.push_back((uint64_t)g.second.size() * std::get<1>(g.first));
  }
  const size_t n_groups = elems.size();
  size_t levels = 0;
  for (auto& el : elems) levels = std::max(levels, el.size() - 1);
  // Jacobian arrays: level 1 of every group, then level 2 of every group, ...
  std::vector<std::vector<uint64_t>> lvl_off(levels + 1, std::vector<uint64_t>(n_groups, 0));
  uint64_t jac_total = 0;
  for (size_t l = 1; l <= levels; ++l) {
    for (size_t g = 0; g < n_groups; ++g) {
      lvl_off[l][g] = jac_total;
      if (l < elems[g].size()) jac_total += rows[g] * elems[g][l];
    }
  }
  const uint64_t items = levels == 0 ? 0 : (levels >= 2 ? lvl_off[2][0] : jac_total);
  std::vector<RedRange> ranges;
  std::vector<uint64_t> fin(num, 0);
  {
    size_t g = 0;
    uint64_t t = 0;
    for (auto& grp : groups) {
      const size_t last = elems[g].size() - 1;
      for (size_t ii = 0; ii < grp.second.size(); ++ii) {
        const uint32_t id = grp.second[ii];
        ranges.push_back(RedRange{t, id, elems[g][1]});
        t += (uint64_t)L.inst[id].Wr * elems[g][1];
        fin[id] = lvl_off[last][g] + (uint64_t)ii * L.inst[id].Wr;
      }
      ++g;
    }
  }
  std::vector<std::vector<LevelSeg>> segs(levels + 1);
  std::vector<uint64_t> seg_threads(levels + 1, 0);
  for (size_t l = 2; l <= levels; ++l) {
    for (size_t g = 0; g < n_groups; ++g) {
      if (l >= elems[g].size()) continue;
      segs[l].push_back(LevelSeg{seg_threads[l], rows[g], elems[g][l - 1], elems[g][l],
                                 lvl_off[l - 1][g], lvl_off[l][g]});
      seg_threads[l] += rows[g] * elems[g][l];
    }
  }
  uint64_t seg_words = 0;
  for (size_t l = 2; l <= levels; ++l) seg_words += up(segs[l].size() * sizeof(LevelSeg));
  // combination order: instances grouped by (rows, window width), so a warp's
  // Horner chains have one length
  std::vector<uint32_t> order(num);
  for (int i = 0; i < num; ++i) order[i] = (uint32_t)i;
  std::stable_sort(order.begin(), order.end(), [&](uint32_t x, uint32_t y) {
    return std::make_pair(L.inst[x].Wr, L.inst[x].c) < std::make_pair(L.inst[y].Wr, L.inst[y].c);
  });
  const uint64_t sz_red = up(ranges.size() * sizeof(RedRange)) + up(num * 8ull) + up(num * 4ull) + seg_words +
                          2 * up(jac_total * sizeof(Jac<F>)) + 4 * up(items * 4) +
                          5 * soa_bytes<F>(std::max<uint64_t>(items, 1)) + 256;
  Scratch rs;
  e = rs.alloc(sz_red, st);
  if (e != cudaSuccess) return e;
  char* q = rs.as<char>();
  auto take_r = [&](uint64_t b) { char* r = q; q += up(b); return r; };
  RedRange* d_ranges = reinterpret_cast<RedRange*>(take_r(ranges.size() * sizeof(RedRange)));
  uint64_t* d_fin = reinterpret_cast<uint64_t*>(take_r(num * 8ull));
  uint32_t* d_order = reinterpret_cast<uint32_t*>(take_r(num * 4ull));
  std::vector<LevelSeg*> d_segs(levels + 1, nullptr);
  for (size_t l = 2; l <= levels; ++l) d_segs[l] = reinterpret_cast<LevelSeg*>(take_r(segs[l].size() * sizeof(LevelSeg)));
  Jac<F>* JR = reinterpret_cast<Jac<F>*>(take_r(jac_total * sizeof(Jac<F>)));
  Jac<F>* JS = reinterpret_cast<Jac<F>*>(take_r(jac_total * sizeof(Jac<F>)));
  uint32_t* cur_e = reinterpret_cast<uint32_t*>(take_r(items * 4));
  uint32_t* cur_a = reinterpret_cast<uint32_t*>(take_r(items * 4));
  uint32_t* lo_b = reinterpret_cast<uint32_t*>(take_r(items * 4));
  uint32_t* rlog = reinterpret_cast<uint32_t*>(take_r(items * 4));
  const uint64_t IT = std::max<uint64_t>(items, 1);
  uint4* rbuf = reinterpret_cast<uint4*>(take_r(5 * soa_bytes<F>(IT)));
  e = upload_words(d_ranges, ranges.data(), ranges.size() * sizeof(RedRange), st);
  if (e != cudaSuccess) return e;
  e = upload_words(d_fin, fin.data(), num * 8ull, st);
  if (e != cudaSuccess) return e;
  e = upload_words(d_order, order.data(), num * 4ull, st);
  if (e != cudaSuccess) return e;
  for (size_t l = 2; l <= levels; ++l) {
    e = upload_words(d_segs[l], segs[l].data(), segs[l].size() * sizeof(LevelSeg), st);
    if (e != cudaSuccess) return e;
  }
  if (items) {
    AffRedArgs<C> r;
    r.inst = d_inst;
    r.ranges = d_ranges;
    r.n_ranges = (uint32_t)ranges.size();
    r.items = items;
    r.poff = poff;
    r.partial = a.partial;
    const uint64_t ss = soa_bytes<F>(IT) / 16;
    r.R = PtSoA<F>{SoA<F>{rbuf, IT}, SoA<F>{rbuf + ss, IT}};
    r.S = PtSoA<F>{SoA<F>{rbuf + 2 * ss, IT}, SoA<F>{rbuf + 3 * ss, IT}};
    r.M = SoA<F>{rbuf + 4 * ss, IT};
    r.cur_e = cur_e;
    r.cur_a = cur_a;
    r.lo_b = lo_b;
    r.rlog = rlog;
    r.out_R = JR;
    r.out_S = JS;
    uint64_t rctas = (uint64_t)device_sm_count() * kGasCtasPerSm;
    uint64_t rper = (items + rctas - 1) / rctas;
    if (rper < 32) rper = 32;
    rctas = (items + rper - 1) / rper;
    r.per_cta = rper;
    const size_t rsmem = N == 8 ? red_smem_bytes<N, kAccBlock>() : smem;
    e = cudaFuncSetAttribute(k_msm_reduce_affine<C, kAccBlock>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rsmem);
    if (e != cudaSuccess) return e;
    k_msm_reduce_affine<C, kAccBlock><<<(unsigned)rctas, kAccBlock, rsmem, st>>>(r);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  for (size_t l = 2; l <= levels; ++l) {
    if (!seg_threads[l]) continue;
    k_msm_reduce_level<C><<<(unsigned)((seg_threads[l] + 63) / 64), 64, 0, st>>>(
        d_segs[l], (uint32_t)segs[l].size(), seg_threads[l], JR, JS);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  phase_mark(4, st);
  // ---- 5: window combination, every instance in one launch
  if (num) {
    k_msm_combine<C><<<(num + 31) / 32, 32, 0, st>>>(d_inst, d_fin, d_order, (uint32_t)num, JS, hdr, out);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  phase_mark(5, st);
  return cudaSuccess;
}

// pre_c > 0: the bases hold precomputed window multiples for width pre_c,
// pre_stride points apart.
inline Layout plan(int curve, uint32_t num, const uint64_t* sizes, const uint64_t* point_off,
            const uint64_t* scalar_off, const int* cs, int pre_c = 0, uint64_t pre_stride = 0) {
  Layout L;
  L.inst.resize(num);
  for (uint32_t i = 0; i < num; ++i) {
    MsmInst& m = L.inst[i];
    m.n = (uint32_t)sizes[i];
    m.c = (uint32_t)(pre_c > 0 ? pre_c : cs && cs[i] > 0 ? cs[i] : msm_window(curve, sizes[i]));
    m.W = (uint32_t)windows_for(curve, (int)m.c);
    m.bucket_base = (uint32_t)L.buckets;
    m.point_off = point_off[i];
    m.scalar_off = scalar_off[i];
    m.pre_stride = pre_c > 0 ? pre_stride : 0;
    m.Wr = pre_c > 0 ? 1u : m.W;
    m.red_log = (uint32_t)std::min<int>(msm_reduce_log(curve, sizes[i]), (int)m.c - 1);
    L.buckets += (uint64_t)m.Wr << (m.c - 1);
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
  (void)total;
  return run_set<C>(curve, L, nullptr, scalars + offsets[0] * 8, out, st, nullptr,
                    points + offsets[0] * 2 * F::N);
}

// The uniform per-instance layout of a device-sized batch (window width c, or
// the library's width for bases with window multiples of width pre_c) with the
// capacity totals: cap scalar rows in num instances.
inline Layout plan_uniform(int curve, uint32_t num, int c, uint64_t cap, int pre_c, uint64_t pre_stride) {
  Layout L;
  MsmInst m{};
  m.c = (uint32_t)(pre_c > 0 ? pre_c : c);
  m.W = (uint32_t)windows_for(curve, (int)m.c);
  m.Wr = pre_c > 0 ? 1u : m.W;
  m.pre_stride = pre_c > 0 ? pre_stride : 0;
  const uint64_t mean = num ? std::max<uint64_t>(cap / num, 2) : 2;
  m.red_log = (uint32_t)std::min<int>(msm_reduce_log(curve, mean), (int)m.c - 1);
  L.inst.assign(num, m);
  for (uint32_t i = 0; i < num; ++i) L.inst[i].bucket_base = (uint32_t)(i * ((uint64_t)m.Wr << (m.c - 1)));
  L.buckets = (uint64_t)num * ((uint64_t)m.Wr << (m.c - 1));
  L.entries_max = cap * m.W;
  L.total_points = cap;
  L.n_chunks = (L.entries_max + kAccChunk - 1) / kAccChunk;
  return L;
}

// Ragged MSMs over caller points with device offsets[num + 1] (offsets[0] = 0),
// at most cap rows, one window width c for every instance.
template <class C>
cudaError_t msm_points_dev(int curve, uint32_t num, uint64_t cap, const uint64_t* offsets, int c,
                           const uint32_t* points, const uint32_t* scalars, uint32_t* out, cudaStream_t st) {
  Layout L = plan_uniform(curve, num, c, cap, 0, 0);
  DevRows dev{offsets, 0, 0, cap};
  return run_set<C>(curve, L, nullptr, scalars, out, st, &dev, points);
}


struct Bases {
  int curve;
  uint64_t n;
  uint32_t* mont;          // AoS Montgomery affine, owned
  uint32_t* pre = nullptr; // window multiples (window-major, window 0 = mont copy), owned
  int pre_c = 0;           // window width of pre (0: none)
};

// Fills bs->pre with 2^(c w) P_i for w < W (W windows of width c).
template <class C>
cudaError_t precompute_t(Bases* bs, int c, cudaStream_t st) {
  using F = typename C::Fp;
  constexpr int N = F::N;
  const uint32_t W = (uint32_t)windows_for(bs->curve, c);
  const uint64_t n = bs->n;
  if ((uint64_t)W * n >= (1ull << 31)) return cudaErrorInvalidValue;  // 31-bit point indices
  uint32_t* pre = nullptr;
  cudaError_t e = cudaMalloc(&pre, std::max<uint64_t>(W * n, 1) * 2 * N * 4);
  if (e != cudaSuccess) return e;
  if (n) e = cudaMemcpyAsync(pre, bs->mont, n * 2 * N * 4, cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess && n && W > 1) {
    Scratch m;
    e = m.alloc(soa_bytes<F>(n), st);
    if (e == cudaSuccess) {
      ShiftArgs<C> a;
      a.pre = pre;
      a.n = n;
      a.W = W;
      a.c = (uint32_t)c;
      a.M = SoA<F>{m.as<uint4>(), n};
      uint64_t ctas = (uint64_t)device_sm_count() * kGasCtasPerSm;
      uint64_t per = (n + ctas - 1) / ctas;
      if (per < 32) per = 32;
      ctas = (n + per - 1) / per;
      a.per_cta = per;
      const size_t smem = sizeof(GasSmem<N, kAccBlock>);
      e = cudaFuncSetAttribute(k_bases_shift<C, kAccBlock>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e == cudaSuccess) {
        k_bases_shift<C, kAccBlock><<<(unsigned)ctas, kAccBlock, smem, st>>>(a);
        e = cudaGetLastError();
      }
    }
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // the old table may be in use until here
  if (e != cudaSuccess) {
    cudaFree(pre);
    return e;
  }
  if (bs->pre) cudaFree(bs->pre);
  bs->pre = pre;
  bs->pre_c = c;
  return cudaSuccess;
}

// Ragged MSMs over resident bases with device sizes[num] (scalar rows back to
// back, at most cap in all), one window width for every instance (the table's
// when the handle has window multiples, else c).
template <class C>
cudaError_t msm_bases_dev_t(Bases* bs, uint32_t num, uint64_t cap, const uint64_t* sizes, int c,
                            const uint32_t* scalars, uint32_t* out, cudaStream_t st) {
  Layout L = plan_uniform(bs->curve, num, c, cap, bs->pre ? bs->pre_c : 0, bs->n);
  DevRows dev{sizes, 1, bs->n, cap};
  return run_set<C>(bs->curve, L, bs->pre ? bs->pre : bs->mont, scalars, out, st, &dev);
}

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
  Layout L = plan(bs->curve, num_vectors, sizes.data(), poff.data(), soff.data(), nullptr,
                  bs->pre ? bs->pre_c : 0, bs->n);
  return run_set<C>(bs->curve, L, bs->pre ? bs->pre : bs->mont, scalars, out, st);
}

}  // namespace msm_detail
}  // namespace ecc
