// K4 (tile sort, clusters of 1..8 CTAs) and the shared-memory merge helpers
// that K5 uses too.  The kernels are templates; k_tile_g2.cu, k_tile_g4.cu
// and k_tile_g8.cu instantiate them for 2, 4 and 8 lanes per odd-even
// transposition group, k_sort2.cu the merge kernels.
//
// K4 for keys of up to 8 u64 words (words of up to 64 letters): phase 3 of
// the paper's method, the sort of each length bucket into ASCII order
// (Section II; Section III step 4).
//
// K4 (k_tile_sort2<CL, G, NTH>) sorts "supertiles".  One CTA of 256 threads holds
// a tile of 2048 u64 words (2048 / W keys) in shared memory, staged by a TMA
// bulk copy, and sorts it with the bubble sort's compare-exchange in its
// parallel form, odd-even transposition:
//   1. each thread sorts its 8 / W keys in registers (odd-even transposition);
//   2. groups of G lanes run G rounds of odd-even transposition between lane
//      neighbours, whole sorted runs exchanged through warp shuffles (the
//      merge-split form of the compare-exchange);
//   3. merge path in shared memory takes those runs up to the tile.
// With CL > 1 the launch uses thread-block clusters of CL CTAs: a cluster
// owns CL consecutive tiles of one bucket and merges them into one run of
// CL tiles through distributed shared memory, each CTA producing its own
// tile of every merge level from slices it copies out of its peers' shared
// memory.  Buckets of up to CL tiles leave K4 fully sorted (and emitted);
// larger ones leave it as runs of CL tiles, and K5 merges those.
#pragma once

#include <cooperative_groups.h>

#include "bsort_dev.cuh"
#include "sort_common.cuh"

namespace cg = cooperative_groups;

namespace bsort {
namespace {

// CTAs per SM that K4's register budget aims for (a build-time tuning
// constant).  The lanes per odd-even transposition group, G (the odd-even /
// merge cutoff: runs of G * KPT keys leave the transposition stage, merges
// take them up to the tile), is a template parameter chosen per launch from
// the tune table.
#ifndef BSORT_K4_MIN_CTAS
#define BSORT_K4_MIN_CTAS 4
#endif

template <int W>
__host__ __device__ constexpr int kpt2() {
  return W >= 8 ? 1 : 8 / W;
}
// Keys per thread when NTH threads share a tile of 2048 u64 words (0: the
// tile is too small for them, keys of W words take NTH / 256 x more).
template <int W, int NTH>
__host__ __device__ constexpr int kptn() {
  return (int)(2048u / (uint32_t)(NTH * W));
}

constexpr int kM2Threads = 256;
// CTAs per SM that K5's register budget aims for (a tuning constant).
#ifndef BSORT_K5_MIN_CTAS
#define BSORT_K5_MIN_CTAS 4
#endif

// Shared-memory layout of a tile: one pad word after every 16 u64 words, so
// that threads reading keys KPT*W words apart (their own runs) or at random
// merge positions spread over all banks.  A key of W <= 16 words never
// straddles a pad (W divides 16), so its words stay contiguous.
__device__ __forceinline__ uint32_t padw(uint32_t w) { return w + (w >> 4); }
__host__ __device__ inline uint32_t padded_words(uint32_t w) { return w + (w >> 4); }

template <int W>
__device__ __forceinline__ const uint64_t* pkey(const uint64_t* buf, uint32_t k) {
  return buf + padw(k * W);
}
template <int W>
__device__ __forceinline__ uint64_t* pkey(uint64_t* buf, uint32_t k) {
  return buf + padw(k * W);
}

// Merge path over two runs given by accessors: how many of the first d
// outputs come from A, ties going to A.
template <int W, class FA, class FB>
__device__ __forceinline__ uint32_t mp_split_f(FA keyA, uint32_t la, FB keyB, uint32_t lb, uint32_t d) {
  uint32_t lo = d > lb ? d - lb : 0u, hi = d < la ? d : la;
  while (lo < hi) {
    const uint32_t m = (lo + hi) >> 1;
    if (klt(keyB(d - 1 - m), keyA(m)))
      hi = m;
    else
      lo = m + 1;
  }
  return lo;
}

// Sequential merge of KPT outputs from (a, b) when both runs sit in one
// padded buffer (A's key i at offA + i, B's at offB + i).  The two heads stay
// in registers and each step loads only the successor of the key it takes;
// an exhausted run's head is +inf (all ones, which no key of letters equals),
// so ties and ends need no bounds test in the compare.
template <int W, int KPT>
__device__ __forceinline__ void merge_run_buf(const uint64_t* buf, uint32_t offA, uint32_t la, uint32_t offB,
                                              uint32_t lb, uint32_t a, uint32_t b, Key<W> (&k)[KPT]) {
  Key<W> ha = a < la ? kload<W>(pkey<W>(buf, offA + a)) : kinf<W>();
  Key<W> hb = b < lb ? kload<W>(pkey<W>(buf, offB + b)) : kinf<W>();
#pragma unroll
  for (int s = 0; s < KPT; ++s) {
    const bool take_a = !klt(hb, ha);
    k[s] = ksel(take_a, ha, hb);
    if (s + 1 < KPT) {
      a += take_a ? 1u : 0u;
      b += take_a ? 0u : 1u;
      const bool more = take_a ? a < la : b < lb;
      const uint32_t pos = take_a ? offA + a : offB + b;
      const Key<W> nx = more ? kload<W>(pkey<W>(buf, pos)) : kinf<W>();
      ha = take_a ? nx : ha;
      hb = take_a ? hb : nx;
    }
  }
}

// Sorts the tile staged (unpadded, by TMA) in buf; the sorted tile is left in
// buf in the padded layout.
template <int W, int G, int NTH>
__device__ void cta_sort(uint64_t* buf) {
  constexpr int KPT = kptn<W, NTH>();
  constexpr uint32_t T = NTH * KPT;
  const int t = threadIdx.x;
  Key<W> k[KPT];
  // The tile is unsorted, so any assignment of keys to threads will do:
  // take them striped, which reads consecutive words across the warp.
#pragma unroll
  for (int i = 0; i < KPT; ++i) k[i] = kload<W>(buf + (size_t)(t + i * NTH) * W);
  oets_registers<W, KPT>(k);
  oets_lanes<W, KPT, G>(k);
#pragma unroll 1
  for (uint32_t R = G * KPT; R < T; R <<= 1) {
    // While both runs of every pair lie in one warp's keys (2R <= 32 KPT),
    // only that warp reads them: a warp barrier suffices (but the first
    // store follows the striped load, which read every warp's keys).
    const bool local = 2 * R <= 32u * KPT && R != (uint32_t)G * KPT;
    if (local)
      __syncwarp();
    else
      __syncthreads();
#pragma unroll
    for (int i = 0; i < KPT; ++i) kstore<W>(pkey<W>(buf, t * KPT + i), k[i]);
    if (2 * R <= 32u * KPT)
      __syncwarp();
    else
      __syncthreads();
    const uint32_t pos = t * KPT;
    const uint32_t base = pos & ~(2 * R - 1);
    const uint32_t d = pos - base;
    auto keyA = [&](uint32_t i) { return kload<W>(pkey<W>(buf, base + i)); };
    auto keyB = [&](uint32_t i) { return kload<W>(pkey<W>(buf, base + R + i)); };
    const uint32_t a = mp_split_f<W>(keyA, R, keyB, R, d);
    merge_run_buf<W, KPT>(buf, base, R, base + R, R, a, d - a, k);
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < KPT; ++i) kstore<W>(pkey<W>(buf, t * KPT + i), k[i]);
  __syncthreads();
}

// Merges the CL sorted tiles of a cluster (CTA q holds supertile positions
// [q*T, (q+1)*T) in its buf0, padded layout) into one sorted run, and returns
// the buffer (buf0 or buf2) that holds this CTA's tile of it.  The levels
// alternate between buf0 and buf2, so one cluster barrier per level suffices:
// a level overwrites the buffer its peers read two levels back.  buf1 takes
// the slices this CTA merges.
template <int W, int CL, int NTH>
__device__ uint64_t* cluster_merge(uint64_t* buf0, uint64_t* buf1, uint64_t* buf2, uint32_t r) {
  constexpr int KPT = kptn<W, NTH>();
  constexpr uint32_t T = NTH * KPT;
  cg::cluster_group cluster = cg::this_cluster();
  const int t = threadIdx.x;
  uint64_t* cur = buf0;  // this level's input tile (every CTA uses the same buffer)
  uint64_t* nxt = buf2;
  auto key_at = [&](uint32_t pos) {  // key `pos` of the supertile, in its owner's shared memory
    return kload<W>(cluster.map_shared_rank(pkey<W>(cur, pos % T), pos / T));
  };
  cluster.sync();
#pragma unroll 1
  for (uint32_t R = T; R < CL * T; R <<= 1) {
    const uint32_t pos0 = r * T;
    const uint32_t pb = pos0 & ~(2 * R - 1);
    const uint32_t d0 = pos0 - pb;
    auto keyA = [&](uint32_t i) { return key_at(pb + i); };
    auto keyB = [&](uint32_t i) { return key_at(pb + R + i); };
    // the two cuts of this CTA's output tile, one warp each, side by side
    __shared__ uint32_t s_cut[2];
    const uint32_t wid = threadIdx.x >> 5;
    if (wid < 2) {
      const uint32_t v = warp_split_fn<W>(keyA, R, keyB, R, d0 + wid * T);
      if ((threadIdx.x & 31) == 0) s_cut[wid] = v;
    }
    __syncthreads();
    const uint32_t a0 = s_cut[0], a1 = s_cut[1];
    const uint32_t na = a1 - a0, b0 = d0 - a0, nb = T - na;
    // copy the two slices into buf1 (keys [0, na) from A, [na, T) from B)
    for (uint32_t e = t; e < T * W; e += NTH) {
      const uint32_t kk = e / W, j = e % W;
      const uint32_t src = kk < na ? pb + a0 + kk : pb + R + b0 + (kk - na);
      buf1[padw(e)] = cluster.map_shared_rank(pkey<W>(cur, src % T), src / T)[j];
    }
    __syncthreads();  // the slices are in
    Key<W> k[KPT];
    const uint32_t pos = t * KPT;
    auto sA = [&](uint32_t i) { return kload<W>(pkey<W>(buf1, i)); };
    auto sB = [&](uint32_t i) { return kload<W>(pkey<W>(buf1, na + i)); };
    const uint32_t a = mp_split_f<W>(sA, na, sB, nb, pos);
    merge_run_buf<W, KPT>(buf1, 0, na, na, nb, a, pos - a, k);
#pragma unroll
    for (int i = 0; i < KPT; ++i) kstore<W>(pkey<W>(nxt, pos + i), k[i]);
    cluster.sync();  // this level's output is visible to the next level's readers
    uint64_t* tmp = cur;
    cur = nxt;
    nxt = tmp;
  }
  return cur;
}

template <int W, int CL, int G, int NTH>
__device__ void sort_supertile(const Segment& sg, uint32_t st, uint32_t r, uint64_t* keys, uint64_t* buf0,
                               uint64_t* buf1, uint64_t* buf2, uint64_t* bar, uint32_t& phase, const EmitOut& eo,
                               Meta* meta, uint64_t wait_limit) {
  constexpr int KPT = kptn<W, NTH>();
  constexpr uint32_t T = NTH * KPT;
  constexpr uint32_t TW = T * W;
  const int t = threadIdx.x;
  const uint64_t j0 = (uint64_t)(st - sg.stile0) * CL * T + (uint64_t)r * T;
  const uint64_t left = j0 < sg.n ? sg.n - j0 : 0ull;
  const uint32_t cnt = left < T ? (uint32_t)left : T;
  uint64_t* g = keys + sg.key_off + j0 * W;
  const uint32_t tma_bytes = (cnt * W * 8u) & ~15u;
  if (t == 0) {
    fence_proxy_async();
    mbar_arrive_expect_tx(bar, tma_bytes);
    if (tma_bytes) tma_load_1d(buf0, g, tma_bytes, bar);
  }
  for (uint32_t e = tma_bytes / 8 + t; e < TW; e += NTH)
    buf0[e] = e < cnt * W ? g[e] : ~0ull;  // odd tail word, then +inf padding
  // The copy's wait has a floor of its own (the caller's wait_limit bounds
  // the waits on other CTAs): a copy of at most 16 KiB lands long before it.
  const uint64_t limit = wait_limit > kCopyWaitFloor ? wait_limit : kCopyWaitFloor;
  const bool ok = mbar_wait_bounded(bar, phase, limit);
  phase ^= 1u;
  const bool lost = __syncthreads_or(!ok);
  if (lost) {
    // The copy did not land in time: report it (the call fails) and give it
    // a second bounded wait to drain.  The CTA neither sorts nor writes this
    // supertile, but stays in step with its cluster (no early exit).
    if (t == 0) {
      atomicAdd(&meta->err_timeout, 1u);
      mbar_wait_bounded(bar, phase ^ 1u, limit);
    }
    __syncthreads();
    // a sorted tile of +inf keys stands in for it, so that the cluster's
    // merge-path cuts stay monotone (every access in bounds)
    for (uint32_t e = t; e < padded_words(TW); e += NTH) buf0[e] = ~0ull;
    __syncthreads();
  } else {
    cta_sort<W, G, NTH>(buf0);
  }
  const uint64_t* res = buf0;
  if constexpr (CL > 1) res = cluster_merge<W, CL, NTH>(buf0, buf1, buf2, r);
  if (lost) {
    // nothing of this supertile is written
  } else if (sg.passes == 0 && !(sg.flags & kSegKeysOut)) {  // the bucket is sorted: its words go straight out
    emit_tile<NTH>(sg, (uint32_t)j0, cnt, [&](uint32_t j, uint32_t q) { return res[padw(j * W + q)]; }, eo);
  } else {  // a run of CL tiles for K5 (or, kSegKeysOut, the sorted keys in place)
    for (uint32_t e = t; e < cnt * W; e += NTH) g[e] = res[padw(e)];
  }
  __syncthreads();
}

template <int CL, int G, int NTH>
__global__ void __launch_bounds__(NTH, BSORT_K4_MIN_CTAS * 256 / NTH) k_tile_sort2(const Segment* __restrict__ segs, uint32_t sbeg,
                                                           uint32_t send, uint32_t nst, uint32_t buf_words,
                                                           uint64_t* keys, EmitOut eo, Meta* meta,
                                                           uint64_t wait_limit) {
  extern __shared__ __align__(128) uint64_t sm[];
  uint64_t* buf0 = sm;
  uint64_t* buf1 = sm + buf_words;
  uint64_t* buf2 = sm + 2 * buf_words;
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t s_seg;
  __shared__ uint32_t s_first[kSegCache];
  const int t = threadIdx.x;
  const bool cached = seg_cache_fill<kByStile0>(segs, sbeg, send, s_first);
  uint32_t r = 0;
  if constexpr (CL > 1) r = cg::this_cluster().block_rank();
  const uint32_t cid = blockIdx.x / CL, ncl = gridDim.x / CL;
  if (t == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  uint32_t phase = 0;
  for (uint32_t st = cid; st < nst; st += ncl) {  // uniform across the cluster
    if (t < 32) {
      const uint32_t v = seg_find_warp<kByStile0>(segs, sbeg, send, s_first, cached, st);
      if (t == 0) s_seg = v;
    }
    __syncthreads();
    const Segment sg = segs[s_seg];
    __syncthreads();
    switch (sg.W) {
      case 1: sort_supertile<1, CL, G, NTH>(sg, st, r, keys, buf0, buf1, buf2, &bar, phase, eo, meta, wait_limit); break;
      case 2: sort_supertile<2, CL, G, NTH>(sg, st, r, keys, buf0, buf1, buf2, &bar, phase, eo, meta, wait_limit); break;
      case 4:
        if constexpr (kptn<4, NTH>() >= 1)
          sort_supertile<4, CL, G, NTH>(sg, st, r, keys, buf0, buf1, buf2, &bar, phase, eo, meta, wait_limit);
        break;
      default:  // (launches with 8-word keys use 256 threads)
        if constexpr (kptn<8, NTH>() >= 1)
          sort_supertile<8, CL, G, NTH>(sg, st, r, keys, buf0, buf1, buf2, &bar, phase, eo, meta, wait_limit);
        break;
    }
  }
}

template <int CL, int G, int NTH>
cudaError_t tile_sort2_cl(const Segment* segs, uint32_t sbeg, uint32_t send, uint32_t nst, int max_grid,
                          int max_width, uint64_t* keys, const EmitOut& eo, Meta* meta, uint64_t wait_limit,
                          cudaStream_t st) {
  (void)max_width;
  const uint32_t buf_words = padded_words(2048u);
  const size_t smem = (size_t)(CL > 1 ? 3 : 1) * buf_words * 8;
  static int attr_done[64];
  static int clusters_cached[64];
  cudaError_t e = once_per_device(attr_done, [&] {
    cudaError_t r = cudaFuncSetAttribute(k_tile_sort2<CL, G, NTH>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (r == cudaSuccess)  // shared memory, not L1, limits how many CTAs fit
      r = cudaFuncSetAttribute(k_tile_sort2<CL, G, NTH>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (r == cudaSuccess && CL > 8)  // clusters of 16 are beyond the portable 8
      r = cudaFuncSetAttribute(k_tile_sort2<CL, G, NTH>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    return r;
  });
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.blockDim = dim3(NTH, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = CL;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int dev = 0;
  cudaGetDevice(&dev);
  int clusters = (dev >= 0 && dev < 64) ? clusters_cached[dev] : 0;
  if (clusters <= 0) {
    cfg.gridDim = dim3(CL, 1, 1);
    e = cudaOccupancyMaxActiveClusters(&clusters, k_tile_sort2<CL, G, NTH>, &cfg);
    if (e != cudaSuccess || clusters <= 0) {
      cudaGetLastError();
      clusters = max(1, max_grid / CL);
    }
    if (dev >= 0 && dev < 64) clusters_cached[dev] = clusters;
  }
  const uint32_t ncl = nst < (uint32_t)clusters * 2u ? nst : (uint32_t)clusters * 2u;
  cfg.gridDim = dim3(ncl * CL, 1, 1);
  return cudaLaunchKernelEx(&cfg, k_tile_sort2<CL, G, NTH>, segs, sbeg, send, nst, buf_words, keys, eo, meta, wait_limit);
}

// All cluster sizes and CTA sizes for one lane count G (each K4 translation
// unit instantiates one G).
template <int G, int NTH>
cudaError_t tile_sort2_cls(int cluster, const Segment* segs, uint32_t sbeg, uint32_t send, uint32_t supertiles,
                           int max_grid, int max_width, uint64_t* keys, const EmitOut& eo, Meta* meta,
                           uint64_t wait_limit, cudaStream_t st) {
  switch (cluster) {
    case 1: return tile_sort2_cl<1, G, NTH>(segs, sbeg, send, supertiles, max_grid, max_width, keys, eo, meta, wait_limit, st);
    case 2: return tile_sort2_cl<2, G, NTH>(segs, sbeg, send, supertiles, max_grid, max_width, keys, eo, meta, wait_limit, st);
    case 4: return tile_sort2_cl<4, G, NTH>(segs, sbeg, send, supertiles, max_grid, max_width, keys, eo, meta, wait_limit, st);
    case 8: return tile_sort2_cl<8, G, NTH>(segs, sbeg, send, supertiles, max_grid, max_width, keys, eo, meta, wait_limit, st);
    case 16: return tile_sort2_cl<16, G, NTH>(segs, sbeg, send, supertiles, max_grid, max_width, keys, eo, meta, wait_limit, st);
    default: return cudaErrorInvalidValue;
  }
}

template <int G>
cudaError_t tile_sort2_lanes(int cluster, int threads, const Segment* segs, uint32_t sbeg, uint32_t send,
                             uint32_t supertiles, int max_grid, int max_width, uint64_t* keys, const EmitOut& eo,
                             Meta* meta, uint64_t wait_limit, cudaStream_t st) {
  if (threads == 512 && max_width <= 4)
    return tile_sort2_cls<G, 512>(cluster, segs, sbeg, send, supertiles, max_grid, max_width, keys, eo, meta,
                                  wait_limit, st);
  return tile_sort2_cls<G, 256>(cluster, segs, sbeg, send, supertiles, max_grid, max_width, keys, eo, meta,
                                wait_limit, st);
}

}  // namespace
}  // namespace bsort
