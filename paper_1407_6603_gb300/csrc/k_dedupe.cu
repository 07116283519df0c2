// Duplicate-aware sort, second half: the expansion.  By now every bucket
// that took the duplicate-aware path has its distinct keys sorted in one
// array, each entry the key's W words followed by its count (the number of
// times the word occurs).  Expanding entry u into count copies of its word,
// in array order, gives the bucket's sorted words: phase 3 of the paper's
// method (Section II; Section III step 4) for a bucket with repeats.
//   k_expand_prefix  per bucket: the exclusive prefix pre[u] of the counts,
//                    and the check that they add up to the word count
//   k_expand_words   per bucket and output tile: each word's entry (a binary
//                    search of the prefix between the entries of the tile's
//                    first and last words), then its letters and offset
#include "bsort_dev.cuh"
#include "sort_common.cuh"

namespace bsort {
namespace {

constexpr int kExThreads = 256;

// A failed consistency check: counted, and its site kept (the first one).
__device__ __forceinline__ void check_failed(Meta* meta, uint32_t site) {
  atomicAdd(&meta->err_internal, 1u);
  atomicCAS(&meta->err_site, 0u, site);
}

// Whether descriptor d stays inside the buffers: its distinct-key entries,
// its prefix, its words and offsets.
__device__ __forceinline__ bool desc_ok(const ExpandDesc& d, const ExpandCaps& caps) {
  const uint32_t W = d.Wp / 2;
  return (W == 1 || W == 2 || W == 4 || W == 8) && d.U >= 1 && d.U <= d.n &&
         d.uniq_off + (uint64_t)d.U * d.Wp <= caps.u_words && d.pre_off + d.U + 1 <= caps.pre &&
         (uint64_t)d.stream_off + (uint64_t)d.n * d.L <= caps.stream && (uint64_t)d.out_word + d.n <= caps.offsets;
}

__device__ __forceinline__ const uint64_t* entries(const ExpandDesc& d, const uint64_t* uA, const uint64_t* uB) {
  return (d.final_buf ? uB : uA) + d.uniq_off;
}

// Per bucket (one CTA): the exclusive prefix pre[u] of the sorted entries'
// counts, and pre[U] = n.  Thread t takes one contiguous slice of entries:
// it sums the slice, thread 0 turns the 256 sums into slice bases in shared
// memory, then each thread writes its slice's prefixes.
__global__ void __launch_bounds__(kExThreads) k_expand_prefix(const ExpandDesc* __restrict__ ed, uint32_t nb,
                                                              const uint64_t* uA, const uint64_t* uB, uint32_t* pre,
                                                              Meta* meta, ExpandCaps caps) {
  __shared__ uint32_t s_base[kExThreads];
  if (blockIdx.x >= nb) return;
  const ExpandDesc d = ed[blockIdx.x];
  if (!desc_ok(d, caps)) {
    if (threadIdx.x == 0) check_failed(meta, 0x101);
    return;
  }
  const uint64_t* P = entries(d, uA, uB);
  const uint32_t W = d.Wp / 2;
  const uint32_t per = (d.U + kExThreads - 1) / kExThreads;
  const uint32_t u0 = min(d.U, threadIdx.x * per), u1 = min(d.U, u0 + per);
  uint32_t sum = 0;
  for (uint32_t u = u0; u < u1; ++u) sum += (uint32_t)P[(uint64_t)u * d.Wp + W];
  s_base[threadIdx.x] = sum;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t run = 0;
    for (int i = 0; i < kExThreads; ++i) {
      const uint32_t v = s_base[i];
      s_base[i] = run;
      run += v;
    }
    pre[d.pre_off + d.U] = run;  // the closing entry: n
    if (run != d.n) check_failed(meta, 0x102);
  }
  __syncthreads();
  uint32_t run = s_base[threadIdx.x];
  for (uint32_t u = u0; u < u1; ++u) {
    pre[d.pre_off + u] = run;
    run += (uint32_t)P[(uint64_t)u * d.Wp + W];
  }
}

// Index of the last entry u in [lo, hi] with pre[u] <= x (pre rises, pre[lo] <= x).
__device__ __forceinline__ uint32_t last_le(const uint32_t* pr, uint32_t lo, uint32_t hi, uint32_t x) {
  while (lo < hi) {
    const uint32_t mid = lo + ((hi - lo + 1) >> 1);
    if (pr[mid] <= x)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

// The words of bucket blockIdx.y, kExpandTileWords / W at a time (tiles
// strided over blockIdx.x): word w0 + j of a tile is a copy of entry u(j),
// the last u with pre[u] <= w0 + j.  Thread 0 finds the entries of the
// tile's first and last words; every entry between them covers at least one
// word of the tile, so each thread finds its words' entries by a search over
// at most cnt of them, then writes each word's letters (big-endian in the
// key words) and its offset.
__global__ void __launch_bounds__(kExThreads) k_expand_words(const ExpandDesc* __restrict__ ed, uint32_t nb,
                                                             const uint64_t* uA, const uint64_t* uB,
                                                             const uint32_t* pre, EmitOut eo, Meta* meta,
                                                             ExpandCaps caps) {
  __shared__ uint32_t s_ua, s_ub;
  if (blockIdx.y >= nb) return;
  const ExpandDesc d = ed[blockIdx.y];
  if (!desc_ok(d, caps)) {
    if (threadIdx.x == 0 && blockIdx.x == 0) check_failed(meta, 0x401);
    return;
  }
  const uint32_t W = d.Wp / 2;
  const uint32_t T = expand_tile(W);
  const uint32_t tiles = (d.n + T - 1) / T;
  const uint32_t* pr = pre + d.pre_off;
  const uint64_t* P = entries(d, uA, uB);
  for (uint32_t it = blockIdx.x; it < tiles; it += gridDim.x) {
    const uint32_t w0 = it * T;
    const uint32_t cnt = min(T, d.n - w0);
    if (threadIdx.x == 0) {
      s_ua = last_le(pr, 0, d.U - 1, w0);
      s_ub = last_le(pr, 0, d.U - 1, w0 + cnt - 1);
    }
    __syncthreads();
    const uint32_t ua = s_ua, ub = s_ub;
    __syncthreads();  // read: the next tile may set them
    if (ub < ua || ub - ua >= cnt) {
      // counts lost to a timed-out insert (already reported): the tile is
      // left unwritten
      if (threadIdx.x == 0) check_failed(meta, 0x402);
      continue;
    }
    for (uint32_t j = threadIdx.x; j < cnt; j += kExThreads) {
      const uint32_t w = w0 + j;
      const uint64_t* e = P + (uint64_t)last_le(pr, ua, ub, w) * d.Wp;
      uint8_t* out = eo.stream + d.stream_off + (size_t)w * d.L;
      for (uint32_t i = 0; i < d.L; ++i) out[i] = (uint8_t)(e[i >> 3] >> (56 - 8 * (i & 7)));
      if (eo.want_offsets) eo.offsets[d.out_word + w] = d.stream_off - d.doc_stream0 + w * d.L;
    }
  }
}

}  // namespace

cudaError_t launch_expand(const ExpandDesc* ed, uint32_t nbuckets, uint32_t max_tiles, const uint64_t* uA,
                          const uint64_t* uB, uint32_t* pre, EmitOut eo, Meta* meta, ExpandCaps caps, cudaStream_t st) {
  if (nbuckets == 0) return cudaSuccess;
  k_expand_prefix<<<nbuckets, kExThreads, 0, st>>>(ed, nbuckets, uA, uB, pre, meta, caps);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || max_tiles == 0) return e;
  const uint32_t gx = max_tiles < 1216u ? max_tiles : 1216u;
  k_expand_words<<<dim3(gx, nbuckets), kExThreads, 0, st>>>(ed, nbuckets, uA, uB, pre, eo, meta, caps);
  return cudaGetLastError();
}

}  // namespace bsort
