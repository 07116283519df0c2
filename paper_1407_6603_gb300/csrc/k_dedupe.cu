// Duplicate-aware sort, second half: the expansion.  By now every bucket
// that took the duplicate-aware path has its distinct keys sorted in one
// array, each entry the key's W words followed by its count (the number of
// times the word occurs).  Expanding entry u into count copies of its word,
// in array order, gives the bucket's sorted words: phase 3 of the paper's
// method (Section II; Section III step 4) for a bucket with repeats.
//   k_expand_sums   per bucket and slice of 4096 entries: the counts' sum
//   k_expand_bases  per bucket: exclusive prefix over its slices' sums, and
//                   the check that the counts add up to the word count
//   k_expand_fill   per slice: the exclusive prefix pre[u] of every entry,
//                   and the entry holding each output tile's first word
//   k_expand_words  per bucket and output tile: each word's entry (a binary
//                   search of the tile's prefix entries, staged in shared
//                   memory), then its offset, and its letters into a shared
//                   copy of the tile's bytes, which go out as 16-byte stores
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
         (uint64_t)d.stream_off + (uint64_t)d.n * d.L <= caps.stream && (uint64_t)d.out_word + d.n <= caps.offsets &&
         (uint64_t)d.tile0 + (d.n + kExpandTileWords / W - 1) / (kExpandTileWords / W) <= caps.tiles;
}

__device__ __forceinline__ const uint64_t* entries(const ExpandDesc& d, const uint64_t* uA, const uint64_t* uB) {
  return (d.final_buf ? uB : uA) + d.uniq_off;
}

// Entries per slice (one CTA) of the prefix kernels, 16 per thread.
constexpr uint32_t kSlice = 4096, kPerThread = kSlice / kExThreads;
static_assert(kPerThread * kExThreads == kSlice, "a slice is 16 entries per thread");

// Sum of the CTA's per-thread values (a tree in shared memory).
__device__ __forceinline__ uint32_t cta_sum(uint32_t v, uint32_t* s_red) {
  s_red[threadIdx.x] = v;
  __syncthreads();
  for (uint32_t w = kExThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) s_red[threadIdx.x] += s_red[threadIdx.x + w];
    __syncthreads();
  }
  const uint32_t tot = s_red[0];
  __syncthreads();
  return tot;
}

// Exclusive prefix of the CTA's per-thread values in thread order (a
// Hillis-Steele scan in shared memory).
__device__ __forceinline__ uint32_t cta_exclusive(uint32_t v, uint32_t* s_red) {
  s_red[threadIdx.x] = v;
  __syncthreads();
  for (uint32_t d = 1; d < kExThreads; d <<= 1) {
    const uint32_t add = threadIdx.x >= d ? s_red[threadIdx.x - d] : 0u;
    __syncthreads();
    s_red[threadIdx.x] += add;
    __syncthreads();
  }
  const uint32_t inc = s_red[threadIdx.x];
  __syncthreads();
  return inc - v;
}

// The prefix is taken in three steps, bucket blockIdx.y, slice blockIdx.x:
// the slices' sums, each bucket's exclusive prefix over them, then every
// entry's prefix pre[u] (and pre[U] = n) from its slice's base.  The last
// step also records, for each output tile, the entry that holds its first
// word: tile k of a bucket starts at word k T inside the entry u with
// pre[u] <= k T < pre[u + 1].
__global__ void __launch_bounds__(kExThreads) k_expand_sums(const ExpandDesc* __restrict__ ed, uint32_t nb,
                                                            uint32_t slices, const uint64_t* uA, const uint64_t* uB,
                                                            uint32_t* ssum, Meta* meta, ExpandCaps caps) {
  __shared__ uint32_t s_red[kExThreads];
  if (blockIdx.y >= nb) return;
  const ExpandDesc d = ed[blockIdx.y];
  if ((uint64_t)blockIdx.x * kSlice >= d.U) return;
  if (!desc_ok(d, caps)) {
    if (threadIdx.x == 0 && blockIdx.x == 0) check_failed(meta, 0x101);
    return;
  }
  const uint64_t* C = entries(d, uA, uB) + d.Wp / 2;  // the count words
  const uint32_t u0 = blockIdx.x * kSlice + threadIdx.x * kPerThread;
  uint32_t v = 0;
#pragma unroll
  for (uint32_t k = 0; k < kPerThread; ++k)
    if (u0 + k < d.U) v += (uint32_t)C[(uint64_t)(u0 + k) * d.Wp];
  const uint32_t tot = cta_sum(v, s_red);
  if (threadIdx.x == 0) ssum[(size_t)blockIdx.y * slices + blockIdx.x] = tot;
}

// One thread per bucket: the exclusive prefix over its slices' sums, in
// place, and the check that the counts add up to the bucket's words.
__global__ void k_expand_bases(const ExpandDesc* __restrict__ ed, uint32_t nb, uint32_t slices, uint32_t* ssum,
                               Meta* meta, ExpandCaps caps) {
  const uint32_t b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nb) return;
  const ExpandDesc d = ed[b];
  if (!desc_ok(d, caps)) return;  // reported by the sums
  const uint32_t ns = (d.U + kSlice - 1) / kSlice;
  uint32_t run = 0;
  for (uint32_t i = 0; i < ns; ++i) {
    const uint32_t v = ssum[(size_t)b * slices + i];
    ssum[(size_t)b * slices + i] = run;
    run += v;
  }
  if (run != d.n) check_failed(meta, 0x102);
}

__global__ void __launch_bounds__(kExThreads) k_expand_fill(const ExpandDesc* __restrict__ ed, uint32_t nb,
                                                            uint32_t slices, const uint64_t* uA, const uint64_t* uB,
                                                            const uint32_t* ssum, uint32_t* pre, uint32_t* tfirst,
                                                            ExpandCaps caps) {
  __shared__ uint32_t s_red[kExThreads];
  if (blockIdx.y >= nb) return;
  const ExpandDesc d = ed[blockIdx.y];
  if ((uint64_t)blockIdx.x * kSlice >= d.U || !desc_ok(d, caps)) return;
  const uint64_t* C = entries(d, uA, uB) + d.Wp / 2;
  const uint32_t T = expand_tile(d.Wp / 2);
  const uint32_t u0 = blockIdx.x * kSlice + threadIdx.x * kPerThread;
  uint32_t cnt[kPerThread];
  uint32_t v = 0;
#pragma unroll
  for (uint32_t k = 0; k < kPerThread; ++k) {
    cnt[k] = u0 + k < d.U ? (uint32_t)C[(uint64_t)(u0 + k) * d.Wp] : 0u;
    v += cnt[k];
  }
  uint32_t run = ssum[(size_t)blockIdx.y * slices + blockIdx.x] + cta_exclusive(v, s_red);
#pragma unroll
  for (uint32_t k = 0; k < kPerThread; ++k) {
    const uint32_t u = u0 + k;
    if (u < d.U) {
      pre[d.pre_off + u] = run;
      // the tiles whose first word lies in this entry's copies (checked
      // against the bucket's tiles: counts that do not add up stay inside)
      const uint32_t end = min(run + cnt[k], d.n);
      for (uint32_t t = (run + T - 1) / T; t * T < end; ++t) tfirst[d.tile0 + t] = u;
      if (u + 1 == d.U) pre[d.pre_off + d.U] = run + cnt[k];  // the closing entry: n
    }
    run += cnt[k];
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

// Bytes of one output tile's letters, staged in shared memory: T keys of W
// words hold at most (2048 / W) * floor(64 W / 6) <= 21845 letters (six-bit
// and case-folded keys spend 6 bits a letter, bytes 8), plus 15 bytes of
// alignment shift.
constexpr uint32_t kExpandStage = 21888;

// The words of bucket blockIdx.y, one output tile of T = kExpandTileWords / W
// at a time (tiles strided over blockIdx.x): word w0 + j of tile k is a copy
// of entry u(j), the last u with pre[u] <= w0 + j.  The entries from the one
// holding the tile's first word to the one holding the next tile's first
// word (every one between covers a word of the tile: at most T + 1 of them)
// have their prefix staged in shared memory; each thread finds its words'
// entries there, writes their offsets, and writes their letters into a
// shared-memory copy of the tile's stream bytes, shifted by the destination's
// offset within 16 bytes; the tile's bytes then go out as aligned 16-byte
// stores (byte stores only at the two ragged ends).
__global__ void __launch_bounds__(kExThreads) k_expand_words(const ExpandDesc* __restrict__ ed, uint32_t nb,
                                                             const uint64_t* uA, const uint64_t* uB,
                                                             const uint32_t* pre, const uint32_t* tfirst, EmitOut eo,
                                                             Meta* meta, ExpandCaps caps) {
  __shared__ uint32_t s_pre[kExpandTileWords + 1];
  __shared__ __align__(16) uint8_t s_out[kExpandStage];
  if (blockIdx.y >= nb) return;
  const ExpandDesc d = ed[blockIdx.y];
  if (!desc_ok(d, caps)) return;  // reported by the prefix kernels
  const uint32_t W = d.Wp / 2;
  const uint32_t T = expand_tile(W);
  const uint32_t tiles = (d.n + T - 1) / T;
  const uint32_t* pr = pre + d.pre_off;
  const uint64_t* P = entries(d, uA, uB);
  for (uint32_t it = blockIdx.x; it < tiles; it += gridDim.x) {
    const uint32_t w0 = it * T;
    const uint32_t cnt = min(T, d.n - w0);
    const uint32_t ua = tfirst[d.tile0 + it];
    const uint32_t ub = it + 1 < tiles ? tfirst[d.tile0 + it + 1] : d.U - 1;
    if (ub < ua || ub - ua > cnt || ub >= d.U) {
      // counts lost to a timed-out insert (already reported): the tile is
      // left unwritten
      if (threadIdx.x == 0) check_failed(meta, 0x402);
      continue;
    }
    for (uint32_t k = threadIdx.x; k <= ub - ua; k += kExThreads) s_pre[k] = pr[ua + k];
    __syncthreads();
    uint8_t* const dst = eo.stream + d.stream_off + (size_t)w0 * d.L;
    const uint32_t nbytes = cnt * d.L;
    const uint32_t sh = (uint32_t)((uintptr_t)dst & 15u);
    const bool staged = sh + nbytes <= kExpandStage;  // (always, for keys of at most 8 words)
    for (uint32_t j = threadIdx.x; j < cnt; j += kExThreads) {
      const uint32_t w = w0 + j;
      const uint64_t* e = P + (uint64_t)(ua + last_le(s_pre, 0, ub - ua, w)) * d.Wp;
      uint8_t* out = staged ? s_out + sh + j * d.L : dst + (size_t)j * d.L;
      for (uint32_t q = 0; q * 8 < d.L; ++q) {
        const uint64_t a = ascii8(eo.codec, d.L, [&](uint32_t x) { return e[x]; }, q);
        for (uint32_t b = 0; b < 8 && q * 8 + b < d.L; ++b) out[q * 8 + b] = (uint8_t)(a >> (56 - 8 * b));
      }
      if (eo.want_offsets) eo.offsets[d.out_word + w] = d.stream_off - d.doc_stream0 + w * d.L;
    }
    __syncthreads();
    if (staged) {
      // dst + head is 16-byte aligned, and so is s_out + sh + head
      const uint32_t head = min(nbytes, (16u - sh) & 15u);
      const uint32_t chunks = (nbytes - head) >> 4;
      const uint32_t tail0 = head + 16u * chunks;
      for (uint32_t c = threadIdx.x; c < chunks; c += kExThreads)
        *reinterpret_cast<uint4*>(dst + head + 16u * c) = *reinterpret_cast<const uint4*>(s_out + sh + head + 16u * c);
      for (uint32_t k = threadIdx.x; k < head + (nbytes - tail0); k += kExThreads) {
        const uint32_t o = k < head ? k : tail0 + (k - head);
        dst[o] = s_out[sh + o];
      }
      __syncthreads();  // s_out and s_pre are read: the next tile may fill them
    }
  }
}

}  // namespace

size_t expand_slices(uint32_t max_U) { return (max_U + kSlice - 1) / kSlice; }

cudaError_t launch_expand(const ExpandDesc* ed, uint32_t nbuckets, uint32_t max_U, uint32_t max_tiles,
                          const uint64_t* uA, const uint64_t* uB, uint32_t* pre, uint32_t* ssum, uint32_t* tfirst,
                          EmitOut eo, Meta* meta, ExpandCaps caps, cudaStream_t st) {
  if (nbuckets == 0) return cudaSuccess;
  const uint32_t slices = (uint32_t)expand_slices(max_U);
  k_expand_sums<<<dim3(slices, nbuckets), kExThreads, 0, st>>>(ed, nbuckets, slices, uA, uB, ssum, meta, caps);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_expand_bases<<<(nbuckets + 127) / 128, 128, 0, st>>>(ed, nbuckets, slices, ssum, meta, caps);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_expand_fill<<<dim3(slices, nbuckets), kExThreads, 0, st>>>(ed, nbuckets, slices, uA, uB, ssum, pre, tfirst, caps);
  if ((e = cudaGetLastError()) != cudaSuccess || max_tiles == 0) return e;
  const uint32_t gx = max_tiles < 1216u ? max_tiles : 1216u;
  k_expand_words<<<dim3(gx, nbuckets), kExThreads, 0, st>>>(ed, nbuckets, uA, uB, pre, tfirst, eo, meta, caps);
  return cudaGetLastError();
}

}  // namespace bsort
