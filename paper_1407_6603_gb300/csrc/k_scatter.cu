// K3 (scatter + pack) and K6 (emit).
//
// K3 is phase 2 of the paper's method (Section II; Section III step 3): each
// word goes to the sub-array of its length.  The paper's chosen layout is a
// 3-D char array, one plane per length (Section III "Approach Second"); here
// each (document, length) bucket is a contiguous array of packed keys, W u64
// words per key, big-endian so that integer order is ASCII order.  A CTA
// takes 2048 words of one document, ranks them per length in shared memory
// and reserves each length's slots with one atomic per length, so the slots
// of a bucket come out in no fixed order (the sort that follows makes the
// result unique anyway).
//
// The sort kernels write each bucket's words as soon as its keys are final
// (emit_tile in bsort_dev.cuh); K3 also writes the per-length counts and each
// document's closing offset, and K6 only emits the buckets of words of 65 or
// more letters, which the narrow-tile kernels sort.
#include "bsort_dev.cuh"
#include "sort_common.cuh"

namespace bsort {
namespace {

constexpr int kWordsPerThread = kWordBlock / kWordThreads;
// Bytes of letters a CTA stages in shared memory (2048 words of up to 16
// letters on average); longer ranges are read from global memory.
constexpr uint32_t kLetterStage = 32768;

__global__ void __launch_bounds__(kWordThreads) k_scatter(
    const uint32_t* __restrict__ starts, const uint8_t* __restrict__ letters, const uint32_t* __restrict__ doc_wbase,
    const uint32_t* __restrict__ doc_lbase, const uint32_t* __restrict__ doc_item0, uint32_t ndocs, uint32_t items,
    const uint32_t* __restrict__ seg_lookup, const Segment* __restrict__ segs, uint32_t* __restrict__ cursor,
    uint64_t* __restrict__ keys, const uint32_t* __restrict__ hist, uint64_t* __restrict__ counts, EmitOut eo) {
  // per-document counts (bin 0 is always 0 in a result) and each document's
  // closing offset; the words themselves are emitted by the sort kernels
  const uint32_t gsz = gridDim.x * blockDim.x;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < ndocs * kHist; i += gsz) {
    const uint32_t d = i / kHist, L = i % kHist;
    counts[i] = L ? hist[i] : 0ull;
    if (L == 0 && eo.want_offsets) eo.offsets[doc_wbase[d + 1] + d] = doc_lbase[d + 1] - doc_lbase[d];
  }
  __shared__ uint32_t cnt[kHist];
  __shared__ uint64_t s_out[kHist];  // word offset in `keys` of the CTA's first slot of each length
  __shared__ uint32_t s_lookup[kHist];
  __shared__ uint32_t s_st[kWordBlock + 1];
  __shared__ __align__(16) uint64_t s_let[kLetterStage / 8 + 2];
  __shared__ uint32_t s_doc;
  const int t = threadIdx.x;
  for (uint32_t it = blockIdx.x; it < items; it += gridDim.x) {
    for (int i = t; i < kHist; i += kWordThreads) cnt[i] = 0;
    if (t < 32) {  // warp 0 finds the item's document
      const uint32_t d0 = ndocs > 1 ? warp_last_le([&](uint32_t i) { return doc_item0[i]; }, ndocs, it) : 0u;
      if (t == 0) s_doc = d0;
    }
    __syncthreads();
    const uint32_t d = s_doc;
    const uint32_t w0 = doc_wbase[d] + (it - doc_item0[d]) * kWordBlock;
    const uint32_t nw = min(w0 + kWordBlock, doc_wbase[d + 1]) - w0;
    // the block's word starts and the document's length -> bucket row
    for (uint32_t i = t; i <= nw; i += kWordThreads) s_st[i] = starts[w0 + i];
    for (int i = t; i < kHist; i += kWordThreads) s_lookup[i] = seg_lookup[(size_t)d * kHist + i];
    __syncthreads();
    // the block's letters, one contiguous range of S, copied in the
    // background (S has 16 bytes of slack past its end) while the words are
    // ranked; a range too long for the stage is read from S directly
    const uint32_t l0 = s_st[0] & ~15u, l1 = (s_st[nw] + 15u) & ~15u;
    const bool staged = l1 - l0 <= kLetterStage;
    if (staged) {
      for (uint32_t i = t; i < (l1 - l0) / 16; i += kWordThreads) cp_async16(s_let + 2 * i, letters + l0 + 16 * i);
      cp_async_commit();
    }
    uint32_t len[kWordsPerThread], rank[kWordsPerThread];
#pragma unroll
    for (int k = 0; k < kWordsPerThread; ++k) {
      const uint32_t i = t + k * kWordThreads;
      uint32_t L = 0;
      if (i < nw) {
        L = s_st[i + 1] - s_st[i];
        if (L > (uint32_t)kMaxLen || s_lookup[L] == kNoSegment) L = 0;
      }
      len[k] = L;
      if (L) rank[k] = atomicAdd(&cnt[L], 1u);
    }
    __syncthreads();
    // one thread per length reserves the CTA's slots in the bucket
    for (int L = t; L < kHist; L += kWordThreads)
      if (cnt[L]) {
        const uint32_t si = s_lookup[L];
        s_out[L] = segs[si].key_off + (uint64_t)atomicAdd(&cursor[si], cnt[L]) * width_of_len(L);
      }
    if (staged) cp_async_wait_all();
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kWordsPerThread; ++k) {
      const uint32_t L = len[k];
      if (L == 0) continue;
      const uint32_t s0 = s_st[t + k * kWordThreads];
      const int W = width_of_len(L);
      uint64_t* out = keys + s_out[L] + (size_t)rank[k] * W;
      // the letters as aligned 8-byte loads, shifted into place, byte-swapped
      // to big-endian and cut at L
      const uint32_t sh = s0 & 7u;
      const uint64_t* src =
          staged ? s_let + ((s0 - l0) >> 3) : reinterpret_cast<const uint64_t*>(letters + (s0 & ~7u));
      uint64_t x0 = src[0];
      for (int q = 0; q < W; ++q) {
        uint64_t v = 0;
        const uint32_t b0 = (uint32_t)q * 8;
        if (b0 < L) {
          const uint64_t x1 = src[q + 1];
          const uint64_t le = sh ? (x0 >> (8 * sh)) | (x1 << (64 - 8 * sh)) : x0;
          x0 = x1;
          v = ((uint64_t)__byte_perm((uint32_t)le, 0, 0x0123) << 32) | __byte_perm((uint32_t)(le >> 32), 0, 0x0123);
          const uint32_t valid = L - b0;
          if (valid < 8) v &= ~0ull << (8 * (8 - valid));
        }
        out[q] = v;
      }
    }
    __syncthreads();
  }
}

// K6: words of the buckets whose keys the narrow-tile kernels sorted (keys of
// 16 and 32 words), from the key buffer they ended in.
__global__ void __launch_bounds__(kSortThreads) k_emit(const Segment* __restrict__ segs, uint32_t sbeg, uint32_t send,
                                                       uint32_t tiles, const uint64_t* __restrict__ keysA,
                                                       const uint64_t* __restrict__ keysB, EmitOut eo) {
  __shared__ uint32_t s_seg;
  __shared__ uint32_t s_first[kSegCache];
  const bool cached = seg_cache_fill<kByEtile0>(segs, sbeg, send, s_first);
  for (uint32_t it = blockIdx.x; it < tiles; it += gridDim.x) {
    if (threadIdx.x < 32) {
      const uint32_t v = seg_find_warp<kByEtile0>(segs, sbeg, send, s_first, cached, it);
      if (threadIdx.x == 0) s_seg = v;
    }
    __syncthreads();
    const Segment sg = segs[s_seg];
    __syncthreads();
    const int W = width_of_len(sg.L);
    const uint32_t T = (uint32_t)tile_of_width(W);
    const uint32_t j0 = (it - sg.etile0) * T;
    const uint32_t cnt = min(T, sg.n - j0);
    const uint64_t* src = (sg.final_buf ? keysB : keysA) + sg.key_off + (size_t)j0 * W;
    emit_tile<kSortThreads>(sg, j0, cnt, [&](uint32_t j, uint32_t q) { return src[(size_t)j * W + q]; }, eo);
  }
}

}  // namespace

cudaError_t launch_scatter(const uint32_t* starts, const uint8_t* letters, const uint32_t* doc_wbase,
                           const uint32_t* doc_lbase, const uint32_t* doc_item0, uint32_t ndocs, uint32_t items,
                           uint32_t grid, const uint32_t* seg_lookup, const Segment* segs, uint32_t* cursor,
                           uint64_t* keys, const uint32_t* hist, uint64_t* counts, EmitOut eo, cudaStream_t st) {
  if (grid == 0) return cudaSuccess;
  k_scatter<<<grid, kWordThreads, 0, st>>>(starts, letters, doc_wbase, doc_lbase, doc_item0, ndocs, items, seg_lookup,
                                           segs, cursor, keys, hist, counts, eo);
  return cudaGetLastError();
}

cudaError_t launch_emit(const Segment* segs, uint32_t sbeg, uint32_t send, uint32_t tiles, uint32_t grid,
                        const uint64_t* keysA, const uint64_t* keysB, EmitOut eo, cudaStream_t st) {
  if (tiles == 0 || grid == 0 || send <= sbeg) return cudaSuccess;
  k_emit<<<grid, kSortThreads, 0, st>>>(segs, sbeg, send, tiles, keysA, keysB, eo);
  return cudaGetLastError();
}

}  // namespace bsort
