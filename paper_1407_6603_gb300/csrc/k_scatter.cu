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
// result unique anyway).  It then packs the words in (length, rank) order,
// so that neighbouring lanes write neighbouring slots of one bucket.
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
// Bytes of letters a CTA stages in shared memory (2048 words of up to 14
// letters on average); longer ranges are read from global memory.  With it a
// CTA holds about 45 KB of shared memory, so five fit on an SM.
constexpr uint32_t kLetterStage = 28672;

// Packs one word into its byte key (kCodeBytes).  Key word q of a word that starts at S offset
// s0 holds its letters 8q..8q+7, first letter in the most significant byte.
// With the letters read as aligned 32-bit words u[] (u[0] at S offset
// `base`), bytes p..p+3 (p = s0 + 8q) lie in u[k], u[k+1] for
// k = (p - base) / 4, and one byte_perm takes them from there already
// reversed (selector nibbles s+3, s+2, s+1, s for s = p % 4).  Bytes past
// the word's last letter are cleared; key words past it are zero.  Reads
// reach at most 11 bytes past the word's last letter.
__device__ __forceinline__ void pack_word(const uint32_t* __restrict__ u, uint32_t base, uint32_t s0, uint32_t L,
                                          uint64_t* __restrict__ out) {
  const uint32_t sel = 0x0123u + (s0 & 3u) * 0x1111u;
  const uint32_t* src = u + ((s0 - base) >> 2);
  uint32_t a = src[0];
  if (L <= 8) {  // one key word: most words; in (length, rank) order a warp's words mostly share L
    const uint32_t b = src[1], c = src[2];
    const uint32_t hi = __byte_perm(a, b, sel) & (~0u << (8 * (4 - min(L, 4u))));
    const uint32_t lo = L > 4 ? __byte_perm(b, c, sel) & (~0u << (8 * (8 - L))) : 0u;
    out[0] = ((uint64_t)hi << 32) | lo;
    return;
  }
  const int W = width_of_len(L);
  for (int q = 0; q < W; ++q) {
    uint64_t v = 0;
    const uint32_t b0 = (uint32_t)q * 8;
    if (b0 < L) {
      const uint32_t b = src[2 * q + 1], c = src[2 * q + 2];
      uint32_t hi = __byte_perm(a, b, sel), lo = __byte_perm(b, c, sel);
      a = c;
      const uint32_t valid = L - b0;
      if (valid < 8) {
        hi &= ~0u << (8 * (4 - min(valid, 4u)));
        lo = valid > 4 ? lo & (~0u << (8 * (8 - valid))) : 0u;
      }
      v = ((uint64_t)hi << 32) | lo;
    }
    out[q] = v;
  }
}

// Packs one word into its key with a letter code (kCodeSix, kCodeFold; see
// bsort_dev.cuh): the codes from the key's most significant bit down, then
// zeros to W words.  Letter i is the byte at S offset s0 + i of the letters
// read as 32-bit words u[] (u[0] at S offset `base`, a multiple of 4).
__device__ __forceinline__ void pack_codes(uint32_t codec, const uint32_t* __restrict__ u, uint32_t base, uint32_t s0,
                                           uint32_t L, uint32_t W, uint64_t* __restrict__ out) {
  uint64_t acc = 0;  // bits not yet written, from the top
  uint32_t nacc = 0, q = 0;
  auto put = [&](uint32_t v, uint32_t nb) {  // appends the nb low bits of v
    if (nacc + nb <= 64) {
      acc |= (uint64_t)v << (64 - nacc - nb);
      nacc += nb;
      if (nacc == 64) {
        out[q++] = acc;
        acc = 0;
        nacc = 0;
      }
    } else {
      const uint32_t first = 64 - nacc;
      out[q++] = acc | ((uint64_t)v >> (nb - first));
      nacc = nb - first;
      acc = (uint64_t)v << (64 - nacc);
    }
  };
  auto letter = [&](uint32_t i) {
    const uint32_t x = s0 + i - base;
    return (u[x >> 2] >> (8 * (x & 3))) & 0xFFu;
  };
  for (uint32_t i = 0; i < L; ++i) {
    const uint32_t c = letter(i);
    if (codec == kCodeSix)
      put(c <= 'Z' ? c - ('A' - 1) : c - ('a' - 27), 6);
    else
      put((c | 0x20u) - ('a' - 1), 5);
  }
  if (codec == kCodeFold)
    for (uint32_t i = 0; i < L; ++i) put((letter(i) >> 5) & 1u, 1);
  if (nacc) out[q++] = acc;
  while (q < W) out[q++] = 0;
}

// A word's key of W words with the given encoding.
__device__ __forceinline__ void pack_key(uint32_t codec, const uint32_t* __restrict__ u, uint32_t base, uint32_t s0,
                                         uint32_t L, uint32_t W, uint64_t* __restrict__ out) {
  if (codec != kCodeBytes) {
    pack_codes(codec, u, base, s0, L, W, out);
    return;
  }
  pack_word(u, base, s0, L, out);
  for (uint32_t q = (uint32_t)width_of_len(L); q < W; ++q) out[q] = 0;  // a wider key (the whole-text order)
}

__global__ void __launch_bounds__(kWordThreads, 5) k_scatter(
    const uint32_t* __restrict__ starts, const uint8_t* __restrict__ letters, const uint32_t* __restrict__ doc_wbase,
    const uint32_t* __restrict__ doc_lbase, const uint32_t* __restrict__ doc_item0, uint32_t ndocs, uint32_t items,
    const uint32_t* __restrict__ seg_lookup, const Segment* __restrict__ segs, uint32_t* __restrict__ cursor,
    uint64_t* __restrict__ keys, const uint32_t* __restrict__ hist, uint64_t* __restrict__ counts, EmitOut eo,
    uint32_t codec) {
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
  __shared__ uint8_t s_w[kHist];  // key width of each length's bucket
  __shared__ uint32_t s_st[kWordBlock + 1];
  __shared__ uint16_t s_idx[kWordBlock];  // the item's words (index in the item) by (length, rank)
  __shared__ uint32_t s_wtot[kWordThreads / 32];
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
    for (int i = t; i < kHist; i += kWordThreads) {
      const uint32_t si = seg_lookup[(size_t)d * kHist + i];
      s_lookup[i] = si;
      s_w[i] = si == kNoSegment ? 0 : (uint8_t)segs[si].W;
    }
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
    // thread t owns length t: it reserves the CTA's slots in the bucket of
    // that length and takes part in the exclusive prefix over lengths of the
    // CTA's counts, which orders the CTA's words by (length, rank)
    static_assert(kHist == kWordThreads, "one length per thread");
    const uint32_t c = cnt[t];
    if (c) {
      const uint32_t si = s_lookup[t];
      s_out[t] = segs[si].key_off + (uint64_t)atomicAdd(&cursor[si], c) * s_w[t];
    }
    uint32_t inc = c;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const uint32_t v = __shfl_up_sync(0xFFFFFFFFu, inc, off);
      if ((t & 31) >= off) inc += v;
    }
    if ((t & 31) == 31) s_wtot[t >> 5] = inc;
    __syncthreads();
    uint32_t before = 0, nv = 0;
#pragma unroll
    for (int w = 0; w < kWordThreads / 32; ++w) {
      const uint32_t x = s_wtot[w];
      before += w < (t >> 5) ? x : 0u;
      nv += x;
    }
    cnt[t] = before + inc - c;  // now: the CTA's words of shorter lengths
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kWordsPerThread; ++k)
      if (len[k]) s_idx[cnt[len[k]] + rank[k]] = (uint16_t)(t + k * kWordThreads);
    if (staged) cp_async_wait_all();
    __syncthreads();
    // the keys in (length, rank) order: neighbouring lanes write neighbouring
    // slots of one bucket, and mostly keys of one width
    auto pack_sorted = [&](const uint32_t* u, uint32_t base) {
      for (uint32_t j = t; j < nv; j += kWordThreads) {
        const uint32_t i = s_idx[j];
        const uint32_t s0 = s_st[i], L = s_st[i + 1] - s0;
        pack_key(codec, u, base, s0, L, s_w[L], keys + s_out[L] + (size_t)(j - cnt[L]) * s_w[L]);
      }
    };
    if (staged)
      pack_sorted(reinterpret_cast<const uint32_t*>(s_let), l0);
    else
      pack_sorted(reinterpret_cast<const uint32_t*>(letters), 0u);
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
    if (sg.flags & kSegKeysOut) continue;  // sorted keys wanted, not words
    const int W = sg.W;
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
                           uint64_t* keys, const uint32_t* hist, uint64_t* counts, EmitOut eo, bool pack,
                           cudaStream_t st) {
  if (grid == 0) return cudaSuccess;
  k_scatter<<<grid, kWordThreads, 0, st>>>(starts, letters, doc_wbase, doc_lbase, doc_item0, ndocs, pack ? items : 0u,
                                           seg_lookup, segs, cursor, keys, hist, counts, eo, eo.codec);
  return cudaGetLastError();
}

cudaError_t launch_emit(const Segment* segs, uint32_t sbeg, uint32_t send, uint32_t tiles, uint32_t grid,
                        const uint64_t* keysA, const uint64_t* keysB, EmitOut eo, cudaStream_t st) {
  if (tiles == 0 || grid == 0 || send <= sbeg) return cudaSuccess;
  k_emit<<<grid, kSortThreads, 0, st>>>(segs, sbeg, send, tiles, keysA, keysB, eo);
  return cudaGetLastError();
}

}  // namespace bsort
