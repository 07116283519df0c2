// K1 (strip + tokenize) and K2 (length histogram).
//
// Phase 1 of the paper's pre-processing (Section II; Section III step 2):
// every byte that is not an ASCII letter is removed, whitespace separates
// words, and words left without letters vanish.  K1 turns the input into
//   S      : the letters of the text back to back (the "stripped" stream), and
//   starts : for word w, the offset in S of its first letter.
// A letter starts a word when the closest preceding letter-or-whitespace byte
// is whitespace (or there is none in the document); other bytes are
// transparent.  Word w then spans S[starts[w] .. starts[w+1]).
//
// Phase 2 (bucketing by length) needs the per-length counts first: K2 builds
// one 256-bin histogram per document from the word lengths.
//
// Each K1 thread owns 64 consecutive bytes.  It classifies them four at a
// time with byte-SIMD compares into two 64-bit masks (letters, whitespace),
// and finds the word starts among its letters with one addition: adding
// (whitespace << 1) to the mask of transparent bytes carries each whitespace
// bit across the transparent run after it and stops on the next letter or
// whitespace byte, so ((T + (Ws << 1)) ^ T) & Letters marks exactly the
// letters whose previous event is whitespace.
#include "bsort_dev.cuh"
#include "tok_common.cuh"

namespace bsort {
namespace {

__device__ __forceinline__ uint32_t find_doc_of_chunk(const DocDesc* docs, uint32_t ndocs, uint32_t c) {
  // last document whose chunk0 <= c among documents that have chunks
  uint32_t lo = 0, hi = ndocs - 1;
  while (lo < hi) {
    const uint32_t mid = (lo + hi + 1) >> 1;
    if (docs[mid].chunk0 <= c)
      lo = mid;
    else
      hi = mid - 1;
  }
  // documents without chunks share chunk0 with the next one; step past them
  while (lo + 1 < ndocs && (docs[lo].nchunks == 0 || c >= docs[lo].chunk0 + docs[lo].nchunks)) ++lo;
  return lo;
}

// Loads this CTA's chunk into shared memory with 16-byte vector loads; bytes
// outside the document read as spaces.  Granules are 16-byte aligned and each
// one read holds at least one byte of the document, so no load leaves the
// caller's allocation.  Returns whether the chunk is its document's first.
__device__ bool load_chunk(const uint8_t* in, const DocDesc* docs, uint32_t ndocs, uint32_t c, uint4* buf) {
  __shared__ uint32_t s_doc;
  if (threadIdx.x == 0) s_doc = ndocs == 1 ? 0u : find_doc_of_chunk(docs, ndocs, c);
  __syncthreads();
  const DocDesc d = docs[s_doc];
  const uintptr_t first = reinterpret_cast<uintptr_t>(in) + d.byte_off;
  const uintptr_t last = first + d.len;  // exclusive
  const uintptr_t base = (first & ~uintptr_t(15)) + uintptr_t(c - d.chunk0) * kChunk;
#pragma unroll
  for (int i = 0; i < kChunk / 16 / kTokThreads; ++i) {
    const int g = threadIdx.x + i * kTokThreads;
    const uintptr_t a = base + uintptr_t(g) * 16;
    uint4 v = make_uint4(0x20202020u, 0x20202020u, 0x20202020u, 0x20202020u);
    if (a + 16 > first && a < last) {
      v = __ldg(reinterpret_cast<const uint4*>(a));
      if (a < first || a + 16 > last) {
        uint32_t* w = reinterpret_cast<uint32_t*>(&v);
#pragma unroll
        for (int b = 0; b < 16; ++b) {
          const uintptr_t p = a + b;
          if (p < first || p >= last) w[b >> 2] = (w[b >> 2] & ~(0xFFu << (8 * (b & 3)))) | (0x20u << (8 * (b & 3)));
        }
      }
    }
    buf[g] = v;
  }
  const bool doc_first = c == d.chunk0;
  __syncthreads();
  return doc_first;
}

// K1a: one summary per chunk.
__global__ void __launch_bounds__(kTokThreads) k_tok_summary(const uint8_t* __restrict__ in,
                                                             const DocDesc* __restrict__ docs, uint32_t ndocs,
                                                             TokSum* __restrict__ sums) {
  __shared__ uint4 buf[kChunk / 16];
  const uint32_t c = blockIdx.x;
  const bool doc_first = load_chunk(in, docs, ndocs, c, buf);
  uint32_t w[16];
  thread_words(buf, w);
  uint64_t lm, sm;
  classify64(w, lm, sm);
  const TokSum mine = seg_summary(lm, sm, doc_first && threadIdx.x == 0);
  TokSum total;
  block_exclusive(mine, &total);
  if (threadIdx.x == 0) sums[c] = total;
}

// K1b: one CTA of 1024 threads scans the chunk summaries (8 per thread per
// round) and derives the per-document bases.
constexpr int kScanThreads = 1024;
constexpr int kScanPer = 8;

__device__ TokSum block_exclusive_1024(const TokSum v, TokSum* total) {
  __shared__ TokSum warp_tot[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const TokSum inc = warp_inclusive(v);
  if (lane == 31) warp_tot[warp] = inc;
  __syncthreads();
  if (warp == 0) warp_tot[lane] = warp_inclusive(warp_tot[lane]);
  __syncthreads();
  TokSum ex = shfl_up_sum(inc, 1);
  if (lane == 0) ex = TokSum{0, 0, 0};
  if (warp > 0) ex = tok_combine(warp_tot[warp - 1], ex);
  *total = warp_tot[31];
  __syncthreads();
  return ex;
}

__global__ void __launch_bounds__(kScanThreads) k_tok_scan(const TokSum* __restrict__ sums, uint32_t nchunks,
                                                           const DocDesc* __restrict__ docs, uint32_t ndocs,
                                                           TokSum* __restrict__ carry, uint32_t* doc_wbase,
                                                           uint32_t* doc_lbase, uint32_t* doc_item0,
                                                           uint32_t* starts, Meta* meta) {
  TokSum run = {0, 0, 0};
  for (uint32_t base = 0; base < nchunks; base += kScanThreads * kScanPer) {
    TokSum loc[kScanPer];
    TokSum acc = {0, 0, 0};
#pragma unroll
    for (int i = 0; i < kScanPer; ++i) {
      const uint32_t c = base + threadIdx.x * kScanPer + i;
      loc[i] = c < nchunks ? sums[c] : TokSum{0, 0, 0};
      acc = tok_combine(acc, loc[i]);
    }
    TokSum total;
    TokSum ex = tok_combine(run, block_exclusive_1024(acc, &total));
#pragma unroll
    for (int i = 0; i < kScanPer; ++i) {
      const uint32_t c = base + threadIdx.x * kScanPer + i;
      if (c < nchunks) carry[c] = ex;
      ex = tok_combine(ex, loc[i]);
    }
    run = tok_combine(run, total);
  }
  if (threadIdx.x == 0) {
    carry[nchunks] = run;
    starts[run.words] = run.letters;  // sentinel: the last word ends at the end of S
    meta->n_total = run.words;
    meta->s_total = run.letters;
  }
  __syncthreads();
  // Per-document bases, and the prefix of 1024-word blocks over documents.
  __shared__ uint32_t s_run;
  if (threadIdx.x == 0) s_run = 0;
  __syncthreads();
  for (uint32_t base = 0; base < ndocs; base += kScanThreads) {
    const uint32_t d = base + threadIdx.x;
    uint32_t items = 0, wb = 0, lb = 0, we = 0;
    if (d < ndocs) {
      const uint32_t c0 = docs[d].chunk0;
      const uint32_t c1 = c0 + docs[d].nchunks;
      wb = carry[c0].words;
      lb = carry[c0].letters;
      we = carry[c1].words;
      items = (we - wb + kWordBlock - 1) / kWordBlock;
    }
    // block exclusive scan of `items` (plain integers)
    __shared__ uint32_t warp_sum[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t inc = items;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const uint32_t u = __shfl_up_sync(kFull, inc, off);
      if (lane >= off) inc += u;
    }
    if (lane == 31) warp_sum[warp] = inc;
    __syncthreads();
    if (warp == 0) {
      uint32_t s = warp_sum[lane];
#pragma unroll
      for (int off = 1; off < 32; off <<= 1) {
        const uint32_t u = __shfl_up_sync(kFull, s, off);
        if (lane >= off) s += u;
      }
      warp_sum[lane] = s;
    }
    __syncthreads();
    const uint32_t ex = inc - items + (warp > 0 ? warp_sum[warp - 1] : 0u) + s_run;
    if (d < ndocs) {
      doc_wbase[d] = wb;
      doc_lbase[d] = lb;
      doc_item0[d] = ex;
    }
    __syncthreads();
    if (threadIdx.x == 0) s_run += warp_sum[31];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    doc_wbase[ndocs] = run.words;
    doc_lbase[ndocs] = run.letters;
    doc_item0[ndocs] = s_run;
    meta->items_total = s_run;
  }
}

// K1c: writes S and starts.  Letters are compacted into shared memory (in the
// space the input occupied, once every thread holds its input in registers)
// and leave as one contiguous run per CTA.
__global__ void __launch_bounds__(kTokThreads) k_tok_write(const uint8_t* __restrict__ in,
                                                           const DocDesc* __restrict__ docs, uint32_t ndocs,
                                                           const TokSum* __restrict__ carry,
                                                           uint8_t* __restrict__ letters_out,
                                                           uint32_t* __restrict__ starts) {
  __shared__ uint4 buf[kChunk / 16];
  const uint32_t c = blockIdx.x;
  const bool doc_first = load_chunk(in, docs, ndocs, c, buf);
  uint32_t w[16];
  thread_words(buf, w);
  uint64_t lm, sm;
  classify64(w, lm, sm);
  const bool my_doc_start = doc_first && threadIdx.x == 0;
  const TokSum mine = seg_summary(lm, sm, my_doc_start);
  TokSum total;
  const TokSum ex = block_exclusive(mine, &total);  // ends with __syncthreads: buf is free
  const TokSum cin = carry[c];
  const TokSum pre = tok_combine(cin, ex);
  // same rule as tok_combine: an undecided first letter starts a word only
  // after an event that is whitespace
  const bool ws_before = my_doc_start || ((pre.flags & kEv) && (pre.flags & kWs));
  uint64_t starts_m = start_mask(lm, sm, ws_before);
  // starts of this thread's words
  uint32_t wpos = pre.words;
  while (starts_m) {
    const int b = __ffsll(starts_m) - 1;
    starts_m &= starts_m - 1;
    const uint64_t below = b ? (lm & (~0ull >> (64 - b))) : 0ull;
    starts[wpos++] = pre.letters + __popcll(below);
  }
  // compact letters into shared memory at their offset within the CTA's run
  uint8_t* stage = reinterpret_cast<uint8_t*>(buf);
  uint32_t lpos = ex.letters;
  uint64_t m = lm;
  while (m) {
    const int b = __ffsll(m) - 1;
    m &= m - 1;
    stage[lpos++] = (uint8_t)(w[b >> 2] >> (8 * (b & 3)));
  }
  __syncthreads();
  const uint32_t out0 = cin.letters;
  for (uint32_t i = threadIdx.x; i < total.letters; i += kTokThreads) letters_out[out0 + i] = stage[i];
}

// K2: per-document length histogram.  Work item i is a block of up to 1024
// consecutive words of one document.  Bin 0 of a document counts its words
// longer than l_cap (a valid result always has counts[0] == 0).
__global__ void __launch_bounds__(kWordThreads) k_hist(const uint32_t* __restrict__ starts,
                                                       const uint32_t* __restrict__ doc_wbase,
                                                       const uint32_t* __restrict__ doc_item0, uint32_t ndocs,
                                                       uint32_t l_cap, uint32_t* __restrict__ hist, Meta* meta) {
  __shared__ uint32_t h[kHist];
  __shared__ uint32_t s_doc;
  const uint32_t items = doc_item0[ndocs];
  for (uint32_t it = blockIdx.x; it < items; it += gridDim.x) {
    for (int i = threadIdx.x; i < kHist; i += kWordThreads) h[i] = 0;
    if (threadIdx.x == 0) {
      uint32_t lo = 0, hi = ndocs - 1;  // last document with doc_item0 <= it
      while (lo < hi) {
        const uint32_t mid = (lo + hi + 1) >> 1;
        if (doc_item0[mid] <= it)
          lo = mid;
        else
          hi = mid - 1;
      }
      s_doc = lo;
    }
    __syncthreads();
    const uint32_t d = s_doc;
    const uint32_t w0 = doc_wbase[d] + (it - doc_item0[d]) * kWordBlock;
    const uint32_t w1 = min(w0 + kWordBlock, doc_wbase[d + 1]);
    uint32_t too_long = 0;
    for (uint32_t wi = w0 + threadIdx.x; wi < w1; wi += kWordThreads) {
      const uint32_t L = starts[wi + 1] - starts[wi];
      if (L > l_cap) {
        ++too_long;
        atomicAdd(&h[0], 1u);
      } else {
        atomicAdd(&h[L], 1u);
      }
    }
    if (too_long) atomicAdd(&meta->err_long, too_long);
    __syncthreads();
    for (int i = threadIdx.x; i < kHist; i += kWordThreads)
      if (h[i]) atomicAdd(&hist[(size_t)d * kHist + i], h[i]);
    __syncthreads();
  }
}

}  // namespace

cudaError_t launch_tok_summary(const uint8_t* in, const DocDesc* docs, uint32_t ndocs, uint32_t nchunks,
                               TokSum* sums, cudaStream_t st) {
  if (nchunks == 0) return cudaSuccess;
  k_tok_summary<<<nchunks, kTokThreads, 0, st>>>(in, docs, ndocs, sums);
  return cudaGetLastError();
}

cudaError_t launch_tok_scan(const TokSum* sums, uint32_t nchunks, const DocDesc* docs, uint32_t ndocs,
                            TokSum* carry, uint32_t* doc_wbase, uint32_t* doc_lbase, uint32_t* doc_item0,
                            uint32_t* starts, Meta* meta, cudaStream_t st) {
  k_tok_scan<<<1, kScanThreads, 0, st>>>(sums, nchunks, docs, ndocs, carry, doc_wbase, doc_lbase, doc_item0, starts,
                                         meta);
  return cudaGetLastError();
}

cudaError_t launch_tok_write(const uint8_t* in, const DocDesc* docs, uint32_t ndocs, uint32_t nchunks,
                             const TokSum* carry, uint8_t* letters, uint32_t* starts, cudaStream_t st) {
  if (nchunks == 0) return cudaSuccess;
  k_tok_write<<<nchunks, kTokThreads, 0, st>>>(in, docs, ndocs, carry, letters, starts);
  return cudaGetLastError();
}

cudaError_t launch_hist(const uint32_t* starts, const uint32_t* doc_wbase, const uint32_t* doc_item0,
                        uint32_t ndocs, uint32_t grid, uint32_t l_cap, uint32_t* hist, Meta* meta,
                        cudaStream_t st) {
  if (grid == 0) return cudaSuccess;
  k_hist<<<grid, kWordThreads, 0, st>>>(starts, doc_wbase, doc_item0, ndocs, l_cap, hist, meta);
  return cudaGetLastError();
}

}  // namespace bsort
