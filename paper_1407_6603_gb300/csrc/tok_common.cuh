// Device helpers of the strip + tokenize step (K1), shared by the one-pass
// kernels of k_tokenize1p.cu (the main path) and k_strip_noalloc.cu.
//
// Each thread owns 64 consecutive bytes.  It classifies them four at a time
// (swar.h) into two 64-bit masks (letters, whitespace), and
// finds the word starts among its letters with one addition: adding
// (whitespace << 1) to the mask of transparent bytes (neither letter nor
// whitespace) carries each whitespace bit across the transparent run after it
// and stops on the next letter or whitespace byte, so
// ((T + (Ws << 1)) ^ T) & Letters marks exactly the letters whose previous
// letter-or-whitespace byte is whitespace.
#pragma once

#include "bsort_dev.cuh"
#include "swar.h"

namespace bsort {
namespace {

constexpr uint32_t kFull = 0xFFFFFFFFu;

// Letter and whitespace bit masks of 64 bytes held as 16 little-endian words.
__device__ __forceinline__ void classify64(const uint32_t (&w)[16], uint64_t& letters, uint64_t& spaces) {
  uint32_t l[2] = {0, 0}, sp[2] = {0, 0};
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    const uint32_t c = class_nibbles(w[i]);
    l[i >> 3] |= (c & 0xFu) << (4 * (i & 7));
    sp[i >> 3] |= (c >> 4) << (4 * (i & 7));
  }
  letters = ((uint64_t)l[1] << 32) | l[0];
  spaces = ((uint64_t)sp[1] << 32) | sp[0];
}

// Letters whose previous letter-or-space byte is a space.  `ws_before` says
// whether the last such byte before these 64 is a space.
__device__ __forceinline__ uint64_t start_mask(uint64_t letters, uint64_t spaces, bool ws_before) {
  const uint64_t transparent = ~(letters | spaces);
  const uint64_t seeds = (spaces << 1) | (ws_before ? 1ull : 0ull);
  return ((transparent + seeds) ^ transparent) & letters;
}

__device__ __forceinline__ TokSum seg_summary(uint64_t letters, uint64_t spaces, bool doc_start) {
  TokSum s;
  s.letters = __popcll(letters);
  s.words = __popcll(start_mask(letters, spaces, doc_start));
  const uint64_t ev = letters | spaces;
  uint32_t flags = 0;
  if (ev) {
    flags |= kEv;
    const int hi = 63 - __clzll(ev);
    if ((spaces >> hi) & 1ull) flags |= kWs;
    const int lo = __ffsll(ev) - 1;
    if (!doc_start && ((letters >> lo) & 1ull)) flags |= kU;
  } else if (doc_start) {
    flags = kEv | kWs;
  }
  s.flags = flags;
  return s;
}

__device__ __forceinline__ TokSum shfl_up_sum(const TokSum& v, int off) {
  TokSum r;
  r.letters = __shfl_up_sync(kFull, v.letters, off);
  r.words = __shfl_up_sync(kFull, v.words, off);
  r.flags = __shfl_up_sync(kFull, v.flags, off);
  return r;
}

__device__ __forceinline__ TokSum warp_inclusive(TokSum v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const TokSum u = shfl_up_sum(v, off);
    if (lane >= off) v = tok_combine(u, v);
  }
  return v;
}

// Exclusive scan over the CTA (blockDim.x == kTokThreads).  Returns this
// thread's exclusive prefix and the CTA total.
__device__ TokSum block_exclusive(const TokSum v, TokSum* total) {
  __shared__ TokSum warp_tot[kTokThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const TokSum inc = warp_inclusive(v);
  if (lane == 31) warp_tot[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    TokSum w = {0, 0, 0};
    if (lane < kTokThreads / 32) w = warp_tot[lane];
    w = warp_inclusive(w);
    if (lane < kTokThreads / 32) warp_tot[lane] = w;
  }
  __syncthreads();
  TokSum ex = shfl_up_sum(inc, 1);
  if (lane == 0) ex = TokSum{0, 0, 0};
  if (warp > 0) ex = tok_combine(warp_tot[warp - 1], ex);
  *total = warp_tot[kTokThreads / 32 - 1];
  __syncthreads();
  return ex;
}

// Packed scan element of a span inside one chunk (one document): letters in
// bits 0..14, words in bits 15..28, the flags EV / WS / U in bits 29..31.  A
// chunk holds at most 16384 letters and 8192 word starts, so no field
// overflows into the next and one 32-bit shuffle carries all three.
constexpr uint32_t kPkWords = 15, kPkFlags = 29, kPkCounts = (1u << kPkFlags) - 1u;
__device__ __forceinline__ uint32_t pk_make(uint32_t letters, uint32_t words, uint32_t flags) {
  return letters | (words << kPkWords) | (flags << kPkFlags);
}
__device__ __forceinline__ uint32_t pk_letters(uint32_t v) { return v & ((1u << kPkWords) - 1u); }
__device__ __forceinline__ uint32_t pk_words(uint32_t v) { return (v & kPkCounts) >> kPkWords; }
__device__ __forceinline__ uint32_t pk_flags(uint32_t v) { return v >> kPkFlags; }
// tok_combine on packed elements (0 is the identity)
__device__ __forceinline__ uint32_t pk_combine(uint32_t a, uint32_t b) {
  const uint32_t fa = a >> kPkFlags, fb = b >> kPkFlags;
  const bool resolve = (fb & kU) && (fa & kEv) && (fa & kWs);
  const uint32_t counts = (a & kPkCounts) + (b & kPkCounts) + (resolve ? (1u << kPkWords) : 0u);
  const uint32_t ev = (fa | fb) & kEv;
  const uint32_t ws = (fb & kEv) ? (fb & kWs) : (fa & kWs);
  const uint32_t u = (fa & kEv) ? (fa & kU) : (fb & kU);
  return counts | ((ev | ws | u) << kPkFlags);
}

// Exclusive scan of packed elements over the CTA; returns this thread's
// prefix and the CTA total.  Ends with a barrier.
__device__ uint32_t block_exclusive_pk(uint32_t v, uint32_t* total) {
  __shared__ uint32_t warp_tot[kTokThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t inc = v;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const uint32_t u = __shfl_up_sync(kFull, inc, off);
    if (lane >= off) inc = pk_combine(u, inc);
  }
  if (lane == 31) warp_tot[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    uint32_t w = lane < kTokThreads / 32 ? warp_tot[lane] : 0u;
#pragma unroll
    for (int off = 1; off < kTokThreads / 32; off <<= 1) {
      const uint32_t u = __shfl_up_sync(kFull, w, off);
      if (lane >= off) w = pk_combine(u, w);
    }
    if (lane < kTokThreads / 32) warp_tot[lane] = w;
  }
  __syncthreads();
  uint32_t ex = __shfl_up_sync(kFull, inc, 1);
  if (lane == 0) ex = 0u;
  if (warp > 0) ex = pk_combine(warp_tot[warp - 1], ex);
  *total = warp_tot[kTokThreads / 32 - 1];
  __syncthreads();
  return ex;
}

// byte_perm selectors that move the bytes of a 4-bit mask, in order, to the
// low end of a word and fill the rest with zero bytes: nibble k of entry m is
// the position of the k-th set bit of m (4 selects a zero byte).  Threads
// 0..15 each fill one entry of a CTA's table.
__device__ __forceinline__ void compact_table_fill(uint32_t* tab) {
  const uint32_t m = threadIdx.x;
  if (m < 16) {
    uint32_t sel = 0x4444u, k = 0;
    for (uint32_t b = 0; b < 4; ++b)
      if ((m >> b) & 1u) {
        sel = (sel & ~(0xFu << (4 * k))) | (b << (4 * k));
        ++k;
      }
    tab[m] = sel;
  }
}

// Writes the letters of the thread's 64 bytes (w, letter mask lm), in order,
// to stage[pos...]: whole aligned 32-bit words where all four bytes are the
// thread's, single bytes at the two ends (which neighbours share).  Pending
// bytes (at most seven) are held in two 32-bit words, the first at byte 0 of
// `lo`, behind the `skew` bytes that precede pos in its word.
__device__ __forceinline__ void stage_letters(const uint32_t (&w)[16], uint64_t lm, uint8_t* stage, uint32_t pos,
                                              const uint32_t* sel_tab) {
  uint32_t* stage32 = reinterpret_cast<uint32_t*>(stage);
  const uint32_t skew = pos & 3u;
  uint32_t lo = 0, hi = 0;
  uint32_t na = skew;  // pending byte count, below 4 at the top of each step
  uint32_t wi = pos >> 2;
  bool first = true;
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    const uint32_t m4 = ((j < 8 ? (uint32_t)lm : (uint32_t)(lm >> 32)) >> (4 * (j & 7))) & 0xFu;
    const uint32_t c = __byte_perm(w[j], 0u, sel_tab[m4]);
    const uint32_t sh = 8 * na;
    hi = __funnelshift_l(c, 0u, sh);  // the bytes of c that pass byte 3
    lo |= c << sh;
    na += __popc(m4);
    if (na >= 4) {
      if (first && skew) {
        for (uint32_t b = skew; b < 4; ++b) stage[4 * wi + b] = (uint8_t)(lo >> (8 * b));
      } else {
        stage32[wi] = lo;
      }
      first = false;
      ++wi;
      lo = hi;
      hi = 0;
      na -= 4;
    }
  }
  for (uint32_t b = first ? skew : 0u; b < na; ++b) stage[4 * wi + b] = (uint8_t)(lo >> (8 * b));
}

// Shared-memory slot of the chunk's 16-byte granule g.  The chunk is loaded
// with granule g in thread g % 256's hands and read back four consecutive
// granules per thread; XOR-ing the low three bits with bits 2..4 spreads
// both access patterns over all eight 16-byte bank groups (no conflicts).
__device__ __forceinline__ uint32_t chunk_slot(uint32_t g) { return g ^ ((g >> 2) & 7u); }

__device__ __forceinline__ void thread_words(const uint4* buf, uint32_t (&w)[16]) {
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const uint4 v = buf[chunk_slot(threadIdx.x * 4 + i)];
    w[4 * i + 0] = v.x;
    w[4 * i + 1] = v.y;
    w[4 * i + 2] = v.z;
    w[4 * i + 3] = v.w;
  }
}

}  // namespace
}  // namespace bsort
