// Internal declarations shared by the CUDA translation units of libbsort.
//
// Data flow of one call (every kernel covers all documents of the call):
//   K1  tokenize      per 16 KiB chunk, one pass (decoupled look-back): the
//                     stripped letter stream S, the S offset of every word
//                     start, the per-document length histograms and bases
//   K2  layout        per document: one segment per (doc, length) with words,
//                     placed in the table by the kernels that sort it; the
//                     host reads back only a fixed-size summary (grid sizes)
//   K3  scatter       per 2048-word block: each word packed into a big-endian
//                     key of W u64 words, written to its segment
//   K4  tile_sort     per tile: odd-even transposition sort, then merges
//                     through distributed shared memory inside a cluster
//   K5  merge_pass    per tile and pass: merge-path merge of run pairs
//   K6  emit          per tile: keys back to bytes, offsets, counts
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "bsort.h"

namespace bsort {

constexpr int kHist = 256;                  // histogram bins: lengths 0..255
constexpr int kMaxLen = 255;                // longest word the key layout holds
constexpr int kTokThreads = 256;            // K1 CTA size
constexpr int kTokSeg = 64;                 // bytes per K1 thread
constexpr int kChunk = kTokThreads * kTokSeg;  // bytes per K1 chunk (16 KiB)
constexpr int kWordBlock = 2048;            // words per K3 work item
constexpr int kWordThreads = 256;
constexpr int kSortThreads = 256;           // K4/K5/K6 CTA size
constexpr int kNumClasses = 6;              // key widths W = 1, 2, 4, 8, 16, 32 u64 words
constexpr uint32_t kNoSegment = 0xFFFFFFFFu;
constexpr uint64_t kDefaultWaitLimit = 1ull << 26;
// Least number of polls a CTA gives one of its own bulk copies into shared
// memory, whatever the configured wait limit: a copy is never abandoned while
// it may still land in memory the CTA goes on to use.
constexpr uint64_t kCopyWaitFloor = 1ull << 26;

// Key width class of a word of L letters: W = next power of two >= ceil(L/8).
__host__ __device__ inline int width_of_len(uint32_t L) {
  // next_pow2(ceil(L / 8)), 1 for L <= 8: without a loop
  const uint32_t k = (L + 7) >> 3;
  if (k <= 1) return 1;
#ifdef __CUDA_ARCH__
  return 1 << (32 - __clz(k - 1));
#else
  return 1 << (32 - __builtin_clz(k - 1));
#endif
}
// Key encodings.  A key is a bit string from the most significant bit of its
// first u64 word, zero past its last letter, so that unsigned order of the W
// words is the order wanted:
//   kCodeBytes  8 bits a letter, its ASCII byte (ASCII order);
//   kCodeSix    6 bits a letter, A..Z -> 1..26 and a..z -> 27..52 (the same
//               order, 10 letters a word instead of 8);
//   kCodeFold   5 bits a letter, its letter case-blind (a/A -> 1 .. z/Z -> 26),
//               then one bit a letter, 0 for upper case (alphabetic order,
//               ties in ASCII order).
// No letter codes to 0, so a word sorts before every longer word it begins
// when keys are padded with zeros to a common width.
constexpr uint32_t kCodeBytes = 0, kCodeSix = 1, kCodeFold = 2;
__host__ __device__ inline uint32_t bits_per_letter(uint32_t codec) { return codec == kCodeBytes ? 8u : 6u; }
// Key width in u64 words of L letters: the next power of two that holds them.
__host__ __device__ inline int key_width(uint32_t codec, uint32_t L) {
  const uint32_t k = (L * bits_per_letter(codec) + 63) / 64;
  if (k <= 1) return 1;
#ifdef __CUDA_ARCH__
  return 1 << (32 - __clz(k - 1));
#else
  return 1 << (32 - __builtin_clz(k - 1));
#endif
}

__host__ __device__ inline int class_of_width(int W) {
  return W == 1 ? 0 : W == 2 ? 1 : W == 4 ? 2 : W == 8 ? 3 : W == 16 ? 4 : 5;
}
__host__ __device__ inline int width_of_class(int c) { return 1 << c; }
// Keys per thread of the sort kernels: a tile holds 2048 u64 words (16 KiB)
// for W <= 8, and 256 keys for the wider classes.
__host__ __device__ inline int kpt_of_width(int W) { return W >= 8 ? 1 : 8 / W; }
__host__ __device__ inline int tile_of_width(int W) { return kSortThreads * kpt_of_width(W); }

struct DocDesc {
  uint64_t byte_off;  // first byte of the document, counted from the input base pointer
  uint64_t len;       // bytes
  uint32_t chunk0;    // first K1 chunk of the document
  uint32_t nchunks;   // K1 chunks (0 for an empty document)
};

// Scan element of K1: what a span of bytes contributes to the word count.
//   letters : letters in the span
//   words   : word starts decided inside the span
//   flags   : bit0 EV  the span has a letter or a whitespace byte
//             bit1 WS  the span's last such byte is whitespace
//             bit2 U   the span's first such byte is a letter, whose being a
//                      word start depends on what precedes the span
struct TokSum {
  uint32_t letters;
  uint32_t words;
  uint32_t flags;
};
constexpr uint32_t kEv = 1u, kWs = 2u, kU = 4u;

__host__ __device__ inline TokSum tok_combine(const TokSum& a, const TokSum& b) {
  TokSum r;
  r.letters = a.letters + b.letters;
  const bool resolve = (b.flags & kU) && (a.flags & kEv) && (a.flags & kWs);
  r.words = a.words + b.words + (resolve ? 1u : 0u);
  const uint32_t ev = (a.flags | b.flags) & kEv;
  const uint32_t ws = (b.flags & kEv) ? (b.flags & kWs) : (a.flags & kWs);
  const uint32_t u = (a.flags & kEv) ? (a.flags & kU) : (b.flags & kU);
  r.flags = ev | ws | u;
  return r;
}

// Device-written summary of K1 that the host reads back.
struct Meta {
  uint32_t n_total;       // words over all documents
  uint32_t s_total;       // letters over all documents
  uint32_t items_total;   // K2/K3 work items
  uint32_t err_long;      // words longer than l_cap
  uint32_t err_timeout;   // bounded waits that ran out: in the sticky copy, those of the sort
                          // kernels (kept until read); in a call's meta, those of its K1
  uint32_t err_prev;      // a call's meta: the sticky count when its K1 ran (earlier calls)
  uint32_t err_internal;  // sticky: a consistency check of the sort kernels failed
  uint32_t err_site;      // sticky: the first such check's site (kernel << 8 | place)
};

// One (document, length) bucket.  K2 orders the table by the K4/K5 kernels
// that sort it (table_order), so that each launch covers a contiguous range
// of it.
struct Segment {
  uint64_t key_off;     // first key, in u64 words, in both key buffers
  uint32_t n;           // words in the bucket
  uint32_t L;           // their length
  uint32_t doc;
  uint32_t tile0;       // first merge tile (K5), numbered over the merge range
  uint32_t etile0;      // first emit tile (K6), numbered over the whole table
  uint32_t stile0;      // first K4 supertile, numbered within its K4 launch
  uint32_t out_word;    // index in offsets[] of the bucket's first word
  uint32_t stream_off;  // byte offset in the output stream of the bucket's first word
  uint32_t doc_stream0; // first stream byte of the document (offsets are per document)
  uint32_t final_buf;   // 0: sorted keys end in buffer A, 1: in buffer B
  uint32_t passes;      // merge passes the bucket needs after K4
  uint32_t run0;        // length of the sorted runs K4 leaves
  uint32_t smp_off;     // pipelined merges: first u64 word of the bucket's merge samples
  uint32_t flags;       // kSegKeysOut, kSegDedupe; bits 8..31: the bucket's dedupe index
  uint32_t W;           // key width in u64 words
  uint32_t pad2[3];
};
static_assert(sizeof(Segment) == 80, "a segment is five 16-byte words");
// Segment flags.  kSegKeysOut: the sorted keys stay in the key buffer (final_buf)
// instead of being emitted as words (the distinct-word arrays of the
// duplicate-aware sort).  kSegDedupe: the hash aggregation kernel (not K4)
// hands the bucket's distinct keys, with their multiplicities, to the
// bucket's hash table.
constexpr uint32_t kSegKeysOut = 1u, kSegDedupe = 2u;
__host__ __device__ inline uint32_t seg_dedupe_index(const Segment& s) { return s.flags >> 8; }

// Duplicate-aware sort (an option of the sort phase; the result is the same):
// a bucket's distinct keys are collected in a hash table with their counts,
// sorted, and expanded by their counts.  Per bucket, for the hash inserts:
struct DedupeIns {
  uint64_t htab_off;  // first u64 word of the bucket's table: 2^hbits slots of 1 + W words
  uint64_t uniq_off;  // first u64 word of its distinct-key array: entries of Wp words
                      // (the key's W words, its count, zeros; while the inserts run, the
                      // slot index after the key or after the count), at most n entries
  uint64_t cnt_off;   // one-word keys: first of its n words of the count array
  uint32_t hbits;
  uint32_t Wp;        // next_pow2(W + 1)
  uint32_t n;         // the bucket's words: the array's capacity in entries
  uint32_t pad;
};
// Per bucket, for the expansion after the distinct keys are sorted:
struct ExpandDesc {
  uint64_t uniq_off;  // the sorted distinct-key array (in the buffer final_buf names)
  uint64_t pre_off;   // u32 index of its exclusive prefix of counts (U + 1 entries)
  uint32_t U;         // distinct keys
  uint32_t n;         // words (the sum of the counts)
  uint32_t L;
  uint32_t Wp;
  uint32_t final_buf;
  uint32_t tile0;     // first output tile, numbered over the expanded buckets
  uint32_t stream_off, out_word, doc_stream0;
  uint32_t pad;
};
constexpr uint32_t kExpandTileWords = 2048;
// words per output tile of the expansion for keys of W u64 words
__host__ __device__ inline uint32_t expand_tile(uint32_t W) { return kExpandTileWords / W; }
// The whole-text order's emission: per document, its bucket of every word
// sorted with zero-padded keys (kept in the key buffer final_buf names).
struct VarDesc {
  uint64_t key_off;
  uint32_t n, W, final_buf;
  uint32_t letters;  // the document's letters: what the words' lengths must add up to
  uint32_t out_word, stream_off, doc_stream0;
  uint32_t pad;
};
// Where the hash inserts go (one call's tables, arrays and counters).
struct DedupeOut {
  const DedupeIns* ins;
  uint64_t* htab;  // every slot zero between calls
  uint64_t* uniq;
  uint32_t* ucnt;  // distinct keys per bucket so far (zeroed per call)
  uint64_t* dcnt;  // one-word keys' counts by distinct-key index (zero between calls)
};

// One output tile of a pipelined merge pass (K5), as the cut kernel leaves it:
// where the tile's slices of the two runs start and where run A ends, how
// many keys it outputs, and where they go.  The tile takes run A's keys up to
// the next tile's a_src (or a_end, whichever comes first) and the rest of its
// outputs from run B.
struct TileJob {
  uint64_t a_src;   // word offset in the source key buffer of the tile's first key of run A
  uint64_t b_src;   // the same for run B
  uint64_t a_end;   // end of run A (its words up to, not including, this offset)
  uint64_t dst;     // word offset in the destination key buffer of the tile's first output
  uint32_t cnt;     // outputs of the tile; 0: nothing to do
  uint32_t L;       // 0: the merged keys go to dst; else this pass finishes the bucket
                    // and its words (of L letters) are emitted:
  uint32_t stream;  //   stream byte offset of the tile's first word
  uint32_t word;    //   offsets[] index of that word
  uint32_t rel;     //   its offset within its document
  uint32_t smp;     // kNoSamples, or the word offset in the sample buffer of the slot of
                    // the tile's first 32 outputs: the merge stores its output at
  uint32_t smp_phase;  // tile positions = smp_phase (mod 32) there, one slot per 32
  uint32_t pad;
};
constexpr uint32_t kNoSamples = 0xFFFFFFFFu;
static_assert(sizeof(TileJob) == 64, "TileJob is four 16-byte copies");

// K4 v2 / K5 v2 geometry (keys of at most 16 u64 words).
constexpr int kSuperCluster = 8;    // CTAs per K4 cluster
// keys per K4 CTA tile: 2048 u64 words, 256 keys of 16 words
__host__ __device__ inline uint32_t tile2_keys(int W) { return (uint32_t)(W >= 16 ? 256 : 2048 / W); }
__host__ __device__ inline uint32_t merge2_keys(int W) { return (uint32_t)(256 * (W >= 8 ? 1 : 8 / W)); }
// keys a single warp sorts on its own (32 lanes x keys per thread)
__host__ __device__ inline uint32_t warp_keys(int W) { return (uint32_t)(32 * (W >= 8 ? 1 : 8 / W)); }

// Sort groups of a bucket of n keys of W words (T = tile2_keys(W)):
//   0..3  W = 1, 2, 4, 8 and more than 8T keys: K4 into runs, then K5 merge
//         passes, or the duplicate-aware sort's hash aggregation; 4 unused
//   5     (4T, 8T] keys: K4 in clusters of 8        6   (2T, 4T]: clusters of 4
//   7     (T, 2T]: clusters of 2                      8   (32 KPT, T]: single CTAs
//   9     at most 32 lanes x KPT keys: one warp each
//   10,11 keys of 16 / 32 words: the narrow-tile kernels of k_sort.cu
constexpr int kGroups = 12;
__host__ __device__ inline int sort_group(uint32_t n, int W) {
  if (W >= 16) return W == 16 ? 10 : 11;
  const uint32_t T = tile2_keys(W);
  if (n <= warp_keys(W)) return 9;
  if (n <= T) return 8;
  if (n <= 2 * T) return 7;
  if (n <= 4 * T) return 6;
  if (n <= (uint32_t)kSuperCluster * T) return 5;
  return class_of_width(W);
}
// CTAs per cluster of the K4 launch that finishes group g (5..8)
__host__ __device__ inline uint32_t group_cluster(int g) { return (uint32_t)kSuperCluster >> (g - 5); }
// merge passes that take runs of `tile` keys to one run of n
__host__ __device__ inline uint32_t merge_passes(uint64_t n, uint64_t tile) {
  uint32_t p = 0;
  while ((tile << p) < n) ++p;
  return p;
}
__host__ __device__ inline uint32_t ceil_log2_u(uint64_t n) {
#ifdef __CUDA_ARCH__
  return n <= 1 ? 0u : (uint32_t)(64 - __clzll((long long)(n - 1)));
#else
  return n <= 1 ? 0u : (uint32_t)(64 - __builtin_clzll(n - 1));
#endif
}
// The segment table's order of the groups, given the run length K4 leaves
// for the merge passes: the groups K4 finishes (clusters of 8, 4, 2, 1), with
// the groups that need merge passes (0..3, and the unused 4) placed just
// before the one whose cluster size makes their runs, so that every K4
// launch and every width's merge chain covers one contiguous range; then
// the warp sort and the wide keys.  order[q] is the group at position q.
__host__ __device__ inline void table_order(uint32_t runs, int* order, int* pos_of) {
  int q = 0;
  for (int gc = 5; gc <= 8; ++gc) {
    if (group_cluster(gc) == runs || (runs > (uint32_t)kSuperCluster && gc == 5))
      for (int g = 0; g < 5; ++g) order[q++] = g;
    order[q++] = gc;
  }
  for (int g = 9; g < kGroups; ++g) order[q++] = g;
  for (int i = 0; i < kGroups; ++i) pos_of[order[i]] = i;
}
// key words per unit of the duplicate-aware sort's hash aggregation
constexpr uint32_t kDedupeUnitWords = 2048;
__host__ __device__ inline uint32_t dedupe_unit_keys(uint32_t W) { return kDedupeUnitWords / W; }

// Work items of the sort and emit kernels are numbered across buckets; a
// CTA finds the bucket of an item by binary search over the buckets' first
// item numbers.  When a launch covers at most kSegCache buckets (every single
// document), the numbers are first copied to shared memory so that the search
// costs no global loads.
constexpr uint32_t kSegCache = 256;

// Where sorted words go: the output stream and per-word offsets, and how
// the keys are encoded.
struct EmitOut {
  uint8_t* stream;
  uint32_t* offsets;
  int want_offsets;
  uint32_t codec;
};

#if defined(__CUDACC__)
// Quotient n / L by one wide multiply with m = ceil(2^32 / L), a 33-bit
// number for L = 1 (division by an invariant integer through its scaled
// reciprocal, after Granlund and Montgomery, 1994).  With e = m L - 2^32 < L,
// n m / 2^32 exceeds n / L by n e / (L 2^32), under 1 / L while n e < 2^32,
// which leaves the floor unchanged: exact for every n < 2^24 and L < 256.
__host__ __device__ __forceinline__ uint64_t recip_of(uint32_t L) { return ((1ull << 32) + L - 1) / L; }
__host__ __device__ __forceinline__ uint32_t quot(uint32_t n, uint64_t m) { return (uint32_t)(((uint64_t)n * m) >> 32); }

// n bits (n <= 32) at bit offset off of a key whose u64 words kw(q) gives.
template <class KW>
__device__ __forceinline__ uint32_t key_bits(KW kw, uint32_t off, uint32_t n) {
  const uint32_t w = off >> 6, sh = off & 63;
  uint64_t v = kw(w) << sh;
  if (sh + n > 64) v |= kw(w + 1) >> (64 - sh);
  return (uint32_t)(v >> (64 - n));
}
// Letters 8q .. 8q + 7 of a key of L letters as big-endian ASCII bytes (zero
// past L), whatever the encoding; kw(q') gives the key's u64 word q'.
template <class KW>
__device__ __forceinline__ uint64_t ascii8(uint32_t codec, uint32_t L, KW kw, uint32_t q) {
  if (codec == kCodeBytes) return kw(q);
  uint64_t r = 0;
  const uint32_t i0 = 8 * q, i1 = min(L, i0 + 8);
  for (uint32_t i = i0; i < i1; ++i) {
    uint32_t ch;
    if (codec == kCodeSix) {
      const uint32_t c = key_bits(kw, 6 * i, 6);
      ch = c <= 26 ? 'A' - 1 + c : 'a' - 27 + c;
    } else {
      const uint32_t c = key_bits(kw, 5 * i, 5);
      ch = (key_bits(kw, 5 * L + i, 1) ? 'a' - 1 : 'A' - 1) + c;
    }
    r |= (uint64_t)ch << (56 - 8 * (i - i0));
  }
  return r;
}

// Emits cnt sorted keys of L letters as the letters of the words (phase 3's
// output, Section II: each length's sorted words, shorter lengths first) at p0
// and, when offs is set, word j's offset within its document, rel0 + j L, at
// offs[j].  key_word(j, q) gives u64 word q of key j, encoded with codec
// (for kCodeBytes: big-endian letters, zero past the word's L letters).  The run's bytes are one contiguous range of the
// stream (at most 2^24 bytes): the NTH threads write its 16-byte aligned
// middle with whole 16-byte stores, each gathering its 16 bytes piece by piece
// (one piece = the rest of one key word, at most 8 bytes), and its ragged ends
// byte by byte, so no byte outside the range is touched and runs never overlap.
template <int NTH, class F>
__device__ __forceinline__ void emit_run(uint32_t L, uint8_t* p0, uint32_t* offs, uint32_t rel0, uint32_t cnt,
                                         F key_word_raw, uint32_t codec) {
  // the key words as ASCII letters, 8 to a word (the keys' own words for kCodeBytes)
  auto key_word = [&](uint32_t j, uint32_t q) -> uint64_t {
    return ascii8(codec, L, [&](uint32_t w) { return key_word_raw(j, w); }, q);
  };
  const uint64_t m = recip_of(L);
  const int t = threadIdx.x;
  const uint32_t nbytes = cnt * L;
  const uint32_t head = min(nbytes, (uint32_t)((16u - ((uintptr_t)p0 & 15u)) & 15u));
  const uint32_t chunks = (nbytes - head) >> 4;
  const uint32_t tail0 = head + chunks * 16u;
  for (uint32_t off = t; off < head + (nbytes - tail0); off += NTH) {  // the ragged ends
    const uint32_t o = off < head ? off : tail0 + (off - head);
    const uint32_t j = quot(o, m), b = o - j * L;
    p0[o] = (uint8_t)(key_word(j, b >> 3) >> (56 - 8 * (b & 7)));
  }
  for (uint32_t c = t; c < chunks; c += NTH) {
    const uint32_t off = head + c * 16u;
    uint32_t j = quot(off, m), b = off - j * L;
    uint64_t hi = 0, lo = 0;  // the chunk, big-endian from the top of hi
    uint32_t nb = 0;          // bytes gathered so far
    do {
      const uint32_t s = b & 7;
      const uint32_t take = min(8u, L - (b & ~7u)) - s;  // letters left in this key word
      const uint64_t v = key_word(j, b >> 3) << (8 * s);
      if (nb < 8) {
        hi |= v >> (8 * nb);
        if (nb) lo |= v << (64 - 8 * nb);
      } else {
        lo |= v >> (8 * (nb - 8));
      }
      nb += take;
      b += take;
      if (b == L) {
        b = 0;
        ++j;
      }
    } while (nb < 16);
    const uint32_t h1 = (uint32_t)(hi >> 32), h0 = (uint32_t)hi, l1 = (uint32_t)(lo >> 32), l0 = (uint32_t)lo;
    *reinterpret_cast<uint4*>(p0 + off) =
        make_uint4(__byte_perm(h1, 0, 0x0123), __byte_perm(h0, 0, 0x0123), __byte_perm(l1, 0, 0x0123),
                   __byte_perm(l0, 0, 0x0123));
  }
  if (offs)
    for (uint32_t j = t; j < cnt; j += NTH) offs[j] = rel0 + j * L;
}

// emit_run for keys [k0, k0 + cnt) of bucket sg.
template <int NTH, class F>
__device__ __forceinline__ void emit_tile(const Segment& sg, uint32_t k0, uint32_t cnt, F key_word,
                                          const EmitOut& eo) {
  emit_run<NTH>(sg.L, eo.stream + sg.stream_off + (size_t)k0 * sg.L,
                eo.want_offsets ? eo.offsets + sg.out_word + k0 : nullptr, sg.stream_off - sg.doc_stream0 + k0 * sg.L,
                cnt, key_word, eo.codec);
}

// The last index d in [0, n) with key(d) <= x, for keys ascending in d and
// key(0) <= x, found by one warp (all 32 lanes call it): every round probes 32
// evenly spaced indexes and keeps the gap after the last one that qualifies,
// so about log32(n) rounds of loads instead of log2(n) one after another.
template <class K>
__device__ __forceinline__ uint32_t warp_last_le(K key, uint32_t n, uint32_t x) {
  const uint32_t lane = threadIdx.x & 31u;
  uint32_t lo = 0, hi = n;  // the answer is in [lo, hi)
  while (hi - lo > 1) {
    const uint32_t step = (hi - lo + 31) / 32;
    const uint32_t p = lo + lane * step;
    const bool ok = p < hi && key(p) <= x;
    const uint32_t m = __ballot_sync(0xffffffffu, ok);
    const uint32_t h = 31u - __clz(m);  // lane 0 always qualifies
    lo = lo + h * step;
    hi = min(lo + step, hi);
  }
  return lo;
}

// Field selector: which first-item number a kernel searches by.
enum SegField { kByTile0, kByStile0, kByEtile0 };
template <SegField F>
__device__ __forceinline__ uint32_t seg_first_item(const Segment& s) {
  return F == kByTile0 ? s.tile0 : F == kByStile0 ? s.stile0 : s.etile0;
}
// Loads the first-item numbers of segments [sbeg, send) into `cache` when
// they fit; returns whether they did.  Call from all threads; ends with a
// barrier.
template <SegField F>
__device__ __forceinline__ bool seg_cache_fill(const Segment* segs, uint32_t sbeg, uint32_t send,
                                               uint32_t* cache) {
  const bool fits = send - sbeg <= kSegCache;
  if (fits)
    for (uint32_t i = threadIdx.x; i < send - sbeg; i += blockDim.x) cache[i] = seg_first_item<F>(segs[sbeg + i]);
  __syncthreads();
  return fits;
}
// Last segment in [sbeg, send) whose first item is <= it.
template <SegField F>
__device__ __forceinline__ uint32_t seg_find(const Segment* segs, uint32_t sbeg, uint32_t send,
                                             const uint32_t* cache, bool cached, uint32_t it) {
  uint32_t lo = 0, hi = send - sbeg - 1;
  while (lo < hi) {
    const uint32_t mid = (lo + hi + 1) >> 1;
    const uint32_t v = cached ? cache[mid] : seg_first_item<F>(segs[sbeg + mid]);
    if (v <= it)
      lo = mid;
    else
      hi = mid - 1;
  }
  return sbeg + lo;
}
// seg_find by one warp (all 32 lanes call it): from the shared-memory cache
// when the launch's segments fit it, else by 32-way rounds over the table in
// global memory (a few dependent loads instead of one per halving).
template <SegField F>
__device__ __forceinline__ uint32_t seg_find_warp(const Segment* segs, uint32_t sbeg, uint32_t send,
                                                  const uint32_t* cache, bool cached, uint32_t it) {
  if (cached) return seg_find<F>(segs, sbeg, send, cache, true, it);
  return sbeg + warp_last_le([&](uint32_t i) { return seg_first_item<F>(segs[sbeg + i]); }, send - sbeg, it);
}
#endif

}  // namespace bsort
// Stops the serving loop of a context, if it runs one (bsort_serve.cu).
struct bsort_ctx;
void bsort_serve_shutdown(const struct bsort_ctx* ctx);
// The serving loop's hand-over of result buffers (bsort_api.cu): a context's
// page-locked result buffers (counts, offsets, stream) move out of it, with
// the results of its last call in them, and a set of earlier buffers moves
// back in for reuse; the context allocates new ones when it has none.
struct bsort_host_out;
struct bsort_host_out* bsort_take_result_buffers(struct bsort_ctx* ctx);
void bsort_give_result_buffers(struct bsort_ctx* ctx, struct bsort_host_out* b);
void bsort_free_result_buffers(struct bsort_host_out* b);
// Grows the context's result buffers to what a bsort_batch of `ndocs`
// documents of `bytes` bytes in all can need (at most: every byte a letter,
// every second one a word), so that the call reallocates none of them:
// freeing page-locked memory waits for the whole device.
bsort_status bsort_reserve_result_buffers(struct bsort_ctx* ctx, uint64_t bytes, uint64_t ndocs);
// Whether a set of result buffers is already large enough for such a batch.
bool bsort_result_buffers_fit(const struct bsort_host_out* b, uint64_t bytes, uint64_t ndocs);
// Ends the hold of a served result (bsort_serve.cu); false if it holds none.
bool bsort_serve_release(const struct bsort_ctx* ctx, const bsort_result* res);
namespace bsort {

// Runs `set` (kernel attribute calls and the like) once per device for the
// calling site instead of before every launch.  Repeating it is harmless, so
// two threads racing on the first call need no lock.
template <class F>
inline cudaError_t once_per_device(int (&done)[64], F set) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev >= 0 && dev < 64 && done[dev]) return cudaSuccess;
  e = set();
  if (e == cudaSuccess && dev >= 0 && dev < 64) done[dev] = 1;
  return e;
}

// -------- launchers (each returns the launch's cudaError_t) --------

// K1's look-back scratch (tokenize1p_scratch_bytes of it) must be zeroed
// before the launch, and meta's histograms too; the caller clears both with
// one memset.
size_t tokenize1p_scratch_bytes(uint32_t nchunks);
// Where K1's last CTA leaves a copy of the meta region for the host: `n16`
// 16-byte words to page-locked host memory at `dst`, then `seq` in *flag
// (after a system-scope fence).  dst == nullptr: no copy (the host reads the
// region with a copy of its own).
struct HostMeta {
  uint4* dst;
  uint32_t n16;
  uint32_t* flag;
  uint32_t seq;
};
// docs: the document table in device memory; with one document K1 takes
// doc0 (passed by value) instead and docs is not read.
cudaError_t launch_tokenize1p(const uint8_t* in, const DocDesc* docs, DocDesc doc0, uint32_t ndocs, uint32_t nchunks,
                              uint8_t* scratch, uint8_t* letters, uint32_t* starts, uint32_t* hist,
                              uint32_t* doc_maxlen, uint32_t* doc_wbase, uint32_t* doc_lbase, uint32_t* doc_item0, Meta* meta,
                              Meta* sticky, uint32_t l_cap, uint64_t wait_limit, HostMeta hm, cudaStream_t st);
// pack = false: only the counts and closing offsets, no keys (the length order).
cudaError_t launch_scatter(const uint32_t* starts, const uint8_t* letters, const uint32_t* doc_wbase,
                           const uint32_t* doc_lbase, const uint32_t* doc_item0, uint32_t ndocs, uint32_t items,
                           uint32_t grid, const uint32_t* seg_lookup, const Segment* segs, uint32_t* cursor,
                           uint64_t* keys, const uint32_t* hist, uint64_t* counts, EmitOut eo, bool pack,
                           cudaStream_t st);
cudaError_t launch_tile_sort(int W, const Segment* segs, uint32_t sbeg, uint32_t send, uint32_t tiles,
                             uint32_t grid, uint64_t* keys, Meta* meta, uint64_t wait_limit, cudaStream_t st);
cudaError_t launch_merge_pass(int W, const Segment* segs, uint32_t sbeg, uint32_t send, uint32_t tiles,
                              uint32_t grid, uint32_t pass, const uint64_t* src, uint64_t* dst, cudaStream_t st);
cudaError_t launch_warp_sort(const Segment* segs, uint32_t sbeg, uint32_t send, uint64_t* keys, EmitOut eo,
                             cudaStream_t st);
// K4 with clusters of `cluster` CTAs of `threads` (256, or 512 when no key
// of the launch is wider than 4 words) and `lanes` (2, 4 or 8) lanes per
// odd-even transposition group.
// The duplicate-aware sort's hash aggregation of segments [sbeg, send) (each
// marked kSegDedupe, with stile0 its first unit of dedupe_unit_keys(W) keys,
// `units` in all): every distinct key of a unit goes to its bucket's table
// with its count; then the `ndd` buckets' distinct-key arrays are completed
// and their tables' claimed slots zeroed.
cudaError_t launch_dedupe_hash(const Segment* segs, uint32_t sbeg, uint32_t send, uint32_t units, uint32_t sm_count,
                               const uint64_t* keys, DedupeOut o, uint32_t ndd, Meta* meta, uint64_t wait_limit,
                               cudaStream_t st);
cudaError_t launch_tile_sort2(int cluster, int lanes, int threads, const Segment* segs, uint32_t sbeg, uint32_t send,
                              uint32_t supertiles, int max_grid, int max_width, uint64_t* keys, EmitOut eo, Meta* meta,
                              uint64_t wait_limit, cudaStream_t st);
cudaError_t launch_tile_sort2_g2(int cluster, int threads, const Segment* segs, uint32_t sbeg, uint32_t send, uint32_t supertiles,
                                 int max_grid, int max_width, uint64_t* keys, EmitOut eo, Meta* meta,
                                 uint64_t wait_limit, cudaStream_t st);
cudaError_t launch_tile_sort2_g4(int cluster, int threads, const Segment* segs, uint32_t sbeg, uint32_t send, uint32_t supertiles,
                                 int max_grid, int max_width, uint64_t* keys, EmitOut eo, Meta* meta,
                                 uint64_t wait_limit, cudaStream_t st);
cudaError_t launch_tile_sort2_g8(int cluster, int threads, const Segment* segs, uint32_t sbeg, uint32_t send, uint32_t supertiles,
                                 int max_grid, int max_width, uint64_t* keys, EmitOut eo, Meta* meta,
                                 uint64_t wait_limit, cudaStream_t st);
// Merge passes pass0 .. pass0 + npass - 1 (keys between kA and kB, pass p
// reading kA when p is even); npass > 1 makes one cooperative launch whose
// passes are separated by grid barriers counted on *barrier (zeroed).
cudaError_t launch_merge_pass2(int W, const Segment* segs, uint32_t sbeg, uint32_t send, uint32_t tiles,
                               uint32_t grid, uint32_t pass0, uint32_t npass, uint64_t* kA, uint64_t* kB, EmitOut eo,
                               uint32_t* barrier, Meta* meta, uint64_t wait_limit, cudaStream_t st);
// Pipelined K5 for passes with many tiles: the cut kernel finds every tile's
// slices (one warp per tile), then the merge kernel streams the tiles through
// two shared-memory buffers, loading one while it merges the other.  Each
// merge pass but a bucket's last also stores one key in 32 of its output in
// `samples` (Segment::smp_off), and the next pass's cut searches those first.
cudaError_t launch_merge_cut(int W, const Segment* segs, uint32_t sbeg, uint32_t send, uint32_t tiles, uint32_t pass,
                             const uint64_t* src, const uint64_t* samples, TileJob* jobs, cudaStream_t st);
cudaError_t launch_merge_piped(int W, const TileJob* jobs, uint32_t tiles, uint32_t grid, const uint64_t* src,
                               uint64_t* dst, uint64_t* samples, EmitOut eo, cudaStream_t st);
// CTAs per SM of the pipelined merge kernel.
int merge_piped_ctas_per_sm();
cudaError_t launch_emit(const Segment* segs, uint32_t sbeg, uint32_t send, uint32_t tiles, uint32_t grid,
                        const uint64_t* keysA, const uint64_t* keysB, EmitOut eo, cudaStream_t st);
// The expansion of the duplicate-aware sort: per bucket the exclusive prefix
// of the sorted distinct keys' counts (max_U: the most distinct keys of one
// bucket), then the words, in output tiles of kExpandTileWords / W
// (max_tiles: the most tiles of one bucket; ExpandDesc::tile0 numbers them
// across buckets).  The counts must add up to each bucket's word count; a
// check marks the call failed otherwise.
// Sizes of the buffers the expansion touches (u64 words of each distinct-key
// buffer, u32 entries of the prefixes, stream bytes, offsets, tiles of the
// tile-start table): every descriptor is checked against them.
struct ExpandCaps {
  uint64_t u_words, pre, stream, offsets, tiles;
};
cudaError_t launch_expand(const ExpandDesc* ed, uint32_t nbuckets, uint32_t max_U, uint32_t max_tiles,
                          const uint64_t* uA, const uint64_t* uB, uint32_t* pre, uint32_t* ssum, uint32_t* tfirst,
                          EmitOut eo, Meta* meta, ExpandCaps caps, cudaStream_t st);
// The length order (Table 1): words grouped by length in input order, from
// the word starts, the letters and the (document, length) buckets' places;
// icnt holds items x 256 counts.
cudaError_t launch_length_order(const uint32_t* starts, const uint8_t* letters, const uint32_t* doc_wbase,
                                const uint32_t* doc_item0, uint32_t ndocs, uint32_t items, const uint32_t* seg_lookup,
                                const Segment* segs, uint32_t* icnt, EmitOut eo, cudaStream_t st);
// The whole-text order's words from nb documents' sorted zero-padded keys
// (max_n: the most words of one document); ssum holds nb x var_slices(max_n).
cudaError_t launch_var_emit(const VarDesc* vd, uint32_t nb, uint32_t max_n, const uint64_t* kA, const uint64_t* kB,
                            uint32_t codec, uint32_t* ssum, Meta* meta, EmitOut eo, cudaStream_t st);
size_t var_slices(uint32_t max_n);
// Entries of the slice sums launch_expand needs per bucket (buffer ssum holds
// nbuckets x expand_slices(max_U)); tfirst holds one entry per output tile.
size_t expand_slices(uint32_t max_U);

// ---- K2: the bucket layout ----
// Per (group, column), the sums K2 builds the table from: segments, key
// words, tiles (merge tiles of groups 0..3, tiles of the wide keys), merge
// sample words, first-K4 supertiles (or hash-aggregation units), and the
// duplicate-aware sort's table, array and count words.
enum LayCol { kColCnt, kColKeyw, kColTile, kColSmp, kColStile, kColHtab, kColUniq, kColDcnt, kLayCols };
constexpr int kMovedPasses = 32;  // merge passes the per-pass byte tags cover
// What the host reads back after K2 (through page-locked memory): the
// call-wide decisions, the table's group sizes, the column totals and the
// per-group figures of the launches' tags.
struct LayoutSummary {
  uint32_t nseg;    // buckets in the table
  uint32_t runs;    // K4 run length (tiles) of the buckets that need merge passes
  uint32_t dd;      // 1: groups 0..3 go to the duplicate-aware sort
  uint32_t dd_beg;  // table position of the first bucket of group 0
  uint32_t group_n[kGroups];
  uint32_t max_w[kGroups];       // widest key of the group's K4-sorted buckets
  uint32_t max_passes[kGroups];  // most merge passes of one bucket (groups 0..3, 10, 11)
  uint32_t max_doc_words;        // whole-text order: most words of one document
  uint32_t seg_over;             // buckets that did not fit the table's capacity
  uint32_t pad[2];
  uint64_t big_tiles;  // merge tiles of the buckets of groups 0..3
  uint64_t dd_bytes;   // key bytes the hash aggregation reads
  uint64_t tot[kGroups][kLayCols];
  uint64_t kb[kGroups], ob[kGroups];  // key bytes; output bytes (words and offsets, or keys kept)
  uint64_t k4_bytes[kGroups];         // what K4 moves for the group's buckets
  uint64_t levels[kGroups];           // key-levels of the group's first sort
  uint64_t moved[6][kMovedPasses];    // bytes per merge pass: groups 0..3, then 10, 11
};
static_assert(sizeof(LayoutSummary) % 16 == 0, "the summary travels as 16-byte words");
struct LayoutWork {
  LayoutSummary s;
  uint32_t ticket;      // K2b's CTAs done
  uint32_t pad[3];
  uint32_t barrier[4];  // grid-barrier counters of the four key widths' merge chains
};
struct LayoutParams {
  uint32_t ndocs, order, codec, off_bytes;
  uint32_t k4_runs, k4_runs_small, dedupe, pad;
  uint64_t piped_tiles;  // merge tiles from which the merges are pipelined
  uint32_t seg_cap;      // entries of the segment table and of the slot cursors
  uint32_t dd_cap;       // entries of the hash-insert descriptors and distinct-key counters
};
// Where K2 writes the table: segments (table order), the (document, length)
// -> segment lookup (every entry written), the slot cursors of K3 and the
// distinct-key counters (written zero), the hash-insert descriptors (by
// table position minus dd_beg), the whole-text order's descriptors (by table
// position); blk holds K2's per-CTA sums (layout_scratch_words).
struct LayoutOut {
  Segment* segs;
  uint32_t* lookup;
  uint32_t* cursor;
  uint32_t* ucnt;
  DedupeIns* ins;
  VarDesc* vdesc;
  uint64_t* blk;
};
size_t layout_scratch_words(uint32_t ndocs);
// Kernels launch_layout starts for ndocs documents (one when one CTA holds them all).
int layout_kernels(uint32_t ndocs);
// K2 over the call's documents, after K1: reads the histograms and bases K1
// left (hist, wbase, lbase, maxlen), accumulates into *work (zeroed before the
// launch), and leaves the summary at hm.dst (n16 16-byte words, then seq in
// *hm.flag) as soon as the table's sizes are known, before the table itself
// is written.
cudaError_t launch_layout(const LayoutParams& p, const uint32_t* hist, const uint32_t* wbase, const uint32_t* lbase,
                          const uint32_t* maxlen, LayoutWork* work, LayoutOut out, HostMeta hm, cudaStream_t st);

}  // namespace bsort
