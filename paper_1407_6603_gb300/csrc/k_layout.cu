// K2: the bucket layout of a call, on the device.
//
// Paper, Section II (pre-processing phase 2) and Section III (step 3): the
// words are put in one sub-array per number of characters, shorter lengths
// first, each sub-array as large as the number of words of its length.  Here
// such a sub-array is a (document, length) bucket with words: one Segment in a
// table that every later kernel reads.  The table is ordered by the kernels
// that sort the buckets (sort_group, table_order), so that each launch covers
// a contiguous range of it, and every field that numbers something across
// buckets (first key word, first tile, first supertile, ...) is an exclusive
// prefix sum in table order.
//
// One warp per document, kLayDocs documents per CTA, in three launches:
//   K2a  the merge tiles of the buckets that need merge passes, summed: the
//        run length K4 leaves and the choice of the duplicate-aware sort
//        follow from that total (choose);
//   K2b  per CTA and (group, column), the sums of its documents' buckets,
//        and the figures of the launches' tags; its last CTA scans the CTA
//        sums, places the groups in table order, folds the group bases into
//        the scan and hands the summary to the host;
//   K2c  each bucket's prefixes = its CTA's scanned base + the documents
//        before it in its CTA + the lengths before it in its document; writes
//        the segment, the lookup entries and the descriptors.
// K2a and K2c read every document's histogram once more than K2b: 1 KiB per
// document, from L2.  When one CTA holds every document, the three phases
// run in one launch (k_layout_one), separated by barriers.
// Inside a warp, lane l holds the bucket of length L0 + l of a chunk of 32
// lengths; the sums and prefixes over the chunk's buckets of one group are
// taken by a sweep of shuffles over the lanes that hold a bucket (peer_sums),
// without atomics.

#include "bsort_dev.cuh"

namespace bsort {
namespace {

constexpr int kLayDocs = 16;
constexpr int kLayThreads = 32 * kLayDocs;
constexpr int kLayEntries = kGroups * kLayCols;
constexpr int kScanParts = kLayThreads / kLayEntries;  // threads per column in the scan
static_assert(kScanParts >= 1, "one thread per (group, column) at least");

__device__ __forceinline__ uint32_t cdiv(uint32_t a, uint32_t b) { return a / b + (a % b != 0u); }
__device__ __forceinline__ uint64_t align16(uint64_t x) { return (x + 15) & ~15ull; }

// The call-wide choices, from the merge tiles of groups 0..3: with enough of
// them for the merges to be pipelined, runs of k4_runs tiles (the passes run
// at HBM speed), else k4_runs_small (fewer passes and launches); and the
// duplicate-aware sort for the same large inputs (dedupe = 1) or always (2),
// for the orders whose buckets hold one length.
struct Choice {
  uint32_t runs;
  bool dd;
};
__device__ __forceinline__ Choice choose(const LayoutParams& p, uint64_t big_tiles) {
  const bool piped = big_tiles >= p.piped_tiles;
  Choice c;
  c.runs = piped ? p.k4_runs : p.k4_runs_small;
  c.dd = p.order <= BSORT_ORDER_FOLDED && (p.dedupe == 2 || (p.dedupe == 1 && piped));
  return c;
}

// The columns a bucket contributes to: the layout's (kLayCols), then the
// tags' figures: key bytes, output bytes, the bytes K4 moves for it, its
// key-levels in its first sort.
enum { kColKb = kLayCols, kColOb, kColK4, kColLev, kSlotCols };
constexpr int kSlotEntries = kGroups * kSlotCols;

// One bucket: its group, how it is sorted, and its column values.
struct Bucket {
  uint32_t n, L, W, g, passes, run0;
  bool dd;
  uint64_t col[kSlotCols];
};
__device__ __forceinline__ Bucket make_bucket(uint32_t n, uint32_t L, uint32_t W, const Choice& ch, bool keys_out,
                                              uint32_t off_bytes) {
  Bucket b;
  b.n = n;
  b.L = L;
  b.W = W;
  const int g = sort_group(n, (int)W);
  b.g = (uint32_t)g;
  b.dd = g < 4 && ch.dd;
  if (g >= 10) {
    b.run0 = (uint32_t)tile_of_width((int)W);
    b.passes = merge_passes(n, b.run0);
  } else if (g < 4) {
    b.run0 = ch.runs * tile2_keys((int)W);
    b.passes = b.dd ? 0u : merge_passes(n, b.run0);
  } else {
    b.run0 = n;
    b.passes = 0;
  }
  const uint64_t nw = (uint64_t)n * W;
  b.col[kColCnt] = 1;
  b.col[kColKeyw] = align16(nw);
  b.col[kColTile] = g < 4 ? cdiv(n, merge2_keys((int)W)) : g >= 10 ? cdiv(n, b.run0) : 0u;
  b.col[kColSmp] = (g < 4 && b.passes) ? (uint64_t)cdiv(n, 32u) * W : 0u;
  uint64_t st = 0;
  uint32_t super = 0;  // keys of one K4 supertile
  if (g < 4) {
    super = ch.runs * tile2_keys((int)W);
    st = b.dd ? cdiv(n, dedupe_unit_keys(W)) : cdiv(n, super);
  } else if (g >= 5 && g <= 8) {
    super = group_cluster(g) * tile2_keys((int)W);
    st = cdiv(n, super);
  }
  b.col[kColStile] = st;
  b.col[kColHtab] = b.dd ? (1ull << ceil_log2_u(2ull * n)) * (W + 1) : 0u;
  b.col[kColUniq] = b.dd ? align16(2 * nw) : 0u;
  b.col[kColDcnt] = (b.dd && W == 1) ? align16(n) : 0u;
  const uint64_t kw = 8 * nw;
  const uint64_t out = keys_out ? kw : (uint64_t)n * (L + off_bytes);
  b.col[kColKb] = kw;
  b.col[kColOb] = out;
  const bool k4 = g <= 8 && !b.dd;  // K4 sorts it: keys in, then runs out for the merges or the words out
  b.col[kColK4] = k4 ? kw + (b.passes ? kw : out) : 0u;
  b.col[kColLev] = k4        ? (uint64_t)n * ceil_log2_u(n < super ? n : super)
                   : g == 9  ? (uint64_t)n * ceil_log2_u(n)
                   : g >= 10 ? (uint64_t)n * ceil_log2_u(n < b.run0 ? n : b.run0)
                             : 0u;
  return b;
}

// A document's buckets, a chunk of 32 lengths at a time (lane l holds length
// L0 + l), in order: f(has, bucket, L, n) on every lane of the warp, once per
// chunk.  The whole-text order has one bucket per document (lane 0): every
// word, keys padded to the longest.
template <class F>
__device__ __forceinline__ void for_doc_buckets(const LayoutParams& p, const Choice& ch, uint32_t d,
                                                const uint32_t* hist, const uint32_t* wbase, uint32_t Lmax,
                                                uint32_t lane, F&& f) {
  const bool keys_out = p.order == BSORT_ORDER_WHOLE;
  if (keys_out) {
    const uint32_t n = wbase[d + 1] - wbase[d];
    const bool has = lane == 0 && n != 0;
    Bucket b{};
    if (has) b = make_bucket(n, Lmax, (uint32_t)key_width(p.codec, Lmax), ch, true, p.off_bytes);
    f(has, b, Lmax, has ? n : 0u);
    return;
  }
  for (uint32_t L0 = 1; L0 <= Lmax; L0 += 32) {
    const uint32_t L = L0 + lane;
    const uint32_t n = L <= Lmax ? hist[(size_t)d * kHist + L] : 0u;
    Bucket b{};
    if (n) b = make_bucket(n, L, (uint32_t)key_width(p.codec, L), ch, false, p.off_bytes);
    f(n != 0, b, L, n);
  }
}

__device__ __forceinline__ bool doc_live(const LayoutParams& p, uint32_t d, const uint32_t* hist) {
  // a document with a word too long (bin 0) has no buckets: the call fails it
  return d < p.ndocs && hist[(size_t)d * kHist] == 0;
}

// Over the lanes that hold a bucket of this lane's group (has, g): the sums
// of the first NC columns of x at the lanes below it (pre, when want_pre)
// and at all of them (tot).  `leader` is set on the lowest such lane.
template <int NC, bool want_pre>
__device__ __forceinline__ void peer_sums(bool has, uint32_t g, uint32_t lane, const uint64_t* x, uint64_t* pre,
                                          uint64_t* tot, bool& leader) {
  const uint32_t any = __ballot_sync(0xFFFFFFFFu, has);
  const uint32_t peers = __match_any_sync(0xFFFFFFFFu, has ? g : 0xFFFFFFFFu);
  const uint32_t mine = has ? peers : 0u;
  const uint32_t below = mine & ((1u << lane) - 1u);
  leader = has && (below == 0);
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    tot[c] = 0;
    if (want_pre) pre[c] = 0;
  }
  for (uint32_t m = any; m; m &= m - 1) {
    const int j = __ffs((int)m) - 1;
    const bool in = (mine >> j) & 1u, lo = (below >> j) & 1u;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      const uint64_t v = __shfl_sync(0xFFFFFFFFu, x[c], j);
      if (in) tot[c] += v;
      if (want_pre && lo) pre[c] += v;
    }
  }
}

// Per-CTA maxima of the tags' figures (shared-memory atomics on 32-bit words).
struct LayMax {
  uint32_t max_w[kGroups], max_passes[kGroups], max_doc_words;
};

// K2a's part for one document: its merge tiles of groups 0..3 (warp-summed).
__device__ __forceinline__ uint64_t doc_tiles(const LayoutParams& p, uint32_t d, const uint32_t* hist,
                                              const uint32_t* wbase, const uint32_t* maxlen, uint32_t lane) {
  uint64_t bt = 0;
  if (doc_live(p, d, hist)) {
    const uint32_t Lmax = min(maxlen[d], (uint32_t)kMaxLen);
    const Choice any{1u, false};  // the groups do not depend on the choices
    for_doc_buckets(p, any, d, hist, wbase, Lmax, lane, [&](bool has, const Bucket& b, uint32_t, uint32_t) {
      if (has && b.g < 4) bt += b.col[kColTile];
    });
  }
  for (int o = 16; o; o >>= 1) bt += __shfl_xor_sync(0xFFFFFFFFu, bt, o);
  return bt;
}

// K2b's part for one document: its sums per (group, column) into slot (this
// warp's), with_stats: the maxima into mx and the per-pass merge bytes into
// the summary (global atomics: only buckets with merge passes have them).
template <bool with_stats>
__device__ __forceinline__ void doc_sums(const LayoutParams& p, const Choice& ch, uint32_t d, const uint32_t* hist,
                                         const uint32_t* wbase, const uint32_t* maxlen, uint32_t lane,
                                         unsigned long long* slot, LayMax* mx, LayoutSummary* S) {
  if (!doc_live(p, d, hist)) return;
  const uint32_t Lmax = min(maxlen[d], (uint32_t)kMaxLen);
  const bool keys_out = p.order == BSORT_ORDER_WHOLE;
  constexpr int NC = with_stats ? kSlotCols : kLayCols;
  for_doc_buckets(p, ch, d, hist, wbase, Lmax, lane, [&](bool has, const Bucket& b, uint32_t, uint32_t) {
    uint64_t tot[NC];
    bool leader;
    peer_sums<NC, false>(has, b.g, lane, b.col, nullptr, tot, leader);
    if (leader) {
#pragma unroll
      for (int c = 0; c < NC; ++c) slot[b.g * kSlotCols + c] += tot[c];
    }
    __syncwarp();
    if (!with_stats || !has) return;
    const int g = (int)b.g;
    if (g <= 8 && !b.dd) atomicMax(&mx->max_w[g], b.W);
    if (g < 4 || g >= 10) atomicMax(&mx->max_passes[g], b.passes);
    if (keys_out) atomicMax(&mx->max_doc_words, b.n);
    const int mg = g < 4 ? g : g >= 10 ? g - 6 : -1;
    if (mg >= 0) {
      const uint64_t kw = b.col[kColKb];
      for (uint32_t q = 0; q < b.passes && q < (uint32_t)kMovedPasses; ++q) {
        // keys in; keys out, or the words at the bucket's last pass
        const bool words = g < 4 && q + 1 == b.passes && !keys_out;
        atomicAdd(reinterpret_cast<unsigned long long*>(&S->moved[mg][q]),
                  (unsigned long long)(kw + (words ? b.col[kColOb] : kw)));
      }
    }
  });
}

// Threads 0..kGroups-1 of the CTA that knows the totals (thread g for group
// g): the groups' table order, each (group, column) base (into base), and
// the summary's scalars (thread 0).  tot holds the layout columns' totals
// per group, kb the key bytes per group.  The caller synchronizes after.
__device__ void plan_groups(const LayoutParams& p, const Choice& ch, const unsigned long long* tot_flat,
                            const unsigned long long* kb, unsigned long long* base_flat, LayoutSummary& S) {
  const int g = (int)threadIdx.x;
  if (g >= kGroups) return;
  const unsigned long long(*tot)[kLayCols] = reinterpret_cast<const unsigned long long(*)[kLayCols]>(tot_flat);
  unsigned long long* base = base_flat + g * kLayCols;
  int order[kGroups], pos_of[kGroups];
  table_order(ch.runs, order, pos_of);
  // segments and key words run across the whole table
  unsigned long long pos = 0, keyw = 0;
  for (int q = 0; q < pos_of[g]; ++q) {
    pos += tot[order[q]][kColCnt];
    keyw += tot[order[q]][kColKeyw];
  }
  for (int c = 0; c < kLayCols; ++c) base[c] = 0;
  base[kColCnt] = pos;
  base[kColKeyw] = keyw;
  // groups 0..3 sit together in table order, ascending: their sample,
  // hash-table, array, count and unit (or supertile) numbering runs across
  // them; tiles are numbered per group
  unsigned long long acc[kLayCols] = {};
  uint64_t ngrp03 = 0, dd_bytes = 0;
  for (int h = 0; h < 4; ++h) {
    if (h < g)
      for (int c = kColSmp; c <= kColDcnt; ++c) acc[c] += tot[h][c];
    ngrp03 += tot[h][kColCnt];
    dd_bytes += kb[h];
  }
  const bool dd = ch.dd && ngrp03 != 0;
  if (g < 4) {
    for (int c = kColSmp; c <= kColDcnt; ++c) base[c] = acc[c];
  } else if (g >= 5 && g <= 8 && !dd && group_cluster(g) == ch.runs) {
    // the K4 launch whose clusters make the merge runs covers groups 0..4
    // first (not when they go to the hash aggregation)
    for (int h = 0; h < 4; ++h) base[kColStile] += tot[h][kColStile];
  }
  S.group_n[g] = (uint32_t)tot[g][kColCnt];
  if (g != 0) return;
  unsigned long long nseg = 0;
  for (int h = 0; h < kGroups; ++h) nseg += tot[h][kColCnt];
  S.nseg = (uint32_t)nseg;
  S.runs = ch.runs;
  S.dd = dd ? 1u : 0u;
  S.dd_beg = (uint32_t)pos;  // group 0's first position
  S.dd_bytes = dd ? dd_bytes : 0u;
  S.seg_over = (nseg > p.seg_cap || (dd && ngrp03 > p.dd_cap)) ? 1u : 0u;
}

// The summary (complete in S, in L2) to the host, then the flag it waits on.
__device__ __forceinline__ void send_summary(const LayoutSummary& S, const HostMeta& hm) {
  __threadfence();
  __syncthreads();
  if (!hm.dst) return;
  const uint4* src = reinterpret_cast<const uint4*>(&S);
  for (uint32_t i = threadIdx.x; i < hm.n16; i += blockDim.x) hm.dst[i] = __ldcg(src + i);
  __threadfence_system();
  __syncthreads();
  if (threadIdx.x == 0) asm volatile("st.release.sys.global.u32 [%0], %1;" ::"l"(hm.flag), "r"(hm.seq) : "memory");
}

// Exclusive-prefix helper: an inclusive warp scan.
__device__ __forceinline__ uint32_t warp_incl32(uint32_t x, uint32_t lane) {
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
    if (lane >= (uint32_t)o) x += y;
  }
  return x;
}

// K2c's part for one document (d < ndocs): run holds this warp's running
// prefixes per (group, layout column), starting at the document's bases.
__device__ __forceinline__ void doc_write(const LayoutParams& p, const Choice& ch, uint32_t dd_beg, uint64_t etile11,
                                          uint32_t d, const uint32_t* hist, const uint32_t* wbase, const uint32_t* lbase,
                                          const uint32_t* maxlen, uint32_t lane, unsigned long long* run,
                                          const LayoutOut& out) {
  uint32_t* lk = out.lookup + (size_t)d * kHist;
  if (!doc_live(p, d, hist)) {
    for (uint32_t L = lane; L < (uint32_t)kHist; L += 32) lk[L] = kNoSegment;
    return;
  }
  const bool whole = p.order == BSORT_ORDER_WHOLE;
  const uint32_t Lmax = min(maxlen[d], (uint32_t)kMaxLen);
  const uint32_t doc_stream0 = lbase[d];
  uint32_t wrun = wbase[d] + d, brun = doc_stream0;  // the next word's offsets index and stream byte
  uint32_t whole_pos = kNoSegment;
  for_doc_buckets(p, ch, d, hist, wbase, Lmax, lane, [&](bool has, const Bucket& b, uint32_t L, uint32_t n) {
    // the bucket's first word and stream byte: the lengths before it
    uint32_t out_word = wrun, stream_off = brun;
    if (!whole) {
      const uint32_t in = warp_incl32(n, lane), ib = warp_incl32(n * L, lane);
      out_word = wrun + (in - n);
      stream_off = brun + (ib - n * L);
      wrun += __shfl_sync(0xFFFFFFFFu, in, 31);
      brun += __shfl_sync(0xFFFFFFFFu, ib, 31);
    }
    // the bucket's prefixes: the document's running sums of its group, plus
    // the buckets of the same group at lower lanes of this chunk
    uint64_t pre[kLayCols], tot[kLayCols];
    bool leader;
    peer_sums<kLayCols, true>(has, b.g, lane, b.col, pre, tot, leader);
    if (has) {
#pragma unroll
      for (int c = 0; c < kLayCols; ++c) pre[c] += run[b.g * kLayCols + c];
    }
    __syncwarp();
    if (leader) {
#pragma unroll
      for (int c = 0; c < kLayCols; ++c) run[b.g * kLayCols + c] += tot[c];
    }
    __syncwarp();
    if (!whole && L < (uint32_t)kHist) lk[L] = has ? (uint32_t)pre[kColCnt] : kNoSegment;
    if (!has) return;
    const uint32_t pos = (uint32_t)pre[kColCnt];
    if (whole) whole_pos = pos;
    if (pos >= p.seg_cap) return;  // the summary reports it; the call fails
    const int g = (int)b.g;
    Segment sg{};
    sg.key_off = pre[kColKeyw];
    sg.n = b.n;
    sg.L = b.L;
    sg.doc = d;
    sg.tile0 = (g < 4 || g >= 10) ? (uint32_t)pre[kColTile] : 0u;
    sg.etile0 = g >= 10 ? (uint32_t)(pre[kColTile] + (g == 11 ? etile11 : 0ull)) : 0u;
    sg.stile0 = (g < 4 || (g >= 5 && g <= 8)) ? (uint32_t)pre[kColStile] : 0u;
    sg.out_word = out_word;
    sg.stream_off = stream_off;
    sg.doc_stream0 = doc_stream0;
    sg.passes = b.passes;
    sg.final_buf = b.passes & 1u;
    sg.run0 = b.run0;
    sg.smp_off = (g < 4 && b.passes) ? (uint32_t)pre[kColSmp] : 0u;
    sg.flags = whole ? kSegKeysOut : 0u;
    sg.W = b.W;
    out.cursor[pos] = 0;
    if (b.dd) {
      const uint32_t di = pos - dd_beg;
      if (di < p.dd_cap) {
        sg.flags |= kSegDedupe | (di << 8);
        DedupeIns in{};
        in.htab_off = pre[kColHtab];
        in.uniq_off = pre[kColUniq];
        in.cnt_off = pre[kColDcnt];
        in.hbits = ceil_log2_u(2ull * b.n);
        in.Wp = 2 * b.W;
        in.n = b.n;
        out.ins[di] = in;
        out.ucnt[di] = 0;
      }
    }
    out.segs[pos] = sg;
    if (whole) {
      VarDesc v{};
      v.key_off = sg.key_off;
      v.n = b.n;
      v.W = b.W;
      v.final_buf = sg.final_buf;
      v.letters = lbase[d + 1] - doc_stream0;
      v.out_word = out_word;
      v.stream_off = stream_off;
      v.doc_stream0 = doc_stream0;
      out.vdesc[pos] = v;
    }
  });
  if (whole) {
    // every length of the document maps to its one bucket
    whole_pos = __shfl_sync(0xFFFFFFFFu, whole_pos, 0);
    for (uint32_t L = lane; L < (uint32_t)kHist; L += 32)
      lk[L] = (whole_pos != kNoSegment && L >= 1 && L <= Lmax && hist[(size_t)d * kHist + L]) ? whole_pos : kNoSegment;
  } else {
    // lengths 0 and above the longest word: no bucket
    for (uint32_t L = lane; L < (uint32_t)kHist; L += 32)
      if (L == 0 || L > Lmax) lk[L] = kNoSegment;
  }
}

__device__ __forceinline__ void clear_shared(unsigned long long* a, uint32_t n) {
  for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) a[i] = 0;
}

__global__ void __launch_bounds__(kLayThreads) k_layout_tiles(LayoutParams p, const uint32_t* __restrict__ hist,
                                                               const uint32_t* __restrict__ wbase,
                                                               const uint32_t* __restrict__ maxlen, LayoutWork* work) {
  const uint32_t lane = threadIdx.x & 31u, d = blockIdx.x * kLayDocs + (threadIdx.x >> 5);
  const uint64_t bt = doc_tiles(p, d, hist, wbase, maxlen, lane);
  if (lane == 0 && bt) atomicAdd(reinterpret_cast<unsigned long long*>(&work->s.big_tiles), (unsigned long long)bt);
}

__global__ void __launch_bounds__(kLayThreads) k_layout_sums(LayoutParams p, const uint32_t* __restrict__ hist,
                                                              const uint32_t* __restrict__ wbase,
                                                              const uint32_t* __restrict__ maxlen, LayoutWork* work,
                                                              unsigned long long* blk, HostMeta hm) {
  __shared__ unsigned long long s_slot[kLayDocs][kSlotEntries];
  __shared__ LayMax s_mx;
  __shared__ unsigned long long s_part[kScanParts][kLayEntries];
  __shared__ unsigned long long s_tot[kLayEntries];
  __shared__ unsigned long long s_base[kLayEntries];
  __shared__ unsigned long long s_kb[kGroups];
  __shared__ bool s_last;
  const uint32_t t = threadIdx.x, lane = t & 31u, warp = t >> 5;
  clear_shared(&s_slot[0][0], kLayDocs * kSlotEntries);
  for (uint32_t i = t; i < sizeof(LayMax) / 4; i += kLayThreads) reinterpret_cast<uint32_t*>(&s_mx)[i] = 0;
  __syncthreads();
  LayoutSummary& S = work->s;
  const Choice ch = choose(p, __ldcg(reinterpret_cast<const unsigned long long*>(&S.big_tiles)));
  doc_sums<true>(p, ch, blockIdx.x * kLayDocs + warp, hist, wbase, maxlen, lane, s_slot[warp], &s_mx, &S);
  __syncthreads();
  // the CTA's sums: the layout columns to blk, the tags' figures to the summary
  for (uint32_t i = t; i < (uint32_t)kSlotEntries; i += kLayThreads) {
    unsigned long long v = 0;
    for (int w = 0; w < kLayDocs; ++w) v += s_slot[w][i];
    const uint32_t g = i / kSlotCols, c = i % kSlotCols;
    if (c < (uint32_t)kLayCols) {
      blk[(size_t)blockIdx.x * kLayEntries + g * kLayCols + c] = v;
    } else if (v) {
      unsigned long long* dst = reinterpret_cast<unsigned long long*>(
          c == kColKb ? S.kb : c == kColOb ? S.ob : c == kColK4 ? S.k4_bytes : S.levels);
      atomicAdd(dst + g, v);
    }
  }
  for (uint32_t i = t; i < (uint32_t)kGroups; i += kLayThreads) {
    if (s_mx.max_w[i]) atomicMax(&S.max_w[i], s_mx.max_w[i]);
    if (s_mx.max_passes[i]) atomicMax(&S.max_passes[i], s_mx.max_passes[i]);
  }
  if (t == 0 && s_mx.max_doc_words) atomicMax(&S.max_doc_words, s_mx.max_doc_words);
  __threadfence();
  __syncthreads();
  if (t == 0) s_last = atomicAdd(&work->ticket, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!s_last) return;
  __threadfence();

  // ---- the last CTA: scan the CTA sums per (group, column) ----
  const uint32_t nblk = gridDim.x;
  const uint32_t per = (nblk + kScanParts - 1) / kScanParts;
  const uint32_t e = t % kLayEntries, part = t / kLayEntries;
  const bool scans = part < (uint32_t)kScanParts;
  const uint32_t b0 = scans ? min(part * per, nblk) : 0u, b1 = scans ? min(b0 + per, nblk) : 0u;
  if (scans) {
    unsigned long long v = 0;
    for (uint32_t b = b0; b < b1; ++b) v += __ldcg(blk + (size_t)b * kLayEntries + e);
    s_part[part][e] = v;
  }
  if (t < (uint32_t)kGroups) s_kb[t] = __ldcg(reinterpret_cast<const unsigned long long*>(&S.kb[t]));
  __syncthreads();
  if (t < (uint32_t)kLayEntries) {
    unsigned long long v = 0;
    for (int q = 0; q < kScanParts; ++q) v += s_part[q][t];
    (&S.tot[0][0])[t] = v;
    s_tot[t] = v;
  }
  __syncthreads();
  plan_groups(p, ch, s_tot, s_kb, s_base, S);
  // the summary to the host as soon as it is complete: the host sizes the
  // later launches while K2c writes the table
  send_summary(S, hm);
  // every CTA's exclusive prefix, with its group base
  if (scans) {
    unsigned long long v = s_base[e];
    for (int q = 0; q < (int)part; ++q) v += s_part[q][e];
    for (uint32_t b = b0; b < b1; ++b) {
      unsigned long long* x = blk + (size_t)b * kLayEntries + e;
      const unsigned long long own = __ldcg(x);
      *x = v;
      v += own;
    }
  }
}

__global__ void __launch_bounds__(kLayThreads) k_layout_write(LayoutParams p, const uint32_t* __restrict__ hist,
                                                               const uint32_t* __restrict__ wbase,
                                                               const uint32_t* __restrict__ lbase,
                                                               const uint32_t* __restrict__ maxlen,
                                                               const LayoutWork* work, LayoutOut out) {
  __shared__ unsigned long long s_slot[kLayDocs][kSlotEntries];
  __shared__ unsigned long long s_run[kLayDocs][kLayEntries];
  const uint32_t t = threadIdx.x, lane = t & 31u, warp = t >> 5;
  clear_shared(&s_slot[0][0], kLayDocs * kSlotEntries);
  __syncthreads();
  const LayoutSummary& S = work->s;
  const Choice ch{S.runs, S.dd != 0};
  const uint32_t d = blockIdx.x * kLayDocs + warp;
  doc_sums<false>(p, ch, d, hist, wbase, maxlen, lane, s_slot[warp], nullptr, nullptr);
  __syncthreads();
  // the document's bases: its CTA's, then the documents before it in the CTA
  for (uint32_t i = lane; i < (uint32_t)kLayEntries; i += 32) {
    const uint32_t g = i / kLayCols, c = i % kLayCols;
    unsigned long long v = __ldcg(reinterpret_cast<const unsigned long long*>(out.blk) + (size_t)blockIdx.x * kLayEntries + i);
    for (uint32_t w = 0; w < warp; ++w) v += s_slot[w][g * kSlotCols + c];
    s_run[warp][i] = v;
  }
  __syncwarp();
  if (d < p.ndocs) doc_write(p, ch, S.dd_beg, S.tot[10][kColTile], d, hist, wbase, lbase, maxlen, lane, s_run[warp], out);
}

// All three phases in one CTA (every document in it): no scratch, no ticket.
// The summary is built in shared memory and stored from there to the host
// and to the work area.
__global__ void __launch_bounds__(kLayThreads) k_layout_one(LayoutParams p, const uint32_t* __restrict__ hist,
                                                             const uint32_t* __restrict__ wbase,
                                                             const uint32_t* __restrict__ lbase,
                                                             const uint32_t* __restrict__ maxlen, LayoutWork* work,
                                                             LayoutOut out, HostMeta hm) {
  __shared__ unsigned long long s_slot[kLayDocs][kSlotEntries];
  __shared__ unsigned long long s_run[kLayDocs][kLayEntries];
  __shared__ unsigned long long s_tot[kLayEntries];
  __shared__ unsigned long long s_base[kLayEntries];
  __shared__ unsigned long long s_kb[kGroups];
  __shared__ unsigned long long s_bt[kLayDocs];
  __shared__ LayMax s_mx;
  __shared__ __align__(16) LayoutSummary s_S;  // (copied as 16-byte words)
  const uint32_t t = threadIdx.x, lane = t & 31u, warp = t >> 5, d = warp;
  clear_shared(&s_slot[0][0], kLayDocs * kSlotEntries);
  for (uint32_t i = t; i < sizeof(LayMax) / 4; i += kLayThreads) reinterpret_cast<uint32_t*>(&s_mx)[i] = 0;
  for (uint32_t i = t; i < sizeof(LayoutSummary) / 16; i += kLayThreads)
    reinterpret_cast<uint4*>(&s_S)[i] = make_uint4(0, 0, 0, 0);
  const uint64_t bt = doc_tiles(p, d, hist, wbase, maxlen, lane);
  if (lane == 0) s_bt[warp] = bt;
  __syncthreads();
  unsigned long long big = 0;
  for (int w = 0; w < kLayDocs; ++w) big += s_bt[w];
  const Choice ch = choose(p, big);
  LayoutSummary& S = s_S;
  doc_sums<true>(p, ch, d, hist, wbase, maxlen, lane, s_slot[warp], &s_mx, &S);
  __syncthreads();
  for (uint32_t i = t; i < (uint32_t)kSlotEntries; i += kLayThreads) {
    unsigned long long v = 0;
    for (int w = 0; w < kLayDocs; ++w) v += s_slot[w][i];
    const uint32_t g = i / kSlotCols, c = i % kSlotCols;
    if (c < (uint32_t)kLayCols) {
      s_tot[g * kLayCols + c] = v;
      S.tot[g][c] = v;
    } else if (c == kColKb) {
      S.kb[g] = v;
      s_kb[g] = v;
    } else if (c == kColOb) {
      S.ob[g] = v;
    } else if (c == kColK4) {
      S.k4_bytes[g] = v;
    } else {
      S.levels[g] = v;
    }
  }
  for (uint32_t i = t; i < (uint32_t)kGroups; i += kLayThreads) {
    S.max_w[i] = s_mx.max_w[i];
    S.max_passes[i] = s_mx.max_passes[i];
  }
  if (t == 0) {
    S.max_doc_words = s_mx.max_doc_words;
    S.big_tiles = big;
  }
  __syncthreads();
  plan_groups(p, ch, s_tot, s_kb, s_base, S);
  __syncthreads();
  {
    // the summary to the work area and to the host, then the flag
    const uint4* src = reinterpret_cast<const uint4*>(&S);
    uint4* dev = reinterpret_cast<uint4*>(&work->s);
    constexpr uint32_t n16 = sizeof(LayoutSummary) / 16;
    for (uint32_t i = t; i < n16; i += kLayThreads) {
      const uint4 v = src[i];
      dev[i] = v;
      if (hm.dst && i < hm.n16) hm.dst[i] = v;
    }
    if (hm.dst) {
      __threadfence_system();
      __syncthreads();
      if (t == 0) asm volatile("st.release.sys.global.u32 [%0], %1;" ::"l"(hm.flag), "r"(hm.seq) : "memory");
    }
  }
  // the documents' bases: the group bases, then the documents before each
  for (uint32_t i = lane; i < (uint32_t)kLayEntries; i += 32) {
    const uint32_t g = i / kLayCols, c = i % kLayCols;
    unsigned long long v = s_base[i];
    for (uint32_t w = 0; w < warp; ++w) v += s_slot[w][g * kSlotCols + c];
    s_run[warp][i] = v;
  }
  __syncwarp();
  const Choice ch2{ch.runs, S.dd != 0};
  if (d < p.ndocs) doc_write(p, ch2, S.dd_beg, s_tot[10 * kLayCols + kColTile], d, hist, wbase, lbase, maxlen, lane,
                             s_run[warp], out);
}

}  // namespace

size_t layout_scratch_words(uint32_t ndocs) {
  const size_t nblk = ndocs ? (ndocs + kLayDocs - 1) / kLayDocs : 1;
  return nblk * kLayEntries;
}

int layout_kernels(uint32_t ndocs) { return ndocs <= (uint32_t)kLayDocs ? 1 : 3; }

cudaError_t launch_layout(const LayoutParams& p, const uint32_t* hist, const uint32_t* wbase, const uint32_t* lbase,
                          const uint32_t* maxlen, LayoutWork* work, LayoutOut out, HostMeta hm, cudaStream_t st) {
  if (p.ndocs <= (uint32_t)kLayDocs) {
    k_layout_one<<<1, kLayThreads, 0, st>>>(p, hist, wbase, lbase, maxlen, work, out, hm);
    return cudaGetLastError();
  }
  const uint32_t grid = (p.ndocs + kLayDocs - 1) / kLayDocs;
  k_layout_tiles<<<grid, kLayThreads, 0, st>>>(p, hist, wbase, maxlen, work);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_layout_sums<<<grid, kLayThreads, 0, st>>>(p, hist, wbase, maxlen, work,
                                               reinterpret_cast<unsigned long long*>(out.blk), hm);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_layout_write<<<grid, kLayThreads, 0, st>>>(p, hist, wbase, lbase, maxlen, work, out);
  return cudaGetLastError();
}

}  // namespace bsort
