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
// Three launches, one warp per document, kLayDocs documents per CTA:
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
// document, from L2.

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

// One bucket: its group, how it is sorted, and its column values.
struct Bucket {
  uint32_t n, L, W, g, passes, run0;
  bool dd;
  uint64_t col[kLayCols];
};
__device__ __forceinline__ Bucket make_bucket(uint32_t n, uint32_t L, uint32_t W, const Choice& ch) {
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
  if (g < 4)
    st = b.dd ? cdiv(n, dedupe_unit_keys(W)) : cdiv(n, ch.runs * tile2_keys((int)W));
  else if (g >= 5 && g <= 8)
    st = cdiv(n, group_cluster(g) * tile2_keys((int)W));
  b.col[kColStile] = st;
  b.col[kColHtab] = b.dd ? (1ull << ceil_log2_u(2ull * n)) * (W + 1) : 0u;
  b.col[kColUniq] = b.dd ? align16(2 * nw) : 0u;
  b.col[kColDcnt] = (b.dd && W == 1) ? align16(n) : 0u;
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
  if (p.order == BSORT_ORDER_WHOLE) {
    const uint32_t n = wbase[d + 1] - wbase[d];
    const bool has = lane == 0 && n != 0;
    Bucket b{};
    if (has) b = make_bucket(n, Lmax, (uint32_t)key_width(p.codec, Lmax), ch);
    f(has, b, Lmax, has ? n : 0u);
    return;
  }
  for (uint32_t L0 = 1; L0 <= Lmax; L0 += 32) {
    const uint32_t L = L0 + lane;
    const uint32_t n = L <= Lmax ? hist[(size_t)d * kHist + L] : 0u;
    Bucket b{};
    if (n) b = make_bucket(n, L, (uint32_t)key_width(p.codec, L), ch);
    f(n != 0, b, L, n);
  }
}

__device__ __forceinline__ bool doc_live(const LayoutParams& p, uint32_t d, const uint32_t* hist) {
  // a document with a word too long (bin 0) has no buckets: the call fails it
  return d < p.ndocs && hist[(size_t)d * kHist] == 0;
}

// The tags' figures, per CTA (shared-memory atomics), then added to the summary.
struct LayStats {
  unsigned long long kb[kGroups], ob[kGroups], k4_bytes[kGroups], levels[kGroups];
  unsigned long long moved[6][kMovedPasses];
  unsigned long long dd_bytes;
  uint32_t max_w[kGroups], max_passes[kGroups], max_doc_words;
};

__device__ __forceinline__ void account(LayStats& s, const Bucket& b, bool keys_out, uint32_t off_bytes,
                                        const Choice& ch) {
  const int g = (int)b.g;
  const unsigned long long kw = 8ull * b.W * b.n;
  const unsigned long long out = keys_out ? kw : (unsigned long long)b.n * (b.L + off_bytes);
  atomicAdd(&s.kb[g], kw);
  atomicAdd(&s.ob[g], out);
  if (g <= 8 && !b.dd) {
    // K4: keys in, then runs out for the merges or the words out
    const uint64_t super = (uint64_t)(g < 4 ? ch.runs : group_cluster(g)) * tile2_keys((int)b.W);
    atomicAdd(&s.k4_bytes[g], kw + (b.passes ? kw : out));
    atomicAdd(&s.levels[g], (unsigned long long)b.n * ceil_log2_u(b.n < super ? b.n : super));
    atomicMax(&s.max_w[g], b.W);
  } else if (g == 9) {
    atomicAdd(&s.levels[g], (unsigned long long)b.n * ceil_log2_u(b.n));
  } else if (g >= 10) {
    atomicAdd(&s.levels[g], (unsigned long long)b.n * ceil_log2_u(b.n < b.run0 ? b.n : b.run0));
  }
  if (b.dd) atomicAdd(&s.dd_bytes, kw);
  if (g < 4 || g >= 10) atomicMax(&s.max_passes[g], b.passes);
  const int mg = g < 4 ? g : g >= 10 ? g - 6 : -1;
  if (mg >= 0)
    for (uint32_t q = 0; q < b.passes && q < (uint32_t)kMovedPasses; ++q) {
      // keys in; keys out, or the words at the bucket's last pass
      const bool words = g < 4 && q + 1 == b.passes && !keys_out;
      atomicAdd(&s.moved[mg][q], kw + (words ? (unsigned long long)b.n * (b.L + off_bytes) : kw));
    }
  if (keys_out) atomicMax(&s.max_doc_words, b.n);
}

__global__ void __launch_bounds__(kLayThreads) k_layout_tiles(LayoutParams p, const uint32_t* __restrict__ hist,
                                                               const uint32_t* __restrict__ wbase,
                                                               const uint32_t* __restrict__ maxlen, LayoutWork* work) {
  const uint32_t lane = threadIdx.x & 31u, d = blockIdx.x * kLayDocs + (threadIdx.x >> 5);
  unsigned long long bt = 0;
  if (doc_live(p, d, hist)) {
    const uint32_t Lmax = min(maxlen[d], (uint32_t)kMaxLen);
    const Choice any{1u, false};  // the groups do not depend on the choices
    for_doc_buckets(p, any, d, hist, wbase, Lmax, lane, [&](bool has, const Bucket& b, uint32_t, uint32_t) {
      if (has && b.g < 4) bt += b.col[kColTile];
    });
  }
  for (int o = 16; o; o >>= 1) bt += __shfl_xor_sync(0xFFFFFFFFu, bt, o);
  if (lane == 0 && bt) atomicAdd(reinterpret_cast<unsigned long long*>(&work->s.big_tiles), bt);
}

__global__ void __launch_bounds__(kLayThreads) k_layout_sums(LayoutParams p, const uint32_t* __restrict__ hist,
                                                              const uint32_t* __restrict__ wbase,
                                                              const uint32_t* __restrict__ maxlen, LayoutWork* work,
                                                              unsigned long long* blk, HostMeta hm) {
  __shared__ unsigned long long s_slot[kLayDocs][kLayEntries];
  __shared__ LayStats s_st;
  __shared__ unsigned long long s_part[kScanParts][kLayEntries];
  __shared__ unsigned long long s_base[kLayEntries];
  __shared__ bool s_last;
  const uint32_t t = threadIdx.x, lane = t & 31u, warp = t >> 5;
  for (uint32_t i = t; i < (uint32_t)(kLayDocs * kLayEntries); i += kLayThreads) (&s_slot[0][0])[i] = 0;
  for (uint32_t i = t; i < sizeof(LayStats) / 4; i += kLayThreads) reinterpret_cast<uint32_t*>(&s_st)[i] = 0;
  __syncthreads();
  const Choice ch = choose(p, __ldcg(reinterpret_cast<const unsigned long long*>(&work->s.big_tiles)));
  const uint32_t d = blockIdx.x * kLayDocs + warp;
  if (doc_live(p, d, hist)) {
    const uint32_t Lmax = min(maxlen[d], (uint32_t)kMaxLen);
    const bool keys_out = p.order == BSORT_ORDER_WHOLE;
    for_doc_buckets(p, ch, d, hist, wbase, Lmax, lane, [&](bool has, const Bucket& b, uint32_t, uint32_t) {
      if (!has) return;
      for (int c = 0; c < kLayCols; ++c)
        if (b.col[c]) atomicAdd(&s_slot[warp][b.g * kLayCols + c], (unsigned long long)b.col[c]);
      account(s_st, b, keys_out, p.off_bytes, ch);
    });
  }
  __syncthreads();
  if (t < (uint32_t)kLayEntries) {
    unsigned long long v = 0;
    for (int w = 0; w < kLayDocs; ++w) v += s_slot[w][t];
    blk[(size_t)blockIdx.x * kLayEntries + t] = v;
  }
  {
    LayoutSummary& S = work->s;
    for (uint32_t i = t; i < (uint32_t)kGroups; i += kLayThreads) {
      if (s_st.kb[i]) atomicAdd(reinterpret_cast<unsigned long long*>(&S.kb[i]), s_st.kb[i]);
      if (s_st.ob[i]) atomicAdd(reinterpret_cast<unsigned long long*>(&S.ob[i]), s_st.ob[i]);
      if (s_st.k4_bytes[i]) atomicAdd(reinterpret_cast<unsigned long long*>(&S.k4_bytes[i]), s_st.k4_bytes[i]);
      if (s_st.levels[i]) atomicAdd(reinterpret_cast<unsigned long long*>(&S.levels[i]), s_st.levels[i]);
      if (s_st.max_w[i]) atomicMax(&S.max_w[i], s_st.max_w[i]);
      if (s_st.max_passes[i]) atomicMax(&S.max_passes[i], s_st.max_passes[i]);
    }
    for (uint32_t i = t; i < 6u * kMovedPasses; i += kLayThreads) {
      const unsigned long long v = (&s_st.moved[0][0])[i];
      if (v) atomicAdd(reinterpret_cast<unsigned long long*>(&S.moved[0][0]) + i, v);
    }
    if (t == 0 && s_st.dd_bytes) atomicAdd(reinterpret_cast<unsigned long long*>(&S.dd_bytes), s_st.dd_bytes);
    if (t == 0 && s_st.max_doc_words) atomicMax(&S.max_doc_words, s_st.max_doc_words);
  }
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
  __syncthreads();
  LayoutSummary& S = work->s;
  if (t < (uint32_t)kLayEntries) {
    unsigned long long v = 0;
    for (int q = 0; q < kScanParts; ++q) v += s_part[q][t];
    (&S.tot[0][0])[t] = v;
    s_slot[0][t] = v;  // the totals, for the bases below
  }
  __syncthreads();
  if (t == 0) {
    const unsigned long long(*tot)[kLayCols] = reinterpret_cast<const unsigned long long(*)[kLayCols]>(&s_slot[0][0]);
    unsigned long long(*base)[kLayCols] = reinterpret_cast<unsigned long long(*)[kLayCols]>(&s_base[0]);
    for (int i = 0; i < kLayEntries; ++i) s_base[i] = 0;
    int order[kGroups], pos_of[kGroups];
    table_order(ch.runs, order, pos_of);
    unsigned long long pos = 0, keyw = 0;
    for (int q = 0; q < kGroups; ++q) {
      const int g = order[q];
      base[g][kColCnt] = pos;
      pos += tot[g][kColCnt];
      base[g][kColKeyw] = keyw;
      keyw += tot[g][kColKeyw];
    }
    // groups 0..3 sit together in table order, ascending: their sample,
    // hash-table, array, count and unit (or supertile) numbering runs across
    // them; tiles are numbered per group
    unsigned long long acc[kLayCols] = {};
    const int across[5] = {kColSmp, kColStile, kColHtab, kColUniq, kColDcnt};
    for (int g = 0; g < 4; ++g)
      for (int k = 0; k < 5; ++k) {
        const int c = across[k];
        base[g][c] = acc[c];
        acc[c] += tot[g][c];
      }
    // the K4 launch whose clusters make the merge runs covers groups 0..4
    // first (not when they go to the hash aggregation)
    uint64_t ngrp03 = 0;
    for (int g = 0; g < 4; ++g) ngrp03 += tot[g][kColCnt];
    const bool dd = ch.dd && ngrp03 != 0;
    for (int g = 5; g <= 8; ++g)
      if (!dd && group_cluster(g) == ch.runs) base[g][kColStile] = acc[kColStile];
    S.nseg = (uint32_t)pos;
    S.runs = ch.runs;
    S.dd = dd ? 1u : 0u;
    S.dd_beg = (uint32_t)base[0][kColCnt];
    for (int g = 0; g < kGroups; ++g) S.group_n[g] = (uint32_t)tot[g][kColCnt];
    S.seg_over = (pos > p.seg_cap || (dd && ngrp03 > p.dd_cap)) ? 1u : 0u;
  }
  __threadfence();
  __syncthreads();
  // the summary to the host as soon as it is complete: the host sizes the
  // later launches while K2c writes the table
  if (hm.dst) {
    const uint4* src = reinterpret_cast<const uint4*>(&S);
    for (uint32_t i = t; i < hm.n16; i += kLayThreads) hm.dst[i] = __ldcg(src + i);
    __threadfence_system();
    __syncthreads();
    if (t == 0) asm volatile("st.release.sys.global.u32 [%0], %1;" ::"l"(hm.flag), "r"(hm.seq) : "memory");
  }
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

// Exclusive-prefix helper: an inclusive warp scan of a 64-bit value.
__device__ __forceinline__ unsigned long long warp_incl(unsigned long long x, uint32_t lane) {
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long y = __shfl_up_sync(0xFFFFFFFFu, x, o);
    if (lane >= (uint32_t)o) x += y;
  }
  return x;
}

__global__ void __launch_bounds__(kLayThreads) k_layout_write(LayoutParams p, const uint32_t* __restrict__ hist,
                                                               const uint32_t* __restrict__ wbase,
                                                               const uint32_t* __restrict__ lbase,
                                                               const uint32_t* __restrict__ maxlen,
                                                               const LayoutWork* work, LayoutOut out) {
  __shared__ unsigned long long s_slot[kLayDocs][kLayEntries];
  __shared__ unsigned long long s_run[kLayDocs][kLayEntries];
  const uint32_t t = threadIdx.x, lane = t & 31u, warp = t >> 5;
  for (uint32_t i = t; i < (uint32_t)(kLayDocs * kLayEntries); i += kLayThreads) (&s_slot[0][0])[i] = 0;
  __syncthreads();
  const LayoutSummary& S = work->s;
  const Choice ch{S.runs, S.dd != 0};
  const uint32_t dd_beg = S.dd_beg;
  const uint64_t etile11 = S.tot[10][kColTile];  // the wide keys' emit tiles: group 10's first
  const uint32_t d = blockIdx.x * kLayDocs + warp;
  const bool live = doc_live(p, d, hist);
  const uint32_t Lmax = live ? min(maxlen[d], (uint32_t)kMaxLen) : 0u;
  if (live)
    for_doc_buckets(p, ch, d, hist, wbase, Lmax, lane, [&](bool has, const Bucket& b, uint32_t, uint32_t) {
      if (!has) return;
      for (int c = 0; c < kLayCols; ++c)
        if (b.col[c]) atomicAdd(&s_slot[warp][b.g * kLayCols + c], (unsigned long long)b.col[c]);
    });
  __syncthreads();
  // the document's bases: its CTA's, then the documents before it in the CTA
  for (uint32_t i = lane; i < (uint32_t)kLayEntries; i += 32) {
    unsigned long long v = __ldcg(reinterpret_cast<const unsigned long long*>(out.blk) + (size_t)blockIdx.x * kLayEntries + i);
    for (uint32_t w = 0; w < warp; ++w) v += s_slot[w][i];
    s_run[warp][i] = v;
  }
  __syncwarp();
  if (d >= p.ndocs) return;
  uint32_t* lk = out.lookup + (size_t)d * kHist;
  const bool whole = p.order == BSORT_ORDER_WHOLE;
  if (!live) {
    for (uint32_t L = lane; L < (uint32_t)kHist; L += 32) lk[L] = kNoSegment;
    return;
  }
  const uint32_t doc_stream0 = lbase[d];
  uint32_t wrun = wbase[d] + d, brun = doc_stream0;  // the next word's offsets index and stream byte
  uint32_t whole_pos = kNoSegment;
  for_doc_buckets(p, ch, d, hist, wbase, Lmax, lane, [&](bool has, const Bucket& b, uint32_t L, uint32_t n) {
    // the bucket's first word and stream byte: the lengths before it
    uint32_t out_word = wrun, stream_off = brun;
    if (!whole) {
      const unsigned long long in = warp_incl(n, lane), ib = warp_incl((unsigned long long)n * L, lane);
      out_word = wrun + (uint32_t)(in - n);
      stream_off = brun + (uint32_t)(ib - (unsigned long long)n * L);
      wrun += (uint32_t)__shfl_sync(0xFFFFFFFFu, in, 31);
      brun += (uint32_t)__shfl_sync(0xFFFFFFFFu, ib, 31);
    }
    // the bucket's prefixes: the document's running sums of its group, plus
    // the buckets of the same group at lower lanes of this chunk
    unsigned long long pre[kLayCols];
    uint32_t todo = __ballot_sync(0xFFFFFFFFu, has);
    while (todo) {
      const uint32_t gl = __shfl_sync(0xFFFFFFFFu, b.g, __ffs(todo) - 1);
      const bool mine = has && b.g == gl;
      todo &= ~__ballot_sync(0xFFFFFFFFu, mine);
      for (int c = 0; c < kLayCols; ++c) {
        const unsigned long long x = mine ? b.col[c] : 0ull;
        const unsigned long long inc = warp_incl(x, lane);
        unsigned long long* r = &s_run[warp][gl * kLayCols + c];
        if (mine) pre[c] = *r + inc - x;
        const unsigned long long all = __shfl_sync(0xFFFFFFFFu, inc, 31);
        __syncwarp();
        if (lane == 0) *r += all;
        __syncwarp();
      }
    }
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

}  // namespace

size_t layout_scratch_words(uint32_t ndocs) {
  const size_t nblk = ndocs ? (ndocs + kLayDocs - 1) / kLayDocs : 1;
  return nblk * kLayEntries;
}

cudaError_t launch_layout(const LayoutParams& p, const uint32_t* hist, const uint32_t* wbase, const uint32_t* lbase,
                          const uint32_t* maxlen, LayoutWork* work, LayoutOut out, HostMeta hm, cudaStream_t st) {
  const uint32_t grid = p.ndocs ? (p.ndocs + kLayDocs - 1) / kLayDocs : 1u;
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
