// K1 in one pass: strip + tokenize + per-document length histogram.
//
// Phase 1 of the paper's pre-processing (Section II; Section III step 2) and
// the counts that phase 2 sizes its sub-arrays with, in one kernel: each CTA
// takes the next 16 KiB chunk from a ticket counter, classifies its bytes
// (letters, whitespace, others), publishes its chunk summary, looks back over
// its predecessors' records until one holds an inclusive prefix (decoupled
// look-back), publishes its own, then writes its letters to S and the S
// offset of every word start.  Tickets are handed out in the order CTAs
// start, so a CTA only ever waits for chunks that running CTAs hold; each
// wait is still bounded and a wait that runs out marks the call as timed out.
//
// Lengths: the thread that holds a word start also knows the start before it
// (carried through the scan as "last start, and its document"), so it emits
// the length of the previous word; the last word of all is emitted by the
// CTA that finishes last.  That CTA also derives each document's word and
// letter bases from the chunk prefixes and the prefix of 2048-word blocks.
#include <cstddef>

#include "bsort_dev.cuh"
#include "tok_common.cuh"

namespace bsort {
namespace {

constexpr uint32_t kHas = 8u;  // the span holds a decided word start

// Scan element: TokSum extended with the last decided word start.
//   fl   bits 0..3: EV WS U HAS; bits 4..31: document of the span's first
//        letter-or-space byte (the document of a start that U may become)
//   last letter offset, within the span, of its last decided word start
//   ldoc document of that start
struct TokAcc {
  uint32_t letters;
  uint32_t words;
  uint32_t fl;
  uint32_t last;
  uint32_t ldoc;
};

__device__ __forceinline__ TokAcc acc_combine(const TokAcc& a, const TokAcc& b) {
  TokAcc r;
  r.letters = a.letters + b.letters;
  const bool resolve = (b.fl & kU) && (a.fl & kEv) && (a.fl & kWs);
  r.words = a.words + b.words + (resolve ? 1u : 0u);
  const uint32_t ev = (a.fl | b.fl) & kEv;
  const uint32_t ws = (b.fl & kEv) ? (b.fl & kWs) : (a.fl & kWs);
  const uint32_t u = (a.fl & kEv) ? (a.fl & kU) : (b.fl & kU);
  const uint32_t udoc = (a.fl & kEv) ? (a.fl >> 4) : (b.fl >> 4);
  uint32_t has;
  if (b.fl & kHas) {
    has = kHas;
    r.last = a.letters + b.last;
    r.ldoc = b.ldoc;
  } else if (resolve) {  // b's first letter becomes a start: it is b's letter 0
    has = kHas;
    r.last = a.letters;
    r.ldoc = b.fl >> 4;
  } else {
    has = a.fl & kHas;
    r.last = a.last;
    r.ldoc = a.ldoc;
  }
  r.fl = ev | ws | u | has | (udoc << 4);
  return r;
}

constexpr TokAcc kAccZero = {0, 0, 0, 0, 0};

struct LookRec {
  uint32_t status;  // 0: not yet, 1: agg published, 2: inc published
  TokAcc agg;
  TokAcc inc;
  uint32_t pad[3];
};
static_assert(sizeof(LookRec) == 56, "look-back record layout");

struct K1Scratch {
  uint32_t ticket;
  uint32_t finished;
  uint32_t pad[30];
  LookRec rec[1];  // [nchunks]
};

__device__ __forceinline__ uint32_t ld_acquire(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(uint32_t* p, uint32_t v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ TokAcc ld_acc(const TokAcc* p) {
  const uint32_t* q = reinterpret_cast<const uint32_t*>(p);
  return TokAcc{__ldcg(q), __ldcg(q + 1), __ldcg(q + 2), __ldcg(q + 3), __ldcg(q + 4)};
}
__device__ __forceinline__ void st_acc(TokAcc* p, const TokAcc& v) {
  uint32_t* q = reinterpret_cast<uint32_t*>(p);
  __stcg(q, v.letters);
  __stcg(q + 1, v.words);
  __stcg(q + 2, v.fl);
  __stcg(q + 3, v.last);
  __stcg(q + 4, v.ldoc);
}

// Adds the last word of the input to its document's histogram (bin 0 counts
// words longer than l_cap, which make the document fail) and to the
// document's longest length.
__device__ __forceinline__ void count_last_word(uint32_t L, uint32_t doc, uint32_t l_cap, uint32_t* hist,
                                                uint32_t* doc_maxlen, Meta* meta) {
  uint32_t bin = L;
  if (L > l_cap || L > (uint32_t)kMaxLen) {
    bin = 0;
    atomicAdd(&meta->err_long, 1u);
  }
  atomicAdd(&hist[(size_t)doc * kHist + bin], 1u);
  if (bin) atomicMax(&doc_maxlen[doc], bin);
}

// Resident CTAs per SM the register budget is sized for (48 registers a
// thread at 5; the shared memory of a CTA, about 34 KB, allows six).  A CTA
// spends much of its time waiting at barriers (for warp 0's look-back), so
// more resident CTAs hide more of it: on a GB300, 5 beat 4 by about 7% on
// large inputs, and 6 (40 registers) lost on small ones.
#ifndef BSORT_K1_MIN_CTAS
#define BSORT_K1_MIN_CTAS 5
#endif

__global__ void __launch_bounds__(kTokThreads, BSORT_K1_MIN_CTAS) k_tokenize1p(
    const uint8_t* __restrict__ in, const DocDesc* __restrict__ docs, DocDesc doc0, uint32_t ndocs, uint32_t nchunks,
    uint8_t* scratch, uint8_t* __restrict__ letters_out, uint32_t* __restrict__ starts, uint32_t* hist,
    uint32_t* doc_maxlen, uint32_t* doc_wbase, uint32_t* doc_lbase, uint32_t* doc_item0, Meta* meta, Meta* sticky,
    uint32_t l_cap, uint64_t wait_limit, HostMeta hm) {
  K1Scratch* s = reinterpret_cast<K1Scratch*>(scratch);
  __shared__ uint4 buf[kChunk / 16 + 1];  // the chunk, then its letters (with up to 15 bytes of lead)
  extern __shared__ uint16_t s_starts[];   // up to kChunk / 2 word starts, as letter offsets in the chunk
  __shared__ uint32_t h_local[kHist];
  __shared__ uint32_t s_c, s_doc, s_last;
  __shared__ TokAcc s_prefix;
  __shared__ uint32_t s_wlast[kTokThreads / 32];
  __shared__ uint32_t s_sel[16];
  const int t = threadIdx.x;
  for (int i = t; i < kHist; i += kTokThreads) h_local[i] = 0;
  compact_table_fill(s_sel);
  if (t < 32) {  // warp 0 takes the ticket and finds the chunk's document
    uint32_t c0 = 0;
    if (t == 0) c0 = atomicAdd(&s->ticket, 1u);
    c0 = __shfl_sync(kFull, c0, 0);
    uint32_t d0 = 0;
    if (c0 < nchunks && ndocs > 1) {
      d0 = warp_last_le([&](uint32_t i) { return docs[i].chunk0; }, ndocs, c0);
      // empty documents share their chunk0 with the next one: step past them
      if (t == 0)
        while (d0 + 1 < ndocs && (docs[d0].nchunks == 0 || c0 >= docs[d0].chunk0 + docs[d0].nchunks)) ++d0;
    }
    if (t == 0) {
      s_c = c0;
      s_doc = d0;
    }
  }
  __syncthreads();
  const uint32_t c = s_c;
  if (c < nchunks) {
    const uint32_t d = s_doc;
    const DocDesc dd = ndocs == 1 ? doc0 : docs[d];
    // 16-byte granules holding at least one byte of the document; the rest reads as spaces
    const uintptr_t first = reinterpret_cast<uintptr_t>(in) + dd.byte_off;
    const uintptr_t last = first + dd.len;
    const uintptr_t base = (first & ~uintptr_t(15)) + uintptr_t(c - dd.chunk0) * kChunk;
#pragma unroll
    for (int i = 0; i < kChunk / 16 / kTokThreads; ++i) {
      const int g = t + i * kTokThreads;
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
      buf[chunk_slot(g)] = v;
    }
    __syncthreads();
    uint32_t w[16];
    thread_words(buf, w);
    uint64_t lm, sm;
    classify64(w, lm, sm);
    const bool doc_start = (c == dd.chunk0) && t == 0;
    const TokSum leaf = seg_summary(lm, sm, doc_start);
    uint32_t total_pk;
    const uint32_t ex = block_exclusive_pk(pk_make(leaf.letters, leaf.words, leaf.flags), &total_pk);
    // The chunk's last word start that its own bytes decide (its first
    // letter, when no whitespace precedes it in the chunk, waits for the
    // chunk's predecessors): one more than its letter offset, 0 for none.
    {
      const uint32_t fe = pk_flags(ex);
      const uint64_t st_loc = start_mask(lm, sm, doc_start || ((fe & kEv) && (fe & kWs)));
      uint32_t my_last = 0;
      if (st_loc) {
        const int hb = 63 - __clzll(st_loc);
        my_last = pk_letters(ex) + (hb ? __popcll(lm & (~0ull >> (64 - hb))) : 0u) + 1u;
      }
      const uint32_t m = __reduce_max_sync(kFull, my_last);
      if ((t & 31) == 0) s_wlast[t >> 5] = m;
    }
    __syncthreads();
    TokAcc total;
    {
      uint32_t last1 = 0;
#pragma unroll
      for (int i = 0; i < kTokThreads / 32; ++i) last1 = max(last1, s_wlast[i]);
      total.letters = pk_letters(total_pk);
      total.words = pk_words(total_pk);
      total.fl = pk_flags(total_pk) | (last1 ? kHas : 0u) | (d << 4);
      total.last = last1 ? last1 - 1u : 0u;
      total.ldoc = d;
    }

    if (t < 32) {
      // warp 0 publishes this chunk's summary, then looks back over 32
      // predecessors per round: lane i reads record c-1-j0-i; the nearest
      // inclusive prefix and the summaries after it are combined in order
      LookRec* rec = s->rec;
      const int lane = t;
      TokAcc acc = kAccZero;
      if (c == 0) {
        if (lane == 0) {
          st_acc(&rec[0].inc, total);
          st_release(&rec[0].status, 2u);
        }
      } else {
        if (lane == 0) {
          st_acc(&rec[c].agg, total);
          st_release(&rec[c].status, 1u);
        }
        int j0 = (int)c - 1;  // newest predecessor the next 32-record read covers
        uint64_t polls = 0;
        for (;;) {
          const int idx = j0 - lane;
          const uint32_t stt = idx >= 0 ? ld_acquire(&rec[idx].status) : 2u;
          const uint32_t inc_mask = __ballot_sync(kFull, stt == 2u);
          const uint32_t ready_mask = __ballot_sync(kFull, stt != 0u);
          // lanes up to (and with) the nearest inclusive record must be ready
          const int upto = inc_mask ? __ffs(inc_mask) - 1 : 31;
          const uint32_t need = upto == 31 ? kFull : ((1u << (upto + 1)) - 1u);
          if ((ready_mask & need) != need) {
            if (++polls >= wait_limit) {  // gave up: the call reports a timeout
              if (lane == 0) atomicAdd(&meta->err_timeout, 1u);
              break;
            }
            __nanosleep(32);
            continue;
          }
          TokAcc v = kAccZero;
          if (lane < upto || (lane == upto && !inc_mask)) v = idx >= 0 ? ld_acc(&rec[idx].agg) : kAccZero;
          if (lane == upto && inc_mask) v = idx >= 0 ? ld_acc(&rec[idx].inc) : kAccZero;
          // ordered reduction: lane 0 ends with v[upto] (+) ... (+) v[0]
#pragma unroll
          for (int off = 1; off < 32; off <<= 1) {
            TokAcc older;
            older.letters = __shfl_down_sync(kFull, v.letters, off);
            older.words = __shfl_down_sync(kFull, v.words, off);
            older.fl = __shfl_down_sync(kFull, v.fl, off);
            older.last = __shfl_down_sync(kFull, v.last, off);
            older.ldoc = __shfl_down_sync(kFull, v.ldoc, off);
            if (lane + off < 32) v = acc_combine(older, v);
          }
          if (lane == 0) acc = acc_combine(v, acc);
          if (inc_mask) break;
          j0 -= 32;
        }
        if (lane == 0) {
          st_acc(&rec[c].inc, acc_combine(acc, total));
          st_release(&rec[c].status, 2u);
        }
      }
      if (lane == 0) s_prefix = acc;
    }
    __syncthreads();
    const TokAcc cin = s_prefix;
    const uint32_t fe = pk_flags(ex);
    const bool cin_ws = (cin.fl & kEv) && (cin.fl & kWs);
    const bool ws_before = doc_start || ((fe & kEv) ? (fe & kWs) != 0 : cin_ws);
    // word starts of this chunk, staged in order (they are contiguous in
    // `starts`); the chunk's first letter counts before this thread when the
    // predecessors end in whitespace
    uint64_t starts_m = start_mask(lm, sm, ws_before);
    uint32_t wpos = pk_words(ex) + (((fe & kU) && cin_ws) ? 1u : 0u);
    while (starts_m) {
      const int b = __ffsll(starts_m) - 1;
      starts_m &= starts_m - 1;
      const uint64_t below = b ? (lm & (~0ull >> (64 - b))) : 0ull;
      s_starts[wpos++] = (uint16_t)(pk_letters(ex) + __popcll(below));
    }
    // letters, staged so that stage[k] lands at global byte (cin.letters & ~15) + k
    const uint32_t lead = cin.letters & 15u;
    uint8_t* const stage = reinterpret_cast<uint8_t*>(buf);
    stage_letters(w, lm, stage, lead + pk_letters(ex), s_sel);
    __syncthreads();
    // letters out: bytes up to the first 16-byte boundary, 16-byte stores, bytes after the last
    {
      const uint32_t n = total.letters, g0 = cin.letters;
      const uint32_t head = lead ? min(16u - lead, n) : 0u;
      if (t < (int)head) letters_out[g0 + t] = stage[lead + t];
      const uint32_t body = (n - head) / 16;
      uint4* dst16 = reinterpret_cast<uint4*>(letters_out + g0 + head);
      const uint4* src16 = reinterpret_cast<const uint4*>(stage + lead + head);
      for (uint32_t i = t; i < body; i += kTokThreads) dst16[i] = src16[i];
      const uint32_t tail0 = head + body * 16;
      if (t < (int)(n - tail0)) letters_out[g0 + tail0 + t] = stage[lead + tail0 + t];
    }
    // word starts out, and the length of every word whose next start is in this
    // chunk (the first one's start comes from the carry), counted with one
    // shared-memory atomic per distinct length in a warp
    // this chunk's starts: its own, plus its first letter when the carry
    // (ending in whitespace) makes that a start
    const uint32_t nw = acc_combine(cin, total).words - cin.words;
    for (uint32_t i = t; i < nw; i += kTokThreads) starts[cin.words + i] = cin.letters + s_starts[i];
    const bool carry_word = (cin.fl & kHas) != 0;
    for (uint32_t i = t; i < nw; i += kTokThreads) {
      if (i == 0 && !carry_word) continue;
      const uint32_t L = i > 0 ? (uint32_t)s_starts[i] - s_starts[i - 1] : cin.letters + s_starts[0] - cin.last;
      const uint32_t pdoc = i > 0 ? d : cin.ldoc;
      uint32_t bin = L;
      if (L > l_cap || L > (uint32_t)kMaxLen) {
        bin = 0;
        atomicAdd(&meta->err_long, 1u);
      }
      if (pdoc != d) {  // a word of an earlier document
        atomicAdd(&hist[(size_t)pdoc * kHist + bin], 1u);
        if (bin) atomicMax(&doc_maxlen[pdoc], bin);
      } else {
        atomicAdd(&h_local[bin], 1u);
      }
    }
    __syncthreads();
    // the histogram and the document's longest length so far (one atomic
    // per warp that holds a non-empty bin)
    static_assert(kHist == kTokThreads, "one bin per thread");
    const uint32_t hv = h_local[t];
    if (hv) atomicAdd(&hist[(size_t)d * kHist + t], hv);
    const uint32_t mx = __reduce_max_sync(kFull, hv && t ? (uint32_t)t : 0u);
    if ((t & 31) == 0 && mx) atomicMax(&doc_maxlen[d], mx);
  }
  // the CTA that finishes last derives the totals and the document bases
  __syncthreads();
  if (t == 0) {
    __threadfence();
    s_last = atomicAdd(&s->finished, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  const TokAcc all = nchunks ? ld_acc(&s->rec[nchunks - 1].inc) : kAccZero;
  if (t == 0) {
    meta->err_prev = ld_acquire(&sticky->err_timeout);  // the host reads it with the counts
    meta->n_total = all.words;
    meta->s_total = all.letters;
    starts[all.words] = all.letters;  // the last word ends at the end of S
    if (all.fl & kHas) count_last_word(all.letters - all.last, all.ldoc, l_cap, hist, doc_maxlen, meta);
    doc_wbase[ndocs] = all.words;
    doc_lbase[ndocs] = all.letters;
  }
  for (uint32_t d = t; d < ndocs; d += kTokThreads) {
    const uint32_t c0 = ndocs == 1 ? doc0.chunk0 : docs[d].chunk0;
    const TokAcc b = c0 ? ld_acc(&s->rec[c0 - 1].inc) : kAccZero;
    doc_wbase[d] = b.words;
    doc_lbase[d] = b.letters;
  }
  __syncthreads();
  // prefix over documents of their 2048-word blocks (work items of K3)
  __shared__ uint32_t warp_sum[kTokThreads / 32];
  __shared__ uint32_t s_run;
  if (t == 0) s_run = 0;
  __syncthreads();
  const int lane = t & 31, warp = t >> 5;
  for (uint32_t base = 0; base < ndocs; base += kTokThreads) {
    const uint32_t d = base + t;
    const uint32_t items = d < ndocs ? (doc_wbase[d + 1] - doc_wbase[d] + kWordBlock - 1) / kWordBlock : 0u;
    uint32_t inc = items;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const uint32_t u = __shfl_up_sync(kFull, inc, off);
      if (lane >= off) inc += u;
    }
    if (lane == 31) warp_sum[warp] = inc;
    __syncthreads();
    uint32_t before = s_run;
    for (int i = 0; i < warp; ++i) before += warp_sum[i];
    if (d < ndocs) doc_item0[d] = before + inc - items;
    __syncthreads();
    if (t == kTokThreads - 1) s_run = before + inc;
    __syncthreads();
  }
  if (t == 0) {
    doc_item0[ndocs] = s_run;
    meta->items_total = s_run;
  }
  if (hm.dst) {
    // the whole meta region (this CTA's writes and the other CTAs' counts,
    // all in L2 by now) to the host, then the flag the host waits on
    __syncthreads();
    const uint4* src = reinterpret_cast<const uint4*>(meta);
    for (uint32_t i = t; i < hm.n16; i += kTokThreads) hm.dst[i] = __ldcg(src + i);
    __threadfence_system();
    __syncthreads();
    if (t == 0) asm volatile("st.release.sys.global.u32 [%0], %1;" ::"l"(hm.flag), "r"(hm.seq) : "memory");
  }
}

}  // namespace

size_t tokenize1p_scratch_bytes(uint32_t nchunks) {
  return offsetof(K1Scratch, rec) + (size_t)(nchunks ? nchunks : 1) * sizeof(LookRec);
}

cudaError_t launch_tokenize1p(const uint8_t* in, const DocDesc* docs, DocDesc doc0, uint32_t ndocs, uint32_t nchunks,
                              uint8_t* scratch, uint8_t* letters, uint32_t* starts, uint32_t* hist,
                              uint32_t* doc_maxlen, uint32_t* doc_wbase, uint32_t* doc_lbase, uint32_t* doc_item0, Meta* meta,
                              Meta* sticky, uint32_t l_cap, uint64_t wait_limit, HostMeta hm, cudaStream_t st) {
  cudaError_t e = cudaSuccess;
  const size_t smem = (size_t)(kChunk / 2) * sizeof(uint16_t);
  static int attr_done[64];
  e = once_per_device(attr_done, [&] {
    return cudaFuncSetAttribute(k_tokenize1p, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  });
  if (e != cudaSuccess) return e;
  k_tokenize1p<<<nchunks ? nchunks : 1u, kTokThreads, smem, st>>>(in, docs, doc0, ndocs, nchunks, scratch, letters, starts,
                                                              hist, doc_maxlen, doc_wbase, doc_lbase, doc_item0, meta, sticky,
                                                              l_cap, wait_limit, hm);
  return cudaGetLastError();
}

}  // namespace bsort
