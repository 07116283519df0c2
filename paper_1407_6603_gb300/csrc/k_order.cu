// The two orders of Table 1 beside the paper's bucketed ASCII sort.
//
// Length order (Table 1, "bubble sort based on the length of the word"):
// the words grouped by length, shorter first, each group in input order (a
// bubble sort that exchanges only on a greater length never reorders equal
// lengths).  No keys and no sort: every word's place follows from counts.
//   k_len_count    per block of 2048 words of a document (K3's work items):
//                  how many words of each length it holds
//   k_len_scan     per document and length: the exclusive prefix of those
//                  counts over the document's blocks
//   k_len_scatter  per block: each word's rank among the block's words of its
//                  length, in input order (warp-synchronous match and count),
//                  then its letters and offset at its place in its bucket
//
// Whole order (Table 1, "bubble sort based on alphabetic order"): one bucket
// per document holding every word, keys zero-padded to the document's
// longest word (a word then sorts before every longer word it begins), sorted
// by the usual kernels with the keys kept (kSegKeysOut).  The words now have
// different lengths, so their places in the stream come from a prefix of the
// lengths in sorted order:
//   k_var_sums   per document and slice of 4096 sorted keys: their letters
//   k_var_bases  per document: the exclusive prefix over its slices
//   k_var_emit   per slice: each key's length and place, then its letters
//                and offset
#include "bsort_dev.cuh"
#include "sort_common.cuh"

namespace bsort {
namespace {

constexpr int kOrdThreads = 256;
constexpr uint32_t kSliceKeys = 4096, kKeysPerThread = kSliceKeys / kOrdThreads;
static_assert(kKeysPerThread * kOrdThreads == kSliceKeys, "16 keys a thread");

// The document of work item `it` (the last with doc_item0 <= it; empty
// documents share their first item with the next one), by warp 0.
__device__ __forceinline__ uint32_t item_doc(const uint32_t* doc_item0, uint32_t ndocs, uint32_t it) {
  return ndocs > 1 ? warp_last_le([&](uint32_t i) { return doc_item0[i]; }, ndocs, it) : 0u;
}

__global__ void __launch_bounds__(kOrdThreads) k_len_count(const uint32_t* __restrict__ starts,
                                                           const uint32_t* __restrict__ doc_wbase,
                                                           const uint32_t* __restrict__ doc_item0, uint32_t ndocs,
                                                           uint32_t items, const uint32_t* __restrict__ seg_lookup,
                                                           uint32_t* __restrict__ icnt) {
  __shared__ uint32_t cnt[kHist];
  __shared__ uint32_t s_doc;
  for (uint32_t it = blockIdx.x; it < items; it += gridDim.x) {
    cnt[threadIdx.x] = 0;
    if (threadIdx.x < 32) {
      const uint32_t d = item_doc(doc_item0, ndocs, it);
      if (threadIdx.x == 0) s_doc = d;
    }
    __syncthreads();
    const uint32_t d = s_doc;
    const uint32_t w0 = doc_wbase[d] + (it - doc_item0[d]) * kWordBlock;
    const uint32_t nw = min(w0 + kWordBlock, doc_wbase[d + 1]) - w0;
    for (uint32_t i = threadIdx.x; i < nw; i += kOrdThreads) {
      const uint32_t L = starts[w0 + i + 1] - starts[w0 + i];
      if (L <= (uint32_t)kMaxLen && seg_lookup[(size_t)d * kHist + L] != kNoSegment) atomicAdd(&cnt[L], 1u);
    }
    __syncthreads();
    icnt[(size_t)it * kHist + threadIdx.x] = cnt[threadIdx.x];
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kOrdThreads) k_len_scan(const uint32_t* __restrict__ doc_item0, uint32_t ndocs,
                                                          uint32_t* __restrict__ icnt) {
  const uint32_t d = blockIdx.x;
  if (d >= ndocs) return;
  uint32_t run = 0;
  for (uint32_t it = doc_item0[d]; it < doc_item0[d + 1]; ++it) {
    const uint32_t v = icnt[(size_t)it * kHist + threadIdx.x];
    icnt[(size_t)it * kHist + threadIdx.x] = run;
    run += v;
  }
}

__global__ void __launch_bounds__(kOrdThreads) k_len_scatter(const uint32_t* __restrict__ starts,
                                                             const uint8_t* __restrict__ letters,
                                                             const uint32_t* __restrict__ doc_wbase,
                                                             const uint32_t* __restrict__ doc_item0, uint32_t ndocs,
                                                             uint32_t items, const uint32_t* __restrict__ seg_lookup,
                                                             const Segment* __restrict__ segs,
                                                             const uint32_t* __restrict__ icnt, EmitOut eo) {
  constexpr uint32_t kWarps = kOrdThreads / 32, kPerWarp = kWordBlock / kWarps, kRounds = kPerWarp / 32;
  __shared__ uint32_t s_st[kWordBlock + 1];
  __shared__ uint16_t wcnt[kWarps][kHist];  // per warp: words of each length, then their base in the block
  __shared__ uint32_t s_doc;
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (uint32_t it = blockIdx.x; it < items; it += gridDim.x) {
    for (uint32_t i = threadIdx.x; i < kWarps * kHist; i += kOrdThreads) (&wcnt[0][0])[i] = 0;
    if (threadIdx.x < 32) {
      const uint32_t d = item_doc(doc_item0, ndocs, it);
      if (threadIdx.x == 0) s_doc = d;
    }
    __syncthreads();
    const uint32_t d = s_doc;
    const uint32_t w0 = doc_wbase[d] + (it - doc_item0[d]) * kWordBlock;
    const uint32_t nw = min(w0 + kWordBlock, doc_wbase[d + 1]) - w0;
    for (uint32_t i = threadIdx.x; i <= nw; i += kOrdThreads) s_st[i] = starts[w0 + i];
    __syncthreads();
    // warp w ranks its 256 consecutive words, 32 a round, in input order
    uint32_t len[kRounds], rank[kRounds];
#pragma unroll
    for (uint32_t r = 0; r < kRounds; ++r) {
      const uint32_t i = warp * kPerWarp + r * 32 + lane;
      uint32_t L = 0;
      if (i < nw) {
        L = s_st[i + 1] - s_st[i];
        if (L > (uint32_t)kMaxLen || seg_lookup[(size_t)d * kHist + L] == kNoSegment) L = 0;
      }
      const uint32_t same = __match_any_sync(0xFFFFFFFFu, L);
      const uint32_t before = wcnt[warp][L];
      rank[r] = before + __popc(same & ((1u << lane) - 1u));
      len[r] = L;
      __syncwarp();
      if (L && lane == (uint32_t)(__ffs(same) - 1)) wcnt[warp][L] = (uint16_t)(before + __popc(same));
      __syncwarp();
    }
    __syncthreads();
    {  // thread t owns length t: the warps' bases for it, in warp order
      uint32_t run = 0;
      for (uint32_t w = 0; w < kWarps; ++w) {
        const uint32_t v = wcnt[w][threadIdx.x];
        wcnt[w][threadIdx.x] = (uint16_t)run;
        run += v;
      }
    }
    __syncthreads();
#pragma unroll
    for (uint32_t r = 0; r < kRounds; ++r) {
      const uint32_t L = len[r];
      if (!L) continue;
      const uint32_t i = warp * kPerWarp + r * 32 + lane;
      const Segment& sg = segs[seg_lookup[(size_t)d * kHist + L]];
      const uint32_t k = icnt[(size_t)it * kHist + L] + wcnt[warp][L] + rank[r];  // place in the bucket
      const uint8_t* src = letters + s_st[i];
      uint8_t* dst = eo.stream + sg.stream_off + (size_t)k * L;
      for (uint32_t b = 0; b < L; ++b) dst[b] = src[b];
      if (eo.want_offsets) eo.offsets[sg.out_word + k] = sg.stream_off - sg.doc_stream0 + k * L;
    }
    __syncthreads();
  }
}

// Letters of a zero-padded key.  The letter codes fill the key from its most
// significant bit as one bit stream (8 or 6 bits a letter) and no code is
// zero, so the key's lowest set bit lies in its last letter: with `used` =
// the bits down to and including it, the key holds ceil(used / bits) letters.
// Every key word before the last letter's holds a whole nonzero code, so the
// first zero word ends the search.
template <int W>
__device__ __forceinline__ uint32_t key_letters(const uint64_t* k, uint32_t codec) {
  uint32_t used = 0;
#pragma unroll
  for (int q = 0; q < W; ++q) {
    const uint64_t v = k[q];
    if (!v) break;
    used = 64u * q + 65u - (uint32_t)__ffsll((long long)v);
  }
  return codec == kCodeSix ? (used + 5u) / 6u : (used + 7u) / 8u;
}

__device__ __forceinline__ uint32_t cta_exclusive(uint32_t v, uint32_t* s_red, uint32_t* total) {
  s_red[threadIdx.x] = v;
  __syncthreads();
  for (uint32_t d = 1; d < kOrdThreads; d <<= 1) {
    const uint32_t add = threadIdx.x >= d ? s_red[threadIdx.x - d] : 0u;
    __syncthreads();
    s_red[threadIdx.x] += add;
    __syncthreads();
  }
  const uint32_t inc = s_red[threadIdx.x];
  *total = s_red[kOrdThreads - 1];
  __syncthreads();
  return inc - v;
}

template <int W>
__device__ void var_sum_slice(const VarDesc& v, uint32_t x, const uint64_t* K, uint32_t codec, uint32_t* s_red,
                              uint32_t* out) {
  const uint32_t u0 = x * kSliceKeys + threadIdx.x * kKeysPerThread;
  uint32_t sum = 0;
  for (uint32_t k = 0; k < kKeysPerThread; ++k)
    if (u0 + k < v.n) sum += key_letters<W>(K + (uint64_t)(u0 + k) * W, codec);
  uint32_t tot;
  cta_exclusive(sum, s_red, &tot);
  if (threadIdx.x == 0) *out = tot;
}

__global__ void __launch_bounds__(kOrdThreads) k_var_sums(const VarDesc* __restrict__ vd, uint32_t nb, uint32_t slices,
                                                          const uint64_t* kA, const uint64_t* kB, uint32_t codec,
                                                          uint32_t* ssum) {
  __shared__ uint32_t s_red[kOrdThreads];
  if (blockIdx.y >= nb) return;
  const VarDesc v = vd[blockIdx.y];
  if ((uint64_t)blockIdx.x * kSliceKeys >= v.n) return;
  const uint64_t* K = (v.final_buf ? kB : kA) + v.key_off;
  uint32_t* out = ssum + (size_t)blockIdx.y * slices + blockIdx.x;
  switch (v.W) {
    case 1: var_sum_slice<1>(v, blockIdx.x, K, codec, s_red, out); break;
    case 2: var_sum_slice<2>(v, blockIdx.x, K, codec, s_red, out); break;
    case 4: var_sum_slice<4>(v, blockIdx.x, K, codec, s_red, out); break;
    case 8: var_sum_slice<8>(v, blockIdx.x, K, codec, s_red, out); break;
    case 16: var_sum_slice<16>(v, blockIdx.x, K, codec, s_red, out); break;
    default: var_sum_slice<32>(v, blockIdx.x, K, codec, s_red, out); break;
  }
}

__global__ void k_var_bases(const VarDesc* __restrict__ vd, uint32_t nb, uint32_t slices, uint32_t* ssum,
                            Meta* meta) {
  const uint32_t b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nb) return;
  const VarDesc v = vd[b];
  const uint32_t ns = (v.n + kSliceKeys - 1) / kSliceKeys;
  uint32_t run = 0;
  for (uint32_t i = 0; i < ns; ++i) {
    const uint32_t x = ssum[(size_t)b * slices + i];
    ssum[(size_t)b * slices + i] = run;
    run += x;
  }
  if (run != v.letters) {  // the keys' letters must be the document's
    atomicAdd(&meta->err_internal, 1u);
    atomicCAS(&meta->err_site, 0u, 0x501u);
  }
}

template <int W>
__device__ void var_emit_slice(const VarDesc& v, uint32_t x, const uint64_t* K, uint32_t codec, uint32_t base,
                               uint32_t* s_red, const EmitOut& eo) {
  const uint32_t u0 = x * kSliceKeys + threadIdx.x * kKeysPerThread;
  uint32_t lens[kKeysPerThread];
  uint32_t sum = 0;
#pragma unroll
  for (uint32_t k = 0; k < kKeysPerThread; ++k) {
    lens[k] = u0 + k < v.n ? key_letters<W>(K + (uint64_t)(u0 + k) * W, codec) : 0u;
    sum += lens[k];
  }
  uint32_t tot;
  uint32_t pos = base + cta_exclusive(sum, s_red, &tot);  // letters before this thread's first key
#pragma unroll
  for (uint32_t k = 0; k < kKeysPerThread; ++k) {
    const uint32_t u = u0 + k;
    if (u >= v.n) break;
    const uint64_t* key = K + (uint64_t)u * W;
    const uint32_t L = lens[k];
    if ((uint64_t)pos + L > v.letters) break;  // (the check above reports keys that do not add up)
    uint8_t* dst = eo.stream + v.stream_off + pos;
    for (uint32_t q = 0; q * 8 < L; ++q) {
      const uint64_t a = ascii8(codec, L, [&](uint32_t w) { return key[w]; }, q);
      for (uint32_t b = 0; b < 8 && q * 8 + b < L; ++b) dst[q * 8 + b] = (uint8_t)(a >> (56 - 8 * b));
    }
    if (eo.want_offsets) eo.offsets[v.out_word + u] = v.stream_off - v.doc_stream0 + pos;
    pos += L;
  }
}

__global__ void __launch_bounds__(kOrdThreads) k_var_emit(const VarDesc* __restrict__ vd, uint32_t nb, uint32_t slices,
                                                          const uint64_t* kA, const uint64_t* kB, uint32_t codec,
                                                          const uint32_t* ssum, EmitOut eo) {
  __shared__ uint32_t s_red[kOrdThreads];
  if (blockIdx.y >= nb) return;
  const VarDesc v = vd[blockIdx.y];
  if ((uint64_t)blockIdx.x * kSliceKeys >= v.n) return;
  const uint64_t* K = (v.final_buf ? kB : kA) + v.key_off;
  const uint32_t base = ssum[(size_t)blockIdx.y * slices + blockIdx.x];
  switch (v.W) {
    case 1: var_emit_slice<1>(v, blockIdx.x, K, codec, base, s_red, eo); break;
    case 2: var_emit_slice<2>(v, blockIdx.x, K, codec, base, s_red, eo); break;
    case 4: var_emit_slice<4>(v, blockIdx.x, K, codec, base, s_red, eo); break;
    case 8: var_emit_slice<8>(v, blockIdx.x, K, codec, base, s_red, eo); break;
    case 16: var_emit_slice<16>(v, blockIdx.x, K, codec, base, s_red, eo); break;
    default: var_emit_slice<32>(v, blockIdx.x, K, codec, base, s_red, eo); break;
  }
}

}  // namespace

cudaError_t launch_length_order(const uint32_t* starts, const uint8_t* letters, const uint32_t* doc_wbase,
                                const uint32_t* doc_item0, uint32_t ndocs, uint32_t items, const uint32_t* seg_lookup,
                                const Segment* segs, uint32_t* icnt, EmitOut eo, cudaStream_t st) {
  if (items == 0) return cudaSuccess;
  const uint32_t grid = items < 152u * 8u ? items : 152u * 8u;
  k_len_count<<<grid, kOrdThreads, 0, st>>>(starts, doc_wbase, doc_item0, ndocs, items, seg_lookup, icnt);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_len_scan<<<ndocs, kOrdThreads, 0, st>>>(doc_item0, ndocs, icnt);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_len_scatter<<<grid, kOrdThreads, 0, st>>>(starts, letters, doc_wbase, doc_item0, ndocs, items, seg_lookup, segs,
                                               icnt, eo);
  return cudaGetLastError();
}

size_t var_slices(uint32_t max_n) { return (max_n + kSliceKeys - 1) / kSliceKeys; }

cudaError_t launch_var_emit(const VarDesc* vd, uint32_t nb, uint32_t max_n, const uint64_t* kA, const uint64_t* kB,
                            uint32_t codec, uint32_t* ssum, Meta* meta, EmitOut eo, cudaStream_t st) {
  if (nb == 0 || max_n == 0) return cudaSuccess;
  const uint32_t slices = (uint32_t)var_slices(max_n);
  k_var_sums<<<dim3(slices, nb), kOrdThreads, 0, st>>>(vd, nb, slices, kA, kB, codec, ssum);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_var_bases<<<(nb + 127) / 128, 128, 0, st>>>(vd, nb, slices, ssum, meta);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_var_emit<<<dim3(slices, nb), kOrdThreads, 0, st>>>(vd, nb, slices, kA, kB, codec, ssum, eo);
  return cudaGetLastError();
}

}  // namespace bsort
