// Duplicate-aware sort, first half: K4's epilogue for the buckets marked
// kSegDedupe.  Text drawn from a Zipf-like vocabulary repeats a few words
// very often, so a large length bucket holds far fewer distinct words than
// words.  Instead of writing a sorted run back for the merge passes, the CTA
// walks its sorted tile, finds every group of equal keys (a binary search for
// the group's end, so a group of any size costs log2(tile) probes), and adds
// (key, group size) to the bucket's hash table in global memory.  The table
// gives each distinct key one entry in the bucket's distinct-key array; its
// count is summed there with 64-bit atomics.  The distinct keys are then
// sorted (the same tile sort and merge passes, keys of key + count words) and
// expanded by their counts (k_dedupe.cu), which gives exactly the words the
// full sort gives, since equal keys are equal words.
#pragma once

#include "bsort_dev.cuh"
#include "sort_common.cuh"

namespace bsort {
namespace {

constexpr uint32_t kSlotBusy = 0xFFFFFFFFu;

__device__ __forceinline__ uint64_t ld_acquire_u64(const uint64_t* p) {
  uint64_t v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ uint64_t ld_relaxed_u64(const uint64_t* p) {
  uint64_t v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_u64(uint64_t* p, uint64_t v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// A 64-bit mix of the key's words (multiply-xorshift rounds).
template <int W>
__device__ __forceinline__ uint64_t key_hash(const Key<W>& k) {
  uint64_t h = 0x6A09E667F3BCC909ull;
#pragma unroll
  for (int q = 0; q < W; ++q) {
    h ^= k.w[q];
    h *= 0x9E3779B97F4A7C15ull;
    h ^= h >> 32;
  }
  h *= 0xD6E8FEB86659FD93ull;
  return h ^ (h >> 29);
}

// Adds `count` copies of key k to the bucket's table.  A slot is 1 + W u64
// words: a header (the call's generation in the high half; in the low half
// kSlotBusy while its first inserter writes the key, then the key's index in
// the distinct-key array) and the key.  A slot stamped with another
// generation is empty, so the table needs no clearing between calls.  The
// wait for a busy slot is bounded; when it runs out the count is dropped and
// the call is marked timed out.
template <int W>
__device__ void hash_add(const Key<W>& k, uint64_t count, const DedupeIns& d, uint32_t di, const DedupeOut& o,
                         Meta* meta, uint64_t wait_limit) {
  uint64_t* tab = o.htab + d.htab_off;
  const uint64_t mask = (1ull << d.hbits) - 1ull;
  const uint64_t gen = (uint64_t)o.gen << 32;
  uint64_t i = key_hash<W>(k) & mask;
  for (uint64_t probes = 0; probes <= mask;) {
    uint64_t* slot = tab + i * (W + 1);
    uint64_t hdr = ld_acquire_u64(slot);
    if ((hdr & 0xFFFFFFFF00000000ull) != gen) {  // empty in this call: claim it
      if (atomicCAS(reinterpret_cast<unsigned long long*>(slot), hdr, gen | kSlotBusy) != hdr) continue;
#pragma unroll
      for (int q = 0; q < W; ++q) slot[1 + q] = k.w[q];
      const uint32_t u = atomicAdd(o.ucnt + di, 1u);
      if (u >= d.n) {  // more distinct keys than words: cannot happen; checked, not written
        atomicAdd(&meta->err_internal, 1u);
        return;
      }
      uint64_t* e = o.uniq + d.uniq_off + (uint64_t)u * d.Wp;
#pragma unroll
      for (int q = 0; q < W; ++q) e[q] = k.w[q];
      e[W] = count;
      for (uint32_t q = W + 1; q < d.Wp; ++q) e[q] = 0ull;
      st_release_u64(slot, gen | u);  // (a release: the key and entry writes above are seen first)
      return;
    }
    if ((uint32_t)hdr == kSlotBusy) {  // another thread is writing this slot's key
      uint64_t polls = 0;
      while ((uint32_t)hdr == kSlotBusy) {
        if (++polls >= wait_limit) {
          atomicAdd(&meta->err_timeout, 1u);
          return;
        }
        __nanosleep(32);
        hdr = ld_acquire_u64(slot);
      }
    }
    bool eq = true;
#pragma unroll
    for (int q = 0; q < W; ++q) eq &= ld_relaxed_u64(slot + 1 + q) == k.w[q];
    if (eq) {
      atomicAdd(reinterpret_cast<unsigned long long*>(o.uniq + d.uniq_off + (uint64_t)(uint32_t)hdr * d.Wp + W),
                (unsigned long long)count);
      return;
    }
    i = (i + 1) & mask;
    ++probes;
  }
  atomicAdd(&meta->err_timeout, 1u);  // a full table (its capacity of 2n keys makes this unreachable)
}

// The epilogue: key_at(i) is the tile's i-th sorted key, i < cnt <= NTH * 8.
// The positions that start a group of equal keys are marked in a bit mask
// (one ballot per warp and round); a group's size is the distance to the next
// marked position.  Thread t adds the groups that start at its positions t,
// t + NTH, ... to the bucket's table.
template <int W, int NTH, class F>
__device__ void rle_insert(F key_at, uint32_t cnt, const Segment& sg, const DedupeOut& o, uint32_t* s_heads,
                           Meta* meta, uint64_t wait_limit) {
  const uint32_t di = seg_dedupe_index(sg);
  const DedupeIns d = o.ins[di];
  const uint32_t words = (cnt + 31) / 32;
  for (uint32_t i0 = 0; i0 < cnt; i0 += NTH) {  // every warp marks 32 consecutive positions per round
    const uint32_t i = i0 + threadIdx.x;
    const bool head = i < cnt && (i == 0 || klt(key_at(i - 1), key_at(i)));
    const uint32_t m = __ballot_sync(0xFFFFFFFFu, head);
    if ((threadIdx.x & 31) == 0 && i < cnt) s_heads[i >> 5] = m;
  }
  __syncthreads();
  for (uint32_t i = threadIdx.x; i < cnt; i += NTH) {
    const uint32_t wi = i >> 5, b = i & 31;
    if (!((s_heads[wi] >> b) & 1u)) continue;
    // the next head after i, or cnt
    uint32_t rest = b == 31 ? 0u : s_heads[wi] >> (b + 1) << (b + 1);
    uint32_t wj = wi;
    while (!rest && ++wj < words) rest = s_heads[wj];
    const uint32_t end = rest ? min(cnt, wj * 32 + (uint32_t)(__ffs(rest) - 1)) : cnt;
    hash_add<W>(key_at(i), end - i, d, di, o, meta, wait_limit);
  }
  __syncthreads();
}

}  // namespace
}  // namespace bsort
