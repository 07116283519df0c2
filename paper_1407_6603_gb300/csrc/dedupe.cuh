// Duplicate-aware sort: the global hash tables of the buckets marked
// kSegDedupe.  Text drawn from a Zipf-like vocabulary repeats a few words very
// often, so a large length bucket holds far fewer distinct words than words.
// Each distinct key of a bucket gets one slot in the bucket's table and one
// entry in its distinct-key array; the hash aggregation kernel
// (k_dedupe_hash.cu) adds every distinct key of a unit of the bucket with its
// count.  The distinct keys are then sorted (the same tile sort and merge
// passes, keys of key + count words) and expanded by their counts
// (k_dedupe.cu), which gives exactly the words the full sort gives, since
// equal keys are equal words.
#pragma once

#include "bsort_dev.cuh"
#include "sort_common.cuh"

namespace bsort {
namespace {

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

// The tables.  Bucket b's table has 2^hbits >= 2 n_b slots and every slot is
// zero between calls: a call's claims are undone by k_dedupe_finish (the
// kernel after the inserts), and the host clears the tables after a call that
// may have left one (a new allocation, a failed consistency check, a
// timeout).  So the layout of the tables may change from call to call.
//   W = 1 (words of up to 8 letters, 10 with six-bit codes: most words): a
//     slot is {key, 1 + the key's index u in the bucket's distinct-key
//     array}.  No key is 0 (every word has a letter), so key 0 marks an
//     empty slot.  A slot is claimed with one compare-and-swap of its key
//     word from 0 to the key; the claimer then takes u and stores it in the
//     slot's second word.  The key word never changes again in the call, so
//     a plain (relaxed) read that finds the key is final; a reader that finds
//     the key before its index waits for the index (boundedly).  The counts
//     are summed with 64-bit atomic adds in a count array indexed by u (also
//     zero between calls), which is compact, so the adds of the many rare
//     words hit the cache instead of a table line each; no fences at all.
//   W >= 2: a slot is {state, key words}: state 0 empty, kStateBusy while
//     the claimer writes the key, then 1 + the key's index in the bucket's
//     distinct-key array, published with a release store after the key (and
//     read with an acquire load).  The count is summed in the array entry.
// Every claimer appends an entry to the bucket's distinct-key array: the key,
// then (W = 1) the slot index, which k_dedupe_finish replaces by the count,
// or (W >= 2) the count so far and the slot index.
constexpr uint64_t kStateBusy = ~0ull;

__device__ __forceinline__ void ld_relaxed_pair(const uint64_t* p, uint64_t& a, uint64_t& b) {
  asm volatile("ld.relaxed.gpu.global.v2.u64 {%0, %1}, [%2];" : "=l"(a), "=l"(b) : "l"(p) : "memory");
}
__device__ __forceinline__ void st_relaxed_u64(uint64_t* p, uint64_t v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Continues the insert of `count` copies of the one-word key k at slot i of
// the bucket's table, whose two words were read as (seen, seen_u).
__device__ void insert1_from(uint64_t k, uint64_t count, uint64_t i, uint64_t seen, uint64_t seen_u,
                             const DedupeIns& d, uint32_t di, const DedupeOut& o, Meta* meta, uint64_t wait_limit) {
  uint64_t* tab = o.htab + d.htab_off;
  const uint64_t mask = (1ull << d.hbits) - 1ull;
  unsigned long long* cnt = reinterpret_cast<unsigned long long*>(o.dcnt + d.cnt_off);
  for (uint64_t probes = 0; probes <= mask; ++probes) {
    uint64_t* slot = tab + 2 * i;
    if (seen == 0) {
      seen = atomicCAS(reinterpret_cast<unsigned long long*>(slot), 0ull, (unsigned long long)k);
      if (seen == 0) {  // claimed
        const uint32_t u = atomicAdd(o.ucnt + di, 1u);
        if (u >= d.n) {  // more distinct keys than words: cannot happen; checked (the host then clears the tables)
          atomicAdd(&meta->err_internal, 1u);
          return;
        }
        uint64_t* e = o.uniq + d.uniq_off + (uint64_t)u * d.Wp;
        e[0] = k;
        e[1] = i;
        st_relaxed_u64(slot + 1, (uint64_t)u + 1);
        atomicAdd(cnt + u, (unsigned long long)count);
        return;
      }
      seen_u = 0;  // (read below)
    }
    if (seen == k) {
      uint64_t polls = 0;
      while (seen_u == 0) {  // claimed, its index not yet stored
        if (++polls >= wait_limit) {
          atomicAdd(&meta->err_timeout, 1u);
          return;
        }
        if (polls > 1) __nanosleep(32);
        seen_u = ld_relaxed_u64(slot + 1);
      }
      if (seen_u > d.n) {  // not an index this call stored: cannot happen; checked
        atomicAdd(&meta->err_internal, 1u);
        return;
      }
      atomicAdd(cnt + seen_u - 1, (unsigned long long)count);
      return;
    }
    i = (i + 1) & mask;
    ld_relaxed_pair(tab + 2 * i, seen, seen_u);
  }
  atomicAdd(&meta->err_timeout, 1u);  // a full table (its capacity of 2n keys makes this unreachable)
}

__device__ __forceinline__ uint64_t first_slot1(uint64_t k, const DedupeIns& d) {
  Key<1> kk;
  kk.w[0] = k;
  return key_hash<1>(kk) & ((1ull << d.hbits) - 1ull);
}

// Adds `count` copies of key k to the bucket's table.  For W >= 2 a reader
// that finds a slot being claimed waits for its key, boundedly: when the
// wait runs out the count is dropped and the call is marked timed out.
template <int W>
__device__ void hash_add(const Key<W>& k, uint64_t count, const DedupeIns& d, uint32_t di, const DedupeOut& o,
                         Meta* meta, uint64_t wait_limit) {
  if constexpr (W == 1) {
    const uint64_t i = first_slot1(k.w[0], d);
    uint64_t seen, seen_u;
    ld_relaxed_pair(o.htab + d.htab_off + 2 * i, seen, seen_u);
    insert1_from(k.w[0], count, i, seen, seen_u, d, di, o, meta, wait_limit);
  } else {
    uint64_t* tab = o.htab + d.htab_off;
    const uint64_t mask = (1ull << d.hbits) - 1ull;
    uint64_t i = key_hash<W>(k) & mask;
    for (uint64_t probes = 0; probes <= mask; ++probes, i = (i + 1) & mask) {
      uint64_t* slot = tab + i * (W + 1);
      uint64_t s = ld_acquire_u64(slot);
      if (s == 0) {
        s = atomicCAS(reinterpret_cast<unsigned long long*>(slot), 0ull, (unsigned long long)kStateBusy);
        if (s == 0) {  // claimed: the key, the entry, then the state
#pragma unroll
          for (int q = 0; q < W; ++q) slot[1 + q] = k.w[q];
          const uint32_t u = atomicAdd(o.ucnt + di, 1u);
          if (u >= d.n) {  // more distinct keys than words: cannot happen; checked (the host then clears the tables)
            atomicAdd(&meta->err_internal, 1u);
            return;
          }
          uint64_t* e = o.uniq + d.uniq_off + (uint64_t)u * d.Wp;
#pragma unroll
          for (int q = 0; q < W; ++q) e[q] = k.w[q];
          e[W] = count;
          e[W + 1] = i;
          for (uint32_t q = W + 2; q < d.Wp; ++q) e[q] = 0ull;
          st_release_u64(slot, (uint64_t)u + 1);  // (a release: the key and entry writes above are seen first)
          return;
        }
        if (s != kStateBusy) s = ld_acquire_u64(slot);  // published meanwhile: read it with acquire
      }
      if (s == kStateBusy) {  // another thread is writing this slot's key
        uint64_t polls = 0;
        while (s == kStateBusy) {
          if (++polls >= wait_limit) {
            atomicAdd(&meta->err_timeout, 1u);
            return;
          }
          __nanosleep(32);
          s = ld_acquire_u64(slot);
        }
      }
      bool eq = true;
#pragma unroll
      for (int q = 0; q < W; ++q) eq &= ld_relaxed_u64(slot + 1 + q) == k.w[q];
      if (eq) {
        atomicAdd(reinterpret_cast<unsigned long long*>(o.uniq + d.uniq_off + (s - 1) * d.Wp + W),
                  (unsigned long long)count);
        return;
      }
    }
    atomicAdd(&meta->err_timeout, 1u);  // a full table (its capacity of 2n keys makes this unreachable)
  }
}

}  // namespace
}  // namespace bsort
