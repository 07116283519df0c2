// Duplicate-aware sort, first half, for the buckets marked kSegDedupe (the
// large buckets of Zipf-like text, where a few words repeat very often).
// Phase 3 of the paper's method (Section II; Section III step 4) sorts every
// length bucket; equal words are byte-identical, so a bucket's sorted words
// are its distinct words in order, each repeated as often as it occurs.  This
// kernel finds the distinct words and their counts without sorting the
// bucket: each unit of 2048 key words (2048 / W keys of one bucket) is
// aggregated in shared memory, then every distinct key of the unit is added
// with its count to the bucket's hash table in global memory (dedupe.cuh).
// The distinct keys are sorted and expanded afterwards (k_dedupe.cu).
//
// Per unit (one CTA at a time, units strided over a persistent grid):
//   1. the unit's keys are copied into shared memory (cp.async, 16 bytes a
//      copy: a bucket's keys start 128-byte aligned and a unit is 16 KiB);
//   2. an open-addressing table of 2 * keys slots (one u32 each: empty, or
//      the index of the slot's first key in the high half and the count of
//      its copies in the low half) takes every key: an empty slot is claimed
//      with a compare-and-swap that sets the count to one, a slot holding an
//      equal key gets an atomic add of one.  The keys never move during the
//      unit, so a slot's key is read where it lies; the table is at most
//      half full, so every probe sequence ends at an empty slot;
//   3. every occupied slot goes to the global table with its count; once all
//      units are done, k_dedupe_finish completes the distinct-key arrays and
//      zeroes the global tables' claimed slots again.
#include "dedupe.cuh"

namespace bsort {
namespace {

constexpr int kHaThreads = 256;
constexpr uint32_t kHaUnitWords = kDedupeUnitWords;  // key words per unit (16 KiB)
constexpr uint32_t kHaSlots = 2 * kHaUnitWords;  // table slots for W = 1 (16 KiB)
constexpr uint32_t kHaEmpty = 0xFFFFFFFFu;
constexpr size_t kHaSmem = 8 * kHaUnitWords + 4 * kHaSlots;
static_assert(kHaUnitWords <= 0xFFFFu, "a slot's key index and count are 16 bits each");

template <int W>
__device__ __forceinline__ Key<W> smem_key(const uint64_t* s_keys, uint32_t i) {
  Key<W> k;
#pragma unroll
  for (int q = 0; q < W; ++q) k.w[q] = s_keys[(size_t)i * W + q];
  return k;
}

template <int W>
__device__ __forceinline__ bool key_eq(const Key<W>& a, const Key<W>& b) {
  bool eq = true;
#pragma unroll
  for (int q = 0; q < W; ++q) eq &= a.w[q] == b.w[q];
  return eq;
}

// Keys [k0, k0 + cnt) of bucket sg (cnt <= kHaUnitWords / W), whose first key
// word is at g.
template <int W>
__device__ void hash_unit(const uint64_t* __restrict__ g, uint32_t cnt, const Segment& sg, uint64_t* s_keys,
                          uint32_t* s_tab, const DedupeOut& o, Meta* meta, uint64_t wait_limit) {
  const uint32_t t = threadIdx.x;
  const uint32_t slots = 2 * (kHaUnitWords / W), mask = slots - 1;
  // 1. the keys (16-byte copies; an odd last word by itself) and an empty table
  const uint32_t words = cnt * W;
  for (uint32_t i = t; i < words / 2; i += kHaThreads) cp_async16(s_keys + 2 * i, g + 2 * i);
  cp_async_commit();
  if ((words & 1u) && t == 0) s_keys[words - 1] = g[words - 1];
  for (uint32_t i = t; i < slots / 4; i += kHaThreads)
    reinterpret_cast<uint4*>(s_tab)[i] = make_uint4(kHaEmpty, kHaEmpty, kHaEmpty, kHaEmpty);
  cp_async_wait_all();
  __syncthreads();
  // 2. every key into the table
  volatile uint32_t* vt = s_tab;
  for (uint32_t i = t; i < cnt; i += kHaThreads) {
    const Key<W> k = smem_key<W>(s_keys, i);
    uint32_t h = (uint32_t)key_hash<W>(k) & mask;
    for (uint32_t probes = 0; probes < slots; ++probes, h = (h + 1) & mask) {
      uint32_t v = vt[h];
      if (v == kHaEmpty) {
        v = atomicCAS(s_tab + h, kHaEmpty, (i << 16) | 1u);
        if (v == kHaEmpty) break;  // claimed, with this key's copy counted
      }
      if (key_eq<W>(smem_key<W>(s_keys, v >> 16), k)) {
        atomicAdd(s_tab + h, 1u);
        break;
      }
    }
  }
  __syncthreads();
  // 3. the unit's distinct keys and their counts to the bucket's table
  const uint32_t di = seg_dedupe_index(sg);
  const DedupeIns d = o.ins[di];
  if constexpr (W == 1) {
    // Each warp first packs the occupied slots of its eighth of the table to
    // the front of that eighth (in place: a packed position never passes the
    // slot it comes from, and the warp reads each round of 32 slots before
    // it writes), then its lanes take the packed distinct keys four at a
    // time: the first probes' loads of the global table are issued together,
    // then each insert goes on from its own.  (Taking the slots as they lie,
    // about half of each round's four would be empty.)
    const uint32_t lane = t & 31u;
    const uint32_t per = slots / (kHaThreads / 32);
    uint32_t* list = s_tab + (t >> 5) * per;
    uint32_t n = 0;
    for (uint32_t b = 0; b < per; b += 32) {
      const uint32_t v = list[b + lane];
      const bool occ = v != kHaEmpty;
      const uint32_t m = __ballot_sync(0xFFFFFFFFu, occ);
      if (occ) list[n + (uint32_t)__popc(m & ((1u << lane) - 1u))] = v;
      n += (uint32_t)__popc(m);
    }
    __syncwarp();
    const uint64_t* gtab = o.htab + d.htab_off;
    for (uint32_t q0 = 0; q0 * 32 < n; q0 += 4) {
      uint64_t seen[4], seen_u[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const uint32_t i = (q0 + j) * 32 + lane;
        seen[j] = seen_u[j] = 0ull;
        if (i < n) ld_relaxed_pair(gtab + 2 * first_slot1(s_keys[list[i] >> 16], d), seen[j], seen_u[j]);
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const uint32_t i = (q0 + j) * 32 + lane;
        if (i < n) {
          const uint32_t v = list[i];
          const uint64_t k = s_keys[v >> 16];
          insert1_from(k, v & 0xFFFFu, first_slot1(k, d), seen[j], seen_u[j], d, di, o, meta, wait_limit);
        }
      }
    }
  } else {
    for (uint32_t h = t; h < slots; h += kHaThreads) {
      const uint32_t v = s_tab[h];
      if (v != kHaEmpty) hash_add<W>(smem_key<W>(s_keys, v >> 16), v & 0xFFFFu, d, di, o, meta, wait_limit);
    }
  }
  __syncthreads();  // the keys and the table are read: the next unit may fill them
}

__global__ void __launch_bounds__(kHaThreads, 4) k_dedupe_hash(const Segment* __restrict__ segs, uint32_t sbeg,
                                                            uint32_t send, uint32_t units,
                                                            const uint64_t* __restrict__ keys, DedupeOut o,
                                                            Meta* meta, uint64_t wait_limit) {
  extern __shared__ __align__(16) uint8_t ha_smem[];
  uint64_t* s_keys = reinterpret_cast<uint64_t*>(ha_smem);
  uint32_t* s_tab = reinterpret_cast<uint32_t*>(ha_smem + 8 * kHaUnitWords);
  __shared__ uint32_t s_first[kSegCache];
  __shared__ uint32_t s_seg;
  const bool cached = seg_cache_fill<kByStile0>(segs, sbeg, send, s_first);
  for (uint32_t it = blockIdx.x; it < units; it += gridDim.x) {
    if (threadIdx.x < 32) {
      const uint32_t v = seg_find_warp<kByStile0>(segs, sbeg, send, s_first, cached, it);
      if (threadIdx.x == 0) s_seg = v;
    }
    __syncthreads();
    const Segment sg = segs[s_seg];
    const uint32_t W = sg.W;
    const uint32_t uk = kHaUnitWords / (W ? W : 1u);
    const uint32_t k0 = (it - sg.stile0) * uk;
    const bool ok = (sg.flags & kSegDedupe) && (W == 1 || W == 2 || W == 4 || W == 8) && k0 < sg.n;
    if (!ok) {  // a unit outside its bucket: a planning error, reported, not run
      if (threadIdx.x == 0) {
        atomicAdd(&meta->err_internal, 1u);
        atomicCAS(&meta->err_site, 0u, 0x601u);
      }
      __syncthreads();
      continue;
    }
    const uint32_t cnt = min(uk, sg.n - k0);
    const uint64_t* g = keys + sg.key_off + (uint64_t)k0 * W;
    switch (W) {
      case 1: hash_unit<1>(g, cnt, sg, s_keys, s_tab, o, meta, wait_limit); break;
      case 2: hash_unit<2>(g, cnt, sg, s_keys, s_tab, o, meta, wait_limit); break;
      case 4: hash_unit<4>(g, cnt, sg, s_keys, s_tab, o, meta, wait_limit); break;
      default: hash_unit<8>(g, cnt, sg, s_keys, s_tab, o, meta, wait_limit); break;
    }
  }
}

// After every insert of the call: each claimed slot of the `ndd` buckets'
// tables is found through its distinct-key entry and zeroed again, and a
// one-word key's count moves from the count array into the entry (in place
// of the slot index; the count array is zeroed again too); a wider key's
// entry drops its slot index.
// Buckets are strided over blockIdx.y, each bucket's entries over blockIdx.x
// and the threads (a bucket may hold hundreds of thousands of distinct keys).
__global__ void __launch_bounds__(kHaThreads) k_dedupe_finish(uint32_t ndd, DedupeOut o, Meta* meta) {
  for (uint32_t b = blockIdx.y; b < ndd; b += gridDim.y) {
    const DedupeIns d = o.ins[b];
    const uint32_t W = d.Wp / 2;
    const uint32_t U = min(o.ucnt[b], d.n);
    uint64_t* E = o.uniq + d.uniq_off;
    uint64_t* tab = o.htab + d.htab_off;
    const uint64_t slots = 1ull << d.hbits;
    for (uint32_t u = blockIdx.x * kHaThreads + threadIdx.x; u < U; u += gridDim.x * kHaThreads) {
      uint64_t* e = E + (uint64_t)u * d.Wp;
      const uint64_t i = W == 1 ? e[1] : e[W + 1];
      if (i >= slots) {
        atomicAdd(&meta->err_internal, 1u);
        atomicCAS(&meta->err_site, 0u, 0x602u);
        continue;
      }
      if (W == 1) {  // the count, from the count array; the slot's two words
        e[1] = o.dcnt[d.cnt_off + u];
        o.dcnt[d.cnt_off + u] = 0;
        tab[2 * i] = 0;
        tab[2 * i + 1] = 0;
      } else {
        e[W + 1] = 0;
        uint64_t* slot = tab + i * (W + 1);
        for (uint32_t q = 0; q <= W; ++q) slot[q] = 0;
      }
    }
  }
}

int attr_done[64];

}  // namespace

cudaError_t launch_dedupe_hash(const Segment* segs, uint32_t sbeg, uint32_t send, uint32_t units, uint32_t sm_count,
                               const uint64_t* keys, DedupeOut o, uint32_t ndd, Meta* meta, uint64_t wait_limit,
                               cudaStream_t st) {
  if (units == 0 || send <= sbeg) return cudaSuccess;
  cudaError_t e = once_per_device(attr_done, [&] {
    return cudaFuncSetAttribute(k_dedupe_hash, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kHaSmem);
  });
  if (e != cudaSuccess) return e;
  // 4 CTAs per SM (registers bound it; 32 KiB of shared memory each): the
  // global inserts are latency-bound, so more warps in flight beat larger
  // units (which would leave fewer distinct keys to insert)
  const uint32_t cap = sm_count * 4u;
  k_dedupe_hash<<<units < cap ? units : cap, kHaThreads, kHaSmem, st>>>(segs, sbeg, send, units, keys, o, meta,
                                                                         wait_limit);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_dedupe_finish<<<dim3(32, ndd < 4096u ? ndd : 4096u), kHaThreads, 0, st>>>(ndd, o, meta);
  return cudaGetLastError();
}

}  // namespace bsort
