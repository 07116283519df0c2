// Sorting building blocks shared by the tile-sort and merge-pass kernels
// (k_sort.cu, k_sort2.cu): packed keys, compare-exchange, the odd-even
// transposition stages, merge path, TMA bulk copies with mbarriers.
#pragma once

#include "bsort_dev.cuh"

namespace bsort {
namespace {

constexpr uint32_t kFull = 0xFFFFFFFFu;

template <int W>
struct Key {
  uint64_t w[W];
};

template <int W>
__device__ __forceinline__ bool klt(const Key<W>& a, const Key<W>& b) {
#pragma unroll
  for (int i = 0; i < W - 1; ++i)
    if (a.w[i] != b.w[i]) return a.w[i] < b.w[i];
  return a.w[W - 1] < b.w[W - 1];
}

template <int W>
__device__ __forceinline__ Key<W> kload(const uint64_t* p) {
  Key<W> k;
#pragma unroll
  for (int i = 0; i < W; ++i) k.w[i] = p[i];
  return k;
}

template <int W>
__device__ __forceinline__ void kstore(uint64_t* p, const Key<W>& k) {
#pragma unroll
  for (int i = 0; i < W; ++i) p[i] = k.w[i];
}

template <int W>
__device__ __forceinline__ Key<W> kinf() {
  Key<W> k;
#pragma unroll
  for (int i = 0; i < W; ++i) k.w[i] = ~0ull;
  return k;
}

template <int W>
__device__ __forceinline__ Key<W> ksel(bool c, const Key<W>& a, const Key<W>& b) {
  Key<W> r;
#pragma unroll
  for (int i = 0; i < W; ++i) r.w[i] = c ? a.w[i] : b.w[i];
  return r;
}

// compare-exchange: afterwards a <= b
template <int W>
__device__ __forceinline__ void cex(Key<W>& a, Key<W>& b) {
  const bool swap = klt(b, a);
  const Key<W> lo = ksel(swap, b, a);
  const Key<W> hi = ksel(swap, a, b);
  a = lo;
  b = hi;
}

__host__ __device__ constexpr int kpt_c(int W) { return W >= 8 ? 1 : 8 / W; }

// ---- TMA bulk copy and mbarrier (inline PTX) ----

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void tma_load_1d(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait: false when `limit` polls pass without the phase completing.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, uint64_t limit) {
  for (uint64_t i = 0; i < limit; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

// ---- asynchronous copies global -> shared (cp.async, per thread) ----
__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// ---- sorting building blocks ----

// 1. odd-even transposition of KPT keys in registers (KPT rounds)
template <int W, int KPT>
__device__ __forceinline__ void oets_registers(Key<W> (&k)[KPT]) {
#pragma unroll
  for (int r = 0; r < KPT; ++r) {
#pragma unroll
    for (int i = r & 1; i + 1 < KPT; i += 2) cex(k[i], k[i + 1]);
  }
}

// 2. odd-even transposition between neighbouring lanes of a G-lane group,
//    G rounds.  In round r the pairs are lanes (g, g+1) with g = r mod 2; the
//    lower lane keeps the KPT smallest of the two runs, the upper lane the
//    KPT largest.  Pairing run a (ascending) with the partner's run reversed
//    gives a bitonic sequence holding exactly those keys, which log2(KPT)
//    half-cleaner stages put in order.
template <int W, int KPT, int G>
__device__ __forceinline__ void oets_lanes(Key<W> (&k)[KPT]) {
  const int lane = threadIdx.x & 31;
  const int g = lane & (G - 1);
#pragma unroll 1
  for (int r = 0; r < G; ++r) {
    const bool lower = ((g & 1) == (r & 1)) && (g + 1 < G);
    const bool upper = (g >= 1) && (((g - 1) & 1) == (r & 1));
    const int partner = lower ? lane + 1 : (upper ? lane - 1 : lane);
    Key<W> p[KPT];
#pragma unroll
    for (int i = 0; i < KPT; ++i)
#pragma unroll
      for (int j = 0; j < W; ++j) p[i].w[j] = __shfl_sync(kFull, k[i].w[j], partner);
    if (lower || upper) {
      Key<W> c[KPT];
#pragma unroll
      for (int i = 0; i < KPT; ++i) {
        const bool plt = klt(p[KPT - 1 - i], k[i]);
        c[i] = ksel(plt == lower, p[KPT - 1 - i], k[i]);
      }
#pragma unroll
      for (int s = KPT / 2; s > 0; s >>= 1)
#pragma unroll
        for (int i = 0; i < KPT; ++i)
          if ((i & s) == 0) cex(c[i], c[i + s]);
#pragma unroll
      for (int i = 0; i < KPT; ++i) k[i] = c[i];
    }
  }
}

// Merge path: how many of the first d outputs of merge(A, B) come from A,
// ties going to A.
template <int W>
__device__ __forceinline__ uint32_t mp_split(const uint64_t* A, uint32_t la, const uint64_t* B, uint32_t lb,
                                             uint32_t d) {
  uint32_t lo = d > lb ? d - lb : 0u, hi = d < la ? d : la;
  while (lo < hi) {
    const uint32_t m = (lo + hi) >> 1;
    if (klt(kload<W>(B + (size_t)(d - 1 - m) * W), kload<W>(A + (size_t)m * W)))
      hi = m;
    else
      lo = m + 1;
  }
  return lo;
}

// Sequential merge of up to KPT outputs starting at (a, b).
template <int W, int KPT>
__device__ __forceinline__ void merge_run(const uint64_t* A, uint32_t la, const uint64_t* B, uint32_t lb, uint32_t a,
                                          uint32_t b, uint32_t n_out, Key<W> (&k)[KPT]) {
#pragma unroll
  for (int s = 0; s < KPT; ++s) {
    if ((uint32_t)s < n_out) {
      const Key<W> ka = a < la ? kload<W>(A + (size_t)a * W) : kinf<W>();
      const Key<W> kb = b < lb ? kload<W>(B + (size_t)b * W) : kinf<W>();
      const bool take_a = a < la && (b >= lb || !klt(kb, ka));
      k[s] = ksel(take_a, ka, kb);
      if (take_a)
        ++a;
      else
        ++b;
    }
  }
}

__device__ __forceinline__ uint32_t find_segment(const Segment* segs, uint32_t sbeg, uint32_t send, uint32_t it) {
  uint32_t lo = sbeg, hi = send - 1;  // last segment with tile0 <= it
  while (lo < hi) {
    const uint32_t mid = (lo + hi + 1) >> 1;
    if (segs[mid].tile0 <= it)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

// Parallel merge-path search: the CTA's NTH threads probe NTH diagonal
// positions at once, keep the interval where the predicate flips, and
// repeat; about log_NTH of the run length rounds.  keyA(i) / keyB(i) return
// the i-th key of each run, wherever it lives (global memory, or the shared
// memory of the CTAs of a cluster).  Uniform across the CTA: every thread
// calls it with the same arguments.
template <int W, int NTH, class FA, class FB>
__device__ uint32_t coop_split_fn(FA keyA, uint32_t la, FB keyB, uint32_t lb, uint32_t d) {
  uint32_t lo = d > lb ? d - lb : 0u, hi = d < la ? d : la;
  while (hi > lo) {
    const uint32_t span = hi - lo;
    if (span <= (uint32_t)NTH) {
      bool f = false;
      if (threadIdx.x < span) {
        const uint32_t m = lo + threadIdx.x;
        f = !klt(keyB(d - 1 - m), keyA(m));
      }
      lo += (uint32_t)__syncthreads_count(f);
      break;
    }
    const uint32_t step = (span + NTH - 1) / NTH;
    const uint32_t m = lo + threadIdx.x * step;
    bool f = false;
    if (m < hi) f = !klt(keyB(d - 1 - m), keyA(m));
    const uint32_t nf = (uint32_t)__syncthreads_count(f);
    const uint32_t nlo = nf == 0 ? lo : lo + (nf - 1) * step + 1;
    const uint32_t nhi = lo + nf * step < hi ? lo + nf * step : hi;
    lo = nlo;
    hi = nhi;
  }
  return lo;
}

// The merge-path search by one warp (all 32 lanes call it): 32 probes per
// round, ballots instead of CTA barriers.  keyA / keyB as in coop_split_fn.
template <int W, class FA, class FB>
__device__ __forceinline__ uint32_t warp_split_fn(FA keyA, uint32_t la, FB keyB, uint32_t lb, uint32_t d) {
  const uint32_t lane = threadIdx.x & 31u;
  uint32_t lo = d > lb ? d - lb : 0u, hi = d < la ? d : la;
  while (hi > lo) {
    const uint32_t span = hi - lo;
    const uint32_t step = span <= 32u ? 1u : (span + 31u) / 32u;
    const uint32_t m = lo + lane * step;
    bool f = false;
    if (m < hi) f = !klt(keyB(d - 1 - m), keyA(m));
    const uint32_t nf = __popc(__ballot_sync(kFull, f));
    const uint32_t nhi = lo + nf * step < hi ? lo + nf * step : hi;
    lo = nf == 0 ? lo : lo + (nf - 1) * step + 1;
    hi = nhi;
  }
  return lo;
}

template <int W, int NTH>
__device__ __forceinline__ uint32_t coop_split(const uint64_t* A, uint32_t la, const uint64_t* B, uint32_t lb,
                                               uint32_t d) {
  return coop_split_fn<W, NTH>([&](uint32_t i) { return kload<W>(A + (size_t)i * W); }, la,
                               [&](uint32_t i) { return kload<W>(B + (size_t)i * W); }, lb, d);
}

}  // namespace
}  // namespace bsort
