// K4 (tile sort) and K5 (merge passes): phase 3 of the paper's method, the
// sort of each length bucket into ASCII order (Section II; Section III step 4).
//
// Keys.  A word of L letters is held as W = next_pow2(ceil(L/8)) u64 words,
// big-endian with zero padding, so that for words of one length the
// lexicographic unsigned byte order is the order of the W-word tuples.
//
// K4 keeps the compare-exchange of bubble sort (Section I: compare adjacent
// items, exchange when out of order) in its parallel form, odd-even
// transposition: rounds alternate between the (even, odd) and (odd, even)
// neighbour pairs, and P rounds sort P items.  A tile of 256 * KPT keys is
// staged in shared memory by a TMA bulk copy, then
//   1. each thread sorts its KPT keys in registers by odd-even transposition;
//   2. groups of G lanes run G rounds of odd-even transposition between lane
//      neighbours, exchanging whole sorted runs through warp shuffles
//      (the merge-split form of the compare-exchange);
//   3. the runs of G*KPT keys are merged up to the tile by merge path in
//      shared memory.
// K5 then merges sorted runs pairwise, pass after pass, until each bucket is
// one run (the bubble sort's n(n-1)/2 comparisons, Section "Bubble sort as
// parallel", are what this avoids).  Each CTA makes one tile of output: it
// finds where its output diagonal cuts the two runs (merge path) with a
// 256-way parallel search in global memory, stages the two slices in shared
// memory and merges them.
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

// ---------------------------------------------------------------- K4 ----
template <int W, int G>
__global__ void __launch_bounds__(kSortThreads) k_tile_sort(const Segment* __restrict__ segs, uint32_t sbeg,
                                                            uint32_t send, uint32_t tiles, uint64_t* keys,
                                                            Meta* meta, uint64_t wait_limit) {
  constexpr int KPT = kpt_c(W);
  constexpr int T = kSortThreads * KPT;
  extern __shared__ __align__(128) uint64_t sm[];  // T keys of W words
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t s_seg;
  const int t = threadIdx.x;
  if (t == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  uint32_t phase = 0;
  for (uint32_t it = blockIdx.x; it < tiles; it += gridDim.x) {
    if (t == 0) s_seg = find_segment(segs, sbeg, send, it);
    __syncthreads();
    const Segment sg = segs[s_seg];
    const uint32_t j0 = (it - sg.tile0) * T;
    const uint32_t cnt = min((uint32_t)T, sg.n - j0);
    uint64_t* g = keys + sg.key_off + (size_t)j0 * W;
    const uint32_t tma_bytes = (cnt * W * 8u) & ~15u;
    if (t == 0) {
      fence_proxy_async();
      mbar_arrive_expect_tx(&bar, tma_bytes);
      if (tma_bytes) tma_load_1d(sm, g, tma_bytes, &bar);
    }
    for (uint32_t e = tma_bytes / 8 + t; e < (uint32_t)(T * W); e += kSortThreads)
      sm[e] = e < cnt * W ? g[e] : ~0ull;  // odd tail word, then +inf padding
    const bool ok = mbar_wait_bounded(&bar, phase, wait_limit);
    phase ^= 1u;
    if (__syncthreads_or(!ok)) {
      // The copy did not land in time: report, let it drain, stop.
      if (t == 0) {
        atomicAdd(&meta->err_timeout, 1u);
        mbar_wait_bounded(&bar, phase ^ 1u, wait_limit);
      }
      __syncthreads();
      return;
    }
    Key<W> k[KPT];
#pragma unroll
    for (int i = 0; i < KPT; ++i) k[i] = kload<W>(sm + (size_t)(t * KPT + i) * W);
    oets_registers<W, KPT>(k);
    oets_lanes<W, KPT, G>(k);
#pragma unroll 1
    for (uint32_t R = G * KPT; R < (uint32_t)T; R <<= 1) {
      __syncthreads();
#pragma unroll
      for (int i = 0; i < KPT; ++i) kstore<W>(sm + (size_t)(t * KPT + i) * W, k[i]);
      __syncthreads();
      const uint32_t pos = t * KPT;
      const uint32_t base = pos & ~(2 * R - 1);
      const uint32_t d = pos - base;
      const uint64_t* A = sm + (size_t)base * W;
      const uint64_t* B = A + (size_t)R * W;
      const uint32_t a = mp_split<W>(A, R, B, R, d);
      merge_run<W, KPT>(A, R, B, R, a, d - a, KPT, k);
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < KPT; ++i) kstore<W>(sm + (size_t)(t * KPT + i) * W, k[i]);
    __syncthreads();
    for (uint32_t e = t; e < cnt * W; e += kSortThreads) g[e] = sm[e];
    __syncthreads();
  }
}

// ---------------------------------------------------------------- K5 ----

// Parallel merge-path search over global memory: the CTA probes 256
// diagonal positions at once, keeps the interval where the predicate flips,
// and repeats; about log_256 of the run length rounds.  Uniform across the
// CTA (every thread calls it with the same arguments).
template <int W>
__device__ uint32_t coop_split(const uint64_t* __restrict__ A, uint32_t la, const uint64_t* __restrict__ B,
                               uint32_t lb, uint32_t d) {
  uint32_t lo = d > lb ? d - lb : 0u, hi = d < la ? d : la;
  while (hi > lo) {
    const uint32_t span = hi - lo;
    if (span <= (uint32_t)kSortThreads) {
      bool f = false;
      if (threadIdx.x < span) {
        const uint32_t m = lo + threadIdx.x;
        f = !klt(kload<W>(B + (size_t)(d - 1 - m) * W), kload<W>(A + (size_t)m * W));
      }
      lo += (uint32_t)__syncthreads_count(f);
      break;
    }
    const uint32_t step = (span + kSortThreads - 1) / kSortThreads;
    const uint32_t m = lo + threadIdx.x * step;
    bool f = false;
    if (m < hi) f = !klt(kload<W>(B + (size_t)(d - 1 - m) * W), kload<W>(A + (size_t)m * W));
    const uint32_t nf = (uint32_t)__syncthreads_count(f);
    const uint32_t nlo = nf == 0 ? lo : lo + (nf - 1) * step + 1;
    const uint32_t nhi = lo + nf * step < hi ? lo + nf * step : hi;
    lo = nlo;
    hi = nhi;
  }
  return lo;
}

template <int W>
__global__ void __launch_bounds__(kSortThreads) k_merge_pass(const Segment* __restrict__ segs, uint32_t sbeg,
                                                             uint32_t send, uint32_t tiles, uint32_t pass,
                                                             const uint64_t* __restrict__ src,
                                                             uint64_t* __restrict__ dst) {
  constexpr int KPT = kpt_c(W);
  constexpr int T = kSortThreads * KPT;
  extern __shared__ __align__(128) uint64_t sm[];
  __shared__ uint32_t s_seg;
  const int t = threadIdx.x;
  for (uint32_t it = blockIdx.x; it < tiles; it += gridDim.x) {
    if (t == 0) s_seg = find_segment(segs, sbeg, send, it);
    __syncthreads();
    const Segment sg = segs[s_seg];
    __syncthreads();
    const uint64_t n = sg.n;
    const uint64_t R = (uint64_t)T << pass;
    if (n <= R) continue;  // this bucket is already one run
    const uint64_t out0 = (uint64_t)(it - sg.tile0) * T;
    const uint64_t ps = out0 / (2 * R) * (2 * R);
    const uint32_t la = (uint32_t)min(R, n - ps);
    const uint32_t lb = n - ps > R ? (uint32_t)min(R, n - ps - R) : 0u;
    const uint32_t d0 = (uint32_t)(out0 - ps);
    const uint32_t cnt = min((uint32_t)T, la + lb - d0);
    const uint32_t d1 = d0 + cnt;
    const uint64_t* A = src + sg.key_off + ps * W;
    const uint64_t* B = A + (size_t)la * W;
    uint64_t* out = dst + sg.key_off + (ps + d0) * W;
    if (lb == 0) {  // odd run at the end of the bucket: carried over
      for (uint32_t e = t; e < cnt * W; e += kSortThreads) out[e] = A[(size_t)d0 * W + e];
      continue;
    }
    const uint32_t a0 = coop_split<W>(A, la, B, lb, d0);
    const uint32_t a1 = coop_split<W>(A, la, B, lb, d1);
    const uint32_t na = a1 - a0, nb = (d1 - a1) - (d0 - a0);
    const uint64_t* gA = A + (size_t)a0 * W;
    const uint64_t* gB = B + (size_t)(d0 - a0) * W;
    for (uint32_t e = t; e < na * W; e += kSortThreads) sm[e] = gA[e];
    for (uint32_t e = t; e < nb * W; e += kSortThreads) sm[na * W + e] = gB[e];
    __syncthreads();
    Key<W> k[KPT];
    const uint32_t pos = t * KPT;
    if (pos < cnt) {
      const uint64_t* SA = sm;
      const uint64_t* SB = sm + (size_t)na * W;
      const uint32_t a = mp_split<W>(SA, na, SB, nb, pos);
      merge_run<W, KPT>(SA, na, SB, nb, a, pos - a, cnt - pos, k);
    }
    __syncthreads();
#pragma unroll
    for (int s = 0; s < KPT; ++s)
      if (pos + s < cnt) kstore<W>(sm + (size_t)(pos + s) * W, k[s]);
    __syncthreads();
    for (uint32_t e = t; e < cnt * W; e += kSortThreads) out[e] = sm[e];
    __syncthreads();
  }
}

template <int W>
size_t sort_smem_bytes() {
  return (size_t)kSortThreads * kpt_c(W) * W * 8;
}

template <int W, int G>
cudaError_t tile_sort_w(const Segment* segs, uint32_t sbeg, uint32_t send, uint32_t tiles, uint32_t grid,
                        uint64_t* keys, Meta* meta, uint64_t wait_limit, cudaStream_t st) {
  const size_t smem = sort_smem_bytes<W>();
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_tile_sort<W, G>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  k_tile_sort<W, G><<<grid, kSortThreads, smem, st>>>(segs, sbeg, send, tiles, keys, meta, wait_limit);
  return cudaGetLastError();
}

template <int W>
cudaError_t merge_pass_w(const Segment* segs, uint32_t sbeg, uint32_t send, uint32_t tiles, uint32_t grid,
                         uint32_t pass, const uint64_t* src, uint64_t* dst, cudaStream_t st) {
  const size_t smem = sort_smem_bytes<W>();
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_merge_pass<W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  k_merge_pass<W><<<grid, kSortThreads, smem, st>>>(segs, sbeg, send, tiles, pass, src, dst);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_tile_sort(int W, const Segment* segs, uint32_t sbeg, uint32_t send, uint32_t tiles, uint32_t grid,
                             uint64_t* keys, Meta* meta, uint64_t wait_limit, cudaStream_t st) {
  if (tiles == 0 || grid == 0) return cudaSuccess;
  switch (W) {
    case 1: return tile_sort_w<1, 32>(segs, sbeg, send, tiles, grid, keys, meta, wait_limit, st);
    case 2: return tile_sort_w<2, 32>(segs, sbeg, send, tiles, grid, keys, meta, wait_limit, st);
    case 4: return tile_sort_w<4, 32>(segs, sbeg, send, tiles, grid, keys, meta, wait_limit, st);
    case 8: return tile_sort_w<8, 32>(segs, sbeg, send, tiles, grid, keys, meta, wait_limit, st);
    case 16: return tile_sort_w<16, 32>(segs, sbeg, send, tiles, grid, keys, meta, wait_limit, st);
    case 32: return tile_sort_w<32, 32>(segs, sbeg, send, tiles, grid, keys, meta, wait_limit, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_merge_pass(int W, const Segment* segs, uint32_t sbeg, uint32_t send, uint32_t tiles,
                              uint32_t grid, uint32_t pass, const uint64_t* src, uint64_t* dst, cudaStream_t st) {
  if (tiles == 0 || grid == 0) return cudaSuccess;
  switch (W) {
    case 1: return merge_pass_w<1>(segs, sbeg, send, tiles, grid, pass, src, dst, st);
    case 2: return merge_pass_w<2>(segs, sbeg, send, tiles, grid, pass, src, dst, st);
    case 4: return merge_pass_w<4>(segs, sbeg, send, tiles, grid, pass, src, dst, st);
    case 8: return merge_pass_w<8>(segs, sbeg, send, tiles, grid, pass, src, dst, st);
    case 16: return merge_pass_w<16>(segs, sbeg, send, tiles, grid, pass, src, dst, st);
    case 32: return merge_pass_w<32>(segs, sbeg, send, tiles, grid, pass, src, dst, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace bsort
