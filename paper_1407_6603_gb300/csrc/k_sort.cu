// K4 and K5 for the widest keys: 16 and 32 u64 words, words of 65..255
// letters (rare in text).  Keys of up to 8 words use k_sort2.cu; these
// kernels keep one CTA of 256 threads per tile of 256 keys (a tile of 32-word
// keys fills 64 KiB of shared memory), the same three odd-even transposition
// stages, and merge-path passes of one tile per CTA.
#include "bsort_dev.cuh"
#include "sort_common.cuh"

namespace bsort {
namespace {

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
    // (the copy's wait has a floor of its own: see sort_supertile)
    const uint64_t limit = wait_limit > kCopyWaitFloor ? wait_limit : kCopyWaitFloor;
    const bool ok = mbar_wait_bounded(&bar, phase, limit);
    phase ^= 1u;
    if (__syncthreads_or(!ok)) {
      // The copy did not land in time: report, give it a second bounded wait
      // to drain, stop without writing anything.
      if (t == 0) {
        atomicAdd(&meta->err_timeout, 1u);
        mbar_wait_bounded(&bar, phase ^ 1u, limit);
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
    const uint32_t a0 = coop_split<W, kSortThreads>(A, la, B, lb, d0);
    const uint32_t a1 = coop_split<W, kSortThreads>(A, la, B, lb, d1);
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
  static int attr_done[64];
  cudaError_t e = once_per_device(attr_done, [&] {
    return smem > 48 * 1024
               ? cudaFuncSetAttribute(k_tile_sort<W, G>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)
               : cudaSuccess;
  });
  if (e != cudaSuccess) return e;
  k_tile_sort<W, G><<<grid, kSortThreads, smem, st>>>(segs, sbeg, send, tiles, keys, meta, wait_limit);
  return cudaGetLastError();
}

template <int W>
cudaError_t merge_pass_w(const Segment* segs, uint32_t sbeg, uint32_t send, uint32_t tiles, uint32_t grid,
                         uint32_t pass, const uint64_t* src, uint64_t* dst, cudaStream_t st) {
  const size_t smem = sort_smem_bytes<W>();
  static int attr_done[64];
  cudaError_t e = once_per_device(attr_done, [&] {
    return smem > 48 * 1024
               ? cudaFuncSetAttribute(k_merge_pass<W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)
               : cudaSuccess;
  });
  if (e != cudaSuccess) return e;
  k_merge_pass<W><<<grid, kSortThreads, smem, st>>>(segs, sbeg, send, tiles, pass, src, dst);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_tile_sort(int W, const Segment* segs, uint32_t sbeg, uint32_t send, uint32_t tiles, uint32_t grid,
                             uint64_t* keys, Meta* meta, uint64_t wait_limit, cudaStream_t st) {
  if (tiles == 0 || grid == 0) return cudaSuccess;
  if (W == 16) return tile_sort_w<16, 32>(segs, sbeg, send, tiles, grid, keys, meta, wait_limit, st);
  if (W != 32) return cudaErrorInvalidValue;
  return tile_sort_w<32, 32>(segs, sbeg, send, tiles, grid, keys, meta, wait_limit, st);
}

cudaError_t launch_merge_pass(int W, const Segment* segs, uint32_t sbeg, uint32_t send, uint32_t tiles,
                              uint32_t grid, uint32_t pass, const uint64_t* src, uint64_t* dst, cudaStream_t st) {
  if (tiles == 0 || grid == 0) return cudaSuccess;
  if (W == 16) return merge_pass_w<16>(segs, sbeg, send, tiles, grid, pass, src, dst, st);
  if (W != 32) return cudaErrorInvalidValue;
  return merge_pass_w<32>(segs, sbeg, send, tiles, grid, pass, src, dst, st);
}

}  // namespace bsort
