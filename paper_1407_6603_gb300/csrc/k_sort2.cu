// K4's warp sort for tiny buckets and K5, the merge passes, for keys of up
// to 8 u64 words: phase 3 of the paper's method, the sort of each length
// bucket into ASCII order (Section II; Section III step 4).  The tile sort
// itself (clusters of CTAs) is in tile_sort2.cuh.
//
// K5 (k_merge_pass2<W>, and the pipelined k_merge_cut<W> + k_merge_piped<W>)
// merges run pairs, one pass per launch and key width, for every bucket of
// that width.  Each CTA produces output tiles; where a tile's output diagonal
// cuts the two runs (merge path) is found by a parallel search in global
// memory, and the tile is merged in shared memory.
#include "tile_sort2.cuh"

namespace bsort {
namespace {

// ------------------------------------------------------- tiny buckets ----
// Buckets of at most 32 * KPT keys: one warp each.  The keys go to registers
// (lane l holds keys l*KPT .. l*KPT+KPT-1, +inf past the end), each lane
// sorts its KPT keys by odd-even transposition, then G lanes, G the smallest
// power of two that holds the bucket, run G rounds of odd-even transposition
// between neighbours.  No shared memory and no barrier.
template <int W, int G>
__device__ void warp_sort_g(const Segment& sg, const uint64_t* g, uint32_t n, const EmitOut& eo) {
  constexpr int KPT = kpt2<W>();
  const int lane = threadIdx.x & 31;
  Key<W> k[KPT];
#pragma unroll
  for (int i = 0; i < KPT; ++i) {
    const uint32_t p = lane * KPT + i;
    k[i] = p < n ? kload<W>(g + (size_t)p * W) : kinf<W>();
  }
  oets_registers<W, KPT>(k);
  if (G > 1) oets_lanes<W, KPT, (G > 1 ? G : 2)>(k);
  if (sg.flags & kSegKeysOut) {  // the sorted keys stay in place
#pragma unroll
    for (int i = 0; i < KPT; ++i) {
      const uint32_t p = lane * KPT + i;
      if (p < n) kstore<W>(const_cast<uint64_t*>(g) + (size_t)p * W, k[i]);
    }
    return;
  }
  // the bucket is sorted: each lane writes its keys' letters and offsets
  const uint32_t L = sg.L;
#pragma unroll
  for (int i = 0; i < KPT; ++i) {
    const uint32_t p = lane * KPT + i;
    if (p < n) {
      uint8_t* dst = eo.stream + sg.stream_off + (size_t)p * L;
      if (eo.codec == kCodeBytes) {
#pragma unroll
        for (int q = 0; q < W; ++q)
#pragma unroll
          for (int b = 0; b < 8; ++b)
            if ((uint32_t)(q * 8 + b) < L) dst[q * 8 + b] = (uint8_t)(k[i].w[q] >> (56 - 8 * b));
      } else {
        uint64_t kw[W];  // (a copy, so that k itself is only indexed by constants)
#pragma unroll
        for (int q = 0; q < W; ++q) kw[q] = k[i].w[q];
        for (uint32_t q = 0; q * 8 < L; ++q) {
          const uint64_t a = ascii8(eo.codec, L, [&](uint32_t w) { return kw[w]; }, q);
          for (uint32_t b = 0; b < 8 && q * 8 + b < L; ++b) dst[q * 8 + b] = (uint8_t)(a >> (56 - 8 * b));
        }
      }
      if (eo.want_offsets) eo.offsets[sg.out_word + p] = sg.stream_off - sg.doc_stream0 + p * L;
    }
  }
}

template <int W>
__device__ void warp_sort(const Segment& sg, const uint64_t* g, uint32_t n, const EmitOut& eo) {
  constexpr int KPT = kpt2<W>();
  const uint32_t lanes = (n + KPT - 1) / KPT;
  if (lanes <= 1)
    warp_sort_g<W, 1>(sg, g, n, eo);
  else if (lanes <= 2)
    warp_sort_g<W, 2>(sg, g, n, eo);
  else if (lanes <= 4)
    warp_sort_g<W, 4>(sg, g, n, eo);
  else if (lanes <= 8)
    warp_sort_g<W, 8>(sg, g, n, eo);
  else if (lanes <= 16)
    warp_sort_g<W, 16>(sg, g, n, eo);
  else
    warp_sort_g<W, 32>(sg, g, n, eo);
}

__global__ void __launch_bounds__(256) k_warp_sort(const Segment* __restrict__ segs, uint32_t sbeg, uint32_t send,
                                                   const uint64_t* keys, EmitOut eo) {
  const uint32_t warps = gridDim.x * (blockDim.x / 32);
  for (uint32_t i = sbeg + blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32; i < send; i += warps) {
    const Segment& sg = segs[i];
    const uint64_t* g = keys + sg.key_off;
    switch (sg.W) {
      case 1: warp_sort<1>(sg, g, sg.n, eo); break;
      case 2: warp_sort<2>(sg, g, sg.n, eo); break;
      case 4: warp_sort<4>(sg, g, sg.n, eo); break;
      default: warp_sort<8>(sg, g, sg.n, eo); break;
    }
  }
}

// ---------------------------------------------------------------- K5 ----

struct SplitCarry {
  uint32_t seg;
  uint32_t d1;
  uint32_t a1;
  uint64_t ps;
};

// One output tile of one merge pass for keys of W words: T = merge2_keys(W)
// keys (2048 u64 words; 4096 for W = 16).  The two input slices sit in sm in
// the padded layout; each thread merges its KPT outputs into registers.
template <int W>
__device__ void merge_tile(const Segment& sg, uint32_t si, uint32_t it, uint32_t pass,
                           const uint64_t* src, uint64_t* dst, uint64_t* sm,
                           SplitCarry& carry, const EmitOut& eo) {
  constexpr int KPT = W >= 8 ? 1 : 8 / W;
  constexpr uint32_t T = kM2Threads * KPT;
  const int t = threadIdx.x;
  const uint64_t n = sg.n;
  const uint64_t R = (uint64_t)sg.run0 << pass;
  const uint64_t out0 = (uint64_t)(it - sg.tile0) * T;
  const uint64_t ps = out0 / (2 * R) * (2 * R);
  const uint32_t la = (uint32_t)min(R, n - ps);
  const uint32_t lb = n - ps > R ? (uint32_t)min(R, n - ps - R) : 0u;
  const uint32_t d0 = (uint32_t)(out0 - ps);
  const uint32_t cnt = min(T, la + lb - d0);
  const uint32_t d1 = d0 + cnt;
  const uint64_t* A = src + sg.key_off + ps * W;
  const uint64_t* B = A + (size_t)la * W;
  uint64_t* out = dst + sg.key_off + (ps + d0) * W;
  // this pass's output is the sorted bucket, whose words go out (unless its
  // sorted keys are what is wanted)
  const bool last = pass + 1 == sg.passes && !(sg.flags & kSegKeysOut);
  if (lb == 0 && last) {  // odd run at the end of the bucket, already in place
    const uint64_t* a = A + (size_t)d0 * W;
    emit_tile<kM2Threads>(sg, (uint32_t)out0, cnt, [&](uint32_t j, uint32_t q) { return a[(size_t)j * W + q]; }, eo);
    return;
  }
  if (lb == 0) {  // odd run at the end of the bucket: carried over
    constexpr int kPer = (T * W + kM2Threads - 1) / kM2Threads;
    const uint64_t* a = A + (size_t)d0 * W;
#pragma unroll
    for (int j0 = 0; j0 < kPer; j0 += 4) {
      uint64_t v[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const uint32_t e = t + (j0 + j) * kM2Threads;
        if (e < cnt * W) v[j] = a[e];
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const uint32_t e = t + (j0 + j) * kM2Threads;
        if (e < cnt * W) out[e] = v[j];
      }
    }
    return;
  }
  // the tile's two cuts, one warp each side by side (the first is the
  // previous tile's second when the CTA just merged that tile)
  __shared__ uint32_t s_cut[2];
  const bool have0 = carry.seg == si && carry.ps == ps && carry.d1 == d0;
  const uint32_t wid = threadIdx.x >> 5;
  if (wid < 2 && !(wid == 0 && have0)) {
    auto kA_ = [&](uint32_t i) { return kload<W>(A + (size_t)i * W); };
    auto kB_ = [&](uint32_t i) { return kload<W>(B + (size_t)i * W); };
    const uint32_t v = warp_split_fn<W>(kA_, la, kB_, lb, wid ? d1 : d0);
    if ((threadIdx.x & 31) == 0) s_cut[wid] = v;
  }
  __syncthreads();
  const uint32_t a0 = have0 ? carry.a1 : s_cut[0];
  const uint32_t a1 = s_cut[1];
  carry = SplitCarry{si, d1, a1, ps};
  // Sorted runs give monotone cuts.  Runs read before their pass finished
  // (a grid barrier that gave up: the call already reports a timeout) may
  // not; such a tile is skipped, so every access stays in bounds.
  if (a1 < a0 || d1 - a1 < d0 - a0) return;
  const uint32_t na = a1 - a0, nb = (d1 - a1) - (d0 - a0);
  const uint64_t* gA = A + (size_t)a0 * W;
  const uint64_t* gB = B + (size_t)(d0 - a0) * W;
  {
    // a thread's loads four at a time before their stores, so they fly together
    constexpr int kPer = (T * W + kM2Threads - 1) / kM2Threads;
    const uint32_t wa = na * W, tot = cnt * W;
#pragma unroll
    for (int j0 = 0; j0 < kPer; j0 += 4) {
      uint64_t v[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const uint32_t e = t + (j0 + j) * kM2Threads;
        if (e < tot) v[j] = e < wa ? gA[e] : gB[e - wa];
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const uint32_t e = t + (j0 + j) * kM2Threads;
        if (e < tot) sm[padw(e)] = v[j];
      }
    }
  }
  __syncthreads();
  Key<W> k[KPT];
  const uint32_t pos = t * KPT;
  if (pos < cnt) {
    auto sA = [&](uint32_t i) { return kload<W>(pkey<W>(sm, i)); };
    auto sB = [&](uint32_t i) { return kload<W>(pkey<W>(sm, na + i)); };
    const uint32_t a = mp_split_f<W>(sA, na, sB, nb, pos);
    merge_run_buf<W, KPT>(sm, 0, na, na, nb, a, pos - a, k);
  }
  __syncthreads();
#pragma unroll
  for (int s = 0; s < KPT; ++s)
    if (pos + s < cnt) kstore<W>(pkey<W>(sm, pos + s), k[s]);
  __syncthreads();
  if (last)
    emit_tile<kM2Threads>(sg, (uint32_t)out0, cnt, [&](uint32_t j, uint32_t q) { return sm[padw(j * W + q)]; }, eo);
  else
    for (uint32_t e = t; e < cnt * W; e += kM2Threads) out[e] = sm[padw(e)];
  __syncthreads();
}

// Grid-wide barrier of a cooperative launch (every CTA resident): CTA
// arrivals counted on `counter`, generation `gen` complete when the count
// reaches (gen + 1) * gridDim.x.  The wait is bounded: when it runs out the
// call is marked timed out and the CTA goes on.
__device__ __forceinline__ void grid_barrier(uint32_t* counter, uint32_t gen, Meta* meta, uint64_t wait_limit) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(counter, 1u);
    const uint32_t target = (gen + 1) * gridDim.x;
    uint64_t polls = 0;
    for (;;) {
      uint32_t v;
      asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(counter) : "memory");
      if (v >= target) break;
      if (++polls >= wait_limit) {
        atomicAdd(&meta->err_timeout, 1u);
        break;
      }
      __nanosleep(64);
    }
    __threadfence();  // the other CTAs' writes of the pass are seen from here on
  }
  __syncthreads();
}

// Merge passes pass0 .. pass0 + npass - 1 over the buckets [sbeg, send) of
// key width W, the keys moving between kA and kB (pass p reads kA when p is
// even).  With npass > 1 the launch is cooperative and the passes are
// separated by grid barriers, one launch for all of them.
template <int W>
__global__ void __launch_bounds__(kM2Threads, BSORT_K5_MIN_CTAS) k_merge_pass2(
    const Segment* __restrict__ segs, uint32_t sbeg, uint32_t send, uint32_t tiles, uint32_t pass0, uint32_t npass,
    uint32_t chunk, uint64_t* kA, uint64_t* kB, EmitOut eo, uint32_t* barrier, Meta* meta, uint64_t wait_limit) {
  extern __shared__ __align__(128) uint64_t sm[];
  __shared__ uint32_t s_seg;
  __shared__ uint32_t s_first[kSegCache];
  const bool cached = seg_cache_fill<kByTile0>(segs, sbeg, send, s_first);
  const uint32_t nchunk = (tiles + chunk - 1) / chunk;
  for (uint32_t q = 0; q < npass; ++q) {
    const uint32_t pass = pass0 + q;
    const uint64_t* src = (pass & 1) ? kB : kA;
    uint64_t* dst = (pass & 1) ? kA : kB;
    if (q > 0) grid_barrier(barrier, q - 1, meta, wait_limit);
    // chunks of `chunk` consecutive tiles, dealt round-robin: within a chunk a
    // tile's start split is the previous tile's end split; with few tiles the
    // host asks for chunks of one so that no CTA serialises several
    SplitCarry carry{~0u, ~0u, 0u, ~0ull};
    for (uint32_t ch = blockIdx.x; ch < nchunk; ch += gridDim.x)
      for (uint32_t it = ch * chunk; it < min(tiles, ch * chunk + chunk); ++it) {
        if (threadIdx.x < 32) {
          const uint32_t v = seg_find_warp<kByTile0>(segs, sbeg, send, s_first, cached, it);
          if (threadIdx.x == 0) s_seg = v;
        }
        __syncthreads();
        const uint32_t si = s_seg;
        const Segment sg = segs[si];
        __syncthreads();
        if (sg.passes <= pass) continue;  // this bucket is already one run
        merge_tile<W>(sg, si, it, pass, src, dst, sm, carry, eo);
      }
  }
}

// ------------------------------------------------- pipelined K5 ----
// The cut kernel: one warp per output tile of the pass finds, by a 32-way
// merge-path search, where the tile's first output cuts the two runs (its end
// is the next tile's start), and lane 0 writes the tile's job.  Entry `tiles`
// is a sentinel whose run-A start lies past every run.
template <int W>
__global__ void __launch_bounds__(256) k_merge_cut(const Segment* __restrict__ segs, uint32_t sbeg, uint32_t send,
                                                   uint32_t tiles, uint32_t pass, const uint64_t* __restrict__ src,
                                                   const uint64_t* __restrict__ samples,
                                                   TileJob* __restrict__ jobs) {
  constexpr int KPT = W >= 8 ? 1 : 8 / W;
  constexpr uint32_t T = kM2Threads * KPT;
  __shared__ uint32_t s_first[kSegCache];
  const bool cached = seg_cache_fill<kByTile0>(segs, sbeg, send, s_first);
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t warps = gridDim.x * (blockDim.x / 32);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    TileJob end{};
    end.a_src = ~0ull;
    jobs[tiles] = end;
  }
  // 32-way search for the first m in [lo, hi) where the monotone predicate
  // f (true, then false) is false; hi if none.  Uniform across the warp.
  auto first_false = [&](uint32_t lo, uint32_t hi, auto f) {
    while (hi > lo) {
      const uint32_t span = hi - lo;
      const uint32_t step = span <= 32u ? 1u : (span + 31u) / 32u;
      const uint32_t m = lo + lane * step;
      const bool t = m < hi && f(m);
      const uint32_t nt = __popc(__ballot_sync(kFull, t));
      // the answer lies after the last probe that holds, up to the next probe
      const uint32_t nhi = lo + nt * step < hi ? lo + nt * step : hi;
      lo = nt == 0 ? lo : lo + (nt - 1) * step + 1;
      hi = nhi;
    }
    return lo;
  };
  for (uint32_t it = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32; it < tiles; it += warps) {
    const uint32_t si = seg_find_warp<kByTile0>(segs, sbeg, send, s_first, cached, it);
    const Segment& sg = segs[si];
    TileJob job{};
    job.smp = kNoSamples;
    const uint32_t passes = sg.passes;
    const uint64_t out0 = (uint64_t)(it - sg.tile0) * T;
    job.a_src = sg.key_off + out0 * W;  // (a bucket already in one run: monotone, no outputs)
    if (passes > pass) {
      const uint64_t n = sg.n, R = (uint64_t)sg.run0 << pass;
      const uint64_t ps = out0 / (2 * R) * (2 * R);
      const uint32_t la = (uint32_t)min(R, n - ps);
      const uint32_t lb = n - ps > R ? (uint32_t)min(R, n - ps - R) : 0u;
      const uint32_t d = (uint32_t)(out0 - ps);
      const uint64_t* A = src + sg.key_off + ps * W;
      const uint64_t* B = A + (size_t)la * W;
      // the cut: the first m where A[m] goes after the diagonal's B key
      // B[d-1-m] (A's keys first among equals)
      uint32_t lo = d > lb ? d - lb : 0u, hi = d < la ? d : la;
      if (pass > 0 && hi > lo) {
        // The previous pass stored this pass's A keys at positions 31 (mod 32)
        // and B keys at positions 0 (mod 32) (run starts and d are multiples
        // of 32), so the probes m = 32i + 31 read A[m] and B[d-1-m] = B[d - 32(i+1)]
        // from the sample buffer.  They pin the cut to 32 positions.
        const uint64_t* sA = samples + sg.smp_off + (ps / 32) * W;
        const uint64_t* sB = samples + sg.smp_off + ((ps + la + d) / 32 - 1) * W;
        const uint32_t i_f = first_false(lo / 32, hi / 32, [&](uint32_t i) {
          return !klt(kload<W>(sB - (size_t)i * W), kload<W>(sA + (size_t)i * W));
        });
        lo = max(lo, 32 * i_f);
        hi = min(hi, 32 * i_f + 31);
      }
      lo = first_false(lo, hi, [&](uint32_t m) {
        return !klt(kload<W>(B + (size_t)(d - 1 - m) * W), kload<W>(A + (size_t)m * W));
      });
      job.a_src = sg.key_off + (ps + lo) * W;
      job.b_src = sg.key_off + (ps + la + (d - lo)) * W;
      job.a_end = sg.key_off + (ps + la) * W;
      job.dst = sg.key_off + out0 * W;
      job.cnt = min(T, la + lb - d);
      if (pass + 1 == passes && (sg.flags & kSegKeysOut)) {
        // the sorted keys themselves are the result: written to dst, no samples
      } else if (pass + 1 == passes) {
        job.L = sg.L;
        job.stream = sg.stream_off + (uint32_t)out0 * sg.L;
        job.word = sg.out_word + (uint32_t)out0;
        job.rel = job.stream - sg.doc_stream0;
      } else {
        // samples for the next pass's cut: the tile lies in one run of that
        // pass (its runs are 2R long, a multiple of T); A runs sample their
        // positions 31 (mod 32), B runs their positions 0 (mod 32)
        job.smp = sg.smp_off + (uint32_t)(out0 / 32) * W;
        job.smp_phase = (out0 / (2 * R)) % 2 == 0 ? 31u : 0u;
      }
    }
    if (lane == 0) jobs[it] = job;
  }
}

// The merge kernel: each CTA takes every gridDim.x-th tile.  Per tile: wait
// for its slices (and the next tile's job), start the copies of the next
// tile's slices into the other buffer and the job after it, then merge this
// tile (merge path per thread in shared memory) and write it out.
template <int W>
__global__ void __launch_bounds__(kM2Threads, BSORT_K5_MIN_CTAS) k_merge_piped(const TileJob* __restrict__ jobs,
                                                                              uint32_t tiles,
                                                                              const uint64_t* __restrict__ src,
                                                                              uint64_t* __restrict__ dst,
                                                                              uint64_t* __restrict__ samples, EmitOut eo) {
  constexpr int KPT = W >= 8 ? 1 : 8 / W;
  constexpr uint32_t TW = kM2Threads * KPT * W;
  extern __shared__ __align__(128) uint64_t sm[];  // two tile buffers, padded layout
  __shared__ __align__(16) TileJob s_job[3];
  __shared__ __align__(8) uint64_t s_next[3];  // the next tile's a_src
  const uint32_t bw = padded_words(TW);
  const int t = threadIdx.x;
  const uint32_t G = gridDim.x;
  auto fetch_job = [&](uint32_t k) {  // the CTA's k-th job into ring slot k % 3
    const uint32_t it = blockIdx.x + k * G;
    if (it < tiles && t < 4)
      cp_async16(reinterpret_cast<uint4*>(&s_job[k % 3]) + t, reinterpret_cast<const uint4*>(jobs + it) + t);
    if (it < tiles && t == 4) cp_async8(&s_next[k % 3], &jobs[it + 1].a_src);
  };
  // keys of the job's tile taken from run A
  auto na_of = [&](uint32_t k) {
    const TileJob& j = s_job[k % 3];
    const uint64_t a1 = s_next[k % 3] < j.a_end ? s_next[k % 3] : j.a_end;
    return (uint32_t)((a1 - j.a_src) / W);
  };
  auto fetch_data = [&](uint32_t k) {  // its slices into buffer k & 1: A's keys, then B's
    if (blockIdx.x + k * G >= tiles) return;
    const TileJob& j = s_job[k % 3];
    const uint32_t wa = j.cnt ? na_of(k) * W : 0u, tot = j.cnt * W;
    uint64_t* buf = sm + (k & 1) * bw;
    for (uint32_t e = t; e < tot; e += kM2Threads) cp_async8(buf + padw(e), src + (e < wa ? j.a_src + e : j.b_src + (e - wa)));
  };
  fetch_job(0);
  cp_async_commit();
  cp_async_wait_all();
  __syncthreads();
  fetch_data(0);
  fetch_job(1);
  cp_async_commit();
  for (uint32_t k = 0; blockIdx.x + k * G < tiles; ++k) {
    cp_async_wait_all();
    __syncthreads();  // tile k's slices and job k+1 are in; tile k-1 is out
    fetch_data(k + 1);
    fetch_job(k + 2);
    cp_async_commit();
    const TileJob& j = s_job[k % 3];
    const uint32_t cnt = j.cnt;
    if (cnt == 0) continue;
    const uint32_t na = na_of(k), nb = cnt - na;
    uint64_t* buf = sm + (k & 1) * bw;
    Key<W> kk[KPT];
    const uint32_t pos = t * KPT;
    if (pos < cnt) {
      auto sA = [&](uint32_t i) { return kload<W>(pkey<W>(buf, i)); };
      auto sB = [&](uint32_t i) { return kload<W>(pkey<W>(buf, na + i)); };
      const uint32_t a = mp_split_f<W>(sA, na, sB, nb, pos);
      merge_run_buf<W, KPT>(buf, 0, na, na, nb, a, pos - a, kk);
      if (j.smp != kNoSamples) {  // one output in 32 for the next pass's cut
#pragma unroll
        for (int s = 0; s < KPT; ++s)
          if ((pos + s) % 32 == j.smp_phase && pos + s < cnt)
            kstore<W>(samples + j.smp + (size_t)((pos + s) / 32) * W, kk[s]);
      }
    }
    __syncthreads();
#pragma unroll
    for (int s = 0; s < KPT; ++s)
      if (pos + s < cnt) kstore<W>(pkey<W>(buf, pos + s), kk[s]);
    __syncthreads();
    const uint32_t L = j.L;
    if (L) {
      emit_run<kM2Threads>(L, eo.stream + j.stream, eo.want_offsets ? eo.offsets + j.word : nullptr, j.rel, cnt,
                           [&](uint32_t q, uint32_t w) { return buf[padw(q * W + w)]; }, eo.codec);
    } else {
      uint64_t* out = dst + j.dst;
      for (uint32_t e = t; e < cnt * W; e += kM2Threads) out[e] = buf[padw(e)];
    }
  }
  cp_async_wait_all();
}

template <int W>
cudaError_t merge_pass2_w(const Segment* segs, uint32_t sbeg, uint32_t send, uint32_t tiles, uint32_t grid,
                          uint32_t pass0, uint32_t npass, uint64_t* kA, uint64_t* kB, const EmitOut& eo,
                          uint32_t* barrier, Meta* meta, uint64_t wait_limit, cudaStream_t st) {
  constexpr uint32_t words = kM2Threads * (W >= 8 ? 1 : 8 / W) * W;
  const size_t smem = (size_t)padded_words(words) * 8;
  // (the default carveout stays: the merge-path probes live in L1)
  static int attr_done[64];
  static int resident[64];  // CTAs per SM, for the cooperative form
  cudaError_t e = once_per_device(attr_done, [&] {
    cudaError_t r = smem > 48 * 1024
                        ? cudaFuncSetAttribute(k_merge_pass2<W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)
                        : cudaSuccess;
    int dev = 0, per_sm = 0;
    if (r == cudaSuccess) r = cudaGetDevice(&dev);
    if (r == cudaSuccess) r = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_merge_pass2<W>, kM2Threads, smem);
    if (r == cudaSuccess && dev >= 0 && dev < 64) resident[dev] = per_sm;
    return r;
  });
  if (e != cudaSuccess) return e;
  const uint32_t chunk = tiles >= 4u * grid ? 4u : 1u;
  const uint32_t nchunk = (tiles + chunk - 1) / chunk;
  uint32_t g = nchunk < grid ? nchunk : grid;
  if (npass <= 1) {
    k_merge_pass2<W><<<g, kM2Threads, smem, st>>>(segs, sbeg, send, tiles, pass0, 1u, chunk, kA, kB, eo, barrier, meta,
                                                 wait_limit);
    return cudaGetLastError();
  }
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return cudaErrorUnknown;
  // at most a quarter of what fits on the device: the chains of the four key
  // widths may each run one of these grids at the same time, and all of them
  // must be resident together
  const uint32_t cap = (uint32_t)(resident[dev >= 0 && dev < 64 ? dev : 0] * sms) / 4;
  if (cap == 0) return cudaErrorCooperativeLaunchTooLarge;
  if (g > cap) g = cap;
  void* args[] = {&segs, &sbeg, &send, &tiles, &pass0, &npass, const_cast<uint32_t*>(&chunk), &kA, &kB,
                  const_cast<EmitOut*>(&eo), &barrier, &meta, &wait_limit};
  return cudaLaunchCooperativeKernel(reinterpret_cast<void*>(k_merge_pass2<W>), dim3(g), dim3(kM2Threads), args, smem,
                                     st);
}

}  // namespace

cudaError_t launch_warp_sort(const Segment* segs, uint32_t sbeg, uint32_t send, uint64_t* keys, EmitOut eo,
                             cudaStream_t st) {
  if (send <= sbeg) return cudaSuccess;
  const uint32_t warps = send - sbeg;
  const uint32_t grid = (warps + 7) / 8 < 152u * 16u ? (warps + 7) / 8 : 152u * 16u;
  k_warp_sort<<<grid, 256, 0, st>>>(segs, sbeg, send, keys, eo);
  return cudaGetLastError();
}

cudaError_t launch_tile_sort2(int cluster, int lanes, int threads, const Segment* segs, uint32_t sbeg, uint32_t send,
                              uint32_t supertiles, int max_grid, int max_width, uint64_t* keys, EmitOut eo, Meta* meta,
                              uint64_t wait_limit, cudaStream_t st) {
  if (supertiles == 0) return cudaSuccess;
  switch (lanes) {
    case 2: return launch_tile_sort2_g2(cluster, threads, segs, sbeg, send, supertiles, max_grid, max_width, keys, eo, meta, wait_limit, st);
    case 4: return launch_tile_sort2_g4(cluster, threads, segs, sbeg, send, supertiles, max_grid, max_width, keys, eo, meta, wait_limit, st);
    case 8: return launch_tile_sort2_g8(cluster, threads, segs, sbeg, send, supertiles, max_grid, max_width, keys, eo, meta, wait_limit, st);
    default: return cudaErrorInvalidValue;
  }
}

int merge_piped_ctas_per_sm() { return BSORT_K5_MIN_CTAS; }

cudaError_t launch_merge_cut(int W, const Segment* segs, uint32_t sbeg, uint32_t send, uint32_t tiles, uint32_t pass,
                             const uint64_t* src, const uint64_t* samples, TileJob* jobs, cudaStream_t st) {
  if (tiles == 0) return cudaSuccess;
  const uint32_t grid = (tiles + 7) / 8;
  switch (W) {
    case 1: k_merge_cut<1><<<grid, 256, 0, st>>>(segs, sbeg, send, tiles, pass, src, samples, jobs); break;
    case 2: k_merge_cut<2><<<grid, 256, 0, st>>>(segs, sbeg, send, tiles, pass, src, samples, jobs); break;
    case 4: k_merge_cut<4><<<grid, 256, 0, st>>>(segs, sbeg, send, tiles, pass, src, samples, jobs); break;
    case 8: k_merge_cut<8><<<grid, 256, 0, st>>>(segs, sbeg, send, tiles, pass, src, samples, jobs); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <int W>
cudaError_t merge_piped_w(const TileJob* jobs, uint32_t tiles, uint32_t grid, const uint64_t* src, uint64_t* dst,
                          uint64_t* samples, const EmitOut& eo, cudaStream_t st) {
  constexpr uint32_t words = kM2Threads * (W >= 8 ? 1 : 8 / W) * W;
  const size_t smem = 2 * (size_t)padded_words(words) * 8;
  static int attr_done[64];
  cudaError_t e = once_per_device(attr_done, [&] {
    return smem > 48 * 1024
               ? cudaFuncSetAttribute(k_merge_piped<W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)
               : cudaSuccess;
  });
  if (e != cudaSuccess) return e;
  k_merge_piped<W><<<grid < tiles ? grid : tiles, kM2Threads, smem, st>>>(jobs, tiles, src, dst, samples, eo);
  return cudaGetLastError();
}

cudaError_t launch_merge_piped(int W, const TileJob* jobs, uint32_t tiles, uint32_t grid, const uint64_t* src,
                               uint64_t* dst, uint64_t* samples, EmitOut eo, cudaStream_t st) {
  if (tiles == 0 || grid == 0) return cudaSuccess;
  switch (W) {
    case 1: return merge_piped_w<1>(jobs, tiles, grid, src, dst, samples, eo, st);
    case 2: return merge_piped_w<2>(jobs, tiles, grid, src, dst, samples, eo, st);
    case 4: return merge_piped_w<4>(jobs, tiles, grid, src, dst, samples, eo, st);
    case 8: return merge_piped_w<8>(jobs, tiles, grid, src, dst, samples, eo, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_merge_pass2(int W, const Segment* segs, uint32_t sbeg, uint32_t send, uint32_t tiles,
                               uint32_t grid, uint32_t pass0, uint32_t npass, uint64_t* kA, uint64_t* kB, EmitOut eo,
                               uint32_t* barrier, Meta* meta, uint64_t wait_limit, cudaStream_t st) {
  if (tiles == 0 || grid == 0) return cudaSuccess;
  switch (W) {
    case 1: return merge_pass2_w<1>(segs, sbeg, send, tiles, grid, pass0, npass, kA, kB, eo, barrier, meta, wait_limit, st);
    case 2: return merge_pass2_w<2>(segs, sbeg, send, tiles, grid, pass0, npass, kA, kB, eo, barrier, meta, wait_limit, st);
    case 4: return merge_pass2_w<4>(segs, sbeg, send, tiles, grid, pass0, npass, kA, kB, eo, barrier, meta, wait_limit, st);
    case 8: return merge_pass2_w<8>(segs, sbeg, send, tiles, grid, pass0, npass, kA, kB, eo, barrier, meta, wait_limit, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace bsort
