// bsort_strip_noalloc: the strip + tokenize step as a single kernel that
// allocates nothing.
//
// Some callers cannot call cudaMalloc: code that runs while a CUDA graph is
// being captured (an allocation there is illegal or would be baked into the
// graph), plugins inside a host framework that owns all device memory and
// forbids other allocators, and processes that must not grow their device
// footprint after start-up.  This entry point serves them: the caller passes
// the input and the output buffers, and the only scratch the kernel needs,
// one look-back record per 16 KiB chunk, lives in the file-scope device
// array below, which every GPU that loads the library holds until exit.
//
// The kernel is a single-document variant of the one-pass K1 of
// k_tokenize1p.cu without the length histogram: each CTA takes the next chunk
// from a ticket counter, publishes its chunk's
// summary, looks back over its predecessors' records until it meets one that
// holds an inclusive prefix (decoupled look-back), publishes its own
// inclusive prefix, and writes its letters and word starts.  Tickets are
// handed out in the order CTAs start, so every chunk a CTA waits for belongs
// to a CTA that is already running; each wait is still bounded, and a wait
// that runs out is counted and reported as BSORT_E_TIMEOUT.
#include <cstddef>
#include <mutex>

#include "bsort.h"
#include "bsort_dev.cuh"
#include "tok_common.cuh"

namespace bsort {
namespace {

constexpr uint32_t kNoAllocMaxChunks = 4096;  // 4096 chunks of 16 KiB: documents below 64 MiB
constexpr uint64_t kNoAllocMaxBytes = (uint64_t)kNoAllocMaxChunks * kChunk - 16;

struct LookbackRec {
  uint32_t status;  // 0: not yet, 1: agg holds the chunk's summary, 2: inc holds the prefix through it
  TokSum agg;
  TokSum inc;
  uint32_t pad;
};
static_assert(sizeof(LookbackRec) == 32, "look-back record is 32 bytes");

struct NoAllocScratch {
  uint32_t ticket;    // next chunk to hand out
  uint32_t finished;  // CTAs done
  uint32_t timeouts;  // look-back waits that ran out
  uint32_t pad[61];
  LookbackRec rec[kNoAllocMaxChunks];
};
constexpr size_t kNoAllocScratchBytes = sizeof(NoAllocScratch);  // 131,328 bytes

// The scratch.  Host code must not take this symbol's address with '&': on
// the host it names a stand-in, not device memory.  The device address comes
// from cudaGetSymbolAddress (see scratch_address below).
static __device__ __align__(256) uint8_t g_strip_scratch[kNoAllocScratchBytes];

__device__ __forceinline__ uint32_t ld_acquire(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(uint32_t* p, uint32_t v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ TokSum ld_sum(const TokSum* p) {
  const uint32_t* q = reinterpret_cast<const uint32_t*>(p);
  return TokSum{__ldcg(q), __ldcg(q + 1), __ldcg(q + 2)};
}
__device__ __forceinline__ void st_sum(TokSum* p, const TokSum& v) {
  uint32_t* q = reinterpret_cast<uint32_t*>(p);
  __stcg(q, v.letters);
  __stcg(q + 1, v.words);
  __stcg(q + 2, v.flags);
}

__global__ void __launch_bounds__(kTokThreads) k_strip_onepass(const uint8_t* __restrict__ in, uint64_t len,
                                                               uint32_t nchunks, uint8_t* scratch,
                                                               uint8_t* __restrict__ letters_out,
                                                               uint32_t* __restrict__ starts, uint32_t* totals,
                                                               uint64_t wait_limit) {
  NoAllocScratch* s = reinterpret_cast<NoAllocScratch*>(scratch);
  __shared__ uint4 buf[kChunk / 16];
  __shared__ uint32_t s_c;
  __shared__ TokSum s_prefix;
  if (threadIdx.x == 0) s_c = atomicAdd(&s->ticket, 1u);
  __syncthreads();
  const uint32_t c = s_c;

  // 16-byte granules that hold at least one byte of the document; the rest
  // (alignment slack, the tail) reads as spaces
  const uintptr_t first = reinterpret_cast<uintptr_t>(in);
  const uintptr_t last = first + len;
  const uintptr_t base = (first & ~uintptr_t(15)) + uintptr_t(c) * kChunk;
#pragma unroll
  for (int i = 0; i < kChunk / 16 / kTokThreads; ++i) {
    const int g = threadIdx.x + i * kTokThreads;
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
  const bool doc_start = c == 0 && threadIdx.x == 0;
  const TokSum mine = seg_summary(lm, sm, doc_start);
  TokSum total;
  const TokSum ex = block_exclusive(mine, &total);  // ends with __syncthreads: buf is free

  if (threadIdx.x == 0) {
    LookbackRec* rec = s->rec;
    TokSum prefix = {0, 0, 0};
    if (c == 0) {
      st_sum(&rec[0].inc, total);
      st_release(&rec[0].status, 2u);
    } else {
      st_sum(&rec[c].agg, total);
      st_release(&rec[c].status, 1u);
      TokSum acc = {0, 0, 0};
      for (int j = (int)c - 1; j >= 0; --j) {
        uint32_t st = 0;
        for (uint64_t it = 0; it < wait_limit; ++it) {
          st = ld_acquire(&rec[j].status);
          if (st) break;
          __nanosleep(32);
        }
        if (st == 0) {  // gave up: the prefix is incomplete, the call reports a timeout
          atomicAdd(&s->timeouts, 1u);
          break;
        }
        if (st == 2) {
          acc = tok_combine(ld_sum(&rec[j].inc), acc);
          break;
        }
        acc = tok_combine(ld_sum(&rec[j].agg), acc);
      }
      prefix = acc;
      st_sum(&rec[c].inc, tok_combine(prefix, total));
      st_release(&rec[c].status, 2u);
    }
    s_prefix = prefix;
  }
  __syncthreads();
  const TokSum cin = s_prefix;
  const TokSum pre = tok_combine(cin, ex);
  const bool ws_before = doc_start || ((pre.flags & kEv) && (pre.flags & kWs));
  uint64_t starts_m = start_mask(lm, sm, ws_before);
  uint32_t wpos = pre.words;
  while (starts_m) {
    const int b = __ffsll(starts_m) - 1;
    starts_m &= starts_m - 1;
    const uint64_t below = b ? (lm & (~0ull >> (64 - b))) : 0ull;
    starts[wpos++] = pre.letters + __popcll(below);
  }
  uint8_t* stage = reinterpret_cast<uint8_t*>(buf);
  uint32_t lpos = ex.letters;
  uint64_t m = lm;
  while (m) {
    const int b = __ffsll(m) - 1;
    m &= m - 1;
    stage[lpos++] = (uint8_t)(w[b >> 2] >> (8 * (b & 3)));
  }
  __syncthreads();
  for (uint32_t i = threadIdx.x; i < total.letters; i += kTokThreads) letters_out[cin.letters + i] = stage[i];
  if (threadIdx.x == 0) {
    if (c == nchunks - 1) {
      const TokSum all = tok_combine(cin, total);
      totals[0] = all.words;
      totals[1] = all.letters;
      starts[all.words] = all.letters;  // the last word ends at the end of the letters
    }
    __threadfence();
    if (atomicAdd(&s->finished, 1u) == nchunks - 1) {  // the last CTA to finish reports the status
      __threadfence();
      totals[2] = atomicAdd(&s->timeouts, 0u) ? (uint32_t)BSORT_E_TIMEOUT : 0u;
    }
  }
}

// Device address of g_strip_scratch, looked up once per device with that
// device current (the host-side name of the array is only a stand-in).
constexpr int kMaxDevices = 64;
void* g_scratch_ptr[kMaxDevices] = {};
std::mutex g_scratch_mutex;

cudaError_t scratch_address(int dev, void** out) {
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_strip_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

}  // namespace
}  // namespace bsort

extern "C" bsort_status bsort_strip_noalloc(const uint8_t* d_bytes, size_t len, void* stream, uint8_t* d_letters,
                                            uint32_t* d_starts, uint32_t* d_totals) {
  using namespace bsort;
  if (!d_totals || !d_starts || (len && (!d_bytes || !d_letters))) return BSORT_E_INVAL;
  if ((uint64_t)len > kNoAllocMaxBytes) return BSORT_E_TOO_LARGE;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return BSORT_E_CUDA;
  }
  void* scratch = nullptr;
  if (scratch_address(dev, &scratch) != cudaSuccess) {
    cudaGetLastError();
    return BSORT_E_CUDA;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const uint64_t mis = reinterpret_cast<uintptr_t>(d_bytes) & 15u;
  const uint32_t nchunks = len ? (uint32_t)((mis + len + kChunk - 1) / kChunk) : 0u;
  cudaError_t e;
  if (nchunks == 0) {
    e = cudaMemsetAsync(d_totals, 0, 3 * sizeof(uint32_t), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_starts, 0, sizeof(uint32_t), st);
  } else {
    // the ticket, the counters and the records that this call uses start at zero
    const size_t used = offsetof(NoAllocScratch, rec) + (size_t)nchunks * sizeof(LookbackRec);
    e = cudaMemsetAsync(scratch, 0, used, st);
    if (e == cudaSuccess) {
      k_strip_onepass<<<nchunks, kTokThreads, 0, st>>>(d_bytes, len, nchunks, static_cast<uint8_t*>(scratch),
                                                       d_letters, d_starts, d_totals, kDefaultWaitLimit);
      e = cudaGetLastError();
    }
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    return BSORT_E_CUDA;
  }
  return BSORT_OK;
}
