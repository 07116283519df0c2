// Host runtime and C ABI of libbsort (declared in include/bsort.h).
//
// One call runs the whole path for one or more documents on one CUDA stream:
//   K1           strip + tokenize and per-document length counts, one pass
//                (paper Section II, phase 1; the counts size phase 2)
//   -- the host reads the counts back and lays out one bucket per
//      (document, length): key offsets, tiles, merge passes --
//   K3           scatter words into buckets as packed keys (phase 2)
//   K4, K5       sort every bucket: odd-even transposition tiles, then
//                merge-path passes (phase 3)
//   K6           write counts, offsets and the sorted stream
// The only host/device synchronisation inside a call is the read of the
// length counts; everything after it is enqueued without waiting.
#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <new>
#include <string>
#include <vector>

#include "bsort.h"
#include "bsort_dev.cuh"
#include "layout_bounds.h"

using namespace bsort;

namespace {

struct DevBuf {
  void* p = nullptr;
  size_t cap = 0;
};
struct HostBuf {
  void* p = nullptr;
  size_t cap = 0;
};

// ceil(log2(n)) for n >= 1 (0 for n <= 1)
double ceil_log2(uint64_t n) { return n <= 1 ? 0.0 : (double)(64 - __builtin_clzll(n - 1)); }

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Tuning chosen per bucket-size class (see bsort_config.tune_table).  The
// built-in values are what the autotuner (autotune.py) picked on a GB300.
struct Tune {
  int k4_lanes[4] = {2, 2, 2, 2};  // clusters of 1, 2, 4, 8 CTAs
  int k4_threads[4] = {256, 256, 256, 256};  // CTA size for the same classes (512: keys of up to 4 words)
  uint32_t piped_min = 1;
  int k4_streams = 1;  // 1: the tile sorts of the smaller classes run on side streams
  int k4_runs = 2;     // cluster size (runs of that many tiles) for buckets that need pipelined merge passes
  int k4_runs_small = 16;  // the same when their merges are too small to pipeline
  int dedupe = 1;          // the duplicate-aware sort for the buckets that need merge passes:
                           // 0 never, 1 on large inputs, 2 always
};

// Parses a tune table; false on an unknown key or a bad value.
bool parse_tune(const char* text, Tune& t) {
  if (!text) return true;
  std::string s(text);
  size_t i = 0;
  auto is_sep = [](char ch) { return ch == ' ' || ch == '\t' || ch == '\n' || ch == '\r' || ch == ';'; };
  while (i < s.size()) {
    if (is_sep(s[i])) {
      ++i;
      continue;
    }
    if (s[i] == '#') {
      while (i < s.size() && s[i] != '\n') ++i;
      continue;
    }
    size_t j = i;
    while (j < s.size() && !is_sep(s[j]) && s[j] != '#') ++j;
    const std::string item = s.substr(i, j - i);
    i = j;
    const size_t eq = item.find('=');
    if (eq == std::string::npos) return false;
    const std::string key = item.substr(0, eq), val = item.substr(eq + 1);
    std::vector<long> nums;
    size_t k = 0;
    while (k <= val.size()) {
      size_t e = val.find(',', k);
      if (e == std::string::npos) e = val.size();
      const std::string tok = val.substr(k, e - k);
      if (tok.empty() || tok.size() > 9 || tok.find_first_not_of("0123456789") != std::string::npos) return false;
      nums.push_back(std::stol(tok));
      k = e + 1;
    }
    if (key == "k4_lanes") {
      if (nums.size() != 4) return false;
      for (int q = 0; q < 4; ++q) {
        if (nums[q] != 2 && nums[q] != 4 && nums[q] != 8) return false;
        t.k4_lanes[q] = (int)nums[q];
      }
    } else if (key == "k4_runs") {
      if (nums.size() != 1 || (nums[0] != 1 && nums[0] != 2 && nums[0] != 4 && nums[0] != 8)) return false;
      t.k4_runs = (int)nums[0];
    } else if (key == "k4_runs_small") {
      if (nums.size() != 1 || (nums[0] != 8 && nums[0] != 16)) return false;
      t.k4_runs_small = (int)nums[0];
    } else if (key == "k4_streams") {
      if (nums.size() != 1 || nums[0] > 1) return false;
      t.k4_streams = (int)nums[0];
    } else if (key == "k4_threads") {
      if (nums.size() != 4) return false;
      for (int q = 0; q < 4; ++q) {
        if (nums[q] != 256 && nums[q] != 512) return false;
        t.k4_threads[q] = (int)nums[q];
      }
    } else if (key == "dedupe") {
      if (nums.size() != 1 || nums[0] > 2) return false;
      t.dedupe = (int)nums[0];
    } else if (key == "piped_min") {
      if (nums.size() != 1 || nums[0] < 1 || nums[0] > 1000000) return false;
      t.piped_min = (uint32_t)nums[0];
    } else {
      return false;
    }
  }
  return true;
}

// The meta region: what K1 leaves for the host (read back in one copy of
// `total` bytes), then K1's look-back scratch and K2's work area (its
// accumulators, its summary, the merge chains' barrier counters); one memset
// clears all three.
struct MetaLayout {
  size_t meta = 0, wbase = 0, lbase = 0, item0 = 0, maxlen = 0, hist = 0, total = 0, scratch = 0, layout = 0,
         cleared = 0;
  void set(uint32_t ndocs, uint32_t chunks) {
    meta = 0;
    wbase = meta + align_up(sizeof(Meta), 128);
    lbase = wbase + align_up((ndocs + 1) * 4ull, 128);
    item0 = lbase + align_up((ndocs + 1) * 4ull, 128);
    maxlen = item0 + align_up((ndocs + 1) * 4ull, 128);
    hist = maxlen + align_up(ndocs * 4ull, 128);
    total = hist + (size_t)ndocs * kHist * 4;
    scratch = align_up(total, 256);
    layout = align_up(scratch + tokenize1p_scratch_bytes(chunks), 256);
    cleared = layout + sizeof(LayoutWork);
  }
};

enum Kind { kTokenize, kScatter, kTileSort, kMerge, kMergeCut, kEmit, kHostGap, kExpand, kDedupe, kLayout, kKinds };
// host_gap is no kernel: the device time between a summary the host waits
// for and the first launch planned from it (the call's round trips: the
// layout's summary, and the distinct-key counts of the duplicate-aware sort)
const char* const kKindName[kKinds] = {"tokenize", "scatter",  "tile_sort", "merge_pass",
                                       "merge_cut", "emit",     "host_gap",  "expand", "dedupe", "layout"};

struct ProfRec {
  int kind;
  cudaEvent_t a, b;
  double bytes;
  uint32_t stream;   // 0: the call's stream; 1.. the side streams
  uint32_t variant;  // tile sort: CTAs per cluster (0: warp sort); merge: key width
  uint32_t kernels;  // kernels the traced call launched
};

}  // namespace

struct bsort_ctx {
  bsort_config cfg{};
  int device = 0;
  int sm_count = 0;
  cudaStream_t own_stream = nullptr;
  static constexpr int kSide = 9;
  static constexpr int kChainSide = 5;        // side[5 + class]: the merge chains of the four key widths
  cudaStream_t side[kSide] = {};              // side[0..4]: the K4 launches after the first, and the warp sort
  cudaEvent_t fork_ev = nullptr, join_ev[kSide] = {};
  cudaEvent_t counts_ev = nullptr;  // the counts of K1 reached the host
  std::string err;
  bool busy = false;
  Tune tune;
  std::string tune_text;  // the caller's tune table, copied
  uint32_t codec = kCodeBytes;  // key encoding (from order and key_pack)

  DevBuf sticky;  // a Meta kept across calls: err_timeout of bounded device waits
  HostBuf h_sticky;
  DevBuf in, docs, meta, starts, letters, plan, keysA, keysB, counts, offsets, stream, jobs, samples;
  HostBuf h_in, h_docs, h_meta, h_lay, h_counts, h_offsets, h_stream;
  // the duplicate-aware sort: hash tables (all slots zero between calls: each
  // call's claims are undone on the device; htab_clean says whether that is
  // known to hold, else the next call clears them), the distinct-key arrays
  // and their ping-pong partner, the second layout, merge scratch and count
  // prefixes
  DevBuf htab, dcnt, uA, uB, plan2, samples2, jobs2, pre, ssum, tfirst, icnt;
  HostBuf h_plan2, h_ucnt, h_dd;  // h_dd: the duplicate-aware buckets' segments and descriptors
  bool htab_clean = false;
  cudaEvent_t dedupe_ev = nullptr;  // the distinct-key counts reached the host
  std::vector<Segment> segv2;
  std::vector<uint8_t> groupv2;
  HostBuf h_flag;     // word 0: K1 raises it once its copy of a small meta region is in h_meta;
                      // word 8: K2 raises it once its summary is in h_lay
  uint32_t seq = 0;   // the value they are raised to: one per call

  // results of the last run (host view)
  MetaLayout ml;
  uint32_t ndocs = 0;
  std::vector<uint32_t> doc_status;

  // tracing
  uint64_t launches = 0;
  uint64_t kind_launches[kKinds] = {};
  double kind_bytes[kKinds] = {};
  double kind_levels[kKinds] = {};  // key-levels of the sort kernels
  std::vector<cudaEvent_t> ev_pool;
  size_t ev_used = 0;
  std::vector<ProfRec> recs;
};

namespace {

bsort_status fail(bsort_ctx* c, bsort_status s, const std::string& msg) {
  c->err = msg;
  return s;
}

bsort_status cuda_fail(bsort_ctx* c, cudaError_t e, const char* what) {
  c->err = std::string(what) + ": " + cudaGetErrorString(e);
  return (e == cudaErrorMemoryAllocation) ? BSORT_E_NOMEM : BSORT_E_CUDA;
}

#define CK(call, what)                                   \
  do {                                                   \
    cudaError_t e_ = (call);                             \
    if (e_ != cudaSuccess) return cuda_fail(c, e_, what); \
  } while (0)

// Host-side fault injection for tests (no GPU fault is involved): the
// environment variable BSORT_FAULT lists, separated by commas,
//   alloc    every device or page-locked host allocation that a call needs
//            fails (the call returns BSORT_E_NOMEM; buffers already large
//            enough are used as they are)
//   timeout  every call whose K1 has run reports a bounded device wait as
//            run out (BSORT_E_TIMEOUT), as a real one would be reported
// It is read on every use, so a test can set and clear it between calls.
bool fault_on(const char* what) {
  const char* f = std::getenv("BSORT_FAULT");
  if (!f || !*f) return false;
  const size_t n = std::strlen(what);
  for (const char* p = f; *p;) {
    const char* e = std::strchr(p, ',');
    const size_t len = e ? (size_t)(e - p) : std::strlen(p);
    if (len == n && std::strncmp(p, what, n) == 0) return true;
    if (!e) break;
    p = e + 1;
  }
  return false;
}

bsort_status grow(bsort_ctx* c, DevBuf& b, size_t bytes, const char* what) {
  if (bytes <= b.cap && b.p) return BSORT_OK;
  if (fault_on("alloc")) {
    c->err = std::string("device allocation for ") + what + " failed (injected by BSORT_FAULT=alloc)";
    return BSORT_E_NOMEM;
  }
  size_t want = std::max<size_t>(bytes, 256);
  want = std::max(want, b.cap + b.cap / 4);  // amortise repeated growth
  if (b.p) {
    cudaFree(b.p);
    b.p = nullptr;
    b.cap = 0;
  }
  cudaError_t e = cudaMalloc(&b.p, want);
  if (e != cudaSuccess) {
    cudaGetLastError();
    b.p = nullptr;
    c->err = std::string("device allocation of ") + std::to_string(want) + " bytes for " + what + " failed";
    return BSORT_E_NOMEM;
  }
  b.cap = want;
  return BSORT_OK;
}

bsort_status grow_host(bsort_ctx* c, HostBuf& b, size_t bytes, const char* what) {
  if (bytes <= b.cap && b.p) return BSORT_OK;
  if (fault_on("alloc")) {
    c->err = std::string("pinned host allocation for ") + what + " failed (injected by BSORT_FAULT=alloc)";
    return BSORT_E_NOMEM;
  }
  size_t want = std::max<size_t>(bytes, 256);
  want = std::max(want, b.cap + b.cap / 4);
  if (b.p) {
    cudaFreeHost(b.p);
    b.p = nullptr;
    b.cap = 0;
  }
  cudaError_t e = cudaMallocHost(&b.p, want);
  if (e != cudaSuccess) {
    cudaGetLastError();
    b.p = nullptr;
    c->err = std::string("pinned host allocation of ") + std::to_string(want) + " bytes for " + what + " failed";
    return BSORT_E_NOMEM;
  }
  b.cap = want;
  return BSORT_OK;
}

#define GROW(buf, bytes, what)                                \
  do {                                                        \
    bsort_status s_ = grow(c, (buf), (bytes), (what));        \
    if (s_ != BSORT_OK) return s_;                            \
  } while (0)
#define GROW_HOST(buf, bytes, what)                           \
  do {                                                        \
    bsort_status s_ = grow_host(c, (buf), (bytes), (what));   \
    if (s_ != BSORT_OK) return s_;                            \
  } while (0)

template <typename T>
T* dptr(const DevBuf& b, size_t byte_off = 0) {
  return reinterpret_cast<T*>(static_cast<char*>(b.p) + byte_off);
}
template <typename T>
T* hptr(const HostBuf& b, size_t byte_off = 0) {
  return reinterpret_cast<T*>(static_cast<char*>(b.p) + byte_off);
}

// Tracing: count every launch; with profiling on, bracket it with events.
cudaEvent_t next_event(bsort_ctx* c) {
  if (c->ev_used == c->ev_pool.size()) {
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    c->ev_pool.push_back(e);
  }
  return c->ev_pool[c->ev_used++];
}

struct Trace {
  bsort_ctx* c;
  cudaStream_t st;
  int kind;
  double bytes;
  double levels;
  uint32_t variant = 0;
  uint32_t kernels = 1;  // kernels the traced call launches
  cudaEvent_t a = nullptr;
  Trace(bsort_ctx* c_, cudaStream_t st_, int kind_, double bytes_, double levels_ = 0.0)
      : c(c_), st(st_), kind(kind_), bytes(bytes_), levels(levels_) {
    if (c->cfg.profile) {
      a = next_event(c);
      if (a) cudaEventRecord(a, st);
    }
  }
  cudaError_t done(cudaError_t e) {
    if (e != cudaSuccess) return e;
    c->launches += kernels;
    c->kind_launches[kind] += kernels;
    c->kind_bytes[kind] += bytes;
    c->kind_levels[kind] += levels;
    if (a) {
      cudaEvent_t b = next_event(c);
      if (b) {
        cudaEventRecord(b, st);
        uint32_t sx = 0;
        for (int i = 0; i < bsort_ctx::kSide; ++i)
          if (st == c->side[i]) sx = (uint32_t)i + 1;
        c->recs.push_back(ProfRec{kind, a, b, bytes, sx, variant, kernels});
      }
    }
    return e;
  }
};

#define LAUNCH(kind, bytes, call, what)                 \
  do {                                                  \
    Trace tr_(c, st, (kind), (double)(bytes));          \
    CK(tr_.done(call), what);                           \
  } while (0)
// the same for a call that launches nk kernels
#define LAUNCHK(kind, bytes, nk, call, what)            \
  do {                                                  \
    Trace tr_(c, st, (kind), (double)(bytes));          \
    tr_.kernels = (nk);                                 \
    CK(tr_.done(call), what);                           \
  } while (0)

// Whether [p, p + len) is page-locked host memory that a copy engine can read
// directly: its first and last bytes both are (a buffer is taken to be one
// allocation; see bsort_text).
bool host_pinned(const void* p, size_t len) {
  if (!p || len == 0) return false;
  for (const void* q : {p, static_cast<const void*>(static_cast<const uint8_t*>(p) + len - 1)}) {
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, q) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    if (a.type != cudaMemoryTypeHost) return false;
  }
  return true;
}

// Waits for an event by polling it (the call's one mid-path wait is short,
// and a poll answers sooner than a blocking wait); after 200 us it blocks.
// Waits until K1 has raised *flag to seq (its copy of the meta region is in
// host memory by then).  Every 64 polls it also asks whether the stream has
// passed `ev` (recorded after K1): a launch that failed or ended without
// raising the flag is then reported instead of waited on.  After 200 us of
// polling it blocks on the event instead, as spin_wait does.
cudaError_t flag_wait(const uint32_t* flag, uint32_t seq, cudaEvent_t ev) {
  const auto t0 = std::chrono::steady_clock::now();
  for (uint32_t n = 1;; ++n) {
    if (__atomic_load_n(flag, __ATOMIC_ACQUIRE) == seq) return cudaSuccess;
    if ((n & 63u) == 0) {
      cudaError_t e = cudaEventQuery(ev);
      if (e == cudaErrorNotReady && std::chrono::steady_clock::now() - t0 > std::chrono::microseconds(200))
        e = cudaEventSynchronize(ev);
      if (e == cudaErrorNotReady) continue;
      if (e != cudaSuccess) return e;
      // the stream is past K1: the flag is up, or the kernel did not raise it
      if (__atomic_load_n(flag, __ATOMIC_ACQUIRE) == seq) return cudaSuccess;
      return cudaErrorLaunchFailure;
    }
  }
}

cudaError_t spin_wait(cudaEvent_t ev) {
  const auto t0 = std::chrono::steady_clock::now();
  for (;;) {
    const cudaError_t e = cudaEventQuery(ev);
    if (e != cudaErrorNotReady) return e;
    if (std::chrono::steady_clock::now() - t0 > std::chrono::microseconds(200)) return cudaEventSynchronize(ev);
  }
}

// ---- sort planning and launching ----
// The (document, length) buckets are laid out by K2 on the device
// (k_layout.cu); the host builds the launch plan from K2's summary
// (plan_from_summary).  The duplicate-aware sort's second phase, the arrays
// of the buckets' distinct keys (a handful of buckets, known only after the
// hash aggregation), is laid out here by plan_sorts, by the same groups
// (sort_group) and table order (table_order).

uint8_t group_of(Segment& sg, uint64_t& big_tiles) {
  const uint32_t n = sg.n;
  const int W = (int)sg.W;
  const int gi = sort_group(n, W);
  sg.run0 = n;
  sg.passes = 0;
  if (gi >= 10) {
    sg.run0 = (uint32_t)tile_of_width(W);
    sg.passes = merge_passes(n, sg.run0);
  } else if (gi < 4) {  // needs merge passes: runs and passes are set by plan_sorts
    big_tiles += (n + merge2_keys(W) - 1) / merge2_keys(W);
  }
  sg.final_buf = sg.passes & 1u;
  return (uint8_t)gi;
}

struct K4Launch {
  int cluster;
  int gc;
  uint32_t sbeg = 0, send = 0;
  uint32_t supertiles = 0;
  int max_w = 1;
  double key_bytes = 0;
  double levels = 0;  // key-levels: each key times log2 of the sorted run it ends in
};

struct SortPlan {
  uint32_t nseg = 0;
  int runs = 2;
  int order[kGroups] = {};
  int pos_of[kGroups] = {};
  uint32_t pbeg[kGroups + 1] = {};
  K4Launch k4[5] = {{8, 5}, {4, 6}, {2, 7}, {1, 8}, {16, -1}};  // the last: clusters of 16, runs only
  uint64_t key_words = 0, smp_words = 0, kb[kGroups] = {};
  double ob[kGroups] = {};
  uint32_t etile = 0, wtiles[2] = {}, wpasses[2] = {}, mtiles[4] = {}, mpasses[4] = {};
  uint64_t jobs_total = 0, job_at[4] = {};
  // the duplicate-aware sort's buckets (groups 0..3 marked kSegDedupe): the
  // hash-aggregation launch covers [dd_beg, dd_end) in dd_units units
  uint32_t dd_units = 0, dd_beg = 0, dd_end = 0;
  double dd_bytes = 0;
  // the tags' figures of the launches that are not per K4 launch: key-levels
  // of the warp sort and the wide keys' tile sorts (groups 9..11), bytes per
  // merge pass (groups 0..3, then 10 and 11)
  double lev[kGroups] = {};
  double moved[6][kMovedPasses] = {};
  uint32_t gb(int g) const { return pbeg[pos_of[g]]; }      // first segment of group g
  uint32_t ge(int g) const { return pbeg[pos_of[g] + 1]; }  // one past its last
};

// Orders the candidates into `out` by the kernels that sort them and fills
// the plan: the run length K4 leaves and the passes of the buckets that need
// merge passes (none for those marked kSegDedupe: their runs go to the hash
// tables), key offsets (kept as given with preset_keys), merge tiles and
// samples, wide-key tiles, the K4 launch ranges and their tags.
void plan_sorts(const bsort_ctx* c, const std::vector<Segment>& cand, const std::vector<uint8_t>& group,
                uint64_t big_tiles, bool preset_keys, uint64_t off_bytes, Segment* out, SortPlan& p) {
  p.nseg = (uint32_t)cand.size();
  uint32_t group_n[kGroups] = {};
  for (uint8_t g : group) ++group_n[g];
  // The buckets that need merge passes leave K4 as runs of k4_runs tiles
  // when their merges are large enough to be pipelined (the passes then run
  // at HBM speed, cheaper than more cluster levels), else as runs of
  // k4_runs_small tiles (fewer passes, fewer launches).
  const uint32_t piped_grid = (uint32_t)(c->sm_count * merge_piped_ctas_per_sm());
  p.runs = big_tiles >= (uint64_t)c->tune.piped_min * piped_grid ? c->tune.k4_runs : c->tune.k4_runs_small;
  // Table order: the groups that K4 finishes (clusters of 8, 4, 2, 1), with
  // the groups that need merge passes (0..3, and the unused 4) placed just
  // before the one whose cluster size makes their runs, so that every K4
  // launch and every width's merge chain covers one contiguous range; then
  // the warp sort and the wide keys.
  table_order((uint32_t)p.runs, p.order, p.pos_of);
  for (int q = 0; q < kGroups; ++q) p.pbeg[q + 1] = p.pbeg[q] + group_n[p.order[q]];
  {  // stable counting sort of the candidates by table position
    uint32_t at[kGroups];
    for (int q = 0; q < kGroups; ++q) at[q] = p.pbeg[q];
    for (uint32_t i = 0; i < p.nseg; ++i) {
      Segment sg = cand[i];
      if (group[i] < 4) {
        if (sg.flags & kSegDedupe) {
          sg.run0 = (uint32_t)p.runs * tile2_keys((int)sg.W);
          sg.passes = 0;
        } else {
          sg.run0 = (uint32_t)p.runs * tile2_keys((int)sg.W);
          sg.passes = merge_passes(sg.n, sg.run0);
        }
        sg.final_buf = sg.passes & 1u;
      }
      out[at[p.pos_of[group[i]]]++] = sg;
    }
  }
  // K4 launches: cluster size, its own group, and the table range it covers
  // (the merge-pass groups too, for the cluster size that makes their runs,
  // unless they go to the duplicate-aware sort's own launch)
  bool dd = false;
  for (uint32_t i = 0; i < p.nseg; ++i) dd |= group[i] < 4 && (cand[i].flags & kSegDedupe);
  const bool runs_in_k4 = !dd;
  for (K4Launch& l : p.k4) {
    if (l.gc < 0) {
      l.sbeg = p.runs == l.cluster && runs_in_k4 ? p.gb(0) : 0u;
      l.send = p.runs == l.cluster && runs_in_k4 ? p.ge(4) : 0u;
    } else {
      l.sbeg = l.cluster == p.runs && runs_in_k4 ? p.gb(0) : p.gb(l.gc);
      l.send = p.ge(l.gc);
    }
  }
  if (dd) {
    p.dd_beg = p.gb(0);
    p.dd_end = p.ge(4);
  }
  auto out_bytes = [&](const Segment& sg) {  // a bucket's output: its letters and offsets
    return (sg.flags & kSegKeysOut) ? 8.0 * sg.W * sg.n : (double)sg.n * (sg.L + off_bytes);
  };
  for (uint32_t i = 0; i < p.nseg; ++i) {
    Segment& sg = out[i];
    const int W = (int)sg.W;
    int q = 0;
    while (i >= p.pbeg[q + 1]) ++q;
    const int gi = p.order[q];
    if (!preset_keys) sg.key_off = p.key_words;
    p.key_words += align_up((size_t)sg.n * W, 16);
    p.kb[gi] += 8ull * W * sg.n;
    p.ob[gi] += out_bytes(sg);
    if (gi >= 10) {  // only the wide keys go through K6
      sg.etile0 = p.etile;
      p.etile += (sg.n + tile_of_width(W) - 1) / tile_of_width(W);
    }
    if (gi < 4 && (sg.flags & kSegDedupe)) {  // the hash-aggregation units
      sg.stile0 = p.dd_units;
      p.dd_units += (sg.n + dedupe_unit_keys(W) - 1) / dedupe_unit_keys(W);
      p.dd_bytes += 8.0 * W * sg.n;
    }
    if (gi < 4) {
      // Every bucket of the group gets its merge tiles, also one that needs
      // no pass (a run of k4_runs_small tiles can hold it, or it went to the
      // hash tables): the merge kernels find a tile's bucket by binary
      // search over tile0, which must rise along the group; they skip the
      // buckets whose passes are done.
      sg.tile0 = p.mtiles[gi];
      p.mtiles[gi] += (sg.n + merge2_keys(W) - 1) / merge2_keys(W);
      p.mpasses[gi] = std::max(p.mpasses[gi], sg.passes);
      if (sg.passes) {  // merge samples: one key in 32 (read by the pipelined merges' cuts)
        sg.smp_off = (uint32_t)p.smp_words;
        p.smp_words += (uint64_t)(sg.n + 31) / 32 * W;
      }
    }
    for (K4Launch& l : p.k4)
      if (i >= l.sbeg && i < l.send) {
        const uint32_t super = (uint32_t)l.cluster * tile2_keys(W);
        sg.stile0 = l.supertiles;
        l.supertiles += (sg.n + super - 1) / super;
        l.max_w = std::max(l.max_w, W);
        // keys in, then runs out for K5, the sorted words out, or (the
        // duplicate-aware sort) nothing but the hash inserts
        l.key_bytes += 8.0 * W * sg.n + ((sg.flags & kSegDedupe) ? 0.0 : sg.passes ? 8.0 * W * sg.n : out_bytes(sg));
        l.levels += (double)sg.n * ceil_log2(std::min<uint64_t>(sg.n, (uint64_t)super));
      }
    if (gi >= 10) {
      sg.tile0 = p.wtiles[gi - 10];
      p.wtiles[gi - 10] += (sg.n + sg.run0 - 1) / sg.run0;
      p.wpasses[gi - 10] = std::max(p.wpasses[gi - 10], sg.passes);
      p.lev[gi] += (double)sg.n * ceil_log2(std::min<uint64_t>(sg.n, sg.run0));
    } else if (gi == 9) {
      p.lev[gi] += (double)sg.n * ceil_log2(sg.n);
    }
    const int mg = gi < 4 ? gi : gi >= 10 ? gi - 6 : -1;
    for (uint32_t q = 0; mg >= 0 && q < sg.passes && q < (uint32_t)kMovedPasses; ++q) {
      // keys in; keys out, or the words at the bucket's last pass
      const double kw = 8.0 * W * sg.n;
      const bool words = gi < 4 && q + 1 == sg.passes && !(sg.flags & kSegKeysOut);
      p.moved[mg][q] += kw + (words ? (double)sg.n * (sg.L + off_bytes) : kw);
    }
  }
  for (int g = 0; g < 4; ++g)
    if (p.mpasses[g] && p.mtiles[g] >= c->tune.piped_min * piped_grid) {
      p.job_at[g] = p.jobs_total;
      p.jobs_total += p.mtiles[g] + 1;  // and the end sentinel
    }
}

// The plan of the (document, length) buckets from K2's summary: the same
// fields plan_sorts fills, from K2's per-group totals.
void plan_from_summary(const bsort_ctx* c, const LayoutSummary& S, SortPlan& p) {
  p.nseg = S.nseg;
  p.runs = (int)S.runs;
  table_order(S.runs, p.order, p.pos_of);
  for (int q = 0; q < kGroups; ++q) p.pbeg[q + 1] = p.pbeg[q] + S.group_n[p.order[q]];
  const bool dd = S.dd != 0;
  for (K4Launch& l : p.k4) {
    const bool runs_here = l.cluster == p.runs && !dd;
    if (l.gc < 0) {
      l.sbeg = runs_here ? p.gb(0) : 0u;
      l.send = runs_here ? p.ge(4) : 0u;
    } else {
      l.sbeg = runs_here ? p.gb(0) : p.gb(l.gc);
      l.send = p.ge(l.gc);
    }
    // its groups: the merge-pass groups when its clusters make their runs, and its own
    for (int g = 0; g < kGroups; ++g) {
      const bool mine = (g < 4 && runs_here) || g == l.gc;
      if (!mine) continue;
      l.supertiles += (uint32_t)S.tot[g][kColStile];
      l.max_w = std::max(l.max_w, (int)S.max_w[g]);
      l.key_bytes += (double)S.k4_bytes[g];
      l.levels += (double)S.levels[g];
    }
  }
  if (dd) {
    p.dd_beg = p.gb(0);
    p.dd_end = p.ge(4);
    for (int g = 0; g < 4; ++g) p.dd_units += (uint32_t)S.tot[g][kColStile];
    p.dd_bytes = (double)S.dd_bytes;
  }
  for (int g = 0; g < kGroups; ++g) {
    p.key_words += S.tot[g][kColKeyw];
    p.kb[g] = (double)S.kb[g];
    p.ob[g] = (double)S.ob[g];
    p.lev[g] = g >= 9 ? (double)S.levels[g] : 0.0;
  }
  for (int g = 0; g < 4; ++g) {
    p.smp_words += S.tot[g][kColSmp];
    p.mtiles[g] = (uint32_t)S.tot[g][kColTile];
    p.mpasses[g] = S.max_passes[g];
  }
  for (int i = 0; i < 2; ++i) {
    p.wtiles[i] = (uint32_t)S.tot[10 + i][kColTile];
    p.wpasses[i] = S.max_passes[10 + i];
  }
  p.etile = p.wtiles[0] + p.wtiles[1];
  for (int m = 0; m < 6; ++m)
    for (int q = 0; q < kMovedPasses; ++q) p.moved[m][q] = (double)S.moved[m][q];
  const uint32_t piped_grid = (uint32_t)(c->sm_count * merge_piped_ctas_per_sm());
  for (int g = 0; g < 4; ++g)
    if (p.mpasses[g] && p.mtiles[g] >= c->tune.piped_min * piped_grid) {
      p.job_at[g] = p.jobs_total;
      p.jobs_total += p.mtiles[g] + 1;  // and the end sentinel
    }
}

bsort_status launch_sorts(bsort_ctx* c, const SortPlan& p, const Segment* d_segs, uint64_t* kA,
                          uint64_t* kB, uint64_t* samples, DevBuf& jobs, uint32_t* barrier_dev, const EmitOut& eo,
                          const DedupeOut& dd, cudaStream_t st, bool side_ok, std::vector<cudaStream_t>& joined,
                          const std::function<bsort_status()>& after_first_k4) {
  const uint32_t grid_cap = (uint32_t)c->sm_count * 16;
  const uint32_t piped_grid = (uint32_t)(c->sm_count * merge_piped_ctas_per_sm());
  Meta* d_sticky = dptr<Meta>(c->sticky);
  // K4: the launch that makes the merge passes' runs first, on the call's
  // stream, so that the merges (which wait for it alone) start as early as
  // they can; then the other launches, largest first, each on a side stream
  // at the same time (they sort other buckets).  (With k4_streams=0 in the
  // tune table every launch stays on the call's stream, one after another:
  // how the autotuner times each class alone.)
  int k4_order[5], n4 = 0;
  for (int i = 0; i < 5; ++i)
    if (p.k4[i].supertiles) k4_order[n4++] = i;
  std::stable_sort(k4_order, k4_order + n4, [&](int a, int b) {
    const bool ra = p.k4[a].cluster == p.runs, rb = p.k4[b].cluster == p.runs;
    if (ra != rb) return ra;
    return p.k4[a].levels > p.k4[b].levels;
  });
  // the warp sort, or more than one launch of K4 and the hash aggregation
  const bool small_work = p.ge(9) > p.gb(9) || n4 + (p.dd_units ? 1 : 0) > 1;
  const bool side = side_ok && small_work && c->tune.k4_streams;
  if (side) CK(cudaEventRecord(c->fork_ev, st), "fork");
  int used = 0;
  auto side_stream = [&]() -> cudaStream_t {
    if (!side) return st;
    cudaStream_t sx = c->side[used++];
    joined.push_back(sx);
    return sx;
  };
  bool first_done = false;
  if (p.dd_units) {
    // the duplicate-aware sort's buckets first, on the call's stream: the
    // distinct-key counts are read back right after it
    Trace tr_(c, st, kDedupe, p.dd_bytes);
    tr_.kernels = 2;  // the aggregation, then the tables' completion
    c->htab_clean = false;  // until the launches that also undo the claims are enqueued
    CK(tr_.done(launch_dedupe_hash(d_segs, p.dd_beg, p.dd_end, p.dd_units, c->sm_count, kA, dd, p.dd_end - p.dd_beg,
                                   d_sticky, c->cfg.wait_limit, st)),
       "duplicate-aware hash aggregation");
    c->htab_clean = true;
    if (after_first_k4) {
      const bsort_status s = after_first_k4();
      if (s != BSORT_OK) return s;
    }
    first_done = true;
  }
  for (int q = 0; q < n4; ++q) {
    const K4Launch& l = p.k4[k4_order[q]];
    cudaStream_t sx = st;
    if ((q > 0 || p.dd_units) && side) {
      sx = side_stream();
      CK(cudaStreamWaitEvent(sx, c->fork_ev, 0), "fork");
    }
    Trace tr_(c, sx, kTileSort, l.key_bytes, l.levels);
    tr_.variant = (uint32_t)l.cluster;
    const int cls = l.cluster == 1 ? 0 : l.cluster == 2 ? 1 : l.cluster == 4 ? 2 : 3;  // 16 as 8
    CK(tr_.done(launch_tile_sort2(l.cluster, c->tune.k4_lanes[cls], c->tune.k4_threads[cls], d_segs, l.sbeg, l.send,
                                  l.supertiles, c->sm_count, l.max_w, kA, eo, d_sticky, c->cfg.wait_limit, sx)),
       "K4 tile_sort");
    if (q == 0 && !first_done && after_first_k4) {
      const bsort_status s = after_first_k4();
      if (s != BSORT_OK) return s;
      first_done = true;
    }
  }
  if (!first_done && after_first_k4) {
    const bsort_status s = after_first_k4();
    if (s != BSORT_OK) return s;
  }
  if (p.ge(9) > p.gb(9)) {
    cudaStream_t sx = side_stream();
    if (side) CK(cudaStreamWaitEvent(sx, c->fork_ev, 0), "fork");
    Trace tr_(c, sx, kTileSort, (double)p.kb[9] + p.ob[9], p.lev[9]);
    CK(tr_.done(launch_warp_sort(d_segs, p.gb(9), p.ge(9), kA, eo, sx)), "K4 warp_sort");
  }
  for (int g = 10; g < 12; ++g) {
    const uint32_t tiles = p.wtiles[g - 10];
    if (!tiles) continue;
    Trace tr_(c, st, kTileSort, 2.0 * p.kb[g], p.lev[g]);
    tr_.variant = 1;
    CK(tr_.done(launch_tile_sort(g == 10 ? 16 : 32, d_segs, p.gb(g), p.ge(g), tiles, std::min(tiles, grid_cap), kA,
                                 d_sticky, c->cfg.wait_limit, st)),
       "K4 tile_sort (wide keys)");
  }
  // K5: merge passes over the buckets that need them, one launch per pass and
  // width.  With at least piped_min tiles per resident CTA the pass is
  // pipelined: a cut kernel lists every tile's slices first, so that the
  // merge kernel can load one tile while it merges another.  The widths'
  // chains of passes are independent: with more than one, each runs on a side
  // stream of its own, so that one chain's latency-bound launches overlap
  // another's merges.
  if (p.jobs_total) GROW(jobs, sizeof(TileJob) * p.jobs_total, "merge jobs");
  int chains = 0;
  for (int g = 0; g < 4; ++g)
    if (p.mpasses[g]) ++chains;
  const bool chain_side = side_ok && chains > 1;
  if (chain_side) CK(cudaEventRecord(c->fork_ev, st), "fork");
  for (int g = 0; g < 4; ++g) {
    if (!p.mpasses[g]) continue;
    const int W = width_of_class(g);
    cudaStream_t sx = st;
    if (chain_side) {
      sx = c->side[bsort_ctx::kChainSide + g];
      joined.push_back(sx);
      CK(cudaStreamWaitEvent(sx, c->fork_ev, 0), "fork");
    }
    auto moved_in = [&](uint32_t pass) { return pass < (uint32_t)kMovedPasses ? p.moved[g][pass] : 0.0; };
    if (p.mtiles[g] >= c->tune.piped_min * piped_grid) {
      for (uint32_t pass = 0; pass < p.mpasses[g]; ++pass) {
        const uint64_t* src = (pass & 1) ? kB : kA;
        uint64_t* dst = (pass & 1) ? kA : kB;
        TileJob* jb = dptr<TileJob>(jobs) + p.job_at[g];
        {
          Trace tr_(c, sx, kMergeCut, 0.0);
          tr_.variant = (uint32_t)W;
          CK(tr_.done(launch_merge_cut(W, d_segs, p.gb(g), p.ge(g), p.mtiles[g], pass, src, samples, jb, sx)),
             "K5 merge cut");
        }
        Trace tr_(c, sx, kMerge, moved_in(pass));
        tr_.variant = (uint32_t)W;
        CK(tr_.done(launch_merge_piped(W, jb, p.mtiles[g], piped_grid, src, dst, samples, eo, sx)), "K5 merge_pass");
      }
    } else {
      // small passes: all of them in one launch, grid barriers between them
      double moved = 0;
      for (uint32_t pass = 0; pass < p.mpasses[g]; ++pass) moved += moved_in(pass);
      Trace tr_(c, sx, kMerge, moved);
      tr_.variant = (uint32_t)W;
      CK(tr_.done(launch_merge_pass2(W, d_segs, p.gb(g), p.ge(g), p.mtiles[g],
                                     std::min<uint32_t>(p.mtiles[g], (uint32_t)c->sm_count * 8), 0, p.mpasses[g], kA, kB,
                                     eo, barrier_dev + g, d_sticky, c->cfg.wait_limit, sx)),
         "K5 merge_pass");
    }
  }
  for (int g = 10; g < 12; ++g) {
    const int W = g == 10 ? 16 : 32;
    const uint32_t tiles = p.wtiles[g - 10];
    for (uint32_t pass = 0; pass < p.wpasses[g - 10]; ++pass) {
      const double moved = pass < (uint32_t)kMovedPasses ? p.moved[g - 6][pass] : 0.0;
      LAUNCH(kMerge, moved,
             launch_merge_pass(W, d_segs, p.gb(g), p.ge(g), tiles, std::min(tiles, grid_cap), pass, (pass & 1) ? kB : kA,
                               (pass & 1) ? kA : kB, st),
             "K5 merge_pass (wide keys)");
    }
  }
  // K6: the words of the wide keys (every other bucket was emitted by its sort)
  if (p.etile) {
    LAUNCH(kEmit, (double)p.kb[10] + p.kb[11] + p.ob[10] + p.ob[11],
           launch_emit(d_segs, p.gb(10), p.ge(11), p.etile, std::min(p.etile, grid_cap), kA, kB, eo, st), "K6 emit");
  }
  return BSORT_OK;
}

// The duplicate-aware sort's second half, once the hash aggregation has
// filled the tables of the `ndd` buckets marked kSegDedupe (dd_segs: host
// copies of their segments, in dedupe-index order; ins: their descriptors): reads
// how many distinct keys each bucket has, sorts every bucket's distinct-key
// array (entries of key + count, kSegKeysOut: the same K4 / K5 kernels, on
// the side streams as the first sorts), then expands the sorted arrays into
// the buckets' words.  The counts' read-back is the call's second round trip.
bsort_status sort_distinct(bsort_ctx* c, const Segment* dd_segs, const DedupeIns* ins, uint32_t ndd,
                           const uint32_t* h_ucnt, const EmitOut& eo, cudaStream_t st) {
  cudaEvent_t gap_a = nullptr;
  if (c->cfg.profile) {
    gap_a = next_event(c);
    if (gap_a) cudaEventRecord(gap_a, st);
  }
  CK(spin_wait(c->dedupe_ev), "wait for distinct-key counts");
  std::vector<Segment>& cand = c->segv2;
  std::vector<uint8_t>& group = c->groupv2;
  cand.clear();
  group.clear();
  uint64_t big_tiles = 0;
  for (uint32_t di = 0; di < ndd; ++di) {
    const uint32_t U = h_ucnt[di];
    if (U == 0) continue;  // every insert dropped: a timeout, which the call reports
    const DedupeIns& d = ins[di];
    Segment u{};
    u.n = U;
    u.L = 8 * d.Wp;  // keys of Wp words: the key, its count, zeros
    u.doc = di;
    u.key_off = d.uniq_off;
    u.W = d.Wp;
    u.flags = kSegKeysOut;
    const uint8_t gi = group_of(u, big_tiles);
    cand.push_back(u);
    group.push_back(gi);
  }
  const uint32_t nseg = (uint32_t)cand.size();
  const size_t seg_bytes = align_up(sizeof(Segment) * std::max<uint32_t>(nseg, 1), 256);
  const size_t barrier_bytes = 256;
  const size_t ed_bytes = align_up(sizeof(ExpandDesc) * std::max<uint32_t>(nseg, 1), 256);
  const size_t plan_bytes = seg_bytes + barrier_bytes + ed_bytes;
  GROW_HOST(c->h_plan2, plan_bytes, "distinct-key layout");
  Segment* const segs2 = hptr<Segment>(c->h_plan2);
  std::memset(hptr<char>(c->h_plan2, seg_bytes), 0, barrier_bytes);
  ExpandDesc* const ed = hptr<ExpandDesc>(c->h_plan2, seg_bytes + barrier_bytes);
  SortPlan p2;
  plan_sorts(c, cand, group, big_tiles, true, c->cfg.want_offsets ? 4 : 0, segs2, p2);
  // expansion descriptors, in the order of the buckets
  std::vector<uint32_t> where(ndd, kNoSegment);
  for (uint32_t i = 0; i < nseg; ++i) where[segs2[i].doc] = i;
  uint32_t ne = 0, max_tiles = 0, tiles = 0, max_U = 0;
  uint64_t pre_words = 0;
  double moved = 0;
  for (uint32_t di = 0; di < ndd; ++di) {
    if (where[di] == kNoSegment) continue;
    const Segment& u = segs2[where[di]];
    const Segment& b = dd_segs[di];
    ExpandDesc& e = ed[ne++];
    e = ExpandDesc{};
    e.uniq_off = ins[di].uniq_off;
    e.pre_off = pre_words;
    pre_words += u.n + 1;
    e.U = u.n;
    e.n = b.n;
    e.L = b.L;
    e.Wp = ins[di].Wp;
    e.final_buf = u.final_buf;
    const uint32_t bt = (b.n + expand_tile(e.Wp / 2) - 1) / expand_tile(e.Wp / 2);
    e.tile0 = tiles;
    tiles += bt;
    max_tiles = std::max(max_tiles, bt);
    max_U = std::max(max_U, u.n);
    e.stream_off = b.stream_off;
    e.out_word = b.out_word;
    e.doc_stream0 = b.doc_stream0;
    // the sorted entries and the prefix read, the words and offsets written
    moved += 8.0 * e.Wp * e.U + 4.0 * (e.U + 1) + (double)b.n * (b.L + (c->cfg.want_offsets ? 4 : 0));
  }
  GROW(c->plan2, plan_bytes, "distinct-key layout");
  GROW(c->samples2, 8 * std::max<uint64_t>(p2.smp_words, 16), "merge samples");
  GROW(c->pre, 4 * std::max<uint64_t>(pre_words, 16), "count prefixes");
  GROW(c->ssum, 4 * std::max<uint64_t>((uint64_t)ne * expand_slices(max_U), 16), "count prefixes");
  GROW(c->tfirst, 4 * std::max<uint64_t>(tiles, 16), "tile starts");
  CK(cudaMemcpyAsync(c->plan2.p, c->h_plan2.p, plan_bytes, cudaMemcpyHostToDevice, st), "copy distinct-key layout");
  if (gap_a) {
    cudaEvent_t gap_b = next_event(c);
    if (gap_b) {
      cudaEventRecord(gap_b, st);
      c->recs.push_back(ProfRec{kHostGap, gap_a, gap_b, 0.0, 0u, 0u, 0u});
      c->kind_launches[kHostGap] += 1;
    }
  }
  const Segment* segs2_dev = dptr<Segment>(c->plan2);
  uint32_t* barrier2 = dptr<uint32_t>(c->plan2, seg_bytes);
  // (the distinct-key sorts use the side streams too: the tile sorts of the
  // size classes, and the merge chains of the key widths, overlap; they are
  // joined back before the expansion)
  std::vector<cudaStream_t> joined2;
  const DedupeOut no_dd{nullptr, nullptr, nullptr, nullptr, nullptr};
  bsort_status s = launch_sorts(c, p2, segs2_dev, dptr<uint64_t>(c->uA), dptr<uint64_t>(c->uB),
                                dptr<uint64_t>(c->samples2), c->jobs2, barrier2, eo, no_dd, st, true, joined2, {});
  if (s != BSORT_OK) return s;
  for (size_t i = 0; i < joined2.size(); ++i) {
    CK(cudaEventRecord(c->join_ev[i], joined2[i]), "join");
    CK(cudaStreamWaitEvent(st, c->join_ev[i], 0), "join");
  }
  const ExpandCaps caps{std::min(c->uA.cap, c->uB.cap) / 8, c->pre.cap / 4, c->stream.cap, c->offsets.cap / 4,
                        c->tfirst.cap / 4};
  LAUNCHK(kExpand, moved, ne == 0 ? 0u : max_tiles == 0 ? 3u : 4u,
         launch_expand(dptr<ExpandDesc>(c->plan2, seg_bytes + barrier_bytes), ne, max_U, max_tiles,
                       dptr<uint64_t>(c->uA), dptr<uint64_t>(c->uB), dptr<uint32_t>(c->pre), dptr<uint32_t>(c->ssum),
                       dptr<uint32_t>(c->tfirst), eo, dptr<Meta>(c->sticky), caps, st),
         "expand");
  return BSORT_OK;
}

// Runs the whole path over `ndocs` documents that sit at d_in + offs[i]
// (lens[i] bytes each) in device memory.  Leaves the outputs in c->counts,
// c->offsets, c->stream and the host copy of the meta region in c->h_meta.
bsort_status run_path(bsort_ctx* c, const uint8_t* d_in, const uint64_t* offs, const uint64_t* lens,
                      uint32_t ndocs, cudaStream_t st) {
  c->ndocs = ndocs;
  c->doc_status.assign(ndocs, BSORT_OK);
  // ---- documents and chunks ----
  GROW_HOST(c->h_docs, sizeof(DocDesc) * ndocs, "document table");
  DocDesc* hd = hptr<DocDesc>(c->h_docs);
  uint64_t chunks = 0, total_len = 0, words_bound = 0, seg_bound = 0;
  for (uint32_t i = 0; i < ndocs; ++i) {
    if (lens[i] >= (1ull << 32))
      return fail(c, BSORT_E_TOO_LARGE, "document of 2^32 bytes or more (offsets are 32-bit)");
    const uint64_t mis = (reinterpret_cast<uintptr_t>(d_in) + offs[i]) & 15u;
    const uint64_t nch = lens[i] ? (mis + lens[i] + kChunk - 1) / kChunk : 0;
    hd[i] = DocDesc{offs[i], lens[i], (uint32_t)chunks, (uint32_t)nch};
    chunks += nch;
    total_len += lens[i];
    const uint64_t wb = lens[i] / 2 + 1;
    words_bound += wb;
    // a bucket per length with words
    seg_bound += std::min<uint64_t>(std::min<uint64_t>(wb, kMaxLen), max_distinct_lengths(lens[i]));
  }
  if (total_len >= (1ull << 32))
    return fail(c, BSORT_E_TOO_LARGE, "2^32 bytes or more in one pass (positions are 32-bit)");
  c->ml.set(ndocs, (uint32_t)chunks);
  const MetaLayout& ml = c->ml;
  const uint32_t order = c->cfg.order;
  GROW(c->docs, sizeof(DocDesc) * ndocs, "document table");
  GROW(c->meta, ml.cleared, "meta");
  GROW(c->starts, 4 * (words_bound + 1), "word starts");
  GROW(c->letters, total_len + 16, "stripped letters");
  GROW_HOST(c->h_meta, ml.total, "meta");
  GROW_HOST(c->h_lay, sizeof(LayoutSummary), "layout summary");
  Meta* d_meta = dptr<Meta>(c->meta, ml.meta);
  Meta* d_sticky = dptr<Meta>(c->sticky);
  uint32_t* d_wbase = dptr<uint32_t>(c->meta, ml.wbase);
  uint32_t* d_lbase = dptr<uint32_t>(c->meta, ml.lbase);
  uint32_t* d_item0 = dptr<uint32_t>(c->meta, ml.item0);
  uint32_t* d_hist = dptr<uint32_t>(c->meta, ml.hist);
  LayoutWork* d_work = dptr<LayoutWork>(c->meta, ml.layout);

  // The table K2 writes, sized by bounds known before the counts: a bucket
  // per (document, length) with words (the whole-text order: per document);
  // a duplicate-aware bucket holds more than 2048 words.
  const uint32_t seg_cap = (uint32_t)std::max<uint64_t>(order == BSORT_ORDER_WHOLE ? ndocs : seg_bound, 1);
  const uint32_t dd_cap = (uint32_t)std::max<uint64_t>(std::min<uint64_t>(seg_cap, words_bound / 2048 + 1), 1);
  const size_t seg_bytes = align_up(sizeof(Segment) * (size_t)seg_cap, 256);
  const size_t lookup_bytes = align_up(4ull * std::max<uint32_t>(ndocs, 1) * kHist, 256);
  const size_t cursor_bytes = align_up(4ull * seg_cap, 256);
  const size_t ucnt_bytes = align_up(4ull * dd_cap, 256);
  const size_t ins_bytes = align_up(sizeof(DedupeIns) * (size_t)dd_cap, 256);
  const size_t var_bytes = order == BSORT_ORDER_WHOLE ? align_up(sizeof(VarDesc) * (size_t)seg_cap, 256) : 0;
  const size_t blk_bytes = align_up(8 * layout_scratch_words(ndocs), 256);
  size_t at = 0;
  const size_t at_segs = at;
  at += seg_bytes;
  const size_t at_lookup = at;
  at += lookup_bytes;
  const size_t at_cursor = at;
  at += cursor_bytes;
  const size_t at_ucnt = at;
  at += ucnt_bytes;
  const size_t at_ins = at;
  at += ins_bytes;
  const size_t at_var = at;
  at += var_bytes;
  const size_t at_blk = at;
  at += blk_bytes;
  GROW(c->plan, at, "layout");
  Segment* const segs_dev = dptr<Segment>(c->plan, at_segs);
  uint32_t* const lookup_dev = dptr<uint32_t>(c->plan, at_lookup);
  uint32_t* const cursor_dev = dptr<uint32_t>(c->plan, at_cursor);
  uint32_t* const ucnt_dev = dptr<uint32_t>(c->plan, at_ucnt);
  DedupeIns* const ins_dev = dptr<DedupeIns>(c->plan, at_ins);
  VarDesc* const var_dev = dptr<VarDesc>(c->plan, at_var);
  uint32_t* const barrier_dev = d_work->barrier;  // one per key width, cleared with meta

  // A small meta region (up to 64 KB: about 60 documents) reaches the host
  // from K1's last CTA directly, without a copy of its own; K2's summary
  // always does (from its last CTA of K2b).
  // (Page-locked host memory is mapped at the same address on the device
  // with unified addressing; where it is not mapped the copy path is taken.)
  bool meta_direct = ml.total <= 65536, lay_direct = true;
  HostMeta hmeta{nullptr, 0, nullptr, 0}, hlay{nullptr, 0, nullptr, 0};
  {
    GROW_HOST(c->h_flag, 64, "flag");
    void* dm = nullptr;
    void* dl = nullptr;
    void* df = nullptr;
    if (cudaHostGetDevicePointer(&dm, c->h_meta.p, 0) != cudaSuccess ||
        cudaHostGetDevicePointer(&dl, c->h_lay.p, 0) != cudaSuccess ||
        cudaHostGetDevicePointer(&df, c->h_flag.p, 0) != cudaSuccess) {
      cudaGetLastError();
      meta_direct = lay_direct = false;
    } else {
      if (++c->seq == 0) ++c->seq;  // 0: the flags' value before any call
      uint32_t* hf = hptr<uint32_t>(c->h_flag);
      __atomic_store_n(hf, 0u, __ATOMIC_RELEASE);
      __atomic_store_n(hf + 8, 0u, __ATOMIC_RELEASE);
      uint32_t* df32 = static_cast<uint32_t*>(df);
      if (meta_direct) hmeta = HostMeta{static_cast<uint4*>(dm), (uint32_t)(ml.total / 16), df32, c->seq};
      hlay = HostMeta{static_cast<uint4*>(dl), (uint32_t)(sizeof(LayoutSummary) / 16), df32 + 8, c->seq};
    }
  }
  // one document travels as a kernel argument; more as a table
  if (ndocs > 1)
    CK(cudaMemcpyAsync(c->docs.p, hd, sizeof(DocDesc) * ndocs, cudaMemcpyHostToDevice, st), "copy document table");
  CK(cudaMemsetAsync(c->meta.p, 0, ml.cleared, st), "clear meta");
  const DocDesc* d_docs = dptr<DocDesc>(c->docs);
  // K1: strip, tokenize and count lengths in one pass.  Its algorithmic bytes
  // (input read, letters and word starts written) are known only after the
  // counts come back; they are added to its tag below.
  LAUNCH(kTokenize, 0,
         launch_tokenize1p(d_in, d_docs, ndocs ? hd[0] : DocDesc{}, ndocs, (uint32_t)chunks, dptr<uint8_t>(c->meta, ml.scratch),
                           dptr<uint8_t>(c->letters), dptr<uint32_t>(c->starts), d_hist,
                           dptr<uint32_t>(c->meta, ml.maxlen), d_wbase, d_lbase, d_item0,
                           d_meta, d_sticky, c->cfg.l_cap, c->cfg.wait_limit, hmeta, st),
         "K1 tokenize");
  if (!meta_direct) CK(cudaMemcpyAsync(c->h_meta.p, c->meta.p, ml.total, cudaMemcpyDeviceToHost, st), "read counts");
  // K2: the bucket layout, from K1's histograms.  Its tag: the histograms
  // read (three times) and the lookup written; the segments written are added
  // once their number is known.
  {
    LayoutParams lp{};
    lp.ndocs = ndocs;
    lp.order = order;
    lp.codec = c->codec;
    lp.off_bytes = c->cfg.want_offsets ? 4u : 0u;
    lp.k4_runs = (uint32_t)c->tune.k4_runs;
    lp.k4_runs_small = (uint32_t)c->tune.k4_runs_small;
    lp.dedupe = (uint32_t)c->tune.dedupe;
    lp.piped_tiles = (uint64_t)c->tune.piped_min * c->sm_count * merge_piped_ctas_per_sm();
    lp.seg_cap = seg_cap;
    lp.dd_cap = dd_cap;
    const LayoutOut lo{segs_dev, lookup_dev, cursor_dev, ucnt_dev, ins_dev, var_dev, dptr<uint64_t>(c->plan, at_blk)};
    Trace tr_(c, st, kLayout, 4.0 * kHist * ndocs * 4);
    tr_.kernels = (uint32_t)layout_kernels(ndocs);
    CK(tr_.done(launch_layout(lp, d_hist, d_wbase, d_lbase, dptr<uint32_t>(c->meta, ml.maxlen), d_work, lo, hlay, st)),
       "K2 layout");
  }
  if (!lay_direct)
    CK(cudaMemcpyAsync(c->h_lay.p, &d_work->s, sizeof(LayoutSummary), cudaMemcpyDeviceToHost, st), "read layout summary");
  cudaEvent_t gap_a = nullptr;
  if (c->cfg.profile) {
    gap_a = next_event(c);
    if (gap_a) cudaEventRecord(gap_a, st);
  }
  CK(cudaEventRecord(c->counts_ev, st), "counts event");
  if (lay_direct) {
    CK(flag_wait(hptr<uint32_t>(c->h_flag) + 8, hlay.seq, c->counts_ev), "wait for the layout");
    if (meta_direct) CK(flag_wait(hptr<uint32_t>(c->h_flag), hmeta.seq, c->counts_ev), "wait for counts");
  } else {
    CK(spin_wait(c->counts_ev), "wait for counts");
  }

  const Meta* hm = hptr<Meta>(c->h_meta, ml.meta);
  const uint32_t* h_hist = hptr<uint32_t>(c->h_meta, ml.hist);
  const LayoutSummary& S = *hptr<LayoutSummary>(c->h_lay);
  // K1's own bounded waits (this call), then the sort kernels' waits of an
  // earlier device call whose status nobody collected (bsort_device_finish)
  if (hm->err_timeout || fault_on("timeout"))
    return fail(c, BSORT_E_TIMEOUT,
                hm->err_timeout ? "a bounded device wait of the tokenize kernel ran out (the call's outputs are not valid)"
                                : "a bounded device wait ran out (injected by BSORT_FAULT=timeout)");
  if (hm->err_prev) {
    c->htab_clean = false;
    CK(cudaMemsetAsync(d_sticky, 0, sizeof(Meta), st), "clear timeout flag");
    return fail(c, BSORT_E_TIMEOUT,
                "a bounded device wait of the sort kernels ran out in an earlier device call on this context, "
                "whose outputs were not valid (bsort_device_finish reports it in time)");
  }
  if (S.seg_over) {
    CK(cudaStreamSynchronize(st), "layout");
    return fail(c, BSORT_E_CUDA, "the bucket layout exceeded its table (a consistency check failed)");
  }
  const uint32_t n_total = hm->n_total, s_total = hm->s_total, items = hm->items_total;
  const uint32_t nseg = S.nseg;
  {
    // K1 reads the input and writes the letters and the word starts; K2
    // writes the segments
    const double k1 = (double)total_len + s_total + 4.0 * n_total;
    const double k2 = (double)sizeof(Segment) * nseg;
    c->kind_bytes[kTokenize] += k1;
    c->kind_bytes[kLayout] += k2;
    bool t1 = false, t2 = false;
    for (auto it = c->recs.rbegin(); it != c->recs.rend() && !(t1 && t2); ++it) {
      if (it->kind == kTokenize && !t1) {
        it->bytes += k1;
        t1 = true;
      } else if (it->kind == kLayout && !t2) {
        it->bytes += k2;
        t2 = true;
      }
    }
  }
  for (uint32_t d = 0; d < ndocs; ++d)
    if (h_hist[(size_t)d * kHist] != 0) c->doc_status[d] = BSORT_E_WORD_TOO_LONG;
  SortPlan p1;
  plan_from_summary(c, S, p1);
  const uint32_t ndd = p1.dd_end - p1.dd_beg;
  uint64_t htab_words = 0, uniq_words = 0, cnt_words = 0;
  for (int g = 0; g < 4; ++g) {
    htab_words += S.tot[g][kColHtab];
    uniq_words += S.tot[g][kColUniq];
    cnt_words += S.tot[g][kColDcnt];
  }
  const uint64_t off_bytes = c->cfg.want_offsets ? 4 : 0;

  // ---- size the key and output buffers ----
  const uint64_t key_words = order == BSORT_ORDER_LENGTH ? 16 : std::max<uint64_t>(p1.key_words, 16);
  GROW(c->keysA, 8 * key_words, "keys");
  GROW(c->keysB, 8 * key_words, "keys");
  GROW(c->samples, 8 * std::max<uint64_t>(p1.smp_words, 16), "merge samples");
  GROW(c->counts, 8ull * ndocs * kHist, "counts");
  GROW(c->offsets, 4ull * ((uint64_t)n_total + ndocs), "offsets");
  GROW(c->stream, (size_t)s_total + 16, "stream");
  DedupeOut ddo{nullptr, nullptr, nullptr, nullptr, nullptr};
  if (ndd) {
    const void* old_tab = c->htab.p;
    const void* old_cnt = c->dcnt.p;
    GROW(c->htab, 8 * htab_words, "hash tables");
    GROW(c->dcnt, 8 * std::max<uint64_t>(cnt_words, 16), "distinct-key counts");
    GROW(c->uA, 8 * std::max<uint64_t>(uniq_words, 16), "distinct keys");
    GROW(c->uB, 8 * std::max<uint64_t>(uniq_words, 16), "distinct keys");
    // a new table or count array, or ones an earlier call may have left dirty
    if (c->htab.p != old_tab || c->dcnt.p != old_cnt || !c->htab_clean) {
      CK(cudaMemsetAsync(c->htab.p, 0, c->htab.cap, st), "clear hash tables");
      CK(cudaMemsetAsync(c->dcnt.p, 0, c->dcnt.cap, st), "clear distinct-key counts");
      c->htab_clean = true;
    }
    ddo = DedupeOut{ins_dev, dptr<uint64_t>(c->htab), dptr<uint64_t>(c->uA), ucnt_dev, dptr<uint64_t>(c->dcnt)};
  }

  if (gap_a) {  // the round trip ends where the first launch after it is enqueued
    cudaEvent_t gap_b = next_event(c);
    if (gap_b) {
      cudaEventRecord(gap_b, st);
      c->recs.push_back(ProfRec{kHostGap, gap_a, gap_b, 0.0, 0u, 0u, 0u});
      c->kind_launches[kHostGap] += 1;
    }
  }
  uint64_t* kA = dptr<uint64_t>(c->keysA);
  uint64_t* kB = dptr<uint64_t>(c->keysB);
  uint64_t key_bytes_all = 0;
  for (int g = 0; g < kGroups; ++g) key_bytes_all += (uint64_t)p1.kb[g];
  const uint32_t grid_cap = (uint32_t)c->sm_count * 16;
  const EmitOut eo{dptr<uint8_t>(c->stream), dptr<uint32_t>(c->offsets), c->cfg.want_offsets, c->codec};
  if (order == BSORT_ORDER_LENGTH) GROW(c->icnt, 4ull * kHist * std::max<uint32_t>(items, 1), "length counts");
  {
    // K3 also writes each document's counts and closing offset, so it runs
    // even when no document has a word (and, for the length order, only that)
    const uint32_t count_grid = std::min<uint32_t>((ndocs * kHist + kWordThreads - 1) / kWordThreads, grid_cap);
    const uint32_t grid = std::max<uint32_t>(std::max(order == BSORT_ORDER_LENGTH ? 0u : items, count_grid), 1u);
    LAUNCH(kScatter,
           (double)s_total + 4.0 * n_total + key_bytes_all + (4.0 + 8.0) * kHist * ndocs + (off_bytes ? 12.0 : 0.0) * ndocs,
           launch_scatter(dptr<uint32_t>(c->starts), dptr<uint8_t>(c->letters), d_wbase, d_lbase, d_item0, ndocs,
                          items, grid, lookup_dev, segs_dev, cursor_dev, kA, d_hist, dptr<uint64_t>(c->counts), eo,
                          order != BSORT_ORDER_LENGTH, st),
           "K3 scatter");
  }
  if (order == BSORT_ORDER_LENGTH) {
    // no sort: every word's place follows from the per-block length counts
    LAUNCHK(kEmit, (double)s_total + 4.0 * n_total + (double)n_total * (off_bytes ? 4.0 : 0.0) + s_total,
           items ? 3u : 0u,
           launch_length_order(dptr<uint32_t>(c->starts), dptr<uint8_t>(c->letters), d_wbase, d_item0, ndocs, items,
                               lookup_dev, segs_dev, dptr<uint32_t>(c->icnt), eo, st),
           "length order");
    return BSORT_OK;
  }
  // K4, K5, K6 of the buckets.  The first launch on the call's stream sorts
  // the buckets that need merge passes (or, for the duplicate-aware sort,
  // aggregates them): the distinct-key counts, with the duplicate-aware
  // buckets' segments and descriptors, are read back right after it, while
  // the other launches run on.
  std::vector<cudaStream_t> joined;
  const uint32_t* h_ucnt = nullptr;
  const Segment* h_ddseg = nullptr;
  const DedupeIns* h_ins = nullptr;
  auto after_first = [&]() -> bsort_status {
    if (!ndd) return BSORT_OK;
    const size_t sb = align_up(sizeof(Segment) * ndd, 64), ib = align_up(sizeof(DedupeIns) * ndd, 64);
    GROW_HOST(c->h_dd, sb + ib, "duplicate-aware buckets");
    GROW_HOST(c->h_ucnt, 4ull * ndd, "distinct-key counts");
    h_ddseg = hptr<Segment>(c->h_dd);
    h_ins = hptr<DedupeIns>(c->h_dd, sb);
    h_ucnt = hptr<uint32_t>(c->h_ucnt);
    CK(cudaMemcpyAsync(hptr<Segment>(c->h_dd), segs_dev + p1.dd_beg, sizeof(Segment) * ndd, cudaMemcpyDeviceToHost, st),
       "read duplicate-aware buckets");
    CK(cudaMemcpyAsync(hptr<DedupeIns>(c->h_dd, sb), ins_dev, sizeof(DedupeIns) * ndd, cudaMemcpyDeviceToHost, st),
       "read duplicate-aware buckets");
    CK(cudaMemcpyAsync(hptr<uint32_t>(c->h_ucnt), ucnt_dev, 4ull * ndd, cudaMemcpyDeviceToHost, st),
       "read distinct-key counts");
    CK(cudaEventRecord(c->dedupe_ev, st), "distinct-key counts event");
    return BSORT_OK;
  };
  bsort_status s = launch_sorts(c, p1, segs_dev, kA, kB, dptr<uint64_t>(c->samples), c->jobs, barrier_dev, eo, ddo, st,
                                true, joined, after_first);
  if (s != BSORT_OK) return s;
  if (ndd) {
    s = sort_distinct(c, h_ddseg, h_ins, ndd, h_ucnt, eo, st);
    if (s != BSORT_OK) return s;
  }
  // the launches on side streams
  for (size_t i = 0; i < joined.size(); ++i) {
    CK(cudaEventRecord(c->join_ev[i], joined[i]), "join");
    CK(cudaStreamWaitEvent(st, c->join_ev[i], 0), "join");
  }
  if (order == BSORT_ORDER_WHOLE && nseg) {
    // the words of the whole-text order, from the sorted keys
    const uint32_t max_doc_words = S.max_doc_words;
    GROW(c->ssum, 4 * std::max<uint64_t>((uint64_t)nseg * var_slices(max_doc_words), 16), "letter prefixes");
    LAUNCHK(kEmit, (double)key_bytes_all + (double)s_total + (double)n_total * (off_bytes ? 4.0 : 0.0),
           max_doc_words ? 3u : 0u,
           launch_var_emit(var_dev, nseg, max_doc_words, kA, kB, c->codec,
                           dptr<uint32_t>(c->ssum), d_sticky, eo, st),
           "whole-text emit");
  }
  return BSORT_OK;
}

// Fills the scalar fields of document d's result from the host meta copy.
void fill_scalars(const bsort_ctx* c, uint32_t d, bsort_result* r) {
  const uint32_t* h_wbase = hptr<uint32_t>(c->h_meta, c->ml.wbase);
  const uint32_t* h_lbase = hptr<uint32_t>(c->h_meta, c->ml.lbase);
  r->max_len = hptr<uint32_t>(c->h_meta, c->ml.maxlen)[d];
  r->n_words = h_wbase[d + 1] - h_wbase[d];
  r->stream_bytes = h_lbase[d + 1] - h_lbase[d];
  r->status = c->doc_status[d];
}

// Copies the outputs of the last run to pinned host memory (offsets and
// stream land at the given bases of the host buffers) and builds the counts.
bsort_status read_back(bsort_ctx* c, cudaStream_t st, size_t off_base, size_t stream_base, size_t counts_base) {
  const uint32_t* h_wbase = hptr<uint32_t>(c->h_meta, c->ml.wbase);
  const uint32_t* h_lbase = hptr<uint32_t>(c->h_meta, c->ml.lbase);
  const uint32_t ndocs = c->ndocs;
  const uint64_t n_off = (uint64_t)h_wbase[ndocs] + ndocs;
  const uint64_t n_bytes = h_lbase[ndocs];
  if (c->cfg.want_offsets && n_off)
    CK(cudaMemcpyAsync(hptr<uint32_t>(c->h_offsets) + off_base, c->offsets.p, 4 * n_off, cudaMemcpyDeviceToHost, st),
       "read offsets");
  if (n_bytes)
    CK(cudaMemcpyAsync(hptr<uint8_t>(c->h_stream) + stream_base, c->stream.p, n_bytes, cudaMemcpyDeviceToHost, st),
       "read stream");
  Meta* hs = hptr<Meta>(c->h_sticky);
  CK(cudaMemcpyAsync(hs, c->sticky.p, sizeof(Meta), cudaMemcpyDeviceToHost, st), "read status");
  uint64_t* hc = hptr<uint64_t>(c->h_counts) + counts_base;
  const uint32_t* hh = hptr<uint32_t>(c->h_meta, c->ml.hist);
  for (size_t i = 0; i < (size_t)ndocs * kHist; ++i) hc[i] = (i % kHist) ? hh[i] : 0;
  CK(cudaStreamSynchronize(st), "wait for results");
  if (hs->err_timeout || hs->err_internal) {
    c->htab_clean = false;  // (a failed check may have left a claimed slot behind)
    CK(cudaMemsetAsync(c->sticky.p, 0, sizeof(Meta), st), "clear timeout flag");
    CK(cudaStreamSynchronize(st), "clear timeout flag");
    if (!hs->err_timeout)
      return fail(c, BSORT_E_CUDA, "a consistency check of the sort kernels failed (site " + std::to_string(hs->err_site) + ")");
    return fail(c, BSORT_E_TIMEOUT, "a bounded device wait ran out");
  }
  return BSORT_OK;
}

struct Busy {
  bsort_ctx* c;
  explicit Busy(bsort_ctx* x) : c(x) { c->busy = true; }
  ~Busy() { c->busy = false; }
};

bsort_status enter(bsort_ctx* c) {
  if (c->busy) return fail(c, BSORT_E_BUSY, "context in use by another call");
  c->err.clear();
  cudaError_t e = cudaSetDevice(c->device);
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaSetDevice");
  return BSORT_OK;
}

}  // namespace

extern "C" {

void bsort_config_default(bsort_config* cfg) {
  if (!cfg) return;
  cfg->l_cap = kMaxLen;
  cfg->want_offsets = 1;
  cfg->device = -1;
  cfg->profile = 0;
  cfg->wait_limit = 0;
  cfg->tune_table = nullptr;
  cfg->order = BSORT_ORDER_ASCII;
  cfg->key_pack = BSORT_KEYS_BYTES;
}

bsort_status bsort_create(bsort_ctx** out, const bsort_config* cfg) {
  if (!out) return BSORT_E_INVAL;
  *out = nullptr;
  bsort_config conf;
  bsort_config_default(&conf);
  if (cfg) conf = *cfg;
  if (conf.l_cap == 0) conf.l_cap = kMaxLen;
  if (conf.l_cap > (uint32_t)kMaxLen) return BSORT_E_INVAL;
  if (conf.wait_limit == 0) conf.wait_limit = kDefaultWaitLimit;
  conf.want_offsets = conf.want_offsets ? 1 : 0;
  conf.profile = conf.profile ? 1 : 0;
  if (conf.order > BSORT_ORDER_LENGTH || conf.key_pack > BSORT_KEYS_LETTERS6) return BSORT_E_INVAL;
  Tune tune;
  if (!parse_tune(conf.tune_table, tune)) return BSORT_E_INVAL;
  int dev = conf.device;
  if (dev < 0 && cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return BSORT_E_CUDA;
  }
  if (cudaSetDevice(dev) != cudaSuccess) {
    cudaGetLastError();
    return BSORT_E_CUDA;
  }
  bsort_ctx* c = new (std::nothrow) bsort_ctx();
  if (!c) return BSORT_E_NOMEM;
  c->cfg = conf;
  c->device = dev;
  c->codec = conf.order == BSORT_ORDER_FOLDED ? kCodeFold : conf.key_pack == BSORT_KEYS_LETTERS6 ? kCodeSix : kCodeBytes;
  c->tune = tune;
  if (conf.tune_table) c->tune_text = conf.tune_table;
  c->cfg.tune_table = conf.tune_table ? c->tune_text.c_str() : nullptr;
  if (cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaStreamCreateWithFlags(&c->own_stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->fork_ev, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->counts_ev, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->dedupe_ev, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    bsort_destroy(c);  // frees whatever was created
    return BSORT_E_CUDA;
  }
  for (int i = 0; i < bsort_ctx::kSide; ++i)
    if (cudaStreamCreateWithFlags(&c->side[i], cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->join_ev[i], cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      bsort_destroy(c);
      return BSORT_E_CUDA;
    }
  // the sticky status word starts cleared
  if (grow(c, c->sticky, sizeof(Meta), "status") != BSORT_OK ||
      grow_host(c, c->h_sticky, sizeof(Meta), "status") != BSORT_OK ||
      cudaMemset(c->sticky.p, 0, sizeof(Meta)) != cudaSuccess) {
    cudaGetLastError();
    bsort_destroy(c);
    return BSORT_E_NOMEM;
  }
  *out = c;
  return BSORT_OK;
}

void bsort_destroy(bsort_ctx* c) {
  if (!c) return;
  bsort_serve_shutdown(c);
  cudaSetDevice(c->device);
  if (c->own_stream) cudaStreamSynchronize(c->own_stream);
  for (DevBuf* b : {&c->sticky, &c->in, &c->docs, &c->meta, &c->starts, &c->letters, &c->plan, &c->keysA, &c->keysB,
                    &c->counts, &c->offsets, &c->stream, &c->jobs, &c->samples, &c->htab, &c->dcnt, &c->uA, &c->uB, &c->plan2,
                    &c->samples2, &c->jobs2, &c->pre, &c->ssum, &c->tfirst, &c->icnt})
    if (b->p) cudaFree(b->p);
  for (HostBuf* b : {&c->h_sticky, &c->h_in, &c->h_docs, &c->h_meta, &c->h_lay, &c->h_counts, &c->h_offsets,
                     &c->h_stream, &c->h_flag, &c->h_plan2, &c->h_ucnt, &c->h_dd})
    if (b->p) cudaFreeHost(b->p);
  for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
  if (c->fork_ev) cudaEventDestroy(c->fork_ev);
  if (c->counts_ev) cudaEventDestroy(c->counts_ev);
  if (c->dedupe_ev) cudaEventDestroy(c->dedupe_ev);
  for (int i = 0; i < bsort_ctx::kSide; ++i) {
    if (c->join_ev[i]) cudaEventDestroy(c->join_ev[i]);
    if (c->side[i]) cudaStreamDestroy(c->side[i]);
  }
  if (c->own_stream) cudaStreamDestroy(c->own_stream);
  delete c;
}

const char* bsort_last_error(const bsort_ctx* c) { return c ? c->err.c_str() : "null context"; }

bsort_status bsort_context_config(const bsort_ctx* c, bsort_config* out) {
  if (!c || !out) return BSORT_E_INVAL;
  *out = c->cfg;
  out->device = c->device;
  return BSORT_OK;
}

bsort_status bsort_text(bsort_ctx* c, const uint8_t* bytes, size_t len, bsort_result* out) {
  if (!c || !out || (!bytes && len)) return c ? fail(c, BSORT_E_INVAL, "null argument") : BSORT_E_INVAL;
  std::memset(out, 0, sizeof(*out));
  bsort_status s = enter(c);
  if (s != BSORT_OK) return s;
  Busy busy(c);
  if ((uint64_t)len >= (1ull << 32)) return fail(c, BSORT_E_TOO_LARGE, "document of 2^32 bytes or more");
  cudaStream_t st = c->own_stream;
  GROW(c->in, len + 16, "input");
  if (len) {
    if (host_pinned(bytes, len)) {  // page-locked: the copy engine reads it directly
      CK(cudaMemcpyAsync(c->in.p, bytes, len, cudaMemcpyHostToDevice, st), "copy input");
    } else {
      GROW_HOST(c->h_in, len + 16, "input staging");
      std::memcpy(c->h_in.p, bytes, len);
      CK(cudaMemcpyAsync(c->in.p, c->h_in.p, len, cudaMemcpyHostToDevice, st), "copy input");
    }
  }
  const uint64_t off = 0, l = len;
  s = run_path(c, dptr<uint8_t>(c->in), &off, &l, 1, st);
  if (s != BSORT_OK) return s;
  if (c->doc_status[0] != BSORT_OK) return fail(c, (bsort_status)c->doc_status[0], "a word is longer than l_cap");
  const uint32_t* h_wbase = hptr<uint32_t>(c->h_meta, c->ml.wbase);
  const uint32_t* h_lbase = hptr<uint32_t>(c->h_meta, c->ml.lbase);
  GROW_HOST(c->h_offsets, 4ull * (h_wbase[1] + 1), "offsets");
  GROW_HOST(c->h_stream, (size_t)h_lbase[1] + 16, "stream");
  GROW_HOST(c->h_counts, 8ull * kHist, "counts");
  s = read_back(c, st, 0, 0, 0);
  if (s != BSORT_OK) return s;
  fill_scalars(c, 0, out);
  out->counts = hptr<uint64_t>(c->h_counts);
  out->offsets = c->cfg.want_offsets ? hptr<uint32_t>(c->h_offsets) : nullptr;
  out->stream = hptr<uint8_t>(c->h_stream);
  return BSORT_OK;
}

bsort_status bsort_text_device(bsort_ctx* c, const uint8_t* d_bytes, size_t len, void* stream, bsort_result* out) {
  if (!c || !out || (!d_bytes && len)) return c ? fail(c, BSORT_E_INVAL, "null argument") : BSORT_E_INVAL;
  std::memset(out, 0, sizeof(*out));
  bsort_status s = enter(c);
  if (s != BSORT_OK) return s;
  Busy busy(c);
  if ((uint64_t)len >= (1ull << 32)) return fail(c, BSORT_E_TOO_LARGE, "document of 2^32 bytes or more");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const uint64_t off = 0, l = len;
  // an empty document still needs a valid (never dereferenced) base pointer
  const uint8_t* base = len ? d_bytes : dptr<uint8_t>(c->meta);
  s = run_path(c, base, &off, &l, 1, st);
  if (s != BSORT_OK) return s;
  if (c->doc_status[0] != BSORT_OK) return fail(c, (bsort_status)c->doc_status[0], "a word is longer than l_cap");
  fill_scalars(c, 0, out);
  out->counts = dptr<uint64_t>(c->counts);
  out->offsets = c->cfg.want_offsets ? dptr<uint32_t>(c->offsets) : nullptr;
  out->stream = dptr<uint8_t>(c->stream);
  return BSORT_OK;
}

bsort_status bsort_batch(bsort_ctx* c, const uint8_t* const* docs, const size_t* lens, size_t n, bsort_result* outs) {
  if (!c || (n && (!docs || !lens || !outs))) return c ? fail(c, BSORT_E_INVAL, "null argument") : BSORT_E_INVAL;
  for (size_t i = 0; i < n; ++i) std::memset(&outs[i], 0, sizeof(bsort_result));
  if (n == 0) return BSORT_OK;
  for (size_t i = 0; i < n; ++i)
    if (!docs[i] && lens[i]) return fail(c, BSORT_E_INVAL, "null document with non-zero length");
  if (n >= (1ull << 24)) return fail(c, BSORT_E_TOO_LARGE, "too many documents in one call");
  bsort_status s = enter(c);
  if (s != BSORT_OK) return s;
  Busy busy(c);
  cudaStream_t st = c->own_stream;
  // Host output buffers for the whole call; documents run in groups of at
  // most 1 GiB of input so that 32-bit positions suffice inside a group.
  uint64_t total = 0, off_total = 0;
  for (size_t i = 0; i < n; ++i) {
    if ((uint64_t)lens[i] >= (1ull << 30)) return fail(c, BSORT_E_TOO_LARGE, "document of 1 GiB or more in a batch");
    total += lens[i];
    off_total += lens[i] / 2 + 2;
  }
  GROW_HOST(c->h_offsets, 4 * off_total, "offsets");
  GROW_HOST(c->h_stream, total + 16, "stream");
  GROW_HOST(c->h_counts, 8ull * kHist * n, "counts");
  const uint64_t kGroupBytes = 1ull << 30;
  std::vector<uint64_t> offs, ls;
  std::vector<uint32_t> first_err;
  size_t g0 = 0, off_base = 0, stream_base = 0;
  bsort_status first = BSORT_OK;
  while (g0 < n) {
    size_t g1 = g0;
    uint64_t bytes = 0;
    while (g1 < n && (g1 == g0 || bytes + align_up(lens[g1], 16) <= kGroupBytes)) bytes += align_up(lens[g1++], 16);
    const uint32_t nd = (uint32_t)(g1 - g0);
    offs.resize(nd);
    ls.resize(nd);
    // Documents that lie back to back in host memory (the empty ones
    // anywhere) move as one region: one copy, read directly when it is
    // page-locked.  Others are gathered into the staging buffer.
    const uint8_t* region = nullptr;
    const uint8_t* region_end = nullptr;
    bool contiguous = true;
    for (size_t i = g0; i < g1 && contiguous; ++i) {
      if (!lens[i]) continue;
      if (!region) region = docs[i];
      else if (docs[i] != region_end) contiguous = false;
      region_end = docs[i] + lens[i];
    }
    if (contiguous && region) {
      const size_t rb = (size_t)(region_end - region);
      GROW(c->in, rb + 16, "input");
      for (uint32_t i = 0; i < nd; ++i) {
        ls[i] = lens[g0 + i];
        offs[i] = ls[i] ? (uint64_t)(docs[g0 + i] - region) : 0;
      }
      if (host_pinned(region, rb)) {
        CK(cudaMemcpyAsync(c->in.p, region, rb, cudaMemcpyHostToDevice, st), "copy input");
      } else {
        GROW_HOST(c->h_in, rb + 16, "input staging");
        std::memcpy(c->h_in.p, region, rb);
        CK(cudaMemcpyAsync(c->in.p, c->h_in.p, rb, cudaMemcpyHostToDevice, st), "copy input");
      }
    } else {
      GROW(c->in, bytes + 16, "input");
      bool all_pinned = true;
      for (size_t i = g0; i < g1 && all_pinned; ++i) all_pinned = !lens[i] || host_pinned(docs[i], lens[i]);
      uint64_t pos = 0;
      if (all_pinned) {  // every document page-locked: the copy engine reads each in place
        for (uint32_t i = 0; i < nd; ++i) {
          offs[i] = pos;
          ls[i] = lens[g0 + i];
          if (ls[i])
            CK(cudaMemcpyAsync(dptr<uint8_t>(c->in, pos), docs[g0 + i], ls[i], cudaMemcpyHostToDevice, st),
               "copy input");
          pos += align_up(ls[i], 16);
        }
      } else {  // gathered into the staging buffer, then one copy
        GROW_HOST(c->h_in, bytes + 16, "input staging");
        for (uint32_t i = 0; i < nd; ++i) {
          offs[i] = pos;
          ls[i] = lens[g0 + i];
          if (ls[i]) std::memcpy(hptr<uint8_t>(c->h_in, pos), docs[g0 + i], ls[i]);
          pos += align_up(ls[i], 16);
        }
        if (bytes) CK(cudaMemcpyAsync(c->in.p, c->h_in.p, bytes, cudaMemcpyHostToDevice, st), "copy input");
      }
    }
    s = run_path(c, dptr<uint8_t>(c->in), offs.data(), ls.data(), nd, st);
    if (s != BSORT_OK) return s;
    s = read_back(c, st, off_base, stream_base, (size_t)g0 * kHist);
    if (s != BSORT_OK) return s;
    const uint32_t* h_wbase = hptr<uint32_t>(c->h_meta, c->ml.wbase);
    const uint32_t* h_lbase = hptr<uint32_t>(c->h_meta, c->ml.lbase);
    for (uint32_t i = 0; i < nd; ++i) {
      bsort_result* r = &outs[g0 + i];
      fill_scalars(c, i, r);
      if (r->status != BSORT_OK) {
        if (first == BSORT_OK) {
          first = (bsort_status)r->status;
          c->err = "document " + std::to_string(g0 + i) + ": a word is longer than l_cap";
        }
        const uint32_t st_keep = r->status;
        std::memset(r, 0, sizeof(*r));
        r->status = st_keep;
        continue;
      }
      r->counts = hptr<uint64_t>(c->h_counts) + (size_t)(g0 + i) * kHist;
      r->offsets = c->cfg.want_offsets ? hptr<uint32_t>(c->h_offsets) + off_base + h_wbase[i] + i : nullptr;
      r->stream = hptr<uint8_t>(c->h_stream) + stream_base + h_lbase[i];
    }
    off_base += (size_t)h_wbase[nd] + nd;
    stream_base += h_lbase[nd];
    g0 = g1;
  }
  return first;
}

int bsort_profile_read(bsort_ctx* c, bsort_kernel_stat* out, int max) {
  if (!c || (!out && max > 0) || max < 0) return -1;
  if (cudaSetDevice(c->device) != cudaSuccess) {
    cudaGetLastError();
    return -1;
  }
  double ms[kKinds] = {};
  for (const ProfRec& r : c->recs) {
    float t = 0.f;
    if (cudaEventSynchronize(r.b) != cudaSuccess || cudaEventElapsedTime(&t, r.a, r.b) != cudaSuccess) {
      cudaGetLastError();
      return -1;
    }
    ms[r.kind] += t;
  }
  int k = 0;
  for (int i = 0; i < kKinds && k < max; ++i) {
    out[k].name = kKindName[i];
    out[k].launches = c->kind_launches[i];
    out[k].ms = ms[i];
    out[k].bytes = c->kind_bytes[i];
    out[k].key_levels = c->kind_levels[i];
    ++k;
  }
  for (int i = 0; i < kKinds; ++i) {
    c->kind_launches[i] = 0;
    c->kind_bytes[i] = 0;
    c->kind_levels[i] = 0;
  }
  c->recs.clear();
  c->ev_used = 0;
  return k;
}

int bsort_trace_read(bsort_ctx* c, bsort_trace_rec* out, int max) {
  if (!c || (!out && max > 0) || max < 0) return -1;
  if (c->recs.empty()) return 0;
  if (cudaSetDevice(c->device) != cudaSuccess) {
    cudaGetLastError();
    return -1;
  }
  const cudaEvent_t t0 = c->recs.front().a;
  int k = 0;
  for (const ProfRec& r : c->recs) {
    if (k < max) {
      float s = 0.f, e = 0.f;
      if (cudaEventSynchronize(r.b) != cudaSuccess || cudaEventElapsedTime(&s, t0, r.a) != cudaSuccess ||
          cudaEventElapsedTime(&e, t0, r.b) != cudaSuccess) {
        cudaGetLastError();
        return -1;
      }
      out[k] = bsort_trace_rec{kKindName[r.kind], s, e, r.bytes, r.stream, r.variant, r.kernels, 0u};
    }
    ++k;
  }
  return k;
}

uint64_t bsort_launch_count(const bsort_ctx* c) { return c ? c->launches : 0; }

bsort_status bsort_batch_device(bsort_ctx* c, const uint8_t* d_base, const uint64_t* offs, const uint64_t* lens,
                                size_t n, void* stream, bsort_result* outs) {
  if (!c || (n && (!offs || !lens || !outs))) return c ? fail(c, BSORT_E_INVAL, "null argument") : BSORT_E_INVAL;
  for (size_t i = 0; i < n; ++i) std::memset(&outs[i], 0, sizeof(bsort_result));
  if (n == 0) return BSORT_OK;
  if (n >= (1ull << 24)) return fail(c, BSORT_E_TOO_LARGE, "too many documents in one call");
  uint64_t total = 0;
  for (size_t i = 0; i < n; ++i) {
    if (!d_base && lens[i]) return fail(c, BSORT_E_INVAL, "null base with a non-empty document");
    total += lens[i];
  }
  if (total >= (1ull << 32)) return fail(c, BSORT_E_TOO_LARGE, "2^32 bytes or more in one batch");
  bsort_status s = enter(c);
  if (s != BSORT_OK) return s;
  Busy busy(c);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const uint8_t* base = d_base ? d_base : dptr<uint8_t>(c->meta);  // never dereferenced when every document is empty
  s = run_path(c, base, offs, lens, (uint32_t)n, st);
  if (s != BSORT_OK) return s;
  const uint32_t* h_wbase = hptr<uint32_t>(c->h_meta, c->ml.wbase);
  const uint32_t* h_lbase = hptr<uint32_t>(c->h_meta, c->ml.lbase);
  bsort_status first = BSORT_OK;
  for (uint32_t i = 0; i < (uint32_t)n; ++i) {
    bsort_result* r = &outs[i];
    fill_scalars(c, i, r);
    if (r->status != BSORT_OK) {
      if (first == BSORT_OK) {
        first = (bsort_status)r->status;
        c->err = "document " + std::to_string(i) + ": a word is longer than l_cap";
      }
      const uint32_t keep = r->status;
      std::memset(r, 0, sizeof(*r));
      r->status = keep;
      continue;
    }
    r->counts = dptr<uint64_t>(c->counts) + (size_t)i * kHist;
    r->offsets = c->cfg.want_offsets ? dptr<uint32_t>(c->offsets) + h_wbase[i] + i : nullptr;
    r->stream = dptr<uint8_t>(c->stream) + h_lbase[i];
  }
  return first;
}

bsort_status bsort_device_finish(bsort_ctx* c, void* stream) {
  if (!c) return BSORT_E_INVAL;
  bsort_status s = enter(c);
  if (s != BSORT_OK) return s;
  Busy busy(c);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Meta* hs = hptr<Meta>(c->h_sticky);
  CK(cudaMemcpyAsync(hs, c->sticky.p, sizeof(Meta), cudaMemcpyDeviceToHost, st), "read status");
  CK(cudaStreamSynchronize(st), "wait for the device work");
  if (hs->err_timeout || hs->err_internal) {
    c->htab_clean = false;  // (a failed check may have left a claimed slot behind)
    CK(cudaMemsetAsync(c->sticky.p, 0, sizeof(Meta), st), "clear timeout flag");
    CK(cudaStreamSynchronize(st), "clear timeout flag");
    if (!hs->err_timeout) return fail(c, BSORT_E_CUDA, "a consistency check of the sort kernels failed");
    return fail(c, BSORT_E_TIMEOUT, "a bounded device wait of the sort kernels ran out (the outputs are not valid)");
  }
  return BSORT_OK;
}

void bsort_result_release(bsort_ctx* c, bsort_result* res) {
  if (!res) return;
  if (c) bsort_serve_release(c, res);  // a served result: its batch's buffers may be reused
  std::memset(res, 0, sizeof(*res));
}

}  // extern "C"

struct bsort_host_out {
  HostBuf counts, offsets, stream;
};

bsort_host_out* bsort_take_result_buffers(bsort_ctx* c) {
  bsort_host_out* b = new bsort_host_out{c->h_counts, c->h_offsets, c->h_stream};
  c->h_counts = HostBuf{};
  c->h_offsets = HostBuf{};
  c->h_stream = HostBuf{};
  return b;
}

void bsort_give_result_buffers(bsort_ctx* c, bsort_host_out* b) {
  for (HostBuf* h : {&c->h_counts, &c->h_offsets, &c->h_stream})
    if (h->p) cudaFreeHost(h->p);
  c->h_counts = b->counts;
  c->h_offsets = b->offsets;
  c->h_stream = b->stream;
  delete b;
}

// (the result buffers a batch of ndocs documents of `bytes` bytes can need)
static uint64_t need_counts(uint64_t ndocs) { return 8ull * kHist * std::max<uint64_t>(ndocs, 1); }
static uint64_t need_offsets(uint64_t bytes, uint64_t ndocs) { return 4ull * (bytes / 2 + 2 * ndocs + 1); }
static uint64_t need_stream(uint64_t bytes) { return bytes + 16; }

bsort_status bsort_reserve_result_buffers(bsort_ctx* c, uint64_t bytes, uint64_t ndocs) {
  GROW_HOST(c->h_counts, need_counts(ndocs), "counts");
  GROW_HOST(c->h_offsets, need_offsets(bytes, ndocs), "offsets");
  GROW_HOST(c->h_stream, need_stream(bytes), "stream");
  return BSORT_OK;
}

bool bsort_result_buffers_fit(const bsort_host_out* b, uint64_t bytes, uint64_t ndocs) {
  return b->counts.cap >= need_counts(ndocs) && b->offsets.cap >= need_offsets(bytes, ndocs) &&
         b->stream.cap >= need_stream(bytes);
}

void bsort_free_result_buffers(bsort_host_out* b) {
  if (!b) return;
  for (HostBuf* h : {&b->counts, &b->offsets, &b->stream})
    if (h->p) cudaFreeHost(h->p);
  delete b;
}
